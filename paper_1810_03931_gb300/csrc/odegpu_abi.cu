// odegpu_abi.cu -- host implementation of the C ABI declared in
// include/odegpu.h: the solver object of Sec. 6.2 (device buffers), the
// LinearSet / RandomSet copies of Sec. 6.3, the Solve call of Sec. 6.4 and
// the iterated Solve of Sec. 7.1.1 as a single launch, read-back (Sec. 6.10)
// and the launch scheduler (per-sweep grid or persistent work-queue grid).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/odegpu.h"
#include "common.cuh"

using namespace odegpu;

namespace odegpu {
bool model_dims(int model, int* n, int* P, int* A, int* E) {
  switch (model) {
    case ODE_DUFFING: *n = 2; *P = 2; *A = 7; *E = 1; return true;
    case ODE_KELLER_MIKSIS: *n = 2; *P = 13; *A = 4; *E = 1; return true;
    case ODE_VALVE: *n = 3; *P = 5; *A = 5; *E = 2; return true;
    case ODE_BOUNCE: *n = 2; *P = 2; *A = 6; *E = 1; return true;
    case ODE_DUFFING_LYAPUNOV: *n = 4; *P = 2; *A = 5; *E = 1; return true;
    default: return false;
  }
}

const void* kernel_for(int model, int scheme, int prec, int persistent) {
  switch (model) {
    case ODE_DUFFING: return kernel_duffing(scheme, prec, persistent);
    case ODE_KELLER_MIKSIS: return kernel_keller_miksis(scheme, prec, persistent);
    case ODE_VALVE: return kernel_valve(scheme, prec, persistent);
    case ODE_BOUNCE: return kernel_bounce(scheme, prec, persistent);
    case ODE_DUFFING_LYAPUNOV: return kernel_duffing_lyapunov(scheme, prec, persistent);
    default: return nullptr;
  }
}
}  // namespace odegpu

struct ode_solver {
  int model, scheme, prec, N, device;
  int n, P, A, E;
  Props pr;
  double* d_td = nullptr;
  double* d_y = nullptr;
  double* d_p = nullptr;
  double* d_acc = nullptr;
  int* d_status = nullptr;
  int* d_ecnt = nullptr;
  long long* d_nacc = nullptr;
  long long* d_nrej = nullptr;
  unsigned int* d_queue = nullptr;
  double* d_records = nullptr;  // staging for host-side records
  size_t records_cap = 0;       // doubles
  double* d_stage = nullptr;    // staging for RandomSet / RandomGet of host data
  size_t stage_cap = 0;         // bytes
  int block_size = 0;           // 0 = automatic
  int persistent = 0;
  int spt = 1;                  // per-sweep launches: systems per thread
  int slices_per_launch = 0;    // ode_run_periods: slices per launch (0 = all in one)
  int warp_sync = 0;            // lanes of a warp start every slice together
  double time_limit_s = 600.0;  // watchdog limit per thread and launch
  std::string err;
};

namespace {

thread_local std::string g_err;  // failures without a solver

int fail(ode_solver* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  g_err = msg;
  return code;
}

int cuda_fail(ode_solver* s, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
  return fail(s, e == cudaErrorMemoryAllocation ? ODE_ERR_OUT_OF_MEMORY : ODE_ERR_CUDA, m);
}

#define CK_CUDA(s, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
  } while (0)

void default_props(ode_solver* s) {
  Props& p = s->pr;
  memset(&p, 0, sizeof(p));
  // ODE properties printed in Sec. 6.5
  for (int i = 0; i < kMaxN; i++) {
    p.rtol[i] = 1e-10;
    p.atol[i] = 1e-10;
  }
  p.hmax = 1.0e6;
  p.hmin = 1.0e-12;
  p.grow = 5.0;
  p.shrink = 0.1;
  // event properties of Sec. 6.6 (disabled until ode_set_events)
  for (int j = 0; j < kMaxE; j++) {
    p.evt_dir[j] = -1;
    p.evt_tol[j] = 1e-6;
    p.evt_stop[j] = 0;
  }
  if (s->model == ODE_VALVE) {
    p.evt_stop[0] = 1;
    p.max_eq = 50;
  }
  p.events_on = 0;
  p.td_mode = kTdKeep;
  p.max_steps = 1000000000LL;
  if (s->model == ODE_DUFFING || s->model == ODE_DUFFING_LYAPUNOV) {
    p.mc[0] = -1.0;  // delta
    p.mc[1] = 1.0;   // c3
    p.mc[2] = 1.0;   // omega
  }
}

int check_solver(ode_solver* s) {
  if (!s) return fail(nullptr, ODE_ERR_INVALID_ARG, "solver is NULL");
  return ODE_OK;
}

// Select the solver's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int ensure_stage(ode_solver* s, size_t bytes) {
  if (bytes <= s->stage_cap) return ODE_OK;
  if (s->d_stage) cudaFree(s->d_stage);
  s->d_stage = nullptr;
  s->stage_cap = 0;
  CK_CUDA(s, cudaMalloc(&s->d_stage, bytes));
  s->stage_cap = bytes;
  return ODE_OK;
}

// Arrays selected by a copy mode: (object array, components).
struct Sel {
  double* obj;
  int comps;
  int flag;
};

void selections(ode_solver* s, Sel out[4]) {
  out[0] = {s->d_td, 2, ODE_TIMEDOMAIN};
  out[1] = {s->d_y, s->n, ODE_STATE};
  out[2] = {s->d_p, s->P, ODE_PARAM};
  out[3] = {s->d_acc, s->A, ODE_ACC};
}

// Gather / scatter between a pool and the object for index lists living on
// the device: obj[c * N + idx_obj[i]] <-> pool[c * pool + idx_pool[i]].
__global__ void random_copy_kernel(double* obj, int N, const double* pool, double* pool_out,
                                   int pool_size, int comps, const int* idx_obj,
                                   const int* idx_pool, int count, int to_object) {
  const long long total = (long long)count * comps;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k % count);
    const int c = (int)(k / count);
    const int io = idx_obj[i], ip = idx_pool[i];
    if (io < 0 || io >= N || ip < 0 || ip >= pool_size) continue;
    if (to_object)
      obj[(size_t)c * N + io] = pool[(size_t)c * pool_size + ip];
    else
      pool_out[(size_t)c * pool_size + ip] = obj[(size_t)c * N + io];
  }
}

// The same for a contiguous staging buffer [comps][count] and object indices.
__global__ void stage_scatter_kernel(double* obj, int N, const double* stage, int comps,
                                     const int* idx_obj, int count, int to_object) {
  const long long total = (long long)count * comps;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k % count);
    const int c = (int)(k / count);
    const int io = idx_obj[i];
    if (io < 0 || io >= N) continue;
    if (to_object)
      obj[(size_t)c * N + io] = stage[(size_t)c * count + i];
    else
      ((double*)stage)[(size_t)c * count + i] = obj[(size_t)c * N + io];
  }
}

int grid_for(long long work) {
  long long g = (work + 255) / 256;
  if (g < 1) g = 1;
  if (g > 65535) g = 65535;
  return (int)g;
}

// Linear copies between the pool and the object for the selected arrays.
int linear_copy(ode_solver* s, int start_obj, int start_pool, int pool_size, int count,
                double* td, double* y, double* p, double* acc, int copy_mode, int ptr_kind,
                void* stream, bool to_object) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (ptr_kind != ODE_PTR_HOST && ptr_kind != ODE_PTR_DEVICE)
    return fail(s, ODE_ERR_INVALID_ARG, "ptr_kind must be ODE_PTR_HOST or ODE_PTR_DEVICE");
  if (copy_mode < 0 || copy_mode > ODE_ALL)
    return fail(s, ODE_ERR_INVALID_ARG, "copy_mode must be a combination of ODE_TIMEDOMAIN..ODE_ACC");
  if (count < 0 || pool_size < 0 || start_obj < 0 || start_pool < 0 ||
      (long long)start_obj + count > s->N || (long long)start_pool + count > pool_size)
    return fail(s, ODE_ERR_INVALID_ARG, "copy range outside the object or the pool");
  double* arrs[4] = {td, y, p, acc};
  Sel sel[4];
  selections(s, sel);
  for (int k = 0; k < 4; k++)
    if ((copy_mode & sel[k].flag) && arrs[k] == nullptr && count > 0)
      return fail(s, ODE_ERR_INVALID_ARG, "an array selected by copy_mode is NULL");
  if (count == 0) return ODE_OK;
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyKind kind = ptr_kind == ODE_PTR_DEVICE
                            ? cudaMemcpyDeviceToDevice
                            : (to_object ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  for (int k = 0; k < 4; k++) {
    if (!(copy_mode & sel[k].flag)) continue;
    // one 2-D copy per array: `comps` rows of `count` doubles
    const size_t row = (size_t)count * sizeof(double);
    double* objp = sel[k].obj + start_obj;
    double* poolp = arrs[k] + start_pool;
    if (to_object)
      CK_CUDA(s, cudaMemcpy2DAsync(objp, (size_t)s->N * sizeof(double), poolp,
                                   (size_t)pool_size * sizeof(double), row, sel[k].comps, kind, st));
    else
      CK_CUDA(s, cudaMemcpy2DAsync(poolp, (size_t)pool_size * sizeof(double), objp,
                                   (size_t)s->N * sizeof(double), row, sel[k].comps, kind, st));
  }
  if (ptr_kind == ODE_PTR_HOST) CK_CUDA(s, cudaStreamSynchronize(st));
  return ODE_OK;
}

int random_copy(ode_solver* s, const int* idx_obj, const int* idx_pool, int pool_size, int count,
                double* td, double* y, double* p, double* acc, int copy_mode, int ptr_kind,
                void* stream, bool to_object) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (ptr_kind != ODE_PTR_HOST && ptr_kind != ODE_PTR_DEVICE)
    return fail(s, ODE_ERR_INVALID_ARG, "ptr_kind must be ODE_PTR_HOST or ODE_PTR_DEVICE");
  if (copy_mode < 0 || copy_mode > ODE_ALL)
    return fail(s, ODE_ERR_INVALID_ARG, "copy_mode must be a combination of ODE_TIMEDOMAIN..ODE_ACC");
  if (count < 0 || pool_size < 0) return fail(s, ODE_ERR_INVALID_ARG, "negative count or pool size");
  if (count == 0) return ODE_OK;
  if (!idx_obj || !idx_pool) return fail(s, ODE_ERR_INVALID_ARG, "index arrays are NULL");
  double* arrs[4] = {td, y, p, acc};
  Sel sel[4];
  selections(s, sel);
  for (int k = 0; k < 4; k++)
    if ((copy_mode & sel[k].flag) && arrs[k] == nullptr)
      return fail(s, ODE_ERR_INVALID_ARG, "an array selected by copy_mode is NULL");
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (ptr_kind == ODE_PTR_DEVICE) {
    for (int k = 0; k < 4; k++) {
      if (!(copy_mode & sel[k].flag)) continue;
      random_copy_kernel<<<grid_for((long long)count * sel[k].comps), 256, 0, st>>>(
          sel[k].obj, s->N, arrs[k], arrs[k], pool_size, sel[k].comps, idx_obj, idx_pool, count,
          to_object ? 1 : 0);
      CK_CUDA(s, cudaGetLastError());
    }
    return ODE_OK;
  }
  // host data: check the indices, gather / scatter through a device staging
  // buffer laid out [comps][count] with the object indices in front of it
  for (int i = 0; i < count; i++) {
    if (idx_obj[i] < 0 || idx_obj[i] >= s->N || idx_pool[i] < 0 || idx_pool[i] >= pool_size)
      return fail(s, ODE_ERR_INVALID_ARG, "index outside the object or the pool");
  }
  int maxc = std::max(std::max(2, s->n), std::max(s->P, s->A));
  size_t idx_bytes = ((size_t)count * sizeof(int) + 255) / 256 * 256;
  if (int rc = ensure_stage(s, idx_bytes + (size_t)maxc * count * sizeof(double))) return rc;
  int* d_idx = (int*)s->d_stage;
  double* d_vals = (double*)((char*)s->d_stage + idx_bytes);
  CK_CUDA(s, cudaMemcpyAsync(d_idx, idx_obj, (size_t)count * sizeof(int), cudaMemcpyHostToDevice, st));
  std::vector<double> host((size_t)maxc * count);
  for (int k = 0; k < 4; k++) {
    if (!(copy_mode & sel[k].flag)) continue;
    const int comps = sel[k].comps;
    if (to_object) {
      for (int c = 0; c < comps; c++)
        for (int i = 0; i < count; i++)
          host[(size_t)c * count + i] = arrs[k][(size_t)c * pool_size + idx_pool[i]];
      CK_CUDA(s, cudaMemcpyAsync(d_vals, host.data(), (size_t)comps * count * sizeof(double),
                                 cudaMemcpyHostToDevice, st));
      stage_scatter_kernel<<<grid_for((long long)count * comps), 256, 0, st>>>(
          sel[k].obj, s->N, d_vals, comps, d_idx, count, 1);
      CK_CUDA(s, cudaGetLastError());
      CK_CUDA(s, cudaStreamSynchronize(st));  // host staging is reused
    } else {
      stage_scatter_kernel<<<grid_for((long long)count * comps), 256, 0, st>>>(
          sel[k].obj, s->N, d_vals, comps, d_idx, count, 0);
      CK_CUDA(s, cudaGetLastError());
      CK_CUDA(s, cudaMemcpyAsync(host.data(), d_vals, (size_t)comps * count * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
      CK_CUDA(s, cudaStreamSynchronize(st));
      for (int c = 0; c < comps; c++)
        for (int i = 0; i < count; i++)
          arrs[k][(size_t)c * pool_size + idx_pool[i]] = host[(size_t)c * count + i];
    }
  }
  return ODE_OK;
}

// Entries of the block-shared RK4 forcing table (Sec. 7.1.1's fixed-step
// loop over forcing periods): 2 n + 1 (cos, sin) pairs cover n steps per
// slice; 2049 pairs (32 KB of shared memory) cover up to 1024 steps.
constexpr int kForcingTable = 2049;

// Table entries for a launch of this solver: binary64 RK4 of a forced model
// whose slices keep their time domain (every slice on the same grid), else 0.
int forcing_table_entries(const ode_solver* s) {
  const bool forced = s->model == ODE_DUFFING || s->model == ODE_DUFFING_LYAPUNOV ||
                      s->model == ODE_KELLER_MIKSIS;
  return (s->scheme == ODE_RK4 && s->prec == ODE_FP64 && forced && s->pr.td_mode == kTdKeep)
             ? kForcingTable : 0;
}

// Blocks per SM and block size for a launch of `fn` with `smem` bytes of
// dynamic shared memory.
int launch_shape(ode_solver* s, const void* fn, int* block, int* blocks_per_sm, int* sms, size_t smem = 0) {
  int bs = s->block_size;
  if (bs <= 0) bs = 128;
  CK_CUDA(s, cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, s->device));
  CK_CUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bs, smem));
  if (*blocks_per_sm < 1)
    return fail(s, ODE_ERR_UNSUPPORTED, "kernel cannot be resident with the requested block size");
  *block = bs;
  return ODE_OK;
}

void finish_props(Props& p) {
  p.err_grow = pow(0.9 / p.grow, 5.0);
  p.err_shrink = pow(0.9 / p.shrink, 5.0);
}

// After the work on `stream` is complete: report a watchdog stop.
int check_watchdog(ode_solver* s, cudaStream_t st) {
  int flag = 0;
  CK_CUDA(s, cudaMemcpyAsync(&flag, (char*)s->d_queue + 64, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK_CUDA(s, cudaStreamSynchronize(st));
  if (flag) {
    CK_CUDA(s, cudaMemsetAsync((char*)s->d_queue + 64, 0, sizeof(int), st));
    return fail(s, ODE_ERR_TIMEOUT,
                "the watchdog stopped systems that ran past the time limit (status ODE_ST_TIMEOUT)");
  }
  return ODE_OK;
}

int integrate(ode_solver* s, double h0, int n_slices, int n_skip, double* records, void* stream) {
  const void* fn = kernel_for(s->model, s->scheme, s->prec, s->persistent ? 1 : 0);
  if (!fn) return fail(s, ODE_ERR_UNSUPPORTED, "no kernel compiled for this model/scheme/precision");
  cudaStream_t st = (cudaStream_t)stream;
  KArgs a;
  a.N = s->N;
  a.ld = s->N;
  a.td = s->d_td;
  a.y = s->d_y;
  a.p = s->d_p;
  a.acc = s->d_acc;
  a.status = s->d_status;
  a.ecnt = s->d_ecnt;
  a.nacc = s->d_nacc;
  a.nrej = s->d_nrej;
  a.records = records;
  a.n_slices = n_slices;
  a.n_skip = n_skip;
  a.h0 = h0;
  a.slices_left = nullptr;
  a.queue_head = s->d_queue;
  a.queue_mode = s->persistent;
  a.spt = s->persistent ? 1 : s->spt;
  a.warp_sync = s->warp_sync;
  a.tab_cap = forcing_table_entries(s);
  const size_t smem = (size_t)a.tab_cap * sizeof(double2);
  a.flags = (int*)((char*)s->d_queue + 64);
  a.time_limit_ns = (long long)(s->time_limit_s * 1e9);
  a.pr = s->pr;
  finish_props(a.pr);
  int block, bps, sms;
  if (int rc = launch_shape(s, fn, &block, &bps, &sms, smem)) return rc;
  long long grid;
  if (s->persistent) {
    CK_CUDA(s, cudaMemsetAsync(s->d_queue, 0, sizeof(unsigned int), st));
    grid = (long long)bps * sms;
    long long need = (s->N + block - 1) / block;
    if (grid > need) grid = need;
  } else {
    const long long per_block = (long long)block * a.spt;
    grid = (s->N + per_block - 1) / per_block;
  }
  if (grid < 1) grid = 1;
  // the queue holds the systems after the grid's first wave (thread i starts
  // with system i)
  a.queue_stride = queue_stride_for((int)std::max(0LL, (long long)s->N - grid * block));
  void* args[] = {&a};
  CK_CUDA(s, cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(block), args, smem, st));
  return ODE_OK;
}

// n_slices slices in launches of at most slices_per_launch slices each (0 =
// one launch).  Every launch stores each system's full state and time
// domain, so the split does not change any result; records of global slice
// g >= n_transient go to index g - n_transient (a launch starting at slice c0
// skips n_transient - c0 slices, which may be negative).
int run_slices(ode_solver* s, double h0, int n_slices, int n_transient, double* records, void* stream) {
  const int L = s->slices_per_launch > 0 ? s->slices_per_launch : n_slices;
  for (int c0 = 0; c0 < n_slices; c0 += L) {
    const int n = std::min(L, n_slices - c0);
    if (int rc = integrate(s, h0, n, n_transient - c0, records, stream)) return rc;
  }
  return ODE_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int ode_create(ode_solver** out, int model, int scheme, int prec, int n_systems, int device) {
  if (!out) return fail(nullptr, ODE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int n, P, A, E;
  if (!model_dims(model, &n, &P, &A, &E)) return fail(nullptr, ODE_ERR_INVALID_ARG, "unknown model");
  if (scheme != ODE_RK4 && scheme != ODE_RKCK45)
    return fail(nullptr, ODE_ERR_INVALID_ARG, "scheme must be ODE_RK4 or ODE_RKCK45");
  if (prec != ODE_FP64 && prec != ODE_FP32_RHS)
    return fail(nullptr, ODE_ERR_INVALID_ARG, "prec must be ODE_FP64 or ODE_FP32_RHS");
  if (prec == ODE_FP32_RHS && (model == ODE_KELLER_MIKSIS || model == ODE_DUFFING_LYAPUNOV))
    return fail(nullptr, ODE_ERR_INVALID_ARG, "the Keller-Miksis and Lyapunov models are binary64 only");
  if (n_systems < 1) return fail(nullptr, ODE_ERR_INVALID_ARG, "n_systems must be >= 1");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(nullptr, ODE_ERR_INVALID_ARG, "no such CUDA device");
  ode_solver* s = new (std::nothrow) ode_solver();
  if (!s) return fail(nullptr, ODE_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->model = model;
  s->scheme = scheme;
  s->prec = prec;
  s->N = n_systems;
  s->device = device;
  s->n = n;
  s->P = P;
  s->A = A;
  s->E = E;
  default_props(s);
  DeviceGuard g(device);
  if (!g.ok) {
    delete s;
    return fail(nullptr, ODE_ERR_CUDA, "cudaSetDevice failed");
  }
  const size_t N = (size_t)n_systems;
  struct {
    void** p;
    size_t bytes;
  } allocs[] = {{(void**)&s->d_td, 2 * N * sizeof(double)},
                {(void**)&s->d_y, n * N * sizeof(double)},
                {(void**)&s->d_p, P * N * sizeof(double)},
                {(void**)&s->d_acc, A * N * sizeof(double)},
                {(void**)&s->d_status, N * sizeof(int)},
                {(void**)&s->d_ecnt, E * N * sizeof(int)},
                {(void**)&s->d_nacc, N * sizeof(long long)},
                {(void**)&s->d_nrej, N * sizeof(long long)},
                {(void**)&s->d_queue, 256}};
  for (auto& al : allocs) {
    e = cudaMalloc(al.p, al.bytes);
    if (e == cudaSuccess) e = cudaMemset(*al.p, 0, al.bytes);
    if (e != cudaSuccess) {
      int rc = cuda_fail(nullptr, e, "ode_create device allocation");
      ode_destroy(s);
      return rc;
    }
  }
  *out = s;
  return ODE_OK;
}

int ode_destroy(ode_solver* s) {
  if (!s) return ODE_OK;
  DeviceGuard g(s->device);
  cudaDeviceSynchronize();
  void* ptrs[] = {s->d_td, s->d_y, s->d_p, s->d_acc, s->d_status, s->d_ecnt, s->d_nacc,
                  s->d_nrej, s->d_queue, s->d_records, s->d_stage};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
  return ODE_OK;
}

int ode_query_dims(const ode_solver* s, int* n_sys, int* n_par, int* n_evt, int* n_acc) {
  if (!s) return fail(nullptr, ODE_ERR_INVALID_ARG, "solver is NULL");
  if (n_sys) *n_sys = s->n;
  if (n_par) *n_par = s->P;
  if (n_evt) *n_evt = s->E;
  if (n_acc) *n_acc = s->A;
  return ODE_OK;
}

int ode_num_systems(const ode_solver* s, int* n_systems) {
  if (!s || !n_systems) return fail(nullptr, ODE_ERR_INVALID_ARG, "NULL argument");
  *n_systems = s->N;
  return ODE_OK;
}

int ode_set_tolerances(ode_solver* s, const double* rtol, const double* atol, double h_max,
                       double h_min, double grow_limit, double shrink_limit) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (!rtol || !atol) return fail(s, ODE_ERR_INVALID_ARG, "rtol / atol are NULL");
  if (!(h_min > 0.0) || !(h_max >= h_min) || !(grow_limit >= 1.0) || !(grow_limit <= 1e4) ||
      !(shrink_limit >= 1e-4) || !(shrink_limit <= 1.0) || !isfinite(h_max))
    return fail(s, ODE_ERR_INVALID_ARG,
                "need 0 < h_min <= h_max < inf, 1 <= grow_limit <= 1e4, 1e-4 <= shrink_limit <= 1");
  for (int i = 0; i < s->n; i++) {
    if (!(rtol[i] >= 0.0) || !(atol[i] >= 0.0) || !(rtol[i] + atol[i] > 0.0) ||
        !isfinite(rtol[i]) || !isfinite(atol[i]))
      return fail(s, ODE_ERR_INVALID_ARG, "tolerances must be finite, >= 0, atol + rtol > 0");
  }
  for (int i = 0; i < s->n; i++) {
    s->pr.rtol[i] = rtol[i];
    s->pr.atol[i] = atol[i];
  }
  s->pr.hmax = h_max;
  s->pr.hmin = h_min;
  s->pr.grow = grow_limit;
  s->pr.shrink = shrink_limit;
  return ODE_OK;
}

int ode_set_events(ode_solver* s, int enabled, const int* direction, const double* tolerance,
                   const int* stop_count, int max_steps_in_zone) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (max_steps_in_zone < 0) return fail(s, ODE_ERR_INVALID_ARG, "max_steps_in_zone must be >= 0");
  if (enabled) {
    if (!direction || !tolerance || !stop_count)
      return fail(s, ODE_ERR_INVALID_ARG, "event property arrays are NULL");
    for (int j = 0; j < s->E; j++) {
      if (direction[j] < -1 || direction[j] > 1)
        return fail(s, ODE_ERR_INVALID_ARG, "event direction must be -1, 0 or +1");
      if (!(tolerance[j] >= 0.0) || !isfinite(tolerance[j]))
        return fail(s, ODE_ERR_INVALID_ARG, "event tolerance must be finite and >= 0");
      if (stop_count[j] < 0) return fail(s, ODE_ERR_INVALID_ARG, "stop count must be >= 0");
    }
    for (int j = 0; j < s->E; j++) {
      s->pr.evt_dir[j] = direction[j];
      s->pr.evt_tol[j] = tolerance[j];
      s->pr.evt_stop[j] = stop_count[j];
    }
  }
  s->pr.events_on = enabled ? 1 : 0;
  s->pr.max_eq = max_steps_in_zone;
  return ODE_OK;
}

int ode_set_model_constants(ode_solver* s, const double* c, int nc) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  const int allowed = (s->model == ODE_DUFFING || s->model == ODE_DUFFING_LYAPUNOV) ? 3 : 0;
  if (nc < 0 || nc > allowed || (nc > 0 && !c))
    return fail(s, ODE_ERR_INVALID_ARG, "wrong number of model constants for this model");
  for (int i = 0; i < nc; i++) {
    if (!isfinite(c[i])) return fail(s, ODE_ERR_INVALID_ARG, "model constants must be finite");
    s->pr.mc[i] = c[i];
  }
  return ODE_OK;
}

int ode_set_time_domain_mode(ode_solver* s, int mode) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (mode < ODE_TD_KEEP || mode > ODE_TD_SHIFT)
    return fail(s, ODE_ERR_INVALID_ARG, "unknown time-domain mode");
  s->pr.td_mode = mode;
  return ODE_OK;
}

int ode_set_step_budget(ode_solver* s, long long max_steps_per_slice) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (max_steps_per_slice < 1) return fail(s, ODE_ERR_INVALID_ARG, "step budget must be >= 1");
  s->pr.max_steps = max_steps_per_slice;
  return ODE_OK;
}

int ode_set_time_limit(ode_solver* s, double seconds) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (!(seconds >= 0.0) || !(seconds < 1e6))
    return fail(s, ODE_ERR_INVALID_ARG, "time limit must be in [0, 1e6) seconds");
  s->time_limit_s = seconds;
  return ODE_OK;
}

int ode_set_launch(ode_solver* s, int block_size, int persistent) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (block_size != 0 && (block_size < 32 || block_size > 256 || block_size % 32))
    return fail(s, ODE_ERR_INVALID_ARG, "block_size must be 0 or a multiple of 32 in [32, 256]");
  if (persistent < 0 || persistent > 2)
    return fail(s, ODE_ERR_INVALID_ARG, "persistent must be 0 (per-sweep), 1 or 2 (queue orders)");
  s->block_size = block_size;
  s->persistent = persistent;
  return ODE_OK;
}

int ode_set_schedule(ode_solver* s, int systems_per_thread, int slices_per_launch, int warp_sync) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (systems_per_thread < 1 || systems_per_thread > 64)
    return fail(s, ODE_ERR_INVALID_ARG, "systems_per_thread must be in [1, 64]");
  if (slices_per_launch < 0) return fail(s, ODE_ERR_INVALID_ARG, "slices_per_launch must be >= 0");
  if (warp_sync != 0 && warp_sync != 1) return fail(s, ODE_ERR_INVALID_ARG, "warp_sync must be 0 or 1");
  s->spt = systems_per_thread;
  s->slices_per_launch = slices_per_launch;
  s->warp_sync = warp_sync;
  return ODE_OK;
}

int ode_linear_set(ode_solver* s, int start_obj, int start_pool, int pool_size, int count,
                   const double* td, const double* y, const double* p, const double* acc,
                   int copy_mode, int ptr_kind, void* stream) {
  return linear_copy(s, start_obj, start_pool, pool_size, count, (double*)td, (double*)y,
                     (double*)p, (double*)acc, copy_mode, ptr_kind, stream, true);
}

int ode_linear_get(ode_solver* s, int start_obj, int start_pool, int pool_size, int count,
                   double* td, double* y, double* p, double* acc, int copy_mode, int ptr_kind,
                   void* stream) {
  return linear_copy(s, start_obj, start_pool, pool_size, count, td, y, p, acc, copy_mode, ptr_kind,
                     stream, false);
}

int ode_random_set(ode_solver* s, const int* idx_obj, const int* idx_pool, int pool_size, int count,
                   const double* td, const double* y, const double* p, const double* acc,
                   int copy_mode, int ptr_kind, void* stream) {
  return random_copy(s, idx_obj, idx_pool, pool_size, count, (double*)td, (double*)y, (double*)p,
                     (double*)acc, copy_mode, ptr_kind, stream, true);
}

int ode_random_get(ode_solver* s, const int* idx_obj, const int* idx_pool, int pool_size, int count,
                   double* td, double* y, double* p, double* acc, int copy_mode, int ptr_kind,
                   void* stream) {
  return random_copy(s, idx_obj, idx_pool, pool_size, count, td, y, p, acc, copy_mode, ptr_kind,
                     stream, false);
}

int ode_solve(ode_solver* s, double h0, void* stream) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (!(h0 > 0.0) || !isfinite(h0)) return fail(s, ODE_ERR_INVALID_ARG, "h0 must be finite and > 0");
  DeviceGuard g(s->device);
  return integrate(s, h0, 1, 1, nullptr, stream);
}

int ode_run_periods(ode_solver* s, double h0, int n_transient, int n_record, double* records,
                    int ptr_kind, void* stream) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (!(h0 > 0.0) || !isfinite(h0)) return fail(s, ODE_ERR_INVALID_ARG, "h0 must be finite and > 0");
  if (n_transient < 0 || n_record < 0)
    return fail(s, ODE_ERR_INVALID_ARG, "n_transient and n_record must be >= 0");
  if (ptr_kind != ODE_PTR_HOST && ptr_kind != ODE_PTR_DEVICE)
    return fail(s, ODE_ERR_INVALID_ARG, "ptr_kind must be ODE_PTR_HOST or ODE_PTR_DEVICE");
  if ((long long)n_transient + n_record > 0x7fffffffLL)
    return fail(s, ODE_ERR_INVALID_ARG, "too many slices");
  const int n_slices = n_transient + n_record;
  if (n_slices == 0) return ODE_OK;
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t R = (size_t)(s->A + s->n + 1);
  const size_t rec_doubles = (size_t)n_record * R * s->N;
  double* dev_rec = nullptr;
  if (records != nullptr && n_record > 0) {
    if (ptr_kind == ODE_PTR_DEVICE) {
      dev_rec = records;
    } else {
      if (rec_doubles > s->records_cap) {
        if (s->d_records) cudaFree(s->d_records);
        s->d_records = nullptr;
        s->records_cap = 0;
        CK_CUDA(s, cudaMalloc(&s->d_records, rec_doubles * sizeof(double)));
        s->records_cap = rec_doubles;
      }
      dev_rec = s->d_records;
    }
  }
  if (int rc = run_slices(s, h0, n_slices, n_transient, dev_rec, stream)) return rc;
  if (records != nullptr && n_record > 0 && ptr_kind == ODE_PTR_HOST) {
    CK_CUDA(s, cudaMemcpyAsync(records, dev_rec, rec_doubles * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    return check_watchdog(s, st);
  }
  return ODE_OK;
}

int ode_synchronize(ode_solver* s) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  DeviceGuard g(s->device);
  CK_CUDA(s, cudaDeviceSynchronize());
  return check_watchdog(s, (cudaStream_t)0);
}

int ode_get_status(ode_solver* s, int* status, long long* accepted, long long* rejected,
                   int* event_counts, int ptr_kind, void* stream) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (ptr_kind != ODE_PTR_HOST && ptr_kind != ODE_PTR_DEVICE)
    return fail(s, ODE_ERR_INVALID_ARG, "ptr_kind must be ODE_PTR_HOST or ODE_PTR_DEVICE");
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyKind kind = ptr_kind == ODE_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t N = (size_t)s->N;
  if (status) CK_CUDA(s, cudaMemcpyAsync(status, s->d_status, N * sizeof(int), kind, st));
  if (accepted) CK_CUDA(s, cudaMemcpyAsync(accepted, s->d_nacc, N * sizeof(long long), kind, st));
  if (rejected) CK_CUDA(s, cudaMemcpyAsync(rejected, s->d_nrej, N * sizeof(long long), kind, st));
  if (event_counts)
    CK_CUDA(s, cudaMemcpyAsync(event_counts, s->d_ecnt, (size_t)s->E * N * sizeof(int), kind, st));
  if (ptr_kind == ODE_PTR_HOST) return check_watchdog(s, st);
  return ODE_OK;
}

int ode_reset_counters(ode_solver* s, void* stream) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  CK_CUDA(s, cudaMemsetAsync(s->d_nacc, 0, (size_t)s->N * sizeof(long long), st));
  CK_CUDA(s, cudaMemsetAsync(s->d_nrej, 0, (size_t)s->N * sizeof(long long), st));
  return ODE_OK;
}

const char* ode_last_error(const ode_solver* s) { return s ? s->err.c_str() : g_err.c_str(); }

int ode_autotune(ode_solver* s, double h0, int n_slices, void* stream, int* block_size,
                 int* persistent, int* systems_per_thread, int* slices_per_launch, int* warp_sync,
                 double* trial_ms) {
  if (check_solver(s)) return ODE_ERR_INVALID_ARG;
  if (!(h0 > 0.0) || !isfinite(h0)) return fail(s, ODE_ERR_INVALID_ARG, "h0 must be finite and > 0");
  if (n_slices < 1 || n_slices > 1000000) return fail(s, ODE_ERR_INVALID_ARG, "n_slices out of range");
  static const int kBlocks[6] = {64, 96, 128, 160, 192, 256};
  // launch forms: (persistent, systems per thread)
  static const int kForms[4][2] = {{0, 1}, {0, 2}, {1, 1}, {2, 1}};
  DeviceGuard g(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)s->N;
  // the trial runs change time domain, state, accessories, status, counters:
  // save them and put them back afterwards
  const size_t dbl = (2 + s->n + s->A) * N, ints = (1 + s->E) * N, lls = 2 * N;
  char* save = nullptr;
  CK_CUDA(s, cudaMalloc(&save, dbl * sizeof(double) + ints * sizeof(int) + lls * sizeof(long long)));
  struct Piece {
    void* p;
    size_t bytes;
  } pieces[] = {{s->d_td, 2 * N * sizeof(double)},     {s->d_y, s->n * N * sizeof(double)},
                {s->d_acc, s->A * N * sizeof(double)},  {s->d_status, N * sizeof(int)},
                {s->d_ecnt, s->E * N * sizeof(int)},    {s->d_nacc, N * sizeof(long long)},
                {s->d_nrej, N * sizeof(long long)}};
  auto copy_all = [&](bool to_save) -> cudaError_t {
    size_t off = 0;
    for (auto& pc : pieces) {
      cudaError_t e = to_save ? cudaMemcpyAsync(save + off, pc.p, pc.bytes, cudaMemcpyDeviceToDevice, st)
                              : cudaMemcpyAsync(pc.p, save + off, pc.bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
      off += pc.bytes;
    }
    return cudaSuccess;
  };
  cudaError_t e = copy_all(true);
  const int old_block = s->block_size, old_pers = s->persistent, old_spt = s->spt,
            old_spl = s->slices_per_launch, old_ws = s->warp_sync;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int rc = ODE_OK;
  // one timed trial of the current shape; ms < 0 when it was not run
  auto trial = [&](float* ms) -> bool {
    *ms = -1.f;
    if ((e = copy_all(false)) != cudaSuccess) return false;
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return false;
    if ((rc = run_slices(s, h0, n_slices, n_slices, nullptr, stream)) != ODE_OK) return false;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return false;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return false;
    return (e = cudaEventElapsedTime(ms, e0, e1)) == cudaSuccess;
  };
  // fastest block per form (one launch, no warp-synchronous slices)
  double form_ms[4] = {1e300, 1e300, 1e300, 1e300};
  int form_b[4] = {0, 0, 0, 0};
  for (int f = 0; f < 4 && e == cudaSuccess && rc == ODE_OK; f++) {
    const int pers = kForms[f][0], spt = kForms[f][1];
    const void* fn = kernel_for(s->model, s->scheme, s->prec, pers ? 1 : 0);
    int max_threads = 1024;
    cudaFuncAttributes at;
    if (fn && cudaFuncGetAttributes(&at, fn) == cudaSuccess) max_threads = at.maxThreadsPerBlock;
    for (int k = 0; k < 6 && e == cudaSuccess && rc == ODE_OK; k++) {
      if (trial_ms) trial_ms[f * 6 + k] = -1.0;
      if (!fn || kBlocks[k] > max_threads) continue;
      int bps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlocks[k], 0) != cudaSuccess || bps < 1)
        continue;
      s->block_size = kBlocks[k];
      s->persistent = pers;
      s->spt = spt;
      s->slices_per_launch = 0;
      s->warp_sync = 0;
      float ms;
      if (!trial(&ms)) break;
      if (trial_ms) trial_ms[f * 6 + k] = ms;
      if (ms < form_ms[f]) {
        form_ms[f] = ms;
        form_b[f] = kBlocks[k];
      }
    }
  }
  // the fastest shape so far (f0) and the overall choice
  int f0 = -1;
  for (int f = 0; f < 4; f++)
    if (form_b[f] > 0 && (f0 < 0 || form_ms[f] < form_ms[f0])) f0 = f;
  double best = f0 >= 0 ? form_ms[f0] : 1e300;
  int best_b = f0 >= 0 ? form_b[f0] : 128, best_p = f0 >= 0 ? kForms[f0][0] : 1,
      best_spt = f0 >= 0 ? kForms[f0][1] : 1, best_spl = 0, best_ws = 0;
  if (trial_ms)
    for (int k = 24; k < 32; k++) trial_ms[k] = -1.0;
  // warp-synchronous slices for every form at its fastest block: whether they
  // pay depends on the form (a persistent queue mixes systems inside a warp)
  for (int f = 0; f < 4 && e == cudaSuccess && rc == ODE_OK; f++) {
    if (form_b[f] == 0) continue;
    s->block_size = form_b[f];
    s->persistent = kForms[f][0];
    s->spt = kForms[f][1];
    s->slices_per_launch = 0;
    s->warp_sync = 1;
    float ms;
    if (!trial(&ms)) break;
    if (trial_ms) trial_ms[28 + f] = ms;
    if (ms < best) {
      best = ms;
      best_b = form_b[f];
      best_p = kForms[f][0];
      best_spt = kForms[f][1];
      best_spl = 0;
      best_ws = 1;
    }
  }
  // the split of the slices for the fastest shape of the first search: one
  // slice per launch and half of the trial's slices per launch
  if (f0 >= 0 && e == cudaSuccess && rc == ODE_OK) {
    if (trial_ms) {
      trial_ms[26] = form_ms[f0];
      trial_ms[27] = trial_ms[28 + f0];
    }
    const int cand_spl[2] = {1, (n_slices + 1) / 2};
    for (int k = 0; k < 2 && e == cudaSuccess && rc == ODE_OK; k++) {
      if (cand_spl[k] >= n_slices || (k == 1 && cand_spl[1] == cand_spl[0])) continue;
      s->block_size = form_b[f0];
      s->persistent = kForms[f0][0];
      s->spt = kForms[f0][1];
      s->slices_per_launch = cand_spl[k];
      s->warp_sync = 0;
      float ms;
      if (!trial(&ms)) break;
      if (trial_ms) trial_ms[24 + k] = ms;
      if (ms < best) {
        best = ms;
        best_b = form_b[f0];
        best_p = kForms[f0][0];
        best_spt = kForms[f0][1];
        best_spl = cand_spl[k];
        best_ws = 0;
      }
    }
  }
  if (e == cudaSuccess) e = copy_all(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (rc != ODE_OK || e != cudaSuccess) {
    s->block_size = old_block;
    s->persistent = old_pers;
    s->spt = old_spt;
    s->slices_per_launch = old_spl;
    s->warp_sync = old_ws;
    return rc != ODE_OK ? rc : cuda_fail(s, e, "ode_autotune");
  }
  s->block_size = best_b;
  s->persistent = best_p;
  s->spt = best_spt;
  s->slices_per_launch = best_spl;
  s->warp_sync = best_ws;
  if (warp_sync) *warp_sync = best_ws;
  if (block_size) *block_size = best_b;
  if (persistent) *persistent = best_p;
  if (systems_per_thread) *systems_per_thread = best_spt;
  if (slices_per_launch) *slices_per_launch = best_spl;
  return check_watchdog(s, st);
}

int ode_km_coefficients(double PA1, double PA2, double omega1, double omega2, double theta,
                        double RE, double Pinf, double pV, double sigma, double mu, double rho,
                        double cL, double gamma, double* C) {
  if (!C) return fail(nullptr, ODE_ERR_INVALID_ARG, "C is NULL");
  if (!(RE > 0) || !(omega1 > 0) || !(rho > 0) || !(cL > 0))
    return fail(nullptr, ODE_ERR_INVALID_ARG, "RE, omega1, rho and cL must be > 0");
  // Eqs. (16)-(28) of the paper; L = 2 pi / (R_E omega_1) is the length-time
  // scale factor that appears squared in most coefficients.
  const double L = 2.0 * M_PI / (RE * omega1);
  const double L2 = L * L;
  const double pg_eq = Pinf - pV + 2.0 * sigma / RE;  // gas pressure at rest
  C[0] = pg_eq * L2 / rho;
  C[1] = (1.0 - 3.0 * gamma) * pg_eq * L / (rho * cL);
  C[2] = (Pinf - pV) * L2 / rho;
  C[3] = 2.0 * sigma * L2 / (rho * RE);
  C[4] = 4.0 * mu * (2.0 * M_PI / omega1) / (rho * RE * RE);
  C[5] = PA1 * L2 / rho;
  C[6] = PA2 * L2 / rho;
  C[7] = RE * omega1 * PA1 * L2 / (rho * cL);
  C[8] = RE * omega2 * PA2 * L2 / (rho * cL);  // omega_2: d/dt of P_A2 sin(omega_2 t)
  C[9] = RE * omega1 / (2.0 * M_PI * cL);
  C[10] = 3.0 * gamma;
  C[11] = omega2 / omega1;
  C[12] = theta;
  return ODE_OK;
}

int ode_kernel_info(int model, int scheme, int prec, int persistent, int block_size, int device,
                    int* regs, int* local_bytes, int* blocks_per_sm) {
  const void* fn = kernel_for(model, scheme, prec, persistent ? 1 : 0);
  if (!fn) return fail(nullptr, ODE_ERR_INVALID_ARG, "no kernel for this model/scheme/precision");
  DeviceGuard g(device);
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, fn);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaFuncGetAttributes");
  if (regs) *regs = at.numRegs;
  if (local_bytes) *local_bytes = (int)at.localSizeBytes;
  if (blocks_per_sm) {
    int bs = block_size > 0 ? block_size : 128;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bs, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  }
  return ODE_OK;
}

}  // extern "C"
