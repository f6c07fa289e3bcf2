// noalloc.cu -- ode_run_periods_noalloc: the iterated integration of
// ode_run_periods without a solver object and without any device allocation.
//
// Some callers cannot call cudaMalloc: a framework that owns all device memory
// through its own pool allocator (a raw cudaMalloc beside it fragments memory
// and can fail under the pool's high-water mark), or a latency-bound loop where
// the implicit device synchronisation of cudaMalloc / cudaFree is not
// acceptable.  Such a caller owns every input and output buffer; the only
// other global memory the persistent integrator kernel needs -- its
// work-queue head, its watchdog flag and its per-system bookkeeping (stop
// status, event counters, accepted / rejected step counters) -- lives in the
// file-scope array below, reserved once when the library's device code is
// loaded on a GPU and kept until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/odegpu.h"
#include "common.cuh"
#include "noalloc_layout.h"

using namespace odegpu;

namespace {

constexpr int kNoAllocMaxSystems = 65536;
// sections on 256-byte boundaries (noalloc_layout.h): 1 835 264 bytes
constexpr size_t kScratchBytes = noalloc_layout(kNoAllocMaxSystems, kMaxE).total;

// Device scratch shared by every call on a device.  In host code this name is
// a host-side stand-in, not a device address: the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current),
// looked up once per device.
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[device] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = (unsigned char*)g_scratch_ptr[device];
  return cudaSuccess;
}

thread_local char g_msg[256];

int bad(const char* m) {
  strncpy(g_msg, m, sizeof(g_msg) - 1);
  g_msg[sizeof(g_msg) - 1] = 0;
  return ODE_ERR_INVALID_ARG;
}

int cuda_bad(cudaError_t e) {
  strncpy(g_msg, cudaGetErrorString(e), sizeof(g_msg) - 1);
  g_msg[sizeof(g_msg) - 1] = 0;
  return e == cudaErrorMemoryAllocation ? ODE_ERR_OUT_OF_MEMORY : ODE_ERR_CUDA;
}

int launch(const ode_noalloc_settings* cfg, const void* fn, int n, int E, int n_systems,
           int device, double h0, int n_transient, int n_record, double* td, double* y,
           const double* p, double* acc, double* records, int* status, long long* accepted,
           cudaStream_t st);

}  // namespace

extern "C" int ode_run_periods_noalloc(const ode_noalloc_settings* cfg, int n_systems, int device,
                                       double h0, int n_transient, int n_record, double* td,
                                       double* y, const double* p, double* acc, double* records,
                                       int* status, long long* accepted, void* stream,
                                       const char** message) {
  if (message) *message = g_msg;
  g_msg[0] = 0;
  if (!cfg) return bad("settings are NULL");
  int n, P, A, E;
  if (!model_dims(cfg->model, &n, &P, &A, &E)) return bad("unknown model");
  if (cfg->scheme != ODE_RK4 && cfg->scheme != ODE_RKCK45) return bad("unknown scheme");
  if (cfg->prec != ODE_FP64 && cfg->prec != ODE_FP32_RHS) return bad("unknown precision");
  const void* fn = kernel_for(cfg->model, cfg->scheme, cfg->prec, 1);
  if (!fn) return bad("no kernel for this model / scheme / precision");
  if (n_systems < 1) return bad("n_systems must be >= 1");
  if (n_systems > kNoAllocMaxSystems)
    return bad("n_systems exceeds the no-allocation maximum of 65536 systems");
  if (device < 0 || device >= kMaxDevices) return bad("device index out of range");
  if (!(h0 > 0.0) || !isfinite(h0)) return bad("h0 must be finite and > 0");
  if (n_transient < 0 || n_record < 0 || (long long)n_transient + n_record > 0x7fffffffLL)
    return bad("bad slice counts");
  if (!td || !y || !p || !acc) return bad("td, y, p and acc are required device arrays");
  if ((uintptr_t)td % alignof(double) || (uintptr_t)y % alignof(double) ||
      (uintptr_t)p % alignof(double) || (uintptr_t)acc % alignof(double) ||
      (uintptr_t)records % alignof(double) || (uintptr_t)status % alignof(int) ||
      (uintptr_t)accepted % alignof(long long))
    return bad("an array is not aligned for its element type");
  if (!(cfg->h_min > 0.0) || !(cfg->h_max >= cfg->h_min) || !isfinite(cfg->h_max) ||
      !(cfg->grow_limit >= 1.0) || !(cfg->grow_limit <= 1e4) || !(cfg->shrink_limit >= 1e-4) ||
      !(cfg->shrink_limit <= 1.0))
    return bad("need 0 < h_min <= h_max < inf, 1 <= grow <= 1e4, 1e-4 <= shrink <= 1");
  for (int i = 0; i < n; i++)
    if (!(cfg->rtol[i] >= 0.0) || !(cfg->atol[i] >= 0.0) || !(cfg->rtol[i] + cfg->atol[i] > 0.0))
      return bad("tolerances must be >= 0 with atol + rtol > 0");
  if (cfg->events_enabled)
    for (int j = 0; j < E; j++)
      if (cfg->direction[j] < -1 || cfg->direction[j] > 1 || !(cfg->tolerance[j] >= 0.0) ||
          cfg->stop_count[j] < 0)
        return bad("bad event properties");
  if (cfg->time_domain_mode < ODE_TD_KEEP || cfg->time_domain_mode > ODE_TD_SHIFT)
    return bad("unknown time-domain mode");
  if (cfg->max_steps_per_slice < 1) return bad("step budget must be >= 1");
  if (!(cfg->time_limit_s >= 0.0) || !(cfg->time_limit_s < 1e6)) return bad("bad time limit");
  for (int i = 0; i < kMaxMC; i++)
    if (!isfinite(cfg->model_constants[i])) return bad("model constants must be finite");
  const int n_slices = n_transient + n_record;
  if (n_slices == 0) return ODE_OK;

  int prev_device = -1;
  if (cudaGetDevice(&prev_device) != cudaSuccess) prev_device = -1;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_bad(e);
  const int rc = launch(cfg, fn, n, E, n_systems, device, h0, n_transient, n_record, td, y, p, acc,
                        records, status, accepted, (cudaStream_t)stream);
  if (prev_device >= 0 && prev_device != device) cudaSetDevice(prev_device);
  return rc;
}

namespace {

int launch(const ode_noalloc_settings* cfg, const void* fn, int n, int E, int n_systems,
           int device, double h0, int n_transient, int n_record, double* td, double* y,
           const double* p, double* acc, double* records, int* status, long long* accepted,
           cudaStream_t st) {
  const int n_slices = n_transient + n_record;
  cudaError_t e;
  unsigned char* scratch = nullptr;
  if ((e = scratch_address(device, &scratch)) != cudaSuccess) return cuda_bad(e);

  const size_t N = (size_t)n_systems;
  const NoAllocLayout lay = noalloc_layout(N, kMaxE);
  if (lay.total > kScratchBytes) return bad("scratch layout exceeds the fixed array");
  long long* d_nacc = (long long*)(scratch + lay.nacc);
  long long* d_nrej = (long long*)(scratch + lay.nrej);
  int* d_status = (int*)(scratch + lay.status);
  int* d_ecnt = (int*)(scratch + lay.ecnt);
  // every section must be aligned for its element type before the kernel
  // touches it (a misaligned 8-byte access is a device fault)
  if ((uintptr_t)scratch % kNoAllocAlign != 0 || (uintptr_t)d_nacc % alignof(long long) != 0 ||
      (uintptr_t)d_nrej % alignof(long long) != 0 || (uintptr_t)d_status % alignof(int) != 0 ||
      (uintptr_t)d_ecnt % alignof(int) != 0)
    return bad("misaligned scratch section");
  // what the kernel accumulates into or tests must start at zero
  if ((e = cudaMemsetAsync(scratch, 0, lay.total, st)) != cudaSuccess) return cuda_bad(e);

  KArgs a;
  memset(&a, 0, sizeof(a));
  a.N = n_systems;
  a.ld = n_systems;
  a.td = td;
  a.y = y;
  a.p = p;
  a.acc = acc;
  a.status = d_status;
  a.ecnt = d_ecnt;
  a.nacc = d_nacc;
  a.nrej = d_nrej;
  a.records = n_record > 0 ? records : nullptr;
  a.n_slices = n_slices;
  a.n_skip = n_transient;
  a.h0 = h0;
  a.queue_head = (unsigned int*)(scratch + lay.head);
  a.queue_mode = 1;
  a.flags = (int*)(scratch + lay.head + 64);
  a.time_limit_ns = (long long)(cfg->time_limit_s * 1e9);
  Props& pr = a.pr;
  for (int i = 0; i < kMaxN; i++) {
    pr.rtol[i] = i < n ? cfg->rtol[i] : 1.0;
    pr.atol[i] = i < n ? cfg->atol[i] : 1.0;
  }
  pr.hmax = cfg->h_max;
  pr.hmin = cfg->h_min;
  pr.grow = cfg->grow_limit;
  pr.shrink = cfg->shrink_limit;
  pr.err_grow = pow(0.9 / pr.grow, 5.0);
  pr.err_shrink = pow(0.9 / pr.shrink, 5.0);
  for (int j = 0; j < kMaxE; j++) {
    pr.evt_dir[j] = j < E ? cfg->direction[j] : -1;
    pr.evt_tol[j] = j < E ? cfg->tolerance[j] : 0.0;
    pr.evt_stop[j] = j < E ? cfg->stop_count[j] : 0;
  }
  pr.max_eq = cfg->max_steps_in_zone;
  pr.events_on = cfg->events_enabled ? 1 : 0;
  pr.td_mode = cfg->time_domain_mode;
  pr.max_steps = cfg->max_steps_per_slice;
  for (int i = 0; i < kMaxMC; i++) pr.mc[i] = cfg->model_constants[i];

  int sms = 0, bps = 0;
  const int block = 128;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return cuda_bad(e);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, block, 0)) != cudaSuccess)
    return cuda_bad(e);
  if (bps < 1) return bad("kernel cannot be resident");
  long long grid = (long long)bps * sms;
  const long long need = (n_systems + block - 1) / block;
  if (grid > need) grid = need;
  // the queue holds the systems after the grid's first wave
  a.queue_stride = queue_stride_for((int)std::max(0LL, (long long)n_systems - grid * block));
  void* args[] = {&a};
  if ((e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(block), args, 0, st)) != cudaSuccess)
    return cuda_bad(e);
  if (status &&
      (e = cudaMemcpyAsync(status, d_status, N * sizeof(int), cudaMemcpyDeviceToDevice, st)) !=
          cudaSuccess)
    return cuda_bad(e);
  if (accepted && (e = cudaMemcpyAsync(accepted, d_nacc, N * sizeof(long long),
                                       cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return cuda_bad(e);
  return ODE_OK;
}

}  // namespace
