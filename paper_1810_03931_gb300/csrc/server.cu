// server.cu -- continuous-batching request loop for parameter-sweep requests.
//
// Each model has a resident pool of system slots in HBM (its size chosen by
// the caller within the server's HBM budget).  A request -- n systems of one
// model, each integrated for a number of periods (slices) -- is admitted when
// a contiguous range of free slots exists; its inputs are copied into the
// range and its state stays resident there until its horizon is done.  An
// admitted request advances in chunks of slices: each chunk is one launch of
// the integrator over the request's slot range (captured once as a CUDA graph
// at admission and replayed), on one of the server's streams.  The chunk
// length is fixed (`slice_periods`) or tuned per request (slice_periods = 0):
// each chunk is timed with events and the next one is sized so that a chunk
// takes about kChunkTargetMs -- long enough to amortise the launch and the
// host's polling, short enough that a finished request is noticed soon.
// Chunks of different requests and models run concurrently on the device; a
// request's next chunk is launched as soon as its previous chunk completes,
// so requests never wait for each other's slow systems.  A finished request is
// copied out asynchronously on its stream; its slots return to the free list
// only once that copy has completed (its event has fired), because the next
// occupant of the range may be admitted on another stream, whose copies and
// launches stream order would not keep behind the pending copy.
//
// Each system's arithmetic does not depend on its slot, its neighbours or the
// chunk boundaries (every slice restarts from its own state), so a request's
// results are the same alone and in any mix.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/odegpu.h"
#include "common.cuh"

using namespace odegpu;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// One-thread-per-system kernel (no work queue) of a model.
const void* kernel_of(int model, int scheme, int prec) { return kernel_for(model, scheme, prec, 0); }

__global__ void fill_int_kernel(int* p, int n, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

enum ReqState { kWaiting = 0, kRunning = 1, kDone = 2 };

struct Request {
  long long ticket = 0;
  int model = 0;
  int n = 0;
  int periods = 0;
  int scheduled = 0;  // periods enqueued in chunks so far
  int chunk = 1;      // slices in the next chunk
  int graph_chunk = 0;  // slices the instantiated graph runs
  cudaGraph_t graph_def = nullptr;  // the captured graph (kept: owns the node)
  cudaGraphNode_t node = nullptr;    // its kernel node
  cudaKernelNodeParams kp;           // the node's launch (function, grid, block)
  KArgs args;                        // its arguments (n_slices updated per chunk)
  int off = -1;       // first slot
  int state = kWaiting;
  bool harvesting = false;
  double t_submit = 0, t_done = 0;
  // pinned host buffers: inputs [2 + n_sys + P][n], outputs
  double* h_in = nullptr;
  double* h_out = nullptr;  // td [2][n], y [n_sys][n], acc [A][n]
  int* h_status = nullptr;
  long long* h_acc_steps = nullptr;
  cudaEvent_t done_ev = nullptr;   // results copied out
  cudaEvent_t chunk_ev = nullptr;  // last chunk finished
  cudaEvent_t start_ev = nullptr;  // last chunk started (tuned chunk length)
  cudaStream_t stream = nullptr;   // borrowed from the server's stream set
  cudaGraphExec_t graph = nullptr; // one chunk of this request
  bool chunk_inflight = false;
};

struct Pool {
  bool on = false;
  int model = 0, scheme = 0, prec = 0;
  int n = 0, P = 0, A = 0, E = 0;
  int cap = 0;
  double h0 = 0;
  Props pr;
  double time_limit_s = 600;
  double *td = nullptr, *y = nullptr, *p = nullptr, *acc = nullptr;
  int *status = nullptr, *ecnt = nullptr, *left = nullptr;
  long long *nacc = nullptr, *nrej = nullptr;
  unsigned char* head = nullptr;  // watchdog flag
  std::map<int, int> free_ranges;  // offset -> length
  std::deque<Request*> waiting;
  std::vector<Request*> running;
  size_t bytes = 0;
  long long chunks = 0;
};

constexpr int kStreams = 32;
constexpr double kChunkTargetMs = 25.0;  // tuned chunks: aimed duration
constexpr int kMaxChunk = 4096;

}  // namespace

struct ode_server {
  int device = 0;
  int slice_periods = 1;
  long long budget = 0;
  long long used = 0;
  Pool pools[kNumModels];
  cudaStream_t streams[kStreams] = {};
  int next_stream = 0;
  std::map<long long, Request*> reqs;
  long long next_ticket = 1;
  std::string err;
};

namespace {

int sfail(ode_server* s, int code, const std::string& m) {
  if (s) s->err = m;
  return code;
}

int scuda(ode_server* s, cudaError_t e, const char* where) {
  return sfail(s, e == cudaErrorMemoryAllocation ? ODE_ERR_OUT_OF_MEMORY : ODE_ERR_CUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

#define SCK(s, call)                                        \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return scuda((s), e_, #call);    \
  } while (0)

size_t per_system_bytes(int n, int P, int A, int E) {
  return sizeof(double) * (2 + n + P + A) + sizeof(int) * (2 + E) + 2 * sizeof(long long);
}

// first-fit range allocator over the pool's slots
int take_range(Pool& pl, int len) {
  for (auto it = pl.free_ranges.begin(); it != pl.free_ranges.end(); ++it) {
    if (it->second >= len) {
      const int off = it->first, rest = it->second - len;
      pl.free_ranges.erase(it);
      if (rest > 0) pl.free_ranges[off + len] = rest;
      return off;
    }
  }
  return -1;
}

void give_range(Pool& pl, int off, int len) {
  auto it = pl.free_ranges.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != pl.free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    pl.free_ranges.erase(nx);
  }
  if (it != pl.free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      pl.free_ranges.erase(it);
    }
  }
}

// Capture one chunk of a request: slice_periods slices (at most the request's
// remaining ones, via the per-slot counts) of its slot range.
int build_request_graph(ode_server* s, Pool& pl, Request* r) {
  const void* fn = kernel_of(pl.model, pl.scheme, pl.prec);
  const size_t off = (size_t)r->off;
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.N = r->n;
  a.ld = pl.cap;
  a.td = pl.td + off;
  a.y = pl.y + off;
  a.p = pl.p + off;
  a.acc = pl.acc + off;
  a.status = pl.status + off;
  a.ecnt = pl.ecnt + off;
  a.nacc = pl.nacc + off;
  a.nrej = pl.nrej + off;
  a.records = nullptr;
  a.n_slices = r->chunk;
  a.n_skip = r->chunk;
  a.h0 = pl.h0;
  a.slices_left = pl.left + off;
  a.queue_head = nullptr;
  a.queue_stride = 1u;
  a.flags = (int*)(pl.head + 64);
  a.time_limit_ns = (long long)(pl.time_limit_s * 1e9);
  a.pr = pl.pr;
  const int block = 64;  // one thread per system, no work queue
  const unsigned grid = (unsigned)((r->n + block - 1) / block);
  cudaGraph_t g = nullptr;
  SCK(s, cudaGraphCreate(&g, 0));
  void* args[] = {&a};
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.func = (void*)fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  cudaError_t e = cudaGraphAddKernelNode(&r->node, g, nullptr, 0, &kp);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&r->graph, g, 0);
  r->graph_def = g;  // kept with the request: its node is updated per chunk
  if (e != cudaSuccess) return scuda(s, e, "chunk graph");
  r->kp = kp;
  r->kp.kernelParams = nullptr;
  r->args = a;
  r->graph_chunk = r->chunk;
  return ODE_OK;
}

void free_request(Request* r) {
  if (r->h_in) cudaFreeHost(r->h_in);
  if (r->h_out) cudaFreeHost(r->h_out);
  if (r->h_status) cudaFreeHost(r->h_status);
  if (r->h_acc_steps) cudaFreeHost(r->h_acc_steps);
  if (r->done_ev) cudaEventDestroy(r->done_ev);
  if (r->chunk_ev) cudaEventDestroy(r->chunk_ev);
  if (r->start_ev) cudaEventDestroy(r->start_ev);
  if (r->graph) cudaGraphExecDestroy(r->graph);
  if (r->graph_def) cudaGraphDestroy(r->graph_def);
  delete r;
}

// Copy a request's inputs into its slot range and arm its slice count.
int launch_chunk(ode_server* s, Pool& pl, Request* r) {
  if (r->chunk != r->graph_chunk) {
    // same node, new slice count: update the executable graph in place
    r->args.n_slices = r->chunk;
    r->args.n_skip = r->chunk;
    void* args[] = {&r->args};
    cudaKernelNodeParams kp = r->kp;
    kp.kernelParams = args;
    SCK(s, cudaGraphExecKernelNodeSetParams(r->graph, r->node, &kp));
    r->graph_chunk = r->chunk;
  }
  if (s->slice_periods == 0) SCK(s, cudaEventRecord(r->start_ev, r->stream));
  SCK(s, cudaGraphLaunch(r->graph, r->stream));
  SCK(s, cudaEventRecord(r->chunk_ev, r->stream));
  r->chunk_inflight = true;
  r->scheduled += r->chunk;
  pl.chunks++;
  return ODE_OK;
}

// Tuned chunk length: scale the last chunk's slice count towards the target
// duration (at most 4x up or down per step).
void retune_chunk(Request* r) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, r->start_ev, r->chunk_ev) != cudaSuccess || !(ms > 0.f)) return;
  double f = kChunkTargetMs / (double)ms;
  f = f > 4.0 ? 4.0 : (f < 0.25 ? 0.25 : f);
  int c = (int)floor(r->chunk * f + 0.5);
  c = c < 1 ? 1 : (c > kMaxChunk ? kMaxChunk : c);
  r->chunk = c;
}

int admit(ode_server* s, Pool& pl, Request* r) {
  const size_t n = (size_t)r->n, cap = (size_t)pl.cap;
  const size_t row = n * sizeof(double), pitch = cap * sizeof(double);
  const double* in = r->h_in;
  r->stream = s->streams[s->next_stream];
  s->next_stream = (s->next_stream + 1) % kStreams;
  cudaStream_t st = r->stream;
  SCK(s, cudaMemcpy2DAsync(pl.td + r->off, pitch, in, row, row, 2, cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpy2DAsync(pl.y + r->off, pitch, in + 2 * n, row, row, pl.n, cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpy2DAsync(pl.p + r->off, pitch, in + (2 + pl.n) * n, row, row, pl.P,
                           cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemsetAsync(pl.nacc + r->off, 0, n * sizeof(long long), st));
  SCK(s, cudaMemsetAsync(pl.nrej + r->off, 0, n * sizeof(long long), st));
  fill_int_kernel<<<(r->n + 255) / 256 < 1024 ? (r->n + 255) / 256 : 1024, 256, 0, st>>>(
      pl.left + r->off, r->n, r->periods);
  SCK(s, cudaGetLastError());
  r->chunk = s->slice_periods > 0 ? s->slice_periods : 1;
  if (int rc = build_request_graph(s, pl, r)) return rc;
  r->state = kRunning;
  r->scheduled = 0;
  pl.running.push_back(r);
  return launch_chunk(s, pl, r);
}

// Copy a finished request's results out (after its last chunk, in stream order).
int harvest(ode_server* s, Pool& pl, Request* r) {
  const size_t n = (size_t)r->n, cap = (size_t)pl.cap;
  const size_t row = n * sizeof(double), pitch = cap * sizeof(double);
  double* out = r->h_out;
  cudaStream_t stream = r->stream;
  SCK(s, cudaMemcpy2DAsync(out, row, pl.td + r->off, pitch, row, 2, cudaMemcpyDeviceToHost, stream));
  SCK(s, cudaMemcpy2DAsync(out + 2 * n, row, pl.y + r->off, pitch, row, pl.n, cudaMemcpyDeviceToHost,
                           stream));
  SCK(s, cudaMemcpy2DAsync(out + (2 + pl.n) * n, row, pl.acc + r->off, pitch, row, pl.A,
                           cudaMemcpyDeviceToHost, stream));
  SCK(s, cudaMemcpyAsync(r->h_status, pl.status + r->off, n * sizeof(int), cudaMemcpyDeviceToHost,
                         stream));
  SCK(s, cudaMemcpyAsync(r->h_acc_steps, pl.nacc + r->off, n * sizeof(long long),
                         cudaMemcpyDeviceToHost, stream));
  SCK(s, cudaEventRecord(r->done_ev, stream));
  r->harvesting = true;
  // the slot range is released in release_harvested(), after done_ev
  return ODE_OK;
}

// Requests whose results have arrived: mark them done and only now return
// their slot ranges to the pool's free list.
int release_harvested(ode_server* s) {
  for (auto& kv : s->reqs) {
    Request* r = kv.second;
    if (!r->harvesting || r->state == kDone) continue;
    cudaError_t q = cudaEventQuery(r->done_ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return scuda(s, q, "harvest");
    r->state = kDone;
    r->t_done = now_s();
    give_range(s->pools[r->model], r->off, r->n);
  }
  return ODE_OK;
}

}  // namespace

extern "C" {

int ode_server_create(ode_server** out, int device, long long hbm_budget_bytes, int slice_periods) {
  if (!out) return ODE_ERR_INVALID_ARG;
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || slice_periods < 0) return ODE_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ODE_ERR_CUDA;
  ode_server* s = new (std::nothrow) ode_server();
  if (!s) return ODE_ERR_OUT_OF_MEMORY;
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->slice_periods = slice_periods;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete s;
    return ODE_ERR_CUDA;
  }
  for (int i = 0; i < kStreams; i++) {
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      ode_server_destroy(s);
      return ODE_ERR_CUDA;
    }
  }
  *out = s;
  return ODE_OK;
}

int ode_server_add_model(ode_server* s, const ode_noalloc_settings* cfg, double h0, int capacity) {
  if (!s) return ODE_ERR_INVALID_ARG;
  if (!cfg) return sfail(s, ODE_ERR_INVALID_ARG, "settings are NULL");
  int n, P, A, E;
  if (!model_dims(cfg->model, &n, &P, &A, &E)) return sfail(s, ODE_ERR_INVALID_ARG, "unknown model");
  Pool& pl = s->pools[cfg->model];
  if (pl.on) return sfail(s, ODE_ERR_INVALID_ARG, "model already added");
  const void* fn = kernel_of(cfg->model, cfg->scheme, cfg->prec);
  if (!fn) return sfail(s, ODE_ERR_INVALID_ARG, "no kernel for this model / scheme / precision");
  if (capacity < 1) return sfail(s, ODE_ERR_INVALID_ARG, "capacity must be >= 1");
  if (!(h0 > 0.0)) return sfail(s, ODE_ERR_INVALID_ARG, "h0 must be > 0");
  if (!(cfg->h_min > 0.0) || !(cfg->h_max >= cfg->h_min) || !(cfg->grow_limit >= 1.0) ||
      !(cfg->grow_limit <= 1e4) || !(cfg->shrink_limit >= 1e-4) || !(cfg->shrink_limit <= 1.0) ||
      cfg->max_steps_per_slice < 1)
    return sfail(s, ODE_ERR_INVALID_ARG, "invalid step-size settings");
  const size_t bytes = per_system_bytes(n, P, A, E) * (size_t)capacity + 256;
  if (s->used + (long long)bytes > s->budget)
    return sfail(s, ODE_ERR_OUT_OF_MEMORY, "pool does not fit in the server's HBM budget");
  if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, ODE_ERR_CUDA, "cudaSetDevice failed");
  pl.model = cfg->model;
  pl.scheme = cfg->scheme;
  pl.prec = cfg->prec;
  pl.n = n;
  pl.P = P;
  pl.A = A;
  pl.E = E;
  pl.cap = capacity;
  pl.h0 = h0;
  pl.time_limit_s = cfg->time_limit_s;
  Props& pr = pl.pr;
  memset(&pr, 0, sizeof(pr));
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
  const size_t C = (size_t)capacity;
  struct {
    void** p;
    size_t b;
  } al[] = {{(void**)&pl.td, 2 * C * sizeof(double)},     {(void**)&pl.y, n * C * sizeof(double)},
            {(void**)&pl.p, P * C * sizeof(double)},      {(void**)&pl.acc, A * C * sizeof(double)},
            {(void**)&pl.status, C * sizeof(int)},         {(void**)&pl.ecnt, E * C * sizeof(int)},
            {(void**)&pl.left, C * sizeof(int)},           {(void**)&pl.nacc, C * sizeof(long long)},
            {(void**)&pl.nrej, C * sizeof(long long)},     {(void**)&pl.head, 256}};
  for (auto& x : al) {
    SCK(s, cudaMalloc(x.p, x.b));
    SCK(s, cudaMemset(*x.p, 0, x.b));
  }
  pl.free_ranges.clear();
  pl.free_ranges[0] = capacity;
  pl.bytes = bytes;
  s->used += (long long)bytes;
  pl.on = true;
  return ODE_OK;
}

int ode_server_submit(ode_server* s, int model, int n_systems, int n_periods, const double* td,
                      const double* y0, const double* p, long long* ticket) {
  if (!s) return ODE_ERR_INVALID_ARG;
  if (model < 0 || model >= kNumModels || !s->pools[model].on)
    return sfail(s, ODE_ERR_INVALID_ARG, "model not served (ode_server_add_model)");
  Pool& pl = s->pools[model];
  if (n_systems < 1 || n_systems > pl.cap)
    return sfail(s, ODE_ERR_INVALID_ARG, "request size outside [1, pool capacity]");
  if (n_periods < 1) return sfail(s, ODE_ERR_INVALID_ARG, "n_periods must be >= 1");
  if (!td || !y0 || !p || !ticket) return sfail(s, ODE_ERR_INVALID_ARG, "NULL argument");
  if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, ODE_ERR_CUDA, "cudaSetDevice failed");
  Request* r = new (std::nothrow) Request();
  if (!r) return sfail(s, ODE_ERR_OUT_OF_MEMORY, "host allocation failed");
  r->model = model;
  r->n = n_systems;
  r->periods = n_periods;
  const size_t n = (size_t)n_systems;
  cudaError_t e = cudaMallocHost(&r->h_in, (2 + pl.n + pl.P) * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&r->h_out, (2 + pl.n + pl.A) * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&r->h_status, n * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&r->h_acc_steps, n * sizeof(long long));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
  // timing events only where the chunk length is tuned
  const unsigned ev_flags = s->slice_periods == 0 ? cudaEventDefault : cudaEventDisableTiming;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->chunk_ev, ev_flags);
  if (e == cudaSuccess && s->slice_periods == 0) e = cudaEventCreateWithFlags(&r->start_ev, ev_flags);
  if (e != cudaSuccess) {
    free_request(r);
    return scuda(s, e, "request buffers");
  }
  memcpy(r->h_in, td, 2 * n * sizeof(double));
  memcpy(r->h_in + 2 * n, y0, pl.n * n * sizeof(double));
  memcpy(r->h_in + (2 + pl.n) * n, p, pl.P * n * sizeof(double));
  r->ticket = s->next_ticket++;
  r->t_submit = now_s();
  s->reqs[r->ticket] = r;
  pl.waiting.push_back(r);
  *ticket = r->ticket;
  return ODE_OK;
}

int ode_server_progress(ode_server* s, int* n_running, int* n_waiting) {
  if (!s) return ODE_ERR_INVALID_ARG;
  if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, ODE_ERR_CUDA, "cudaSetDevice failed");
  int running = 0, waiting = 0;
  // 0. finished copies out free their slots before anything is admitted
  if (int rc = release_harvested(s)) return rc;
  for (Pool& pl : s->pools) {
    if (!pl.on) continue;
    // 1. requests whose chunk finished: next chunk, or copy out when done
    std::vector<Request*> still;
    for (Request* r : pl.running) {
      if (r->chunk_inflight) {
        cudaError_t q = cudaEventQuery(r->chunk_ev);
        if (q == cudaErrorNotReady) {
          still.push_back(r);
          continue;
        }
        if (q != cudaSuccess) return scuda(s, q, "chunk");
        r->chunk_inflight = false;
        if (s->slice_periods == 0) retune_chunk(r);
      }
      if (r->scheduled >= r->periods) {
        if (int rc = harvest(s, pl, r)) return rc;
      } else {
        if (int rc = launch_chunk(s, pl, r)) return rc;
        still.push_back(r);
      }
    }
    pl.running.swap(still);
    // 2. admit waiting requests in arrival order while slots are free
    while (!pl.waiting.empty()) {
      Request* r = pl.waiting.front();
      const int off = take_range(pl, r->n);
      if (off < 0) break;
      r->off = off;
      pl.waiting.pop_front();
      if (int rc = admit(s, pl, r)) return rc;
    }
    running += (int)pl.running.size();
    waiting += (int)pl.waiting.size();
  }
  // 3. requests whose results have arrived in this pass
  if (int rc = release_harvested(s)) return rc;
  if (n_running) *n_running = running;
  if (n_waiting) *n_waiting = waiting;
  return ODE_OK;
}

int ode_server_poll(ode_server* s, long long ticket, int* state) {
  if (!s || !state) return ODE_ERR_INVALID_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(s, ODE_ERR_INVALID_ARG, "unknown ticket");
  *state = it->second->state;
  return ODE_OK;
}

int ode_server_result(ode_server* s, long long ticket, double* td, double* y, double* acc,
                      int* status, long long* accepted, double* latency_s) {
  if (!s) return ODE_ERR_INVALID_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(s, ODE_ERR_INVALID_ARG, "unknown ticket");
  Request* r = it->second;
  if (r->state != kDone) return sfail(s, ODE_ERR_NOT_READY, "request not finished");
  const Pool& pl = s->pools[r->model];
  const size_t n = (size_t)r->n;
  if (td) memcpy(td, r->h_out, 2 * n * sizeof(double));
  if (y) memcpy(y, r->h_out + 2 * n, pl.n * n * sizeof(double));
  if (acc) memcpy(acc, r->h_out + (2 + pl.n) * n, pl.A * n * sizeof(double));
  if (status) memcpy(status, r->h_status, n * sizeof(int));
  if (accepted) memcpy(accepted, r->h_acc_steps, n * sizeof(long long));
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  s->reqs.erase(it);
  free_request(r);
  return ODE_OK;
}

int ode_server_destroy(ode_server* s) {
  if (!s) return ODE_OK;
  cudaSetDevice(s->device);
  for (int i = 0; i < kStreams; i++)
    if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
  for (auto& kv : s->reqs) free_request(kv.second);
  for (Pool& pl : s->pools) {
    void* ptrs[] = {pl.td, pl.y, pl.p, pl.acc, pl.status, pl.ecnt, pl.left, pl.nacc, pl.nrej, pl.head};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  for (int i = 0; i < kStreams; i++)
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
  delete s;
  return ODE_OK;
}

const char* ode_server_last_error(const ode_server* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
