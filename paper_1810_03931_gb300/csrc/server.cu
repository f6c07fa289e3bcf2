// server.cu -- continuous-batching request loop for parameter-sweep requests,
// built on the resident serving kernel of serve.cuh.
//
// Each served model has a pool of system slots in HBM (capacity chosen by the
// caller within the server's HBM budget: admission by footprint) and, while
// it has work, one or more resident instances of its serving kernel.  A
// request -- n systems of one model, each integrated over n_periods slices --
// waits (FIFO per model) until a contiguous range of n free slots exists.
// Admission copies its inputs, slice budgets and request-table entry into the
// range; its slot indices are then published to the model's ring, from which
// the kernel's threads take systems the moment they free up.  A thread runs a
// system for its whole horizon (or for slice_periods slices, after which the
// system goes back through the host to the ring: time slicing), stores it
// and counts it in its request's done counter.  When a request's count
// reaches n, its results are copied out (pinned D2H) and, once that copy has
// completed, its slots return to the free list.  Requests that arrive while
// others run are merged into the same launch: there is one launch per model
// and residency, not per request.
//
// The host side never blocks: ode_server_progress takes one asynchronous
// snapshot of the done counters and the yield list per call, publishes ring
// entries, starts kernel instances and copies results out.  Blocks are split
// between models with work in equal shares; a model that gets work while the
// others hold the GPU has them stop at their next slice boundary (their
// systems come back through the yield list) and all are relaunched with the
// new split.  Every system's arithmetic is that of ode_run_periods, so a
// request's results are the same alone and in any mix.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <climits>
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

enum ReqState { kWaiting = 0, kRunning = 1, kDone = 2 };

constexpr int kMaxReq = 4096;         // request-table entries per model (done counters)
constexpr int kTailWords = 256;       // pinned words for ring-tail publishes
constexpr int kThreads = 128;         // threads per block of the serving kernel
constexpr long long kIdleNs = 2000000;  // a warp without work exits after 2 ms

// Pinned host buffers are recycled by size class instead of freed:
// cudaFreeHost waits for the device, which would stall every request's result
// behind the resident kernels.  Buffers go back to the server's cache and are
// released only when the server is destroyed.
struct PinnedCache {
  std::map<size_t, std::vector<void*>> free_lists;
  static size_t klass(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
  }
  cudaError_t get(void** p, size_t bytes) {
    auto& fl = free_lists[klass(bytes)];
    if (!fl.empty()) {
      *p = fl.back();
      fl.pop_back();
      return cudaSuccess;
    }
    return cudaMallocHost(p, klass(bytes));
  }
  void put(void* p, size_t bytes) {
    if (p) free_lists[klass(bytes)].push_back(p);
  }
  void release() {
    for (auto& kv : free_lists)
      for (void* p : kv.second) cudaFreeHost(p);
    free_lists.clear();
  }
};

struct Request {
  long long ticket = 0;
  int model = 0;
  int n = 0;
  int periods = 0;
  int off = -1;            // first slot
  int tix = -1;            // request-table entry
  unsigned int base = 0;   // done counter value when admitted
  int fresh = 0;           // systems admitted but not yet published to the ring
  std::deque<int> yielded; // its slots handed back by the kernel, to publish again
  bool in_feed = false;
  int state = kWaiting;
  bool harvesting = false;
  double t_submit = 0, t_done = 0;
  // pinned host buffers: inputs [2 + n_sys + P][n], budgets and table
  // entries [2][n] (int), zero counters [2][n] (long long), outputs
  double* h_in = nullptr;
  int* h_meta = nullptr;
  long long* h_zero = nullptr;
  double* h_out = nullptr;  // td [2][n], y [n_sys][n], acc [A][n]
  int* h_status = nullptr;
  long long* h_acc_steps = nullptr;
  cudaEvent_t done_ev = nullptr;  // results copied out
  size_t b_in = 0, b_meta = 0, b_zero = 0, b_out = 0, b_status = 0, b_steps = 0;  // buffer sizes
};

struct Instance {
  cudaEvent_t ev = nullptr;  // completion
  int blocks = 0;
  int lanes_per_warp = 32;   // threads per warp that take systems
  bool live = false;
};

struct Pool {
  bool on = false;
  int model = 0, scheme = 0, prec = 0;
  int n = 0, P = 0, A = 0, E = 0;
  int cap = 0;
  double h0 = 0;
  Props pr;
  double time_limit_s = 600;
  const void* fn = nullptr;
  int bps = 0;  // resident blocks per SM of the serving kernel
  // device
  double *td = nullptr, *y = nullptr, *p = nullptr, *acc = nullptr;
  int *status = nullptr, *ecnt = nullptr, *left = nullptr, *owner = nullptr;
  long long *nacc = nullptr, *nrej = nullptr;
  unsigned int* ring = nullptr;
  unsigned int* ctl = nullptr;
  unsigned long long* yl = nullptr;
  unsigned int* done = nullptr;
  unsigned int ring_cap = 0, yl_cap = 0;
  // host
  std::map<int, int> free_ranges;  // offset -> length
  std::vector<int> free_tix;
  std::vector<unsigned int> tix_base;  // done counter value after the last occupant
  std::deque<Request*> waiting;
  std::vector<Request*> running;       // admitted, not finished
  std::deque<Request*> feed;           // admitted requests with systems to publish (round robin)
  std::vector<Request*> slot_req;      // request holding each slot
  unsigned int tail = 0;               // ring entries published
  unsigned int yl_read = 0;            // yield-list entries taken back
  unsigned int* h_ring = nullptr;      // pinned staging of ring entries [ring_cap]
  unsigned int* h_tail = nullptr;      // pinned words for tail publishes [kTailWords]
  cudaEvent_t tail_ev[kTailWords] = {};
  int tail_next = 0;
  unsigned int* h_ctl = nullptr;       // pinned snapshot of the control block
  unsigned int* h_done = nullptr;      // pinned snapshot of the done counters
  unsigned long long* h_yl = nullptr;  // pinned snapshot of the yield list [yl_cap]
  unsigned int snap_yl_lo = 0, snap_yl_hi = 0;  // yield-list range in the snapshot
  unsigned int* h_flag = nullptr;      // pinned stop-flag words [2]: 0 and 1
  cudaEvent_t snap_ev = nullptr;
  bool snap_inflight = false;
  bool snap_valid = false;
  unsigned int known_yield_tail = 0;   // from the last snapshot
  cudaStream_t cstream = nullptr;      // the server's copy stream (shared by the pools)
  cudaStream_t kstream = nullptr;      // the serving kernel's stream
  Instance inst;                       // the resident instance (at most one)
  bool stopping = false;               // stop flag raised for a rebalance
  int target_blocks = 0;
  long long unfinished = 0;            // systems admitted and not yet counted done
  size_t bytes = 0;
  long long launches = 0;   // serving-kernel instances started
  long long stops = 0;      // stop requests (rebalancing)
  long long yielded = 0;    // systems taken back from the yield list
  long long snapshots = 0;  // snapshots read
  long long published = 0;  // ring entries published
  long long finished = 0;   // requests copied out
  unsigned int flags = 0;   // watchdog / bounds flags seen
};

}  // namespace

struct ode_server {
  int device = 0;
  int slice_periods = 0;
  int sms = 0;
  // Few streams on purpose: streams share the device's hardware work queues,
  // and a copy queued behind a resident kernel in the same queue would wait
  // for the kernel to end.  One copy stream for all pools and one kernel
  // stream per pool stay within the default number of queues.
  cudaStream_t cstream = nullptr;
  long long budget = 0;
  long long used = 0;
  Pool pools[kNumModels];
  PinnedCache pinned;
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

// device bytes per slot: time domain, state, parameters, accessories, status,
// event counters, slice budget, owner, two step counters, a ring entry and a
// yield-list entry
size_t per_system_bytes(int n, int P, int A, int E) {
  return sizeof(double) * (2 + n + P + A) + sizeof(int) * (3 + E) + 2 * sizeof(long long) +
         sizeof(unsigned int) + sizeof(unsigned long long);
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

void free_request(PinnedCache& pc, Request* r) {
  pc.put(r->h_in, r->b_in);
  pc.put(r->h_meta, r->b_meta);
  pc.put(r->h_zero, r->b_zero);
  pc.put(r->h_out, r->b_out);
  pc.put(r->h_status, r->b_status);
  pc.put(r->h_acc_steps, r->b_steps);
  if (r->done_ev) cudaEventDestroy(r->done_ev);
  delete r;
}

}  // namespace

namespace {

// Copy a request's inputs, slice budgets, request-table entry and zero step
// counters into its slot range (on the pool's copy stream).
int admit(ode_server* s, Pool& pl, Request* r) {
  const size_t n = (size_t)r->n, cap = (size_t)pl.cap;
  const size_t row = n * sizeof(double), pitch = cap * sizeof(double);
  const size_t irow = n * sizeof(int), ipitch = cap * sizeof(int);
  cudaStream_t st = s->cstream;
  r->tix = pl.free_tix.back();
  pl.free_tix.pop_back();
  r->base = pl.tix_base[r->tix];
  for (size_t i = 0; i < n; i++) {
    r->h_meta[i] = r->periods;        // slice budget
    r->h_meta[n + i] = r->tix;        // request-table entry
  }
  const double* in = r->h_in;
  SCK(s, cudaMemcpy2DAsync(pl.td + r->off, pitch, in, row, row, 2, cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpy2DAsync(pl.y + r->off, pitch, in + 2 * n, row, row, pl.n, cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpy2DAsync(pl.p + r->off, pitch, in + (2 + pl.n) * n, row, row, pl.P,
                           cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpyAsync(pl.left + r->off, r->h_meta, irow, cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpyAsync(pl.owner + r->off, r->h_meta + n, irow, cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpyAsync(pl.nacc + r->off, r->h_zero, n * sizeof(long long), cudaMemcpyHostToDevice, st));
  SCK(s, cudaMemcpyAsync(pl.nrej + r->off, r->h_zero + n, n * sizeof(long long), cudaMemcpyHostToDevice, st));
  (void)ipitch;
  r->state = kRunning;
  r->fresh = r->n;
  for (int i = 0; i < r->n; i++) pl.slot_req[r->off + i] = r;
  pl.running.push_back(r);
  r->in_feed = true;
  pl.feed.push_back(r);
  pl.unfinished += r->n;
  return ODE_OK;
}

// From the last snapshot: ring entries published but not yet taken, and the
// threads of the running instance without a system (claimed entries minus
// systems finished -- the sum of the monotone done counters -- minus systems
// handed back).
unsigned int ring_outstanding(const Pool& pl) {
  const unsigned int head = pl.snap_valid ? pl.h_ctl[kCtlRingHead] : 0u;
  return pl.tail - head;
}

long long idle_threads(const Pool& pl) {
  const long long lanes =
      pl.inst.live ? (long long)pl.inst.blocks * (kThreads / 32) * pl.inst.lanes_per_warp : 0;
  if (!pl.snap_valid) return lanes;
  unsigned int done = 0;
  for (int t = 0; t < kMaxReq; t++) done += pl.h_done[t];
  const unsigned int in_flight = pl.h_ctl[kCtlRingHead] - done - pl.h_ctl[kCtlYieldTail];
  return std::max(0LL, lanes - (long long)in_flight);
}

// Publish slots to the ring, round robin over the requests that have systems
// to run (their yielded systems first, then fresh ones), in chunks of
// kChunk, and only as many as the running instance has idle threads plus a
// margin: a request that arrives later is then never queued behind the whole
// of an earlier one.  Entries are staged in pinned memory at their ring
// positions and copied, then the new tail is copied from a pinned word of
// its own (a word is reused only after its copy has completed).
int publish(ode_server* s, Pool& pl) {
  const int w = pl.tail_next;
  if (pl.tail_ev[w]) {
    cudaError_t q = cudaEventQuery(pl.tail_ev[w]);
    if (q == cudaErrorNotReady) return ODE_OK;  // try again on the next pass
    if (q != cudaSuccess) return scuda(s, q, "ring tail copy");
  }
  constexpr long long kMargin = 512;
  constexpr int kChunk = 256;
  long long room = idle_threads(pl) + kMargin - (long long)ring_outstanding(pl);
  const unsigned int first = pl.tail;
  unsigned int k = 0;
  while (room > 0 && !pl.feed.empty()) {
    Request* r = pl.feed.front();
    pl.feed.pop_front();
    int take = 0;
    while (take < kChunk && room > 0 && !r->yielded.empty()) {
      pl.h_ring[(first + k) % pl.ring_cap] = (unsigned int)r->yielded.front();
      r->yielded.pop_front();
      k++, take++, room--;
    }
    while (take < kChunk && room > 0 && r->fresh > 0) {
      pl.h_ring[(first + k) % pl.ring_cap] = (unsigned int)(r->off + (r->n - r->fresh));
      r->fresh--;
      k++, take++, room--;
    }
    r->in_feed = r->fresh > 0 || !r->yielded.empty();
    if (r->in_feed) pl.feed.push_back(r);
  }
  if (k == 0) return ODE_OK;
  // one or two contiguous segments of the ring
  const unsigned int a0 = first % pl.ring_cap;
  const unsigned int n0 = std::min(k, pl.ring_cap - a0);
  SCK(s, cudaMemcpyAsync(pl.ring + a0, pl.h_ring + a0, n0 * sizeof(unsigned int), cudaMemcpyHostToDevice,
                         s->cstream));
  if (n0 < k)
    SCK(s, cudaMemcpyAsync(pl.ring, pl.h_ring, (k - n0) * sizeof(unsigned int), cudaMemcpyHostToDevice,
                           s->cstream));
  pl.tail = first + k;
  pl.published += k;
  pl.h_tail[w] = pl.tail;
  SCK(s, cudaMemcpyAsync(pl.ctl + kCtlRingTail, pl.h_tail + w, sizeof(unsigned int), cudaMemcpyHostToDevice,
                         s->cstream));
  SCK(s, cudaEventRecord(pl.tail_ev[w], s->cstream));
  pl.tail_next = (w + 1) % kTailWords;
  return ODE_OK;
}

// Copy a finished request's results out (pinned D2H on the copy stream).
int harvest(ode_server* s, Pool& pl, Request* r) {
  const size_t n = (size_t)r->n, cap = (size_t)pl.cap;
  const size_t row = n * sizeof(double), pitch = cap * sizeof(double);
  double* out = r->h_out;
  cudaStream_t st = s->cstream;
  SCK(s, cudaMemcpy2DAsync(out, row, pl.td + r->off, pitch, row, 2, cudaMemcpyDeviceToHost, st));
  SCK(s, cudaMemcpy2DAsync(out + 2 * n, row, pl.y + r->off, pitch, row, pl.n, cudaMemcpyDeviceToHost, st));
  SCK(s, cudaMemcpy2DAsync(out + (2 + pl.n) * n, row, pl.acc + r->off, pitch, row, pl.A,
                           cudaMemcpyDeviceToHost, st));
  SCK(s, cudaMemcpyAsync(r->h_status, pl.status + r->off, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  SCK(s, cudaMemcpyAsync(r->h_acc_steps, pl.nacc + r->off, n * sizeof(long long), cudaMemcpyDeviceToHost,
                         st));
  SCK(s, cudaEventRecord(r->done_ev, st));
  r->harvesting = true;
  pl.unfinished -= r->n;
  pl.finished++;
  return ODE_OK;
}

// Requests whose results have arrived: mark them done and only now return
// their slots and request-table entries (the copy out has completed, so a
// later admission into the same range cannot overwrite results in flight).
int release_harvested(ode_server* s) {
  for (auto& kv : s->reqs) {
    Request* r = kv.second;
    if (!r->harvesting || r->state == kDone) continue;
    cudaError_t q = cudaEventQuery(r->done_ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return scuda(s, q, "harvest");
    r->state = kDone;
    r->t_done = now_s();
    Pool& pl = s->pools[r->model];
    give_range(pl, r->off, r->n);
    pl.tix_base[r->tix] = r->base + (unsigned int)r->n;
    pl.free_tix.push_back(r->tix);
  }
  return ODE_OK;
}

// Start an asynchronous snapshot of the control block, the done counters and
// the yield-list entries reserved up to the previous snapshot.
int start_snapshot(ode_server* s, Pool& pl) {
  cudaStream_t st = s->cstream;
  SCK(s, cudaMemcpyAsync(pl.h_ctl, pl.ctl, kCtlWords * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  SCK(s, cudaMemcpyAsync(pl.h_done, pl.done, kMaxReq * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  pl.snap_yl_lo = pl.yl_read;
  pl.snap_yl_hi = pl.known_yield_tail;
  const unsigned int k = pl.snap_yl_hi - pl.snap_yl_lo;
  if (k > 0) {
    const unsigned int a0 = pl.snap_yl_lo % pl.yl_cap;
    const unsigned int n0 = std::min(k, pl.yl_cap - a0);
    SCK(s, cudaMemcpyAsync(pl.h_yl + a0, pl.yl + a0, n0 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           st));
    if (n0 < k)
      SCK(s, cudaMemcpyAsync(pl.h_yl, pl.yl, (k - n0) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             st));
  }
  SCK(s, cudaEventRecord(pl.snap_ev, st));
  pl.snap_inflight = true;
  return ODE_OK;
}

// A completed snapshot: take back yielded slots, copy out finished requests.
int take_snapshot(ode_server* s, Pool& pl) {
  pl.snap_inflight = false;
  pl.snap_valid = true;
  pl.snapshots++;
  pl.flags |= pl.h_ctl[kCtlFlags];
  pl.known_yield_tail = pl.h_ctl[kCtlYieldTail];
  while (pl.yl_read != pl.snap_yl_hi) {
    const unsigned int pos = pl.yl_read;
    const unsigned long long e = pl.h_yl[pos % pl.yl_cap];
    if ((unsigned int)(e >> 32) != pos / pl.yl_cap + 1u) break;  // reserved, not yet written
    const int slot = (int)(e & 0xffffffffu);
    pl.yl_read++;
    Request* r = (slot >= 0 && slot < pl.cap) ? pl.slot_req[slot] : nullptr;
    if (r && r->state == kRunning && !r->harvesting) {
      r->yielded.push_back(slot);
      if (!r->in_feed) {
        r->in_feed = true;
        pl.feed.push_back(r);
      }
    }
    pl.yielded++;
  }
  std::vector<Request*> still;
  for (Request* r : pl.running) {
    const unsigned int cnt = pl.h_done[r->tix] - r->base;
    if (cnt >= (unsigned int)r->n) {
      if (int rc = harvest(s, pl, r)) return rc;
    } else {
      still.push_back(r);
    }
  }
  pl.running.swap(still);
  return ODE_OK;
}

}  // namespace

namespace {

double share_of(const Pool& pl, int blocks, int sms) {
  return pl.bps > 0 ? (double)blocks / ((double)pl.bps * sms) : 0.0;
}

int live_blocks(const Pool& pl) { return pl.inst.live ? pl.inst.blocks : 0; }

// Write the stop flag of a pool (0 or 1) on its copy stream.
int set_stop(ode_server* s, Pool& pl, int v) {
  SCK(s, cudaMemcpyAsync(pl.ctl + kCtlStop, pl.h_flag + (v ? 1 : 0), sizeof(unsigned int),
                         cudaMemcpyHostToDevice, s->cstream));
  pl.stopping = v != 0;
  if (v) pl.stops++;
  return ODE_OK;
}

// Launch the pool's serving kernel with `blocks` blocks on its kernel stream,
// ordered after everything on the copy stream so far (the cleared stop flag,
// admissions, ring entries).
int launch_instance(ode_server* s, Pool& pl, int blocks, int lanes_per_warp) {
  if (pl.inst.live || blocks < 1) return ODE_OK;
  cudaEvent_t ready = nullptr;
  SCK(s, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ready, s->cstream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(pl.kstream, ready, 0);
  cudaEventDestroy(ready);
  if (e != cudaSuccess) return scuda(s, e, "instance ordering");
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.N = pl.cap;
  a.ld = pl.cap;
  a.td = pl.td;
  a.y = pl.y;
  a.p = pl.p;
  a.acc = pl.acc;
  a.status = pl.status;
  a.ecnt = pl.ecnt;
  a.nacc = pl.nacc;
  a.nrej = pl.nrej;
  a.records = nullptr;
  a.n_slices = s->slice_periods > 0 ? s->slice_periods : INT_MAX;  // residency quantum
  a.n_skip = INT_MAX;
  a.h0 = pl.h0;
  a.slices_left = pl.left;
  a.flags = (int*)(pl.ctl + kCtlFlags);
  a.time_limit_ns = (long long)(pl.time_limit_s * 1e9);
  a.pr = pl.pr;
  ServeArgs sv;
  memset(&sv, 0, sizeof(sv));
  sv.ring = pl.ring;
  sv.ring_cap = pl.ring_cap;
  sv.ctl = pl.ctl;
  sv.yl = pl.yl;
  sv.yl_cap = pl.yl_cap;
  sv.done_cnt = pl.done;
  sv.done_cap = kMaxReq;
  sv.owner = pl.owner;
  sv.idle_ns = kIdleNs;
  sv.lanes_per_warp = lanes_per_warp;
  void* args[] = {&a, &sv};
  SCK(s, cudaLaunchKernel(pl.fn, dim3((unsigned)blocks), dim3(kThreads), args, 0, pl.kstream));
  SCK(s, cudaEventRecord(pl.inst.ev, pl.kstream));
  pl.inst.live = true;
  pl.inst.blocks = blocks;
  pl.inst.lanes_per_warp = lanes_per_warp;
  pl.launches++;
  return ODE_OK;
}

// Split the GPU between the models that have work, max-min fair in two
// passes: first the dense demand (the share of the SMs a model's unfinished
// systems fill at one thread per system), smallest first, each model getting
// at most an equal part of what is left; then what is left over goes, the
// same way, to the spread demand (one system per warp).  An instance takes
// systems on as many threads per warp as its share needs.  A model below
// 0.8 x its share is started, or stopped and relaunched larger if the GPU has
// room; otherwise the models above 1.5 x their share stop at their next
// slice boundary (their systems come back through the yield list) and are
// relaunched at their share once their instance has exited.
int manage_instances(ode_server* s) {
  double demand[kNumModels] = {0}, spread[kNumModels] = {0}, target[kNumModels] = {0};
  int order[kNumModels], with_work = 0;
  for (int m = 0; m < kNumModels; m++) {
    Pool& pl = s->pools[m];
    if (!pl.on) continue;
    if (pl.inst.live) {
      cudaError_t q = cudaEventQuery(pl.inst.ev);
      if (q == cudaSuccess) pl.inst.live = false;
      else if (q != cudaErrorNotReady) return scuda(s, q, "serving kernel");
    }
    if (pl.unfinished > 0) {
      const double blocks = ceil((double)pl.unfinished / kThreads);
      demand[m] = std::min(1.0, blocks / ((double)pl.bps * s->sms));
      // spread demand: one system per warp, so that a few slow systems (the
      // tail of a long request) get a scheduler each instead of sharing one
      const double wblocks = ceil((double)pl.unfinished / (kThreads / 32));
      spread[m] = std::min(1.0, wblocks / ((double)pl.bps * s->sms));
      order[with_work++] = m;
    }
  }
  // max-min fair split of the dense demand; what is left over goes to the
  // spread demand (dense packing while the GPU is busy, spreading when SMs
  // would otherwise idle)
  double left = 1.0;
  for (int pass = 0; pass < 2; pass++) {
    double want[kNumModels];
    for (int i = 0; i < with_work; i++) {
      const int m = order[i];
      want[m] = pass == 0 ? demand[m] : std::max(0.0, spread[m] - target[m]);
    }
    std::sort(order, order + with_work, [&](int a, int b) { return want[a] < want[b]; });
    for (int i = 0; i < with_work; i++) {
      const int m = order[i];
      const double g = std::min(want[m], left / (with_work - i));
      target[m] += g;
      left -= g;
    }
  }
  double used = 0.0;
  for (Pool& pl : s->pools)
    if (pl.on) used += share_of(pl, live_blocks(pl), s->sms);
  for (int m = 0; m < kNumModels; m++) {
    Pool& pl = s->pools[m];
    if (!pl.on) continue;
    const int lb = live_blocks(pl);
    if (pl.stopping) {
      if (lb > 0) continue;
      if (int rc = set_stop(s, pl, 0)) return rc;
    }
    if (pl.unfinished <= 0) continue;
    const double have = share_of(pl, lb, s->sms);
    // a running instance whose claiming threads are far fewer than the
    // model's unfinished systems is relaunched (more threads per warp)
    if (pl.inst.live && pl.inst.lanes_per_warp < 32 &&
        (double)pl.unfinished > 2.0 * lb * (kThreads / 32) * pl.inst.lanes_per_warp) {
      if (int rc = set_stop(s, pl, 1)) return rc;
      continue;
    }
    if (have >= 0.8 * target[m]) continue;
    const double want = target[m] - have;
    if (pl.inst.live) {
      // one instance per model: a running one below its share is stopped and
      // relaunched at the share once it has exited (it is not stopped for
      // less than a quarter of the GPU)
      if (want >= 0.25 && used + want <= 1.02)
        if (int rc = set_stop(s, pl, 1)) return rc;
      continue;
    }
    if (used + want <= 1.02) {
      const int blocks = std::max(1, (int)ceil(target[m] * pl.bps * s->sms));
      const long long warps = (long long)blocks * (kThreads / 32);
      const int lpw = (int)std::min<long long>(32, std::max<long long>(1, (pl.unfinished + warps - 1) / warps));
      if (int rc = launch_instance(s, pl, blocks, lpw)) return rc;
      used += share_of(pl, blocks, s->sms);
    } else {
      for (int o = 0; o < kNumModels; o++) {
        Pool& po = s->pools[o];
        if (!po.on || o == m || po.stopping) continue;
        if (share_of(po, live_blocks(po), s->sms) > 1.5 * target[o] + 1e-9)
          if (int rc = set_stop(s, po, 1)) return rc;
      }
    }
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
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return ODE_ERR_CUDA;
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
  const void* fn = kernel_for(cfg->model, cfg->scheme, cfg->prec, 3);
  if (!fn) return sfail(s, ODE_ERR_INVALID_ARG, "no kernel for this model / scheme / precision");
  if (capacity < 1) return sfail(s, ODE_ERR_INVALID_ARG, "capacity must be >= 1");
  if (!(h0 > 0.0)) return sfail(s, ODE_ERR_INVALID_ARG, "h0 must be > 0");
  if (!(cfg->h_min > 0.0) || !(cfg->h_max >= cfg->h_min) || !(cfg->grow_limit >= 1.0) ||
      !(cfg->grow_limit <= 1e4) || !(cfg->shrink_limit >= 1e-4) || !(cfg->shrink_limit <= 1.0) ||
      cfg->max_steps_per_slice < 1)
    return sfail(s, ODE_ERR_INVALID_ARG, "invalid step-size settings");
  const size_t bytes = per_system_bytes(n, P, A, E) * (size_t)capacity + kCtlWords * 4 + kMaxReq * 4;
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
  pl.fn = fn;
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
  SCK(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl.bps, fn, kThreads, 0));
  if (pl.bps < 1) return sfail(s, ODE_ERR_UNSUPPORTED, "serving kernel cannot be resident");
  const size_t C = (size_t)capacity;
  pl.ring_cap = (unsigned int)capacity;
  pl.yl_cap = (unsigned int)capacity;
  struct {
    void** p;
    size_t b;
  } al[] = {{(void**)&pl.td, 2 * C * sizeof(double)},   {(void**)&pl.y, n * C * sizeof(double)},
            {(void**)&pl.p, P * C * sizeof(double)},    {(void**)&pl.acc, A * C * sizeof(double)},
            {(void**)&pl.status, C * sizeof(int)},       {(void**)&pl.ecnt, E * C * sizeof(int)},
            {(void**)&pl.left, C * sizeof(int)},         {(void**)&pl.owner, C * sizeof(int)},
            {(void**)&pl.nacc, C * sizeof(long long)},   {(void**)&pl.nrej, C * sizeof(long long)},
            {(void**)&pl.ring, C * sizeof(unsigned int)},
            {(void**)&pl.yl, C * sizeof(unsigned long long)},
            {(void**)&pl.ctl, kCtlWords * sizeof(unsigned int)},
            {(void**)&pl.done, kMaxReq * sizeof(unsigned int)}};
  for (auto& x : al) {
    SCK(s, cudaMalloc(x.p, x.b));
    SCK(s, cudaMemset(*x.p, 0, x.b));
  }
  SCK(s, cudaMallocHost(&pl.h_ring, C * sizeof(unsigned int)));
  SCK(s, cudaMallocHost(&pl.h_tail, kTailWords * sizeof(unsigned int)));
  SCK(s, cudaMallocHost(&pl.h_ctl, kCtlWords * sizeof(unsigned int)));
  SCK(s, cudaMallocHost(&pl.h_done, kMaxReq * sizeof(unsigned int)));
  SCK(s, cudaMallocHost(&pl.h_yl, C * sizeof(unsigned long long)));
  SCK(s, cudaMallocHost(&pl.h_flag, 2 * sizeof(unsigned int)));
  memset(pl.h_ctl, 0, kCtlWords * sizeof(unsigned int));
  pl.h_flag[0] = 0;
  pl.h_flag[1] = 1;
  SCK(s, cudaStreamCreateWithFlags(&pl.kstream, cudaStreamNonBlocking));
  SCK(s, cudaEventCreateWithFlags(&pl.inst.ev, cudaEventDisableTiming));
  for (int i = 0; i < kTailWords; i++) SCK(s, cudaEventCreateWithFlags(&pl.tail_ev[i], cudaEventDisableTiming));
  SCK(s, cudaEventCreateWithFlags(&pl.snap_ev, cudaEventDisableTiming));
  pl.free_ranges.clear();
  pl.free_ranges[0] = capacity;
  pl.free_tix.clear();
  for (int i = kMaxReq - 1; i >= 0; i--) pl.free_tix.push_back(i);
  pl.slot_req.assign(C, nullptr);
  pl.tix_base.assign(kMaxReq, 0u);
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
  r->b_in = (2 + pl.n + pl.P) * n * sizeof(double);
  r->b_meta = 2 * n * sizeof(int);
  r->b_zero = 2 * n * sizeof(long long);
  r->b_out = (2 + pl.n + pl.A) * n * sizeof(double);
  r->b_status = n * sizeof(int);
  r->b_steps = n * sizeof(long long);
  PinnedCache& pc = s->pinned;
  cudaError_t e = pc.get((void**)&r->h_in, r->b_in);
  if (e == cudaSuccess) e = pc.get((void**)&r->h_meta, r->b_meta);
  if (e == cudaSuccess) e = pc.get((void**)&r->h_zero, r->b_zero);
  if (e == cudaSuccess) e = pc.get((void**)&r->h_out, r->b_out);
  if (e == cudaSuccess) e = pc.get((void**)&r->h_status, r->b_status);
  if (e == cudaSuccess) e = pc.get((void**)&r->h_acc_steps, r->b_steps);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_request(pc, r);
    return scuda(s, e, "request buffers");
  }
  memcpy(r->h_in, td, 2 * n * sizeof(double));
  memcpy(r->h_in + 2 * n, y0, pl.n * n * sizeof(double));
  memcpy(r->h_in + (2 + pl.n) * n, p, pl.P * n * sizeof(double));
  memset(r->h_zero, 0, 2 * n * sizeof(long long));
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
  // 0. finished copies out free their slots before anything is admitted
  if (int rc = release_harvested(s)) return rc;
  int running = 0, waiting = 0;
  for (Pool& pl : s->pools) {
    if (!pl.on) continue;
    // 1. a completed snapshot: yielded systems back, finished requests out
    if (pl.snap_inflight) {
      cudaError_t q = cudaEventQuery(pl.snap_ev);
      if (q == cudaSuccess) {
        if (int rc = take_snapshot(s, pl)) return rc;
      } else if (q != cudaErrorNotReady) {
        return scuda(s, q, "snapshot");
      }
    }
    // 2. admit waiting requests in arrival order while slots are free
    while (!pl.waiting.empty() && !pl.free_tix.empty()) {
      Request* r = pl.waiting.front();
      const int off = take_range(pl, r->n);
      if (off < 0) break;
      r->off = off;
      pl.waiting.pop_front();
      if (int rc = admit(s, pl, r)) return rc;
    }
    // 3. publish systems to the ring
    if (int rc = publish(s, pl)) return rc;
  }
  // 4. kernel instances: relaunch, grow, or stop to rebalance
  if (int rc = manage_instances(s)) return rc;
  for (Pool& pl : s->pools) {
    if (!pl.on) continue;
    // 5. the next snapshot
    if (!pl.snap_inflight && (pl.unfinished > 0 || pl.yl_read != pl.known_yield_tail))
      if (int rc = start_snapshot(s, pl)) return rc;
    running += (int)pl.running.size();
    waiting += (int)pl.waiting.size();
  }
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
  free_request(s->pinned, r);
  return ODE_OK;
}

int ode_server_destroy(ode_server* s) {
  if (!s) return ODE_OK;
  cudaSetDevice(s->device);
  // running instances stop at their next slice boundary and exit
  for (Pool& pl : s->pools)
    if (pl.on && s->cstream) set_stop(s, pl, 1);
  if (s->cstream) cudaStreamSynchronize(s->cstream);
  for (Pool& pl : s->pools)
    if (pl.kstream) cudaStreamSynchronize(pl.kstream);
  for (auto& kv : s->reqs) free_request(s->pinned, kv.second);
  s->pinned.release();
  for (Pool& pl : s->pools) {
    void* ptrs[] = {pl.td, pl.y, pl.p, pl.acc, pl.status, pl.ecnt, pl.left, pl.owner, pl.nacc, pl.nrej,
                    pl.ring, pl.yl, pl.ctl, pl.done};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    void* hp[] = {pl.h_ring, pl.h_tail, pl.h_ctl, pl.h_done, pl.h_yl, pl.h_flag};
    for (void* p : hp)
      if (p) cudaFreeHost(p);
    if (pl.inst.ev) cudaEventDestroy(pl.inst.ev);
    if (pl.kstream) cudaStreamDestroy(pl.kstream);
    for (int i = 0; i < kTailWords; i++)
      if (pl.tail_ev[i]) cudaEventDestroy(pl.tail_ev[i]);
    if (pl.snap_ev) cudaEventDestroy(pl.snap_ev);
  }
  if (s->cstream) cudaStreamDestroy(s->cstream);
  delete s;
  return ODE_OK;
}

int ode_server_stats(const ode_server* s, int model, long long* out) {
  if (!s || !out || model < 0 || model >= kNumModels) return ODE_ERR_INVALID_ARG;
  const Pool& pl = s->pools[model];
  out[0] = pl.launches;
  out[1] = pl.stops;
  out[2] = pl.yielded;
  out[3] = pl.snapshots;
  out[4] = pl.published;
  out[5] = pl.finished;
  out[6] = (long long)pl.flags;
  out[7] = pl.unfinished;
  return ODE_OK;
}

const char* ode_server_last_error(const ode_server* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
