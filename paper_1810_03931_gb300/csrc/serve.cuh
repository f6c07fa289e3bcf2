// serve.cuh -- the resident serving kernel: a persistent integrator whose
// threads take systems from a ring of slot indices that the host keeps
// filling while the kernel runs (continuous batching of sweep requests into
// one launch; the refill of Sec. 7.2's "clustering" remark and of the device
// work queue taken to requests that arrive over time).
//
// Protocol (all waits bounded):
//  * The host writes a system's inputs into its slot, then the slot index
//    into ring[tail % ring_cap], then the new tail (ctl[kCtlRingTail]), each
//    copy ordered after the previous one on one stream.  Threads read the
//    tail and the entries through L2 and claim entries with compare-and-swap
//    on ctl[kCtlRingHead]; a claimed system is loaded through L2 as well (L1
//    is not coherent with those copies).
//  * A thread runs its system for at most a.n_slices slices (the residency
//    quantum, or until the system's own slice budget slices_left runs out),
//    stores the whole state back, and then either counts the system as
//    finished -- a system-scope fence, then done_cnt[owner[slot]] += 1 -- or,
//    with slices left, appends (lap << 32 | slot) to the yield list for the
//    host to put back into the ring.
//  * ctl[kCtlStop] != 0 makes threads yield at their next slice boundary and
//    take no new work; a warp with no work exits once the stop flag is seen
//    or after idle_ns without work.  The host relaunches when work remains.
//  * Watchdog: a system that runs longer than a.time_limit_ns in one
//    residency stops with kStTimeout and counts as finished.
// Each system's arithmetic is that of ode_kernel (the same Lane state
// machine), so a served result equals a plain integration of the system.
#pragma once

namespace odegpu {

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

template <class M, int SCHEME, int PREC>
__global__ void __launch_bounds__(ODEGPU_MAX_THREADS_OF(M), ODEGPU_MIN_BLOCKS_OF(M))
    serve_kernel(const KArgs a, const ServeArgs sv) {
  using L_t = Lane<M, SCHEME, PREC>;
  using T = typename L_t::T;
  L_t L;
#pragma unroll
  for (int m = 0; m < 3; m++) L.mct[m] = (T)a.pr.mc[m];
  {
    double mcd[3] = {a.pr.mc[0], a.pr.mc[1], a.pr.mc[2]};
    L.w = M::omega(mcd);
  }
  L.tab = nullptr;
  L.tab_n = 0;
  L.tab_t0 = L.tab_t1 = 0.0;
  L.use_tab = false;

  unsigned int* head = sv.ctl + kCtlRingHead;
  const unsigned int* tail = sv.ctl + kCtlRingTail;
  const unsigned int* stop = sv.ctl + kCtlStop;
  bool active = false, fresh = false, stopping = false;
  unsigned long long t_sys = 0;

  // Claim the next ring entry: slot index, -1 when the ring is empty, -2
  // when the host asked the kernel to stop.  A failed compare-and-swap means
  // another thread claimed that entry; at most 64 attempts per call.
  const bool claims = (int)(threadIdx.x & 31) < sv.lanes_per_warp;
  auto claim = [&]() -> int {
    if (ld_volatile_u32(stop) != 0u) return -2;
    if (!claims) return -1;
    unsigned int h = ld_volatile_u32(head);
    for (int it = 0; it < 64; it++) {
      const unsigned int t = ld_volatile_u32(tail);
      if ((int)(t - h) <= 0) return -1;
      const unsigned int prev = atomicCAS(head, h, h + 1u);
      if (prev == h) {
        const unsigned int slot = __ldcg(sv.ring + (h % sv.ring_cap));
        if (slot < (unsigned int)a.N) return (int)slot;
        atomicExch(sv.ctl + kCtlFlags, 2);  // an entry outside the pool: skipped, reported
        return -1;
      }
      h = prev;
    }
    return -1;
  };
  auto next_system = [&]() {
    if (stopping) {
      active = false;
      return;
    }
    const int r = claim();
    if (r >= 0) {
      L.sys = r;
      active = true;
      fresh = true;
      t_sys = globaltimer_ns();
    } else {
      active = false;
      stopping = (r == -2);
    }
  };
  // the system in L.sys has been stored: finished or handed back
  auto release = [&](bool finished) {
    __threadfence_system();
    if (finished) {
      const unsigned int o = (unsigned int)__ldcg(sv.owner + L.sys);
      if (o < sv.done_cap) atomicAdd(sv.done_cnt + o, 1u);
      else atomicExch(sv.ctl + kCtlFlags, 2);
    } else {
      const unsigned int pos = atomicAdd(sv.ctl + kCtlYieldTail, 1u);
      const unsigned long long lap = (unsigned long long)(pos / sv.yl_cap + 1u);
      sv.yl[pos % sv.yl_cap] = (lap << 32) | (unsigned long long)(unsigned int)L.sys;
    }
  };
  auto settle = [&]() {
    while (active) {
      if (fresh) {
        fresh = false;
        if (!L.template load<true>(a)) {  // nothing left for this slot
          release(true);
          next_system();
          continue;
        }
        L.begin_slice(a);
      }
      if (L.status == kStNone) return;
      L.end_slice(a);
      if (L.slice < L.my_slices && ld_volatile_u32(stop) == 0u) {
        L.begin_slice(a);
        continue;
      }
      L.template store<true>(a);  // slices_left[slot] = loaded budget - slices run
      release(L.left0 - L.slice <= 0);
      next_system();
    }
  };

  next_system();
  settle();
  unsigned long long idle_since = 0;  // 0: the warp had work at its last check
  unsigned int wd = 0, poll = 0;
  for (;;) {
    if (!__any_sync(0xffffffffu, active)) {
      // The whole warp is without work (a warp-uniform branch): exit when a
      // thread saw the stop flag or after idle_ns without work; otherwise
      // sleep, look at the ring once per warp, and claim entries if any.
      if (__any_sync(0xffffffffu, stopping)) break;
      int quit = 0, work = 0;
      if ((threadIdx.x & 31) == 0) {
        const unsigned long long now = globaltimer_ns();
        if (idle_since == 0) idle_since = now;
        quit = now - idle_since > (unsigned long long)sv.idle_ns;
        work = (int)(ld_volatile_u32(tail) - ld_volatile_u32(head)) > 0 || ld_volatile_u32(stop) != 0u;
      }
      if (__shfl_sync(0xffffffffu, quit, 0)) break;
      if (__shfl_sync(0xffffffffu, work, 0)) {
        next_system();
        settle();
      } else {
        __nanosleep(20000);
      }
      continue;
    }
    idle_since = 0;
    if (active) {
      L.trial(a);
      if (L.status != kStNone) settle();
      if (active && a.time_limit_ns > 0 && ((++wd & 1023u) == 0u) &&
          globaltimer_ns() - t_sys > (unsigned long long)a.time_limit_ns) {
        L.status = kStTimeout;
        L.template store<true>(a);
        atomicExch(sv.ctl + kCtlFlags, 1);
        release(true);
        next_system();
        settle();
      }
    } else if (((++poll) & 63u) == 0u) {
      // an idle thread in a busy warp looks for work now and then
      next_system();
      settle();
    }
  }
}

template <class M>
const void* lookup_serve_kernel(int scheme, int prec) {
  if (prec == kFP64)
    return scheme == kRK4 ? (const void*)serve_kernel<M, kRK4, kFP64>
                          : (const void*)serve_kernel<M, kRKCK45, kFP64>;
  if constexpr (M::kHasFP32)
    return scheme == kRK4 ? (const void*)serve_kernel<M, kRK4, kFP32RHS>
                          : (const void*)serve_kernel<M, kRKCK45, kFP32RHS>;
  return nullptr;
}

}  // namespace odegpu
