// noalloc_layout.h -- byte layout of the fixed scratch array used by
// ode_run_periods_noalloc.  Plain host C++ (no CUDA), so that a CPU test can
// compile it on its own and check the arithmetic for every size.
//
// The array holds, for a call on n systems:
//   [0, 256)  queue head (unsigned int at byte 0) and watchdog flag (int at 64)
//   nacc      accepted-step counters, long long [n]
//   nrej      rejected-step counters, long long [n]
//   status    stop status, int [n]
//   ecnt      event counters, int [max_events][n]
// Every section starts on a 256-byte boundary, so each one is aligned for its
// element type (and for full-segment warp accesses) whatever n is.
#pragma once

#include <stddef.h>

namespace odegpu {

struct NoAllocLayout {
  size_t head;    // queue head + watchdog flag (256 bytes)
  size_t nacc;    // long long [n]
  size_t nrej;    // long long [n]
  size_t status;  // int [n]
  size_t ecnt;    // int [max_events][n]
  size_t total;   // bytes used, a multiple of 256
};

constexpr size_t kNoAllocAlign = 256;
constexpr size_t kNoAllocHeadBytes = 256;

constexpr size_t noalloc_align_up(size_t x) {
  return (x + kNoAllocAlign - 1) / kNoAllocAlign * kNoAllocAlign;
}

constexpr NoAllocLayout noalloc_layout(size_t n, size_t max_events) {
  NoAllocLayout L{0, 0, 0, 0, 0, 0};
  L.head = 0;
  L.nacc = noalloc_align_up(L.head + kNoAllocHeadBytes);
  L.nrej = noalloc_align_up(L.nacc + n * sizeof(long long));
  L.status = noalloc_align_up(L.nrej + n * sizeof(long long));
  L.ecnt = noalloc_align_up(L.status + n * sizeof(int));
  L.total = noalloc_align_up(L.ecnt + max_events * n * sizeof(int));
  return L;
}

}  // namespace odegpu
