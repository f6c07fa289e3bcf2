// cluster.cu -- host-side ordering of systems along a Z-order (Morton) curve
// of their governing parameters, so that the systems a warp integrates
// together need similar numbers of steps (the "clustering" the paper
// recommends against thread divergence, Sec. 7.2).  Plain host code.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/odegpu.h"

namespace {

// Spread the low `bits` bits of v so that bit i lands at position i * K + d.
uint64_t interleave(uint64_t v, int bits, int K, int d) {
  uint64_t out = 0;
  for (int i = 0; i < bits; i++)
    if (v >> i & 1u) out |= (uint64_t)1 << (i * K + d);
  return out;
}

}  // namespace

extern "C" int ode_cluster_order(const double* keys, int K, int N, int* perm) {
  if (K < 1 || K > 8 || N < 0 || (N > 0 && (!keys || !perm))) return ODE_ERR_INVALID_ARG;
  if (N == 0) return ODE_OK;
  const int bits = 63 / K < 31 ? 63 / K : 31;  // bits per key
  const double top = (double)(((uint64_t)1 << bits) - 1);
  std::vector<uint64_t> code((size_t)N, 0);
  std::vector<unsigned char> bad((size_t)N, 0);
  for (int d = 0; d < K; d++) {
    const double* kd = keys + (size_t)d * N;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < N; i++)
      if (isfinite(kd[i])) {
        lo = kd[i] < lo ? kd[i] : lo;
        hi = kd[i] > hi ? kd[i] : hi;
      }
    const bool used = hi > lo;  // a constant (or all non-finite) key orders nothing
    for (int i = 0; i < N; i++) {
      if (!isfinite(kd[i])) {
        bad[i] = 1;
        continue;
      }
      if (!used) continue;
      const double u = (kd[i] - lo) / (hi - lo);  // [0, 1]
      const uint64_t q = (uint64_t)floor(u * top + 0.5);
      code[i] |= interleave(q, bits, K, d);
    }
  }
  for (int i = 0; i < N; i++) perm[i] = i;
  // non-finite keys last, then by Morton code, ties by index (deterministic)
  std::stable_sort(perm, perm + N, [&](int a, int b) {
    if (bad[a] != bad[b]) return bad[a] < bad[b];
    return code[a] < code[b];
  });
  return ODE_OK;
}
