// kern_duffing_lyapunov.cu -- integrator kernels of the Duffing model with
// its polar linearisation (binary64 only, both schemes and launch forms),
// compiled in their own translation unit so the models build in parallel.
#include "integrator.cuh"

namespace odegpu {
const void* kernel_duffing_lyapunov(int scheme, int prec, int persistent) {
  return lookup_kernel<DuffingLyapunov>(scheme, prec, persistent);
}
}  // namespace odegpu
