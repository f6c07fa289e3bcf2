// kern_bounce.cu -- integrator kernels of the Bounce model (every scheme,
// precision and launch form), compiled in their own translation unit so the
// models build in parallel.
#include "integrator.cuh"

namespace odegpu {
const void* kernel_bounce(int scheme, int prec, int persistent) {
  return lookup_kernel<Bounce>(scheme, prec, persistent);
}
}  // namespace odegpu
