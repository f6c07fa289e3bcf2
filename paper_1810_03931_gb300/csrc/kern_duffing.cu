// kern_duffing.cu -- integrator kernels of the Duffing model (every scheme,
// precision and launch form), compiled in their own translation unit so the
// models build in parallel.
#include "integrator.cuh"

namespace odegpu {
const void* kernel_duffing(int scheme, int prec, int persistent) {
  return lookup_kernel<Duffing>(scheme, prec, persistent);
}
}  // namespace odegpu
