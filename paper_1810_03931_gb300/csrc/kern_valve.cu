// kern_valve.cu -- integrator kernels of the Valve model (every scheme,
// precision and launch form), compiled in their own translation unit so the
// models build in parallel.
#include "integrator.cuh"

namespace odegpu {
const void* kernel_valve(int scheme, int prec, int persistent) {
  return lookup_kernel<Valve>(scheme, prec, persistent);
}
}  // namespace odegpu
