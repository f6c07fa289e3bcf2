// kern_keller_miksis.cu -- integrator kernels of the KellerMiksis model (every scheme,
// precision and launch form), compiled in their own translation unit so the
// models build in parallel.
#include "integrator.cuh"

namespace odegpu {
const void* kernel_keller_miksis(int scheme, int prec, int persistent) {
  return lookup_kernel<KellerMiksis>(scheme, prec, persistent);
}
}  // namespace odegpu
