// The integration kernel with the ROS34PW2 W-method stepper (option "method" = 1),
// instantiated in its own translation unit so that the two steppers compile in
// parallel; the device code is shared with chem_kernels.cu through chem_device.cuh.

#include "chem_device.cuh"

namespace chem {

cudaError_t launch_integrate_w(const IntegrateArgs& a, int block, int prec, int grid, cudaStream_t st) {
#define LW(P)                                                                       \
  do {                                                                              \
    if (block == 64) return launch_integrate_m<2, P, METHOD_ROS34PW2>(a, grid, st);  \
    if (block == 256) return launch_integrate_m<8, P, METHOD_ROS34PW2>(a, grid, st); \
    return launch_integrate_m<4, P, METHOD_ROS34PW2>(a, grid, st);                   \
  } while (0)
  if (prec == PREC_FP64) LW(PREC_FP64);
  if (prec == PREC_MIXED) LW(PREC_MIXED);
  LW(PREC_FP32ASM);
#undef LW
}

}  // namespace chem
