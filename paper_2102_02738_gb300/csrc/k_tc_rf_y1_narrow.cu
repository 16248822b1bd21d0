// k_tc_rf_y1_narrow.cu -- instantiations of k_tc_rf for scatterers off the azimuth plane
// (Y != 0, delta with the Eq. 14 exponent) and sinc arguments up to 3.2.
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_y1_narrow(bool linear) {
    return linear ? k_tc_rf<true, 1, true> : k_tc_rf<true, 1, false>;
}
}  // namespace simus
