// k_tc_rf_y1_narrow.cu -- instantiations of k_tc_rf for scatterers off the azimuth plane
// (Y != 0, delta with the Eq. 14 exponent) and sinc arguments up to 3.2.
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_y1_narrow(bool linear, bool split) {
    if (split) return tc_kernel_bf16_y1_narrow(linear);
    return linear ? k_tc_rf<true, 1, true, false> : k_tc_rf<true, 1, false, false>;
}
}  // namespace simus
