// k_tc_rf_y0_narrow.cu -- instantiations of k_tc_rf for scatterers at Y = 0 and sinc
// arguments up to 3.2 (narrow sub-elements).
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_y0_narrow(bool linear, bool split) {
    if (split) return tc_kernel_bf16_y0_narrow(linear);
    return linear ? k_tc_rf<false, 1, true, false> : k_tc_rf<false, 1, false, false>;
}
}  // namespace simus
