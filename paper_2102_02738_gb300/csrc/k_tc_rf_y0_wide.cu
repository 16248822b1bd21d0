// k_tc_rf_y0_wide.cu -- instantiations of k_tc_rf for scatterers at Y = 0 and sinc
// arguments of any size (sub-elements wider than the Eq. 21 rule gives).
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_y0_wide(bool linear, bool split) {
    if (split) return tc_kernel_bf16_y0_wide(linear);
    return linear ? k_tc_rf<false, 0, true, false> : k_tc_rf<false, 0, false, false>;
}
}  // namespace simus
