// k_tc_rf_y0_mid.cu -- instantiations of k_tc_rf for scatterers at Y = 0 and sinc
// arguments up to 4.6 (every probe split by Eq. 21 with a bandwidth up to 75 %).
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_y0_mid(bool linear, bool split) {
    if (split) return tc_kernel_bf16_y0_mid(linear);
    return linear ? k_tc_rf<false, 2, true, false> : k_tc_rf<false, 2, false, false>;
}
}  // namespace simus
