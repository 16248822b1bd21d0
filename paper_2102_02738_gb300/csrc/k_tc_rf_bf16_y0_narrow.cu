// k_tc_rf_bf16_y0_narrow.cu -- instantiations of k_tc_rf with split BF16 operands (leading
// part + remainder, three products per GEMM) for scatterers at Y = 0 and sinc arguments up
// to 3.2.
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_bf16_y0_narrow(bool linear) {
    return linear ? k_tc_rf<false, 1, true, true> : k_tc_rf<false, 1, false, true>;
}
}  // namespace simus
