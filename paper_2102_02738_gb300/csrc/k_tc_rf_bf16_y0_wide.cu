// k_tc_rf_bf16_y0_wide.cu -- instantiations of k_tc_rf with split BF16 operands (leading
// part + remainder, three products per GEMM) for scatterers at Y = 0 and sinc arguments
// beyond 4.6.
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_bf16_y0_wide(bool linear) {
    return linear ? k_tc_rf<false, 0, true, true> : k_tc_rf<false, 0, false, true>;
}
}  // namespace simus
