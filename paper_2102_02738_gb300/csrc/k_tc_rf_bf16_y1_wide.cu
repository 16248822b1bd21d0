// k_tc_rf_bf16_y1_wide.cu -- instantiations of k_tc_rf with split BF16 operands (leading
// part + remainder, three products per GEMM) for scatterers off the azimuth plane and sinc
// arguments beyond 3.2.
#include "k_tc_kernel.cuh"

namespace simus {
TcKernelFn tc_kernel_bf16_y1_wide(bool linear) {
    return linear ? k_tc_rf<true, 0, true, true> : k_tc_rf<true, 0, false, true>;
}
}  // namespace simus
