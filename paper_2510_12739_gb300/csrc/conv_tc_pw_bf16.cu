// Tensor-core 1x1 convs (the pointwise half of a depthwise-separable residual block) with
// BF16 operands, for the 2 x 32, 3 x 64 and 4 x 96 residual networks.
#include "conv_tc.cuh"

namespace conet {

int launch_conv_tc_pw_bf16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a,
                           cudaStream_t s) {
  constexpr int kind = 0;
  TC_PW_CASE(0, 2, 32)
  TC_PW_CASE(0, 3, 64)
  TC_PW_CASE(0, 4, 96)
  return fail(CONET_ERR_UNSUPPORTED, "tensor-core 1x1 conv kind=%d branches=%d C=%d not instantiated", kind, nb, cout);
}

}  // namespace conet
