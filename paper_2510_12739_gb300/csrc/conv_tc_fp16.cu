// Tensor-core conv instantiations with FP16 operands (kind::f16, the BF16 rate with 11-bit
// significands).
// One translation unit per operand type, so the build compiles them in parallel.
#include "conv_tc.cuh"

namespace conet {

int launch_conv_tc_fp16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  constexpr int kind = 3;
  TC_CASE(3, 2, 16, 32)
  TC_CASE(3, 2, 32, 32)
  TC_CASE(3, 3, 16, 64)
  TC_CASE(3, 3, 64, 64)
  TC_CASE(3, 4, 16, 96)
  TC_CASE(3, 4, 96, 96)
  TC_CASE(3, 3, 16, 32)
  TC_CASE(3, 3, 32, 32)
  TC_CASE(3, 1, 16, 112)
  TC_CASE(3, 1, 112, 112)
  return fail(CONET_ERR_UNSUPPORTED, "tensor-core conv kind=%d branches=%d Cin=%d Cout=%d not instantiated", kind, nb,
              cin, cout);
}

}  // namespace conet
