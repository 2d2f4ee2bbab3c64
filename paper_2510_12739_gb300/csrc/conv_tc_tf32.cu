// Tensor-core conv instantiations with split-TF32 operands (kind::tf32, three MMAs per K
// slice: FP32-accurate products).
// One translation unit per operand type, so the build compiles them in parallel.
#include "conv_tc.cuh"

namespace conet {

int launch_conv_tc_tf32(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  constexpr int kind = 1;
  TC_CASE(1, 2, 16, 32)
  TC_CASE(1, 2, 32, 32)
  TC_CASE(1, 3, 16, 64)
  TC_CASE(1, 3, 64, 64)
  TC_CASE(1, 4, 16, 96)
  TC_CASE(1, 4, 96, 96)
  TC_CASE(1, 3, 16, 32)
  TC_CASE(1, 3, 32, 32)
  TC_CASE(1, 1, 16, 112)
  TC_CASE(1, 1, 112, 112)
  return fail(CONET_ERR_UNSUPPORTED, "tensor-core conv kind=%d branches=%d Cin=%d Cout=%d not instantiated", kind, nb,
              cin, cout);
}

}  // namespace conet
