// Tensor-core conv instantiations with BF16 operands (kind::f16); input layers take 16 padded
// channels (32-byte rows).
// One translation unit per operand type, so the build compiles them in parallel.
#include "conv_tc.cuh"

namespace conet {

int launch_conv_tc_bf16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  constexpr int kind = 0;
  TC_CASE(0, 2, 16, 32)
  TC_CASE(0, 2, 32, 32)
  TC_CASE(0, 3, 16, 64)
  TC_CASE(0, 3, 64, 64)
  TC_CASE(0, 4, 16, 96)
  TC_CASE(0, 4, 96, 96)
  TC_CASE(0, 1, 16, 64)
  TC_CASE(0, 1, 64, 64)
  TC_CASE(0, 3, 16, 16)
  TC_CASE(0, 3, 16, 32)
  TC_CASE(0, 3, 32, 32)
  TC_CASE(0, 1, 16, 112)
  TC_CASE(0, 1, 112, 112)
  TC_CASE(0, 4, 16, 64)
  TC_CASE(0, 4, 64, 64)
  TC_CASE(0, 1, 16, 96)
  TC_CASE(0, 1, 96, 96)
  return fail(CONET_ERR_UNSUPPORTED, "tensor-core conv kind=%d branches=%d Cin=%d Cout=%d not instantiated", kind, nb,
              cin, cout);
}

}  // namespace conet
