// Tensor-core conv instantiations with E4M3 operands (kind::f8f6f4); input layers take 32 padded
// channels (32-byte rows).
// One translation unit per operand type, so the build compiles them in parallel.
#include "conv_tc.cuh"

namespace conet {

int launch_conv_tc_e4m3(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  constexpr int kind = 2;
  TC_CASE(2, 2, 32, 32)
  TC_CASE(2, 3, 32, 32)
  TC_CASE(2, 3, 32, 64)
  TC_CASE(2, 3, 64, 64)
  TC_CASE(2, 4, 32, 96)
  TC_CASE(2, 4, 96, 96)
  TC_CASE(2, 1, 32, 64)
  TC_CASE(2, 1, 64, 64)
  return fail(CONET_ERR_UNSUPPORTED, "tensor-core conv kind=%d branches=%d Cin=%d Cout=%d not instantiated", kind, nb,
              cin, cout);
}

}  // namespace conet
