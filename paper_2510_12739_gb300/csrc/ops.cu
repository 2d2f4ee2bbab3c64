// Standalone layer operations of the C ABI that run without a receiver handle.
#include "common.cuh"
#include "kernels.cuh"

using namespace conet;

extern "C" int conet_conv3x3_wgrad(const float* x, const float* dz, int B, int T, int F, int cin, int cout,
                                   float* dW, float* db, void* stream) {
  if (!x || !dz || !dW) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1 || T < 1 || F < 1) return fail(CONET_ERR_SHAPE, "empty grid B=%d T=%d F=%d", B, T, F);
  if (cin < 4 || cin > 128 || cin % 4 || cout < 4 || cout > 128 || cout % 4)
    return fail(CONET_ERR_SHAPE, "cin=%d cout=%d: multiples of 4 in 4..128 required", cin, cout);
  cudaStream_t s = (cudaStream_t)stream;
  const long long M = (long long)B * T * F;
  const size_t part_floats = wgrad_partial_floats(M, cin, cout, 1);
  const size_t ew_floats = (size_t)EW_PART_CTAS * cout;
  float* part = nullptr;
  CONET_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&part), (part_floats + ew_floats) * sizeof(float), s));
  WgradArgs a = {};
  a.x[0] = x;
  a.g[0] = dz;
  a.dW[0] = dW;
  a.cin_src[0] = cin;
  a.part = part;
  a.cin = cin;
  a.cout = cout;
  a.n_br = 1;
  a.T = T;
  a.F = F;
  a.M = M;
  int rc = launch_wgrad(a, s);
  if (rc == CONET_OK && db) {
    float* ew = part + part_floats;
    rc = launch_channel_sums(dz, M, cout, ew, s);
    if (rc == CONET_OK) rc = launch_reduce_partials(ew, ew_grid(M), cout, db, 0, s);
  }
  const cudaError_t fe = cudaFreeAsync(part, s);
  if (rc != CONET_OK) return rc;
  return check_cuda(fe, "cudaFreeAsync");
}
