// Shared device helpers of libconet: Philox4x32-10, uniform / Gaussian draws, Gray QAM,
// warp reductions, and the error plumbing of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>
#include <cstdio>
#include <string>

#include "../../include/conet.h"

namespace conet {

// ------------------------------------------------------------------ error plumbing
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);
int check_launch(const char* what);
// The process-wide count of kernel launches (conet_launch_count), and an adjustment of it:
// a replayed CUDA graph adds its kernels, a capture takes back the launches it recorded.
unsigned long long launch_count();
void launch_count_add(long long n);

#define CONET_TRY(expr)            \
  do {                             \
    int _rc = (expr);              \
    if (_rc != CONET_OK) return _rc; \
  } while (0)

#define CONET_CUDA(call) CONET_TRY(::conet::check_cuda((call), #call))
#define CONET_LAUNCHED(name) CONET_TRY(::conet::check_launch(name))

inline int grid_for(long long n, int threads, int cap = 152 * 32) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11: 10 rounds of (multiply-high/low of c0 and c2 by the round
// multipliers, swap and xor with the key), key bumped by the Weyl constants.
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return {c0, c1, c2, c3};
}

// Uniform in (0, 1), exactly ((w >> 9) + 0.5) * 2^-23 (representable in float32).
__device__ __forceinline__ float u01(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// Philox stream tags (counter word c3).
enum : uint32_t {
  TAG_SLOT = 1,
  TAG_BITS = 2,
  TAG_PILOT = 3,
  TAG_CHAN = 4,
  TAG_ICHAN = 5,
  TAG_NOISE = 6,
  TAG_IBITS = 7,
  TAG_INIT = 8
};

// Gray-mapped square QAM of unit energy: bit k of `word` is b_k; even positions label
// the in-phase axis, odd positions the quadrature axis, most significant first; the
// label is the binary-reflected Gray code of the PAM level index.
__device__ __forceinline__ float2 qam_map(uint32_t word, int q) {
  const int half = q >> 1;
  uint32_t li = 0, lq = 0;
  for (int i = 0; i < half; ++i) {
    li = (li << 1) | ((word >> (2 * i)) & 1u);
    lq = (lq << 1) | ((word >> (2 * i + 1)) & 1u);
  }
  uint32_t ii = li, iq = lq;
  for (uint32_t s = li >> 1; s; s >>= 1) ii ^= s;
  for (uint32_t s = lq >> 1; s; s >>= 1) iq ^= s;
  const float P = (float)(1 << half);
  const float scale = rsqrtf(2.0f * (float)((1 << q) - 1) / 3.0f);
  return make_float2((2.0f * (float)ii - (P - 1.0f)) * scale, (2.0f * (float)iq - (P - 1.0f)) * scale);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace conet
