// Per-RE elementwise stage between convolution layers (Sec. III): Hadamard fusion of the
// main and support activations, LayerNorm over channels after the fusion, the
// pre-activation (LN ->) ReLU that feeds the next block's first conv, and the 1x1 LLR
// head.  One warp per RE; lanes stride the channels, so every load is a coalesced
// 128-byte row segment and the LayerNorm statistics are warp-shuffle reductions.
#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

constexpr int CPL = 4;   // channels per lane: C <= 128

__device__ __forceinline__ void layer_norm(float (&x)[CPL], int lane, int C, const float* g, const float* b,
                                           float (&y)[CPL]) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < CPL; ++j) s += (lane + 32 * j < C) ? x[j] : 0.f;
  const float mean = warp_sum(s) / (float)C;
  float q = 0.f;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const float d = (lane + 32 * j < C) ? x[j] - mean : 0.f;
    q += d * d;
  }
  const float rstd = rsqrtf(warp_sum(q) / (float)C + 1e-5f);
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j;
    y[j] = c < C ? (x[j] - mean) * rstd * __ldg(g + c) + __ldg(b + c) : 0.f;
  }
}

__global__ void fuse_kernel(FuseArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C;
  for (long long m = warp0; m < a.M; m += nwarps) {
    float u[MAX_BR][CPL];
#pragma unroll
    for (int b = 0; b < MAX_BR; ++b)
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        u[b][j] = (b < a.n_br && c < C) ? a.u[b][m * C + c] : 0.f;
      }
    float x0[CPL];
    if (a.fuse) {
      float p[CPL];
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        p[j] = u[0][j];
#pragma unroll
        for (int b = 1; b < MAX_BR; ++b)
          if (b < a.n_br) p[j] *= u[b][j];
      }
      if (a.fuse_g) {
        layer_norm(p, lane, C, a.fuse_g, a.fuse_b, x0);
      } else {
#pragma unroll
        for (int j = 0; j < CPL; ++j) x0[j] = p[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) x0[j] = u[0][j];
    }
    if (a.x0_out) {
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        if (c < C) a.x0_out[m * C + c] = x0[j];
      }
    }
#pragma unroll
    for (int b = 0; b < MAX_BR; ++b) {
      if (b >= a.n_br || !a.h_out[b]) continue;
      float xb[CPL], h[CPL];
#pragma unroll
      for (int j = 0; j < CPL; ++j) xb[j] = b == 0 ? x0[j] : u[b][j];
      if (a.ln1_g[b]) {
        layer_norm(xb, lane, C, a.ln1_g[b], a.ln1_b[b], h);
      } else {
#pragma unroll
        for (int j = 0; j < CPL; ++j) h[j] = xb[j];
      }
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        if (c < C) a.h_out[b][m * C + c] = fmaxf(h[j], 0.f);
      }
    }
    if (a.head_w) {
      for (int q = 0; q < a.Q; ++q) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int c = lane + 32 * j;
          if (c < C) s += __ldg(a.head_w + q * C + c) * x0[j];
        }
        s = warp_sum(s);
        if (lane == 0) a.llr[m * a.Q + q] = s + __ldg(a.head_b + q);
      }
    }
  }
}

}  // namespace

int launch_fuse(const FuseArgs& a, cudaStream_t s) {
  if (a.C > 32 * CPL) return fail(CONET_ERR_UNSUPPORTED, "width %d > %d", a.C, 32 * CPL);
  fuse_kernel<<<grid_for(a.M * 32, 256, 152 * 16), 256, 0, s>>>(a);
  return check_launch("fuse_kernel");
}

}  // namespace conet
