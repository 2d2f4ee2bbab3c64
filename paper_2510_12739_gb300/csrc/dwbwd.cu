// Backward of a depthwise-separable block conv on the FP32 path (Sec. II-A / III): the
// per-channel 3x3 z = dw(x, Wd) followed by the 1x1 y = W1 z + b.  Given g = dL/dy:
//   dW1[co][ci] = sum_m g[m][co] z[m][ci]              (wgrad1x1_kernel, split over REs)
//   dz[m][ci]   = sum_co g[m][co] W1[co][ci]           (the FP32 conv with one tap)
//   dWd[c][tap] = sum_m dz[m][c] x[m + shift(tap)][c]  (dw_wgrad_kernel, split over REs)
//   dx          = dw(dz, Wd rotated by 180 degrees)    (dwconv3x3_kernel, flip = 1)
// Both weight gradients write per-CTA partial sums that launch_reduce_partials adds up.
#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

constexpr int W1_ROWS = 32;   // REs per shared-memory tile of the 1x1 weight gradient

// grid (S splits, n_br); 256 threads as a 16 x 16 grid, each owning an R x R block of the
// C x C gradient (R = C / 16); partial sums to part[(b * S + split)][C][C]
template <int C>
__global__ void __launch_bounds__(256) wgrad1x1_kernel(const __grid_constant__ Wgrad1x1Args a, int S) {
  constexpr int R = C / 16;
  __shared__ float gs[W1_ROWS][C];
  __shared__ float zs[W1_ROWS][C];
  const int b = blockIdx.y, split = blockIdx.x;
  const float* __restrict__ g = a.g[b];
  const float* __restrict__ z = a.z[b];
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  float acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.f;
  const long long per = (a.M + S - 1) / S;
  const long long m_beg = split * per, m_end = m_beg + per < a.M ? m_beg + per : a.M;
  for (long long m0 = m_beg; m0 < m_end; m0 += W1_ROWS) {
    __syncthreads();
    for (int i = threadIdx.x; i < W1_ROWS * C; i += 256) {
      const int r = i / C, c = i % C;
      const long long m = m0 + r;
      gs[r][c] = m < m_end ? g[m * C + c] : 0.f;
      zs[r][c] = m < m_end ? z[m * C + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < W1_ROWS; ++r) {
      float gv[R], zv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        gv[i] = gs[r][tr * R + i];
        zv[i] = zs[r][tc * R + i];
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fmaf(gv[i], zv[j], acc[i][j]);
    }
  }
  float* out = a.part + ((size_t)b * S + split) * C * C;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) out[(tr * R + i) * C + tc * R + j] = acc[i][j];
}

// grid (S splits, n_br); blockDim = L x C threads (channel c = tid % C, RE lane tid / C);
// partial sums to part[(b * S + split)][C][9]
__global__ void __launch_bounds__(256) dw_wgrad_kernel(const __grid_constant__ DwWgradArgs a, int S) {
  extern __shared__ float red[];   // [lanes][C][9]
  const int b = blockIdx.y, split = blockIdx.x, C = a.C;
  const int lanes = blockDim.x / C, c = threadIdx.x % C, lane = threadIdx.x / C;
  const float* __restrict__ x = a.x[b];
  const float* __restrict__ dz = a.dz[b];
  float acc[9];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) acc[tap] = 0.f;
  const int TF = a.T * a.F;
  const long long per = (a.M + S - 1) / S;
  const long long m_beg = split * per, m_end = m_beg + per < a.M ? m_beg + per : a.M;
  for (long long m = m_beg + lane; m < m_end; m += lanes) {
    const float d = dz[m * C + c];
    const int r = (int)(m % TF), t = r / a.F, f = r % a.F;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int tt = t + tap / 3 - 1, ff = f + tap % 3 - 1;
      if (tt < 0 || tt >= a.T || ff < 0 || ff >= a.F) continue;
      acc[tap] = fmaf(d, __ldg(x + (m + (long long)(tap / 3 - 1) * a.F + (tap % 3 - 1)) * C + c), acc[tap]);
    }
  }
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) red[(lane * C + c) * 9 + tap] = acc[tap];
  __syncthreads();
  float* out = a.part + ((size_t)b * S + split) * C * 9;
  for (int i = threadIdx.x; i < C * 9; i += blockDim.x) {
    float s = 0.f;
    for (int l = 0; l < lanes; ++l) s += red[l * C * 9 + i];
    out[i] = s;
  }
}

}  // namespace

int dw_bwd_splits(int n_br) { return 152 * 4 / (n_br > 0 ? n_br : 1); }

int launch_wgrad1x1(const Wgrad1x1Args& a, cudaStream_t s) {
  const int S = dw_bwd_splits(a.n_br);
  const dim3 grid((unsigned)S, (unsigned)a.n_br);
  switch (a.C) {
    case 16: wgrad1x1_kernel<16><<<grid, 256, 0, s>>>(a, S); break;
    case 32: wgrad1x1_kernel<32><<<grid, 256, 0, s>>>(a, S); break;
    case 64: wgrad1x1_kernel<64><<<grid, 256, 0, s>>>(a, S); break;
    case 96: wgrad1x1_kernel<96><<<grid, 256, 0, s>>>(a, S); break;
    case 112: wgrad1x1_kernel<112><<<grid, 256, 0, s>>>(a, S); break;
    default: return fail(CONET_ERR_UNSUPPORTED, "1x1 weight gradient of width %d", a.C);
  }
  CONET_LAUNCHED("wgrad1x1_kernel");
  for (int b = 0; b < a.n_br; ++b)
    CONET_TRY(launch_reduce_partials(a.part + (size_t)b * S * a.C * a.C, S, a.C * a.C, a.dW[b], 0, s));
  return CONET_OK;
}

int launch_dw_wgrad(const DwWgradArgs& a, cudaStream_t s) {
  if (a.C < 1 || a.C > 256) return fail(CONET_ERR_UNSUPPORTED, "depthwise weight gradient of width %d", a.C);
  const int S = dw_bwd_splits(a.n_br);
  const int lanes = 256 / a.C;
  const size_t smem = (size_t)lanes * a.C * 9 * sizeof(float);
  dw_wgrad_kernel<<<dim3((unsigned)S, (unsigned)a.n_br), lanes * a.C, smem, s>>>(a, S);
  CONET_LAUNCHED("dw_wgrad_kernel");
  for (int b = 0; b < a.n_br; ++b)
    CONET_TRY(launch_reduce_partials(a.part + (size_t)b * S * a.C * 9, S, a.C * 9, a.dWd[b], 0, s));
  return CONET_OK;
}

}  // namespace conet
