// Backward pass of the CoNet receiver (the training of Sec. IV) and the Adam update:
//  - head backward (1x1 conv): dX0 = dLLR W_h, partial dW_h / db_h per CTA;
//  - Hadamard-fusion backward with the post-fusion LayerNorm and the ReLU mask of the
//    fused activations: d a_j = d p * prod_{i != j} a_i (+ the branch's own gradient);
//  - LayerNorm(+ReLU) backward of the pre-activations inside RB / MRB blocks;
//  - 3x3 weight gradient dW[co][tap][ci] = sum_RE dz[RE][co] x[RE + shift(tap)][ci],
//    split over RE ranges into per-split partials that a second kernel sums in a fixed
//    order (deterministic);
//  - per-channel sums (bias gradients) and the partial-sum reduction;
//  - bias-corrected Adam.
// The data gradient of a 3x3 conv reuses the forward conv kernel with the weights
// rotated by 180 degrees and transposed (see launch_weights_dgrad_layout).
#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

// CPL: channels per lane, C <= 32 CPL (kernels are instantiated for CPL = 1 .. 4).
constexpr int EW_THREADS = 256;
constexpr int EW_WARPS = EW_THREADS / 32;

template <int CPL>
__device__ __forceinline__ void load_row(const float* __restrict__ p, long long m, int C, int lane, float (&x)[CPL]) {
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j;
    x[j] = c < C ? p[m * C + c] : 0.f;
  }
}

template <int CPL>
__device__ __forceinline__ void store_row(float* __restrict__ p, long long m, int C, int lane, const float (&x)[CPL]) {
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j;
    if (c < C) p[m * C + c] = x[j];
  }
}

// LayerNorm backward for one RE held by a warp.  x: LN input, gy: grad wrt the LN output
// (before the affine gain is applied, gy is the grad of y = g*xhat + b).
// Returns dx; accumulates dgamma (gy*xhat) and dbeta (gy) in the lane's registers.
template <int CPL>
__device__ __forceinline__ void ln_backward(const float (&x)[CPL], const float (&gy)[CPL], const float* __restrict__ g,
                                            int C, int lane, float (&dx)[CPL], float (&dg)[CPL], float (&db)[CPL]) {
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
  float xh[CPL], gxh[CPL];
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j;
    xh[j] = c < C ? (x[j] - mean) * rstd : 0.f;
    gxh[j] = c < C ? gy[j] * __ldg(g + c) : 0.f;
    dg[j] += gy[j] * xh[j];
    db[j] += gy[j];
    s1 += gxh[j];
    s2 += gxh[j] * xh[j];
  }
  const float m1 = warp_sum(s1) / (float)C, m2 = warp_sum(s2) / (float)C;
#pragma unroll
  for (int j = 0; j < CPL; ++j) dx[j] = rstd * (gxh[j] - m1 - xh[j] * m2);
}

// Block reduction of per-lane channel partials [n_vec][CPL] into part[blockIdx][n_vec * C].
template <int NV, int CPL>
__device__ void block_store_partials(float (&v)[NV][CPL], int C, float* __restrict__ part) {
  __shared__ float red[EW_WARPS][NV][128];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      if (c < C) red[w][k][c] = v[k][j];
    }
  __syncthreads();
  for (int i = threadIdx.x; i < NV * C; i += blockDim.x) {
    const int k = i / C, c = i % C;
    float s = 0.f;
    for (int ww = 0; ww < EW_WARPS; ++ww) s += red[ww][k][c];
    part[(size_t)blockIdx.x * NV * C + i] = s;
  }
}

template <int CPL>
__global__ void __launch_bounds__(EW_THREADS) fuse_bwd_kernel(FuseBwdArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C;
  float pv[2][CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) pv[0][j] = pv[1][j] = 0.f;
  for (long long m = warp0; m < a.M; m += nwarps) {
    float u[MAX_BR][CPL], gx0[CPL];
#pragma unroll
    for (int b = 0; b < MAX_BR; ++b) {
      if (b < a.n_br) load_row(a.u[b], m, C, lane, u[b]);
      else
#pragma unroll
        for (int j = 0; j < CPL; ++j) u[b][j] = 1.f;
    }
    load_row(a.gx0, m, C, lane, gx0);
    float gu[MAX_BR][CPL];
#pragma unroll
    for (int b = 1; b < MAX_BR; ++b) {
      if (b < a.n_br && a.gxs[b]) load_row(a.gxs[b], m, C, lane, gu[b]);
      else
#pragma unroll
        for (int j = 0; j < CPL; ++j) gu[b][j] = 0.f;
    }
    if (a.fuse) {
      // Example II's feedback: a support's stored activation is its next input a_b + a_0,
      // which fed the next layer; the fusion and the ReLU masks read a_b, and a_0 also
      // receives every support's input gradient
      float gfb[CPL];
#pragma unroll
      for (int j = 0; j < CPL; ++j) gfb[j] = 0.f;
      if (a.feedback) {
#pragma unroll
        for (int b = 1; b < MAX_BR; ++b) {
          if (b >= a.n_br) continue;
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
            u[b][j] -= u[0][j];
            gfb[j] += gu[b][j];
          }
        }
      }
      float gp[CPL];
      if (a.ln_g) {
        float p[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          if (a.op == 1) {
            p[j] = 0.f;
#pragma unroll
            for (int b = 0; b < MAX_BR; ++b)
              if (b < a.n_br) p[j] += u[b][j];
          } else {
            p[j] = u[0][j] * u[1][j] * u[2][j] * u[3][j];
          }
        }
        ln_backward(p, gx0, a.ln_g, C, lane, gp, pv[0], pv[1]);
      } else {
#pragma unroll
        for (int j = 0; j < CPL; ++j) gp[j] = gx0[j];
      }
#pragma unroll
      for (int b = 0; b < MAX_BR; ++b) {
        if (b >= a.n_br) continue;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          float o = gp[j];
          if (a.op != 1) {
#pragma unroll
            for (int i = 0; i < MAX_BR; ++i)
              if (i != b) o *= u[i][j];
          }
          gu[b][j] = (b == 0 ? gfb[j] : gu[b][j]) + o;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) gu[0][j] = gx0[j];
    }
#pragma unroll
    for (int b = 0; b < MAX_BR; ++b) {
      if (b >= a.n_br) continue;
      if (a.relu_mask)
#pragma unroll
        for (int j = 0; j < CPL; ++j) gu[b][j] = u[b][j] > 0.f ? gu[b][j] : 0.f;
      store_row(a.gu[b], m, C, lane, gu[b]);
    }
  }
  if (a.part) block_store_partials<2, CPL>(pv, C, a.part);
}

template <int CPL>
__global__ void __launch_bounds__(EW_THREADS) ln_relu_bwd_kernel(LnReluBwdArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C;
  float pv[2][CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) pv[0][j] = pv[1][j] = 0.f;
  for (long long m = warp0; m < a.M; m += nwarps) {
    float x[CPL], g[CPL], out[CPL];
    load_row(a.x, m, C, lane, x);
    load_row(a.g, m, C, lane, g);
    if (a.ln_g) {
      // recompute y = LN(x) * gamma + beta to get the ReLU mask, then LN backward
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
      float gy[CPL];
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        const float y = c < C ? (x[j] - mean) * rstd * __ldg(a.ln_g + c) + __ldg(a.ln_b + c) : 0.f;
        gy[j] = y > 0.f ? g[j] : 0.f;
      }
      ln_backward(x, gy, a.ln_g, C, lane, out, pv[0], pv[1]);
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) out[j] = x[j] > 0.f ? g[j] : 0.f;
    }
    if (a.add) {
      float ad[CPL];
      load_row(a.add, m, C, lane, ad);
#pragma unroll
      for (int j = 0; j < CPL; ++j) out[j] += ad[j];
    }
    store_row(a.out, m, C, lane, out);
  }
  if (a.part) block_store_partials<2, CPL>(pv, C, a.part);
}

template <int CPL>
__global__ void __launch_bounds__(EW_THREADS) head_bwd_kernel(HeadBwdArgs a) {
  constexpr int QMAX = 8;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C, Q = a.Q;
  float pw[QMAX][CPL], pb[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    pb[q] = 0.f;
#pragma unroll
    for (int j = 0; j < CPL; ++j) pw[q][j] = 0.f;
  }
  for (long long m = warp0; m < a.M; m += nwarps) {
    float x[CPL], g[CPL];
    load_row(a.x0, m, C, lane, x);
#pragma unroll
    for (int j = 0; j < CPL; ++j) g[j] = 0.f;
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      if (q >= Q) continue;
      const float d = __ldg(a.dllr + m * Q + q);
      pb[q] += d;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        if (c < C) {
          g[j] += d * __ldg(a.w + q * C + c);
          pw[q][j] += d * x[j];
        }
      }
    }
    store_row(a.gx0, m, C, lane, g);
  }
  __shared__ float red[EW_WARPS][QMAX * 128 + QMAX];
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      if (q < Q && c < C) red[w][q * C + c] = pw[q][j];
    }
    if (lane == 0 && q < Q) red[w][QMAX * 128 + q] = pb[q];
  }
  __syncthreads();
  const int n = Q * C + Q;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int src = i < Q * C ? i : QMAX * 128 + (i - Q * C);
    float s = 0.f;
    for (int ww = 0; ww < EW_WARPS; ++ww) s += red[ww][src];
    a.part[(size_t)blockIdx.x * n + i] = s;
  }
}

template <int CPL>
__global__ void __launch_bounds__(EW_THREADS) channel_sums_kernel(const float* __restrict__ g, long long M, int C,
                                                                  float* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  float pv[1][CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) pv[0][j] = 0.f;
  for (long long m = warp0; m < M; m += nwarps) {
    float x[CPL];
    load_row(g, m, C, lane, x);
#pragma unroll
    for (int j = 0; j < CPL; ++j) pv[0][j] += x[j];
  }
  block_store_partials<1, CPL>(pv, C, part);
}

// out[j] (+)= sum_i part[i * n + j].  One CTA per group of 32 consecutive j: its 8 warps
// stride the partial rows (lane = j, so every load is one coalesced row segment) and are
// combined in a fixed order, so the sum is deterministic.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const float* __restrict__ part, int n_part, int n,
                                                              float* __restrict__ out, int accumulate) {
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < n)
    for (int i = w; i < n_part; i += 8) s += part[(size_t)i * n + j];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < n) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    out[j] = accumulate ? out[j] + t : t;
  }
}

// Weight gradient of a 3x3 conv for one tap per blockIdx.y, one branch per blockIdx.z and
// one RE range per blockIdx.x.  256 threads = 64 (4 ci x 4 co) output blocks x 4 RE lanes;
// blocks beyond the (CIN/4)(COUT/4) grid are handled by further CTAs (blk chunk in y).
constexpr int WG_CHUNK = 32;
__global__ void __launch_bounds__(256) wgrad_kernel(WgradArgs a) {
  extern __shared__ float4 wg_smem4[];
  float* xs = reinterpret_cast<float*>(wg_smem4);          // [WG_CHUNK][CIN]
  const int CIN = a.cin, COUT = a.cout;
  float* gs = xs + WG_CHUNK * CIN;                          // [WG_CHUNK][COUT]
  const int br = blockIdx.z;
  const int tap = blockIdx.y % 9, chunk = blockIdx.y / 9;
  const int dt = tap / 3 - 1, df = tap % 3 - 1;
  const int slot = threadIdx.x & 63, lane_r = threadIdx.x >> 6;
  const int nblk_co = COUT / 4;
  const int blk = chunk * 64 + slot;
  const bool active = blk < (CIN / 4) * nblk_co;
  const int ci0 = active ? (blk / nblk_co) * 4 : 0, co0 = active ? (blk % nblk_co) * 4 : 0;
  const long long per = (a.M + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per, r1 = min(a.M, r0 + per);
  const float* __restrict__ x = a.x[br];
  const float* __restrict__ g = a.g[br];
  const int TF = a.T * a.F;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (long long rc = r0; rc < r1; rc += WG_CHUNK) {
    const int n = (int)min((long long)WG_CHUNK, r1 - rc);
    __syncthreads();
    for (int i = threadIdx.x; i < WG_CHUNK * CIN / 4; i += blockDim.x) {
      const int r = i / (CIN / 4), q = i % (CIN / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < n) {
        const long long m = rc + r;
        const int rr = (int)(m % TF), t = rr / a.F + dt, f = rr % a.F + df;
        if (t >= 0 && t < a.T && f >= 0 && f < a.F)
          v = __ldg(reinterpret_cast<const float4*>(x + (m + (long long)dt * a.F + df) * CIN) + q);
      }
      reinterpret_cast<float4*>(xs)[i] = v;
    }
    for (int i = threadIdx.x; i < WG_CHUNK * COUT / 4; i += blockDim.x) {
      const int r = i / (COUT / 4), q = i % (COUT / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < n) v = __ldg(reinterpret_cast<const float4*>(g + (rc + r) * COUT) + q);
      reinterpret_cast<float4*>(gs)[i] = v;
    }
    __syncthreads();
    if (active) {
      for (int r = lane_r; r < n; r += 4) {
        const float4 xv = *reinterpret_cast<const float4*>(xs + r * CIN + ci0);
        const float4 gv = *reinterpret_cast<const float4*>(gs + r * COUT + co0);
        const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
        const float ga[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], ga[j], acc[i][j]);
      }
    }
  }
  // reduce the 4 RE lanes through shared memory, then write this split's partial
  __syncthreads();
  float* red = xs;   // [4][64][16]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) red[(lane_r * 64 + slot) * 16 + i * 4 + j] = acc[i][j];
  __syncthreads();
  if (lane_r == 0 && active) {
    float* out = a.part + ((((size_t)blockIdx.x * a.n_br + br) * 9 + tap) * CIN) * COUT;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float s = 0.f;
#pragma unroll
        for (int l = 0; l < 4; ++l) s += red[(l * 64 + slot) * 16 + i * 4 + j];
        out[(size_t)(ci0 + i) * COUT + co0 + j] = s;
      }
  }
}

// Sum the per-split partials [S][n_br][9][CIN][COUT] of branch `br` into the master
// gradient layout [COUT][3][3][cin_src] (padded input channels dropped).
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int S, int n_br, int br, int cin, int cout,
                                    int cin_src, float* __restrict__ dW) {
  const int n = cout * 9 * cin_src;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i / (9 * cin_src), rem = i % (9 * cin_src), tap = rem / cin_src, ci = rem % cin_src;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += part[((((size_t)k * n_br + br) * 9 + tap) * cin + ci) * cout + co];
    dW[i] = s;
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// dgrad weights: Wd[tap'][co][ci] = W[co][8 - tap'][ci]  (conv of dz with the kernel
// rotated by 180 degrees, input and output channels exchanged) for W [cout][3][3][cin]
__global__ void weights_dgrad_kernel(const float* __restrict__ w, int cout, int cin, float* __restrict__ out) {
  const int n = 9 * cout * cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin, rem = i / cin, co = rem % cout, tp = rem / cout;
    out[i] = w[((size_t)co * 9 + (8 - tp)) * cin + ci];
  }
}

// Backward of the concatenation interaction (op 2) of a plain network: the main's fused
// activation x = [u_0, u_1, ...] (W = n_br x C channels, the supports' rows with the main's
// subtracted again when Example II's feedback added it in place) with the gradient gx0
// [M][W]; through the LayerNorm over W when ln_g is set, each branch's slice goes back to
// its activation, plus the support's own stream gradient gxs[b], plus (feedback) every
// support's stream gradient into the main; then the ReLU mask of the activation.
__global__ void __launch_bounds__(EW_THREADS) concat_fuse_bwd_kernel(FuseBwdArgs a) {
  constexpr int CPL = 4;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C, W = a.n_br * a.C;
  float pv[2][CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) pv[0][j] = pv[1][j] = 0.f;
  for (long long m = warp0; m < a.M; m += nwarps) {
    float x[CPL], g[CPL], dx[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      x[j] = g[j] = 0.f;
      if (c < W) {
        const int b = c / C, cc = c % C;
        float v = a.u[b][m * C + cc];
        if (a.feedback && b > 0) v -= a.u[0][m * C + cc];
        x[j] = v;
        g[j] = a.gx0[m * W + c];
      }
    }
    if (a.ln_g) {
      ln_backward(x, g, a.ln_g, W, lane, dx, pv[0], pv[1]);
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) dx[j] = g[j];
    }
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      if (c >= W) continue;
      const int b = c / C, cc = c % C;
      float o = dx[j];
      if (b > 0 && a.gxs[b]) o += a.gxs[b][m * C + cc];
      if (b == 0 && a.feedback)
        for (int s = 1; s < a.n_br; ++s)
          if (a.gxs[s]) o += a.gxs[s][m * C + cc];
      if (a.relu_mask && !(x[j] > 0.f)) o = 0.f;
      a.gu[b][m * C + cc] = o;
    }
  }
  if (a.part) block_store_partials<2, CPL>(pv, W, a.part);
}

}  // namespace

int ew_grid(long long M) { return grid_for(M * 32, EW_THREADS, EW_PART_CTAS); }

int launch_fuse_bwd(const FuseBwdArgs& a, cudaStream_t s) {
  if (a.fuse && a.op == 2) {
    if (a.n_br * a.C > 128) return fail(CONET_ERR_UNSUPPORTED, "concatenated width %d > 128", a.n_br * a.C);
    concat_fuse_bwd_kernel<<<ew_grid(a.M), EW_THREADS, 0, s>>>(a);
    return check_launch("concat_fuse_bwd_kernel");
  }
  const int cpl = (a.C + 31) / 32;
  if (cpl < 1 || cpl > 4) return fail(CONET_ERR_UNSUPPORTED, "width %d > 128", a.C);
  const int g = ew_grid(a.M);
  if (cpl == 1) fuse_bwd_kernel<1><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 2) fuse_bwd_kernel<2><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 3) fuse_bwd_kernel<3><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 4) fuse_bwd_kernel<4><<<g, EW_THREADS, 0, s>>>(a);
  return check_launch("fuse_bwd_kernel");
}

int launch_ln_relu_bwd(const LnReluBwdArgs& a, cudaStream_t s) {
  const int cpl = (a.C + 31) / 32;
  if (cpl < 1 || cpl > 4) return fail(CONET_ERR_UNSUPPORTED, "width %d > 128", a.C);
  const int g = ew_grid(a.M);
  if (cpl == 1) ln_relu_bwd_kernel<1><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 2) ln_relu_bwd_kernel<2><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 3) ln_relu_bwd_kernel<3><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 4) ln_relu_bwd_kernel<4><<<g, EW_THREADS, 0, s>>>(a);
  return check_launch("ln_relu_bwd_kernel");
}

int launch_head_bwd(const HeadBwdArgs& a, cudaStream_t s) {
  if (a.Q > 8) return fail(CONET_ERR_UNSUPPORTED, "Q > 8");
  const int cpl = (a.C + 31) / 32;
  if (cpl < 1 || cpl > 4) return fail(CONET_ERR_UNSUPPORTED, "width %d > 128", a.C);
  const int g = ew_grid(a.M);
  if (cpl == 1) head_bwd_kernel<1><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 2) head_bwd_kernel<2><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 3) head_bwd_kernel<3><<<g, EW_THREADS, 0, s>>>(a);
  if (cpl == 4) head_bwd_kernel<4><<<g, EW_THREADS, 0, s>>>(a);
  return check_launch("head_bwd_kernel");
}

int launch_channel_sums(const float* gr, long long M, int C, float* part, cudaStream_t s) {
  const int cpl = (C + 31) / 32;
  if (cpl < 1 || cpl > 4) return fail(CONET_ERR_UNSUPPORTED, "width %d > 128", C);
  const int g = ew_grid(M);
  if (cpl == 1) channel_sums_kernel<1><<<g, EW_THREADS, 0, s>>>(gr, M, C, part);
  if (cpl == 2) channel_sums_kernel<2><<<g, EW_THREADS, 0, s>>>(gr, M, C, part);
  if (cpl == 3) channel_sums_kernel<3><<<g, EW_THREADS, 0, s>>>(gr, M, C, part);
  if (cpl == 4) channel_sums_kernel<4><<<g, EW_THREADS, 0, s>>>(gr, M, C, part);
  return check_launch("channel_sums_kernel");
}

int launch_reduce_partials(const float* part, int n_part, int n, float* out, int accumulate, cudaStream_t s) {
  reduce_partials_kernel<<<(n + 31) / 32, 256, 0, s>>>(part, n_part, n, out, accumulate);
  return check_launch("reduce_partials_kernel");
}

// Weight gradient on the FP32 FMA pipes as a split-K GEMM: one CTA per (RE range, branch)
// computes the whole [tap][ci] x [co] block (9 CIN x COUT) of that range, each thread an
// 8 x 8 sub-block (8 input channels of one tap x 8 output channels) with packed two-lane
// FMAs.  REs go through shared memory in chunks of RC: the grad rows of the chunk and, per
// symbol shift dt, the input rows m + dt F - 1 .. m + dt F + RC (the subcarrier halo),
// with a per-RE mask of the taps whose shifted position lies in the grid (zero padding).
// Partials go to part[split][branch][tap][ci][co], summed in a fixed order afterwards.
namespace {

constexpr int WT_RC = 64;

__device__ __forceinline__ unsigned long long wt_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ void wt_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ void wt_fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

template <int CIN, int COUT>
__global__ void __launch_bounds__((9 * CIN / 8) * (COUT / 8)) wgrad_tiled_kernel(WgradArgs a, int S) {
  constexpr int NT = (9 * CIN / 8) * (COUT / 8);
  constexpr int XR = WT_RC + 2;          // input rows per symbol shift
  constexpr int XS = CIN + 4;            // padded row (shifts rows across banks)
  extern __shared__ float4 wt_smem4[];
  float* xs = reinterpret_cast<float*>(wt_smem4);   // [3][XR][XS]
  float* gs = xs + 3 * XR * XS;                     // [WT_RC][COUT]
  int* mk = reinterpret_cast<int*>(gs + WT_RC * COUT);   // [WT_RC]
  const int br = blockIdx.y, split = blockIdx.x, tid = threadIdx.x;
  const int rbk = tid / (COUT / 8), cbk = tid % (COUT / 8);
  const int tap = rbk / (CIN / 8), ci0 = (rbk % (CIN / 8)) * 8, co0 = cbk * 8;
  const int dt = tap / 3 - 1, df = tap % 3 - 1;
  const long long M = a.M;
  const int T = a.T, F = a.F, TF = T * F;
  const float* __restrict__ x = a.x[br];
  const float* __restrict__ g = a.g[br];
  const long long per = ((M + S - 1) / S + WT_RC - 1) / WT_RC * WT_RC;
  const long long r0 = (long long)split * per, r1 = r0 + per < M ? r0 + per : M;
  unsigned long long acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[i][p] = 0ull;
  for (long long c0 = r0; c0 < r1; c0 += WT_RC) {
    const int n = r1 - c0 < WT_RC ? (int)(r1 - c0) : WT_RC;
    __syncthreads();
    for (int idx = tid; idx < 3 * XR * (CIN / 4); idx += NT) {
      const int sft = idx / (XR * (CIN / 4)), rem = idx % (XR * (CIN / 4)), i = rem / (CIN / 4), q = rem % (CIN / 4);
      const long long row = c0 + (long long)(sft - 1) * F - 1 + i;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i <= n + 1 && row >= 0 && row < M) v = __ldg(reinterpret_cast<const float4*>(x + row * CIN) + q);
      *reinterpret_cast<float4*>(xs + (sft * XR + i) * XS + 4 * q) = v;
    }
    for (int idx = tid; idx < WT_RC * (COUT / 4); idx += NT) {
      const int i = idx / (COUT / 4), q = idx % (COUT / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < n) v = __ldg(reinterpret_cast<const float4*>(g + (c0 + i) * COUT) + q);
      *reinterpret_cast<float4*>(gs + i * COUT + 4 * q) = v;
    }
    for (int i = tid; i < WT_RC; i += NT) {
      int bits = 0;
      if (i < n) {
        const int tf = (int)((c0 + i) % TF), t = tf / F, f = tf % F;
#pragma unroll
        for (int tp = 0; tp < 9; ++tp) {
          const int tt = t + tp / 3 - 1, ff = f + tp % 3 - 1;
          if (tt >= 0 && tt < T && ff >= 0 && ff < F) bits |= 1 << tp;
        }
      }
      mk[i] = bits;
    }
    __syncthreads();
    const float* xrow = xs + (dt + 1) * XR * XS + (1 + df) * XS + ci0;
    for (int i = 0; i < n; ++i) {
      const bool on = (mk[i] >> tap) & 1;
      float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
      if (on) {
        xa = *reinterpret_cast<const float4*>(xrow + i * XS);
        xb = *reinterpret_cast<const float4*>(xrow + i * XS + 4);
      }
      const float4 ga = *reinterpret_cast<const float4*>(gs + i * COUT + co0);
      const float4 gb = *reinterpret_cast<const float4*>(gs + i * COUT + co0 + 4);
      const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
      const unsigned long long gp[4] = {wt_pack(ga.x, ga.y), wt_pack(ga.z, ga.w), wt_pack(gb.x, gb.y),
                                        wt_pack(gb.z, gb.w)};
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const unsigned long long xd = wt_pack(xv[r], xv[r]);
#pragma unroll
        for (int p = 0; p < 4; ++p) wt_fma2(acc[r][p], xd, gp[p]);
      }
    }
  }
  float* out = a.part + ((((size_t)split * a.n_br + br) * 9 + tap) * CIN + ci0) * COUT + co0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float v[8];
#pragma unroll
    for (int p = 0; p < 4; ++p) wt_unpack(acc[r][p], v[2 * p], v[2 * p + 1]);
    reinterpret_cast<float4*>(out + r * COUT)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(out + r * COUT)[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

template <int CIN, int COUT>
int launch_wgrad_tiled_t(const WgradArgs& a, int S, cudaStream_t s) {
  constexpr int NT = (9 * CIN / 8) * (COUT / 8);
  constexpr size_t smem = (size_t)(3 * (WT_RC + 2) * (CIN + 4) + WT_RC * COUT) * sizeof(float) + WT_RC * sizeof(int);
  static bool attr = false;
  if (!attr) {
    CONET_CUDA(cudaFuncSetAttribute(wgrad_tiled_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    attr = true;
  }
  wgrad_tiled_kernel<CIN, COUT><<<dim3(S, a.n_br), NT, smem, s>>>(a, S);
  return check_launch("wgrad_tiled_kernel");
}

}  // namespace

int wgrad_tiled_splits(long long M, int n_br) {
  long long s = (long long)WG_TILED_MAX_CTAS / n_br;
  const long long by_size = (M + 4 * WT_RC - 1) / (4 * WT_RC);   // >= 256 REs per split
  if (s > by_size) s = by_size;
  return s < 1 ? 1 : (int)s;
}

// dW[co][tap][ci] (ci < cin_src) = sum over splits k of part[k][br][tap][ci][co]: CTAs over
// groups of 32 consecutive (tap, ci, co), 8 warps striding the splits, a fixed combine order.
__global__ void __launch_bounds__(256) wgrad_reduce_rows_kernel(const float* __restrict__ part, int S, int n_br,
                                                                int br, int cin, int cout, int cin_src,
                                                                float* __restrict__ dW) {
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = 9 * cin * cout;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < n)
    for (int k = w; k < S; k += 8) s += part[((size_t)k * n_br + br) * n + j];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < n) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    const int co = j % cout, rem = j / cout, ci = rem % cin, tap = rem / cin;
    if (ci < cin_src) dW[((size_t)co * 9 + tap) * cin_src + ci] = t;
  }
}

int launch_wgrad_reduce(const float* part, int S, int n_br, int br, int cin, int cout, int cin_src, float* dW,
                        cudaStream_t s) {
  wgrad_reduce_rows_kernel<<<(9 * cin * cout + 31) / 32, 256, 0, s>>>(part, S, n_br, br, cin, cout, cin_src, dW);
  return check_launch("wgrad_reduce_rows_kernel");
}

int launch_wgrad_tiled(const WgradArgs& a, cudaStream_t s) {
  const int S = wgrad_tiled_splits(a.M, a.n_br);
  int rc = CONET_ERR_UNSUPPORTED;
#define WT_CASE(CI, CO) \
  else if (a.cin == CI && a.cout == CO) rc = launch_wgrad_tiled_t<CI, CO>(a, S, s);
  if (false) {
  }
  WT_CASE(8, 16)
  WT_CASE(16, 16)
  WT_CASE(8, 32)
  WT_CASE(32, 32)
  WT_CASE(8, 64)
  WT_CASE(64, 64)
#undef WT_CASE
  else return launch_wgrad(a, s);   // other shapes: the general kernel
  CONET_TRY(rc);
  for (int b = 0; b < a.n_br; ++b) {
    wgrad_reduce_rows_kernel<<<(9 * a.cin * a.cout + 31) / 32, 256, 0, s>>>(a.part, S, a.n_br, b, a.cin, a.cout,
                                                                             a.cin_src[b], a.dW[b]);
    CONET_LAUNCHED("wgrad_reduce_rows_kernel");
  }
  return CONET_OK;
}

int wgrad_splits(long long M, int cin, int cout, int n_br) {
  const int chunks = ((cin / 4) * (cout / 4) + 63) / 64;
  long long s = (152LL * 4) / (9LL * chunks * n_br);
  if (s < 1) s = 1;
  if (s > WG_MAX_SPLITS) s = WG_MAX_SPLITS;
  const long long by_size = (M + 4 * WG_CHUNK - 1) / (4 * WG_CHUNK);   // >= 128 REs per split
  if (s > by_size) s = by_size < 1 ? 1 : by_size;
  return (int)s;
}

size_t wgrad_partial_floats(long long M, int cin, int cout, int n_br) {
  return (size_t)wgrad_splits(M, cin, cout, n_br) * n_br * 9 * cin * cout;
}

int launch_wgrad(const WgradArgs& a, cudaStream_t s) {
  if (a.cin % 4 || a.cout % 4 || a.cin > 128 || a.cout > 128) return fail(CONET_ERR_UNSUPPORTED, "wgrad channels");
  const int S = wgrad_splits(a.M, a.cin, a.cout, a.n_br);
  const int chunks = ((a.cin / 4) * (a.cout / 4) + 63) / 64;
  const size_t smem = (size_t)WG_CHUNK * (a.cin + a.cout) * sizeof(float);
  const size_t red = 4 * 64 * 16 * sizeof(float);
  const size_t sm = smem > red ? smem : red;
  dim3 grid(S, 9 * chunks, a.n_br);
  wgrad_kernel<<<grid, 256, sm, s>>>(a);
  CONET_LAUNCHED("wgrad_kernel");
  for (int b = 0; b < a.n_br; ++b) {
    wgrad_reduce_kernel<<<grid_for((long long)a.cout * 9 * a.cin_src[b], 256, 512), 256, 0, s>>>(
        a.part, S, a.n_br, b, a.cin, a.cout, a.cin_src[b], a.dW[b]);
    CONET_LAUNCHED("wgrad_reduce_kernel");
  }
  return CONET_OK;
}

int launch_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                float bc1, float bc2, cudaStream_t s) {
  adam_kernel<<<grid_for((long long)n, 256, 152 * 8), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
  return check_launch("adam_kernel");
}

int launch_weights_dgrad_layout(const float* w, int cout, float* out, cudaStream_t s, int cin) {
  if (cin <= 0) cin = cout;
  weights_dgrad_kernel<<<grid_for(9LL * cout * cin, 256, 512), 256, 0, s>>>(w, cout, cin, out);
  return check_launch("weights_dgrad_kernel");
}

__global__ void zero_input_channels_kernel(float* __restrict__ w, int n, int cin, unsigned keep) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!((keep >> (i % cin)) & 1u)) w[i] = 0.f;
}

int launch_zero_input_channels(float* w, int cout, int cin, unsigned keep, cudaStream_t s) {
  if (cin > 32) return fail(CONET_ERR_ARG, "input channel mask over %d channels", cin);
  const int n = cout * 9 * cin;
  zero_input_channels_kernel<<<grid_for(n, 256), 256, 0, s>>>(w, n, cin, keep);
  return check_launch("zero_input_channels_kernel");
}

}  // namespace conet
