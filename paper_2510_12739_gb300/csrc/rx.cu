// Receiver-side DSP kernels: network input assembly (Sec. II-A), the LS-LMMSE baseline
// receiver with exact / max-log demapping (Sec. I, Sec. IV baselines), and the fused
// BCE-loss / bit-error counter over data REs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace conet {

// One thread per RE: channels Re Y_n, Im Y_n, mask, Re/Im of the antenna-averaged LS
// estimate y conj(p) / |p|^2 at pilots; zero padding up to c_pad channels (<= 16).
template <typename Out>
__global__ void assemble_kernel(const float2* __restrict__ Y, const uint8_t* __restrict__ mask,
                                const float2* __restrict__ psym, int B, int N, int T, int F, int c_pad,
                                Out* __restrict__ X0) {
  const long long TF = (long long)T * F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * TF;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / TF, r = i % TF;
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.f;
    const bool pil = mask[r] != 0;
    const float2 p = psym[r];
    const float inv = pil ? 1.0f / (p.x * p.x + p.y * p.y) : 0.f;
    float hr = 0.f, hi = 0.f;
    for (int n = 0; n < N; ++n) {
      const float2 y = Y[(b * N + n) * TF + r];
      v[n] = y.x;
      v[N + n] = y.y;
      hr += (y.x * p.x + y.y * p.y) * inv;     // y conj(p) / |p|^2
      hi += (y.y * p.x - y.x * p.y) * inv;
    }
    v[2 * N] = pil ? 1.f : 0.f;
    v[2 * N + 1] = hr / (float)N;
    v[2 * N + 2] = hi / (float)N;
    Out* o = X0 + i * c_pad;
    if constexpr (sizeof(Out) == 4) {
      if (c_pad % 4 == 0) {
        for (int c = 0; c < c_pad; c += 4)
          *reinterpret_cast<float4*>(o + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
      } else {
        for (int c = 0; c < c_pad; ++c) o[c] = v[c];
      }
    } else {
      for (int c = 0; c < c_pad; c += 8) {
        __align__(16) Out h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = Out(v[c + j]);
        *reinterpret_cast<uint4*>(o + c) = *reinterpret_cast<uint4*>(h);
      }
    }
  }
}

int launch_assemble(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F, int c_pad,
                    float* X0, cudaStream_t s) {
  const long long n = (long long)B * T * F;
  assemble_kernel<float><<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float2*>(Y), mask,
                                                          reinterpret_cast<const float2*>(psym), B, N, T, F,
                                                          c_pad, X0);
  return check_launch("assemble_kernel");
}

int launch_assemble_16(int kind, const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                       int c_pad, void* X0, cudaStream_t s) {
  const long long n = (long long)B * T * F;
  if (kind == 3)
    assemble_kernel<__half><<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float2*>(Y), mask,
                                                             reinterpret_cast<const float2*>(psym), B, N, T, F, c_pad,
                                                             reinterpret_cast<__half*>(X0));
  else
    assemble_kernel<__nv_bfloat16><<<grid_for(n, 256), 256, 0, s>>>(
        reinterpret_cast<const float2*>(Y), mask, reinterpret_cast<const float2*>(psym), B, N, T, F, c_pad,
        reinterpret_cast<__nv_bfloat16*>(X0));
  return check_launch("assemble_kernel_16");
}

// Same channels as assemble_kernel, written as TF32 hi parts and FP32 lo = x - hi.
__global__ void assemble_split_kernel(const float2* __restrict__ Y, const uint8_t* __restrict__ mask,
                                      const float2* __restrict__ psym, int B, int N, int T, int F, int c_pad,
                                      float* __restrict__ hi, float* __restrict__ lo) {
  const long long TF = (long long)T * F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * TF;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / TF, r = i % TF;
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.f;
    const bool pil = mask[r] != 0;
    const float2 p = psym[r];
    const float inv = pil ? 1.0f / (p.x * p.x + p.y * p.y) : 0.f;
    float hr = 0.f, hq = 0.f;
    for (int n = 0; n < N; ++n) {
      const float2 y = Y[(b * N + n) * TF + r];
      v[n] = y.x;
      v[N + n] = y.y;
      hr += (y.x * p.x + y.y * p.y) * inv;
      hq += (y.y * p.x - y.x * p.y) * inv;
    }
    v[2 * N] = pil ? 1.f : 0.f;
    v[2 * N + 1] = hr / (float)N;
    v[2 * N + 2] = hq / (float)N;
    for (int c = 0; c < c_pad; c += 4) {
      float h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v[c + j]));
        h[j] = __uint_as_float(u);
        l[j] = v[c + j] - h[j];
      }
      *reinterpret_cast<float4*>(hi + i * c_pad + c) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(lo + i * c_pad + c) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

int launch_assemble_split(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                          int c_pad, float* hi, float* lo, cudaStream_t s) {
  const long long n = (long long)B * T * F;
  assemble_split_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float2*>(Y), mask,
                                                         reinterpret_cast<const float2*>(psym), B, N, T, F, c_pad,
                                                         hi, lo);
  return check_launch("assemble_split_kernel");
}

// Same channels as assemble_kernel (c_pad <= 32), written as E4M3 of value * qinv[0]; with
// X0 == NULL the kernel only folds the largest |value| into *amax.
__global__ void assemble_fp8_kernel(const float2* __restrict__ Y, const uint8_t* __restrict__ mask,
                                    const float2* __restrict__ psym, int B, int N, int T, int F, int c_pad,
                                    const float* __restrict__ qinv, uint8_t* __restrict__ X0,
                                    unsigned* __restrict__ amax) {
  const long long TF = (long long)T * F;
  const float qi = X0 ? *qinv : 1.f;
  float mx = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * TF;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / TF, r = i % TF;
    float v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = 0.f;
    const bool pil = mask[r] != 0;
    const float2 p = psym[r];
    const float inv = pil ? 1.0f / (p.x * p.x + p.y * p.y) : 0.f;
    float hr = 0.f, hq = 0.f;
    for (int n = 0; n < N; ++n) {
      const float2 y = Y[(b * N + n) * TF + r];
      v[n] = y.x;
      v[N + n] = y.y;
      hr += (y.x * p.x + y.y * p.y) * inv;
      hq += (y.y * p.x - y.x * p.y) * inv;
    }
    v[2 * N] = pil ? 1.f : 0.f;
    v[2 * N + 1] = hr / (float)N;
    v[2 * N + 2] = hq / (float)N;
    if (!X0) {
#pragma unroll
      for (int c = 0; c < 32; ++c) mx = fmaxf(mx, fabsf(v[c]));
      continue;
    }
    for (int c = 0; c < c_pad; c += 16) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[c + 4 * j] * qi, v[c + 4 * j + 1] * qi),
                                                     __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[c + 4 * j + 2] * qi, v[c + 4 * j + 3] * qi),
                                                     __NV_SATFINITE, __NV_E4M3);
        w[j] = (lo & 0xFFFFu) | (hi << 16);
      }
      *reinterpret_cast<uint4*>(X0 + i * c_pad + c) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  if (!X0) {
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(amax, __float_as_uint(mx));
  }
}

int launch_assemble_fp8(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                        int c_pad, const float* qinv, uint8_t* X0, unsigned* amax, cudaStream_t s) {
  if (c_pad != 32 || 2 * N + 3 > 32) return fail(CONET_ERR_UNSUPPORTED, "E4M3 input assembly pads to 32 channels");
  const long long n = (long long)B * T * F;
  assemble_fp8_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float2*>(Y), mask,
                                                       reinterpret_cast<const float2*>(psym), B, N, T, F, c_pad, qinv,
                                                       X0, amax);
  return check_launch("assemble_fp8_kernel");
}

// ------------------------------------------------------------------ LS-LMMSE
__device__ __forceinline__ float2 cmul_conj(float2 y, float2 p) {   // y conj(p)
  return make_float2(y.x * p.x + y.y * p.y, y.y * p.x - y.x * p.y);
}

__device__ __forceinline__ float2 ls_at(const LmmseArgs& a, const float2* Yn, int tp, int f) {
  const int r = tp * a.F + f;
  const float2 p = reinterpret_cast<const float2*>(a.psym)[r];
  const float inv = 1.0f / (p.x * p.x + p.y * p.y);
  const float2 v = cmul_conj(Yn[r], p);
  return make_float2(v.x * inv, v.y * inv);
}

// Linear interpolation across the pilot comb of symbol tp (constant beyond the last).
__device__ __forceinline__ float2 ls_row(const LmmseArgs& a, const float2* Yn, int tp, int f) {
  const int c = a.comb;
  const int f0 = (f / c) * c;
  if (f0 == f) return ls_at(a, Yn, tp, f);
  const int f1 = f0 + c;
  const float2 v0 = ls_at(a, Yn, tp, f0);
  if (f1 >= a.F) return v0;
  const float2 v1 = ls_at(a, Yn, tp, f1);
  const float w = (float)(f - f0) / (float)c;
  return make_float2(v0.x + w * (v1.x - v0.x), v0.y + w * (v1.y - v0.y));
}

// Per-axis demapping of square Gray QAM: the quadrature factor cancels in the LLR of an
// in-phase bit (and vice versa), so each axis needs only its sqrt(M) PAM levels.
__device__ void demap_axis(float xv, float mu, float nu, int half, float scale, int exact, float* out,
                           int stride) {
  const int P = 1 << half;
  float m1[4], m0[4], s1[4], s0[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    m1[j] = m0[j] = -INFINITY;
    s1[j] = s0[j] = 0.f;
  }
  for (int i = 0; i < P; ++i) {
    const float lv = (2.0f * (float)i - (float)(P - 1)) * scale;
    const float d = xv - mu * lv;
    const float e = -d * d / nu;
    const int g = i ^ (i >> 1);
    for (int j = 0; j < half; ++j) {
      const int bit = (g >> (half - 1 - j)) & 1;
      float& m = bit ? m1[j] : m0[j];
      float& s = bit ? s1[j] : s0[j];
      if (exact) {
        if (e > m) {
          s = s * __expf(m - e) + 1.0f;
          m = e;
        } else {
          s += __expf(e - m);
        }
      } else {
        m = fmaxf(m, e);
      }
    }
  }
  for (int j = 0; j < half; ++j)
    out[j * stride] = exact ? (m1[j] + logf(s1[j])) - (m0[j] + logf(s0[j])) : m1[j] - m0[j];
}

__global__ void ls_lmmse_kernel(LmmseArgs a) {
  const long long TF = (long long)a.T * a.F;
  const int half = a.Q / 2;
  const float scale = rsqrtf(2.0f * (float)((1 << a.Q) - 1) / 3.0f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)a.B * TF;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / TF;
    const int r = (int)(i % TF), t = r / a.F, f = r % a.F;
    // time interpolation weights between pilot symbols (constant outside)
    int j0 = 0, j1 = 0;
    float wt = 0.f;
    const int np = a.n_pilot_syms;
    if (t <= a.pilot_syms[0]) {
      j0 = j1 = 0;
    } else if (t >= a.pilot_syms[np - 1]) {
      j0 = j1 = np - 1;
    } else {
      for (int j = 0; j + 1 < np; ++j)
        if (a.pilot_syms[j] <= t && t < a.pilot_syms[j + 1]) {
          j0 = j;
          j1 = j + 1;
          wt = (float)(t - a.pilot_syms[j]) / (float)(a.pilot_syms[j + 1] - a.pilot_syms[j]);
        }
    }
    float g = 0.f, nr = 0.f, ni = 0.f;
    for (int n = 0; n < a.N; ++n) {
      const float2* Yn = reinterpret_cast<const float2*>(a.Y) + (b * a.N + n) * TF;
      float2 h;
      if (a.Hp) {
        h = reinterpret_cast<const float2*>(a.Hp)[(b * a.N + n) * TF + r];
      } else {
        const float2 h0 = ls_row(a, Yn, a.pilot_syms[j0], f);
        const float2 h1 = j1 == j0 ? h0 : ls_row(a, Yn, a.pilot_syms[j1], f);
        h = make_float2(h0.x + wt * (h1.x - h0.x), h0.y + wt * (h1.y - h0.y));
      }
      const float2 y = Yn[r];
      g += h.x * h.x + h.y * h.y;
      nr += h.x * y.x + h.y * y.y;    // conj(h) y
      ni += h.x * y.y - h.y * y.x;
    }
    float s2 = a.noise_var[b];
    if (a.interf_var) s2 += a.interf_var[b];
    const float den = g + s2;
    const float xr = nr / den, xi = ni / den;
    const float mu = g / den;
    const float nu = fmaxf(mu * (1.0f - mu), 1e-12f);
    float* out = a.llr + i * a.Q;
    demap_axis(xr, mu, nu, half, scale, a.exact, out, 2);       // b_0, b_2, ...
    demap_axis(xi, mu, nu, half, scale, a.exact, out + 1, 2);   // b_1, b_3, ...
  }
}

int launch_ls_lmmse(const LmmseArgs& a, cudaStream_t s) {
  const long long n = (long long)a.B * a.T * a.F;
  ls_lmmse_kernel<<<grid_for(n, 256), 256, 0, s>>>(a);
  return check_launch("ls_lmmse_kernel");
}

// ------------------------------------------------------------------ BCE + bit errors
__global__ void loss_ber_kernel(const float* __restrict__ llr, const uint8_t* __restrict__ bits,
                                const uint8_t* __restrict__ mask, long long n_re, int TF, int Q,
                                float grad_scale, float* __restrict__ dllr, double* loss_sum,
                                unsigned long long* err, unsigned long long* nbits) {
  double loss = 0.0;
  unsigned long long e = 0, nb = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_re;
       i += (long long)gridDim.x * blockDim.x) {
    const bool pil = mask[i % TF] != 0;
    for (int q = 0; q < Q; ++q) {
      const long long o = i * Q + q;
      if (pil) {
        if (dllr) dllr[o] = 0.f;
        continue;
      }
      const float L = llr[o];
      const float b = bits[o] ? 1.f : 0.f;
      loss += (double)(fmaxf(L, 0.f) - b * L + log1pf(__expf(-fabsf(L))));
      e += ((L > 0.f) ? 1u : 0u) != (unsigned)bits[o];
      nb += 1;
      if (dllr) dllr[o] = (1.0f / (1.0f + __expf(-L)) - b) * grad_scale;
    }
  }
  __shared__ double sl[32];
  __shared__ unsigned long long se[32], sn[32];
  loss = warp_sum_d(loss);
  e = warp_sum_u64(e);
  nb = warp_sum_u64(nb);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sl[wid] = loss;
    se[wid] = e;
    sn[wid] = nb;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    loss = lane < nw ? sl[lane] : 0.0;
    e = lane < nw ? se[lane] : 0ull;
    nb = lane < nw ? sn[lane] : 0ull;
    loss = warp_sum_d(loss);
    e = warp_sum_u64(e);
    nb = warp_sum_u64(nb);
    if (lane == 0) {
      if (loss_sum) atomicAdd(loss_sum, loss);
      if (err) atomicAdd(err, e);
      if (nbits) atomicAdd(nbits, nb);
    }
  }
}

int launch_loss_ber(const float* llr, const uint8_t* bits, const uint8_t* mask, int B, int T, int F, int Q,
                    float grad_scale, float* dllr, double* loss_sum, unsigned long long* err,
                    unsigned long long* nbits, cudaStream_t s) {
  const long long n = (long long)B * T * F;
  loss_ber_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(llr, bits, mask, n, T * F, Q, grad_scale, dllr,
                                                            loss_sum, err, nbits);
  return check_launch("loss_ber_kernel");
}

}  // namespace conet
