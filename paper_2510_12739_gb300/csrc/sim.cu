// Device-side synthetic OFDM link (Sec. II, Eq. 1 of CoNet-Rx): uniform bits -> Gray QAM,
// fixed QPSK pilots, TDL Rayleigh channel with sum-of-sinusoids Doppler, optional
// co-channel QAM interferer with a random time offset, AWGN.  Also the fixed pilot grid
// and the He-normal weight initialiser, which draw from the same Philox generator.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace conet {

__device__ __forceinline__ bool is_pilot(int t, int f, const PilotGrid& pg) {
  if (f % pg.comb) return false;
  for (int i = 0; i < pg.n_syms; ++i)
    if (pg.syms[i] == t) return true;
  return false;
}

__device__ __forceinline__ float2 pilot_symbol(int r, const PilotGrid& pg) {
  const u32x4 w = philox((uint32_t)r, 0u, 0u, TAG_PILOT, pg.k0, pg.k1);
  const float a = 0.70710678118654752f;
  return make_float2((w.x & 1u) ? -a : a, (w.x & 2u) ? -a : a);
}

__global__ void pilots_kernel(int T, int F, PilotGrid pg, uint8_t* mask, float2* psym) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= T * F) return;
  const int t = r / F, f = r % F;
  const bool p = is_pilot(t, f, pg);
  mask[r] = p ? 1 : 0;
  psym[r] = p ? pilot_symbol(r, pg) : make_float2(0.f, 0.f);
}

int launch_pilots(int T, int F, const PilotGrid& pg, uint8_t* mask, float* psym, cudaStream_t s) {
  pilots_kernel<<<(T * F + 255) / 256, 256, 0, s>>>(T, F, pg, mask, reinterpret_cast<float2*>(psym));
  return check_launch("pilots_kernel");
}

// Uniform i (0 = theta, 1..S = phi_s) of tap (n, l): Philox block j = i / 4, word i % 4.
__device__ __forceinline__ float chan_uniform(int i, uint32_t c0, uint32_t slot, uint32_t tag,
                                              uint32_t k0, uint32_t k1) {
  const u32x4 w = philox(c0, (uint32_t)(i >> 2), slot, tag, k0, k1);
  const uint32_t v = (i & 3) == 0 ? w.x : (i & 3) == 1 ? w.y : (i & 3) == 2 ? w.z : w.w;
  return u01(v);
}

// a_{n,l}(t) = sqrt(P_l / S) sum_s exp(j 2 pi (f_D cos(alpha_s) t T_sym + u_s)),
// alpha_s = 2 pi (s + theta) / S.
__device__ float2 tap_gain(int n, int l, int t, float fd, const SimArgs& a, uint32_t slot, uint32_t tag) {
  const uint32_t c0 = (uint32_t)(n * 256 + l);
  const int S = a.n_sin;
  const float theta = chan_uniform(0, c0, slot, tag, a.k0, a.k1);
  const float tt = (float)t * a.t_sym;
  float re = 0.f, im = 0.f;
  for (int s = 0; s < S; ++s) {
    const float ca = cospif(2.0f * ((float)s + theta) / (float)S);
    const float turns = fd * ca * tt + chan_uniform(1 + s, c0, slot, tag, a.k0, a.k1);
    float sn, cs;
    sincospif(2.0f * turns, &sn, &cs);
    re += cs;
    im += sn;
  }
  return make_float2(re * a.amp[l], im * a.amp[l]);
}

constexpr int SIM_TF = 128;   // subcarriers per CTA

__global__ void __launch_bounds__(SIM_TF) sim_kernel(SimArgs a) {
  extern __shared__ float2 sm[];
  const int L = a.n_taps, T = a.T, F = a.F;
  float2* tapH = sm;                         // [L][T]
  float2* tapG = tapH + L * T;               // [L][T] (interferer)
  float2* ef = tapG + L * T;                 // [L][SIM_TF]
  const int n = blockIdx.y, b = blockIdx.z, f0 = blockIdx.x * SIM_TF;
  const uint32_t slot = (uint32_t)(a.slot0 + (uint64_t)b);

  const u32x4 sp = philox(0u, 0u, slot, TAG_SLOT, a.k0, a.k1);
  const float snr = a.fixed_snr ? a.snr_fixed : (a.snr_lo == a.snr_hi ? a.snr_lo : a.snr_lo + (a.snr_hi - a.snr_lo) * u01(sp.x));
  const float fd = a.fd_lo == a.fd_hi ? a.fd_lo : a.fd_lo + (a.fd_hi - a.fd_lo) * u01(sp.y);
  const float sir = a.sir_lo == a.sir_hi ? a.sir_lo : a.sir_lo + (a.sir_hi - a.sir_lo) * u01(sp.z);
  const float delta = (9.0f / 128.0f) * u01(sp.w);
  const float sigma2 = exp10f(-snr / 10.0f);
  const float p_i = a.interferer ? exp10f(-sir / 10.0f) : 0.0f;

  if (!a.awgn) {
    for (int i = threadIdx.x; i < L * T; i += blockDim.x) {
      const int l = i / T, t = i % T;
      tapH[i] = tap_gain(n, l, t, fd, a, slot, TAG_CHAN);
      if (a.interferer) tapG[i] = tap_gain(n, l, t, fd, a, slot, TAG_ICHAN);
    }
    for (int i = threadIdx.x; i < L * SIM_TF; i += blockDim.x) {
      const int l = i / SIM_TF, f = f0 + i % SIM_TF;
      // exp(-j 2 pi k rho_l), k = f - F/2: the phase is reduced to one turn in FP64
      double turns = (double)(f - F / 2) * a.rho[l];
      turns -= rint(turns);
      float sn, cs;
      sincospif(2.0f * (float)turns, &sn, &cs);
      ef[i] = make_float2(cs, -sn);
    }
  }
  __syncthreads();

  const int f = f0 + threadIdx.x;
  if (f >= F) return;
  const float nstd = sqrtf(sigma2 * 0.5f);
  const float istd = sqrtf(p_i);
  float sr = 0.f, cr = 1.f;
  if (a.interferer) sincospif(-2.0f * (float)(f - F / 2) * delta, &sr, &cr);
  for (int t = 0; t < T; ++t) {
    const int r = t * F + f;
    float2 x;
    const bool pil = is_pilot(t, f, a.pg);
    const u32x4 wb = philox((uint32_t)r, 0u, slot, TAG_BITS, a.k0, a.k1);
    if (pil) {
      x = pilot_symbol(r, a.pg);
    } else {
      x = qam_map(wb.x, a.Q);
    }
    float2 h = make_float2(1.f, 0.f), g = make_float2(1.f, 0.f);
    if (!a.awgn) {
      h = make_float2(0.f, 0.f);
      g = make_float2(0.f, 0.f);
      for (int l = 0; l < L; ++l) {
        const float2 e = ef[l * SIM_TF + threadIdx.x];
        const float2 th = tapH[l * T + t];
        h.x += th.x * e.x - th.y * e.y;
        h.y += th.x * e.y + th.y * e.x;
        if (a.interferer) {
          const float2 tg = tapG[l * T + t];
          g.x += tg.x * e.x - tg.y * e.y;
          g.y += tg.x * e.y + tg.y * e.x;
        }
      }
    }
    float yr = h.x * x.x - h.y * x.y;
    float yi = h.x * x.y + h.y * x.x;
    if (a.interferer) {
      const u32x4 wz = philox((uint32_t)r, 0u, slot, TAG_IBITS, a.k0, a.k1);
      const float2 z = qam_map(wz.x, a.iQ);
      const float zr = z.x * cr - z.y * sr, zi = z.x * sr + z.y * cr;   // z e^{-j 2 pi k delta}
      yr += istd * (g.x * zr - g.y * zi);
      yi += istd * (g.x * zi + g.y * zr);
    }
    const u32x4 wn = philox((uint32_t)r, (uint32_t)n, slot, TAG_NOISE, a.k0, a.k1);
    const float rad = sqrtf(-2.0f * logf(u01(wn.x)));
    float s1, c1;
    sincospif(2.0f * u01(wn.y), &s1, &c1);
    yr += nstd * rad * c1;
    yi += nstd * rad * s1;
    const size_t o = (((size_t)b * a.N + n) * T + t) * (size_t)F + f;
    reinterpret_cast<float2*>(a.Y)[o] = make_float2(yr, yi);
    if (a.H) reinterpret_cast<float2*>(a.H)[o] = h;
    if (n == 0) {
      uint8_t* bp = a.bits + ((size_t)b * T * F + r) * a.Q;
      for (int k = 0; k < a.Q; ++k) bp[k] = pil ? 0 : (uint8_t)((wb.x >> k) & 1u);
    }
  }
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    a.noise_var[b] = sigma2;
    if (a.interf_var) a.interf_var[b] = p_i;
  }
}

int launch_sim(const SimArgs& a, int B, cudaStream_t s) {
  if (a.n_taps > MAX_TAPS) return fail(CONET_ERR_UNSUPPORTED, "n_taps > %d", MAX_TAPS);
  const size_t smem = (size_t)(2 * a.n_taps * a.T + a.n_taps * SIM_TF) * sizeof(float2);
  dim3 grid((a.F + SIM_TF - 1) / SIM_TF, a.N, B);
  sim_kernel<<<grid, SIM_TF, smem, s>>>(a);
  return check_launch("sim_kernel");
}

// He-normal initialiser for one parameter segment: value = std * N(0,1) (Box-Muller on
// Philox(TAG_INIT, global index)), or a constant when std < 0 (value = -std - 1 encoding
// avoided: `constant` carries it).
__global__ void init_segment_kernel(float* p, size_t off, size_t n, float std, float constant, int normal,
                                    uint32_t k0, uint32_t k1) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float v = constant;
    if (normal) {
      const size_t gi = off + i;
      const u32x4 w = philox((uint32_t)gi, (uint32_t)(gi >> 32), 0u, TAG_INIT, k0, k1);
      const float rad = sqrtf(-2.0f * logf(u01(w.x)));
      v = std * rad * cospif(2.0f * u01(w.y));
    }
    p[off + i] = v;
  }
}

int launch_init_segment(float* p, size_t off, size_t n, float std, float constant, int normal, uint64_t seed,
                        cudaStream_t s) {
  init_segment_kernel<<<grid_for((long long)n, 256, 1024), 256, 0, s>>>(
      p, off, n, std, constant, normal, (uint32_t)seed, (uint32_t)(seed >> 32));
  return check_launch("init_segment_kernel");
}

}  // namespace conet
