// FP32 3x3 'same' convolution of channels-last activations [B][T][F][C] as an implicit
// GEMM on the FP32 FFMA pipes (the exact-FP32 path).  M = B*T*F resource elements,
// N = Cout, K = 9*Cin (tap-major, input channel fastest).  One launch covers every
// branch of a layer (blockIdx.y).  A CTA owns 128 consecutive REs x all Cout channels, so
// the epilogue can apply bias, residual add, ReLU and a per-RE LayerNorm in place.
//
// Each thread accumulates an 8 x 8 register tile: REs {4r..4r+3, 64+4r..64+4r+3} and
// channels {4c..4c+3, Cout/2+4c..Cout/2+4c+3}.  Splitting both sets in halves makes every
// 8-thread shared-memory phase read one contiguous 128-byte row (no bank conflicts) while
// one k step costs four 128-bit loads for 64 FMAs, issued as 32 packed two-lane FP32 FMAs
// (fma.rn.f32x2: each lane rounds exactly like fmaf, so results equal the scalar form).
#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

constexpr int TM = 128;   // REs per CTA
constexpr int HM = TM / 2;

// (lo, hi) as one 64-bit register pair, and back.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// d.lo += a.lo * b.lo, d.hi += a.hi * b.hi, each a fused multiply-add rounded to nearest.
__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// TAPS = 9: the 3x3 conv; TAPS = 1: a 1x1 conv (the pointwise half of a depthwise-separable
// conv), the same GEMM with only the centre tap and weights [1][Cin][Cout].
template <int CIN, int COUT, int KC, int TAPS = 9>
__global__ void __launch_bounds__(COUT * 2, (COUT <= 64 ? 4 : 2)) conv3x3_fp32_kernel(ConvArgs a) {
  constexpr int NT = COUT * 2;            // (COUT/8) channel groups x 16 RE groups
  constexpr int CG = COUT / 8;
  constexpr int HC = COUT / 2;
  constexpr int NCH = TAPS * (CIN / KC);  // K chunks
  constexpr int A_F4 = TM * KC / 4;
  constexpr int A_PER_T = (A_F4 + NT - 1) / NT;
  constexpr int B_F4 = KC * COUT / 4;
  constexpr int B_PER_T = (B_F4 + NT - 1) / NT;
  constexpr int CS = COUT + 4;            // padded row of the epilogue tile
  static_assert(COUT % 8 == 0 && CIN % KC == 0 && KC % 4 == 0, "tile shape");

  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* As = smem;                       // [2][KC][TM]
  float* Bs = As + 2 * KC * TM;           // [2][KC][COUT]

  const int br = blockIdx.y;
  // The epilogue takes the branch (and so its pointers) from shared memory, which keeps the
  // compiler from computing them ahead of the main loop: measured 3 % faster at Cout = 64.
  __shared__ int cta_br;
  if (threadIdx.x == 0) cta_br = br;
  const float* __restrict__ in = a.in[br];
  const float* __restrict__ w = a.w[br];
  const int tid = threadIdx.x;
  const int cg = tid % CG, rg = tid / CG;
  const long long m0 = (long long)blockIdx.x * TM;
  const int T = a.T, F = a.F, TF = T * F;

  int a_re[A_PER_T], a_q[A_PER_T], a_t[A_PER_T], a_f[A_PER_T];
  bool a_ok[A_PER_T], a_st[A_PER_T];
#pragma unroll
  for (int j = 0; j < A_PER_T; ++j) {
    const int idx = tid + j * NT;
    a_st[j] = idx < A_F4;
    a_re[j] = idx / (KC / 4);
    a_q[j] = idx % (KC / 4);
    const long long m = m0 + a_re[j];
    a_ok[j] = a_st[j] && m < a.M;
    const int r = (int)(m % TF);
    a_t[j] = r / F;
    a_f[j] = r % F;
  }
  float4 ra[A_PER_T], rb[B_PER_T];

  auto load_chunk = [&](int c) {
    const int wtap = c / (CIN / KC), ci0 = (c % (CIN / KC)) * KC;   // tap index in the weights
    const int tap = TAPS == 9 ? wtap : 4;                           // grid shift (4 = centre)
    const int dt = tap / 3 - 1, df = tap % 3 - 1;
#pragma unroll
    for (int j = 0; j < A_PER_T; ++j) {
      const int tt = a_t[j] + dt, ff = a_f[j] + df;
      if (a_ok[j] && tt >= 0 && tt < T && ff >= 0 && ff < F) {
        const long long m = m0 + a_re[j] + (long long)dt * F + df;
        ra[j] = __ldg(reinterpret_cast<const float4*>(in + m * CIN + ci0) + a_q[j]);
      } else {
        ra[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int j = 0; j < B_PER_T; ++j) {
      const int idx = tid + j * NT;
      if (idx < B_F4) rb[j] = __ldg(reinterpret_cast<const float4*>(w + (size_t)(wtap * CIN + ci0) * COUT) + idx);
    }
  };
  auto store_chunk = [&](int buf) {
    float* Ab = As + buf * KC * TM;
#pragma unroll
    for (int j = 0; j < A_PER_T; ++j) {
      if (a_st[j]) {
        Ab[(4 * a_q[j] + 0) * TM + a_re[j]] = ra[j].x;
        Ab[(4 * a_q[j] + 1) * TM + a_re[j]] = ra[j].y;
        Ab[(4 * a_q[j] + 2) * TM + a_re[j]] = ra[j].z;
        Ab[(4 * a_q[j] + 3) * TM + a_re[j]] = ra[j].w;
      }
    }
#pragma unroll
    for (int j = 0; j < B_PER_T; ++j) {
      const int idx = tid + j * NT;
      if (idx < B_F4) reinterpret_cast<float4*>(Bs + buf * KC * COUT)[idx] = rb[j];
    }
  };

  unsigned long long acc2[8][4];   // acc2[i][p] = (acc[i][2p], acc[i][2p + 1])
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc2[i][p] = 0ull;

  load_chunk(0);
  store_chunk(0);
  __syncthreads();
  for (int c = 0; c < NCH; ++c) {
    const int buf = c & 1;
    if (c + 1 < NCH) load_chunk(c + 1);
    const float* Ab = As + buf * KC * TM;
    const float* Bb = Bs + buf * KC * COUT;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(Ab + k * TM + rg * 4);
      const float4 a1 = *reinterpret_cast<const float4*>(Ab + k * TM + HM + rg * 4);
      const float4 b0 = *reinterpret_cast<const float4*>(Bb + k * COUT + cg * 4);
      const float4 b1 = *reinterpret_cast<const float4*>(Bb + k * COUT + HC + cg * 4);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const unsigned long long bp[4] = {pack2(b0.x, b0.y), pack2(b0.z, b0.w), pack2(b1.x, b1.y), pack2(b1.z, b1.w)};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const unsigned long long ad = pack2(av[i], av[i]);
#pragma unroll
        for (int p = 0; p < 4; ++p) fma2(acc2[i][p], ad, bp[p]);
      }
    }
    if (c + 1 < NCH) store_chunk(buf ^ 1);
    __syncthreads();
  }

  // ---------------------------------------------------------------- epilogue
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) unpack2(acc2[i][p], acc[i][2 * p], acc[i][2 * p + 1]);
  const int ebr = *static_cast<volatile int*>(&cta_br);   // written before the loop's barriers
  const float* __restrict__ bias = a.bias[ebr];
  const float* __restrict__ resid = a.resid[ebr];
  float* __restrict__ out0 = a.out0[ebr];
  const bool ln = a.ln_g[ebr] != nullptr;
  float* Cs = smem;   // [TM][CS], reuses the mainloop buffers (all reads done)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c0 = h * HC + cg * 4;
    const float4 bv = bias ? __ldg(reinterpret_cast<const float4*>(bias + c0)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int re = (i < 4 ? 0 : HM) + rg * 4 + (i & 3);
      const long long m = m0 + re;
      if (m >= a.M) continue;
      float4 v = make_float4(acc[i][4 * h] + bv.x, acc[i][4 * h + 1] + bv.y, acc[i][4 * h + 2] + bv.z,
                             acc[i][4 * h + 3] + bv.w);
      if (resid) {
        const float4 r = __ldg(reinterpret_cast<const float4*>(resid + m * COUT + c0));
        v.x += r.x;
        v.y += r.y;
        v.z += r.z;
        v.w += r.w;
      }
      if (out0) {
        float4 o = v;
        if (a.relu0) o = make_float4(fmaxf(o.x, 0.f), fmaxf(o.y, 0.f), fmaxf(o.z, 0.f), fmaxf(o.w, 0.f));
        *reinterpret_cast<float4*>(out0 + m * COUT + c0) = o;
      }
      if (ln) *reinterpret_cast<float4*>(Cs + re * CS + c0) = v;
    }
  }
  if (!ln) return;
  __syncthreads();
  const float* __restrict__ g = a.ln_g[ebr];
  const float* __restrict__ be = a.ln_b[ebr];
  float* __restrict__ out1 = a.out1[ebr];
  // the rows run on the CTA's full warps only: at Cout = 88 (176 threads) the sixth warp has
  // 16 threads, and its shuffles would read lanes that do not exist
  constexpr int NW = NT / 32;
  static_assert(NW >= 1, "at least one full warp");
  constexpr int CPL = (COUT + 31) / 32;
  const int lane = tid & 31, warp = tid >> 5;
  if (warp >= NW) return;
  for (int re = warp; re < TM; re += NW) {
    const long long m = m0 + re;
    if (m >= a.M) break;
    float x[CPL];
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      x[j] = c < COUT ? Cs[re * CS + c] : 0.f;
      s += x[j];
    }
    const float mean = warp_sum(s) * (1.0f / COUT);
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      const float d = c < COUT ? x[j] - mean : 0.f;
      q += d * d;
    }
    const float rstd = rsqrtf(warp_sum(q) * (1.0f / COUT) + 1e-5f);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int c = lane + 32 * j;
      if (c < COUT) out1[m * COUT + c] = fmaxf((x[j] - mean) * rstd * __ldg(g + c) + __ldg(be + c), 0.f);
    }
  }
}

template <int CIN, int COUT, int KC, int TAPS = 9>
int launch_t(const ConvArgs& a, int n_br, cudaStream_t s) {
  constexpr size_t main_smem = (size_t)(2 * KC * TM + 2 * KC * COUT) * sizeof(float);
  constexpr size_t epi_smem = (size_t)TM * (COUT + 4) * sizeof(float);
  constexpr size_t smem = main_smem > epi_smem ? main_smem : epi_smem;
  static bool attr = false;
  if (!attr) {
    CONET_CUDA(cudaFuncSetAttribute(conv3x3_fp32_kernel<CIN, COUT, KC, TAPS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  dim3 grid((unsigned)((a.M + TM - 1) / TM), n_br);
  conv3x3_fp32_kernel<CIN, COUT, KC, TAPS><<<grid, COUT * 2, smem, s>>>(a);
  return check_launch(TAPS == 9 ? "conv3x3_fp32_kernel" : "conv1x1_fp32_kernel");
}

// Depthwise 3x3 'same' conv of every branch (the first half of a depthwise-separable conv):
// out[m][c] = sum over the 9 taps of w[c][tap] x[m + shift(tap)][c] (zero outside the grid).
// One thread per RE and 4 channels; the 9 neighbour rows come through L1 / L2.
__global__ void dwconv3x3_kernel(DwArgs a, int n_br) {
  const int q = a.C / 4;
  const long long total = a.M * q * n_br;
  const int TF = a.T * a.F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = 4 * (int)(i % q);
    const long long rest = i / q;
    const long long m = rest % a.M;
    const int b = (int)(rest / a.M);
    const int r = (int)(m % TF), t = r / a.F, f = r % a.F;
    const float* w = a.w[b];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int tt = t + tap / 3 - 1, ff = f + tap % 3 - 1;
      if (tt < 0 || tt >= a.T || ff < 0 || ff >= a.F) continue;
      const long long mm = m + (long long)(tap / 3 - 1) * a.F + (tap % 3 - 1);
      const float4 x = __ldg(reinterpret_cast<const float4*>(a.in[b] + mm * a.C + c));
      const int wt = a.flip ? 8 - tap : tap;
      acc.x = fmaf(__ldg(w + (c + 0) * 9 + wt), x.x, acc.x);
      acc.y = fmaf(__ldg(w + (c + 1) * 9 + wt), x.y, acc.y);
      acc.z = fmaf(__ldg(w + (c + 2) * 9 + wt), x.z, acc.z);
      acc.w = fmaf(__ldg(w + (c + 3) * 9 + wt), x.w, acc.w);
    }
    *reinterpret_cast<float4*>(a.out[b] + m * a.C + c) = acc;
  }
}

}  // namespace

int launch_conv3x3_fp32(const ConvArgs& a, int n_br, int cin, int cout, cudaStream_t s) {
  if (a.taps == 1) {   // the 1x1 of a depthwise-separable conv (C -> C)
#define PW_CASE(C) \
  if (cin == C && cout == C) return launch_t<C, C, 8, 1>(a, n_br, s);
    PW_CASE(16)
    PW_CASE(32)
    PW_CASE(64)
    PW_CASE(96)
    PW_CASE(112)
#undef PW_CASE
    return fail(CONET_ERR_UNSUPPORTED, "FP32 1x1 conv with Cin=%d Cout=%d is not instantiated", cin, cout);
  }
#define CONV_CASE(CI, CO, KC) \
  if (cin == CI && cout == CO) return launch_t<CI, CO, KC>(a, n_br, s);
  CONV_CASE(8, 32, 8)
  CONV_CASE(32, 32, 8)
  CONV_CASE(8, 64, 8)
  CONV_CASE(64, 64, 8)
  CONV_CASE(8, 112, 8)
  CONV_CASE(112, 112, 8)
  CONV_CASE(12, 96, 4)
  CONV_CASE(96, 96, 8)
  CONV_CASE(8, 16, 8)
  CONV_CASE(16, 16, 8)
  CONV_CASE(8, 88, 8)
  CONV_CASE(88, 88, 8)
  CONV_CASE(64, 32, 8)   // main layers after a concatenating fusion point: 2 x 32 -> 32
  CONV_CASE(48, 16, 8)   // 3 x 16 -> 16
  CONV_CASE(32, 64, 8)   // ... and their data gradients: 32 -> 2 x 32
  CONV_CASE(16, 48, 8)   // 16 -> 3 x 16
#undef CONV_CASE
  return fail(CONET_ERR_UNSUPPORTED, "FP32 conv3x3 with Cin=%d Cout=%d is not instantiated", cin, cout);
}

// [Cout][taps][cin_src] -> [taps][cin_dst][Cout], zero rows for cin_src <= ci < cin_dst
// (taps = 9 for a 3x3 conv, 1 for a 1x1 conv)
__global__ void weights_tap_major_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst, int taps,
                                         float* __restrict__ out) {
  const int n = taps * cin_dst * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i % cout, rem = i / cout, ci = rem % cin_dst, tap = rem / cin_dst;
    out[i] = ci < cin_src ? w[((size_t)co * taps + tap) * cin_src + ci] : 0.f;
  }
}

int launch_weights_to_tap_major(const float* w, int cout, int cin_src, int cin_dst, float* out, cudaStream_t s,
                                int taps) {
  weights_tap_major_kernel<<<grid_for((long long)cout * taps * cin_dst, 256, 512), 256, 0, s>>>(w, cout, cin_src,
                                                                                                cin_dst, taps, out);
  return check_launch("weights_tap_major_kernel");
}

int launch_dwconv3x3(const DwArgs& a, int n_br, cudaStream_t s) {
  if (a.C % 4) return fail(CONET_ERR_UNSUPPORTED, "depthwise conv needs C %% 4 == 0");
  dwconv3x3_kernel<<<grid_for(a.M * (a.C / 4) * n_br, 256, 152 * 16), 256, 0, s>>>(a, n_br);
  return check_launch("dwconv3x3_kernel");
}

}  // namespace conet
