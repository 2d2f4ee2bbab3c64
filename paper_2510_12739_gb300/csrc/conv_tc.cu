// 3x3 'same' convolution of every CoNet branch as an implicit GEMM on the 5th-generation
// tensor cores (tcgen05) with TMEM accumulators and TMA-fed shared-memory operands.
//
// Tile: 128 resource elements = 128 consecutive subcarriers of one OFDM symbol of one slot
// (rows of the MMA), all Cout channels of every branch (one MMA N = Cout per branch, the
// branches' accumulators side by side in TMEM).  K runs over the 9 taps x Cin channels in
// chunks of KC channels: for tap (dt, df) the A operand is the TMA box of the input
// shifted by (dt, df); rows or subcarriers outside the grid come back as TMA zero fill,
// which is exactly the conv's zero padding.  The B operand is the tap's [Cout][KC] weight
// slice, both K-major.
//
// Warp roles (192 threads): warp 0 issues TMA loads into a ring of shared-memory stages,
// warp 1 issues tcgen05.mma from one thread and commits each stage back to the producer,
// warps 2-5 (one TMEM lane quarter each, one RE per thread) run the fused epilogue:
// bias, residual add, ReLU / LayerNorm, the Hadamard fusion of the branches with its
// LayerNorm, the next layer's pre-activation, and the 1x1 LLR head.  Two TMEM accumulator
// sets (when they fit) let the epilogue of one tile overlap the MMAs of the next.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace conet {

namespace {

constexpr int TILE_M = 128;
constexpr int CW = 8;                             // accumulator columns per epilogue chunk
constexpr size_t SMEM_LIMIT = 227 * 1024;
constexpr int HEAD_QMAX = 8;
// Per epilogue warp: shared scratch used in turn for the LayerNorm moment exchange
// ((NB + 1) x 2 x 32 floats) and the head's partial sums (HEAD_QMAX x 32 floats).
constexpr int SCR_WARP_FLOATS = 320;
static_assert((4 + 1) * 2 * 32 <= SCR_WARP_FLOATS && HEAD_QMAX * 32 <= SCR_WARP_FLOATS, "epilogue scratch");

// The epilogue's per-channel parameters, copied once per CTA into shared memory: every tile
// reads all of them, and from global memory they would share the few KB of L1 left beside
// the operand stages with the streaming residual traffic (and mostly miss).  Layout in
// floats: the fused LayerNorm's gamma and beta, the head's [HEAD_QMAX][Cout] weights and
// HEAD_QMAX biases, the E4M3 output scales 1 / s of up to 8 branches, then per branch its
// bias, LN2 gamma and beta, LN1 gamma and beta and E4M3 dequantisation factors.
enum { PF_BIAS, PF_LN2G, PF_LN2B, PF_LN1G, PF_LN1B, PF_DQ, PF_N };
static_assert(MAX_BR <= 8, "E4M3 output scales");
template <int COUT>
struct ParLayout {
  static constexpr int LNFG = 0, LNFB = COUT, HEADW = 2 * COUT, HEADB = HEADW + HEAD_QMAX * COUT,
                       QINV = HEADB + HEAD_QMAX, BR = QINV + 8;
  static constexpr int at(int b, int f) { return BR + (PF_N * b + f) * COUT; }
};
__host__ __device__ constexpr size_t par_bytes(int nb, int cout) {
  return ((size_t)((2 + HEAD_QMAX) * cout + HEAD_QMAX + 8 + PF_N * nb * cout) * sizeof(float) + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t scr_bytes(int ep) { return (size_t)4 * ep * SCR_WARP_FLOATS * sizeof(float); }

__host__ __device__ constexpr int pow2_ceil(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

__host__ __device__ constexpr int elt_of(int kind) { return kind == 1 ? 4 : kind == 2 ? 1 : 2; }
__host__ __device__ constexpr int nsplit_of(int kind) { return kind == 1 ? 2 : 1; }

// Shared-memory bytes of one pipeline stage: per branch (and split part) an A box of
// a_rows rows and `taps` weight slices of cout rows, rows of `row` bytes; 1 KB aligned.
__host__ __device__ constexpr size_t stage_bytes(int kind, int nb, int cout, int row, int a_rows, int taps) {
  return ((size_t)nb * nsplit_of(kind) * ((size_t)a_rows * row + (size_t)taps * cout * row) + 1023) / 1024 * 1024;
}

__host__ __device__ constexpr int stages_fit(int kind, int nb, int cout, int row, int a_rows, int taps, int ep,
                                             size_t par) {
  return (int)((SMEM_LIMIT - 1024 - 256 - scr_bytes(ep) - par) / stage_bytes(kind, nb, cout, row, a_rows, taps));
}

// K chunk (channels per operand row) and stage shape of an instantiation.  Preferred: the
// "halo" stage -- one TMA box of TILE_M + 2 subcarriers serves the three subcarrier taps of
// one symbol row through descriptors shifted by 0, 1, 2 rows, with the three taps' weights
// -- at the longest operand row (128, 64, 32 bytes) that divides Cin and leaves >= 3
// stages.  Else one tap per stage at the longest row that leaves >= 2 stages.
constexpr int HALO_ROWS = TILE_M + 8;   // smem rows reserved for a halo box (a whole swizzle atom)
__host__ __device__ constexpr int kc_min(int kind) { return 32 / elt_of(kind); }   // one MMA K step

// Branch groups per tile: 1 when two accumulator sets of all branches fit in TMEM's 512
// columns; else 2 when half the branches double-buffer and a COUT-column stash for the
// running Hadamard product still fits (4 branches x 96 channels: 2 x 192 + 96 = 480).
// Split TF32 runs 3-branch networks one branch at a time: a one-branch stage takes
// operand rows twice as long, which its TMA-bound main loop needs (measured: +10 %; the
// 16-bit and E4M3 paths are faster as one group).
__host__ __device__ constexpr int tc_groups(int kind, int nb, int cout) {
  return kind == 1 && nb == 3 ? 3
         : 2 * pow2_ceil(nb * cout) <= 512 ? 1
                                            : (nb % 2 == 0 && nb * cout + cout <= 512 ? 2 : 1);
}

// Epilogue warps per TMEM lane quarter (channel parts): 4 (18 warps, up to 96 registers
// each), except 3 (14 warps, up to 128 registers) for single-group E4M3 epilogues of three
// or more branches, whose dequantisation state does not fit 96 registers (measured on the
// 14x624 network: 4 parts are 5 % faster with 16-bit operands, 6 % slower with E4M3).
__host__ __device__ constexpr int epi_parts(int kind, int nb, int cout) {
  return tc_groups(kind, nb, cout) == 1 && kind == 2 && nb >= 3 ? 3 : 4;
}

__host__ __device__ constexpr int tc_plan(int kind, int nb_all, int cin, int cout, bool want_halo) {
  // returns KC for the requested stage shape, 0 if none fits; a stage holds one branch group
  const int nb = nb_all / tc_groups(kind, nb_all, cout);
  const int ep = epi_parts(kind, nb_all, cout);
  const size_t par = par_bytes(nb_all, cout);
  for (int row = 128; row >= 32; row >>= 1) {
    const int kc = row / elt_of(kind);
    if (kc < kc_min(kind) || cin % kc) continue;
    if (want_halo ? stages_fit(kind, nb, cout, row, HALO_ROWS, 3, ep, par) >= 3
                  : stages_fit(kind, nb, cout, row, TILE_M, 1, ep, par) >= 2)
      return kc;
  }
  return 0;
}

__host__ __device__ constexpr int tc_halo(int kind, int nb, int cin, int cout) {
  return tc_plan(kind, nb, cin, cout, true) > 0 ? 1 : 0;
}

__host__ __device__ constexpr int tc_kc(int kind, int nb, int cin, int cout) {
  return tc_halo(kind, nb, cin, cout) ? tc_plan(kind, nb, cin, cout, true) : tc_plan(kind, nb, cin, cout, false);
}

template <int KIND, int NB, int CIN, int COUT, int KC, int HALO>
struct Cfg {
  static constexpr int ELT = elt_of(KIND);
  static constexpr int ROW = KC * ELT;                  // bytes per operand row (= swizzle span)
  static_assert(ROW == 32 || ROW == 64 || ROW == 128, "row bytes");
  static constexpr int SLICES = ROW / 32;               // MMAs (32 bytes of K each) per chunk
  static constexpr int NSPLIT = nsplit_of(KIND);        // split TF32: hi and lo copies of A and B
  static constexpr int TAPS = HALO ? 3 : 1;             // weight taps (subcarrier shifts) per stage
  static constexpr int A_BOX = HALO ? TILE_M + 2 : TILE_M;
  static constexpr int A_PART = (HALO ? HALO_ROWS : TILE_M) * ROW;
  static constexpr int B_PART = TAPS * COUT * ROW;
  static constexpr int A_BYTES = NSPLIT * A_PART;
  static constexpr int B_BYTES = NSPLIT * B_PART;
  static constexpr int NG = tc_groups(KIND, NB, COUT); // branch groups per tile
  static constexpr int G = NB / NG;                     // branches per MMA unit (one stage holds G)
  static constexpr int STAGE_TX = G * NSPLIT * (A_BOX * ROW + B_PART);
  static constexpr int STAGE = (int)stage_bytes(KIND, G, COUT, ROW, HALO ? HALO_ROWS : TILE_M, TAPS);
  static constexpr int K_ITERS = (9 / TAPS) * (CIN / KC);
  static constexpr int COLS = NG == 1 ? pow2_ceil(NB * COUT) : G * COUT;   // stride of accumulator sets
  static constexpr int N_ACC = NG == 1 ? (2 * COLS <= 512 ? 2 : 1) : 2;
  static constexpr int STASH = NG == 1 ? 0 : 2 * G * COUT;                 // running-product columns
  static constexpr int TMEM_COLS = NG == 1 ? N_ACC * COLS : 512;
  static_assert(NG == 1 || STASH + COUT <= 512, "TMEM columns for the product stash");
  static constexpr int EP = epi_parts(KIND, NB, COUT);  // channel parts per lane quarter
  static constexpr int EPI_WARPS = 4 * EP;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr size_t SCR = scr_bytes(EP);
  static constexpr size_t PAR = par_bytes(NB, COUT);
  static constexpr int STAGES_FIT = (int)((SMEM_LIMIT - 1024 - 256 - SCR - PAR) / STAGE);
  static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256 + SCR + PAR;
  static constexpr uint32_t IDESC = tc::instr_desc(KIND == 0 ? 1 : KIND == 1 ? 2 : 0, COUT);   // BF16 / TF32 / F16, E4M3
  static_assert(STAGES >= 2, "not enough shared memory for two stages");
  static_assert(COUT % 16 == 0 && COUT <= 256 && COUT % CW == 0, "MMA N");
  static_assert(NB * COUT <= 512, "TMEM columns");
  static_assert(CIN % KC == 0, "K chunking");
  static_assert(A_PART % 1024 == 0 || (A_PART % 512 == 0 && ROW <= 64) || (A_PART % 256 == 0 && ROW == 32),
                "A part must hold whole swizzle atoms");
};

// Chan et al.'s pairwise rule: fold the part (nb, mb, Mb) -- count, mean and sum of
// squared deviations -- into the running (na, ma, Ma).
__device__ __forceinline__ void chan_fold(float& na, float& ma, float& Ma, float nb, float mb, float Mb) {
  if (nb == 0.f) return;
  const float n = na + nb;
  const float d = mb - ma;
  ma += d * (nb / n);
  Ma += Mb + d * d * (na * nb / n);
  na = n;
}

__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Barrier over `threads` threads that also returns whether `ok` held in all of them, so the
// warps of an epilogue quarter always take the same branch (a lone warp would otherwise wait
// at the next named barrier for partners that already left).
__device__ __forceinline__ bool barrier_all(int id, int threads, bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(id), "r"(threads)
      : "memory");
  return r != 0;
}

// 8 consecutive floats (32-byte aligned: one whole sector) in one 256-bit access: loads of
// residual rows, read once, so they bypass L1 (no_allocate; measured 5 % faster on the
// 14x624 BF16 network than allocating them), and stores of FP32 output rows.
__device__ __forceinline__ void ldg8(const float* p, float (&x)[8]) {
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
      : "l"(p));
}

__device__ __forceinline__ void stg8(float* p, const float (&x)[8]) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(x[0]), "f"(x[1]), "f"(x[2]),
               "f"(x[3]), "f"(x[4]), "f"(x[5]), "f"(x[6]), "f"(x[7])
               : "memory");
}

// 8 (or 1) parameter floats from the shared-memory copy; every lane reads the same address
// (a broadcast).  Volatile keeps the loads after the barrier that publishes the copy.
__device__ __forceinline__ void lds8(const float* p, float (&x)[8]) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]) : "r"(s));
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4 + 16];" : "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7]) : "r"(s));
}

__device__ __forceinline__ float lds1(const float* p) {
  float x;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x) : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return x;
}

// Copy of the epilogue parameters (layout ParLayout) by threads i0, i0 + stride, ...; null
// or unused entries read as 0.
template <int KIND, int NB, int COUT>
__device__ void stage_params(const TcConvArgs& a, float* par, int i0, int stride) {
  using PL = ParLayout<COUT>;
  constexpr int N = PL::at(NB, 0);
  const int qn = a.Q < HEAD_QMAX ? a.Q : HEAD_QMAX;
  for (int i = i0; i < N; i += stride) {
    const float* src = nullptr;
    int k = 0;
    if (i < PL::HEADW) {
      src = i < PL::LNFB ? a.lnf_g : a.lnf_b;
      k = i % COUT;
    } else if (i < PL::HEADB) {
      k = i - PL::HEADW;
      if (k < qn * COUT) src = a.head_w;
    } else if (i < PL::QINV) {
      k = i - PL::HEADB;
      if (k < qn) src = a.head_b;
    } else if (i < PL::BR) {
      const int b = i - PL::QINV;
      if (KIND == 2 && b < NB) src = a.qinv[b];
    } else {
      const int r = i - PL::BR, b = r / (PF_N * COUT), f = (r / COUT) % PF_N;
      k = r % COUT;
      src = f == PF_BIAS   ? a.bias[b]
            : f == PF_LN2G ? a.ln2_g[b]
            : f == PF_LN2B ? a.ln2_b[b]
            : f == PF_LN1G ? a.ln1_g[b]
            : f == PF_LN1B ? a.ln1_b[b]
                           : (KIND == 2 ? a.dq[b] : nullptr);
    }
    par[i] = src ? src[k] : 0.f;
  }
}

// v_b = acc_b (x dq_b on the E4M3 path) + bias_b (+ resid_b) for the 8 channels of chunk j
// of every branch (add = false: the raw TMEM columns, when an earlier pass wrote v back).
// (Branches b0 .. b0 + NB - 1, accumulators at TMEM columns 0, COUT, ... from tacc.)
template <int KIND, int NB, int COUT>
__device__ __forceinline__ void load_chunk(const TcConvArgs& a, const float* par, uint32_t tacc, int b0, int j,
                                           bool valid, long long m, float (&v)[NB][CW], bool add) {
  using PL = ParLayout<COUT>;
  uint32_t r[NB][CW];
#pragma unroll
  for (int b = 0; b < NB; ++b) tc::tmem_ld8_nowait(tacc + (uint32_t)(b * COUT + CW * j), r[b]);
  tc::tmem_wait_ld();
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int c = 0; c < CW; ++c) v[b][c] = __uint_as_float(r[b][c]);
  if (!add) return;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float x[CW];
    if constexpr (KIND == 2) {
      lds8(par + PL::at(b0 + b, PF_DQ) + CW * j, x);
#pragma unroll
      for (int c = 0; c < CW; ++c) v[b][c] *= x[c];
    }
    lds8(par + PL::at(b0 + b, PF_BIAS) + CW * j, x);
#pragma unroll
    for (int c = 0; c < CW; ++c) v[b][c] += x[c];
    if (a.resid[b0 + b] && valid) {
      ldg8(a.resid[b0 + b] + m * COUT + CW * j, x);
#pragma unroll
      for (int c = 0; c < CW; ++c) v[b][c] += x[c];
    }
  }
}

// One 8-column chunk of a single TMEM column range (the product stash).
__device__ __forceinline__ void tmem_get8(uint32_t taddr, float (&x)[CW]) {
  uint32_t r[CW];
  tc::tmem_ld8_nowait(taddr, r);
  tc::tmem_wait_ld();
#pragma unroll
  for (int c = 0; c < CW; ++c) x[c] = __uint_as_float(r[c]);
}

// Round to the nearest TF32 value (10 explicit mantissa bits; low 13 bits zero).
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// 8 values as 16-bit floats (one 16-byte store) or as E4M3 of value x qinv (one 8-byte store).
template <typename H>
__device__ __forceinline__ void store8_h(H* p, const float (&x)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if constexpr (std::is_same<H, __half>::value) {
      const __half2 h = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&h);
    } else {
      const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
  }
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void store8_e4m3(uint8_t* p, const float (&x)[8], float qinv) {
  uint32_t w[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(x[4 * i] * qinv, x[4 * i + 1] * qinv), __NV_SATFINITE,
                                                 __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(x[4 * i + 2] * qinv, x[4 * i + 3] * qinv),
                                                 __NV_SATFINITE, __NV_E4M3);
    w[i] = (lo & 0xFFFFu) | (hi << 16);
  }
  *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
}

// Chunks [first, first + count) of COUT / CW owned by channel part p (near-equal split).
template <int COUT, int EP>
__device__ __forceinline__ void part_chunks(int p, int& first, int& count) {
  constexpr int CH = COUT / CW, base = CH / EP, rem = CH % EP;
  first = p * base + (p < rem ? p : rem);
  count = base + (p < rem ? 1 : 0);
}

// The fused epilogue for one RE (this thread's TMEM lane) and one part of its channels.
// Pass 1 (when a LayerNorm is applied) folds each branch's values, and the fused product,
// into shifted first and second moments; the parts of a lane quarter publish theirs in
// their shared scratch and each part merges all of them in the same order (Chan et al.), so
// every part normalises with identical statistics.  Pass 1 also writes the biased (and
// residual-added) values back into TMEM.  Pass 2 applies the pre-activation, the Hadamard
// fusion and its LayerNorm, writes the residual stream and the next conv's input, and
// accumulates the head's partial sums, which part 0 reduces through the scratch.
template <int KIND, int NB, int COUT, int EP>
__device__ __forceinline__ void tc_epilogue(const TcConvArgs& a, const float* par, uint32_t tacc, bool valid,
                                            long long m, int part, int quarter, int lane, float* scr_all) {
  constexpr int QMAX = HEAD_QMAX;
  using PL = ParLayout<COUT>;
  float* scr = scr_all + (size_t)(4 * part + ((quarter + 2) & 3)) * SCR_WARP_FLOATS;
  int j_lo, n_ch;
  part_chunks<COUT, EP>(part, j_lo, n_ch);
  const int j_hi = j_lo + n_ch;
  const bool pre_ln = a.pre == 2;
  const bool fuse_ln = a.fuse && a.lnf_g != nullptr;
  bool any_ln1 = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) any_ln1 = any_ln1 || a.post[b] == 2;
  const bool stats = pre_ln || fuse_ln || any_ln1;
  const bool add2 = !stats;   // pass 2 adds bias / residual itself unless pass 1 wrote v back

  float mean_b[NB], rstd_b[NB], mean_p = 0.f, rstd_p = 1.f;
  if (stats) {
    // shifted sums: shift = the part's first value of each statistic
    float k_b[NB], s1_b[NB], s2_b[NB], k_p = 0.f, s1_p = 0.f, s2_p = 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) k_b[b] = s1_b[b] = s2_b[b] = 0.f;
    for (int j = j_lo; j < j_hi; ++j) {
      float v[NB][CW];
      __syncwarp();
      load_chunk<KIND, NB, COUT>(a, par, tacc, 0, j, valid, m, v, true);
      __syncwarp();   // tcgen05.st is warp-collective: reconverge after the per-row residual loads
#pragma unroll
      for (int b = 0; b < NB; ++b) tc::tmem_st8_nowait(tacc + (uint32_t)(b * COUT + CW * j), v[b]);
      // the statistic of branch b is over v_b (pre_ln) or over pre(v_b) (the next block's
      // LN1); the fused product is over pre(v_b).  pre = 1 is ReLU, applied in place here
      // (pass 2 re-reads the unactivated values from TMEM).
      if (a.pre == 1) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int c = 0; c < CW; ++c) v[b][c] = fmaxf(v[b][c], 0.f);
      }
      if (j == j_lo) {
        float p0 = 1.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          k_b[b] = v[b][0];
          p0 *= v[b][0];
        }
        k_p = p0;
      }
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        float p = 1.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const float d = v[b][c] - k_b[b];
          s1_b[b] += d;
          s2_b[b] = fmaf(d, d, s2_b[b]);
          p *= v[b][c];
        }
        if (fuse_ln) {
          const float d = p - k_p;
          s1_p += d;
          s2_p = fmaf(d, d, s2_p);
        }
      }
    }
    __syncwarp();
    tc::tmem_wait_st();
    // publish (mean, M2) of this part, then fold all parts in order
    const float n_mine = (float)(CW * n_ch);
#pragma unroll
    for (int s = 0; s <= NB; ++s) {
      const float k = s < NB ? k_b[s] : k_p, s1 = s < NB ? s1_b[s] : s1_p, s2 = s < NB ? s2_b[s] : s2_p;
      const float m1 = n_ch ? s1 / n_mine : 0.f;
      scr[(2 * s) * 32 + lane] = k + m1;
      scr[(2 * s + 1) * 32 + lane] = fmaxf(s2 - s1 * m1, 0.f);
    }
    named_barrier(1 + quarter, 32 * EP);
#pragma unroll
    for (int s = 0; s <= NB; ++s) {
      float n = 0.f, mu = 0.f, M2 = 0.f;
#pragma unroll
      for (int pp = 0; pp < EP; ++pp) {
        int f0, cnt;
        part_chunks<COUT, EP>(pp, f0, cnt);
        const float* o = scr_all + (size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_WARP_FLOATS;
        chan_fold(n, mu, M2, (float)(CW * cnt), o[(2 * s) * 32 + lane], o[(2 * s + 1) * 32 + lane]);
      }
      const float rs = rsqrtf(M2 / (float)COUT + 1e-5f);
      if (s < NB) {
        mean_b[s] = mu;
        rstd_b[s] = rs;
      } else {
        mean_p = mu;
        rstd_p = rs;
      }
    }
    named_barrier(1 + quarter, 32 * EP);   // scratch free for the stores
  }

  float hq[QMAX];
#pragma unroll
  for (int qq = 0; qq < QMAX; ++qq) hq[qq] = 0.f;
  float amx[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) amx[b] = 0.f;
  for (int j = j_lo; j < j_hi; ++j) {
    float v[NB][CW];
    __syncwarp();
    load_chunk<KIND, NB, COUT>(a, par, tacc, 0, j, valid, m, v, add2);
    const int c0 = CW * j;
    // rows past the grid edge compute on don't-care values and store nothing
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (valid && a.t_out[b]) stg8(a.t_out[b] + m * COUT + c0, v[b]);
    // a_b = pre(v_b), in place
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (a.pre == 1) {
#pragma unroll
        for (int c = 0; c < CW; ++c) v[b][c] = fmaxf(v[b][c], 0.f);
      } else if (pre_ln) {
        float g[CW], be[CW];
        lds8(par + PL::at(b, PF_LN2G) + c0, g);
        lds8(par + PL::at(b, PF_LN2B) + c0, be);
        const float mu = mean_b[b], rs = rstd_b[b];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[b][c] = fmaxf((v[b][c] - mu) * rs * g[c] + be[c], 0.f);
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (valid && a.a_out[b]) stg8(a.a_out[b] + m * COUT + c0, v[b]);
    // x_0 = fused (and normalised) product, or a_0; it replaces v[0] from here on
    if (a.fuse) {
#pragma unroll
      for (int c = 0; c < CW; ++c) {
#pragma unroll
        for (int b = 1; b < NB; ++b) v[0][c] *= v[b][c];
      }
      if (fuse_ln) {
        float g[CW], be[CW];
        lds8(par + PL::LNFG + c0, g);
        lds8(par + PL::LNFB + c0, be);
#pragma unroll
        for (int c = 0; c < CW; ++c) v[0][c] = (v[0][c] - mean_p) * rstd_p * g[c] + be[c];
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (valid && a.xs_out[b] && !a.measure) stg8(a.xs_out[b] + m * COUT + c0, v[b]);
      if (a.nx_out[b]) {
        float o[CW];
        if (a.post[b] == 2) {
          float g[CW], be[CW];
          lds8(par + PL::at(b, PF_LN1G) + c0, g);
          lds8(par + PL::at(b, PF_LN1B) + c0, be);
          const float mu = mean_b[b], rs = rstd_b[b];
#pragma unroll
          for (int c = 0; c < CW; ++c) o[c] = fmaxf((v[b][c] - mu) * rs * g[c] + be[c], 0.f);
        } else if (a.post[b] == 1) {
#pragma unroll
          for (int c = 0; c < CW; ++c) o[c] = fmaxf(v[b][c], 0.f);
        } else {
#pragma unroll
          for (int c = 0; c < CW; ++c) o[c] = v[b][c];
        }
        if constexpr (KIND == 2) {
          if (a.amax[b] && valid) {
#pragma unroll
            for (int c = 0; c < CW; ++c) amx[b] = fmaxf(amx[b], fabsf(o[c]));
          }
          if (valid && !a.measure)
            store8_e4m3(reinterpret_cast<uint8_t*>(a.nx_out[b]) + m * COUT + c0, o, lds1(par + PL::QINV + b));
        } else if constexpr (KIND == 1) {
          float lo[CW];
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            const float hi = tf32_round(o[c]);
            lo[c] = o[c] - hi;
            o[c] = hi;
          }
          if (valid) {
            stg8(reinterpret_cast<float*>(a.nx_out[b]) + m * COUT + c0, o);
            stg8(a.nx_lo[b] + m * COUT + c0, lo);
          }
        } else if constexpr (KIND == 3) {
          if (valid) store8_h(reinterpret_cast<__half*>(a.nx_out[b]) + m * COUT + c0, o);
        } else {
          if (valid) store8_h(reinterpret_cast<__nv_bfloat16*>(a.nx_out[b]) + m * COUT + c0, o);
        }
      }
    }
    if (a.head_w) {
#pragma unroll
      for (int qq = 0; qq < QMAX; ++qq) {
        if (qq >= a.Q) break;
        float hw[CW];
        lds8(par + PL::HEADW + qq * COUT + c0, hw);
        float sacc = 0.f;
#pragma unroll
        for (int c = 0; c < CW; ++c) sacc = fmaf(hw[c], v[0][c], sacc);
        hq[qq] += sacc;
      }
    }
  }
  if constexpr (KIND == 2) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!a.amax[b]) continue;
      float mx = amx[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(a.amax[b], __float_as_uint(mx));
    }
  }
  if (a.head_w) {
    __syncwarp();
    for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) scr[qq * 32 + lane] = hq[qq];
    named_barrier(5 + quarter, 32 * EP);
    if (part == 0 && valid && !a.measure) {
      for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) {
        float sum = 0.f;
#pragma unroll
        for (int pp = 0; pp < EP; ++pp)
          sum += scr_all[(size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_WARP_FLOATS + qq * 32 + lane];
        a.llr[m * a.Q + qq] = sum + lds1(par + PL::HEADB + qq);
      }
    }
  }
}

// Epilogue of branch group g (branches g*G .. g*G + G - 1) of a tile whose branches are
// computed G at a time: the MMAs of one group overlap the epilogue of the previous one, and
// TMEM columns [tstash, tstash + COUT) carry the running Hadamard product from group to
// group.  Per-branch work (bias, residual, pre-activation, the branches' own LayerNorms and
// outputs) happens in the branch's group; branch 0's output -- the fused, normalised
// product x_0 -- is formed in the last group (in group 0 when this layer does not fuse),
// which also accumulates the head.  Statistics are merged across the lane quarter's parts
// as in tc_epilogue.  Fused layers have pre-activation none or ReLU, so the product can be
// formed in the statistics pass.
template <int KIND, int NB, int COUT, int G, int EP>
__device__ __forceinline__ void tc_epilogue_group(const TcConvArgs& a, const float* par, uint32_t tacc,
                                                  uint32_t tstash, int g, bool valid, long long m, int part,
                                                  int quarter, int lane, float* scr_all) {
  constexpr int QMAX = HEAD_QMAX;
  using PL = ParLayout<COUT>;
  constexpr int NG = NB / G;
  float* scr = scr_all + (size_t)(4 * part + ((quarter + 2) & 3)) * SCR_WARP_FLOATS;
  int j_lo, n_ch;
  part_chunks<COUT, EP>(part, j_lo, n_ch);
  const int j_hi = j_lo + n_ch;
  const int b0 = g * G;
  const bool first = g == 0, last = g == NG - 1;
  const bool pre_ln = a.pre == 2;
  const bool fuse = a.fuse != 0;
  const bool fuse_ln = fuse && a.lnf_g != nullptr;
  const bool main_here = fuse ? last : first;   // the group that forms branch 0's output
  bool any_b = false;
#pragma unroll
  for (int bb = 0; bb < G; ++bb) any_b = any_b || pre_ln || a.post[b0 + bb] == 2;
  const bool prod_stats = last && fuse_ln;
  const bool stats = any_b || prod_stats;

  float mean_b[G], rstd_b[G], mean_p = 0.f, rstd_p = 1.f;
  if (stats) {
    float k_b[G], s1_b[G], s2_b[G], k_p = 0.f, s1_p = 0.f, s2_p = 0.f;
#pragma unroll
    for (int bb = 0; bb < G; ++bb) k_b[bb] = s1_b[bb] = s2_b[bb] = 0.f;
    for (int j = j_lo; j < j_hi; ++j) {
      float v[G][CW];
      __syncwarp();
      load_chunk<KIND, G, COUT>(a, par, tacc, b0, j, valid, m, v, true);
      __syncwarp();
#pragma unroll
      for (int bb = 0; bb < G; ++bb) tc::tmem_st8_nowait(tacc + (uint32_t)(bb * COUT + CW * j), v[bb]);
      if (a.pre == 1) {
#pragma unroll
        for (int bb = 0; bb < G; ++bb)
#pragma unroll
          for (int c = 0; c < CW; ++c) v[bb][c] = fmaxf(v[bb][c], 0.f);
      }
      if (j == j_lo) {
#pragma unroll
        for (int bb = 0; bb < G; ++bb) k_b[bb] = v[bb][0];
      }
#pragma unroll
      for (int c = 0; c < CW; ++c) {
#pragma unroll
        for (int bb = 0; bb < G; ++bb) {
          const float d = v[bb][c] - k_b[bb];
          s1_b[bb] += d;
          s2_b[bb] = fmaf(d, d, s2_b[bb]);
        }
      }
      if (fuse) {
        float q[CW];
        if (first) {
#pragma unroll
          for (int c = 0; c < CW; ++c) q[c] = 1.f;
        } else {
          tmem_get8(tstash + (uint32_t)(CW * j), q);
        }
#pragma unroll
        for (int c = 0; c < CW; ++c)
#pragma unroll
          for (int bb = 0; bb < G; ++bb) q[c] *= v[bb][c];
        if (prod_stats) {
          if (j == j_lo) k_p = q[0];
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            const float d = q[c] - k_p;
            s1_p += d;
            s2_p = fmaf(d, d, s2_p);
          }
        }
        tc::tmem_st8_nowait(tstash + (uint32_t)(CW * j), q);
      }
    }
    __syncwarp();
    tc::tmem_wait_st();
    const float n_mine = (float)(CW * n_ch);
#pragma unroll
    for (int s = 0; s <= G; ++s) {
      const float k = s < G ? k_b[s] : k_p, s1 = s < G ? s1_b[s] : s1_p, s2 = s < G ? s2_b[s] : s2_p;
      const float m1 = n_ch ? s1 / n_mine : 0.f;
      scr[(2 * s) * 32 + lane] = k + m1;
      scr[(2 * s + 1) * 32 + lane] = fmaxf(s2 - s1 * m1, 0.f);
    }
    named_barrier(1 + quarter, 32 * EP);
#pragma unroll
    for (int s = 0; s <= G; ++s) {
      float n = 0.f, mu = 0.f, M2 = 0.f;
#pragma unroll
      for (int pp = 0; pp < EP; ++pp) {
        int f0, cnt;
        part_chunks<COUT, EP>(pp, f0, cnt);
        const float* o = scr_all + (size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_WARP_FLOATS;
        chan_fold(n, mu, M2, (float)(CW * cnt), o[(2 * s) * 32 + lane], o[(2 * s + 1) * 32 + lane]);
      }
      const float rs = rsqrtf(M2 / (float)COUT + 1e-5f);
      if (s < G) {
        mean_b[s] = mu;
        rstd_b[s] = rs;
      } else {
        mean_p = mu;
        rstd_p = rs;
      }
    }
    named_barrier(1 + quarter, 32 * EP);
  }

  float hq[QMAX];
#pragma unroll
  for (int qq = 0; qq < QMAX; ++qq) hq[qq] = 0.f;
  float amx_b[G], amx0 = 0.f;
#pragma unroll
  for (int bb = 0; bb < G; ++bb) amx_b[bb] = 0.f;
  for (int j = j_lo; j < j_hi; ++j) {
    float v[G][CW];
    __syncwarp();
    load_chunk<KIND, G, COUT>(a, par, tacc, b0, j, valid, m, v, !stats);
    const int c0 = CW * j;
#pragma unroll
    for (int bb = 0; bb < G; ++bb)
      if (valid && a.t_out[b0 + bb]) stg8(a.t_out[b0 + bb] + m * COUT + c0, v[bb]);
#pragma unroll
    for (int bb = 0; bb < G; ++bb) {
      if (a.pre == 1) {
#pragma unroll
        for (int c = 0; c < CW; ++c) v[bb][c] = fmaxf(v[bb][c], 0.f);
      } else if (pre_ln) {
        float gm[CW], be[CW];
        lds8(par + PL::at(b0 + bb, PF_LN2G) + c0, gm);
        lds8(par + PL::at(b0 + bb, PF_LN2B) + c0, be);
        const float mu = mean_b[bb], rs = rstd_b[bb];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[bb][c] = fmaxf((v[bb][c] - mu) * rs * gm[c] + be[c], 0.f);
      }
    }
#pragma unroll
    for (int bb = 0; bb < G; ++bb)
      if (valid && a.a_out[b0 + bb]) stg8(a.a_out[b0 + bb] + m * COUT + c0, v[bb]);
    // x_0: the fused product (from the stash when the statistics pass formed it), normalised
    float x0[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) x0[c] = 0.f;
    if (fuse) {
      __syncwarp();
      if (stats) {
        if (last) tmem_get8(tstash + (uint32_t)c0, x0);
      } else {
        float q[CW];
        if (first) {
#pragma unroll
          for (int c = 0; c < CW; ++c) q[c] = 1.f;
        } else {
          tmem_get8(tstash + (uint32_t)c0, q);
        }
#pragma unroll
        for (int c = 0; c < CW; ++c)
#pragma unroll
          for (int bb = 0; bb < G; ++bb) q[c] *= v[bb][c];
        if (last) {
#pragma unroll
          for (int c = 0; c < CW; ++c) x0[c] = q[c];
        } else {
          __syncwarp();
          tc::tmem_st8_nowait(tstash + (uint32_t)c0, q);
        }
      }
      if (last && fuse_ln) {
        float gm[CW], be[CW];
        lds8(par + PL::LNFG + c0, gm);
        lds8(par + PL::LNFB + c0, be);
#pragma unroll
        for (int c = 0; c < CW; ++c) x0[c] = (x0[c] - mean_p) * rstd_p * gm[c] + be[c];
      }
    } else if (first) {
#pragma unroll
      for (int c = 0; c < CW; ++c) x0[c] = v[0][c];
    }
    // outputs: the group's branches other than branch 0, then branch 0 where it is formed
#pragma unroll
    for (int bb = 0; bb <= G; ++bb) {
      const bool is_main = bb == G;
      const int b = is_main ? 0 : b0 + bb;
      if (is_main ? !main_here : b == 0) continue;
      const float(&y)[CW] = is_main ? x0 : v[bb < G ? bb : 0];
      if (valid && a.xs_out[b] && !a.measure) stg8(a.xs_out[b] + m * COUT + c0, y);
      if (!a.nx_out[b]) continue;
      float o[CW];
      if (a.post[b] == 2) {
        float gm[CW], be[CW];
        lds8(par + PL::at(b, PF_LN1G) + c0, gm);
        lds8(par + PL::at(b, PF_LN1B) + c0, be);
        const float mu = mean_b[bb < G ? bb : 0], rs = rstd_b[bb < G ? bb : 0];
#pragma unroll
        for (int c = 0; c < CW; ++c) o[c] = fmaxf((y[c] - mu) * rs * gm[c] + be[c], 0.f);
      } else if (a.post[b] == 1) {
#pragma unroll
        for (int c = 0; c < CW; ++c) o[c] = fmaxf(y[c], 0.f);
      } else {
#pragma unroll
        for (int c = 0; c < CW; ++c) o[c] = y[c];
      }
      if constexpr (KIND == 2) {
        if (a.amax[b] && valid) {
          float& mx = is_main ? amx0 : amx_b[bb < G ? bb : 0];
#pragma unroll
          for (int c = 0; c < CW; ++c) mx = fmaxf(mx, fabsf(o[c]));
        }
        if (valid && !a.measure)
          store8_e4m3(reinterpret_cast<uint8_t*>(a.nx_out[b]) + m * COUT + c0, o, lds1(par + PL::QINV + b));
      } else if constexpr (KIND == 1) {
        float lo[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const float hi = tf32_round(o[c]);
          lo[c] = o[c] - hi;
          o[c] = hi;
        }
        if (valid) {
          stg8(reinterpret_cast<float*>(a.nx_out[b]) + m * COUT + c0, o);
          stg8(a.nx_lo[b] + m * COUT + c0, lo);
        }
      } else if constexpr (KIND == 3) {
        if (valid) store8_h(reinterpret_cast<__half*>(a.nx_out[b]) + m * COUT + c0, o);
      } else {
        if (valid) store8_h(reinterpret_cast<__nv_bfloat16*>(a.nx_out[b]) + m * COUT + c0, o);
      }
    }
    if (main_here && a.head_w) {
#pragma unroll
      for (int qq = 0; qq < QMAX; ++qq) {
        if (qq >= a.Q) break;
        float hw[CW];
        lds8(par + PL::HEADW + qq * COUT + c0, hw);
        float sacc = 0.f;
#pragma unroll
        for (int c = 0; c < CW; ++c) sacc = fmaf(hw[c], x0[c], sacc);
        hq[qq] += sacc;
      }
    }
  }
  __syncwarp();
  tc::tmem_wait_st();
  if constexpr (KIND == 2) {
#pragma unroll
    for (int bb = 0; bb <= G; ++bb) {
      const bool is_main = bb == G;
      const int b = is_main ? 0 : b0 + bb;
      if ((is_main ? !main_here : b == 0) || !a.amax[b]) continue;
      float mx = is_main ? amx0 : amx_b[bb < G ? bb : 0];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(a.amax[b], __float_as_uint(mx));
    }
  }
  if (main_here && a.head_w) {
    __syncwarp();
    for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) scr[qq * 32 + lane] = hq[qq];
    named_barrier(5 + quarter, 32 * EP);
    if (part == 0 && valid && !a.measure) {
      for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) {
        float sum = 0.f;
#pragma unroll
        for (int pp = 0; pp < EP; ++pp)
          sum += scr_all[(size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_WARP_FLOATS + qq * 32 + lane];
        a.llr[m * a.Q + qq] = sum + lds1(par + PL::HEADB + qq);
      }
    }
  }
}

__device__ __forceinline__ void decode_tile(int tile, int T, int nfb, int& slot, int& t, int& fb) {
  fb = tile % nfb;
  const int st = tile / nfb;
  t = st % T;
  slot = st / T;
}

// Start moving the residual rows of branches b0 .. b0 + NB - 1 of a tile (contiguous:
// consecutive subcarriers of one symbol) from HBM into L2, so that the epilogue's loads of
// them wait on L2 rather than on DRAM.  Issued one MMA unit ahead: earlier, part of it is
// evicted again by the streaming traffic before use.
template <int NB, int COUT>
__device__ __forceinline__ void prefetch_resid(const TcConvArgs& a, int tile, int b0) {
  if (tile >= a.n_tiles) return;
  int slot, t, fb;
  decode_tile(tile, a.T, a.nfb, slot, t, fb);
  const int rows = a.F - fb * TILE_M < TILE_M ? a.F - fb * TILE_M : TILE_M;
  const long long m0 = ((long long)slot * a.T + t) * a.F + (long long)fb * TILE_M;
#pragma unroll
  for (int b = b0; b < b0 + NB; ++b)
    if (a.resid[b]) tc::prefetch_l2(a.resid[b] + m0 * COUT, (uint32_t)(rows * COUT * sizeof(float)));
}

template <int KIND, int NB, int CIN, int COUT, int KC, int HALO>
// 2 + 4 x EP warps: 14 (at most 4 per SM sub-partition, up to 128 registers each) or 18
// (up to 96 registers each).
__global__ void __launch_bounds__((Cfg<KIND, NB, CIN, COUT, KC, HALO>::THREADS), 1)
    conv_tc_kernel(const __grid_constant__ TcMaps maps, TcConvArgs a) {
  using K = Cfg<KIND, NB, CIN, COUT, KC, HALO>;
  constexpr int EP = K::EP;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)K::STAGES * K::STAGE);
  uint64_t* empty = full + K::STAGES;
  uint64_t* tfull = empty + K::STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  float* scr_all = reinterpret_cast<float*>(smem + (size_t)K::STAGES * K::STAGE + 256);
  float* par = reinterpret_cast<float*>(smem + (size_t)K::STAGES * K::STAGE + 256 + K::SCR);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < K::STAGES; ++s) {
        tc::mbar_init(&full[s], 1);
        tc::mbar_init(&empty[s], 1);
      }
      for (int i = 0; i < 2; ++i) {
        tc::mbar_init(&tfull[i], 1);
        tc::mbar_init(&tempty[i], K::EPI_WARPS);
      }
      tc::fence_mbar_init();
      for (int b = 0; b < NB; ++b) {
        tc::prefetch_tmap(&maps.a[b]);
        tc::prefetch_tmap(&maps.w[b]);
      }
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, K::TMEM_COLS);
  } else if (warp >= 2) {
    stage_params<KIND, NB, COUT>(a, par, threadIdx.x - 64, K::THREADS - 64);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_slot;
  int* err = a.err;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int s = 0;
    uint32_t ph = 0;
    uint32_t last_par[8];
    bool used[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) used[i] = false;
    bool ok = true;
    for (int unit = blockIdx.x * K::NG; ok && unit < a.n_tiles * K::NG;
         unit += (K::NG == 1 || unit % K::NG == K::NG - 1) ? (int)gridDim.x * K::NG - (K::NG - 1) : 1) {
      const int tile = unit / K::NG, g0 = (unit % K::NG) * K::G;   // tile and its branch group
      int slot, t, fb;
      decode_tile(tile, a.T, a.nfb, slot, t, fb);
      for (int k = 0; k < K::K_ITERS; ++k) {
        if (!tc::mbar_wait(&empty[s], ph ^ 1u, err, 1)) {
          ok = false;
          break;
        }
        tc::mbar_arrive_expect_tx(&full[s], K::STAGE_TX);
        // halo stage: symbol row t + dt, subcarriers from one before the tile, taps
        // (dt, -1..1); else one tap (dt, df) with the tile's rows shifted by df
        const int grp = k / (CIN / KC), ch = (k % (CIN / KC)) * KC;
        const int dt = HALO ? grp - 1 : grp / 3 - 1;
        const int f0 = HALO ? fb * TILE_M - 1 : fb * TILE_M + grp % 3 - 1;
        const int tap0 = HALO ? 3 * grp : grp;
        uint8_t* st = smem + (size_t)s * K::STAGE;
#pragma unroll
        for (int i = 0; i < K::G; ++i) {
          const int b = g0 + i;
          uint8_t* ab = st + i * K::A_BYTES;
          uint8_t* bb = st + K::G * K::A_BYTES + i * K::B_BYTES;
          tc::tma_load_4d(ab, &maps.a[b], &full[s], ch, f0, t + dt, slot);
          tc::tma_load_3d(bb, &maps.w[b], &full[s], ch, 0, tap0);
          if constexpr (K::NSPLIT == 2) {
            tc::tma_load_4d(ab + K::A_PART, &maps.a_lo[b], &full[s], ch, f0, t + dt, slot);
            tc::tma_load_3d(bb + K::B_PART, &maps.w_lo[b], &full[s], ch, 0, tap0);
          }
        }
        used[s] = true;
        last_par[s] = ph;
        if (++s == K::STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    // drain: every issued load has landed before the CTA may exit
    for (int i = 0; i < K::STAGES; ++i)
      if (used[i]) tc::mbar_wait(&full[i], last_par[i], err, 9);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    int s = 0;
    uint32_t ph = 0;
    int it = 0;
    bool ok = true;
    for (int unit = blockIdx.x * K::NG; ok && unit < a.n_tiles * K::NG;
         unit += (K::NG == 1 || unit % K::NG == K::NG - 1) ? (int)gridDim.x * K::NG - (K::NG - 1) : 1, ++it) {
      const int acc = it % K::N_ACC;
      const uint32_t aph = (uint32_t)(it / K::N_ACC) & 1u;
      if (!tc::mbar_wait(&tempty[acc], aph ^ 1u, err, 2)) break;
      tc::fence_after_sync();
      const uint32_t dcol = tbase + (uint32_t)(acc * K::COLS);
      for (int k = 0; k < K::K_ITERS; ++k) {
        if (!tc::mbar_wait(&full[s], ph, err, 3)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t st = tc::smem_u32(smem + (size_t)s * K::STAGE);
#pragma unroll
        for (int b = 0; b < K::G; ++b) {
#pragma unroll
          for (int d = 0; d < K::TAPS; ++d) {
#pragma unroll
            for (int j = 0; j < K::SLICES; ++j) {
              // tap d of a halo stage reads the box from row d: the swizzle pattern is a
              // function of the shared-memory address, so a whole-row shift of the
              // descriptor's start selects the shifted rows
              const uint32_t aa = st + b * K::A_BYTES + d * K::ROW + 32 * j;
              const uint32_t ba = st + K::G * K::A_BYTES + b * K::B_BYTES + d * COUT * K::ROW + 32 * j;
              const uint64_t ad = tc::smem_desc(aa, K::ROW);
              const uint64_t bd = tc::smem_desc(ba, K::ROW);
              tc::mma<KIND>(dcol + (uint32_t)(b * COUT), ad, bd, K::IDESC, (k | d | j) != 0);
              if constexpr (K::NSPLIT == 2) {
                // FP32-accurate product from TF32 parts: hi*hi + hi*lo + lo*hi
                tc::mma<KIND>(dcol + (uint32_t)(b * COUT), ad, tc::smem_desc(ba + K::B_PART, K::ROW), K::IDESC, 1u);
                tc::mma<KIND>(dcol + (uint32_t)(b * COUT), tc::smem_desc(aa + K::A_PART, K::ROW), bd, K::IDESC, 1u);
              }
            }
          }
        }
        tc::mma_commit(&empty[s]);
        if (++s == K::STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
      tc::mma_commit(&tfull[acc]);
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ fused epilogue
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int part = (warp - 2) / 4;        // which share of the channels this warp handles
    const int row = 32 * q + lane;
    const bool prefetcher = warp == 2 && lane == 0;
    if (prefetcher) prefetch_resid<K::G, COUT>(a, blockIdx.x, 0);
    int it = 0;
    for (int unit = blockIdx.x * K::NG; unit < a.n_tiles * K::NG;
         unit += (K::NG == 1 || unit % K::NG == K::NG - 1) ? (int)gridDim.x * K::NG - (K::NG - 1) : 1, ++it) {
      const int tile = unit / K::NG, g = unit % K::NG;
      const int acc = it % K::N_ACC;
      const uint32_t aph = (uint32_t)(it / K::N_ACC) & 1u;
      if (prefetcher) {
        if (g + 1 < K::NG)
          prefetch_resid<K::G, COUT>(a, tile, (g + 1) * K::G);
        else
          prefetch_resid<K::G, COUT>(a, tile + gridDim.x, 0);
      }
      const bool got = tc::mbar_wait(&tfull[acc], aph, err, 4);
      if (!barrier_all(1 + q, 32 * EP, got)) break;
      tc::fence_after_sync();
      int slot, t, fb;
      decode_tile(tile, a.T, a.nfb, slot, t, fb);
      const int f = fb * TILE_M + row;
      const bool valid = f < a.F;
      const long long m = ((long long)slot * a.T + t) * a.F + f;
      const uint32_t lanes = (uint32_t)(32 * q) << 16;
      const uint32_t tacc = tbase + (uint32_t)(acc * K::COLS) + lanes;
      if constexpr (K::NG == 1)
        tc_epilogue<KIND, NB, COUT, EP>(a, par, tacc, valid, m, part, q, lane, scr_all);
      else
        tc_epilogue_group<KIND, NB, COUT, K::G, EP>(a, par, tacc, tbase + (uint32_t)K::STASH + lanes, g, valid, m,
                                                    part, q, lane, scr_all);
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[acc]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, K::TMEM_COLS);
  }
}

template <int KIND, int NB, int CIN, int COUT, int KC, int HALO>
int launch_tc_t(const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  using K = Cfg<KIND, NB, CIN, COUT, KC, HALO>;
  static int attr_done = 0;
  if (!attr_done) {
    CONET_CUDA(cudaFuncSetAttribute(conv_tc_kernel<KIND, NB, CIN, COUT, KC, HALO>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM));
    attr_done = 1;
  }
  int dev = 0, n_sm = 0;
  CONET_CUDA(cudaGetDevice(&dev));
  CONET_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = a.n_tiles < n_sm ? a.n_tiles : n_sm;
  conv_tc_kernel<KIND, NB, CIN, COUT, KC, HALO><<<grid, K::THREADS, K::SMEM, s>>>(maps, a);
  return check_launch("conv_tc_kernel");
}

}  // namespace

int launch_conv_tc(int kind, int nb, int cin, int cout, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  // the branch-group epilogue forms the fused product in its statistics pass and gives the
  // fused branch 0 no LayerNorm of its own
  if (a.fuse && (a.pre == 2 || (tc_groups(kind, nb, cout) > 1 && a.post[0] == 2)))
    return fail(CONET_ERR_UNSUPPORTED, "fused layer with a LayerNorm pre-activation or a normalised fused branch");
#define TC_CASE(KI, NBV, CI, CO)                                                                          \
  if (kind == KI && nb == NBV && cin == CI && cout == CO)                                                  \
    return launch_tc_t<KI, NBV, CI, CO, tc_kc(KI, NBV, CI, CO), tc_halo(KI, NBV, CI, CO)>(maps, a, s);
  // BF16 (kind::f16): input layers take 16 padded channels (32-byte rows)
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
  // FP16 operands (kind::f16, same rate, 11-bit significands)
  TC_CASE(3, 2, 16, 32)
  TC_CASE(3, 2, 32, 32)
  TC_CASE(3, 3, 16, 64)
  TC_CASE(3, 3, 64, 64)
  TC_CASE(3, 4, 16, 96)
  TC_CASE(3, 4, 96, 96)
  TC_CASE(3, 3, 16, 32)
  TC_CASE(3, 3, 32, 32)
  // split TF32 (kind::tf32, three MMAs per K slice): FP32-accurate products
  TC_CASE(1, 2, 16, 32)
  TC_CASE(1, 2, 32, 32)
  TC_CASE(1, 3, 16, 64)
  TC_CASE(1, 3, 64, 64)
  TC_CASE(1, 4, 16, 96)
  TC_CASE(1, 4, 96, 96)
  TC_CASE(1, 3, 16, 32)
  TC_CASE(1, 3, 32, 32)
  TC_CASE(1, 1, 16, 112)
  TC_CASE(1, 1, 112, 112)
  // the matched single-branch ResNet (width 112) in 16-bit operands
  TC_CASE(0, 1, 16, 112)
  TC_CASE(0, 1, 112, 112)
  TC_CASE(3, 1, 16, 112)
  TC_CASE(3, 1, 112, 112)
  // E4M3 operands (kind::f8f6f4): input layers take 32 padded channels (32-byte rows)
  TC_CASE(2, 2, 32, 32)
  TC_CASE(2, 3, 32, 32)
  TC_CASE(2, 3, 32, 64)
  TC_CASE(2, 3, 64, 64)
  TC_CASE(2, 4, 32, 96)
  TC_CASE(2, 4, 96, 96)
  TC_CASE(2, 1, 32, 64)
  TC_CASE(2, 1, 64, 64)
#undef TC_CASE
  return fail(CONET_ERR_UNSUPPORTED, "tensor-core conv kind=%d branches=%d Cin=%d Cout=%d not instantiated", kind, nb,
              cin, cout);
}

// ------------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

static CUtensorMapSwizzle swizzle_of(int row_bytes) {
  return row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                          : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

static CUtensorMapDataType dtype_of(int kind) {
  if (kind == 3) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                   : kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
}

int make_act_map(CUtensorMap* map, int kind, const void* base, int C, int F, int T, int slots, int kc, int taps) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(CONET_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int e = (kind == 0 || kind == 3) ? 2 : kind == 1 ? 4 : 1;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)F, (cuuint64_t)T, (cuuint64_t)slots};
  const cuuint64_t strides[3] = {(cuuint64_t)C * e, (cuuint64_t)F * C * e, (cuuint64_t)T * F * C * e};
  const cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)(taps == 3 ? TILE_M + 2 : TILE_M), 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = enc(map, dtype_of(kind), 4, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(kc * e), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CONET_ERR_CUDA, "activation tensor map encode failed (%d)", (int)r);
  return CONET_OK;
}

int make_weight_map(CUtensorMap* map, int kind, const void* base, int cin, int cout, int kc, int taps) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(CONET_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int e = (kind == 0 || kind == 3) ? 2 : kind == 1 ? 4 : 1;
  const cuuint64_t dims[3] = {(cuuint64_t)cin, (cuuint64_t)cout, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)cin * e, (cuuint64_t)cout * cin * e};
  const cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)cout, (cuuint32_t)taps};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, dtype_of(kind), 3, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(kc * e), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CONET_ERR_CUDA, "weight tensor map encode failed (%d)", (int)r);
  return CONET_OK;
}

// Channels per K chunk and taps per stage of the instantiation for (kind, nb, cin, cout).
int tc_chunk(int kind, int nb, int cin, int cout) { return tc_kc(kind, nb, cin, cout); }
int tc_taps(int kind, int nb, int cin, int cout) { return tc_halo(kind, nb, cin, cout) ? 3 : 1; }

// [Cout][3][3][cin_src] FP32 master -> [9][Cout][cin_dst] TF32 hi and FP32 lo = w - hi
__global__ void weights_split_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst,
                                     float* __restrict__ hi, float* __restrict__ lo) {
  const int n = 9 * cout * cin_dst;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin_dst, rem = i / cin_dst, co = rem % cout, tap = rem / cout;
    const float v = ci < cin_src ? w[((size_t)co * 9 + tap) * cin_src + ci] : 0.f;
    const float h = tf32_round(v);
    hi[i] = h;
    lo[i] = v - h;
  }
}

int launch_weights_split(const float* w, int cout, int cin_src, int cin_dst, float* hi, float* lo, cudaStream_t s) {
  weights_split_kernel<<<grid_for(9LL * cout * cin_dst, 256, 512), 256, 0, s>>>(w, cout, cin_src, cin_dst, hi, lo);
  return check_launch("weights_split_kernel");
}

// [Cout][3][3][cin_src] FP32 master -> [9][Cout][cin_dst] BF16, zero padded input channels
__global__ void weights_bf16_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst,
                                    __nv_bfloat16* __restrict__ out) {
  const int n = 9 * cout * cin_dst;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin_dst, rem = i / cin_dst, co = rem % cout, tap = rem / cout;
    out[i] = __float2bfloat16_rn(ci < cin_src ? w[((size_t)co * 9 + tap) * cin_src + ci] : 0.f);
  }
}

__global__ void weights_f16_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst,
                                   __half* __restrict__ out) {
  const int n = 9 * cout * cin_dst;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin_dst, rem = i / cin_dst, co = rem % cout, tap = rem / cout;
    out[i] = __float2half_rn(ci < cin_src ? w[((size_t)co * 9 + tap) * cin_src + ci] : 0.f);
  }
}

int launch_weights_16(int kind, const float* w, int cout, int cin_src, int cin_dst, void* out, cudaStream_t s) {
  if (kind == 3)
    weights_f16_kernel<<<grid_for(9LL * cout * cin_dst, 256, 512), 256, 0, s>>>(w, cout, cin_src, cin_dst,
                                                                                reinterpret_cast<__half*>(out));
  else
    weights_bf16_kernel<<<grid_for(9LL * cout * cin_dst, 256, 512), 256, 0, s>>>(
        w, cout, cin_src, cin_dst, reinterpret_cast<__nv_bfloat16*>(out));
  return check_launch("weights_16_kernel");
}

// Smallest power of two s with t / s <= 448, the largest finite E4M3 value (1 for t <= 0):
// with t = m 2^e, m in [0.5, 1), and 448 = 0.875 x 2^9, s = 2^(e - 9) if m <= 0.875 else
// 2^(e - 8).  Power-of-two scales make scaling and unscaling exact.
__device__ __forceinline__ float e4m3_pow2_scale(float t) {
  if (!(t > 0.f)) return 1.f;
  int e;
  const float m = frexpf(t, &e);
  return ldexpf(1.f, m <= 0.875f ? e - 9 : e - 8);
}

// One CTA per output channel: the channel's scale is the power of two that maps its largest
// |w| into (224, 448], so that each channel's E4M3 weights use the format's full range
// (per-output-channel scaling).
__global__ void weights_fp8_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst,
                                   uint8_t* __restrict__ out, float* __restrict__ wscale) {
  __shared__ float red[32];
  const int co = blockIdx.x;
  const int n = 9 * cin_src;
  const float* wc = w + (size_t)co * n;
  float mx = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(wc[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) red[0] = mx;
  }
  __syncthreads();
  const float scale = e4m3_pow2_scale(red[0]);
  const float inv = 1.f / scale;   // exact: a power of two
  if (threadIdx.x == 0) wscale[co] = scale;
  for (int i = threadIdx.x; i < 9 * cin_dst; i += blockDim.x) {
    const int tap = i / cin_dst, ci = i % cin_dst;
    const float v = ci < cin_src ? wc[(size_t)tap * cin_src + ci] * inv : 0.f;
    out[((size_t)tap * cout + co) * cin_dst + ci] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

int launch_weights_fp8(const float* w, int cout, int cin_src, int cin_dst, uint8_t* out, float* wscale,
                       cudaStream_t s) {
  weights_fp8_kernel<<<cout, 128, 0, s>>>(w, cout, cin_src, cin_dst, out, wscale);
  return check_launch("weights_fp8_kernel");
}

__global__ void fp8_scales_kernel(Fp8ScaleArgs a, int cout, float margin) {
  const int b = blockIdx.x;
  const float scale = e4m3_pow2_scale(margin * __uint_as_float(*a.amax[b]));
  if (threadIdx.x == 0) {
    *a.scale[b] = scale;
    *a.qinv[b] = 1.f / scale;
  }
  for (int c = threadIdx.x; c < cout; c += blockDim.x) a.dq[b][c] = scale * a.wscale[b][c];
}

int launch_fp8_scales(const Fp8ScaleArgs& a, int nb, int cout, float margin, cudaStream_t s) {
  fp8_scales_kernel<<<nb, 128, 0, s>>>(a, cout, margin);
  return check_launch("fp8_scales_kernel");
}

}  // namespace conet
