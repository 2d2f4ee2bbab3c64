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
// CTA pairs: the kernel runs in clusters of two CTAs that compute two tiles with one
// tcgen05.mma.cta_group::2 of M = 256 per K step.  Each CTA TMA-loads its own tile's A box and
// one half (Cout / 2 rows) of the weight slices; the MMA reads B across both CTAs' shared
// memory, so L2 serves every weight byte once per pair and each SM holds half the weights.
//
// Warp roles: warp 0 of each CTA issues that CTA's TMA loads into a ring of shared-memory
// stages (completion counted on the first CTA's barrier); warp 1 of the first CTA issues the
// pair's MMAs from one thread and commits each stage back to both producers; the epilogue
// warps of each CTA (4 TMEM lane quarters x 3 or 4 channel parts, one RE per thread) run the
// fused epilogue on their own CTA's accumulators: bias, residual add, ReLU / LayerNorm, the
// Hadamard fusion of the branches with its LayerNorm, the next layer's pre-activation, and
// the 1x1 LLR head.  Two TMEM accumulator sets (when they fit) let the epilogue of one tile
// overlap the MMAs of the next.
#pragma once

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

// Shared-memory bytes of one pipeline stage of one CTA of a pair: per branch (and split part)
// an A box of a_rows rows and `taps` weight slices of this CTA's cout / 2 rows, rows of `row`
// bytes; 1 KB aligned.
__host__ __device__ constexpr size_t stage_bytes(int kind, int nb, int cout, int row, int a_rows, int taps) {
  return ((size_t)nb * nsplit_of(kind) * ((size_t)a_rows * row + (size_t)taps * (cout / 2) * row) + 1023) / 1024 *
         1024;
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
// each), or 3 (14 warps, up to 128 registers) for the branch-group epilogues and for the
// single-group E4M3 epilogues of three or more branches whose Cout splits evenly in three
// (measured: 4 parts 5 % faster than 3 with 16-bit operands on the 14x624 network; on the
// 14x3276 branch-group network 3 parts are 3.5 % faster; on the 14x624 E4M3 network four
// even parts of 16 channels, which the fast fixed-shape epilogues need, beat three uneven
// ones by 26 %).
__host__ __device__ constexpr int epi_parts(int kind, int nb, int cout) {
  return (tc_groups(kind, nb, cout) == 1 && kind == 2 && nb >= 3 && (cout / 8) % 3 == 0) ||
                 tc_groups(kind, nb, cout) > 1
             ? 3
             : 4;
}

// Staged output stores of the fixed layer shapes (MODE 1..3, below): each epilogue warp
// writes its 32 rows x PW channels (PW = Cout / channel parts) of one output branch -- the
// FP32 stream and the next conv's input -- into two swizzled shared-memory boxes that two
// TMA stores write out, instead of storing 32 row segments 1 to 3 lines apart per store
// instruction (measured on the 14x3276 network: the scattered stream and next-input stores
// cost a third of the body convs' time).  Needs equal parts whose rows span 16, 32, 64 or
// 128 bytes in both types; not on the split-TF32 path (its next input has two FP32 parts).
__host__ __device__ constexpr int part_width(int kind, int nb, int cout) {
  return (cout / CW) % epi_parts(kind, nb, cout) == 0 ? cout / epi_parts(kind, nb, cout) : 0;
}
__host__ __device__ constexpr bool box_row_ok(int bytes) {
  return bytes == 16 || bytes == 32 || bytes == 64 || bytes == 128;
}
// the layer shapes with fixed-shape epilogues: residual-block body convs and the input
// layers of residual networks of three or more branches
__host__ __device__ constexpr bool fixed_shapes(int nb, int cin, int cout) {
  return (cin == cout && nb >= 2) || (cin != cout && nb >= 3);
}
__host__ __device__ constexpr bool staged_ok(int kind, int nb, int cin, int cout) {
  return kind != 1 && fixed_shapes(nb, cin, cout) && part_width(kind, nb, cout) > 0 &&
         box_row_ok(part_width(kind, nb, cout) * 4) && box_row_ok(part_width(kind, nb, cout) * elt_of(kind));
}
__host__ __device__ constexpr size_t kb_ceil(size_t x) { return (x + 1023) / 1024 * 1024; }
// per epilogue warp: the FP32 box, then the next-input box, each 1 KB aligned
__host__ __device__ constexpr size_t stg_xs_bytes(int kind, int nb, int cout) {
  return kb_ceil((size_t)32 * part_width(kind, nb, cout) * 4);
}
__host__ __device__ constexpr size_t stg_nx_bytes(int kind, int nb, int cout) {
  return kb_ceil((size_t)32 * part_width(kind, nb, cout) * elt_of(kind));
}
__host__ __device__ constexpr size_t stg_bytes(int kind, int nb, int cin, int cout) {
  return staged_ok(kind, nb, cin, cout)
             ? (size_t)4 * epi_parts(kind, nb, cout) * (stg_xs_bytes(kind, nb, cout) + stg_nx_bytes(kind, nb, cout))
             : 0;
}

__host__ __device__ constexpr int tc_plan(int kind, int nb_all, int cin, int cout, bool want_halo) {
  // returns KC for the requested stage shape, 0 if none fits; a stage holds one branch group
  const int nb = nb_all / tc_groups(kind, nb_all, cout);
  const int ep = epi_parts(kind, nb_all, cout);
  const size_t stg = stg_bytes(kind, nb_all, cin, cout);
  const size_t par = par_bytes(nb_all, cout) + (stg ? 1024 + stg : 0);
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

// HALO: 1 = the halo stage of a 3x3 conv (three subcarrier taps per stage), 0 = one 3x3 tap
// per stage, 2 = a 1x1 conv (the pointwise half of a depthwise-separable conv: only the
// centre tap, weights [1][Cout][Cin], CIN / KC K steps per tile).
template <int KIND, int NB, int CIN, int COUT, int KC, int HALO, int MODE = 0>
struct Cfg {
  static constexpr int ELT = elt_of(KIND);
  static constexpr int ROW = KC * ELT;                  // bytes per operand row (= swizzle span)
  static_assert(ROW == 32 || ROW == 64 || ROW == 128, "row bytes");
  static constexpr int SLICES = ROW / 32;               // MMAs (32 bytes of K each) per chunk
  static constexpr int NSPLIT = nsplit_of(KIND);        // split TF32: hi and lo copies of A and B
  static constexpr int TAPS = HALO == 1 ? 3 : 1;        // weight taps (subcarrier shifts) per stage
  static constexpr int A_BOX = HALO == 1 ? TILE_M + 2 : TILE_M;
  static constexpr int A_PART = (HALO == 1 ? HALO_ROWS : TILE_M) * ROW;
  static constexpr int B_ROWS = COUT / 2;               // weight rows (output channels) per CTA
  static constexpr int B_PART = TAPS * B_ROWS * ROW;
  static constexpr int A_BYTES = NSPLIT * A_PART;
  static constexpr int B_BYTES = NSPLIT * B_PART;
  static constexpr int NG = tc_groups(KIND, NB, COUT); // branch groups per tile
  static constexpr int G = NB / NG;                     // branches per MMA unit (one stage holds G)
  static constexpr int STAGE_TX = G * NSPLIT * (A_BOX * ROW + B_PART);   // bytes one CTA loads per stage
  static constexpr int STAGE = (int)stage_bytes(KIND, G, COUT, ROW, HALO == 1 ? HALO_ROWS : TILE_M, TAPS);
  static constexpr int K_ITERS = (HALO == 2 ? 1 : 9 / TAPS) * (CIN / KC);
  static constexpr int COLS = NG == 1 ? pow2_ceil(NB * COUT) : G * COUT;   // stride of accumulator sets
  static constexpr int N_ACC = NG == 1 ? (2 * COLS <= 512 ? 2 : 1) : 2;
  static constexpr int STASH = NG == 1 ? 0 : 2 * G * COUT;                 // running-product columns
  static constexpr int TMEM_COLS = NG == 1 ? N_ACC * COLS : 512;
  static_assert(NG == 1 || STASH + COUT <= 512, "TMEM columns for the product stash");
  static constexpr int EP = epi_parts(KIND, NB, COUT);  // channel parts per lane quarter
  static constexpr int EPI_WARPS = 4 * EP;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr size_t PAR = par_bytes(NB, COUT);
  // Staged output stores (fixed layer shapes only): each epilogue warp owns a 1 KB-aligned
  // region holding its FP32 box and its next-input box (conv1 of a block, MODE 1, writes no
  // stream: no FP32 box).  The region also serves as the warp's LayerNorm-moment scratch,
  // which is dead while the boxes are in use.
  static constexpr bool STAGED = MODE != 0 && staged_ok(KIND, NB, CIN, COUT);
  static constexpr int PW = part_width(KIND, NB, COUT);
  // (MODE 4 stores through no box: the region is its scratch only)
  static constexpr size_t XS_B = (MODE == 1 || MODE == 4) ? 0 : stg_xs_bytes(KIND, NB, COUT),
                          NX_B = MODE == 4 ? 0 : stg_nx_bytes(KIND, NB, COUT);
  static constexpr size_t REG_B =
      kb_ceil(XS_B + NX_B > SCR_WARP_FLOATS * sizeof(float) ? XS_B + NX_B : SCR_WARP_FLOATS * sizeof(float));
  static constexpr size_t SCR = STAGED ? 0 : scr_bytes(EP);
  static constexpr int SCR_STRIDE = STAGED ? (int)(REG_B / sizeof(float)) : SCR_WARP_FLOATS;   // floats per warp
  static constexpr size_t STG = STAGED ? (size_t)EPI_WARPS * REG_B : 0;
  static constexpr size_t fixed_end(int st) {
    return STAGED ? kb_ceil((size_t)st * STAGE + 256 + SCR + PAR) : (size_t)st * STAGE + 256 + SCR + PAR;
  }
  static constexpr int stages_max() {
    int st = 1;
    while (st < 8 && 1024 + fixed_end(st + 1) + STG <= SMEM_LIMIT) ++st;
    return st;
  }
  static constexpr int STAGES = stages_max();
  static constexpr size_t STG_OFF = fixed_end(STAGES);
  static constexpr size_t SMEM = 1024 + STG_OFF + STG;
  static constexpr uint32_t IDESC = tc::instr_desc(KIND == 0 ? 1 : KIND == 1 ? 2 : 0, COUT, 256);   // BF16 / TF32 / F16, E4M3
  static_assert(STAGES >= 2 && SMEM <= SMEM_LIMIT, "not enough shared memory for two stages");
  static_assert(COUT % 16 == 0 && COUT <= 256 && COUT % CW == 0, "MMA N");
  static_assert(B_ROWS % 8 == 0, "each CTA's weight half holds whole swizzle atoms");
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

// Layer shape seen by an epilogue.  MODE 0 reads every flag and output pointer at run time;
// MODE 1 (first conv of a residual block: LN2 + ReLU, next input only), MODE 2 (second conv
// of a fused residual block: residual add, fusion + LN, the stream, LN1 + ReLU of the
// supports and ReLU of the main branch, next input) and MODE 3 (input layer of a fused
// residual network: MODE 2 with a ReLU pre-activation and no residual) fix them at compile
// time, so their epilogues test no absent output and take no run-time branch on the layer
// type.  MODE 4 (the last conv2 of a fused residual network at inference: residual add,
// fusion + LN and the 1x1 head; no stream or next input) runs only where the fast
// epilogue (conv2_part) serves the shape (tc_mode).
template <int MODE>
struct Lay {
  static constexpr bool FUSED = MODE == 2 || MODE == 3 || MODE == 4;
  __device__ static bool pre_relu(const TcConvArgs& a) { return MODE == 0 ? a.pre == 1 : MODE == 3; }
  __device__ static bool pre_ln(const TcConvArgs& a) { return MODE == 0 ? a.pre == 2 : MODE == 1; }
  __device__ static bool fuse(const TcConvArgs& a) { return MODE == 0 ? a.fuse != 0 : FUSED; }
  __device__ static bool fuse_ln(const TcConvArgs& a) {
    return MODE == 0 ? (a.fuse != 0 && a.lnf_g != nullptr) : FUSED;
  }
  __device__ static int post(const TcConvArgs& a, int b) { return MODE == 0 ? a.post[b] : FUSED ? (b == 0 ? 1 : 2) : 0; }
  __device__ static bool resid(const TcConvArgs& a, int b) {
    return MODE == 0 ? a.resid[b] != nullptr : (MODE == 2 || MODE == 4);
  }
  __device__ static bool t_out(const TcConvArgs& a, int b) { return MODE == 0 && a.t_out[b] != nullptr; }
  __device__ static bool a_out(const TcConvArgs& a, int b) { return MODE == 0 && a.a_out[b] != nullptr; }
  __device__ static bool xs_out(const TcConvArgs& a, int b) {
    return MODE == 0 ? a.xs_out[b] != nullptr : (FUSED && MODE != 4);
  }
  __device__ static bool nx_out(const TcConvArgs& a, int b) { return MODE == 0 ? a.nx_out[b] != nullptr : MODE != 4; }
  __device__ static bool head(const TcConvArgs& a) { return MODE == 0 ? a.head_w != nullptr : MODE == 4; }
  __device__ static bool measure(const TcConvArgs& a) { return MODE == 0 && a.measure != 0; }
  __device__ static bool amax(const TcConvArgs& a, int b) { return MODE == 0 && a.amax[b] != nullptr; }
};

// v_b = acc_b (x dq_b on the E4M3 path) + bias_b (+ resid_b) for the 8 channels of chunk j
// of every branch (add = false: the raw TMEM columns, when an earlier pass wrote v back).
// (Branches b0 .. b0 + NB - 1, accumulators at TMEM columns 0, COUT, ... from tacc.)
template <int KIND, int NB, int COUT, int MODE>
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
    if (Lay<MODE>::resid(a, b0 + b) && valid) {
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

// A warp's staged output boxes (fixed layer shapes): its two shared-memory boxes, the
// output tensors' maps ([symbols][F][Cout] per branch) and the boxes' coordinates there
// (first channel, first subcarrier, symbol).  ok = false: a tile past the last one or rows
// wholly past the grid edge, nothing to store.  Rows past F inside a box are clipped by TMA.
struct StoreBox {
  uint8_t* xs;
  uint8_t* nx;
  const CUtensorMap* xs_map;
  const CUtensorMap* nx_map;
  int c0, f0, st;
  bool ok;
};

// Address of 16-byte chunk k of row r of a 1 KB-aligned box with rows of rb bytes, laid
// out in TMA's swizzle for that row length: the chunk index XOR row bits 0-2 (128-byte
// rows), 1-2 (64), 2 (32), none (16).  A warp writing one chunk column of 32 rows then
// touches every bank group evenly.
__device__ __forceinline__ uint8_t* box_chunk(uint8_t* box, int rb, int r, int k) {
  const int x = rb == 128 ? (r & 7) : rb == 64 ? ((r >> 1) & 3) : rb == 32 ? ((r >> 2) & 1) : 0;
  return box + r * rb + 16 * (k ^ x);
}

// Chunk jj (8 channels) of row r of a warp's boxes: FP32 stream values (two 16-byte chunks)
// and next-input values (16-bit: one 16-byte chunk; E4M3 of value x qinv: half of one).
template <int PW>
__device__ __forceinline__ void stage_xs8(uint8_t* box, int r, int jj, const float (&y)[CW]) {
  *reinterpret_cast<float4*>(box_chunk(box, PW * 4, r, 2 * jj)) = make_float4(y[0], y[1], y[2], y[3]);
  *reinterpret_cast<float4*>(box_chunk(box, PW * 4, r, 2 * jj + 1)) = make_float4(y[4], y[5], y[6], y[7]);
}
template <int KIND, int PW>
__device__ __forceinline__ void stage_nx8(uint8_t* box, int r, int jj, const float (&o)[CW], float qinv) {
  if constexpr (KIND == 2)
    store8_e4m3(box_chunk(box, PW, r, jj >> 1) + 8 * (jj & 1), o, qinv);
  else if constexpr (KIND == 3)
    store8_h(reinterpret_cast<__half*>(box_chunk(box, PW * 2, r, jj)), o);
  else
    store8_h(reinterpret_cast<__nv_bfloat16*>(box_chunk(box, PW * 2, r, jj)), o);
}

// a_b = pre(v_b) of the fixed layer shapes: relu(LN2_b(v_b)) (MODE 1), relu(v_b) (MODE 3),
// v_b (MODE 2); chunk c0 of branch b, LN2 statistics (mu, rs).
template <int MODE, int COUT>
__device__ __forceinline__ void pre_fixed(const float* par, int b, int c0, float mu, float rs, float (&v)[CW]) {
  using PL = ParLayout<COUT>;
  if constexpr (MODE == 1) {
    float g[CW], be[CW];
    lds8(par + PL::at(b, PF_LN2G) + c0, g);
    lds8(par + PL::at(b, PF_LN2B) + c0, be);
#pragma unroll
    for (int c = 0; c < CW; ++c) v[c] = fmaxf((v[c] - mu) * rs * g[c] + be[c], 0.f);
  } else if constexpr (MODE == 3) {
#pragma unroll
    for (int c = 0; c < CW; ++c) v[c] = fmaxf(v[c], 0.f);
  }
}

// next_b = post(x_b) of the fixed layer shapes: x_b (MODE 1); relu(x_0) for the fused main
// branch and relu(LN1_b(x_b)) for a support (MODE 2, 3), LN1 statistics (mu, rs).
template <int MODE, int COUT>
__device__ __forceinline__ void post_fixed(const float* par, int b, int c0, float mu, float rs, const float (&x)[CW],
                                           float (&o)[CW]) {
  using PL = ParLayout<COUT>;
  if constexpr (MODE == 1) {
#pragma unroll
    for (int c = 0; c < CW; ++c) o[c] = x[c];
  } else if (b == 0) {
#pragma unroll
    for (int c = 0; c < CW; ++c) o[c] = fmaxf(x[c], 0.f);
  } else {
    float g[CW], be[CW];
    lds8(par + PL::at(b, PF_LN1G) + c0, g);
    lds8(par + PL::at(b, PF_LN1B) + c0, be);
#pragma unroll
    for (int c = 0; c < CW; ++c) o[c] = fmaxf((x[c] - mu) * rs * g[c] + be[c], 0.f);
  }
}

// Before a warp rewrites its boxes: the TMA stores issued from them have read them.
__device__ __forceinline__ void boxes_free(int lane) {
  if (lane == 0) tc::bulk_wait_read();
  __syncwarp();
}

// After the warp has written its boxes: make the writes visible to TMA and store branch b's
// boxes (has_xs: the stream box too).
__device__ __forceinline__ void boxes_store(const StoreBox& sb, int b, bool has_xs, int lane) {
  tc::fence_proxy_async();
  __syncwarp();
  if (lane == 0 && sb.ok) {
    if (has_xs) tc::tma_store_3d(sb.xs_map + b, sb.xs, sb.c0, sb.f0, sb.st);
    tc::tma_store_3d(sb.nx_map + b, sb.nx, sb.c0, sb.f0, sb.st);
    tc::bulk_commit();
  }
}

// Two 16-bit values of max(x, 0) in one register (lo in the low half).
template <int KIND>
__device__ __forceinline__ uint32_t relu_pack2(float lo, float hi) {
  uint32_t r;
  if constexpr (KIND == 3)
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  else
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Next-input values of chunk k (8 channels) of row r of a warp's box, max(o, 0) first:
// 16-bit pairs packed with the ReLU in the conversion; E4M3 codes of value x qinv.
template <int KIND, int PC>
__device__ __forceinline__ void put_next8(uint8_t* box, int r, int k, const float (&o)[CW], float qinv) {
  if constexpr (KIND == 2) {
    float t[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) t[c] = fmaxf(o[c], 0.f);
    store8_e4m3(box_chunk(box, PC, r, k >> 1) + 8 * (k & 1), t, qinv);
  } else {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = relu_pack2<KIND>(o[2 * e], o[2 * e + 1]);
    *reinterpret_cast<uint4*>(box_chunk(box, PC * 2, r, k)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Epilogue of the first conv of a residual block (MODE 1), for a warp whose part is PC = 16
// or 32 channels of G branches (a branch group, or all branches): v_b = acc_b (x dq_b,
// E4M3) + bias_b, next_b = relu(LN2_b(v_b)).  The part's columns of every branch come out
// of TMEM with one wait and stay in registers through the moment exchange (no write-back,
// no second read), and the arithmetic runs on two-lane FP32 instructions: a quarter of the
// waits and half the FP32 instructions of the general epilogue, whose per-group time
// otherwise exceeds the group's MMA time.
template <int KIND, int G, int COUT, int EP, int SCR_STRIDE, int PC>
__device__ __forceinline__ void conv1_part(const float* par, uint32_t tacc, int b0, int part, int quarter, int lane,
                                           float* scr_all, const StoreBox& sb) {
  using PL = ParLayout<COUT>;
  static_assert(COUT == EP * PC && (PC == 16 || PC == 32), "equal parts of 16 or 32 channels");
  const int c0 = PC * part;
  float v[G][PC];
  {
    uint32_t r[G][PC / 16][16];
    __syncwarp();
#pragma unroll
    for (int bb = 0; bb < G; ++bb)
#pragma unroll
      for (int h = 0; h < PC / 16; ++h) tc::tmem_ld16_nowait(tacc + (uint32_t)(bb * COUT + c0 + 16 * h), r[bb][h]);
    tc::tmem_wait_ld();
#pragma unroll
    for (int bb = 0; bb < G; ++bb)
#pragma unroll
      for (int h = 0; h < PC / 16; ++h)
#pragma unroll
        for (int i = 0; i < 16; ++i) v[bb][16 * h + i] = __uint_as_float(r[bb][h][i]);
  }
  // (dequantise,) + bias; shifted moments of each branch over the part (shift: its first
  // value), summed in two interleaved lanes
  float* scr = scr_all + (size_t)(4 * part + ((quarter + 2) & 3)) * SCR_STRIDE;
  boxes_free(lane);   // the scratch shares the boxes of the last stores
#pragma unroll
  for (int bb = 0; bb < G; ++bb) {
#pragma unroll
    for (int k = 0; k < PC / CW; ++k) {
      float x[CW];
      if constexpr (KIND == 2) {
        lds8(par + PL::at(b0 + bb, PF_DQ) + c0 + CW * k, x);
#pragma unroll
        for (int c = 0; c < CW; ++c) v[bb][CW * k + c] *= x[c];
      }
      lds8(par + PL::at(b0 + bb, PF_BIAS) + c0 + CW * k, x);
#pragma unroll
      for (int c = 0; c < CW; ++c) v[bb][CW * k + c] += x[c];
    }
    const float k0 = v[bb][0];
    const unsigned long long kk = tc::f2pack(k0, k0);
    unsigned long long s1 = 0ull, s2 = 0ull;
#pragma unroll
    for (int c = 0; c < PC; c += 2) {
      const unsigned long long d = tc::f2sub(tc::f2pack(v[bb][c], v[bb][c + 1]), kk);
      s1 = tc::f2add(s1, d);
      s2 = tc::f2fma(d, d, s2);
    }
    float a1, b1, a2, b2;
    tc::f2unpack(s1, a1, b1);
    tc::f2unpack(s2, a2, b2);
    const float t1 = a1 + b1, t2 = a2 + b2, m1 = t1 / (float)PC;
    scr[(2 * bb) * 32 + lane] = k0 + m1;
    scr[(2 * bb + 1) * 32 + lane] = fmaxf(t2 - t1 * m1, 0.f);
  }
  named_barrier(1 + quarter, 32 * EP);
  float mean[G], rstd[G];
#pragma unroll
  for (int bb = 0; bb < G; ++bb) {
    float n = 0.f, mu = 0.f, M2 = 0.f;
#pragma unroll
    for (int pp = 0; pp < EP; ++pp) {
      const float* o = scr_all + (size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE;
      chan_fold(n, mu, M2, (float)PC, o[(2 * bb) * 32 + lane], o[(2 * bb + 1) * 32 + lane]);
    }
    mean[bb] = mu;
    rstd[bb] = rsqrtf(M2 / (float)COUT + 1e-5f);
  }
  named_barrier(1 + quarter, 32 * EP);
  // next_b = relu((v_b - mu) * rs * g + beta), one branch at a time through the warp's box
#pragma unroll
  for (int bb = 0; bb < G; ++bb) {
    const int b = b0 + bb;
    const float qinv = KIND == 2 ? lds1(par + PL::QINV + b) : 0.f;
    const unsigned long long mu2 = tc::f2pack(mean[bb], mean[bb]), rs2 = tc::f2pack(rstd[bb], rstd[bb]);
    boxes_free(lane);
#pragma unroll
    for (int k = 0; k < PC / CW; ++k) {
      float gm[CW], be[CW], o[CW];
      lds8(par + PL::at(b, PF_LN2G) + c0 + CW * k, gm);
      lds8(par + PL::at(b, PF_LN2B) + c0 + CW * k, be);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = CW * k + 2 * e;
        unsigned long long t = tc::f2mul(tc::f2sub(tc::f2pack(v[bb][c], v[bb][c + 1]), mu2), rs2);
        t = tc::f2fma(t, tc::f2pack(gm[2 * e], gm[2 * e + 1]), tc::f2pack(be[2 * e], be[2 * e + 1]));
        tc::f2unpack(t, o[2 * e], o[2 * e + 1]);
      }
      put_next8<KIND, PC>(sb.nx, lane, k, o, qinv);
    }
    boxes_store(sb, b, false, lane);
  }
}

// Epilogue of the fused fixed shapes (MODE 2: second conv of a residual block; MODE 3: the
// input layer, a_b = relu(v_b) and no residual; MODE 4: the last block's second conv, with
// the head instead of stream and next input), for a warp whose part is PC = 16 or 32
// channels of G branches b0 .. b0 + G - 1 (a branch group: first / last say which; or all
// branches: both).  Pass 1: v_b = acc_b (x dq_b, E4M3) + bias_b (+ resid_b), a_b = v_b
// (MODE 3: relu(v_b)), written back to TMEM; the running Hadamard product of the a_b in the
// TMEM stash; the LN1 moments of the support branches and, in the last group, those of the
// product.  Pass 2, one output at a time through the warp's boxes: each support's stream
// x_b = a_b and next input relu(LN1_b(a_b)); in the last group branch 0's stream x_0 =
// LN_f(product) and next input relu(x_0).  MODE 4 writes nothing back and takes no support
// moments; its pass 2 forms the head's partial sums of LN_f(product) over the part, and the
// quarter's part 0 adds them up through the scratch into the LLRs.  Pass 1 goes in 8-column steps whose residual rows and TMEM loads are
// all issued before the step's one wait (16-column steps spill at the 128-register budget
// of a 14-warp CTA and measured 6 % slower); pass 2 reads 16 columns per wait; the
// arithmetic runs on two-lane FP32 instructions.
template <int KIND, int G, int COUT, int EP, int SCR_STRIDE, int PC, int MODE>
__device__ __forceinline__ void conv2_part(const TcConvArgs& a, const float* par, uint32_t tacc, uint32_t tstash,
                                           int b0, bool first, bool last, bool valid, long long m, int part,
                                           int quarter, int lane, float* scr_all, const StoreBox& sb) {
  using PL = ParLayout<COUT>;
  static_assert(COUT == EP * PC && (PC == 16 || PC == 32), "equal parts of 16 or 32 channels");
  static_assert(MODE == 2 || MODE == 3 || MODE == 4, "fused fixed shapes");
  constexpr bool RESID = MODE != 3, PRE_RELU = MODE == 3, HEAD = MODE == 4;
  const int c0 = PC * part;
  // shifted moments: slot bb < G for support branch b0 + bb, slot G for the product
  float ks[G + 1];
  unsigned long long s1[G + 1], s2[G + 1];
#pragma unroll
  for (int i = 0; i <= G; ++i) {
    ks[i] = 0.f;
    s1[i] = s2[i] = 0ull;
  }
#pragma unroll
  for (int j = 0; j < PC / CW; ++j) {
    const int ch = c0 + CW * j;
    float r[G][CW];
#pragma unroll
    for (int bb = 0; bb < G; ++bb) {
      if (RESID && valid) {
        ldg8(a.resid[b0 + bb] + m * COUT + ch, r[bb]);
      } else {
#pragma unroll
        for (int c = 0; c < CW; ++c) r[bb][c] = 0.f;
      }
    }
    uint32_t acc[G][CW], qr[CW];
    __syncwarp();
#pragma unroll
    for (int bb = 0; bb < G; ++bb) tc::tmem_ld8_nowait(tacc + (uint32_t)(bb * COUT + ch), acc[bb]);
    if (!first) tc::tmem_ld8_nowait(tstash + (uint32_t)ch, qr);
    tc::tmem_wait_ld();
    unsigned long long q[CW / 2];
#pragma unroll
    for (int i = 0; i < CW / 2; ++i)
      q[i] = first ? tc::f2pack(1.f, 1.f) : tc::f2pack(__uint_as_float(qr[2 * i]), __uint_as_float(qr[2 * i + 1]));
    float bi[G][CW];
#pragma unroll
    for (int bb = 0; bb < G; ++bb) lds8(par + PL::at(b0 + bb, PF_BIAS) + ch, bi[bb]);
#pragma unroll
    for (int bb = 0; bb < G; ++bb) {
      float dq[CW];
      if constexpr (KIND == 2) lds8(par + PL::at(b0 + bb, PF_DQ) + ch, dq);
      float v[CW];
#pragma unroll
      for (int e = 0; e < CW / 2; ++e) {
        unsigned long long t = tc::f2pack(__uint_as_float(acc[bb][2 * e]), __uint_as_float(acc[bb][2 * e + 1]));
        if constexpr (KIND == 2) t = tc::f2mul(t, tc::f2pack(dq[2 * e], dq[2 * e + 1]));
        t = tc::f2add(t, tc::f2pack(bi[bb][2 * e], bi[bb][2 * e + 1]));
        if constexpr (RESID) t = tc::f2add(t, tc::f2pack(r[bb][2 * e], r[bb][2 * e + 1]));
        tc::f2unpack(t, v[2 * e], v[2 * e + 1]);
        if constexpr (PRE_RELU) {
          v[2 * e] = fmaxf(v[2 * e], 0.f);
          v[2 * e + 1] = fmaxf(v[2 * e + 1], 0.f);
        }
      }
      if constexpr (!HEAD) tc::tmem_st8_nowait(tacc + (uint32_t)(bb * COUT + ch), v);
      if (!HEAD && b0 + bb != 0) {
        if (j == 0) ks[bb] = v[0];
        const unsigned long long kk = tc::f2pack(ks[bb], ks[bb]);
#pragma unroll
        for (int i = 0; i < CW / 2; ++i) {
          const unsigned long long d = tc::f2sub(tc::f2pack(v[2 * i], v[2 * i + 1]), kk);
          s1[bb] = tc::f2add(s1[bb], d);
          s2[bb] = tc::f2fma(d, d, s2[bb]);
        }
      }
#pragma unroll
      for (int i = 0; i < CW / 2; ++i) q[i] = tc::f2mul(q[i], tc::f2pack(v[2 * i], v[2 * i + 1]));
    }
    float qf[CW];
#pragma unroll
    for (int i = 0; i < CW / 2; ++i) tc::f2unpack(q[i], qf[2 * i], qf[2 * i + 1]);
    if (last) {
      if (j == 0) ks[G] = qf[0];
      const unsigned long long kk = tc::f2pack(ks[G], ks[G]);
#pragma unroll
      for (int i = 0; i < CW / 2; ++i) {
        const unsigned long long d = tc::f2sub(q[i], kk);
        s1[G] = tc::f2add(s1[G], d);
        s2[G] = tc::f2fma(d, d, s2[G]);
      }
    }
    tc::tmem_st8_nowait(tstash + (uint32_t)ch, qf);
  }
  __syncwarp();
  tc::tmem_wait_st();
  // publish, then merge over the quarter's parts (Chan), the slots in use
  float* scr = scr_all + (size_t)(4 * part + ((quarter + 2) & 3)) * SCR_STRIDE;
  boxes_free(lane);   // the scratch shares the boxes of the last stores
#pragma unroll
  for (int i = 0; i <= G; ++i) {
    if (i < G ? b0 + i == 0 : !last) continue;
    float a1, c1, a2, c2;
    tc::f2unpack(s1[i], a1, c1);
    tc::f2unpack(s2[i], a2, c2);
    const float t1 = a1 + c1, t2 = a2 + c2, m1 = t1 / (float)PC;
    scr[(2 * i) * 32 + lane] = ks[i] + m1;
    scr[(2 * i + 1) * 32 + lane] = fmaxf(t2 - t1 * m1, 0.f);
  }
  named_barrier(1 + quarter, 32 * EP);
  float mean[G + 1], rstd[G + 1];
#pragma unroll
  for (int i = 0; i <= G; ++i) {
    mean[i] = 0.f;
    rstd[i] = 1.f;
    if (i < G ? b0 + i == 0 : !last) continue;
    float n = 0.f, mu = 0.f, M2 = 0.f;
#pragma unroll
    for (int pp = 0; pp < EP; ++pp) {
      const float* o = scr_all + (size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE;
      chan_fold(n, mu, M2, (float)PC, o[(2 * i) * 32 + lane], o[(2 * i + 1) * 32 + lane]);
    }
    mean[i] = mu;
    rstd[i] = rsqrtf(M2 / (float)COUT + 1e-5f);
  }
  named_barrier(1 + quarter, 32 * EP);
  if constexpr (HEAD) {
    // the head on x_0 = LN_f(product): partial sums over the part, then part 0 adds the parts
    if (!last) return;
    float hq[HEAD_QMAX];
#pragma unroll
    for (int qq = 0; qq < HEAD_QMAX; ++qq) hq[qq] = 0.f;
    const unsigned long long mu2 = tc::f2pack(mean[G], mean[G]), rs2 = tc::f2pack(rstd[G], rstd[G]);
#pragma unroll
    for (int h = 0; h < PC / 16; ++h) {
      const int ch = c0 + 16 * h;
      uint32_t xr[16];
      __syncwarp();
      tc::tmem_ld16_nowait(tstash + (uint32_t)ch, xr);
      tc::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int cc = ch + CW * k;
        float gm[CW], be[CW], x0[CW];
        lds8(par + PL::LNFG + cc, gm);
        lds8(par + PL::LNFB + cc, be);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = CW * k + 2 * e;
          unsigned long long t = tc::f2mul(
              tc::f2sub(tc::f2pack(__uint_as_float(xr[c]), __uint_as_float(xr[c + 1])), mu2), rs2);
          t = tc::f2fma(t, tc::f2pack(gm[2 * e], gm[2 * e + 1]), tc::f2pack(be[2 * e], be[2 * e + 1]));
          tc::f2unpack(t, x0[2 * e], x0[2 * e + 1]);
        }
#pragma unroll
        for (int qq = 0; qq < HEAD_QMAX; ++qq) {
          if (qq >= a.Q) break;
          float hw[CW];
          lds8(par + PL::HEADW + qq * COUT + cc, hw);
          float sacc = 0.f;
#pragma unroll
          for (int c = 0; c < CW; ++c) sacc = fmaf(hw[c], x0[c], sacc);
          hq[qq] += sacc;
        }
      }
    }
    __syncwarp();
    for (int qq = 0; qq < a.Q && qq < HEAD_QMAX; ++qq) scr[qq * 32 + lane] = hq[qq];
    named_barrier(5 + quarter, 32 * EP);
    if (part == 0 && valid) {
      for (int qq = 0; qq < a.Q && qq < HEAD_QMAX; ++qq) {
        float sum = 0.f;
#pragma unroll
        for (int pp = 0; pp < EP; ++pp) sum += scr_all[(size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE + qq * 32 + lane];
        const float v = sum + lds1(par + PL::HEADB + qq);
        a.llr[m * a.Q + qq] = v;
        if (!(fabsf(v) <= FLT_MAX)) *a.nonfinite = 1;
      }
    }
    return;
  }
  // pass 2: the supports of the group, then (last group) branch 0
#pragma unroll
  for (int ob = 0; ob <= G; ++ob) {
    const bool is_main = ob == G;
    const int b = is_main ? 0 : b0 + ob;
    if (is_main ? !last : b == 0) continue;
    const float qinv = KIND == 2 ? lds1(par + PL::QINV + b) : 0.f;
    const unsigned long long mu2 = tc::f2pack(mean[ob], mean[ob]), rs2 = tc::f2pack(rstd[ob], rstd[ob]);
    boxes_free(lane);
#pragma unroll
    for (int h = 0; h < PC / 16; ++h) {
      const int ch = c0 + 16 * h;
      uint32_t xr[16];
      __syncwarp();
      tc::tmem_ld16_nowait(is_main ? tstash + (uint32_t)ch : tacc + (uint32_t)(ob * COUT + ch), xr);
      tc::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int cc = ch + CW * k;
        float gm[CW], be[CW], y[CW], o[CW];
        lds8(par + (is_main ? PL::LNFG : PL::at(b, PF_LN1G)) + cc, gm);
        lds8(par + (is_main ? PL::LNFB : PL::at(b, PF_LN1B)) + cc, be);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = CW * k + 2 * e;
          const unsigned long long x2 = tc::f2pack(__uint_as_float(xr[c]), __uint_as_float(xr[c + 1]));
          // LayerNorm: of the product for branch 0 (its stream), of v_b for a support (its
          // next input); a support's stream is v_b itself
          unsigned long long t = tc::f2mul(tc::f2sub(x2, mu2), rs2);
          t = tc::f2fma(t, tc::f2pack(gm[2 * e], gm[2 * e + 1]), tc::f2pack(be[2 * e], be[2 * e + 1]));
          tc::f2unpack(is_main ? t : x2, y[2 * e], y[2 * e + 1]);
          tc::f2unpack(t, o[2 * e], o[2 * e + 1]);
        }
        stage_xs8<PC>(sb.xs, lane, (cc - c0) / CW, y);
        put_next8<KIND, PC>(sb.nx, lane, (cc - c0) / CW, o, qinv);
      }
    }
    boxes_store(sb, b, true, lane);
  }
}

// The fused epilogue for one RE (this thread's TMEM lane) and one part of its channels.
// Pass 1 (when a LayerNorm is applied) folds each branch's values, and the fused product,
// into shifted first and second moments; the parts of a lane quarter publish theirs in
// their shared scratch and each part merges all of them in the same order (Chan et al.), so
// every part normalises with identical statistics.  Pass 1 also writes the biased (and
// residual-added) values back into TMEM.  Pass 2 applies the pre-activation, the Hadamard
// fusion and its LayerNorm, writes the residual stream and the next conv's input, and
// accumulates the head's partial sums, which part 0 reduces through the scratch.
template <int KIND, int NB, int COUT, int EP, int MODE, int PW, int SCR_STRIDE>
__device__ __forceinline__ void tc_epilogue(const TcConvArgs& a, const float* par, uint32_t tacc, bool valid,
                                            long long m, int part, int quarter, int lane, float* scr_all,
                                            const StoreBox& sb) {
  constexpr int QMAX = HEAD_QMAX;
  using PL = ParLayout<COUT>;
  // the fixed residual-block shapes with equal 16- or 32-channel parts (conv1: when the
  // part's columns of all branches fit the 96 registers of an 18-warp CTA beside the rest;
  // conv2: when the accumulator set's unused columns can hold the product)
  if constexpr (MODE == 1 && (PW == 16 || PW == 32) && NB * PW <= 48) {
    conv1_part<KIND, NB, COUT, EP, SCR_STRIDE, PW>(par, tacc, 0, part, quarter, lane, scr_all, sb);
    return;
  }
  if constexpr ((MODE == 2 || MODE == 3 || MODE == 4) && (PW == 16 || PW == 32) &&
                pow2_ceil(NB * COUT) >= NB * COUT + COUT) {
    conv2_part<KIND, NB, COUT, EP, SCR_STRIDE, PW, MODE>(a, par, tacc, tacc + (uint32_t)(NB * COUT), 0, true, true,
                                                         valid, m, part, quarter, lane, scr_all, sb);
    return;
  }
  float* scr = scr_all + (size_t)(4 * part + ((quarter + 2) & 3)) * SCR_STRIDE;
  int j_lo, n_ch;
  part_chunks<COUT, EP>(part, j_lo, n_ch);
  const int j_hi = j_lo + n_ch;
  using LY = Lay<MODE>;
  const bool pre_ln = LY::pre_ln(a), fuse_ln = LY::fuse_ln(a);
  bool any_ln1 = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) any_ln1 = any_ln1 || LY::post(a, b) == 2;
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
      load_chunk<KIND, NB, COUT, MODE>(a, par, tacc, 0, j, valid, m, v, true);
      __syncwarp();   // tcgen05.st is warp-collective: reconverge after the per-row residual loads
#pragma unroll
      for (int b = 0; b < NB; ++b) tc::tmem_st8_nowait(tacc + (uint32_t)(b * COUT + CW * j), v[b]);
      // the statistic of branch b is over v_b (pre_ln) or over pre(v_b) (the next block's
      // LN1); the fused product is over pre(v_b).  pre = 1 is ReLU, applied in place here
      // (pass 2 re-reads the unactivated values from TMEM).
      if (LY::pre_relu(a)) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int c = 0; c < CW; ++c) v[b][c] = fmaxf(v[b][c], 0.f);
      }
      // run-time layers with the sum interaction or Example II's feedback: the fused
      // statistic is over the sum of the a_b, and a support's (LN1) statistic over a_b + a_0
      const bool sum_op = MODE == 0 && a.op == 1, fb = MODE == 0 && a.feedback && LY::fuse(a);
      if (j == j_lo) {
        float p0 = sum_op ? 0.f : 1.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          k_b[b] = fb && b > 0 ? v[b][0] + v[0][0] : v[b][0];
          p0 = sum_op ? p0 + v[b][0] : p0 * v[b][0];
        }
        k_p = p0;
      }
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        float p = sum_op ? 0.f : 1.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const float x_b = fb && b > 0 ? v[b][c] + v[0][c] : v[b][c];
          const float d = x_b - k_b[b];
          s1_b[b] += d;
          s2_b[b] = fmaf(d, d, s2_b[b]);
          p = sum_op ? p + v[b][c] : p * v[b][c];
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
    if constexpr (PW > 0) boxes_free(lane);   // the scratch shares the boxes of the last stores
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
        const float* o = scr_all + (size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE;
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

  if constexpr (PW > 0) {
    // pass 2 of the fixed layer shapes, staged (PW channels per part): one output branch at
    // a time through the warp's boxes.  Their statistics pass wrote v_b back to TMEM; they
    // have no head and measure nothing.
    static_assert(MODE != 0, "staged stores serve the fixed layer shapes");
#pragma unroll
    for (int ob = 0; ob < NB; ++ob) {
      const bool has_xs = LY::xs_out(a, ob);
      const float qinv = KIND == 2 ? lds1(par + PL::QINV + ob) : 0.f;
      boxes_free(lane);
      for (int j = j_lo; j < j_hi; ++j) {
        float v[NB][CW];
        __syncwarp();
        load_chunk<KIND, NB, COUT, MODE>(a, par, tacc, 0, j, valid, m, v, false);
        const int c0 = CW * j;
        float x[CW];
        if (LY::fuse(a) && ob == 0) {
          // x_0 = LN_f(prod_b a_b)
#pragma unroll
          for (int b = 0; b < NB; ++b) pre_fixed<MODE, COUT>(par, b, c0, mean_b[b], rstd_b[b], v[b]);
          float g[CW], be[CW];
          lds8(par + PL::LNFG + c0, g);
          lds8(par + PL::LNFB + c0, be);
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            float p = v[0][c];
#pragma unroll
            for (int b = 1; b < NB; ++b) p *= v[b][c];
            x[c] = (p - mean_p) * rstd_p * g[c] + be[c];
          }
        } else {
          pre_fixed<MODE, COUT>(par, ob, c0, mean_b[ob], rstd_b[ob], v[ob]);
#pragma unroll
          for (int c = 0; c < CW; ++c) x[c] = v[ob][c];
        }
        if (has_xs) stage_xs8<PW>(sb.xs, lane, j - j_lo, x);
        float o[CW];
        post_fixed<MODE, COUT>(par, ob, c0, mean_b[ob], rstd_b[ob], x, o);
        stage_nx8<KIND, PW>(sb.nx, lane, j - j_lo, o, qinv);
      }
      boxes_store(sb, ob, has_xs, lane);
    }
    return;
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
    load_chunk<KIND, NB, COUT, MODE>(a, par, tacc, 0, j, valid, m, v, add2);
    const int c0 = CW * j;
    // rows past the grid edge compute on don't-care values and store nothing
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (valid && LY::t_out(a, b)) stg8(a.t_out[b] + m * COUT + c0, v[b]);
    // a_b = pre(v_b), in place
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (LY::pre_relu(a)) {
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
      if (valid && LY::a_out(a, b)) stg8(a.a_out[b] + m * COUT + c0, v[b]);
    // x_0 = fused (and normalised) product or sum, or a_0; it replaces v[0] from here on;
    // with Example II's feedback the supports continue with a_b + a_0
    if (LY::fuse(a)) {
      if constexpr (MODE == 0) {
        const bool sum_op = a.op == 1;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const float a0 = v[0][c];
#pragma unroll
          for (int b = 1; b < NB; ++b) v[0][c] = sum_op ? v[0][c] + v[b][c] : v[0][c] * v[b][c];
          if (a.feedback) {
#pragma unroll
            for (int b = 1; b < NB; ++b) v[b][c] += a0;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < CW; ++c) {
#pragma unroll
          for (int b = 1; b < NB; ++b) v[0][c] *= v[b][c];
        }
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
      if (valid && LY::xs_out(a, b) && !LY::measure(a)) stg8(a.xs_out[b] + m * COUT + c0, v[b]);
      if (LY::nx_out(a, b)) {
        float o[CW];
        if (LY::post(a, b) == 2) {
          float g[CW], be[CW];
          lds8(par + PL::at(b, PF_LN1G) + c0, g);
          lds8(par + PL::at(b, PF_LN1B) + c0, be);
          const float mu = mean_b[b], rs = rstd_b[b];
#pragma unroll
          for (int c = 0; c < CW; ++c) o[c] = fmaxf((v[b][c] - mu) * rs * g[c] + be[c], 0.f);
        } else if (LY::post(a, b) == 1) {
#pragma unroll
          for (int c = 0; c < CW; ++c) o[c] = fmaxf(v[b][c], 0.f);
        } else {
#pragma unroll
          for (int c = 0; c < CW; ++c) o[c] = v[b][c];
        }
        if constexpr (KIND == 2) {
          if (LY::amax(a, b) && valid) {
#pragma unroll
            for (int c = 0; c < CW; ++c) amx[b] = fmaxf(amx[b], fabsf(o[c]));
          }
          if (valid && !LY::measure(a))
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
    if (LY::head(a)) {
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
      if (!LY::amax(a, b)) continue;
      float mx = amx[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(a.amax[b], __float_as_uint(mx));
    }
  }
  if (LY::head(a)) {
    __syncwarp();
    for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) scr[qq * 32 + lane] = hq[qq];
    named_barrier(5 + quarter, 32 * EP);
    if (part == 0 && valid && !LY::measure(a)) {
      for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) {
        float sum = 0.f;
#pragma unroll
        for (int pp = 0; pp < EP; ++pp)
          sum += scr_all[(size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE + qq * 32 + lane];
        const float v = sum + lds1(par + PL::HEADB + qq);
        a.llr[m * a.Q + qq] = v;
        if (!(fabsf(v) <= FLT_MAX)) *a.nonfinite = 1;
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
template <int KIND, int NB, int COUT, int G, int EP, int MODE, int PW, int SCR_STRIDE>
__device__ __forceinline__ void tc_epilogue_group(const TcConvArgs& a, const float* par, uint32_t tacc,
                                                  uint32_t tstash, int g, bool valid, long long m, int part,
                                                  int quarter, int lane, float* scr_all, const StoreBox& sb) {
  constexpr int QMAX = HEAD_QMAX;
  using PL = ParLayout<COUT>;
  constexpr int NG = NB / G;
  if constexpr (MODE == 1 && (PW == 16 || PW == 32)) {
    conv1_part<KIND, G, COUT, EP, SCR_STRIDE, PW>(par, tacc, g * G, part, quarter, lane, scr_all, sb);
    return;
  }
  if constexpr ((MODE == 2 || MODE == 3 || MODE == 4) && (PW == 16 || PW == 32)) {
    conv2_part<KIND, G, COUT, EP, SCR_STRIDE, PW, MODE>(a, par, tacc, tstash, g * G, g == 0, g == NB / G - 1, valid,
                                                        m, part, quarter, lane, scr_all, sb);
    return;
  }
  float* scr = scr_all + (size_t)(4 * part + ((quarter + 2) & 3)) * SCR_STRIDE;
  int j_lo, n_ch;
  part_chunks<COUT, EP>(part, j_lo, n_ch);
  const int j_hi = j_lo + n_ch;
  const int b0 = g * G;
  const bool first = g == 0, last = g == NG - 1;
  using LY = Lay<MODE>;
  const bool pre_ln = LY::pre_ln(a), fuse = LY::fuse(a), fuse_ln = LY::fuse_ln(a);
  const bool main_here = fuse ? last : first;   // the group that forms branch 0's output
  bool any_b = false;
#pragma unroll
  for (int bb = 0; bb < G; ++bb) any_b = any_b || pre_ln || LY::post(a, b0 + bb) == 2;
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
      load_chunk<KIND, G, COUT, MODE>(a, par, tacc, b0, j, valid, m, v, true);
      __syncwarp();
#pragma unroll
      for (int bb = 0; bb < G; ++bb) tc::tmem_st8_nowait(tacc + (uint32_t)(bb * COUT + CW * j), v[bb]);
      if (LY::pre_relu(a)) {
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
    if constexpr (PW > 0) boxes_free(lane);   // the scratch shares the boxes of the last stores
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
        const float* o = scr_all + (size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE;
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

  if constexpr (PW > 0) {
    // pass 2 of the fixed layer shapes, staged: the group's support branches, then branch 0
    // where it is formed, one at a time through the warp's boxes (statistics were taken:
    // TMEM holds v_b and, in the last group of a fused layer, the stash the product)
    static_assert(MODE != 0, "staged stores serve the fixed layer shapes");
#pragma unroll
    for (int ob = 0; ob <= G; ++ob) {
      const bool is_main = ob == G;
      const int b = is_main ? 0 : b0 + ob;
      if (is_main ? !main_here : b == 0) continue;
      const int si = is_main ? 0 : ob;   // statistics slot (not fused: branch 0 is slot 0 of group 0)
      const bool has_xs = LY::xs_out(a, b);
      const float qinv = KIND == 2 ? lds1(par + PL::QINV + b) : 0.f;
      boxes_free(lane);
      for (int j = j_lo; j < j_hi; ++j) {
        const int c0 = CW * j;
        float x[CW];
        __syncwarp();
        if (is_main && fuse) {
          tmem_get8(tstash + (uint32_t)c0, x);   // the fused product
          float gm[CW], be[CW];
          lds8(par + PL::LNFG + c0, gm);
          lds8(par + PL::LNFB + c0, be);
#pragma unroll
          for (int c = 0; c < CW; ++c) x[c] = (x[c] - mean_p) * rstd_p * gm[c] + be[c];
        } else {
          tmem_get8(tacc + (uint32_t)(si * COUT + c0), x);
          pre_fixed<MODE, COUT>(par, b, c0, mean_b[si], rstd_b[si], x);
        }
        if (has_xs) stage_xs8<PW>(sb.xs, lane, j - j_lo, x);
        float o[CW];
        post_fixed<MODE, COUT>(par, b, c0, mean_b[si], rstd_b[si], x, o);
        stage_nx8<KIND, PW>(sb.nx, lane, j - j_lo, o, qinv);
      }
      boxes_store(sb, b, has_xs, lane);
    }
    return;
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
    load_chunk<KIND, G, COUT, MODE>(a, par, tacc, b0, j, valid, m, v, !stats);
    const int c0 = CW * j;
#pragma unroll
    for (int bb = 0; bb < G; ++bb)
      if (valid && LY::t_out(a, b0 + bb)) stg8(a.t_out[b0 + bb] + m * COUT + c0, v[bb]);
#pragma unroll
    for (int bb = 0; bb < G; ++bb) {
      if (LY::pre_relu(a)) {
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
      if (valid && LY::a_out(a, b0 + bb)) stg8(a.a_out[b0 + bb] + m * COUT + c0, v[bb]);
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
      if (valid && LY::xs_out(a, b) && !LY::measure(a)) stg8(a.xs_out[b] + m * COUT + c0, y);
      if (!LY::nx_out(a, b)) continue;
      float o[CW];
      if (LY::post(a, b) == 2) {
        float gm[CW], be[CW];
        lds8(par + PL::at(b, PF_LN1G) + c0, gm);
        lds8(par + PL::at(b, PF_LN1B) + c0, be);
        const float mu = mean_b[bb < G ? bb : 0], rs = rstd_b[bb < G ? bb : 0];
#pragma unroll
        for (int c = 0; c < CW; ++c) o[c] = fmaxf((y[c] - mu) * rs * gm[c] + be[c], 0.f);
      } else if (LY::post(a, b) == 1) {
#pragma unroll
        for (int c = 0; c < CW; ++c) o[c] = fmaxf(y[c], 0.f);
      } else {
#pragma unroll
        for (int c = 0; c < CW; ++c) o[c] = y[c];
      }
      if constexpr (KIND == 2) {
        if (LY::amax(a, b) && valid) {
          float& mx = is_main ? amx0 : amx_b[bb < G ? bb : 0];
#pragma unroll
          for (int c = 0; c < CW; ++c) mx = fmaxf(mx, fabsf(o[c]));
        }
        if (valid && !LY::measure(a))
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
    if (main_here && LY::head(a)) {
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
      if ((is_main ? !main_here : b == 0) || !LY::amax(a, b)) continue;
      float mx = is_main ? amx0 : amx_b[bb < G ? bb : 0];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(a.amax[b], __float_as_uint(mx));
    }
  }
  if (main_here && LY::head(a)) {
    __syncwarp();
    for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) scr[qq * 32 + lane] = hq[qq];
    named_barrier(5 + quarter, 32 * EP);
    if (part == 0 && valid && !LY::measure(a)) {
      for (int qq = 0; qq < a.Q && qq < QMAX; ++qq) {
        float sum = 0.f;
#pragma unroll
        for (int pp = 0; pp < EP; ++pp)
          sum += scr_all[(size_t)(4 * pp + ((quarter + 2) & 3)) * SCR_STRIDE + qq * 32 + lane];
        const float v = sum + lds1(par + PL::HEADB + qq);
        a.llr[m * a.Q + qq] = v;
        if (!(fabsf(v) <= FLT_MAX)) *a.nonfinite = 1;
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

template <int KIND, int NB, int CIN, int COUT, int KC, int HALO, int MODE>
// 2 + 4 x EP warps: 14 (at most 4 per SM sub-partition, up to 128 registers each) or 18
// (up to 96 registers each).  MODE: the epilogue's layer shape (Lay).
__global__ void __launch_bounds__((Cfg<KIND, NB, CIN, COUT, KC, HALO>::THREADS), 1)
    conv_tc_kernel(const __grid_constant__ TcMaps maps, TcConvArgs a) {
  using K = Cfg<KIND, NB, CIN, COUT, KC, HALO, MODE>;
  constexpr int EP = K::EP;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)K::STAGES * K::STAGE);
  uint64_t* empty = full + K::STAGES;
  uint64_t* tfull = empty + K::STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  // the LayerNorm-moment scratch: its own block, or (staged) inside the warps' box regions
  float* scr_all = reinterpret_cast<float*>(smem + (K::STAGED ? K::STG_OFF : (size_t)K::STAGES * K::STAGE + 256));
  float* par = reinterpret_cast<float*>(smem + (size_t)K::STAGES * K::STAGE + 256 + K::SCR);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // The pair computes tiles 2u and 2u + 1 of every pair-unit u it owns: this CTA (rank 0 or 1)
  // the one of its rank.  Both CTAs walk the same units; a tile past the last one (odd tile
  // counts) computes on zero-filled operands and stores nothing.
  const uint32_t rank = tc::cluster_ctarank();
  const int pair = (int)(blockIdx.x >> 1), n_pairs = (int)(gridDim.x >> 1);
  const int pair_units = (a.n_tiles + 1) / 2 * K::NG;
  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < K::STAGES; ++s) {
        tc::mbar_init(&full[s], 1);    // the first CTA's producer; both CTAs' TMA bytes
        tc::mbar_init(&empty[s], 1);   // the pair's MMA commit
      }
      for (int i = 0; i < 2; ++i) {
        tc::mbar_init(&tfull[i], 1);
        tc::mbar_init(&tempty[i], 2 * K::EPI_WARPS);   // both CTAs' epilogue warps
      }
      tc::fence_mbar_init();
      for (int b = 0; b < NB; ++b) {
        tc::prefetch_tmap(&maps.a[b]);
        tc::prefetch_tmap(&maps.w[b]);
      }
    }
    __syncwarp();
    tc::tmem_alloc_pair(tmem_slot, K::TMEM_COLS);
  } else if (warp >= 2) {
    stage_params<KIND, NB, COUT>(a, par, threadIdx.x - 64, K::THREADS - 64);
  }
  tc::fence_before_sync();
  tc::cluster_sync();   // both CTAs' barriers are initialised before any remote signal
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_slot;
  int* err = a.err;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer (each CTA)
    const uint32_t full0 = tc::mapa(tc::smem_u32(&full[0]), 0);   // the first CTA's full barriers
    int s = 0;
    uint32_t ph = 0;
    uint32_t last_par[8];
    bool used[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) used[i] = false;
    bool ok = true;
    for (int unit = pair * K::NG; ok && unit < pair_units;
         unit += (K::NG == 1 || unit % K::NG == K::NG - 1) ? n_pairs * K::NG - (K::NG - 1) : 1) {
      const int tile = 2 * (unit / K::NG) + (int)rank, g0 = (unit % K::NG) * K::G;   // tile and branch group
      int slot, t, fb;
      decode_tile(tile, a.T, a.nfb, slot, t, fb);
      for (int k = 0; k < K::K_ITERS; ++k) {
        if (!tc::mbar_wait(&empty[s], ph ^ 1u, err, 1)) {
          ok = false;
          break;
        }
        if (rank == 0) tc::mbar_arrive_expect_tx(&full[s], 2 * K::STAGE_TX);
        const uint32_t fb_s = full0 + (uint32_t)(s * sizeof(uint64_t));
        // halo stage: symbol row t + dt, subcarriers from one before the tile, taps
        // (dt, -1..1); else one tap (dt, df) with the tile's rows shifted by df; a 1x1 conv
        // reads the tile's own rows and its single weight tap
        const int grp = k / (CIN / KC), ch = (k % (CIN / KC)) * KC;
        const int dt = HALO == 1 ? grp - 1 : HALO == 2 ? 0 : grp / 3 - 1;
        const int f0 = HALO == 1 ? fb * TILE_M - 1 : HALO == 2 ? fb * TILE_M : fb * TILE_M + grp % 3 - 1;
        const int tap0 = HALO == 1 ? 3 * grp : HALO == 2 ? 0 : grp;
        const int r0 = (int)rank * K::B_ROWS;   // this CTA's half of the output channels
        uint8_t* st = smem + (size_t)s * K::STAGE;
#pragma unroll
        for (int i = 0; i < K::G; ++i) {
          const int b = g0 + i;
          uint8_t* ab = st + i * K::A_BYTES;
          uint8_t* bb = st + K::G * K::A_BYTES + i * K::B_BYTES;
          tc::tma_load_4d_pair(ab, &maps.a[b], fb_s, ch, f0, t + dt, slot);
          if constexpr (K::NSPLIT == 2) tc::tma_load_4d_pair(ab + K::A_PART, &maps.a_lo[b], fb_s, ch, f0, t + dt, slot);
          tc::tma_load_3d_pair(bb, &maps.w[b], fb_s, ch, r0, tap0);
          if constexpr (K::NSPLIT == 2) tc::tma_load_3d_pair(bb + K::B_PART, &maps.w_lo[b], fb_s, ch, r0, tap0);
        }
        used[s] = true;
        last_par[s] = ph;
        if (++s == K::STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    // drain: the pair's MMAs have released every stage this CTA filled (so every load into
    // it has landed and been read, and every commit to it has arrived) before it may exit
    for (int i = 0; i < K::STAGES; ++i)
      if (used[i]) tc::mbar_wait(&empty[i], last_par[i], err, 9);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------ MMA issuer (first CTA)
    int s = 0;
    uint32_t ph = 0;
    int it = 0;
    bool ok = true;
    for (int unit = pair * K::NG; ok && unit < pair_units;
         unit += (K::NG == 1 || unit % K::NG == K::NG - 1) ? n_pairs * K::NG - (K::NG - 1) : 1, ++it) {
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
              const uint32_t ba = st + K::G * K::A_BYTES + b * K::B_BYTES + d * K::B_ROWS * K::ROW + 32 * j;
              const uint64_t ad = tc::smem_desc(aa, K::ROW);
              const uint64_t bd = tc::smem_desc(ba, K::ROW);
              tc::mma_pair<KIND>(dcol + (uint32_t)(b * COUT), ad, bd, K::IDESC, (k | d | j) != 0);
              if constexpr (K::NSPLIT == 2) {
                // FP32-accurate product from TF32 parts: hi*hi + hi*lo + lo*hi
                tc::mma_pair<KIND>(dcol + (uint32_t)(b * COUT), ad, tc::smem_desc(ba + K::B_PART, K::ROW), K::IDESC,
                                   1u);
                tc::mma_pair<KIND>(dcol + (uint32_t)(b * COUT), tc::smem_desc(aa + K::A_PART, K::ROW), bd, K::IDESC,
                                   1u);
              }
            }
          }
        }
        tc::mma_commit_pair(&empty[s]);   // the stage is free again in both CTAs
        if (++s == K::STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
      tc::mma_commit_pair(&tfull[acc]);     // both CTAs' accumulators are complete
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ fused epilogue (each CTA)
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int part = (warp - 2) / 4;        // which share of the channels this warp handles
    const int row = 32 * q + lane;
    const bool prefetcher = warp == 2 && lane == 0;
    // the first CTA's tempty barriers, where both CTAs' epilogue warps report a drained set
    const uint32_t tempty0 = tc::mapa(tc::smem_u32(&tempty[0]), 0);
    if (prefetcher) prefetch_resid<K::G, COUT>(a, 2 * pair + (int)rank, 0);
    int it = 0;
    for (int unit = pair * K::NG; unit < pair_units;
         unit += (K::NG == 1 || unit % K::NG == K::NG - 1) ? n_pairs * K::NG - (K::NG - 1) : 1, ++it) {
      const int tile = 2 * (unit / K::NG) + (int)rank, g = unit % K::NG;
      const int acc = it % K::N_ACC;
      const uint32_t aph = (uint32_t)(it / K::N_ACC) & 1u;
      if (prefetcher) {
        if (g + 1 < K::NG)
          prefetch_resid<K::G, COUT>(a, tile, (g + 1) * K::G);
        else
          prefetch_resid<K::G, COUT>(a, tile + 2 * n_pairs, 0);
      }
      const bool got = tc::mbar_wait(&tfull[acc], aph, err, 4);
      if (!barrier_all(1 + q, 32 * EP, got)) break;
      tc::fence_after_sync();
      int slot, t, fb;
      decode_tile(tile, a.T, a.nfb, slot, t, fb);
      const int f = fb * TILE_M + row;
      const bool valid = tile < a.n_tiles && f < a.F;
      const long long m = ((long long)slot * a.T + t) * a.F + f;
      const uint32_t lanes = (uint32_t)(32 * q) << 16;
      const uint32_t tacc = tbase + (uint32_t)(acc * K::COLS) + lanes;
      StoreBox sb = {};
      if constexpr (K::STAGED) {
        sb.xs = smem + K::STG_OFF + (size_t)(warp - 2) * K::REG_B;
        sb.nx = sb.xs + K::XS_B;
        sb.xs_map = maps.xs;
        sb.nx_map = maps.nx;
        sb.c0 = part * K::PW;
        sb.f0 = fb * TILE_M + 32 * q;
        sb.st = slot * a.T + t;
        sb.ok = tile < a.n_tiles && sb.f0 < a.F;
      }
      constexpr int PW = K::STAGED ? K::PW : 0;
      if constexpr (K::NG == 1)
        tc_epilogue<KIND, NB, COUT, EP, MODE, PW, K::SCR_STRIDE>(a, par, tacc, valid, m, part, q, lane, scr_all, sb);
      else
        tc_epilogue_group<KIND, NB, COUT, K::G, EP, MODE, PW, K::SCR_STRIDE>(
            a, par, tacc, tbase + (uint32_t)K::STASH + lanes, g, valid, m, part, q, lane, scr_all, sb);
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive_cluster(tempty0 + (uint32_t)(acc * sizeof(uint64_t)));
    }
    // the staged stores have written global memory and read the boxes before the CTA ends
    if constexpr (K::STAGED)
      if (lane == 0) tc::bulk_wait_all();
  }
  // neither CTA deallocates or leaves while the pair may still read its shared memory or
  // TMEM or signal its barriers
  tc::fence_before_sync();
  __syncthreads();
  tc::cluster_sync();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc_pair(tbase, K::TMEM_COLS);
  }
}

template <int KIND, int NB, int CIN, int COUT, int KC, int HALO, int MODE>
int launch_tc_t(const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  using K = Cfg<KIND, NB, CIN, COUT, KC, HALO, MODE>;
  auto* kern = conv_tc_kernel<KIND, NB, CIN, COUT, KC, HALO, MODE>;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(K::THREADS);
  cfg.dynamicSmemBytes = K::SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // persistent grid: as many CTA pairs as can be resident at once (one CTA per SM)
  static int max_pairs = 0;
  if (!max_pairs) {
    CONET_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM));
    int dev = 0, n_sm = 0, n_cl = 0;
    CONET_CUDA(cudaGetDevice(&dev));
    CONET_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    cfg.gridDim = dim3((unsigned)(n_sm / 2 * 2));
    CONET_CUDA(cudaOccupancyMaxActiveClusters(&n_cl, kern, &cfg));
    if (n_cl < 1) return fail(CONET_ERR_CUDA, "conv_tc_kernel: no CTA pair fits an SM pair");
    max_pairs = n_cl < n_sm / 2 ? n_cl : n_sm / 2;
  }
  const int want = (a.n_tiles + 1) / 2;
  cfg.gridDim = dim3((unsigned)(2 * (want < max_pairs ? want : max_pairs)));
  CONET_CUDA(cudaLaunchKernelEx(&cfg, kern, maps, a));
  return check_launch("conv_tc_kernel");
}

// Whether the fast fused epilogue (conv2_part) serves a shape: equal 16- or 32-channel parts,
// staged stores, and room for the product (a branch-group stash, or spare accumulator columns).
__host__ __device__ constexpr bool fast_fused(int kind, int nb, int cin, int cout) {
  return staged_ok(kind, nb, cin, cout) &&
         (part_width(kind, nb, cout) == 16 || part_width(kind, nb, cout) == 32) &&
         (tc_groups(kind, nb, cout) > 1 || pow2_ceil(nb * cout) >= nb * cout + cout);
}

// The compile-time layer shape (Lay) that a launch's arguments match, 0 if none.
int tc_mode(int kind, int nb, int cin, int cout, const TcConvArgs& a) {
  if (a.measure || nb < 2 || a.op || a.feedback) return 0;
  if (a.head_w) {
    // the last conv2 of a fused residual network, at inference, where the fast epilogue runs
    bool m4 = a.pre == 0 && a.fuse && a.lnf_g && a.llr && cin == cout && fast_fused(kind, nb, cin, cout);
    for (int b = 0; b < nb; ++b)
      m4 = m4 && a.resid[b] && !a.nx_out[b] && !a.t_out[b] && !a.a_out[b] && !a.amax[b];
    return m4 ? 4 : 0;
  }
  bool m1 = a.pre == 2 && !a.fuse, m2 = a.pre == 0 && a.fuse && a.lnf_g, m3 = a.pre == 1 && a.fuse && a.lnf_g;
  for (int b = 0; b < nb; ++b) {
    if (a.t_out[b] || a.a_out[b] || !a.nx_out[b] || a.amax[b]) return 0;
    if (kind == 1 && !a.nx_lo[b]) return 0;
    if (kind == 2 && !a.qinv[b]) return 0;
    m1 = m1 && !a.resid[b] && a.post[b] == 0 && !a.xs_out[b];
    const bool fused_out = a.post[b] == (b == 0 ? 1 : 2) && a.xs_out[b] && (b == 0 || (a.ln1_g[b] && a.ln1_b[b]));
    m2 = m2 && a.resid[b] && fused_out;
    m3 = m3 && !a.resid[b] && fused_out;
  }
  return m1 ? 1 : m2 ? 2 : m3 ? 3 : 0;
}

}  // namespace

// Launch of one instantiated shape (used by the per-type dispatchers below): every shape
// with its run-time epilogue (Lay<0>); the body convs of residual networks (Cin = Cout, two
// or more branches) also with the two fixed residual-block shapes (measured: 14x624 E4M3
// +13 %, BF16 +1 %, split TF32 +2 %; 14x3276 E4M3 +22 %, BF16 +1 %), and the input layers
// of the 3- and 4-branch residual networks with the fixed input-layer shape.
#define TC_CASE(KI, NBV, CI, CO)                                                                                  \
  if (kind == KI && nb == NBV && cin == CI && cout == CO) {                                                        \
    constexpr int KC_ = tc_kc(KI, NBV, CI, CO), HALO_ = tc_halo(KI, NBV, CI, CO);                                  \
    constexpr bool BODY_ = CI == CO && NBV >= 2, INPUT_ = CI != CO && NBV >= 3;                                    \
    if (BODY_ && mode == 1) return launch_tc_t<KI, NBV, CI, CO, KC_, HALO_, BODY_ ? 1 : 0>(maps, a, s);            \
    if (BODY_ && mode == 2) return launch_tc_t<KI, NBV, CI, CO, KC_, HALO_, BODY_ ? 2 : 0>(maps, a, s);            \
    if (BODY_ && mode == 4) return launch_tc_t<KI, NBV, CI, CO, KC_, HALO_, BODY_ ? 4 : 0>(maps, a, s);            \
    if (INPUT_ && mode == 3) return launch_tc_t<KI, NBV, CI, CO, KC_, HALO_, INPUT_ ? 3 : 0>(maps, a, s);          \
    return launch_tc_t<KI, NBV, CI, CO, KC_, HALO_, 0>(maps, a, s);                                                \
  }

// The 1x1 conv (C -> C) of a depthwise-separable residual block of NBV branches: the body
// conv's layer shapes with the pointwise stage (HALO = 2).
#define TC_PW_CASE(KI, NBV, C)                                                                                    \
  if (kind == KI && nb == NBV && cin == C && cout == C) {                                                          \
    constexpr int KC_ = tc_plan(KI, NBV, C, C, false);                                                             \
    if (mode == 1) return launch_tc_t<KI, NBV, C, C, KC_, 2, 1>(maps, a, s);                                        \
    if (mode == 2) return launch_tc_t<KI, NBV, C, C, KC_, 2, 2>(maps, a, s);                                        \
    if (mode == 4) return launch_tc_t<KI, NBV, C, C, KC_, 2, 4>(maps, a, s);                                        \
    return launch_tc_t<KI, NBV, C, C, KC_, 2, 0>(maps, a, s);                                                      \
  }

// Dispatchers of the instantiated shapes of one operand type (conv_tc_<type>.cu); mode is
// tc_mode's classification.  CONET_ERR_UNSUPPORTED for a shape that is not instantiated.
int launch_conv_tc_bf16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s);
int launch_conv_tc_fp16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s);
int launch_conv_tc_tf32(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s);
int launch_conv_tc_e4m3(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s);
// the 1x1 convs of depthwise-separable blocks (conv_tc_pw_<type>.cu)
int launch_conv_tc_pw_bf16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a,
                           cudaStream_t s);
int launch_conv_tc_pw_fp16(int nb, int cin, int cout, int mode, const TcMaps& maps, const TcConvArgs& a,
                           cudaStream_t s);

}  // namespace conet
