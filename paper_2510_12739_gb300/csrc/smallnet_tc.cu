// Whole-network kernel for the small plain CoNets (the 14 x 72 class: 2 branches of 32
// channels, plain conv + ReLU layers with Hadamard fusion, Sec. III Fig. "Example I"), BF16
// or E4M3 operands on the tensor cores, FP32 accumulation.
//
// Layer by layer, these networks are launch- and L2-bound: a slot's 1008 REs x 64 channels
// are a few hundred KB per layer, so every layer launch pays a ramp and a round trip to L2.
// Here one persistent CTA per SM takes whole slots and keeps every layer's activations in
// shared memory:
//   * each branch's activations live in a padded grid of (T + 2) x (F + 1) rows of 32
//     channels (BF16: 64 bytes, 64-byte swizzle; E4M3: 32 bytes, 32-byte swizzle), zero
//     outside the slot: row P(t, f) = (t + 1)
//     (F + 1) + (f + 1) for t in -1..T, f in -1..F-1.  The column f = -1 of row t + 1 is also
//     the right-hand neighbour of f = F - 1 of row t, so one zero column pads both sides;
//   * a 3x3 tap (dt, df) of every output row P is then the same grid at row P + dt (F + 1) +
//     df: one MMA operand descriptor per tap, shifted by whole rows;
//   * all T (F + 1) output rows (F + 1 <= 1024 / T) are 8 tiles of 128 rows, whose
//     accumulators for both branches fill TMEM exactly (8 x 64 columns);
//   * per layer, warp 1 issues M = 128, N = 32 MMAs (2 branches x 8 tiles x 9 taps x K steps)
//     and commits; eight epilogue warps then dequantise (E4M3: the input scale times the
//     output channel's weight scale), add the bias, apply ReLU, form the Hadamard product (and
//     its LayerNorm when the network has one) and write the next layer's inputs back into the
//     grids (E4M3 of value / the next input's scale), zero at padding rows, or, after the last
//     layer, the 1x1 head's LLRs to global memory;
//   * warp 0 TMA-loads the next layer's weights while the epilogue runs, and the next slot's
//     input grid once the first layer has read it: the assembled input (BF16 x 16 or E4M3 x 32
//     channels: 32-byte rows), repacked in global memory into the same padded row order (zero
//     at the padding), comes in as 256-row boxes that land on 8 KB boundaries.
// Calls of few slots split a slot over a cluster of S = 2, 4 or 8 CTAs (one per SM), CTA r
// computing tiles [r 8/S, (r + 1) 8/S) of every layer.  A tile's taps reach W + 1 <= 128 rows
// beyond it, so each CTA writes the first and last W + 1 rows of its outputs also into its
// neighbours' grids (distributed shared memory).  Per layer, a CTA writes into a neighbour
// only after the neighbour's MMAs of that layer are complete (`ndone`, signalled remotely),
// and a CTA's next-layer MMAs start only after both neighbours' writes (`hfull`, release /
// acquire at cluster scope, with an async-proxy fence on the writing side).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace conet {
namespace {

constexpr int SN_C = 32;             // channels per branch
constexpr int SN_NB = 2;             // branches
constexpr int SN_XROW = 32;          // input-grid row bytes (16 BF16 or 32 E4M3 channels)
constexpr int SN_TILES = 8;          // 128-row output tiles (8 x 2 x 32 = 512 TMEM columns)
constexpr int SN_G = 1;              // guard row before a branch grid (tap (-1, -1) of the first row)
constexpr int SN_GX = 8;             // guard rows before the input grid (keeps its TMA boxes 256-byte aligned)
constexpr int SN_XBOX = 256;         // input-grid rows per TMA box
constexpr int SN_THREADS = 320;      // TMA warp, MMA warp, 8 epilogue warps
// Operand geometry per kind (0 = BF16 kind::f16, 2 = E4M3 kind::f8f6f4)
template <int KIND>
struct SnK {
  static constexpr int ARow = KIND == 2 ? 32 : 64;                       // branch-grid row bytes
  __host__ __device__ static constexpr int w_row(int l) { return KIND == 2 ? 32 : (l == 0 ? 32 : 64); }
  __host__ __device__ static constexpr int ksteps(int l) { return KIND == 2 ? 1 : (l == 0 ? 1 : 2); }
  static constexpr uint32_t IDESC = tc::instr_desc(KIND == 2 ? 0 : 1, SN_C, 128);
};

struct SnMaps {
  CUtensorMap x0;                          // padded input [slots][(T + 2)(F + 1)][32 B], box {row, 256, 1}
  CUtensorMap w[SN_MAX_LAYERS][SN_NB];     // [9][32][Cin] per layer and branch, box {Cin, 32, 9}
};

// Shared-memory layout (byte offsets from the 1 KB aligned base), chosen on the host.
struct SnLayout {
  int rows;                                // grid rows incl. guards
  int a_off[SN_NB], x_off, w_off, bar_off, bytes;
};

__host__ __device__ inline SnLayout sn_layout(int T, int F, int a_row) {
  SnLayout L;
  const int W = F + 1;
  // rows the MMAs read: the 8 output tiles from P(0, -1), each tap up to W + 1 rows away
  const int span = W + SN_TILES * 128 + W + 2;
  const int grid_rows = (T + 2) * W + 8 > span ? (T + 2) * W + 8 : span;
  L.rows = (SN_G + grid_rows + 7) / 8 * 8;
  int o = 0;
  for (int b = 0; b < SN_NB; ++b) {
    L.a_off[b] = o;
    o += (L.rows * a_row + 1023) / 1024 * 1024;
  }
  L.x_off = o;
  const int xboxed = ((T + 2) * W + SN_XBOX - 1) / SN_XBOX * SN_XBOX;
  const int xrows = SN_GX + (xboxed > span ? xboxed : span);
  o += (xrows * SN_XROW + 1023) / 1024 * 1024;
  L.w_off = o;
  o += SN_NB * 9 * SN_C * a_row;
  L.bar_off = o;
  o += 256;
  L.bytes = o;
  return L;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- cluster-split slots: distributed shared memory and cluster-scope barriers
// generic-proxy writes to any CTA's shared memory become visible to the async proxy
__device__ __forceinline__ void fence_proxy_async_cluster() {
  asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}
// 16 bytes into shared::cluster address caddr (this CTA's or another of the cluster)
__device__ __forceinline__ void st_cluster16(uint32_t caddr, uint4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(caddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
// arrive on another CTA's mbarrier, releasing this thread's prior writes at cluster scope
__device__ __forceinline__ void mbar_arrive_release_cluster(uint32_t caddr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
// bounded wait on this CTA's mbarrier with cluster-scope acquire (records `where` on timeout)
__device__ __forceinline__ bool mbar_wait_acq_cluster(uint64_t* bar, uint32_t parity, int* err, int where) {
  const uint64_t t0 = tc::globaltimer_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::smem_u32(bar)), "r"(parity), "r"(tc::WAIT_HINT_NS)
        : "memory");
    if (ok) return true;
    if (tc::globaltimer_ns() - t0 > tc::WAIT_NS) break;
  }
  atomicCAS(err, 0, where);
  return false;
}

template <int KIND, int S>
__global__ void __launch_bounds__(SN_THREADS, 1) smallnet_kernel(const __grid_constant__ SnMaps maps, SmallNetArgs a) {
  using K = SnK<KIND>;
  constexpr int TPC = SN_TILES / S;          // output tiles per CTA
  constexpr uint32_t TCOLS = TPC * SN_NB * SN_C;   // TMEM columns (a power of two >= 64)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const SnLayout L = sn_layout(a.T, a.F, K::ARow);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* xfull = bars + 0;    // the slot's input grid landed (TMA bytes)
  uint64_t* xempty = bars + 1;   // the first layer's MMAs have read it
  uint64_t* wfull = bars + 2;    // the layer's weights landed
  uint64_t* wempty = bars + 3;   // the layer's MMAs have read them
  uint64_t* dfull = bars + 4;    // the layer's accumulators are complete
  uint64_t* afull = bars + 5;    // the epilogue drained TMEM and wrote the next inputs (8 warps)
  uint64_t* ndone = bars + 6;    // (S > 1) the neighbours' MMAs of the layer are complete
  uint64_t* hfull = bars + 7;    // (S > 1) the neighbours' halo rows of the layer's outputs are written
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  uint64_t* dfull_t = bars + 16; // (S = 1) tiles 0 .. t of the layer are complete (one per tile)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = a.T, F = a.F, W = F + 1, D = a.depth;
  const int p0 = W;              // first output row: P(0, -1)
  const int rank = S > 1 ? (int)tc::cluster_ctarank() : 0;
  const int cid = (int)blockIdx.x / S, ncl = (int)gridDim.x / S;   // cluster (slot group) index
  const int nn = (rank > 0 ? 1 : 0) + (rank < S - 1 ? 1 : 0);       // neighbours in the cluster

  // zero both grids and the input grid (their padding rows must read as zero), then init
  for (int i = threadIdx.x; i < (L.w_off) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    if (lane == 0) {
      tc::mbar_init(xfull, 1);
      tc::mbar_init(xempty, 1);
      tc::mbar_init(wfull, 1);
      tc::mbar_init(wempty, 1);
      tc::mbar_init(dfull, 1);
      tc::mbar_init(afull, 8);
      for (int i = 0; i < TPC; ++i) tc::mbar_init(&dfull_t[i], 1);
      tc::mbar_init(ndone, nn > 0 ? nn : 1);
      tc::mbar_init(hfull, nn > 0 ? 8 * nn : 1);
      tc::fence_mbar_init();
      tc::prefetch_tmap(&maps.x0);
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, TCOLS);
  }
  fence_proxy_async_smem();      // the zeroes are visible to TMA and the tensor cores
  tc::fence_before_sync();
  if constexpr (S > 1)
    tc::cluster_sync();          // every CTA's grids are zero and its barriers initialised
  else
    __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_slot;
  int* err = a.err;
  const int n_iter = a.B > cid ? (a.B - 1 - cid) / ncl + 1 : 0;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    bool ok = true;
    for (int it = 0; ok && it < n_iter; ++it) {
      const int slot = cid + it * ncl;
      // the input grid of this slot, once the previous slot's first layer has read the last one
      if (!tc::mbar_wait(xempty, (uint32_t)(it & 1) ^ 1u, err, 31)) break;
      const int nbox = ((T + 2) * W + SN_XBOX - 1) / SN_XBOX;
      tc::mbar_arrive_expect_tx(xfull, (uint32_t)(nbox * SN_XBOX * SN_XROW));
      for (int k = 0; k < nbox; ++k)
        tc::tma_load_3d(smem + L.x_off + (SN_GX + k * SN_XBOX) * SN_XROW, &maps.x0, xfull, 0, k * SN_XBOX, slot);
      for (int l = 0; l < D; ++l) {
        const int g = it * D + l;
        if (!tc::mbar_wait(wempty, (uint32_t)(g & 1) ^ 1u, err, 32)) {
          ok = false;
          break;
        }
        const int wrow = K::w_row(l);
        tc::mbar_arrive_expect_tx(wfull, (uint32_t)(SN_NB * 9 * SN_C * wrow));
        for (int b = 0; b < SN_NB; ++b)
          tc::tma_load_3d(smem + L.w_off + b * 9 * SN_C * wrow, &maps.w[l][b], wfull, 0, 0, 0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    bool ok = true;
    for (int it = 0; ok && it < n_iter; ++it) {
      for (int l = 0; l < D; ++l) {
        const int g = it * D + l;
        if (!tc::mbar_wait(wfull, (uint32_t)(g & 1), err, 33)) {
          ok = false;
          break;
        }
        if (l == 0 && !tc::mbar_wait(xfull, (uint32_t)(it & 1), err, 34)) {
          ok = false;
          break;
        }
        if (g > 0 && !tc::mbar_wait(afull, (uint32_t)((g - 1) & 1), err, 35)) {   // TMEM free, inputs written
          ok = false;
          break;
        }
        // the neighbours' halo rows of this layer's inputs (phases count layers 0 .. D - 2)
        if (S > 1 && l > 0 && !mbar_wait_acq_cluster(hfull, (uint32_t)((it * (D - 1) + l - 1) & 1), err, 37)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        fence_proxy_async_smem();
        const int row_b = l == 0 ? SN_XROW : K::ARow;   // operand row bytes (input grid / branch grids)
        const int ksteps = K::ksteps(l);
        const int guard = l == 0 ? SN_GX : SN_G;
        const uint32_t wsm = tc::smem_u32(smem + L.w_off);
        // tile by tile (one slot per CTA: each tile's completion is signalled, so the epilogue
        // of a tile overlaps the next tiles' MMAs)
        for (int ml = 0; ml < TPC; ++ml) {
          const int mt = rank * TPC + ml;
          for (int b = 0; b < SN_NB; ++b) {
            const uint32_t asm_b = tc::smem_u32(smem + (l == 0 ? L.x_off : L.a_off[b]));
            const uint32_t wb = wsm + (uint32_t)(b * 9 * SN_C * row_b);
            const uint32_t d = tbase + (uint32_t)(ml * SN_NB * SN_C + b * SN_C);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
              const int shift = (tap / 3 - 1) * W + (tap % 3 - 1);
              const uint32_t arow = asm_b + (uint32_t)((guard + p0 + mt * 128 + shift) * row_b);
              for (int j = 0; j < ksteps; ++j) {
                const uint64_t ad = tc::smem_desc(arow + 32 * j, row_b);
                const uint64_t bd = tc::smem_desc(wb + (uint32_t)(tap * SN_C * row_b + 32 * j), row_b);
                tc::mma<KIND>(d, ad, bd, K::IDESC, (tap | j) != 0 ? 1u : 0u);
              }
            }
          }
          if (S == 1) tc::mma_commit(&dfull_t[ml]);
        }
        tc::mma_commit(dfull);
        tc::mma_commit(wempty);
        if (l == 0) tc::mma_commit(xempty);
      }
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue (8 warps)
    const int q = warp & 3;                         // TMEM lane quarter
    const int half = (warp - 2) >> 2;               // local tiles half, 2 * k + half
    // (S > 1) this CTA's output rows, the rows its neighbours read, and their grids' addresses
    const int row0 = p0 + rank * TPC * 128, row1 = row0 + TPC * 128;
    uint32_t nbr_grid[2][SN_NB] = {};
    uint32_t nbr_ndone[2] = {}, nbr_hfull[2] = {};
    if constexpr (S > 1) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int nr = side == 0 ? rank - 1 : rank + 1;
        if (nr < 0 || nr >= S) continue;
#pragma unroll
        for (int b = 0; b < SN_NB; ++b) nbr_grid[side][b] = tc::mapa(tc::smem_u32(smem + L.a_off[b]), (uint32_t)nr);
        nbr_ndone[side] = tc::mapa(tc::smem_u32(ndone), (uint32_t)nr);
        nbr_hfull[side] = tc::mapa(tc::smem_u32(hfull), (uint32_t)nr);
      }
    }
    bool ok = true;
    for (int it = 0; ok && it < n_iter; ++it) {
      const int slot = cid + it * ncl;
      for (int l = 0; l < D; ++l) {
        const int g = it * D + l;
        if (S > 1) {   // (one slot per CTA: per-tile waits below)
          const bool got = tc::mbar_wait(dfull, (uint32_t)(g & 1), err, 36);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
        }
        const bool last = l == D - 1;
        const bool halo = S > 1 && !last;
        if (halo) {
          // this CTA's MMAs of the layer are complete: its neighbours may write into its grids;
          // then wait until theirs are, before writing into theirs
          if (warp == 2 && lane == 0) {
            if (nbr_ndone[0]) mbar_arrive_release_cluster(nbr_ndone[0]);
            if (nbr_ndone[1]) mbar_arrive_release_cluster(nbr_ndone[1]);
          }
          const bool nd = mbar_wait_acq_cluster(ndone, (uint32_t)((it * (D - 1) + l) & 1), err, 38);
          if (!__all_sync(0xffffffffu, nd)) {
            ok = false;
            break;
          }
        }
        for (int ml = half; ml < TPC; ml += 2) {
          const int mt = rank * TPC + ml;
          const int P = p0 + mt * 128 + 32 * q + lane;
          const int t = P / W - 1, f = P % W - 1;
          const bool valid = t >= 0 && t < T && f >= 0 && f < F;
          if (S == 1) {   // this tile's accumulators are complete
            const bool got = tc::mbar_wait(&dfull_t[ml], (uint32_t)(g & 1), err, 36);
            if (!__all_sync(0xffffffffu, got)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
          }
          float x[SN_NB][SN_C];
          {
            uint32_t r[SN_NB][2][16];
            __syncwarp();
#pragma unroll
            for (int b = 0; b < SN_NB; ++b)
#pragma unroll
              for (int h = 0; h < 2; ++h)
                tc::tmem_ld16_nowait(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(ml * SN_NB * SN_C + b * SN_C + 16 * h),
                                     r[b][h]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int b = 0; b < SN_NB; ++b)
#pragma unroll
              for (int c = 0; c < SN_C; ++c) x[b][c] = __uint_as_float(r[b][c >> 4][c & 15]);
          }
#pragma unroll
          for (int b = 0; b < SN_NB; ++b) {
            const float4* bias4 = reinterpret_cast<const float4*>(a.bias[l][b]);
            if constexpr (KIND == 2) {
              const float4* dq4 = reinterpret_cast<const float4*>(a.dq[l][b]);
#pragma unroll
              for (int c = 0; c < SN_C; c += 4) {                                             // dequantise
                const float4 d = __ldg(dq4 + c / 4);
                x[b][c] *= d.x;
                x[b][c + 1] *= d.y;
                x[b][c + 2] *= d.z;
                x[b][c + 3] *= d.w;
              }
            }
#pragma unroll
            for (int c = 0; c < SN_C; c += 4) {                                               // a_b = ReLU(conv + bias)
              const float4 bv = __ldg(bias4 + c / 4);
              x[b][c] = fmaxf(x[b][c] + bv.x, 0.f);
              x[b][c + 1] = fmaxf(x[b][c + 1] + bv.y, 0.f);
              x[b][c + 2] = fmaxf(x[b][c + 2] + bv.z, 0.f);
              x[b][c + 3] = fmaxf(x[b][c + 3] + bv.w, 0.f);
            }
          }
          if (a.fuse[l]) {
#pragma unroll
            for (int c = 0; c < SN_C; ++c) x[0][c] *= x[1][c];                 // Hadamard fusion
            if (a.lnf_g[l]) {
              float mean = 0.f;
#pragma unroll
              for (int c = 0; c < SN_C; ++c) mean += x[0][c];
              mean *= 1.0f / SN_C;
              float var = 0.f;
#pragma unroll
              for (int c = 0; c < SN_C; ++c) var = fmaf(x[0][c] - mean, x[0][c] - mean, var);
              const float rs = rsqrtf(var * (1.0f / SN_C) + 1e-5f);
#pragma unroll
              for (int c = 0; c < SN_C; ++c)
                x[0][c] = (x[0][c] - mean) * rs * __ldg(a.lnf_g[l] + c) + __ldg(a.lnf_b[l] + c);
            }
          }
          if (S == 1 && !last && ml + 1 < TPC) {
            // the next tile's MMAs read this tile's last W + 1 rows: they finish before the
            // rows are overwritten (the previous tile's finished before this tile's)
            const bool got = tc::mbar_wait(&dfull_t[ml + 1], (uint32_t)(g & 1), err, 39);
            if (!__all_sync(0xffffffffu, got)) {
              ok = false;
              break;
            }
          }
          if (!last) {
            // the next layer's inputs into both grids, zero at padding rows.  BF16: 64-byte rows,
            // 64-byte swizzle (16-byte chunk k of row r at chunk k ^ ((r >> 1) & 3)); E4M3 of
            // value / scale: 32-byte rows, 32-byte swizzle (chunk k at k ^ ((r >> 2) & 1))
            const int r = SN_G + P;
#pragma unroll
            for (int b = 0; b < SN_NB; ++b) {
              uint8_t* row = smem + L.a_off[b] + (size_t)r * K::ARow;
              if constexpr (KIND == 2) {
                const float qi = __ldg(a.qinv[l + 1][b]);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                  uint32_t w4[4] = {0u, 0u, 0u, 0u};
                  if (valid) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                      const float* v = &x[b][16 * k + 4 * e];
                      const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[0] * qi, v[1] * qi), __NV_SATFINITE, __NV_E4M3);
                      const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[2] * qi, v[3] * qi), __NV_SATFINITE, __NV_E4M3);
                      w4[e] = (lo & 0xFFFFu) | (hi << 16);
                    }
                  }
                  const int off = r * K::ARow + 16 * (k ^ ((r >> 2) & 1));
                  const uint4 v4 = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                  *reinterpret_cast<uint4*>(row + 16 * (k ^ ((r >> 2) & 1))) = v4;
                  if (halo && P - row0 <= W && nbr_grid[0][b]) st_cluster16(nbr_grid[0][b] + (uint32_t)off, v4);
                  if (halo && row1 - 1 - P <= W && nbr_grid[1][b]) st_cluster16(nbr_grid[1][b] + (uint32_t)off, v4);
                }
              } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  uint32_t w4[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 h2 = valid ? __floats2bfloat162_rn(x[b][8 * k + 2 * e], x[b][8 * k + 2 * e + 1])
                                                    : __floats2bfloat162_rn(0.f, 0.f);
                    w4[e] = *reinterpret_cast<const uint32_t*>(&h2);
                  }
                  const int off = r * K::ARow + 16 * (k ^ ((r >> 1) & 3));
                  const uint4 v4 = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                  *reinterpret_cast<uint4*>(row + 16 * (k ^ ((r >> 1) & 3))) = v4;
                  if (halo && P - row0 <= W && nbr_grid[0][b]) st_cluster16(nbr_grid[0][b] + (uint32_t)off, v4);
                  if (halo && row1 - 1 - P <= W && nbr_grid[1][b]) st_cluster16(nbr_grid[1][b] + (uint32_t)off, v4);
                }
              }
            }
          } else if (valid) {
            // 1x1 head on the fused main activation
            const long long m = ((long long)slot * T + t) * F + f;
            for (int qq = 0; qq < a.Q; ++qq) {
              float s = __ldg(a.head_b + qq);
#pragma unroll
              for (int c = 0; c < SN_C; ++c) s = fmaf(__ldg(a.head_w + qq * SN_C + c), x[0][c], s);
              a.llr[m * a.Q + qq] = s;
              if (!(fabsf(s) <= FLT_MAX)) *a.nonfinite = 1;
            }
          }
        }
        if (!ok) break;
        fence_proxy_async_smem();   // the grids written here are read by the next layer's MMAs
        if (halo) fence_proxy_async_cluster();   // ... and the neighbours' grids, by theirs
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(afull);
          if (halo) {
            if (nbr_hfull[0]) mbar_arrive_release_cluster(nbr_hfull[0]);
            if (nbr_hfull[1]) mbar_arrive_release_cluster(nbr_hfull[1]);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  if constexpr (S > 1)
    tc::cluster_sync();   // no CTA leaves while a neighbour may still write its grids or barriers
  else
    __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, TCOLS);
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

}  // namespace

bool smallnet_eligible(int kind, int T, int F, int nb, int C, int depth, int Q) {
  if (kind != 0 && kind != 2) return false;
  if (nb != SN_NB || C != SN_C || depth < 1 || depth > SN_MAX_LAYERS || Q < 1 || Q > 8) return false;
  if (T < 1 || F < 1 || T * (F + 1) > SN_TILES * 128 || F > 256) return false;
  return (size_t)sn_layout(T, F, kind == 2 ? SnK<2>::ARow : SnK<0>::ARow).bytes + 1024 <= 227 * 1024;
}

size_t smallnet_input_bytes(int slots, int T, int F) { return (size_t)slots * (T + 2) * (F + 1) * SN_XROW; }

// The padded input's 32-byte rows as 32 bytes (E4M3 channels) or 16 BF16.
int make_smallnet_input_map(CUtensorMap* map, int kind, const void* xp, int slots, int T, int F) {
  EncodeFn enc = encoder();
  if (!enc) return fail(CONET_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int e = kind == 2 ? 1 : 2, n = SN_XROW / e;
  const cuuint64_t R = (cuuint64_t)(T + 2) * (F + 1);
  const cuuint64_t dims[3] = {(cuuint64_t)n, R, (cuuint64_t)slots};
  const cuuint64_t strides[2] = {(cuuint64_t)SN_XROW, R * SN_XROW};
  const cuuint32_t box[3] = {(cuuint32_t)n, (cuuint32_t)SN_XBOX, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, kind == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                         const_cast<void*>(xp), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CONET_ERR_CUDA, "whole-network input map encode failed (%d)", (int)r);
  return CONET_OK;
}

// [slots][T][F] rows of 32 bytes (16 BF16 or 32 E4M3 channels) -> the padded row order
// [slots][(T + 2)(F + 1)]; padding rows are never written (the buffer is zeroed once).  One
// thread per RE and 16 bytes.
__global__ void smallnet_pad_kernel(const uint4* __restrict__ x, uint4* __restrict__ xp, int slots, int T, int F) {
  const long long n = (long long)slots * T * F * 2;
  const int W = F + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(i & 1);
    const long long re = i >> 1;
    const int f = (int)(re % F);
    const long long st = re / F;
    const int t = (int)(st % T);
    const long long slot = st / T;
    const long long P = (long long)(t + 1) * W + (f + 1);
    xp[(slot * (T + 2) * W + P) * 2 + h] = x[i];
  }
}

int launch_smallnet_pad(const void* x, void* xp, int slots, int T, int F, cudaStream_t s) {
  smallnet_pad_kernel<<<grid_for((long long)slots * T * F * 2, 256, 152 * 8), 256, 0, s>>>(
      static_cast<const uint4*>(x), static_cast<uint4*>(xp), slots, T, F);
  return check_launch("smallnet_pad_kernel");
}

// Cluster size S for a call of B slots: the largest of 8, 4, 2 whose clusters of the kernel
// can all be resident at once (one slot each), else 1 (one slot per CTA, persistent).  A
// split needs a tile's halo, W + 1 rows, within the neighbouring CTA's tiles.
template <int KIND, int S>
int cluster_capacity(size_t smem) {
  static int cap = -1;
  static size_t cap_smem = 0;
  if (cap < 0 || cap_smem != smem) {
    auto* kern = smallnet_kernel<KIND, S>;
    CONET_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, n_sm = 0, n_cl = 0;
    CONET_CUDA(cudaGetDevice(&dev));
    CONET_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    if (S == 1) {
      n_cl = n_sm;
    } else {
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = S;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(n_sm / S * S));
      cfg.blockDim = dim3(SN_THREADS);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      CONET_CUDA(cudaOccupancyMaxActiveClusters(&n_cl, kern, &cfg));
    }
    cap = n_cl;
    cap_smem = smem;
  }
  return cap;
}

template <int KIND, int S>
int launch_smallnet_s(const SnMaps& maps, const SmallNetArgs& a, size_t smem, int n_cl, cudaStream_t s) {
  auto* kern = smallnet_kernel<KIND, S>;
  const int ncl = a.B < n_cl ? a.B : n_cl;
  if (S == 1) {
    kern<<<ncl, SN_THREADS, smem, s>>>(maps, a);
    return check_launch("smallnet_kernel");
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(S * ncl));
  cfg.blockDim = dim3(SN_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CONET_CUDA(cudaLaunchKernelEx(&cfg, kern, maps, a));
  return check_launch("smallnet_kernel (cluster)");
}

template <int KIND>
int launch_smallnet_t(const SnMaps& maps, const SmallNetArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)sn_layout(a.T, a.F, SnK<KIND>::ARow).bytes + 1024;
  const bool split_ok = a.F + 2 <= 128;   // W + 1 halo rows within one neighbouring tile
  int cap = 0;
  if (split_ok) {
    if ((cap = cluster_capacity<KIND, 8>(smem)) < 0) return CONET_ERR_CUDA;
    if (a.B <= cap) return launch_smallnet_s<KIND, 8>(maps, a, smem, cap, s);
    if ((cap = cluster_capacity<KIND, 4>(smem)) < 0) return CONET_ERR_CUDA;
    if (a.B <= cap) return launch_smallnet_s<KIND, 4>(maps, a, smem, cap, s);
    if ((cap = cluster_capacity<KIND, 2>(smem)) < 0) return CONET_ERR_CUDA;
    if (a.B <= cap) return launch_smallnet_s<KIND, 2>(maps, a, smem, cap, s);
  }
  if ((cap = cluster_capacity<KIND, 1>(smem)) < 0) return CONET_ERR_CUDA;
  return launch_smallnet_s<KIND, 1>(maps, a, smem, cap, s);
}

int launch_smallnet(int kind, const CUtensorMap& x0_map, const CUtensorMap (*w_maps)[2], const SmallNetArgs& a,
                    cudaStream_t s) {
  SnMaps maps;
  maps.x0 = x0_map;
  for (int l = 0; l < a.depth; ++l)
    for (int b = 0; b < SN_NB; ++b) maps.w[l][b] = w_maps[l][b];
  if (kind == 2) return launch_smallnet_t<2>(maps, a, s);
  return launch_smallnet_t<0>(maps, a, s);
}

}  // namespace conet
