// Weight gradient of the 3x3 convs on the tensor cores (BF16 training handles):
//   dW[co][tap][ci] = sum over REs m of g[m][co] x[m + shift(tap)][ci]
// is a GEMM whose reduction runs over the REs.  tcgen05 operands are K-major, so a first
// pass writes BF16 copies of both operands with the REs innermost: the gradient as
// GT[co][slot][t F + f] and the layer input as three copies XT[df][ci][slot][t F + f] =
// x[slot][t][f + df][ci] (zero where f + df leaves the grid), one per subcarrier shift.  The
// symbol shift dt is then a TMA coordinate offset of dt F along the flattened (t, f) axis,
// whose out-of-range rows (t + dt outside the slot) TMA fills with zeros; F is a multiple
// of 8, so every such offset stays on a 16-byte boundary.
//
// Kernel: CTA s of branch b reduces a contiguous range of 64-RE chunks.  Per chunk, warp 0
// TMA-loads the nine shifted [CIN][64] input boxes stacked as the rows [tap][ci] of the A
// operand and the [COUT][64] gradient box as B; warp 1 issues M = 128 x N = COUT x K = 16
// MMAs (FP32 accumulators in TMEM: one [128][COUT] tile per 128 rows of [tap][ci]); after
// the CTA's last chunk, four epilogue warps copy the accumulators into the CTA's split
// partial in the layout [tap][ci][co], which a fixed-order reduction over the splits turns
// into the master [co][3][3][ci] gradient (deterministic).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace conet {
namespace {

constexpr int WK = 64;                 // REs per chunk (K per stage): one 128-byte BF16 row
constexpr int WG_THREADS = 192;        // TMA warp, MMA warp, 4 epilogue warps

template <int CIN, int COUT>
struct WCfg {
  static_assert(CIN % 8 == 0 && COUT % 16 == 0 && COUT <= 128, "wgrad tile");
  static constexpr int ROWS = 9 * CIN;                         // [tap][ci] rows of A
  static constexpr int NMT = (ROWS + 127) / 128;               // M tiles
  static constexpr int A_BYTES = NMT * 128 * 128;
  static constexpr int B_BYTES = COUT * 128;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int TX = ROWS * 128 + B_BYTES;              // bytes TMA delivers per stage
  static constexpr int STAGES_FIT = (int)((227 * 1024 - 1024 - 256) / STAGE);
  static constexpr int STAGES = STAGES_FIT > 4 ? 4 : STAGES_FIT;
  static_assert(STAGES >= 2, "wgrad stages");
  static constexpr int COLS = NMT * COUT;
  static constexpr int TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static_assert(COLS <= 512, "wgrad TMEM");
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
  static constexpr uint32_t IDESC = tc::instr_desc(1, COUT, 128);   // BF16 x BF16 -> FP32
};

struct WgMaps {
  CUtensorMap xt[MAX_BR][3];   // XT[df] of each branch: dims {T F, slots, CIN}, box {64, 1, CIN}
  CUtensorMap gt[MAX_BR];      // GT of each branch: dims {T F, slots, COUT}, box {64, 1, COUT}
};

struct WgTcArgs {
  float* part;                 // [S][n_br][9 CIN][COUT]
  int* err;
  int S, n_br, slots, T, F;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS, 1) wgrad_tc_kernel(const __grid_constant__ WgMaps maps, WgTcArgs a) {
  using K = WCfg<CIN, COUT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)K::STAGES * K::STAGE);
  uint64_t* empty = full + K::STAGES;
  uint64_t* done = empty + K::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s_id = blockIdx.x, b = blockIdx.y;
  const int TF = a.T * a.F;
  const int nmc = (TF + WK - 1) / WK;                 // chunks per slot
  const long long total = (long long)a.slots * nmc;
  const long long per = (total + a.S - 1) / a.S;
  const long long c0 = (long long)s_id * per, c1 = c0 + per < total ? c0 + per : total;
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < K::STAGES; ++i) {
        tc::mbar_init(&full[i], 1);
        tc::mbar_init(&empty[i], 1);
      }
      tc::mbar_init(done, 1);
      tc::fence_mbar_init();
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, K::TMEM_COLS);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tmem_slot;
  int* err = a.err;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    int s = 0;
    uint32_t ph = 0;
    for (long long c = c0; c < c1; ++c) {
      if (!tc::mbar_wait(&empty[s], ph ^ 1u, err, 21)) break;
      tc::mbar_arrive_expect_tx(&full[s], K::TX);
      const int slot = (int)(c / nmc), m0 = (int)(c % nmc) * WK;
      uint8_t* st = smem + (size_t)s * K::STAGE;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dt = tap / 3 - 1, df = tap % 3 - 1;
        tc::tma_load_3d(st + tap * CIN * 128, &maps.xt[b][df + 1], &full[s], m0 + dt * a.F, slot, 0);
      }
      tc::tma_load_3d(st + K::A_BYTES, &maps.gt[b], &full[s], m0, slot, 0);
      if (++s == K::STAGES) {
        s = 0;
        ph ^= 1u;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (long long c = c0; c < c1; ++c) {
      if (!tc::mbar_wait(&full[s], ph, err, 22)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t st = tc::smem_u32(smem + (size_t)s * K::STAGE);
#pragma unroll
      for (int mt = 0; mt < K::NMT; ++mt) {
#pragma unroll
        for (int j = 0; j < WK / 16; ++j) {
          const uint64_t ad = tc::smem_desc(st + mt * 128 * 128 + 32 * j, 128);
          const uint64_t bd = tc::smem_desc(st + K::A_BYTES + 32 * j, 128);
          tc::mma<0>(tbase + (uint32_t)(mt * COUT), ad, bd, K::IDESC, (c != c0 || j != 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&empty[s]);
      if (++s == K::STAGES) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (ok && c1 > c0) tc::mma_commit(done);
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue: partials
    const int q = warp & 3;
    const bool have = c1 > c0;
    bool got = true;
    if (have) {
      got = tc::mbar_wait(done, 0u, err, 23);
      tc::fence_after_sync();
    }
    float* out = a.part + ((size_t)s_id * a.n_br + b) * (size_t)K::ROWS * COUT;
#pragma unroll
    for (int mt = 0; mt < K::NMT; ++mt) {
      const int r = mt * 128 + 32 * q + lane;
#pragma unroll
      for (int c = 0; c < COUT; c += 16) {
        float v[16];
        if (have && got) {
          tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(mt * COUT + c), v);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if (r < K::ROWS) {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4*>(out + (size_t)r * COUT + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
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

// x [M][x_ld] FP32 (channels cin_src used, CIN written with zero padding), g [M][COUT] FP32 ->
// XT[3][CIN][slots][ld] and GT[COUT][slots][ld] BF16 (ld >= T F).  One CTA per 64 consecutive
// REs of one slot's flattened (t, f) axis: it stages the 66 input rows around them (one RE of
// halo on each side for the subcarrier shifts) and their 64 gradient rows in shared memory with
// coalesced row reads, then writes every channel's 64 REs as one contiguous 128-byte run of each
// output plane.
constexpr int OP_MAXC = 64;

struct WgOpArgs {
  const float* x;
  const float* g;
  __nv_bfloat16* xt;
  __nv_bfloat16* gt;
  int x_ld, cin_src, cin, cout, slots, T, F, ld;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(256) wgrad_operands_kernel(WgOpArgs a) {
  static_assert(CIN % 4 == 0 && COUT % 4 == 0 && CIN <= OP_MAXC && COUT <= OP_MAXC, "operand tile");
  __shared__ float xs[WK + 2][CIN + 1];
  __shared__ float gs[WK][COUT + 1];
  const int TF = a.T * a.F;
  const int nmc = (TF + WK - 1) / WK;
  const int slot = blockIdx.x / nmc, m0 = (blockIdx.x % nmc) * WK;
  const long long base = (long long)slot * TF;
  // stage rows m0 - 1 .. m0 + WK of x (inside the slot) and m0 .. m0 + WK - 1 of g, four
  // channels per thread per step
  for (int i = threadIdx.x; i < (WK + 2) * (CIN / 4); i += blockDim.x) {
    const int r = i / (CIN / 4), c = 4 * (i % (CIN / 4)), m = m0 - 1 + r;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (m >= 0 && m < TF) {
      const float* src = a.x + (base + m) * a.x_ld + c;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = c + k < a.cin_src ? src[k] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) xs[r][c + k] = v[k];
  }
  for (int i = threadIdx.x; i < WK * (COUT / 4); i += blockDim.x) {
    const int r = i / (COUT / 4), c = 4 * (i % (COUT / 4)), m = m0 + r;
    const float4 v = m < TF ? *reinterpret_cast<const float4*>(a.g + (base + m) * COUT + c) : make_float4(0, 0, 0, 0);
    gs[r][c] = v.x;
    gs[r][c + 1] = v.y;
    gs[r][c + 2] = v.z;
    gs[r][c + 3] = v.w;
  }
  __syncthreads();
  const size_t plane = (size_t)a.slots * a.ld;
  const size_t col0 = (size_t)slot * a.ld + m0;
  const int n = m0 + WK <= TF ? WK : TF - m0;           // REs of this chunk inside the slot
  // one warp per output row (df, c): each lane writes two consecutive REs (4 bytes), so a
  // warp stores the row's 64 REs as one 128-byte run
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = 2 * lane;
  const int f0 = (m0 + r) % a.F, f1 = (m0 + r + 1) % a.F;
  for (int row = warp; row < 3 * CIN + COUT; row += blockDim.x / 32) {
    float v0, v1;
    __nv_bfloat16* dst;
    if (row < 3 * CIN) {
      // XT[df][c][slot][m] = x[m + df] when the shifted subcarrier stays in the symbol, else 0
      const int df = row / CIN - 1, c = row % CIN;
      v0 = (f0 + df >= 0 && f0 + df < a.F) ? xs[r + 1 + df][c] : 0.f;
      v1 = (f1 + df >= 0 && f1 + df < a.F) ? xs[r + 2 + df][c] : 0.f;
      dst = a.xt + (size_t)row * plane + col0 + r;
    } else {
      const int c = row - 3 * CIN;
      v0 = gs[r][c];
      v1 = gs[r + 1][c];
      dst = a.gt + (size_t)c * plane + col0 + r;
    }
    if (r + 1 < n) {
      *reinterpret_cast<__nv_bfloat162*>(dst) = __floats2bfloat162_rn(v0, v1);
    } else if (r < n) {
      dst[0] = __float2bfloat16_rn(v0);
    }
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

// [rows][slots][ld] BF16 plane stack, box {64 REs, 1 slot, rows}, 128-byte swizzle.
int make_plane_map(CUtensorMap* map, const void* base, int rows, int slots, int TF, int ld) {
  EncodeFn enc = encoder();
  if (!enc) return fail(CONET_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t dims[3] = {(cuuint64_t)TF, (cuuint64_t)slots, (cuuint64_t)rows};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)slots * ld * 2};
  const cuuint32_t box[3] = {(cuuint32_t)WK, 1, (cuuint32_t)rows};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CONET_ERR_CUDA, "wgrad tensor map encode failed (%d)", (int)r);
  return CONET_OK;
}

template <int CIN, int COUT>
int launch_wgrad_tc_t(const WgMaps& maps, const WgTcArgs& a, cudaStream_t s) {
  using K = WCfg<CIN, COUT>;
  static bool attr = false;
  if (!attr) {
    CONET_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)K::SMEM));
    attr = true;
  }
  wgrad_tc_kernel<CIN, COUT><<<dim3(a.S, a.n_br), WG_THREADS, K::SMEM, s>>>(maps, a);
  return check_launch("wgrad_tc_kernel");
}

}  // namespace

size_t wgrad_tc_scratch_bytes(long long slots, int T, int F, int cin_max, int cout) {
  const size_t ld = ((size_t)T * F + 7) / 8 * 8;
  return ((size_t)3 * cin_max + cout) * (size_t)slots * ld * sizeof(__nv_bfloat16);
}

int wgrad_tc_splits(long long slots, int T, int F, int n_br) {
  const long long chunks = slots * ((T * F + WK - 1) / WK);
  long long s = 2LL * 152 / n_br;
  if (s > chunks) s = chunks;
  if (s > WG_TILED_MAX_CTAS / n_br) s = WG_TILED_MAX_CTAS / n_br;
  return s < 1 ? 1 : (int)s;
}

bool wgrad_tc_supported(int cin, int cout, int F) {
  const int cinp = (cin + 7) / 8 * 8;
  if (F % 8 != 0 || cinp > OP_MAXC || cout > OP_MAXC) return false;
  if (cout == 32) return cinp == 8 || cinp == 16 || cinp == 32;
  if (cout == 64) return cinp == 8 || cinp == 16 || cinp == 64;
  return false;
}

// Weight and bias-free gradient of one conv layer of every branch on the tensor cores:
// writes the split partials into a.part (wgrad_tc_splits x n_br x 9 CINP x cout floats),
// then the fixed-order reduction into a.dW.  `scratch` holds the BF16 operand copies of one
// branch at a time (wgrad_tc_scratch_bytes).
int launch_wgrad_tc(const WgradArgs& a, int slots, void* scratch, int* err, cudaStream_t s) {
  const int cinp = (a.cin + 7) / 8 * 8;
  if (!wgrad_tc_supported(a.cin, a.cout, a.F)) return fail(CONET_ERR_UNSUPPORTED, "tensor-core wgrad shape");
  const int TF = a.T * a.F;
  const int ld = (TF + 7) / 8 * 8;
  const size_t plane = (size_t)slots * ld;
  const int S = wgrad_tc_splits(slots, a.T, a.F, a.n_br);
  for (int b = 0; b < a.n_br; ++b) {
    // operands of branch b (the scratch holds one branch), then its split partials
    __nv_bfloat16* xt = static_cast<__nv_bfloat16*>(scratch);
    __nv_bfloat16* gt = xt + (size_t)3 * cinp * plane;
    WgOpArgs o = {};
    o.x = a.x[b];
    o.g = a.g[b];
    o.xt = xt;
    o.gt = gt;
    o.x_ld = a.cin;
    o.cin_src = a.cin_src[b];
    o.cin = cinp;
    o.cout = a.cout;
    o.slots = slots;
    o.T = a.T;
    o.F = a.F;
    o.ld = ld;
    const int grid = slots * ((TF + WK - 1) / WK);
    if (cinp == 8 && a.cout == 32) wgrad_operands_kernel<8, 32><<<grid, 256, 0, s>>>(o);
    else if (cinp == 16 && a.cout == 32) wgrad_operands_kernel<16, 32><<<grid, 256, 0, s>>>(o);
    else if (cinp == 32 && a.cout == 32) wgrad_operands_kernel<32, 32><<<grid, 256, 0, s>>>(o);
    else if (cinp == 8 && a.cout == 64) wgrad_operands_kernel<8, 64><<<grid, 256, 0, s>>>(o);
    else if (cinp == 16 && a.cout == 64) wgrad_operands_kernel<16, 64><<<grid, 256, 0, s>>>(o);
    else wgrad_operands_kernel<64, 64><<<grid, 256, 0, s>>>(o);
    CONET_LAUNCHED("wgrad_operands_kernel");
    WgMaps maps = {};
    for (int df = 0; df < 3; ++df)
      CONET_TRY(make_plane_map(&maps.xt[0][df], xt + (size_t)df * cinp * plane, cinp, slots, TF, ld));
    CONET_TRY(make_plane_map(&maps.gt[0], gt, a.cout, slots, TF, ld));
    WgTcArgs t = {};
    t.part = a.part + (size_t)b * S * 9 * cinp * a.cout;
    t.err = err;
    t.S = S;
    t.n_br = 1;
    t.slots = slots;
    t.T = a.T;
    t.F = a.F;
    int rc = CONET_ERR_UNSUPPORTED;
    if (cinp == 8 && a.cout == 32) rc = launch_wgrad_tc_t<8, 32>(maps, t, s);
    else if (cinp == 16 && a.cout == 32) rc = launch_wgrad_tc_t<16, 32>(maps, t, s);
    else if (cinp == 32 && a.cout == 32) rc = launch_wgrad_tc_t<32, 32>(maps, t, s);
    else if (cinp == 8 && a.cout == 64) rc = launch_wgrad_tc_t<8, 64>(maps, t, s);
    else if (cinp == 16 && a.cout == 64) rc = launch_wgrad_tc_t<16, 64>(maps, t, s);
    else if (cinp == 64 && a.cout == 64) rc = launch_wgrad_tc_t<64, 64>(maps, t, s);
    CONET_TRY(rc);
    CONET_TRY(launch_wgrad_reduce(a.part + (size_t)b * S * 9 * cinp * a.cout, S, 1, 0, cinp, a.cout, a.cin_src[b],
                                  a.dW[b], s));
  }
  return CONET_OK;
}

}  // namespace conet
