// Host side of the tensor-core conv: dispatch to the per-operand-type instantiations
// (conv_tc_<type>.cu; the kernel itself is in conv_tc.cuh), the TMA tensor maps of its
// operands, and the weight conversion and E4M3 scale kernels.
#include "conv_tc.cuh"

namespace conet {

int launch_conv_tc(int kind, int nb, int cin, int cout, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s) {
  // the branch-group epilogue forms the fused product in its statistics pass and gives the
  // fused branch 0 no LayerNorm of its own
  if (a.fuse && (a.pre == 2 || (tc_groups(kind, nb, cout) > 1 && a.post[0] == 2)))
    return fail(CONET_ERR_UNSUPPORTED, "fused layer with a LayerNorm pre-activation or a normalised fused branch");
  const int mode = tc_mode(kind, nb, cin, cout, a);
  if (a.taps == 1) {
    if (kind == 0) return launch_conv_tc_pw_bf16(nb, cin, cout, mode, maps, a, s);
    if (kind == 3) return launch_conv_tc_pw_fp16(nb, cin, cout, mode, maps, a, s);
    return fail(CONET_ERR_UNSUPPORTED, "tensor-core 1x1 conv kind %d", kind);
  }
  switch (kind) {
    case 0: return launch_conv_tc_bf16(nb, cin, cout, mode, maps, a, s);
    case 1: return launch_conv_tc_tf32(nb, cin, cout, mode, maps, a, s);
    case 2: return launch_conv_tc_e4m3(nb, cin, cout, mode, maps, a, s);
    case 3: return launch_conv_tc_fp16(nb, cin, cout, mode, maps, a, s);
    default: return fail(CONET_ERR_UNSUPPORTED, "tensor-core conv kind %d", kind);
  }
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

int make_weight_map(CUtensorMap* map, int kind, const void* base, int cin, int cout, int kc, int rows, int taps,
                    int n_taps) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(CONET_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if (taps > n_taps) return fail(CONET_ERR_ARG, "weight box of %d taps over a tensor of %d", taps, n_taps);
  const int e = (kind == 0 || kind == 3) ? 2 : kind == 1 ? 4 : 1;
  const cuuint64_t dims[3] = {(cuuint64_t)cin, (cuuint64_t)cout, (cuuint64_t)n_taps};
  const cuuint64_t strides[2] = {(cuuint64_t)cin * e, (cuuint64_t)cout * cin * e};
  const cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)rows, (cuuint32_t)taps};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, dtype_of(kind), 3, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(kc * e), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CONET_ERR_CUDA, "weight tensor map encode failed (%d)", (int)r);
  return CONET_OK;
}

int tc_branch_groups(int kind, int nb, int cout) { return tc_groups(kind, nb, cout); }

// Channels per K chunk and taps per stage of the instantiation for (kind, nb, cin, cout).
int tc_chunk(int kind, int nb, int cin, int cout) { return tc_kc(kind, nb, cin, cout); }
int tc_chunk_pw(int kind, int nb, int c) { return tc_plan(kind, nb, c, c, false); }
int tc_taps(int kind, int nb, int cin, int cout) { return tc_halo(kind, nb, cin, cout) ? 3 : 1; }
int tc_wbox_rows(int kind, int nb, int cin, int cout) { return cout / 2; }   // one CTA's half of a pair's B
int tc_wbox_taps(int kind, int nb, int cin, int cout) { return tc_taps(kind, nb, cin, cout); }
int tc_store_cols(int kind, int nb, int cin, int cout) {
  return staged_ok(kind, nb, cin, cout) ? part_width(kind, nb, cout) : 0;
}

int make_out_map(CUtensorMap* map, int out_kind, void* base, int C, int F, int symbols, int cols) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(CONET_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int e = out_kind < 0 ? 4 : elt_of(out_kind);
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)F, (cuuint64_t)symbols};
  const cuuint64_t strides[2] = {(cuuint64_t)C * e, (cuuint64_t)F * C * e};
  const cuuint32_t box[3] = {(cuuint32_t)cols, 32, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const int rb = cols * e;
  const CUtensorMapSwizzle sw = rb == 16 ? CU_TENSOR_MAP_SWIZZLE_NONE : swizzle_of(rb);
  const CUresult r = enc(map, out_kind < 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : dtype_of(out_kind), 3, base, dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CONET_ERR_CUDA, "output tensor map encode failed (%d)", (int)r);
  return CONET_OK;
}

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
__global__ void weights_bf16_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst, int taps,
                                    __nv_bfloat16* __restrict__ out) {
  const int n = taps * cout * cin_dst;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin_dst, rem = i / cin_dst, co = rem % cout, tap = rem / cout;
    out[i] = __float2bfloat16_rn(ci < cin_src ? w[((size_t)co * taps + tap) * cin_src + ci] : 0.f);
  }
}

__global__ void weights_dgrad_bf16_kernel(const float* __restrict__ w, int C, __nv_bfloat16* __restrict__ out) {
  const int n = 9 * C * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int in = i % C, rem = i / C, o = rem % C, tp = rem / C;
    out[i] = __float2bfloat16_rn(w[((size_t)in * 9 + (8 - tp)) * C + o]);
  }
}

struct GradsBf16Args {
  const float* in[MAX_BR];
  __nv_bfloat16* out[MAX_BR];
};

// 8 values per thread step (n a multiple of 8: rows of C = 16k channels)
__global__ void grads_bf16_kernel(GradsBf16Args a, int nb, long long n8) {
  const long long total = n8 * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / n8);
    const long long k = i - (long long)b * n8;
    const float4 x0 = __ldg(reinterpret_cast<const float4*>(a.in[b]) + 2 * k);
    const float4 x1 = __ldg(reinterpret_cast<const float4*>(a.in[b]) + 2 * k + 1);
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x0.x, x0.y), h1 = __floats2bfloat162_rn(x0.z, x0.w);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(x1.x, x1.y), h3 = __floats2bfloat162_rn(x1.z, x1.w);
    uint4 o;
    o.x = *reinterpret_cast<const uint32_t*>(&h0);
    o.y = *reinterpret_cast<const uint32_t*>(&h1);
    o.z = *reinterpret_cast<const uint32_t*>(&h2);
    o.w = *reinterpret_cast<const uint32_t*>(&h3);
    reinterpret_cast<uint4*>(a.out[b])[k] = o;
  }
}

__global__ void weights_f16_kernel(const float* __restrict__ w, int cout, int cin_src, int cin_dst, int taps,
                                   __half* __restrict__ out) {
  const int n = taps * cout * cin_dst;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin_dst, rem = i / cin_dst, co = rem % cout, tap = rem / cout;
    out[i] = __float2half_rn(ci < cin_src ? w[((size_t)co * taps + tap) * cin_src + ci] : 0.f);
  }
}

int launch_weights_dgrad_bf16(const float* w, int C, void* out, cudaStream_t s) {
  weights_dgrad_bf16_kernel<<<grid_for(9LL * C * C, 256, 512), 256, 0, s>>>(w, C,
                                                                            static_cast<__nv_bfloat16*>(out));
  return check_launch("weights_dgrad_bf16_kernel");
}

int launch_grads_bf16(const float* const* in, void* const* out, int nb, long long n, cudaStream_t s) {
  if (nb < 1 || nb > MAX_BR || n % 8) return fail(CONET_ERR_UNSUPPORTED, "grads_bf16: nb %d, n %lld", nb, n);
  GradsBf16Args a = {};
  for (int b = 0; b < nb; ++b) {
    a.in[b] = in[b];
    a.out[b] = static_cast<__nv_bfloat16*>(out[b]);
  }
  grads_bf16_kernel<<<grid_for(n / 8 * nb, 256, 152 * 8), 256, 0, s>>>(a, nb, n / 8);
  return check_launch("grads_bf16_kernel");
}

int launch_weights_16(int kind, const float* w, int cout, int cin_src, int cin_dst, void* out, cudaStream_t s,
                      int taps) {
  if (kind == 3)
    weights_f16_kernel<<<grid_for((long long)taps * cout * cin_dst, 256, 512), 256, 0, s>>>(
        w, cout, cin_src, cin_dst, taps, reinterpret_cast<__half*>(out));
  else
    weights_bf16_kernel<<<grid_for((long long)taps * cout * cin_dst, 256, 512), 256, 0, s>>>(
        w, cout, cin_src, cin_dst, taps, reinterpret_cast<__nv_bfloat16*>(out));
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
