// Depthwise 3x3 'same' conv of every branch on 16-bit activations (the first half of a
// depthwise-separable conv on the BF16 / FP16 tensor-core path, Sec. II-A / III):
// out[m][c] = round16(sum over the taps, in order, of w[c][tap] x[m + shift(tap)][c]) with
// FP32 weights and FP32 accumulation, zero outside the grid.
//
// Memory-bound (2 x C x 2 bytes per RE and branch).  A CTA takes tiles of one symbol row x
// DW_TF subcarriers x all channels: it copies the tile's three input rows (with the one-
// subcarrier halo, zero outside the grid) into shared memory with 16-byte loads, every
// thread issuing its share at once, so each input vector leaves DRAM / L2 once per tile;
// then each thread computes DW_NO consecutive outputs of 4 channels from shared memory,
// with the branch's weights staged there too, in two-lane FP32 FMAs (fma.rn.f32x2, each
// lane rounding like fmaf).  Several CTAs per SM keep enough loads in flight.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

// The two 16-bit values packed in a 32-bit word (low half first) as floats, and back
// (round to nearest even), without taking the word's address.
template <typename T16>
__device__ __forceinline__ float2 unpack16x2(uint32_t u);
template <>
__device__ __forceinline__ float2 unpack16x2<__nv_bfloat16>(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <>
__device__ __forceinline__ float2 unpack16x2<__half>(uint32_t u) {
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}

template <typename T16>
__device__ __forceinline__ uint32_t pack16x2(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack16x2<__nv_bfloat16>(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}
template <>
__device__ __forceinline__ uint32_t pack16x2<__half>(float lo, float hi) {
  return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
}

__device__ __forceinline__ unsigned long long f2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ float2 un2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

constexpr int DW_TF = 64;     // subcarriers per tile
constexpr int DW_NO = 4;      // consecutive outputs per thread
constexpr int DW_THREADS = 256;

__host__ __device__ constexpr int dw_smem_bytes(int C) { return 3 * (DW_TF + 2) * C * 2 + 9 * C * 4; }

// grid (x: tile groups, y: branch).  The loads of the next tile are issued into registers
// before the current tile is computed from shared memory, so they overlap.
template <typename T16, int C>
__global__ void __launch_bounds__(DW_THREADS, C <= 64 ? 3 : 2) dwconv3x3_16_kernel(const __grid_constant__ DwArgs16 a) {
  constexpr int q8 = C / 8, q4 = C / 4;
  constexpr int N_VEC = 3 * (DW_TF + 2) * q8;                 // 16-byte vectors of a tile's three rows
  constexpr int PER = (N_VEC + DW_THREADS - 1) / DW_THREADS;   // per thread
  constexpr int N_UNIT = q4 * (DW_TF / DW_NO);
  extern __shared__ uint4 dw_smem[];
  const int b = blockIdx.y;
  uint4* xs = dw_smem;                                                  // [3][DW_TF + 2][q8]
  float* ws = reinterpret_cast<float*>(dw_smem + N_VEC);                // [9][C]
  const T16* __restrict__ in = static_cast<const T16*>(a.in[b]);
  T16* __restrict__ out = static_cast<T16*>(a.out[b]);
  const int T = a.T, F = a.F;
  const int ntf = (F + DW_TF - 1) / DW_TF;
  const long long n_tiles = a.M / F * ntf;
  {
    const float* __restrict__ w = a.w[b];
    for (int i = threadIdx.x; i < 9 * C; i += DW_THREADS) ws[i] = __ldg(w + (i % C) * 9 + i / C);
  }
  uint4 reg[PER];
  auto load_tile = [&](long long tile) {
    const long long row = tile / ntf;
    const int f0 = (int)(tile % ntf) * DW_TF, t = (int)(row % T);
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int e = (int)threadIdx.x + it * DW_THREADS;
      const int v = e % q8, k = (e / q8) % (DW_TF + 2), r = e / (q8 * (DW_TF + 2));
      const int f = f0 + k - 1, tt = t + r - 1;
      reg[it] = make_uint4(0u, 0u, 0u, 0u);
      if (e < N_VEC && tt >= 0 && tt < T && f >= 0 && f < F)
        reg[it] = __ldg(reinterpret_cast<const uint4*>(in + ((row + r - 1) * F + f) * C) + v);
    }
  };
  long long tile = blockIdx.x;
  if (tile < n_tiles) load_tile(tile);
  for (; tile < n_tiles; tile += gridDim.x) {
    const long long row = tile / ntf;
    const int f0 = (int)(tile % ntf) * DW_TF;
    __syncthreads();   // the previous tile's reads of xs are done (and ws is written)
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int e = (int)threadIdx.x + it * DW_THREADS;
      if (e < N_VEC) xs[e] = reg[it];
    }
    __syncthreads();
    if (tile + gridDim.x < n_tiles) load_tile(tile + gridDim.x);
    const uint2* xs2 = reinterpret_cast<const uint2*>(xs);   // 4-channel vectors: [3][DW_TF + 2][q4]
    for (int u = threadIdx.x; u < N_UNIT; u += DW_THREADS) {
      const int g = u % q4, j0 = (u / q4) * DW_NO, c = 4 * g;
      if (f0 + j0 >= F) continue;
      unsigned long long acc01[DW_NO], acc23[DW_NO];
#pragma unroll
      for (int j = 0; j < DW_NO; ++j) acc01[j] = acc23[j] = 0ull;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        unsigned long long w01[3], w23[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float4 wv = *reinterpret_cast<const float4*>(ws + (3 * r + d) * C + c);
          w01[d] = f2(wv.x, wv.y);
          w23[d] = f2(wv.z, wv.w);
        }
        // each input vector of the row unpacked once and added into the outputs that use it,
        // so every output takes its taps in order 0..8
#pragma unroll
        for (int k = 0; k < DW_NO + 2; ++k) {
          const uint2 raw = xs2[(r * (DW_TF + 2) + j0 + k) * q4 + g];
          const float2 p = unpack16x2<T16>(raw.x), p2 = unpack16x2<T16>(raw.y);
          const unsigned long long x01 = f2(p.x, p.y), x23 = f2(p2.x, p2.y);
#pragma unroll
          for (int d = 0; d < 3; ++d) {   // output j = k - d takes this column as tap (r, d)
            const int j = k - d;
            if (j < 0 || j >= DW_NO) continue;
            fma2(acc01[j], w01[d], x01);
            fma2(acc23[j], w23[d], x23);
          }
        }
      }
      T16* o = out + (row * F + f0 + j0) * C + c;
#pragma unroll
      for (int j = 0; j < DW_NO; ++j) {
        if (f0 + j0 + j >= F) break;
        const float2 o01 = un2(acc01[j]), o23 = un2(acc23[j]);
        *reinterpret_cast<uint2*>(o + (long long)j * C) =
            make_uint2(pack16x2<T16>(o01.x, o01.y), pack16x2<T16>(o23.x, o23.y));
      }
    }
  }
}

template <typename T16, int C>
int launch_dw16(const DwArgs16& a, int n_br, cudaStream_t s) {
  const long long n_tiles = a.M / a.F * ((a.F + DW_TF - 1) / DW_TF);
  const int smem = dw_smem_bytes(C);
  // one wave of resident CTAs, shared by the branches (each CTA then walks its tiles)
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 0, per_sm = 0;
    CONET_CUDA(cudaGetDevice(&dev));
    CONET_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CONET_CUDA(cudaFuncSetAttribute(dwconv3x3_16_kernel<T16, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CONET_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dwconv3x3_16_kernel<T16, C>, DW_THREADS, smem));
    resident = sms * (per_sm > 0 ? per_sm : 1);
  }
  // (rounded down: a CTA past the resident wave would run alone after it)
  const int gx = grid_for(n_tiles, 1, resident / n_br > 0 ? resident / n_br : 1);
  dwconv3x3_16_kernel<T16, C><<<dim3((unsigned)gx, (unsigned)n_br), DW_THREADS, smem, s>>>(a);
  return check_launch("dwconv3x3_16_kernel");
}

}  // namespace

int launch_dwconv3x3_16(int kind, const DwArgs16& a, int n_br, cudaStream_t s) {
  if (n_br < 1 || a.F < 1 || a.M % a.F) return fail(CONET_ERR_ARG, "depthwise conv: %d branches, %lld REs", n_br, a.M);
  if (kind != 0 && kind != 3) return fail(CONET_ERR_UNSUPPORTED, "16-bit depthwise conv kind %d", kind);
#define DW_CASE(CC)                                                                                 \
  if (a.C == CC)                                                                                    \
    return kind == 3 ? launch_dw16<__half, CC>(a, n_br, s) : launch_dw16<__nv_bfloat16, CC>(a, n_br, s);
  DW_CASE(32)
  DW_CASE(64)
  DW_CASE(96)
  DW_CASE(128)
#undef DW_CASE
  return fail(CONET_ERR_UNSUPPORTED, "16-bit depthwise conv of width %d is not instantiated", a.C);
}

}  // namespace conet
