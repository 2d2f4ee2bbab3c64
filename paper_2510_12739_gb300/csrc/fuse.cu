// Per-RE elementwise stage between convolution layers (Sec. III): Hadamard fusion of the
// main and support activations, LayerNorm over channels after the fusion, the
// pre-activation (LN ->) ReLU that feeds the next block's first conv, and the 1x1 LLR
// head.  One warp per RE; lanes stride the channels, so every load is a coalesced row
// segment and the LayerNorm statistics are warp-shuffle reductions.
#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

// Each lane holds NV vectors of VW consecutive channels: channel c = VW * (lane + 32 * v) + e.
// VW = 2 serves the 64-channel networks with one 8-byte access per lane per row; VW = 1,
// NV = 4 any width up to 128.
template <int VW, int NV>
struct Lane {
  float x[NV][VW];
};

template <int VW, int NV>
__device__ __forceinline__ int chan(int lane, int v, int e) { return VW * (lane + 32 * v) + e; }

template <int VW, int NV>
__device__ __forceinline__ void load_row(const float* p, int lane, int C, Lane<VW, NV>& r) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int c = chan<VW, NV>(lane, v, 0);
    if constexpr (VW == 2) {
      const float2 t = c < C ? *reinterpret_cast<const float2*>(p + c) : make_float2(0.f, 0.f);
      r.x[v][0] = t.x;
      r.x[v][1] = t.y;
    } else {
      r.x[v][0] = c < C ? p[c] : 0.f;
    }
  }
}

template <int VW, int NV>
__device__ __forceinline__ void store_row(float* p, int lane, int C, const Lane<VW, NV>& r) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int c = chan<VW, NV>(lane, v, 0);
    if (c >= C) continue;
    if constexpr (VW == 2)
      *reinterpret_cast<float2*>(p + c) = make_float2(r.x[v][0], r.x[v][1]);
    else
      p[c] = r.x[v][0];
  }
}

template <int VW, int NV>
__device__ __forceinline__ void layer_norm(const Lane<VW, NV>& x, int lane, int C, const float* g, const float* b,
                                           Lane<VW, NV>& y) {
  float s = 0.f;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) s += chan<VW, NV>(lane, v, e) < C ? x.x[v][e] : 0.f;
  const float mean = warp_sum(s) / (float)C;
  float q = 0.f;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const float d = chan<VW, NV>(lane, v, e) < C ? x.x[v][e] - mean : 0.f;
      q += d * d;
    }
  const float rstd = rsqrtf(warp_sum(q) / (float)C + 1e-5f);
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int c = chan<VW, NV>(lane, v, e);
      y.x[v][e] = c < C ? (x.x[v][e] - mean) * rstd * __ldg(g + c) + __ldg(b + c) : 0.f;
    }
}

template <int VW, int NV>
__global__ void fuse_kernel(FuseArgs a) {
  using L = Lane<VW, NV>;
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C;
  for (long long m = warp0; m < a.M; m += nwarps) {
    L u[MAX_BR];
#pragma unroll
    for (int b = 0; b < MAX_BR; ++b) {
      if (b < a.n_br) {
        load_row(a.u[b] + m * C, lane, C, u[b]);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int e = 0; e < VW; ++e) u[b].x[v][e] = 0.f;
      }
    }
    L x0;
    if (a.fuse) {
      // the interaction: product (op 0) or sum (op 1) of all branches
      L p = u[0];
#pragma unroll
      for (int b = 1; b < MAX_BR; ++b)
        if (b < a.n_br) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int e = 0; e < VW; ++e) p.x[v][e] = a.op ? p.x[v][e] + u[b].x[v][e] : p.x[v][e] * u[b].x[v][e];
        }
      if (a.fuse_g)
        layer_norm(p, lane, C, a.fuse_g, a.fuse_b, x0);
      else
        x0 = p;
      if (a.feedback) {
        // Example II: each support continues with its activation plus the main's, written
        // back over its own row (its stream / next input)
#pragma unroll
        for (int b = 1; b < MAX_BR; ++b) {
          if (b >= a.n_br) continue;
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int e = 0; e < VW; ++e) u[b].x[v][e] += u[0].x[v][e];
          store_row(const_cast<float*>(a.u[b]) + m * C, lane, C, u[b]);
        }
      }
    } else {
      x0 = u[0];
    }
    if (a.x0_out) store_row(a.x0_out + m * C, lane, C, x0);
#pragma unroll
    for (int b = 0; b < MAX_BR; ++b) {
      if (b >= a.n_br || !a.h_out[b]) continue;
      const L& xb = b == 0 ? x0 : u[b];
      L h;
      if (a.ln1_g[b])
        layer_norm(xb, lane, C, a.ln1_g[b], a.ln1_b[b], h);
      else
        h = xb;
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int e = 0; e < VW; ++e) h.x[v][e] = fmaxf(h.x[v][e], 0.f);
      store_row(a.h_out[b] + m * C, lane, C, h);
    }
    if (a.head_w) {
      for (int q = 0; q < a.Q; ++q) {
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            const int c = chan<VW, NV>(lane, v, e);
            if (c < C) s += __ldg(a.head_w + q * C + c) * x0.x[v][e];
          }
        s = warp_sum(s);
        if (lane == 0) {
          const float v = s + __ldg(a.head_b + q);
          a.llr[m * a.Q + q] = v;
          if (!(fabsf(v) <= FLT_MAX)) *a.nonfinite = 1;
        }
      }
    }
  }
}

}  // namespace

int launch_fuse(const FuseArgs& a, cudaStream_t s) {
  if (a.C > 128) return fail(CONET_ERR_UNSUPPORTED, "width %d > 128", a.C);
  if (a.C == 64)
    fuse_kernel<2, 1><<<grid_for(a.M * 32, 256, 152 * 16), 256, 0, s>>>(a);
  else
    fuse_kernel<1, 4><<<grid_for(a.M * 32, 256, 152 * 16), 256, 0, s>>>(a);
  return check_launch("fuse_kernel");
}

}  // namespace conet
