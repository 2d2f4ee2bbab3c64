// Per-RE elementwise stage between convolution layers (Sec. III) of the FP32 path: the
// interaction, its LayerNorm, the pre-activations of the next block and the LLR head
// (fuse_quad, four REs per warp step, for widths that are multiples of 32; else
// fuse_row, one RE per warp step).  The forward and the backward's recompute of a
// block's input both launch it; the concatenation interaction runs concat_fuse_kernel.
#include "common.cuh"
#include "kernels.cuh"

namespace conet {

namespace {

// ------------------------------------------------------------------ one RE per warp
// Each lane holds NV vectors of VW consecutive channels: channel c = VW * (lane + 32 * v) + e.
// The launcher uses VW = 1, NV = 4 (any width up to 128) for the widths fuse_quad does not
// serve.
template <int VW, int NV>
struct Lane {
  float x[NV][VW];
};

template <int VW, int NV>
__device__ __forceinline__ int chan(int lane, int v, int e) { return VW * (lane + 32 * v) + e; }

// The branch activations are read once, past L1 (ld.global.cg).
template <int VW, int NV>
__device__ __forceinline__ void load_row(const float* p, int lane, int C, Lane<VW, NV>& r) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int c = chan<VW, NV>(lane, v, 0);
    if constexpr (VW == 2) {
      const float2 t = c < C ? __ldcg(reinterpret_cast<const float2*>(p + c)) : make_float2(0.f, 0.f);
      r.x[v][0] = t.x;
      r.x[v][1] = t.y;
    } else {
      r.x[v][0] = c < C ? __ldcg(p + c) : 0.f;
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

// The stage for resource element m (all 32 lanes of the warp take part).
template <int VW, int NV>
__device__ __forceinline__ void fuse_row(const FuseArgs& a, long long m, int lane) {
  using L = Lane<VW, NV>;
  const int C = a.C;
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

// ------------------------------------------------------------------ four REs per warp
// The same stage for widths C = 32 * NV4 (32, 64, 96, 128) with a group of eight lanes per
// RE: lane j of a group holds the float4 chunks {32 k + 4 j .. 32 k + 4 j + 3}, so a group's
// row access is one contiguous 128-byte segment per k, and a LayerNorm reduction is three
// shuffles instead of five for four REs at once: about a third of fuse_row's instructions
// per RE.
template <int NV4>
struct Quad {
  float4 x[NV4];
};

__device__ __forceinline__ float group8_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

template <int NV4>
__device__ __forceinline__ void q_load(const float* row, int j, bool ok, Quad<NV4>& r) {
#pragma unroll
  for (int k = 0; k < NV4; ++k)
    r.x[k] = ok ? __ldcg(reinterpret_cast<const float4*>(row + 32 * k + 4 * j)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int NV4>
__device__ __forceinline__ void q_store(float* row, int j, bool ok, const Quad<NV4>& r) {
  if (!ok) return;
#pragma unroll
  for (int k = 0; k < NV4; ++k) *reinterpret_cast<float4*>(row + 32 * k + 4 * j) = r.x[k];
}

__device__ __forceinline__ float f4_sum(float4 v) { return (v.x + v.y) + (v.z + v.w); }

// y = LN(x) * g + b over the C = 32 * NV4 channels of the group's RE (two passes: the mean,
// then the mean square deviation), optionally followed by ReLU.
template <int NV4>
__device__ __forceinline__ void q_layer_norm(const Quad<NV4>& x, int j, const float* g, const float* b, bool relu,
                                             Quad<NV4>& y) {
  constexpr float inv_c = 1.0f / (32 * NV4);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NV4; ++k) s += f4_sum(x.x[k]);
  const float mean = group8_sum(s) * inv_c;
  float q = 0.f;
#pragma unroll
  for (int k = 0; k < NV4; ++k) {
    const float4 d = make_float4(x.x[k].x - mean, x.x[k].y - mean, x.x[k].z - mean, x.x[k].w - mean);
    q += (d.x * d.x + d.y * d.y) + (d.z * d.z + d.w * d.w);
  }
  const float rstd = rsqrtf(group8_sum(q) * inv_c + 1e-5f);
#pragma unroll
  for (int k = 0; k < NV4; ++k) {
    const float4 gv = __ldg(reinterpret_cast<const float4*>(g + 32 * k + 4 * j));
    const float4 bv = __ldg(reinterpret_cast<const float4*>(b + 32 * k + 4 * j));
    float4 o = make_float4((x.x[k].x - mean) * rstd * gv.x + bv.x, (x.x[k].y - mean) * rstd * gv.y + bv.y,
                           (x.x[k].z - mean) * rstd * gv.z + bv.z, (x.x[k].w - mean) * rstd * gv.w + bv.w);
    if (relu) o = make_float4(fmaxf(o.x, 0.f), fmaxf(o.y, 0.f), fmaxf(o.z, 0.f), fmaxf(o.w, 0.f));
    y.x[k] = o;
  }
}

// The stage for resource element m, computed by the eight lanes of one group (j = lane % 8);
// all 32 lanes of the warp call it together (ok = false for a group past the end).
template <int NV4>
__device__ __forceinline__ void fuse_quad(const FuseArgs& a, long long m, bool ok, int j) {
  using Q4 = Quad<NV4>;
  constexpr int C = 32 * NV4;
  Q4 u[MAX_BR];
#pragma unroll
  for (int b = 0; b < MAX_BR; ++b)
    if (b < a.n_br) q_load(a.u[b] + m * C, j, ok, u[b]);
  Q4 x0 = u[0];
  if (a.fuse) {
    Q4 p = u[0];
#pragma unroll
    for (int b = 1; b < MAX_BR; ++b) {
      if (b >= a.n_br) continue;
#pragma unroll
      for (int k = 0; k < NV4; ++k) {
        float4& v = p.x[k];
        const float4 w = u[b].x[k];
        v = a.op ? make_float4(v.x + w.x, v.y + w.y, v.z + w.z, v.w + w.w)
                 : make_float4(v.x * w.x, v.y * w.y, v.z * w.z, v.w * w.w);
      }
    }
    if (a.fuse_g)
      q_layer_norm(p, j, a.fuse_g, a.fuse_b, false, x0);
    else
      x0 = p;
    if (a.feedback) {
#pragma unroll
      for (int b = 1; b < MAX_BR; ++b) {
        if (b >= a.n_br) continue;
#pragma unroll
        for (int k = 0; k < NV4; ++k) {
          float4& v = u[b].x[k];
          const float4 w = u[0].x[k];
          v = make_float4(v.x + w.x, v.y + w.y, v.z + w.z, v.w + w.w);
        }
        q_store(const_cast<float*>(a.u[b]) + m * C, j, ok, u[b]);
      }
    }
  }
  if (a.x0_out) q_store(a.x0_out + m * C, j, ok, x0);
#pragma unroll
  for (int b = 0; b < MAX_BR; ++b) {
    if (b >= a.n_br || !a.h_out[b]) continue;
    const Q4& xb = b == 0 ? x0 : u[b];
    Q4 h;
    if (a.ln1_g[b]) {
      q_layer_norm(xb, j, a.ln1_g[b], a.ln1_b[b], true, h);
    } else {
#pragma unroll
      for (int k = 0; k < NV4; ++k)
        h.x[k] = make_float4(fmaxf(xb.x[k].x, 0.f), fmaxf(xb.x[k].y, 0.f), fmaxf(xb.x[k].z, 0.f),
                             fmaxf(xb.x[k].w, 0.f));
    }
    q_store(a.h_out[b] + m * C, j, ok, h);
  }
  if (a.head_w) {
    for (int q = 0; q < a.Q; ++q) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < NV4; ++k) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(a.head_w + q * C + 32 * k + 4 * j));
        s += (w.x * x0.x[k].x + w.y * x0.x[k].y) + (w.z * x0.x[k].z + w.w * x0.x[k].w);
      }
      s = group8_sum(s);
      if (ok && j == 0) {
        const float v = s + __ldg(a.head_b + q);
        a.llr[m * a.Q + q] = v;
        if (!(fabsf(v) <= FLT_MAX)) *a.nonfinite = 1;
      }
    }
  }
}


// NV4 > 0: widths 32 * NV4, four REs per warp step (fuse_quad); NV4 = 0: any width up
// to 128, one RE per warp step (fuse_row).
template <int NV4>
__global__ void fuse_kernel(FuseArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  if constexpr (NV4 > 0) {
    const int grp = lane >> 3, j = lane & 7;
    for (long long q = warp0; 4 * q < a.M; q += nwarps) {
      const long long m = 4 * q + grp;
      const bool ok = m < a.M;
      fuse_quad<NV4>(a, ok ? m : 4 * q, ok, j);
    }
  } else {
    for (long long m = warp0; m < a.M; m += nwarps) fuse_row<1, 4>(a, m, lane);
  }
}

// ------------------------------------------------------------------ concatenation
// The concatenation interaction (op 2) of a plain network: the main's next input is the
// branches' rows side by side, W = n_br x C <= 128 channels, normalised over all W when
// fuse_g is set, written to x0_out [M][W]; the head (at the last layer) reads all W.  One
// warp per RE, lane l holding channels l + 32 v.  With feedback the supports' rows get the
// main's added in place.
__global__ void concat_fuse_kernel(FuseArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int C = a.C, W = a.n_br * a.C;
  for (long long m = warp0; m < a.M; m += nwarps) {
    float x[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = lane + 32 * v;
      x[v] = c < W ? __ldcg(a.u[c / C] + m * C + c % C) : 0.f;
    }
    if (a.feedback) {
      // Example II: each support continues with its activation plus the main's (the
      // concatenation above keeps the values before this)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int c = lane + 32 * v;
        if (c >= C && c < W)
          const_cast<float*>(a.u[c / C])[m * C + c % C] = x[v] + __ldcg(a.u[0] + m * C + c % C);
      }
    }
    if (a.fuse_g) {
      float s = 0.f;
#pragma unroll
      for (int v = 0; v < 4; ++v) s += x[v];
      const float mean = warp_sum(s) / (float)W;
      float q = 0.f;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float d = lane + 32 * v < W ? x[v] - mean : 0.f;
        q += d * d;
      }
      const float rstd = rsqrtf(warp_sum(q) / (float)W + 1e-5f);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int c = lane + 32 * v;
        x[v] = c < W ? (x[v] - mean) * rstd * __ldg(a.fuse_g + c) + __ldg(a.fuse_b + c) : 0.f;
      }
    }
    if (a.x0_out) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int c = lane + 32 * v;
        if (c < W) a.x0_out[m * W + c] = x[v];
      }
    }
    if (a.head_w) {
      for (int q = 0; q < a.Q; ++q) {
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = lane + 32 * v;
          if (c < W) s += __ldg(a.head_w + q * W + c) * x[v];
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
  if (a.fuse && a.op == 2) {
    if (a.n_br * a.C > 128) return fail(CONET_ERR_UNSUPPORTED, "concatenated width %d > 128", a.n_br * a.C);
    concat_fuse_kernel<<<grid_for(a.M * 32, 256, 152 * 16), 256, 0, s>>>(a);
    return check_launch("concat_fuse_kernel");
  }
  if (a.C > 128) return fail(CONET_ERR_UNSUPPORTED, "width %d > 128", a.C);
  const int g = grid_for(a.M * 32, 256, 152 * 16);
  switch (a.C) {
    case 32: fuse_kernel<1><<<g, 256, 0, s>>>(a); break;
    case 64: fuse_kernel<2><<<g, 256, 0, s>>>(a); break;
    case 96: fuse_kernel<3><<<g, 256, 0, s>>>(a); break;
    case 128: fuse_kernel<4><<<g, 256, 0, s>>>(a); break;
    default: fuse_kernel<0><<<g, 256, 0, s>>>(a); break;
  }
  return check_launch("fuse_kernel");
}

}  // namespace conet
