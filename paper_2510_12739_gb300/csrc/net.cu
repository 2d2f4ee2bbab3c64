// Host orchestration of the CoNet forward pass (Sec. III): input assembly, one conv launch
// per layer covering every branch, then the per-RE fusion / LayerNorm / pre-activation
// stage, and the 1x1 head fused into the last fusion stage.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"
#include "net.cuh"

namespace conet {

int dev_alloc(conet_s* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CONET_ERR_NOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  return CONET_OK;
}

void prof_begin(conet_s* h, int kind, cudaStream_t s) {
  if (!h->prof_on || h->prof_kind.size() >= PROF_CAP) return;
  const size_t i = h->prof_kind.size();
  while (h->prof_ev.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    h->prof_ev.push_back(e);
  }
  cudaEventRecord(h->prof_ev[2 * i], s);
  h->prof_open = kind;
}

void prof_end(conet_s* h, cudaStream_t s) {
  if (h->prof_open < 0) return;
  const size_t i = h->prof_kind.size();
  cudaEventRecord(h->prof_ev[2 * i + 1], s);
  h->prof_kind.push_back(h->prof_open);
  h->prof_open = -1;
}

namespace {

// Activation buffers.  Inference keeps two residual-stream buffers per branch (ping-pong)
// plus the two conv inputs of a block; training keeps every layer's tensors for backward.
struct Acts {
  conet_s* h;
  bool train() const { return h->cfg.train != 0; }
  float* at(size_t i) const { return h->act[i]; }
  int nb() const { return h->nb; }
  int depth() const { return h->cfg.depth; }
  // plain networks
  float* A(int l, int b) const { return train() ? at((size_t)l * nb() + b) : at((size_t)(l & 1) * nb() + b); }
  float* XM(int l) const { return train() ? at((size_t)depth() * nb() + l) : A(l, 0); }
  // residual networks
  float* A0(int b) const { return at(b); }
  float* RXM(int k) const {    // main residual stream entering block k (k = depth: head input)
    return train() ? at(nb() + k) : at((size_t)(k & 1) * nb());
  }
  size_t rbase() const { return (size_t)nb() + depth() + 1; }
  float* H1(int k, int b) const { return train() ? at(rbase() + ((size_t)k * 4 + 0) * nb() + b) : at(2 * nb() + b); }
  float* T1(int k, int b) const { return train() ? at(rbase() + ((size_t)k * 4 + 1) * nb() + b) : nullptr; }
  float* H2(int k, int b) const { return train() ? at(rbase() + ((size_t)k * 4 + 2) * nb() + b) : at(3 * nb() + b); }
  float* U(int k, int b) const { return train() ? at(rbase() + ((size_t)k * 4 + 3) * nb() + b) : at((size_t)((k + 1) & 1) * nb() + b); }
  float* XS(int k, int b) const {   // residual stream entering block k
    if (b == 0) return RXM(k);
    return k == 0 ? A0(b) : U(k - 1, b);
  }
  static size_t count(const conet_s* h) {
    const int nb = h->nb, d = h->cfg.depth;
    if (!h->cfg.residual) return h->cfg.train ? (size_t)d * nb + d : 2 * (size_t)nb;
    return h->cfg.train ? (size_t)nb + d + 1 + 4 * (size_t)d * nb : 4 * (size_t)nb;
  }
};

const float* P(const conet_s* h, long off) { return off < 0 ? nullptr : h->params + off; }
const float* W(const conet_s* h, long off) { return h->wt + h->wt_off.at((size_t)off); }

}  // namespace

int net_setup(conet_s* h) {
  const size_t n = h->L.total;
  CONET_TRY(dev_alloc_t(h, &h->params, n));
  CONET_TRY(dev_alloc_t(h, &h->grads, n));
  CONET_TRY(dev_alloc_t(h, &h->adam_m, n));
  CONET_TRY(dev_alloc_t(h, &h->adam_v, n));
  size_t wt = 0;
  for (const auto& c : h->L.convs) {
    const int cin_dst = c.cin == h->cin ? h->c_pad : c.cin;
    h->wt_off[c.off] = wt;
    wt += (size_t)9 * cin_dst * c.cout;
  }
  h->wt_total = wt;
  CONET_TRY(dev_alloc_t(h, &h->wt, wt));
  CONET_TRY(dev_alloc_t(h, &h->mask, (size_t)h->T * h->F));
  CONET_TRY(dev_alloc_t(h, &h->psym, (size_t)h->T * h->F * 2));
  const size_t re = (size_t)h->cfg.max_batch * h->T * h->F;
  CONET_TRY(dev_alloc_t(h, &h->X0, re * h->c_pad));
  const size_t na = Acts::count(h);
  h->act.resize(na);
  for (size_t i = 0; i < na; ++i) CONET_TRY(dev_alloc_t(h, &h->act[i], re * h->C));
  CONET_TRY(dev_alloc_t(h, &h->d_loss, 1));
  CONET_TRY(dev_alloc_t(h, &h->d_cnt, 2));
  CONET_CUDA(cudaMemset(h->params, 0, n * sizeof(float)));
  CONET_CUDA(cudaMemset(h->grads, 0, n * sizeof(float)));
  CONET_CUDA(cudaMemset(h->adam_m, 0, n * sizeof(float)));
  CONET_CUDA(cudaMemset(h->adam_v, 0, n * sizeof(float)));
  CONET_CUDA(cudaMemset(h->wt, 0, wt * sizeof(float)));
  PilotGrid pg;
  for (int i = 0; i < 4; ++i) pg.syms[i] = i < h->cfg.n_pilot_syms ? h->cfg.pilot_syms[i] : -1;
  pg.n_syms = h->cfg.n_pilot_syms;
  pg.comb = h->cfg.pilot_comb;
  pg.k0 = (uint32_t)h->cfg.pilot_seed;
  pg.k1 = (uint32_t)(h->cfg.pilot_seed >> 32);
  CONET_TRY(launch_pilots(h->T, h->F, pg, h->mask, h->psym, 0));
  CONET_CUDA(cudaDeviceSynchronize());
  return CONET_OK;
}

int net_weights_changed(conet_s* h, cudaStream_t s) {
  for (const auto& c : h->L.convs) {
    const int cin_dst = c.cin == h->cin ? h->c_pad : c.cin;
    CONET_TRY(launch_weights_to_tap_major(h->params + c.off, c.cout, c.cin, cin_dst, h->wt + h->wt_off.at(c.off), s));
  }
  return CONET_OK;
}

static int conv_layer(conet_s* h, ConvArgs& a, int cin, cudaStream_t s) {
  prof_begin(h, cin == h->C ? PK_CONV : PK_CONV_IN, s);
  const int rc = launch_conv3x3_fp32(a, h->nb, cin, h->C, s);
  prof_end(h, s);
  return rc;
}

static int fuse_stage(conet_s* h, const FuseArgs& f, cudaStream_t s) {
  prof_begin(h, PK_FUSE, s);
  const int rc = launch_fuse(f, s);
  prof_end(h, s);
  return rc;
}

static ConvArgs conv_args(conet_s* h, int B) {
  ConvArgs a = {};
  a.M = B * h->T * h->F;
  a.T = h->T;
  a.F = h->F;
  return a;
}

static FuseArgs fuse_args(conet_s* h, int B) {
  FuseArgs f = {};
  f.n_br = h->nb;
  f.C = h->C;
  f.Q = h->Q;
  f.M = (long long)B * h->T * h->F;
  return f;
}

int net_forward(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s) {
  if (h->prec != CONET_FP32) return fail(CONET_ERR_UNSUPPORTED, "precision %d forward not built yet", h->prec);
  const Acts A{h};
  const Layout& L = h->L;
  const int nb = h->nb, depth = h->cfg.depth;
  prof_begin(h, PK_ASSEMBLE, s);
  CONET_TRY(launch_assemble(Y, mask, h->psym, B, h->N, h->T, h->F, h->c_pad, h->X0, s));
  prof_end(h, s);
  if (!h->cfg.residual) {
    for (int l = 0; l < depth; ++l) {
      ConvArgs c = conv_args(h, B);
      for (int b = 0; b < nb; ++b) {
        c.in[b] = l == 0 ? h->X0 : (b == 0 ? A.XM(l - 1) : A.A(l - 1, b));
        c.w[b] = W(h, l == 0 ? L.in_w[b] : L.lw[b][l - 1]);
        c.bias[b] = P(h, l == 0 ? L.in_b[b] : L.lb[b][l - 1]);
        c.out0[b] = A.A(l, b);
      }
      c.relu0 = 1;
      CONET_TRY(conv_layer(h, c, l == 0 ? h->c_pad : h->C, s));
      FuseArgs f = fuse_args(h, B);
      for (int b = 0; b < nb; ++b) f.u[b] = A.A(l, b);
      f.fuse = fused_at(h->cfg, l);
      f.fuse_g = P(h, L.fg[l]);
      f.fuse_b = P(h, L.fb[l]);
      f.x0_out = A.XM(l);
      if (l == depth - 1) {
        f.head_w = P(h, L.hw);
        f.head_b = P(h, L.hb);
        f.llr = llr;
      }
      CONET_TRY(fuse_stage(h, f, s));
    }
  } else {
    ConvArgs c = conv_args(h, B);
    for (int b = 0; b < nb; ++b) {
      c.in[b] = h->X0;
      c.w[b] = W(h, L.in_w[b]);
      c.bias[b] = P(h, L.in_b[b]);
      c.out0[b] = A.A0(b);
    }
    c.relu0 = 1;
    CONET_TRY(conv_layer(h, c, h->c_pad, s));
    for (int k = 0; k <= depth; ++k) {
      // fusion after the input layer (k = 0) or after block k-1, then the next block's
      // pre-activation (or the head after the last block)
      FuseArgs f = fuse_args(h, B);
      for (int b = 0; b < nb; ++b) f.u[b] = k == 0 ? A.A0(b) : A.U(k - 1, b);
      f.fuse = fused_at(h->cfg, k);
      f.fuse_g = P(h, L.fg[k]);
      f.fuse_b = P(h, L.fb[k]);
      f.x0_out = A.RXM(k);
      if (k < depth) {
        for (int b = 0; b < nb; ++b) {
          f.h_out[b] = A.H1(k, b);
          f.ln1_g[b] = P(h, L.blk[b][k].ln1g);
          f.ln1_b[b] = P(h, L.blk[b][k].ln1b);
        }
      } else {
        f.head_w = P(h, L.hw);
        f.head_b = P(h, L.hb);
        f.llr = llr;
      }
      CONET_TRY(fuse_stage(h, f, s));
      if (k == depth) break;
      ConvArgs c1 = conv_args(h, B);
      for (int b = 0; b < nb; ++b) {
        c1.in[b] = A.H1(k, b);
        c1.w[b] = W(h, L.blk[b][k].c1w);
        c1.bias[b] = P(h, L.blk[b][k].c1b);
        c1.out0[b] = A.T1(k, b);
        c1.out1[b] = A.H2(k, b);
        c1.ln_g[b] = P(h, L.blk[b][k].ln2g);
        c1.ln_b[b] = P(h, L.blk[b][k].ln2b);
      }
      CONET_TRY(conv_layer(h, c1, h->C, s));
      ConvArgs c2 = conv_args(h, B);
      for (int b = 0; b < nb; ++b) {
        c2.in[b] = A.H2(k, b);
        c2.w[b] = W(h, L.blk[b][k].c2w);
        c2.bias[b] = P(h, L.blk[b][k].c2b);
        c2.resid[b] = A.XS(k, b);
        c2.out0[b] = A.U(k, b);
      }
      CONET_TRY(conv_layer(h, c2, h->C, s));
    }
  }
  h->fwd_B = B;
  return CONET_OK;
}

int net_backward(conet_s* h, const float* dllr, int B, cudaStream_t s) {
  (void)h; (void)dllr; (void)B; (void)s;
  return fail(CONET_ERR_UNSUPPORTED, "backward not built yet");
}

int net_adam(conet_s* h, float lr, int step, cudaStream_t s) {
  (void)h; (void)lr; (void)step; (void)s;
  return fail(CONET_ERR_UNSUPPORTED, "Adam not built yet");
}

int net_train_step(conet_s* h, const SimArgs& a, uint64_t step, int B, float lr, double* loss_out, cudaStream_t s) {
  (void)h; (void)a; (void)step; (void)B; (void)lr; (void)loss_out; (void)s;
  return fail(CONET_ERR_UNSUPPORTED, "train step not built yet");
}

}  // namespace conet
