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
// plus the two conv inputs of a block; training keeps every layer's tensors for backward,
// or (residual networks with recompute) the streams of every block and one block's inner
// tensors (H1, T1, H2), which the backward pass recomputes block by block.
struct Acts {
  conet_s* h;
  bool train() const { return h->cfg.train != 0; }
  bool rc() const { return train() && h->cfg.residual && h->cfg.recompute; }
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
  float* H1(int k, int b) const {
    return rc() ? at(rbase() + b) : train() ? at(rbase() + ((size_t)k * 4 + 0) * nb() + b) : at(2 * nb() + b);
  }
  float* T1(int k, int b) const {
    return rc() ? at(rbase() + nb() + b) : train() ? at(rbase() + ((size_t)k * 4 + 1) * nb() + b) : nullptr;
  }
  float* H2(int k, int b) const {
    return rc() ? at(rbase() + 2 * nb() + b) : train() ? at(rbase() + ((size_t)k * 4 + 2) * nb() + b) : at(3 * nb() + b);
  }
  float* U(int k, int b) const {
    return rc()      ? at(rbase() + ((size_t)3 + k) * nb() + b)
           : train() ? at(rbase() + ((size_t)k * 4 + 3) * nb() + b)
                     : at((size_t)((k + 1) & 1) * nb() + b);
  }
  float* XS(int k, int b) const {   // residual stream entering block k
    if (b == 0) return RXM(k);
    return k == 0 ? A0(b) : U(k - 1, b);
  }
  static size_t count(const conet_s* h) {
    const int nb = h->nb, d = h->cfg.depth;
    const bool tc = h->prec != CONET_FP32;   // tensor-core inference keeps its conv inputs in 16 bits
    if (!h->cfg.residual) return h->cfg.train ? (size_t)d * nb + d : (tc ? 0 : 2 * (size_t)nb);
    if (h->cfg.train && h->cfg.recompute) return (size_t)nb + d + 1 + (3 + (size_t)d) * nb;
    return h->cfg.train ? (size_t)nb + d + 1 + 4 * (size_t)d * nb : (tc ? 2 : 4) * (size_t)nb;
  }
};

const float* P(const conet_s* h, long off) { return off < 0 ? nullptr : h->params + off; }

// Plain networks with the concatenation interaction: whether the main activation after
// layer l is n_branches x width wide, and its buffer (one per layer when training).
bool wide_at(const conet_s* h, int l) { return l >= 0 && fused_width(h->cfg, l) != h->C; }
float* xcat_at(const conet_s* h, int l) {
  return h->xcat + (h->cfg.train ? (size_t)l * h->chunk * h->T * h->F * h->nb * h->C : 0);
}
const float* W(const conet_s* h, long off) { return h->wt + h->wt_off.at((size_t)off); }

}  // namespace

int tc_setup(conet_s* h);
int tc_weights_changed(conet_s* h, cudaStream_t s);
int net_forward_tc(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s);

int net_setup(conet_s* h) {
  // (Example II's feedback adds the main activation into the supports' rows in place, so a
  // per-block recompute would add it twice; the tensor-core epilogue's training tape holds a
  // support's activation before the feedback, so BF16 handles train the sum interaction only)
  if (h->cfg.train && ((h->cfg.feedback && (h->prec != CONET_FP32 || (h->cfg.residual && h->cfg.recompute))) ||
                       (h->cfg.fuse_op == 1 && h->prec != CONET_FP32 && h->prec != CONET_BF16)))
    return fail(CONET_ERR_UNSUPPORTED,
                "training: the sum interaction on FP32 / BF16 handles, Example II feedback on FP32 handles "
                "without recompute");
  if (h->cfg.fuse_op == 2 && h->prec != CONET_FP32)
    return fail(CONET_ERR_UNSUPPORTED, "concatenation (fuse_op 2): FP32 handles only");
  if (h->cfg.depthwise && (!h->cfg.residual || (h->cfg.train && h->prec != CONET_FP32) ||
                            (h->prec != CONET_FP32 && h->prec != CONET_BF16 && h->prec != CONET_FP16)))
    return fail(CONET_ERR_UNSUPPORTED,
                "depthwise-separable convs: residual networks, FP32 training, FP32 / BF16 / FP16 inference");
  const size_t n = h->L.total;
  CONET_TRY(dev_alloc_t(h, &h->params, n));
  if (h->cfg.support_inputs) CONET_TRY(dev_alloc_t(h, &h->params_eff, n));
  CONET_TRY(dev_alloc_t(h, &h->grads, n));
  CONET_TRY(dev_alloc_t(h, &h->adam_m, n));
  CONET_TRY(dev_alloc_t(h, &h->adam_v, n));
  size_t wt = 0;
  for (const auto& c : h->L.convs) {
    const int cin_dst = c.cin == h->cin ? h->c_pad : c.cin;
    h->wt_off[c.off] = wt;
    wt += (size_t)c.taps * cin_dst * c.cout;
  }
  h->wt_total = wt;
  CONET_TRY(dev_alloc_t(h, &h->wt, wt));
  CONET_TRY(dev_alloc_t(h, &h->mask, (size_t)h->T * h->F));
  CONET_TRY(dev_alloc_t(h, &h->psym, (size_t)h->T * h->F * 2));
  // Tensor-core inference streams the batch through activation buffers sized for a chunk of
  // slots (at most ~48 GB of activations); FP32 and training keep the whole batch.
  const size_t na = Acts::count(h);
  h->chunk = h->cfg.max_batch;
  if (h->prec != CONET_FP32 && !h->cfg.train) {
    // bytes per conv-input value (hi + lo for split TF32)
    const double opnd = h->prec == CONET_TF32X3 ? 8.0 : h->prec == CONET_FP8E4M3 ? 1.0 : 2.0;
    const double n_in = h->cfg.depthwise ? 3.0 : 2.0;   // 16-bit conv inputs per branch (+ depthwise output)
    const double per_slot = (double)h->T * h->F * ((double)na * h->C * 4 + n_in * h->nb * h->C * opnd + 32 * opnd);
    const double fit = 48e9 / per_slot;
    h->chunk = fit < 1 ? 1 : (fit < h->cfg.max_batch ? (int)fit : h->cfg.max_batch);
  }
  const size_t re = (size_t)h->chunk * h->T * h->F;
  const bool need_x0 = h->prec == CONET_FP32 || h->cfg.train;
  CONET_TRY(dev_alloc_t(h, &h->X0, need_x0 ? re * h->c_pad : 4));
  h->act.resize(na);
  for (size_t i = 0; i < na; ++i) CONET_TRY(dev_alloc_t(h, &h->act[i], re * h->C));
  if (h->cfg.depthwise && h->prec == CONET_FP32)
    for (int b = 0; b < h->nb; ++b) CONET_TRY(dev_alloc_t(h, &h->dw_out[b], re * h->C));
  // concatenated main activations: one buffer, or (training) one per layer for the backward
  if (h->cfg.fuse_op == 2)
    CONET_TRY(dev_alloc_t(h, &h->xcat, re * h->nb * h->C * (h->cfg.train ? h->cfg.depth : 1)));
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
  h->n_pilot_re = 0;
  for (int t = 0; t < h->T; ++t) {
    bool p = false;
    for (int i = 0; i < h->cfg.n_pilot_syms; ++i) p = p || h->cfg.pilot_syms[i] == t;
    if (p) h->n_pilot_re += (h->F + h->cfg.pilot_comb - 1) / h->cfg.pilot_comb;
  }
  if (h->cfg.train) {
    size_t wd = 0;
    for (const auto& c : h->L.convs) {
      if (c.cin == h->cin) continue;   // the input conv needs no data gradient
      h->wd_off[c.off] = wd;
      wd += (size_t)9 * c.cin * c.cout;
    }
    CONET_TRY(dev_alloc_t(h, &h->wd, wd ? wd : 1));
    h->tc_dgrad = h->prec == CONET_BF16;
    if (h->tc_dgrad) {
      const int cinp0 = (h->c_pad + 7) / 8 * 8;
      CONET_TRY(dev_alloc(h, &h->wg_tc,
                          wgrad_tc_scratch_bytes(h->cfg.max_batch, h->T, h->F, h->C > cinp0 ? h->C : cinp0, h->C)));
      CONET_TRY(dev_alloc(h, &h->wd16, (wd ? wd : 1) * sizeof(uint16_t)));
      for (int b = 0; b < h->nb; ++b) CONET_TRY(dev_alloc(h, &h->g16[b], re * h->C * sizeof(uint16_t)));
      CONET_TRY(dev_alloc_t(h, &h->zero_c, (size_t)h->C));
      CONET_CUDA(cudaMemset(h->zero_c, 0, (size_t)h->C * sizeof(float)));
    }
    for (int k = 0; k < 3; ++k)
      for (int b = 0; b < h->nb; ++b) CONET_TRY(dev_alloc_t(h, &h->G[k][b], re * h->C));
    const size_t cw = (size_t)(h->cfg.fuse_op == 2 ? h->nb * h->C : h->C);   // widest fused activation
    CONET_TRY(dev_alloc_t(h, &h->ew_part, (size_t)EW_PART_CTAS * (h->Q * cw + h->Q + 2 * cw)));
    if (h->cfg.fuse_op == 2) CONET_TRY(dev_alloc_t(h, &h->gcat, re * cw));
    // split partials of the weight gradient, sized for the largest split count of either kernel
    const size_t splits = (size_t)(WG_MAX_SPLITS * h->nb > WG_TILED_MAX_CTAS ? WG_MAX_SPLITS * h->nb : WG_TILED_MAX_CTAS);
    const size_t wg = splits * 9 * (size_t)(h->C > h->c_pad ? h->C : h->c_pad) * h->C;
    CONET_TRY(dev_alloc_t(h, &h->wg_part, wg));
    CONET_TRY(dev_alloc_t(h, &h->sim_Y, re * h->N * 2));
    CONET_TRY(dev_alloc_t(h, &h->sim_bits, re * h->Q));
    CONET_TRY(dev_alloc_t(h, &h->sim_nv, (size_t)h->cfg.max_batch));
    CONET_TRY(dev_alloc_t(h, &h->llr, re * h->Q));
    CONET_TRY(dev_alloc_t(h, &h->dllr, re * h->Q));
  }
  // device status words: [0] the site of the first timed-out pipeline wait, [1] set when a
  // forward pass wrote a non-finite LLR (both read and cleared by conet_sync)
  CONET_TRY(dev_alloc_t(h, &h->d_err, 2));
  CONET_CUDA(cudaMemset(h->d_err, 0, 2 * sizeof(int)));
  CONET_TRY(tc_setup(h));
  CONET_CUDA(cudaDeviceSynchronize());
  return CONET_OK;
}

// Selective support inputs (Sec. III): the support nets' input-layer weights on the
// withheld channels -- by default the received signal (the first 2 N of the input), else
// every channel outside support_mask -- held at zero in `w` (the master parameters'
// effective copy, or their gradient).
static int zero_withheld_inputs(const conet_s* h, float* w, cudaStream_t s) {
  if (!h->cfg.support_inputs) return CONET_OK;
  const unsigned keep = h->cfg.support_mask ? h->cfg.support_mask : 7u << (2 * h->N);   // mask, Re / Im LS
  for (int b = 1; b < h->nb; ++b) CONET_TRY(launch_zero_input_channels(w + h->L.in_w[b], h->C, h->cin, keep, s));
  return CONET_OK;
}

// The parameters the kernels' weight layouts are made from.
static const float* eff_params(const conet_s* h) { return h->cfg.support_inputs ? h->params_eff : h->params; }

int net_weights_changed(conet_s* h, cudaStream_t s) {
  if (h->cfg.support_inputs) {
    CONET_CUDA(cudaMemcpyAsync(h->params_eff, h->params, h->L.total * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CONET_TRY(zero_withheld_inputs(h, h->params_eff, s));
  }
  const float* pe = eff_params(h);
  for (const auto& c : h->L.convs) {
    const int cin_dst = c.cin == h->cin ? h->c_pad : c.cin;
    CONET_TRY(launch_weights_to_tap_major(pe + c.off, c.cout, c.cin, cin_dst, h->wt + h->wt_off.at(c.off), s,
                                          c.taps));
    if (h->cfg.train && c.cin != h->cin && c.taps == 9) {
      if (h->tc_dgrad)
        CONET_TRY(launch_weights_dgrad_bf16(h->params + c.off, c.cout,
                                            static_cast<uint16_t*>(h->wd16) + h->wd_off.at(c.off), s));
      else
        CONET_TRY(launch_weights_dgrad_layout(h->params + c.off, c.cout, h->wd + h->wd_off.at(c.off), s, c.cin));
    }
  }
  return tc_weights_changed(h, s);
}

static int conv_layer(conet_s* h, ConvArgs& a, int cin, cudaStream_t s, int n_br = 0) {
  prof_begin(h, cin == h->C || n_br ? PK_CONV : PK_CONV_IN, s);
  const int rc = launch_conv3x3_fp32(a, n_br ? n_br : h->nb, cin, h->C, s);
  prof_end(h, s);
  return rc;
}

// A plain layer whose main input is the concatenation of the previous layer's activations
// (fuse_op 2): the main branch's conv reads n_branches x width channels, so it launches on
// its own, the supports' convs together.
static int conv_layer_concat(conet_s* h, const ConvArgs& a, cudaStream_t s) {
  ConvArgs m = a, sup = a;
  CONET_TRY(conv_layer(h, m, h->nb * h->C, s, 1));
  for (int b = 1; b < h->nb; ++b) {
    sup.in[b - 1] = a.in[b];
    sup.w[b - 1] = a.w[b];
    sup.bias[b - 1] = a.bias[b];
    sup.out0[b - 1] = a.out0[b];
  }
  return conv_layer(h, sup, h->C, s, h->nb - 1);
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
  f.nonfinite = h->d_err + 1;
  f.op = h->cfg.fuse_op;
  f.feedback = h->cfg.feedback;
  return f;
}

void net_graph_reset(conet_s* h) {
  if (h->g_exec) cudaGraphExecDestroy(h->g_exec);
  h->g_exec = nullptr;
  h->g_Y = h->g_mask = h->g_llr = nullptr;
  h->g_B = 0;
}

// The forward as a replayed CUDA graph where that is sound: an inference handle, no launch
// profiling, and (E4M3) activation scales already calibrated, since a calibrating pass
// changes host state.  Any capture failure falls back to the eager forward for good.
int net_forward_replay(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s) {
  const bool eligible = h->graphs && !h->cfg.train && !h->prof_on &&
                        !(h->prec == CONET_FP8E4M3 && !h->fp8_calibrated);
  if (!eligible) {
    net_graph_reset(h);
    return net_forward(h, Y, mask, B, llr, s);
  }
  const bool same = h->g_Y == Y && h->g_mask == mask && h->g_llr == llr && h->g_B == B;
  if (same && h->g_exec) {
    CONET_CUDA(cudaGraphLaunch(h->g_exec, s));
    launch_count_add(h->g_kernels);
    h->fwd_B = B;
    return CONET_OK;
  }
  if (!same) {
    net_graph_reset(h);
    h->g_Y = Y;
    h->g_mask = mask;
    h->g_llr = llr;
    h->g_B = B;
    return net_forward(h, Y, mask, B, llr, s);
  }
  if ((!h->g_stream && cudaStreamCreateWithFlags(&h->g_stream, cudaStreamNonBlocking) != cudaSuccess) ||
      cudaStreamBeginCapture(h->g_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    net_graph_reset(h);
    h->graphs = false;
    return net_forward(h, Y, mask, B, llr, s);
  }
  cudaGraph_t g = nullptr;
  const unsigned long long n0 = launch_count();
  const int rc = net_forward(h, Y, mask, B, llr, h->g_stream);
  const cudaError_t e = cudaStreamEndCapture(h->g_stream, &g);
  const long long n_cap = (long long)(launch_count() - n0);
  launch_count_add(-n_cap);   // recorded, not run
  cudaGetLastError();
  cudaGraphExec_t ex = nullptr;
  const bool ok = rc == CONET_OK && e == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    net_graph_reset(h);
    h->graphs = false;
    return net_forward(h, Y, mask, B, llr, s);
  }
  h->g_exec = ex;
  h->g_kernels = n_cap;
  CONET_CUDA(cudaGraphLaunch(h->g_exec, s));
  launch_count_add(h->g_kernels);
  h->fwd_B = B;
  return CONET_OK;
}

// One stage of the FP32 residual forward: the fusion after the input layer (k = 0) or after
// block k-1, then block k's pre-activation (or the head after the last block).
static int resid_fuse(conet_s* h, int k, int B, float* llr, cudaStream_t s) {
  const Acts A{h};
  const Layout& L = h->L;
  const int nb = h->nb, depth = h->cfg.depth;
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
  return fuse_stage(h, f, s);
}

// A depthwise-separable block conv's per-channel 3x3 (into dw_out); the 1x1 that follows
// runs as the block conv itself with taps = 1 (same epilogue).
static int resid_dw(conet_s* h, int B, float* const* in, const long* dw_off, cudaStream_t s) {
  DwArgs d = {};
  for (int b = 0; b < h->nb; ++b) {
    d.in[b] = in[b];
    d.w[b] = P(h, dw_off[b]);
    d.out[b] = h->dw_out[b];
  }
  d.C = h->C;
  d.T = h->T;
  d.F = h->F;
  d.M = (long long)B * h->T * h->F;
  prof_begin(h, PK_CONV, s);
  const int rc = launch_dwconv3x3(d, h->nb, s);
  prof_end(h, s);
  return rc;
}

// Block k's first conv (LN2 + ReLU epilogue) and second conv (residual add).
static int resid_conv1(conet_s* h, int k, int B, cudaStream_t s) {
  const Acts A{h};
  const Layout& L = h->L;
  ConvArgs c1 = conv_args(h, B);
  if (h->cfg.depthwise) {
    float* in[MAX_BR];
    long d[MAX_BR];
    for (int b = 0; b < h->nb; ++b) {
      in[b] = A.H1(k, b);
      d[b] = L.blk[b][k].c1d;
    }
    CONET_TRY(resid_dw(h, B, in, d, s));
    c1.taps = 1;
  }
  for (int b = 0; b < h->nb; ++b) {
    c1.in[b] = h->cfg.depthwise ? h->dw_out[b] : A.H1(k, b);
    c1.w[b] = W(h, L.blk[b][k].c1w);
    c1.bias[b] = P(h, L.blk[b][k].c1b);
    c1.out0[b] = A.T1(k, b);
    c1.out1[b] = A.H2(k, b);
    c1.ln_g[b] = P(h, L.blk[b][k].ln2g);
    c1.ln_b[b] = P(h, L.blk[b][k].ln2b);
  }
  return conv_layer(h, c1, h->C, s);
}

static int resid_conv2(conet_s* h, int k, int B, cudaStream_t s) {
  const Acts A{h};
  const Layout& L = h->L;
  ConvArgs c2 = conv_args(h, B);
  if (h->cfg.depthwise) {
    float* in[MAX_BR];
    long d[MAX_BR];
    for (int b = 0; b < h->nb; ++b) {
      in[b] = A.H2(k, b);
      d[b] = L.blk[b][k].c2d;
    }
    CONET_TRY(resid_dw(h, B, in, d, s));
    c2.taps = 1;
  }
  for (int b = 0; b < h->nb; ++b) {
    c2.in[b] = h->cfg.depthwise ? h->dw_out[b] : A.H2(k, b);
    c2.w[b] = W(h, L.blk[b][k].c2w);
    c2.bias[b] = P(h, L.blk[b][k].c2b);
    c2.resid[b] = A.XS(k, b);
    c2.out0[b] = A.U(k, b);
  }
  return conv_layer(h, c2, h->C, s);
}

int net_forward(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s) {
  if (h->prec == CONET_BF16 || h->prec == CONET_FP16 || h->prec == CONET_TF32X3 || h->prec == CONET_FP8E4M3)
    return net_forward_tc(h, Y, mask, B, llr, s);
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
      // the main activation after a concatenating fusion point is n_branches x width wide
      const bool wide_in = l > 0 && fused_width(h->cfg, l - 1) != h->C;
      for (int b = 0; b < nb; ++b) {
        c.in[b] = l == 0 ? h->X0 : (b == 0 ? (wide_in ? xcat_at(h, l - 1) : A.XM(l - 1)) : A.A(l - 1, b));
        c.w[b] = W(h, l == 0 ? L.in_w[b] : L.lw[b][l - 1]);
        c.bias[b] = P(h, l == 0 ? L.in_b[b] : L.lb[b][l - 1]);
        c.out0[b] = A.A(l, b);
      }
      c.relu0 = 1;
      if (wide_in)
        CONET_TRY(conv_layer_concat(h, c, s));
      else
        CONET_TRY(conv_layer(h, c, l == 0 ? h->c_pad : h->C, s));
      FuseArgs f = fuse_args(h, B);
      for (int b = 0; b < nb; ++b) f.u[b] = A.A(l, b);
      f.fuse = fused_at(h->cfg, l);
      f.fuse_g = P(h, L.fg[l]);
      f.fuse_b = P(h, L.fb[l]);
      f.x0_out = wide_at(h, l) ? xcat_at(h, l) : A.XM(l);
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
      CONET_TRY(resid_fuse(h, k, B, llr, s));
      if (k == depth) break;
      CONET_TRY(resid_conv1(h, k, B, s));
      CONET_TRY(resid_conv2(h, k, B, s));
    }
  }
  h->fwd_B = B;
  return CONET_OK;
}

// ------------------------------------------------------------------ tensor-core paths
namespace {

// tcgen05 operand kind of the handle's precision: 0 BF16, 3 FP16, 1 split TF32, 2 E4M3;
// -1 = SIMT path.
int tc_kind(const conet_s* h) {
  switch (h->prec) {
    case CONET_BF16: return 0;
    case CONET_FP16: return 3;
    case CONET_TF32X3: return 1;
    case CONET_FP8E4M3: return 2;
    default: return -1;
  }
}

int tc_elt(int kind) { return kind == 1 ? 4 : kind == 2 ? 1 : 2; }

// Padded input channels of the input layer: one MMA K step (32 bytes) of E4M3, 16 otherwise.
int tc_cin0(int kind) { return kind == 2 ? 32 : 16; }

// low part of the input buffer of conv launch idx (split TF32)
const void* tc_conv_in_lo(const conet_s* h, int idx, int b) {
  if (idx == 0) return h->X0b_lo;
  if (!h->cfg.residual) return h->nxb_lo[(idx - 1) & 1][b];
  return h->nxb_lo[(idx - 1) % 2 == 0 ? 0 : 1][b];
}

// conv launch index -> (per branch) master weight offset
long tc_conv_w(const conet_s* h, int idx, int b) {
  const Layout& L = h->L;
  if (idx == 0) return L.in_w[b];
  if (!h->cfg.residual) return L.lw[b][idx - 1];
  const int k = (idx - 1) / 2;
  return (idx - 1) % 2 == 0 ? L.blk[b][k].c1w : L.blk[b][k].c2w;
}

int tc_n_convs(const conet_s* h) { return h->cfg.residual ? 1 + 2 * h->cfg.depth : h->cfg.depth; }

// input buffer of conv launch idx for branch b
const void* tc_conv_in(const conet_s* h, int idx, int b) {
  if (idx == 0) return h->X0b;
  if (!h->cfg.residual) return h->nxb[(idx - 1) & 1][b];
  return h->nxb[(idx - 1) % 2 == 0 ? 0 : 1][b];
}

// E4M3 activation scales of the input of conv launch idx, branch b: records of C + 8 floats
// (scale, 1 / scale, padding, then dq[C] on a 32-byte boundary for the epilogue's 256-bit loads)
constexpr int FP8_REC_PAD = 8;
size_t fp8_rec(const conet_s* h, int idx, int b) { return ((size_t)idx * h->nb + b) * (size_t)(h->C + FP8_REC_PAD); }
float* fp8_scale(const conet_s* h, int idx, int b) { return h->fp8_act + fp8_rec(h, idx, b); }
float* fp8_qinv(const conet_s* h, int idx, int b) { return h->fp8_act + fp8_rec(h, idx, b) + 1; }
float* fp8_dq(const conet_s* h, int idx, int b) { return h->fp8_act + fp8_rec(h, idx, b) + FP8_REC_PAD; }
unsigned* fp8_amax(const conet_s* h, int idx, int b) { return h->fp8_amax + (size_t)idx * h->nb + b; }

}  // namespace

static TcConvArgs tc_args(conet_s* h, int idx, float* llr);

int tc_setup(conet_s* h) {
  if (tc_kind(h) < 0) return CONET_OK;
  const int kind = tc_kind(h);
  const int cin0 = tc_cin0(kind);
  if (h->cin > cin0) return fail(CONET_ERR_UNSUPPORTED, "tensor-core path takes at most %d input channels", cin0);
  if (h->C % 16) return fail(CONET_ERR_UNSUPPORTED, "tensor-core path needs width %% 16 == 0");
  if (kind == 2 && h->C % 32) return fail(CONET_ERR_UNSUPPORTED, "E4M3 path needs width %% 32 == 0");
  if (kind == 2 && h->cfg.train) return fail(CONET_ERR_UNSUPPORTED, "E4M3 handles are inference-only (train = 0)");
  if ((h->cfg.fuse_op || h->cfg.feedback) && tc_branch_groups(kind, h->nb, h->C) > 1)
    return fail(CONET_ERR_UNSUPPORTED, "sum interaction / feedback on a branch-group network (%d x %d)", h->nb, h->C);
  const size_t re = (size_t)h->chunk * h->T * h->F;
  const size_t e = (size_t)tc_elt(kind);
  const bool split = kind == 1;
  CONET_TRY(dev_alloc(h, &h->X0b, re * cin0 * e));
  if (split) CONET_TRY(dev_alloc(h, &h->X0b_lo, re * cin0 * e));
  for (int i = 0; i < 2; ++i)
    for (int b = 0; b < h->nb; ++b) {
      CONET_TRY(dev_alloc(h, &h->nxb[i][b], re * h->C * e));
      if (split) CONET_TRY(dev_alloc_t(h, &h->nxb_lo[i][b], re * h->C));
    }
  if (h->cfg.depthwise)
    for (int b = 0; b < h->nb; ++b) CONET_TRY(dev_alloc(h, &h->dwb[b], re * h->C * e));
  size_t wb = 0, ws = 0;
  for (const auto& c : h->L.convs) {
    const int cin_dst = c.cin == h->cin ? cin0 : c.cin;
    h->wb_off[c.off] = wb;
    wb += (size_t)c.taps * cin_dst * c.cout;
    h->fp8_ws_off[c.off] = ws;
    ws += (size_t)c.cout;
  }
  CONET_TRY(dev_alloc(h, &h->wb, wb * e));
  CONET_CUDA(cudaMemset(h->wb, 0, wb * e));
  if (split) {
    CONET_TRY(dev_alloc_t(h, &h->wb_lo, wb));
    CONET_CUDA(cudaMemset(h->wb_lo, 0, wb * sizeof(float)));
  }
  const int n = tc_n_convs(h);
  if (kind == 2) {
    CONET_TRY(dev_alloc_t(h, &h->fp8_wscale, ws));
    CONET_TRY(dev_alloc_t(h, &h->fp8_act, (size_t)n * h->nb * (h->C + FP8_REC_PAD)));
    CONET_TRY(dev_alloc_t(h, &h->fp8_amax, (size_t)n * h->nb));
    CONET_CUDA(cudaMemset(h->fp8_act, 0, (size_t)n * h->nb * (h->C + FP8_REC_PAD) * sizeof(float)));
  }
  // the whole-network kernel for small plain BF16 / E4M3 inference networks
  h->sn = (kind == 0 || kind == 2) && !h->cfg.train && !h->cfg.residual && !h->cfg.fuse_op && !h->cfg.feedback &&
          smallnet_eligible(kind, h->T, h->F, h->nb, h->C, h->cfg.depth, h->Q);
  if (h->sn) {
    const size_t xb = smallnet_input_bytes(h->chunk, h->T, h->F);
    CONET_TRY(dev_alloc(h, &h->sn_x, xb));
    CONET_CUDA(cudaMemset(h->sn_x, 0, xb));   // padding rows stay zero
    CONET_TRY(make_smallnet_input_map(&h->sn_xmap, kind, h->sn_x, h->chunk, h->T, h->F));
    for (int l = 0; l < h->cfg.depth; ++l)
      for (int b = 0; b < h->nb; ++b) {
        const int cin = l == 0 ? cin0 : h->C;
        const size_t woff = h->wb_off.at((size_t)tc_conv_w(h, l, b));
        CONET_TRY(make_weight_map(&h->sn_wmaps[l][b], kind, static_cast<const uint8_t*>(h->wb) + woff * e, cin, h->C,
                                  cin, h->C, 9));
      }
  }
  h->tcmaps.resize(n);
  for (int idx = 0; idx < n; ++idx) {
    const int cin = idx == 0 ? cin0 : h->C;
    // a depthwise-separable block conv: the 1x1 reads the depthwise output with one-tap boxes
    const bool pw = h->cfg.depthwise && idx > 0;
    const int kc = pw ? tc_chunk_pw(kind, h->nb, h->C) : tc_chunk(kind, h->nb, cin, h->C);
    const int taps = pw ? 1 : tc_taps(kind, h->nb, cin, h->C);
    const int wrows = tc_wbox_rows(kind, h->nb, cin, h->C), wtaps = pw ? 1 : tc_wbox_taps(kind, h->nb, cin, h->C);
    if (kc <= 0) return fail(CONET_ERR_UNSUPPORTED, "no tensor-core stage fits (kind %d, Cin %d, C %d)", kind, cin, h->C);
    for (int b = 0; b < h->nb; ++b) {
      const size_t woff = h->wb_off.at((size_t)tc_conv_w(h, idx, b));
      CONET_TRY(make_act_map(&h->tcmaps[idx].a[b], kind, pw ? h->dwb[b] : tc_conv_in(h, idx, b), cin, h->F, h->T,
                             h->chunk, kc, taps));
      CONET_TRY(make_weight_map(&h->tcmaps[idx].w[b], kind, static_cast<const uint8_t*>(h->wb) + woff * e, cin,
                                h->C, kc, wrows, wtaps, pw ? 1 : 9));
      if (split) {
        CONET_TRY(make_act_map(&h->tcmaps[idx].a_lo[b], kind, tc_conv_in_lo(h, idx, b), cin, h->F, h->T, h->chunk,
                               kc, taps));
        CONET_TRY(make_weight_map(&h->tcmaps[idx].w_lo[b], kind, h->wb_lo + woff, cin, h->C, kc, wrows, wtaps));
      }
    }
    // the staged stores' output maps (used by the fixed layer shapes only)
    const int cols = tc_store_cols(kind, h->nb, cin, h->C);
    if (cols > 0) {
      const TcConvArgs oa = tc_args(h, idx, nullptr);
      for (int b = 0; b < h->nb; ++b) {
        if (oa.xs_out[b])
          CONET_TRY(make_out_map(&h->tcmaps[idx].xs[b], -1, oa.xs_out[b], h->C, h->F, h->chunk * h->T, cols));
        if (oa.nx_out[b])
          CONET_TRY(make_out_map(&h->tcmaps[idx].nx[b], kind, oa.nx_out[b], h->C, h->F, h->chunk * h->T, cols));
      }
    }
  }
  return CONET_OK;
}

int tc_weights_changed(conet_s* h, cudaStream_t s) {
  const int kind = tc_kind(h);
  if (kind < 0) return CONET_OK;
  const float* pe = eff_params(h);
  for (const auto& c : h->L.convs) {
    const int cin_dst = c.cin == h->cin ? tc_cin0(kind) : c.cin;
    const size_t wo = h->wb_off.at(c.off);
    if (kind == 1)
      CONET_TRY(launch_weights_split(pe + c.off, c.cout, c.cin, cin_dst, static_cast<float*>(h->wb) + wo,
                                     h->wb_lo + wo, s));
    else if (kind == 2)
      CONET_TRY(launch_weights_fp8(pe + c.off, c.cout, c.cin, cin_dst, static_cast<uint8_t*>(h->wb) + wo,
                                   h->fp8_wscale + h->fp8_ws_off.at(c.off), s));
    else
      CONET_TRY(launch_weights_16(kind, pe + c.off, c.cout, c.cin, cin_dst, static_cast<uint16_t*>(h->wb) + wo, s,
                                  c.taps));
  }
  h->fp8_calibrated = false;   // activation ranges change with the weights
  return CONET_OK;
}

static int tc_conv(conet_s* h, int idx, TcConvArgs& a, int B, cudaStream_t s) {
  a.T = h->T;
  a.F = h->F;
  a.nfb = (h->F + 127) / 128;
  a.n_tiles = B * h->T * a.nfb;
  a.Q = h->Q;
  a.err = h->d_err;
  a.nonfinite = h->d_err + 1;
  const int cin = idx == 0 ? tc_cin0(tc_kind(h)) : h->C;
  prof_begin(h, idx == 0 ? PK_CONV_IN : PK_CONV, s);
  const int rc = launch_conv_tc(tc_kind(h), h->nb, cin, h->C, h->tcmaps[idx], a, s);
  prof_end(h, s);
  return rc;
}

// Arguments of conv launch idx of the forward pass over B slots.
static TcConvArgs tc_args(conet_s* h, int idx, float* llr) {
  const Acts A{h};
  const Layout& L = h->L;
  const int nb = h->nb, depth = h->cfg.depth;
  const bool train = h->cfg.train != 0;
  TcConvArgs a = {};
  if (!h->cfg.residual) {
    const int l = idx;
    for (int b = 0; b < nb; ++b) {
      a.bias[b] = P(h, l == 0 ? L.in_b[b] : L.lb[b][l - 1]);
      if (l + 1 < depth) {
        a.nx_out[b] = h->nxb[l & 1][b];
        a.nx_lo[b] = h->nxb_lo[l & 1][b];
      }
      if (train) a.a_out[b] = A.A(l, b);
    }
    if (train) a.xs_out[0] = A.XM(l);
    a.pre = 1;
    a.fuse = fused_at(h->cfg, l);
    a.op = a.fuse ? h->cfg.fuse_op : 0;
    a.feedback = a.fuse ? h->cfg.feedback : 0;
    a.lnf_g = P(h, L.fg[l]);
    a.lnf_b = P(h, L.fb[l]);
    if (l == depth - 1) {
      a.head_w = P(h, L.hw);
      a.head_b = P(h, L.hb);
      a.llr = llr;
    }
  } else {
    // input layer, then per block conv1 (LN2 + ReLU epilogue) and conv2 (residual add,
    // Hadamard fusion + LN, next pre-activation or head)
    const int k = (idx - 1) / 2;
    const bool conv1 = idx > 0 && (idx - 1) % 2 == 0;
    if (conv1) {
      for (int b = 0; b < nb; ++b) {
        a.bias[b] = P(h, L.blk[b][k].c1b);
        a.ln2_g[b] = P(h, L.blk[b][k].ln2g);
        a.ln2_b[b] = P(h, L.blk[b][k].ln2b);
        a.nx_out[b] = h->nxb[1][b];
        a.nx_lo[b] = h->nxb_lo[1][b];
      }
      a.pre = 2;
    } else {
      const int point = idx == 0 ? 0 : k + 1;        // fusion point after this conv
      for (int b = 0; b < nb; ++b) {
        a.bias[b] = P(h, idx == 0 ? L.in_b[b] : L.blk[b][k].c2b);
        if (idx > 0) a.resid[b] = h->act[(size_t)(k & 1) * nb + b];
        a.xs_out[b] = h->act[(size_t)(point & 1) * nb + b];
        if (point < depth) {
          a.nx_out[b] = h->nxb[0][b];
          a.nx_lo[b] = h->nxb_lo[0][b];
          const long g = L.blk[b][point].ln1g;
          a.post[b] = g >= 0 ? 2 : 1;
          a.ln1_g[b] = P(h, g);
          a.ln1_b[b] = P(h, L.blk[b][point].ln1b);
        }
      }
      a.pre = idx == 0 ? 1 : 0;
      a.fuse = fused_at(h->cfg, point);
      a.op = a.fuse ? h->cfg.fuse_op : 0;
      a.feedback = a.fuse ? h->cfg.feedback : 0;
      a.lnf_g = P(h, L.fg[point]);
      a.lnf_b = P(h, L.fb[point]);
      if (point == depth) {
        a.head_w = P(h, L.hw);
        a.head_b = P(h, L.hb);
        a.llr = llr;
      }
    }
  }
  if (tc_kind(h) == 2) {
    for (int b = 0; b < nb; ++b) {
      a.dq[b] = fp8_dq(h, idx, b);
      if (a.nx_out[b]) a.qinv[b] = fp8_qinv(h, idx + 1, b);
    }
  }
  return a;
}

// Activation scales of conv launch idx's input from the amax recorded for it.
static int fp8_set_scales(conet_s* h, int idx, float margin, cudaStream_t s) {
  Fp8ScaleArgs sa = {};
  for (int b = 0; b < h->nb; ++b) {
    sa.amax[b] = fp8_amax(h, idx, idx == 0 ? 0 : b);      // the input grid is shared by all branches
    sa.wscale[b] = h->fp8_wscale + h->fp8_ws_off.at((size_t)tc_conv_w(h, idx, b));
    sa.scale[b] = fp8_scale(h, idx, b);
    sa.qinv[b] = fp8_qinv(h, idx, b);
    sa.dq[b] = fp8_dq(h, idx, b);
  }
  return launch_fp8_scales(sa, h->nb, h->C, margin, s);
}

static int net_forward_tc_chunk(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, bool calibrate,
                                cudaStream_t s) {
  const int kind = tc_kind(h);
  const int n = tc_n_convs(h);
  const bool train = h->cfg.train != 0;
  if (train && h->cfg.residual) return fail(CONET_ERR_UNSUPPORTED, "tensor-core training of residual networks");
  prof_begin(h, PK_ASSEMBLE, s);
  if (kind == 1) {
    CONET_TRY(launch_assemble_split(Y, mask, h->psym, B, h->N, h->T, h->F, tc_cin0(kind), static_cast<float*>(h->X0b),
                                    static_cast<float*>(h->X0b_lo), s));
  } else if (kind == 2) {
    if (calibrate) {
      CONET_CUDA(cudaMemsetAsync(h->fp8_amax, 0, (size_t)n * h->nb * sizeof(unsigned), s));
      CONET_TRY(launch_assemble_fp8(Y, mask, h->psym, B, h->N, h->T, h->F, tc_cin0(kind), nullptr, nullptr,
                                    fp8_amax(h, 0, 0), s));
      CONET_TRY(fp8_set_scales(h, 0, h->fp8_margin, s));
    }
    CONET_TRY(launch_assemble_fp8(Y, mask, h->psym, B, h->N, h->T, h->F, tc_cin0(kind), fp8_qinv(h, 0, 0),
                                  static_cast<uint8_t*>(h->X0b), nullptr, s));
  } else {
    CONET_TRY(launch_assemble_16(kind, Y, mask, h->psym, B, h->N, h->T, h->F, tc_cin0(kind), h->X0b, s));
  }
  if (train) CONET_TRY(launch_assemble(Y, mask, h->psym, B, h->N, h->T, h->F, h->c_pad, h->X0, s));
  if (h->sn && llr && !calibrate && (h->whole_net == 2 || (h->whole_net == 1 && B >= CONET_WHOLE_NET_MIN_SLOTS))) {
    CONET_TRY(launch_smallnet_pad(h->X0b, h->sn_x, B, h->T, h->F, s));
    prof_end(h, s);
    // every layer and the head in one persistent kernel
    const Layout& L = h->L;
    SmallNetArgs sa = {};
    for (int l = 0; l < h->cfg.depth; ++l) {
      for (int b = 0; b < h->nb; ++b) sa.bias[l][b] = P(h, l == 0 ? L.in_b[b] : L.lb[b][l - 1]);
      sa.fuse[l] = fused_at(h->cfg, l);
      sa.lnf_g[l] = P(h, L.fg[l]);
      sa.lnf_b[l] = P(h, L.fb[l]);
      if (kind == 2)
        for (int b = 0; b < h->nb; ++b) {
          sa.dq[l][b] = fp8_dq(h, l, b);
          if (l > 0) sa.qinv[l][b] = fp8_qinv(h, l, b);
        }
    }
    sa.head_w = P(h, L.hw);
    sa.head_b = P(h, L.hb);
    sa.llr = llr;
    sa.err = h->d_err;
    sa.nonfinite = h->d_err + 1;
    sa.B = B;
    sa.T = h->T;
    sa.F = h->F;
    sa.Q = h->Q;
    sa.depth = h->cfg.depth;
    prof_begin(h, PK_CONV, s);
    const int rc = launch_smallnet(kind, h->sn_xmap, h->sn_wmaps, sa, s);
    prof_end(h, s);
    CONET_TRY(rc);
    h->fwd_B = B;
    return CONET_OK;
  }
  prof_end(h, s);
  for (int idx = 0; idx < n; ++idx) {
    TcConvArgs a = tc_args(h, idx, llr);
    if (calibrate && idx + 1 < n) {
      // measuring pass: the outputs' largest magnitude per branch, then the next input's scales
      TcConvArgs m = a;
      m.measure = 1;
      for (int b = 0; b < h->nb; ++b) m.amax[b] = m.nx_out[b] ? fp8_amax(h, idx + 1, b) : nullptr;
      CONET_TRY(tc_conv(h, idx, m, B, s));
      CONET_TRY(fp8_set_scales(h, idx + 1, h->fp8_margin, s));
    }
    if (idx + 1 == n && !llr) break;     // calibration only: the head's output is not needed
    if (h->cfg.depthwise && idx > 0) {
      // depthwise-separable block conv: the per-channel 3x3 into dwb, then the 1x1 below
      const int k = (idx - 1) / 2;
      DwArgs16 d = {};
      for (int b = 0; b < h->nb; ++b) {
        d.in[b] = tc_conv_in(h, idx, b);
        d.w[b] = P(h, (idx - 1) % 2 == 0 ? h->L.blk[b][k].c1d : h->L.blk[b][k].c2d);
        d.out[b] = h->dwb[b];
      }
      d.C = h->C;
      d.T = h->T;
      d.F = h->F;
      d.M = (long long)B * h->T * h->F;
      prof_begin(h, PK_CONV, s);
      const int rc = launch_dwconv3x3_16(kind, d, h->nb, s);
      prof_end(h, s);
      CONET_TRY(rc);
      a.taps = 1;
    }
    CONET_TRY(tc_conv(h, idx, a, B, s));
  }
  h->fwd_B = B;
  return CONET_OK;
}

int net_forward_tc(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s) {
  for (int c0 = 0; c0 < B; c0 += h->chunk) {
    const int Bc = B - c0 < h->chunk ? B - c0 : h->chunk;
    const bool calibrate = tc_kind(h) == 2 && !h->fp8_calibrated;
    CONET_TRY(net_forward_tc_chunk(h, Y + (size_t)c0 * h->N * h->T * h->F * 2, mask, Bc,
                                   llr + (size_t)c0 * h->T * h->F * h->Q, calibrate, s));
    if (calibrate) h->fp8_calibrated = true;
  }
  h->fwd_B = B;
  return CONET_OK;
}

// E4M3 activation scales from B slots (at most one chunk): the forward pass up to the last
// conv, every conv run once more beforehand to measure its outputs' range.
int net_calibrate(conet_s* h, const float* Y, const uint8_t* mask, int B, float margin, cudaStream_t s) {
  if (tc_kind(h) != 2) return CONET_OK;
  h->fp8_margin = margin;
  const int Bc = B < h->chunk ? B : h->chunk;
  CONET_TRY(net_forward_tc_chunk(h, Y, mask, Bc, nullptr, true, s));
  h->fp8_calibrated = true;
  h->fwd_B = 0;
  return CONET_OK;
}

// ------------------------------------------------------------------ backward
namespace {

struct Bwd {
  conet_s* h;
  cudaStream_t s;
  long long M;

  int reduce_ew(int n, long off) {   // sum the elementwise kernels' partials into grads[off..off+n)
    return launch_reduce_partials(h->ew_part, ew_grid(M), n, h->grads + off, 0, s);
  }
  int bias(const float* g, long off) {
    CONET_TRY(launch_channel_sums(g, M, h->C, h->ew_part, s));
    return reduce_ew(h->C, off);
  }
  // weight + bias gradients of one conv layer of every branch (or of branches b0 .. b0 +
  // nbr - 1, whose input has cin channels: the main's layer after a concatenation)
  int wgrad(const float* const* x, const float* const* g, bool input_layer, const long* w_off, const long* b_off,
            int b0 = 0, int nbr = 0, int cin = 0) {
    if (!nbr) nbr = h->nb;
    const int cin_pad = cin ? cin : input_layer ? h->c_pad : h->C;
    WgradArgs w = {};
    for (int i = 0; i < nbr; ++i) {
      const int b = b0 + i;
      w.x[i] = x[b];
      w.g[i] = g[b];
      w.dW[i] = h->grads + w_off[b];
      w.cin_src[i] = cin ? cin : input_layer ? h->cin : h->C;
    }
    w.part = h->wg_part;
    w.cin = cin_pad;
    w.cout = h->C;
    w.n_br = nbr;
    w.T = h->T;
    w.F = h->F;
    w.M = M;
    prof_begin(h, PK_BACKWARD, s);
    // BF16 training: BF16 operands on the tensor cores where the shape is instantiated
    const int rc = h->tc_dgrad && wgrad_tc_supported(cin_pad, h->C, h->F)
                       ? launch_wgrad_tc(w, (int)(M / ((long long)h->T * h->F)), h->wg_tc, h->d_err, s)
                       : launch_wgrad_tiled(w, s);
    prof_end(h, s);
    CONET_TRY(rc);
    for (int b = b0; b < b0 + nbr; ++b) CONET_TRY(bias(g[b], b_off[b]));
    return CONET_OK;
  }
  // tensor maps of the BF16 dgrad conv of one layer (built on first use; host-side encoding)
  int dg_maps_for(const long* w_off, const TcMaps** out) {
    auto it = h->dg_index.find((size_t)w_off[0]);
    if (it == h->dg_index.end()) {
      TcMaps m = {};
      const int C = h->C, nb = h->nb;
      const int kc = tc_chunk(0, nb, C, C), taps = tc_taps(0, nb, C, C);
      const int wrows = tc_wbox_rows(0, nb, C, C), wtaps = tc_wbox_taps(0, nb, C, C);
      if (kc <= 0) return fail(CONET_ERR_UNSUPPORTED, "no tensor-core stage fits the dgrad conv (C %d)", C);
      for (int b = 0; b < nb; ++b) {
        CONET_TRY(make_act_map(&m.a[b], 0, h->g16[b], C, h->F, h->T, h->chunk, kc, taps));
        CONET_TRY(make_weight_map(&m.w[b], 0, static_cast<const uint16_t*>(h->wd16) + h->wd_off.at((size_t)w_off[b]),
                                  C, C, kc, wrows, wtaps));
      }
      h->dg_maps.push_back(m);
      it = h->dg_index.emplace((size_t)w_off[0], h->dg_maps.size() - 1).first;
    }
    *out = &h->dg_maps[it->second];
    return CONET_OK;
  }
  // data gradient of a body conv of every branch: out = conv3x3(g, rotated W); with BF16
  // training on the tensor cores (BF16 operands, FP32 accumulation and output).  FP32: or of
  // branches b0 .. b0 + nbr - 1 with cout-channel outputs (the main's concatenated input).
  int dgrad(float* const* g, const long* w_off, float* const* out, int b0 = 0, int nbr = 0, int cout = 0) {
    if (h->tc_dgrad) {
      const TcMaps* maps = nullptr;
      CONET_TRY(dg_maps_for(w_off, &maps));
      CONET_TRY(launch_grads_bf16(g, h->g16, h->nb, M * h->C, s));
      TcConvArgs a = {};
      a.T = h->T;
      a.F = h->F;
      a.nfb = (h->F + 127) / 128;
      a.n_tiles = (int)(M / ((long long)h->T * h->F)) * h->T * a.nfb;
      a.Q = h->Q;
      a.err = h->d_err;
      a.nonfinite = h->d_err + 1;
      for (int b = 0; b < h->nb; ++b) {
        a.bias[b] = h->zero_c;
        a.t_out[b] = out[b];
      }
      prof_begin(h, PK_BACKWARD, s);
      const int rc = launch_conv_tc(0, h->nb, h->C, h->C, *maps, a, s);
      prof_end(h, s);
      return rc;
    }
    if (!nbr) nbr = h->nb;
    ConvArgs c = {};
    c.M = (int)M;
    c.T = h->T;
    c.F = h->F;
    for (int i = 0; i < nbr; ++i) {
      c.in[i] = g[b0 + i];
      c.w[i] = h->wd + h->wd_off.at((size_t)w_off[b0 + i]);
      c.out0[i] = out[b0 + i];
    }
    prof_begin(h, PK_BACKWARD, s);
    const int rc = launch_conv3x3_fp32(c, nbr, h->C, cout ? cout : h->C, s);
    prof_end(h, s);
    return rc;
  }
  // gradients of a depthwise-separable block conv of every branch (x: its input, g: the
  // gradient of its output, out: the gradient of x), with dw_out as the scratch of the
  // per-channel 3x3's output z and then of its gradient dz
  int sep(const float* const* x, float* const* g, const long* d_off, const long* w_off, const long* b_off,
          float* const* out) {
    const int nb = h->nb, C = h->C;
    DwArgs z = {};
    for (int b = 0; b < nb; ++b) {
      z.in[b] = x[b];
      z.w[b] = P(h, d_off[b]);
      z.out[b] = h->dw_out[b];
    }
    z.C = C;
    z.T = h->T;
    z.F = h->F;
    z.M = M;
    Wgrad1x1Args w = {};
    DwWgradArgs v = {};
    ConvArgs c = {};
    DwArgs d = z;
    for (int b = 0; b < nb; ++b) {
      w.g[b] = g[b];
      w.z[b] = h->dw_out[b];
      w.dW[b] = h->grads + w_off[b];
      c.in[b] = g[b];
      c.w[b] = P(h, w_off[b]);   // master [Cout][Cin]: the one-tap conv's [1][K = Cout][N = Cin]
      c.out0[b] = h->dw_out[b];
      v.x[b] = x[b];
      v.dz[b] = h->dw_out[b];
      v.dWd[b] = h->grads + d_off[b];
      d.in[b] = h->dw_out[b];
      d.out[b] = out[b];
    }
    w.part = v.part = h->wg_part;
    w.C = v.C = C;
    w.n_br = v.n_br = nb;
    w.M = v.M = M;
    v.T = h->T;
    v.F = h->F;
    c.M = (int)M;
    c.T = h->T;
    c.F = h->F;
    c.taps = 1;
    d.flip = 1;
    prof_begin(h, PK_BACKWARD, s);
    int rc = launch_dwconv3x3(z, nb, s);                                  // z
    if (rc == CONET_OK) rc = launch_wgrad1x1(w, s);                        // d W1
    if (rc == CONET_OK) rc = launch_conv3x3_fp32(c, nb, C, C, s);          // dz = g W1
    if (rc == CONET_OK) rc = launch_dw_wgrad(v, s);                        // d Wd
    if (rc == CONET_OK) rc = launch_dwconv3x3(d, nb, s);                   // dx
    prof_end(h, s);
    CONET_TRY(rc);
    for (int b = 0; b < nb; ++b) CONET_TRY(bias(g[b], b_off[b]));
    return CONET_OK;
  }
  int fuse(const float* const* u, const float* gx0, float* const* gxs, float* const* gu, int point, int relu_mask) {
    FuseBwdArgs f = {};
    for (int b = 0; b < h->nb; ++b) {
      f.u[b] = u[b];
      f.gu[b] = gu[b];
      f.gxs[b] = b ? gxs[b] : nullptr;
    }
    f.gx0 = gx0;
    f.ln_g = P(h, h->L.fg[point]);
    f.part = f.ln_g ? h->ew_part : nullptr;
    f.n_br = h->nb;
    f.fuse = fused_at(h->cfg, point);
    f.relu_mask = relu_mask;
    f.op = h->cfg.fuse_op;
    f.feedback = h->cfg.feedback;
    f.C = h->C;
    f.M = M;
    CONET_TRY(launch_fuse_bwd(f, s));
    if (f.ln_g) CONET_TRY(reduce_ew(2 * fused_width(h->cfg, point), h->L.fg[point]));
    return CONET_OK;
  }
  int ln_relu(const float* g, const float* x, long lng, long lnb, const float* add, float* out) {
    LnReluBwdArgs a = {};
    a.g = g;
    a.x = x;
    a.ln_g = P(h, lng);
    a.ln_b = P(h, lnb);
    a.add = add;
    a.out = out;
    a.part = a.ln_g ? h->ew_part : nullptr;
    a.C = h->C;
    a.M = M;
    CONET_TRY(launch_ln_relu_bwd(a, s));
    if (a.ln_g) CONET_TRY(reduce_ew(2 * h->C, lng));
    return CONET_OK;
  }
};

}  // namespace

int net_backward(conet_s* h, const float* dllr, int B, cudaStream_t s) {
  if (h->prec != CONET_FP32 && (h->prec == CONET_FP8E4M3 || h->cfg.residual))
    return fail(CONET_ERR_UNSUPPORTED, "precision %d backward of this network not built yet", h->prec);
  const Acts A{h};
  const Layout& L = h->L;
  const int nb = h->nb, depth = h->cfg.depth, C = h->C;
  Bwd bw{h, s, (long long)B * h->T * h->F};
  float* const* G0 = h->G[0];
  float* const* G1 = h->G[1];
  float* const* G2 = h->G[2];
  float* nulw[MAX_BR] = {};
  // head: grad wrt the head input, dW_h and db_h (stored contiguously)
  // (plain networks whose last layer concatenates: the head reads n_branches x width channels)
  const bool wide_head = !h->cfg.residual && wide_at(h, depth - 1);
  const int head_c = wide_head ? nb * C : C;
  HeadBwdArgs hb = {};
  hb.dllr = dllr;
  hb.x0 = h->cfg.residual ? A.RXM(depth) : wide_head ? xcat_at(h, depth - 1) : A.XM(depth - 1);
  hb.w = P(h, L.hw);
  hb.gx0 = wide_head ? h->gcat : G0[0];
  hb.part = h->ew_part;
  hb.C = head_c;
  hb.Q = h->Q;
  hb.M = bw.M;
  CONET_TRY(launch_head_bwd(hb, s));
  CONET_TRY(bw.reduce_ew(h->Q * head_c + h->Q, L.hw));
  long w_off[MAX_BR], b_off[MAX_BR];
  if (!h->cfg.residual) {
    float* const* gxs = nulw;   // support gradients entering the top layer: zero
    // with the concatenation interaction the main's fused activations and their gradients
    // (gcat) are n_branches x width wide, and the main's convs after them run on their own
    float* gmain[MAX_BR];
    for (int b = 0; b < nb; ++b) gmain[b] = G0[b];
    for (int l = depth - 1; l >= 0; --l) {
      const float* u[MAX_BR];
      for (int b = 0; b < nb; ++b) u[b] = A.A(l, b);
      CONET_TRY(bw.fuse(u, wide_at(h, l) ? h->gcat : G0[0], gxs, G1, l, 1));
      const bool wide_in = l > 0 && wide_at(h, l - 1);
      const float* x[MAX_BR];
      for (int b = 0; b < nb; ++b) {
        x[b] = l == 0 ? h->X0 : (b == 0 ? (wide_in ? xcat_at(h, l - 1) : A.XM(l - 1)) : A.A(l - 1, b));
        w_off[b] = l == 0 ? L.in_w[b] : L.lw[b][l - 1];
        b_off[b] = l == 0 ? L.in_b[b] : L.lb[b][l - 1];
      }
      if (wide_in) {
        CONET_TRY(bw.wgrad(x, G1, false, w_off, b_off, 0, 1, nb * C));
        CONET_TRY(bw.wgrad(x, G1, false, w_off, b_off, 1, nb - 1));
      } else {
        CONET_TRY(bw.wgrad(x, G1, l == 0, w_off, b_off));
      }
      if (l > 0) {
        if (wide_in) {
          gmain[0] = h->gcat;
          CONET_TRY(bw.dgrad(G1, w_off, gmain, 0, 1, nb * C));
          CONET_TRY(bw.dgrad(G1, w_off, G0, 1, nb - 1));
        } else {
          CONET_TRY(bw.dgrad(G1, w_off, G0));
        }
        gxs = G0;
      }
    }
  } else {
    float* const* gxs = nulw;
    for (int k = depth; k >= 1; --k) {
      const int blk = k - 1;
      if (A.rc()) {
        // this block's pre-activation, first conv and normalisation again, from the stored
        // streams, by the forward's own kernels (bitwise the forward's values)
        CONET_TRY(resid_fuse(h, blk, B, nullptr, s));
        CONET_TRY(resid_conv1(h, blk, B, s));
      }
      const float* u[MAX_BR];
      for (int b = 0; b < nb; ++b) u[b] = A.U(blk, b);
      CONET_TRY(bw.fuse(u, G0[0], gxs, G1, k, 0));                       // G1 = d u
      const float* x[MAX_BR];
      long d_off[MAX_BR];
      const bool sep = h->cfg.depthwise != 0;
      // conv2: input h2, output gradient d u
      for (int b = 0; b < nb; ++b) {
        x[b] = A.H2(blk, b);
        w_off[b] = L.blk[b][blk].c2w;
        b_off[b] = L.blk[b][blk].c2b;
        d_off[b] = L.blk[b][blk].c2d;
      }
      if (sep) {
        CONET_TRY(bw.sep(x, G1, d_off, w_off, b_off, G2));               // G2 = d h2
      } else {
        CONET_TRY(bw.wgrad(x, G1, false, w_off, b_off));
        CONET_TRY(bw.dgrad(G1, w_off, G2));                             // G2 = d h2
      }
      for (int b = 0; b < nb; ++b)                                      // G0 = d t1
        CONET_TRY(bw.ln_relu(G2[b], A.T1(blk, b), L.blk[b][blk].ln2g, L.blk[b][blk].ln2b, nullptr, G0[b]));
      for (int b = 0; b < nb; ++b) {
        x[b] = A.H1(blk, b);
        w_off[b] = L.blk[b][blk].c1w;
        b_off[b] = L.blk[b][blk].c1b;
        d_off[b] = L.blk[b][blk].c1d;
      }
      if (sep) {
        CONET_TRY(bw.sep(x, G0, d_off, w_off, b_off, G2));               // G2 = d h1
      } else {
        CONET_TRY(bw.wgrad(x, G0, false, w_off, b_off));
        CONET_TRY(bw.dgrad(G0, w_off, G2));                             // G2 = d h1
      }
      for (int b = 0; b < nb; ++b)                                      // G0 = d x (skip + pre-act)
        CONET_TRY(bw.ln_relu(G2[b], A.XS(blk, b), L.blk[b][blk].ln1g, L.blk[b][blk].ln1b, G1[b], G0[b]));
      gxs = G0;
    }
    const float* u[MAX_BR];
    for (int b = 0; b < nb; ++b) u[b] = A.A0(b);
    CONET_TRY(bw.fuse(u, G0[0], gxs, G1, 0, 1));
    const float* x[MAX_BR];
    for (int b = 0; b < nb; ++b) {
      x[b] = h->X0;
      w_off[b] = L.in_w[b];
      b_off[b] = L.in_b[b];
    }
    CONET_TRY(bw.wgrad(x, G1, true, w_off, b_off));
  }
  return zero_withheld_inputs(h, h->grads, s);   // their gradient is zero
}

int net_adam(conet_s* h, float lr, int step, cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - pow(b1, step)), bc2 = (float)(1.0 - pow(b2, step));
  prof_begin(h, PK_ADAM, s);
  const int rc = launch_adam(h->params, h->grads, h->adam_m, h->adam_v, h->L.total, lr, (float)b1, (float)b2, 1e-8f,
                             bc1, bc2, s);
  prof_end(h, s);
  CONET_TRY(rc);
  return net_weights_changed(h, s);
}

int net_train_step(conet_s* h, const SimArgs& a0, uint64_t step, int B, float lr, double* loss_out, cudaStream_t s) {
  SimArgs a = a0;
  a.Y = h->sim_Y;
  a.bits = h->sim_bits;
  a.H = nullptr;
  a.noise_var = h->sim_nv;
  a.interf_var = nullptr;
  CONET_TRY(launch_sim(a, B, s));
  CONET_TRY(net_forward(h, h->sim_Y, h->mask, B, h->llr, s));
  const double count = (double)B * ((double)h->T * h->F - h->n_pilot_re) * h->Q;
  CONET_CUDA(cudaMemsetAsync(h->d_loss, 0, sizeof(double), s));
  CONET_TRY(launch_loss_ber(h->llr, h->sim_bits, h->mask, B, h->T, h->F, h->Q, (float)(1.0 / count), h->dllr,
                            h->d_loss, nullptr, nullptr, s));
  CONET_TRY(net_backward(h, h->dllr, B, s));
  CONET_TRY(net_adam(h, lr, (int)(step + 1), s));
  if (loss_out) {
    double v = 0.0;
    CONET_CUDA(cudaMemcpyAsync(&v, h->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    CONET_CUDA(cudaStreamSynchronize(s));
    *loss_out = v / count;
    if (!isfinite(*loss_out)) return fail(CONET_ERR_NONFINITE, "training loss is not finite");
  }
  return CONET_OK;
}

}  // namespace conet
