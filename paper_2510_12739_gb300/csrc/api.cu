// C ABI of libconet (include/conet.h): handle lifecycle, parameter layout, and the host
// orchestration of the device kernels for each entry point.  Host code validates every
// argument before the first launch; the kernels do all the arithmetic of the path.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "net.cuh"

namespace conet {

static thread_local std::string g_err = "no error";

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CONET_OK;
  return fail(CONET_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static unsigned long long g_launches = 0;   // host-side count of kernel launches

int check_launch(const char* what) {
  __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
  return check_cuda(cudaGetLastError(), what);
}

unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
void launch_count_add(long long n) { __atomic_add_fetch(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }

// ------------------------------------------------------------------ parameter layout
bool fused_at(const conet_config& c, int i) {
  if (c.resnet_baseline || c.n_branches < 2) return false;
  if (c.fuse_mask < 0) return true;
  return (c.fuse_mask >> i) & 1;
}

// Channels of the main activation after fusion point i: n_branches x width where the point
// concatenates (fuse_op 2, plain networks), else width.
int fused_width(const conet_config& c, int i) {
  return c.fuse_op == 2 && fused_at(c, i) ? c.n_branches * c.width : c.width;
}

Layout build_layout(const conet_config& c) {
  Layout L;
  const int C = c.width, Q = c.qam_bits, cin = 2 * c.n_rx + 3;
  size_t o = 0;
  auto take = [&](size_t n, int kind, float stdv) {
    L.segs.push_back({o, n, kind, stdv});
    const size_t r = o;
    o += n;
    return (long)r;
  };
  auto conv = [&](int ci, int co, long* w, long* b) {
    *w = take((size_t)co * 9 * ci, 0, sqrtf(2.0f / (9.0f * ci)));
    *b = take((size_t)co, 2, 0.f);
    L.convs.push_back({(size_t)*w, co, ci, 9});
  };
  // depthwise-separable: per-channel 3x3 [C][3][3] (He, fan-in 9), then 1x1 [C][C] + bias
  auto sep_conv = [&](long* d, long* w, long* b) {
    *d = take((size_t)C * 9, 0, sqrtf(2.0f / 9.0f));
    *w = take((size_t)C * C, 0, sqrtf(2.0f / C));
    *b = take((size_t)C, 2, 0.f);
    L.convs.push_back({(size_t)*w, C, C, 1});
  };
  auto ln = [&](long* g, long* b) {
    *g = take((size_t)C, 1, 0.f);
    *b = take((size_t)C, 2, 0.f);
  };
  for (int b = 0; b < c.n_branches; ++b) {
    conv(cin, C, &L.in_w[b], &L.in_b[b]);
    if (!c.residual) {
      for (int l = 1; l < c.depth; ++l) {
        long w, bb;
        conv(b == 0 ? fused_width(c, l - 1) : C, C, &w, &bb);
        L.lw[b].push_back(w);
        L.lb[b].push_back(bb);
      }
    } else {
      for (int k = 0; k < c.depth; ++k) {
        BlockOff B;
        if (b >= 1 || c.resnet_baseline) ln(&B.ln1g, &B.ln1b);
        if (c.depthwise) sep_conv(&B.c1d, &B.c1w, &B.c1b);
        else conv(C, C, &B.c1w, &B.c1b);
        ln(&B.ln2g, &B.ln2b);
        if (c.depthwise) sep_conv(&B.c2d, &B.c2w, &B.c2b);
        else conv(C, C, &B.c2w, &B.c2b);
        L.blk[b].push_back(B);
      }
    }
  }
  const int n_points = c.residual ? c.depth + 1 : c.depth;
  for (int i = 0; i < n_points; ++i) {
    long g = -1, bb = -1;
    if (c.norm && fused_at(c, i)) {
      g = take((size_t)fused_width(c, i), 1, 0.f);
      bb = take((size_t)fused_width(c, i), 2, 0.f);
    }
    L.fg.push_back(g);
    L.fb.push_back(bb);
  }
  const int head_c = c.residual ? C : fused_width(c, c.depth - 1);
  L.hw = take((size_t)Q * head_c, 0, sqrtf(2.0f / head_c));
  L.hb = take((size_t)Q, 2, 0.f);
  L.total = o;
  return L;
}

static int validate_config(const conet_config* c) {
  if (!c) return fail(CONET_ERR_ARG, "config is NULL");
  if (c->n_rx < 1 || c->n_rx > 6) return fail(CONET_ERR_ARG, "n_rx %d outside 1..6", c->n_rx);
  if (c->n_sym < 1 || c->n_sc < 1) return fail(CONET_ERR_ARG, "empty grid %dx%d", c->n_sym, c->n_sc);
  if (c->qam_bits < 2 || c->qam_bits > 8 || (c->qam_bits & 1))
    return fail(CONET_ERR_ARG, "qam_bits %d not in {2,4,6,8}", c->qam_bits);
  if (c->n_branches < 1 || c->n_branches > MAX_BR) return fail(CONET_ERR_ARG, "n_branches %d outside 1..4", c->n_branches);
  if (c->depth < 1 || c->depth > 64) return fail(CONET_ERR_ARG, "depth %d outside 1..64", c->depth);
  if (c->width < 1 || c->width > 128) return fail(CONET_ERR_ARG, "width %d outside 1..128", c->width);
  if (c->resnet_baseline && (c->n_branches != 1 || !c->residual))
    return fail(CONET_ERR_ARG, "resnet_baseline needs n_branches = 1 and residual = 1");
  if (c->n_pilot_syms < 1 || c->n_pilot_syms > 4) return fail(CONET_ERR_ARG, "n_pilot_syms %d outside 1..4", c->n_pilot_syms);
  for (int i = 0; i < c->n_pilot_syms; ++i) {
    if (c->pilot_syms[i] < 0 || c->pilot_syms[i] >= c->n_sym) return fail(CONET_ERR_ARG, "pilot symbol %d outside grid", c->pilot_syms[i]);
    if (i && c->pilot_syms[i] <= c->pilot_syms[i - 1]) return fail(CONET_ERR_ARG, "pilot symbols must increase");
  }
  if (c->pilot_comb < 1) return fail(CONET_ERR_ARG, "pilot_comb %d < 1", c->pilot_comb);
  if (c->fuse_op < 0 || c->fuse_op > 2) return fail(CONET_ERR_ARG, "fuse_op %d not in {0, 1, 2}", c->fuse_op);
  if (c->fuse_op == 2 && c->residual)
    return fail(CONET_ERR_ARG, "concatenation (fuse_op 2) fuses plain networks only");
  if (c->fuse_op == 2 && c->n_branches * c->width > 128)
    return fail(CONET_ERR_ARG, "concatenated width %d > 128", c->n_branches * c->width);
  if (c->feedback < 0 || c->feedback > 1) return fail(CONET_ERR_ARG, "feedback %d not in {0, 1}", c->feedback);
  if (c->depthwise < 0 || c->depthwise > 1) return fail(CONET_ERR_ARG, "depthwise %d not in {0, 1}", c->depthwise);
  if (c->support_inputs < 0 || c->support_inputs > 1)
    return fail(CONET_ERR_ARG, "support_inputs %d not in {0, 1}", c->support_inputs);
  if (c->support_inputs && c->n_branches < 2) return fail(CONET_ERR_ARG, "support_inputs needs a support net");
  if (c->support_mask && !c->support_inputs) return fail(CONET_ERR_ARG, "support_mask needs support_inputs = 1");
  if (c->support_mask >> (2 * c->n_rx + 3))
    return fail(CONET_ERR_ARG, "support_mask 0x%x names channels beyond the %d inputs", c->support_mask, 2 * c->n_rx + 3);
  return CONET_OK;
}

static PilotGrid pilot_grid_of(const conet_config& c) {
  PilotGrid pg;
  for (int i = 0; i < 4; ++i) pg.syms[i] = i < c.n_pilot_syms ? c.pilot_syms[i] : -1;
  pg.n_syms = c.n_pilot_syms;
  pg.comb = c.pilot_comb;
  pg.k0 = (uint32_t)c.pilot_seed;
  pg.k1 = (uint32_t)(c.pilot_seed >> 32);
  return pg;
}

}  // namespace conet

using namespace conet;

extern "C" {

const char* conet_last_error(void) { return g_err.c_str(); }

unsigned long long conet_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int conet_sync(conet_t h, void* stream) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  CONET_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int e[2] = {0, 0};
  CONET_CUDA(cudaMemcpy(e, h->d_err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e[0] || e[1]) CONET_CUDA(cudaMemset(h->d_err, 0, sizeof(e)));
  if (e[0]) return fail(CONET_ERR_TIMEOUT, "a device pipeline wait timed out (site %d)", e[0]);
  if (e[1]) return fail(CONET_ERR_NONFINITE, "a forward pass wrote a NaN or infinite LLR");
  return CONET_OK;
}

int conet_profile_enable(conet_t h, int enable) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  CONET_CUDA(cudaDeviceSynchronize());
  h->prof_kind.clear();
  h->prof_open = -1;
  h->prof_on = enable != 0;
  return CONET_OK;
}

int conet_profile_read(conet_t h, int kind, double* total_ms, long long* launches) {
  if (!h || !total_ms || !launches) return fail(CONET_ERR_ARG, "NULL argument");
  if (kind < 0 || kind >= PK_N) return fail(CONET_ERR_ARG, "profile kind %d outside 0..%d", kind, PK_N - 1);
  CONET_CUDA(cudaDeviceSynchronize());
  double ms = 0.0;
  long long n = 0;
  for (size_t i = 0; i < h->prof_kind.size(); ++i) {
    if (h->prof_kind[i] != kind) continue;
    float e = 0.f;
    CONET_CUDA(cudaEventElapsedTime(&e, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    ms += e;
    ++n;
  }
  *total_ms = ms;
  *launches = n;
  return CONET_OK;
}

int conet_param_count(const conet_config* cfg, size_t* n_out) {
  CONET_TRY(validate_config(cfg));
  if (!n_out) return fail(CONET_ERR_ARG, "n_out is NULL");
  *n_out = build_layout(*cfg).total;
  return CONET_OK;
}

void conet_destroy(conet_t h) {
  if (!h) return;
  net_graph_reset(h);
  if (h->g_stream) cudaStreamDestroy(h->g_stream);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

int conet_create(const conet_config* cfg, int precision, conet_t* out) {
  CONET_TRY(validate_config(cfg));
  if (!out) return fail(CONET_ERR_ARG, "out is NULL");
  if (cfg->max_batch < 1) return fail(CONET_ERR_SHAPE, "max_batch %d < 1", cfg->max_batch);
  if (precision != CONET_FP32 && precision != CONET_BF16 && precision != CONET_FP8E4M3 && precision != CONET_FP16 &&
      precision != CONET_TF32X3)
    return fail(CONET_ERR_ARG, "unknown precision %d", precision);
  conet_s* h = new conet_s();
  h->cfg = *cfg;
  h->prec = precision;
  h->L = build_layout(*cfg);
  h->T = cfg->n_sym;
  h->F = cfg->n_sc;
  h->N = cfg->n_rx;
  h->Q = cfg->qam_bits;
  h->C = cfg->width;
  h->nb = cfg->n_branches;
  h->cin = 2 * cfg->n_rx + 3;
  h->c_pad = (h->cin + 3) / 4 * 4;
  int rc = net_setup(h);
  if (rc != CONET_OK) {
    const std::string msg = g_err;
    conet_destroy(h);
    g_err = msg;
    return rc;
  }
  *out = h;
  return CONET_OK;
}

int conet_init_he(conet_t h, uint64_t seed, void* stream) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  for (const auto& sg : h->L.segs) {
    CONET_TRY(launch_init_segment(h->params, sg.off, sg.n, sg.stdv, sg.kind == 1 ? 1.f : 0.f, sg.kind == 0, seed, s));
  }
  CONET_CUDA(cudaMemsetAsync(h->adam_m, 0, h->L.total * sizeof(float), s));
  CONET_CUDA(cudaMemsetAsync(h->adam_v, 0, h->L.total * sizeof(float), s));
  return net_weights_changed(h, s);
}

int conet_load_weights(conet_t h, const float* host_params, size_t n) {
  if (!h || !host_params) return fail(CONET_ERR_ARG, "NULL argument");
  if (n != h->L.total) return fail(CONET_ERR_WEIGHTS, "weight vector has %zu floats, network needs %zu", n, h->L.total);
  CONET_CUDA(cudaMemcpy(h->params, host_params, n * sizeof(float), cudaMemcpyHostToDevice));
  CONET_CUDA(cudaMemset(h->adam_m, 0, n * sizeof(float)));
  CONET_CUDA(cudaMemset(h->adam_v, 0, n * sizeof(float)));
  CONET_TRY(net_weights_changed(h, 0));
  CONET_CUDA(cudaDeviceSynchronize());
  return CONET_OK;
}

int conet_save_weights(conet_t h, float* host_params, size_t n) {
  if (!h || !host_params) return fail(CONET_ERR_ARG, "NULL argument");
  if (n != h->L.total) return fail(CONET_ERR_WEIGHTS, "buffer has %zu floats, network has %zu", n, h->L.total);
  CONET_CUDA(cudaDeviceSynchronize());
  CONET_CUDA(cudaMemcpy(host_params, h->params, n * sizeof(float), cudaMemcpyDeviceToHost));
  return CONET_OK;
}

int conet_params_device(conet_t h, float** p, size_t* n) {
  if (!h || !p || !n) return fail(CONET_ERR_ARG, "NULL argument");
  *p = h->params;
  *n = h->L.total;
  return CONET_OK;
}

int conet_params_updated(conet_t h, void* stream) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  return net_weights_changed(h, (cudaStream_t)stream);
}

int conet_grads_device(conet_t h, float** p, size_t* n) {
  if (!h || !p || !n) return fail(CONET_ERR_ARG, "NULL argument");
  *p = h->grads;
  *n = h->L.total;
  return CONET_OK;
}

int conet_forward(conet_t h, const float* Y, const uint8_t* pilot_mask, const float* noise_var, int B, float* llr,
                  void* stream) {
  (void)noise_var;
  if (!h || !Y || !pilot_mask || !llr) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1 || B > h->cfg.max_batch) return fail(CONET_ERR_SHAPE, "B = %d outside 1..max_batch (%d)", B, h->cfg.max_batch);
  return net_forward_replay(h, Y, pilot_mask, B, llr, (cudaStream_t)stream);
}

int conet_whole_network(conet_t h, int enable, int* available) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  net_graph_reset(h);
  if (enable < 0 || enable > 2) return fail(CONET_ERR_ARG, "enable = %d outside 0..2", enable);
  h->whole_net = enable;
  if (available) *available = h->sn ? 1 : 0;
  return CONET_OK;
}

int conet_graphs(conet_t h, int enable) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  net_graph_reset(h);
  h->graphs = enable != 0;
  return CONET_OK;
}

int conet_calibrate(conet_t h, const float* Y, const uint8_t* pilot_mask, int B, float margin, void* stream) {
  if (!h || !Y || !pilot_mask) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1 || B > h->cfg.max_batch) return fail(CONET_ERR_SHAPE, "B = %d outside 1..max_batch (%d)", B, h->cfg.max_batch);
  if (!(margin >= 1.f) || !(margin <= 448.f)) return fail(CONET_ERR_ARG, "margin %g outside [1, 448]", (double)margin);
  return net_calibrate(h, Y, pilot_mask, B, margin, (cudaStream_t)stream);
}

int conet_backward(conet_t h, const float* dllr, int B, void* stream) {
  if (!h || !dllr) return fail(CONET_ERR_ARG, "NULL argument");
  if (!h->cfg.train) return fail(CONET_ERR_ARG, "handle was created with train = 0");
  if (B != h->fwd_B) return fail(CONET_ERR_ARG, "backward B = %d but the last forward had B = %d", B, h->fwd_B);
  return net_backward(h, dllr, B, (cudaStream_t)stream);
}

int conet_adam_step(conet_t h, float lr, int step, void* stream) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  if (step < 1) return fail(CONET_ERR_ARG, "Adam step %d < 1", step);
  if (!(lr >= 0.f)) return fail(CONET_ERR_ARG, "learning rate must be >= 0");
  return net_adam(h, lr, step, (cudaStream_t)stream);
}

static int fill_sim_args(const conet_config* cfg, const conet_sim_params* sp, uint64_t seed, uint64_t slot0,
                         float fixed_snr_db, SimArgs* a) {
  if (!sp) return fail(CONET_ERR_ARG, "sim params NULL");
  if (sp->n_taps < 1 || sp->n_taps > MAX_TAPS) return fail(CONET_ERR_ARG, "n_taps %d outside 1..%d", sp->n_taps, MAX_TAPS);
  if (sp->n_sinusoids < 1 || sp->n_sinusoids > 64) return fail(CONET_ERR_ARG, "n_sinusoids outside 1..64");
  if (!(sp->scs_hz > 0.f)) return fail(CONET_ERR_ARG, "scs_hz must be > 0");
  if (sp->interferer && (sp->iqam_bits < 2 || sp->iqam_bits > 8 || (sp->iqam_bits & 1)))
    return fail(CONET_ERR_ARG, "iqam_bits %d not in {2,4,6,8}", sp->iqam_bits);
  *a = SimArgs();
  a->N = cfg->n_rx;
  a->T = cfg->n_sym;
  a->F = cfg->n_sc;
  a->Q = cfg->qam_bits;
  a->iQ = sp->iqam_bits;
  a->n_taps = sp->n_taps;
  a->n_sin = sp->n_sinusoids;
  // exponential PDP P_l ~ e^-l, delays l * d with d chosen so the rms delay spread is exact
  double P[MAX_TAPS], sum = 0.0, m1 = 0.0, m2 = 0.0;
  for (int l = 0; l < sp->n_taps; ++l) sum += (P[l] = exp(-(double)l));
  for (int l = 0; l < sp->n_taps; ++l) {
    P[l] /= sum;
    m1 += l * P[l];
    m2 += (double)l * l * P[l];
  }
  const double sig = sqrt(fmax(m2 - m1 * m1, 0.0));
  const double d = sp->n_taps > 1 ? (double)sp->delay_spread_s / sig : 0.0;
  for (int l = 0; l < sp->n_taps; ++l) {
    a->amp[l] = (float)sqrt(P[l] / sp->n_sinusoids);
    a->rho[l] = (double)sp->scs_hz * l * d;
  }
  a->t_sym = (float)((1.0 + 9.0 / 128.0) / (double)sp->scs_hz);
  a->fd_lo = sp->fd_lo;
  a->fd_hi = sp->fd_hi;
  a->snr_lo = sp->snr_lo;
  a->snr_hi = sp->snr_hi;
  a->sir_lo = sp->sir_lo;
  a->sir_hi = sp->sir_hi;
  a->fixed_snr = !isnan(fixed_snr_db);
  a->snr_fixed = fixed_snr_db;
  a->interferer = sp->interferer;
  a->awgn = sp->awgn;
  a->k0 = (uint32_t)seed;
  a->k1 = (uint32_t)(seed >> 32);
  a->slot0 = slot0;
  a->pg = pilot_grid_of(*cfg);
  return CONET_OK;
}

int conet_sim_generate(const conet_config* cfg, const conet_sim_params* sim, uint64_t seed, uint64_t slot0, int B,
                       float fixed_snr_db, float* Y, uint8_t* bits, float* H, float* noise_var, float* interf_var,
                       void* stream) {
  CONET_TRY(validate_config(cfg));
  if (!Y || !bits || !noise_var) return fail(CONET_ERR_ARG, "NULL output");
  if (B < 1 || B > 65535) return fail(CONET_ERR_SHAPE, "B = %d outside 1..65535", B);
  SimArgs a;
  CONET_TRY(fill_sim_args(cfg, sim, seed, slot0, fixed_snr_db, &a));
  a.Y = Y;
  a.bits = bits;
  a.H = H;
  a.noise_var = noise_var;
  a.interf_var = interf_var;
  return launch_sim(a, B, (cudaStream_t)stream);
}

int conet_pilots(const conet_config* cfg, uint8_t* mask, float* pilot_sym, void* stream) {
  CONET_TRY(validate_config(cfg));
  if (!mask || !pilot_sym) return fail(CONET_ERR_ARG, "NULL output");
  return launch_pilots(cfg->n_sym, cfg->n_sc, pilot_grid_of(*cfg), mask, pilot_sym, (cudaStream_t)stream);
}

int conet_assemble_input(const conet_config* cfg, const float* Y, const uint8_t* pilot_mask, const float* pilot_sym,
                         int B, float* X0, void* stream) {
  CONET_TRY(validate_config(cfg));
  if (!Y || !pilot_mask || !pilot_sym || !X0) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1) return fail(CONET_ERR_SHAPE, "B = %d < 1", B);
  return launch_assemble(Y, pilot_mask, pilot_sym, B, cfg->n_rx, cfg->n_sym, cfg->n_sc, 2 * cfg->n_rx + 3, X0,
                         (cudaStream_t)stream);
}

int conet_ls_lmmse(const conet_config* cfg, const float* Y, const uint8_t* pilot_mask, const float* pilot_sym,
                   const float* noise_var, const float* interf_var, const float* H_perfect, int demap_exact, int B,
                   float* llr, void* stream) {
  CONET_TRY(validate_config(cfg));
  if (!Y || !pilot_mask || !pilot_sym || !noise_var || !llr) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1) return fail(CONET_ERR_SHAPE, "B = %d < 1", B);
  LmmseArgs a;
  a.Y = Y;
  a.mask = pilot_mask;
  a.psym = pilot_sym;
  a.noise_var = noise_var;
  a.interf_var = interf_var;
  a.Hp = H_perfect;
  a.llr = llr;
  a.B = B;
  a.N = cfg->n_rx;
  a.T = cfg->n_sym;
  a.F = cfg->n_sc;
  a.Q = cfg->qam_bits;
  a.exact = demap_exact ? 1 : 0;
  for (int i = 0; i < 4; ++i) a.pilot_syms[i] = cfg->pilot_syms[i];
  a.n_pilot_syms = cfg->n_pilot_syms;
  a.comb = cfg->pilot_comb;
  return launch_ls_lmmse(a, (cudaStream_t)stream);
}

int conet_loss_ber(const float* llr, const uint8_t* bits, const uint8_t* pilot_mask, int B, int T, int F, int Q,
                   float grad_scale, float* dllr, double* loss_sum, unsigned long long* err_bits,
                   unsigned long long* n_bits, void* stream) {
  if (!llr || !bits || !pilot_mask) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1 || T < 1 || F < 1 || Q < 1 || Q > 16) return fail(CONET_ERR_SHAPE, "bad sizes B=%d T=%d F=%d Q=%d", B, T, F, Q);
  return launch_loss_ber(llr, bits, pilot_mask, B, T, F, Q, grad_scale, dllr, loss_sum, err_bits, n_bits,
                         (cudaStream_t)stream);
}

int conet_ber_count(const float* llr, const uint8_t* bits, const uint8_t* pilot_mask, int B, int T, int F, int Q,
                    unsigned long long* err_bits, unsigned long long* n_bits, void* stream) {
  return conet_loss_ber(llr, bits, pilot_mask, B, T, F, Q, 0.f, nullptr, nullptr, err_bits, n_bits, stream);
}

// ------------------------------------------------------------------ checkpoints
// Version-1 layout: a 64-byte header, then the FP32 master parameters, Adam's first and
// second moments (n floats each, the flat parameter layout).
namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  uint64_t config_hash;
  uint64_t n_params;
  uint64_t adam_step;
  uint32_t precision;
  uint32_t flags;
  uint8_t reserved[16];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header");
constexpr char CKPT_MAGIC[8] = {'C', 'O', 'N', 'E', 'T', 'C', 'K', 0};
constexpr uint32_t CKPT_VERSION = 1;
constexpr uint32_t CKPT_HAS_ADAM = 1;

// FNV-1a (64-bit) over the fields that give the parameters their meaning: the network
// shape and the fixed pilot grid (each value folded in as 8 little-endian bytes).
uint64_t config_hash(const conet_config& c) {
  uint64_t h = 0xcbf29ce484222325ull;
  auto mix = [&](int64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (uint64_t)((v >> (8 * i)) & 0xff);
      h *= 0x100000001b3ull;
    }
  };
  const int f[] = {c.n_rx, c.n_sym, c.n_sc, c.qam_bits, c.n_branches, c.depth, c.width,
                   c.residual, c.norm, c.fuse_mask, c.resnet_baseline, c.n_pilot_syms, c.pilot_comb,
                   c.fuse_op, c.feedback, c.depthwise};
  for (int v : f) mix(v);
  if (c.support_inputs) mix(0x5e1ec7 + c.support_inputs);   // (absent from hashes of full-input networks)
  if (c.support_mask) mix(0x5a3c0000ull + c.support_mask);
  for (int i = 0; i < c.n_pilot_syms && i < 4; ++i) mix(c.pilot_syms[i]);
  mix((int64_t)c.pilot_seed);
  return h;
}

size_t ckpt_bytes(const conet_s* h) { return sizeof(CkptHeader) + 3 * h->L.total * sizeof(float); }

}  // namespace

int conet_checkpoint_hash(const conet_config* cfg, uint64_t* hash) {
  CONET_TRY(validate_config(cfg));
  if (!hash) return fail(CONET_ERR_ARG, "hash is NULL");
  *hash = config_hash(*cfg);
  return CONET_OK;
}

int conet_checkpoint_bytes(conet_t h, size_t* bytes) {
  if (!h || !bytes) return fail(CONET_ERR_ARG, "NULL argument");
  *bytes = ckpt_bytes(h);
  return CONET_OK;
}

int conet_save_checkpoint(conet_t h, uint64_t adam_step, void* host_buf, size_t bytes) {
  if (!h || !host_buf) return fail(CONET_ERR_ARG, "NULL argument");
  if (bytes != ckpt_bytes(h)) return fail(CONET_ERR_WEIGHTS, "checkpoint buffer has %zu bytes, needs %zu", bytes, ckpt_bytes(h));
  CkptHeader hd = {};
  memcpy(hd.magic, CKPT_MAGIC, sizeof(hd.magic));
  hd.version = CKPT_VERSION;
  hd.header_bytes = sizeof(CkptHeader);
  hd.config_hash = config_hash(h->cfg);
  hd.n_params = h->L.total;
  hd.adam_step = adam_step;
  hd.precision = (uint32_t)h->prec;
  hd.flags = CKPT_HAS_ADAM;
  uint8_t* out = static_cast<uint8_t*>(host_buf);
  const size_t nb = h->L.total * sizeof(float);
  CONET_CUDA(cudaDeviceSynchronize());
  CONET_CUDA(cudaMemcpy(out + sizeof(CkptHeader), h->params, nb, cudaMemcpyDeviceToHost));
  CONET_CUDA(cudaMemcpy(out + sizeof(CkptHeader) + nb, h->adam_m, nb, cudaMemcpyDeviceToHost));
  CONET_CUDA(cudaMemcpy(out + sizeof(CkptHeader) + 2 * nb, h->adam_v, nb, cudaMemcpyDeviceToHost));
  memcpy(out, &hd, sizeof(hd));
  return CONET_OK;
}

int conet_load_checkpoint(conet_t h, const void* host_buf, size_t bytes, uint64_t* adam_step) {
  if (!h || !host_buf) return fail(CONET_ERR_ARG, "NULL argument");
  if (bytes < sizeof(CkptHeader)) return fail(CONET_ERR_WEIGHTS, "checkpoint of %zu bytes has no header", bytes);
  CkptHeader hd;
  memcpy(&hd, host_buf, sizeof(hd));
  if (memcmp(hd.magic, CKPT_MAGIC, sizeof(hd.magic)) != 0) return fail(CONET_ERR_WEIGHTS, "not a CoNet checkpoint");
  if (hd.version != CKPT_VERSION || hd.header_bytes != sizeof(CkptHeader) || !(hd.flags & CKPT_HAS_ADAM))
    return fail(CONET_ERR_WEIGHTS, "checkpoint version %u (header %u bytes) is not readable by version %u", hd.version,
                hd.header_bytes, CKPT_VERSION);
  if (hd.config_hash != config_hash(h->cfg) || hd.n_params != h->L.total)
    return fail(CONET_ERR_WEIGHTS, "checkpoint was written for a different network (hash %016llx, %llu parameters)",
                (unsigned long long)hd.config_hash, (unsigned long long)hd.n_params);
  if (bytes != ckpt_bytes(h)) return fail(CONET_ERR_WEIGHTS, "checkpoint has %zu bytes, needs %zu", bytes, ckpt_bytes(h));
  const uint8_t* in = static_cast<const uint8_t*>(host_buf);
  const size_t nb = h->L.total * sizeof(float);
  CONET_CUDA(cudaDeviceSynchronize());
  CONET_CUDA(cudaMemcpy(h->params, in + sizeof(CkptHeader), nb, cudaMemcpyHostToDevice));
  CONET_CUDA(cudaMemcpy(h->adam_m, in + sizeof(CkptHeader) + nb, nb, cudaMemcpyHostToDevice));
  CONET_CUDA(cudaMemcpy(h->adam_v, in + sizeof(CkptHeader) + 2 * nb, nb, cudaMemcpyHostToDevice));
  CONET_TRY(net_weights_changed(h, 0));
  CONET_CUDA(cudaDeviceSynchronize());
  if (adam_step) *adam_step = hd.adam_step;
  return CONET_OK;
}

int conet_train_step(conet_t h, const conet_sim_params* sim, uint64_t seed, uint64_t step, int B, float lr,
                     double* loss_out, void* stream) {
  if (!h || !sim) return fail(CONET_ERR_ARG, "NULL argument");
  if (!h->cfg.train) return fail(CONET_ERR_ARG, "handle was created with train = 0");
  if (B < 1 || B > h->cfg.max_batch) return fail(CONET_ERR_SHAPE, "B = %d outside 1..max_batch (%d)", B, h->cfg.max_batch);
  SimArgs a;
  CONET_TRY(fill_sim_args(&h->cfg, sim, seed, step * (uint64_t)B, NAN, &a));
  return net_train_step(h, a, step, B, lr, loss_out, (cudaStream_t)stream);
}

}  // extern "C"
