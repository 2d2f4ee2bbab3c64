// Handle state and network orchestration of libconet (host side).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <vector>

#include "../../include/conet.h"
#include "kernels.cuh"

namespace conet {

struct BlockOff {
  long ln1g = -1, ln1b = -1, c1w = -1, c1b = -1, ln2g = -1, ln2b = -1, c2w = -1, c2b = -1;
  long c1d = -1, c2d = -1;   // depthwise 3x3 weights [C][3][3] of depthwise-separable convs
};

struct Seg {
  size_t off, n;
  int kind;      // 0 He-normal, 1 ones, 2 zeros
  float stdv;
};

struct ConvT {
  size_t off;
  int cout, cin;
  int taps;      // 9 = a 3x3 conv [Cout][3][3][Cin]; 1 = the 1x1 of a depthwise-separable conv [Cout][Cin]
};

// Offsets (in floats) of every tensor in the flat parameter vector; -1 = absent.
struct Layout {
  long in_w[MAX_BR] = {}, in_b[MAX_BR] = {};
  std::vector<long> lw[MAX_BR], lb[MAX_BR];   // plain layers 1..depth-1
  std::vector<BlockOff> blk[MAX_BR];          // residual blocks
  std::vector<long> fg, fb;                   // fusion LayerNorm per fusion point
  long hw = 0, hb = 0;
  size_t total = 0;
  std::vector<Seg> segs;
  std::vector<ConvT> convs;
};

bool fused_at(const conet_config& c, int i);
int fused_width(const conet_config& c, int i);
Layout build_layout(const conet_config& c);

}  // namespace conet

struct conet_s {
  conet_config cfg;
  int prec = 0;
  conet::Layout L;
  int T = 0, F = 0, N = 0, Q = 0, C = 0, nb = 0, cin = 0, c_pad = 0;
  float* params = nullptr;
  float* params_eff = nullptr;               // support_inputs: params with the withheld weights zero
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* wt = nullptr;                       // conv weights in [9][Cin_pad][Cout] order
  std::map<size_t, size_t> wt_off;           // master offset -> wt offset
  size_t wt_total = 0;
  uint8_t* mask = nullptr;                   // fixed pilot grid [T][F]
  float* psym = nullptr;                     // pilot symbols [T][F][2]
  float* X0 = nullptr;                       // assembled input [B][T][F][c_pad]
  std::vector<float*> act;                   // activation buffers, max_batch*T*F*C floats each
  float* wd = nullptr;                       // body conv weights for dgrad: [9][Cout][Cin], rotated
  std::map<size_t, size_t> wd_off;
  float* G[3][conet::MAX_BR] = {};           // gradient buffers (train), max_batch*T*F*C each
  float* ew_part = nullptr;                  // partial sums of the elementwise backward kernels
  float* wg_part = nullptr;                  // split partials of the weight gradient
  float* dw_out[conet::MAX_BR] = {};         // depthwise-separable convs: the depthwise output
  void* wg_tc = nullptr;                     // BF16 training: transposed operand copies of the tensor-core wgrad
  int n_pilot_re = 0;
  // tensor-core (BF16) path
  void* X0b = nullptr;                       // assembled input, BF16 [B][T][F][16]
  void* nxb[2][conet::MAX_BR] = {};          // BF16 conv inputs (ping-pong / H1, H2)
  void* dwb[conet::MAX_BR] = {};             // 16-bit depthwise outputs (depthwise-separable blocks)
  void* X0b_lo = nullptr;                    // split-TF32 path: low parts of X0b / nxb / wb
  float* nxb_lo[2][conet::MAX_BR] = {};
  float* wb_lo = nullptr;
  void* wb = nullptr;                        // BF16 weights [9][Cout][Cin_pad] per conv
  std::map<size_t, size_t> wb_off;
  std::vector<conet::TcMaps> tcmaps;         // tensor maps per conv launch
  // BF16 training: the data gradient of each body conv runs on the tensor cores as the conv
  // of a BF16 copy of the incoming gradient with the rotated, transposed BF16 weights
  bool tc_dgrad = false;
  void* wd16 = nullptr;                      // [9][Cin][Cout] per body conv, offsets wd_off
  void* g16[conet::MAX_BR] = {};             // BF16 copies of the incoming data gradients
  float* zero_c = nullptr;                   // C zeros: the dgrad conv has no bias
  std::vector<conet::TcMaps> dg_maps;        // per body conv (in wd_off order)
  std::map<size_t, size_t> dg_index;         // branch 0's conv weight offset -> dg_maps index
  float* xcat = nullptr;                     // FP32 plain networks, fuse_op 2: the concatenated main input
  float* gcat = nullptr;                     // ... and, training, the gradient of a concatenated activation
  int* d_err = nullptr;                      // device error word of the tensor-core kernels
  // E4M3 path
  float* fp8_wscale = nullptr;               // per conv: [Cout] per-output-channel weight scales
  std::map<size_t, size_t> fp8_ws_off;       // master offset -> offset in fp8_wscale
  float* fp8_act = nullptr;                  // per conv launch and branch: scale, 1/scale, pad to 8, dq[C]
  unsigned* fp8_amax = nullptr;              // per conv launch and branch: largest |input| (float bits)
  bool fp8_calibrated = false;               // activation scales valid for the current weights
  float fp8_margin = 2.f;                    // scale = margin * amax / 448
  float* sim_Y = nullptr;                    // training-step slots
  uint8_t* sim_bits = nullptr;
  float* sim_nv = nullptr;
  float* llr = nullptr;
  float* dllr = nullptr;
  double* d_loss = nullptr;
  unsigned long long* d_cnt = nullptr;
  int fwd_B = 0;
  int chunk = 1;                             // slots per pass (activation buffers hold this many)
  std::vector<void*> allocs;
  // Inference forward replayed as a CUDA graph: the first call with a given (Y, mask, B, llr)
  // runs eagerly, the second identical call captures its launches into a graph (on an
  // internal stream), later identical calls launch that graph on the caller's stream.
  bool graphs = true;                        // conet_graphs
  // whole-network kernel (small plain BF16 networks): padded input grid and its tensor maps
  bool sn = false;                           // the handle's network qualifies
  int whole_net = 1;                         // conet_whole_network: 0 never, 1 automatic, 2 always
  void* sn_x = nullptr;
  CUtensorMap sn_xmap;
  CUtensorMap sn_wmaps[conet::SN_MAX_LAYERS][2];
  cudaGraphExec_t g_exec = nullptr;
  cudaStream_t g_stream = nullptr;           // capture stream
  const void* g_Y = nullptr;
  const void* g_mask = nullptr;
  const void* g_llr = nullptr;
  int g_B = 0;
  long long g_kernels = 0;                   // kernel launches the graph holds
  bool prof_on = false;                      // CUDA-event timing of launches by kind
  std::vector<cudaEvent_t> prof_ev;          // 2 events per recorded launch
  std::vector<int> prof_kind;
  int prof_open = -1;
};

namespace conet {

int dev_alloc(conet_s* h, void** p, size_t bytes);

enum ProfKind { PK_CONV = 0, PK_CONV_IN = 1, PK_FUSE = 2, PK_ASSEMBLE = 3, PK_BACKWARD = 4, PK_ADAM = 5, PK_N = 6 };
constexpr size_t PROF_CAP = 65536;
void prof_begin(conet_s* h, int kind, cudaStream_t s);
void prof_end(conet_s* h, cudaStream_t s);
template <typename Tp>
inline int dev_alloc_t(conet_s* h, Tp** p, size_t count) {
  return dev_alloc(h, reinterpret_cast<void**>(p), count * sizeof(Tp));
}

int net_setup(conet_s* h);
int net_weights_changed(conet_s* h, cudaStream_t s);
int net_forward(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s);
int net_forward_replay(conet_s* h, const float* Y, const uint8_t* mask, int B, float* llr, cudaStream_t s);
void net_graph_reset(conet_s* h);
int net_backward(conet_s* h, const float* dllr, int B, cudaStream_t s);
int net_adam(conet_s* h, float lr, int step, cudaStream_t s);
int net_train_step(conet_s* h, const SimArgs& a, uint64_t step, int B, float lr, double* loss_out, cudaStream_t s);
int net_calibrate(conet_s* h, const float* Y, const uint8_t* mask, int B, float margin, cudaStream_t s);

}  // namespace conet
