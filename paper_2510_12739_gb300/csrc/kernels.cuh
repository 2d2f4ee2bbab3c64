// Internal kernel launchers of libconet and their argument blocks.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace conet {

constexpr int MAX_TAPS = 24;
constexpr int MAX_BR = 4;

struct PilotGrid {
  int syms[4];
  int n_syms;
  int comb;
  uint32_t k0, k1;   // Philox key of the pilot seed
};

struct SimArgs {
  float* Y;
  float* H;
  uint8_t* bits;
  float* noise_var;
  float* interf_var;
  int N, T, F, Q, iQ;
  int n_taps, n_sin;
  float amp[MAX_TAPS];      // sqrt(P_l / S)
  double rho[MAX_TAPS];     // scs * tau_l: phase turns per subcarrier
  float t_sym;
  float fd_lo, fd_hi, snr_lo, snr_hi, sir_lo, sir_hi;
  int fixed_snr;
  float snr_fixed;
  int interferer, awgn;
  uint32_t k0, k1;
  uint64_t slot0;
  PilotGrid pg;
};

int launch_pilots(int T, int F, const PilotGrid& pg, uint8_t* mask, float* psym, cudaStream_t s);
int launch_sim(const SimArgs& a, int B, cudaStream_t s);
int launch_init_segment(float* p, size_t off, size_t n, float std, float constant, int normal, uint64_t seed,
                        cudaStream_t s);

// ---------------------------------------------------------------- receiver DSP
int launch_assemble(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                    int c_pad, float* X0, cudaStream_t s);
int launch_assemble_16(int kind, const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                       int c_pad, void* X0, cudaStream_t s);

struct LmmseArgs {
  const float* Y;
  const uint8_t* mask;
  const float* psym;
  const float* noise_var;
  const float* interf_var;
  const float* Hp;
  float* llr;
  int B, N, T, F, Q, exact;
  int pilot_syms[4];
  int n_pilot_syms;
  int comb;
};
int launch_ls_lmmse(const LmmseArgs& a, cudaStream_t s);

int launch_loss_ber(const float* llr, const uint8_t* bits, const uint8_t* mask, int B, int T, int F, int Q,
                    float grad_scale, float* dllr, double* loss_sum, unsigned long long* err,
                    unsigned long long* nbits, cudaStream_t s);

// ---------------------------------------------------------------- FP32 convolution
// One launch runs the same 3x3 conv layer for every branch (blockIdx.y = branch).
// Epilogue per RE: v = conv + bias (+ resid);  out0 = relu0 ? max(v, 0) : v;
// out1 = relu(LN(v) * gamma + beta) when ln_g is set.
struct ConvArgs {
  const float* in[MAX_BR];
  const float* w[MAX_BR];      // [9][Cin][Cout]  (tap-major, output channel fastest)
  const float* bias[MAX_BR];
  const float* resid[MAX_BR];
  float* out0[MAX_BR];
  float* out1[MAX_BR];
  const float* ln_g[MAX_BR];
  const float* ln_b[MAX_BR];
  int relu0;
  int M, T, F;                 // M = B * T * F resource elements
  int taps;                    // 0 or 9: 3x3 conv; 1: 1x1 conv (w = [1][Cin][Cout])
};
int launch_conv3x3_fp32(const ConvArgs& a, int n_br, int cin, int cout, cudaStream_t s);

// Depthwise 3x3 'same' conv per branch: out[m][c] = sum_tap w[c][tap'] in[m + shift(tap)][c]
// with tap' = tap, or 8 - tap when flip is set (the kernel rotated by 180 degrees: the data
// gradient of the conv).
struct DwArgs {
  const float* in[MAX_BR];
  const float* w[MAX_BR];      // [C][3][3]
  float* out[MAX_BR];
  int C, T, F;
  long long M;
  int flip;
};
int launch_dwconv3x3(const DwArgs& a, int n_br, cudaStream_t s);
// The same conv on 16-bit activations (kind 0 BF16, 3 FP16) with FP32 weights [C][3][3]:
// products accumulated in FP32 over the taps in order, the sum rounded once to the format.
struct DwArgs16 {
  const void* in[MAX_BR];
  const float* w[MAX_BR];
  void* out[MAX_BR];
  int C, T, F;
  long long M;
};
int launch_dwconv3x3_16(int kind, const DwArgs16& a, int n_br, cudaStream_t s);

// ---------------------------------------------------------------- fusion / LN / head
// Per RE (fuse_quad / fuse_row in csrc/fuse.cu):
// x0 = fuse ? LN?(prod_b u_b or sum_b u_b) : u_0 (written to x0_out);
// h_b = relu(LN1_b(x_b)) or relu(x_b) (written to h_out[b] when set);
// llr = head_w x0 + head_b when head_w is set.
struct FuseArgs {
  const float* u[MAX_BR];
  float* x0_out;
  float* h_out[MAX_BR];
  const float* ln1_g[MAX_BR];
  const float* ln1_b[MAX_BR];
  const float* fuse_g;
  const float* fuse_b;
  const float* head_w;
  const float* head_b;
  float* llr;
  int* nonfinite;              // set to 1 when an LLR written is NaN or infinite
  int n_br, fuse, C, Q;
  int op;                      // interaction: 0 = product, 1 = sum
  int feedback;                // Example II: u[b] += u[0] (in place) for the supports
  long long M;
};
int launch_fuse(const FuseArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- backward
constexpr int EW_PART_CTAS = 512;     // CTAs (hence partial rows) of the elementwise bwd kernels
constexpr int WG_MAX_SPLITS = 64;
constexpr int WG_TILED_MAX_CTAS = 152 * 6;   // split-K CTAs (all branches) of the tiled weight gradient

// Hadamard fusion backward (+ post-fusion LN, + ReLU mask of the fused activations):
// gu_0 = dp prod_{i>0} u_i,  gu_b = gxs_b + dp prod_{i!=b} u_i  (fuse), else gu_b = gx_b.
struct FuseBwdArgs {
  const float* u[MAX_BR];
  const float* gx0;
  const float* gxs[MAX_BR];   // [0] unused; NULL = zero
  float* gu[MAX_BR];
  const float* ln_g;          // post-fusion LN gain or NULL
  float* part;                // [grid][2][C] dgamma / dbeta partials (when ln_g)
  int n_br, fuse, relu_mask, C;
  int op;                     // interaction: 0 = product, 1 = sum, 2 = concatenation (gx0 and
                              // the LN partials then n_br x C wide)
  int feedback;               // Example II: the supports' u hold a_b + a_0 (their next input)
  long long M;
};
int launch_fuse_bwd(const FuseBwdArgs& a, cudaStream_t s);

// out = add + d/dx relu(LN(x)*g + b) . g_out   (or add + [x > 0] g_out without LN)
struct LnReluBwdArgs {
  const float* g;
  const float* x;
  const float* ln_g;
  const float* ln_b;
  const float* add;
  float* out;
  float* part;                // [grid][2][C] dgamma / dbeta partials (when ln_g)
  int C;
  long long M;
};
int launch_ln_relu_bwd(const LnReluBwdArgs& a, cudaStream_t s);

struct HeadBwdArgs {
  const float* dllr;
  const float* x0;
  const float* w;
  float* gx0;
  float* part;                // [grid][Q*C + Q]
  int C, Q;
  long long M;
};
int launch_head_bwd(const HeadBwdArgs& a, cudaStream_t s);
int launch_channel_sums(const float* g, long long M, int C, float* part, cudaStream_t s);
int launch_reduce_partials(const float* part, int n_part, int n, float* out, int accumulate, cudaStream_t s);
int ew_grid(long long M);

struct WgradArgs {
  const float* x[MAX_BR];     // conv input [M][cin]
  const float* g[MAX_BR];     // grad wrt conv output [M][cout]
  float* dW[MAX_BR];          // master layout [cout][3][3][cin_src]
  int cin_src[MAX_BR];
  float* part;                // split partials
  int cin, cout, n_br, T, F;
  long long M;
};
int wgrad_splits(long long M, int cin, int cout, int n_br);
size_t wgrad_partial_floats(long long M, int cin, int cout, int n_br);
int launch_wgrad(const WgradArgs& a, cudaStream_t s);
// The same gradient through the tiled split-K kernel where instantiated (cin, cout in
// {8/16, 16/16, 8/32, 32/32, 8/64, 64/64}), else launch_wgrad; partials need
// wgrad_tiled_splits(M, n_br) * n_br * 9 * cin * cout floats.
int launch_wgrad_tiled(const WgradArgs& a, cudaStream_t s);
// Weight gradients of a depthwise-separable block conv (FP32 path, csrc/dwbwd.cu): the 1x1's
// dW[co][ci] = sum_m g[m][co] z[m][ci] (z = the per-channel 3x3's output) and the per-channel
// 3x3's dWd[c][tap] = sum_m dz[m][c] x[m + shift(tap)][c]; both overwrite dW / dWd (master
// layouts [C][C] and [C][3][3]) through per-CTA partials in `part` (dw_bwd_splits(n_br) x
// n_br x C x C floats at most).
struct Wgrad1x1Args {
  const float* g[MAX_BR];
  const float* z[MAX_BR];
  float* dW[MAX_BR];
  float* part;
  int C, n_br;
  long long M;
};
struct DwWgradArgs {
  const float* x[MAX_BR];
  const float* dz[MAX_BR];
  float* dWd[MAX_BR];
  float* part;
  int C, n_br, T, F;
  long long M;
};
int dw_bwd_splits(int n_br);
int launch_wgrad1x1(const Wgrad1x1Args& a, cudaStream_t s);
int launch_dw_wgrad(const DwWgradArgs& a, cudaStream_t s);
int wgrad_tiled_splits(long long M, int n_br);
// Fixed-order sum over S split partials [S][n_br][9][cin][cout] of branch br into the master
// layout dW [cout][3][3][cin_src].
// w [cout][3][3][cin] (cin <= 32): the entries of the input channels whose bit in `keep` is
// clear set to zero (the support nets' withheld inputs, Sec. III selective inputs).
int launch_zero_input_channels(float* w, int cout, int cin, unsigned keep, cudaStream_t s);
int launch_wgrad_reduce(const float* part, int S, int n_br, int br, int cin, int cout, int cin_src, float* dW,
                        cudaStream_t s);
// The weight gradient on the tensor cores from BF16 copies of the operands (wgrad_tc.cu):
// shapes with F % 8 == 0 and (cin padded to 8, cout) in {8, 16, 32} x {32} or {8, 16, 64} x {64};
// a.part needs wgrad_tc_splits(...) x n_br x 9 x cin_padded x cout floats, `scratch`
// wgrad_tc_scratch_bytes(...) bytes.
bool wgrad_tc_supported(int cin, int cout, int F);
int wgrad_tc_splits(long long slots, int T, int F, int n_br);
size_t wgrad_tc_scratch_bytes(long long slots, int T, int F, int cin_max, int cout);
int launch_wgrad_tc(const WgradArgs& a, int slots, void* scratch, int* err, cudaStream_t s);

int launch_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                float bc1, float bc2, cudaStream_t s);
// (cin = 0: square, cin = cout)
int launch_weights_dgrad_layout(const float* w, int cout, float* out, cudaStream_t s, int cin = 0);

// ---------------------------------------------------------------- tensor-core convolution
struct TcMaps {
  CUtensorMap a[MAX_BR];       // activations [slots][T][F][Cin], box {KC, 128, 1, 1}
  CUtensorMap w[MAX_BR];       // weights [9][Cout][Cin], box {KC, Cout, 1}
  CUtensorMap a_lo[MAX_BR];    // split-TF32 path: low parts of the same tensors
  CUtensorMap w_lo[MAX_BR];
  // staged output stores of the fixed layer shapes: the FP32 stream xs_out[b] and the next
  // input nx_out[b] as [slots x T][F][Cout], box {channels per epilogue part, 32, 1}
  CUtensorMap xs[MAX_BR];
  CUtensorMap nx[MAX_BR];
};

// Fused epilogue, per RE and branch b:
//   v_b = conv_b + bias_b (+ resid_b)                  -> t_out[b]   (FP32, optional)
//   a_b = v_b | relu(v_b) | relu(LN2_b(v_b))            (pre = 0 | 1 | 2)
//   x_0 = fuse ? LN_f?(prod_b a_b) : a_0;  x_b = a_b    -> xs_out[b]  (FP32, optional)
//   next_b = x_b | relu(x_b) | relu(LN1_b(x_b))         (post[b] = 0 | 1 | 2) -> nx_out[b]
//   llr = head_w x_0 + head_b                           (when head_w)
struct TcConvArgs {
  int n_tiles, T, F, nfb;
  const float* bias[MAX_BR];
  const float* resid[MAX_BR];
  int pre;
  const float* ln2_g[MAX_BR];
  const float* ln2_b[MAX_BR];
  int fuse;
  const float* lnf_g;
  const float* lnf_b;
  float* t_out[MAX_BR];
  float* a_out[MAX_BR];        // a_b (FP32, optional; kept for backward)
  float* xs_out[MAX_BR];
  void* nx_out[MAX_BR];
  float* nx_lo[MAX_BR];        // split-TF32 path: nx_out holds hi = tf32(next), nx_lo = next - hi
  int post[MAX_BR];
  const float* ln1_g[MAX_BR];
  const float* ln1_b[MAX_BR];
  const float* head_w;
  const float* head_b;
  float* llr;
  int Q;
  int* err;                    // device error word (first timed-out wait)
  int* nonfinite;              // set to 1 when an LLR written is NaN or infinite
  // E4M3 path: accumulator column c of branch b is dequantised by dq[b][c] (= the input's
  // per-tensor scale x the weights' per-output-channel scale); nx_out[b] is written as
  // E4M3 of next / scale, with qinv[b] = 1 / scale (device scalars); amax[b], when set,
  // receives the largest |next| (float bits, atomicMax); measure = 1 writes no activation.
  const float* dq[MAX_BR];
  const float* qinv[MAX_BR];
  unsigned* amax[MAX_BR];
  int measure;
  int op;                      // fused layers: 0 = product, 1 = sum of the branches
  int feedback;                // fused layers, Example II: supports continue with a_b + a_0
  int taps;                    // 0: the 3x3 conv; 1: a 1x1 conv (maps built with tc_chunk_pw,
                               // one-tap boxes and [1][Cout][Cin] weights; BF16 / FP16)
};
int launch_conv_tc(int kind, int nb, int cin, int cout, const TcMaps& maps, const TcConvArgs& a, cudaStream_t s);
// TMA maps of one conv operand: activations [slots][T][F][C] read in boxes of kc channels x
// (TILE_M, or TILE_M + 2 when taps == 3) subcarriers; weights [n_taps][cout][cin] (9, or 1
// for a 1x1 conv) in boxes of kc x rows x taps (rows = tc_wbox_rows, taps = tc_wbox_taps of
// the conv's shape; 1 for a 1x1 conv).
int make_act_map(CUtensorMap* map, int kind, const void* base, int C, int F, int T, int slots, int kc, int taps);
int make_weight_map(CUtensorMap* map, int kind, const void* base, int cin, int cout, int kc, int rows, int taps,
                    int n_taps = 9);
int tc_chunk(int kind, int nb, int cin, int cout);
int tc_chunk_pw(int kind, int nb, int c);   // channels per K chunk of the 1x1 conv (C -> C)
int tc_branch_groups(int kind, int nb, int cout);   // branch groups per tile (1: all branches at once)
// BF16 tensor-core dgrad operands: Wd[tap'][o][i] = W[i][8 - tap'][o] (the kernel rotated by
// 180 degrees, input and output channels exchanged; input channel fastest) from the FP32
// master [C][9][C]; and the BF16 copies of n values of each of nb gradient tensors.
int launch_weights_dgrad_bf16(const float* w, int C, void* out, cudaStream_t s);
int launch_grads_bf16(const float* const* in, void* const* out, int nb, long long n, cudaStream_t s);
int tc_taps(int kind, int nb, int cin, int cout);
int tc_wbox_rows(int kind, int nb, int cin, int cout);   // output channels per weight box
int tc_wbox_taps(int kind, int nb, int cin, int cout);   // taps per weight box
// channels per epilogue part of the staged output stores of the fixed layer shapes, 0 when
// the shape stores unstaged
int tc_store_cols(int kind, int nb, int cin, int cout);
// output map of a staged store: [slots x T][F][C] elements of `out_kind` (-1: FP32; else an
// operand kind), box {cols, 32, 1}, swizzled for rows of cols elements
int make_out_map(CUtensorMap* map, int out_kind, void* base, int C, int F, int symbols, int cols);
// [Cout][taps][cin_src] FP32 master -> [taps][Cout][cin_dst] BF16 (kind 0) / FP16 (kind 3)
int launch_weights_16(int kind, const float* w, int cout, int cin_src, int cin_dst, void* out, cudaStream_t s,
                      int taps = 9);
int launch_weights_split(const float* w, int cout, int cin_src, int cin_dst, float* hi, float* lo, cudaStream_t s);
int launch_assemble_split(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                          int c_pad, float* hi, float* lo, cudaStream_t s);
// E4M3 input assembly: X0 [B][T][F][c_pad] = E4M3(channel value * qinv[0]); X0 == NULL only
// accumulates the largest |channel value| into *amax (float bits).
int launch_assemble_fp8(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
                        int c_pad, const float* qinv, uint8_t* X0, unsigned* amax, cudaStream_t s);
// [Cout][3][3][cin_src] FP32 master -> [9][Cout][cin_dst] E4M3 with one scale per output
// channel, wscale[co] = the smallest power of two >= max_{tap,ci} |w| / 448 (1 for an
// all-zero channel).
int launch_weights_fp8(const float* w, int cout, int cin_src, int cin_dst, uint8_t* out, float* wscale,
                       cudaStream_t s);
// Activation scales of one conv launch from the recorded amax: per branch b, scale = the
// smallest power of two >= margin * amax[b] / 448 (1 when amax is 0), qinv[b] = 1 / scale
// and dq[b][c] = scale * wscale[b][c] for c < cout.
struct Fp8ScaleArgs {
  const unsigned* amax[MAX_BR];
  const float* wscale[MAX_BR];
  float* scale[MAX_BR];
  float* qinv[MAX_BR];
  float* dq[MAX_BR];
};
int launch_fp8_scales(const Fp8ScaleArgs& a, int nb, int cout, float margin, cudaStream_t s);

// ---------------------------------------------------------------- whole-network kernel
// Small plain CoNets (2 branches x 32 channels, T (F + 1) <= 1024): every layer of a slot in
// one persistent kernel, activations in shared memory (smallnet_tc.cu).
constexpr int SN_MAX_LAYERS = 8;
struct SmallNetArgs {
  const float* bias[SN_MAX_LAYERS][2];
  const float* lnf_g[SN_MAX_LAYERS];   // LayerNorm after the fusion of layer l, or NULL
  const float* lnf_b[SN_MAX_LAYERS];
  int fuse[SN_MAX_LAYERS];
  const float* head_w;
  const float* head_b;
  const float* dq[SN_MAX_LAYERS][2];   // E4M3: dequantisation [32] of layer l's accumulators
  const float* qinv[SN_MAX_LAYERS][2]; // E4M3: 1 / scale of layer l's input (device scalar)
  float* llr;
  int* err;
  int* nonfinite;
  int B, T, F, Q, depth;
};
// kind: 0 BF16, 2 E4M3
bool smallnet_eligible(int kind, int T, int F, int nb, int C, int depth, int Q);
size_t smallnet_input_bytes(int slots, int T, int F);   // the padded input grid
int make_smallnet_input_map(CUtensorMap* map, int kind, const void* xp, int slots, int T, int F);
int launch_smallnet_pad(const void* x, void* xp, int slots, int T, int F, cudaStream_t s);
int launch_smallnet(int kind, const CUtensorMap& x0_map, const CUtensorMap (*w_maps)[2], const SmallNetArgs& a,
                    cudaStream_t s);

// ---------------------------------------------------------------- weights
// Re-layout of the FP32 master conv weights [Cout][3][3][cin_src] into the kernels'
// [9][cin_dst][Cout] order (input channels zero-padded to cin_dst).
int launch_weights_to_tap_major(const float* w, int cout, int cin_src, int cin_dst, float* out, cudaStream_t s,
                                int taps = 9);

}  // namespace conet
