// Internal kernel launchers of libconet and their argument blocks.
#pragma once

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
int launch_assemble_bf16(const float* Y, const uint8_t* mask, const float* psym, int B, int N, int T, int F,
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
};
int launch_conv3x3_fp32(const ConvArgs& a, int n_br, int cin, int cout, cudaStream_t s);

// ---------------------------------------------------------------- fusion / LN / head
// Per RE (one warp): x0 = fuse ? LN?(prod_b u_b) : u_0 (written to x0_out);
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
  int n_br, fuse, C, Q;
  long long M;
};
int launch_fuse(const FuseArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- weights
// Re-layout of the FP32 master conv weights [Cout][3][3][cin_src] into the kernels'
// [9][cin_dst][Cout] order (input channels zero-padded to cin_dst).
int launch_weights_to_tap_major(const float* w, int cout, int cin_src, int cin_dst, float* out, cudaStream_t s);

}  // namespace conet
