/*
 * conet.h -- C ABI of libconet, a GB300 (sm_103a) implementation of the hot path of
 * "CoNet-Rx: Collaborative Neural Networks for OFDM Receivers": the collaborative
 * network receiver's forward pass (received grid -> per-bit LLRs), the backward pass
 * and optimiser step that train it, the synthetic OFDM link that feeds it, and the
 * LS-LMMSE receiver it is compared against.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Tensor arguments marked "dev" are device pointers in caller-owned memory on the
 *    current CUDA device; "host" pointers are ordinary host memory.  The library never
 *    frees caller memory.  All device tensors are dense, row-major, with the layouts
 *    given per argument, and 16-byte aligned (as cudaMalloc / torch allocations are).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *    are asynchronous on that stream unless they say they synchronise.
 *  - Complex values are interleaved (re, im) float32 pairs: a complex [..] tensor is a
 *    float [.., 2] tensor.
 *  - Grid axes: B slots, N receive antennas, T OFDM symbols per slot (14), F
 *    subcarriers, Q bits per QAM symbol.  A resource element (RE) is one (t, f).
 *  - LLR sign: LLR = log P(b = 1) / P(b = 0); the hard decision is b = [LLR > 0].
 *  - Every function returns CONET_OK (0) or a negative conet_status.  Argument and
 *    shape errors are detected on the host before any launch and leave outputs
 *    untouched; CUDA errors surface as CONET_ERR_CUDA.  conet_last_error() returns a
 *    thread-local message for the last failure.
 */
#ifndef CONET_H
#define CONET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct conet_s* conet_t;   /* opaque: owns weights, gradients, Adam state, workspace */

typedef enum {
  CONET_OK = 0,
  CONET_ERR_ARG = -1,          /* null pointer or invalid value */
  CONET_ERR_SHAPE = -2,        /* sizes out of range (e.g. B > max_batch) */
  CONET_ERR_CUDA = -3,         /* a CUDA runtime call or launch failed */
  CONET_ERR_NOMEM = -4,        /* device allocation failed at create time */
  CONET_ERR_WEIGHTS = -5,      /* weight vector of the wrong size */
  CONET_ERR_NONFINITE = -6,    /* NaN / Inf met in a loss or written as an LLR */
  CONET_ERR_TIMEOUT = -7,      /* a bounded device-side wait gave up */
  CONET_ERR_UNSUPPORTED = -8   /* valid request this build does not implement */
} conet_status;

typedef enum {
  CONET_FP32 = 0,              /* FP32 storage, FP32 FFMA convolutions */
  CONET_BF16 = 1,              /* BF16 activations / weights, FP32 accumulate (tcgen05) */
  CONET_FP8E4M3 = 2,           /* E4M3 weights (per-output-channel scales) and activations
                                  (per-tensor scales from calibration), FP32 accumulate
                                  (tcgen05 kind::f8f6f4); inference only */
  CONET_FP16 = 3,              /* FP16 activations / weights, FP32 accumulate (tcgen05) */
  CONET_TF32X3 = 4             /* FP32-accurate on tensor cores: operands split into TF32 hi +
                                  lo parts, hi*hi + hi*lo + lo*hi accumulated in FP32 (tcgen05) */
} conet_precision;

/*
 * Network and grid description (Sec. III, Fig. "Example I"; Sec. II for the grid).
 *   n_rx, n_sym, n_sc, qam_bits : N, T, F, Q.  Input channels C_in = 2 N + 3:
 *       Re Y_1..N, Im Y_1..N, pilot mask, Re / Im of the antenna-averaged LS estimate.
 *   n_branches       : 1 main net + (n_branches - 1) support nets (Sec. III, M nets).
 *   depth            : conv layers per branch (plain) or residual blocks (residual).
 *   width            : channels per conv layer in every branch.
 *   residual         : 0 plain conv+ReLU branches; 1 support = RB, main = MRB blocks.
 *   norm             : 1 = LayerNorm over channels after each Hadamard fusion.
 *   fuse_mask        : bit i = fuse after layer / block i (bit 0 = input layer);
 *                      -1 = every layer.
 *   resnet_baseline  : 1 = single pre-activation ResNet branch without fusion.
 *   max_batch        : largest B any later call may pass (sizes the workspace).
 *   train            : 1 = keep every layer's activations so that conet_backward and
 *                      conet_train_step can run (more workspace); 0 = inference only.
 *   pilot_syms[0..n_pilot_syms-1], pilot_comb, pilot_seed : the fixed pilot grid
 *       (Sec. II-A: pilots are fixed) -- QPSK pilots on symbols pilot_syms, every
 *       pilot_comb-th subcarrier starting at 0, drawn once from pilot_seed.
 *   recompute        : residual training handles only: 1 = keep, per block, only the
 *                      residual streams and recompute each block's inner activations (its
 *                      pre-activation, first conv and normalisation) from them during the
 *                      backward pass, per branch and block, instead of storing all four
 *                      tensors of every block (about 3.5x less activation memory for one
 *                      more fusion and conv launch per block).  The recomputation runs the
 *                      same kernels on the same inputs, so gradients are bitwise those of
 *                      recompute = 0.  Ignored by inference handles and plain networks.
 *   fuse_op          : the interaction at a fusion point (Sec. III: multiplication,
 *                      addition or concatenation of the subnets' activations): 0 = the
 *                      element-wise product (default), 1 = the element-wise sum, 2 = the
 *                      concatenation over channels (plain networks, n_branches x width <=
 *                      128, FP32 handles only, inference and training): the main's next conv and the
 *                      head then read n_branches x width channels, so in the flat layout
 *                      the main's layer weights after a fused layer are [C][3][3][nb C],
 *                      the fusion LayerNorm's gamma / beta [nb C] and the head [Q][nb C].
 *   feedback         : 1 = Example II (Sec. III, Fig. "conet2"): at every fusion point each
 *                      support net continues with its own activation plus the main net's
 *                      (taken before the fusion).
 *   fuse_op = 1 trains on FP32 and BF16 handles, feedback = 1 on FP32 handles without recompute
 *   (train = 1 otherwise returns CONET_ERR_UNSUPPORTED), and on the tensor-core paths (inference) need
 *   a network whose accumulators fit TMEM twice (not the 4 x 96 network).
 *   depthwise        : residual networks: 1 = every conv inside an RB / MRB is depthwise-
 *                      separable (Sec. II-A, Sec. III): a per-channel 3x3 'same' conv without
 *                      bias, then a 1x1 conv with bias.  Flat layout of such a conv: depthwise
 *                      W [C][3][3], then 1x1 W [C][C], bias [C] (in place of W, bias below).
 *                      Inference handles of precision FP32, BF16 or FP16 and FP32 training
 *                      handles (else CONET_ERR_UNSUPPORTED); BF16 / FP16 run the per-channel 3x3 on the
 *                      16-bit activations (FP32 weights and accumulation, output rounded to
 *                      the format) and the 1x1 on the tensor cores, for the 2 x 32, 3 x 64
 *                      and 4 x 96 networks (other widths: CONET_ERR_UNSUPPORTED at the
 *                      first forward).
 *   support_inputs   : 1 = selective inputs (Sec. III): the support nets (branches 1..) are
 *                      fed only the pilot information -- the pilot mask and the LS estimate
 *                      at the pilots -- and not the received signal: their input layers'
 *                      weights on the Re / Im Y channels (the first 2 n_rx of the flat
 *                      layout's c_in) act as zero whatever the parameters hold, and their
 *                      gradients are zero.  Needs n_branches >= 2 (else CONET_ERR_ARG).
 *   support_mask     : with support_inputs = 1, another subset of the inputs for the support
 *                      nets: bit j set = input channel j (of the 2 n_rx + 3 assembled
 *                      channels: Re Y per antenna, Im Y per antenna, pilot mask, Re and Im of
 *                      the LS estimate) is fed; the other channels' weights act as zero and
 *                      get zero gradients.  0 = the pilot information (bits 2 n_rx .. 2 n_rx
 *                      + 2).  Bits at or above 2 n_rx + 3, or a mask without support_inputs,
 *                      give CONET_ERR_ARG.
 */
typedef struct {
  int n_rx, n_sym, n_sc, qam_bits;
  int n_branches, depth, width;
  int residual, norm, fuse_mask, resnet_baseline;
  int max_batch;
  int train;                   /* 1 = keep every layer's activations for backward */
  int pilot_syms[4];
  int n_pilot_syms;
  int pilot_comb;
  uint64_t pilot_seed;
  int recompute;               /* 1 = recompute block activations in backward (training) */
  int fuse_op;                 /* 0 = product, 1 = sum at every fusion point */
  int feedback;                /* 1 = Example II: supports add the main net's activation */
  int depthwise;               /* 1 = depthwise-separable convs inside RB / MRB blocks */
  int support_inputs;          /* 1 = support nets see only the pilot information */
  unsigned support_mask;       /* with support_inputs: the input channels they see (0: pilots) */
} conet_config;

/*
 * Synthetic link of Sec. II, Eq. (1): y = h x + g z + n, per receive antenna.
 *   scs_hz                 subcarrier spacing (OFDM symbol = (1 + 9/128) / scs_hz).
 *   n_taps, delay_spread_s TDL with exponential power-delay profile e^-l whose rms
 *                          delay spread equals delay_spread_s.
 *   fd_lo..fd_hi           max Doppler shift, drawn uniformly per slot (Hz).
 *   snr_lo..snr_hi         Es/N0 per antenna, drawn uniformly per slot (dB);
 *                          +inf gives a noiseless grid.
 *   interferer             1 = add a co-channel QAM interferer (iqam_bits) through an
 *                          independent TDL channel, SIR drawn in sir_lo..sir_hi dB, with
 *                          a random time offset inside the cyclic prefix.
 *   awgn                   1 = replace the fading channel by h = 1.
 *   n_sinusoids            sum-of-sinusoids terms per tap (16).
 */
typedef struct {
  float scs_hz;
  int n_taps;
  float delay_spread_s;
  float fd_lo, fd_hi;
  float snr_lo, snr_hi;
  int interferer;
  float sir_lo, sir_hi;
  int iqam_bits;
  int awgn;
  int n_sinusoids;
} conet_sim_params;

/* ---------------------------------------------------------------- lifecycle */

/* Number of float parameters of the network `cfg` describes (flat layout below). */
int conet_param_count(const conet_config* cfg, size_t* n_out);

/*
 * Create a receiver.  Allocates all device memory the handle will ever need (weights
 * in every precision, gradients, Adam moments, activations for max_batch slots) on
 * the current device; later calls allocate nothing.  precision: conet_precision.
 * Flat parameter layout (FP32, the order save/load use), per branch b = 0..n_br-1:
 *   input conv W [C][3][3][C_in], bias [C];
 *   plain: layers l = 1..depth-1: W [C][3][3][C], bias [C];
 *   residual: blocks k: (support or resnet only) ln1 gain [C], ln1 shift [C];
 *             conv1 W, bias; ln2 gain, shift; conv2 W, bias;
 * then (norm = 1) one LayerNorm gain [C], shift [C] per fusion point in order;
 * then head W [Q][C], bias [Q].
 */
int conet_create(const conet_config* cfg, int precision, conet_t* out);
void conet_destroy(conet_t h);

/* He-normal weights (std sqrt(2 / fan_in)), zero biases, LayerNorm gain 1 / shift 0,
 * drawn on the device from Philox4x32-10 with the given seed; zeroes Adam state. */
int conet_init_he(conet_t h, uint64_t seed, void* stream);

/* Copy n floats (must equal conet_param_count) from / to host memory; synchronises.
 * A wrong n returns CONET_ERR_WEIGHTS and changes nothing.  Load zeroes Adam state. */
int conet_load_weights(conet_t h, const float* host_params, size_t n);
int conet_save_weights(conet_t h, float* host_params, size_t n);

/*
 * Versioned training checkpoint, so that an interrupted run resumes exactly: a 64-byte
 * header (magic "CONETCK", format version 1, a 64-bit FNV-1a hash of the network shape and
 * pilot grid, the parameter count n, the caller's Adam step, the handle's precision), then
 * n FP32 master parameters, n Adam first moments and n Adam second moments in the flat
 * layout above.  The training workflow of Sec. IV needs the optimiser state as well as the
 * weights; the paper specifies no file format.
 *   conet_checkpoint_hash   the header's hash of a config (host only, no handle needed).
 *   conet_checkpoint_bytes  size of a checkpoint of this handle.
 *   conet_save_checkpoint   host_buf (host, exactly that size) <- the handle's state, with
 *                           adam_step recorded (the `step` a following conet_train_step
 *                           takes); synchronises the device.
 *   conet_load_checkpoint   the handle's parameters and Adam moments <- host_buf, re-deriving
 *                           the kernels' weight layouts; *adam_step (may be NULL) <- the
 *                           recorded step; synchronises.  A buffer that is not a version-1
 *                           checkpoint of a network with the same hash and parameter count,
 *                           or of the wrong size, returns CONET_ERR_WEIGHTS and changes
 *                           nothing.
 * Resuming with the loaded state and the recorded step continues bitwise as the
 * uninterrupted run would (every training kernel reduces in a fixed order).
 */
int conet_checkpoint_hash(const conet_config* cfg, uint64_t* hash);
int conet_checkpoint_bytes(conet_t h, size_t* bytes);
int conet_save_checkpoint(conet_t h, uint64_t adam_step, void* host_buf, size_t bytes);
int conet_load_checkpoint(conet_t h, const void* host_buf, size_t bytes, uint64_t* adam_step);

/* Views of the library's FP32 master parameters and their gradients (device, n floats,
 * flat layout above), valid until conet_destroy. */
int conet_params_device(conet_t h, float** dev_params, size_t* n);
int conet_grads_device(conet_t h, float** dev_grads, size_t* n);

/* After the caller changed the master parameters in place (through conet_params_device,
 * e.g. with its own optimiser), re-derive the kernels' weight layouts from them, on
 * `stream`; conet_load_weights, conet_init_he and conet_adam_step do this themselves.  E4M3
 * handles recalibrate their activation scales on the next forward. */
int conet_params_updated(conet_t h, void* stream);

/* ---------------------------------------------------------------- forward / backward */

/*
 * Receive B slots: input assembly (Sec. II-A) -> all CoNet branches with Hadamard
 * fusion (Sec. III) -> 1x1 head, writing per-RE per-bit LLRs.
 *   Y          dev float [B][N][T][F][2]   received grid
 *   pilot_mask dev uint8 [T][F]            1 on pilot REs (must match the config's grid)
 *   noise_var  dev float [B] or NULL       per-slot noise variance (unused by the
 *                                          network inputs; accepted for the ABI)
 *   llr        dev float [B][T][F][Q]      output (pilot REs hold values that
 *                                          loss and BER ignore)
 * 0 < B <= max_batch, else CONET_ERR_SHAPE.  Keeps the activations for a following
 * conet_backward on the same handle.
 */
int conet_forward(conet_t h, const float* Y, const uint8_t* pilot_mask, const float* noise_var,
                  int B, float* llr, void* stream);

/*
 * CUDA-graph replay of conet_forward (on by default for inference handles).  The first
 * call with given (Y, pilot_mask, B, llr) pointers and batch runs eagerly; a second
 * identical call captures its launches into a CUDA graph on an internal stream and
 * launches it on the caller's stream; later identical calls only launch the graph, so a
 * launch-bound small batch costs one graph launch instead of one launch per kernel.
 * Results are identical to the eager forward: the graph runs the same kernels on the same
 * buffers (weights loaded later are read from those buffers).  Training handles, launch
 * profiling and an E4M3 pass that still calibrates always run eagerly; a capture that
 * fails turns replay off for the handle.  enable = 0 turns it off (and drops the graph).
 */
int conet_graphs(conet_t h, int enable);

/*
 * Whole-network kernel for small plain networks (2 branches x 32 channels, T (F + 1) <=
 * 1024, up to 8 layers, BF16 or calibrated E4M3 inference handles, product fusion): every
 * layer and the head of a slot run in one kernel whose activations stay in shared memory,
 * instead of one launch per layer (the 14 x 72 networks of the paper's Example I, Sec. III,
 * are launch- and L2-bound layer by layer).  Large calls run one slot per CTA; calls of few
 * slots split each slot over a cluster of 8, 4 or 2 CTAs (one per SM) that exchange the
 * rows at their tile boundaries through distributed shared memory (grids of F + 2 <= 128
 * columns).  Results equal the layer-by-layer path of the same precision up to FP32
 * accumulation order (and, for E4M3, the rare activation code that order moves).
 * enable: 0 = never (layer by layer), 1 = automatic (the default: forward calls of at least
 * CONET_WHOLE_NET_MIN_SLOTS slots), 2 = every forward call.  An E4M3 forward that
 * calibrates runs layer by layer.  *available (may be NULL) <- 1 when the handle's network
 * qualifies.  Errors: CONET_ERR_ARG for a NULL handle or enable outside 0..2.
 */
#define CONET_WHOLE_NET_MIN_SLOTS 1
int conet_whole_network(conet_t h, int enable, int* available);

/*
 * Activation scales of a CONET_FP8E4M3 handle.  Every conv input (the assembled grid and each
 * branch's activation entering each conv) is stored as E4M3 of value / s with one scale s per
 * tensor; the weights of each output channel carry their own scale (the smallest power of
 * two >= largest |w| / 448), and the FP32 accumulator is multiplied back by s x that channel
 * scale before the bias (the FP8 variant of the convolutions of Sec. III).  E4M3 values are
 * rounded to nearest even and saturate at +-448.  This call runs the forward pass on the
 * first min(B, activation chunk) of the given slots and sets each s = the smallest power of
 * two >= margin x (largest |value| of that tensor on them) / 448; larger values met later
 * saturate at +-448 s.  Arguments as for
 * conet_forward; margin in [1, 448], else CONET_ERR_ARG.  Handles of other precisions
 * return CONET_OK and change nothing.  A forward pass on an FP8 handle whose weights changed
 * since its last calibration (or that was never calibrated) first calibrates on its own
 * first chunk with margin 2.  Writes no caller memory; asynchronous on `stream`.
 */
int conet_calibrate(conet_t h, const float* Y, const uint8_t* pilot_mask, int B, float margin, void* stream);

/*
 * Backward of the last conet_forward on this handle for upstream gradient dllr (dev
 * float [B][T][F][Q], same B).  Writes the parameter gradient (flat layout) into the
 * buffer conet_grads_device exposes (overwritten, not accumulated).
 * CONET_ERR_ARG if no forward with this B preceded it or the handle was created with
 * train = 0.
 */
int conet_backward(conet_t h, const float* dllr, int B, void* stream);

/*
 * Weight and bias gradient of one 3x3 'same' convolution layer (zero padding 1 on the
 * symbol and subcarrier axes, as every CoNet conv of Sec. III), the weight-gradient step of
 * conet_backward exposed for callers that run their own backward pass:
 *   dW[co][kh][kw][ci] = sum_{b,t,f} dz[b][t][f][co] x[b][t+kh-1][f+kw-1][ci]   (0 outside)
 *   db[co]             = sum_{b,t,f} dz[b][t][f][co]
 *   x  dev float [B][T][F][cin]     layer input, channels last
 *   dz dev float [B][T][F][cout]    gradient w.r.t. the layer output (pre-activation)
 *   dW dev float [cout][3][3][cin]  overwritten;  db dev float [cout] or NULL
 * cin and cout are multiples of 4 in 4..128.  The split partial sums live in scratch that
 * this call allocates and frees stream-ordered (cudaMallocAsync / cudaFreeAsync on `stream`);
 * the sum over splits runs in a fixed order, so results are deterministic.
 */
int conet_conv3x3_wgrad(const float* x, const float* dz, int B, int T, int F, int cin, int cout, float* dW,
                        float* db, void* stream);

/*
 * The same weight and bias gradient for callers that cannot allocate device memory when
 * they need it: a real-time receiver or training loop that plans all memory at start-up, code
 * running inside a CUDA graph capture, or an embedding that only owns its own buffers.  The
 * paper has no counterpart: this is a deployment variant of the library's own op.
 * Arguments, layouts and results are those of conet_conv3x3_wgrad; the call allocates and
 * frees nothing.  Its partial sums live in one array compiled into the library (about
 * 4.25 MiB, held by every GPU that loads the library until the process exits); a size whose
 * partials would not fit returns CONET_ERR_SHAPE (never the case for cin, cout <= 128 with
 * the library's split rule).  The first call on each device, with that device current,
 * looks up the array's device address once (cudaGetSymbolAddress) and keeps it: make that
 * first call before any stream capture.  The kept address is valid until the device is reset;
 * do not call this entry point on a device after cudaDeviceReset in the same process.  All
 * calls share the array, so calls that overlap on the GPU (other streams, other host threads)
 * race; serialise them.
 */
int conet_conv3x3_wgrad_noalloc(const float* x, const float* dz, int B, int T, int F, int cin, int cout,
                                float* dW, float* db, void* stream);

/* One bias-corrected Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the master
 * parameters with the current gradient; `step` counts from 1. */
int conet_adam_step(conet_t h, float lr, int step, void* stream);

/*
 * One training step on freshly simulated slots (the paper trains on simulated TDL
 * slots, Sec. IV): simulate B slots (seed, global slots step*B .. step*B+B-1) ->
 * forward -> mean BCE-with-logits over data REs -> backward -> Adam (step + 1).
 * loss_out (host, may be NULL): when non-NULL the call synchronises and returns the
 * mean loss; CONET_ERR_NONFINITE if it is not finite.
 */
int conet_train_step(conet_t h, const conet_sim_params* sim, uint64_t seed, uint64_t step, int B,
                     float lr, double* loss_out, void* stream);

/* ---------------------------------------------------------------- link and DSP */

/* Fixed pilot grid of `cfg`: mask dev uint8 [T][F], pilot symbols dev float [T][F][2]
 * (0 on data REs). */
int conet_pilots(const conet_config* cfg, uint8_t* mask, float* pilot_sym, void* stream);

/*
 * Simulate B slots of Eq. (1) (global slot ids slot0 .. slot0+B-1) with Philox4x32-10
 * keyed by `seed`.  fixed_snr_db: NaN = draw per slot from sim->snr_lo..snr_hi.
 *   Y dev float [B][N][T][F][2]; bits dev uint8 [B][T][F][Q] (0 on pilot REs);
 *   H dev float [B][N][T][F][2] or NULL; noise_var dev float [B]; interf_var dev
 *   float [B] or NULL (P_I, 0 without interferer).
 */
int conet_sim_generate(const conet_config* cfg, const conet_sim_params* sim, uint64_t seed,
                       uint64_t slot0, int B, float fixed_snr_db, float* Y, uint8_t* bits,
                       float* H, float* noise_var, float* interf_var, void* stream);

/*
 * Network input of Sec. II-A: X0 dev float [B][T][F][C_in] with channels Re Y_n,
 * Im Y_n (n = 1..N), pilot mask, Re / Im of (1/N) sum_n y_n conj(p) / |p|^2 at pilot
 * REs (0 elsewhere).  pilot_sym dev float [T][F][2].
 */
int conet_assemble_input(const conet_config* cfg, const float* Y, const uint8_t* pilot_mask,
                         const float* pilot_sym, int B, float* X0, void* stream);

/*
 * LS-LMMSE receiver (the conventional baseline of Sec. I and Sec. IV): LS at pilots,
 * linear interpolation across subcarriers then symbols, SIMO LMMSE with
 * s2 = noise_var (+ interf_var, interference as noise), then exact (demap_exact = 1)
 * or max-log demapping.  H_perfect (dev [B][N][T][F][2]) replaces the estimate when
 * non-NULL (perfect CSI).  llr dev float [B][T][F][Q].
 */
int conet_ls_lmmse(const conet_config* cfg, const float* Y, const uint8_t* pilot_mask,
                   const float* pilot_sym, const float* noise_var, const float* interf_var,
                   const float* H_perfect, int demap_exact, int B, float* llr, void* stream);

/*
 * Mean-BCE loss and bit-error counters over data REs (hard decision [LLR > 0]).
 * Accumulates into caller-owned device counters (zero them first):
 *   loss_sum  dev double[1]  += sum of softplus(L) - b L
 *   err_bits  dev u64[1]     += hard-decision errors;  n_bits dev u64[1] += bits counted.
 * dllr (dev float [B][T][F][Q] or NULL) receives (sigmoid(L) - b) * grad_scale on data
 * REs and 0 on pilots.  Any of loss_sum / err_bits / n_bits may be NULL.
 */
int conet_loss_ber(const float* llr, const uint8_t* bits, const uint8_t* pilot_mask, int B, int T,
                   int F, int Q, float grad_scale, float* dllr, double* loss_sum,
                   unsigned long long* err_bits, unsigned long long* n_bits, void* stream);

/*
 * Bit-error counting alone (the BER of Sec. IV's figures): over the data REs of llr (dev
 * float [B][T][F][Q], pilot REs where pilot_mask [T][F] is 1 are skipped) the hard
 * decisions [LLR > 0] are compared with bits (dev u8 [B][T][F][Q]); err_bits += the
 * errors, n_bits += the bits compared (caller-owned device u64 counters, zero them first;
 * either may be NULL).  The same kernel and counts as conet_loss_ber with no loss or
 * gradient.  CONET_ERR_ARG / CONET_ERR_SHAPE on the host for NULL inputs or bad sizes.
 */
int conet_ber_count(const float* llr, const uint8_t* bits, const uint8_t* pilot_mask, int B, int T, int F,
                    int Q, unsigned long long* err_bits, unsigned long long* n_bits, void* stream);

/* ---------------------------------------------------------------- diagnostics */

/*
 * Per-kernel timing of a handle's launches with CUDA events recorded on the launch
 * stream (no synchronisation while enabled).  kind: 0 = body 3x3 convolutions
 * (C -> C), 1 = input convolution, 2 = fusion / LayerNorm / head stage, 3 = input
 * assembly, 4 = backward kernels, 5 = Adam.  conet_profile_read synchronises the
 * device, returns the summed milliseconds and the launch count of that kind since the
 * last enable, and leaves profiling on.  At most 65536 launches are recorded.
 */
int conet_profile_enable(conet_t h, int enable);
int conet_profile_read(conet_t h, int kind, double* total_ms, long long* launches);

/*
 * Wait for `stream` and report device-side failures of this handle's kernels since the
 * last call: CONET_ERR_TIMEOUT when a bounded pipeline wait gave up, CONET_ERR_NONFINITE
 * when a forward pass wrote a NaN or infinite LLR (both status words are then cleared; a
 * timeout is reported first), CONET_ERR_CUDA for an asynchronous CUDA error.
 */
int conet_sync(conet_t h, void* stream);

/*
 * Failure-detection self-test: launches one kernel on `stream` that waits, with the same
 * bounded mbarrier wait as the tensor-core pipelines but a limit of limit_s seconds
 * (1e-6 .. 1, else CONET_ERR_ARG), for a phase that nothing completes.  The wait gives up,
 * records its site (100) in the handle's status word and the kernel returns, so the next
 * conet_sync returns CONET_ERR_TIMEOUT and the context stays usable.  Diagnostics only:
 * the paper has no counterpart.
 */
int conet_selftest_timeout(conet_t h, double limit_s, void* stream);

/* Kernel launches issued by this library in this process so far (all handles); a replayed
 * forward graph (conet_graphs) counts the kernels it runs. */
unsigned long long conet_launch_count(void);

/* Thread-local text of the last error (never NULL). */
const char* conet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CONET_H */
