// Host-side logic of the tensor-core conv, compiled and run on the CPU by
// tests/test_host_logic.py (no kernel is launched): the stage plan of every instantiated
// shape fits shared memory and TMEM, and tc_mode picks the fixed-shape epilogues exactly
// for the argument patterns they assume.
#include <cstdio>

#include "../../paper_2510_12739_gb300/csrc/conv_tc.cuh"

using namespace conet;

static int failures = 0;
#define CHECK(cond)                                                       \
  do {                                                                    \
    if (!(cond)) {                                                        \
      std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #cond);         \
      ++failures;                                                         \
    }                                                                     \
  } while (0)

template <int KI, int NB, int CI, int CO>
void check_plan() {
  constexpr int KC = tc_kc(KI, NB, CI, CO), HALO = tc_halo(KI, NB, CI, CO);
  static_assert(KC > 0, "a stage plan exists");
  using K = Cfg<KI, NB, CI, CO, KC, HALO>;
  CHECK(K::SMEM <= SMEM_LIMIT);
  CHECK(K::STAGES >= (HALO ? 3 : 2));
  CHECK(K::TMEM_COLS <= 512);
  CHECK(K::THREADS == 64 + 128 * K::EP);
  CHECK((long)K::THREADS * (K::EP == 3 ? 128 : 96) <= 65536);
}

// The one-tap stage of the 1x1 convs of depthwise-separable blocks (HALO = 2): the tile's
// own rows and one weight tap per stage, Cin / KC K steps per tile, with the same fixed
// epilogue shapes as the 3x3 body convs.
template <int KI, int NB, int C>
void check_pointwise_plan() {
  constexpr int KC = tc_plan(KI, NB, C, C, false);
  static_assert(KC > 0, "a one-tap stage plan exists");
  using K = Cfg<KI, NB, C, C, KC, 2, 2>;
  using K3 = Cfg<KI, NB, C, C, tc_kc(KI, NB, C, C), tc_halo(KI, NB, C, C), 2>;
  CHECK(K::TAPS == 1 && K::A_BOX == TILE_M);
  CHECK(K::K_ITERS == C / KC);
  CHECK(K::STAGE_TX == K::G * (TILE_M * K::ROW + (C / 2) * K::ROW));   // both TMA boxes of a stage
  CHECK(K::SMEM <= SMEM_LIMIT && K::STAGES >= 2);
  CHECK(K::TMEM_COLS == K3::TMEM_COLS && K::EP == K3::EP && K::STAGED == K3::STAGED);
}

static TcConvArgs base_args(int nb) {
  static float f[64];
  static float out[64];
  static unsigned short h[64];
  TcConvArgs a = {};
  for (int b = 0; b < nb; ++b) {
    a.bias[b] = f;
    a.nx_out[b] = h;
  }
  (void)out;
  return a;
}

int main() {
  check_pointwise_plan<0, 2, 32>();
  check_pointwise_plan<0, 3, 64>();
  check_pointwise_plan<0, 4, 96>();
  check_pointwise_plan<3, 3, 64>();
  check_plan<0, 3, 16, 64>();
  check_plan<0, 3, 64, 64>();
  check_plan<0, 4, 16, 96>();
  check_plan<0, 4, 96, 96>();
  check_plan<0, 2, 32, 32>();
  check_plan<3, 3, 64, 64>();
  check_plan<1, 3, 64, 64>();
  check_plan<1, 4, 96, 96>();
  check_plan<1, 1, 112, 112>();
  check_plan<2, 3, 64, 64>();
  check_plan<2, 4, 96, 96>();
  check_plan<2, 2, 32, 32>();
  check_plan<0, 4, 16, 64>();
  check_plan<0, 4, 64, 64>();
  check_plan<0, 1, 16, 96>();
  check_plan<0, 1, 96, 96>();

  static float buf[64];
  // conv1 of a residual block: LN2 + ReLU, next input only
  TcConvArgs a = base_args(3);
  a.pre = 2;
  for (int b = 0; b < 3; ++b) {
    a.ln2_g[b] = buf;
    a.ln2_b[b] = buf;
  }
  CHECK(tc_mode(0, 3, 64, 64, a) == 1);
  a.a_out[1] = buf;                          // an extra output: run-time epilogue
  CHECK(tc_mode(0, 3, 64, 64, a) == 0);

  // conv2 of a fused residual block
  TcConvArgs c = base_args(3);
  c.pre = 0;
  c.fuse = 1;
  c.lnf_g = buf;
  c.lnf_b = buf;
  for (int b = 0; b < 3; ++b) {
    c.resid[b] = buf;
    c.xs_out[b] = buf;
    c.post[b] = b == 0 ? 1 : 2;
    if (b) {
      c.ln1_g[b] = buf;
      c.ln1_b[b] = buf;
    }
  }
  CHECK(tc_mode(0, 3, 64, 64, c) == 2);
  TcConvArgs d = c;
  d.head_w = buf;                            // the last block feeds the head, and still has outputs
  CHECK(tc_mode(0, 3, 64, 64, d) == 0);
  for (int b = 0; b < 3; ++b) d.nx_out[b] = nullptr;
  d.llr = buf;                               // only the head: the fast head shape where it serves
  CHECK(tc_mode(0, 3, 64, 64, d) == 4);
  TcConvArgs d4 = d;
  d4.resid[3] = buf;
  d4.xs_out[3] = buf;
  CHECK(tc_mode(0, 4, 96, 96, d4) == 4);     // branch groups: the stash holds the product
  CHECK(tc_mode(0, 4, 64, 64, d4) == 0);     // no spare accumulator columns for the product
  CHECK(tc_mode(2, 3, 64, 64, d) == 4);      // E4M3: four even parts of 16 channels
  CHECK(tc_mode(1, 3, 64, 64, d) == 0);      // split TF32: no staged epilogue
  d.a_out[0] = buf;                          // training outputs: run-time epilogue
  CHECK(tc_mode(0, 3, 64, 64, d) == 0);
  d = c;
  d.post[0] = 2;                             // a normalised main branch is not the fixed shape
  CHECK(tc_mode(0, 3, 64, 64, d) == 0);
  d = c;
  d.measure = 1;                             // E4M3 calibration passes stay run-time
  CHECK(tc_mode(2, 3, 64, 64, d) == 0);
  CHECK(tc_mode(2, 3, 64, 64, c) == 0);              // E4M3 needs its output scales
  for (int b = 0; b < 3; ++b) d.qinv[b] = buf;
  d.measure = 0;
  CHECK(tc_mode(2, 3, 64, 64, d) == 2);
  CHECK(tc_mode(1, 3, 64, 64, c) == 0);              // split TF32 needs the low parts
  for (int b = 0; b < 3; ++b) d.nx_lo[b] = buf;
  CHECK(tc_mode(1, 3, 64, 64, d) == 2);

  // input layer of a fused residual network: ReLU pre-activation, no residual
  TcConvArgs e = c;
  e.pre = 1;
  for (int b = 0; b < 3; ++b) e.resid[b] = nullptr;
  CHECK(tc_mode(0, 3, 16, 64, e) == 3);
  e.resid[2] = buf;                          // partly residual: neither shape
  CHECK(tc_mode(0, 3, 16, 64, e) == 0);

  // one branch never takes a fixed shape (no fusion)
  CHECK(tc_mode(0, 1, 64, 64, a) == 0);

  if (failures) return 1;
  std::printf("host logic ok\n");
  return 0;
}
