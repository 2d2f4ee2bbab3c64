"""GPU parity of the E4M3 tensor-core path (CONET_FP8E4M3: tcgen05 kind::f8f6f4 convolutions,
per-output-channel weight scales, per-tensor activation scales calibrated on the batch,
FP32 accumulation and epilogue).

Two references:
* the oracle's E4M3 emulation of the same network (oracle/fp8.py: the same quantisation
  points, power-of-two scales from the same calibration rule, FP64 arithmetic elsewhere).
  This is the parity check proper: the GPU and the emulation round the same values to the
  same E4M3 codes, except where an FP32 value and its FP64 counterpart fall on opposite
  sides of a rounding boundary (a few in 10^5 elements, each moving one code).
  On networks with a LayerNorm after a Hadamard fusion the normalisation amplifies such a
  one-code difference (and the FP32-vs-FP64 differences that decide it) by up to
  1/sqrt(eps) ~ 316 at He initialisation, where the fused products' variance sits near the
  LN epsilon: the element-wise maximum bar there is 0.2 (measured up to 0.15 on the 17-conv
  96-channel network, median 1e-7); at trained weights it is 0.15
  (test_gpu_trained_parity.py);
* the unquantised FP64 oracle, against which the format's own error is stated: 3 mantissa
  bits give a relative rounding error up to 2^-4 per operand, and on the plain 14 x 72
  networks the E4M3 network's LLRs sit within 6e-2 of the largest LLR at the 99th
  percentile (max ~0.1-0.2, the same in the emulation: the format, not the kernel).
"""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, torch
from workloads import WORKLOADS, replace

pytestmark = pytest.mark.gpu
TOL_EMU = 1e-2          # vs the E4M3 emulation, normwise (measured <= 3.4e-4 on plain networks)
MAX_EMU_LN = 0.2        # vs the E4M3 emulation, normwise maximum, LayerNorm-fused networks at He init
MED_EMU = 1e-5          # vs the E4M3 emulation, median element error / max |L|
TOL_FP8 = 6e-2          # vs FP64, the normwise accuracy target for E4M3


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def run_fp8(net, sim, B, seed=1, wseed=2, perturb=0.0, params=None):
    from oracle import net as onet, pipeline
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(net, sim, seed, 0, B)
    if params is None:
        params = onet.init_params(net, wseed)
        if perturb:
            params = params + perturb * np.random.default_rng(wseed).standard_normal(params.size)
    params = np.asarray(params, dtype=np.float32)
    rx = api.Receiver(net, precision="fp8", max_batch=B)
    rx.load_weights(params)
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).cpu().numpy()
    rx.sync()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    p64 = params.astype(np.float64)
    L_emu = pipeline.receive_fp8(net, p64, Yd, ref["pilot_sym"], ref["pilot_mask"], margin=2.0)
    L_ref = pipeline.receive(net, p64, Yd, ref["pilot_sym"], ref["pilot_mask"])
    return L, L_emu, L_ref


def ln_fused(net):
    return bool(net.norm or net.residual) and net.n_branches >= 2


def check_emu(L, L_emu, net, ln_max=MAX_EMU_LN, med=MED_EMU):
    assert np.all(np.isfinite(L))
    scale = np.max(np.abs(L_emu))
    err = np.abs(L - L_emu) / scale
    tol = ln_max if ln_fused(net) else TOL_EMU
    assert err.max() < tol, err.max()
    assert np.median(err) < med, np.median(err)
    sure = np.abs(L_emu) > tol * scale
    assert np.mean((L > 0)[sure] == (L_emu > 0)[sure]) >= 0.999


def check_fp64_plain(L, L_ref):
    """The format's own error against FP64 on the plain 14 x 72 networks: the
    6e-2 normwise target is not met by post-training E4M3 at He init (measured max 0.09-0.18,
    the emulation shows the same: 3 mantissa bits per operand over 4 layers), so the maximum
    is held to 0.25 and the 6e-2 bar is an expected failure (test_fp8_6e2_bar_plain).
    Hard decisions agree on >= 99.5 % of the bits whose FP64 LLR exceeds 6e-2 of the largest:
    a relative operand error up to 2^-4 flips more near-boundary decisions than BF16's 2^-8."""
    scale = np.max(np.abs(L_ref))
    err = normwise(L, L_ref)
    assert err < 0.25, err
    sure = np.abs(L_ref) > TOL_FP8 * scale
    assert np.mean((L > 0)[sure] == (L_ref > 0)[sure]) >= 0.995


def test_fp8_interference_14x72_b16():
    """The FP8 interference workload's network (1 Rx, 2 branches x 4 conv x 32) on slots with
    a co-channel 64-QAM interferer."""
    w = WORKLOADS["interf_14x72_b512_fp8"]
    L, L_emu, L_ref = run_fp8(w.net, w.sim, 16)
    check_emu(L, L_emu, w.net)
    check_fp64_plain(L, L_ref)


@pytest.mark.xfail(reason="post-training E4M3 on the plain 14x72 network: max 0.09-0.18 > 6e-2", strict=False)
def test_fp8_6e2_bar_plain():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    L, _, L_ref = run_fp8(w.net, w.sim, 8, perturb=0.02)
    assert normwise(L, L_ref) < TOL_FP8


def test_fp8_plain_14x72_perturbed():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    L, L_emu, L_ref = run_fp8(w.net, w.sim, 8, perturb=0.02)
    check_emu(L, L_emu, w.net)
    check_fp64_plain(L, L_ref)


@pytest.mark.parametrize("F", [1, 129, 200])
def test_fp8_ragged_grids(F):
    """One RE per tile, a one-column last tile, and a partial last tile of 128."""
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_branches=3, width=32, depth=3, n_sc=F)
    L, L_emu, L_ref = run_fp8(net, w.sim, 2, perturb=0.02)
    check_emu(L, L_emu, net)


def test_fp8_plain_with_layernorm():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, norm=1, depth=3, n_sc=150)
    L, L_emu, _ = run_fp8(net, w.sim, 2, perturb=0.02)
    check_emu(L, L_emu, net)


def test_fp8_residual_64_ragged():
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37)
    L, L_emu, _ = run_fp8(net, w.sim, 2, perturb=0.02)
    check_emu(L, L_emu, net)


def test_fp8_residual_96_four_antennas():
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    net = replace(w.net, n_sc=29, depth=2)
    L, L_emu, _ = run_fp8(net, w.sim, 1, perturb=0.02)
    check_emu(L, L_emu, net)


def test_fp8_one_branch_64():
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_branches=1, n_sc=40, depth=2)
    L, L_emu, _ = run_fp8(net, w.sim, 2, perturb=0.02)
    check_emu(L, L_emu, net)


def test_per_output_channel_weight_scales():
    """Scaling output channel c of the main branch's last conv (weights and bias) by 2^-k_c,
    k_c up to 23, and the head's column c by 2^k_c leaves the network unchanged.  With one
    scale per output channel the E4M3 codes and the dequantised products are the same, so the
    LLRs must be bitwise equal; a per-tensor weight scale would flush those rows to zero."""
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["interf_14x72_b512_fp8"]
    net = w.net
    p = onet.init_params(net, 2).astype(np.float32)
    P = onet.unflatten(net, p.copy())
    k = np.arange(net.width) % 24
    last = net.depth - 1
    P[f"b0.l{last}.w"][...] *= (2.0 ** -k)[:, None, None, None]
    P[f"b0.l{last}.b"][...] *= 2.0 ** -k
    P["head.w"][...] *= (2.0 ** k)[None, :]
    p2 = np.concatenate([P[n].ravel() for n, _ in onet.param_layout(net)]).astype(np.float32)
    ref = oracle_inputs(net, w.sim, 3, 0, 4)
    out = []
    for params in (p, p2):
        rx = api.Receiver(net, precision="fp8", max_batch=4)
        rx.load_weights(params)
        out.append(rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])))
        rx.sync()
    assert torch.equal(out[0], out[1])


def test_calibration_rules():
    """Explicit calibration on the forward's own slots equals the automatic first-forward
    calibration; new weights trigger a new calibration; bad margins are rejected."""
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS["interf_14x72_b512_fp8"]
    net = w.net
    s = api.sim_generate(net, w.sim, 4, 0, 8)
    mask, _ = api.pilots(net)
    a = api.Receiver(net, precision="fp8", max_batch=8)
    a.init_he(1)
    La = a.forward(s["Y"], mask)
    b = api.Receiver(net, precision="fp8", max_batch=8)
    b.whole_network(False)     # bitwise comparisons: the same (layer-by-layer) kernels as a's calibrating pass
    b.load_weights(a.save_weights())
    b.calibrate(s["Y"], mask, margin=2.0)
    assert torch.equal(b.forward(s["Y"], mask), La)
    # other weights: a calibrated handle recalibrates after load_weights
    c = api.Receiver(net, precision="fp8", max_batch=8)
    c.init_he(2)
    Lc = c.forward(s["Y"], mask)
    b.load_weights(c.save_weights())
    assert torch.equal(b.forward(s["Y"], mask), Lc)
    # a larger margin leaves more headroom: different codes, still close
    b.calibrate(s["Y"], mask, margin=8.0)
    L8 = b.forward(s["Y"], mask)
    assert normwise(L8.cpu().numpy(), Lc.cpu().numpy()) < 0.3
    with pytest.raises(ConetError):
        b.calibrate(s["Y"], mask, margin=0.5)
    b.sync()


def test_fp8_interference_full_batch_sampled_slots():
    """The FP8 interference workload at its full batch of 512 slots (scales calibrated on all
    of them): sampled slots against the emulation calibrated on the same 512 slots."""
    from oracle import fp8, net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["interf_14x72_b512_fp8"]
    B = w.batch
    ref = oracle_inputs(w.net, w.sim, 5, 0, B)
    params = onet.init_params(w.net, 6).astype(np.float32)
    rx = api.Receiver(w.net, precision="fp8", max_batch=B)
    rx.load_weights(params)
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).cpu().numpy()
    rx.sync()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    L_emu = fp8.forward_fp8(w.net, params.astype(np.float64), X0)
    for b in (0, 255, B - 1):
        check_emu(L[b:b + 1], L_emu[b:b + 1], w.net)


def _calibrated_pair(w, B, n_cal, wseed):
    """A handle calibrated explicitly on the first n_cal slots, then run on all B slots (the
    workload's batch, as the benchmark runs it); the oracle's scales from the same slots."""
    from oracle import net as onet, pipeline
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(w.net, w.sim, 7, 0, B)
    params = onet.init_params(w.net, wseed).astype(np.float32)
    rx = api.Receiver(w.net, precision="fp8", max_batch=B)
    rx.load_weights(params)
    Y, mask = dev(ref["Y32"]), dev(ref["pilot_mask"])
    rx.calibrate(Y[:n_cal].contiguous(), mask, margin=2.0)
    L = rx.forward(Y, mask).cpu().numpy()
    rx.sync()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    p64 = params.astype(np.float64)
    scales = pipeline.calibrate_fp8(w.net, p64, Yd[:n_cal], ref["pilot_sym"], ref["pilot_mask"])
    return L, ref, Yd, p64, scales


def test_fp8_resid_14x624_full_batch_calibrated_on_four_slots():
    """The 14 x 624 residual network in E4M3 at the benchmark's batch of 256, scales
    calibrated on 4 slots: sampled slots against the emulation with the oracle's scales
    from the same 4 slots."""
    from oracle import pipeline
    w = WORKLOADS["resid_14x624_b256_fp32"]
    L, ref, Yd, p64, scales = _calibrated_pair(w, w.batch, 4, 8)
    for b in (0, 131, w.batch - 1):
        L_emu = pipeline.receive_fp8(w.net, p64, Yd[b:b + 1], ref["pilot_sym"], ref["pilot_mask"], scales=scales)
        check_emu(L[b:b + 1], L_emu, w.net)


def test_fp8_resid_14x3276_sampled_res_calibrated_on_one_slot():
    """The 14 x 3276, 4-branch x 96 network in E4M3 (branch groups of two), B = 6, scales
    calibrated on one slot: sampled subcarriers against the emulation on the exact
    receptive-field crop with the oracle's scales from that slot.

    This network is 17 convs deep with a LayerNorm after each of its 9 fusions.  An output's
    receptive field holds millions of quantised values, so the rare codes that FP32 and FP64
    round to opposite sides of a boundary are many, and their normalised effect spreads
    over the whole distribution.  Measured on 896 LLRs: median 2.5e-4, 99th percentile
    3.9e-2, max 7.4e-2, hard decisions all equal.  The E4M3 format's own error against FP64
    on these networks is ~100x the median.  The bar is 1e-3 at the median and 0.15 at the
    element-wise maximum."""
    from gpu_util import receptive_radius
    from oracle import fp8, rx as orx
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    L, ref, Yd, p64, scales = _calibrated_pair(w, 6, 1, 9)
    R = receptive_radius(w.net)
    got, want = [], []
    for b, f in [(0, 0), (3, 1637), (5, 3275), (1, 128), (2, 2000)]:
        lo, hi = max(0, f - R), min(w.net.n_sc, f + R + 1)
        X0 = orx.assemble_input(Yd[b:b + 1, :, :, lo:hi], ref["pilot_sym"][:, lo:hi], ref["pilot_mask"][:, lo:hi])
        crop = replace(w.net, n_sc=hi - lo)
        Lc = fp8.forward_fp8(crop, p64, X0, scales=scales)
        got.append(L[b, :, f, :])
        want.append(Lc[0, :, f - lo, :])
    check_emu(np.array(got), np.array(want), w.net, ln_max=0.15, med=1e-3)
