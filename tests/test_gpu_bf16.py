"""GPU parity of the 16-bit tensor-core paths (tcgen05 implicit-GEMM convolutions with the
fused Hadamard / LayerNorm / head epilogue, BF16 or FP16 operands, FP32 accumulation).

Networks without a LayerNorm after a Hadamard fusion: LLRs within 2e-2 of the largest FP64
oracle LLR at every element (normwise maximum), and >= 99.9 % hard-decision agreement on
every bit whose oracle LLR is not itself within that error of zero.

Networks with a LayerNorm after a fusion (the residual CoNets, plain ones with norm = 1),
here at random initialisation: the fused product is a product of several ReLU outputs, and
its variance over channels sits below 100 x the LN epsilon (1e-5) at most REs and reaches 0
at some; the normalisation divides by sqrt(var + eps), so the 16-bit format's own rounding
is amplified up to 1/sqrt(eps) ~ 316 there, and the FP64 distance at He init is the format's
conditioning, not the kernel's (measured up to 5.5e-2 BF16 / 1.2e-2 FP16 on the 6-block 64-
channel network, and on the 8-block 96-channel one a fused variance of exactly 0).  These
tests therefore compare against the oracle's emulation of the same 16-bit receiver
(oracle.half: the same operands rounded, FP64 elsewhere), element-wise maximum, with bars
from the worst measured He-init case with a margin (BF16 6.2e-2 -> 0.1, FP16 1.7e-2 ->
3e-2, both on single slots of the full 256-slot 14 x 624 batch); the FP64 bars of the
precision target (2e-2) are asserted on trained weights, where the fused products are well
conditioned, in test_gpu_trained_parity.py (measured there: BF16 1.1e-2, FP16 1.8e-3 against
FP64; BF16 4.5e-3, FP16 8.9e-4 against the emulation)."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, oracle_llr_at, torch
from workloads import WORKLOADS, replace

pytestmark = pytest.mark.gpu
TOL_16 = 2e-2
# Against the oracle's 16-bit emulation (oracle.half) the GPU differs only by FP32 rounding
# and the rare 16-bit rounding decision it flips.  Measured on plain networks: 1.7e-6 (BF16)
# and 1.9e-4 (FP16) max normwise; bar with a 5x margin.  On LayerNorm-fused networks at He
# init the amplification above applies to those flips: element-wise maximum bars per format.
EMU_MAX = 1e-3
EMU_MAX_LN = {"bf16": 0.1, "fp16": 3e-2}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def ln_fused(net):
    """A LayerNorm follows a Hadamard fusion (or normalises RB / MRB inputs)."""
    return bool(net.norm or net.residual) and net.n_branches >= 2


def check_16(L, L_ref, net, precision="fp16", L_emu=None):
    """Networks without a LayerNorm after a fusion: maximum error against FP64 within 2e-2.
    LayerNorm-fused networks: maximum error against the 16-bit emulation within the format's
    bar.  Hard decisions must agree on >= 99.9 % of the bits the bar cannot flip."""
    assert np.all(np.isfinite(L))
    if ln_fused(net):
        assert L_emu is not None
        ref, tol = L_emu, EMU_MAX_LN[precision]
    else:
        ref, tol = L_ref, TOL_16
    err = normwise(L, ref)
    assert err < tol, err
    sure = np.abs(ref) > tol * np.max(np.abs(ref))
    agree = np.mean((L > 0)[sure] == (ref > 0)[sure])
    assert agree >= 0.999, agree
    return err


def run_16(net, sim, B, precision, seed=1, wseed=2, perturb=0.02):
    """GPU LLRs, the FP64 oracle's, and (LayerNorm-fused networks) the 16-bit emulation's."""
    from oracle import half, net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(net, sim, seed, 0, B)
    params = onet.init_params(net, wseed)
    params = (params + perturb * np.random.default_rng(wseed).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, precision=precision, max_batch=B)
    rx.load_weights(params)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    rx.sync()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    p64 = params.astype(np.float64)
    L_ref = onet.forward(net, p64, X0)
    L_emu = half.forward_16(net, p64, X0, precision) if ln_fused(net) else None
    return llr.cpu().numpy(), L_ref, L_emu


PREC = ["bf16", "fp16"]


@pytest.mark.parametrize("precision", PREC)
def test_plain_smallest(precision):
    net = replace(WORKLOADS["plain_14x72_b16_fp32"].net, n_branches=3, width=32, depth=2, n_sc=17)
    L, L_ref, L_emu = run_16(net, WORKLOADS["plain_14x72_b16_fp32"].sim, 2, precision)
    check_16(L, L_ref, net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_plain_14x72_b16(precision):
    w = WORKLOADS["plain_14x72_b16_fp32"]
    L, L_ref, L_emu = run_16(w.net, w.sim, 16, precision)
    check_16(L, L_ref, w.net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
@pytest.mark.parametrize("F", [1, 129, 200])
def test_plain_ragged_grids(precision, F):
    """One RE per tile, a one-column last tile, and a partial last tile of 128."""
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_branches=3, width=32, depth=3, n_sc=F)
    L, L_ref, L_emu = run_16(net, w.sim, 2, precision)
    check_16(L, L_ref, net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_plain_two_branches_with_layernorm(precision):
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, norm=1, depth=3, n_sc=150)
    L, L_ref, L_emu = run_16(net, w.sim, 2, precision)
    check_16(L, L_ref, net, precision, L_emu)


EMU_CASES = [("plain_14x72_b16_fp32", dict(n_branches=3, width=32, depth=3, n_sc=40), 4),
             ("resid_14x624_b256_fp32", dict(n_sc=37, depth=2), 2),
             ("resid_14x3276_b1024_bf16", dict(n_sc=29, depth=2), 1)]


@pytest.mark.parametrize("precision", PREC)
@pytest.mark.parametrize("key,kw,B", EMU_CASES)
def test_matches_16bit_emulation(precision, key, kw, B):
    """Against the oracle's emulation of the 16-bit receiver (oracle.half: conv inputs and
    weights rounded to the 16-bit format, everything else exact) the GPU differs only by its
    FP32 arithmetic and the rare 16-bit rounding decision that flips.  That is much closer
    than to the FP64 network."""
    from oracle import half, net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS[key]
    net = replace(w.net, **kw)
    ref = oracle_inputs(net, w.sim, 1, 0, B)
    params = onet.init_params(net, 2)
    params = (params + 0.02 * np.random.default_rng(2).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, precision=precision, max_batch=B)
    rx.load_weights(params)
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    L_emu = half.forward_16(net, params.astype(np.float64), X0, precision)
    L_ref = onet.forward(net, params.astype(np.float64), X0)
    err, err_ref = normwise(L, L_emu), normwise(L, L_ref)
    print(f"{key} {precision}: vs emulation max {err:.2e}; vs FP64 {err_ref:.2e}")
    assert err < (EMU_MAX_LN[precision] if ln_fused(net) else EMU_MAX), err
    assert err < err_ref or err < 1e-4


@pytest.mark.parametrize("precision", PREC)
@pytest.mark.parametrize("n_sym,pilots,B", [(3, (1,), 1), (7, (1, 5), 23)])
def test_odd_tile_counts(precision, n_sym, pilots, B):
    """Odd numbers of 128-RE tiles (one per symbol of a slot here).  The conv kernels run in
    CTA pairs that share the weight loads, so a pair's second CTA then runs units past the
    last tile (zero operands, no stores): in the first round (3 tiles) or in the second
    persistent round (161 tiles on 152 SMs)."""
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_sym=n_sym, pilot_syms=pilots, n_sc=40, depth=3, n_branches=3, width=32)
    L, L_ref, L_emu = run_16(net, w.sim, B, precision)
    check_16(L, L_ref, net, precision, L_emu)


def test_residual_odd_tile_count():
    """The residual network's fixed-shape epilogues on 161 tiles (7 symbols x 23 slots, one
    tile each): the second CTA of the last active pair runs a unit past the last tile."""
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sym=7, pilot_syms=(1, 5), n_sc=37, depth=2)
    L, L_ref, L_emu = run_16(net, w.sim, 23, "bf16")
    check_16(L, L_ref, net, "bf16", L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_residual_64_ragged(precision):
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37)
    L, L_ref, L_emu = run_16(net, w.sim, 2, precision)
    check_16(L, L_ref, net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_residual_14x624_full_depth_he_init(precision):
    w = WORKLOADS["resid_14x624_b256_fp32"]
    L, L_ref, L_emu = run_16(w.net, w.sim, 1, precision, perturb=0.0)
    check_16(L, L_ref, w.net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_residual_96_four_antennas(precision):
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    net = replace(w.net, n_sc=29, depth=2)
    L, L_ref, L_emu = run_16(net, w.sim, 1, precision)
    check_16(L, L_ref, net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_resnet_112(precision):
    w = WORKLOADS["resnet_14x624_b256_fp32"]
    net = replace(w.net, n_sc=40, depth=3)
    L, L_ref, L_emu = run_16(net, w.sim, 1, precision)
    check_16(L, L_ref, net, precision, L_emu)


@pytest.mark.parametrize("precision", PREC)
def test_resid_14x3276_full_grid_sampled_res(precision):
    """Full 14 x 3276 grid, 8 blocks, 4 branches x 96: sampled subcarriers of sampled
    slots against the oracle evaluated on the exact receptive-field crop."""
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    B = 8
    ref = oracle_inputs(w.net, w.sim, 6, 500, B)
    params = onet.init_params(w.net, 4).astype(np.float32)
    rx = api.Receiver(w.net, precision=precision, max_batch=B)
    rx.load_weights(params)
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).cpu().numpy()
    rx.sync()
    p64 = params.astype(np.float64)
    got, emu = [], []
    for b, f in [(0, 0), (3, 1637), (7, 3275), (5, 128), (2, 127), (1, 2000), (4, 640), (6, 3)]:
        got.append(L[b, :, f, :])
        emu.append(oracle_llr_at(w.net, p64, ref["Y32"][b], ref["pilot_sym"], ref["pilot_mask"], f, fmt=precision))
    check_16(np.array(got), None, w.net, precision, np.array(emu))


def test_chunked_batch_matches_single_pass():
    """A handle whose activation buffers hold fewer slots than the batch streams it in
    chunks; every slot's result is bitwise the one a single-slot handle computes."""
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    B = 300
    s = api.sim_generate(w.net, w.sim, 2, 0, B)
    mask, _ = api.pilots(w.net)
    rx = api.Receiver(w.net, precision="bf16", max_batch=B)
    rx.init_he(3)
    full = rx.forward(s["Y"], mask)
    one = api.Receiver(w.net, precision="bf16", max_batch=1)
    one.load_weights(rx.save_weights())
    for b in (0, B // 2, B - 1):
        single = one.forward(s["Y"][b:b + 1].contiguous(), mask)
        assert torch.equal(single[0], full[b])
    rx.sync()


@pytest.mark.parametrize("precision", PREC)
def test_resid_14x624_full_batch_sampled_slots(precision):
    """The 14 x 624 residual workload at its full batch of 256 slots (the benchmark's launch
    configuration), sampled slots against the oracle."""
    from oracle import half, net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["resid_14x624_b256_fp32"]
    B = w.batch
    ref = oracle_inputs(w.net, w.sim, 4, 1000, B)
    params = onet.init_params(w.net, 9).astype(np.float32)
    rx = api.Receiver(w.net, precision=precision, max_batch=B)
    rx.load_weights(params)
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).cpu().numpy()
    rx.sync()
    for b in (0, 131, B - 1):
        Yd = ref["Y32"][b:b + 1, ..., 0].astype(np.float64) + 1j * ref["Y32"][b:b + 1, ..., 1]
        X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
        L_emu = half.forward_16(w.net, params.astype(np.float64), X0, precision)
        check_16(L[b:b + 1], None, w.net, precision, L_emu)


@pytest.mark.parametrize("key", ["conet_d14_14x624_bf16", "resnet_d24_14x624_bf16"])
def test_depth_comparison_networks(key):
    """The 4-branch x 64 CoNet and the 1-branch x 96 ResNet of the depth comparison."""
    w = WORKLOADS[key]
    net = replace(w.net, n_sc=29, depth=2)
    L, L_ref, L_emu = run_16(net, w.sim, 1, "bf16")
    check_16(L, L_ref, net, "bf16", L_emu)
