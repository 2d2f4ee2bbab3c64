"""GPU parity of the CoNet forward pass (input assembly -> all branches with Hadamard
fusion -> 1x1 head) against the FP64 oracle on oracle-simulated slots and oracle He
weights, through the C ABI.  FP32 LLRs must agree within 1e-4 normwise (the FP32
tolerance of the method's precision targets)."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, torch
from workloads import WORKLOADS, NetConfig, SimConfig, replace

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-4


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def run_pair(net, sim, B, seed=1, wseed=2, precision="fp32", slot0=0, perturb=0.0):
    from oracle import net as onet, pipeline
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(net, sim, seed, slot0, B)
    params = onet.init_params(net, wseed)
    if perturb:
        params = params + perturb * np.random.default_rng(wseed + 1).standard_normal(params.size)
    params32 = params.astype(np.float32)
    rx = api.Receiver(net, precision=precision, max_batch=B)
    rx.load_weights(params32)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]), dev(ref["noise_var"].astype(np.float32)))
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    L_ref = pipeline.receive(net, params32.astype(np.float64), Yd, ref["pilot_sym"], ref["pilot_mask"])
    return llr.cpu().numpy(), L_ref, rx


def check_fp32(L, L_ref):
    assert np.all(np.isfinite(L))
    err = normwise(L, L_ref)
    assert err < FP32_TOL, err
    amb = np.abs(L_ref) <= 1e-4 * np.max(np.abs(L_ref))
    assert np.all(((L > 0) == (L_ref > 0)) | amb)


def test_plain_14x72_b16():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    L, L_ref, _ = run_pair(w.net, w.sim, 16)
    check_fp32(L, L_ref)


@pytest.mark.parametrize("F", [1, 2, 3, 17, 129])
def test_plain_odd_grids(F):
    net = replace(WORKLOADS["plain_14x72_b16_fp32"].net, n_sc=F, width=16, n_branches=3, depth=3)
    L, L_ref, _ = run_pair(net, WORKLOADS["plain_14x72_b16_fp32"].sim, 3)
    check_fp32(L, L_ref)


def test_plain_with_layernorm_and_partial_fusion():
    net = replace(WORKLOADS["plain_14x72_b16_fp32"].net, norm=1, fuse_mask=0b1010, n_sc=40)
    L, L_ref, _ = run_pair(net, WORKLOADS["plain_14x72_b16_fp32"].sim, 2, perturb=0.05)
    check_fp32(L, L_ref)


def test_residual_64_ragged():
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37)
    L, L_ref, _ = run_pair(net, w.sim, 2, perturb=0.02)
    check_fp32(L, L_ref)


def test_resnet_112():
    w = WORKLOADS["resnet_14x624_b256_fp32"]
    net = replace(w.net, n_sc=20, depth=3)
    L, L_ref, _ = run_pair(net, w.sim, 1, perturb=0.02)
    check_fp32(L, L_ref)


@pytest.mark.parametrize("width,nb,kw", [(16, 3, dict()), (32, 2, dict()), (88, 2, dict()),
                                         (88, 1, dict(resnet_baseline=1))])
def test_residual_every_conv_width(width, nb, kw):
    """Residual LayerNorm networks at the other widths the FP32 conv is built for, so that
    every instantiation's LayerNorm rows and its stage between layers run: at 88 channels a
    CTA has 176 threads, five full warps and a half one (the width of the matched ResNet of
    the interference study)."""
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37, depth=2, width=width, n_branches=nb, **kw)
    L, L_ref, _ = run_pair(net, w.sim, 2, perturb=0.02)
    check_fp32(L, L_ref)


def test_repeated_and_smaller_batches_agree_bitwise():
    """Repeated calls agree bitwise, and a smaller batch afterwards gives the first slot's
    LLRs of the larger one bitwise: every RE's arithmetic is independent of the tiling and of
    the launch's other slots."""
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37, depth=2)
    ref = oracle_inputs(net, w.sim, 5, 0, 3)
    rx = api.Receiver(net, precision="fp32", max_batch=3)
    rx.load_weights(onet.init_params(net, 3).astype(np.float32))
    Y, M = dev(ref["Y32"]), dev(ref["pilot_mask"])
    L1 = rx.forward(Y, M).cpu().numpy()
    L2 = rx.forward(Y, M).cpu().numpy()
    np.testing.assert_array_equal(L1, L2)
    L3 = rx.forward(Y[:1].contiguous(), M).cpu().numpy()
    np.testing.assert_array_equal(L3, L1[:1])
    L4 = rx.forward(Y, M).cpu().numpy()
    np.testing.assert_array_equal(L4, L1)


def test_residual_96_four_antennas():
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    net = replace(w.net, n_sc=29, depth=2)
    L, L_ref, _ = run_pair(net, w.sim, 1, perturb=0.02)
    check_fp32(L, L_ref)


def test_resid_14x624_full_batch_sampled_slots():
    """The benchmarked launch (B = 256 slots of 14 x 624) against the oracle on sampled slots."""
    from oracle import net as onet, pipeline
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["resid_14x624_b256_fp32"]
    B = w.batch
    ref = oracle_inputs(w.net, w.sim, 4, 1000, B)
    params32 = onet.init_params(w.net, 9).astype(np.float32)
    rx = api.Receiver(w.net, precision="fp32", max_batch=B)
    rx.load_weights(params32)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]), dev(ref["noise_var"].astype(np.float32)))
    L = llr.cpu().numpy()
    assert np.all(np.isfinite(L))
    for b in (0, 131, B - 1):
        Yd = ref["Y32"][b:b + 1, ..., 0].astype(np.float64) + 1j * ref["Y32"][b:b + 1, ..., 1]
        L_ref = pipeline.receive(w.net, params32.astype(np.float64), Yd, ref["pilot_sym"], ref["pilot_mask"])
        check_fp32(L[b:b + 1], L_ref)


def test_forward_rejects_oversized_batch():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS["plain_14x72_b16_fp32"]
    rx = api.Receiver(w.net, max_batch=2)
    Y = torch.zeros((3, 1, 14, 72, 2), device="cuda")
    m = torch.zeros((14, 72), dtype=torch.uint8, device="cuda")
    with pytest.raises(ConetError) as e:
        rx.forward(Y, m)
    assert e.value.code == -2
    with pytest.raises(ConetError) as e:
        rx.load_weights(np.zeros(10, dtype=np.float32))
    assert e.value.code == -5
