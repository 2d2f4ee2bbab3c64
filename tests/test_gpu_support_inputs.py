"""GPU parity of selective inputs to the support nets (Sec. III, support_inputs = 1: the
support nets are fed only the pilot information, not the received signal) on every path
that reads the conv weights: the FP32 path, the tensor-core layer path (16-bit and E4M3),
the whole-network kernel of the small plain networks, and the FP32 / BF16 backward.

Bars are the ones of the full-input tests: FP32 1e-4 normwise against the FP64 oracle;
16-bit 1e-3 against the oracle's emulation on plain networks and the He-init LayerNorm bars
on residual ones; E4M3 1e-2 against its emulation.  Beside parity: the network equals, on
the same kernels and bitwise, the full-input network whose support input layers have zero
weights on the signal channels, and the withheld weights' gradients are exactly zero, so an
Adam step leaves them where they were."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs
from workloads import WORKLOADS, random_grid, replace

pytestmark = pytest.mark.gpu
EMU_MAX_LN = {"bf16": 0.1, "fp16": 3e-2}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _params(net, wseed=2, perturb=0.02):
    from oracle import net as onet
    p = onet.init_params(net, wseed)
    return (p + perturb * np.random.default_rng(wseed).standard_normal(p.size)).astype(np.float32)


def _in_w(net, flat, b):
    from oracle import net as onet
    o = 0
    for name, shape in onet.param_layout(net):
        n = int(np.prod(shape))
        if name == f"b{b}.in.w":
            return flat[o:o + n].reshape(shape)
        o += n
    raise KeyError(b)


def _forward(net, sim, B, precision, params):
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(net, sim, 1, 0, B)
    rx = api.Receiver(net, precision=precision, max_batch=B)
    rx.load_weights(params)
    Y, M = dev(ref["Y32"]), dev(ref["pilot_mask"])
    L = rx.forward(Y, M).cpu().numpy()
    if precision == "fp8":           # past the calibrating pass (the whole-network kernel, where it applies)
        L = rx.forward(Y, M).cpu().numpy()
    rx.sync()
    return L, ref


def _reference(net, ref, params, precision):
    from oracle import fp8, half, net as onet, rx as orx
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    p64 = params.astype(np.float64)
    if precision == "fp32":
        return onet.forward(net, p64, X0)
    if precision == "fp8":
        return fp8.forward_fp8(net, p64, X0)
    return half.forward_16(net, p64, X0, precision)


PLAIN = [("plain_14x72_b16_fp32", dict(), 16), ("plain_14x72_b16_fp32", dict(n_branches=3, depth=3, n_sc=40), 2)]


@pytest.mark.parametrize("key,kw,B", PLAIN)
@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16", "fp8"])
def test_plain_network(key, kw, B, precision):
    w = WORKLOADS[key]
    net = replace(w.net, support_inputs=1, **kw)
    params = _params(net)
    L, ref = _forward(net, w.sim, B, precision, params)
    R = _reference(net, ref, params, precision)
    err = normwise(L, R)
    print(f"support inputs, plain {kw} B={B} {precision}: {err:.2e}")
    assert np.all(np.isfinite(L)) and err < {"fp32": 1e-4, "bf16": 1e-3, "fp16": 1e-3, "fp8": 1e-2}[precision], err
    # bitwise the full-input network with the support nets' signal weights zero
    full = replace(net, support_inputs=0)
    zeroed = params.copy()
    for b in range(1, net.n_branches):
        _in_w(net, zeroed, b)[..., :2 * net.n_rx] = 0.0
    L0, _ = _forward(full, w.sim, B, precision, zeroed)
    np.testing.assert_array_equal(L, L0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_support_mask_subset(precision):
    """support_mask names another subset of the inputs for the support nets (here Re Y, Im Y
    and the Im part of the LS estimate): parity with the oracle, and bitwise the full-input
    network whose support input layers have zero weights on the other channels."""
    w = WORKLOADS["plain_14x72_b16_fp32"]
    keep = 0b10011
    net = replace(w.net, n_branches=3, depth=3, n_sc=40, support_inputs=1, support_mask=keep)
    params = _params(net)
    L, ref = _forward(net, w.sim, 2, precision, params)
    err = normwise(L, _reference(net, ref, params, precision))
    print(f"support mask {keep:#b} {precision}: {err:.2e}")
    assert np.all(np.isfinite(L)) and err < {"fp32": 1e-4, "bf16": 1e-3}[precision], err
    full = replace(net, support_inputs=0, support_mask=0)
    zeroed = params.copy()
    for b in range(1, net.n_branches):
        wb = _in_w(net, zeroed, b)
        for j in range(net.c_in):
            if not (keep >> j) & 1:
                wb[..., j] = 0.0
    L0, _ = _forward(full, w.sim, 2, precision, zeroed)
    np.testing.assert_array_equal(L, L0)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_residual_network(precision):
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37, depth=2, support_inputs=1)
    params = _params(net)
    L, ref = _forward(net, w.sim, 2, precision, params)
    err = normwise(L, _reference(net, ref, params, precision))
    print(f"support inputs, residual {precision}: {err:.2e}")
    assert np.all(np.isfinite(L)) and err < {"fp32": 1e-4, **EMU_MAX_LN}[precision], err


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_gradients_and_adam_keep_the_withheld_weights(precision):
    from oracle import net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=24, n_branches=3, depth=3, width=16, support_inputs=1)
    B = 3
    ref = oracle_inputs(net, w.sim, 3, 0, B)
    params = _params(net, 4, 0.05)
    rx = api.Receiver(net, precision=precision, max_batch=B, train=True)
    rx.load_weights(params)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    dllr = random_grid(13, llr.shape, scale=1e-3)
    rx.backward(dev(dllr))
    g = rx.grads_device().cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    _, tape = onet.forward(net, params.astype(np.float64), X0, keep_tape=True)
    g_ref, _ = onet.backward(net, tape, dllr.astype(np.float64))
    for b in range(1, net.n_branches):
        assert np.all(_in_w(net, g, b)[..., :2 * net.n_rx] == 0.0)
    if precision == "fp32":
        o = 0
        for name, shape in onet.param_layout(net):
            n = int(np.prod(shape))
            assert normwise(g[o:o + n], g_ref[o:o + n]) < 2e-4, name
            o += n
    rx.adam_step(1e-2, 1)
    p1 = rx.save_weights()
    for b in range(1, net.n_branches):
        np.testing.assert_array_equal(_in_w(net, p1, b)[..., :2 * net.n_rx], _in_w(net, params, b)[..., :2 * net.n_rx])
    assert not np.array_equal(_in_w(net, p1, 1)[..., 2 * net.n_rx:], _in_w(net, params, 1)[..., 2 * net.n_rx:])
