"""Pins of the oracle's 16-bit emulation (oracle.half): the rounding against independent
implementations and hand-derived cases, and the forward's hook against the exact forward."""
import numpy as np
import pytest

from oracle import half, net as onet
from workloads import WORKLOADS, replace

torch = pytest.importorskip("torch")


def test_bf16_representable_values_are_fixed_points():
    m = np.arange(128)
    vals = np.concatenate([(1 + m / 128.0) * 2.0 ** e for e in range(-20, 21)])
    vals = np.concatenate([vals, -vals, [0.0]])
    assert np.array_equal(half.round16(vals, "bf16"), vals)


def test_bf16_ties_to_even_hand_cases():
    # spacing 2^-7 on [1, 2): 1 + 2^-8 lies halfway between 1 (even) and 1 + 2^-7 (odd)
    cases = {1 + 2.0 ** -8: 1.0,
             1 + 3 * 2.0 ** -8: 1 + 2.0 ** -6,              # between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
             1 + 2.0 ** -8 + 2.0 ** -20: 1 + 2.0 ** -7,     # just above the tie
             -(2 + 2.0 ** -7): -2.0,                         # spacing 2^-6 on [2, 4)
             3.0 * 2.0 ** -130: 3.0 * 2.0 ** -130}          # subnormal, exactly representable
    for x, want in cases.items():
        assert half.round16(x, "bf16") == want, x


def test_bf16_matches_torch_on_float32_inputs():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-30, 30, 200_000))).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(half.round16(x.astype(np.float64), "bf16"), want)


def test_fp16_matches_numpy_including_subnormals_and_overflow():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(200_000) * np.exp(rng.uniform(-20, 12, 200_000))
    x = np.concatenate([x, [65504.0, 65519.9, 65520.0, 7e4, -7e4, 2.0 ** -24, 3 * 2.0 ** -26]])
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(half.round16(x, "fp16"), want)


def test_rounding_error_bound():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(100_000) * np.exp(rng.uniform(-10, 10, 100_000))
    for fmt, bits in (("bf16", 8), ("fp16", 11)):
        y = x[np.abs(x) > 2.0 ** -14] if fmt == "fp16" else x
        y = y[np.abs(y) < 6e4]
        r = half.round16(y, fmt)
        spacing = np.ldexp(1.0, np.frexp(np.abs(y))[1] - 1 - (bits - 1))
        assert np.all(np.abs(r - y) <= 0.5 * spacing)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_hook_rounds_only_conv_operands(fmt):
    """With every weight and input already representable, the emulated forward is the exact
    forward; with arbitrary ones it stays within a few 16-bit roundings of it."""
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_sc=12, depth=3, width=8, n_sym=6, pilot_syms=(1, 4))
    rng = np.random.default_rng(3)
    flat = onet.init_params(net, 5)
    X0 = rng.standard_normal((2, net.n_sym, net.n_sc, 2 * net.n_rx + 3))
    exact = onet.forward(net, half.round16(flat, fmt), half.round16(X0, fmt))
    # rounded weights and input are fixed points, so only the rounding of inner activations differs
    L = half.forward_16(net, half.round16(flat, fmt), half.round16(X0, fmt), fmt)
    unit = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -11
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(L - exact)) <= 20 * unit * scale
    assert not np.array_equal(L, exact) or net.depth == 1   # inner activations were rounded
    L_all = half.forward_16(net, flat, X0, fmt)
    assert np.max(np.abs(L_all - onet.forward(net, flat, X0))) <= 40 * unit * np.max(np.abs(L_all))


def test_training_conv_reduces_to_the_exact_conv_pieces():
    """conv3x3_rounded (a 16-bit training step's conv) is assembled from the brute-force-pinned
    conv3x3: its output is conv3x3 of the rounded input and weight, its data gradient is
    conv3x3's data gradient at the rounded weight for the rounded upstream gradient, and its
    weight gradient is conv3x3's at the rounded input for the rounded upstream gradient."""
    from oracle import net as onet
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2, 4, 5, 3))
    W = rng.standard_normal((6, 3, 3, 3))
    bias = rng.standard_normal(6)
    G = rng.standard_normal((2, 4, 5, 6))
    q = half.Round16Train("bf16")
    tp = onet.Tape()
    x, w, b = tp.leaf(X), tp.leaf(W), tp.leaf(bias)
    y = onet.conv3x3_rounded(tp, x, w, b, q)
    dX, dW, db = tp.recs[y][1](G)
    ref = onet.Tape()
    xq, wq, bq = ref.leaf(half.round16(X)), ref.leaf(half.round16(W)), ref.leaf(bias)
    yq = onet.conv3x3(ref, xq, wq, bq)
    assert np.allclose(tp[y], ref[yq], rtol=1e-13, atol=1e-13)
    dX_ref, dW_ref, _ = ref.recs[yq][1](half.round16(G))
    assert np.allclose(dX, dX_ref, rtol=1e-13, atol=1e-13)
    assert np.allclose(dW, dW_ref, rtol=1e-13, atol=1e-13) and np.allclose(db, G.sum(axis=(0, 1, 2)))
    # the misreadings "weight gradient from the unrounded input or gradient" are distinguishable
    ref2 = onet.Tape()
    y2 = onet.conv3x3(ref2, ref2.leaf(X), ref2.leaf(W), ref2.leaf(bias))
    _, dW_wrong, _ = ref2.recs[y2][1](G)
    assert not np.allclose(dW, dW_wrong, rtol=1e-6)
    _, dW_wrong2, _ = ref.recs[yq][1](G)
    assert not np.allclose(dW, dW_wrong2, rtol=1e-6)


def test_training_gradient_with_identity_rounding_is_the_exact_gradient():
    """With roundings that change nothing, grad_16's hooks give the finite-difference-pinned
    exact gradient of oracle.net (all layers, fusion, LayerNorm, head)."""
    from oracle import net as onet
    from workloads import tiny_net
    for kw in (dict(), dict(norm=1), dict(residual=1, norm=1, n_branches=3)):
        cfg = tiny_net(**kw)
        rng = np.random.default_rng(5)
        flat = onet.init_params(cfg, 2) + 0.1 * rng.standard_normal(onet.param_count(cfg))
        X0 = rng.standard_normal((2, cfg.n_sym, cfg.n_sc, cfg.c_in))
        L, tape = onet.forward(cfg, flat, X0, keep_tape=True)
        dllr = rng.standard_normal(L.shape)
        g_ref, _ = onet.backward(cfg, tape, dllr)
        _, tape_i = onet.forward(cfg, flat, X0, keep_tape=True, quant=half.Round16Train(identity=True))
        g_id, _ = onet.backward(cfg, tape_i, dllr)
        assert np.allclose(g_id, g_ref, rtol=1e-12, atol=1e-14), kw
        g16 = half.grad_16(cfg, flat, X0, dllr)
        assert not np.allclose(g16, g_ref, rtol=1e-4)       # BF16 rounding does move it


class _Recorder:
    """Identity quantisation hooks that record what they are handed."""

    def __init__(self):
        self.acts, self.weights = [], []

    def act(self, x):
        self.acts.append(np.array(x, dtype=np.float64))
        return np.asarray(x, dtype=np.float64)

    def weight(self, w):
        self.weights.append(np.array(w, dtype=np.float64))
        return np.asarray(w, dtype=np.float64)


def _dw_brute(X, W):
    B, T, F, C = X.shape
    out = np.zeros_like(X)
    Xp = np.zeros((B, T + 2, F + 2, C))
    Xp[:, 1:-1, 1:-1] = X
    for kh in range(3):
        for kw in range(3):
            out += Xp[:, kh:kh + T, kw:kw + F] * W[:, kh, kw]
    return out


def test_depthwise_blocks_round_the_separable_operands():
    """Reading R8, pinned through recording hooks: the reduced-precision forward of a
    depthwise-separable network passes to the rounding hooks exactly the input layer's
    operands and, per block conv, the conv's input, the per-channel 3x3's output (which is the
    3x3 of the rounded input, by brute force) and the 1x1 weight, never the per-channel
    weights; with identity hooks it is the exact forward, and with 16-bit rounding it stays
    within a few roundings of it."""
    from workloads import tiny_net
    cfg = replace(tiny_net(residual=1, norm=1, depthwise=1, width=8), n_sc=10)
    rng = np.random.default_rng(7)
    flat = onet.init_params(cfg, 4) + 0.05 * rng.standard_normal(onet.param_count(cfg))
    X0 = rng.standard_normal((2, cfg.n_sym, cfg.n_sc, cfg.c_in))
    rec = _Recorder()
    L = onet.forward(cfg, flat, X0, quant=rec)
    assert np.array_equal(L, onet.forward(cfg, flat, X0))
    nb, C, D = cfg.n_branches, cfg.width, cfg.depth
    params, o = {}, 0
    for name, shape in onet.param_layout(cfg):
        n = int(np.prod(shape))
        params[name] = flat[o:o + n].reshape(shape)
        o += n
    assert [w.shape for w in rec.weights] == [(C, 3, 3, cfg.c_in)] * nb + [(C, C)] * (2 * D * nb)
    assert len(rec.acts) == nb + 2 * 2 * D * nb
    blocks = rec.acts[nb:]
    i = 0
    for k in range(D):
        for b in range(nb):
            for conv in ("c1", "c2"):
                x_in, dw_out = blocks[i], blocks[i + 1]
                assert np.allclose(dw_out, _dw_brute(x_in, params[f"b{b}.k{k}.{conv}.dw"]), rtol=0, atol=1e-12)
                i += 2
    for fmt, unit in (("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)):
        L16 = half.forward_16(cfg, flat, X0, fmt)
        assert not np.array_equal(L16, L)
        assert np.max(np.abs(L16 - L)) <= 200 * unit * np.max(np.abs(L))
