"""Pins of the oracle's CoNet network: brute-force 3x3 convolution on tiny tensors,
1x1 / identity special cases, LayerNorm moments, structural invariants of the
Hadamard fusion (support nets that output 1 leave the main net alone; support nets
commute), identity residual blocks, central finite differences of the whole
forward + BCE loss (rel. err <= 1e-6), and Adam's closed-form first step."""
import itertools

import numpy as np
import pytest

from oracle import net as onet
from workloads import tiny_net, replace


def brute_conv(x, w, b):
    B, T, F, Ci = x.shape
    Co = w.shape[0]
    out = np.zeros((B, T, F, Co))
    for bb, t, f, o in itertools.product(range(B), range(T), range(F), range(Co)):
        acc = b[o]
        for kh, kw, i in itertools.product(range(3), range(3), range(Ci)):
            tt, ff = t + kh - 1, f + kw - 1
            if 0 <= tt < T and 0 <= ff < F:
                acc += w[o, kh, kw, i] * x[bb, tt, ff, i]
        out[bb, t, f, o] = acc
    return out


def run_conv(x, w, b):
    tp = onet.Tape()
    return tp[onet.conv3x3(tp, tp.leaf(x), tp.leaf(w), tp.leaf(b))]


def test_conv3x3_matches_brute_force():
    g = np.random.default_rng(0)
    x = g.standard_normal((2, 4, 5, 3))
    w = g.standard_normal((2, 3, 3, 3))
    b = g.standard_normal(2)
    assert np.allclose(run_conv(x, w, b), brute_conv(x, w, b), atol=1e-12)


def test_conv3x3_special_cases():
    g = np.random.default_rng(1)
    x = g.standard_normal((1, 3, 4, 3))
    w = np.zeros((3, 3, 3, 3))
    M = g.standard_normal((3, 3))
    w[:, 1, 1, :] = M
    assert np.allclose(run_conv(x, w, np.zeros(3)), x @ M.T)          # centre tap only = 1x1
    wi = np.zeros((3, 3, 3, 3))
    wi[:, 1, 1, :] = np.eye(3)
    assert np.allclose(run_conv(x, wi, np.zeros(3)), x)
    ws = np.zeros((1, 3, 3, 1))
    ws[0, 0, 0, 0] = 1.0                                               # picks x[t-1, f-1]
    y = run_conv(x[..., :1], ws, np.zeros(1))
    assert np.allclose(y[0, 1:, 1:, 0], x[0, :-1, :-1, 0]) and np.all(y[0, 0, :, 0] == 0)


def test_layernorm_moments():
    g = np.random.default_rng(2)
    x = g.standard_normal((2, 3, 4, 16)) * 3 + 1
    tp = onet.Tape()
    y = tp[onet.layernorm(tp, tp.leaf(x), tp.leaf(np.ones(16)), tp.leaf(np.zeros(16)))]
    assert np.allclose(y.mean(-1), 0, atol=1e-12)
    assert np.allclose(y.var(-1), x.var(-1) / (x.var(-1) + onet.LN_EPS), atol=1e-12)


def _inputs(cfg, seed, B=2):
    g = np.random.default_rng(seed)
    X0 = g.standard_normal((B, cfg.n_sym, cfg.n_sc, cfg.c_in))
    mask = np.zeros((cfg.n_sym, cfg.n_sc), dtype=np.uint8)
    mask[list(cfg.pilot_syms), ::2] = 1
    bits = g.integers(0, 2, (B, cfg.n_sym, cfg.n_sc, cfg.qam_bits)).astype(np.uint8)
    bits[:, mask.astype(bool)] = 0
    return X0, bits, mask


def _set(cfg, flat, name, value):
    P = onet.unflatten(cfg, flat)
    P[name][...] = value


def test_support_branches_outputting_one_leave_the_main_net():
    cfg = tiny_net(n_branches=3, depth=3, width=4)
    single = replace(cfg, n_branches=1)
    flat = onet.init_params(cfg, 5)
    for b in (1, 2):
        for l in range(cfg.depth):
            key = "in" if l == 0 else f"l{l}"
            _set(cfg, flat, f"b{b}.{key}.w", 0.0)
            _set(cfg, flat, f"b{b}.{key}.b", 1.0)
    P = onet.unflatten(cfg, flat)
    flat1 = np.concatenate([P[n].ravel() for n, _ in onet.param_layout(single)])
    X0, _, _ = _inputs(cfg, 3)
    assert np.allclose(onet.forward(cfg, flat, X0), onet.forward(single, flat1, X0), atol=1e-12)


@pytest.mark.parametrize("residual", [0, 1])
def test_support_branches_commute(residual):
    cfg = tiny_net(n_branches=3, depth=2, width=4, residual=residual, norm=residual)
    flat = onet.init_params(cfg, 8)
    P = onet.unflatten(cfg, flat)
    swapped = flat.copy()
    Q = onet.unflatten(cfg, swapped)
    for n in P:
        if n.startswith("b1."):
            Q[n][...] = P["b2." + n[3:]]
            Q["b2." + n[3:]][...] = P[n]
    X0, _, _ = _inputs(cfg, 4)
    assert np.allclose(onet.forward(cfg, flat, X0), onet.forward(cfg, swapped, X0), atol=1e-12)
    # swapping main with a support branch changes the result (the main net is special)
    M = flat.copy()
    R = onet.unflatten(cfg, M)
    for n in P:
        if n.startswith("b1.") and ("b0." + n[3:]) in P:
            R[n][...] = P["b0." + n[3:]]
            R["b0." + n[3:]][...] = P[n]
    assert not np.allclose(onet.forward(cfg, flat, X0), onet.forward(cfg, M, X0))


def test_sum_fusion_with_silent_supports_leaves_the_main_net():
    """Sum interaction (fuse_op = 1): support branches whose activations are 0 (weights and
    biases 0, so ReLU gives 0) add nothing, and the CoNet is the main net alone."""
    cfg = tiny_net(n_branches=3, depth=3, width=4, fuse_op=1)
    single = replace(cfg, n_branches=1)
    flat = onet.init_params(cfg, 5)
    for b in (1, 2):
        for l in range(cfg.depth):
            key = "in" if l == 0 else f"l{l}"
            _set(cfg, flat, f"b{b}.{key}.w", 0.0)
            _set(cfg, flat, f"b{b}.{key}.b", 0.0)
    P = onet.unflatten(cfg, flat)
    flat1 = np.concatenate([P[n].ravel() for n, _ in onet.param_layout(single)])
    X0, _, _ = _inputs(cfg, 3)
    assert np.allclose(onet.forward(cfg, flat, X0), onet.forward(single, flat1, X0), atol=1e-12)


def test_sum_fusion_and_feedback_by_hand():
    """One fused input layer (depth 1 would fuse once and feed the head): with two branches
    and brute-force convs, x_main = a0 + a1 (sum interaction) or a0 * a1, and after a second
    layer Example II's support input is a1 + a0 (feedback) rather than a1."""
    for fuse_op in (0, 1):
        for feedback in (0, 1):
            cfg = tiny_net(n_branches=2, depth=2, width=3, fuse_op=fuse_op, feedback=feedback)
            flat = onet.init_params(cfg, 21) + 0.05
            P = onet.unflatten(cfg, flat)
            X0, _, _ = _inputs(cfg, 22)
            a = [np.maximum(brute_conv(X0, P[f"b{b}.in.w"], P[f"b{b}.in.b"]), 0) for b in range(2)]
            x0 = a[0] + a[1] if fuse_op else a[0] * a[1]
            x1 = a[1] + a[0] if feedback else a[1]
            c = [np.maximum(brute_conv(x0, P["b0.l1.w"], P["b0.l1.b"]), 0),
                 np.maximum(brute_conv(x1, P["b1.l1.w"], P["b1.l1.b"]), 0)]
            y0 = c[0] + c[1] if fuse_op else c[0] * c[1]
            want = y0 @ P["head.w"].T + P["head.b"]
            assert np.allclose(onet.forward(cfg, flat, X0), want, atol=1e-10), (fuse_op, feedback)


def test_identity_residual_blocks_reduce_to_fused_input_layer():
    cfg = tiny_net(n_branches=2, depth=2, width=4, residual=1, norm=1)
    flat = onet.init_params(cfg, 9)
    P = onet.unflatten(cfg, flat)
    g = np.random.default_rng(10)
    for n in P:
        if ".c2." in n:
            P[n][...] = 0.0
        if n.startswith("f") and n.endswith(".b"):
            P[n][...] = g.standard_normal(P[n].shape)
    X0, _, _ = _inputs(cfg, 11)

    def ln(v, gam, bet):
        mu = v.mean(-1, keepdims=True)
        return (v - mu) / np.sqrt(((v - mu) ** 2).mean(-1, keepdims=True) + 1e-5) * gam + bet

    a = [np.maximum(brute_conv(X0, P[f"b{b}.in.w"], P[f"b{b}.in.b"]), 0) for b in range(2)]
    x0 = ln(a[0] * a[1], P["f0.g"], P["f0.b"])
    for i in (1, 2):
        x0 = ln(x0 * a[1], P[f"f{i}.g"], P[f"f{i}.b"])
    want = x0 @ P["head.w"].T + P["head.b"]
    assert np.allclose(onet.forward(cfg, flat, X0), want, atol=1e-10)


FD_CASES = [
    dict(),
    dict(norm=1),
    dict(n_branches=3, depth=3),
    dict(residual=1, norm=1),
    dict(residual=1, norm=1, n_branches=3, depth=1),
    dict(n_branches=1, residual=1, norm=1, resnet_baseline=1, width=4),
    dict(fuse_mask=0b01),
    dict(fuse_op=1, norm=1, n_branches=3),
    dict(feedback=1, n_branches=3),
    dict(feedback=1, fuse_op=1, residual=1, norm=1),
    dict(depthwise=1, residual=1, norm=1, width=4),
    dict(support_inputs=1, n_branches=3),
    dict(support_inputs=1, residual=1, norm=1),
    dict(support_inputs=1, support_mask=0b10011, n_branches=3),
    dict(fuse_op=2, norm=1, n_branches=3),
    dict(fuse_op=2, fuse_mask=0b01),
    dict(fuse_op=2, feedback=1, norm=1),
]


@pytest.mark.parametrize("kw", FD_CASES)
def test_gradient_central_finite_differences(kw):
    cfg = tiny_net(**kw)
    flat = onet.init_params(cfg, 12)
    flat = flat + 0.1 * np.random.default_rng(13).standard_normal(flat.size)
    X0, bits, mask = _inputs(cfg, 14)
    loss, g, _ = onet.loss_and_grad(cfg, flat, X0, bits, mask)
    idx = np.random.default_rng(15).choice(flat.size, size=min(40, flat.size), replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(flat[i]))
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = onet.bce_loss(onet.forward(cfg, fp, X0), bits, mask)
        lm, _ = onet.bce_loss(onet.forward(cfg, fm, X0), bits, mask)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3) + 1e-9, (i, fd, g[i])


def test_bce_closed_forms():
    mask = np.zeros((1, 2), dtype=np.uint8)
    llr = np.zeros((1, 1, 2, 3))
    bits = np.zeros((1, 1, 2, 3), dtype=np.uint8)
    loss, d = onet.bce_loss(llr, bits, mask)
    assert np.isclose(loss, np.log(2.0)) and np.allclose(d, 0.5 / 6)
    llr = np.array([[[[40.0, -40.0]]]])
    loss, _ = onet.bce_loss(llr, np.array([[[[1, 0]]]], dtype=np.uint8), np.zeros((1, 1), np.uint8))
    assert loss < 1e-15


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w = np.ones(4)
    w1, m, v = onet.adam_step(w, g, np.zeros(4), np.zeros(4), 1, 1e-3)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_param_counts_of_named_networks():
    from workloads import WORKLOADS
    n2 = onet.param_count(WORKLOADS["resid_14x624_b256_fp32"].net)
    r2 = onet.param_count(WORKLOADS["resnet_14x624_b256_fp32"].net)
    assert abs(n2 - r2) / r2 < 0.02          # matched model size (Sec. III, last paragraph)
    assert onet.param_count(WORKLOADS["plain_14x72_b16_fp32"].net) == 2 * (9 * 5 * 32 + 32 + 3 * (9 * 32 * 32 + 32)) + 32 * 4 + 4


@pytest.mark.parametrize("name,kw", [("plain_14x72_b16_fp32", {}), ("resid_14x624_b256_fp32", dict(n_sc=60, depth=2))])
def test_cropped_receptive_field_is_exact(name, kw):
    """A depth-L stack of 3x3 convs (LayerNorm and fusion act per RE) sees L subcarriers on
    each side: the oracle on the crop f-L..f+L reproduces the full-grid LLR at f.  The GPU
    tests use this to check full-size grids RE by RE."""
    from gpu_util import oracle_inputs, oracle_llr_at
    from oracle import pipeline
    from workloads import WORKLOADS
    w = WORKLOADS[name]
    net = replace(w.net, **kw)
    ref = oracle_inputs(net, w.sim, 1, 0, 1)
    p = onet.init_params(net, 3)
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    full = pipeline.receive(net, p, Yd, ref["pilot_sym"], ref["pilot_mask"])
    for f in (0, 1, net.n_sc // 2, net.n_sc - 1):
        crop = oracle_llr_at(net, p, ref["Y32"][0], ref["pilot_sym"], ref["pilot_mask"], f)
        assert np.max(np.abs(crop - full[0, :, f, :])) < 1e-12


def test_depthwise_conv_matches_brute_force():
    g = np.random.default_rng(31)
    X = g.standard_normal((2, 4, 5, 3))
    W = g.standard_normal((3, 3, 3))
    tp = onet.Tape()
    y = tp[onet.dwconv3x3(tp, tp.leaf(X), tp.leaf(W))]
    want = np.zeros_like(X)
    for b, t, f, c in itertools.product(range(2), range(4), range(5), range(3)):
        for kh in range(3):
            for kw in range(3):
                tt, ff = t + kh - 1, f + kw - 1
                if 0 <= tt < 4 and 0 <= ff < 5:
                    want[b, t, f, c] += X[b, tt, ff, c] * W[c, kh, kw]
    assert np.allclose(y, want, atol=1e-12)
    # a depthwise conv equals the standard conv whose weight is diagonal in the channels
    Wfull = np.zeros((3, 3, 3, 3))
    for c in range(3):
        Wfull[c, :, :, c] = W[c]
    assert np.allclose(y, brute_conv(X, Wfull, np.zeros(3)), atol=1e-12)


def test_depthwise_block_is_the_separable_composition():
    """A depthwise residual network's block conv is the per-channel 3x3 then the 1x1 with
    bias: with the 1x1 weight the identity and zero bias, the block conv is the depthwise
    conv alone; the parameter count is 9 C + C^2 + C per block conv."""
    cfg = tiny_net(residual=1, norm=1, depthwise=1, width=4)
    std = replace(cfg, depthwise=0)
    C = cfg.width
    per_conv_dw, per_conv_std = 9 * C + C * C + C, 9 * C * C + C
    n_convs = 2 * cfg.depth * cfg.n_branches
    assert onet.param_count(std) - onet.param_count(cfg) == n_convs * (per_conv_std - per_conv_dw)
    names = [n for n, _ in onet.param_layout(cfg)]
    assert "b0.k0.c1.dw" in names and "b1.k1.c2.w" in names


def _support_in_w(cfg, flat, b):
    """View of branch b's input-layer weights [C, 3, 3, c_in] in a flat parameter vector."""
    o = 0
    for name, shape in onet.param_layout(cfg):
        n = int(np.prod(shape))
        if name == f"b{b}.in.w":
            return flat[o:o + n].reshape(shape)
        o += n
    raise KeyError(b)


@pytest.mark.parametrize("kw", [dict(n_branches=3), dict(residual=1, norm=1, n_branches=3), dict(n_rx=2)])
def test_selective_support_inputs_are_zeroed_signal_weights(kw):
    """Support nets fed only the pilot information (Sec. III): the network equals the
    full-input network whose support input layers have zero weights on the Re / Im Y
    channels of every antenna; the main net keeps them; and the received signal then
    reaches the LLRs only through the main net."""
    cfg = tiny_net(support_inputs=1, **kw)
    full = replace(cfg, support_inputs=0)
    flat = onet.init_params(cfg, 21) + 0.1 * np.random.default_rng(22).standard_normal(onet.param_count(cfg))
    X0, _, _ = _inputs(cfg, 23)
    zeroed = flat.copy()
    for b in range(1, cfg.n_branches):
        _support_in_w(cfg, zeroed, b)[..., :2 * cfg.n_rx] = 0.0
    np.testing.assert_array_equal(onet.forward(cfg, flat, X0), onet.forward(full, zeroed, X0))
    assert not np.array_equal(onet.forward(cfg, flat, X0), onet.forward(full, flat, X0))
    # the main net's signal weights matter: zeroing them too changes the output
    main0 = zeroed.copy()
    _support_in_w(cfg, main0, 0)[..., :2 * cfg.n_rx] = 0.0
    assert not np.allclose(onet.forward(full, main0, X0), onet.forward(full, zeroed, X0))


def test_selective_support_inputs_gradient_is_zero_on_withheld_channels():
    cfg = tiny_net(support_inputs=1, n_branches=3)
    flat = onet.init_params(cfg, 31) + 0.1 * np.random.default_rng(32).standard_normal(onet.param_count(cfg))
    X0, bits, mask = _inputs(cfg, 33)
    _, g, _ = onet.loss_and_grad(cfg, flat, X0, bits, mask)
    for b in range(cfg.n_branches):
        gw = _support_in_w(cfg, g, b)
        if b == 0:
            assert np.abs(gw[..., :2 * cfg.n_rx]).max() > 0
        else:
            assert np.all(gw[..., :2 * cfg.n_rx] == 0.0)
            assert np.abs(gw[..., 2 * cfg.n_rx:]).max() > 0


def test_concatenation_with_zero_support_weights_is_the_unfused_main():
    """Concatenation (fuse_op 2, reading R9) without LayerNorm: when the main's wide layers and
    the head give zero weight to the support channels (input channels C.. of the concatenated
    activation), the LLRs are those of the same network without fusion whose main weights are
    the first C input channels; the parameter count grows by the support channels' weights."""
    cfg = tiny_net(fuse_op=2, n_sc=7)
    plain = replace(cfg, fuse_mask=0)
    C, nb = cfg.width, cfg.n_branches
    rng = np.random.default_rng(21)
    flat = onet.init_params(cfg, 5) + 0.1 * rng.standard_normal(onet.param_count(cfg))
    P = onet.unflatten(cfg, flat)
    for l in range(1, cfg.depth):
        P[f"b0.l{l}.w"][..., C:] = 0.0
    P["head.w"][:, C:] = 0.0
    Q = {name: (P[name][..., :C] if name.startswith("b0.l") and name.endswith(".w") else
                P[name][:, :C] if name == "head.w" else P[name]) for name, _ in onet.param_layout(cfg)}
    flat_c = np.concatenate([P[name].ravel() for name, _ in onet.param_layout(cfg)])
    flat_p = np.concatenate([Q[name].ravel() for name, _ in onet.param_layout(plain)])
    X0, _, _ = _inputs(cfg, 3)
    assert np.allclose(onet.forward(cfg, flat_c, X0), onet.forward(plain, flat_p, X0), rtol=0, atol=1e-12)
    extra = (cfg.depth - 1) * C * 9 * (nb - 1) * C + cfg.qam_bits * (nb - 1) * C
    assert onet.param_count(cfg) - onet.param_count(plain) == extra
    with pytest.raises(ValueError):
        onet.forward(replace(cfg, residual=1, norm=1), onet.init_params(replace(cfg, residual=1, norm=1), 1), X0)


def test_support_mask_names_the_fed_channels():
    """support_mask: the default subset is the pilot information (channels 2 N .. 2 N + 2), so
    naming those bits gives the default network exactly; a mask keeping only channel j makes
    the support nets' input layers blind to every other channel (changing them changes
    nothing), while changing channel j does."""
    cfg = tiny_net(support_inputs=1, n_branches=3)
    flat = onet.init_params(cfg, 6)
    X0, _, _ = _inputs(cfg, 7)
    pil = 7 << (2 * cfg.n_rx)
    assert np.array_equal(onet.forward(cfg, flat, X0), onet.forward(replace(cfg, support_mask=pil), flat, X0))
    j = 1
    one = replace(cfg, support_mask=1 << j, fuse_mask=0b01)
    L = onet.forward(one, flat, X0)
    # only the support nets' view of the input matters through the fusion; perturb their
    # other channels' weights, then channel j's
    P = onet.unflatten(one, flat.copy())
    for b in (1, 2):
        P[f"b{b}.in.w"][..., [c for c in range(cfg.c_in) if c != j]] += 1.0
    flat2 = np.concatenate([P[n].ravel() for n, _ in onet.param_layout(one)])
    assert np.array_equal(onet.forward(one, flat2, X0), L)
    P[f"b1.in.w"][..., j] += 1.0
    flat3 = np.concatenate([P[n].ravel() for n, _ in onet.param_layout(one)])
    assert not np.allclose(onet.forward(one, flat3, X0), L)
