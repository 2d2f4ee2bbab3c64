"""Pins of the oracle's E4M3 emulation (oracle/fp8.py) against the format definition,
an independent library conversion, exactly representable networks and the rounding
error bound."""
import numpy as np
import pytest

from oracle import fp8, net as onet
from workloads import WORKLOADS, replace, tiny_net

torch = pytest.importorskip("torch")


def test_value_set_from_bit_patterns():
    v = fp8.e4m3_values()
    assert v.size == 127                       # 0, 7 subnormals, 15 x 8 normals minus NaN
    assert v[0] == 0 and v[1] == 2.0 ** -9 and v[-1] == 448.0
    assert 2.0 ** -6 in v and 1.125 in v and 1.0 + 2 ** -4 not in v
    # every representable value is a fixed point, the midpoints round to the even neighbour
    assert np.array_equal(fp8.e4m3_round(v), v)
    assert np.array_equal(fp8.e4m3_round(-v), -v)


def test_ties_to_even_and_saturation():
    assert fp8.e4m3_round(1.0625) == 1.0       # halfway 1 .. 1.125 -> even mantissa 000
    assert fp8.e4m3_round(1.1875) == 1.25      # halfway 1.125 .. 1.25 -> mantissa 010
    assert fp8.e4m3_round(2.0 ** -10) == 0.0   # half the smallest subnormal -> 0 (even)
    assert fp8.e4m3_round(3 * 2.0 ** -10) == 2.0 ** -8
    assert fp8.e4m3_round(460.0) == 448.0 and fp8.e4m3_round(1e6) == 448.0
    assert fp8.e4m3_round(-1e6) == -448.0


def test_matches_torch_float8_e4m3fn():
    """torch's float8_e4m3fn cast rounds to nearest even; inside the finite range it must
    agree exactly."""
    g = np.random.default_rng(0)
    x = np.concatenate([g.standard_normal(20000) * 10.0 ** g.uniform(-4, 2.6, 20000),
                        fp8.e4m3_values()[1:] * (1 + 2.0 ** -5), fp8.e4m3_values()[1:] * (1 - 2.0 ** -5)])
    x = x[np.abs(x) <= 448.0].astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(fp8.e4m3_round(x), ref)


def test_pow2_scale():
    for t in [1e-7, 0.3, 1.0, 223.9, 224.0, 224.1, 447.0, 448.0, 448.5, 896.0, 897.0, 3.3e4]:
        s = fp8.pow2_scale(t)
        assert np.log2(s) == np.round(np.log2(s))
        assert t / s <= 448.0 and t / s > 224.0
    assert fp8.pow2_scale(0.0) == 1.0


def test_weight_rows_scaled_separately():
    """A row 2^-20 smaller than another keeps its own relative precision."""
    g = np.random.default_rng(1)
    w = g.standard_normal((4, 3, 3, 5))
    w[1] *= 2.0 ** -20
    q = fp8.quantize_weight(w)
    rel = np.abs(q - w) / np.abs(w)
    assert np.max(rel[np.abs(w) > 2.0 ** -6 * np.max(np.abs(w), axis=(1, 2, 3), keepdims=True)]) <= 2.0 ** -4


def _representable_net(residual):
    """A network whose conv inputs and weights are exactly representable in E4M3 after
    pow2 scaling: single centre taps copying one channel, biases 0."""
    net = tiny_net(residual=residual)
    p = onet.init_params(net, 0)
    P = onet.unflatten(net, p)
    for name, arr in P.items():
        if name.endswith(".w") and arr.ndim == 4:
            arr[...] = 0.0
            for co in range(arr.shape[0]):
                arr[co, 1, 1, co % arr.shape[3]] = 2.0 ** (co % 3 - 1)
        elif name.endswith(".b") and not name.startswith("head") and ".ln" not in name and not name.startswith("f"):
            arr[...] = 0.0
    return net, np.concatenate([P[n].ravel() for n, _ in onet.param_layout(net)])


def test_representable_network_is_unchanged():
    net, p = _representable_net(0)
    g = np.random.default_rng(2)
    X0 = g.integers(-3, 4, size=(2, net.n_sym, net.n_sc, net.c_in)).astype(np.float64)
    assert np.array_equal(fp8.forward_fp8(net, p, X0), onet.forward(net, p, X0))


def _conv(x, w):
    tp = onet.Tape()
    y = onet.conv3x3(tp, tp.leaf(x), tp.leaf(w), tp.leaf(np.zeros(w.shape[0])))
    return tp[y]


def test_single_conv_error_bound():
    """One conv with E4M3 input and weights: |y_q - y| <= sum |w||x| ((1 + u)^2 - 1)
    + subnormal terms, u = 2^-4 (half the spacing of a 3-bit mantissa)."""
    net = tiny_net()
    g = np.random.default_rng(3)
    p = onet.init_params(net, 4)
    X0 = g.standard_normal((2, net.n_sym, net.n_sc, net.c_in))
    w = onet.unflatten(net, p)["b0.in.w"]
    q = fp8.E4M3Quant(margin=1.0)
    err = np.abs(_conv(q.act(X0), q.weight(w)) - _conv(X0, w))
    u = 2.0 ** -4
    sx = fp8.pow2_scale(np.max(np.abs(X0)))
    sw = max(fp8.pow2_scale(np.max(np.abs(w[co]))) for co in range(w.shape[0]))
    tail = 9 * net.c_in * 2.0 ** -10 * (sx * np.max(np.abs(w)) + np.max(np.abs(X0)) * sw) * (1 + u)
    bound = _conv(np.abs(X0), np.abs(w)) * ((1 + u) ** 2 - 1) + tail
    assert np.all(err <= bound + 1e-12)
    assert np.max(err) > 0                     # quantisation did happen
    # a dropped quantisation step would make the emulated conv exact
    assert np.mean(err) > 1e-4 * np.mean(np.abs(_conv(X0, w)))


def test_recorded_scales_replay_and_count():
    """Calibration records one scale per conv input, in forward order; replaying them on the
    same batch reproduces the calibrated forward exactly; the input layer's scale from a
    subset of the slots is at most the whole batch's (its amax is over fewer values)."""
    from workloads import replace
    net = replace(tiny_net(residual=1), depth=2)
    p = onet.init_params(net, 3)
    g = np.random.default_rng(4)
    X0 = g.standard_normal((3, net.n_sym, net.n_sc, net.c_in))
    scales = fp8.calibrate_fp8(net, p, X0)
    n_convs = net.n_branches * (1 + 2 * net.depth)
    assert len(scales) == n_convs
    assert np.array_equal(fp8.forward_fp8(net, p, X0, scales=scales), fp8.forward_fp8(net, p, X0))
    own = fp8.calibrate_fp8(net, p, X0[:1])
    assert len(own) == n_convs
    assert all(own[b] <= scales[b] for b in range(net.n_branches))
