"""GPU parity of the other interaction operations of Sec. III (f2): the element-wise sum at
the fusion points (fuse_op = 1) and Example II's feedback (Fig. "conet2": every support net
continues with its own activation plus the main net's), on the FP32 fusion stage and the
tensor-core run-time epilogue, and their backward on FP32 plain networks, against the oracle (FP64, and its 16-bit / E4M3 emulations
for the reduced-precision paths).  Bars as in the product-fusion tests: FP32 1e-4 normwise
against FP64; 16-bit 1e-3 against the emulation on plain networks and the He-init
LayerNorm bars on residual ones; E4M3 1e-2 against its emulation on plain networks."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs
from workloads import WORKLOADS, replace

pytestmark = pytest.mark.gpu
VARIANTS = [dict(fuse_op=1), dict(feedback=1), dict(fuse_op=1, feedback=1)]
EMU_MAX_LN = {"bf16": 0.1, "fp16": 3e-2}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _run(net, sim, B, precision, wseed=2, perturb=0.02):
    from oracle import fp8, half, net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(net, sim, 1, 0, B)
    params = onet.init_params(net, wseed)
    params = (params + perturb * np.random.default_rng(wseed).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, precision=precision, max_batch=B)
    rx.load_weights(params)
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).cpu().numpy()
    rx.sync()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    p64 = params.astype(np.float64)
    if precision == "fp32":
        R = onet.forward(net, p64, X0)
    elif precision == "fp8":
        R = fp8.forward_fp8(net, p64, X0)
    else:
        R = half.forward_16(net, p64, X0, precision)
    return L, R


@pytest.mark.parametrize("kw", VARIANTS)
@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16", "fp8"])
def test_plain_network(kw, precision):
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_branches=3, depth=3, n_sc=40, **kw)
    L, R = _run(net, w.sim, 2, precision)
    err = normwise(L, R)
    print(f"plain {kw} {precision}: {err:.2e}")
    assert np.all(np.isfinite(L)) and err < {"fp32": 1e-4, "bf16": 1e-3, "fp16": 1e-3, "fp8": 1e-2}[precision], err


@pytest.mark.parametrize("kw", VARIANTS)
@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_residual_network(kw, precision):
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=37, depth=2, **kw)
    L, R = _run(net, w.sim, 2, precision)
    err = normwise(L, R)
    print(f"residual {kw} {precision}: {err:.2e}")
    assert np.all(np.isfinite(L)) and err < {"fp32": 1e-4, **EMU_MAX_LN}[precision], err


def test_unsupported_combinations_are_refused():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS["resid_14x3276_b1024_bf16"]
    with pytest.raises(ConetError) as e:                  # branch-group network on the tensor cores
        api.Receiver(replace(w.net, n_sc=29, feedback=1), "bf16", max_batch=1)
    assert e.value.code == -8
    with pytest.raises(ConetError) as e:                  # training with feedback: FP32 only
        api.Receiver(replace(WORKLOADS["plain_14x72_b16_fp32"].net, feedback=1), "bf16", max_batch=1, train=True)
    assert e.value.code == -8
    with pytest.raises(ConetError) as e:                  # feedback adds in place: no per-block recompute
        api.Receiver(replace(WORKLOADS["resid_14x624_b256_fp32"].net, n_sc=37, feedback=1), "fp32", max_batch=1,
                     train=True, recompute=True)
    assert e.value.code == -8


@pytest.mark.parametrize("kw", VARIANTS + [dict(fuse_op=1, norm=1), dict(feedback=1, norm=1, fuse_mask=0b0101),
                                dict(fuse_op=1, residual=1, norm=1), dict(feedback=1, residual=1, norm=1),
                                dict(fuse_op=1, feedback=1, residual=1, norm=1, fuse_mask=0b101),
                                dict(fuse_op=2), dict(fuse_op=2, norm=1), dict(fuse_op=2, feedback=1, norm=1, fuse_mask=0b101)])
def test_training_gradients_fp32(kw):
    """Backward of the sum interaction and of Example II's feedback (FP32 plain and residual
    networks) and of the concatenation (plain networks: the fusion backward splits the
    gradient of the wide activation back to the branches, the main's wide conv has its own
    weight and data gradients): the GPU gradient against the FP64 oracle's, per parameter
    tensor, within the product-fusion bar (2e-4 normwise)."""
    from oracle import net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    from workloads import random_grid
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=24, n_branches=3, depth=3, width=16, **kw)
    B = 3
    ref = oracle_inputs(net, w.sim, 3, 0, B)
    params = onet.init_params(net, 4)
    params = (params + 0.05 * np.random.default_rng(4).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, precision="fp32", max_batch=B, train=True)
    rx.load_weights(params)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    dllr = random_grid(13, llr.shape, scale=1e-3)
    rx.backward(dev(dllr))
    g = rx.grads_device().cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    L_ref, tape = onet.forward(net, params.astype(np.float64), X0, keep_tape=True)
    g_ref, _ = onet.backward(net, tape, dllr.astype(np.float64))
    assert normwise(llr.cpu().numpy(), L_ref) < 1e-4
    o, worst = 0, (0.0, None)
    for name, shape in onet.param_layout(net):
        n = int(np.prod(shape))
        e = normwise(g[o:o + n], g_ref[o:o + n])
        worst = max(worst, (e, name))
        o += n
    print(f"training {kw}: worst gradient tensor {worst}")
    assert worst[0] < 2e-4, worst


@pytest.mark.parametrize("key,kw", [("resid_14x624_b256_fp32", dict(n_sc=37, depth=2)),
                                    ("resid_14x624_b256_fp32", dict(n_sc=130, depth=1, n_branches=2, width=32)),
                                    ("resnet_14x624_b256_fp32", dict(n_sc=21, depth=2))])
def test_depthwise_separable_blocks_fp32(key, kw):
    """Depthwise-separable RB / MRB convs (f3: per-channel 3x3, then 1x1 with bias) on the FP32
    path (depthwise kernel + the implicit-GEMM kernel with only the centre tap), against the
    FP64 oracle at 1e-4 normwise; also with the sum interaction and Example II feedback."""
    w = WORKLOADS[key]
    for extra in (dict(), dict(fuse_op=1, feedback=1)):
        if extra and w.net.resnet_baseline:
            continue
        net = replace(w.net, depthwise=1, **kw, **extra)
        L, R = _run(net, w.sim, 2, "fp32")
        err = normwise(L, R)
        print(f"depthwise {key} {kw} {extra}: {err:.2e}")
        assert np.all(np.isfinite(L)) and err < 1e-4, err


@pytest.mark.parametrize("key,kw", [("resid_14x624_b256_fp32", dict(n_sc=37, depth=2)),
                                    ("resid_14x624_b256_fp32", dict(n_sc=130, depth=1, n_branches=2, width=32)),
                                    ("resid_14x3276_b1024_bf16", dict(n_sc=29, depth=2))])
@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_depthwise_separable_blocks_16bit(key, kw, precision):
    """Depthwise-separable blocks on the 16-bit tensor-core path (f3, reading R8): the
    per-channel 3x3 on 16-bit activations (FP32 weights and accumulation, output rounded to
    the format), then the 1x1 as a one-tap tcgen05 conv with the body convs' fused epilogues,
    against the oracle's emulation at the He-init LayerNorm bars; also with the sum
    interaction and Example II feedback where the network runs as one branch group."""
    w = WORKLOADS[key]
    extras = [dict()] if w.net.n_branches * w.net.width > 256 else [dict(), dict(fuse_op=1, feedback=1)]
    for extra in extras:
        net = replace(w.net, depthwise=1, **kw, **extra)
        L, R = _run(net, w.sim, 2, precision)
        err = normwise(L, R)
        print(f"depthwise {key} {kw} {extra} {precision}: {err:.2e}")
        assert np.all(np.isfinite(L)) and err < EMU_MAX_LN[precision], err


@pytest.mark.parametrize("kw", [dict(fuse_op=2), dict(fuse_op=2, norm=1), dict(fuse_op=2, norm=1, fuse_mask=0b0101),
                                dict(fuse_op=2, feedback=1, norm=1), dict(fuse_op=2, n_branches=3, width=16, norm=1)])
def test_concatenation_fp32(kw):
    """The concatenation interaction (reading R9) on the FP32 path: the stage writes the
    branches' activations side by side (normalised over all of them), the main's next conv
    reads n_branches x width channels in a launch of its own, and the head the same width
    after the last layer; against the FP64 oracle at the FP32 bar (1e-4 normwise)."""
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_sc=40, **kw)
    L, R = _run(net, w.sim, 2, "fp32")
    err = normwise(L, R)
    print(f"concatenation {kw}: {err:.2e}")
    assert np.all(np.isfinite(L)) and err < 1e-4, err


def test_concatenation_refused_outside_fp32():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    net = replace(WORKLOADS["plain_14x72_b16_fp32"].net, fuse_op=2, n_sc=40)
    for prec, train in (("bf16", False), ("fp8", False), ("bf16", True)):
        with pytest.raises(ConetError) as e:
            api.Receiver(net, prec, max_batch=1, train=train)
        assert e.value.code == -8


@pytest.mark.parametrize("kw,recompute", [(dict(), False), (dict(n_branches=2, width=32), True),
                                          (dict(n_branches=1, width=16, resnet_baseline=1), False)])
def test_depthwise_training_gradients_fp32(kw, recompute):
    """Backward of depthwise-separable blocks on the FP32 path (the 1x1's weight gradient, its
    data gradient as a one-tap conv, the per-channel 3x3's weight gradient and its data
    gradient as the rotated 3x3), against the FP64 oracle's gradient per parameter tensor
    at the 2e-4 normwise bar of the other FP32 gradients; also with per-block recompute and
    on the single-branch ResNet; one Adam step then moves the per-channel weights."""
    from oracle import net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    from workloads import random_grid
    w = WORKLOADS["resid_14x624_b256_fp32"]
    net = replace(w.net, n_sc=21, depth=2, depthwise=1, **kw)
    B = 2
    ref = oracle_inputs(net, w.sim, 3, 0, B)
    params = onet.init_params(net, 4)
    params = (params + 0.05 * np.random.default_rng(4).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, precision="fp32", max_batch=B, train=True, recompute=recompute)
    rx.load_weights(params)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    dllr = random_grid(13, llr.shape, scale=1e-3)
    rx.backward(dev(dllr))
    g = rx.grads_device().cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    L_ref, tape = onet.forward(net, params.astype(np.float64), X0, keep_tape=True)
    g_ref, _ = onet.backward(net, tape, dllr.astype(np.float64))
    assert normwise(llr.cpu().numpy(), L_ref) < 1e-4
    o, worst = 0, (0.0, None)
    for name, shape in onet.param_layout(net):
        n = int(np.prod(shape))
        e = normwise(g[o:o + n], g_ref[o:o + n])
        worst = max(worst, (e, name))
        o += n
    print(f"depthwise training {kw} recompute={recompute}: worst gradient tensor {worst}")
    assert worst[0] < 2e-4, worst
    rx.adam_step(1e-2, 1)
    p1 = rx.save_weights()
    o = 0
    for name, shape in onet.param_layout(net):
        n = int(np.prod(shape))
        if name.endswith(".dw"):
            assert not np.array_equal(p1[o:o + n], params[o:o + n]), name
        o += n


def test_depthwise_refused_outside_its_paths():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    net = replace(WORKLOADS["resid_14x624_b256_fp32"].net, depthwise=1, n_sc=37, depth=1)
    for prec, train in (("fp8", False), ("tf32x3", False), ("bf16", True)):
        with pytest.raises(ConetError) as e:
            api.Receiver(net, prec, max_batch=1, train=train)
        assert e.value.code == -8
