"""GPU parity of the backward pass, Adam and the training step against the FP64 oracle
(through the C ABI).  The upstream LLR gradient is a seeded random tensor fed to both
sides.  Gradients agree per parameter tensor within 2e-4 normwise: FP32 accumulation
over B*T*F*9 products per weight with partial sums per split keeps the relative error
near 1e-6 * sqrt(terms), two decades below the bar."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, torch
from workloads import WORKLOADS, random_grid, replace

pytestmark = pytest.mark.gpu
GRAD_TOL = 2e-4


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def grad_pair(net, sim, B, seed=3, wseed=4, perturb=0.05, precision="fp32"):
    from oracle import net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    ref = oracle_inputs(net, sim, seed, 0, B)
    params = onet.init_params(net, wseed)
    params = (params + perturb * np.random.default_rng(wseed).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, precision=precision, max_batch=B, train=True)
    rx.load_weights(params)
    llr = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    dllr = random_grid(seed + 10, llr.shape, scale=1e-3)
    rx.backward(dev(dllr))
    g = rx.grads_device().cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    L_ref, tape = onet.forward(net, params.astype(np.float64), X0, keep_tape=True)
    g_ref, _ = onet.backward(net, tape, dllr.astype(np.float64))
    return llr.cpu().numpy(), L_ref, g, g_ref


def check_grads(net, g, g_ref, tol=GRAD_TOL):
    from oracle import net as onet
    o = 0
    worst = (0.0, None)
    for name, shape in onet.param_layout(net):
        n = int(np.prod(shape))
        e = normwise(g[o:o + n], g_ref[o:o + n])
        if e > worst[0]:
            worst = (e, name)
        o += n
    assert worst[0] < tol, worst
    return worst


@pytest.mark.parametrize("kw", [dict(), dict(norm=1, fuse_mask=0b1011), dict(n_branches=3, depth=3, width=16)])
def test_plain_gradients(kw):
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=24, **kw)
    L, L_ref, g, g_ref = grad_pair(net, w.sim, 3)
    assert normwise(L, L_ref) < 1e-4
    check_grads(net, g, g_ref)


def test_plain_gradients_full_grid():
    w = WORKLOADS["train_14x72_b128_bf16"]
    L, L_ref, g, g_ref = grad_pair(w.net, w.sim, 8)
    check_grads(w.net, g, g_ref)


@pytest.mark.parametrize("n_sc,B", [(24, 3), (72, 8)])
def test_bf16_training_gradients(n_sc, B):
    """A BF16 training handle: every conv's math on the tensor cores with BF16 operands and
    FP32 accumulation -- the forward convs, the body convs' data gradients (BF16 copies of the
    incoming gradient and of the rotated weights) and the weight gradients (BF16 copies of
    the incoming gradient and of the conv's input, split over REs, reduced in a fixed order)
    -- and everything else in FP32.  The oracle's 16-bit training emulation
    (oracle.half.grad_16) rounds exactly those operands and computes the rest in FP64, so the
    GPU gradient differs from it only by FP32 rounding: accumulation error of order 1e-6,
    plus the rare BF16 rounding decision that an FP32-vs-FP64 difference flips (about 3e-5 of
    the rounded values, each by one BF16 step of 2^-8, diluted over the 9 C terms of every
    downstream sum to ~2e-4 of a tensor's largest entry).  Bar: 2e-3 normwise per parameter
    tensor."""
    from oracle import half, net as onet, rx as orx
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=n_sc)
    L, L_ref, g, g_ref = grad_pair(net, w.sim, B, precision="bf16")
    ref = oracle_inputs(net, w.sim, 3, 0, B)
    params = onet.init_params(net, 4)
    params = (params + 0.05 * np.random.default_rng(4).standard_normal(params.size)).astype(np.float32)
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    assert normwise(L, half.forward_16(net, params.astype(np.float64), X0)) < 1e-3
    dllr = random_grid(3 + 10, L.shape, scale=1e-3)
    g16 = half.grad_16(net, params.astype(np.float64), X0, dllr.astype(np.float64))
    check_grads(net, g, g16, tol=2e-3)


@pytest.mark.parametrize("kw", [dict(fuse_op=1), dict(fuse_op=1, fuse_mask=0b1011)])
def test_bf16_training_gradients_sum_interaction(kw):
    """A BF16 training handle with the sum interaction at the fusion points (the tensor-core
    run-time epilogue forms the sum; the FP32 fusion backward passes the gradient to every
    branch unchanged): against the oracle's 16-bit training emulation at the BF16 bar."""
    from oracle import half, net as onet, rx as orx
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=24, **kw)
    B = 3
    L, _, g, _ = grad_pair(net, w.sim, B, precision="bf16")
    ref = oracle_inputs(net, w.sim, 3, 0, B)
    params = onet.init_params(net, 4)
    params = (params + 0.05 * np.random.default_rng(4).standard_normal(params.size)).astype(np.float32)
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    assert normwise(L, half.forward_16(net, params.astype(np.float64), X0)) < 1e-3
    dllr = random_grid(3 + 10, L.shape, scale=1e-3)
    g16 = half.grad_16(net, params.astype(np.float64), X0, dllr.astype(np.float64))
    print(f"bf16 training {kw}: worst {check_grads(net, g, g16, tol=2e-3)}")


@pytest.mark.parametrize("name,kw", [("resid_14x624_b256_fp32", dict(n_sc=21, depth=2)),
                                     ("resnet_14x624_b256_fp32", dict(n_sc=13, depth=2)),
                                     ("resid_14x3276_b1024_bf16", dict(n_sc=11, depth=1))])
def test_residual_gradients(name, kw):
    w = WORKLOADS[name]
    net = replace(w.net, **kw)
    L, L_ref, g, g_ref = grad_pair(net, w.sim, 2, perturb=0.02)
    assert normwise(L, L_ref) < 1e-4
    check_grads(net, g, g_ref)


def test_adam_step_matches_oracle():
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=8)
    rx = api.Receiver(net, max_batch=1, train=True)
    p0 = onet.init_params(net, 5).astype(np.float32)
    rx.load_weights(p0)
    g = rx.grads_device()
    gv = random_grid(6, g.shape, scale=1e-2)
    g.copy_(dev(gv))
    m = np.zeros(p0.size)
    v = np.zeros(p0.size)
    p = p0.astype(np.float64)
    for step in (1, 2, 3):
        rx.adam_step(1e-3, step)
        p, m, v = onet.adam_step(p, gv.astype(np.float64), m, v, step, 1e-3)
    got = rx.save_weights()
    assert np.max(np.abs(got - p)) < 1e-6


def test_train_step_loss_and_gradient_match_oracle():
    from oracle import net as onet, rx as orx, sim as osim
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["train_14x72_b128_bf16"]
    B, seed, step = 8, 21, 3
    rx = api.Receiver(w.net, max_batch=B, train=True)
    p0 = onet.init_params(w.net, 7).astype(np.float32)
    rx.load_weights(p0)
    loss = rx.train_step(w.sim, seed, step, B, 0.0)          # lr 0: parameters unchanged
    g = rx.grads_device().cpu().numpy()
    s = osim.simulate(w.net, w.sim, seed, step * B, B)
    X0 = orx.assemble_input(s["Y"], s["pilot_sym"], s["pilot_mask"])
    loss_ref, g_ref, _ = onet.loss_and_grad(w.net, p0.astype(np.float64), X0, s["bits"], s["pilot_mask"])
    assert abs(loss - loss_ref) < 1e-5 * loss_ref
    assert normwise(g, g_ref) < 1e-3             # float32 simulator input vs float64
    assert np.array_equal(rx.save_weights(), p0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_training_reduces_loss(precision):
    """The loss first falls to log 2 (all LLRs shrink to 0), then below it as the network
    learns to detect; 300 steps of 128 slots go well below."""
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["train_14x72_b128_bf16"]
    rx = api.Receiver(w.net, precision=precision, max_batch=w.batch, train=True)
    rx.init_he(1)
    losses = [rx.train_step(w.sim, 5, i, w.batch, 1e-3, want_loss=(i < 5 or i >= 280)) for i in range(300)]
    first = [l for l in losses[:5]]
    last = [l for l in losses[280:]]
    assert np.all(np.isfinite(first + last))
    assert np.mean(last) < 0.85 * np.log(2.0) and np.mean(last) < 0.8 * np.mean(first), (first, last)


def test_trained_conet_beats_ls_lmmse():
    """The learned part earns its place: after 3000 steps on device-simulated slots, the
    14 x 72 CoNet's uncoded BER at 10 dB is below the LS-LMMSE receiver's on the same held-out
    slots (the paper's comparison against the conventional receiver, Sec. IV)."""
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["train_14x72_b128_bf16"]
    rx = api.Receiver(w.net, precision="fp32", max_batch=w.batch, train=True)
    rx.init_he(1)
    for i in range(3000):
        rx.train_step(w.sim, 5, i, w.batch, 3e-3, want_loss=False)
    mask, psym = api.pilots(w.net)
    s = api.sim_generate(w.net, w.sim, 999, 10_000_000, 256, fixed_snr_db=10.0)
    ev = api.Receiver(w.net, precision="fp32", max_batch=256)
    ev.load_weights(rx.save_weights())
    _, c_net, _ = api.loss_ber(ev.forward(s["Y"], mask, s["noise_var"]), s["bits"], mask)
    _, c_ls, _ = api.loss_ber(api.ls_lmmse(w.net, s["Y"], mask, psym, s["noise_var"]), s["bits"], mask)
    ber_net = c_net[0].item() / c_net[1].item()
    ber_ls = c_ls[0].item() / c_ls[1].item()
    n = c_net[1].item()
    sd = np.sqrt(ber_ls * (1 - ber_ls) / n)
    assert ber_net < ber_ls - 4 * sd, (ber_net, ber_ls)


def test_backward_requires_train_handle_and_matching_batch():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS["plain_14x72_b16_fp32"]
    rx = api.Receiver(w.net, max_batch=2)
    with pytest.raises(ConetError):
        rx.backward(torch.zeros((2, 14, 72, 4), device="cuda"))
    rt = api.Receiver(w.net, max_batch=2, train=True)
    rt.init_he(0)
    m = torch.zeros((14, 72), dtype=torch.uint8, device="cuda")
    rt.forward(torch.zeros((2, 1, 14, 72, 2), device="cuda"), m)
    with pytest.raises(ConetError):
        rt.backward(torch.zeros((1, 14, 72, 4), device="cuda"))


@pytest.mark.parametrize("name,kw", [("resid_14x624_b256_fp32", dict(n_sc=40, depth=3)),
                                     ("resnet_14x624_b256_fp32", dict(n_sc=24, depth=2))])
def test_recompute_gives_bitwise_identical_gradients(name, kw):
    """Residual training with per-block recompute (conet_config.recompute = 1) keeps only the
    residual streams of every block and reruns each block's pre-activation, first conv and
    normalisation during the backward pass: the same kernels on the same inputs, so the
    parameter gradient and the training trajectory are bitwise those of storing everything."""
    from paper_2510_12739_gb300 import api
    w = WORKLOADS[name]
    net = replace(w.net, **kw)
    out = []
    for rc in (False, True):
        rx = api.Receiver(net, "fp32", max_batch=3, train=True, recompute=rc)
        rx.init_he(4)
        for i in range(3):
            rx.train_step(w.sim, 12, i, 3, 1e-3, want_loss=False)
        s = api.sim_generate(net, w.sim, 8, 0, 3)
        mask, _ = api.pilots(net)
        llr = rx.forward(s["Y"], mask)
        rx.backward(dev(random_grid(14, tuple(llr.shape), scale=1e-3)))
        out.append((rx.save_weights(), rx.grads_device().cpu().numpy(), llr.cpu().numpy()))
        rx.sync()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
