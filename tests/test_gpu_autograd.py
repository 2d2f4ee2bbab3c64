"""The torch.autograd binding (CoNetFn, CoNet): loss.backward() through the library's own
backward kernels must give the parameter gradient of conet_backward and of the FP64 oracle,
and an in-place torch optimiser step followed by params_updated() must take effect in the
next forward exactly as if the weights had been loaded."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, torch
from workloads import WORKLOADS, random_grid, replace

pytestmark = pytest.mark.gpu
GRAD_TOL = 2e-4   # the FP32 backward's bar (test_gpu_backward)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _case(n_sc=24, B=3):
    from oracle import net as onet
    w = WORKLOADS["train_14x72_b128_bf16"]
    net = replace(w.net, n_sc=n_sc)
    ref = oracle_inputs(net, w.sim, 3, 0, B)
    params = onet.init_params(net, 4)
    params = (params + 0.05 * np.random.default_rng(4).standard_normal(params.size)).astype(np.float32)
    return net, ref, params


def test_autograd_gradient_matches_oracle():
    from oracle import net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    net, ref, params = _case()
    B = ref["Y32"].shape[0]
    model = api.CoNet(net, precision="fp32", max_batch=B)
    model.rx.load_weights(params)
    assert np.array_equal(model.weight.detach().cpu().numpy(), params)   # the Parameter aliases the library
    llr = model(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    assert llr.requires_grad
    dllr = random_grid(13, tuple(llr.shape), scale=1e-3)
    (llr * dev(dllr)).sum().backward()
    g = model.weight.grad.cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    _, tape = onet.forward(net, params.astype(np.float64), X0, keep_tape=True)
    g_ref, _ = onet.backward(net, tape, dllr.astype(np.float64))
    o = 0
    for name, shape in onet.param_layout(net):
        n = int(np.prod(shape))
        assert normwise(g[o:o + n], g_ref[o:o + n]) < GRAD_TOL, name
        o += n


def test_torch_optimiser_step_then_params_updated():
    from paper_2510_12739_gb300 import api
    net, ref, params = _case()
    B = ref["Y32"].shape[0]
    Y, mask = dev(ref["Y32"]), dev(ref["pilot_mask"])
    model = api.CoNet(net, precision="fp32", max_batch=B)
    model.rx.load_weights(params)
    opt = torch.optim.SGD([model.weight], lr=1.0)
    llr0 = model(Y, mask)
    (llr0 * dev(random_grid(13, tuple(llr0.shape), scale=1e-3))).sum().backward()
    opt.step()
    model.params_updated()
    with torch.no_grad():
        llr1 = model(Y, mask)
    new = model.weight.detach().cpu().numpy()
    assert not np.array_equal(new, params)
    rx = api.Receiver(net, precision="fp32", max_batch=B)
    rx.load_weights(new)
    want = rx.forward(Y, mask)
    rx.sync()
    assert np.all(np.isfinite(llr1.detach().cpu().numpy()))
    assert normwise(llr1.detach().cpu().numpy(), want.cpu().numpy()) < 1e-6
    assert not np.array_equal(llr1.detach().cpu().numpy(), llr0.detach().cpu().numpy())   # the step took effect
