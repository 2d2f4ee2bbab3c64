"""GPU parity of the whole-network kernel (conet_whole_network): every layer and the head of
a small plain BF16 or E4M3 CoNet (2 branches x 32 channels, the 14 x 72 networks of Example I) in
one persistent kernel with the activations in shared memory.

Against the oracle's BF16 emulation (oracle.half: conv inputs and weights rounded to BF16,
everything else exact) the kernel differs only by FP32 accumulation order and the rare BF16
rounding decision that flips: 1e-3 normwise per 4 layers, the layer-by-layer kernels' bar on
plain networks.  Against the layer-by-layer path of the same handle (the same BF16 operands,
another FP32 summation order) it must agree to 1e-5 (measured 4e-8 to 2e-7).
Cases cover the full 14 x 72 grid at the benchmark batches, more slots than SMs, narrower
grids (fewer than eight 128-row tiles of real rows), 1..8 layers, partial fusion and a
LayerNorm after the fusion.  Calls of few slots split each slot over a cluster of 8, 4 or 2
CTAs that exchange halo rows through distributed shared memory (1-24 slots: 8 or 4; 60: 4
or 2, depending on how many clusters fit), larger calls run one slot per CTA (200, 300).

E4M3: the first forward calibrates the activation scales on the layer-by-layer path; later
forwards run the whole-network kernel with those scales.  Against the oracle's E4M3 emulation
(same calibration rule on the same batch) the bars are those of the layer-by-layer kernels;
against the layer path with the same scales the two differ only where an FP32 summation-order
difference moves a value across an E4M3 rounding boundary (a few elements in 10^5)."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, torch
from workloads import WORKLOADS, replace

pytestmark = pytest.mark.gpu
EMU_MAX = 1e-3


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


CASES = [(dict(), 16), (dict(), 1), (dict(), 200), (dict(), 24), (dict(), 60), (dict(n_sc=40), 3), (dict(n_sc=17), 2), (dict(n_sym=7, pilot_syms=(1, 5), n_sc=40), 2),
         (dict(depth=2), 4), (dict(depth=8), 2), (dict(fuse_mask=0b0101), 3), (dict(norm=1, depth=3), 2)]


@pytest.mark.parametrize("kw,B", CASES)
def test_whole_network_matches_emulation_and_layer_path(kw, B):
    from oracle import half, net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, **kw)
    ref = oracle_inputs(net, w.sim, 5, 0, B)
    params = onet.init_params(net, 3)
    params = (params + 0.02 * np.random.default_rng(3).standard_normal(params.size)).astype(np.float32)
    rx = api.Receiver(net, "bf16", max_batch=B)
    rx.load_weights(params)
    rx.graphs(False)
    assert rx.whole_network(True)
    n0 = api.launch_count()
    L = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"])).clone()
    rx.sync()
    launches = api.launch_count() - n0
    rx.whole_network(False)
    L_layers = rx.forward(dev(ref["Y32"]), dev(ref["pilot_mask"]))
    rx.sync()
    L, L_layers = L.cpu().numpy(), L_layers.cpu().numpy()
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    X0 = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    L_emu = half.forward_16(net, params.astype(np.float64), X0, "bf16")
    e_emu, e_lay = normwise(L, L_emu), normwise(L, L_layers)
    print(f"whole net {kw} B={B}: vs emulation {e_emu:.2e}, vs layer path {e_lay:.2e}, {launches} launches")
    assert np.all(np.isfinite(L))
    # LayerNorm after the fusion at He init: see test_gpu_bf16.  The flipped BF16 rounding
    # decisions accumulate over layers: 8 layers measured 1.6e-3 against the emulation, on
    # both paths alike (the two paths agree to 1.4e-7)
    # With a LayerNorm after the fusion the two paths' FP32 summation orders flip a few more
    # BF16 roundings of the normalised products (measured 9.6e-5 between them)
    bar = 0.1 if net.norm else EMU_MAX * max(1.0, net.depth / 4)
    assert e_emu < bar, e_emu
    assert e_lay < (1e-3 if net.norm else 1e-5), e_lay
    assert launches == 3                   # assembly, padding, the network


def test_whole_network_availability():
    from paper_2510_12739_gb300 import api
    net = WORKLOADS["plain_14x72_b16_fp32"].net
    assert not api.Receiver(replace(net, n_branches=3), "bf16", max_batch=1).whole_network(True)
    assert not api.Receiver(net, "fp16", max_batch=1).whole_network(True)
    assert not api.Receiver(replace(net, n_sc=80), "bf16", max_batch=1).whole_network(True)   # 14 x 81 > 1024 rows
    assert api.Receiver(net, "bf16", max_batch=1).whole_network(True)
    assert api.Receiver(net, "fp8", max_batch=1).whole_network(True)


FP8_CASES = [("plain_14x72_b16_fp32", dict(), 16), ("interf_14x72_b512_fp8", dict(), 300),
             ("plain_14x72_b16_fp32", dict(n_sc=40, depth=6), 3), ("plain_14x72_b16_fp32", dict(fuse_mask=0b0101), 2)]


@pytest.mark.parametrize("wl,kw,B", FP8_CASES)
def test_whole_network_e4m3(wl, kw, B):
    from oracle import net as onet, pipeline
    from paper_2510_12739_gb300 import api
    w = WORKLOADS[wl]
    net = replace(w.net, **kw)
    ref = oracle_inputs(net, w.sim, 7, 0, B)
    params = onet.init_params(net, 4).astype(np.float32)
    rx = api.Receiver(net, "fp8", max_batch=B)
    rx.load_weights(params)
    rx.graphs(False)
    assert rx.whole_network(True)
    Y, M = dev(ref["Y32"]), dev(ref["pilot_mask"])
    L_cal = rx.forward(Y, M).clone()          # calibrates on the layer path
    n0 = api.launch_count()
    L = rx.forward(Y, M).clone()
    rx.sync()
    launches = api.launch_count() - n0
    rx.whole_network(False)
    L_layers = rx.forward(Y, M)
    rx.sync()
    L, L_layers, L_cal = L.cpu().numpy(), L_layers.cpu().numpy(), L_cal.cpu().numpy()
    assert np.array_equal(L_layers, L_cal)    # the same scales on both layer-path passes
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    L_emu = pipeline.receive_fp8(net, params.astype(np.float64), Yd, ref["pilot_sym"], ref["pilot_mask"], margin=2.0)
    scale = np.max(np.abs(L_emu))
    e_emu = np.abs(L - L_emu) / scale
    e_lay = np.abs(L - L_layers) / scale
    print(f"whole net e4m3 {wl} {kw} B={B}: vs emulation max {e_emu.max():.2e} median {np.median(e_emu):.1e}, "
          f"vs layer path max {e_lay.max():.2e} median {np.median(e_lay):.1e}, {launches} launches")
    assert np.all(np.isfinite(L))
    assert e_emu.max() < 1e-2 and np.median(e_emu) < 1e-5
    assert e_lay.max() < 1e-2 and np.median(e_lay) < 1e-6
    assert launches == 3
