"""The named workloads carry the shapes and link ranges of the five measured configurations,
and the ResNet comparison network matches the CoNet's parameter count."""
import numpy as np
import pytest

from oracle import net as onet
from workloads import WORKLOADS


def _n_params(net):
    return sum(int(np.prod(shape)) for _, shape in onet.param_layout(net))


@pytest.mark.parametrize("name,rx,sc,bits,nb,depth,width,residual,batch,cin", [
    ("plain_14x72_b16_fp32", 1, 72, 4, 2, 4, 32, 0, 16, 5),
    ("resid_14x624_b256_fp32", 2, 624, 6, 3, 6, 64, 1, 256, 7),
    ("train_14x72_b128_bf16", 1, 72, 4, 2, 4, 32, 0, 128, 5),
    ("resid_14x3276_b1024_bf16", 4, 3276, 8, 4, 8, 96, 1, 1024, 11),
    ("interf_14x72_b512_fp8", 1, 72, 4, 2, 4, 32, 0, 512, 5)])
def test_network_and_grid_shapes(name, rx, sc, bits, nb, depth, width, residual, batch, cin):
    w = WORKLOADS[name]
    n = w.net
    assert (n.n_rx, n.n_sc, n.qam_bits, n.n_branches, n.depth, n.width, n.residual) == \
        (rx, sc, bits, nb, depth, width, residual)
    assert n.n_sym == 14 and n.pilot_syms == (2, 11) and n.pilot_comb == 2
    assert n.c_in == cin and w.batch == batch
    assert all(n.fused(i) for i in range(n.depth + 1))          # Hadamard interaction at every point


@pytest.mark.parametrize("name,taps,ds,fd,snr,interferer", [
    ("plain_14x72_b16_fp32", 6, 100e-9, (0, 100), (0, 20), 0),
    ("resid_14x624_b256_fp32", 12, 300e-9, (0, 300), (-5, 25), 0),
    ("train_14x72_b128_bf16", 6, 100e-9, (0, 400), (-5, 25), 0),
    ("resid_14x3276_b1024_bf16", 12, 300e-9, (0, 300), (0, 30), 0),
    ("interf_14x72_b512_fp8", 6, 100e-9, (0, 400), (-5, 25), 1)])
def test_link_ranges(name, taps, ds, fd, snr, interferer):
    s = WORKLOADS[name].sim
    assert s.n_taps == taps and s.delay_spread_s == ds and not s.awgn
    assert (s.fd_lo, s.fd_hi) == fd and (s.snr_lo, s.snr_hi) == snr and s.interferer == interferer
    if interferer:
        assert (s.sir_lo, s.sir_hi) == (0, 20) and s.iqam_bits == 6      # 64-QAM interferer


def test_training_and_fp8_workloads_reuse_the_14x72_network():
    base = WORKLOADS["plain_14x72_b16_fp32"].net
    assert WORKLOADS["train_14x72_b128_bf16"].net == base and WORKLOADS["train_14x72_b128_bf16"].train
    assert WORKLOADS["interf_14x72_b512_fp8"].net == base


def test_resnet_matches_the_conet_parameter_count():
    conet = WORKLOADS["resid_14x624_b256_fp32"].net
    resnet = WORKLOADS["resnet_14x624_b256_fp32"].net
    assert resnet.resnet_baseline and resnet.n_branches == 1 and resnet.depth == conet.depth
    ratio = _n_params(resnet) / _n_params(conet)
    assert abs(ratio - 1) < 0.05, ratio


def test_depth_comparison_networks():
    """The 14-layer CoNet and the 24-layer ResNet of the depth comparison (Sec. IV, Fig.
    "InferenceD"): sequential layers = input conv + 2 per block + head, both near 1.9 M
    parameters and within 5 % of each other."""
    c = WORKLOADS["conet_d14_14x624_bf16"].net
    r = WORKLOADS["resnet_d24_14x624_bf16"].net
    assert 1 + 2 * c.depth + 1 == 14 and 1 + 2 * r.depth + 1 == 24
    assert c.n_branches > 1 and r.resnet_baseline and r.n_branches == 1
    nc, nr = _n_params(c), _n_params(r)
    assert 1.7e6 < nc < 2.1e6 and 1.7e6 < nr < 2.1e6 and abs(nc / nr - 1) < 0.05, (nc, nr)
