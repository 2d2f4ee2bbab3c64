"""Pins of the oracle's link simulator against facts fixed outside the oracle:
published Philox vectors and an independent Philox implementation, QAM algebra,
channel statistics (power, Jakes autocorrelation, PDP Fourier transform), noise
statistics and the noiseless identity y = H x."""
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import philox, sim as osim
from workloads import NetConfig, SimConfig, WORKLOADS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    for r in rows:
        out = philox.philox4x32(*r[:6])
        assert [int(o) for o in out] == r[6:]


def test_philox_matches_triton_interpreter():
    """Cross-check against Triton's own Philox4x32-10 (run in its CPU interpreter)."""
    pytest.importorskip("triton")
    import subprocess
    import sys
    code = r'''
import os
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out_ptr, seed, BLOCK: tl.constexpr):
    off = tl.arange(0, BLOCK)
    c0 = off.to(tl.uint32) * 977
    z = tl.zeros_like(c0)
    a, b, c, d = tl.philox(seed, c0, z + 7, z + 123456, z + 5)
    for i, v in enumerate((a, b, c, d)):
        tl.store(out_ptr + off * 4 + i, v.to(tl.int32, bitcast=True))
out = torch.zeros(256, dtype=torch.int32)
k[(1,)](out, 0x0123456789ABCDEF, BLOCK=64)
print(",".join(str(int(x) & 0xFFFFFFFF) for x in out))
'''
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    ref = np.array([int(x) for x in res.stdout.strip().split(",")], dtype=np.uint64)
    k0, k1 = philox.key_of(0x0123456789ABCDEF)
    got = np.stack(philox.philox4x32(np.arange(64, dtype=np.uint64) * 977, 7, 123456, 5, k0, k1), 1).reshape(-1)
    assert np.array_equal(got.astype(np.uint64), ref)


def test_uniform23_range_and_float32_exact():
    w = np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.uniform23(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 0.5 * 2.0 ** -23 and u[-1] == 1 - 0.5 * 2.0 ** -23


@pytest.mark.parametrize("q", [2, 4, 6, 8])
def test_qam_unit_energy_and_gray(q):
    pts, labels = osim.constellation(q)
    assert len(np.unique(np.round(pts, 12))) == 1 << q
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-12
    # nearest neighbours on the square grid differ in exactly one bit
    step = np.min(np.abs(np.diff(np.unique(np.round(pts.real, 12)))))
    for i in range(len(pts)):
        d = np.abs(pts - pts[i])
        nn = np.nonzero(np.abs(d - step) < 1e-9)[0]
        assert len(nn) >= 2
        for j in nn:
            assert np.sum(labels[i] != labels[j]) == 1


def test_qam_textbook_cases():
    pts, labels = osim.constellation(2)
    # QPSK: b = 0 -> -1/sqrt(2) on each axis
    for p, lab in zip(pts, labels):
        assert np.isclose(p.real, (2 * int(lab[0]) - 1) / np.sqrt(2))
        assert np.isclose(p.imag, (2 * int(lab[1]) - 1) / np.sqrt(2))
    pts16, _ = osim.constellation(4)
    assert np.allclose(np.sort(np.unique(np.round(pts16.real * np.sqrt(10), 9))), [-3, -1, 1, 3])


def test_pilot_grid_counts_and_fixedness():
    mask, p = osim.pilot_grid(14, 72, (2, 11), 2, 12739)
    assert mask.sum() == 72 and 14 * 72 - mask.sum() == 936
    assert np.allclose(np.abs(p[mask == 1]), 1.0) and np.all(p[mask == 0] == 0)
    mask2, p2 = osim.pilot_grid(14, 72, (2, 11), 2, 12739)
    assert np.array_equal(p, p2)
    assert np.all(mask[2, 1::2] == 0) and np.all(mask[[0, 1, 3], :] == 0)


@pytest.mark.parametrize("L,ds", [(6, 100e-9), (12, 300e-9), (1, 0.0)])
def test_tdl_profile_rms_spread(L, ds):
    P, tau = osim.tdl_profile(L, ds)
    assert abs(P.sum() - 1) < 1e-14
    m = np.sum(P * tau)
    assert abs(np.sqrt(np.sum(P * tau ** 2) - m * m) - ds) < 1e-18
    assert np.all(np.diff(P) < 0) if L > 1 else True


def _net(**kw):
    base = dict(n_rx=1, n_sc=72, qam_bits=4, n_branches=2, depth=4, width=32)
    base.update(kw)
    return NetConfig(**base)


def test_channel_power_and_static_and_flat():
    net = _net(n_rx=2)
    sim = SimConfig(n_taps=6, delay_spread_s=300e-9, fd_lo=0, fd_hi=300)
    slots = np.arange(400, dtype=np.uint64)
    fd = np.full(400, 0.0)
    H = osim.tdl_channel(sim, 2, 14, 72, 7, slots, osim.TAG_CHAN, fd)
    assert abs(np.mean(np.abs(H) ** 2) - 1.0) < 0.05
    assert np.allclose(H[:, :, 0:1, :], H)                       # f_D = 0: constant in time
    flat = osim.tdl_channel(SimConfig(n_taps=1, delay_spread_s=0.0), 1, 14, 72, 7, slots, osim.TAG_CHAN, fd + 200)
    assert np.allclose(flat[..., 0:1], flat)                     # one tap: flat across f


def test_channel_time_autocorrelation_is_jakes():
    """E[a(0) a*(t)] = J0(2 pi f_D t T_sym) for uniformly rotated sum-of-sinusoids."""
    sim = SimConfig(n_taps=1, delay_spread_s=0.0, scs_hz=30e3)
    n = 6000
    fd = np.full(n, 1500.0)
    H = osim.tdl_channel(sim, 1, 14, 1, 11, np.arange(n, dtype=np.uint64), osim.TAG_CHAN, fd)[:, 0, :, 0]
    Tsym = (1 + osim.CP_FRACTION) / sim.scs_hz
    for t in range(0, 14, 2):
        r = np.mean(H[:, 0] * np.conj(H[:, t])).real
        assert abs(r - special.j0(2 * np.pi * 1500.0 * t * Tsym)) < 0.06, t


def test_channel_frequency_correlation_is_pdp_transform():
    sim = SimConfig(n_taps=6, delay_spread_s=300e-9)
    n = 5000
    H = osim.tdl_channel(sim, 1, 1, 72, 5, np.arange(n, dtype=np.uint64), osim.TAG_CHAN, np.zeros(n))[:, 0, 0, :]
    P, tau = osim.tdl_profile(6, 300e-9)
    for dk in (1, 4, 16, 40):
        emp = np.mean(H[:, 10] * np.conj(H[:, 10 + dk]))
        theo = np.sum(P * np.exp(2j * np.pi * dk * 30e3 * tau))
        assert abs(emp - theo) < 0.06, (dk, emp, theo)


def test_noiseless_grid_is_h_times_x_and_bits():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    sim = SimConfig(**{**w.sim.__dict__, "snr_lo": np.inf, "snr_hi": np.inf})
    s = osim.simulate(w.net, sim, 3, 100, 4)
    assert np.all(s["noise_var"] == 0)
    assert np.allclose(s["Y"], s["H"] * s["x"][:, None])
    m = s["pilot_mask"].astype(bool)
    assert np.all(s["bits"][:, m] == 0)
    assert np.allclose(s["x"][:, m], s["pilot_sym"][m][None])
    assert abs(s["bits"][:, ~m].mean() - 0.5) < 0.02


def test_noise_variance_matches_snr():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    sim = SimConfig(**{**w.sim.__dict__, "snr_lo": 3.0, "snr_hi": 3.0})
    s = osim.simulate(w.net, sim, 9, 0, 64)
    n = s["Y"] - s["H"] * s["x"][:, None]
    k = n.size
    est = np.sum(np.abs(n) ** 2) / k
    sigma2 = 10 ** -0.3
    # 2 k est / sigma2 ~ chi^2 with 2k degrees of freedom
    lo, hi = stats.chi2.ppf([1e-4, 1 - 1e-4], 2 * k) * sigma2 / (2 * k)
    assert lo < est < hi
    assert np.allclose(s["noise_var"], sigma2)


def test_slot_draws_in_range_and_deterministic():
    w = WORKLOADS["interf_14x72_b512_fp8"]
    a = osim.simulate(w.net, w.sim, 5, 1000, 8)
    b = osim.simulate(w.net, w.sim, 5, 1004, 4)
    assert np.array_equal(a["Y"][4:], b["Y"]) and np.array_equal(a["bits"][4:], b["bits"])
    assert np.all((a["snr_db"] >= -5) & (a["snr_db"] <= 25))
    assert np.all((a["interf_var"] >= 10 ** -2) & (a["interf_var"] <= 1))
    c = osim.simulate(w.net, w.sim, 6, 1000, 8)
    assert not np.allclose(a["Y"], c["Y"])
