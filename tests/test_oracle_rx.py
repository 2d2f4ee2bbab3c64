"""Pins of the oracle's receiver DSP: exact LS at noiseless pilots, exact linear
interpolation of a linear channel, the QPSK closed-form LLR, and the closed-form
uncoded BER of Gray-mapped square QAM on AWGN with perfect CSI."""
import numpy as np
import pytest
from scipy import special

from oracle import rx as orx, sim as osim
from workloads import SimConfig, WORKLOADS, replace


@pytest.mark.parametrize("name,c", [("plain_14x72_b16_fp32", 5), ("resid_14x624_b256_fp32", 7),
                                    ("resid_14x3276_b1024_bf16", 11)])
def test_input_channel_counts(name, c):
    assert WORKLOADS[name].net.c_in == c


def _noiseless(sim):
    return replace(sim, snr_lo=np.inf, snr_hi=np.inf)


@pytest.mark.parametrize("n_rx", [1, 2])
def test_ls_exact_at_pilots_without_noise(n_rx):
    w = WORKLOADS["plain_14x72_b16_fp32"]
    net = replace(w.net, n_rx=n_rx)
    s = osim.simulate(net, _noiseless(w.sim), 1, 0, 3)
    X = orx.assemble_input(s["Y"], s["pilot_sym"], s["pilot_mask"])
    m = s["pilot_mask"].astype(bool)
    Hbar = s["H"].mean(axis=1)
    assert X.shape[-1] == 2 * n_rx + 3
    assert np.allclose(X[:, m, 2 * n_rx + 1], Hbar[:, m].real, atol=1e-12)
    assert np.allclose(X[:, m, 2 * n_rx + 2], Hbar[:, m].imag, atol=1e-12)
    assert np.all(X[:, ~m, 2 * n_rx + 1:] == 0)
    assert np.all(X[..., 2 * n_rx] == m[None].astype(float))
    for n in range(n_rx):
        assert np.array_equal(X[..., n], s["Y"][:, n].real)
        assert np.array_equal(X[..., n_rx + n], s["Y"][:, n].imag)


def test_interpolation_reproduces_a_linear_channel():
    T, F = 14, 24
    mask, p = osim.pilot_grid(T, F, (2, 11), 2, 77)
    t = np.arange(T)[:, None]
    f = np.arange(F)[None, :]
    H = (0.3 + 0.1j) + (0.02 - 0.01j) * f + (-0.05 + 0.03j) * t
    Y = (H * np.where(mask, p, 1.0))[None, None]
    est = orx.interpolate_ls(Y, p, mask, (2, 11))[0, 0]
    inner = (slice(2, 12), slice(0, F - 1))      # between pilot symbols and pilot subcarriers
    assert np.allclose(est[inner], H[inner], atol=1e-12)
    assert np.allclose(est[0], est[2]) and np.allclose(est[13], est[11])
    assert np.allclose(est[:, F - 1], est[:, F - 2])


def test_lmmse_noiseless_static_flat_channel_is_error_free():
    w = WORKLOADS["plain_14x72_b16_fp32"]
    sim = replace(_noiseless(w.sim), n_taps=1, delay_spread_s=0.0, fd_lo=0.0, fd_hi=0.0)
    s = osim.simulate(w.net, sim, 4, 0, 4)
    llr = orx.ls_lmmse(s["Y"], s["noise_var"], s["pilot_sym"], s["pilot_mask"], (2, 11), 4)
    e, n = orx.bit_errors(llr, s["bits"], s["pilot_mask"])
    assert e == 0 and n == 4 * 936 * 4
    assert np.min(np.abs(llr[:, ~s["pilot_mask"].astype(bool)])) > 1e3


def test_exact_qpsk_llr_closed_form():
    rng = np.random.default_rng(0)
    xhat = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    mu = rng.uniform(0.2, 0.9, 50)
    nu = mu * (1 - mu)
    llr = orx.demap(xhat, mu, nu, 2, exact=True)
    a = 1 / np.sqrt(2)
    assert np.allclose(llr[:, 0], 4 * mu * a * xhat.real / nu, rtol=1e-10)
    assert np.allclose(llr[:, 1], 4 * mu * a * xhat.imag / nu, rtol=1e-10)


def gray_pam_ber(q, snr_db):
    """Exact per-bit error probability of nearest-point detection of Gray square QAM
    (binary-reflected Gray code per axis, unit average energy) on AWGN CN(0, s2)."""
    half = q // 2
    P = 1 << half
    d = 1 / np.sqrt(2 * ((1 << q) - 1) / 3)
    lv = (2 * np.arange(P) - (P - 1)) * d
    s = np.sqrt(10 ** (-snr_db / 10) / 2)
    edges = np.concatenate([[-np.inf], (lv[:-1] + lv[1:]) / 2, [np.inf]])
    gray = np.arange(P) ^ (np.arange(P) >> 1)
    Qf = lambda x: 0.5 * special.erfc(x / np.sqrt(2))
    tot = 0.0
    for j in range(half):
        bit = (gray >> (half - 1 - j)) & 1
        for i in range(P):
            for r in range(P):
                if bit[r] != bit[i]:
                    tot += (Qf((edges[r] - lv[i]) / s) - Qf((edges[r + 1] - lv[i]) / s)) / P
    return tot / half


@pytest.mark.parametrize("q,snr", [(2, 4.0), (4, 10.0), (6, 16.0), (8, 22.0)])
def test_awgn_perfect_csi_ber_matches_closed_form(q, snr):
    net = replace(WORKLOADS["plain_14x72_b16_fp32"].net, qam_bits=q)
    sim = SimConfig(awgn=1, snr_lo=snr, snr_hi=snr)
    errs = bits = 0
    for chunk in range(4):
        s = osim.simulate(net, sim, 21, chunk * 64, 64)
        llr = orx.ls_lmmse(s["Y"], s["noise_var"], s["pilot_sym"], s["pilot_mask"], (2, 11), q,
                           H_perfect=s["H"], exact=False)
        e, n = orx.bit_errors(llr, s["bits"], s["pilot_mask"])
        errs += e
        bits += n
    p = gray_pam_ber(q, snr)
    sd = np.sqrt(p * (1 - p) / bits)
    assert abs(errs / bits - p) < 4.5 * sd, (errs / bits, p, sd)


def test_bit_error_count_on_known_decisions():
    mask = np.zeros((2, 3), dtype=np.uint8)
    mask[0, 0] = 1
    bits = np.zeros((1, 2, 3, 2), dtype=np.uint8)
    llr = -np.ones((1, 2, 3, 2))
    llr[0, 0, 0, :] = 5.0          # pilot RE: ignored
    llr[0, 1, 2, 1] = 0.5          # one error
    llr[0, 1, 1, 0] = 0.0          # tie decides 0: correct
    assert orx.bit_errors(llr, bits, mask) == (1, 10)
