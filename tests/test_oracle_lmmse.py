"""Statistical pins of the oracle's LMMSE equaliser and exact demapper (the LS-LMMSE
receiver of Sec. I and Sec. IV, the BER reference of every trained-network test).

With the channel known, y = h x + n per antenna, n ~ CN(0, s2 I), the SIMO LMMSE output is
x_hat = h^H y / (|h|^2 + s2) = mu x + e with mu = |h|^2 / (|h|^2 + s2) and e a circular
Gaussian of variance |h|^2 s2 / (|h|^2 + s2)^2 = mu (1 - mu).  These tests measure mu and
var(e) by Monte Carlo on symbols drawn uniformly from the Gray QAM alphabet, so a wrong bias
term or error variance in ``lmmse_equalise`` fails them; the hard-decision and QPSK tests
elsewhere do not depend on nu.  Because e is exactly Gaussian and x uniform, the exact LLR
is the true posterior log-ratio: the empirical frequency of b = 1 among bits whose LLR falls
near l must follow the logistic curve 1 / (1 + e^-l), which pins the demapper's scale and
sign together with mu and nu."""
import numpy as np
import pytest
from scipy import stats

from oracle import rx as orx
from oracle.sim import constellation


def _draw(q, n_sym, h, s2, seed):
    """n_sym uniform QAM symbols through the fixed SIMO channel h [N] with noise CN(0, s2)."""
    rng = np.random.default_rng(seed)
    pts, labels = constellation(q)
    idx = rng.integers(0, len(pts), n_sym)
    x = pts[idx]
    N = len(h)
    n = np.sqrt(s2 / 2) * (rng.standard_normal((N, n_sym)) + 1j * rng.standard_normal((N, n_sym)))
    y = h[:, None] * x[None, :] + n                                   # [N, n_sym]
    # lmmse_equalise takes [B, N, T, F] grids and a per-slot variance: one slot, one symbol row
    Y = y[None, :, None, :]
    H = np.broadcast_to(h[None, :, None, None], Y.shape)
    xhat, mu, nu = orx.lmmse_equalise(Y, H, np.array([s2]))
    return x, labels[idx], xhat[0, 0], mu[0, 0], nu[0, 0]


CASES = [(4, np.array([0.9 - 0.4j]), 0.5), (4, np.array([0.3 + 0.2j, -0.5 + 0.1j]), 0.2),
         (6, np.array([1.1 + 0.3j, 0.2 - 0.7j]), 1.5), (2, np.array([0.6j]), 0.05)]


@pytest.mark.parametrize("q,h,s2", CASES)
def test_lmmse_bias_and_error_variance(q, h, s2):
    n_sym = 400_000
    x, _, xhat, mu, nu = _draw(q, n_sym, h, s2, 7)
    g = float(np.sum(np.abs(h) ** 2))
    mu_true = g / (g + s2)
    nu_true = g * s2 / (g + s2) ** 2
    assert np.allclose(mu, mu_true, rtol=1e-12) and np.allclose(nu, nu_true, rtol=1e-12)
    # the bias: least-squares slope of x_hat on x; e is independent of x with variance nu
    slope = np.vdot(x, xhat) / np.vdot(x, x)
    se = np.sqrt(nu_true / np.vdot(x, x).real)
    assert abs(slope - mu_true) < 5 * se, (slope, mu_true, se)
    # the error: x_hat - mu x has mean 0 and variance nu (chi-square interval on 2 n_sym dof)
    e = xhat - mu_true * x
    assert abs(e.mean()) < 5 * np.sqrt(nu_true / n_sym)
    dof = 2 * n_sym
    ratio = np.sum(np.abs(e) ** 2) / nu_true * 2              # ~ chi2(dof) when var(e) = nu
    lo, hi = stats.chi2.ppf([1e-6, 1 - 1e-6], dof)
    assert lo < ratio < hi, (ratio / dof, nu_true)
    # the two misreadings this guards against are far outside that interval
    for wrong in (1 - mu_true, mu_true):
        assert not (lo < np.sum(np.abs(e) ** 2) / wrong * 2 < hi)


@pytest.mark.parametrize("q,h,s2", CASES[:3])
def test_exact_llr_is_calibrated(q, h, s2):
    """P(b = 1 | LLR in a bin) = mean over the bin of 1 / (1 + e^-LLR), within binomial error."""
    x, bits, xhat, mu, nu = _draw(q, 300_000, h, s2, 11)
    mu, nu = float(mu.flat[0]), float(nu.flat[0])        # the channel is fixed: one value each
    llr = orx.demap(xhat[None], np.full((1, len(xhat)), mu), np.full((1, len(xhat)), nu), q, exact=True)[0]
    L = llr.ravel()
    b = bits.ravel().astype(np.float64)
    edges = np.array([-8, -4, -2, -1, -0.5, 0, 0.5, 1, 2, 4, 8], dtype=np.float64)
    checked = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (L >= lo) & (L < hi)
        n = int(sel.sum())
        if n < 2000:
            continue
        p_model = float(np.mean(1 / (1 + np.exp(-L[sel]))))
        p_emp = float(b[sel].mean())
        sd = np.sqrt(p_model * (1 - p_model) / n)
        assert abs(p_emp - p_model) < 5 * sd + 1e-3, (lo, hi, p_emp, p_model, n)
        checked += 1
    assert checked >= 6
    # a demapper with the error variance misread as 1 - mu is visibly miscalibrated
    wrong = orx.demap(xhat[None], np.full((1, len(xhat)), mu), np.full((1, len(xhat)), 1 - mu), q, exact=True)[0]
    Lw = wrong.ravel()
    sel = (Lw >= 1) & (Lw < 2)
    if sel.sum() > 2000 and abs(nu - (1 - mu)) > 0.05:
        p_model = float(np.mean(1 / (1 + np.exp(-Lw[sel]))))
        sd = np.sqrt(p_model * (1 - p_model) / sel.sum())
        assert abs(float(b[sel].mean()) - p_model) > 5 * sd
