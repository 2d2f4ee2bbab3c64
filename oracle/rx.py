"""FP64 oracle of the receiver-side DSP around CoNet.

* ``assemble_input``: the network input of Sec. II-A -- the complex grid Y split into
  real and imaginary channels per antenna -- plus the pilot mask and the LS channel
  estimate at the pilots, averaged over antennas (O6 reading: C_in = 2N + 3).
* ``ls_lmmse``: the conventional receiver the paper compares against (Sec. I, Sec. IV:
  LS channel estimation at the pilots and LMMSE equalisation, with imperfect or
  perfect CSI), followed by exact or max-log demapping.
* ``bit_errors``: hard decisions b = [LLR > 0] and error counts over data REs
  (the BER metric of Sec. IV, uncoded).

LLR sign convention: LLR = log P(b = 1) / P(b = 0).
"""
from __future__ import annotations

import numpy as np

from .sim import constellation


def ls_estimate(Y, pilot_sym, pilot_mask):
    """Per-antenna LS estimate y conj(p) / |p|^2 at pilot REs, 0 elsewhere. Y [B,N,T,F]."""
    m = pilot_mask.astype(bool)
    p = np.where(m, pilot_sym, 1.0)
    return np.where(m[None, None], Y * np.conj(p) / np.abs(p) ** 2, 0.0)


def assemble_input(Y, pilot_sym, pilot_mask):
    """Network input X0 [B, T, F, 2N+3]: Re Y_0..N-1, Im Y_0..N-1, mask, Re/Im of the
    antenna-averaged LS estimate (channels last)."""
    B, N, T, F = Y.shape
    Hls = ls_estimate(Y, pilot_sym, pilot_mask).mean(axis=1)          # [B, T, F]
    X = np.zeros((B, T, F, 2 * N + 3))
    for n in range(N):
        X[..., n] = Y[:, n].real
        X[..., N + n] = Y[:, n].imag
    X[..., 2 * N] = pilot_mask[None]
    X[..., 2 * N + 1] = Hls.real
    X[..., 2 * N + 2] = Hls.imag
    return X


def interpolate_ls(Y, pilot_sym, pilot_mask, pilot_syms):
    """Full-grid channel estimate from the LS pilots: linear interpolation across
    subcarriers between pilot subcarriers (constant beyond the outermost ones), then
    linearly across OFDM symbols between the pilot symbols (constant outside)."""
    B, N, T, F = Y.shape
    Hls = ls_estimate(Y, pilot_sym, pilot_mask)
    f = np.arange(F)
    rows = []
    for tp in pilot_syms:
        fp = np.nonzero(pilot_mask[tp])[0]
        v = Hls[:, :, tp, fp]                                             # [B, N, P]
        re = np.apply_along_axis(lambda r: np.interp(f, fp, r), -1, v.real)
        im = np.apply_along_axis(lambda r: np.interp(f, fp, r), -1, v.imag)
        rows.append(re + 1j * im)                                         # [B, N, F]
    rows = np.stack(rows, axis=2)                                         # [B, N, P_t, F]
    tp = np.asarray(pilot_syms, dtype=np.float64)
    out = np.zeros((B, N, T, F), dtype=np.complex128)
    for t in range(T):
        if len(tp) == 1 or t <= tp[0]:
            out[:, :, t] = rows[:, :, 0]
        elif t >= tp[-1]:
            out[:, :, t] = rows[:, :, -1]
        else:
            j = np.searchsorted(tp, t, side="right") - 1
            w = (t - tp[j]) / (tp[j + 1] - tp[j])
            out[:, :, t] = (1 - w) * rows[:, :, j] + w * rows[:, :, j + 1]
    return out


def lmmse_equalise(Y, Hhat, var_eff):
    """SIMO LMMSE per RE: x_hat = h^H y / (|h|^2 + s2), mu = |h|^2 / (|h|^2 + s2);
    x_hat = mu x + e with var(e) = mu (1 - mu) for E|x|^2 = 1."""
    s2 = np.asarray(var_eff, dtype=np.float64)[:, None, None]
    g = np.sum(np.abs(Hhat) ** 2, axis=1)                                 # [B, T, F]
    num = np.sum(np.conj(Hhat) * Y, axis=1)
    den = g + s2
    xhat = num / den
    mu = g / den
    nu = mu * (1.0 - mu)
    return xhat, mu, nu


def demap(xhat, mu, nu, q, exact=True, nu_floor=1e-12):
    """LLR_k = log sum_{s: b_k=1} exp(-|x - mu s|^2 / nu) - log sum_{s: b_k=0} (...)
    (exact), or the max-log version with min distances."""
    pts, labels = constellation(q)
    nu = np.maximum(nu, nu_floor)
    d = -np.abs(xhat[..., None] - mu[..., None] * pts) ** 2 / nu[..., None]   # [..., M]
    llr = np.zeros(xhat.shape + (q,))
    for k in range(q):
        one = labels[:, k] == 1
        d1, d0 = d[..., one], d[..., ~one]
        if exact:
            m1, m0 = d1.max(-1), d0.max(-1)
            l1 = m1 + np.log(np.exp(d1 - m1[..., None]).sum(-1))
            l0 = m0 + np.log(np.exp(d0 - m0[..., None]).sum(-1))
            llr[..., k] = l1 - l0
        else:
            llr[..., k] = d1.max(-1) - d0.max(-1)
    return llr


def ls_lmmse(Y, noise_var, pilot_sym, pilot_mask, pilot_syms, q, interf_var=None,
             H_perfect=None, exact=True):
    """LS-LMMSE receiver (imperfect CSI), or LMMSE with the true channel when
    ``H_perfect`` is given.  Interference is treated as noise: s2 = sigma^2 + P_I."""
    var_eff = np.asarray(noise_var, dtype=np.float64)
    if interf_var is not None:
        var_eff = var_eff + np.asarray(interf_var, dtype=np.float64)
    Hhat = H_perfect if H_perfect is not None else interpolate_ls(Y, pilot_sym, pilot_mask, pilot_syms)
    xhat, mu, nu = lmmse_equalise(Y, Hhat, var_eff)
    return demap(xhat, mu, nu, q, exact=exact)


def bit_errors(llr, bits, pilot_mask):
    """(errors, bits counted) over data REs; hard decision b_hat = [LLR > 0]."""
    data = ~pilot_mask.astype(bool)
    hard = (llr > 0).astype(np.uint8)
    err = (hard != bits)[:, data, :]
    return int(err.sum()), int(err.size)
