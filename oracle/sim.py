"""FP64 oracle of the synthetic OFDM uplink (Sec. II and Eq. 1 of the CoNet-Rx paper).

Per slot (one TTI of T = 14 OFDM symbols x F subcarriers) and receive antenna n:

    y_n[t, f] = h_n[t, f] x[t, f] + sqrt(P_I) g_n[t, f] z[t, f] e^{-j 2 pi k delta} + n_n[t, f]

with x the Gray-mapped QAM data (uniform random bits, Sec. II) or the fixed QPSK
pilots (Sec. II-A: pilots are fixed from slot to slot), h and g independent TDL
Rayleigh channels with Doppler (Sec. IV: TDL channels with random delay spread /
UE speed), z a random-data QAM interferer with a random time offset delta and
random SIR (Sec. II), and n circular Gaussian noise.

The time-domain IFFT / cyclic prefix / FFT chain of Sec. II is replaced by its exact
frequency-domain equivalent y = H x per resource element, which holds while the
cyclic prefix covers the channel's delay spread (inter-carrier interference from
Doppler is neglected; f_D / scs stays below 1.4 %).

Random draws come from Philox4x32-10 with key = seed and counter
(c0, c1, c2 = slot, c3 = stream tag); see ``TAG_*`` for the layout.
"""
from __future__ import annotations

import numpy as np

from .philox import key_of, philox4x32, uniform23

TAG_SLOT = 1     # c0 = 0, c1 = 0: words -> SNR, Doppler, SIR, interferer offset
TAG_BITS = 2     # c0 = t*F + f: low Q bits of word 0 are b_0 .. b_{Q-1}
TAG_PILOT = 3    # key = pilot_seed, c2 = 0, c0 = t*F + f: bits 0/1 of word 0
TAG_CHAN = 4     # c0 = n*256 + l, c1 = j: uniforms 4j..4j+3 (theta, then phi_s)
TAG_ICHAN = 5    # same layout for the interferer's channel
TAG_NOISE = 6    # c0 = t*F + f, c1 = n: words 0, 1 -> Box-Muller pair
TAG_IBITS = 7    # c0 = t*F + f: interferer symbol bits

CP_FRACTION = 9.0 / 128.0      # normal cyclic prefix, ~7 % of the useful symbol


def qam_amplitudes(bits: np.ndarray, q: int) -> np.ndarray:
    """Gray-mapped square QAM of unit average energy (O2 reading of Sec. II mapping).

    ``bits[..., k]`` for k = 0..q-1; even positions label the in-phase axis and odd
    positions the quadrature axis, most significant first.  Each axis label is a
    binary-reflected Gray code of the PAM level index i, amplitude
    (2 i - (P - 1)) / sqrt(2 (M - 1) / 3) with P = 2**(q/2), M = 2**q.
    """
    half = q // 2
    P = 1 << half
    M = 1 << q
    scale = 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)

    def axis(sel):
        label = np.zeros(bits.shape[:-1], dtype=np.int64)
        for i, k in enumerate(sel):
            label |= bits[..., k].astype(np.int64) << (half - 1 - i)
        idx = label.copy()
        shift = label >> 1
        while np.any(shift):
            idx ^= shift
            shift >>= 1
        return (2.0 * idx - (P - 1)) * scale

    return axis(range(0, q, 2)) + 1j * axis(range(1, q, 2))


def constellation(q: int):
    """All 2**q points and their bit labels (label row k = bits of point k)."""
    M = 1 << q
    labels = ((np.arange(M)[:, None] >> np.arange(q)[None, :]) & 1).astype(np.uint8)
    return qam_amplitudes(labels, q), labels


def pilot_grid(n_sym: int, n_sc: int, pilot_syms, comb: int, pilot_seed: int):
    """Fixed pilot mask [T, F] and QPSK pilot symbols [T, F] (0 on data REs)."""
    mask = np.zeros((n_sym, n_sc), dtype=np.uint8)
    for t in pilot_syms:
        mask[t, ::comb] = 1
    r = np.arange(n_sym * n_sc, dtype=np.uint64)
    k0, k1 = key_of(pilot_seed)
    w0 = philox4x32(r, 0, 0, TAG_PILOT, k0, k1)[0].astype(np.int64)
    u0 = w0 & 1
    u1 = (w0 >> 1) & 1
    p = ((1 - 2 * u0) + 1j * (1 - 2 * u1)) / np.sqrt(2.0)
    p = p.reshape(n_sym, n_sc) * mask
    return mask, p


def tdl_profile(n_taps: int, delay_spread_s: float):
    """Exponential power-delay profile P_l ~ e^{-l}, delays tau_l = l d scaled so that
    the rms delay spread equals ``delay_spread_s`` exactly (O4 reading)."""
    l = np.arange(n_taps, dtype=np.float64)
    P = np.exp(-l)
    P /= P.sum()
    if n_taps == 1:
        return P, np.zeros(1)
    mean = np.sum(l * P)
    sig = np.sqrt(np.sum(l * l * P) - mean * mean)
    return P, l * (delay_spread_s / sig)


def slot_params(sim, seed: int, slots: np.ndarray):
    k0, k1 = key_of(seed)
    w = philox4x32(0, 0, slots, TAG_SLOT, k0, k1)
    u = [uniform23(x) for x in w]
    def draw(lo, hi, x):                       # a degenerate range is the value itself
        return np.full(x.shape, float(lo)) if lo == hi else lo + (hi - lo) * x
    snr_db = draw(sim.snr_lo, sim.snr_hi, u[0])
    fd = draw(sim.fd_lo, sim.fd_hi, u[1])
    sir_db = draw(sim.sir_lo, sim.sir_hi, u[2])
    delta = CP_FRACTION * u[3]
    return snr_db, fd, sir_db, delta


def tdl_channel(sim, n_rx, n_sym, n_sc, seed, slots, tag, fd):
    """H[b, n, t, f] of a sum-of-sinusoids TDL Rayleigh channel (O4 reading of Sec. IV).

    a_{n,l}(t) = sqrt(P_l / S) sum_s exp(j (2 pi f_D cos(alpha_s) t T_sym + phi_s)),
    alpha_s = 2 pi (s + theta) / S, and H = sum_l a_l(t) exp(-j 2 pi k scs tau_l) with
    k = f - F // 2 and T_sym = (1 + CP) / scs.
    """
    B = len(slots)
    if sim.awgn:
        return np.ones((B, n_rx, n_sym, n_sc), dtype=np.complex128)
    S = sim.n_sinusoids
    L = sim.n_taps
    P, tau = tdl_profile(L, sim.delay_spread_s)
    k0, k1 = key_of(seed)
    n_words = S + 1
    n_blocks = (n_words + 3) // 4
    T_sym = (1.0 + CP_FRACTION) / sim.scs_hz
    t = np.arange(n_sym, dtype=np.float64)
    kf = np.arange(n_sc, dtype=np.float64) - (n_sc // 2)
    H = np.zeros((B, n_rx, n_sym, n_sc), dtype=np.complex128)
    for n in range(n_rx):
        for l in range(L):
            c0 = n * 256 + l
            u = np.zeros((B, 4 * n_blocks))
            for j in range(n_blocks):
                w = philox4x32(c0, j, slots, tag, k0, k1)
                for i in range(4):
                    u[:, 4 * j + i] = uniform23(w[i])
            theta = u[:, 0]
            phi = 2.0 * np.pi * u[:, 1:S + 1]                               # [B, S]
            alpha = 2.0 * np.pi * (np.arange(S)[None, :] + theta[:, None]) / S
            dop = fd[:, None] * np.cos(alpha)                               # [B, S] Hz
            ph = 2.0 * np.pi * dop[:, :, None] * (t[None, None, :] * T_sym) + phi[:, :, None]
            a = np.sqrt(P[l] / S) * np.exp(1j * ph).sum(axis=1)             # [B, T]
            e = np.exp(-2j * np.pi * kf * sim.scs_hz * tau[l])              # [F]
            H[:, n] += a[:, :, None] * e[None, None, :]
    return H


def data_bits(seed, slots, n_sym, n_sc, q, tag=TAG_BITS):
    k0, k1 = key_of(seed)
    r = np.arange(n_sym * n_sc, dtype=np.uint64)
    w0 = philox4x32(r[None, :], 0, slots[:, None], tag, k0, k1)[0].astype(np.int64)
    bits = ((w0[..., None] >> np.arange(q)) & 1).astype(np.uint8)
    return bits.reshape(len(slots), n_sym, n_sc, q)


def noise(seed, slots, n_rx, n_sym, n_sc):
    """Unit-variance circular Gaussian samples by Box-Muller on Philox uniforms."""
    k0, k1 = key_of(seed)
    r = np.arange(n_sym * n_sc, dtype=np.uint64)
    g = np.zeros((len(slots), n_rx, n_sym * n_sc), dtype=np.complex128)
    for n in range(n_rx):
        w = philox4x32(r[None, :], n, slots[:, None], TAG_NOISE, k0, k1)
        u0, u1 = uniform23(w[0]), uniform23(w[1])
        rad = np.sqrt(-2.0 * np.log(u0))
        g[:, n] = rad * np.cos(2 * np.pi * u1) + 1j * rad * np.sin(2 * np.pi * u1)
    return g.reshape(len(slots), n_rx, n_sym, n_sc)


def simulate(net, sim, seed: int, slot0: int, batch: int, fixed_snr_db=None):
    """Generate ``batch`` slots (global slot ids slot0 .. slot0+batch-1).

    Returns a dict with Y [B,N,T,F] complex, bits [B,T,F,Q] uint8 (0 on pilot REs),
    H [B,N,T,F], x [B,T,F], noise_var [B] (= sigma^2 = 10^(-SNR/10), Es/N0 per
    antenna with E|x|^2 = E|h|^2 = 1), interf_var [B] (= P_I), pilot_mask, pilot_sym.
    ``fixed_snr_db`` overrides the per-slot SNR draw (BER sweeps)."""
    T, F, N, Q = net.n_sym, net.n_sc, net.n_rx, net.qam_bits
    slots = (np.arange(batch, dtype=np.uint64) + np.uint64(slot0)) & np.uint64(0xFFFFFFFF)
    mask, psym = pilot_grid(T, F, net.pilot_syms, net.pilot_comb, net.pilot_seed)
    snr_db, fd, sir_db, delta = slot_params(sim, seed, slots)
    if fixed_snr_db is not None:
        snr_db = np.full(batch, float(fixed_snr_db))
    sigma2 = 10.0 ** (-snr_db / 10.0)
    bits = data_bits(seed, slots, T, F, Q)
    bits[:, mask.astype(bool)] = 0
    x = qam_amplitudes(bits, Q)
    x = np.where(mask.astype(bool)[None], psym[None], x)
    H = tdl_channel(sim, N, T, F, seed, slots, TAG_CHAN, fd)
    Y = H * x[:, None]
    p_i = np.zeros(batch)
    if sim.interferer:
        p_i = 10.0 ** (-sir_db / 10.0)
        zb = data_bits(seed, slots, T, F, sim.iqam_bits, tag=TAG_IBITS)
        z = qam_amplitudes(zb, sim.iqam_bits)
        G = tdl_channel(sim, N, T, F, seed, slots, TAG_ICHAN, fd)
        kf = np.arange(F, dtype=np.float64) - (F // 2)
        ramp = np.exp(-2j * np.pi * kf[None, :] * delta[:, None])          # [B, F]
        Y = Y + np.sqrt(p_i)[:, None, None, None] * G * (z * ramp[:, None, :])[:, None]
    Y = Y + np.sqrt(sigma2 / 2.0)[:, None, None, None] * noise(seed, slots, N, T, F)
    return dict(Y=Y, bits=bits, H=H, x=x, noise_var=sigma2, interf_var=p_i, snr_db=snr_db,
                fd=fd, pilot_mask=mask, pilot_sym=psym)
