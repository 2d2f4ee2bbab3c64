"""FP64 emulation of the CoNet forward pass with FP8 E4M3 convolution operands.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU baseline use
this package; the library never calls it.

E4M3 (OCP 8-bit floating point, the "FN" variant): 1 sign bit, 4 exponent bits with
bias 7, 3 mantissa bits; normal values (1 + m/8) 2^(e-7) for e = 1..15 except the
all-ones pattern S.1111.111 (NaN), subnormals (m/8) 2^-6; no infinities.  The largest
finite value is 1.75 x 2^8 = 448, the smallest subnormal 2^-9.  Conversion here rounds to
nearest with ties to even and saturates to +-448 (the "satfinite" conversion).

Quantised network (the precision recipe of the FP8 receiver: E4M3 convolutions with one
scale per output channel for the weights and one per tensor for the activations, FP32
accumulation, everything else in full precision):
  * every 3x3 conv input x (the assembled grid for the input layer, else the branch's
    activation entering the conv) becomes s_x e4m3(x / s_x), s_x = pow2_scale(margin
    max|x|) with the maximum over the whole tensor (all slots of the batch);
  * every conv weight row W[co] becomes s_co e4m3(W[co] / s_co), s_co =
    pow2_scale(max |W[co]|);
  * biases, LayerNorms, the Hadamard fusion, the residual stream and the 1x1 head stay
    unquantised, and so does the last conv's output (it feeds the head).
Scales are powers of two (reading F1), so scaling and unscaling are exact.
"""
from __future__ import annotations

import numpy as np

from . import net as onet

E4M3_MAX = 448.0
E4M3_MIN_NORMAL = 2.0 ** -6
E4M3_MIN_SUBNORMAL = 2.0 ** -9


def e4m3_round(x):
    """Round to the nearest E4M3 value (ties to even), saturating to +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    # exponent of the binade [2^e, 2^(e+1)) holding |x|; below the normal range the
    # spacing is that of the subnormals, 2^-9 = 2^(-6-3)
    _, e = np.frexp(np.where(a > 0, a, 1.0))          # a = m 2^e, m in [0.5, 1)
    e = np.maximum(e - 1, -6)
    quantum = np.ldexp(1.0, e - 3)
    r = np.round(a / quantum) * quantum                # numpy rounds halves to even
    r = np.minimum(r, E4M3_MAX)
    return np.copysign(r, x)


def e4m3_values():
    """All finite non-negative E4M3 values, from the bit patterns."""
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue                               # NaN
            vals.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(sorted(set(vals)))


def pow2_scale(t):
    """Smallest power of two s with t / s <= 448 (1 for t == 0): t = m 2^e with m in
    [0.5, 1) and 448 = 0.875 x 2^9, so s = 2^(e - 9) when m <= 0.875, else 2^(e - 8)."""
    t = float(t)
    if t <= 0.0:
        return 1.0
    m, e = np.frexp(t)
    return float(np.ldexp(1.0, e - 9 if m <= 0.875 else e - 8))


def quantize(x, s):
    return s * e4m3_round(np.asarray(x, dtype=np.float64) / s)


def quantize_weight(w):
    """Per-output-channel E4M3 of a [Cout][3][3][Cin] conv weight."""
    w = np.asarray(w, dtype=np.float64)
    out = np.empty_like(w)
    for co in range(w.shape[0]):
        out[co] = quantize(w[co], pow2_scale(np.max(np.abs(w[co]))))
    return out


class E4M3Quant:
    """Quantisation hooks for oracle.net.forward (conv inputs and conv weights).

    Activation scales are calibrated on the tensor each hook call sees (the whole batch),
    or, with ``scales``, taken in call order from a list recorded by an earlier calibration
    (``used`` records the scales of this pass, in the forward's conv order)."""

    def __init__(self, margin: float = 2.0, scales=None):
        self.margin = float(margin)
        self.scales = None if scales is None else list(scales)
        self.used = []

    def act(self, x):
        if self.scales is not None:
            s = self.scales[len(self.used)]
        else:
            s = pow2_scale(self.margin * np.max(np.abs(x)))
        self.used.append(s)
        return quantize(x, s)

    def weight(self, w):
        return quantize_weight(w)


def forward_fp8(cfg, flat, X0, margin: float = 2.0, scales=None):
    """LLR [B, T, F, Q] of the CoNet with E4M3 conv operands: activation scales calibrated on
    X0's batch, or the given ones (as calibrate_fp8 returns them)."""
    return onet.forward(cfg, flat, X0, quant=E4M3Quant(margin, scales))


def calibrate_fp8(cfg, flat, X0, margin: float = 2.0):
    """Activation scales of every conv input, in forward order, calibrated on X0's batch."""
    q = E4M3Quant(margin)
    onet.forward(cfg, flat, X0, quant=q)
    return q.used
