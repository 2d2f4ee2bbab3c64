"""FP64 emulation of the CoNet forward pass with 16-bit (BF16 or FP16) convolution operands,
and of the gradient of a 16-bit training step.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU baseline use
this package; the library never calls it.

The 16-bit receivers keep every 3x3 conv input (the assembled grid for the input layer,
else the branch's activation entering the conv) and every conv weight as 16-bit floats and
accumulate the products in FP32; biases, LayerNorms, the Hadamard fusion, the residual
stream and the 1x1 head stay in FP32.  The emulation rounds exactly those operands to the
16-bit format and computes everything else in FP64, so it differs from the GPU only by the
GPU's FP32 rounding (and the rare 16-bit rounding decision that this flips).

A 16-bit training step (grad_16) also runs each body conv's data gradient on 16-bit operands
(the incoming gradient and the weights) and each conv's weight gradient on 16-bit operands
(the incoming gradient and the conv's input), accumulating in FP32; the emulation rounds the
same operands.

Formats (round to nearest, ties to even):
  * BF16: 8 significant bits (1 implicit + 7 stored), FP32's exponent range; in the binade
    [2^e, 2^(e+1)) the spacing is 2^(e-7).
  * FP16 (IEEE binary16): 11 significant bits, normal binades e >= -14, subnormal spacing
    2^-24, largest finite value 65504 (larger magnitudes round to infinity, as the GPU's
    conversion does).
"""
from __future__ import annotations

import numpy as np

from . import net as onet

FORMATS = {"bf16": dict(bits=8, emin=-126, max=None), "fp16": dict(bits=11, emin=-14, max=65504.0)}


def round16(x, fmt: str = "bf16"):
    """Round to the nearest value of the 16-bit format ``fmt`` (ties to even)."""
    f = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(np.where(a > 0, a, 1.0))          # a = m 2^e with m in [0.5, 1)
    e = np.maximum(e - 1, f["emin"])                    # binade [2^e, 2^(e+1)), clamped to the normal range
    quantum = np.ldexp(1.0, e - (f["bits"] - 1))
    r = np.round(a / quantum) * quantum                 # numpy rounds halves to even
    if f["max"] is not None:
        # beyond the largest finite value (by more than half a spacing) the conversion overflows
        r = np.where(a >= f["max"] + 0.5 * np.ldexp(1.0, 15 - (f["bits"] - 1)), np.inf, np.minimum(r, f["max"]))
    return np.copysign(r, x)


class Round16:
    """Quantisation hooks for oracle.net.forward: conv inputs and weights to a 16-bit format."""

    def __init__(self, fmt: str = "bf16"):
        self.fmt = fmt

    def act(self, x):
        return round16(x, self.fmt)

    def weight(self, w):
        return round16(w, self.fmt)


class Round16Train(Round16):
    """Hooks of a 16-bit training step (oracle.net.conv3x3_rounded): conv inputs, weights and
    the upstream gradients of every conv are rounded to the format, in the forward and in
    both gradients.  identity=True rounds nothing (for pins)."""

    def __init__(self, fmt: str = "bf16", identity: bool = False):
        super().__init__(fmt)
        self.identity = identity

    def act(self, x):
        return np.asarray(x, dtype=np.float64) if self.identity else super().act(x)

    def weight(self, w):
        return np.asarray(w, dtype=np.float64) if self.identity else super().weight(w)

    def grad(self, g):
        return np.asarray(g, dtype=np.float64) if self.identity else round16(g, self.fmt)


def grad_16(cfg, flat, X0, dllr, fmt: str = "bf16"):
    """Parameter gradient of a 16-bit training step for the upstream LLR gradient dllr:
    forward on 16-bit conv operands, data and weight gradients from 16-bit gradients, weights
    and inputs, everything else exact (FP64)."""
    _, tape = onet.forward(cfg, flat, X0, keep_tape=True, quant=Round16Train(fmt))
    g, _ = onet.backward(cfg, tape, dllr)
    return g


def forward_16(cfg, flat, X0, fmt: str = "bf16"):
    """LLR [B, T, F, Q] of the CoNet with 16-bit conv operands and exact arithmetic elsewhere."""
    return onet.forward(cfg, flat, X0, quant=Round16(fmt))
