"""FP64 oracle of the end-to-end steps: receive (input assembly -> CoNet -> LLR),
bit-error counting, and one training step (simulate -> forward -> BCE -> backward ->
Adam) on freshly simulated slots, the training set-up of the CoNet-Rx evaluation
(Sec. IV: the network is trained on simulated TDL slots)."""
from __future__ import annotations

import numpy as np

from . import net as onet
from . import rx as orx
from . import sim as osim


def receive(cfg, params, Y, pilot_sym, pilot_mask):
    X0 = orx.assemble_input(Y, pilot_sym, pilot_mask)
    return onet.forward(cfg, params, X0)


def receive_fp8(cfg, params, Y, pilot_sym, pilot_mask, margin: float = 2.0, scales=None):
    """receive() with E4M3 conv operands (oracle.fp8): scales calibrated on this batch, or
    the given ones (from calibrate_fp8 on another batch)."""
    from . import fp8
    X0 = orx.assemble_input(Y, pilot_sym, pilot_mask)
    return fp8.forward_fp8(cfg, params, X0, margin, scales)


def calibrate_fp8(cfg, params, Y, pilot_sym, pilot_mask, margin: float = 2.0):
    from . import fp8
    X0 = orx.assemble_input(Y, pilot_sym, pilot_mask)
    return fp8.calibrate_fp8(cfg, params, X0, margin)


def train_step(cfg, sim, params, m, v, step: int, seed: int, batch: int, lr: float):
    """Slots seed/(step*batch .. step*batch+batch-1); returns (params, m, v, loss)."""
    s = osim.simulate(cfg, sim, seed, step * batch, batch)
    X0 = orx.assemble_input(s["Y"], s["pilot_sym"], s["pilot_mask"])
    loss, g, _ = onet.loss_and_grad(cfg, params, X0, s["bits"], s["pilot_mask"])
    params, m, v = onet.adam_step(params, g, m, v, step + 1, lr)
    return params, m, v, loss


def ber(llr, bits, pilot_mask):
    e, n = orx.bit_errors(llr, bits, pilot_mask)
    return e / max(n, 1), e, n
