"""Thin Python binding of libconet with the C ABI's names.

torch provides the device memory and the stream; every step of the path runs in the
library's kernels.  Tensors passed in must be contiguous CUDA tensors of the dtype and
layout given in include/conet.h.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from ._lib import check, conet_config, conet_sim_params, lib

PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3, "tf32x3": 4}


def make_config(net, max_batch: int = 1, train: bool = False, recompute: bool = False) -> conet_config:
    c = conet_config()
    c.n_rx, c.n_sym, c.n_sc, c.qam_bits = net.n_rx, net.n_sym, net.n_sc, net.qam_bits
    c.n_branches, c.depth, c.width = net.n_branches, net.depth, net.width
    c.residual, c.norm, c.fuse_mask, c.resnet_baseline = net.residual, net.norm, net.fuse_mask, net.resnet_baseline
    c.max_batch, c.train = int(max_batch), int(bool(train))
    ps = list(net.pilot_syms)
    for i in range(4):
        c.pilot_syms[i] = ps[i] if i < len(ps) else -1
    c.n_pilot_syms, c.pilot_comb, c.pilot_seed = len(ps), net.pilot_comb, net.pilot_seed
    c.recompute = int(bool(recompute))
    c.fuse_op = int(getattr(net, "fuse_op", 0))
    c.feedback = int(getattr(net, "feedback", 0))
    c.depthwise = int(getattr(net, "depthwise", 0))
    c.support_inputs = int(getattr(net, "support_inputs", 0))
    c.support_mask = int(getattr(net, "support_mask", 0))
    return c


def make_sim(sim) -> conet_sim_params:
    s = conet_sim_params()
    s.scs_hz, s.n_taps, s.delay_spread_s = sim.scs_hz, sim.n_taps, sim.delay_spread_s
    s.fd_lo, s.fd_hi, s.snr_lo, s.snr_hi = sim.fd_lo, sim.fd_hi, sim.snr_lo, sim.snr_hi
    s.interferer, s.sir_lo, s.sir_hi, s.iqam_bits = sim.interferer, sim.sir_lo, sim.sir_hi, sim.iqam_bits
    s.awgn, s.n_sinusoids = sim.awgn, sim.n_sinusoids
    return s


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def param_count(net) -> int:
    n = C.c_size_t()
    check(lib().conet_param_count(C.byref(make_config(net)), C.byref(n)))
    return n.value


class _DevView:
    """__cuda_array_interface__ wrapper that lets torch alias a library-owned buffer."""

    def __init__(self, ptr, n, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None, "stream": None}
        self._owner = owner


class Receiver:
    """A CoNet receiver handle (conet_create ... conet_destroy)."""

    def __init__(self, net, precision: str = "fp32", max_batch: int = 1, train: bool = False,
                 recompute: bool = False):
        self.net = net
        self.precision = precision
        self.cfg = make_config(net, max_batch, train, recompute)
        h = C.c_void_p()
        check(lib().conet_create(C.byref(self.cfg), PRECISIONS[precision], C.byref(h)))
        self.h = h
        self.n_params = param_count(net)

    def close(self):
        if getattr(self, "h", None):
            lib().conet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_he(self, seed: int, stream=None):
        check(lib().conet_init_he(self.h, seed, _stream(stream)))

    def load_weights(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(lib().conet_load_weights(self.h, p.ctypes.data_as(C.c_void_p), p.size))

    def save_weights(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        check(lib().conet_save_weights(self.h, out.ctypes.data_as(C.c_void_p), out.size))
        return out

    def save_checkpoint(self, adam_step: int) -> bytes:
        """Versioned checkpoint: parameters, Adam moments and the Adam step to resume at."""
        n = C.c_size_t()
        check(lib().conet_checkpoint_bytes(self.h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        check(lib().conet_save_checkpoint(self.h, int(adam_step), C.cast(buf, C.c_void_p), n.value))
        return buf.raw

    def load_checkpoint(self, blob: bytes) -> int:
        """Restore a checkpoint; returns the Adam step it recorded."""
        step = C.c_uint64()
        buf = C.create_string_buffer(bytes(blob), len(blob))
        check(lib().conet_load_checkpoint(self.h, C.cast(buf, C.c_void_p), len(blob), C.byref(step)))
        return step.value

    def selftest_timeout(self, limit_s: float = 1e-3, stream=None):
        """Launch the failure-detection self-test (a bounded wait that gives up)."""
        check(lib().conet_selftest_timeout(self.h, float(limit_s), _stream(stream)))

    def params_device(self) -> torch.Tensor:
        p, n = C.c_void_p(), C.c_size_t()
        check(lib().conet_params_device(self.h, C.byref(p), C.byref(n)))
        return torch.as_tensor(_DevView(p.value, n.value, self), device="cuda")

    def grads_device(self) -> torch.Tensor:
        p, n = C.c_void_p(), C.c_size_t()
        check(lib().conet_grads_device(self.h, C.byref(p), C.byref(n)))
        return torch.as_tensor(_DevView(p.value, n.value, self), device="cuda")

    def params_updated(self, stream=None):
        """Re-derive the kernels' weight layouts after an in-place change of params_device()."""
        check(lib().conet_params_updated(self.h, _stream(stream)))

    def forward(self, Y, pilot_mask, noise_var=None, llr=None, stream=None) -> torch.Tensor:
        B = Y.shape[0]
        if llr is None:
            llr = torch.empty((B, self.net.n_sym, self.net.n_sc, self.net.qam_bits), device=Y.device,
                              dtype=torch.float32)
        check(lib().conet_forward(self.h, _ptr(Y), _ptr(pilot_mask), _ptr(noise_var), B, _ptr(llr),
                                  _stream(stream)))
        return llr

    def whole_network(self, mode=True) -> bool:
        """Single-kernel path for small plain BF16 / E4M3 networks: True or "always" runs
        every forward through it, "auto" (the default) forward calls of at least
        CONET_WHOLE_NET_MIN_SLOTS slots, False never.  Returns whether this handle's network
        qualifies for it."""
        m = {False: 0, True: 2, "never": 0, "auto": 1, "always": 2}[mode]
        avail = C.c_int()
        check(lib().conet_whole_network(self.h, m, C.byref(avail)))
        return bool(avail.value)

    def graphs(self, enable: bool = True):
        """CUDA-graph replay of repeated identical forward calls (on by default)."""
        check(lib().conet_graphs(self.h, int(bool(enable))))

    def calibrate(self, Y, pilot_mask, margin: float = 2.0, stream=None):
        """E4M3 activation scales from these slots (no-op for other precisions)."""
        check(lib().conet_calibrate(self.h, _ptr(Y), _ptr(pilot_mask), Y.shape[0], margin, _stream(stream)))

    def backward(self, dllr, stream=None):
        check(lib().conet_backward(self.h, _ptr(dllr), dllr.shape[0], _stream(stream)))

    def adam_step(self, lr: float, step: int, stream=None):
        check(lib().conet_adam_step(self.h, lr, step, _stream(stream)))

    def sync(self, stream=None):
        """Wait for the stream; raise on a device-side timeout or CUDA error."""
        check(lib().conet_sync(self.h, _stream(stream)))

    def profile_enable(self, enable: bool = True):
        check(lib().conet_profile_enable(self.h, int(bool(enable))))

    def profile_read(self, kind: int):
        """(summed milliseconds, launches) of one kernel kind since profile_enable."""
        ms, n = C.c_double(), C.c_longlong()
        check(lib().conet_profile_read(self.h, kind, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def train_step(self, sim, seed: int, step: int, B: int, lr: float, want_loss=True, stream=None):
        loss = C.c_double()
        check(lib().conet_train_step(self.h, C.byref(make_sim(sim)), seed, step, B, lr,
                                     C.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None


class CoNetFn(torch.autograd.Function):
    """LLRs = CoNet(Y) as an autograd node over the flat master parameters.

    ``params`` must be the handle's own parameter buffer (``Receiver.params_device()``, as
    ``CoNet.weight`` holds it): the forward reads the weights from the library, not from the
    tensor.  Forward saves only the handle (the library keeps the activations); backward
    runs conet_backward on the incoming LLR gradient and returns a copy of the library's
    parameter gradient.  There is no gradient with respect to Y or the pilot mask."""

    @staticmethod
    def forward(ctx, params, rx, Y, pilot_mask):
        ctx.rx = rx
        return rx.forward(Y, pilot_mask)

    @staticmethod
    def backward(ctx, dllr):
        ctx.rx.backward(dllr.contiguous())
        return ctx.rx.grads_device().clone(), None, None, None


class CoNet(torch.nn.Module):
    """A trainable CoNet receiver: ``weight`` is an nn.Parameter aliasing the library's FP32
    master parameters, so ``loss.backward()`` fills ``weight.grad`` through CoNetFn.  Update
    the weights with ``adam_step`` (the library's Adam), or change ``weight`` in place with a
    torch optimiser and then call ``params_updated()``."""

    def __init__(self, net, precision: str = "fp32", max_batch: int = 1, seed: int = 0):
        super().__init__()
        self.rx = Receiver(net, precision=precision, max_batch=max_batch, train=True)
        self.rx.init_he(seed)
        self.weight = torch.nn.Parameter(self.rx.params_device(), requires_grad=True)

    def forward(self, Y, pilot_mask):
        return CoNetFn.apply(self.weight, self.rx, Y, pilot_mask)

    def adam_step(self, lr: float, step: int):
        self.rx.adam_step(lr, step)

    def params_updated(self):
        self.rx.params_updated()


def pilots(net, device="cuda", stream=None):
    mask = torch.empty((net.n_sym, net.n_sc), dtype=torch.uint8, device=device)
    psym = torch.empty((net.n_sym, net.n_sc, 2), dtype=torch.float32, device=device)
    check(lib().conet_pilots(C.byref(make_config(net)), _ptr(mask), _ptr(psym), _stream(stream)))
    return mask, psym


def sim_generate(net, sim, seed: int, slot0: int, B: int, fixed_snr_db=None, want_H=False,
                 want_interf=False, device="cuda", stream=None):
    T, F, N, Q = net.n_sym, net.n_sc, net.n_rx, net.qam_bits
    Y = torch.empty((B, N, T, F, 2), dtype=torch.float32, device=device)
    bits = torch.empty((B, T, F, Q), dtype=torch.uint8, device=device)
    H = torch.empty_like(Y) if want_H else None
    nv = torch.empty(B, dtype=torch.float32, device=device)
    iv = torch.empty(B, dtype=torch.float32, device=device) if want_interf else None
    snr = float("nan") if fixed_snr_db is None else float(fixed_snr_db)
    check(lib().conet_sim_generate(C.byref(make_config(net)), C.byref(make_sim(sim)), seed, slot0, B, snr,
                                   _ptr(Y), _ptr(bits), _ptr(H), _ptr(nv), _ptr(iv), _stream(stream)))
    return dict(Y=Y, bits=bits, H=H, noise_var=nv, interf_var=iv)


def assemble_input(net, Y, pilot_mask, pilot_sym, stream=None):
    B = Y.shape[0]
    X0 = torch.empty((B, net.n_sym, net.n_sc, net.c_in), dtype=torch.float32, device=Y.device)
    check(lib().conet_assemble_input(C.byref(make_config(net)), _ptr(Y), _ptr(pilot_mask), _ptr(pilot_sym), B,
                                     _ptr(X0), _stream(stream)))
    return X0


def ls_lmmse(net, Y, pilot_mask, pilot_sym, noise_var, interf_var=None, H_perfect=None, exact=True, stream=None):
    B = Y.shape[0]
    llr = torch.empty((B, net.n_sym, net.n_sc, net.qam_bits), dtype=torch.float32, device=Y.device)
    check(lib().conet_ls_lmmse(C.byref(make_config(net)), _ptr(Y), _ptr(pilot_mask), _ptr(pilot_sym),
                               _ptr(noise_var), _ptr(interf_var), _ptr(H_perfect), int(bool(exact)), B,
                               _ptr(llr), _stream(stream)))
    return llr


def loss_ber(llr, bits, pilot_mask, grad_scale: float = 0.0, want_grad=False, stream=None):
    B, T, F, Q = llr.shape
    dev = llr.device
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    dllr = torch.empty_like(llr) if want_grad else None
    check(lib().conet_loss_ber(_ptr(llr), _ptr(bits), _ptr(pilot_mask), B, T, F, Q, grad_scale, _ptr(dllr),
                               _ptr(loss), C.c_void_p(cnt.data_ptr()), C.c_void_p(cnt.data_ptr() + 8),
                               _stream(stream)))
    return loss, cnt, dllr


def ber_count(llr, bits, pilot_mask, stream=None) -> torch.Tensor:
    """Hard-decision bit errors and bits counted over the data REs: int64 [2] on the device."""
    B, T, F, Q = llr.shape
    cnt = torch.zeros(2, dtype=torch.int64, device=llr.device)
    check(lib().conet_ber_count(_ptr(llr), _ptr(bits), _ptr(pilot_mask), B, T, F, Q, C.c_void_p(cnt.data_ptr()),
                                C.c_void_p(cnt.data_ptr() + 8), _stream(stream)))
    return cnt


def conv3x3_wgrad(x, dz, want_bias=True, stream=None):
    """(dW [Cout][3][3][Cin], db [Cout]) of one 3x3 'same' conv: x [B,T,F,Cin], dz [B,T,F,Cout]."""
    B, T, F, cin = x.shape
    cout = dz.shape[-1]
    dW = torch.empty((cout, 3, 3, cin), dtype=torch.float32, device=x.device)
    db = torch.empty(cout, dtype=torch.float32, device=x.device) if want_bias else None
    check(lib().conet_conv3x3_wgrad(_ptr(x), _ptr(dz), B, T, F, cin, cout, _ptr(dW), _ptr(db), _stream(stream)))
    return dW, db


def checkpoint_hash(net) -> int:
    """The checkpoint header's hash of a network description."""
    h = C.c_uint64()
    check(lib().conet_checkpoint_hash(C.byref(make_config(net)), C.byref(h)))
    return h.value


def launch_count() -> int:
    return int(lib().conet_launch_count())


PROFILE_KINDS = {"conv": 0, "conv_in": 1, "fuse": 2, "assemble": 3, "backward": 4, "adam": 5}
# conet.h's CONET_WHOLE_NET_MIN_SLOTS: in automatic mode, forward calls of at least this many
# slots run the whole-network kernel
WHOLE_NET_MIN_SLOTS = 1
