"""ctypes declarations of libconet's C ABI (include/conet.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libconet.so")


class ConetError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libconet error {code}: {msg}")
        self.code = code


class conet_config(C.Structure):
    _fields_ = [("n_rx", C.c_int), ("n_sym", C.c_int), ("n_sc", C.c_int), ("qam_bits", C.c_int),
                ("n_branches", C.c_int), ("depth", C.c_int), ("width", C.c_int),
                ("residual", C.c_int), ("norm", C.c_int), ("fuse_mask", C.c_int), ("resnet_baseline", C.c_int),
                ("max_batch", C.c_int), ("train", C.c_int),
                ("pilot_syms", C.c_int * 4), ("n_pilot_syms", C.c_int), ("pilot_comb", C.c_int),
                ("pilot_seed", C.c_uint64), ("recompute", C.c_int), ("fuse_op", C.c_int), ("feedback", C.c_int),
                ("depthwise", C.c_int), ("support_inputs", C.c_int), ("support_mask", C.c_uint)]


class conet_sim_params(C.Structure):
    _fields_ = [("scs_hz", C.c_float), ("n_taps", C.c_int), ("delay_spread_s", C.c_float),
                ("fd_lo", C.c_float), ("fd_hi", C.c_float), ("snr_lo", C.c_float), ("snr_hi", C.c_float),
                ("interferer", C.c_int), ("sir_lo", C.c_float), ("sir_hi", C.c_float), ("iqam_bits", C.c_int),
                ("awgn", C.c_int), ("n_sinusoids", C.c_int)]


P = C.c_void_p
I = C.c_int
SZ = C.c_size_t
U64 = C.c_uint64
F32 = C.c_float
CFG = C.POINTER(conet_config)
SIM = C.POINTER(conet_sim_params)

SIGNATURES = {
    "conet_param_count": (I, [CFG, C.POINTER(SZ)]),
    "conet_create": (I, [CFG, I, C.POINTER(P)]),
    "conet_destroy": (None, [P]),
    "conet_init_he": (I, [P, U64, P]),
    "conet_load_weights": (I, [P, P, SZ]),
    "conet_save_weights": (I, [P, P, SZ]),
    "conet_checkpoint_hash": (I, [CFG, C.POINTER(U64)]),
    "conet_checkpoint_bytes": (I, [P, C.POINTER(SZ)]),
    "conet_save_checkpoint": (I, [P, U64, P, SZ]),
    "conet_load_checkpoint": (I, [P, P, SZ, C.POINTER(U64)]),
    "conet_params_device": (I, [P, C.POINTER(P), C.POINTER(SZ)]),
    "conet_grads_device": (I, [P, C.POINTER(P), C.POINTER(SZ)]),
    "conet_params_updated": (I, [P, P]),
    "conet_forward": (I, [P, P, P, P, I, P, P]),
    "conet_graphs": (I, [P, I]),
    "conet_whole_network": (I, [P, I, C.POINTER(I)]),
    "conet_calibrate": (I, [P, P, P, I, F32, P]),
    "conet_backward": (I, [P, P, I, P]),
    "conet_adam_step": (I, [P, F32, I, P]),
    "conet_conv3x3_wgrad": (I, [P, P, I, I, I, I, I, P, P, P]),
    "conet_conv3x3_wgrad_noalloc": (I, [P, P, I, I, I, I, I, P, P, P]),
    "conet_train_step": (I, [P, SIM, U64, U64, I, F32, C.POINTER(C.c_double), P]),
    "conet_pilots": (I, [CFG, P, P, P]),
    "conet_sim_generate": (I, [CFG, SIM, U64, U64, I, F32, P, P, P, P, P, P]),
    "conet_assemble_input": (I, [CFG, P, P, P, I, P, P]),
    "conet_ls_lmmse": (I, [CFG, P, P, P, P, P, P, I, I, P, P]),
    "conet_loss_ber": (I, [P, P, P, I, I, I, I, F32, P, P, P, P, P]),
    "conet_ber_count": (I, [P, P, P, I, I, I, I, P, P, P]),
    "conet_profile_enable": (I, [P, I]),
    "conet_profile_read": (I, [P, I, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "conet_launch_count": (C.c_ulonglong, []),
    "conet_sync": (I, [P, P]),
    "conet_selftest_timeout": (I, [P, C.c_double, P]),
    "conet_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libconet.so (built in-tree by ``paper_2510_12739_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libconet.so is not built ({LIB_PATH}); run python -m paper_2510_12739_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != 0:
        raise ConetError(rc, lib().conet_last_error().decode())
