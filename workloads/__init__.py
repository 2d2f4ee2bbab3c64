"""Workload definitions and seeded input generators shared by the CUDA path and the oracle.

This module holds no arithmetic of the method: only the named network / link
configurations (shapes, ranges, seeds) and plain seeded random-number helpers.
Both the product package and ``oracle/`` may import it; neither imports the
other.

The five named workloads follow the network and link descriptions of the
CoNet-Rx paper (Sec. II system model, Sec. III architecture, Sec. IV set-up),
restated at the sizes this library is measured on.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field, replace

import numpy as np

# Pilot symbols never change from slot to slot (Sec. II-A: the pilots are fixed),
# so one library-wide pilot seed defines them.
DEFAULT_PILOT_SEED = 12739


@dataclass(frozen=True)
class NetConfig:
    """Shape of one CoNet receiver (Sec. III, Fig. "Example I").

    n_branches: 1 main net + (n_branches - 1) support nets (Sec. III, M support nets).
    depth: number of 3x3 conv layers (plain) or of residual blocks after the
        input layer (residual).
    residual: 0 = plain CNN branches; 1 = RB support branches and MRB main branch.
    norm: 1 = LayerNorm over channels after every fusion (and inside RB/MRB).
    fuse_mask: bit i set = Hadamard fusion after layer/block i (bit 0 = input layer).
    resnet_baseline: 1 = a single pre-activation ResNet branch, no fusion (the
        DeepRx-style comparison network).
    fuse_op: the interaction operation at a fusion point (Sec. III lists multiplication,
        addition and concatenation): 0 = element-wise product, 1 = element-wise sum, 2 =
        concatenation over channels (plain networks; the main's next layer and the head then
        read n_branches x width channels).
    feedback: 1 = Example II (Sec. III, Fig. "conet2"): at every fusion point each support
        net continues with its own activation plus the main net's (before the fusion).
    depthwise: 1 = the convs inside RB / MRB blocks are depthwise-separable: a per-channel
        3x3 conv followed by a 1x1 conv with bias (Sec. II-A, Sec. III).
    support_inputs: 1 = the support nets are fed only the pilot information (pilot mask and
        LS estimate at the pilots), not the received signal (Sec. III, selective inputs).
    support_mask: with support_inputs = 1, another subset: bit j = input channel j of the
        assembled grid is fed to the support nets (0 = the pilot information).
    """
    n_rx: int
    n_sc: int
    qam_bits: int
    n_branches: int
    depth: int
    width: int
    residual: int = 0
    norm: int = 0
    fuse_mask: int = -1
    resnet_baseline: int = 0
    fuse_op: int = 0
    feedback: int = 0
    depthwise: int = 0
    support_inputs: int = 0
    support_mask: int = 0
    n_sym: int = 14
    pilot_syms: tuple = (2, 11)
    pilot_comb: int = 2
    pilot_seed: int = DEFAULT_PILOT_SEED

    @property
    def c_in(self) -> int:
        # Re/Im of Y per antenna, pilot mask, Re/Im of the antenna-averaged LS estimate.
        return 2 * self.n_rx + 3

    def fused(self, i: int) -> bool:
        if self.resnet_baseline or self.n_branches < 2:
            return False
        return bool((self.fuse_mask >> i) & 1) if self.fuse_mask >= 0 else True


@dataclass(frozen=True)
class SimConfig:
    """Synthetic OFDM link (Sec. II, Eq. 1): TDL Rayleigh channel, AWGN, optional interferer."""
    scs_hz: float = 30e3
    n_taps: int = 6
    delay_spread_s: float = 100e-9
    fd_lo: float = 0.0
    fd_hi: float = 100.0
    snr_lo: float = 0.0
    snr_hi: float = 20.0
    interferer: int = 0
    sir_lo: float = 0.0
    sir_hi: float = 20.0
    iqam_bits: int = 6
    awgn: int = 0            # 1 = H == 1 (no fading), used by closed-form BER checks
    n_sinusoids: int = 16


@dataclass(frozen=True)
class Workload:
    name: str
    net: NetConfig
    sim: SimConfig
    batch: int
    precision: str           # "fp32" | "bf16" | "fp8"
    train: bool = False
    description: str = ""


_NET1 = NetConfig(n_rx=1, n_sc=72, qam_bits=4, n_branches=2, depth=4, width=32)
_SIM1 = SimConfig(n_taps=6, delay_spread_s=100e-9, fd_lo=0.0, fd_hi=100.0, snr_lo=0.0, snr_hi=20.0)

_NET2 = NetConfig(n_rx=2, n_sc=624, qam_bits=6, n_branches=3, depth=6, width=64, residual=1, norm=1)
_NET2_RESNET = replace(_NET2, n_branches=1, width=112, resnet_baseline=1)
_SIM2 = SimConfig(n_taps=12, delay_spread_s=300e-9, fd_lo=0.0, fd_hi=300.0, snr_lo=-5.0, snr_hi=25.0)

_SIM3 = replace(_SIM1, snr_lo=-5.0, snr_hi=25.0, fd_hi=400.0)

_NET4 = NetConfig(n_rx=4, n_sc=3276, qam_bits=8, n_branches=4, depth=8, width=96, residual=1, norm=1)
_SIM4 = replace(_SIM2, snr_lo=0.0, snr_hi=30.0)

_SIM5 = replace(_SIM3, interferer=1, sir_lo=0.0, sir_hi=20.0, iqam_bits=6)

# Depth comparison of Sec. IV (Fig. "InferenceD"): a CoNet of 14 sequential layers (input
# conv, 6 RB / MRB blocks of two convs, 1x1 head) against a single-branch pre-activation
# ResNet of 24 (input conv, 11 blocks, head), both near 1.9 M parameters, on the 14 x 624 link.
_NET_D14 = NetConfig(n_rx=2, n_sc=624, qam_bits=6, n_branches=4, depth=6, width=64, residual=1, norm=1)
_NET_D24 = NetConfig(n_rx=2, n_sc=624, qam_bits=6, n_branches=1, depth=11, width=96, residual=1, norm=1,
                     resnet_baseline=1)

WORKLOADS = {
    "plain_14x72_b16_fp32": Workload(
        "plain_14x72_b16_fp32", _NET1, _SIM1, 16, "fp32",
        description="1 Rx, 14x72 grid, 16-QAM, 2 branches x 4 conv3x3 x 32, Hadamard, 1x1 head"),
    "resid_14x624_b256_fp32": Workload(
        "resid_14x624_b256_fp32", _NET2, _SIM2, 256, "fp32",
        description="2 Rx, 14x624 grid, 64-QAM, 3 branches x (input + 6 RB/MRB) x 64, LN, Hadamard"),
    "resnet_14x624_b256_fp32": Workload(
        "resnet_14x624_b256_fp32", _NET2_RESNET, _SIM2, 256, "fp32",
        description="matched-FLOP single-branch pre-activation ResNet, width 112, 6 RB"),
    "train_14x72_b128_bf16": Workload(
        "train_14x72_b128_bf16", _NET1, _SIM3, 128, "bf16", train=True,
        description="training of the 14x72 plain CoNet on device-generated slots, BCE + Adam"),
    "resid_14x3276_b1024_bf16": Workload(
        "resid_14x3276_b1024_bf16", _NET4, _SIM4, 1024, "bf16",
        description="4 Rx, 14x3276 grid, 256-QAM, 4 branches x (input + 8 RB/MRB) x 96"),
    "interf_14x72_b512_fp8": Workload(
        "interf_14x72_b512_fp8", _NET1, _SIM5, 512, "fp8",
        description="14x72 plain CoNet with a co-channel 64-QAM interferer, SIR U(0,20) dB"),
    "conet_d14_14x624_bf16": Workload(
        "conet_d14_14x624_bf16", _NET_D14, _SIM2, 256, "bf16",
        description="14-layer CoNet, 4 branches x (input + 6 RB/MRB) x 64, 1.78 M parameters"),
    "resnet_d24_14x624_bf16": Workload(
        "resnet_d24_14x624_bf16", _NET_D24, _SIM2, 256, "bf16",
        description="24-layer pre-activation ResNet, 1 branch x (input + 11 RB) x 96, 1.83 M parameters"),
    "resid_dw_14x624_b256_bf16": Workload(
        "resid_dw_14x624_b256_bf16", replace(_NET2, depthwise=1), _SIM2, 256, "bf16",
        description="the 14x624 residual CoNet with depthwise-separable block convs (per-channel 3x3 + 1x1)"),
}


def tiny_net(**kw) -> NetConfig:
    """Small network shapes for brute-force and finite-difference checks."""
    base = dict(n_rx=1, n_sc=6, qam_bits=2, n_branches=2, depth=2, width=3, n_sym=4,
                pilot_syms=(1, 2))
    base.update(kw)
    return NetConfig(**base)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_grid(seed: int, shape, scale: float = 1.0, dtype=np.float32) -> np.ndarray:
    """Seeded standard-normal tensor (used as a stand-in received grid or gradient)."""
    return (rng(seed).standard_normal(shape) * scale).astype(dtype)


def random_bits(seed: int, shape) -> np.ndarray:
    return rng(seed).integers(0, 2, size=shape, dtype=np.uint8)


def asdict(x) -> dict:
    return dataclasses.asdict(x)
