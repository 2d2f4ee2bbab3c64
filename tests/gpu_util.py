"""Helpers shared by the GPU parity tests: oracle-side inputs as float32 arrays and the
normwise error measure used by every floating-point comparison."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_12739_gb300 import api  # noqa: F401  (fails loudly when libconet is missing)


def cplx_to_f32(z):
    return np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1).astype(np.float32))


def oracle_inputs(net, sim, seed, slot0, B, **kw):
    """Slots simulated by the oracle (float64), plus their float32 interleaved copies."""
    from oracle import sim as osim
    s = osim.simulate(net, sim, seed, slot0, B, **kw)
    s["Y32"] = cplx_to_f32(s["Y"])
    s["H32"] = cplx_to_f32(s["H"])
    return s


def receptive_radius(net):
    """Subcarriers on each side that one output RE depends on (one per 3x3 conv)."""
    return 1 + (2 * net.depth if net.residual else net.depth - 1)


def oracle_llr_at(net, params64, Y32_slot, pilot_sym, pilot_mask, f, fmt=None):
    """Exact oracle LLRs of one slot at subcarrier f (all symbols), computed on the crop
    f - R .. f + R of the grid: positions farther than R from the crop edge see exactly
    the receptive field they see in the full grid.  fmt = "bf16" / "fp16": the oracle's
    emulation of that 16-bit receiver instead of the FP64 network."""
    from oracle import half, net as onet, rx as orx
    from workloads import replace
    R = receptive_radius(net)
    F = Y32_slot.shape[-2]
    lo, hi = max(0, f - R), min(F, f + R + 1)
    Yc = Y32_slot[None, :, :, lo:hi, 0].astype(np.float64) + 1j * Y32_slot[None, :, :, lo:hi, 1]
    crop = replace(net, n_sc=hi - lo)
    X0 = orx.assemble_input(Yc, pilot_sym[:, lo:hi], pilot_mask[:, lo:hi])
    L = half.forward_16(crop, params64, X0, fmt) if fmt else onet.forward(crop, params64, X0)
    return L[0, :, f - lo, :]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def normwise(got, ref):
    """max |got - ref| / max |ref| (normwise infinity-norm relative error)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / (den if den > 0 else 1.0))


def ill_conditioned_res(net, taps, k=100.0, eps=1e-5):
    """REs whose LLRs depend on a LayerNorm of a nearly constant fused product.

    A LayerNorm after a Hadamard fusion divides by sqrt(var + eps); where the product's
    variance over channels is below k eps it multiplies absolute rounding differences by up
    to 1 / sqrt(eps) ~ 316 instead of at most 1 / sqrt((k + 1) eps).  From the oracle's
    per-RE fused variances (oracle.net.forward's taps), flag those REs at every fusion point
    and grow the flags by one RE on both grid axes (the 3 x 3 neighbourhood) for every
    main-branch 3x3 conv that follows that point: the receptive field through which the
    difference reaches the LLRs.  Returns a boolean [B, T, F]."""
    out = None
    for i, var in taps.items():
        flag = var < k * eps
        convs_after = 2 * (net.depth - i) if net.residual else (net.depth - 1 - i)
        for _ in range(convs_after):
            p = np.pad(flag, ((0, 0), (1, 1), (1, 1)))
            T, F = flag.shape[1], flag.shape[2]
            flag = np.zeros_like(flag)
            for dt in range(3):
                for df in range(3):
                    flag |= p[:, dt:dt + T, df:df + F]
        out = flag if out is None else (out | flag)
    if out is None:
        raise ValueError("the network has no LayerNorm after a fusion")
    return out
