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


def oracle_llr_at(net, params64, Y32_slot, pilot_sym, pilot_mask, f):
    """Exact oracle LLRs of one slot at subcarrier f (all symbols), computed on the crop
    f - R .. f + R of the grid: positions farther than R from the crop edge see exactly
    the receptive field they see in the full grid."""
    from oracle import pipeline
    from workloads import replace
    R = receptive_radius(net)
    F = Y32_slot.shape[-2]
    lo, hi = max(0, f - R), min(F, f + R + 1)
    Yc = Y32_slot[None, :, :, lo:hi, 0].astype(np.float64) + 1j * Y32_slot[None, :, :, lo:hi, 1]
    L = pipeline.receive(replace(net, n_sc=hi - lo), params64, Yc, pilot_sym[:, lo:hi], pilot_mask[:, lo:hi])
    return L[0, :, f - lo, :]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def normwise(got, ref):
    """max |got - ref| / max |ref| (normwise infinity-norm relative error)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / (den if den > 0 else 1.0))
