"""GPU parity of the link simulator, pilot grid, input assembly, LS-LMMSE receiver and the
loss / bit-error counter against the FP64 oracle (called through the C ABI).

Tolerances: bits, masks and counts bit-exact; float32 results within a normwise
relative error derived from float32 rounding (2^-24 ~ 6e-8 per operation over at most a
few hundred accumulated terms, so 2e-5 leaves two decades of headroom)."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, oracle_inputs, torch
from workloads import WORKLOADS, SimConfig, replace

pytestmark = pytest.mark.gpu
SIM_TOL = 2e-5


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_pilot_grid_bit_exact(name):
    from oracle import sim as osim
    from paper_2510_12739_gb300 import api
    net = WORKLOADS[name].net
    mask, psym = api.pilots(net)
    m_ref, p_ref = osim.pilot_grid(net.n_sym, net.n_sc, net.pilot_syms, net.pilot_comb, net.pilot_seed)
    assert np.array_equal(mask.cpu().numpy(), m_ref)
    p = psym.cpu().numpy()
    assert np.array_equal(p[..., 0], p_ref.real.astype(np.float32))
    assert np.array_equal(p[..., 1], p_ref.imag.astype(np.float32))


SIM_CASES = [
    ("plain_14x72_b16_fp32", 4, {}),
    ("resid_14x624_b256_fp32", 2, {}),
    ("train_14x72_b128_bf16", 6, {}),
    ("interf_14x72_b512_fp8", 4, {}),
    ("resid_14x3276_b1024_bf16", 1, {}),
    ("plain_14x72_b16_fp32", 3, dict(awgn=1)),
    ("plain_14x72_b16_fp32", 3, dict(snr_lo=float("inf"), snr_hi=float("inf"))),
    ("plain_14x72_b16_fp32", 2, dict(n_taps=1, delay_spread_s=0.0)),
]


@pytest.mark.parametrize("name,B,over", SIM_CASES)
def test_simulator_matches_oracle(name, B, over):
    from paper_2510_12739_gb300 import api
    w = WORKLOADS[name]
    sim = replace(w.sim, **over)
    slot0 = 12345
    g = api.sim_generate(w.net, sim, 77, slot0, B, want_H=True, want_interf=True)
    ref = oracle_inputs(w.net, sim, 77, slot0, B)
    assert np.array_equal(g["bits"].cpu().numpy(), ref["bits"])
    assert np.allclose(g["noise_var"].cpu().numpy(), ref["noise_var"], rtol=1e-6, atol=0)
    assert np.allclose(g["interf_var"].cpu().numpy(), ref["interf_var"], rtol=1e-6, atol=0)
    Y = g["Y"].cpu().numpy()
    H = g["H"].cpu().numpy()
    for b in range(B):
        assert normwise(Y[b], ref["Y32"][b]) < SIM_TOL, b
        assert normwise(H[b], ref["H32"][b]) < SIM_TOL, b


def test_simulator_fixed_snr_and_large_slot_ids():
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["resid_14x624_b256_fp32"]
    g = api.sim_generate(w.net, w.sim, 3, 2**32 - 2, 2, fixed_snr_db=7.5)
    ref = oracle_inputs(w.net, w.sim, 3, 2**32 - 2, 2, fixed_snr_db=7.5)
    assert np.array_equal(g["bits"].cpu().numpy(), ref["bits"])
    assert np.allclose(g["noise_var"].cpu().numpy(), 10 ** -0.75, rtol=1e-6)
    for b in range(2):
        assert normwise(g["Y"].cpu().numpy()[b], ref["Y32"][b]) < SIM_TOL


@pytest.mark.parametrize("name", ["plain_14x72_b16_fp32", "resid_14x624_b256_fp32", "resid_14x3276_b1024_bf16"])
def test_input_assembly_matches_oracle(name):
    from oracle import rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS[name]
    ref = oracle_inputs(w.net, w.sim, 5, 0, 2)
    Y32 = ref["Y32"]
    X = api.assemble_input(w.net, dev(Y32), dev(ref["pilot_mask"]),
                           dev(np.stack([ref["pilot_sym"].real, ref["pilot_sym"].imag], -1).astype(np.float32)))
    Yd = Y32[..., 0].astype(np.float64) + 1j * Y32[..., 1]
    X_ref = orx.assemble_input(Yd, ref["pilot_sym"], ref["pilot_mask"])
    assert X.shape[-1] == w.net.c_in
    assert normwise(X.cpu().numpy(), X_ref) < 1e-6


def _psym32(p):
    return np.stack([p.real, p.imag], -1).astype(np.float32)


@pytest.mark.parametrize("name,exact,perfect", [("plain_14x72_b16_fp32", True, False),
                                                ("plain_14x72_b16_fp32", False, False),
                                                ("resid_14x624_b256_fp32", True, False),
                                                ("resid_14x624_b256_fp32", True, True),
                                                ("interf_14x72_b512_fp8", True, False),
                                                ("resid_14x3276_b1024_bf16", False, True)])
def test_ls_lmmse_matches_oracle(name, exact, perfect):
    from oracle import rx as orx
    from paper_2510_12739_gb300 import api
    w = WORKLOADS[name]
    ref = oracle_inputs(w.net, w.sim, 8, 40, 2)
    Yd = ref["Y32"][..., 0].astype(np.float64) + 1j * ref["Y32"][..., 1]
    Hd = ref["H32"][..., 0].astype(np.float64) + 1j * ref["H32"][..., 1]
    nv = ref["noise_var"].astype(np.float32)
    iv = ref["interf_var"].astype(np.float32) if w.sim.interferer else None
    llr = api.ls_lmmse(w.net, dev(ref["Y32"]), dev(ref["pilot_mask"]), dev(_psym32(ref["pilot_sym"])), dev(nv),
                       dev(iv) if iv is not None else None, dev(ref["H32"]) if perfect else None, exact=exact)
    L_ref = orx.ls_lmmse(Yd, nv.astype(np.float64), ref["pilot_sym"], ref["pilot_mask"], w.net.pilot_syms,
                         w.net.qam_bits, interf_var=None if iv is None else iv.astype(np.float64),
                         H_perfect=Hd if perfect else None, exact=exact)
    L = llr.cpu().numpy()
    assert normwise(L, L_ref) < 1e-4
    # hard decisions agree except where the reference LLR is within rounding of 0
    amb = np.abs(L_ref) <= 1e-4 * np.max(np.abs(L_ref))
    assert np.all(((L > 0) == (L_ref > 0)) | amb)


def test_loss_and_bit_errors_match_oracle():
    from oracle import net as onet, rx as orx
    from paper_2510_12739_gb300 import api
    from workloads import random_bits, random_grid
    w = WORKLOADS["train_14x72_b128_bf16"]
    ref = oracle_inputs(w.net, w.sim, 2, 0, 1)
    B, T, F, Q = 37, 14, 72, 4
    llr = random_grid(11, (B, T, F, Q), scale=3.0)
    bits = random_bits(12, (B, T, F, Q))
    mask = ref["pilot_mask"]
    bits[:, mask.astype(bool)] = 0
    loss, cnt, dllr = api.loss_ber(dev(llr), dev(bits), dev(mask), grad_scale=0.25, want_grad=True)
    e_ref, n_ref = orx.bit_errors(llr.astype(np.float64), bits, mask)
    assert int(cnt[0]) == e_ref and int(cnt[1]) == n_ref
    l_ref, d_ref = onet.bce_loss(llr.astype(np.float64), bits, mask)
    assert abs(loss.item() / n_ref - l_ref) < 1e-6 * l_ref
    assert normwise(dllr.cpu().numpy(), d_ref * n_ref * 0.25) < 1e-6
    # the counting-only entry point: the same counts, bit-exact
    cnt2 = api.ber_count(dev(llr), dev(bits), dev(mask))
    assert int(cnt2[0]) == e_ref and int(cnt2[1]) == n_ref
