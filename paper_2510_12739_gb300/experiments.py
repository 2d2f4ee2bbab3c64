"""Training runs and BER tables built on the library's public API.

The paper's figure of merit is the uncoded BER over an SNR (or SINR) grid, of the trained
CoNet against the conventional LS-LMMSE receiver (Sec. IV).  These helpers train a receiver
on slots that the library's device simulator regenerates every step (conet_train_step), and
count bit errors of several receivers on the same seeded held-out slots, so that precisions
are compared pairwise on identical inputs.  Everything runs in libconet's kernels; this
module only sequences calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import api

PRECISIONS = ("fp32", "bf16", "fp16", "fp8")


def train_receiver(net, sim, steps: int, batch: int = 128, precision: str = "bf16", lr: float = 1e-3,
                   seed: int = 5, init_seed: int = 1, lr_schedule: str = "const", log_every: int = 0):
    """Train a CoNet on device-simulated slots with the library's BCE + Adam step.

    lr_schedule "const" keeps lr; "cos" decays it to 0 on a half cosine.  Returns the FP32
    master parameters (numpy) and the list of (step, loss) samples taken every log_every steps."""
    rx = api.Receiver(net, precision=precision, max_batch=batch, train=True)
    rx.init_he(init_seed)
    losses = []
    for i in range(steps):
        a = lr if lr_schedule == "const" else lr * 0.5 * (1.0 + math.cos(math.pi * i / steps))
        want = bool(log_every) and (i + 1) % log_every == 0
        l = rx.train_step(sim, seed, i, batch, a, want_loss=want)
        if want:
            losses.append((i + 1, l))
    params = rx.save_weights()
    rx.close()
    return params, losses


def ber_table(net, sim, params, snrs, slots: int = 2048, chunk: int = 512, precisions=PRECISIONS,
              seed: int = 999, slot0: int = 10_000_000, calib_seed: int = 4242, sinr_share=None):
    """Uncoded BER of the CoNet (``params``) in each precision and of LS-LMMSE, per SNR point.

    Every receiver sees the same seeded slots at each point (paired comparison).  E4M3
    receivers are calibrated once on `chunk` slots of the training distribution drawn with
    calib_seed.  LS-LMMSE treats the interferer as noise when the link has one.  With
    sinr_share = s (interference links only), each grid point is an SINR: the noise and the
    interferer take (1 - s) and s of the noise-plus-interference power.  Returns
    {snr: {receiver: (errors, bits)}}."""
    mask, psym = api.pilots(net)
    evs = {}
    for p in precisions:
        ev = api.Receiver(net, p, max_batch=chunk)
        ev.load_weights(params)
        if p == "fp8":
            cal = api.sim_generate(net, sim, calib_seed, 0, chunk, want_interf=True)
            ev.calibrate(cal["Y"], mask)
        evs[p] = ev
    out = {}
    for snr in snrs:
        point_sim, fixed = sim, float(snr)
        if sinr_share is not None:
            total = 10.0 ** (-snr / 10.0)
            n_db = -10.0 * math.log10((1.0 - sinr_share) * total)
            i_db = -10.0 * math.log10(sinr_share * total)
            point_sim = _replace(sim, sir_lo=i_db, sir_hi=i_db)
            fixed = n_db
        tot = {}
        for c in range(0, slots, chunk):
            B = min(chunk, slots - c)
            s = api.sim_generate(net, point_sim, seed, slot0 + c, B, fixed_snr_db=fixed, want_interf=True)
            for p, ev in evs.items():
                llr = ev.forward(s["Y"], mask, s["noise_var"])
                _, cnt, _ = api.loss_ber(llr, s["bits"], mask)
                _acc(tot, p, cnt)
            iv = s["interf_var"] if sim.interferer else None
            llr = api.ls_lmmse(net, s["Y"], mask, psym, s["noise_var"], interf_var=iv)
            _, cnt, _ = api.loss_ber(llr, s["bits"], mask)
            _acc(tot, "ls_lmmse", cnt)
        out[snr] = {k: (int(v[0]), int(v[1])) for k, v in tot.items()}
    for ev in evs.values():
        ev.close()
    return out


def _acc(tot, key, cnt):
    c = cnt.cpu().numpy()
    t = tot.setdefault(key, [0, 0])
    t[0] += int(c[0])
    t[1] += int(c[1])


def _replace(sim, **kw):
    import dataclasses
    return dataclasses.replace(sim, **kw)


def relative_gap(table, ref: str = "fp32"):
    """{snr: {receiver: (BER_receiver - BER_ref) / BER_ref}} from ber_table's counts."""
    out = {}
    for snr, row in table.items():
        e0, n0 = row[ref]
        b0 = e0 / n0
        out[snr] = {k: ((e / n) - b0) / b0 if b0 > 0 else float("nan") for k, (e, n) in row.items()}
    return out


def sinr_at_ber(table, receiver: str, target: float):
    """SINR (dB) at which a receiver's BER crosses `target`, by linear interpolation of
    log10(BER) between grid points; None when the curve does not cross it."""
    pts = sorted((snr, row[receiver][0] / row[receiver][1]) for snr, row in table.items())
    for (s0, b0), (s1, b1) in zip(pts, pts[1:]):
        if b0 >= target >= b1 and b0 > 0 and b1 > 0:
            l0, l1, lt = np.log10(b0), np.log10(b1), np.log10(target)
            return s0 + (s1 - s0) * (l0 - lt) / (l0 - l1) if l0 != l1 else s0
    return None



# ------------------------------------------------------------------ Sec. IV experiments
def interference_study(steps: int = 6000, batch: int = 64, slots: int = 1024, shares=(0.3, 0.8),
                       sinrs=tuple(np.arange(0.0, 30.1, 2.5)), width_conet: int = 64, width_resnet: int = 88,
                       log=print):
    """CoNet against a parameter-matched single-branch ResNet under co-channel interference
    (Sec. IV, Figs. "Res_0109", "highInterf", "lowInterf"), on the library's own link: 1 Rx,
    14 x 72 grid, 64-QAM, a 64-QAM interferer through an independent TDL channel, 6 taps at
    300 ns, Doppler U(0, 175) Hz (15 m/s at 3.5 GHz).  Both networks have an input layer, 4
    residual blocks and the 1x1 head (the paper's depth); the CoNet has 2 branches of
    `width_conet` channels with Hadamard fusion + LayerNorm, the ResNet one branch of
    `width_resnet` (parameter counts within a few per cent).  Both train with the library's
    FP32 training step on slots with SNR U(5, 30) dB and SIR U(0, 25) dB (interference shares
    of the noise-plus-interference power from about 3 % to 99 %), then decode the same seeded
    slots at every SINR of `sinrs` for each interference share, beside LS-LMMSE (interference
    treated as noise).  Returns the BER tables, the parameter counts and the SINR each
    receiver needs for BER 0.2, 0.1, 0.05 and 0.03 (None where its curve does not cross it)."""
    import dataclasses

    from workloads import NetConfig, SimConfig

    sim = SimConfig(n_taps=6, delay_spread_s=300e-9, fd_lo=0.0, fd_hi=175.0, snr_lo=5.0, snr_hi=30.0,
                    interferer=1, sir_lo=0.0, sir_hi=25.0, iqam_bits=6)
    nets = {"conet": NetConfig(n_rx=1, n_sc=72, qam_bits=6, n_branches=2, depth=4, width=width_conet, residual=1,
                               norm=1),
            "resnet": NetConfig(n_rx=1, n_sc=72, qam_bits=6, n_branches=1, depth=4, width=width_resnet, residual=1,
                                norm=1, resnet_baseline=1)}
    out = {"link": dataclasses.asdict(sim), "steps": steps, "batch": batch, "slots_per_point": slots,
           "params": {k: api.param_count(n) for k, n in nets.items()}, "tables": {}}
    trained = {}
    for name, net in nets.items():
        params, losses = train_receiver(net, sim, steps, batch=batch, precision="fp32", lr=1e-3, lr_schedule="cos",
                                        seed=21, init_seed=2, log_every=max(1, steps // 4))
        trained[name] = params
        out.setdefault("train_loss", {})[name] = losses
        log(f"trained {name}: {losses}")
    for share in shares:
        tab = {}
        for name, net in nets.items():
            t = ber_table(net, sim, trained[name], list(sinrs), slots=slots, precisions=("fp32",),
                          sinr_share=share)
            for snr, row in t.items():
                tab.setdefault(float(snr), {})[name] = row["fp32"]
                tab[float(snr)]["ls_lmmse"] = row["ls_lmmse"]
        key = f"share_{int(round(100 * share))}"
        out["tables"][key] = {str(k): {r: v[0] / v[1] for r, v in row.items()} for k, row in tab.items()}
        need = {}
        for r in ("conet", "resnet", "ls_lmmse"):
            need[r] = {str(t): sinr_at_ber({k: {r: v[r]} for k, v in tab.items()}, r, t) for t in (0.2, 0.1, 0.05, 0.03)}
        out["tables"][key + "_sinr_needed"] = need
        log(f"{key}: {need}")
    return out


if __name__ == "__main__":
    import json
    import sys

    if len(sys.argv) > 1 and sys.argv[1] == "interference":
        steps = int(sys.argv[2]) if len(sys.argv) > 2 else 6000
        res = interference_study(steps=steps)
        print(json.dumps(res))
