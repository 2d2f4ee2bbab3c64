#!/usr/bin/env python
"""Throughput benchmark of the CoNet-Rx receiver on GB300.

One step = one pass of the inference hot path over one batch of synthetic slots already
resident in HBM: input assembly -> every CoNet branch with Hadamard fusion -> 1x1 LLR
head -> BCE loss and bit-error counters against the transmitted bits.  The slots come
from the library's own device-side link simulator before the timed region.  The
headline workload is the 2-Rx, 14 x 624 subcarrier, 64-QAM slot batch (B = 256) through
the 3-branch x (input + 6 RB/MRB) x 64-channel residual CoNet in FP32.

The same line carries, under "variants", the other precisions of that workload, the
4-Rx 14 x 3276 BF16 / FP16 workload, the matched single-branch ResNet, and training
throughput (simulate -> forward -> BCE -> backward -> Adam per step).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import ctypes as C
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import WORKLOADS  # noqa: E402

L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP32_LANES_PER_SM = 128             # FFMA lanes per SM (4 SMSPs x 32)
SM_MAX_MHZ = 2070.0
METRIC = "conet_infer_slots_per_s"
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
NOMINAL_FP8_OVER_BF16 = 4.5 / 2.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="resid_14x624_b256_fp32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    p.add_argument("--no-variants", action="store_true", help="headline workload only")
    p.add_argument("--no-ber", action="store_true", help="skip the trained-network BER table")
    p.add_argument("--batch", type=int, default=0, help="override the workload's batch (profiling runs)")
    p.add_argument("--precision", choices=["fp32", "bf16", "fp16", "tf32x3", "fp8"], default=None,
                   help="override the workload's conv precision")
    return p.parse_args()


def conv_flops(net, B):
    """Algorithmic FLOPs (2 x MACs) of one body conv layer over B slots (all branches): the 3x3
    conv, or the depthwise-separable conv's per-channel 3x3 plus 1x1."""
    C = net.width
    per_re = 9 * C + C * C if getattr(net, "depthwise", 0) else 9 * C * C
    return 2.0 * B * net.n_sym * net.n_sc * per_re * net.n_branches


def n_body_convs(net):
    """Body (C -> C) 3x3 conv layers per branch."""
    return 2 * net.depth if net.residual else net.depth - 1


def net_flops_per_re(net):
    C, nb = net.width, net.n_branches
    body = 9 * C + C * C if getattr(net, "depthwise", 0) else 9 * C * C
    return 2 * 9 * net.c_in * C * nb + n_body_convs(net) * 2 * body * nb + 2 * C * net.qam_bits


def tensor_peak():
    """Dense BF16/FP16 tensor peak in TFLOP/s: the measured sustained cuBLAS figure
    (the conv is timed inside a long step), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback sustained BF16 1.7 PFLOP/s (of fallback)"


def measure_fp8_peak(torch, n=8192, burst=10, sustain_s=3.0):
    """Dense E4M3 tensor throughput on this GPU, measured: cuBLASLt's FP8 GEMM
    (torch._scaled_mm, unit scales, BF16 output) at n x n x n, 2 n^3 FLOP per call; burst =
    best of `burst` single calls, sustained = back-to-back calls for sustain_s seconds.
    An "unavailable" entry instead when this torch build has no FP8 GEMM for the device."""
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()     # column-major operand
        one = torch.ones((), device="cuda")

        def mm():
            return torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)

        for _ in range(3):
            mm()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(burst):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mm()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        k = max(1, int(sustain_s / best))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            mm()
        e1.record()
        torch.cuda.synchronize()
        sus = e0.elapsed_time(e1) / 1e3 / k
        f = 2.0 * n ** 3
        del a, b
        return {"burst_tflops": f / best / 1e12, "sustained_tflops": f / sus / 1e12, "n": n,
                "how": f"torch._scaled_mm e4m3 x e4m3 -> bf16, {n}^3, best of {burst} / {k} back to back"}
    except (RuntimeError, AttributeError, TypeError) as e:
        return {"unavailable": str(e).splitlines()[0][:200]}


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(w, budget_s=12.0, max_slots=64):
    """The FP64 oracle (as it stands) on host cores: slots/s over a bounded sample."""
    from oracle import net as onet, pipeline, sim as osim
    params = onet.init_params(w.net, 0)
    done, t_used = 0, 0.0
    while done < max_slots and t_used < budget_s:
        s = osim.simulate(w.net, w.sim, 1, done, 1)
        t0 = time.perf_counter()
        llr = pipeline.receive(w.net, params, s["Y"], s["pilot_sym"], s["pilot_mask"])
        pipeline.ber(llr, s["bits"], s["pilot_mask"])
        t_used += time.perf_counter() - t0
        done += 1
    return done / t_used, done, t_used


def reference_arm(args, rank, world):
    w = WORKLOADS[args.workload]
    if rank != 0:
        return 0
    from oracle import net as onet, pipeline, sim as osim
    params = onet.init_params(w.net, 0)
    slots = [osim.simulate(w.net, w.sim, 1, i, 1) for i in range(args.steps + args.warmup)]

    def step(s):
        llr = pipeline.receive(w.net, params, s["Y"], s["pilot_sym"], s["pilot_mask"])
        pipeline.ber(llr, s["bits"], s["pilot_mask"])

    for i in range(args.warmup):
        step(slots[i])
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(slots[args.warmup + i])
    dt = time.perf_counter() - t0
    v = args.steps / dt
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": v, "unit": "slots/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "batch_per_step": 1, "note": "one slot of the workload per step"},
            "cpu_baseline": {"value": v, "unit": "slots/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} slots of {w.name}, one per step"},
            "e2e": {"value": v, "unit": "slots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


RANK_SLOT_STRIDE = 1_000_000   # slot ids of rank r start at r * RANK_SLOT_STRIDE (disjoint shards)


def rank_slot0(rank: int) -> int:
    return rank * RANK_SLOT_STRIDE


def max_over_ranks(v: float, dist=None, device="cpu") -> float:
    """The largest v over all ranks (the job's step time is its slowest rank's)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


class Ctx:
    def __init__(self, rank, world, local, dist):
        import torch
        self.torch = torch
        self.rank, self.world, self.local, self.dist = rank, world, local, dist
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, v):
        return max_over_ranks(v, self.dist, "cuda")

    def timed(self, fn, steps):
        """Per-step CUDA-event times on the launch stream, L2 flushed between steps."""
        torch = self.torch
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            self.flush.zero_()
            evs[i][0].record(self.stream)
            fn()
            evs[i][1].record(self.stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]


FP8_PEAK = {}   # filled by main() with measure_fp8_peak's result before the E4M3 variants


def roofline_of(w, net, B, rx, steps, n_sm):
    from paper_2510_12739_gb300 import api
    conv_ms, conv_n = rx.profile_read(api.PROFILE_KINDS["conv"])
    avg_s = (conv_ms / max(conv_n, 1)) / 1e3
    per_step = conv_n / max(1, steps)
    # the whole-network kernel runs every layer and the head of the batch in one launch
    whole = rx.whole_network("auto") and B >= api.WHOLE_NET_MIN_SLOTS
    if whole:
        flops_per_launch = net_flops_per_re(net) * B * net.n_sym * net.n_sc / max(1e-9, per_step)
    else:
        flops_per_launch = conv_flops(net, B) * n_body_convs(net) / max(1e-9, per_step)
    achieved = flops_per_launch / avg_s / 1e12 if conv_n else None
    if w.precision == "fp32":
        peak = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        bound, src = "alu", f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x {SM_MAX_MHZ:.0f} MHz"
        kname = f"conv3x3_fp32_kernel<{net.width},{net.width},8> (body 3x3 conv, {net.n_branches} branches per launch)"
    else:
        peak, src = tensor_peak()
        bound = "tensor"
        if w.precision == "tf32x3":
            # TF32 runs at the nominal 1.1 / 2.25 of the BF16 rate and issues 3 MMAs per product
            peak = peak * NOMINAL_TF32_OVER_BF16 / 3.0
            src += " x 1.1/2.25 (nominal TF32/BF16) / 3 MMAs per useful product (split TF32)"
        elif w.precision == "fp8":
            if FP8_PEAK.get("sustained_tflops"):
                peak = FP8_PEAK["sustained_tflops"]
                src = "measured dense E4M3 GEMM, sustained (" + FP8_PEAK["how"] + ") (of measured)"
            else:
                peak = peak * NOMINAL_FP8_OVER_BF16
                src += " x 4.5/2.25 (nominal FP8/BF16 dense)"
        if whole:
            kname = (f"smallnet_kernel<{w.precision}> (tcgen05 whole network: every layer and the head, "
                     f"one slot per CTA; FLOPs of all layers)")
        elif getattr(net, "depthwise", 0):
            kname = (f"dwconv3x3_16_kernel + conv_tc_kernel<{w.precision},{net.n_branches},{net.width},"
                     f"{net.width}> 1x1 (depthwise-separable body conv: two launches, FLOPs of both)")
        else:
            kname = (f"conv_tc_kernel<{w.precision},{net.n_branches},{net.width},{net.width}> "
                     f"(tcgen05 body 3x3 conv, {net.n_branches} branches per launch)")
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic_per_launch(w, net, B, per_step),
            "kernel": kname, "peak_source": src, "launches": conv_n, "avg_launch_ms": avg_s * 1e3}


def measure_inference(ctx, w, B, steps, warmup, clocks=False, e2e=False):
    """Device-resident inference throughput (and optionally host-buffer end to end)."""
    torch = ctx.torch
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import check, lib
    net = w.net
    T, F, Q = net.n_sym, net.n_sc, net.qam_bits
    rx = api.Receiver(net, precision=w.precision, max_batch=B)
    rx.init_he(0)
    mask, _ = api.pilots(net)
    s = api.sim_generate(net, w.sim, 1, rank_slot0(ctx.rank), B)     # each rank its own slots
    Y, bits, nv = s["Y"], s["bits"], s["noise_var"]
    llr = torch.empty((B, T, F, Q), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = ctx.stream

    def count(l):
        check(lib().conet_loss_ber(C.c_void_p(l.data_ptr()), C.c_void_p(bits.data_ptr()),
                                   C.c_void_p(mask.data_ptr()), B, T, F, Q, 0.0, None,
                                   C.c_void_p(loss.data_ptr()), C.c_void_p(cnt.data_ptr()),
                                   C.c_void_p(cnt.data_ptr() + 8), C.c_void_p(stream.cuda_stream)))

    def step():
        rx.forward(Y, mask, nv, llr)
        count(llr)

    for _ in range(warmup):
        step()
    rx.sync()
    ctx.barrier()
    sampler = ClockSampler(ctx.local) if clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    n0 = api.launch_count()
    times = ctx.timed(step, steps)   # repeated identical forwards replay one CUDA graph
    n_launch = api.launch_count() - n0
    ctx.barrier()
    clk = sampler.stop() if sampler else None
    ms = ctx.max_over_ranks(statistics.mean(times))
    # the per-kernel roofline comes from a second, event-timed pass (eager launches)
    rx.profile_enable(True)
    ctx.timed(step, steps)
    n_sm = torch.cuda.get_device_properties(ctx.local).multi_processor_count
    roof = roofline_of(w, net, B, rx, steps, n_sm)
    rx.profile_enable(False)
    rx.sync()
    out = {"value": job_rate(B, ctx.world, ms), "ms_per_step": ms, "roofline": roof, "gpu_launches": n_launch,
           "clocks": clk, "step_ms": {"min": min(times), "max": max(times)}}
    if e2e:
        Y_h = Y.cpu().pin_memory()
        nv_h = nv.cpu().pin_memory()
        llr_h = torch.empty(llr.shape, dtype=llr.dtype, pin_memory=True)
        cnt_h = torch.empty(2, dtype=torch.int64, pin_memory=True)
        Yd, nvd = torch.empty_like(Y), torch.empty_like(nv)

        def e2e_step():
            Yd.copy_(Y_h, non_blocking=True)
            nvd.copy_(nv_h, non_blocking=True)
            rx.forward(Yd, mask, nvd, llr)
            count(llr)
            llr_h.copy_(llr, non_blocking=True)
            cnt_h.copy_(cnt, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ctx.barrier()
        ms_e2e = ctx.max_over_ranks(statistics.mean(ctx.timed(e2e_step, steps)))
        out["e2e"] = {"value": job_rate(B, ctx.world, ms_e2e), "unit": "slots/s",
                      "h2d_bytes_per_step": int(Y.nbytes + nv.nbytes),
                      "d2h_bytes_per_step": int(llr.nbytes + cnt.nbytes)}
    rx.close()
    return out


def measure_training(ctx, w, steps, warmup):
    """Train slots/s: each step simulates B slots on the device, runs forward, BCE,
    backward and Adam (conet_train_step)."""
    from paper_2510_12739_gb300 import api
    B = w.batch
    rx = api.Receiver(w.net, precision=w.precision, max_batch=B, train=True)
    rx.init_he(1)
    it = [0]

    def step():
        rx.train_step(w.sim, 7, rank_slot0(ctx.rank) + it[0], B, 1e-3, want_loss=False)
        it[0] += 1

    for _ in range(warmup):
        step()
    rx.sync()
    times = ctx.timed(step, steps)
    loss = rx.train_step(w.sim, 7, rank_slot0(ctx.rank) + it[0], B, 1e-3, want_loss=True)
    ms = ctx.max_over_ranks(statistics.mean(times))
    rx.close()
    return {"value": job_rate(B, ctx.world, ms), "unit": "train slots/s", "ms_per_step": ms,
            "precision": w.precision, "loss_after": loss}


def measure_depth(ctx):
    """Sec. IV depth comparison (Fig. "InferenceD"): a 14-layer CoNet (4 branches x 64, input
    + 6 RB/MRB + head) against a 24-layer ResNet (1 x 96, input + 11 RB + head), 1.80 M and
    1.84 M parameters, on the 2-Rx 14 x 624 link in BF16: latency of one slot (B = 1) and
    throughput at B = 256, with the library's kernels."""
    out = {}
    for name in ("conet_d14_14x624_bf16", "resnet_d24_14x624_bf16"):
        w = WORKLOADS[name]
        for B, steps in ((1, 50), (w.batch, 10)):
            r = measure_inference(ctx, w, B, steps, 3)
            out[f"{name}@B{B}"] = {"ms_per_step": r["ms_per_step"], "slots_per_s": r["value"]}
    c1, r1 = out["conet_d14_14x624_bf16@B1"]["ms_per_step"], out["resnet_d24_14x624_bf16@B1"]["ms_per_step"]
    c2, r2 = (out["conet_d14_14x624_bf16@B256"]["ms_per_step"], out["resnet_d24_14x624_bf16@B256"]["ms_per_step"])
    out["latency_reduction_B1"] = 1.0 - c1 / r1
    out["time_reduction_B256"] = 1.0 - c2 / r2
    return out


BER_GRIDS = {"plain_14x72": ("plain_14x72_b16_fp32", range(0, 21, 5)),
             "train_14x72": ("train_14x72_b128_bf16", range(-5, 26, 5)),
             "interf_14x72": ("interf_14x72_b512_fp8", range(0, 21, 5))}


def measure_ber(steps=20_000):
    """Matched BER: the 14 x 72 CoNet trained on device-simulated slots (BF16 training handle,
    `steps` steps of 128 slots, Adam 1e-3), then FP32 / BF16 / FP16 / E4M3 and LS-LMMSE on the
    same 2048 seeded held-out slots per grid point; BER and the gap to FP32 per receiver."""
    from paper_2510_12739_gb300 import experiments as ex
    w = WORKLOADS["train_14x72_b128_bf16"]
    t0 = time.perf_counter()
    params, losses = ex.train_receiver(w.net, w.sim, steps, batch=w.batch, precision="bf16", lr=1e-3,
                                       log_every=steps // 4)
    out = {"network": "14x72 plain CoNet, 2 branches x 4 conv x 32", "train_steps": steps, "batch": w.batch,
           "train_s": time.perf_counter() - t0, "train_loss": losses, "slots_per_point": 2048, "grids": {}}
    for name, (wl, snrs) in BER_GRIDS.items():
        tab = ex.ber_table(w.net, WORKLOADS[wl].sim, params, list(snrs))
        gap = ex.relative_gap(tab)
        out["grids"][name] = {str(snr): {k: {"ber": e / n, "errors": e, "gap_vs_fp32": gap[snr][k]}
                                         for k, (e, n) in row.items()} for snr, row in tab.items()}
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_12739_gb300 import api  # noqa: F401  (fails loudly without libconet)
    ctx = Ctx(rank, world, local, dist)

    w = WORKLOADS[args.workload]
    if args.precision:
        w = dataclasses.replace(w, precision=args.precision)
    B = args.batch or w.batch
    head = measure_inference(ctx, w, B, args.steps, args.warmup, clocks=True, e2e=not args.no_e2e)

    variants = {}
    if (not args.no_variants and not args.batch) or w.precision == "fp8":
        FP8_PEAK.update(measure_fp8_peak(torch))
        if w.precision == "fp8":      # the headline's roofline used the nominal ratio: redo it
            head = measure_inference(ctx, w, B, args.steps, args.warmup, clocks=True, e2e=not args.no_e2e)
    if not args.no_variants and not args.batch:
        for name, prec, steps in [("resid_14x624_b256_fp32", "tf32x3", 10), ("resid_14x624_b256_fp32", "bf16", 10),
                                  ("resid_14x624_b256_fp32", "fp16", 10), ("resnet_14x624_b256_fp32", "fp32", 5),
                                  ("resid_14x624_b256_fp32", "fp8", 10),
                                  ("resid_14x3276_b1024_bf16", "bf16", 3), ("resid_14x3276_b1024_bf16", "fp16", 3),
                                  ("resid_14x3276_b1024_bf16", "fp8", 3),
                                  ("interf_14x72_b512_fp8", "fp8", 20), ("interf_14x72_b512_fp8", "bf16", 20),
                                  ("interf_14x72_b512_fp8", "fp32", 20),
                                  ("plain_14x72_b16_fp32", "fp32", 20), ("plain_14x72_b16_fp32", "bf16", 20),
                                  ("resid_dw_14x624_b256_bf16", "bf16", 10), ("resid_dw_14x624_b256_bf16", "fp32", 5)]:
            vw = dataclasses.replace(WORKLOADS[name], precision=prec)
            r = measure_inference(ctx, vw, vw.batch, steps, 2)
            variants[f"{name}:{prec}"] = {"value": r["value"], "unit": "slots/s", "ms_per_step": r["ms_per_step"],
                                          "conv_tflops": r["roofline"]["achieved"],
                                          "roofline_frac": r["roofline"]["frac"], "bound": r["roofline"]["bound"]}
        for prec in ("bf16", "fp32"):
            tw = dataclasses.replace(WORKLOADS["train_14x72_b128_bf16"], precision=prec)
            variants[f"train_14x72_b128:{prec}"] = measure_training(ctx, tw, 20, 3)
        variants["depth_comparison"] = measure_depth(ctx)

    ber = None
    if rank == 0 and not args.no_ber and not args.batch:
        ber = measure_ber()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, secs = cpu_oracle_rate(w)
        cpu = {"value": rate, "unit": "slots/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} slots of {w.name} (FP64 numpy oracle, receive + BER), {secs:.1f} s"}

    if rank == 0:
        net = w.net
        line = {"metric": METRIC, "value": head["value"], "unit": "slots/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "tf32x3": "f32 (tf32x3 split)",
                          "fp8": "e4m3"}[w.precision],
                "data": "synthetic",
                "config": {"workload": w.name, "global_batch": B * world, "batch_per_gpu": B, "n_rx": net.n_rx,
                           "grid": f"{net.n_sym}x{net.n_sc}", "qam_bits": net.qam_bits,
                           "branches": net.n_branches, "blocks": net.depth, "width": net.width,
                           "flop_per_slot": net_flops_per_re(net) * net.n_sym * net.n_sc,
                           "l2": "flushed (512 MB write) between timed steps", "parallelism": f"replicas{world}"},
                "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head.get("e2e"),
                "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "step_ms": head["step_ms"],
                "fp8_peak": FP8_PEAK or None, "ber": ber, "variants": variants}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def traffic_per_launch(w, net, B, launches_per_step):
    """DRAM bytes per body-conv launch from the committed ncu summary, scaled to this
    launch's REs, when it was taken on the current kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            recs = json.load(f)
    except (OSError, ValueError):
        return None
    rec = recs.get(w.precision)
    if not rec or rec.get("workload") != w.name:
        return None
    src = os.path.join(ROOT, "paper_2510_12739_gb300", "csrc", rec["source"])
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != rec.get("sha256"):
        return None
    res_per_launch = B * net.n_sym * net.n_sc * n_body_convs(net) / max(1e-9, launches_per_step)
    return rec["bytes_per_launch"] / rec["res_per_launch"] * res_per_launch


if __name__ == "__main__":
    sys.exit(main())
