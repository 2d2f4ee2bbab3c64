#!/usr/bin/env python
"""Throughput benchmark of the CoNet-Rx receiver on GB300.

One step = one pass of the inference hot path over one batch of synthetic slots already
resident in HBM: input assembly -> every CoNet branch with Hadamard fusion -> 1x1 LLR
head -> BCE loss and bit-error counters against the transmitted bits.  The slots come
from the library's own device-side link simulator before the timed region.  The
default workload is the 2-Rx, 14 x 624 subcarrier, 64-QAM slot batch (B = 256) through
the 3-branch x (input + 6 RB/MRB) x 64-channel residual CoNet in FP32.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import WORKLOADS  # noqa: E402

L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP32_LANES_PER_SM = 128             # FFMA lanes per SM (4 SMSPs x 32)
SM_MAX_MHZ = 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="resid_14x624_b256_fp32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    p.add_argument("--batch", type=int, default=0, help="override the workload's batch (profiling runs)")
    p.add_argument("--precision", choices=["fp32", "bf16", "fp16"], default=None,
                   help="override the workload's conv precision")
    return p.parse_args()


def conv_flops(net, B):
    """Algorithmic FLOPs (2 x MACs) of one body 3x3 conv launch (all branches)."""
    M = B * net.n_sym * net.n_sc
    return 2.0 * M * 9 * net.width * net.width * net.n_branches


def n_body_convs(net):
    """Body (C -> C) 3x3 conv layers per branch."""
    return 2 * net.depth if net.residual else net.depth - 1


def tensor_peak():
    """Dense BF16/FP16 tensor peak in TFLOP/s: the measured sustained cuBLAS figure
    (the conv is timed inside a long step), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback sustained BF16 1.7 PFLOP/s (of fallback)"


def net_flops_per_re(net):
    C, nb = net.width, net.n_branches
    f = 2 * 9 * net.c_in * C * nb
    body = (2 * net.depth) if net.residual else (net.depth - 1)
    f += body * 2 * 9 * C * C * nb
    return f + 2 * C * net.qam_bits


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
    line = {"metric": "conet_infer_slots_per_s", "value": v, "unit": "slots/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "batch_per_step": 1, "note": "one slot of the workload per step"},
            "cpu_baseline": {"value": v, "unit": "slots/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} slots of {w.name}, one per step"},
            "e2e": {"value": v, "unit": "slots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    from paper_2510_12739_gb300 import api

    w = WORKLOADS[args.workload]
    if args.precision:
        import dataclasses
        w = dataclasses.replace(w, precision=args.precision)
    net, B = w.net, (args.batch or w.batch)
    T, F, Q = net.n_sym, net.n_sc, net.qam_bits
    rx = api.Receiver(net, precision=w.precision, max_batch=B)
    rx.init_he(0)
    mask, psym = api.pilots(net)
    s = api.sim_generate(net, w.sim, 1, rank * 1_000_000, B)     # each rank its own slots
    Y, bits, nv = s["Y"], s["bits"], s["noise_var"]
    llr = torch.empty((B, T, F, Q), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    from paper_2510_12739_gb300._lib import check, lib
    import ctypes as C

    def count(l):
        check(lib().conet_loss_ber(C.c_void_p(l.data_ptr()), C.c_void_p(bits.data_ptr()),
                                   C.c_void_p(mask.data_ptr()), B, T, F, Q, 0.0, None,
                                   C.c_void_p(loss.data_ptr()), C.c_void_p(cnt.data_ptr()),
                                   C.c_void_p(cnt.data_ptr() + 8), C.c_void_p(stream.cuda_stream)))

    def step():
        rx.forward(Y, mask, nv, llr)
        count(llr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---------------------------------------------------------------- device-resident timing
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    rx.profile_enable(True)
    n0 = api.launch_count()
    for i in range(args.steps):
        flush.zero_()                                   # evict L2 between steps
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    n_launch = api.launch_count() - n0
    barrier()
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.mean(times)
    conv_ms, conv_n = rx.profile_read(api.PROFILE_KINDS["conv"])
    rx.profile_enable(False)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, rx, count, Y, nv, mask, llr, cnt, flush, stream, B, world, dist, barrier)
    return finish(args, rank, world, local, w, net, B, T, F, Q, ms, times, conv_ms, conv_n, clk, n_launch, e2e, dist)


def end_to_end(args, rx, count, Y, nv, mask, llr, cnt, flush, stream, B, world, dist, barrier):
    import torch
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
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        flush.zero_()
        ev2[i][0].record(stream)
        e2e_step()
        ev2[i][1].record(stream)
    torch.cuda.synchronize()
    ms_e2e = statistics.mean(a.elapsed_time(b) for a, b in ev2)
    if dist is not None:
        t = torch.tensor([ms_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    return {"value": B * world / (ms_e2e / 1e3), "unit": "slots/s",
            "h2d_bytes_per_step": int(Y.nbytes + nv.nbytes),
            "d2h_bytes_per_step": int(llr.nbytes + cnt.nbytes)}


def finish(args, rank, world, local, w, net, B, T, F, Q, ms, times, conv_ms, conv_n, clk, n_launch, e2e, dist):
    import torch
    value = B * world / (ms / 1e3)
    # ---------------------------------------------------------------- roofline of the body conv
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    avg_conv_s = (conv_ms / max(conv_n, 1)) / 1e3
    # one launch per body layer and batch chunk: spread the step's body-conv FLOPs over them
    launches_per_step = conv_n / max(1, args.steps)
    flops_per_launch = conv_flops(net, B) * n_body_convs(net) / max(1e-9, launches_per_step)
    achieved = flops_per_launch / avg_conv_s / 1e12 if conv_n else None
    if w.precision == "fp32":
        peak = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        bound, src = "alu", f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x {SM_MAX_MHZ:.0f} MHz"
        kname = f"conv3x3_fp32_kernel<{net.width},{net.width},8> (body 3x3 conv, {net.n_branches} branches per launch)"
    else:
        peak, src = tensor_peak()
        bound = "tensor"
        kname = (f"conv_tc_kernel<{w.precision},{net.n_branches},{net.width},{net.width}> "
                 f"(tcgen05 body 3x3 conv, {net.n_branches} branches per launch)")
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic_per_launch(net, B),
                "kernel": kname, "peak_source": src, "launches": conv_n, "avg_launch_ms": avg_conv_s * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, secs = cpu_oracle_rate(w)
        cpu = {"value": rate, "unit": "slots/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} slots of {w.name} (FP64 numpy oracle, receive + BER), {secs:.1f} s"}

    if rank == 0:
        line = {"metric": "conet_infer_slots_per_s", "value": value, "unit": "slots/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3"}[w.precision],
                "data": "synthetic",
                "config": {"workload": w.name, "global_batch": B * world, "batch_per_gpu": B, "n_rx": net.n_rx,
                           "grid": f"{T}x{F}", "qam_bits": Q, "branches": net.n_branches, "blocks": net.depth,
                           "width": net.width, "flop_per_slot": net_flops_per_re(net) * T * F,
                           "l2": "flushed (512 MB write) between timed steps", "parallelism": f"replicas{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch,
                "clocks": clk, "step_ms": {"min": min(times), "max": max(times)}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def traffic_per_launch(net, B):
    """DRAM bytes per body-conv launch from the committed ncu summary, when it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    import hashlib
    src = os.path.join(ROOT, "paper_2510_12739_gb300", "csrc", rec.get("source", ""))
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != rec.get("sha256"):
        return None
    per_re = rec["bytes_per_launch"] / rec["res_per_launch"]
    return per_re * B * net.n_sym * net.n_sc


if __name__ == "__main__":
    sys.exit(main())
