#!/usr/bin/env python
"""Throughput of the natively periodic FMM solve on GB300.

One step = one full solve (mean removal, P2M, M2M, M2L at every level, L2L,
L2P and the near-zone sum) of a seeded synthetic 256^3 density field,
order p = 6, with the input already resident in HBM.  Prints ONE JSON line.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]
                    [--n 256 --L 5 --p 6 --precision fp32|bf16|bf16x3]

Under torchrun (N > 1) every rank solves its own field (independent replicas,
no communication); the value is the cells of all ranks over the slowest rank's
time.  ``--impl reference`` times the FP64 CPU oracle instead (rank 0 only).
"""
import argparse
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

METRIC = "FMM cells/s at 256^3 p=6: mixed-prec+learned vs plain FP32, L2 err ≤1e-4 vs PM"
UNIT = "cells/s"
FP32_FMA_PER_SM_PER_CLK = 128        # FP32 lanes per SM (4 partitions x 32)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_density(n, field):
    from paper_2011_07099_gb300 import inputs
    # the headline workload: 1 + 0.5 lognormal(sigma = 0.5), k^-2 Gaussian field,
    # seeded per rank
    return inputs.lognormal(n, sigma=0.5, seed=5000 + field)


def p2p_flops(N, L):
    S = N >> L
    return (8 ** L) * (S ** 3) * 27 * (S ** 3) * 8.0      # 4 FMA per pair


def m2l_flops(L, p):
    tot = 0.0
    for lev in range(2, L + 1):
        n_off = 37 if lev == 2 else 189
        tot += 2.0 * 4 * p ** 3 * p ** 3 * n_off * 8 ** lev
    return tot


def cpu_baseline():
    """The FP64 oracle, as it stands, on the host cores: full solve of a 64^3
    lognormal field with the same order (p = 6) and leaf size (S = 8, L = 3),
    whose per-cell arithmetic matches the 256^3 p = 6 L = 5 workload within a
    few percent."""
    import numpy as np  # noqa: F401
    from oracle import fmm as ofmm
    rho = workload_density(64, 0)
    t = time.perf_counter()
    ofmm.solve(rho, 3, 6)
    dt = time.perf_counter() - t
    return {"value": 64 ** 3 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "seconds": dt,
            "sample": "full oracle solve of a 64^3 lognormal field, p=6, L=3 (S=8), numpy FP64 on all host cores"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import fmm as ofmm
    n, L, p = 32, 2, 6
    rho = workload_density(n, 0)
    for _ in range(args.warmup):
        ofmm.solve(rho, L, p)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        ofmm.solve(rho, L, p)
        times.append(time.perf_counter() - t)
    ms = 1000.0 * statistics.mean(times)
    value = n ** 3 / (ms / 1000.0)
    sample = (f"FP64 numpy oracle, full solve of a {n}^3 lognormal field per step with order p={p} and leaf "
              f"size S=8 (L={L}), host cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"oracle sample: {n}^3 lognormal sigma=0.5, p={p}, L={L}", "N": n, "L": L,
                       "order": p},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2011_07099_gb300 import binding, build

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()
    B = binding
    n, L, p = args.n, args.L, args.p
    prec = {"fp32": B.FMM_PREC_FP32, "bf16": B.FMM_PREC_BF16, "bf16x3": B.FMM_PREC_BF16X3}[args.precision]
    plan = B.Plan(n, L, p)
    if prec != B.FMM_PREC_FP32:
        plan.set_precision(prec)
    rho = torch.from_numpy(workload_density(n, rank)).to(dev)
    phi = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    acc = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan.solve(rho, phi, acc)
    torch.cuda.synchronize()
    B.fmm_plan_set_timing(plan.handle, True)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    step_ms, stage = [], []
    launches_per_solve = 2 + 1 + (L - 2) + (L - 1) + (L - 2) + 1
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            l2_flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.solve(rho, phi, acc)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            stage.append(B.fmm_plan_stage_times(plan.handle))
        torch.cuda.synchronize()
        barrier()
    wall = time.perf_counter() - wall0
    B.fmm_plan_set_timing(plan.handle, False)
    ms = statistics.mean(step_ms)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * n ** 3 / (ms / 1000.0)

    # per-stage means over the timed steps
    nslot = len(stage[0])
    st = [statistics.mean(s[i] for s in stage) for i in range(nslot)]
    names = ["mean", "p2m", "m2m", "m2l", "l2l", "p2p_l2p"]
    stage_ms = {names[i]: st[i] for i in range(6)}
    for lev in range(2, L + 1):
        stage_ms[f"m2l_level{lev}"] = st[B.FMM_TIME_M2L_LEVEL0 + lev]
    peaks, src = _peaks()
    dominant = max(names, key=lambda k: stage_ms[k])
    if dominant == "p2p_l2p":
        clk_mhz = SM_MAX_MHZ
        peak = SM_COUNT * FP32_FMA_PER_SM_PER_CLK * 2 * clk_mhz * 1e6 / 1e12
        ach = p2p_flops(n, L) / (stage_ms["p2p_l2p"] / 1000.0) / 1e12
        roof = {"kernel": "k_p2p (fused L2P + near-zone sum)", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": f"152 SMs x 128 FP32 FMA/clk x 2 flop x {clk_mhz:.0f} MHz (derived)"}
    else:
        ach = m2l_flops(L, p) / (stage_ms["m2l"] / 1000.0) / 1e12
        if prec == B.FMM_PREC_FP32:
            peak = SM_COUNT * FP32_FMA_PER_SM_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
            roof = {"kernel": "k_m2l_fp32", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None,
                    "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz (derived)"}
        else:
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            roof = {"kernel": "m2l tensor", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None, "peak_source": f"bf16_tflops_sustained ({src})"}

    # end to end through the public host-buffer entry point
    hin = torch.from_numpy(workload_density(n, rank)).pin_memory()
    hphi = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    hacc = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    B.fmm_solve_host(plan.handle, hin, hphi, hacc, stream)
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.fmm_solve_host(plan.handle, hin, hphi, hacc, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == B.FMM_PREC_FP32 else args.precision,
        "data": "synthetic",
        "config": {"workload": f"{n}^3 lognormal sigma=0.5 (seeded), order p={p}, L={L} (S={n >> L}), "
                               f"M2L {args.precision}",
                   "N": n, "L": L, "order": p, "precision": args.precision,
                   "l2_flush": "256 MB buffer written between timed steps",
                   "parallelism": f"replicas x{ws}"},
        "stage_ms": stage_ms,
        "wall_s": wall,
        "roofline": roof,
        "e2e": {"value": ws * n ** 3 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * n ** 3,
                "d2h_bytes_per_step": 16 * n ** 3},
        "gpu_launches": launches_per_solve * args.steps,
        "clocks": clocks,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--L", type=int, default=5)
    ap.add_argument("--p", type=int, default=6)
    ap.add_argument("--precision", choices=["fp32", "bf16", "bf16x3"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
