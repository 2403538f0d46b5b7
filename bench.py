#!/usr/bin/env python
"""Throughput of the natively periodic FMM solve on GB300.

One step = one full solve (mean removal, P2M, M2M, M2L at every level, L2L,
L2P and the near-zone sum) of a seeded synthetic 256^3 density field,
order p = 6, with the input already resident in HBM.  The timed form is the
mixed-precision one (tensor-core bf16x3 M2L at levels >= 4); the plain FP32
form is timed on the same field in the same run, and the result's error
against PM is stated twice: by the library (fmm_plan_error_stats, exact at
256 sampled cells) and, with the CPU baseline, over every cell by the FP64
oracle's FFT PM.  Prints ONE JSON line.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]
                    [--n 256 --L 5 --p 6 --precision fp32|bf16|bf16x3]

Under torchrun (N > 1) every rank solves its own field (independent replicas,
no communication); the value is the cells of all ranks over the slowest rank's
time.  ``--impl reference`` times the FP64 CPU oracle instead (rank 0 only).
"""
import argparse
import json

import numpy as np
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
# weights of the learned M2L table correction trained by
# `python -m paper_2011_07099_gb300.learn` (order 6, 64^3 training fields)
DEFAULT_CORRECTION = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2011_07099_gb300", "data",
                                  "correction_p6.npz")
UNIT = "cells/s"
FP32_FMA_PER_SM_PER_CLK = 128        # FP32 lanes per SM (4 partitions x 32)
SM_MAX_MHZ = 2070.0                  # used only when neither nvidia-smi nor MEASURED_PEAKS.json gives it


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


def slowest_rank_ms(ms, ws, device=None):
    """The step time of the whole job: the maximum over the ranks (one
    independent field per rank, no data-path collective; this all-reduce
    only aggregates the timing)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_cells_per_s(ws, n, ms):
    """Cells of all ranks over the slowest rank's step time (weak scaling)."""
    return ws * n ** 3 / (ms / 1000.0)


def workload_density(n, field):
    from paper_2011_07099_gb300 import inputs
    # the headline workload: 1 + 0.5 lognormal(sigma = 0.5), k^-2 Gaussian field,
    # seeded per rank
    return inputs.lognormal(n, sigma=0.5, seed=5000 + field)


# DRAM bytes (read + write) of one k_p2p launch, from an ncu capture of the
# current kernel at 256^3, p = 6, L = 5 (dram__bytes_read.sum +
# dram__bytes_write.sum); not measured in this run
P2P_TRAFFIC = {(256, 5, 6): 419.3e6}
# DRAM bytes (read + write) of one launch of the tensor-core M2L at the leaf
# level and of the three near-zone FFT kernels together, from ncu captures
# of the current kernels at 256^3 p=6 (profiles/); None where not captured
M2L_TC_TRAFFIC = {(256, 5, 6): 1603.3e6}
M2L_TC_TRAFFIC_SOURCE = ("ncu capture of the current k_m2l_tc at 256^3 p=6, level 5 (dram__bytes read 1503.1 MB + "
                         "write 100.2 MB), not measured in this run")
NEAR_FFT_TRAFFIC = {(256, 5, 6): 6942.5e6}
NEAR_FFT_TRAFFIC_SOURCE = ("ncu capture of the current k_nz_fwd + k_nz_mac + k_nz_l2p + k_nz_inv at 256^3 p=6 "
                           "(dram__bytes read+write summed), not measured in this run")
P2P_TRAFFIC_SOURCE = ("ncu capture of the current k_p2p at 256^3 p=6 (dram__bytes read 197.6 MB + write 221.7 MB), "
                      "not measured in this run")


def measure_fp32_peak(B, dev, stream, reps=40):
    """The FP32 CUDA-core peak of this device, measured: the library's FMA
    probe (dependent FMA chains only, 2 CTAs of 1024 threads per SM), each
    launch timed with CUDA events on the launching stream, median of `reps`
    launches after 3 warm-ups; SM clocks are sampled meanwhile."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 2 * sms, 20000
    out = torch.empty(blocks, dtype=torch.float32, device=dev)
    for _ in range(3):
        flops = B.fmm_probe_fma(out, blocks, iters, stream)
    torch.cuda.synchronize(dev)
    ms = []
    with ClockSampler(dev.index) as clk:
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.fmm_probe_fma(out, blocks, iters, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    med = statistics.median(ms)
    c = clk.summary() or {}
    max_mhz = c.get("sm_max_mhz") or SM_MAX_MHZ
    derived = sms * FP32_FMA_PER_SM_PER_CLK * 2 * max_mhz * 1e6 / 1e12
    return {"tflops": flops / (med / 1e3) / 1e12, "launch_ms": med, "sm_count": sms,
            "sm_mhz_median": c.get("sm_mhz"), "sm_max_mhz": max_mhz, "clock_reasons": c.get("reasons"),
            "derived_at_max_clock_tflops": derived,
            "how": f"fmm_probe_fma: {blocks} CTAs x 1024 threads x 8 FMA chains x {iters} x 16, CUDA events, "
                   f"median of {reps}"}


def p2p_flops(N, L):
    S = N >> L
    return (8 ** L) * (S ** 3) * 27 * (S ** 3) * 8.0      # 4 FMA per pair


def m2l_flops(L, p):
    tot = 0.0
    for lev in range(2, L + 1):
        n_off = 37 if lev == 2 else 189
        tot += 2.0 * 4 * p ** 3 * p ** 3 * n_off * 8 ** lev
    return tot


def near_fft_flops(N, L, p):
    """Arithmetic of the near zone by FFT per solve, counted as the kernels do
    it (direct DFTs per axis, 8-cell leaves, 16^3 padded transforms): the
    spectral sums (27 offsets x 4 fields x 2304 frequencies, 8 flop per complex
    multiply-add), the forward transform of the masses and the four inverse
    transforms that keep only the leaf's cells."""
    leaves = 8 ** L
    mac = 27 * 4 * 2304 * 8
    fwd = 2 * (64 * 9 * 8 * 2 + 8 * 16 * 9 * 8 * 4 + 16 * 16 * 9 * 8 * 4)        # FMA x 2 per axis pass
    inv = 4 * 2 * (8 * 16 * 9 * 16 * 4 + 8 * 8 * 9 * 16 * 4 + 512 * 8 * 2)   # per field, 4 fields
    return float(leaves * (mac + fwd + inv))


def cpu_baseline():
    """The FP64 oracle, as it stands, on the host cores: full solve of a 64^3
    lognormal field with the same order (p = 6) and leaf size (S = 8, L = 3),
    whose per-cell arithmetic matches the 256^3 p = 6 L = 5 workload within a
    few percent."""
    import numpy as np  # noqa: F401
    from oracle import fmm as ofmm
    rho = workload_density(64, 0)
    t, c = time.perf_counter(), time.process_time()
    ofmm.solve(rho, 3, 6)
    dt, cpu = time.perf_counter() - t, time.process_time() - c
    return {"value": 64 ** 3 / dt, "unit": UNIT, "cores": effective_cores(cpu, dt), "kind": "oracle",
            "cores_available": os.cpu_count(), "seconds": dt,
            "sample": "full oracle solve of a 64^3 lognormal field, p=6, L=3 (S=8), numpy FP64 on the host cores"}


def effective_cores(cpu_seconds, wall_seconds):
    """Threads the oracle kept busy on average: process CPU time over wall
    time (numpy's BLAS decides how many it starts)."""
    return round(cpu_seconds / wall_seconds, 1) if wall_seconds > 0 else 0.0


def pm_references(rho):
    """Part of the oracle leg: PM with the same Green's function (FFT
    convolution, FP64 host) and, secondary, the spectral PM with G_K."""
    import numpy as np
    from oracle import green, pm
    n = rho.shape[0]
    m = pm.masses(rho.astype(np.float64))
    return pm.pm(m, green.g_s1, green.grad_g_s1, green.self_term(n)), pm.pm_gk(m)


def accuracy_vs_pm(refs, phi, acc):
    """Relative L2 over all cells of a result against PM(G_S1) (primary: the
    same G in PM and FMM) and PM(G_K) (secondary)."""
    import numpy as np
    (pphi, pg), (kphi, kg) = refs
    rel = lambda a, b: float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))
    return {"vs_pm_gs1": {"phi": rel(phi, pphi), "g": rel(acc, pg)},
            "vs_pm_gk": {"phi": rel(phi - phi.mean(), kphi - kphi.mean()), "g": rel(acc, kg)},
            "note": "relative L2 over all cells; PM(G_S1) is the primary reference (same G in PM and FMM)"}


def learned_correction(args):
    """The learned table correction the headline workload applies: the
    shipped order-6 weights (or --correction) in the tensor-core forms,
    None otherwise.  The weights file path is under "path"."""
    wpath = args.correction or (DEFAULT_CORRECTION if args.p == 6 else None)
    if args.precision == "fp32" or args.no_correction or not wpath or not os.path.exists(wpath):
        return None
    here = os.path.dirname(os.path.abspath(__file__))
    return {"path": wpath, "weights": os.path.relpath(wpath, here), "inference": "bf16",
            "applied_to": "M2L tables, levels 2..L"}


def near_fft_used(args):
    """The near zone by FFT (Sec. 3's doubled-grid convolution) needs 8-cell leaves."""
    return args.near == "fft" and (args.n >> args.L) == 8


def headline_config(args, learned, ws):
    """The `config` object of the headline workload; both arms print it."""
    n, L, p = args.n, args.L, args.p
    near = "near zone by FFT on the doubled grid" if near_fft_used(args) else "near zone by direct sum"
    return {"workload": f"{n}^3 lognormal sigma=0.5 (seeded), order p={p}, L={L} (S={n >> L}), "
                        f"M2L levels>=4 {args.precision}, levels 2-3 extended-precision CUDA-core, {near}"
                        + (", learned table correction" if learned else ""),
            "N": n, "L": L, "order": p, "precision": args.precision, "near_zone": args.near if near_fft_used(args)
            else "direct",
            "learned_correction": None if learned is None else {k: v for k, v in learned.items() if k != "path"},
            "l2_flush": "256 MB buffer written between timed steps",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import fmm as ofmm
    n, L, p = 64, 3, 6            # the cpu_baseline sample: levels 2 and 3, M2M and L2L, S = 8
    rho = workload_density(64, 0)
    for _ in range(args.warmup):
        ofmm.solve(rho, L, p)
    times = []
    c = time.process_time()
    for _ in range(args.steps):
        t = time.perf_counter()
        ofmm.solve(rho, L, p)
        times.append(time.perf_counter() - t)
    cores = effective_cores(time.process_time() - c, sum(times))
    ms = 1000.0 * statistics.mean(times)
    value = n ** 3 / (ms / 1000.0)
    sample = (f"FP64 numpy oracle (plain method, no correction), full solve of a {n}^3 lognormal sigma=0.5 "
              f"field per step with order p={p} and the workload's leaf size S=8 (L={L}); cells/s of the "
              f"sample stand for the {args.n}^3 workload")
    line = {"impl": "reference", "method": "the plain method in FP64 (CPU oracle): no tensor cores, no "
                                          "mixed precision, no learned correction",
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(args, learned_correction(args), ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cores_available": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def _time_solves(B, plan, rho, phi, acc, steps, warmup, l2_flush, stream, barrier, timing=True):
    """W untimed solves, then `steps` solves each bracketed by CUDA events on
    the launching stream, with an L2 flush (256 MB write) between them.  The
    timed solves run as a user's do (the library overlaps independent stages
    on its own streams); the per-stage times come from two more solves with
    the library's stage timing on (which runs the stages one after another),
    outside the timed region.  Returns (per-step ms list, per-stage-time
    lists, wall seconds)."""
    import torch
    for _ in range(warmup):
        plan.solve(rho, phi, acc)
    torch.cuda.synchronize()
    step_ms, stage = [], []
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(steps):
        l2_flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.solve(rho, phi, acc)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    if timing:
        B.fmm_plan_set_timing(plan.handle, True)
        for _ in range(2):
            l2_flush.zero_()
            plan.solve(rho, phi, acc)
            stage.append(B.fmm_plan_stage_times(plan.handle))
        B.fmm_plan_set_timing(plan.handle, False)
    return step_ms, stage, wall


def device_check(B, plan):
    """fmm_plan_check after a loop of solves: "ok", or the error it reports
    (a bounded device wait that ran out makes those results invalid)."""
    rc = B.lib().fmm_plan_check(plan.handle)
    return "ok" if rc == B.FMM_OK else B.lib().fmm_error_string(rc).decode()


def launches_per_solve(L, tc, p=6, near_fft=False):
    # mean (2) + P2M + M2M per level + M2L per level + L2L per level + P2P
    # (four kernels with the near zone by FFT: forward, sums, L2P, inverse);
    # M2L of the coarse levels (2-3, and every level above the leaves at
    # order >= 7) adds the FP64 range-sum kernel, tensor-core levels the
    # BF16 split kernel
    wide = lambda lev: lev <= 3 or (p >= 7 and lev < L)
    tc_first = max(4, L) if p >= 7 else 4
    m2l = sum(2 if (wide(lev) or (tc and lev >= tc_first)) else 1 for lev in range(2, L + 1))
    return 2 + 1 + (L - 2) + m2l + (L - 2) + (4 if near_fft else 1)


def solve_roofline(n, L, p, tc, ms, peaks, fp32_tflops, near_fft=False):
    """Ideal time of the whole solve (each step at its own bound: FP32 FMA,
    BF16 tensor (executed products), HBM bytes) against the measured step.
    With the near zone by FFT its term is the larger of its arithmetic at the
    FP32 peak and its spectra's HBM round trips (source spectra written and
    read, target spectra written and read: 2 x (18 + 74) KB per leaf)."""
    fp32 = fp32_tflops * 1e12
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0) * 1e12
    hbm = peaks.get("hbm_gbs", 6500.0) * 1e9
    p3 = p ** 3
    tc_first = max(4, L) if p >= 7 else 4
    if near_fft:
        near = max(near_fft_flops(n, L, p) / fp32, (8 ** L) * 2 * (18432 + 73728) / peaks.get("hbm_gbs", 6500.0) / 1e9)
        t = {"near_fft": near, "m2l_cuda_cores": 0.0, "m2l_tensor": 0.0}
    else:
        t = {"p2p": p2p_flops(n, L) / fp32, "m2l_cuda_cores": 0.0, "m2l_tensor": 0.0}
    for lev in range(2, L + 1):
        f = 2.0 * 4 * p3 * p3 * (37 if lev == 2 else 189) * 8 ** lev
        if tc and lev >= tc_first:
            t["m2l_tensor"] += 3 * f / bf16
        else:
            t["m2l_cuda_cores"] += f / fp32
    bytes_ = 4 * n ** 3 * 2 + 4 * p3 * 8 ** L                              # mean + P2M
    bytes_ += sum(9 * 4 * p3 * 8 ** lev for lev in range(2, L))          # M2M
    bytes_ += sum(4 * 4 * p3 * 8 ** lev * 17 for lev in range(2, L))     # L2L (parent + children read/write)
    t["hbm_passes"] = bytes_ / hbm
    ideal = sum(t.values()) * 1e3
    return {"ideal_ms": ideal, "measured_ms": ms, "frac": ideal / ms,
            "terms_ms": {k: v * 1e3 for k, v in t.items()},
            "peaks": f"FP32 {fp32_tflops:.1f} TFLOP/s (measured, fmm_probe_fma), BF16 sustained and HBM from "
                     "MEASURED_PEAKS.json"}


def run_ours(args):
    import numpy as np
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
    tc = prec != B.FMM_PREC_FP32

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    rho_host = workload_density(n, rank)
    rho = torch.from_numpy(rho_host).to(dev)
    phi = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    acc = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    plan = B.Plan(n, L, p)
    if tc:
        plan.set_precision(prec)
    learned = learned_correction(args)
    if learned is not None:
        w = torch.from_numpy(np.load(learned["path"])["w"].astype(np.float32)).to(dev)
        B.fmm_plan_set_correction(plan.handle, w)   # tabulated once at plan time; BF16 inference
    near_fft = near_fft_used(args)
    if near_fft:
        B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_FFT)
    # the tensor-core tile of each level, autotuned at plan time (outside the timed region)
    tc_tiles = B.fmm_plan_autotune_tiles(plan.handle, rho)[:L + 1] if tc else None
    with ClockSampler(dev.index) as clk:
        step_ms, stage, wall = _time_solves(B, plan, rho, phi, acc, args.steps, args.warmup, l2_flush, stream,
                                            barrier)
    checks = {"timed_solves": device_check(B, plan)}
    ms = slowest_rank_ms(statistics.mean(step_ms), ws, dev)
    value = whole_job_cells_per_s(ws, n, ms)
    host_leg = rank == 0 and ws == 1 and not args.no_cpu_baseline
    result_phi = phi.cpu().numpy() if host_leg else None
    result_acc = acc.cpu().numpy() if host_leg else None
    # the library's own statement of this result's error against PM with
    # G_S1, measured exactly at sampled cells (outside the timed region)
    stmt_cells = 256

    def statement_of(pl, ph, ac):
        try:
            e_phi, e_g = pl.error_stats(rho, ph, ac, samples=stmt_cells, seed=1)
            return {"vs_pm_gs1": {"phi": e_phi, "g": e_g}, "cells": stmt_cells,
                    "source": "fmm_plan_error_stats (exact direct sum at sampled cells, GPU)"}
        except B.FMMError as e:   # reported in the line; the timed numbers stand
            return {"failed": str(e)}

    statement = statement_of(plan, phi, acc)
    checks["error_statement"] = device_check(B, plan)

    # what the learned correction gains on the timed field: the same form
    # without the correction, solved once (outside the timed region)
    gain = None
    if learned is not None:
        nplan = B.Plan(n, L, p)
        if tc:
            nplan.set_precision(prec)
        if near_fft:
            B.fmm_plan_set_near_algorithm(nplan.handle, B.FMM_NEAR_FFT)
        nphi = torch.empty_like(phi)
        nacc = torch.empty_like(acc)
        nplan.solve(rho, nphi, nacc)
        torch.cuda.synchronize(dev)
        checks["without_correction"] = device_check(B, nplan)
        gain = {"with_correction": statement.get("vs_pm_gs1"),
                "without_correction": statement_of(nplan, nphi, nacc).get("vs_pm_gs1"),
                "measured_by": f"fmm_plan_error_stats, {stmt_cells} cells (seed 1), same cells for both"}
        if host_leg:
            gain["without_correction_host_pm"] = ("pending", nphi.cpu().numpy(), nacc.cpu().numpy())
        nplan.close()
        del nphi, nacc

    # per-stage means over the timed steps
    nslot = len(stage[0])
    st = [statistics.mean(s[i] for s in stage) for i in range(nslot)]
    names = ["mean", "p2m", "m2m", "m2l", "l2l", "p2p_l2p"]
    stage_ms = {names[i]: st[i] for i in range(6)}
    for lev in range(2, L + 1):
        stage_ms[f"m2l_level{lev}"] = st[B.FMM_TIME_M2L_LEVEL0 + lev]

    # the plain FP32 form on the same field, same run (the comparison the metric
    # names: FP32 M2L, near zone by direct sum), and the two forms between it
    # and the headline (one change each), so the speed-up can be split up
    def time_form(form_prec, form_fft, form_learned):
        fplan = B.Plan(n, L, p)
        if form_prec != B.FMM_PREC_FP32:
            fplan.set_precision(form_prec)
        if form_learned is not None:
            B.fmm_plan_set_correction(fplan.handle, w)
        if form_fft:
            B.fmm_plan_set_near_algorithm(fplan.handle, B.FMM_NEAR_FFT)
        fms, fstage, _ = _time_solves(B, fplan, rho, phi, acc, max(1, min(args.steps, 3)),
                                      max(1, min(args.warmup, 2)), l2_flush, stream, barrier)
        fm = slowest_rank_ms(statistics.mean(fms), ws, dev)
        res = {"value": whole_job_cells_per_s(ws, n, fm), "ms_per_step": fm,
               "m2l_ms": statistics.mean(s_[B.FMM_TIME_M2L] for s_ in fstage),
               "p2p_ms": statistics.mean(s_[B.FMM_TIME_P2P] for s_ in fstage),
               "device_check": device_check(B, fplan)}
        fplan.close()
        return res

    plain = None
    forms = {}
    if tc and not args.no_plain:
        plain = time_form(B.FMM_PREC_FP32, False, None)
        checks["plain_fp32"] = plain.pop("device_check")
        if near_fft:
            forms["plain_fp32_near_fft"] = time_form(B.FMM_PREC_FP32, True, None)
            forms["mixed_near_direct"] = time_form(prec, False, learned)
        # phi/acc now hold the last form's result: the timed result was
        # copied to the host (host leg) and measured (error statement) above

    peaks, src = _peaks()
    fma = measure_fp32_peak(B, dev, stream)
    fp32_peak = fma["tflops"]
    dominant = max(names, key=lambda k: stage_ms[k])
    roof_p2p = roof_near = None
    if near_fft:
        near_ach = near_fft_flops(n, L, p) / (stage_ms["p2p_l2p"] / 1000.0) / 1e12
        roof_near = {"kernel": "k_nz_fwd + k_nz_mac + k_nz_l2p + k_nz_inv (near zone by FFT and L2P; the whole stage)",
                     "bound": "alu", "achieved": near_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": near_ach / fp32_peak, "traffic": NEAR_FFT_TRAFFIC.get((n, L, p)),
                     "traffic_source": NEAR_FFT_TRAFFIC_SOURCE if NEAR_FFT_TRAFFIC.get((n, L, p)) else None,
                     "peak_source": "measured (of measured): " + fma["how"]}
    else:
        p2p_ach = p2p_flops(n, L) / (stage_ms["p2p_l2p"] / 1000.0) / 1e12
        traffic = P2P_TRAFFIC.get((n, L, p))
        roof_p2p = {"kernel": "k_p2p (fused L2P + near-zone sum)", "bound": "alu", "achieved": p2p_ach,
                    "peak": fp32_peak, "unit": "TFLOP/s", "frac": p2p_ach / fp32_peak,
                    "traffic": traffic, "traffic_source": P2P_TRAFFIC_SOURCE if traffic else None,
                    "peak_source": "measured (of measured): " + fma["how"], "fp32_probe": fma}
    roof_m2l = None
    if tc:
        # the leaf level's launch: the longest single launch of the mixed forms
        tc_ms = stage_ms[f"m2l_level{L}"]
        alg = 2.0 * 4 * p ** 3 * p ** 3 * 189 * 8 ** L
        ach = alg / (tc_ms / 1000.0) / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        traffic = M2L_TC_TRAFFIC.get((n, L, p))
        roof_m2l = {"kernel": f"k_m2l_tc (level {L}, one launch)", "bound": "tensor",
                    "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                    "traffic_source": M2L_TC_TRAFFIC_SOURCE if traffic else None,
                    "executed_tflops": ach * (3 if prec == B.FMM_PREC_BF16X3 else 1),
                    "executed_frac": ach * (3 if prec == B.FMM_PREC_BF16X3 else 1) / peak,
                    "peak_source": f"bf16_tflops_sustained ({src}, of measured); achieved counts the algorithmic "
                                   "contraction (2 x 4p^3 x p^3 x 189 flop per node), bf16x3 executes 3 MMAs per "
                                   "product"}
    if near_fft:
        roof = roof_m2l if roof_m2l is not None else roof_near
    else:
        roof = roof_p2p if (dominant == "p2p_l2p" or roof_m2l is None) else roof_m2l

    # end to end through the public host-buffer entry point
    hin = torch.from_numpy(rho_host).pin_memory()
    hphi = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    hacc = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    B.fmm_solve_host(plan.handle, hin, hphi, hacc, stream)
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.fmm_solve_host(plan.handle, hin, hphi, hacc, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    checks["e2e"] = device_check(B, plan)
    plan.close()

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if not tc else ("bf16x3" if prec == B.FMM_PREC_BF16X3 else "bf16"),
        "data": "synthetic",
        "config": dict(headline_config(args, learned, ws), tc_tiles=tc_tiles),
        "stage_ms": stage_ms,
        "stage_ms_source": "two solves with the library's stage timing on, which runs the stages one after another; "
                           "the timed steps overlap the CUDA-core M2L levels and the near zone's forward transform "
                           "with the tensor-core levels",
        "wall_s": wall,
        "roofline": roof,
        "roofline_p2p": roof_p2p,
        "roofline_near_fft": roof_near,
        "roofline_m2l": roof_m2l,
        "e2e": {"value": ws * n ** 3 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * n ** 3,
                "d2h_bytes_per_step": 16 * n ** 3},
        "gpu_launches": launches_per_solve(L, tc, p, near_fft) * args.steps,
        "solve_roofline": solve_roofline(n, L, p, tc, ms, peaks, fp32_peak, near_fft),
        "clocks": clocks,
        "error_statement": statement,
        "device_checks": checks,
    }
    if plain is not None:
        line["plain_fp32"] = plain
        line["speedup_vs_plain_fp32"] = plain["ms_per_step"] / ms
    if forms:
        line["forms"] = forms
    if host_leg:
        line["cpu_baseline"] = cpu_baseline()
        refs = pm_references(rho_host)
        line["accuracy"] = accuracy_vs_pm(refs, result_phi, result_acc)
        if gain is not None:
            _, gphi, gacc = gain.pop("without_correction_host_pm")
            gain["whole_mesh"] = {"with_correction": line["accuracy"],
                                  "without_correction": accuracy_vs_pm(refs, gphi, gacc)}
    if gain is not None:
        line["learned_gain"] = gain
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """The batching workload: 64 independent periodic fields with N drawn from
    {32, 48, 64, 96, 128}, order 4 or 6, lognormal sigma in [0.3, 1.5]
    (seeded), leaf levels autotuned, solved as one CUDA-graph launch."""
    import torch
    from paper_2011_07099_gb300 import binding as B, build, inputs
    torch.cuda.set_device(0)
    build.build()
    rng = np.random.Generator(np.random.PCG64(2000))
    nf = args.fields
    Ns = [int(x) for x in rng.choice([32, 48, 64, 96, 128], nf)]
    ps = [int(x) for x in rng.choice([4, 6], nf)]
    sig = rng.uniform(0.3, 1.5, nf)
    import tempfile
    os.environ.setdefault("FMM_AUTOTUNE_CACHE", os.path.join(tempfile.gettempdir(), "fmm_autotune.jsonl"))
    t0 = time.perf_counter()
    # with the near zone by FFT the fields whose N is 8 x a power of two take
    # 8-cell leaves (its leaf size); the others are autotuned (L = 0)
    near_fft = args.near == "fft"
    Ls = [(n // 8).bit_length() - 1 if near_fft and n % 8 == 0 and (n // 8) & (n // 8 - 1) == 0 and n >= 32 else 0
          for n in Ns]
    batch = B.Batch(Ns, Ls, ps, precision=B.FMM_PREC_BF16X3)
    if near_fft:
        B.fmm_batch_set_near_algorithm(batch.handle, B.FMM_NEAR_FFT)
    tune_s = time.perf_counter() - t0
    d = [torch.from_numpy(inputs.lognormal(n, sigma=float(s_), seed=2000 + i)).cuda() for i, (n, s_) in
         enumerate(zip(Ns, sig))]
    pots = [torch.empty((n, n, n), device="cuda") for n in Ns]
    accs = [torch.empty((3, n, n, n), device="cuda") for n in Ns]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.solve(d, pots, accs)
    torch.cuda.synchronize()
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    times = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            l2_flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.solve(d, pots, accs)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    batch.check()
    ms = statistics.mean(times)
    cells = sum(n ** 3 for n in Ns)
    line = {"metric": "FMM cells/s, batch of 64 uneven periodic fields (one graph launch)", "value": cells / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": f"{nf} fields, N in {{32,48,64,96,128}}, p in {{4,6}}, lognormal sigma U[0.3,1.5]"
                                   + (", near zone by FFT where the leaves hold 8 cells" if near_fft else ""),
                       "cells": cells, "levels": batch.levels, "N": Ns, "order": ps, "autotune_s": tune_s},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def run_full512(args):
    """The full-scale workload: 512^3 (134M cells), order 8, L = 6 (S = 8),
    density 1 + lognormal(sigma 1.5) plus 4096 Plummer clumps; the mixed form
    (tensor-core bf16x3 M2L) against the plain FP32 form, errors against PM
    with G_S1 (libfmm mesh Green's function + cuFFT)."""
    import torch
    from paper_2011_07099_gb300 import binding as B, build, inputs, learn
    torch.cuda.set_device(0)
    build.build()
    n, L, p = 512, 6, 8
    dev = torch.device("cuda", 0)
    rho = inputs.config_density_torch(4, dev)
    out = {}
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    tphi, tacc = learn.pm_target(rho, n)
    with ClockSampler(0) as clk:
        for name, prec in (("mixed_bf16x3", B.FMM_PREC_BF16X3), ("plain_fp32", B.FMM_PREC_FP32)):
            plan = B.Plan(n, L, p)
            if prec:
                plan.set_precision(prec)
            if prec != B.FMM_PREC_FP32 and args.near == "fft":
                B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_FFT)   # the plain form keeps the direct sum
            phi = torch.empty((n, n, n), device=dev)
            acc = torch.empty((3, n, n, n), device=dev)
            ms, stage, _ = _time_solves(B, plan, rho, phi, acc, args.steps, max(1, args.warmup), l2_flush, stream,
                                        lambda: None)
            e_phi = float(((phi.double() - tphi.double()) ** 2).sum().sqrt() / (tphi.double() ** 2).sum().sqrt())
            e_g = float(((acc.double() - tacc.double()) ** 2).sum().sqrt() / (tacc.double() ** 2).sum().sqrt())
            st = [statistics.mean(s_[i] for s_ in stage) for i in range(len(stage[0]))]
            out[name] = {"ms_per_step": statistics.mean(ms), "cells_per_s": n ** 3 / (statistics.mean(ms) / 1e3),
                         "m2l_ms": st[B.FMM_TIME_M2L], "p2p_ms": st[B.FMM_TIME_P2P],
                         "vs_pm_gs1": {"phi": e_phi, "g": e_g}, "device_check": device_check(B, plan)}
            plan.close()
            del phi, acc
    line = {"metric": "FMM cells/s at 512^3 p=8 (full scale)", "value": out["mixed_bf16x3"]["cells_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["mixed_bf16x3"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": "512^3, p=8, L=6 (S=8), 1 + lognormal(sigma=1.5) + 4096 Plummer clumps; mixed form: "
                                   "bf16x3 leaf-level M2L, bf16x6 level 5 (FP64 fields), double-float levels 2-4"
                                   + (", near zone by FFT" if args.near == "fft" else ""),
                       "forms": out}, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--precision", choices=["fp32", "bf16", "bf16x3"], default="bf16x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP32 form")
    ap.add_argument("--workload", choices=["headline", "batch", "full512"], default="headline")
    ap.add_argument("--fields", type=int, default=64)
    ap.add_argument("--correction", default=None,
                    help="weights (.npz with 'w') of the learned table correction for the mixed form; "
                         "default: the trained order-6 weights shipped with the package, when p = 6")
    ap.add_argument("--no-correction", action="store_true", help="time the mixed form without the correction")
    ap.add_argument("--near", choices=["fft", "direct"], default="fft",
                    help="near zone of the timed form: FFT convolution on the doubled grid (Sec. 3; 8-cell "
                         "leaves) or the direct sum; the plain FP32 form always uses the direct sum")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "full512":
        return run_full512(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
