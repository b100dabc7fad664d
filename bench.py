#!/usr/bin/env python
"""Benchmark: chemistry cells/s per flow step dt on one GB300 (per GPU under torchrun).

Workload (the one the metric is quoted on): 262,144 cells of a 53-species /
325-reaction synthetic mechanism, bimodal field (45 % cold ambient, 45 %
burnt near-equilibrium, 10 % flame front), p = 20 bar, dt = 1e-5 s, rtol
1e-5, atol 1e-8 (the paper's ODE tolerances, Sec. 4.1), FP64, mapping
tolerance 1e-4 on T and Y. One step is one call of the whole hot path:
mapping classification (one reference per state bucket), cost-key sort,
the persistent Rosenbrock integrator pulling cells longest-first, mapping
scatter. Cost keys are the previous call's step counts. The comparison
forms (plain FP64 without mapping, one reference cell, mixed precision) are
timed on the same field after the headline.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream; L2 is flushed (256 MB write) between timed steps.
value = cells / (device ms per step). e2e repeats the same step through the
host-buffer entry point (dlbchem_integrate_host) with the host<->device
copies inside the timed region. The CPU baseline and the reference arm time
the FP64 oracle on a bounded random sample of the same field.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import read_mech, states  # noqa: E402

NSP, NRX, SEED = 53, 325, 0
NCELLS = 262144
DT, RTOL, ATOL = 1e-5, 1e-5, 1e-8
MAP_TOL = 1e-4
HEADLINE_MAPPING = 2   # 1: one reference cell per field; 2: one reference per state bucket
METRIC = "chemistry cells/s per dt at stated T/Y error vs FP64 oracle; frac of FP64 roofline"
# FP64 peak derived from unit counts and clocks: 152 SMs x 2.07 GHz x 2 FP64
# FMA lanes per clock per SM x 2 flop (= the 1.25 TFLOP/s nominal figure).
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12
# dram__bytes_read.sum + dram__bytes_write.sum of one FP64 integrator launch
# (rosenbrock_kernel<2, false>) from ncu per integrated cell (4,040,960 B
# read, 0 written, 912 cells integrated on the 8,192-cell bimodal field with
# bucket mapping), scaled by the cells the benchmark's launch integrates; None
# whenever the kernel has changed since the capture.
INTEGRATOR_TRAFFIC_BYTES_PER_CELL = 4040960 / 912
N_F = 3   # function evaluations per Rosenbrock step (stage 4 reuses stage 3's)
PAPER_CONTEXT = ("paper (DLBFoam, arXiv 2011.07978): load balancing + reference mapping speed the CPU "
                 "chemistry step up by about 10x (Spray A, 256 MPI ranks on 2x64-core AMD EPYC Rome nodes, "
                 "FP64; chi_su 9.87 LB+RM, 2.57 LB only); context, not a target")


def flops_per_step(m) -> float:
    """Algorithmic FP64 flops of one attempted step of the 4-stage Rosenbrock
    method: (2/3) N^3 for the LU of the iteration matrix, 8 N^2 for its four
    pairs of triangular solves, n_f (25 R + 15 N_sp) for the n_f = 3 rate and
    right-hand-side evaluations, 90 R + 3 N^2 for the analytic Jacobian and
    the assembly of the iteration matrix. exp and log are not flops here;
    transcendentals_per_step counts them."""
    nsp, nrx = m.nsp, m.nrx
    N = nsp + 1
    return (2.0 / 3.0) * N**3 + 8.0 * N**2 + N_F * (25 * nrx + 15 * nsp) + 90 * nrx + 3 * N**2


def transcendentals_per_step(m) -> dict:
    """exp and log per attempted step, counted apart from the flops: a forward
    rate constant per reaction and evaluation plus a reverse one per
    reaction and evaluation and one for the Jacobian, a log per species."""
    return {"exp": (2 * N_F + 1) * m.nrx, "log": m.nsp}


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(T, p, Y, n_sample, seed, mapping=HEADLINE_MAPPING, idx=None):
    """Time the FP64 oracle on a random sample of cells (or the given cells),
    all host cores."""
    import oracle
    if idx is None:
        idx = np.sort(np.random.default_rng(seed + 99).choice(T.size, size=n_sample, replace=False))
    orc = oracle.Oracle(states.mech_path(NSP, NRX, SEED))
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = orc.integrate(T[idx], p[idx], np.ascontiguousarray(Y[:, idx]), DT, rtol=RTOL, atol=ATOL,
                        nthreads=cores, mapping=mapping, map_Ttol=MAP_TOL, map_Ytol=MAP_TOL)
    wall = time.perf_counter() - t0
    return idx, res, wall, cores


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over the ranks (the slowest rank sets the job's time);
    x itself when there is one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job cells/s: every rank integrates its own field of cells_per_rank
    (replicas, weak scaling) within the slowest rank's time per step."""
    return world * cells_per_rank / (ms_per_step / 1e3)


def reference_arm(args):
    """--impl reference: the FP64 oracle on the host cores (rank 0 only)."""
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    T, p, Y, cls = states.bimodal_states(NSP, NRX, NCELLS, SEED)
    n_sample = 384
    for w in range(args.warmup):
        cpu_oracle_sample(T, p, Y, n_sample, 1000 + w)
    walls = []
    cores = os.cpu_count() or 1
    for k in range(args.steps):
        _, _, wall, cores = cpu_oracle_sample(T, p, Y, n_sample, k)
        walls.append(wall)
    v = n_sample / (sum(walls) / len(walls))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_sample / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "bimodal 262144 cells, 53 species / 325 reactions, p 20 bar, dt 1e-5 s, "
                                   "rtol 1e-5, atol 1e-8, mapping tol 1e-4 (one reference per state bucket)",
                       "sample_cells_per_step": n_sample},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n_sample} random cells of the 262144-cell field per step"},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def conservation(mech, T, Y, To, Yo):
    """Largest changes of the linear invariants over the field (on the GPU,
    outside the timed region): |sum_k Y'_k - sum_k Y_k| per cell, and the
    relative change of each element's total sum_k a_ek Y_k / W_k."""
    import torch
    aW = torch.tensor(mech.atoms.T / mech.W[None, :], dtype=torch.float64, device=Y.device)   # [4, nsp]
    e0 = aW @ Y
    e1 = aW @ Yo
    rel = ((e1 - e0).abs() / e0.abs().clamp_min(1e-300))[e0 > 0]
    return {"mass_defect_max": float((Yo.sum(0) - Y.sum(0)).abs().max()),
            "sum_Y_minus_1_max": float((Yo.sum(0) - 1.0).abs().max()),
            "element_defect_max_rel": float(rel.max()) if rel.numel() else 0.0}


def time_form(dlbchem, mech_path, fstep, Td, pd, Yd, To, Yo, stream, *, schedule, mapping, precision, warm=1):
    """One comparison form on the full field: warm-up calls (the first gives
    the queue's cost keys), then one call timed with CUDA events."""
    import torch
    n = Td.numel()
    ctx = dlbchem.Context(mech_path, rtol=RTOL, atol=ATOL, schedule=schedule, mapping=mapping,
                          map_Ttol=MAP_TOL, map_Ytol=MAP_TOL, timing=1, precision=precision)
    steps = torch.zeros(n, dtype=torch.int32, device=Td.device)
    status = torch.zeros(n, dtype=torch.int32, device=Td.device)
    for _ in range(warm):
        ctx.integrate(Td, pd, Yd, DT, T_out=To, Y_out=Yo, steps=steps, status=status, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.integrate(Td, pd, Yd, DT, T_out=To, Y_out=Yo, steps=steps, status=status, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    integ = ctx.last_timing()["integrator_ms"]
    st = ctx.last_stats()
    total = int(steps.sum().item())
    ach = fstep * total / (integ / 1e3) / 1e12
    return {"cells_per_s": n / (ms / 1e3), "ms": ms, "integrator_ms": integ, "attempted_steps": total,
            "roofline_frac": ach / FP64_PEAK_TFLOPS, "achieved_tflops": ach, "integrated": st["integrated"],
            "mapped": st["mapped"], "failed": int((status < 0).sum().item()),
            "fp64_fallbacks": st["fp64_fallbacks"] if precision else None}


def mlp_forward_rate(dlbchem, dev, stream, n):
    """Forward pass of the 13 -> 256 -> 256 -> 256 -> 12 network on n cells
    (random weights), timed with CUDA events: TFLOP/s of its GEMMs against
    the measured BF16 peak."""
    import torch
    net = dlbchem.MLP(13, 256, 12)
    g = torch.Generator(device="cpu").manual_seed(0)
    net.set_params((torch.randn(net.nparams, generator=g) * 0.05).to(dev))
    X = torch.randn(n, 13, generator=g).to(dev)
    out = torch.empty(n, 12, dtype=torch.float32, device=dev)

    def timed(reps=5):
        for _ in range(2):
            net.forward(X, out, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            net.forward(X, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    fused = net.fused
    ms = timed()
    net.set_fused(False)
    ms_layered = timed()
    net.set_fused(True)
    flops = 2.0 * n * (13 * 256 + 2 * 256 * 256 + 256 * 12)
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(peaks))["bf16_tflops"] if os.path.exists(peaks) else 1900.0
    tf = flops / (ms / 1e3) / 1e12
    net.close()
    return {"cells": n, "ms": ms, "achieved_tflops": tf, "peak_bf16_tflops": peak, "frac": tf / peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops" if os.path.exists(peaks) else "fallback 1.9 PFLOP/s",
            "kernel": ("mlp_fused_forward_kernel (whole network per 128 rows; tcgen05.mma kind::f16, TMEM "
                       "accumulator, weights by cp.async.bulk)") if fused else "gemm_tc_kernel per layer",
            "layered_ms": ms_layered,
            "layered_kernel": "gemm_tc_kernel per layer (FP32 activations in HBM)"}


def fp64_probe(dlbchem, dev, stream):
    """Measured FP64 FMA throughput (TFLOP/s) of this GPU, best of 3 launches."""
    import torch
    out = torch.empty(152 * 8 * 256, dtype=torch.float64, device=dev)
    dlbchem.fp64_fma_probe(2000, out, stream)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = dlbchem.fp64_fma_probe(20000, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def class_errors(cls, To_h, Yo_h, idx, res, sel_mask):
    """max / p99 of |dT|/T and |dY| per cell class on the sampled cells."""
    dT = np.abs(To_h[idx] - res[0]) / res[0]
    dY = np.abs(Yo_h[:, idx] - res[1]).max(axis=0)
    err = {}
    for c, name in ((0, "cold"), (1, "burnt"), (2, "front")):
        sel = (cls[idx] == c) & sel_mask
        if sel.any():
            err[name] = {"max_rel_T": float(dT[sel].max()), "p99_rel_T": float(np.percentile(dT[sel], 99)),
                         "max_abs_Y": float(dY[sel].max()), "p99_abs_Y": float(np.percentile(dY[sel], 99)),
                         "cells": int(sel.sum())}
    return err


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dlbchem", choices=["dlbchem", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-arms", action="store_true", help="skip the comparison forms (plain, mixed, ...)")
    ap.add_argument("--schedule", default="queue", choices=["queue", "plain"])
    ap.add_argument("--mapping", type=int, default=HEADLINE_MAPPING, choices=[0, 1, 2],
                    help="0 none, 1 one reference cell, 2 one reference per state bucket")
    ap.add_argument("--ncells", type=int, default=NCELLS)
    ap.add_argument("--team-warps", type=int, default=0, choices=[0, 1, 2, 4],
                    help="warps per cell (0 = the library's automatic choice)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: FP32 LU of the iteration matrix with FP64 refinement")
    ap.add_argument("--mlp-only", type=int, default=0, metavar="CELLS",
                    help="only time the network's forward pass on CELLS rows and print its JSON")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.mlp_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        from paper_2011_07978_gb300 import dlbchem
        dev = torch.device("cuda:0")
        torch.cuda.set_device(dev)
        print(json.dumps(mlp_forward_rate(dlbchem, dev, torch.cuda.current_stream(dev), args.mlp_only)))
        return 0
    args.warmup = max(args.warmup, 3)

    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07978_gb300 import dlbchem

    n = args.ncells
    T, p, Y, cls = states.bimodal_states(NSP, NRX, n, SEED + rank)
    mech_path = states.mech_path(NSP, NRX, SEED)
    mech = read_mech(mech_path)
    sched = dlbchem.SCHED_QUEUE if args.schedule == "queue" else dlbchem.SCHED_PLAIN
    prec = 1 if args.precision == "mixed" else 0
    ctx = dlbchem.Context(mech_path, rtol=RTOL, atol=ATOL, schedule=sched,
                          mapping=args.mapping, map_Ttol=MAP_TOL, map_Ytol=MAP_TOL, timing=1,
                          team_warps=args.team_warps, precision=prec)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    Td, pd, Yd = d(T), d(p), d(Y)
    To, Yo = torch.empty_like(Td), torch.empty_like(Yd)
    steps = torch.zeros(n, dtype=torch.int32, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        ctx.integrate(Td, pd, Yd, DT, T_out=To, Y_out=Yo, steps=steps, status=status, stream=stream)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    integ_ms, launches, total_steps = [], 0, 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            ctx.integrate(Td, pd, Yd, DT, T_out=To, Y_out=Yo, steps=steps, status=status, stream=stream)
            ev[k][1].record(stream)
            integ_ms.append(ctx.last_timing()["integrator_ms"])
            st = ctx.last_stats()
            launches += st["launches"]
            total_steps += int(steps.sum().item())
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = max_over_ranks(float(np.sum(step_ms)), world, dev)
    ms_per_step = dev_ms / args.steps
    value = job_throughput(n, world, ms_per_step)

    # roofline of the integrator kernel (algorithmic flops / its event-timed duration)
    fstep = flops_per_step(mech)
    flops_launch = fstep * total_steps / args.steps
    integ_avg_ms = float(np.mean(integ_ms))
    achieved = flops_launch / (integ_avg_ms / 1e3) / 1e12
    stats = ctx.last_stats()
    status_h = status.cpu().numpy()
    cons = conservation(mech, Td, Yd, To, Yo)
    peak_measured = fp64_probe(dlbchem, dev, stream)

    # e2e: same step through the host-buffer entry point, copies inside the timed region
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    Th, ph, Yh = pin(T), pin(p), pin(Y)
    Toh, Yoh = pin(np.zeros(n)), pin(np.zeros_like(Y))
    sth = pin(steps.cpu().numpy())
    stath = pin(np.zeros(n, dtype=np.int32))
    ctx.set_options(timing=0)
    ctx.integrate_host(Th, ph, Yh, DT, Toh, Yoh, steps=sth, status=stath, stream=stream)   # warm
    e2e_walls = []
    for k in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.integrate_host(Th, ph, Yh, DT, Toh, Yoh, steps=sth, status=stath, stream=stream)
        e2e_walls.append(time.perf_counter() - t1)
    e2e_value = world * n / float(np.mean(e2e_walls))
    h2d = Th.nbytes + ph.nbytes + Yh.nbytes + sth.nbytes
    d2h = Toh.nbytes + Yoh.nbytes + sth.nbytes + stath.nbytes
    To_h, Yo_h = To.cpu().numpy(), Yo.cpu().numpy()

    map_names = {0: "none", 1: "one reference cell", 2: "one reference per state bucket"}
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64 (LU in f32, f64 refinement)",
        "data": "synthetic",
        "config": {"workload": f"bimodal {n} cells, 53 species / 325 reactions (seeded synthetic), p 20 bar, "
                               f"dt 1e-5 s, rtol 1e-5, atol 1e-8, {'FP64' if args.precision == 'fp64' else 'mixed precision'}",
                   "schedule": args.schedule, "precision": args.precision,
                   "mapping": map_names[args.mapping], "mapping_tol": MAP_TOL, "cells_per_gpu": n,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": (INTEGRATOR_TRAFFIC_BYTES_PER_CELL * stats["integrated"]
                                 if args.precision == "fp64" and INTEGRATOR_TRAFFIC_BYTES_PER_CELL else None),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per integrated cell, "
                                       "8,192-cell capture, scaled by the cells integrated per launch",
                     "kernel": "rosenbrock_kernel", "flops_per_step": fstep,
                     "flops_formula": "(2/3)N^3 + 8N^2 + 3(25R + 15Nsp) + 90R + 3N^2, N = Nsp + 1",
                     "transcendentals_per_step": transcendentals_per_step(mech),
                     "steps_per_launch": total_steps / args.steps, "launch_ms": integ_avg_ms,
                     "peak_source": "derived: 152 SMs x 2.07 GHz x 2 FP64 FMA/clk/SM x 2",
                     "peak_measured": peak_measured, "frac_of_measured": achieved / peak_measured,
                     "peak_measured_source": "dlbchem_fp64_fma_probe in this run (8 FMA chains per thread, "
                                             "152 x 8 blocks of 256 threads), best of 3"},
        "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "cells": {"integrated": stats["integrated"], "mapped": stats["mapped"],
                  "failed": int((status_h < 0).sum())},
        "conservation": cons,
        "wall_s_timed": wall,
        "paper_context": PAPER_CONTEXT,
    }
    # the network's forward pass on the field: its GEMMs on the tensor cores
    # against the BF16 peak (algorithmic 2 (13*256 + 2*256^2 + 256*12) flops per cell)
    line["mlp_forward"] = mlp_forward_rate(dlbchem, dev, stream, n)
    if not args.no_arms:
        arms = {}
        scratch_T, scratch_Y = torch.empty_like(Td), torch.empty_like(Yd)
        forms = [("plain_fp64", dict(schedule=dlbchem.SCHED_PLAIN, mapping=0, precision=0, warm=1)),
                 ("queue_one_reference_fp64", dict(schedule=dlbchem.SCHED_QUEUE, mapping=1, precision=0, warm=2)),
                 ("queue_buckets_fp64", dict(schedule=dlbchem.SCHED_QUEUE, mapping=2, precision=0, warm=2)),
                 ("queue_buckets_mixed", dict(schedule=dlbchem.SCHED_QUEUE, mapping=2, precision=1, warm=2))]
        for name, kw in forms:
            same = (kw["schedule"] == sched and kw["mapping"] == args.mapping and kw["precision"] == prec)
            if same or (kw["mapping"] == 2 and HEADLINE_MAPPING != 2):
                continue
            arms[name] = time_form(dlbchem, mech_path, fstep, Td, pd, Yd, scratch_T, scratch_Y, stream, **kw)
        line["forms"] = arms
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        # the CPU baseline: the oracle running the same method (mapping as the
        # headline) on a random sample of the field
        idx_m, res_m, cwall, cores = cpu_oracle_sample(T, p, Y, 1024, 0, mapping=args.mapping)
        # error of this field's GPU result vs the oracle: integrated cells (up
        # to 256 per class among the cells this call integrated; the cold
        # class is mostly mapped, so its integrated cells are the bucket
        # references) against the oracle integrating them; mapped cells (a
        # sample per class) against the oracle integrating them instead of
        # mapping them (the mapping approximation)
        rng = np.random.default_rng(7)
        integ = np.flatnonzero(status_h == 0)
        pick = [rng.choice(c_idx, size=min(256, c_idx.size), replace=False)
                for c_idx in (integ[cls[integ] == c] for c in (0, 1, 2)) if c_idx.size]
        idx_i = np.sort(np.concatenate(pick)) if pick else np.zeros(0, dtype=np.int64)
        idx, res, _, cores = cpu_oracle_sample(T, p, Y, 0, 1, mapping=0, idx=idx_i)
        line["error_vs_oracle"] = class_errors(cls, To_h, Yo_h, idx, res, np.ones(idx.size, dtype=bool))
        # the oracle without mapping on a random sample of the field (a baseline figure)
        idx_u, _, uwall, _ = cpu_oracle_sample(T, p, Y, 1024, 1, mapping=0)
        mapped = np.flatnonzero(status_h == 1)
        if mapped.size:
            rng = np.random.default_rng(7)
            pick = np.sort(np.concatenate([rng.choice(mapped[cls[mapped] == c], size=min(256, int((cls[mapped] == c).sum())),
                                                      replace=False) for c in (0, 1, 2) if (cls[mapped] == c).any()]))
            orc = oracle.Oracle(mech_path)
            resm = orc.integrate(T[pick], p[pick], np.ascontiguousarray(Y[:, pick]), DT, rtol=RTOL, atol=ATOL,
                                 nthreads=cores)
            line["mapped_error_vs_unmapped_oracle"] = class_errors(cls, To_h, Yo_h, pick, resm,
                                                                   np.ones(pick.size, bool))
        # single-threaded oracle on a stratified sample (cold, burnt, front), no mapping
        one = states.stratified_sample(cls, 16, 3)
        t1 = time.perf_counter()
        oracle.Oracle(mech_path).integrate(T[one], p[one], np.ascontiguousarray(Y[:, one]), DT, rtol=RTOL,
                                           atol=ATOL, nthreads=1)
        w1 = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": idx_m.size / cwall, "unit": "cells/s", "cores": cores, "kind": "oracle",
                                "sample": f"{idx_m.size} random cells of the field, mapping {map_names[args.mapping]} "
                                          f"within the sample, {cwall:.1f} s wall",
                                "no_mapping": {"value": idx_u.size / uwall, "unit": "cells/s",
                                               "sample": f"{idx_u.size} random cells, {uwall:.1f} s wall"},
                                "single_thread": {"value": one.size / w1, "unit": "cells/s",
                                                  "sample": f"{one.size} cells, 16 per class, no mapping, "
                                                            f"{w1:.1f} s wall"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
