"""Batched uneven launch: several meshes over two mechanisms in one CUDA graph.

Three meshes of uneven sizes over the 53-species / 325-reaction and the
100-species / 1000-reaction mechanisms (65,536 cells of 53/325 at dt 1e-6 s,
262,144 of 100/1000 at 1e-5 s, 1,048,576 of 53/325 at 1e-5 s, all divided by
--scale), states drawn as for the 10-species case (T U[300, 2500] K,
Dirichlet(0.5) Y, 1 atm). The autotuner picks team size and queue chunk per
mechanism class, the graph is captured once and replayed; the same cells are
also integrated by one dlbchem_integrate call per mesh in sequence (each
with the team size the tuner chose) for the comparison. Prints one JSON line.

    python -m paper_2011_07978_gb300.batched [--scale 16]
"""
from __future__ import annotations

import numpy as np

from . import dlbchem


def main(argv=None):
    import argparse
    import json
    import time

    import torch

    from synth import states
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=16, help="divide every mesh's cell count by this")
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--atol", type=float, default=1e-10)
    ap.add_argument("--replays", type=int, default=2)
    args = ap.parse_args(argv)
    dev = torch.device("cuda")
    m53, m100 = states.mech_path(53, 325, 0), states.mech_path(100, 1000, 1)
    spec = [(m53, 53, 65536 // args.scale, 1e-6, 41), (m100, 100, 262144 // args.scale, 1e-5, 42),
            (m53, 53, 1048576 // args.scale, 1e-5, 43)]
    dd = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    b = dlbchem.Batch(rtol=args.rtol, atol=args.atol)
    meshes = []
    for mech, nsp, n, dt, seed in spec:
        T, p, Y = states.uniform_states(nsp, n, seed)
        a = dict(T=dd(T), p=dd(p), Y=dd(Y), To=torch.empty(n, dtype=torch.float64, device=dev),
                 Yo=torch.empty((nsp, n), dtype=torch.float64, device=dev),
                 st=torch.zeros(n, dtype=torch.int32, device=dev), ss=torch.zeros(n, dtype=torch.int32, device=dev))
        b.add(mech, a["T"], a["p"], a["Y"], dt, a["To"], a["Yo"], steps=a["st"], status=a["ss"])
        meshes.append((mech, nsp, n, dt, a))
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    b.tune(sample_cells=1024, stream=stream)
    tune_s = time.perf_counter() - t0
    b.capture(stream)
    info = [b.info(c) for c in range(2)]
    b.launch(stream)                       # warm-up; fills steps[] (the next replay's cost keys)
    stream.synchronize()
    graph_ms = []
    for _ in range(args.replays):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.launch(stream)
        e1.record(stream)
        stream.synchronize()
        graph_ms.append(e0.elapsed_time(e1))
    steps_total = int(sum(int(a["st"].sum()) for *_, a in meshes))
    failed = int(sum(int((a["ss"] < 0).sum()) for *_, a in meshes))
    # the same cells, one call per mesh in sequence, each with the tuned team size and queue
    seq_ms = 0.0
    identical = True
    for mech, nsp, n, dt, a in meshes:
        i = info[0 if mech == m53 else 1]
        ctx = dlbchem.Context(mech, rtol=args.rtol, atol=args.atol, team_warps=i["team_warps"],
                              schedule=dlbchem.SCHED_QUEUE, chunk=i["chunk"])
        st = a["st"].clone()
        ctx.integrate(a["T"], a["p"], a["Y"], dt, steps=st)          # warm-up, cost keys
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        To, Yo = ctx.integrate(a["T"], a["p"], a["Y"], dt, steps=st)
        e1.record()
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
        identical &= bool(torch.equal(To, a["To"]) and torch.equal(Yo, a["Yo"]))
    cells = sum(n for _, _, n, _, _ in meshes)
    g = float(np.mean(graph_ms))
    line = {"config": f"batched uneven launch: meshes {[n for _, _, n, _, _ in meshes]} cells "
                      f"(53/325 dt 1e-6, 100/1000 dt 1e-5, 53/325 dt 1e-5; the full sizes divided by {args.scale}), "
                      f"T U[300,2500] K, Dirichlet Y, 1 atm, rtol {args.rtol}, atol {args.atol}, FP64",
            "classes": info, "tune_s": tune_s,
            "graph": {"ms": g, "cells_per_s": cells / (g / 1e3), "replays_ms": graph_ms},
            "sequential_calls": {"ms": seq_ms, "cells_per_s": cells / (seq_ms / 1e3)},
            "graph_speedup": seq_ms / g, "identical_to_single_calls": identical,
            "attempted_steps": steps_total, "failed_cells": failed}
    b.close()
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
