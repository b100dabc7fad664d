"""The batched uneven launch at full size (configuration C4): meshes of
65,536 cells (53 species / 325 reactions, dt 1e-6 s), 262,144 cells (100 /
1000, dt 1e-5 s) and 1,048,576 cells (53 / 325, dt 1e-5 s), states as for
the 10-species case, rtol 1e-6, atol 1e-10, one captured CUDA graph with the
autotuned team size and queue chunk per mechanism. It takes about twenty
minutes of GPU time, so it runs only with DLBCHEM_C4_FULL=1. It prints one
JSON line (tuner choice, time of one replay, cells/s) and checks 256 sampled
cells of every mesh against the oracle."""
import json
import os
import time

import numpy as np
import pytest

import oracle
from synth import states
from tests.test_gpu_parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("DLBCHEM_C4_FULL") != "1", reason="full-size C4: DLBCHEM_C4_FULL=1")]
DEV = "cuda:0"


def test_c4_full_size_graph_against_oracle():
    from paper_2011_07978_gb300 import build, dlbchem as d
    build.build()
    m53, m100 = states.mech_path(53, 325, 0), states.mech_path(100, 1000, 1)
    spec = [(m53, 53, 65536, 1e-6, 41), (m100, 100, 262144, 1e-5, 42), (m53, 53, 1048576, 1e-5, 43)]
    dd = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
    b = d.Batch(rtol=1e-6, atol=1e-10)
    meshes = []
    for mech, nsp, n, dt, seed in spec:
        T, p, Y = states.uniform_states(nsp, n, seed)
        a = dict(T=dd(T), p=dd(p), Y=dd(Y), To=torch.empty(n, dtype=torch.float64, device=DEV),
                 Yo=torch.empty((nsp, n), dtype=torch.float64, device=DEV),
                 st=torch.zeros(n, dtype=torch.int32, device=DEV), ss=torch.zeros(n, dtype=torch.int32, device=DEV))
        b.add(mech, a["T"], a["p"], a["Y"], dt, a["To"], a["Yo"], steps=a["st"], status=a["ss"])
        meshes.append((mech, nsp, n, dt, a))
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    b.tune(sample_cells=1024, stream=stream)
    tune_s = time.perf_counter() - t0
    b.capture(stream)
    info = [b.info(c) for c in range(2)]
    b.launch(stream)                                  # first replay: index order, fills the cost keys
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.launch(stream)                                  # timed replay: longest first by the first one's steps
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    cells = sum(n for _, _, n, _, _ in meshes)
    steps = int(sum(int(a["st"].sum()) for *_, a in meshes))
    line = {"config": "C4 full size: 65536 (53/325, dt 1e-6) + 262144 (100/1000, dt 1e-5) + 1048576 "
                      "(53/325, dt 1e-5) cells, uniform states, rtol 1e-6, atol 1e-10, FP64, one graph",
            "classes": info, "tune_s": tune_s, "replay_ms": ms, "cells_per_s": cells / (ms / 1e3),
            "attempted_steps": steps, "failed_cells": int(sum(int((a["ss"] < 0).sum()) for *_, a in meshes))}
    errs = []
    for mech, nsp, n, dt, a in meshes:
        assert (a["ss"] == 0).all()
        idx = np.sort(np.random.default_rng(n).choice(n, size=256, replace=False))
        T0, p0, Y0 = (a[k].cpu().numpy() for k in ("T", "p", "Y"))
        orc = oracle.Oracle(mech)
        o = orc.integrate(T0[idx], p0[idx], Y0[:, idx], dt, rtol=1e-6, atol=1e-10)
        tight = orc.integrate(T0[idx], p0[idx], Y0[:, idx], dt, rtol=1e-10, atol=1e-16)
        g = (a["To"].cpu().numpy()[idx], a["Yo"].cpu().numpy()[:, idx], a["st"].cpu().numpy()[idx],
             a["ss"].cpu().numpy()[idx])
        dT, dY, frac = assert_parity(g, o, min_tight=0.95, tight_ref=tight[:2])
        errs.append({"cells": n, "max_rel_T": dT, "max_abs_Y": dY, "within_1e-9": frac})
    line["error_vs_oracle"] = errs
    print(json.dumps(line), flush=True)
    b.close()
