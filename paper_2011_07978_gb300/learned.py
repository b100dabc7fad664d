"""Training and use of the learned cost predictor / surrogate.

Host orchestration only: the training targets come from the library's FP64
integrator, and every forward, backward and optimiser step runs in the
library's BF16 tensor-core kernels (dlbchem_mlp_*). The feature definition
matches the inference kernel: x = [T/1000, ln p, Y_1..Y_nsp, ln dt],
y = [ln attempted steps, dT, dY_1..dY_nsp]. A residual network instead
learns the increment minus the explicit Euler step dt f(y) (f from
dlbchem_rhs); the gate then tries y + dt f(y) + its output (surrogate = 2).
"""
from __future__ import annotations

import numpy as np

from . import dlbchem

N_HIDDEN = 256


def features(T, p, Y, dt):
    """[n, nsp + 3] float32 network inputs (physical, not normalised)."""
    n = T.size
    x = np.empty((n, Y.shape[0] + 3), dtype=np.float32)
    x[:, 0] = T * 1e-3
    x[:, 1] = np.log(p)
    x[:, 2:-1] = Y.T
    x[:, -1] = np.log(dt)
    return x


def targets(T, Y, To, Yo, steps):
    n = T.size
    y = np.empty((n, Y.shape[0] + 2), dtype=np.float32)
    y[:, 0] = np.log(np.maximum(steps, 1))
    y[:, 1] = To - T
    y[:, 2:] = (Yo - Y).T
    return y


def generate(ctx, T, p, Y, dt_cells, device="cuda", residual=False):
    """Integrate every cell over its own dt with the FP64 integrator (cells
    grouped by dt value) and return (features, targets, steps, status). With
    residual, the increment targets are the increments minus dt f(y)."""
    import torch
    n = T.size
    To = np.empty(n)
    Yo = np.empty_like(Y)
    steps = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    euler_T = np.zeros(n)
    euler_Y = np.zeros_like(Y)
    for dt in np.unique(dt_cells):
        idx = np.flatnonzero(dt_cells == dt)
        d = lambda a: torch.tensor(np.ascontiguousarray(a), device=device)
        st = torch.zeros(idx.size, dtype=torch.int32, device=device)
        ss = torch.zeros(idx.size, dtype=torch.int32, device=device)
        Td, pd, Yd = d(T[idx]), d(p[idx]), d(Y[:, idx])
        a, b = ctx.integrate(Td, pd, Yd, float(dt), steps=st, status=ss)
        if residual:
            fT, fY = ctx.rhs(Td, pd, Yd)
            euler_T[idx] = float(dt) * fT.cpu().numpy()
            euler_Y[:, idx] = float(dt) * fY.cpu().numpy()
        torch.cuda.synchronize()
        To[idx] = a.cpu().numpy()
        Yo[:, idx] = b.cpu().numpy()
        steps[idx] = st.cpu().numpy()
        status[idx] = ss.cpu().numpy()
    y = targets(T, Y, To, Yo, steps)
    if residual:
        y[:, 1] -= euler_T
        y[:, 2:] -= euler_Y.T
    return features(T, p, Y, dt_cells), y, steps, status


def dt_buckets(n, seed, nbuckets=64, lo=1e-6, hi=1e-5):
    """dt log-uniform on [lo, hi], drawn from nbuckets log-spaced values."""
    rng = np.random.default_rng(seed + 15485863)
    grid = np.exp(np.linspace(np.log(lo), np.log(hi), nbuckets))
    return grid[rng.integers(nbuckets, size=n)]


def normalisation(X, Y):
    mu_x, sd_x = X.mean(0), X.std(0)
    mu_y, sd_y = Y.mean(0), Y.std(0)
    sd_x = np.where(sd_x > 1e-12, sd_x, 1.0).astype(np.float32)
    sd_y = np.where(sd_y > 1e-12, sd_y, 1.0).astype(np.float32)
    return mu_x.astype(np.float32), sd_x, mu_y.astype(np.float32), sd_y


def init_params(n_in, n_out, seed, n_hidden=N_HIDDEN):
    """He-normal weights, zero biases, flat [W1 b1 ... W4 b4] (float32)."""
    rng = np.random.default_rng(seed)
    dims = [n_in, n_hidden, n_hidden, n_hidden, n_out]
    parts = []
    for a, b in zip(dims[:-1], dims[1:]):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / a), a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def train(X, Y, epochs=10, batch=4096, lr=1e-3, seed=0, device="cuda", log=None):
    """Train a fresh network on (X, Y) (physical units) with the library's
    kernels; returns the dlbchem.MLP with its normalisation set."""
    import torch
    n_in, n_out = X.shape[1], Y.shape[1]
    mu_x, sd_x, mu_y, sd_y = normalisation(X, Y)
    Xn = ((X - mu_x) / sd_x).astype(np.float32)
    Yn = ((Y - mu_y) / sd_y).astype(np.float32)
    perm = np.random.default_rng(seed).permutation(X.shape[0])
    Xd = torch.tensor(Xn[perm], device=device)
    Yd = torch.tensor(Yn[perm], device=device)
    net = dlbchem.MLP(n_in, N_HIDDEN, n_out)
    net.set_params(torch.tensor(init_params(n_in, n_out, seed), device=device))
    net.set_norm(mu_x, sd_x, mu_y, sd_y)
    loss = torch.zeros(1, dtype=torch.float32, device=device)
    nb = X.shape[0] // batch
    history = []
    for ep in range(epochs):
        lr_ep = lr * (0.5 ** (ep // max(1, epochs // 3)))
        acc = 0.0
        for b in range(nb):
            net.train_step(Xd[b * batch:(b + 1) * batch], Yd[b * batch:(b + 1) * batch], lr_ep, loss=loss)
            if b % 16 == 0:
                acc += float(loss.item())
        history.append(acc / max(1, (nb + 15) // 16))
        if log:
            log(f"epoch {ep}: mean loss {history[-1]:.4e}")
    net.history = history
    return net


def evaluate(mech, nets, T, p, Y, dt_cells, rtol=1e-6, atol=1e-10, device="cuda"):
    """Cells/s of the queue without a network (index order: a fresh field has
    no previous steps), with the predictor, and with predictor + surrogate,
    on the same cells (grouped by dt); plus the surrogate's acceptance and
    its error against the integrated result. nets: {"increment": net,
    "residual": net} (either may be missing)."""
    import torch
    out = {}
    ref = {}
    modes = [("queue", None, dict())]
    if "increment" in nets:
        modes += [("queue+predictor", nets["increment"], dict(predictor=1)),
                  ("queue+predictor+surrogate", nets["increment"], dict(predictor=1, surrogate=1))]
    if "residual" in nets:
        modes += [("queue+predictor+residual surrogate", nets["residual"], dict(predictor=1, surrogate=2))]
    for name, net, kw in modes:
        ctx = dlbchem.Context(mech, rtol=rtol, atol=atol, schedule=dlbchem.SCHED_QUEUE, **kw)
        if net is not None:
            ctx.attach_mlp(net)
        total_ms, accepted, worst_dy, worst_dt, identical = 0.0, 0, 0.0, 0.0, True
        for dt in np.unique(dt_cells):
            idx = np.flatnonzero(dt_cells == dt)
            d = lambda a: torch.tensor(np.ascontiguousarray(a), device=device)
            Td, pd, Yd = d(T[idx]), d(p[idx]), d(Y[:, idx])
            st = torch.zeros(idx.size, dtype=torch.int32, device=device)
            ss = torch.zeros(idx.size, dtype=torch.int32, device=device)
            ctx.integrate(Td, pd, Yd, float(dt), steps=torch.zeros_like(st))          # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            To, Yo = ctx.integrate(Td, pd, Yd, float(dt), steps=st, status=ss)
            e1.record()
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            To, Yo, ss = To.cpu().numpy(), Yo.cpu().numpy(), ss.cpu().numpy()
            if name == "queue":
                ref[float(dt)] = (To, Yo)
            else:
                Tr, Yr = ref[float(dt)]
                acc = ss == dlbchem.CELL_SURROGATE
                accepted += int(acc.sum())
                integ = ~acc
                identical &= bool(np.array_equal(To[integ], Tr[integ]) and np.array_equal(Yo[:, integ], Yr[:, integ]))
                if acc.any():
                    worst_dy = max(worst_dy, float(np.abs(Yo[:, acc] - Yr[:, acc]).max()))
                    worst_dt = max(worst_dt, float((np.abs(To[acc] - Tr[acc]) / Tr[acc]).max()))
        out[name] = {"cells_per_s": T.size / (total_ms / 1e3), "ms": total_ms, "accepted": accepted,
                     "integrated_identical_to_queue": identical, "accepted_max_abs_dY": worst_dy,
                     "accepted_max_rel_dT": worst_dt}
    return out


def main(argv=None):
    """Train the network on integrator trajectories of the 10-species case
    and report what it gains on a fresh field; prints one JSON line."""
    import argparse
    import json
    import time

    import torch

    from synth import states
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-cells", type=int, default=2_000_000)
    ap.add_argument("--eval-cells", type=int, default=262_144)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    args = ap.parse_args(argv)
    mech = states.mech_path(10, 20, 0)
    ctx = dlbchem.Context(mech, rtol=1e-6, atol=1e-10, schedule=dlbchem.SCHED_QUEUE)
    T, p, Y = states.uniform_states(10, args.train_cells, 100)
    dts = dt_buckets(args.train_cells, 100)
    nets, train_info = {}, {}
    for kind in ("increment", "residual"):
        t0 = time.perf_counter()
        X, Yt, steps, status = generate(ctx, T, p, Y, dts, residual=(kind == "residual"))
        t_gen = time.perf_counter() - t0
        t0 = time.perf_counter()
        net = train(X, Yt, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=1)
        torch.cuda.synchronize()
        nets[kind] = net
        train_info[kind] = {"generate_s": t_gen, "train_s": time.perf_counter() - t0, "epochs": args.epochs,
                            "loss_first_epoch": net.history[0], "loss_last_epoch": net.history[-1],
                            "failed_cells": int((status != 0).sum())}
    Te, pe, Ye = states.uniform_states(10, args.eval_cells, 1)
    dte = dt_buckets(args.eval_cells, 1, nbuckets=8)
    ev = evaluate(mech, nets, Te, pe, Ye, dte)
    base = ev["queue"]["cells_per_s"]
    line = {"config": "learned predictor + surrogate: 10 species / 20 reactions, trained on "
                      f"{args.train_cells} integrator trajectories (T U[300,2500] K, Dirichlet Y, dt log-U "
                      "[1e-6, 1e-5] s), evaluated on a fresh field of "
                      f"{args.eval_cells} cells, gate 1e-4, FP64 fallback",
            "train": train_info, "eval": ev,
            "predictor_gain": ev["queue+predictor"]["cells_per_s"] / base,
            "surrogate_gain": ev["queue+predictor+surrogate"]["cells_per_s"] / base,
            "residual_surrogate_gain": ev["queue+predictor+residual surrogate"]["cells_per_s"] / base}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
