"""Training and use of the learned cost predictor / surrogate.

Host orchestration only: the training targets come from the library's FP64
integrator, and every forward, backward and optimiser step runs in the
library's BF16 tensor-core kernels (dlbchem_mlp_*). The feature definition
matches the inference kernel: x = [T/1000, ln p, Y_1..Y_nsp, ln dt],
y = [ln attempted steps, dT, dY_1..dY_nsp].
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


def generate(ctx, T, p, Y, dt_cells, device="cuda"):
    """Integrate every cell over its own dt with the FP64 integrator (cells
    grouped by dt value) and return (features, targets, steps, status)."""
    import torch
    n = T.size
    To = np.empty(n)
    Yo = np.empty_like(Y)
    steps = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    for dt in np.unique(dt_cells):
        idx = np.flatnonzero(dt_cells == dt)
        d = lambda a: torch.tensor(np.ascontiguousarray(a), device=device)
        st = torch.zeros(idx.size, dtype=torch.int32, device=device)
        ss = torch.zeros(idx.size, dtype=torch.int32, device=device)
        a, b = ctx.integrate(d(T[idx]), d(p[idx]), d(Y[:, idx]), float(dt), steps=st, status=ss)
        torch.cuda.synchronize()
        To[idx] = a.cpu().numpy()
        Yo[:, idx] = b.cpu().numpy()
        steps[idx] = st.cpu().numpy()
        status[idx] = ss.cpu().numpy()
    return features(T, p, Y, dt_cells), targets(T, Y, To, Yo, steps), steps, status


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
