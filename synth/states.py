"""Seeded cell states (T, p, Y) for the workloads the paper's cases stand for.

Layout: T[n], p[n] (Pa) and Y[nsp, n] species-major, all float64.

* ``uniform_states``: T ~ U[300, 2500] K, p = 1 atm, Y ~ Dirichlet(0.5)
  (the 10-species / 1024-cell case and the batched meshes).
* ``bimodal_states``: the 262,144-cell, 20 bar case that mimics a
  partially burnt flow field (the paper's shear layer and spray, whose
  fields are not available): 45 % cold ambient cells drawn from 8 ambient
  states (T ~ U[300, 600], fixed Dirichlet Y) with relative noise 2e-5,
  45 % burnt cells taken from stored near-equilibrium base states with
  relative noise 1e-6, and 10 % flame-front cells with T ~ U[900, 1600] and
  Dirichlet Y. The classes are interleaved in random order, as spatial
  mixing would leave them.
"""
from __future__ import annotations

import os

import numpy as np

P_ATM = 101325.0
DATA = os.path.join(os.path.dirname(__file__), "data")
COLD, BURNT, FRONT = 0, 1, 2


def mech_path(nsp: int, nrx: int, seed: int) -> str:
    return os.path.join(DATA, f"mech_{nsp}_{nrx}_s{seed}.bin")


def burnt_base_path(nsp: int, nrx: int, seed: int) -> str:
    return os.path.join(DATA, f"burnt_base_{nsp}_{nrx}_s{seed}.npz")


def _renorm(Y: np.ndarray) -> np.ndarray:
    return Y / Y.sum(axis=0, keepdims=True)


def uniform_states(nsp: int, n: int, seed: int, p: float = P_ATM,
                   Tlo: float = 300.0, Thi: float = 2500.0):
    rng = np.random.default_rng(seed)
    T = rng.uniform(Tlo, Thi, n)
    Y = np.ascontiguousarray(rng.dirichlet(np.full(nsp, 0.5), size=n).T)
    return T, np.full(n, float(p)), Y


def burnt_seed_states(nsp: int, nbase: int, seed: int):
    """Starting points that are equilibrated at frozen T to make burnt bases."""
    rng = np.random.default_rng(seed + 7919)
    T = rng.uniform(1800.0, 2300.0, nbase)
    Y = np.ascontiguousarray(rng.dirichlet(np.full(nsp, 0.5), size=nbase).T)
    return T, Y


def bimodal_states(nsp: int, nrx: int, n: int, seed: int, p: float = 20e5,
                   n_ambient: int = 8, cold_noise: float = 2e-5, burnt_noise: float = 1e-6,
                   mech_seed: int = 0):
    """seed draws the field; mech_seed names the mechanism whose stored burnt
    base states are used."""
    path = burnt_base_path(nsp, nrx, mech_seed)
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} missing: it is written by oracle/make_burnt_base.py")
    base = np.load(path)
    Tb, Yb = base["T"], base["Y"]
    rng = np.random.default_rng(seed)
    ncold = int(round(0.45 * n))
    nburnt = int(round(0.45 * n))
    nfront = n - ncold - nburnt
    cls = np.concatenate([np.full(ncold, COLD), np.full(nburnt, BURNT), np.full(nfront, FRONT)])
    cls = cls[rng.permutation(n)].astype(np.int32)
    T = np.empty(n)
    Y = np.empty((nsp, n))
    # cold ambient
    Ta = rng.uniform(300.0, 600.0, n_ambient)
    Ya = rng.dirichlet(np.full(nsp, 0.5), size=n_ambient).T
    ic = np.flatnonzero(cls == COLD)
    which = rng.integers(n_ambient, size=ic.size)
    T[ic] = Ta[which] * (1.0 + rng.uniform(-cold_noise, cold_noise, ic.size))
    Y[:, ic] = _renorm(Ya[:, which] * (1.0 + rng.uniform(-cold_noise, cold_noise, (nsp, ic.size))))
    # burnt near-equilibrium
    ib = np.flatnonzero(cls == BURNT)
    which = rng.integers(Tb.size, size=ib.size)
    T[ib] = Tb[which] * (1.0 + rng.uniform(-burnt_noise, burnt_noise, ib.size))
    Y[:, ib] = _renorm(Yb[:, which] * (1.0 + rng.uniform(-burnt_noise, burnt_noise, (nsp, ib.size))))
    # flame front
    iff = np.flatnonzero(cls == FRONT)
    T[iff] = rng.uniform(900.0, 1600.0, iff.size)
    Y[:, iff] = rng.dirichlet(np.full(nsp, 0.5), size=iff.size).T
    return T, np.full(n, float(p)), np.ascontiguousarray(Y), cls


def temperature_class(T: np.ndarray) -> np.ndarray:
    """Cell class by temperature: 0 below 900 K, 1 above 1600 K, 2 between."""
    c = np.full(T.shape, FRONT, dtype=np.int32)
    c[T < 900.0] = COLD
    c[T > 1600.0] = BURNT
    return c


def stratified_sample(cls: np.ndarray, per_class: int, seed: int) -> np.ndarray:
    """Sorted indices: up to ``per_class`` random cells from every class."""
    rng = np.random.default_rng(seed + 104729)
    out = []
    for c in np.unique(cls):
        idx = np.flatnonzero(cls == c)
        take = min(per_class, idx.size)
        out.append(rng.choice(idx, size=take, replace=False))
    return np.sort(np.concatenate(out))


def log_uniform_dt(n: int, seed: int, lo: float = 1e-6, hi: float = 1e-5) -> np.ndarray:
    rng = np.random.default_rng(seed + 15485863)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))
