"""Write the near-equilibrium base states of the bimodal 262,144-cell workload.

Burnt cells of that workload stand for the fully reacted regions of the
paper's shear-layer and spray cases (Sec. 4). Each base state is a seeded
draw (T ~ U[1800, 2300] K, Dirichlet(0.5) Y) integrated by the oracle at
frozen T and p = 20 bar for 1 s, which brings it to chemical equilibrium at
that T. The input generator then perturbs these bases by a relative 1e-6.

Usage: python -m oracle.make_burnt_base [nsp nrx seed nbase]
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from synth import states  # noqa: E402


def make(nsp: int = 53, nrx: int = 325, seed: int = 0, nbase: int = 64) -> str:
    orc = oracle.Oracle(states.mech_path(nsp, nrx, seed))
    T, Y = states.burnt_seed_states(nsp, nbase, seed)
    Tout, Yout, steps, status = orc.integrate(T, 20e5, Y, 1.0, rtol=1e-8, atol=1e-14, isothermal=True)
    if (status != 0).any():
        raise RuntimeError(f"equilibration failed: {np.unique(status, return_counts=True)}")
    path = states.burnt_base_path(nsp, nrx, seed)
    np.savez(path, T=Tout, Y=Yout / Yout.sum(axis=0, keepdims=True), steps=steps)
    return path


if __name__ == "__main__":
    args = [int(a) for a in sys.argv[1:]]
    print(make(*args))
