"""Hand-built 2-3 species mechanisms whose solutions have closed forms."""
from __future__ import annotations

import numpy as np

from synth import Mechanism, write_mech


def make(path, species, reactions, eff=(), falloff=(), plog=()):
    """species: list of dicts (atoms, hf, s0, a, b); reactions: dicts with
    reac, prod [(k, nu)], lnA, beta, Ea, rev, tb."""
    atoms = np.array([s["atoms"] for s in species])
    W = atoms @ np.array([12.011, 1.008, 15.999, 14.007])
    m = Mechanism(W=W, cp_a=np.array([s["a"] for s in species], float),
                  cp_b=np.array([s["b"] for s in species], float),
                  hf=np.array([s["hf"] for s in species], float),
                  s0=np.array([s["s0"] for s in species], float), atoms=atoms,
                  lnA=np.array([r["lnA"] for r in reactions], float),
                  beta=np.array([r.get("beta", 0.0) for r in reactions], float),
                  Ea=np.array([r.get("Ea", 0.0) for r in reactions], float),
                  reac=[r["reac"] for r in reactions], prod=[r["prod"] for r in reactions],
                  reversible=np.array([r.get("rev", 1) for r in reactions]),
                  thirdbody=np.array([r.get("tb", 0) for r in reactions]), eff=list(eff),
                  falloff=list(falloff), plog=list(plog))
    write_mech(str(path), m)
    return m
