"""Seeded synthetic element-balanced mechanisms.

Recipe (the paper names a 54-species n-dodecane mechanism that is not
available here; these mechanisms stand in for its size and structure):

* Species are atom vectors over (C, H, O, N) with counts 0..3. The set is
  grown greedily from two single-atom species: each new species is the
  candidate vector that adds the most new element-balanced pairs of
  1- or 2-species multisets, ties broken by the seeded generator. This gives
  the small-lattice structure of real mechanisms (H, O, OH, H2O, HO2, ...)
  so that even 10 species carry 20+ balanced reactions.
* Thermo per species: cp = a + b*T with a ~ U[25, 45] J/(mol K),
  b ~ U[0, 0.01] J/(mol K^2); h_f ~ U[-150, 50] kJ/mol; s0 = 100 + 40*n_atoms
  + U[-15, 15] J/(mol K). Tying s0 to the atom count (as for real species:
  H 115, OH 184, H2O 189, H2O2 233) keeps reaction entropies physical: about
  +100 J/(mol K) for A <=> B + C and about 0 for A + B <=> C + D. Entropies
  drawn independently per species give |dS| up to 40 R, equilibrium
  constants off by e^40 and reverse rate constants above 1e20 per second.
* Reactions are drawn uniformly without replacement from all pairs of
  distinct multisets with equal element sums (types A <=> B + C and
  A + B <=> C + D). round(0.1*R) of them are third-body reactions
  A + B (+M) <=> C (+M), efficiency 1 for every species.
* Each reaction is oriented so that its forward direction is exothermic at
  298.15 K (sum of nu*h_f <= 0); then A is log-uniform on [1e6, 1e14]
  (mol, cm^3, s units), beta ~ U[-1, 1], Ea ~ U[0, 200] kJ/mol.
* Every species must take part in at least one reaction; the reaction draw
  is repeated (same stream) until it does.
"""
from __future__ import annotations

import itertools

import numpy as np

from .mechfile import ATOMIC_MASS, Mechanism

_CANDIDATES = np.array([v for v in itertools.product(range(4), repeat=4) if sum(v) > 0], dtype=np.int64)


def _key(v) -> tuple:
    return tuple(int(x) for x in v)


def _grow_species(nsp: int, rng: np.random.Generator) -> np.ndarray:
    els = rng.permutation(4)[:2]
    species = [np.eye(4, dtype=np.int64)[e] for e in els]
    # count[sum] = number of 1- and 2-species multisets with that element sum
    count: dict = {}

    def add_counts(vs):
        for v in vs:
            count[_key(v)] = count.get(_key(v), 0) + 1

    add_counts([species[0], species[1], 2 * species[0], 2 * species[1], species[0] + species[1]])
    while len(species) < nsp:
        have = {_key(s) for s in species}
        best, best_gain = [], -1
        for v in _CANDIDATES:
            if _key(v) in have:
                continue
            # new multisets {v}, {v,v}, {v,s}: each pairs with every existing
            # multiset of the same sum (they cannot collide with each other)
            gain = count.get(_key(v), 0) + count.get(_key(2 * v), 0)
            for s in species:
                gain += count.get(_key(v + s), 0)
            if gain > best_gain:
                best, best_gain = [v], gain
            elif gain == best_gain:
                best.append(v)
        v = best[int(rng.integers(len(best)))]
        add_counts([v, 2 * v] + [v + s for s in species])
        species.append(v)
    return np.array(species)


def _candidate_pairs(atoms: np.ndarray):
    """All unordered pairs of distinct multisets (size 1 or 2) with equal sums."""
    nsp = len(atoms)
    groups: dict = {}
    for i in range(nsp):
        groups.setdefault(_key(atoms[i]), []).append((i,))
        for j in range(i, nsp):
            groups.setdefault(_key(atoms[i] + atoms[j]), []).append((i, j))
    pairs = []
    for key in sorted(groups):
        ms = groups[key]
        for a, b in itertools.combinations(ms, 2):
            pairs.append((a, b))
    return pairs


def _side(ms) -> list:
    out: dict = {}
    for k in ms:
        out[k] = out.get(k, 0) + 1
    return sorted(out.items())


def generate_mechanism(nsp: int, nrx: int, seed: int, tb_fraction: float = 0.1) -> Mechanism:
    rng = np.random.default_rng(seed)
    atoms = _grow_species(nsp, rng)
    W = atoms @ ATOMIC_MASS
    cp_a = rng.uniform(25.0, 45.0, nsp)
    cp_b = rng.uniform(0.0, 0.01, nsp)
    hf = rng.uniform(-150e3, 50e3, nsp)
    s0 = 100.0 + 40.0 * atoms.sum(axis=1) + rng.uniform(-15.0, 15.0, nsp)

    pairs = _candidate_pairs(atoms)
    if len(pairs) < nrx:
        raise ValueError(f"only {len(pairs)} balanced reactions exist for {nsp} species")
    one_two = [i for i, (a, b) in enumerate(pairs) if len(a) != len(b)]
    ntb = int(round(tb_fraction * nrx))
    if len(one_two) < ntb:
        raise ValueError("too few A <=> B + C candidates for the third-body share")
    for _attempt in range(1000):
        tb_sel = [one_two[i] for i in rng.choice(len(one_two), size=ntb, replace=False)]
        rest = np.setdiff1d(np.arange(len(pairs)), tb_sel)
        other = list(rng.choice(rest, size=nrx - ntb, replace=False))
        chosen = tb_sel + [int(i) for i in other]
        used = set()
        for i in chosen:
            a, b = pairs[i]
            used.update(a)
            used.update(b)
        if len(used) == nsp:
            break
    else:
        raise ValueError("could not cover every species with reactions")

    reac, prod, tb = [], [], []
    for n, i in enumerate(chosen):
        a, b = pairs[i]
        if n < ntb and len(a) == 2:     # third-body: write as A + B (+M) <=> C (+M)
            a, b = b, a
        ra, pb = _side(a), _side(b)
        dh = sum(nu * hf[k] for k, nu in pb) - sum(nu * hf[k] for k, nu in ra)
        if dh > 0.0:
            ra, pb = pb, ra
        reac.append(ra)
        prod.append(pb)
        tb.append(1 if n < ntb else 0)
    lnA = rng.uniform(np.log(1e6), np.log(1e14), nrx)
    beta = rng.uniform(-1.0, 1.0, nrx)
    Ea = rng.uniform(0.0, 200e3, nrx)
    perm = rng.permutation(nrx)   # interleave third-body and plain reactions
    return Mechanism(W=W, cp_a=cp_a, cp_b=cp_b, hf=hf, s0=s0, atoms=atoms,
                     lnA=lnA[perm], beta=beta[perm], Ea=Ea[perm],
                     reac=[reac[i] for i in perm], prod=[prod[i] for i in perm],
                     reversible=np.ones(nrx, dtype=np.int64),
                     thirdbody=np.array([tb[i] for i in perm], dtype=np.int64), eff=[])


def with_falloff(m: Mechanism, seed: int) -> Mechanism:
    """A copy of m whose third-body reactions become pressure-dependent
    (fall-off) reactions, cycling through Lindemann, three- and four-parameter
    Troe forms, each with listed efficiencies for two species. The low-
    pressure limit is drawn so that the reduced pressure is of order one at
    the concentrations of 1-20 bar: A0 = A * U[1e4, 1e6] cm^3/mol,
    beta0 = beta - U[0, 1.5], Ea0 = max(0, Ea - U[0, 20] kJ/mol); Troe
    a ~ U[0.2, 0.9], T3 ~ U[100, 500] K, T1 ~ U[1000, 3000] K, T2 ~ U[2000,
    6000] K. (Stand-in for real mechanisms' fall-off data, which is not
    available here; only the seeded draw lives in this package.)"""
    import copy
    rng = np.random.default_rng(seed + 777)
    out = copy.deepcopy(m)
    tb = np.flatnonzero(np.asarray(m.thirdbody) != 0)
    falloff, eff = [], [e for e in m.eff if e[0] not in set(tb.tolist())]
    for i, j in enumerate(tb):
        kind = 1 + i % 3
        lnA0 = m.lnA[j] + np.log(rng.uniform(1e4, 1e6))
        beta0 = m.beta[j] - rng.uniform(0.0, 1.5)
        Ea0 = max(0.0, m.Ea[j] - rng.uniform(0.0, 20e3))
        a, T3, T1, T2 = rng.uniform(0.2, 0.9), rng.uniform(100, 500), rng.uniform(1000, 3000), rng.uniform(2000, 6000)
        falloff.append((int(j), kind, lnA0, beta0, Ea0, a, T3, T1, T2))
        for k in rng.choice(m.nsp, size=2, replace=False):
            eff.append((int(j), int(k), float(rng.uniform(0.3, 3.0))))
    out.falloff = falloff
    out.eff = eff
    return out


def with_plog(m: Mechanism, seed: int, frac: float = 0.15) -> Mechanism:
    """A copy of m in which a seeded fraction of the reactions that are
    neither third-body nor fall-off become pressure-dependent Arrhenius
    (PLOG) reactions with 2-4 points at pressures drawn from 0.1-100 bar
    (sorted), each point's parameters perturbed from the reaction's own:
    A * U[0.2, 5], beta + U[-0.3, 0.3], Ea + U[-8, 8] kJ/mol (at least 0).
    (Stand-in for real mechanisms' PLOG data, which is not available here.)"""
    import copy
    rng = np.random.default_rng(seed + 4242)
    out = copy.deepcopy(m)
    fall_rx = {int(r[0]) for r in m.falloff}
    grid = np.array([1e4, 3e4, 1e5, 3e5, 1e6, 3e6, 1e7])
    plog = []
    for j in range(m.nrx):
        if m.thirdbody[j] or j in fall_rx or rng.uniform() >= frac:
            continue
        n = int(rng.integers(2, 5))
        ps = np.sort(rng.choice(grid, size=n, replace=False))
        pts = [(float(pp), float(m.lnA[j] + np.log(rng.uniform(0.2, 5.0))), float(m.beta[j] + rng.uniform(-0.3, 0.3)),
                float(max(0.0, m.Ea[j] + rng.uniform(-8e3, 8e3)))) for pp in ps]
        plog.append((j, pts))
    out.plog = plog
    return out



def nasa7_of_linear(m: Mechanism, Tmid: float = 1000.0) -> np.ndarray:
    """NASA-7 data [nsp, 17] that reproduce m's linear thermo exactly
    (cp = a + b T, h(T0) = hf, s(T0) = s0; both ranges the same)."""
    R, T0 = 8.314462618, 298.15
    out = np.zeros((m.nsp, 17))
    for k in range(m.nsp):
        a1, a2 = m.cp_a[k] / R, m.cp_b[k] / R
        a6 = T0 * (m.hf[k] / (R * T0) - a1 - a2 * T0 / 2)
        a7 = m.s0[k] / R - a1 * np.log(T0) - a2 * T0
        c = [a1, a2, 0.0, 0.0, 0.0, a6, a7]
        out[k] = [200.0, Tmid, 6000.0, *c, *c]
    return out


def with_nasa7(m: Mechanism, seed: int) -> Mechanism:
    """A copy of m with NASA-7 thermo: each species keeps h(T0) = hf and
    s(T0) = s0 and its linear cp plus curvature, cp/R += a3 T^2 + a4 T^3 +
    a5 T^4 with a3 ~ U[-2e-7, 2e-7], a4 ~ U[-5e-11, 5e-11], a5 ~ U[-5e-15, 5e-15]
    below Tmid (a few tenths of cp/R at 3000 K); above Tmid a3 changes by U[-1e-7, 1e-7] and a1 so that cp
    is continuous at Tmid, and a6, a7 so that h and s are. Tmid is 1000 K for
    most species and 1200 K for every fifth. (Stand-in for real
    mechanisms' NASA-7 data, which is not available here.)"""
    import copy
    R, T0 = 8.314462618, 298.15
    rng = np.random.default_rng(seed + 9090)
    out = copy.deepcopy(m)
    nasa = np.zeros((m.nsp, 17))

    def poly_h(c, T):   # h/(R T) without the a6 term
        return c[0] + c[1] * T / 2 + c[2] * T ** 2 / 3 + c[3] * T ** 3 / 4 + c[4] * T ** 4 / 5

    def poly_s(c, T):   # s/R without a7
        return c[0] * np.log(T) + c[1] * T + c[2] * T ** 2 / 2 + c[3] * T ** 3 / 3 + c[4] * T ** 4 / 4

    for k in range(m.nsp):
        Tmid = 1200.0 if k % 5 == 4 else 1000.0
        lo = np.zeros(7)
        lo[0], lo[1] = m.cp_a[k] / R, m.cp_b[k] / R
        lo[2:5] = rng.uniform(-2e-7, 2e-7), rng.uniform(-5e-11, 5e-11), rng.uniform(-5e-15, 5e-15)
        lo[5] = T0 * (m.hf[k] / (R * T0) - poly_h(lo, T0))
        lo[6] = m.s0[k] / R - poly_s(lo, T0)
        hi = lo.copy()
        g = rng.uniform(-1e-7, 1e-7)
        hi[2] += g
        hi[0] -= g * Tmid ** 2
        hi[5] = lo[5] + Tmid * (poly_h(lo, Tmid) - poly_h(hi, Tmid))
        hi[6] = lo[6] + poly_s(lo, Tmid) - poly_s(hi, Tmid)
        nasa[k] = [200.0, Tmid, 6000.0, *lo, *hi]
    out.nasa = nasa
    return out
