"""Symbolic sparse-LU analysis of the iteration matrix (dlbchem_lu_stats,
host only, CPU test): its counts against a plain numpy re-derivation from the
mechanism file, the dense counts against their closed forms, and the limit
where every species is coupled to every other (sparse = dense)."""
import numpy as np
import pytest

from synth import read_mech, states
from tests import tinymech


def lib():
    from paper_2011_07978_gb300 import build, dlbchem
    build.build()
    return dlbchem


def _by_hand(path):
    m = read_mech(path)
    nsp, N = m.nsp, m.nsp + 1
    A = np.eye(nsp, dtype=bool)
    effs = {}
    for j, k, e in m.eff:
        effs.setdefault(j, []).append(k)
    for r in range(m.nrx):
        nu = {}
        for k, v in m.reac[r]:
            nu[k] = nu.get(k, 0) - v
        for k, v in m.prod[r]:
            nu[k] = nu.get(k, 0) + v
        dep = [k for k, _ in m.reac[r]] + ([k for k, _ in m.prod[r]] if m.reversible[r] else [])
        if m.thirdbody[r]:
            dep += effs.get(r, [])
        for k, v in nu.items():
            if v != 0:
                for j in dep:
                    A[k, j] = A[j, k] = True
    nnz = int(A.sum())
    done = np.zeros(nsp, bool)
    lu = tri = filled = 0
    for _ in range(nsp):
        deg = [(int((A[v] & ~done).sum()) - 1, v) for v in range(nsp) if not done[v]]
        d, v = min(deg)
        nb = [u for u in range(nsp) if u != v and not done[u] and A[v, u]]
        for a in nb:
            for b in nb:
                A[a, b] = True
        lu += (len(nb) + 1) ** 2
        tri += 2 * (len(nb) + 1)
        filled += 2 * len(nb) + 1
        done[v] = True
    lu_dense = sum((N - 1 - k) ** 2 for k in range(N))
    rank1 = tri + N + 8 * N
    return dict(N=N, block_nnz=nnz, factor_nnz=filled, lu_dense=lu_dense, lu_sparse=lu, solve_dense=N * (N - 1),
                solve_sparse=tri, rank1=rank1, step_dense=lu_dense + 4 * N * (N - 1), step_sparse=lu + 4 * tri + rank1)


@pytest.mark.parametrize("mech", [(10, 20), (53, 325)])
def test_counts_match_a_rederivation(mech):
    path = states.mech_path(*mech, 0)
    got = lib().lu_stats(path)
    assert got == _by_hand(path)
    N = mech[0] + 1
    assert got["lu_dense"] == (N - 1) * N * (2 * N - 1) // 6          # sum of squares
    assert got["lu_sparse"] <= got["lu_dense"]
    print(mech, got)


def test_fully_coupled_mechanism_gives_the_dense_count(tmp_path):
    """A + B + C <=> D couples every species to every other: no sparsity."""
    sp = [dict(atoms=(1, 0, 0, 0), hf=0.0, s0=150.0, a=30.0, b=0.0),
          dict(atoms=(0, 1, 0, 0), hf=0.0, s0=150.0, a=30.0, b=0.0),
          dict(atoms=(0, 0, 1, 0), hf=0.0, s0=150.0, a=30.0, b=0.0),
          dict(atoms=(1, 1, 1, 0), hf=-100e3, s0=300.0, a=60.0, b=0.0)]
    path = tmp_path / "full.bin"
    tinymech.make(path, sp, [dict(reac=[(0, 1), (1, 1), (2, 1)], prod=[(3, 1)], lnA=np.log(1e10))])
    got = lib().lu_stats(str(path))
    assert got["block_nnz"] == 16 and got["factor_nnz"] == 16
    assert got["lu_sparse"] == got["lu_dense"] and got["solve_sparse"] == got["solve_dense"]
