"""Host checks of the mechanism tables (CPU only, through the C ABI).

dlbchem_table_stats builds the round tables the integrator's gathers use and
checks them against the mechanism file (every entry once, no target twice in a
round, no target in two warps, each target's entries in order). Here the
round counts are also held to bounds computed independently from the
mechanism: the whole-mechanism rounds of a one-warp team must reach the lower
bound max(largest per-target count, ceil(entries / 32)) exactly."""
from collections import Counter

import numpy as np
import pytest

from synth import mechfile, states

MECHS = [(10, 20, 0), (53, 325, 0), (100, 1000, 1)]


def dlb():
    from paper_2011_07978_gb300 import dlbchem
    try:
        dlbchem.load()
    except ImportError as e:
        pytest.skip(f"library not built: {e}")
    return dlbchem


def incidence_counts(m):
    """Per species, the number of reactions with a nonzero net coefficient."""
    nr, npd = m.nu_matrix()
    nu = npd - nr
    return (nu != 0).sum(axis=1)


@pytest.mark.parametrize("nsp,nrx,seed", MECHS)
@pytest.mark.parametrize("wpc", [1, 2, 4])
def test_tables_pass_the_host_check(nsp, nrx, seed, wpc):
    d = dlb()
    st = d.table_stats(states.mech_path(nsp, nrx, seed), wpc)
    assert st["nsp"] == nsp and st["nrx"] == nrx
    assert st["chunk_size"] == 32 * wpc and st["chunks"] == -(-nrx // (32 * wpc))
    assert st["split_off"] >= nsp + 1


@pytest.mark.parametrize("nsp,nrx,seed", MECHS)
def test_whole_mechanism_rounds_reach_the_bound(nsp, nrx, seed):
    d = dlb()
    m = mechfile.read_mech(states.mech_path(nsp, nrx, seed))
    mult = incidence_counts(m)
    n = int(mult.sum())
    for wpc in (1, 2, 4):
        st = d.table_stats(states.mech_path(nsp, nrx, seed), wpc)
        share = -(-n // (32 * wpc))
        split = mult > share
        assert st["nsplit"] == int(split.sum())
        # after splitting, a species' largest accumulator holds ceil(m/2) entries
        largest = int(np.where(split, -(-mult // 2), mult).max())
        lower = max(largest, -(-n // (32 * wpc)))
        if wpc == 1:
            assert st["all_rounds_max_warp"] == max(largest, -(-n // 32))
        else:
            assert lower <= st["all_rounds_max_warp"] <= max(largest, -(-n // 32))


def test_table_check_rejects_a_bad_path():
    d = dlb()
    with pytest.raises(d.DlbchemError):
        d.table_stats("/nonexistent/mechanism.bin", 1)
    with pytest.raises(d.DlbchemError):
        d.table_stats(states.mech_path(10, 20, 0), 3)
