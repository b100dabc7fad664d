"""Pins of the oracle's reference mapping with one reference per state bucket
(Sec. 2.3 generalised from one reference cell to one per bucket; CPU only).

Reading: a cell's bucket key is (the IEEE bits of T shifted right by s, s the
largest integer with 2^(s-52) <= T_tol; floor(Y_k / Y_tol) per species); the
reference of a bucket is its lowest-index eligible cell; another cell of the
bucket is mapped to it when it meets the Sec. 2.3 criterion against it
(max_k |Y_k - Yr_k| < Y_tol, |T - Tr| < T_tol Tr). Mapped cells take the
reference's increment, written as T' = T'_r + (T - T_r), Y' = Y'_r + (Y - Y_r).
"""
import numpy as np
import pytest

import oracle
from synth import states
from tests import tinymech

ISO = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)


def _two_species(tmp_path):
    path = tmp_path / "two.bin"
    tinymech.make(path, [ISO, ISO], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=np.log(1e3), rev=0)])
    return oracle.Oracle(str(path))


def test_worked_example(tmp_path):
    """T_tol = 0.01: s = 45, so T sits on a grid of 4 K in [512, 1024) and
    [1000, 1004) is one bin. Y_tol = 0.1: Y_1 bins of width 0.1."""
    orc = _two_species(tmp_path)
    T = np.array([1001.0, 1002.5, 1004.5, 1003.0, 1001.5, 1003.9, 1002.0, np.nan, 1000.5])
    Y1 = np.array([0.25, 0.26, 0.25, 0.29, 0.31, 0.305, 0.25, 0.25, 0.255])
    Y = np.vstack([Y1, 1 - Y1])
    ref, flag = orc.map_buckets(T, Y, 0.01, 0.1)
    # bins: 0 (T bin, 2, 7); 1 same -> 0; 2 next T bin; 3 -> 0; 4 (Y bin 3, 6); 5 -> 4;
    # 6 -> 0; 7 not finite; 8 -> 0
    np.testing.assert_array_equal(ref, [-1, 0, -1, 0, -1, 4, 0, -1, 0])
    np.testing.assert_array_equal(flag, ref >= 0)
    # below a temperature threshold only: cells with T >= 1002 are not eligible
    ref, flag = orc.map_buckets(T, Y, 0.01, 0.1, Tmax=1002.0)
    np.testing.assert_array_equal(ref, [-1, -1, -1, -1, -1, -1, -1, -1, 0])
    # T_tol = 2^-10: s = 42, the T grid is 0.5 K wide in [512, 1024) and no two
    # of these cells share a T bin, so nothing is mapped
    ref, flag = orc.map_buckets(T, Y, 2.0**-10, 0.1)
    np.testing.assert_array_equal(ref, np.full(T.size, -1))
    # the same key also requires the Sec. 2.3 criterion against the reference
    # (it can fail only within rounding of a bin edge); identical cells map
    ref, flag = orc.map_buckets(np.full(3, 1500.0), np.vstack([np.full(3, 0.4), np.full(3, 0.6)]), 1e-4, 1e-4)
    np.testing.assert_array_equal(ref, [-1, 0, 0])


def _keys(T, Y, Ttol, Ytol):
    """Bucket keys written out from the definition with numpy."""
    s = min(62, max(0, 51 + int(np.frexp(Ttol)[1])))
    kT = (T.view(np.uint64) >> np.uint64(s)).astype(np.int64)
    q = np.floor(Y * (1.0 / Ytol)).astype(np.int64)
    return np.vstack([kT[None, :], q]).T


@pytest.mark.parametrize("tol", [1e-4, 1e-3])
def test_buckets_by_brute_force_on_a_bimodal_field(orc_c2, tol):
    T, p, Y, cls = states.bimodal_states(53, 325, 3000, 9)
    ref, flag = orc_c2.map_buckets(T, Y, tol, tol)
    keys = _keys(T, Y, tol, tol)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.ravel()
    first = np.full(uniq.shape[0], T.size)
    np.minimum.at(first, inv, np.arange(T.size))
    r_expect = first[inv]
    ok = (np.abs(Y - Y[:, r_expect]).max(axis=0) < tol) & (np.abs(T - T[r_expect]) < tol * T[r_expect])
    want = (r_expect != np.arange(T.size)) & ok
    np.testing.assert_array_equal(flag.astype(bool), want)
    np.testing.assert_array_equal(ref[want], r_expect[want])
    assert (ref[~want] == -1).all()
    assert not flag[ref[want]].any()          # references are integrated, never mapped
    assert want[cls == states.COLD].mean() > 0.9 and want[cls == states.FRONT].sum() == 0


def test_mapped_cells_take_the_reference_increment(orc_c2):
    T, p, Y, cls = states.bimodal_states(53, 325, 600, 10)
    To, Yo, steps, st = orc_c2.integrate(T, p, Y, 1e-5, rtol=1e-5, atol=1e-8, mapping=2,
                                         map_Ttol=1e-4, map_Ytol=1e-4)
    ref, flag = orc_c2.map_buckets(T, Y, 1e-4, 1e-4)
    m = flag.astype(bool)
    r = ref[m]
    assert m.sum() > 100
    np.testing.assert_array_equal(To[m], To[r] + (T[m] - T[r]))
    np.testing.assert_array_equal(Yo[:, m], Yo[:, r] + (Y[:, m] - Y[:, r]))
    np.testing.assert_array_equal(st[m], oracle.ST_MAPPED)
    np.testing.assert_array_equal(steps[m], 0)
    plain = orc_c2.integrate(T, p, Y, 1e-5, rtol=1e-5, atol=1e-8)
    np.testing.assert_array_equal(To[~m], plain[0][~m])
    np.testing.assert_array_equal(Yo[:, ~m], plain[1][:, ~m])


def test_zero_tolerance_maps_nothing(orc_c1):
    T, p, Y = states.uniform_states(10, 200, 4)
    T[:50] = T[0]
    Y[:, :50] = Y[:, :1]
    for Ttol, Ytol in ((0.0, 1e-4), (1e-4, 0.0), (0.0, 0.0)):
        ref, flag = orc_c1.map_buckets(T, Y, Ttol, Ytol)
        assert flag.sum() == 0
    a = orc_c1.integrate(T, p, Y, 1e-6, mapping=2, map_Ttol=0.0, map_Ytol=0.0)
    b = orc_c1.integrate(T, p, Y, 1e-6)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_power_of_two_tolerances_nest_and_the_error_falls(orc_c2):
    """Halving both tolerances (powers of two, so the grids nest exactly)
    splits buckets: the mapped set shrinks to a subset, and the mapping error
    against the unmapped integration does not grow."""
    T, p, Y, cls = states.bimodal_states(53, 325, 400, 12, cold_noise=2e-3)
    plain = orc_c2.integrate(T, p, Y, 1e-5, rtol=1e-5, atol=1e-8)
    prev_set, prev_err = None, None
    for e in (-7, -9, -11, -13):
        tol = 2.0 ** e
        res = orc_c2.integrate(T, p, Y, 1e-5, rtol=1e-5, atol=1e-8, mapping=2, map_Ttol=tol, map_Ytol=tol)
        m = res[3] == oracle.ST_MAPPED
        err = float(np.abs(res[1] - plain[1]).max()) if m.any() else 0.0
        if prev_set is not None:
            assert not (m & ~prev_set).any()
            assert err <= prev_err
        prev_set, prev_err = m, err
    assert prev_set.sum() < 0.5 * (res[3] >= 0).sum()
