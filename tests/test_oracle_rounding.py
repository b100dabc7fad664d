"""How far two correct FP64 integrations of the same cells can disagree (CPU only).

The adaptive Rosenbrock step sequence is a chain of floating-point decisions
(a step is accepted when its error norm is <= 1). Where a decision is taken
at a norm within rounding of 1, any change in rounding can flip it, and the
cell then follows another, equally valid, step sequence. This file measures
that spread with the oracle alone, so it says nothing about the GPU:

* two builds of the same oracle.cpp that differ only in FMA contraction
  (-ffp-contract=off against =fast; on x86-64 the second also needs -mfma);
* one build, with every input temperature moved by one unit in the last place.

Measured on the 10-species case (1024 cells, dt 1e-6, rtol 1e-6, atol 1e-10):
37 cells (3.6 %) differ by more than 1e-9 in some mass fraction, by at most
2.6e-8, and 57 cells change their step count; at rtol 1e-8 every cell agrees
within 1.5e-10. On 1500 cold cells of the 262,144-cell bimodal field (53
species, rtol 1e-5, atol 1e-8), 27 cells (1.8 %) differ by more than 1e-9, by
at most 2.1e-9. These are the facts behind the parity bars of the GPU tests:
1e-9 on every cell where the step sequence is not rounding-sensitive, and on
a stated fraction of cells where it is.
"""
import os
import platform

import numpy as np
import pytest

import oracle
from synth import states


def _has_fma() -> bool:
    if platform.machine() != "x86_64":
        return True
    try:
        with open("/proc/cpuinfo") as f:
            return " fma " in f.read().replace("\n", " ")
    except OSError:
        return False


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    if not _has_fma():
        pytest.skip("this CPU has no FMA instruction")
    d = tmp_path_factory.mktemp("orc")
    off = oracle.build_variant(str(d / "orc_off.so"), ["-ffp-contract=off"])
    fast = ["-ffp-contract=fast"] + (["-mfma"] if platform.machine() == "x86_64" else [])
    on = oracle.build_variant(str(d / "orc_fma.so"), fast)
    return oracle.load_variant(off), oracle.load_variant(on)


def _spread(a, b):
    dY = np.abs(a[1] - b[1]).max(axis=0)
    dT = np.abs(a[0] - b[0]) / a[0]
    return dT, dY


def test_fma_contraction_changes_c1_results_above_the_bar(builds):
    off, on = builds
    mech = states.mech_path(10, 20, 0)
    T, p, Y = states.uniform_states(10, 1024, 0)
    a = oracle.Oracle(mech, lib=off).integrate(T, p, Y, 1e-6, rtol=1e-6, atol=1e-10)
    b = oracle.Oracle(mech, lib=on).integrate(T, p, Y, 1e-6, rtol=1e-6, atol=1e-10)
    assert (a[3] == 0).all() and (b[3] == 0).all()
    dT, dY = _spread(a, b)
    frac = (dY > 1e-9).mean()
    print(f"c1 rtol 1e-6: {int((dY > 1e-9).sum())} cells over 1e-9 ({frac:.4f}), max |dY| {dY.max():.3e}, "
          f"steps differ on {int((a[2] != b[2]).sum())}")
    assert 0.01 <= frac <= 0.10
    assert 1e-9 < dY.max() < 1e-7
    assert dT.max() < 1e-7


def test_fma_contraction_within_the_bar_at_rtol_1e8(builds):
    off, on = builds
    mech = states.mech_path(10, 20, 0)
    T, p, Y = states.uniform_states(10, 1024, 0)
    a = oracle.Oracle(mech, lib=off).integrate(T, p, Y, 1e-6, rtol=1e-8, atol=1e-12)
    b = oracle.Oracle(mech, lib=on).integrate(T, p, Y, 1e-6, rtol=1e-8, atol=1e-12)
    dT, dY = _spread(a, b)
    assert dY.max() < 1e-9, dY.max()


def test_fma_contraction_on_cold_bimodal_cells(builds):
    off, on = builds
    mech = states.mech_path(53, 325, 0)
    T, p, Y, cls = states.bimodal_states(53, 325, 262144, 0)
    idx = states.stratified_sample(cls, 1500, 0)
    idx = idx[cls[idx] == states.COLD][:400]
    args = (T[idx], p[idx], np.ascontiguousarray(Y[:, idx]), 1e-5)
    a = oracle.Oracle(mech, lib=off).integrate(*args, rtol=1e-5, atol=1e-8)
    b = oracle.Oracle(mech, lib=on).integrate(*args, rtol=1e-5, atol=1e-8)
    dT, dY = _spread(a, b)
    n_over = int((dY > 1e-9).sum())
    print(f"bimodal cold: {n_over} of {idx.size} cells over 1e-9, max |dY| {dY.max():.3e}")
    assert 1 <= n_over <= 0.05 * idx.size
    assert dY.max() < 1e-8


def test_one_ulp_change_of_the_inputs_moves_c1_results_above_the_bar():
    """The same sensitivity without a second build: T moved by one ulp."""
    mech = states.mech_path(10, 20, 0)
    T, p, Y = states.uniform_states(10, 1024, 0)
    orc = oracle.Oracle(mech)
    a = orc.integrate(T, p, Y, 1e-6, rtol=1e-6, atol=1e-10)
    b = orc.integrate(np.nextafter(T, np.inf), p, Y, 1e-6, rtol=1e-6, atol=1e-10)
    dT, dY = _spread(a, b)
    frac = (dY > 1e-9).mean()
    assert 0.01 <= frac <= 0.10, frac
    assert 1e-9 < dY.max() < 1e-7
