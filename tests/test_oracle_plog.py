"""Pins of the oracle's pressure-dependent Arrhenius (PLOG) reactions (CPU only).

Definition (the logarithmic pressure interpolation of real mechanisms): each
listed pressure p_i has its own Arrhenius form k_i(T); between the two listed
pressures that bracket p, ln k = ln k_i + (ln k_{i+1} - ln k_i) w with
w = ln(p / p_i) / ln(p_{i+1} / p_i); below the first and above the last listed
pressure, that point's k (reading: clamp, not extrapolate). Pinned by
bit-identity with a plain Arrhenius mechanism at a listed pressure and outside
the range, the first-order decay exp(-k t) at the geometric mean of two
listed pressures (k = sqrt(k_i k_{i+1})) and elsewhere, the equilibrium
constant left unchanged, the linear invariants, and central differences of
the analytic Jacobian.
"""
import numpy as np
import pytest

import oracle
from synth import read_mech, states, with_plog, write_mech
from tests import tinymech

R = 8.314462618
ISO = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)
PTS = [(1e5, np.log(2e6), 0.4, 25e3), (1e6, np.log(5e7), -0.2, 31e3), (1e7, np.log(8e8), 0.1, 40e3)]


def _iso(path, pts=PTS, rev=0):
    tinymech.make(path, [ISO, ISO], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=0.0, rev=rev)], plog=[(0, pts)])
    return oracle.Oracle(str(path))


def _plain(path, pt, rev=0):
    tinymech.make(path, [ISO, ISO], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=pt[1], beta=pt[2], Ea=pt[3], rev=rev)])
    return oracle.Oracle(str(path))


def _k(pt, T):
    return np.exp(pt[1] + pt[2] * np.log(T) - pt[3] / (R * T))


@pytest.mark.parametrize("p,i", [(1e6, 1), (1e5, 0), (1e7, 2), (1e3, 0), (1e9, 2)])
def test_listed_pressure_and_outside_the_range_equal_plain_arrhenius(tmp_path, p, i):
    """At a listed pressure the interpolation weight is exactly 0, and outside
    the range the nearest point is used: the integration is bit-identical to
    a mechanism with that point's Arrhenius form."""
    orc = _iso(tmp_path / "plog.bin")
    ref = _plain(tmp_path / "plain.bin", PTS[i])
    T = np.array([900.0, 1300.0, 1700.0])
    Y = np.array([[1.0, 0.7, 0.5], [0.0, 0.3, 0.5]])
    a = orc.integrate(T, np.full(3, p), Y, 1e-5, rtol=1e-8, atol=1e-14)
    b = ref.integrate(T, np.full(3, p), Y, 1e-5, rtol=1e-8, atol=1e-14)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("p", [np.sqrt(1e5 * 1e6), np.sqrt(1e6 * 1e7), 2.5e5, 7e6])
def test_first_order_decay_between_listed_pressures(tmp_path, p):
    """A -> B between isomers (T stays constant): Y_A = Y_A0 exp(-k dt) with
    k = k_i^(1 - w) k_{i+1}^w, w = ln(p/p_i)/ln(p_{i+1}/p_i); at the geometric
    mean of p_i and p_{i+1}, k = sqrt(k_i k_{i+1})."""
    orc = _iso(tmp_path / "plog.bin")
    T = np.array([900.0, 1300.0])
    Y = np.array([[1.0, 0.6], [0.0, 0.4]])
    dt = 3e-5
    To, Yo, steps, st = orc.integrate(T, np.full(2, p), Y, dt, rtol=1e-10, atol=1e-16)
    assert (st == 0).all()
    i = 0 if p < 1e6 else 1
    w = np.log(p / PTS[i][0]) / np.log(PTS[i + 1][0] / PTS[i][0])
    k = _k(PTS[i], T) ** (1 - w) * _k(PTS[i + 1], T) ** w
    if np.isclose(w, 0.5):
        np.testing.assert_allclose(k, np.sqrt(_k(PTS[i], T) * _k(PTS[i + 1], T)), rtol=1e-13)
    assert (k * dt > 0.05).any()                       # the reaction does visible work
    np.testing.assert_allclose(Yo[0], Y[0] * np.exp(-k * dt), rtol=1e-7, atol=1e-14)
    np.testing.assert_allclose(To, T, rtol=1e-13)


def test_rate_constant_across_pressures(tmp_path):
    """The oracle's rate constant along a pressure sweep: continuous at the
    listed pressures, log-linear in ln p between them, flat outside."""
    orc = _iso(tmp_path / "plog.bin")
    T = 1100.0
    ps = np.geomspace(1e3, 1e9, 61)
    kf = np.array([orc.rates(p, np.array([T, 1.0, 0.0]))[1][0] for p in ps])
    lnk = [np.log(_k(pt, T)) for pt in PTS]
    lnp = [np.log(pt[0]) for pt in PTS]
    want = np.exp(np.interp(np.log(ps), lnp, lnk))   # np.interp clamps outside the range
    np.testing.assert_allclose(kf, want, rtol=1e-12)


def test_plog_keeps_the_equilibrium_constant(tmp_path):
    """A reversible PLOG reaction A <=> B between isomers with different
    formation enthalpies: k_f / k_r = K_c(T) at every pressure."""
    B = dict(ISO, hf=-25e3, s0=205.0)
    path = tmp_path / "rev.bin"
    tinymech.make(path, [ISO, B], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=0.0, rev=1)], plog=[(0, PTS)])
    orc = oracle.Oracle(str(path))
    T = 1250.0
    ratios = []
    for p in (3e4, 1e5, 4e5, 1e6, 5e7):
        c, kf, kr, q = orc.rates(p, np.array([T, 0.5, 0.5]))
        ratios.append(kf[0] / kr[0])
    # dnu = 0: K_c = K_p = exp(-dG/(R T)) with dG = dH - T dS (same cp for both)
    Kc = np.exp(-((-25e3 + 10e3) - T * (205.0 - 200.0)) / (R * T))
    np.testing.assert_allclose(ratios, Kc, rtol=1e-12)


@pytest.fixture(scope="module")
def plog_c1(tmp_path_factory):
    path = tmp_path_factory.mktemp("plog") / "c1_plog.bin"
    m = with_plog(read_mech(states.mech_path(10, 20, 0)), 0, frac=0.5)
    assert len(m.plog) >= 4
    write_mech(str(path), m)
    return oracle.Oracle(str(path)), str(path)


def test_plog_file_round_trip(plog_c1):
    _, path = plog_c1
    m = read_mech(path)
    for j, pts in m.plog:
        assert not m.thirdbody[j] and 2 <= len(pts) <= 4
        ps = [q[0] for q in pts]
        assert ps == sorted(ps)


@pytest.mark.parametrize("p", [5e3, 2e5, 1.3e6, 4e7])
def test_plog_jacobian_against_central_differences(plog_c1, p):
    """Analytic Jacobian (d ln k / dT of the interpolated form) against
    fourth-order central differences, inside and outside the listed range."""
    orc, _ = plog_c1
    T, _, Y = states.uniform_states(10, 3, 8)
    for i in range(3):
        y = np.concatenate([[T[i]], Y[:, i]])
        J = orc.jacobian(p, y, False)
        Jfd = np.zeros_like(J)
        for j in range(y.size):
            hh = 1e-3 * max(abs(y[j]), 1e-3 if j > 0 else 1.0)
            e = np.zeros(y.size)
            e[j] = hh
            f = lambda d: orc.rhs(p, y + d * e, False)
            Jfd[:, j] = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * hh)
        rowmax = np.abs(J).max(1, keepdims=True)
        rowmax[rowmax == 0] = 1.0
        assert (np.abs(J - Jfd) / rowmax).max() < 1e-8


def test_plog_invariants(plog_c1):
    """sum Y and the element totals are kept with PLOG reactions."""
    orc, path = plog_c1
    m = read_mech(path)
    T, p, Y = states.uniform_states(10, 48, 12)
    p[:] = np.geomspace(3e3, 3e7, 48)
    To, Yo, steps, st = orc.integrate(T, p, Y, 1e-5, rtol=1e-8, atol=1e-14)
    assert (st == 0).all()
    np.testing.assert_allclose(Yo.sum(0), 1.0, atol=1e-12)
    aW = m.atoms.T / m.W[None, :]
    np.testing.assert_allclose(aW @ Yo, aW @ Y, rtol=1e-10, atol=1e-14)
