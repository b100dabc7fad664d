"""Pins of the oracle's pressure-dependent (fall-off) reactions (CPU only).

Forms (Lindemann; Troe's broadening, Gilbert, Luther and Troe 1983):
k = k_inf Pr / (1 + Pr) F, Pr = k_0 [M] / k_inf, F = 1 (Lindemann) or
log10 F = log10 Fcent / (1 + f^2), f = (log10 Pr + c) / (n - 0.14 (log10 Pr + c)),
c = -0.4 - 0.67 log10 Fcent, n = 0.75 - 1.27 log10 Fcent,
Fcent = (1 - a) e^(-T/T3) + a e^(-T/T1) [+ e^(-T2/T)]; [M] enters only
through Pr. Pinned by a closed-form decay in the low- and high-pressure
limits and in between, Troe's centre point (F = Fcent where
log10 Pr = -c), the equilibrium constant left unchanged, the linear
invariants, and central differences of the analytic Jacobian on a
mechanism with fall-off reactions and listed efficiencies.
"""
import numpy as np
import pytest

import oracle
from synth import read_mech, states, with_falloff, write_mech
from tests import tinymech

R = 8.314462618
ISO = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)


def _iso_falloff(path, kind, lnA, lnA0, Ea=30e3, Ea0=10e3, beta=0.0, beta0=-1.0, a=0.6, T3=300.0, T1=2000.0,
                 T2=5000.0):
    tinymech.make(path, [ISO, ISO], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=lnA, beta=beta, Ea=Ea, rev=0, tb=1)],
                  falloff=[(0, kind, lnA0, beta0, Ea0, a, T3, T1, T2)])
    return oracle.Oracle(str(path))


@pytest.mark.parametrize("p", [1e2, 1e5, 1e11])
def test_lindemann_decay_closed_form(tmp_path, p):
    """A (+M) -> B between isomers: T and [M] = p/(R T) stay constant, so Y_A
    decays as exp(-k t) with k = k_inf Pr/(1 + Pr); at low pressure k -> k_0 [M],
    at high pressure k -> k_inf."""
    lnA, lnA0 = np.log(1e7), np.log(1e12)
    orc = _iso_falloff(tmp_path / "l.bin", 1, lnA, lnA0)
    T = np.array([900.0, 1300.0])
    Y = np.array([[1.0, 0.8], [0.0, 0.2]])
    dt = 2e-5
    To, Yo, steps, st = orc.integrate(T, np.full(2, p), Y, dt, rtol=1e-9, atol=1e-15)
    assert (st == 0).all()
    kinf = np.exp(lnA - 30e3 / (R * T))
    k0 = np.exp(lnA0 - np.log(T) - 10e3 / (R * T))
    M = 1e-6 * p / (R * T)
    Pr = k0 * M / kinf
    k = kinf * Pr / (1 + Pr)
    np.testing.assert_allclose(Yo[0], Y[0] * np.exp(-k * dt), rtol=1e-7)
    np.testing.assert_allclose(To, T, rtol=1e-13)
    if p == 1e2:
        np.testing.assert_allclose(k, k0 * M, rtol=1e-3)
    if p == 1e11:
        np.testing.assert_allclose(k, kinf, rtol=1e-3)


@pytest.mark.parametrize("kind", [2, 3])
def test_troe_centre_point(tmp_path, kind):
    """Where log10 Pr = -c (c = -0.4 - 0.67 log10 Fcent) the Troe factor is
    Fcent exactly, for the three- and the four-parameter Fcent."""
    lnA, lnA0 = np.log(1e7), np.log(1e12)
    a, T3, T1, T2 = 0.6, 300.0, 2000.0, 5000.0
    orc = _iso_falloff(tmp_path / f"t{kind}.bin", kind, lnA, lnA0, a=a, T3=T3, T1=T1, T2=T2)
    for T in (800.0, 1100.0, 1700.0):
        Fcent = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + (np.exp(-T2 / T) if kind == 3 else 0.0)
        c = -0.4 - 0.67 * np.log10(Fcent)
        kinf = np.exp(lnA - 30e3 / (R * T))
        k0 = np.exp(lnA0 - np.log(T) - 10e3 / (R * T))
        M = 10.0 ** (-c) * kinf / k0                     # log10 Pr + c = 0
        c_, kf, kr, q = orc.rates(M * 1e6 * R * T, np.array([T, 1.0, 0.0]))
        Pr = k0 * c_.sum() / kinf
        assert np.log10(Pr) + c == pytest.approx(0.0, abs=1e-12)
        assert kf[0] == pytest.approx(kinf * Pr / (1 + Pr) * Fcent, rel=1e-12)
        assert abs(np.log10(Fcent)) > 0.05               # the broadening is not negligible here


@pytest.fixture(scope="module")
def fall_c1(tmp_path_factory):
    path = tmp_path_factory.mktemp("fall") / "c1_fall.bin"
    m = with_falloff(read_mech(states.mech_path(10, 20, 0)), 0)
    assert len(m.falloff) == 2 and {r[1] for r in m.falloff} == {1, 2}
    write_mech(str(path), m)
    return oracle.Oracle(str(path)), str(path)


@pytest.mark.parametrize("iso", [False, True])
def test_falloff_jacobian_against_central_differences(fall_c1, iso):
    orc, _ = fall_c1
    T, p, Y = states.uniform_states(10, 4, 5)
    p = np.array([1e4, 1e5, 2e6, 5e5])
    for i in range(4):
        y = np.concatenate([[T[i]], Y[:, i]])
        J = orc.jacobian(p[i], y, iso)
        Jfd = np.zeros_like(J)
        for j in range(y.size):
            hh = 1e-3 * max(abs(y[j]), 1e-3 if j > 0 else 1.0)
            e = np.zeros(y.size)
            e[j] = hh
            f = lambda d: orc.rhs(p[i], y + d * e, iso)
            Jfd[:, j] = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * hh)
        rowmax = np.abs(J).max(1, keepdims=True)
        rowmax[rowmax == 0] = 1.0
        assert (np.abs(J - Jfd) / rowmax).max() < 1e-8
        big = np.abs(J) > 1e-3 * rowmax
        assert (np.abs(J - Jfd)[big] / np.abs(J)[big]).max() < 1e-6


@pytest.mark.parametrize("kind", [1, 3])
def test_falloff_keeps_the_equilibrium_constant(tmp_path, kind):
    """A + B (+M) <=> C as a fall-off reaction, dh = 0, ds = -60 J/(mol K):
    the reverse rate is k_f / K_c, so at equilibrium X_C / (X_A X_B) =
    K_p p / p0 with K_p = exp(ds/R), whatever k_f's pressure dependence."""
    A = dict(atoms=(1, 0, 0, 0), hf=-50e3, s0=150.0, a=30.0, b=0.002)
    B = dict(atoms=(0, 1, 0, 0), hf=-20e3, s0=130.0, a=25.0, b=0.001)
    C = dict(atoms=(1, 1, 0, 0), hf=-70e3, s0=220.0, a=55.0, b=0.003)
    path = tmp_path / f"abc_fall{kind}.bin"
    m = tinymech.make(path, [A, B, C], [dict(reac=[(0, 1), (1, 1)], prod=[(2, 1)], lnA=np.log(1e12), tb=1)],
                      eff=[(0, 2, 2.0)], falloff=[(0, kind, np.log(1e17), -0.5, 0.0, 0.5, 200.0, 1500.0, 4000.0)])
    orc = oracle.Oracle(str(path))
    Kp = np.exp(-60.0 / R)
    for p in (101325.0, 20e5):
        T = np.array([1200.0])
        Y = np.array([[0.4], [0.3], [0.3]])
        To, Yo, _, st = orc.integrate(T, p, Y, 1e-2, rtol=1e-10, atol=1e-16)
        assert st[0] == 0
        X = (Yo[:, 0] / m.W) / (Yo[:, 0] / m.W).sum()
        assert X[2] / (X[0] * X[1]) == pytest.approx(Kp * p / 101325.0, rel=1e-6)


def test_falloff_invariants(fall_c1):
    """sum Y and the element totals are kept with fall-off reactions."""
    orc, path = fall_c1
    m = read_mech(path)
    T, p, Y = states.uniform_states(10, 64, 11)
    p[:] = np.geomspace(1e4, 5e6, 64)
    To, Yo, steps, st = orc.integrate(T, p, Y, 1e-5, rtol=1e-8, atol=1e-14)
    assert (st == 0).all()
    np.testing.assert_allclose(Yo.sum(0), 1.0, atol=1e-12)
    aW = m.atoms.T / m.W[None, :]
    np.testing.assert_allclose(aW @ Yo, aW @ Y, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_isolated_falloff_jacobian_against_central_differences(tmp_path, kind):
    """One reversible fall-off reaction A + B (+M) <=> C with listed
    efficiencies, heat release and T-dependent Fcent, at pressures across the
    fall-off region: every Jacobian entry, the T column (d k / dT through k_0,
    k_inf and Fcent) and the [M] columns included, against fourth-order
    central differences of the right-hand side."""
    A = dict(atoms=(1, 0, 0, 0), hf=-50e3, s0=150.0, a=30.0, b=0.002)
    B = dict(atoms=(0, 1, 0, 0), hf=-20e3, s0=130.0, a=25.0, b=0.001)
    C = dict(atoms=(1, 1, 0, 0), hf=-170e3, s0=220.0, a=55.0, b=0.003)
    path = tmp_path / f"iso_fall{kind}.bin"
    tinymech.make(path, [A, B, C], [dict(reac=[(0, 1), (1, 1)], prod=[(2, 1)], lnA=np.log(3e12), beta=0.3,
                                         Ea=40e3, tb=1)],
                  eff=[(0, 0, 2.5), (0, 2, 0.4)],
                  falloff=[(0, kind, np.log(1e18), -1.2, 5e3, 0.55, 250.0, 1800.0, 3500.0)])
    orc = oracle.Oracle(str(path))
    for T, p in ((900.0, 1e3), (1200.0, 1e5), (1500.0, 3e6), (2000.0, 1e8)):
        y = np.array([T, 0.3, 0.25, 0.45])
        J = orc.jacobian(p, y, False)
        Jfd = np.zeros_like(J)
        for j in range(y.size):
            hh = 1e-4 * max(abs(y[j]), 1e-3 if j > 0 else 1.0)
            e = np.zeros(y.size)
            e[j] = hh
            f = lambda d: orc.rhs(p, y + d * e, False)
            Jfd[:, j] = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * hh)
        scale = np.abs(J).max()
        assert np.abs(J - Jfd).max() < 1e-7 * scale, (T, p, np.abs(J - Jfd).max() / scale)
        big = np.abs(J) > 1e-4 * scale
        assert (np.abs(J - Jfd)[big] / np.abs(J)[big]).max() < 1e-6, (T, p)
