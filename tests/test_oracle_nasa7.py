"""Pins of the oracle's NASA-7 thermo (CPU only).

Definition (the two-range polynomials of real mechanisms' thermo data):
cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4, h/(R T) = a1 + a2 T/2 + a3 T^2/3
+ a4 T^3/4 + a5 T^4/5 + a6/T, s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3
+ a5 T^4/4 + a7, the low set below each species' Tmid, the high set from Tmid
up. Pinned by: equality with the (already pinned) linear thermo when the
polynomials reproduce it; h and s as the integrals of cp and cp/T (numerical
quadrature, across Tmid); continuity of the generated data at Tmid; the
equilibrium constant of a reaction from quadrature of cp; conservation of the
mixture enthalpy in adiabatic integration; central differences of the
analytic Jacobian (where dcp/dT and h(T) enter).
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
from synth import nasa7_of_linear, read_mech, states, with_nasa7, write_mech
from tests import tinymech

R = 8.314462618
T0 = 298.15


@pytest.fixture(scope="module")
def c1_pair(tmp_path_factory):
    d = tmp_path_factory.mktemp("nasa")
    base = read_mech(states.mech_path(10, 20, 0))
    lin = base
    import copy
    same = copy.deepcopy(base)
    same.nasa = nasa7_of_linear(base)
    curved = with_nasa7(base, 0)
    paths = {}
    for name, m in (("same", same), ("curved", curved)):
        paths[name] = str(d / f"c1_{name}.bin")
        write_mech(paths[name], m)
    return states.mech_path(10, 20, 0), paths, curved


def test_polynomials_of_the_linear_thermo_reproduce_it(c1_pair):
    """NASA-7 data that encode cp = a + b T, h(T0) = hf, s(T0) = s0 give the
    linear thermo's cp, h, s and the same integration, to rounding."""
    lin, paths, _ = c1_pair
    a, b = oracle.Oracle(lin), oracle.Oracle(paths["same"])
    for T in (300.0, 999.0, 1000.0, 1700.0, 2600.0):
        for x, y in zip(a.thermo(T), b.thermo(T)):
            np.testing.assert_allclose(y, x, rtol=1e-12, atol=1e-9)
    T, p, Y = states.uniform_states(10, 200, 3)
    ra = a.integrate(T, p, Y, 1e-6, rtol=1e-8, atol=1e-12)
    rb = b.integrate(T, p, Y, 1e-6, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(rb[0], ra[0], rtol=1e-10)
    np.testing.assert_allclose(rb[1], ra[1], atol=1e-10)


def test_h_and_s_are_integrals_of_cp(c1_pair):
    """h(T) - h(T0) = int cp dT and s(T) - s(T0) = int cp/T dT (quadrature of
    the oracle's own cp, piecewise at each species' Tmid)."""
    _, paths, m = c1_pair
    orc = oracle.Oracle(paths["curved"])
    cp = lambda T: orc.thermo(T)[0]
    h0, s0 = orc.thermo(T0)[1], orc.thermo(T0)[2]
    for T in (650.0, 1000.0, 1150.0, 1900.0, 2800.0):
        h, s = orc.thermo(T)[1], orc.thermo(T)[2]
        for k in range(m.nsp):
            pts = [t for t in (m.nasa[k, 1],) if T0 < t < T]
            dh = integrate.quad(lambda t: cp(t)[k], T0, T, points=pts, epsabs=0, epsrel=1e-13, limit=200)[0]
            ds = integrate.quad(lambda t: cp(t)[k] / t, T0, T, points=pts, epsabs=0, epsrel=1e-13, limit=200)[0]
            assert h[k] - h0[k] == pytest.approx(dh, rel=1e-9, abs=1e-6)
            assert s[k] - s0[k] == pytest.approx(ds, rel=1e-9, abs=1e-9)


def test_generated_data_are_continuous_at_tmid(c1_pair):
    _, paths, m = c1_pair
    orc = oracle.Oracle(paths["curved"])
    for k in range(m.nsp):
        Tm = m.nasa[k, 1]
        lo, hi = orc.thermo(np.nextafter(Tm, 0)), orc.thermo(Tm)
        for x, y in zip(lo, hi):
            assert y[k] == pytest.approx(x[k], rel=1e-11, abs=1e-8)
    assert len({float(t) for t in m.nasa[:, 1]}) == 2        # two different Tmid in use


def test_equilibrium_constant_from_quadrature_of_cp(tmp_path):
    """A + B <=> C with NASA-7 thermo: at equilibrium X_C/(X_A X_B) = K_p p/p0,
    K_p = exp(-dG/(R T)) with dG from h and s obtained by integrating the
    species' cp polynomials numerically from T0."""
    A = dict(atoms=(1, 0, 0, 0), hf=-50e3, s0=150.0, a=30.0, b=0.002)
    B = dict(atoms=(0, 1, 0, 0), hf=-20e3, s0=130.0, a=25.0, b=0.001)
    C = dict(atoms=(1, 1, 0, 0), hf=-70e3, s0=220.0, a=55.0, b=0.003)
    path = tmp_path / "abc.bin"
    m = tinymech.make(path, [A, B, C], [dict(reac=[(0, 1), (1, 1)], prod=[(2, 1)], lnA=np.log(1e12))])
    m = with_nasa7(m, 3)
    write_mech(str(path), m)
    orc = oracle.Oracle(str(path))
    T, p = 1400.0, 5e5

    def cp_poly(k, t):
        c = m.nasa[k, 3:8] if t < m.nasa[k, 1] else m.nasa[k, 10:15]
        return R * (c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3 + c[4] * t ** 4)

    g = []
    for k, sp in enumerate((A, B, C)):
        pts = [m.nasa[k, 1]]
        h = sp["hf"] + integrate.quad(lambda t: cp_poly(k, t), T0, T, points=pts, epsrel=1e-13)[0]
        s = sp["s0"] + integrate.quad(lambda t: cp_poly(k, t) / t, T0, T, points=pts, epsrel=1e-13)[0]
        g.append(h - T * s)
    Kp = np.exp(-(g[2] - g[0] - g[1]) / (R * T))
    Y = np.array([[0.4], [0.3], [0.3]])
    To, Yo, _, st = orc.integrate(np.array([T]), p, Y, 1e-2, rtol=1e-10, atol=1e-16, isothermal=True)
    assert st[0] == 0
    X = (Yo[:, 0] / m.W) / (Yo[:, 0] / m.W).sum()
    assert X[2] / (X[0] * X[1]) == pytest.approx(Kp * p / 101325.0, rel=1e-6)


def test_adiabatic_integration_keeps_the_mixture_enthalpy(c1_pair):
    """At constant p with no heat loss, sum_k Y_k h_k(T) / W_k is constant:
    the temperature equation and the NASA-7 h and cp agree."""
    _, paths, m = c1_pair
    orc = oracle.Oracle(paths["curved"])
    T, p, Y = states.uniform_states(10, 60, 5)
    To, Yo, steps, st = orc.integrate(T, p, Y, 1e-5, rtol=1e-9, atol=1e-14)
    assert (st == 0).all()
    for i in range(T.size):
        h0 = (Y[:, i] * orc.thermo(T[i])[1] / m.W).sum()
        h1 = (Yo[:, i] * orc.thermo(To[i])[1] / m.W).sum()
        scale = (np.abs(Y[:, i] * orc.thermo(T[i])[1] / m.W)).sum()
        assert abs(h1 - h0) <= 1e-8 * scale, (i, h0, h1)
    assert np.abs(To - T).max() > 10.0                       # the test sees real heat release


@pytest.mark.parametrize("iso", [False, True])
def test_nasa7_jacobian_against_central_differences(c1_pair, iso):
    _, paths, _ = c1_pair
    orc = oracle.Oracle(paths["curved"])
    T, p, Y = states.uniform_states(10, 4, 9)
    T[:] = [700.0, 990.0, 1150.0, 2200.0]   # stencils stay inside one range (cp' jumps at Tmid)
    for i in range(4):
        y = np.concatenate([[T[i]], Y[:, i]])
        J = orc.jacobian(p[i], y, iso)
        Jfd = np.zeros_like(J)
        for j in range(y.size):
            hh = 1e-3 * max(abs(y[j]), 1e-3 if j > 0 else 0.02)
            e = np.zeros(y.size)
            e[j] = hh
            f = lambda d: orc.rhs(p[i], y + d * e, iso)
            Jfd[:, j] = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * hh)
        rowmax = np.abs(J).max(1, keepdims=True)
        rowmax[rowmax == 0] = 1.0
        assert (np.abs(J - Jfd) / rowmax).max() < 1e-8, (i, (np.abs(J - Jfd) / rowmax).max())
