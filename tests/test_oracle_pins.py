"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a fact that the mathematics or a library
fixes: Rosenbrock order conditions, closed-form solutions, equilibrium
constants from the drawn thermo, quadrature, finite differences, a library
stiff solver and a library linear solve.
"""
import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from synth import read_mech, states
from tests import tinymech

R = 8.314462618
RC = 82.05736
P_ATM = 101325.0
T0 = 298.15


# ---------------------------------------------------------------- coefficients
def _untransform(c):
    """Transformed (a, c, m, e) coefficients -> (alpha, strict beta, b, bhat)."""
    g = c["gamma"]
    C = np.zeros((4, 4))
    C[1, 0] = c["c21"]; C[2, 0] = c["c31"]; C[2, 1] = c["c32"]
    C[3, 0] = c["c41"]; C[3, 1] = c["c42"]; C[3, 2] = c["c43"]
    A = np.zeros((4, 4))
    A[1, 0] = c["a21"]; A[2, 0] = c["a31"]; A[2, 1] = c["a32"]; A[3, 0] = c["a31"]; A[3, 1] = c["a32"]
    Gam = np.linalg.inv(np.diag(np.full(4, 1.0 / g)) - C)
    alpha = A @ Gam
    b = c["m"] @ Gam
    bhat = (c["m"] - c["e"]) @ Gam
    beta_strict = alpha + Gam - np.diag(np.diag(Gam))
    return g, Gam, alpha, beta_strict, b, bhat


def _order_residuals(g, alpha, bs, b):
    """Hairer-Wanner II, Table 7.1: the 8 conditions up to order 4."""
    al = alpha.sum(1)
    bp = bs.sum(1)
    return np.array([
        b.sum() - 1,
        b @ bp - (0.5 - g),
        b @ al**2 - 1 / 3,
        b @ (bs @ bp) - (1 / 6 - g + g * g),
        b @ al**3 - 1 / 4,
        b @ (al * (alpha @ bp)) - (1 / 8 - g / 3),
        b @ (bs @ al**2) - (1 / 12 - g / 3),
        b @ (bs @ (bs @ bp)) - (1 / 24 - g / 2 + 1.5 * g * g - g**3),
    ])


def test_ros4_order_conditions():
    g, Gam, alpha, bs, b, bhat = _untransform(oracle.ros4_coefficients())
    assert np.allclose(np.diag(Gam), g, rtol=0, atol=1e-14)
    assert np.abs(_order_residuals(g, alpha, bs, b)).max() < 1e-13
    emb = _order_residuals(g, alpha, bs, bhat)
    assert np.abs(emb[:4]).max() < 1e-13          # embedded method: order 3
    assert np.abs(emb[4:]).max() > 1e-3           # ... and not order 4
    # stage 4 reuses the stage-3 argument
    assert np.allclose(alpha[3], alpha[2]) and alpha.sum(1)[3] == pytest.approx(alpha.sum(1)[2])


def test_ros4_stability_function():
    g, Gam, alpha, bs, b, bhat = _untransform(oracle.ros4_coefficients())
    B = bs + np.diag(np.full(4, g))
    one = np.ones(4)

    def Rz(z):
        return 1 + z * b @ np.linalg.solve(np.eye(4) - z * B, one)

    # L-stability: R(inf) = 1 - b^T B^-1 1; the published gamma 0.57282 is the
    # L-stability root 0.5728160624821349 rounded, so R(inf) is 1.5e-5, not 0.
    Rinf = 1 - b @ np.linalg.solve(B, one)
    assert abs(Rinf) < 2e-5
    assert abs(Rz(-1e12)) < 2e-5
    # A-stability: |R(iy)| <= 1 on the imaginary axis, and on the left half plane samples
    ys = np.concatenate([-np.logspace(-3, 6, 200), np.logspace(-3, 6, 200)])
    assert max(abs(Rz(1j * y)) for y in ys) <= 1 + 1e-12
    rng = np.random.default_rng(0)
    zs = -rng.exponential(10, 200) + 1j * rng.normal(0, 30, 200)
    assert max(abs(Rz(z)) for z in zs) <= 1 + 1e-12
    # order 4: R(z) - e^z = O(z^5)
    z = 1e-2
    assert abs(Rz(z) - np.exp(z)) < 1e-10 * 10


# ---------------------------------------------------------------- thermo
def test_thermo_against_quadrature(orc_c1):
    m = read_mech(states.mech_path(10, 20, 0))
    for T in (300.0, 1000.0, 2500.0):
        cp, h, s, g = orc_c1.thermo(T)
        for k in range(m.nsp):
            cpf = lambda t: m.cp_a[k] + m.cp_b[k] * t
            assert cp[k] == pytest.approx(cpf(T), rel=1e-14)
            dh = integrate.quad(cpf, T0, T, epsabs=1e-10, epsrel=1e-13)[0]
            ds = integrate.quad(lambda t: cpf(t) / t, T0, T, epsabs=1e-12, epsrel=1e-13)[0]
            assert h[k] == pytest.approx(m.hf[k] + dh, rel=1e-12, abs=1e-6)
            assert s[k] == pytest.approx(m.s0[k] + ds, rel=1e-12)
            assert g[k] == pytest.approx(h[k] - T * s[k], rel=1e-12, abs=1e-6)


# ---------------------------------------------------------------- closed forms
ISO = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)


def test_first_order_decay_closed_form(tmp_path):
    """A -> B, isomers with equal thermo: Y_A = Y_A0 exp(-k t), T constant."""
    path = tmp_path / "decay.bin"
    lnA, beta, Ea = np.log(1e6), 0.5, 20e3
    tinymech.make(path, [ISO, ISO], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=lnA, beta=beta, Ea=Ea, rev=0)])
    orc = oracle.Oracle(str(path))
    T = np.array([800.0, 1000.0, 1300.0])
    Y = np.array([[0.9, 0.6, 1.0], [0.1, 0.4, 0.0]])
    dt, rtol = 1e-6, 1e-8
    To, Yo, steps, st = orc.integrate(T, P_ATM, Y, dt, rtol=rtol, atol=1e-14)
    assert (st == 0).all()
    k = np.exp(lnA) * T**beta * np.exp(-Ea / (R * T))
    exact = Y[0] * np.exp(-k * dt)
    assert np.all(k * dt > 0.3)
    np.testing.assert_allclose(Yo[0], exact, rtol=10 * rtol)
    np.testing.assert_allclose(To, T, rtol=1e-13)


def test_second_order_decay_closed_form(tmp_path):
    """2A -> B with h_B = 2 h_A (isothermal). At constant p, T:
    dY/dt = -4 k P' Y^2 / (T (1+Y)), P' = 1e-6 p / R, so
    ln Y - 1/Y = ln Y0 - 1/Y0 - 4 k P' t / T."""
    path = tmp_path / "dimer.bin"
    A_sp = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)
    B_sp = dict(atoms=(2, 2, 0, 0), hf=-20e3, s0=400.0, a=60.0, b=0.004)
    lnA = np.log(4e10)
    tinymech.make(path, [A_sp, B_sp], [dict(reac=[(0, 2)], prod=[(1, 1)], lnA=lnA, rev=0)])
    orc = oracle.Oracle(str(path))
    T = np.array([1000.0, 1500.0])
    Y0 = np.array([1.0, 0.7])
    Y = np.vstack([Y0, 1 - Y0])
    dt, rtol = 1e-6, 1e-8
    To, Yo, steps, st = orc.integrate(T, P_ATM, Y, dt, rtol=rtol, atol=1e-14)
    assert (st == 0).all()
    kap = 4 * np.exp(lnA) * (1e-6 * P_ATM / R) / T
    for i in range(2):
        F = lambda y: np.log(y) - 1 / y - (np.log(Y0[i]) - 1 / Y0[i] - kap[i] * dt)
        ye = optimize.brentq(F, 1e-12, Y0[i], xtol=1e-16, rtol=1e-15)
        assert Yo[0, i] == pytest.approx(ye, rel=10 * rtol)
        assert ye < 0.8 * Y0[i]
    np.testing.assert_allclose(To, T, rtol=1e-13)


def test_reversible_relaxation_and_Kc(tmp_path):
    """A <=> B, dh = 0, ds = 5 J/(mol K): K = exp(ds/R);
    Y_A(t) = Y_inf + (Y_A0 - Y_inf) exp(-(kf + kr) t), Y_inf = 1/(1+K)."""
    path = tmp_path / "iso.bin"
    Bs = dict(ISO, s0=ISO["s0"] + 5.0)
    kf = 2e6
    tinymech.make(path, [ISO, Bs], [dict(reac=[(0, 1)], prod=[(1, 1)], lnA=np.log(kf))])
    orc = oracle.Oracle(str(path))
    K = np.exp(5.0 / R)
    kr = kf / K
    T = np.array([600.0, 1800.0])
    Y = np.array([[1.0, 0.2], [0.0, 0.8]])
    for dt in (3e-7, 1e-3):
        To, Yo, _, st = orc.integrate(T, P_ATM, Y, dt, rtol=1e-9, atol=1e-15)
        assert (st == 0).all()
        Yinf = 1 / (1 + K)
        exact = Yinf + (Y[0] - Yinf) * np.exp(-(kf + kr) * dt)
        np.testing.assert_allclose(Yo[0], exact, rtol=1e-7)
    np.testing.assert_allclose(Yo[1] / Yo[0], K, rtol=1e-8)


@pytest.mark.parametrize("reverse", [False, True])
def test_pressure_dependent_equilibrium(tmp_path, reverse):
    """A + B <=> C with dh = 0 and ds = -60 J/(mol K): at equilibrium
    X_C / (X_A X_B) = K_p * p / p0, K_p = exp(ds/R). reverse=True writes the
    same reaction as C <=> A + B (delta nu = +1)."""
    path = tmp_path / f"abc{int(reverse)}.bin"
    A = dict(atoms=(1, 0, 0, 0), hf=-50e3, s0=150.0, a=30.0, b=0.002)
    B = dict(atoms=(0, 1, 0, 0), hf=-20e3, s0=130.0, a=25.0, b=0.001)
    C = dict(atoms=(1, 1, 0, 0), hf=-70e3, s0=220.0, a=55.0, b=0.003)
    rx = dict(reac=[(0, 1), (1, 1)], prod=[(2, 1)], lnA=np.log(1e12))
    if reverse:
        rx = dict(reac=[(2, 1)], prod=[(0, 1), (1, 1)], lnA=np.log(1e7))
    m = tinymech.make(path, [A, B, C], [rx])
    orc = oracle.Oracle(str(path))
    Kp = np.exp(-60.0 / R)
    for p in (P_ATM, 20e5):
        T = np.array([1200.0])
        Y = np.array([[0.4], [0.3], [0.3]])
        To, Yo, _, st = orc.integrate(T, p, Y, 1e-2, rtol=1e-10, atol=1e-16)
        assert st[0] == 0
        X = (Yo[:, 0] / m.W) / (Yo[:, 0] / m.W).sum()
        assert X[2] / (X[0] * X[1]) == pytest.approx(Kp * p / P_ATM, rel=1e-6)
        assert To[0] == pytest.approx(1200.0, rel=1e-12)


# ---------------------------------------------------------------- equilibrium of a random mechanism
@pytest.mark.parametrize("iso", [True, False])
def test_detailed_balance_at_long_dt(orc_c1, iso):
    """After 1 s at T >= 1800 K every reaction whose species are resolved
    (Y >= 1e-15, far above atol) satisfies k_r prod c'' = k_f prod c' with
    K_c from the species' Gibbs energies, and the state is stationary.
    (Below ~600 K many reactions are frozen over 1 s; species far below atol
    carry uncontrolled fluxes of 1e-35 mol/cm^3/s and are left out.)"""
    m = read_mech(states.mech_path(10, 20, 0))
    nr, npd = m.nu_matrix()
    T, p, Y = states.uniform_states(10, 2, 11)
    T[:] = [1900.0, 2300.0]
    To, Yo, steps, st = orc_c1.integrate(T, p, Y, 1.0, rtol=1e-10, atol=1e-22, max_steps=2000000, isothermal=iso)
    assert (st == 0).all()
    for i in range(2):
        y = np.concatenate([[To[i]], Yo[:, i]])
        c, kf, kr, q = orc_c1.rates(p[i], y)
        fwd = kf * np.prod(c[:, None] ** nr, axis=0)
        rev = kr * np.prod(c[:, None] ** npd, axis=0)
        resolved = np.array([(Yo[(nr[:, j] + npd[:, j]) > 0, i] >= 1e-15).all() for j in range(m.nrx)])
        assert resolved.sum() >= 3
        assert np.abs(1 - rev / fwd)[resolved].max() < 1e-4
        T2, Y2, _, st2 = orc_c1.integrate(To[i:i + 1], p[i], Yo[:, i:i + 1], 1e-3, rtol=1e-10, atol=1e-22,
                                          isothermal=iso)
        assert st2[0] == 0
        assert abs(T2[0] - To[i]) < 1e-8 * To[i]
        assert np.abs(Y2[:, 0] - Yo[:, i]).max() < 1e-12


# ---------------------------------------------------------------- invariants
def test_linear_and_enthalpy_invariants(orc_c1):
    m = read_mech(states.mech_path(10, 20, 0))
    T, p, Y = states.uniform_states(10, 256, 3)
    rtol = 1e-6
    To, Yo, steps, st = orc_c1.integrate(T, p, Y, 1e-6, rtol=rtol, atol=1e-10)
    assert (st == 0).all()
    np.testing.assert_allclose(Yo.sum(0), 1.0, rtol=0, atol=1e-12)
    elem0 = m.atoms.T @ (Y / m.W[:, None])
    elem1 = m.atoms.T @ (Yo / m.W[:, None])
    assert np.abs(elem1 - elem0).max() <= 1e-12 * np.abs(elem0).max()
    # mixture enthalpy sum_k Y_k h_k(T) / W_k is conserved (adiabatic, constant p)
    for i in range(0, 256, 17):
        h0 = orc_c1.thermo(T[i])[1] / m.W
        h1 = orc_c1.thermo(To[i])[1] / m.W
        scale = np.abs(Y[:, i] * h0).sum()
        assert abs(Yo[:, i] @ h1 - Y[:, i] @ h0) <= 10 * rtol * scale


# ---------------------------------------------------------------- brute force
def test_nonisothermal_against_library_stiff_solver(tmp_path):
    """A + B <=> C, exothermic (dh = -80 kJ/mol): the temperature moves by tens
    of kelvin (up where C forms, down where it dissociates). The
    reference integrates the same physics written out for this system with
    scipy's Radau at rtol 1e-12."""
    path = tmp_path / "exo.bin"
    sp = [dict(atoms=(1, 0, 0, 0), hf=-30e3, s0=150.0, a=30.0, b=0.002),
          dict(atoms=(0, 1, 0, 0), hf=-10e3, s0=130.0, a=25.0, b=0.004),
          dict(atoms=(1, 1, 0, 0), hf=-120e3, s0=190.0, a=45.0, b=0.003)]
    lnA, beta, Ea = np.log(3e12), 0.3, 40e3
    m = tinymech.make(path, sp, [dict(reac=[(0, 1), (1, 1)], prod=[(2, 1)], lnA=lnA, beta=beta, Ea=Ea)])
    orc = oracle.Oracle(str(path))
    a, b, hf, s0, W = m.cp_a, m.cp_b, m.hf, m.s0, m.W
    p = 5 * P_ATM

    def h(T):
        return hf + a * (T - T0) + 0.5 * b * (T * T - T0 * T0)

    def s(T):
        return s0 + a * np.log(T / T0) + b * (T - T0)

    def f(t, y):
        T, Yv = y[0], y[1:]
        rho = 1e-6 * p / (R * T * np.sum(Yv / W))
        c = rho * Yv / W
        kf = np.exp(lnA + beta * np.log(T) - Ea / (R * T))
        g = h(T) - T * s(T)
        Kp = np.exp(-(g[2] - g[0] - g[1]) / (R * T))
        Kc = Kp * (1.0 / (RC * T)) ** (-1)
        q = kf * c[0] * c[1] - kf / Kc * c[2]
        w = np.array([-q, -q, q])
        cpm = np.sum(Yv * (a + b * T) / W)
        return np.concatenate([[-np.sum(h(T) * w) / (rho * cpm)], W * w / rho])

    T = np.array([900.0, 1100.0])
    Y = np.array([[0.5, 0.3], [0.4, 0.3], [0.1, 0.4]])
    dt, rtol = 2e-6, 1e-8
    To, Yo, _, st = orc.integrate(T, p, Y, dt, rtol=rtol, atol=1e-14)
    assert (st == 0).all()
    for i in range(2):
        y0 = np.concatenate([[T[i]], Y[:, i]])
        sol = integrate.solve_ivp(f, (0, dt), y0, method="Radau", rtol=1e-12, atol=1e-16)
        ref = sol.y[:, -1]
        assert abs(ref[0] - T[i]) > 20.0      # a real temperature change
        assert To[i] == pytest.approx(ref[0], rel=10 * rtol)
        np.testing.assert_allclose(Yo[:, i], ref[1:], rtol=0, atol=10 * rtol)


# ---------------------------------------------------------------- Jacobian
@pytest.mark.parametrize("which,iso", [("c1", False), ("c1", True), ("c2", False)])
def test_jacobian_against_central_differences(which, iso, orc_c1, orc_c2):
    orc, nsp = (orc_c1, 10) if which == "c1" else (orc_c2, 53)
    T, p, Y = states.uniform_states(nsp, 4, 5)
    for i in range(4):
        y = np.concatenate([[T[i]], Y[:, i]])
        J = orc.jacobian(p[i], y, iso)
        # fourth-order central differences, step 1e-3 * max(|y_j|, scale_j)
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
        big = np.abs(J) > 1e-3 * rowmax          # well-scaled entries
        assert (np.abs(J - Jfd)[big] / np.abs(J)[big]).max() < 1e-6


# ---------------------------------------------------------------- linear solve
def test_lu_solve_against_library():
    rng = np.random.default_rng(2)
    for n in (1, 2, 11, 54, 101):
        A = rng.normal(size=(n, n))
        if n > 2:
            A[0, 0] = 0.0        # forces a row exchange
        x0 = rng.normal(size=n)
        b = A @ x0
        x = oracle.lu_solve(A, b)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)
        assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(x) * n


# ---------------------------------------------------------------- convergence order
def test_fixed_step_convergence_order(tmp_path):
    """Fixed steps on the nonlinear 2A -> B problem: the error falls as h^4."""
    path = tmp_path / "dimer.bin"
    A_sp = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)
    B_sp = dict(atoms=(2, 2, 0, 0), hf=-20e3, s0=400.0, a=60.0, b=0.004)
    lnA = np.log(4e10)
    tinymech.make(path, [A_sp, B_sp], [dict(reac=[(0, 2)], prod=[(1, 1)], lnA=lnA, rev=0)])
    orc = oracle.Oracle(str(path))
    T = np.array([1000.0])
    Y = np.array([[1.0], [0.0]])
    dt = 1e-6
    kap = 4 * np.exp(lnA) * (1e-6 * P_ATM / R) / T[0]
    F = lambda y: np.log(y) - 1 / y - (0.0 - 1.0 - kap * dt)
    ye = optimize.brentq(F, 1e-12, 1.0, xtol=1e-17, rtol=1e-15)
    errs = []
    ns = [8, 16, 32, 64]
    for n in ns:
        _, Yo, steps, st = orc.integrate(T, P_ATM, Y, dt, fixed_h=dt / n)
        assert steps[0] == n
        errs.append(abs(Yo[0, 0] - ye))
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert -4.2 <= slope <= -3.8, (errs, slope)


# ---------------------------------------------------------------- reference mapping
def test_map_classification_worked_example(orc_c1):
    """Cells built to lie inside / outside the criteria (Sec. 2.3 reading):
    qualify = max|Y - Yref| < Ytol; reference = first qualifying cell; mapped =
    other qualifying cells with |T - T_ref| < Ttol * T_ref."""
    rng = np.random.default_rng(4)
    Yref = rng.dirichlet(np.full(10, 0.5))
    n = 8
    Y = np.repeat(Yref[:, None], n, axis=1)
    T = np.full(n, 500.0)
    Y[:, 0] = rng.dirichlet(np.full(10, 0.5))        # far in composition
    Y[3, 2] += 2e-4; Y[4, 2] -= 2e-4                 # just outside Ytol
    Y[3, 4] += 5e-5; Y[4, 4] -= 5e-5                 # inside Ytol
    T[1] = 500.0                                     # reference (first qualifying)
    T[5] = 500.0 * (1 + 2e-4)                        # outside Ttol
    T[6] = 500.0 * (1 + 5e-5)                        # inside Ttol
    ref, flag = orc_c1.map_classify(T, Y, Yref, 1e-4, 1e-4)
    assert ref == 1
    assert flag.tolist() == [0, 0, 0, 1, 1, 0, 1, 1]
    ref0, flag0 = orc_c1.map_classify(T, Y, Yref, 0.0, 0.0)
    assert ref0 == -1 and flag0.sum() == 0
    # T_max gate excludes everything hotter
    ref2, flag2 = orc_c1.map_classify(T, Y, Yref, 1e-4, 1e-4, Tmax=400.0)
    assert ref2 == -1 and flag2.sum() == 0


def test_mapping_copies_reference_increment(orc_c1):
    T, p, Y = states.uniform_states(10, 6, 8)
    T[:] = 450.0
    Y[:] = Y[:, :1]
    Y[:, 3] = Y[:, 3] * (1 + 1e-6); Y[:, 3] /= Y[:, 3].sum()
    To, Yo, steps, st = orc_c1.integrate(T, p, Y, 1e-6, mapping=True, map_Ttol=1e-4, map_Ytol=1e-4)
    assert st[0] == 0 and (st[1:] == 1).all() and (steps[1:] == 0).all()
    np.testing.assert_allclose(To[1:] - T[1:], To[0] - T[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(Yo[:, 1:] - Y[:, 1:], np.broadcast_to(Yo[:, :1] - Y[:, :1], (10, 5)),
                               rtol=0, atol=1e-15)
    To2, Yo2, _, st2 = orc_c1.integrate(T, p, Y, 1e-6, mapping=True, map_Ttol=0.0, map_Ytol=0.0)
    To3, Yo3, _, st3 = orc_c1.integrate(T, p, Y, 1e-6)
    assert (st2 == 0).all()
    np.testing.assert_array_equal(To2, To3)
    np.testing.assert_array_equal(Yo2, Yo3)


# ---------------------------------------------------------------- status handling
def test_status_codes(orc_c1):
    T, p, Y = states.uniform_states(10, 4, 1)
    T[1] = np.nan
    T[2] = -5.0
    To, Yo, steps, st = orc_c1.integrate(T, p, Y, 1e-6, max_steps=3)
    assert st[1] == oracle.ST_NONFINITE and st[2] == oracle.ST_NONFINITE
    assert st[0] == oracle.ST_MAX_STEPS and steps[0] == 3


def test_trapezoid_gate_rejects_even_exact_increments_of_stiff_cells(orc_c1):
    """The surrogate gate accepts a proposed (T', Y') only when its trapezoid
    defect y' - y - dt/2 (f(y) + f(y')) is within the gate. Applied to the
    oracle's own (tight-tolerance) solution of the 10-species cells over
    dt = 1e-6 s, the defect is far above 1e-4 on every cell: their fast
    reactions relax within the step (dt |f(y)| ~ 1e0..1e6 at any T), so no
    proposal, however exact, passes. Near-equilibrium cells do pass (the
    bimodal field's burnt cells: the GPU test of the gate's accept branch)."""
    T, p, Y = states.uniform_states(10, 64, 7)
    dt = 1e-6
    To, Yo, steps, st = orc_c1.integrate(T, p, Y, dt, rtol=1e-10, atol=1e-16)
    for i in range(T.size):
        y0 = np.concatenate([[T[i]], Y[:, i]])
        y1 = np.concatenate([[To[i]], Yo[:, i]])
        d = y1 - y0 - 0.5 * dt * (orc_c1.rhs(p[i], y0) + orc_c1.rhs(p[i], y1))
        assert max(abs(d[0]) / T[i], np.abs(d[1:]).max()) > 1e-2
