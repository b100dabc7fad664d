"""End-to-end pin of the oracle's integration on the full mechanisms (CPU
only): the right-hand side written out again in numpy from the mechanism
file (ideal gas, linear-cp thermo, mass action with third bodies and
efficiencies, K_c from the Gibbs energies) and integrated by scipy's Radau
at tight tolerance, against the oracle's Rosenbrock result on cells of the
10-species case and of the three classes of the 53-species bimodal field.
Independent code and an independent method: a mistake in either the
oracle's rate, thermo or temperature equation or in its step control shows
up as a difference far above the tolerances."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from synth import read_mech, states

R = 8.314462618
RC = 82.05736      # cm^3 atm / (mol K)
T0 = 298.15


def numpy_rhs(m, p):
    nr, npd = m.nu_matrix()
    nu = (npd - nr).astype(float)
    dnu = nu.sum(axis=0)
    E = np.zeros((m.nrx, m.nsp))
    E[np.asarray(m.thirdbody) != 0] = 1.0
    for j, k, e in m.eff:
        E[j, k] = e
    tb = np.asarray(m.thirdbody) != 0
    rev = np.asarray(m.reversible) != 0
    a, b, W = m.cp_a, m.cp_b, m.W

    def f(t, y):
        T, Y = y[0], y[1:]
        rho = 1e-6 * p * 1.0 / (R * T * np.sum(Y / W))            # g/cm^3
        c = rho * Y / W                                           # mol/cm^3
        h = m.hf + a * (T - T0) + 0.5 * b * (T * T - T0 * T0)
        s = m.s0 + a * np.log(T / T0) + b * (T - T0)
        g = h - T * s
        kf = np.exp(m.lnA + m.beta * np.log(T) - m.Ea / (R * T))
        Kc = np.exp(-(nu.T @ g) / (R * T)) * (1.0 / (RC * T)) ** dnu
        fwd = kf * np.prod(c[:, None] ** nr, axis=0)
        bwd = np.where(rev, kf / Kc * np.prod(c[:, None] ** npd, axis=0), 0.0)
        M = np.where(tb, E @ c, 1.0)
        w = nu @ (M * (fwd - bwd))
        cpm = np.sum(Y * (a + b * T) / W)
        return np.concatenate([[-np.sum(h * w) / (rho * cpm)], W * w / rho])
    return f


def _check(mech, T, p, Y, dt, rtol, atol):
    orc = oracle.Oracle(mech)
    To, Yo, steps, st = orc.integrate(T, p, Y, dt, rtol=rtol, atol=atol)
    assert (st == 0).all()
    m = read_mech(mech)
    worst_T, worst_Y = 0.0, 0.0
    for i in range(T.size):
        f = numpy_rhs(m, p[i])
        y0 = np.concatenate([[T[i]], Y[:, i]])
        sol = integrate.solve_ivp(f, (0.0, dt), y0, method="Radau", rtol=1e-11, atol=1e-15)
        assert sol.success
        ref = sol.y[:, -1]
        worst_T = max(worst_T, abs(To[i] - ref[0]) / ref[0])
        worst_Y = max(worst_Y, np.abs(Yo[:, i] - ref[1:]).max())
    return worst_T, worst_Y, To, T


def test_ten_species_cells_against_radau():
    T, p, Y = states.uniform_states(10, 12, 21)
    wT, wY, To, T0_ = _check(states.mech_path(10, 20, 0), T, p, Y, 1e-6, 1e-9, 1e-13)
    print(f"10 species: max |dT|/T {wT:.2e}, max |dY| {wY:.2e}")
    assert np.abs(To - T0_).max() > 1.0            # the chemistry changes the state
    assert wT < 1e-8 and wY < 1e-8


def test_fiftythree_species_bimodal_cells_against_radau():
    T, p, Y, cls = states.bimodal_states(53, 325, 3000, 22)
    idx = np.concatenate([np.flatnonzero(cls == c)[:2] for c in (states.COLD, states.BURNT, states.FRONT)])
    wT, wY, To, T0_ = _check(states.mech_path(53, 325, 0), T[idx], p[idx], np.ascontiguousarray(Y[:, idx]), 1e-5,
                             1e-8, 1e-12)
    print(f"53 species: max |dT|/T {wT:.2e}, max |dY| {wY:.2e}")
    assert wT < 1e-7 and wY < 1e-7
