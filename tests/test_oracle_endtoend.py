"""End-to-end pin of the oracle's integration on the full mechanisms (CPU
only): the right-hand side written out again in numpy from the mechanism
file (ideal gas, linear-cp or NASA-7 thermo, mass action with third bodies
and efficiencies, fall-off and PLOG, K_c from the Gibbs energies) and
integrated by scipy's Radau at tight tolerance, against the oracle's Rosenbrock result on cells of the
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


def _thermo(m, T):
    """molar cp, h, s of every species: NASA-7 when the mechanism has it, else linear cp"""
    if m.nasa is None:
        a, b = m.cp_a, m.cp_b
        return (a + b * T, m.hf + a * (T - T0) + 0.5 * b * (T * T - T0 * T0),
                m.s0 + a * np.log(T / T0) + b * (T - T0))
    c = np.where((T < m.nasa[:, 1])[:, None], m.nasa[:, 3:10], m.nasa[:, 10:17])
    cp = R * (c[:, 0] + c[:, 1] * T + c[:, 2] * T ** 2 + c[:, 3] * T ** 3 + c[:, 4] * T ** 4)
    h = R * T * (c[:, 0] + c[:, 1] * T / 2 + c[:, 2] * T ** 2 / 3 + c[:, 3] * T ** 3 / 4 + c[:, 4] * T ** 4 / 5
                 + c[:, 5] / T)
    s = R * (c[:, 0] * np.log(T) + c[:, 1] * T + c[:, 2] * T ** 2 / 2 + c[:, 3] * T ** 3 / 3
             + c[:, 4] * T ** 4 / 4 + c[:, 6])
    return cp, h, s


def numpy_rhs(m, p):
    """f(T, Y) at pressure p from the mechanism's definitions: ideal gas,
    mass action, K_c from the Gibbs energies, third bodies with
    efficiencies, Lindemann/Troe fall-off, PLOG log-pressure interpolation."""
    nr, npd = m.nu_matrix()
    nu = (npd - nr).astype(float)
    dnu = nu.sum(axis=0)
    E = np.zeros((m.nrx, m.nsp))
    E[np.asarray(m.thirdbody) != 0] = 1.0
    for j, k, e in m.eff:
        E[j, k] = e
    tb = np.asarray(m.thirdbody) != 0
    rev = np.asarray(m.reversible) != 0
    fall = {int(r[0]): r for r in m.falloff}
    plog = {int(j): pts for j, pts in m.plog}
    W = m.W

    def arrhenius(lnA, beta, Ea, T):
        return np.exp(lnA + beta * np.log(T) - Ea / (R * T))

    def f(t, y):
        T, Y = y[0], y[1:]
        rho = 1e-6 * p / (R * T * np.sum(Y / W))                  # g/cm^3
        c = rho * Y / W                                           # mol/cm^3
        cp, h, s = _thermo(m, T)
        g = h - T * s
        kf = arrhenius(m.lnA, m.beta, m.Ea, T)
        M = np.where(tb, E @ c, 1.0)
        for j, pts in plog.items():                               # ln k linear in ln p, clamped
            lnk = [lp[1] + lp[2] * np.log(T) - lp[3] / (R * T) for lp in pts]
            kf[j] = np.exp(np.interp(np.log(p), [np.log(q[0]) for q in pts], lnk))
        for j, r in fall.items():
            k0 = arrhenius(r[2], r[3], r[4], T)
            Pr = k0 * M[j] / kf[j]
            F = 1.0
            if r[1] >= 2:
                Fc = (1 - r[5]) * np.exp(-T / r[6]) + r[5] * np.exp(-T / r[7]) + (np.exp(-r[8] / T) if r[1] == 3 else 0)
                cc, nn = -0.4 - 0.67 * np.log10(Fc), 0.75 - 1.27 * np.log10(Fc)
                x = np.log10(Pr) + cc
                F = 10 ** (np.log10(Fc) / (1 + (x / (nn - 0.14 * x)) ** 2))
            kf[j] *= Pr / (1 + Pr) * F
            M[j] = 1.0
        Kc = np.exp(-(nu.T @ g) / (R * T)) * (1.0 / (RC * T)) ** dnu
        fwd = kf * np.prod(c[:, None] ** nr, axis=0)
        bwd = np.where(rev, kf / Kc * np.prod(c[:, None] ** npd, axis=0), 0.0)
        w = nu @ (M * (fwd - bwd))
        cpm = np.sum(Y * cp / W)
        return np.concatenate([[-np.sum(h * w) / (rho * cpm)], W * w / rho])
    return f


def _check(mech, T, p, Y, dt, rtol, atol, m=None):
    orc = oracle.Oracle(mech)
    To, Yo, steps, st = orc.integrate(T, p, Y, dt, rtol=rtol, atol=atol)
    assert (st == 0).all()
    m = m if m is not None else read_mech(mech)
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


def test_real_mechanism_features_against_radau(tmp_path):
    """The 10-species mechanism with NASA-7 thermo, fall-off (Lindemann and
    Troe, listed efficiencies) and PLOG reactions, at pressures across the
    PLOG range and the fall-off region."""
    from synth import with_falloff, with_nasa7, with_plog, write_mech
    m = with_plog(with_falloff(with_nasa7(read_mech(states.mech_path(10, 20, 0)), 0), 0), 0, frac=0.5)
    assert m.falloff and m.plog and m.nasa is not None
    path = str(tmp_path / "all.bin")
    write_mech(path, m)
    T, p, Y = states.uniform_states(10, 6, 23)
    p = np.geomspace(5e3, 5e7, 6)
    wT, wY, To, T0_ = _check(path, T, p, Y, 1e-6, 1e-9, 1e-13)
    print(f"10 species, NASA-7 + fall-off + PLOG: max |dT|/T {wT:.2e}, max |dY| {wY:.2e}")
    assert np.abs(To - T0_).max() > 1.0
    assert wT < 1e-8 and wY < 1e-8

