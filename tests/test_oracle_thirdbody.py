"""Pins of the oracle's third-body factor [M] (CPU only).

A third-body reaction's net rate is multiplied by [M] = sum_k eff_k c_k, with
c_k in mol/cm^3 (the unit convention of the mechanism constants). These tests
fix both the magnitude of [M] and the handling of efficiencies with closed
forms that do not go through the oracle's own formula:

* unit efficiencies: [M] is the total molar concentration, which for an ideal
  gas is p / (R T) whatever the composition (1e-6 p / (R T) mol/cm^3, p in Pa);
* a uniform efficiency e: [M] = e p / (R T);
* efficiency 0 for the product of 2A (+M) -> B and 1 for A: [M] = c_A, so
  the rate law becomes third order in A, with its own closed form.

The reaction is the dimerisation 2A (+M) -> B with W_B = 2 W_A and
h_B = 2 h_A (isothermal at constant p). With a = 2 P'/T, P' = 1e-6 p / R and
Y the mass fraction of A, c_A = a Y / (1 + Y) and rho = a W_A / (1 + Y), so
dY/dt = -2 W_A q / rho gives
  q = k [M] c_A^2, [M] = e P'/T:  ln Y - 1/Y = C - 2 k e a (P'/T) t
  q = k c_A^3 ([M] = c_A):        ln Y - 2/Y - 1/(2 Y^2) = C - 2 k a^2 t
A slip in the units of [M] (mol/m^3 for mol/cm^3), in its temperature
dependence or in the efficiencies changes the decay by orders of magnitude.
"""
import numpy as np
import pytest
from scipy import optimize

import oracle
from tests import tinymech

R = 8.314462618
P_ATM = 101325.0

A_SP = dict(atoms=(1, 1, 0, 0), hf=-10e3, s0=200.0, a=30.0, b=0.002)
B_SP = dict(atoms=(2, 2, 0, 0), hf=-20e3, s0=400.0, a=60.0, b=0.004)


def _dimer(path, lnA, eff=()):
    tinymech.make(path, [A_SP, B_SP], [dict(reac=[(0, 2)], prod=[(1, 1)], lnA=lnA, rev=0, tb=1)], eff=eff)
    return oracle.Oracle(str(path))


def _run(orc, T, p, Y0, dt, rtol=1e-8):
    Y = np.vstack([Y0, 1 - Y0])
    To, Yo, steps, st = orc.integrate(T, p, Y, dt, rtol=rtol, atol=1e-14)
    assert (st == 0).all()
    np.testing.assert_allclose(To, T, rtol=1e-13)
    return Yo[0]


@pytest.mark.parametrize("e", [1.0, 2.5, 0.4])
def test_uniform_efficiency_closed_form(tmp_path, e):
    """[M] = e p/(R T): the second-order closed form with k -> k e P'/T."""
    lnA = np.log(3e15)
    eff = [] if e == 1.0 else [(0, 0, e), (0, 1, e)]
    orc = _dimer(tmp_path / "m.bin", lnA, eff)
    T = np.array([1000.0, 1500.0, 1200.0])
    p = np.array([P_ATM, P_ATM, 20e5])
    Y0 = np.array([1.0, 0.7, 0.9])
    dt, rtol = 1e-6, 1e-8
    Yo = _run(orc, T, p, Y0, dt, rtol)
    Pp = 1e-6 * p / R
    kap = 4.0 * np.exp(lnA) * e * (Pp / T) * Pp / T
    for i in range(T.size):
        F = lambda y: np.log(y) - 1 / y - (np.log(Y0[i]) - 1 / Y0[i] - kap[i] * dt)
        ye = optimize.brentq(F, 1e-12, Y0[i], xtol=1e-16, rtol=1e-15)
        assert ye < 0.95 * Y0[i]                       # the reaction does visible work
        assert Yo[i] == pytest.approx(ye, rel=10 * rtol)


def test_zero_efficiency_of_the_product_makes_the_rate_third_order(tmp_path):
    """eff_B = 0, eff_A = 1: [M] = c_A, q = k c_A^3."""
    lnA = np.log(2e20)
    orc = _dimer(tmp_path / "m.bin", lnA, eff=[(0, 1, 0.0)])
    T = np.array([1000.0, 1400.0])
    p = np.array([P_ATM, 5 * P_ATM])
    Y0 = np.array([1.0, 0.8])
    dt, rtol = 1e-6, 1e-8
    Yo = _run(orc, T, p, Y0, dt, rtol)
    a = 2e-6 * p / (R * T)
    kap = 2.0 * np.exp(lnA) * a * a
    G = lambda y: np.log(y) - 2 / y - 0.5 / (y * y)
    for i in range(T.size):
        ye = optimize.brentq(lambda y: G(y) - (G(Y0[i]) - kap[i] * dt), 1e-9, Y0[i], xtol=1e-16, rtol=1e-15)
        assert ye < 0.95 * Y0[i]
        assert Yo[i] == pytest.approx(ye, rel=10 * rtol)


def test_initial_rate_matches_ideal_gas_third_body(tmp_path):
    """Over a tiny dt the change of Y_B is dt W_B q / rho with
    q = k [M] c_A^2; here [M], c_A and rho come from the ideal gas law and the
    mole fractions, never from the oracle, for mixed efficiencies (A 1.7,
    B 0.3) where [M] = (P'/T)(1.7 X_A + 0.3 X_B)."""
    lnA = np.log(1e15)
    orc = _dimer(tmp_path / "m.bin", lnA, eff=[(0, 0, 1.7), (0, 1, 0.3)])
    T = np.array([900.0, 1300.0])
    p = np.array([P_ATM, 10 * P_ATM])
    Y0 = np.array([0.6, 0.35])
    WA = 12.011 + 1.008
    WB = 2 * WA
    dt = 1e-15                                 # the rate changes by ~1e-8 over dt
    Y = np.vstack([Y0, 1 - Y0])
    To, Yo, steps, st = orc.integrate(T, p, Y, dt, rtol=1e-10, atol=1e-20)
    assert (st == 0).all()
    nA, nB = Y0 / WA, (1 - Y0) / WB
    XA, XB = nA / (nA + nB), nB / (nA + nB)
    ctot = 1e-6 * p / (R * T)                  # mol/cm^3
    M = ctot * (1.7 * XA + 0.3 * XB)
    cA = ctot * XA
    rho = ctot * (XA * WA + XB * WB)            # g/cm^3
    q = np.exp(lnA) * M * cA * cA
    rate = (Yo[1] - Y[1]) / dt
    np.testing.assert_allclose(rate, WB * q / rho, rtol=2e-7)
    # the same concentrations through the oracle's rate evaluation
    for i in range(T.size):
        c, kf, kr, qo = orc.rates(p[i], np.array([T[i], Y0[i], 1 - Y0[i]]))
        np.testing.assert_allclose(c, [cA[i], ctot[i] * XB[i]], rtol=1e-13)
        assert qo[0] == pytest.approx(q[i], rel=1e-12)
