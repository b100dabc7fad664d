"""The seeded generators: stored mechanisms match their recipe, states are valid."""
import numpy as np
import pytest

from synth import generate_mechanism, read_mech, states


@pytest.mark.parametrize("nsp,nrx,seed", [(10, 20, 0), (53, 325, 0), (100, 1000, 1)])
def test_stored_mechanism_recipe(nsp, nrx, seed):
    m = read_mech(states.mech_path(nsp, nrx, seed))
    assert (m.nsp, m.nrx) == (nsp, nrx)
    nr, npd = m.nu_matrix()
    assert np.abs(m.atoms.T @ (npd - nr)).max() == 0            # element balance
    assert ((nr + npd).sum(1) > 0).all()                        # every species reacts
    assert m.atoms.min() >= 0 and m.atoms.max() <= 3
    assert len({tuple(a) for a in m.atoms}) == nsp              # distinct species
    assert m.thirdbody.sum() == round(0.1 * nrx)
    assert ((npd - nr).T @ m.hf <= 0).all()                    # forward exothermic at T0
    assert np.all((np.exp(m.lnA) >= 1e6 * (1 - 1e-12)) & (np.exp(m.lnA) <= 1e14 * (1 + 1e-12)))
    assert np.all(np.abs(m.beta) <= 1) and np.all((m.Ea >= 0) & (m.Ea <= 200e3))
    np.testing.assert_allclose(m.W, m.atoms @ np.array([12.011, 1.008, 15.999, 14.007]), rtol=1e-14)


def test_generator_is_deterministic_and_matches_stored():
    a = generate_mechanism(10, 20, 0)
    b = read_mech(states.mech_path(10, 20, 0))
    np.testing.assert_array_equal(a.lnA, b.lnA)
    assert a.reac == [list(map(tuple, r)) for r in b.reac]


def test_bimodal_states():
    n = 4096
    T, p, Y, cls = states.bimodal_states(53, 325, n, 0)
    assert Y.shape == (53, n) and (p == 20e5).all()
    np.testing.assert_allclose(Y.sum(0), 1.0, atol=1e-13)
    frac = np.bincount(cls, minlength=3) / n
    np.testing.assert_allclose(frac, [0.45, 0.45, 0.10], atol=1e-3)
    assert T[cls == 0].min() >= 300 * (1 - 3e-5) and T[cls == 0].max() <= 600 * (1 + 3e-5)
    assert T[cls == 1].min() >= 1800 * (1 - 2e-6) and T[cls == 1].max() <= 2300 * (1 + 2e-6)
    assert T[cls == 2].min() >= 900 and T[cls == 2].max() <= 1600
    # cold cells come from 8 ambient states: they cluster within the mapping tolerance
    Tc = np.sort(np.unique(np.round(T[cls == 0], 0)))
    assert len(np.unique(np.round(T[cls == 0] / 10))) <= 8 * 2


def test_uniform_states():
    T, p, Y = states.uniform_states(10, 1024, 0)
    assert T.min() >= 300 and T.max() <= 2500 and (p == 101325.0).all()
    np.testing.assert_allclose(Y.sum(0), 1.0, atol=1e-13)
