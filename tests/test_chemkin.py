"""CHEMKIN-format text reader (CPU only): a written-out generated mechanism
reads back to the same mechanism (round trip through the text, NASA-7 thermo,
third bodies with efficiencies, fall-off, PLOG), a hand-written text with the
syntax variants reads to the values written in it, and what the reader does
not take is refused."""
import math

import numpy as np
import pytest

import oracle
from synth import read_mech, states, with_falloff, with_nasa7, with_plog, write_mech
from synth.chemkin import read_chemkin, write_chemkin


def test_round_trip_of_a_generated_mechanism(tmp_path):
    m = with_plog(with_falloff(with_nasa7(read_mech(states.mech_path(10, 20, 0)), 0), 0), 0, frac=0.5)
    assert m.falloff and m.plog and m.eff
    text = write_chemkin(m)
    r = read_chemkin(text)
    assert r.nsp == m.nsp and r.nrx == m.nrx
    np.testing.assert_array_equal(r.atoms, m.atoms)
    np.testing.assert_allclose(r.W, m.W, rtol=1e-15)
    np.testing.assert_allclose(r.nasa, m.nasa, rtol=1e-8, atol=1e-12)   # 9 significant digits in THERMO
    np.testing.assert_allclose(r.lnA, m.lnA, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r.beta, m.beta, rtol=1e-15)
    np.testing.assert_allclose(r.Ea, m.Ea, rtol=1e-15)
    assert r.reac == m.reac and r.prod == m.prod
    np.testing.assert_array_equal(r.reversible, m.reversible)
    np.testing.assert_array_equal(r.thirdbody, m.thirdbody)
    assert sorted(r.eff) == pytest.approx(sorted(m.eff))
    assert [f[:2] for f in r.falloff] == [f[:2] for f in m.falloff]
    for a, b in zip(r.falloff, m.falloff):       # the parameters each form uses (Lindemann: no Troe ones)
        used = {1: 5, 2: 8, 3: 9}[b[1]]
        np.testing.assert_allclose(a[2:used], b[2:used], rtol=1e-13, atol=1e-12)
    assert [j for j, _ in r.plog] == [j for j, _ in m.plog]
    for (_, a), (_, b) in zip(r.plog, m.plog):
        np.testing.assert_allclose(np.array(a), np.array(b), rtol=1e-13, atol=1e-12)
    # and the same chemistry
    pa, pb = str(tmp_path / "orig.bin"), str(tmp_path / "read.bin")
    write_mech(pa, m)
    write_mech(pb, r)
    T, p, Y = states.uniform_states(10, 64, 2)
    p[:] = np.geomspace(1e4, 2e7, 64)
    oa = oracle.Oracle(pa).integrate(T, p, Y, 1e-6, rtol=1e-8, atol=1e-12)
    ob = oracle.Oracle(pb).integrate(T, p, Y, 1e-6, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(ob[0], oa[0], rtol=1e-8)
    np.testing.assert_allclose(ob[1], oa[1], atol=1e-8)


THERMO = """THERMO ALL
   300.000  1000.000  5000.000
AX                      C   1H   1          G   300.000  5000.000 1000.00      1
 3.00000000E+00 1.00000000E-03 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
-1.00000000E+03 2.00000000E+00 3.50000000E+00 5.00000000E-04 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00-1.20000000E+03 4.00000000E+00                   4
BY                      O   2               G   300.000  5000.000 1200.00      1
 4.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
-2.00000000E+03 1.00000000E+00 4.00000000E+00 0.00000000E+00 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00-2.00000000E+03 1.00000000E+00                   4
CZ                      C   1H   1O   2     G   300.000  5000.000              1
 6.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
-5.00000000E+03 3.00000000E+00 6.00000000E+00 0.00000000E+00 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00-5.00000000E+03 3.00000000E+00                   4
END
"""

MECH = """! a made-up three-species mechanism with every form the reader takes
ELEMENTS
C H O
END
SPECIES AX BY
CZ
END
REACTIONS KCAL/MOLE
AX + BY <=> CZ        1.0E13  0.0   10.0   ! plain, reversible
AX+BY+M=>CZ+M         2.0E15 -1.0   0.0
   BY/2.5/ CZ/0.0/
AX+BY(+M) = CZ(+M)    3.0E12  0.5   5.0
   LOW / 4.0E18 -1.5 1.0 /
   TROE / 0.6 300.0 2000.0 /
CZ => AX + BY         5.0E9   0.0   20.0
   PLOG / 0.1 1.0E8 0.0 18.0 /
   PLOG / 10.0 1.0E10 0.2 21.0 /
CZ => AX + BY         1.0E9   0.0   25.0
   DUPLICATE
END
"""


def test_hand_written_text_reads_to_its_values():
    m = read_chemkin(MECH, THERMO)
    assert m.nsp == 3 and m.nrx == 5
    np.testing.assert_array_equal(m.atoms, [[1, 1, 0, 0], [0, 0, 2, 0], [1, 1, 2, 0]])
    cal = 4184.0
    assert m.reac[0] == [(0, 1), (1, 1)] and m.prod[0] == [(2, 1)] and m.reversible[0] == 1
    assert m.lnA[0] == pytest.approx(math.log(1e13)) and m.Ea[0] == pytest.approx(10.0 * cal)
    assert m.reac[1] == [(0, 1), (1, 1)] and m.prod[1] == [(2, 1)] and m.reversible[1] == 0 and m.thirdbody[1] == 1
    assert sorted(e for e in m.eff if e[0] == 1) == [(1, 1, 2.5), (1, 2, 0.0)]
    assert m.thirdbody[2] == 1 and m.reversible[2] == 1
    (j, kind, lnA0, b0, E0, a, T3, T1, T2), = m.falloff
    assert (j, kind) == (2, 2)
    assert lnA0 == pytest.approx(math.log(4e18)) and b0 == -1.5 and E0 == pytest.approx(1.0 * cal)
    assert (a, T3, T1) == (0.6, 300.0, 2000.0)
    (j, pts), = m.plog
    assert j == 3
    np.testing.assert_allclose(pts, [(0.1 * 101325.0, math.log(1e8), 0.0, 18.0 * cal),
                                     (10.0 * 101325.0, math.log(1e10), 0.2, 21.0 * cal)])
    assert m.reac[4] == [(2, 1)] and m.prod[4] == [(0, 1), (1, 1)]
    # thermo: high set first in the text, Tmid from the entry or the THERMO ALL line
    np.testing.assert_allclose(m.nasa[0], [300, 1000, 5000, 3.5, 5e-4, 0, 0, 0, -1200, 4.0,
                                           3.0, 1e-3, 0, 0, 0, -1000, 2.0])
    assert m.nasa[1, 1] == 1200.0 and m.nasa[2, 1] == 1000.0


@pytest.mark.parametrize("bad", [
    MECH.replace("C H O", "C H O AR"),
    MECH.replace("AX+BY+M=>CZ+M", "AX+BY+M=>CZ"),
    MECH.replace("AX+BY+M=>CZ+M", "3AX+BY+M=>CZ+M"),
    MECH.replace("AX+BY+M=>CZ+M", "2AX+M=>CZ+AX+M"),
    MECH.replace("   DUPLICATE", "   REV / 1.0E9 0.0 5.0 /"),
    MECH.replace("AX + BY <=> CZ", "0.5AX + BY <=> CZ"),
    MECH.replace("AX+BY(+M) = CZ(+M)", "AX+BY(+BY) = CZ(+BY)"),
    MECH.replace("REACTIONS KCAL/MOLE", "REACTIONS MOLECULES"),
    MECH.replace("   LOW / 4.0E18 -1.5 1.0 /\n", ""),
])
def test_refuses_what_it_does_not_read(bad):
    with pytest.raises(ValueError):
        read_chemkin(bad, THERMO)


def test_command_line_writes_a_mechanism_file(tmp_path):
    """python -m synth.chemkin mech.inp thermo.dat out.bin: the file the
    oracle then loads and integrates (element totals kept)."""
    import subprocess
    import sys
    mech, thermo, out = tmp_path / "m.inp", tmp_path / "t.dat", tmp_path / "m.bin"
    mech.write_text(MECH)
    thermo.write_text(THERMO)
    r = subprocess.run([sys.executable, "-m", "synth.chemkin", str(mech), str(thermo), str(out)],
                       capture_output=True, text=True, cwd=str(__import__("pathlib").Path(__file__).parents[1]))
    assert r.returncode == 0, r.stderr
    assert "3 species, 5 reactions, 1 fall-off, 1 PLOG" in r.stdout
    m = read_mech(str(out))
    T = np.array([1200.0, 1500.0])
    Y = np.array([[0.5, 0.2], [0.3, 0.5], [0.2, 0.3]])
    To, Yo, _, st = oracle.Oracle(str(out)).integrate(T, np.array([1e5, 2e6]), Y, 1e-5, rtol=1e-8, atol=1e-12)
    assert (st == 0).all()
    aW = m.atoms.T / m.W[None, :]
    np.testing.assert_allclose(aW @ Yo, aW @ Y, rtol=1e-10, atol=1e-14)
