"""Reference mapping in the oracle (Sec. 2.3 reading; CPU only): the error it
introduces falls as the tolerance falls, and vanishes at tolerance 0.

Cold cells of the bimodal field around one ambient state, the first of them
supplying the reference composition. It qualifies at any positive tolerance,
so the reference cell is the same for every tolerance and the mapped sets
are nested: the largest difference between mapped and integrated results
cannot grow as the tolerance shrinks, and at 0 nothing maps and the result is
the unmapped run bit for bit."""
import numpy as np

import oracle
from synth import states


def test_mapping_error_falls_with_the_tolerance():
    mech = states.mech_path(53, 325, 0)
    T, p, Y, cls = states.bimodal_states(53, 325, 4096, 3)
    cold = np.flatnonzero(cls == 0)
    c0 = cold[0]
    dist = np.maximum(np.abs(Y[:, cold] - Y[:, [c0]]).max(axis=0), np.abs(T[cold] - T[c0]) / T[c0])
    near = cold[np.argsort(dist, kind="stable")[:96]]            # c0 first (distance 0)
    assert near[0] == c0
    sel = np.concatenate([near, cold[np.argsort(dist, kind="stable")[-24:]]])
    orc = oracle.Oracle(mech)
    args = (T[sel], p[sel], Y[:, sel], 1e-5)
    base = orc.integrate(*args, rtol=1e-5, atol=1e-8)
    assert (base[3] == 0).all()
    errs, counts, prev_mapped = [], [], None
    for tol in (1e-3, 1e-4, 3e-5, 1e-5, 3e-6, 0.0):
        r = orc.integrate(*args, rtol=1e-5, atol=1e-8, mapping=True, map_Ttol=tol, map_Ytol=tol)
        mapped = r[3] == 1
        assert r[3][0] == 0                                        # the reference is integrated
        if prev_mapped is not None:
            assert not (mapped & ~prev_mapped).any()               # nested as the tolerance shrinks
        prev_mapped = mapped
        err = 0.0
        if mapped.any():
            err = max(float(np.abs(r[1][:, mapped] - base[1][:, mapped]).max()),
                      float((np.abs(r[0][mapped] - base[0][mapped]) / base[0][mapped]).max()))
            # integrated cells are untouched by mapping
            np.testing.assert_array_equal(r[0][~mapped], base[0][~mapped])
        errs.append(err)
        counts.append(int(mapped.sum()))
    assert counts[0] > counts[-2] > 0 and counts[-1] == 0, counts
    assert all(a >= b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] == 0.0
    r0 = orc.integrate(*args, rtol=1e-5, atol=1e-8, mapping=True, map_Ttol=0.0, map_Ytol=0.0)
    np.testing.assert_array_equal(r0[0], base[0])
    np.testing.assert_array_equal(r0[1], base[1])
