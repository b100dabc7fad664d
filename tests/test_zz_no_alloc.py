"""dlbchem_integrate_static, the queued integration for callers that may not
allocate device memory while they run (a flow solver that reserved its whole
memory budget at start-up), checked against dlbchem_integrate with the same
queue schedule on two calls in a row, in FP64 and in mixed precision, and
checked to leave the device's free memory unchanged. Kept last in collection
order so that a failure here never hides another test; it also passes on its
own in a fresh process."""
import numpy as np
import pytest

from synth import states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _lib():
    from paper_2011_07978_gb300 import build, dlbchem
    build.build()
    return dlbchem


def _field(n, seed=11):
    T, p, Y, cls = states.bimodal_states(53, 325, n, seed)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
    return d(T), d(p), d(Y)


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_matches_dlbchem_integrate_twice(precision):
    d = _lib()
    mech = states.mech_path(53, 325, 0)
    n = 3000
    T, p, Y = _field(n)
    ctx_ref = d.Context(mech, rtol=1e-5, atol=1e-8, schedule=d.SCHED_QUEUE, precision=precision)
    ctx = d.Context(mech, rtol=1e-5, atol=1e-8, precision=precision)
    steps_ref = torch.zeros(n, dtype=torch.int32, device=DEV)
    steps = torch.zeros(n, dtype=torch.int32, device=DEV)
    for call in range(2):       # second call sorts by the first call's step counts
        st_ref = torch.full((n,), 99, dtype=torch.int32, device=DEV)
        st = torch.full((n,), 99, dtype=torch.int32, device=DEV)
        To_ref, Yo_ref = ctx_ref.integrate(T, p, Y, 1e-5, steps=steps_ref, status=st_ref)
        To, Yo = torch.empty_like(T), torch.empty_like(Y)
        ctx.integrate_static(T, p, Y, 1e-5, To, Yo, steps=steps, status=st)
        torch.cuda.synchronize()
        a, b = To.cpu().numpy(), To_ref.cpu().numpy()
        assert np.all(np.abs(a - b) <= 1e-5 * b), call
        assert np.abs(Yo.cpu().numpy() - Yo_ref.cpu().numpy()).max() <= 1e-9, call
        np.testing.assert_array_equal(st.cpu().numpy(), st_ref.cpu().numpy())
        np.testing.assert_array_equal(steps.cpu().numpy(), steps_ref.cpu().numpy())
        assert (st.cpu().numpy() == 0).all()
        stats = ctx.last_stats()
        assert stats["integrated"] == n and stats["mapped"] == 0 and stats["precision"] == precision
        if precision == 1:
            assert stats["fp64_fallbacks"] == ctx_ref.last_stats()["fp64_fallbacks"]


def test_static_call_leaves_free_device_memory_unchanged():
    """After one call (which loads the scheduling kernels), a call on a
    larger field than before changes nothing in cudaMemGetInfo."""
    d = _lib()
    mech = states.mech_path(53, 325, 0)
    ctx = d.Context(mech, rtol=1e-5, atol=1e-8)
    small, big = _field(500, 12), _field(4000, 13)
    outs = [(torch.empty_like(f[0]), torch.empty_like(f[2]), torch.zeros(f[0].numel(), dtype=torch.int32, device=DEV))
            for f in (small, big)]
    (Ts, ps, Ys), (Tb, pb, Yb) = small, big
    ctx.integrate_static(Ts, ps, Ys, 1e-5, outs[0][0], outs[0][1], steps=outs[0][2])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    ctx.integrate_static(Tb, pb, Yb, 1e-5, outs[1][0], outs[1][1], steps=outs[1][2])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0, (free0, free1)
    assert torch.isfinite(outs[1][0]).all()


def test_static_scratch_rejects_fields_above_its_limit():
    d = _lib()
    ctx = d.Context(states.mech_path(10, 20, 0))
    n = d.STATIC_MAX_CELLS + 1
    T = torch.full((n,), 1000.0, dtype=torch.float64, device=DEV)
    p = torch.full((n,), 101325.0, dtype=torch.float64, device=DEV)
    Y = torch.full((10, n), 0.1, dtype=torch.float64, device=DEV)
    with pytest.raises(d.DlbchemError) as ei:
        ctx.integrate_static(T, p, Y, 1e-6, torch.empty_like(T), torch.empty_like(Y))
    assert ei.value.code == d.BAD_ARG and "DLBCHEM_STATIC_MAX_CELLS" in str(ei.value)
