"""The learned cost predictor and surrogate (needs a GB300).

* The BF16 tensor-core network's loss and gradients match the FP64 CPU
  oracle network (oracle/mlp.py) per tensor within 2e-2 relative, cosine
  >= 0.999; the whole-network forward kernel matches the layer-by-layer one
  and the oracle.
* Trained on integrator trajectories of the 10-species case, the predicted
  step counts order the queue better than index order (makespan of greedy
  scheduling on the true costs), cells that fail the gate are integrated
  bit-identically to the plain path, and accepted cells satisfy the gate.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from synth import read_mech, states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def lib():
    from paper_2011_07978_gb300 import build, dlbchem
    build.build()
    return dlbchem


def _per_tensor(theta, shapes):
    out, o = [], 0
    for a, b in shapes:
        out.append(theta[o:o + a * b]); o += a * b
        out.append(theta[o:o + b]); o += b
    return out


@pytest.mark.parametrize("B", [96, 1000])
def test_network_gradients_match_fp64_oracle(B):
    """Forward and backward on the tensor cores (tcgen05, BF16, FP32
    accumulator in tensor memory) against the FP64 oracle network: B = 96 is a
    partial 128-row tile, B = 1000 spans eight row tiles and, for the weight
    gradients, sixteen accumulated k-tiles."""
    d = lib()
    n_in, n_out = 13, 12
    shapes = omlp.layer_shapes(n_in, 256, n_out)
    rng = np.random.default_rng(3)
    theta = omlp.init_params(n_in, 256, n_out, seed=5) + rng.normal(0, 0.02, omlp.n_params(n_in, 256, n_out))
    theta = theta.astype(np.float32).astype(np.float64)
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    Y = rng.normal(size=(B, n_out)).astype(np.float32)
    loss_ref, g_ref = omlp.loss_and_grad(theta, X.astype(np.float64), Y.astype(np.float64), shapes)
    out_ref, _ = omlp.forward(theta, X.astype(np.float64), shapes)
    net = d.MLP(n_in, 256, n_out)
    assert net.nparams == theta.size
    net.set_params(torch.tensor(theta.astype(np.float32), device=DEV))
    Xd, Yd = torch.tensor(X, device=DEV), torch.tensor(Y, device=DEV)
    out = net.forward(Xd, torch.empty((B, n_out), dtype=torch.float32, device=DEV))
    g = torch.zeros(net.nparams, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    net.grad(Xd, Yd, grad=g, loss=loss)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    assert np.linalg.norm(out - out_ref) <= 2e-2 * np.linalg.norm(out_ref)
    assert abs(float(loss.item()) - loss_ref) <= 2e-2 * loss_ref
    for gg, gr in zip(_per_tensor(g.cpu().numpy().astype(np.float64), shapes), _per_tensor(g_ref, shapes)):
        rel = np.linalg.norm(gg - gr) / np.linalg.norm(gr)
        cos = gg @ gr / (np.linalg.norm(gg) * np.linalg.norm(gr))
        assert rel <= 2e-2 and cos >= 0.999, (rel, cos)


@pytest.mark.parametrize("n_in,hidden,n_out,B", [(13, 256, 12, 96), (13, 256, 12, 5000), (56, 256, 55, 777),
                                                  (13, 128, 12, 1000)])
def test_fused_forward_matches_layered_and_oracle(n_in, hidden, n_out, B):
    """The whole-network forward kernel (activations kept in shared memory,
    weights streamed as packed BF16 k-tiles by bulk copy) against the
    layer-by-layer tensor-core forward (same BF16 operands, FP32 accumulation
    over k-tiles of 64, FP32 bias and SiLU) and against the FP64 oracle
    network. Batches end in a partial 128-row tile except at 5000 - 4992 = 8."""
    d = lib()
    shapes = omlp.layer_shapes(n_in, hidden, n_out)
    rng = np.random.default_rng(11)
    theta = omlp.init_params(n_in, hidden, n_out, seed=7) + rng.normal(0, 0.02, omlp.n_params(n_in, hidden, n_out))
    theta = theta.astype(np.float32).astype(np.float64)
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    out_ref, _ = omlp.forward(theta, X.astype(np.float64), shapes)
    net = d.MLP(n_in, hidden, n_out)
    assert net.fused
    net.set_params(torch.tensor(theta.astype(np.float32), device=DEV))
    Xd = torch.tensor(X, device=DEV)
    fused = net.forward(Xd, torch.full((B, n_out), float("nan"), dtype=torch.float32, device=DEV)).cpu().numpy()
    net.set_fused(False)
    assert not net.fused
    layered = net.forward(Xd, torch.full((B, n_out), float("nan"), dtype=torch.float32, device=DEV)).cpu().numpy()
    net.set_fused(True)
    again = net.forward(Xd, torch.full((B, n_out), float("nan"), dtype=torch.float32, device=DEV)).cpu().numpy()
    assert np.isfinite(fused).all() and np.isfinite(layered).all()
    np.testing.assert_array_equal(again, fused)                       # repacked weights are reused
    scale = np.abs(layered).max()
    assert np.abs(fused - layered).max() <= 1e-5 * scale, np.abs(fused - layered).max() / scale
    for o in (fused, layered):
        assert np.linalg.norm(o - out_ref) <= 2e-2 * np.linalg.norm(out_ref)
    # new parameters are repacked before the next fused forward
    net.set_params(torch.tensor((theta * 0.5).astype(np.float32), device=DEV))
    half = net.forward(Xd, torch.empty((B, n_out), dtype=torch.float32, device=DEV)).cpu().numpy()
    out_half, _ = omlp.forward(theta * 0.5, X.astype(np.float64), shapes)
    assert np.linalg.norm(half - out_half) <= 2e-2 * np.linalg.norm(out_half)
    net.close()


def test_fused_forward_declines_other_shapes():
    """A hidden width that is not a multiple of 64 runs layer by layer."""
    d = lib()
    net = d.MLP(13, 96, 12)
    assert not net.fused
    shapes = omlp.layer_shapes(13, 96, 12)
    theta = omlp.init_params(13, 96, 12, seed=2).astype(np.float32).astype(np.float64)
    X = np.random.default_rng(4).normal(size=(300, 13)).astype(np.float32)
    net.set_params(torch.tensor(theta.astype(np.float32), device=DEV))
    out = net.forward(torch.tensor(X, device=DEV), torch.empty((300, 12), dtype=torch.float32, device=DEV)).cpu().numpy()
    ref, _ = omlp.forward(theta, X.astype(np.float64), shapes)
    assert np.linalg.norm(out - ref) <= 2e-2 * np.linalg.norm(ref)
    net.close()


def test_adam_step_matches_oracle():
    d = lib()
    net = d.MLP(13, 256, 12)
    rng = np.random.default_rng(0)
    theta = rng.normal(size=net.nparams).astype(np.float32)
    g = rng.normal(size=net.nparams).astype(np.float32)
    net.set_params(torch.tensor(theta, device=DEV))
    net.adam(1e-3, grad=torch.tensor(g, device=DEV))
    out = net.get_params(torch.empty(net.nparams, dtype=torch.float32, device=DEV)).cpu().numpy()
    ref, _, _ = omlp.adam_step(theta.astype(np.float64), g.astype(np.float64), np.zeros(net.nparams),
                               np.zeros(net.nparams), 1, 1e-3)
    np.testing.assert_allclose(out, ref, rtol=1e-5, atol=1e-7)


def _greedy_makespan(costs, P):
    """List scheduling: each cost goes to the team that frees up first."""
    import heapq
    heap = [0.0] * P
    for c in costs:
        t = heapq.heappop(heap)
        heapq.heappush(heap, t + c)
    return max(heap)


@pytest.fixture(scope="module")
def trained():
    d = lib()
    from paper_2011_07978_gb300 import learned
    mech = states.mech_path(10, 20, 0)
    ctx = d.Context(mech, rtol=1e-6, atol=1e-10)
    n = 49152
    T, p, Y = states.uniform_states(10, n, 100)
    dt = learned.dt_buckets(n, 100, nbuckets=8)
    X, Yt, steps, status = learned.generate(ctx, T, p, Y, dt)
    assert (status == 0).all()
    net = learned.train(X, Yt, epochs=12, batch=2048, lr=2e-3, seed=1)
    assert net.history[-1] < 0.5 * net.history[0]
    return d, learned, net, mech


def test_predictor_orders_the_queue_and_keeps_results(trained):
    d, learned, net, mech = trained
    n = 6000
    T, p, Y = states.uniform_states(10, n, 1)            # a fresh field: no previous steps
    dt = 4e-6
    dd = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
    plain = d.Context(mech, rtol=1e-6, atol=1e-10)
    st0 = torch.zeros(n, dtype=torch.int32, device=DEV)
    To0, Yo0 = plain.integrate(dd(T), dd(p), dd(Y), dt, steps=st0)
    ctx = d.Context(mech, rtol=1e-6, atol=1e-10, schedule=d.SCHED_QUEUE, predictor=1)
    ctx.attach_mlp(net)
    st = torch.zeros(n, dtype=torch.int32, device=DEV)
    To, Yo = ctx.integrate(dd(T), dd(p), dd(Y), dt, steps=st)
    wl = torch.zeros(n, dtype=torch.int32, device=DEV)
    m = ctx.last_worklist(wl)
    torch.cuda.synchronize()
    assert torch.equal(To, To0) and torch.equal(Yo, Yo0) and torch.equal(st, st0)
    cost = st0.cpu().numpy().astype(float)
    order = wl.cpu().numpy()[:m]
    P = 608
    span_index = _greedy_makespan(cost, P)
    span_pred = _greedy_makespan(cost[order], P)
    span_lpt = _greedy_makespan(np.sort(cost)[::-1], P)
    print(f"makespan in steps: index order {span_index:.0f}, predicted order {span_pred:.0f}, "
          f"exact LPT {span_lpt:.0f}")
    assert span_pred < span_index
    rank = np.corrcoef(np.argsort(np.argsort(-cost[order])), np.arange(m))[0, 1]
    assert rank > 0.3


def test_surrogate_gate_and_fallback(trained):
    d, learned, net, mech = trained
    n = 4000
    T, p, Y = states.uniform_states(10, n, 2)
    T[: n // 2] = np.random.default_rng(0).uniform(300, 420, n // 2)   # some nearly inert cold cells
    dt = 2e-6
    dd = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
    plain = d.Context(mech, rtol=1e-6, atol=1e-10)
    To0, Yo0 = plain.integrate(dd(T), dd(p), dd(Y), dt)
    gate = 1e-4
    ctx = d.Context(mech, rtol=1e-6, atol=1e-10, surrogate=1, gate=gate)
    ctx.attach_mlp(net)
    st = torch.zeros(n, dtype=torch.int32, device=DEV)
    ss = torch.zeros(n, dtype=torch.int32, device=DEV)
    To, Yo = ctx.integrate(dd(T), dd(p), dd(Y), dt, steps=st, status=ss)
    torch.cuda.synchronize()
    ss, To, Yo, To0, Yo0 = ss.cpu().numpy(), To.cpu().numpy(), Yo.cpu().numpy(), To0.cpu().numpy(), Yo0.cpu().numpy()
    acc = ss == d.CELL_SURROGATE
    integ = ss == 0
    assert acc.sum() + integ.sum() == n
    np.testing.assert_array_equal(To[integ], To0[integ])
    np.testing.assert_array_equal(Yo[:, integ], Yo0[:, integ])
    orc = oracle.Oracle(mech)
    m = read_mech(mech)
    for i in np.flatnonzero(acc)[:50]:
        y0 = np.concatenate([[T[i]], Y[:, i]])
        y1 = np.concatenate([[To[i]], Yo[:, i]])
        defect = y1 - y0 - 0.5 * dt * (orc.rhs(p[i], y0) + orc.rhs(p[i], y1))
        assert abs(defect[0]) <= gate * T[i] * 1.001 and np.abs(defect[1:]).max() <= gate * 1.001
        assert abs(Yo[:, i].sum() - 1) <= gate * 1.001
    err = np.abs(Yo[:, acc] - Yo0[:, acc]).max(axis=0) if acc.any() else np.zeros(0)
    print(f"surrogate accepted {acc.sum()} of {n} cells; max |dY| vs integrator on accepted "
          f"{err.max() if err.size else 0:.2e}")


def test_gate_accept_branch_with_a_host_built_network():
    """Drives the gate's accept branch with a network built on the host: all
    weights and biases zero and output normalisation mu = 0, sd = 1, so its
    output is exactly zero. With surrogate = 1 it proposes a zero increment,
    with surrogate = 2 the explicit Euler step y + dt f(y) and then the zero
    increment. On the bimodal
    field's near-equilibrium burnt cells (53 species, dt 1e-5) the gate
    accepts them, and never a flame-front cell. Accepted cells meet the gate
    against the oracle's right-hand side, their error against the oracle's
    integration (the increment they skip) is stated and at most twice the
    gate, and the other cells are integrated exactly as without the
    surrogate."""
    d = lib()
    mech = states.mech_path(53, 325, 0)
    T, p, Y, cls = states.bimodal_states(53, 325, 4000, 21)
    keep = np.flatnonzero(cls != states.COLD)          # burnt and front cells
    T, p, Y, cls = T[keep], p[keep], np.ascontiguousarray(Y[:, keep]), cls[keep]
    n, dt, gate = T.size, 1e-5, 1e-4
    net = d.MLP(56, 256, 55)
    net.set_params(torch.zeros(net.nparams, dtype=torch.float32, device=DEV))
    net.set_norm(np.zeros(56), np.ones(56), np.zeros(55), np.ones(55))
    dd = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
    plain = d.Context(mech, rtol=1e-5, atol=1e-8)
    To0, Yo0 = plain.integrate(dd(T), dd(p), dd(Y), dt)
    To0, Yo0 = To0.cpu().numpy(), Yo0.cpu().numpy()
    orc = oracle.Oracle(mech)
    accepted = {}
    for mode in (1, 2):
        ctx = d.Context(mech, rtol=1e-5, atol=1e-8, surrogate=mode, gate=gate)
        ctx.attach_mlp(net)
        st = torch.zeros(n, dtype=torch.int32, device=DEV)
        ss = torch.zeros(n, dtype=torch.int32, device=DEV)
        To, Yo = ctx.integrate(dd(T), dd(p), dd(Y), dt, steps=st, status=ss)
        torch.cuda.synchronize()
        ss, st, To, Yo = ss.cpu().numpy(), st.cpu().numpy(), To.cpu().numpy(), Yo.cpu().numpy()
        acc = ss == d.CELL_SURROGATE
        accepted[mode] = acc
        assert acc[cls == states.BURNT].mean() > 0.5 and not acc[cls == states.FRONT].any()
        assert ((ss == 0) | acc).all() and (st[acc] == 0).all()
        np.testing.assert_array_equal(To[~acc], To0[~acc])
        np.testing.assert_array_equal(Yo[:, ~acc], Yo0[:, ~acc])
        if mode == 1:
            np.testing.assert_array_equal(To[acc], T[acc])
            np.testing.assert_array_equal(Yo[:, acc], Y[:, acc])
        for i in np.flatnonzero(acc)[:300]:
            y0 = np.concatenate([[T[i]], Y[:, i]])
            y1 = np.concatenate([[To[i]], Yo[:, i]])
            f0, f1 = orc.rhs(p[i], y0), orc.rhs(p[i], y1)
            defect = y1 - y0 - 0.5 * dt * (f0 + f1)
            assert abs(defect[0]) <= gate * T[i] * (1 + 1e-6) and np.abs(defect[1:]).max() <= gate * (1 + 1e-6)
            assert abs(Yo[:, i].sum() - 1) <= gate and Yo[:, i].min() >= -gate
            # not stiff along the increment: dt |f(y') - f(y)| <= |y' - y| + 2 gate (T relative)
            w = np.concatenate([[1.0 / T[i]], np.ones(Y.shape[0])])
            lip, inc = (dt * np.abs(f1 - f0) * w).max(), (np.abs(y1 - y0) * w).max()
            assert lip <= (inc + 2 * gate) * (1 + 1e-6) + 1e-12
        sel = np.flatnonzero(acc)
        o = orc.integrate(T[sel], p[sel], Y[:, sel], dt, rtol=1e-5, atol=1e-8)
        err_T = np.abs(To[sel] - o[0]) / o[0]
        err_Y = np.abs(Yo[:, sel] - o[1]).max(axis=0)
        print(f"surrogate mode {mode} (zero network): accepted {sel.size} of {n} cells "
              f"({int(acc[cls == states.BURNT].sum())} of {int((cls == states.BURNT).sum())} burnt); vs the oracle's "
              f"integration max |dT|/T {err_T.max():.2e}, max |dY| {err_Y.max():.2e}")
        assert err_Y.max() <= 2 * gate and err_T.max() <= 2 * gate
    assert accepted[2].sum() >= accepted[1].sum()


def test_rhs_matches_oracle():
    """dlbchem_rhs against the oracle's right-hand side, cell by cell, on the
    10- and the 53-species mechanisms, fall-off and PLOG variants of the
    10-species one at 0.01 to 300 bar, and a NASA-7 variant of the 53-species
    one. The two sides evaluate rates, thermo
    and f in different orders, so they agree to rounding of the terms that
    make up each component: for f_Y_k the scale is W_k / rho times the sum of
    |nu_kr| [M]_r (forward_r + reverse_r) over the reactions (near
    equilibrium those cancel), for f_T that scale times |h_k| / cp."""
    d = lib()
    import tempfile
    from synth import with_falloff, with_nasa7, with_plog, write_mech
    fall = tempfile.NamedTemporaryFile(suffix=".bin", delete=False).name
    write_mech(fall, with_falloff(read_mech(states.mech_path(10, 20, 0)), 0))
    plog = tempfile.NamedTemporaryFile(suffix=".bin", delete=False).name
    write_mech(plog, with_plog(read_mech(states.mech_path(10, 20, 0)), 0, frac=0.5))
    Tf, pf, Yf = states.uniform_states(10, 300, 6)
    pf = np.geomspace(1e3, 1e7, 300)
    Tp, pp, Yp = states.uniform_states(10, 300, 7)
    pp = np.geomspace(3e3, 3e7, 300)
    nasa = tempfile.NamedTemporaryFile(suffix=".bin", delete=False).name
    write_mech(nasa, with_nasa7(read_mech(states.mech_path(53, 325, 0)), 0))
    for mech, (T, p, Y) in ((states.mech_path(10, 20, 0), states.uniform_states(10, 500, 3)),
                            (fall, (Tf, pf, Yf)), (plog, (Tp, pp, Yp)),
                            (nasa, states.bimodal_states(53, 325, 400, 5)[:3]),
                            (states.mech_path(53, 325, 0), states.bimodal_states(53, 325, 600, 4)[:3])):
        ctx = d.Context(mech)
        dd = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
        fT, fY = ctx.rhs(dd(T), dd(p), dd(Y))
        torch.cuda.synchronize()
        fT, fY = fT.cpu().numpy(), fY.cpu().numpy()
        orc = oracle.Oracle(mech)
        m = read_mech(mech)
        nr, npd = m.nu_matrix()
        absnu = np.abs(npd - nr).astype(float)
        for i in range(T.size):
            y0 = np.concatenate([[T[i]], Y[:, i]])
            fo = orc.rhs(p[i], y0)
            c, kf, kr, q = orc.rates(p[i], y0)
            fwd = kf * np.prod(c[:, None] ** nr, axis=0)
            rev = kr * np.prod(c[:, None] ** npd, axis=0)
            M = np.where(m.thirdbody != 0, c.sum(), 1.0)
            for rec in m.falloff:                     # fall-off: [M] is inside k_f, not a factor
                M[rec[0]] = 1.0
            rho = (c * m.W).sum()
            termY = m.W / rho * (absnu @ (M * (fwd + rev)))
            cp, h, s_, g = orc.thermo(T[i])
            cpm = (Y[:, i] * cp / m.W).sum()
            termT = (np.abs(h) / m.W * termY).sum() / cpm
            assert np.all(np.abs(fY[:, i] - fo[1:]) <= 1e-12 * termY + 1e-300), i
            assert abs(fT[i] - fo[0]) <= 1e-12 * termT + 1e-300, (i, fT[i], fo[0])
    bad = dd(np.array([np.nan, 1000.0]))
    fT, fY = ctx.rhs(bad, dd(np.array([1e5, -1.0])), dd(np.full((53, 2), 1.0 / 53)))
    assert torch.isnan(fT).all() and torch.isnan(fY).all()
