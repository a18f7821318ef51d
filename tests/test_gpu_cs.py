"""Cucker--Smale on the GPU through the C ABI against the FP64 oracle.

Tolerances (FP32 state and sums):
* direct RHS and CIA with a constant feature map: ||dv_gpu - dv_ref||_inf /
  ||dv_ref||_inf <= 1e-5 (FP32 arithmetic), positions' derivative = v exactly;
* CIA with a non-constant learned map: the device rounds hidden activations
  and features to BF16, and a rounding decision the device takes in FP32 can
  differ from the oracle's FP64 one; the test bounds the difference by one
  BF16 spacing of every feature (relative 2^-7) propagated through the dense
  sum, and checks momentum conservation (sum_m v_m' = 0), which holds for any
  symmetric pair weight.
"""
import numpy as np
import pytest

from helpers import cuda_available

pytestmark = pytest.mark.gpu

H, R = 128, 64


@pytest.fixture(scope="module")
def P():
    if not cuda_available():
        pytest.skip("no CUDA device")
    import paper_2203_16657_gb300 as P
    from paper_2203_16657_gb300 import build
    build.build()
    return P


def _workload(scale=0.125):
    import synthetic as S
    return S.cucker_smale(scale)


def _x0(w):
    return np.concatenate([w.s0, w.v0], axis=1)


def _params(seed, w2=None, b2=0.1, const=False):
    rng = np.random.default_rng(seed)
    w2 = 1.0 / np.sqrt(H) if w2 is None else w2
    p = {"W1": rng.normal(0, 0.5, (H, 2)), "b1": rng.normal(0, 0.5, H),
         "W2": rng.normal(0, w2, (R, H)), "b2": rng.normal(0, b2, R)}
    if const:
        p["W2"][:] = 0.0
    return p


def _plan(P, w, *, K=None, beta=None, build_direct=True, tile_nodes=0):
    g = w.graph
    return P.Plan(g.rowptr, g.col, g.labels, None, K=w.K if K is None else K, sigma=w.sigma,
                  beta=w.beta if beta is None else beta, precision="fp32",
                  model="cucker_smale", build_direct=build_direct, tile_nodes=tile_nodes)


def _rel_v(got, ref):
    return float(np.abs(got[:, 2:] - ref[:, 2:]).max() / np.abs(ref[:, 2:]).max())


def test_bookkeeping_and_info(P):
    w = _workload()
    plan = _plan(P, w)
    inf = plan.info()
    assert inf["model"] == 2 and inf["state_dim"] == 4 and inf["tile_nodes"] == 128
    perm, off = plan.permutation()
    assert sorted(perm.tolist()) == list(range(w.graph.n))


def test_direct_rhs(P, oracle_mod):
    import torch
    w = _workload()
    plan = _plan(P, w)
    x = _x0(w)
    out = plan.rhs(torch.from_numpy(x.ravel()).cuda(), method="direct").cpu().numpy().reshape(-1, 4)
    ref = oracle_mod.cs_direct(w.graph.rowptr, w.graph.col, x, w.K, w.sigma, w.beta)
    np.testing.assert_array_equal(out[:, :2], x[:, 2:])
    assert _rel_v(out, ref) <= 1e-5


@pytest.mark.parametrize("tile_nodes", [0, 64, 96])
def test_cia_constant_features_equals_direct(P, oracle_mod, tile_nodes):
    """W2 = 0: phi = b2 for every agent, stored in BF16, phi.phi = |bf16(b2)|^2.
    With beta = 0 and K = |bf16(b2)|^2 the exact weight is the same constant,
    so the CIA reaches the direct sum to rounding (moments, dense term and
    both halves of S)."""
    import torch
    w = _workload()
    p = _params(21, const=True)
    vec = oracle_mod.pack_params(p).astype(np.float32)
    b2 = oracle_mod.bf16_round(vec[-R:])   # the plan stores features in BF16
    K = float((b2 * b2).sum())
    plan = _plan(P, w, K=K, beta=0.0, tile_nodes=tile_nodes)
    basis = P.Basis(vec)
    plan.set_basis(basis)
    x = _x0(w)
    out = plan.rhs(torch.from_numpy(x.ravel()).cuda()).cpu().numpy().reshape(-1, 4)
    ref = oracle_mod.cs_direct(w.graph.rowptr, w.graph.col, x, K, w.sigma, 0.0)
    np.testing.assert_array_equal(out[:, :2], x[:, 2:])
    assert _rel_v(out, ref) <= 1e-5


def _oracle_features(oracle_mod, vec, x_perm, off):
    """phi of every community node at its position minus the community centroid
    (BF16 hidden activations and BF16 features, as the device evaluates them)."""
    p = oracle_mod.unpack_params(np.asarray(vec, dtype=np.float32).astype(np.float64))
    p["W2"] = oracle_mod.bf16_round(p["W2"])
    feat = np.zeros((len(x_perm), R))
    for c in range(len(off) - 1):
        s = x_perm[off[c]:off[c + 1], :2]
        if len(s) == 0:
            continue
        rel = s - s.mean(axis=0)
        f, _ = oracle_mod.mlp_forward(p, rel, hidden_round=oracle_mod.bf16_round)
        feat[off[c]:off[c + 1]] = oracle_mod.bf16_round(f)
    return feat


def _oracle_features_shifted(oracle_mod, vec, x_perm, off, shift):
    """phi of every community node at its position minus a given per-community shift."""
    p = oracle_mod.unpack_params(np.asarray(vec, dtype=np.float32).astype(np.float64))
    p["W2"] = oracle_mod.bf16_round(p["W2"])
    feat = np.zeros((len(x_perm), R))
    for c in range(len(off) - 1):
        if off[c + 1] > off[c]:
            f, _ = oracle_mod.mlp_forward(p, x_perm[off[c]:off[c + 1], :2] - shift[c],
                                          hidden_round=oracle_mod.bf16_round)
            feat[off[c]:off[c + 1]] = oracle_mod.bf16_round(f)
    return feat


def _dense_bf16_bound(feat, xp, off, N):
    """Per node: one BF16 spacing of every feature (relative 2^-7) propagated
    through the dense sum sum_r phi_r(m) (H_cr - U_cr v_m)."""
    bound = np.zeros(len(xp))
    for c in range(len(off) - 1):
        a, b = off[c], off[c + 1]
        F = np.abs(feat[a:b])
        v = xp[a:b, 2:]
        absU = F.sum(axis=0) / N
        absH = (F[:, :, None] * np.abs(v)[:, None, :]).sum(axis=0) / N
        U = feat[a:b].sum(axis=0) / N
        Hm = (feat[a:b][:, :, None] * v[:, None, :]).sum(axis=0) / N
        for i in range(b - a):
            t1 = F[i] @ np.abs(Hm - U[:, None] * v[i][None, :])
            t2 = F[i] @ (absH + absU[:, None] * np.abs(v[i])[None, :])
            bound[a + i] = (2.0 ** -7) * (t1 + t2).max()
    return bound


def test_integrate_learned_cia_uses_the_step_shift(P, oracle_mod):
    """RK4 with a learned (non-constant) basis.  The four stages of a step
    evaluate phi with the centroid of the step's initial state as the shift
    (stages 1-3 compute the next stage's features in their own launch); the
    FP64 oracle RK4 below takes the same reading, calling cs_cia with the
    features of each stage state at that shift.  Bound: one BF16 spacing of
    every feature through the dense sum per stage (the single-RHS bound at
    the initial state, doubled for the later stage states), accumulated as
    dt per step.  dt = 0.5 moves the stage states far enough that features
    left from the step's first stage exceed the bound 3-fold on about a
    quarter of the nodes (checked with the oracle on the CPU).  The stage
    state's own centroid as the shift stays within a quarter of the bound:
    the two readings are numerically equivalent here."""
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(22)).astype(np.float32)
    plan = _plan(P, w)
    plan.set_basis(P.Basis(vec))
    x = _x0(w)
    dt, steps = 0.5, 2
    xd = torch.from_numpy(x.ravel().copy()).cuda()
    plan.integrate(xd, dt, steps)
    plan.sync()
    got = xd.cpu().numpy().reshape(-1, 4)
    perm, off = plan.permutation()
    sp = oracle_mod.split(w.graph.rowptr, w.graph.col, w.graph.labels)
    assert (sp.perm == perm).all()
    M = len(off) - 1

    def rk4_step(y):
        yp = y[perm]
        shift = [yp[off[c]:off[c + 1], :2].mean(axis=0) if off[c + 1] > off[c] else np.zeros(2) for c in range(M)]

        def f(z):
            zp = z[perm]
            out = np.empty_like(z)
            out[perm] = oracle_mod.cs_cia(sp, zp, _oracle_features_shifted(oracle_mod, vec, zp, off, shift),
                                          w.K, w.sigma, w.beta)
            return out

        k1 = f(y)
        k2 = f(y + 0.5 * dt * k1)
        k3 = f(y + 0.5 * dt * k2)
        k4 = f(y + dt * k3)
        return y + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    ref = x.copy()
    for _ in range(steps):
        ref = rk4_step(ref)
    xp = x[perm]
    feat0 = _oracle_features(oracle_mod, vec, xp, off)
    bound = np.empty(len(x))
    bound[perm] = 2.0 * _dense_bf16_bound(feat0, xp, off, len(x))
    vscale = np.abs(ref[:, 2:]).max()
    dv = np.abs(got[:, 2:] - ref[:, 2:]).max(axis=1)
    assert (dv <= steps * dt * bound + 1e-5 * vscale).all(), float(((dv - steps * dt * bound) / vscale).max())
    ds = np.abs(got[:, :2] - ref[:, :2]).max()
    assert ds <= steps * dt * dt * bound.max() + 1e-5 * np.abs(ref[:, :2]).max(), ds
    # the steps moved the velocities by several times the allowed difference
    assert np.abs(ref[:, 2:] - x[:, 2:]).max() > 4.0 * (steps * dt * bound.max())


def test_cia_learned_features_within_bf16_bound(P, oracle_mod):
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(22)).astype(np.float32)
    plan = _plan(P, w)
    basis = P.Basis(vec)
    plan.set_basis(basis)
    x = _x0(w)
    out = plan.rhs(torch.from_numpy(x.ravel()).cuda()).cpu().numpy().reshape(-1, 4)
    perm, off = plan.permutation()
    sp = oracle_mod.split(w.graph.rowptr, w.graph.col, w.graph.labels)
    assert (sp.perm == perm).all()
    xp = x[perm]
    feat = _oracle_features(oracle_mod, vec, xp, off)
    ref = oracle_mod.cs_cia(sp, xp, feat, w.K, w.sigma, w.beta)
    got = out[perm]
    # one BF16 spacing per feature (relative 2^-7) through the dense sum
    N = len(x)
    bound = np.zeros(N)
    for c in range(len(off) - 1):
        a, b = off[c], off[c + 1]
        F = np.abs(feat[a:b])
        v = xp[a:b, 2:]
        absU = F.sum(axis=0) / N
        absH = (F[:, :, None] * np.abs(v)[:, None, :]).sum(axis=0) / N
        U = feat[a:b].sum(axis=0) / N
        Hm = (feat[a:b][:, :, None] * v[:, None, :]).sum(axis=0) / N
        for i in range(b - a):
            t1 = F[i] @ np.abs(Hm - U[:, None] * v[i][None, :])
            t2 = F[i] @ (absH + absU[:, None] * np.abs(v[i])[None, :])
            bound[a + i] = (2.0 ** -7) * (t1 + t2).max()
    scale = np.abs(ref[:, 2:]).max()
    diff = np.abs(got[:, 2:] - ref[:, 2:]).max(axis=1)
    assert (diff <= bound + 1e-5 * scale).all(), float(((diff - bound) / scale).max())
    # most of the difference is far below the worst case
    assert np.median(diff) <= 1e-3 * scale
    # momentum: sum of v' over all agents vanishes for symmetric weights
    mom = np.abs(got[:, 2:].sum(axis=0)).max()
    assert mom <= 1e-5 * np.abs(got[:, 2:]).sum(axis=0).max()


def test_integrate_direct_matches_oracle(P, oracle_mod):
    import torch
    w = _workload()
    plan = _plan(P, w)
    x = _x0(w)
    steps = 20
    xd = torch.from_numpy(x.ravel().copy()).cuda()
    plan.integrate(xd, w.dt, steps, method="direct")
    got = xd.cpu().numpy().reshape(-1, 4)
    rhs = lambda y: oracle_mod.cs_direct(w.graph.rowptr, w.graph.col, y, w.K, w.sigma, w.beta)
    ref, _ = oracle_mod.integrate(rhs, x, w.dt, steps, wrap=False)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err


def test_integrate_cia_constant_features_matches_direct_oracle(P, oracle_mod):
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(23, const=True)).astype(np.float32)
    b2 = oracle_mod.bf16_round(vec[-R:])   # the plan stores features in BF16
    K = float((b2 * b2).sum())
    plan = _plan(P, w, K=K, beta=0.0)
    plan.set_basis(P.Basis(vec))
    x = _x0(w)
    steps = 20
    xd = torch.from_numpy(x.ravel().copy()).cuda()
    plan.integrate(xd, w.dt, steps)
    plan.sync()
    got = xd.cpu().numpy().reshape(-1, 4)
    rhs = lambda y: oracle_mod.cs_direct(w.graph.rowptr, w.graph.col, y, K, w.sigma, 0.0)
    ref, _ = oracle_mod.integrate(rhs, x, w.dt, steps, wrap=False)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err


def test_state_resume_is_bit_exact(P, oracle_mod):
    """2k steps in one call == k steps, store, load, k steps (learned CIA)."""
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(24)).astype(np.float32)
    plan = _plan(P, w)
    plan.set_basis(P.Basis(vec))
    x = torch.from_numpy(_x0(w).ravel().copy()).cuda()
    a = x.clone()
    plan.integrate(a, w.dt, 10)
    b = x.clone()
    plan.integrate(b, w.dt, 5)
    plan.integrate(b, w.dt, 5)
    plan.sync()
    # the resumed run restarts its stage state from the FP64 master: equal to
    # the uninterrupted run because every step starts from (float) master too
    assert torch.equal(a, b)


def test_check_falls_back_to_direct(P, oracle_mod):
    """An untrained basis with a tight bound fails the check before step 0:
    the whole run is the direct method (bit-identical to method='direct')."""
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(25)).astype(np.float32)
    plan = _plan(P, w)
    plan.set_basis(P.Basis(vec))
    plan.set_check(every=5, bound=1e-3)
    x = torch.from_numpy(_x0(w).ravel().copy()).cuda()
    a = x.clone()
    plan.integrate(a, w.dt, 10)
    rep = plan.check_report()
    assert rep["fell_back"] == 1 and rep["fallback_step"] == 0 and rep["checks"] == 1
    assert rep["last_error"] > 1e-3
    assert "direct method" in plan.last_fallback
    b = x.clone()
    plan.integrate(b, w.dt, 10, method="direct")
    plan.sync()
    assert torch.equal(a, b)


def test_check_value_matches_oracle(P, oracle_mod):
    """The check's err/ref against the same quantity from the oracle."""
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(26)).astype(np.float32)
    plan = _plan(P, w)
    plan.set_basis(P.Basis(vec))
    plan.set_check(every=1, bound=1e9)
    x = _x0(w)
    plan.integrate(torch.from_numpy(x.ravel().copy()).cuda(), w.dt, 1)
    rep = plan.check_report()
    assert rep["checks"] == 1 and rep["fell_back"] == 0
    perm, off = plan.permutation()
    xp = x[perm]
    feat = _oracle_features(oracle_mod, vec, xp, off)
    sp = oracle_mod.split(w.graph.rowptr, w.graph.col, w.graph.labels)
    cia = oracle_mod.cs_cia(sp, xp, feat, w.K, w.sigma, w.beta)
    direct = oracle_mod.cs_direct(w.graph.rowptr, w.graph.col, x, w.K, w.sigma, w.beta)[perm]
    nc = off[-1]
    cnt = min(512, nc)
    nodes = [(2 * k + 1) * nc // (2 * cnt) for k in range(cnt)]
    err = np.abs(cia[nodes, 2:] - direct[nodes, 2:]).max()
    ref = np.abs(direct[nodes, 2:]).max()
    assert abs(rep["last_error"] - err / ref) <= 0.05 * (err / ref) + 1e-5


def test_sample_pairs(P, oracle_mod):
    import torch
    w = _workload()
    plan = _plan(P, w)
    x = _x0(w)
    plan.state_load(torch.from_numpy(x.ravel().copy()).cuda())
    pairs = plan.sample_pairs(4096, seed=9).cpu().numpy().astype(np.float64)
    d2 = ((pairs[:, 0:2] - pairs[:, 2:4]) ** 2).sum(axis=1)
    np.testing.assert_allclose(pairs[:, 4], oracle_mod.cs_kernel_weight(d2, w.K, w.sigma, w.beta),
                               rtol=1e-5)
    # positions are relative to a centroid: both members of a pair are real
    # agents of one community, whose centroid is subtracted
    perm, off = plan.permutation()
    xp = x[perm]
    cen = np.array([xp[off[c]:off[c + 1], :2].mean(axis=0) for c in range(len(off) - 1)])
    pts = {tuple(np.round(p, 4)) for c in range(len(off) - 1)
           for p in (xp[off[c]:off[c + 1], :2] - cen[c]).astype(np.float32)}
    hits = sum(tuple(np.round(p.astype(np.float32), 4)) in pts for p in pairs[:200, 0:2])
    assert hits >= 190
    again = plan.sample_pairs(4096, seed=9).cpu().numpy()
    np.testing.assert_array_equal(again, pairs.astype(np.float32))


def test_learn_fit_gains_over_untrained(P, oracle_mod):
    """A basis learned from direct trajectories brings the CIA closer to the
    direct right-hand side than the same network untrained."""
    import torch
    w = _workload()
    vec = oracle_mod.pack_params(_params(27, w2=0.02, b2=0.02)).astype(np.float32)
    plan = _plan(P, w)
    basis = P.Basis(vec)
    plan.set_basis(basis)
    plan.set_check(every=1, bound=1e9)
    x = torch.from_numpy(_x0(w).ravel().copy()).cuda()
    plan.integrate(x.clone(), w.dt, 1)
    before = plan.check_report()["last_error"]
    rep = plan.learn_fit(basis, x, dt=w.dt, steps=20, snapshots=4, pairs=400000, seed=3,
                         batch=8192, epochs=3, lr=2e-3)
    assert rep["pairs"] == 400000 and rep["last_epoch_loss"] < 0.1 * rep["first_loss"], rep
    plan.set_check(every=1, bound=1e9)
    plan.integrate(x.clone(), w.dt, 1)
    after = plan.check_report()["last_error"]
    assert after < 0.2 * before, (before, after)


def test_full_size_direct_and_constant_cia(P, oracle_mod):
    """The N = 131072 workload in the bench's launch configuration: the direct
    RHS against the FP64 oracle, and the CIA with a constant feature map (exact
    for a constant weight) against the oracle's direct sum."""
    import torch
    import synthetic as S
    w = S.cached("cucker_smale", 1.0)
    g = w.graph
    x = _x0(w)
    xd = torch.from_numpy(x.ravel()).cuda()
    plan = _plan(P, w)
    out = plan.rhs(xd, method="direct").cpu().numpy().reshape(-1, 4)
    ref = oracle_mod.cs_direct(g.rowptr, g.col, x, w.K, w.sigma, w.beta)
    assert _rel_v(out, ref) <= 1e-5
    vec = oracle_mod.pack_params(_params(28, const=True)).astype(np.float32)
    b2 = oracle_mod.bf16_round(vec[-R:])   # the plan stores features in BF16
    K = float((b2 * b2).sum())
    plan2 = _plan(P, w, K=K, beta=0.0, build_direct=False)
    plan2.set_basis(P.Basis(vec))
    out2 = plan2.rhs(xd).cpu().numpy().reshape(-1, 4)
    ref2 = oracle_mod.cs_direct(g.rowptr, g.col, x, K, w.sigma, 0.0)
    assert _rel_v(out2, ref2) <= 1e-5


def test_learned_basis_beats_fourier_at_equal_rank(P, oracle_mod):
    """What the trained network gains over the paper's own basis: at rank 64
    the learned feature map brings the CIA closer to the exact right-hand side
    than the 64 strongest Fourier modes of the weight on the box that holds
    every in-community difference (App. A.6), both judged by the FP64 oracle."""
    import torch
    w = _workload()
    x = _x0(w)
    g = w.graph
    eta = lambda d2: oracle_mod.cs_kernel_weight(d2, w.K, w.sigma, w.beta)
    ref = oracle_mod.cs_direct(g.rowptr, g.col, x, w.K, w.sigma, w.beta)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    xp = x[sp.perm]
    L = 10.0
    alpha, c = oracle_mod.fourier_basis(oracle_mod.radial(eta), L, rank=64)
    F = oracle_mod.fourier_features(xp[:, :2], alpha, c, L)
    assert F.shape[1] <= 64
    four = oracle_mod.cs_cia(sp, xp, F, w.K, w.sigma, w.beta)
    inv = np.empty_like(sp.perm)
    inv[sp.perm] = np.arange(len(sp.perm))
    e_fourier = _rel_v(four[inv], ref)
    # the network starts as the Fourier basis (sine units are plane waves) and
    # is trained on pairs from direct trajectories
    vec = P.Basis.params_fourier(w.K, w.sigma, w.beta, L, seed=5)
    plan = _plan(P, w)
    basis = P.Basis(vec)
    xd = torch.from_numpy(x.ravel().copy()).cuda()
    plan.learn_fit(basis, xd, dt=w.dt, steps=20, snapshots=4, pairs=1_000_000, seed=5,
                   batch=8192, epochs=8, lr=3e-4, lr_final=1e-5)
    got = plan.rhs(xd).cpu().numpy().reshape(-1, 4)
    e_learned = _rel_v(got, ref)
    assert e_learned < e_fourier, (e_learned, e_fourier)


@pytest.mark.parametrize("case", ["free_nodes", "singletons", "no_edges", "all_free"])
def test_cia_degenerate_graphs(P, oracle_mod, case):
    """Unlabelled agents (all their links sparse), one-agent communities,
    an empty graph and a graph without communities: with a constant feature
    map (exact for a constant weight) the CIA equals the direct sum."""
    import torch
    import synthetic as S
    if case == "free_nodes":
        g = S.random_labels_graph(90, 0.2, 4, seed=41, free_frac=0.3)
    elif case == "singletons":
        g = S.random_labels_graph(40, 0.3, 1, seed=42, free_frac=0.0)
        g.labels = np.arange(g.n, dtype=np.int32)
    elif case == "no_edges":
        g = S.random_labels_graph(30, 0.0, 3, seed=43, free_frac=0.1)
    else:
        g = S.random_labels_graph(50, 0.3, 1, seed=44, free_frac=1.0)
    rng = np.random.default_rng(45)
    x = S.as_fp32_values(np.concatenate([rng.uniform(0, 10, (g.n, 2)), rng.normal(size=(g.n, 2))], axis=1))
    vec = oracle_mod.pack_params(_params(46, const=True)).astype(np.float32)
    b2 = oracle_mod.bf16_round(vec[-R:])
    K = float((b2 * b2).sum())
    plan = P.Plan(g.rowptr, g.col, g.labels, None, K=K, sigma=1.0, beta=0.0, precision="fp32",
                  model="cucker_smale", build_direct=True, tile_nodes=32)
    plan.set_basis(P.Basis(vec))
    xd = torch.from_numpy(x.ravel().copy()).cuda()
    ref = oracle_mod.cs_direct(g.rowptr, g.col, x, K, 1.0, 0.0)
    # FP32 rounding is relative to the terms summed: a whole community's block
    # (K lambda max|v| / N) even where the exact result is zero (no links)
    lam = np.bincount(g.labels[g.labels >= 0]).max() if (g.labels >= 0).any() else 1
    terms = K * lam * np.abs(x[:, 2:]).max() / g.n
    for method in ("cia", "direct"):
        out = plan.rhs(xd, method=method).cpu().numpy().reshape(-1, 4)
        np.testing.assert_array_equal(out[:, :2], x[:, 2:])
        tol = 1e-5 * max(np.abs(ref[:, 2:]).max(), terms)
        assert np.abs(out[:, 2:] - ref[:, 2:]).max() <= tol, method
    # a few steps through the stage kernels (features launch included)
    xs = xd.clone()
    plan.integrate(xs, 0.01, 3)
    plan.sync()
    rhs = lambda y: oracle_mod.cs_direct(g.rowptr, g.col, y, K, 1.0, 0.0)
    want, _ = oracle_mod.integrate(rhs, x, 0.01, 3, wrap=False)
    assert np.abs(xs.cpu().numpy().reshape(-1, 4) - want).max() <= 1e-5 * np.abs(want).max()
