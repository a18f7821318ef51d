"""Ensembles of independent Kuramoto networks in one plan (batched launches,
per-instance K / N_i and order parameters), CUDA-graph replay, re-tiling and
the autotuner, against the FP64 oracle run instance by instance.

Tolerances: FP32 right-hand side 1e-5 relative on the coupling part (per
instance); after 20 RK4 steps the phases within 1e-4 and r(t) within 1e-5
(the stated r tolerance is 1e-3).  Two paths running the same kernels on the
same inputs (graph replay vs plain launches; an ensemble of one vs the single
plan) must agree bit for bit.
"""
import numpy as np
import pytest

from helpers import coupling_rel_err, cuda_available

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not cuda_available():
        pytest.skip("no CUDA device")
    import paper_2203_16657_gb300 as P
    from paper_2203_16657_gb300 import build
    build.build()
    return P


def _small(B=8, n_range=(64, 600)):
    import synthetic as S
    return S.kuramoto_ensemble(B, n_range=n_range)


def _with_free_nodes(B=5, seed=31):
    """Instances with labels -1 (no community) mixed in: free-node tiles must
    never span two instances."""
    import synthetic as S
    out = []
    for i in range(B):
        g = S.random_labels_graph(40 + 17 * i, 0.2, 3, seed=seed + i, free_frac=0.3)
        rng = np.random.default_rng(seed + 100 + i)
        om = S.as_fp32_values(rng.normal(size=g.n))
        th = S.as_fp32_values(rng.uniform(0, 2 * np.pi, g.n))
        out.append((g, om, th))
    return out


def _batch_plan(P, inst, **kw):
    return P.Plan.batch([(w.graph.rowptr, w.graph.col) for w in inst],
                        [w.graph.labels for w in inst], [w.omega for w in inst],
                        K=4.0, precision="fp32", **kw)


def _concat(xs):
    return np.concatenate(xs)


def test_batch_rhs_matches_each_instance(P, oracle_mod):
    import torch
    e = _small()
    plan = _batch_plan(P, e.instances, build_direct=True)
    assert plan.info()["instances"] == len(e.instances)
    x = torch.from_numpy(_concat([w.theta0 for w in e.instances])).cuda()
    for method in ("cia", "direct"):
        out = plan.rhs(x, method=method).cpu().numpy()
        o = 0
        for w in e.instances:
            n = w.graph.n
            ref = oracle_mod.kuramoto_direct(w.graph.rowptr, w.graph.col, w.theta0, w.omega, 4.0)
            assert coupling_rel_err(out[o:o + n], ref, w.omega) <= 1e-5, (method, w.name)
            o += n


def test_batch_with_free_nodes(P, oracle_mod):
    import torch
    inst = _with_free_nodes()
    plan = P.Plan.batch([(g.rowptr, g.col) for g, _, _ in inst], [g.labels for g, _, _ in inst],
                        [om for _, om, _ in inst], K=3.0, precision="fp32", tile_nodes=32)
    x = torch.from_numpy(_concat([th for _, _, th in inst])).cuda()
    out = plan.rhs(x).cpu().numpy()
    o = 0
    for g, om, th in inst:
        ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 3.0)
        assert coupling_rel_err(out[o:o + g.n], ref, om) <= 1e-5
        o += g.n
    # order parameters per instance after 3 steps, free nodes included
    xs = x.clone()
    r = torch.zeros(3 * len(inst), dtype=torch.float64, device="cuda")
    plan.integrate(xs, 0.01, 3, r_out=r)
    r = r.cpu().numpy().reshape(3, len(inst))
    for i, (g, om, th) in enumerate(inst):
        rhs = lambda y: oracle_mod.kuramoto_direct(g.rowptr, g.col, y, om, 3.0)
        _, rr = oracle_mod.integrate(rhs, th, 0.01, 3, wrap=True, observe=oracle_mod.order_parameter)
        np.testing.assert_allclose(r[:, i], rr, rtol=0, atol=1e-5)


def test_batch_integrate_and_order_parameters(P, oracle_mod):
    import torch
    e = _small()
    plan = _batch_plan(P, e.instances)
    B, steps = len(e.instances), 20
    x = torch.from_numpy(_concat([w.theta0 for w in e.instances])).cuda()
    r = torch.zeros(steps * B, dtype=torch.float64, device="cuda")
    plan.integrate(x, e.dt, steps, r_out=r)
    plan.sync()
    got = x.cpu().numpy()
    r = r.cpu().numpy().reshape(steps, B)
    o = 0
    for i, w in enumerate(e.instances):
        n = w.graph.n
        rhs = lambda y: oracle_mod.kuramoto_direct(w.graph.rowptr, w.graph.col, y, w.omega, 4.0)
        ref, rr = oracle_mod.integrate(rhs, w.theta0, e.dt, steps, wrap=True,
                                       observe=oracle_mod.order_parameter)
        assert np.abs(oracle_mod.angle_diff(got[o:o + n], ref)).max() <= 1e-4, w.name
        np.testing.assert_allclose(r[:, i], rr, rtol=0, atol=1e-5)
        o += n


def test_host_buffer_integration_of_an_ensemble(P):
    """cia_integrate_host on an ensemble returns steps x instances order
    parameters; from pinned and from pageable memory it equals cia_integrate
    on device buffers bit for bit, twice in a row."""
    import torch
    e = _small(5)
    B, steps = len(e.instances), 7
    x0 = _concat([w.theta0 for w in e.instances])
    plan = _batch_plan(P, e.instances)
    xd = torch.from_numpy(x0.copy()).cuda()
    rd = torch.zeros(steps * B, dtype=torch.float64, device="cuda")
    want = []
    for _ in range(2):
        plan.integrate(xd, e.dt, steps, r_out=rd)
        plan.sync()
        want.append((xd.cpu().numpy().copy(), rd.cpu().numpy().copy()))
    for pinned in (True, False):
        xh = torch.from_numpy(x0.copy())
        rh = torch.zeros(steps * B, dtype=torch.float64)
        if pinned:
            xh, rh = xh.pin_memory(), rh.pin_memory()
        xn, rn = xh.numpy(), rh.numpy()
        for k in range(2):
            plan.integrate_host(xn, e.dt, steps, r_out=rn)
            np.testing.assert_array_equal(xn, want[k][0])
            np.testing.assert_array_equal(rn, want[k][1])
            assert (rn > 0).all()


def test_graph_replay_is_bit_identical_to_plain_launches(P):
    import torch
    e = _small(6)
    a_plan = _batch_plan(P, e.instances, use_graphs=True)
    b_plan = _batch_plan(P, e.instances, use_graphs=False)
    x0 = torch.from_numpy(_concat([w.theta0 for w in e.instances])).cuda()
    ra = torch.zeros(15 * 6, dtype=torch.float64, device="cuda")
    rb = torch.zeros_like(ra)
    xa, xb = x0.clone(), x0.clone()
    a_plan.integrate(xa, e.dt, 15, r_out=ra)
    b_plan.integrate(xb, e.dt, 15, r_out=rb)
    # twice more through the cached graph (no re-capture)
    a_plan.integrate(xa, e.dt, 15, r_out=ra)
    b_plan.integrate(xb, e.dt, 15, r_out=rb)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(ra, rb)


def test_ensemble_of_one_equals_single_plan(P):
    import torch
    e = _small(1, n_range=(500, 500))
    w = e.instances[0]
    single = P.Plan(w.graph.rowptr, w.graph.col, w.graph.labels, w.omega, K=4.0, precision="fp32")
    batch = _batch_plan(P, e.instances)
    xa = torch.from_numpy(w.theta0.copy()).cuda()
    xb = xa.clone()
    single.integrate(xa, e.dt, 10)
    batch.integrate(xb, e.dt, 10)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb)


@pytest.mark.parametrize("tile_nodes,tib,staging", [(64, 4096, "plain"), (256, 16384, "pipeline"),
                                                   (128, 49152, "auto"), (256, 8192, "window"),
                                                   (256, 24576, "stream"), (128, 8192, "stream")])
def test_retile_keeps_results(P, oracle_mod, tile_nodes, tib, staging):
    import torch
    e = _small(4)
    plan = _batch_plan(P, e.instances)
    plan.retile(tile_nodes, tib, staging)
    x = torch.from_numpy(_concat([w.theta0 for w in e.instances])).cuda()
    out = plan.rhs(x).cpu().numpy()
    o = 0
    for w in e.instances:
        n = w.graph.n
        ref = oracle_mod.kuramoto_direct(w.graph.rowptr, w.graph.col, w.theta0, w.omega, 4.0)
        assert coupling_rel_err(out[o:o + n], ref, w.omega) <= 1e-5
        o += n
    # advancing needs a fresh state load after a re-tiling
    with pytest.raises(P.CiaError):
        plan.advance(e.dt, 1)
    plan.state_load(x)
    plan.advance(e.dt, 2)
    plan.sync()


def test_autotune_picks_a_working_tiling(P, oracle_mod):
    import torch
    e = _small(8)
    plan = _batch_plan(P, e.instances)
    x = torch.from_numpy(_concat([w.theta0 for w in e.instances])).cuda()
    rep = plan.autotune(x, e.dt, steps=4)
    assert rep["candidates"] >= 3
    assert 0 < rep["best_ms_per_step"] <= rep["worst_ms_per_step"]
    inf = plan.info()
    assert inf["tile_nodes"] == rep["tile_nodes"]
    steps = 5
    xs = x.clone()
    plan.integrate(xs, e.dt, steps)
    got = xs.cpu().numpy()
    o = 0
    for w in e.instances:
        n = w.graph.n
        rhs = lambda y: oracle_mod.kuramoto_direct(w.graph.rowptr, w.graph.col, y, w.omega, 4.0)
        ref, _ = oracle_mod.integrate(rhs, w.theta0, e.dt, steps, wrap=True)
        assert np.abs(oracle_mod.angle_diff(got[o:o + n], ref)).max() <= 1e-4
        o += n


def test_largest_ensemble_instances(P, oracle_mod):
    """The instances of the full ensemble with the largest communities (N_i
    above 15000 in M_i = 2 communities of about 8000 nodes), batched with a
    small one: every node's FP32 right-hand side against the oracle."""
    import torch
    import synthetic as S
    big = [i for i in range(4096)
           if S.ensemble_instance_shape(i)[1] == 2 and S.ensemble_instance_shape(i)[0] >= 15000][:3]
    assert len(big) == 3
    inst = [S.ensemble_instance(i) for i in [0] + big]
    assert max(w.graph.sizes.max() for w in inst) >= 7500
    plan = _batch_plan(P, inst)
    x = torch.from_numpy(_concat([w.theta0 for w in inst])).cuda()
    out = plan.rhs(x).cpu().numpy()
    o = 0
    for w in inst:
        n = w.graph.n
        ref = oracle_mod.kuramoto_direct(w.graph.rowptr, w.graph.col, w.theta0, w.omega, 4.0)
        assert coupling_rel_err(out[o:o + n], ref, w.omega) <= 1e-5, w.name
        o += n


def test_bench_sized_ensemble_sampled(P, oracle_mod):
    """The 32 instances the measurement uses (full per-instance size
    distribution): CIA right-hand side of every instance against the oracle."""
    import torch
    import synthetic as S
    e = S.kuramoto_ensemble(32)
    plan = _batch_plan(P, e.instances)
    x = torch.from_numpy(_concat([w.theta0 for w in e.instances])).cuda()
    out = plan.rhs(x).cpu().numpy()
    o = 0
    for w in e.instances:
        n = w.graph.n
        ref = oracle_mod.kuramoto_direct(w.graph.rowptr, w.graph.col, w.theta0, w.omega, 4.0)
        assert coupling_rel_err(out[o:o + n], ref, w.omega) <= 1e-5, w.name
        o += n


def test_streamed_plan_equals_batch_plan(P):
    """An ensemble planned instance by instance (cia_plan_batch_begin/add/
    finish) has the one-call plan's layout: the same permutation, split of S
    and tiling, and an integration with order parameters bit for bit equal."""
    import torch
    inst = [(w.graph, w.omega, w.theta0) for w in _small(5).instances] + _with_free_nodes(3)
    a = P.Plan.batch([(g.rowptr, g.col) for g, _, _ in inst], [g.labels for g, _, _ in inst],
                     [om for _, om, _ in inst], K=4.0, precision="fp32")
    b = P.Plan.streamed(((g.rowptr, g.col, g.labels, om) for g, om, _ in inst), K=4.0, precision="fp32")
    ia, ib = a.info(), b.info()
    for key in ("n", "M", "n_free", "nnz_graph", "nnz_missing", "nnz_inter", "n_tiles", "instances", "staging"):
        assert ia[key] == ib[key], key
    pa, oa = a.permutation()
    pb, ob = b.permutation()
    assert np.array_equal(pa, pb) and np.array_equal(oa, ob)
    for x, y in zip(a.split(), b.split()):
        assert np.array_equal(x, y)
    x0 = torch.from_numpy(_concat([th for _, _, th in inst])).cuda()
    xa, xb = x0.clone(), x0.clone()
    ra = torch.zeros(8 * len(inst), dtype=torch.float64, device="cuda")
    rb = torch.zeros_like(ra)
    a.integrate(xa, 0.01, 8, r_out=ra)
    b.integrate(xb, 0.01, 8, r_out=rb)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(ra, rb)
