"""Parity of the CUDA Kuramoto path (libcia via its C ABI) with the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
  FP64 plans: coupling part within 1e-12 relative (norm-wise, inf-norm);
  FP32 plans: within 1e-5 relative; order parameter r(t) within 1e-3 over
  the horizon; integer bookkeeping (permutation, offsets, split of S)
  bit-exact.
"""
import numpy as np
import pytest

import synthetic as S
from helpers import coupling_rel_err, cuda_available, split_halves

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

FP64_TOL = 1e-12
FP32_TOL = 1e-5
R_TOL = 1e-3


@pytest.fixture(scope="module")
def cia():
    import paper_2203_16657_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    torch.cuda.init()
    return torch


def make_plan(cia, g, omega, K, d_sin=(1.0,), d_cos=(0.0,), precision="fp64", **kw):
    return cia.Plan(g.rowptr, g.col, g.labels, omega, K=K, d_sin=d_sin, d_cos=d_cos,
                    precision=precision, build_direct=True, **kw)


def gpu_rhs(torch_mod, plan, x, method):
    xd = torch_mod.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    out = plan.rhs(xd, method=method)
    torch_mod.cuda.synchronize()
    return out.cpu().numpy()


# ------------------------------------------------------------------ bookkeeping

def check_bookkeeping(oracle_mod, plan, g):
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    perm, off = plan.permutation()
    assert np.array_equal(perm.astype(np.int64), sp.perm)
    assert np.array_equal(off, sp.off)
    mrp, mcol, irp, icol = plan.split()
    omrp, omcol, oirp, oicol = split_halves(sp)
    assert np.array_equal(mrp, omrp) and np.array_equal(mcol, omcol)
    assert np.array_equal(irp, oirp) and np.array_equal(icol, oicol)
    info = plan.info()
    assert info["nnz_missing"] == len(omcol) and info["nnz_inter"] == len(oicol)
    return sp


@pytest.mark.parametrize("seed", range(4))
def test_bookkeeping_random_labels(cia, oracle_mod, seed):
    g = S.random_labels_graph(45, 0.25, 5, seed=seed, free_frac=0.2)
    plan = make_plan(cia, g, None, 1.0)
    check_bookkeeping(oracle_mod, plan, g)


def test_bookkeeping_small_sbm(cia, oracle_mod):
    w = S.kuramoto_sbm_small()
    plan = make_plan(cia, w.graph, w.omega, w.K)
    check_bookkeeping(oracle_mod, plan, w.graph)


# ------------------------------------------------------------------ RHS parity

@pytest.mark.parametrize("method", ["cia", "direct"])
def test_rhs_fp64_small_sbm(cia, oracle_mod, torch_mod, method):
    w = S.kuramoto_sbm_small()
    g = w.graph
    plan = make_plan(cia, g, w.omega, w.K)
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, w.theta0, w.omega, w.K)
    got = gpu_rhs(torch_mod, plan, w.theta0, method)
    assert coupling_rel_err(got, ref, w.omega) < FP64_TOL


@pytest.mark.parametrize("staging", ["pipeline", "window", "stream"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rhs_harmonics(cia, oracle_mod, torch_mod, p, precision, staging):
    rng = np.random.default_rng(p)
    g = S.sbm_graph([40, 70, 33, 64], 0.8, inter_degree=5.0, seed=50 + p, n_free=9)
    d_sin, d_cos = rng.normal(size=p), rng.normal(size=p)
    th = S.as_fp32_values(rng.uniform(-np.pi, np.pi, g.n))
    om = S.as_fp32_values(rng.normal(size=g.n))
    plan = make_plan(cia, g, om, 2.0, d_sin, d_cos, precision, tile_nodes=32, staging=staging)
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 2.0, d_sin, d_cos)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    for method in ("cia", "direct"):
        assert coupling_rel_err(gpu_rhs(torch_mod, plan, th, method), ref, om) < tol, method


@pytest.mark.parametrize("staging", ["auto", "plain", "window", "pipeline", "stream"])
@pytest.mark.parametrize("group_size", [4, 8, 16, 32])
@pytest.mark.parametrize("tile_nodes,tile_index_bytes", [(32, 0), (96, 0), (1024, 0), (256, 256),
                                                         (1024, 4096)])
def test_rhs_launch_shapes(cia, oracle_mod, torch_mod, group_size, tile_nodes, tile_index_bytes,
                           staging):
    """Several tiles per community with a ragged tail, every group width,
    index budgets that cut tiles at single rows, TMA staging and plain loads."""
    g = S.sbm_graph([300, 129, 31, 700], 0.9, inter_degree=6.0, seed=7, n_free=40)
    rng = np.random.default_rng(1)
    th = rng.uniform(0, 2 * np.pi, g.n)
    om = rng.normal(size=g.n)
    plan = make_plan(cia, g, om, 3.0, tile_nodes=tile_nodes, group_size=group_size,
                     tile_index_bytes=tile_index_bytes, staging=staging)
    # the pipelined TMA kernel and the window kernel take tiles of at most 256 rows
    want = {"auto": 2, "plain": 1, "window": 2, "pipeline": 3, "stream": 4}[staging]
    assert plan.info()["staging"] == (want if tile_nodes <= 256 else 1)
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 3.0)
    for method in ("cia", "direct"):
        assert coupling_rel_err(gpu_rhs(torch_mod, plan, th, method), ref, om) < FP64_TOL


@pytest.mark.parametrize("case", ["all_free", "no_edges", "single_node", "empty_labels",
                                  "singletons", "complete"])
def test_rhs_degenerate_graphs(cia, oracle_mod, torch_mod, case):
    rng = np.random.default_rng(3)
    if case == "all_free":
        g = S.random_labels_graph(30, 0.3, 1, seed=1, free_frac=1.0)
    elif case == "no_edges":
        g = S.random_labels_graph(20, 0.0, 3, seed=2, free_frac=0.1)
    elif case == "single_node":
        g = S.Graph(1, np.array([0, 0], np.int64), np.zeros(0, np.int32),
                    np.array([0], np.int32), np.array([1], np.int64))
    elif case == "empty_labels":
        g = S.random_labels_graph(40, 0.4, 3, seed=4, free_frac=0.0)
        g.labels = (g.labels * 3 + 2).astype(np.int32)    # labels 2, 5, 8: gaps
    elif case == "singletons":
        g = S.random_labels_graph(25, 0.5, 1, seed=5, free_frac=0.0)
        g.labels = np.arange(g.n, dtype=np.int32)
    else:
        g = S.complete_graph_communities([17, 5, 1], seed=6)
    th = rng.uniform(-3, 3, g.n)
    om = rng.normal(size=g.n)
    plan = make_plan(cia, g, om, 1.5, (0.6, 0.2), (0.3, -0.4))
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 1.5, (0.6, 0.2), (0.3, -0.4))
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, th, method)
        if np.abs(ref - om).max() == 0:
            assert np.abs(got - ref).max() < 1e-15
        else:
            assert coupling_rel_err(got, ref, om) < FP64_TOL


@pytest.mark.parametrize("staging", ["auto", "plain", "window", "pipeline", "stream"])
def test_rhs_fp32_lognormal_reduced(cia, oracle_mod, torch_mod, staging):
    w = S.kuramoto_lognormal(scale=1 / 16)
    g = w.graph
    plan = make_plan(cia, g, w.omega, w.K, precision="fp32", staging=staging)
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, w.theta0, w.omega, w.K)
    for method in ("cia", "direct"):
        assert coupling_rel_err(gpu_rhs(torch_mod, plan, w.theta0, method), ref, w.omega) < FP32_TOL


def test_rhs_fp32_lognormal_full_size(cia, oracle_mod, torch_mod):
    """The full N = 262144 lognormal workload (256 communities, p_in 0.95,
    inter degree 8) in the launch configuration the measurement times: FP32
    CIA right-hand side against the FP64 oracle's direct sum, element-wise
    on the coupling part."""
    w = S.cached("kuramoto_lognormal")
    g = w.graph
    plan = make_plan(cia, g, w.omega, w.K, precision="fp32")
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, w.theta0, w.omega, w.K)
    assert coupling_rel_err(gpu_rhs(torch_mod, plan, w.theta0, "direct"), ref, w.omega) < FP32_TOL
    # every CIA kernel, the persistent ones with several tiles per CTA
    for staging, tib, want in [("window", 0, 2), ("stream", 49152, 4), ("stream", 24576, 4),
                               ("pipeline", 32768, 3)]:
        plan.retile(0, tib, staging)
        assert plan.info()["staging"] == want
        got = gpu_rhs(torch_mod, plan, w.theta0, "cia")
        assert coupling_rel_err(got, ref, w.omega) < FP32_TOL, staging


def test_stream_kernel_many_rounds_integrate(cia, oracle_mod, torch_mod):
    """The persistent per-tile kernel with far more tiles than resident CTAs
    (every CTA runs several rounds: descriptors fetched ahead, the copy
    barrier's phases reused), through all four RK4 stage modes: 20 steps of
    r(t) and the final phases against the oracle's RK4 of its CIA."""
    w = S.kuramoto_lognormal(scale=1 / 8, steps=20)
    g = w.graph
    plan = make_plan(cia, g, w.omega, w.K, precision="fp32", tile_nodes=32, tile_index_bytes=8192,
                     staging="stream")
    assert plan.info()["staging"] == 4 and plan.info()["n_tiles"] > 4 * 152
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    omp = w.omega[sp.perm]
    rhs = lambda x: oracle_mod.kuramoto_cia(sp, x, omp, w.K)
    ref, r_ref = oracle_mod.integrate(rhs, w.theta0[sp.perm], w.dt, w.steps, wrap=True,
                                      observe=oracle_mod.order_parameter)
    x = torch_mod.from_numpy(w.theta0.copy()).cuda()
    r = torch_mod.zeros(w.steps, dtype=torch_mod.float64, device="cuda")
    plan.integrate(x, w.dt, w.steps, r_out=r)
    plan.sync()
    assert np.abs(r.cpu().numpy() - np.array(r_ref)).max() < 1e-5
    got = x.cpu().numpy()[sp.perm]
    assert np.abs(oracle_mod.angle_diff(got, ref)).max() < 1e-4


@pytest.mark.parametrize("lam,staging", [(20000, 2), (50000, 1)])
def test_rhs_fp32_large_communities(cia, oracle_mod, torch_mod, lam, staging):
    """Communities above 10^4 nodes in FP32 (p_in 0.95, inter degree 8, a few
    unlabelled nodes): the community observable of lam unit phasors summed by
    32-term warp trees in FP32 and in FP64 above them must keep the coupling
    part within the FP32 bar.  lam = 20000 still takes the shared-memory window
    (160 KB); lam = 50000 does not fit it, so the whole plan takes the
    plain-load kernel."""
    g = S.hash_sbm_graph([lam, 1500, 37], 0.95, seed=70 + lam // 10000, inter_degree=8.0, n_free=13)
    rng = np.random.default_rng(lam)
    th = S.as_fp32_values(rng.uniform(-np.pi, np.pi, g.n))
    th[:lam] = S.as_fp32_values(0.3 * rng.standard_normal(lam))   # partly synchronised: |Z| ~ lam
    om = S.as_fp32_values(0.5 * rng.standard_cauchy(g.n))
    plan = cia.Plan(g.rowptr, g.col, g.labels, om, K=2.0, precision="fp32")
    assert plan.info()["staging"] == staging
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 2.0)
    got = gpu_rhs(torch_mod, plan, th, "cia")
    assert coupling_rel_err(got, ref, om) < FP32_TOL
    # the nodes of the large community alone (their coupling is the largest)
    assert coupling_rel_err(got[:lam], ref[:lam], om[:lam]) < FP32_TOL


# ------------------------------------------------------------------ integration

def test_integrate_fp64_small_sbm(cia, oracle_mod, torch_mod):
    """The full small workload: FP64, RK4 dt = 0.01, 100 steps."""
    w = S.kuramoto_sbm_small()
    g = w.graph
    rhs = lambda x: oracle_mod.kuramoto_direct(g.rowptr, g.col, x, w.omega, w.K)
    ref, r_ref = oracle_mod.integrate(rhs, w.theta0, w.dt, w.steps, wrap=True,
                                      observe=oracle_mod.order_parameter)
    plan = make_plan(cia, g, w.omega, w.K)
    for method in ("cia", "direct"):
        x = torch_mod.from_numpy(w.theta0.copy()).cuda()
        r = torch_mod.zeros(w.steps, dtype=torch_mod.float64, device="cuda")
        plan.integrate(x, w.dt, w.steps, method=method, r_out=r)
        got = x.cpu().numpy()
        assert np.abs(oracle_mod.angle_diff(got, ref)).max() < 1e-10, method
        assert np.abs(r.cpu().numpy() - np.array(r_ref)).max() < 1e-12, method
        assert np.all(np.abs(got) <= np.pi + 1e-12)


def test_integrate_host_buffers(cia, oracle_mod, torch_mod):
    w = S.kuramoto_sbm_small()
    g = w.graph
    plan = make_plan(cia, g, w.omega, w.K)
    x_dev = torch_mod.from_numpy(w.theta0.copy()).cuda()
    plan.integrate(x_dev, w.dt, 10)
    x_host = w.theta0.copy()
    r = np.zeros(10)
    plan.integrate_host(x_host, w.dt, 10, r_out=r)
    assert np.array_equal(x_host, x_dev.cpu().numpy())
    assert 0.0 < r.min() and r.max() <= 1.0


def test_integrate_fp32_lognormal_reduced_horizon(cia, oracle_mod, torch_mod):
    """Reduced lognormal workload over its full 2000-step horizon: r(t)
    within 1e-3 of the FP64 oracle at every step."""
    w = S.kuramoto_lognormal(scale=1 / 32)
    g = w.graph
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    omp = w.omega[sp.perm]
    rhs = lambda x: oracle_mod.kuramoto_cia(sp, x, omp, w.K)
    _, r_ref = oracle_mod.integrate(rhs, w.theta0[sp.perm], w.dt, w.steps, wrap=True,
                                    observe=oracle_mod.order_parameter)
    plan = make_plan(cia, g, w.omega, w.K, precision="fp32")
    x = torch_mod.from_numpy(w.theta0.copy()).cuda()
    r = torch_mod.zeros(w.steps, dtype=torch_mod.float64, device="cuda")
    plan.integrate(x, w.dt, w.steps, r_out=r)
    assert np.abs(r.cpu().numpy() - np.array(r_ref)).max() < R_TOL


def test_fp64_master_keeps_large_frequencies(cia, torch_mod):
    """Uncoupled oscillators with huge frequencies: theta(T) = wrap(theta0 +
    omega T) exactly up to FP64 rounding in both precisions (the time
    accumulation is FP64 even for FP32 plans)."""
    n = 64
    g = S.Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32),
                np.full(n, -1, np.int32), np.zeros(0, np.int64))
    om = S.as_fp32_values(np.geomspace(1.0, 3e4, n))
    th0 = np.linspace(-3, 3, n)
    for prec in ("fp64", "fp32"):
        plan = make_plan(cia, g, om, 1.0, precision=prec)
        x = torch_mod.from_numpy(th0.copy()).cuda()
        plan.integrate(x, 0.01, 500)
        want = np.remainder(th0 + om * 5.0 + np.pi, 2 * np.pi) - np.pi
        diff = np.remainder(x.cpu().numpy() - want + np.pi, 2 * np.pi) - np.pi
        assert np.abs(diff).max() < 1e-9, prec


# ------------------------------------------------------------------ errors

def test_error_paths(cia, torch_mod):
    w = S.kuramoto_sbm_small()
    g = w.graph
    plan = cia.Plan(g.rowptr, g.col, g.labels, w.omega, K=w.K)     # no build_direct
    x = torch_mod.from_numpy(w.theta0.copy()).cuda()
    with pytest.raises(cia.CiaError) as e:
        plan.rhs(x, method="direct")
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"
    with pytest.raises(cia.CiaError) as e:
        plan.integrate(x, float("nan"), 3)
    assert e.value.status_name == "CIA_ERR_NUMERIC"


def test_bounded_wait_reports_timeout_and_context_survives(cia, oracle_mod, torch_mod):
    """Failure detection without a fault: a wait that nothing completes gives
    up after its bound, the next sync reports CIA_ERR_TIMEOUT once, and the
    plan keeps computing correct results afterwards."""
    w = S.kuramoto_sbm_small()
    g = w.graph
    plan = cia.Plan(g.rowptr, g.col, g.labels, w.omega, K=w.K)
    plan.selftest_bounded_wait(2_000_000)      # 2 ms
    with pytest.raises(cia.CiaError) as e:
        plan.sync()
    assert e.value.status_name == "CIA_ERR_TIMEOUT"
    plan.sync()                                # the flag was cleared
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, w.theta0, w.omega, w.K)
    assert coupling_rel_err(gpu_rhs(torch_mod, plan, w.theta0, "cia"), ref, w.omega) < FP64_TOL
    with pytest.raises(cia.CiaError) as e:
        plan.selftest_bounded_wait(10)         # out of range
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"


def test_partition_choice_beats_the_s_minimal_partition(cia, torch_mod):
    """Step P1's communities-vs-cost trade-off, measured: 4096 communities of
    16 nodes (p_in 0.95) in groups of 8 linked at density 0.45, so that the
    S-minimal partition keeps the small communities (one short tile each)
    while merging a group adds only a few entries to S and removes 7 tiles.
    The chosen partition must be coarser and faster, as measured, than the
    partition with mu = 0."""
    g = S.hierarchical_sbm_graph(512, 8, 16, 0.95, 0.45, seed=3, inter_degree=4.0)
    rng = np.random.default_rng(0)
    x0 = rng.uniform(-np.pi, np.pi, g.n)
    om = rng.normal(size=g.n)
    labels, rep = cia.choose_partition(g.rowptr, g.col, om, x0, 0.01, steps=10, K=2.0)
    ms = rep["ms_per_step"]
    assert rep["communities"][0] >= 2048            # mu = 0 keeps (nearly all) small communities
    assert rep["chosen"] != 0
    c = rep["chosen"]
    assert rep["communities"][c] < rep["communities"][0] and ms[c] < ms[0]
    assert rep["per_tile_us"] > 0 and rep["community_cost"] > 0
    assert len(np.unique(labels[labels >= 0])) == rep["communities"][c]


def test_single_steps_replay_the_captured_graph_bit_exactly(cia, torch_mod):
    """advance(dt, 2) captures the step graph; later one-step calls with the
    same dt replay it from their first step.  Five steps taken that way (2 +
    1 + 1 + 1), and with r(t) through the host-buffer call (one two-step call,
    then one-step calls), equal five steps of plain launches bit for bit."""
    g = S.sbm_graph([300, 200, 120], 0.9, inter_degree=4.0, seed=41, n_free=9)
    rng = np.random.default_rng(42)
    omega = S.as_fp32_values(rng.normal(size=g.n))
    theta0 = S.as_fp32_values(rng.uniform(0.0, 2.0 * np.pi, g.n))
    dt = 0.01
    states = {}
    for graphs in (True, False):
        plan = make_plan(cia, g, omega, 2.0, precision="fp32", use_graphs=graphs, tile_nodes=64)
        x = torch_mod.from_numpy(theta0.copy()).cuda()
        plan.state_load(x)
        plan.advance(dt, 2)
        for _ in range(3):
            plan.advance(dt, 1)
        plan.state_store(x)
        xh = theta0.copy()
        r = np.zeros(5)
        plan.integrate_host(xh, dt, 2, r_out=r[:2])
        for k in range(3):
            plan.integrate_host(xh, dt, 1, r_out=r[2 + k:3 + k])
        states[graphs] = (x.cpu().numpy(), xh, r)
    for a, b in zip(states[True], states[False]):
        np.testing.assert_array_equal(a, b)
