"""Parity of the CUDA general-coupling path (polynomial moments, App. A.3;
Desai--Zwanzig, App. A.5; rank-one weights; real 2-D Fourier series) with the
FP64 oracle, through the C ABI.

Tolerances (written here, derived from the arithmetic): the path is FP64
throughout; the moment expansion cancels terms of size lambda max|x|^p against
each other, so the coupling part of the RHS is compared norm-wise within
1e-12 relative (inf-norm); trajectories of 100 RK4 steps within 1e-11 of the
largest state; the linear-consensus closed form within 1e-12.
"""
import numpy as np
import pytest

import synthetic as S
from helpers import coupling_rel_err, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

FP64_TOL = 1e-12
DW_DV = (0.0, -1.0, 0.0, 1.0)      # V(x) = x^4/4 - x^2/2: V'(x) = x^3 - x


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


def make_plan(cia, g, K, c, dv, **kw):
    return cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial", K=K, poly_c=c, dV=dv,
                    precision="fp64", build_direct=True, **kw)


def gpu_rhs(torch_mod, plan, x, method):
    xd = torch_mod.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    out = plan.rhs(xd, method=method)
    torch_mod.cuda.synchronize()
    return out.cpu().numpy()


def coupling_err(oracle_mod, g, x, got, ref, c, dv):
    # the potential term alone: the oracle with K = 0
    pot = oracle_mod.poly_direct(g.rowptr, g.col, x, 0.0, c, dv)
    return coupling_rel_err(got, ref, pot)


# ------------------------------------------------------------------ RHS parity

@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_rhs_degrees(cia, oracle_mod, torch_mod, p):
    rng = np.random.default_rng(100 + p)
    g = S.sbm_graph([40, 70, 33, 64], 0.8, inter_degree=5.0, seed=70 + p, n_free=9)
    c = rng.normal(size=p + 1)
    dv = rng.normal(size=5)
    x = rng.normal(size=g.n)
    plan = make_plan(cia, g, 1.7, c, dv, tile_nodes=32)
    ref = oracle_mod.poly_direct(g.rowptr, g.col, x, 1.7, c, dv)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        if p == 0:
            # h constant: the coupling is K/N c_0 deg(m), no cancellation
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), method
        else:
            assert coupling_err(oracle_mod, g, x, got, ref, c, dv) < FP64_TOL, method


@pytest.mark.parametrize("staging", ["auto", "plain"])
@pytest.mark.parametrize("group_size", [4, 16, 32])
@pytest.mark.parametrize("tile_nodes,tile_index_bytes", [(32, 0), (96, 0), (256, 0), (256, 256),
                                                         (128, 4096)])
def test_rhs_launch_shapes(cia, oracle_mod, torch_mod, group_size, tile_nodes, tile_index_bytes,
                           staging):
    """Several tiles per community with a ragged tail, index budgets that cut
    tiles at single rows, every group width of the direct kernel, the community
    window in shared memory (auto) and read from global memory (plain)."""
    g = S.sbm_graph([300, 129, 31, 700], 0.9, inter_degree=6.0, seed=7, n_free=40)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1.5, 1.5, g.n)
    c, dv = (0.1, 1.0, -0.3, 0.2), DW_DV
    plan = make_plan(cia, g, 2.5, c, dv, tile_nodes=tile_nodes, group_size=group_size,
                     tile_index_bytes=tile_index_bytes, staging=staging)
    assert plan.info()["staging"] == (1 if staging == "plain" else 2)
    ref = oracle_mod.poly_direct(g.rowptr, g.col, x, 2.5, c, dv)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        assert coupling_err(oracle_mod, g, x, got, ref, c, dv) < FP64_TOL, method


@pytest.mark.parametrize("case", ["all_free", "no_edges", "single_node", "empty_labels",
                                  "singletons", "complete"])
def test_rhs_degenerate_graphs(cia, oracle_mod, torch_mod, case):
    rng = np.random.default_rng(5)
    if case == "all_free":
        g = S.random_labels_graph(30, 0.3, 1, seed=1, free_frac=1.0)
    elif case == "no_edges":
        g = S.random_labels_graph(20, 0.0, 3, seed=2, free_frac=0.1)
    elif case == "single_node":
        g = S.Graph(1, np.array([0, 0], np.int64), np.zeros(0, np.int32),
                    np.array([0], np.int32), np.array([1], np.int64))
    elif case == "empty_labels":
        g = S.random_labels_graph(40, 0.4, 3, seed=4, free_frac=0.0)
        g.labels = (g.labels * 3 + 2).astype(np.int32)
    elif case == "singletons":
        g = S.random_labels_graph(25, 0.5, 1, seed=5, free_frac=0.0)
        g.labels = np.arange(g.n, dtype=np.int32)
    else:
        g = S.complete_graph_communities([17, 5, 1], seed=6)
    x = rng.normal(size=g.n)
    c, dv = (0.2, -1.0, 0.5, 0.25, -0.1), (0.3, -1.0, 0.1, 1.0, 0.05)
    plan = make_plan(cia, g, 1.5, c, dv)
    ref = oracle_mod.poly_direct(g.rowptr, g.col, x, 1.5, c, dv)
    pot = oracle_mod.poly_direct(g.rowptr, g.col, x, 0.0, c, dv)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        if np.abs(ref - pot).max() == 0:
            assert np.abs(got - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max()), method
        else:
            assert coupling_rel_err(got, ref, pot) < FP64_TOL, method


@pytest.mark.parametrize("staging", ["auto", "plain"])
def test_rhs_wide_dynamic_range_and_zero_communities(cia, oracle_mod, torch_mod, staging):
    """States spanning eight decades inside one community (the shared-memory
    window holds fixed-point powers scaled by the community's largest one),
    and a community whose states are all zero."""
    g = S.sbm_graph([300, 129, 64], 0.9, inter_degree=6.0, seed=17, n_free=20)
    rng = np.random.default_rng(12)
    x = rng.choice([-1.0, 1.0], g.n) * 10.0 ** rng.uniform(-6, 2, g.n)
    x[g.labels == 2] = 0.0
    c, dv = (0.3, -1.0, 0.2, 0.01), (0.0, 1.0)
    plan = make_plan(cia, g, 1.0, c, dv, staging=staging)
    ref = oracle_mod.poly_direct(g.rowptr, g.col, x, 1.0, c, dv)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        assert coupling_err(oracle_mod, g, x, got, ref, c, dv) < FP64_TOL, method
    G = rng.normal(size=(4, 4))
    gplan = make_general(cia, g, 1.0, G, dv, staging=staging)
    gref = oracle_mod.polyg_direct(g.rowptr, g.col, x, 1.0, G, dv)
    assert general_err(oracle_mod, g, x, gpu_rhs(torch_mod, gplan, x, "cia"), gref, G, dv) < FP64_TOL


def test_rhs_matches_oracle_cia_permuted(cia, oracle_mod, torch_mod):
    """The oracle's own moment formula (permuted order) agrees with the device
    CIA too: the same E1/E2 split, evaluated independently."""
    g = S.sbm_graph([64, 200, 90], 0.85, inter_degree=4.0, seed=12, n_free=11)
    rng = np.random.default_rng(8)
    x = rng.normal(size=g.n)
    c, dv = (0.0, 1.0, 0.0, -0.2), DW_DV
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    ref = oracle_mod.poly_cia(sp, x[sp.perm], 0.9, c, dv)[sp.iperm]
    plan = make_plan(cia, g, 0.9, c, dv)
    got = gpu_rhs(torch_mod, plan, x, "cia")
    assert coupling_err(oracle_mod, g, x, got, ref, c, dv) < FP64_TOL


# ------------------------------------------------------------------ integration

def test_integrate_desai_zwanzig(cia, oracle_mod, torch_mod):
    """Double-well units (V' = x^3 - x) with linear attraction on a community
    graph: 100 RK4 steps of dt = 0.01 against the oracle's RK4 of the direct sum."""
    g = S.sbm_graph([120, 300, 57, 200], 0.7, inter_degree=5.0, seed=21, n_free=23)
    rng = np.random.default_rng(9)
    x0 = rng.normal(0.0, 1.2, g.n)
    c, K, dt, steps = (0.0, 1.0), 4.0, 0.01, 100
    rhs = lambda y: oracle_mod.poly_direct(g.rowptr, g.col, y, K, c, DW_DV)
    ref, _ = oracle_mod.integrate(rhs, x0, dt, steps, wrap=False)
    plan = make_plan(cia, g, K, c, DW_DV)
    for method in ("cia", "direct"):
        x = torch_mod.from_numpy(x0.copy()).cuda()
        plan.integrate(x, dt, steps, method=method)
        got = x.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max(), method


def test_integrate_cubic_coupling_graph_replay(cia, oracle_mod, torch_mod):
    """A cubic h on a larger graph (several tiles per community) through
    several advance calls: CUDA-graph replay and plain launches agree with the
    oracle's RK4."""
    g = S.sbm_graph([700, 300, 129], 0.9, inter_degree=6.0, seed=31, n_free=17)
    rng = np.random.default_rng(10)
    x0 = rng.uniform(-1.0, 1.0, g.n)
    c, dv, K, dt = (0.0, 0.5, 0.0, -0.3), (0.0, -1.0, 0.0, 1.0), 3.0, 0.02
    rhs = lambda y: oracle_mod.poly_direct(g.rowptr, g.col, y, K, c, dv)
    ref, _ = oracle_mod.integrate(rhs, x0, dt, 40, wrap=False)
    for graphs in (True, False):
        plan = make_plan(cia, g, K, c, dv, tile_nodes=128, use_graphs=graphs)
        x = torch_mod.from_numpy(x0.copy()).cuda()
        plan.state_load(x)
        for _ in range(4):
            plan.advance(dt, 10)
        plan.state_store(x)
        got = x.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max(), graphs


def test_linear_consensus_closed_form(cia, torch_mod):
    """V' = 0, h(x) = x on one complete community: x' = K (mean - x_m) exactly,
    so each RK4 step keeps the mean and scales every deviation by the RK4
    stability polynomial R(-K dt)."""
    n, K, dt, steps = 300, 1.3, 0.05, 25
    g = S.complete_graph_communities([n], seed=1)
    x0 = np.random.default_rng(4).normal(size=n)
    plan = make_plan(cia, g, K, (0.0, 1.0), (0.0,))
    z = -K * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    want = x0.mean() + (x0 - x0.mean()) * R ** steps
    for method in ("cia", "direct"):
        x = torch_mod.from_numpy(x0.copy()).cuda()
        plan.integrate(x, dt, steps, method=method)
        assert np.abs(x.cpu().numpy() - want).max() < 1e-12, method


def test_integrate_host_buffers(cia, torch_mod):
    g = S.sbm_graph([50, 80], 0.8, inter_degree=3.0, seed=3, n_free=5)
    x0 = np.random.default_rng(6).normal(size=g.n)
    plan = make_plan(cia, g, 2.0, (0.0, 1.0), DW_DV)
    x_dev = torch_mod.from_numpy(x0.copy()).cuda()
    plan.integrate(x_dev, 0.01, 10)
    x_host = x0.copy()
    plan.integrate_host(x_host, 0.01, 10)
    assert np.array_equal(x_host, x_dev.cpu().numpy())


# ------------------------------------------------------------------ general g(x_l, x_m)

def make_general(cia, g, K, G, dv, **kw):
    return cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial_general", K=K, poly_g=G,
                    dV=dv, precision="fp64", build_direct=True, **kw)


def general_err(oracle_mod, g, x, got, ref, G, dv):
    pot = oracle_mod.polyg_direct(g.rowptr, g.col, x, 0.0, G, dv)
    return coupling_rel_err(got, ref, pot)


@pytest.mark.parametrize("staging", ["auto", "plain"])
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_general_rhs_degrees(cia, oracle_mod, torch_mod, p, staging):
    rng = np.random.default_rng(200 + p)
    g = S.sbm_graph([40, 70, 33, 64], 0.8, inter_degree=5.0, seed=90 + p, n_free=9)
    G = rng.normal(size=(p + 1, p + 1))
    dv = rng.normal(size=4)
    x = rng.uniform(-1.2, 1.2, g.n)
    plan = make_general(cia, g, 1.4, G, dv, tile_nodes=32, staging=staging)
    assert plan.info()["model"] == 4
    ref = oracle_mod.polyg_direct(g.rowptr, g.col, x, 1.4, G, dv)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        assert general_err(oracle_mod, g, x, got, ref, G, dv) < FP64_TOL, method


@pytest.mark.parametrize("tile_nodes,tile_index_bytes", [(64, 0), (256, 256), (128, 4096)])
def test_general_rhs_launch_shapes(cia, oracle_mod, torch_mod, tile_nodes, tile_index_bytes):
    g = S.sbm_graph([300, 129, 31, 700], 0.9, inter_degree=6.0, seed=8, n_free=40)
    rng = np.random.default_rng(3)
    G = rng.normal(size=(4, 4))
    x = rng.uniform(-1.0, 1.0, g.n)
    plan = make_general(cia, g, 2.0, G, DW_DV, tile_nodes=tile_nodes, tile_index_bytes=tile_index_bytes)
    ref = oracle_mod.polyg_direct(g.rowptr, g.col, x, 2.0, G, DW_DV)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        assert general_err(oracle_mod, g, x, got, ref, G, DW_DV) < FP64_TOL, method


@pytest.mark.parametrize("case", ["all_free", "single_node", "singletons", "complete"])
def test_general_rhs_degenerate_graphs(cia, oracle_mod, torch_mod, case):
    if case == "all_free":
        g = S.random_labels_graph(30, 0.3, 1, seed=1, free_frac=1.0)
    elif case == "single_node":
        g = S.Graph(1, np.array([0, 0], np.int64), np.zeros(0, np.int32),
                    np.array([0], np.int32), np.array([1], np.int64))
    elif case == "singletons":
        g = S.random_labels_graph(25, 0.5, 1, seed=5, free_frac=0.0)
        g.labels = np.arange(g.n, dtype=np.int32)
    else:
        g = S.complete_graph_communities([17, 5, 1], seed=6)
    rng = np.random.default_rng(6)
    G = rng.normal(size=(3, 3))
    x = rng.normal(size=g.n)
    plan = make_general(cia, g, 1.5, G, (0.3, -1.0))
    ref = oracle_mod.polyg_direct(g.rowptr, g.col, x, 1.5, G, (0.3, -1.0))
    pot = oracle_mod.polyg_direct(g.rowptr, g.col, x, 0.0, G, (0.3, -1.0))
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        if np.abs(ref - pot).max() == 0:
            assert np.abs(got - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max()), method
        else:
            assert coupling_rel_err(got, ref, pot) < FP64_TOL, method


def test_general_matches_difference_plan(cia, torch_mod):
    """g(u, y) = h(u - y) written out as G_ab = c_{a+b} binom(a+b, a) (-1)^b:
    the general and the difference plans agree on the device."""
    from math import comb
    g = S.sbm_graph([200, 90, 31], 0.85, inter_degree=4.0, seed=13, n_free=7)
    c = (0.2, 1.0, -0.5, 0.3)
    p = len(c) - 1
    G = np.zeros((p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1 - a):
            G[a, b] = c[a + b] * comb(a + b, a) * (-1) ** b
    x = np.random.default_rng(5).uniform(-1, 1, g.n)
    gen = gpu_rhs(torch_mod, make_general(cia, g, 1.2, G, DW_DV), x, "cia")
    dif = gpu_rhs(torch_mod, make_plan(cia, g, 1.2, c, DW_DV), x, "cia")
    assert np.abs(gen - dif).max() < 1e-12 * np.abs(dif).max()


def test_general_integrate(cia, oracle_mod, torch_mod):
    g = S.sbm_graph([120, 300, 57], 0.7, inter_degree=5.0, seed=22, n_free=13)
    rng = np.random.default_rng(11)
    x0 = rng.uniform(-0.8, 0.8, g.n)
    G = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, -0.2], [0.1, 0.0, 0.0]])
    K, dt, steps = 2.0, 0.01, 60
    rhs = lambda y: oracle_mod.polyg_direct(g.rowptr, g.col, y, K, G, DW_DV)
    ref, _ = oracle_mod.integrate(rhs, x0, dt, steps, wrap=False)
    plan = make_general(cia, g, K, G, DW_DV)
    for method in ("cia", "direct"):
        x = torch_mod.from_numpy(x0.copy()).cuda()
        plan.integrate(x, dt, steps, method=method)
        assert np.abs(x.cpu().numpy() - ref).max() < 1e-11 * np.abs(ref).max(), method


# ------------------------------------------------------------------ rank-one link weights

def difference_as_general(c):
    from math import comb
    p = len(c) - 1
    G = np.zeros((p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1 - a):
            G[a, b] = c[a + b] * comb(a + b, a) * (-1) ** b
    return G


@pytest.mark.parametrize("staging", ["auto", "plain"])
@pytest.mark.parametrize("form,p", [("difference", 1), ("difference", 3), ("general", 2), ("general", 4)])
def test_weighted_rhs(cia, oracle_mod, torch_mod, form, p, staging):
    g = S.sbm_graph([300, 129, 31, 200], 0.85, inter_degree=6.0, seed=40 + p, n_free=25)
    rng = np.random.default_rng(60 + p)
    x = rng.uniform(-1.2, 1.2, g.n)
    al = rng.uniform(0.5, 2.0, g.n)
    be = rng.normal(size=g.n)
    be[::7] = 0.0
    dv = (0.1, -1.0, 0.0, 1.0)
    if form == "difference":
        c = rng.normal(size=p + 1)
        G = difference_as_general(c)
        plan = make_plan(cia, g, 1.3, c, dv, tile_nodes=128, staging=staging)
    else:
        G = rng.normal(size=(p + 1, p + 1))
        plan = make_general(cia, g, 1.3, G, dv, tile_nodes=128, staging=staging)
    plan.set_weights(al, be)
    assert plan.info()["staging"] == (1 if staging == "plain" else 2)
    ref = oracle_mod.polyw_direct(g.rowptr, g.col, x, 1.3, G, dv, al, be)
    pot = oracle_mod.polyw_direct(g.rowptr, g.col, x, 0.0, G, dv, al, be)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        assert coupling_rel_err(got, ref, pot) < FP64_TOL, method


def test_weighted_one_sided_and_removed(cia, oracle_mod, torch_mod):
    """alpha alone, beta alone, then no weights: the unweighted plan's values."""
    g = S.sbm_graph([150, 90], 0.8, inter_degree=4.0, seed=3, n_free=10)
    rng = np.random.default_rng(7)
    x = rng.normal(size=g.n)
    c, dv = (0.0, 1.0, -0.2), DW_DV
    G = difference_as_general(c)
    plan = make_plan(cia, g, 2.0, c, dv)
    base = gpu_rhs(torch_mod, plan, x, "cia")
    ones = np.ones(g.n)
    al, be = rng.uniform(0, 2, g.n), rng.uniform(-1, 1, g.n)
    pot = oracle_mod.polyw_direct(g.rowptr, g.col, x, 0.0, G, dv, ones, ones)
    for a_, b_ in ((al, None), (None, be)):
        plan.set_weights(a_, b_)
        ref = oracle_mod.polyw_direct(g.rowptr, g.col, x, 2.0, G, dv,
                                      a_ if a_ is not None else ones, b_ if b_ is not None else ones)
        assert coupling_rel_err(gpu_rhs(torch_mod, plan, x, "cia"), ref, pot) < FP64_TOL
    plan.set_weights(None, None)
    assert np.array_equal(gpu_rhs(torch_mod, plan, x, "cia"), base)


def test_weighted_integrate(cia, oracle_mod, torch_mod):
    """Rank-one weighted Desai-Zwanzig network, 50 RK4 steps, CUDA-graph replay."""
    g = S.sbm_graph([400, 200, 77], 0.8, inter_degree=5.0, seed=50, n_free=19)
    rng = np.random.default_rng(13)
    x0 = rng.normal(size=g.n)
    al, be = rng.uniform(0.5, 1.5, g.n), rng.uniform(0.0, 2.0, g.n)
    K, dt, steps = 3.0, 0.01, 50
    G = difference_as_general((0.0, 1.0))
    rhs = lambda y: oracle_mod.polyw_direct(g.rowptr, g.col, y, K, G, DW_DV, al, be)
    ref, _ = oracle_mod.integrate(rhs, x0, dt, steps, wrap=False)
    plan = make_plan(cia, g, K, (0.0, 1.0), DW_DV)
    plan.set_weights(al, be)
    for method in ("cia", "direct"):
        x = torch_mod.from_numpy(x0.copy()).cuda()
        plan.integrate(x, dt, steps, method=method)
        assert np.abs(x.cpu().numpy() - ref).max() < 1e-11 * np.abs(ref).max(), method


def test_weights_rejections(cia, torch_mod):
    g = S.sbm_graph([40, 30], 0.8, inter_degree=2.0, seed=1, n_free=3)
    kplan = cia.Plan(g.rowptr, g.col, g.labels, np.zeros(g.n), K=1.0)
    with pytest.raises(cia.CiaError, match="polynomial"):
        kplan.set_weights(np.ones(g.n), None)
    plan = make_plan(cia, g, 1.0, (0.0, 1.0), DW_DV)
    with pytest.raises(cia.CiaError, match="finite"):
        plan.set_weights(np.full(g.n, np.inf), None)
    with pytest.raises(ValueError):
        plan.set_weights(np.ones(g.n + 1), None)
    x = torch_mod.zeros(g.n, dtype=torch_mod.float64, device="cuda")
    plan.state_load(x)
    plan.set_weights(None, np.ones(g.n))
    with pytest.raises(cia.CiaError, match="load"):
        plan.advance(0.01, 1)


# ------------------------------------------------------------------ general real 2-D Fourier coupling

def make_fourier(cia, g, K, L, C, dv, **kw):
    return cia.Plan(g.rowptr, g.col, g.labels, None, model="fourier_general", K=K, fourier_L=L,
                    fourier_C=C, dV=dv, precision="fp64", build_direct=True, **kw)


def fourier_err(oracle_mod, g, x, got, ref, L, C, dv):
    pot = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 0.0, L, C, dv)
    return coupling_rel_err(got, ref, pot)


@pytest.mark.parametrize("staging", ["auto", "plain"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fourier_rhs_harmonics(cia, oracle_mod, torch_mod, p, staging):
    g = S.sbm_graph([300, 129, 31, 200], 0.85, inter_degree=6.0, seed=90 + p, n_free=25)
    rng = np.random.default_rng(300 + p)
    C = [rng.normal(size=(p + 1, p + 1)) for _ in range(4)]
    dv = (0.2, -1.0, 0.0, 0.5)
    L = 2.0
    x = rng.uniform(-2.5, 2.5, g.n)
    plan = make_fourier(cia, g, 1.4, L, C, dv, tile_nodes=128, staging=staging)
    info = plan.info()
    assert info["model"] == 5 and info["staging"] == (1 if staging == "plain" else 2)
    ref = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 1.4, L, C, dv)
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        assert fourier_err(oracle_mod, g, x, got, ref, L, C, dv) < FP64_TOL, method


def test_fourier_window_runs_by_community_size(cia, oracle_mod, torch_mod):
    """Two harmonics (four window rows of 8 bytes per node): the tiles of the
    6400-node community fit no window and read features from global memory,
    the 2000-, 1000- and 500-node communities fit windows for 2, 3 and 4
    resident CTAs, and the small community and the free nodes share the last
    run.  Every run against the oracle, in one right-hand side and through
    an RK4 step replayed as a CUDA graph."""
    g = S.hash_sbm_graph([6400, 2000, 1000, 500, 100], 0.9, seed=61, inter_degree=4.0, n_free=37)
    rng = np.random.default_rng(62)
    C = [rng.normal(size=(3, 3)) for _ in range(4)]
    dv = (0.1, -1.0, 0.0, 0.4)
    L = 2.0
    x = rng.uniform(-2.5, 2.5, g.n)
    plan = make_fourier(cia, g, 1.1, L, C, dv)
    assert plan.info()["staging"] == 2
    ref = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 1.1, L, C, dv)
    got = gpu_rhs(torch_mod, plan, x, "cia")
    assert fourier_err(oracle_mod, g, x, got, ref, L, C, dv) < FP64_TOL
    dt = 0.01
    rhs = lambda y: oracle_mod.fourierg_direct(g.rowptr, g.col, y, 1.1, L, C, dv)
    want, _ = oracle_mod.integrate(rhs, x, dt, 2, wrap=False)
    xd = torch_mod.from_numpy(x.copy()).cuda()
    plan.state_load(xd)
    plan.advance(dt, 1)
    plan.advance(dt, 1)
    plan.state_store(xd)
    assert np.abs(xd.cpu().numpy() - want).max() < 1e-11 * np.abs(want).max()


def test_fourier_sine_of_difference_matches_kuramoto_plan(cia, torch_mod):
    """sin(w(u - y)) through the general series equals the FP64 Kuramoto plan
    on the phases w x."""
    g = S.sbm_graph([200, 90, 31], 0.85, inter_degree=4.0, seed=14, n_free=7)
    L = 1.5
    x = np.random.default_rng(15).uniform(-L, L, g.n)
    C = [np.zeros((2, 2)) for _ in range(4)]
    C[2][1, 1], C[1][1, 1] = 1.0, -1.0
    four = gpu_rhs(torch_mod, make_fourier(cia, g, 2.0, L, C, (0.0,)), x, "cia")
    kplan = cia.Plan(g.rowptr, g.col, g.labels, np.zeros(g.n), K=2.0, precision="fp64")
    kur = gpu_rhs(torch_mod, kplan, np.pi * x / L, "cia")
    assert np.abs(four - kur).max() < 1e-12 * np.abs(kur).max()


@pytest.mark.parametrize("case", ["all_free", "single_node", "singletons", "complete"])
def test_fourier_rhs_degenerate_graphs(cia, oracle_mod, torch_mod, case):
    if case == "all_free":
        g = S.random_labels_graph(30, 0.3, 1, seed=1, free_frac=1.0)
    elif case == "single_node":
        g = S.Graph(1, np.array([0, 0], np.int64), np.zeros(0, np.int32),
                    np.array([0], np.int32), np.array([1], np.int64))
    elif case == "singletons":
        g = S.random_labels_graph(25, 0.5, 1, seed=5, free_frac=0.0)
        g.labels = np.arange(g.n, dtype=np.int32)
    else:
        g = S.complete_graph_communities([17, 5, 1], seed=6)
    rng = np.random.default_rng(16)
    C = [rng.normal(size=(3, 3)) for _ in range(4)]
    x = rng.uniform(-3, 3, g.n)
    plan = make_fourier(cia, g, 1.5, 3.0, C, (0.3, -1.0))
    ref = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 1.5, 3.0, C, (0.3, -1.0))
    pot = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 0.0, 3.0, C, (0.3, -1.0))
    for method in ("cia", "direct"):
        got = gpu_rhs(torch_mod, plan, x, method)
        if np.abs(ref - pot).max() == 0:
            assert np.abs(got - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max()), method
        else:
            assert coupling_rel_err(got, ref, pot) < FP64_TOL, method


def test_fourier_integrate(cia, oracle_mod, torch_mod):
    """40 RK4 steps of a two-harmonic coupling with a confining potential,
    CUDA-graph replay and plain launches, against the oracle's RK4."""
    g = S.sbm_graph([400, 200, 77], 0.8, inter_degree=5.0, seed=51, n_free=19)
    rng = np.random.default_rng(17)
    x0 = rng.uniform(-1.5, 1.5, g.n)
    C = [0.5 * rng.normal(size=(3, 3)) for _ in range(4)]
    K, L, dt = 2.0, 2.0, 0.01
    rhs = lambda y: oracle_mod.fourierg_direct(g.rowptr, g.col, y, K, L, C, DW_DV)
    ref, _ = oracle_mod.integrate(rhs, x0, dt, 40, wrap=False)
    for graphs in (True, False):
        plan = make_fourier(cia, g, K, L, C, DW_DV, use_graphs=graphs)
        for method in ("cia", "direct"):
            x = torch_mod.from_numpy(x0.copy()).cuda()
            plan.state_load(x)
            for _ in range(4):
                plan.advance(dt, 10, method=method)
            plan.state_store(x)
            assert np.abs(x.cpu().numpy() - ref).max() < 1e-11 * np.abs(ref).max(), (graphs, method)


def test_fourier_rejections(cia):
    g = S.sbm_graph([40, 30], 0.8, inter_degree=2.0, seed=1, n_free=3)
    C = [np.zeros((2, 2)) for _ in range(4)]
    with pytest.raises(cia.CiaError, match="fourier_L"):
        make_fourier(cia, g, 1.0, 0.0, C, (0.0,))
    with pytest.raises(ValueError):
        make_fourier(cia, g, 1.0, 1.0, [np.zeros((1, 1))] * 4, (0.0,))
    with pytest.raises(ValueError):
        make_fourier(cia, g, 1.0, 1.0, C[:3], (0.0,))
    bad = [c.copy() for c in C]
    bad[3][1, 1] = np.nan
    with pytest.raises(cia.CiaError, match="finite"):
        make_fourier(cia, g, 1.0, 1.0, bad, (0.0,))
    plan = make_fourier(cia, g, 1.0, 1.0, C, (0.0,))
    with pytest.raises(cia.CiaError, match="polynomial"):
        plan.set_weights(np.ones(g.n), None)


# ------------------------------------------------------------------ errors

def test_plan_rejections(cia, torch_mod):
    g = S.sbm_graph([40, 30], 0.8, inter_degree=2.0, seed=1, n_free=3)
    with pytest.raises(cia.CiaError, match="omega"):
        cia.Plan(g.rowptr, g.col, g.labels, np.zeros(g.n), model="polynomial", poly_c=(0.0, 1.0))
    with pytest.raises(cia.CiaError, match="FP64"):
        cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial", precision="fp32")
    with pytest.raises(cia.CiaError, match="tile_nodes"):
        cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial", tile_nodes=512)
    with pytest.raises(ValueError):
        cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial", poly_c=tuple(range(6)))
    with pytest.raises(ValueError):
        cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial_general", poly_g=np.zeros((2, 3)))
    with pytest.raises(cia.CiaError, match="finite"):
        cia.Plan(g.rowptr, g.col, g.labels, None, model="polynomial_general",
                 poly_g=np.array([[0.0, np.nan], [1.0, 0.0]]))
    plan = make_plan(cia, g, 1.0, (0.0, 1.0), DW_DV)
    x = torch_mod.zeros(g.n, dtype=torch_mod.float64, device="cuda")
    r = torch_mod.zeros(3, dtype=torch_mod.float64, device="cuda")
    with pytest.raises(cia.CiaError, match="r_out"):
        plan.integrate(x, 0.01, 3, r_out=r)
    with pytest.raises(cia.CiaError):
        plan.autotune(x, 0.01, 1)
