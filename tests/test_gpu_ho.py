"""Parity of the higher-order (triadic) Kuramoto path with the FP64 oracle.

The triadic term lives on the complete hyperedges of each community
(App. A.7 with lambda = (1, 1, -2)); the oracle's brute-force sum over ordered
pairs is the reference, its moment formula (pinned to the brute force) gives the
long runs.  Tolerances as for the pairwise model: FP64 1e-12, FP32 1e-5
(coupling part, inf-norm relative)."""
import numpy as np
import pytest

import synthetic as S
from helpers import coupling_rel_err, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def ho_reference(oracle_mod, g, th, om, K, K2, nodes=None):
    """omega + pairwise direct + triadic brute force (original order);
    with `nodes` (original ids) only those entries are valid."""
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    pair = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, K)
    phi = th[sp.perm]
    if nodes is None:
        tri = oracle_mod.ho_triadic_direct(sp, phi, K2, np.arange(g.n))[sp.iperm]
        return pair + tri
    tri = oracle_mod.ho_triadic_direct(sp, phi, K2, sp.iperm[nodes])
    out = pair.copy()
    out[nodes] += tri
    return out


def gpu_rhs(plan, x, method):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.rhs(xd, method=method)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(3))
def test_ho_rhs_small(oracle_mod, precision, seed):
    import paper_2203_16657_gb300 as cia
    rng = np.random.default_rng(seed)
    g = S.sbm_graph([int(rng.integers(5, 60)) for _ in range(4)], 0.8, inter_degree=4.0,
                    seed=seed, n_free=5)
    th = S.as_fp32_values(rng.uniform(-np.pi, np.pi, g.n))
    om = S.as_fp32_values(rng.normal(size=g.n))
    K, K2 = 1.3, 2.0
    plan = cia.Plan(g.rowptr, g.col, g.labels, om, K=K, model="kuramoto_ho", K2=K2,
                    precision=precision, build_direct=True, tile_nodes=32)
    ref = ho_reference(oracle_mod, g, th, om, K, K2)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for method in ("cia", "direct"):
        assert coupling_rel_err(gpu_rhs(plan, th, method), ref, om) < tol, method


def test_ho_rhs_reduced_workload(oracle_mod):
    """The higher-order workload at 1/16 of its communities (4 x 64 nodes)."""
    import paper_2203_16657_gb300 as cia
    w = S.kuramoto_ho(scale=1 / 16)
    g = w.graph
    plan = cia.Plan(g.rowptr, g.col, g.labels, w.omega, K=w.K, model="kuramoto_ho", K2=w.K2,
                    precision="fp32", build_direct=True)
    ref = ho_reference(oracle_mod, g, w.theta0, w.omega, w.K, w.K2)
    for method in ("cia", "direct"):
        assert coupling_rel_err(gpu_rhs(plan, w.theta0, method), ref, w.omega) < 1e-5, method


def test_ho_rhs_full_size_sampled(oracle_mod):
    """Full size (N = 65536, 64 x 1024): the CIA right-hand side at 512
    sampled nodes against the oracle's pair-by-pair triadic sum."""
    import paper_2203_16657_gb300 as cia
    w = S.kuramoto_ho()
    g = w.graph
    plan = cia.Plan(g.rowptr, g.col, g.labels, w.omega, K=w.K, model="kuramoto_ho", K2=w.K2,
                    precision="fp32")
    got = gpu_rhs(plan, w.theta0, "cia")
    nodes = np.random.default_rng(2).choice(g.n, 512, replace=False)
    ref = ho_reference(oracle_mod, g, w.theta0, w.omega, w.K, w.K2, nodes=nodes)
    assert coupling_rel_err(got[nodes], ref[nodes], w.omega[nodes]) < 1e-5


def test_ho_integrate_fp64(oracle_mod):
    """RK4 with the triadic term: 50 steps on a small planted graph, FP64,
    against the oracle's RK4 with its (pinned) moment formula."""
    import torch
    import paper_2203_16657_gb300 as cia
    g = S.sbm_graph([40, 25, 31], 0.9, inter_degree=3.0, seed=12, n_free=3)
    rng = np.random.default_rng(4)
    th0 = rng.uniform(0, 2 * np.pi, g.n)
    om = rng.normal(size=g.n)
    K, K2, dt, steps = 1.0, 3.0, 0.01, 50
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)

    def rhs(x):
        pair = oracle_mod.kuramoto_direct(g.rowptr, g.col, x, om, K)
        return pair + oracle_mod.ho_triadic_cia(sp, x[sp.perm], K2)[sp.iperm]

    ref, _ = oracle_mod.integrate(rhs, th0, dt, steps, wrap=True)
    plan = cia.Plan(g.rowptr, g.col, g.labels, om, K=K, model="kuramoto_ho", K2=K2,
                    build_direct=True)
    for method in ("cia", "direct"):
        x = torch.from_numpy(th0.copy()).cuda()
        plan.integrate(x, dt, steps, method=method)
        assert np.abs(oracle_mod.angle_diff(x.cpu().numpy(), ref)).max() < 1e-10, method
