"""The allocation-free right-hand side (cia_rhs_kuramoto_static).

Some callers cannot let the library allocate device memory: their host
application owns the device-memory pool, or their loop may not call
cudaMalloc, which can synchronise the device.  cia_rhs_kuramoto_static serves
them from a fixed scratch array inside the library.  These tests call it
through the C ABI, two calls in a row on different states, and check each
result against the FP64 oracle's direct sum (eq. GeneralNetworkSystem) and
against cia_rhs on the same state, within the FP64 parity tolerance of the
other tests; they also cover the branches the header promises (no
communities, omega NULL, empty halves of S with NULL column arrays) and the
capacity limit on both sides.  The file is named so that pytest collects it
last.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from helpers import coupling_rel_err, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

FP64_TOL = 1e-12
CAPACITY = 327680          # complex entries of the scratch array: p * (n + M) at most


def _coupling(abi, K, d_sin, d_cos):
    cp = abi.Coupling()
    cp.model = abi.MODEL["kuramoto"]
    cp.p = len(d_sin)
    for k in range(len(d_sin)):
        cp.d_sin[k] = float(d_sin[k])
        cp.d_cos[k] = float(d_cos[k])
    cp.K = float(K)
    return cp


def _static_calls(oracle_mod, g, K, d_sin, d_cos, omega, calls=2, seed=7, check_plan=True):
    """Call the entry point `calls` times on fresh states and compare each
    result with the oracle's direct sum and with cia_rhs."""
    import torch
    import paper_2203_16657_gb300 as cia
    from paper_2203_16657_gb300 import _abi

    rng = np.random.default_rng(seed)
    plan = cia.Plan(g.rowptr, g.col, g.labels, omega, K=K, d_sin=d_sin, d_cos=d_cos)
    perm, off = plan.permutation()
    mrp, mcol, irp, icol = plan.split()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None
    d_off, d_mrp, d_mcol, d_irp, d_icol = dev(off), dev(mrp), dev(mcol), dev(irp), dev(icol)
    d_om = dev(np.asarray(omega)[perm]) if omega is not None else None
    cp = _coupling(_abi, K, d_sin, d_cos)
    lib = cia.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    om = np.zeros(g.n) if omega is None else np.asarray(omega)
    for call in range(calls):
        x = rng.uniform(-np.pi, np.pi, g.n)
        want = oracle_mod.kuramoto_direct(g.rowptr, g.col, x, om, K, d_sin, d_cos)
        out = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.cia_rhs_kuramoto_static(g.n, len(off) - 1, ptr(d_off), ptr(d_mrp), ptr(d_mcol),
                                         ptr(d_irp), ptr(d_icol), ptr(dev(x[perm])), ptr(d_om),
                                         ctypes.byref(cp), ptr(out), stream)
        _abi.check(st)
        torch.cuda.synchronize()
        got = np.empty(g.n)
        got[perm] = out.cpu().numpy()
        assert np.isfinite(got).all(), call
        assert coupling_rel_err(got, want, om) < FP64_TOL, call
        if check_plan:                                     # the existing entry point
            ref = plan.rhs(dev(x)).cpu().numpy()
            assert coupling_rel_err(got, ref, om) < FP64_TOL, call
    return len(mcol), len(icol), len(off) - 1


@pytest.mark.parametrize("d_sin,d_cos", [((1.0,), (0.0,)), ((0.7, -0.3, 0.2), (0.1, 0.4, -0.5))])
def test_static_rhs_matches_oracle_and_cia_rhs_twice(oracle_mod, d_sin, d_cos):
    g = S.sbm_graph([120, 75, 200, 33], 0.85, inter_degree=5.0, seed=31, n_free=17)
    omega = np.random.default_rng(3).normal(size=g.n)
    nm, ni, M = _static_calls(oracle_mod, g, 2.5, d_sin, d_cos, omega)
    assert nm > 0 and ni > 0 and M == 4


def test_static_rhs_without_communities_and_omega(oracle_mod):
    """M = 0 (every node unlabelled, so every link is an inter link and no
    observable is formed), omega NULL (zero), missing-link columns NULL."""
    g = S.sbm_graph([40, 30], 0.5, inter_degree=3.0, seed=5)
    g.labels[:] = -1
    nm, ni, M = _static_calls(oracle_mod, g, 1.5, (0.6, 0.2), (-0.3, 0.1), None)
    assert (nm, M) == (0, 0) and ni > 0


def test_static_rhs_with_empty_split(oracle_mod):
    """Complete communities and no links between them: both halves of S are
    empty (NULL column arrays) and the RHS is the dense term alone."""
    g = S.sbm_graph([25, 40, 7], 1.0, p_out=0.0, seed=9)
    omega = np.random.default_rng(4).normal(size=g.n)
    nm, ni, M = _static_calls(oracle_mod, g, 3.0, (1.0, 0.5), (0.0, 0.25), omega)
    assert (nm, ni, M) == (0, 0, 3)


def test_static_rhs_at_capacity_edge(oracle_mod):
    """p * (n + M) equal to the capacity exactly: p = 4, 8192 communities of 9
    nodes, n + M = 81920."""
    g = S.sbm_graph([9] * 8192, 0.9, inter_degree=2.0, seed=12)
    assert 4 * (g.n + 8192) == CAPACITY
    omega = np.random.default_rng(5).normal(size=g.n)
    _static_calls(oracle_mod, g, 2.0, (0.5, 0.3, -0.2, 0.1), (0.2, -0.1, 0.05, 0.3), omega,
                  check_plan=False)


@pytest.mark.parametrize("n,M,p", [(CAPACITY, 1, 1),                 # one entry over, p = 1
                                   (CAPACITY // 4 - 7, 8, 4),         # one entry over, p = 4
                                   (400000, 1, 1),
                                   (1 << 62, 0, 4),                   # p * n wraps in 64 bits
                                   (16, 1 << 62, 4)])
def test_static_rhs_rejects_sizes_beyond_capacity(n, M, p):
    import paper_2203_16657_gb300 as cia
    from paper_2203_16657_gb300 import _abi

    lib = cia.load()
    cp = _coupling(_abi, 1.0, (1.0,) * p, (0.0,) * p)
    dummy = ctypes.c_void_p(16)        # never dereferenced: the size check comes first
    st = lib.cia_rhs_kuramoto_static(n, M, dummy, dummy, None, dummy, None, dummy, None,
                                     ctypes.byref(cp), dummy, None)
    assert _abi.STATUS[st] == "CIA_ERR_INVALID_ARG"
    assert "capacity" in lib.cia_last_error().decode()
