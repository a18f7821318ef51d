"""The allocation-free right-hand side (cia_rhs_kuramoto_static) against cia_rhs.

Some callers cannot let the library allocate device memory (their host
application owns the device-memory pool, or their loop may not call cudaMalloc,
which can synchronise the device).  cia_rhs_kuramoto_static serves them from a
fixed scratch array inside the library.  This test calls it through the C ABI
twice in a row on different states, with the split of S taken from a plan, and
checks each result against cia_rhs on the same state within the FP64 parity
tolerance of the other tests.  The file is named so that pytest collects it
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


def _coupling(abi, K, d_sin, d_cos):
    cp = abi.Coupling()
    cp.model = abi.MODEL["kuramoto"]
    cp.p = len(d_sin)
    for k in range(len(d_sin)):
        cp.d_sin[k] = float(d_sin[k])
        cp.d_cos[k] = float(d_cos[k])
    cp.K = float(K)
    return cp


@pytest.mark.parametrize("d_sin,d_cos", [((1.0,), (0.0,)), ((0.7, -0.3, 0.2), (0.1, 0.4, -0.5))])
def test_static_rhs_matches_cia_rhs_twice(d_sin, d_cos):
    import torch
    import paper_2203_16657_gb300 as cia
    from paper_2203_16657_gb300 import _abi

    g = S.sbm_graph([120, 75, 200, 33], 0.85, inter_degree=5.0, seed=31, n_free=17)
    rng = np.random.default_rng(7)
    omega = rng.normal(size=g.n)
    K = 2.5
    plan = cia.Plan(g.rowptr, g.col, g.labels, omega, K=K, d_sin=d_sin, d_cos=d_cos)
    perm, off = plan.permutation()
    mrp, mcol, irp, icol = plan.split()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_off, d_mrp, d_mcol, d_irp, d_icol = dev(off), dev(mrp), dev(mcol), dev(irp), dev(icol)
    d_om = dev(omega[perm])
    cp = _coupling(_abi, K, d_sin, d_cos)
    lib = cia.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t.numel() else None

    for call in range(2):
        x = rng.uniform(-np.pi, np.pi, g.n)
        want = plan.rhs(dev(x)).cpu().numpy()                 # existing entry point
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        st = lib.cia_rhs_kuramoto_static(g.n, len(off) - 1, ptr(d_off), ptr(d_mrp), ptr(d_mcol),
                                         ptr(d_irp), ptr(d_icol), ptr(dev(x[perm])), ptr(d_om),
                                         ctypes.byref(cp), ptr(out), stream)
        _abi.check(st)
        torch.cuda.synchronize()
        got = np.empty(g.n)
        got[perm] = out.cpu().numpy()
        assert coupling_rel_err(got, want, omega) < FP64_TOL, call


def test_static_rhs_rejects_sizes_beyond_capacity():
    import paper_2203_16657_gb300 as cia
    from paper_2203_16657_gb300 import _abi

    lib = cia.load()
    cp = _coupling(_abi, 1.0, (1.0,), (0.0,))
    dummy = ctypes.c_void_p(16)        # never dereferenced: the size check comes first
    st = lib.cia_rhs_kuramoto_static(400000, 1, dummy, dummy, None, dummy, None, dummy, None,
                                     ctypes.byref(cp), dummy, None)
    assert _abi.STATUS[st] == "CIA_ERR_INVALID_ARG"
    assert "capacity" in lib.cia_last_error().decode()
