"""Host-side checks of the streamed ensemble plan (cia_plan_batch_begin/add):
option checks, per-instance validation with the instance named in the
message, and the state machine.  No device work happens before finish."""
import ctypes

import numpy as np
import pytest

import synthetic as S


@pytest.fixture(scope="module")
def lib():
    import paper_2203_16657_gb300 as cia
    return cia.load()


def _coupling(abi):
    cp = abi.Coupling()
    cp.model = abi.MODEL["kuramoto"]
    cp.p = 1
    cp.d_sin[0] = 1.0
    cp.K = 4.0
    return cp


def _begin(lib, abi, build_direct=0):
    opt = abi.Options(abi.PRECISION["fp32"], build_direct, 0, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    st = lib.cia_plan_batch_begin(ctypes.byref(_coupling(abi)), ctypes.byref(opt), ctypes.byref(h))
    return st, h


def _add(lib, abi, h, g, labels=None):
    lb = np.ascontiguousarray(g.labels if labels is None else labels, dtype=np.int32)
    gr = abi.Graph(g.n, g.rowptr.ctypes.data, g.col.ctypes.data)
    return lib.cia_plan_batch_add(h, ctypes.byref(gr), lb.ctypes.data, None)


def test_streamed_plan_rejects_the_direct_method(lib):
    from paper_2203_16657_gb300 import _abi
    st, h = _begin(lib, _abi, build_direct=1)
    assert _abi.STATUS[st] == "CIA_ERR_UNSUPPORTED" and not h.value
    assert "direct" in lib.cia_last_error().decode()


def test_streamed_plan_validates_each_instance(lib):
    from paper_2203_16657_gb300 import _abi
    st, h = _begin(lib, _abi)
    assert _abi.STATUS[st] == "CIA_OK"
    try:
        good = S.sbm_graph([20, 15], 0.8, inter_degree=2.0, seed=3)
        assert _abi.STATUS[_add(lib, _abi, h, good)] == "CIA_OK"
        # instance 1: a link without its reverse
        bad = S.sbm_graph([12, 9], 0.9, inter_degree=2.0, seed=4)
        row = int(np.argmax(np.diff(bad.rowptr) > 0))
        col = bad.col.copy()
        j = int(col[bad.rowptr[row]])
        # drop the reverse link j -> row by moving it to another column of row j
        seg = col[bad.rowptr[j]:bad.rowptr[j + 1]]
        k = int(np.searchsorted(seg, row))
        free = sorted(set(range(bad.n)) - set(seg.tolist()) - {j, row})
        seg[k] = free[0]
        col[bad.rowptr[j]:bad.rowptr[j + 1]] = np.sort(seg)
        bad = S.Graph(bad.n, bad.rowptr, col, bad.labels, bad.sizes)
        st = _add(lib, _abi, h, bad)
        assert _abi.STATUS[st] == "CIA_ERR_INVALID_GRAPH"
        msg = lib.cia_last_error().decode()
        assert msg.startswith("instance 1:") and "reverse" in msg
        # labels below -1
        st = _add(lib, _abi, h, good, labels=np.full(good.n, -2))
        assert _abi.STATUS[st] == "CIA_ERR_INVALID_ARG"
        # the failed adds left the plan as it was: one more good instance is fine
        assert _abi.STATUS[_add(lib, _abi, h, good)] == "CIA_OK"
    finally:
        lib.cia_plan_destroy(h)


def test_streamed_plan_state_machine(lib):
    from paper_2203_16657_gb300 import _abi
    st, h = _begin(lib, _abi)
    try:
        assert _abi.STATUS[lib.cia_plan_batch_finish(h)] == "CIA_ERR_INVALID_ARG"   # no instance
        assert "no instance" in lib.cia_last_error().decode()
    finally:
        lib.cia_plan_destroy(h)
    g = S.sbm_graph([6, 4], 0.8, inter_degree=1.0, seed=5)
    assert _abi.STATUS[_add(lib, _abi, None, g)] == "CIA_ERR_INVALID_ARG"
