"""The C ABI without a GPU: the library builds, loads, exports every entry
point that include/*.h declares, and rejects bad input on the host before
any CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_16657_gb300 import build
    build.build()
    import paper_2203_16657_gb300 as P
    return P


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cia_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "cia_plan_create" in names and "cia_integrate" in names
    so = ctypes.CDLL(lib._abi.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(lib._abi.SIGNATURES), set(names) - set(lib._abi.SIGNATURES)


def test_status_strings(lib):
    for code, name in lib._abi.STATUS.items():
        assert lib.status_string(code) == name


def _plan(lib, rowptr, col, labels, omega=None, **kw):
    return lib.Plan(np.array(rowptr), np.array(col), np.array(labels), omega, **kw)


@pytest.mark.parametrize("rowptr,col,why", [
    ([0, 1, 1], [1], "asymmetric"),
    ([0, 0, 1], [0], "asymmetric: link 1->0"),                 # a link below the diagonal alone
    ([0, 2, 3, 4], [1, 2, 0, 1], "asymmetric: link 0->2"),     # 2 lists 1, not 0
    ([0, 1, 2], [0, 0], "self loop"),
    ([0, 2, 3, 4], [2, 1, 0, 0], "not strictly increasing"),
    ([0, 1, 2], [5, 0], "out of range"),
    ([0, 2, 2], [1, 1], "not strictly increasing"),
])
def test_invalid_graphs_rejected(lib, rowptr, col, why):
    n = len(rowptr) - 1
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, rowptr, col, [0] * n)
    assert e.value.status_name == "CIA_ERR_INVALID_GRAPH"
    assert why in str(e.value)


def test_non_finite_inputs_rejected(lib):
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], np.array([0.0, np.nan]))
    assert e.value.status_name == "CIA_ERR_NUMERIC"
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], K=float("inf"))
    assert e.value.status_name == "CIA_ERR_NUMERIC"


def test_bad_options_rejected(lib):
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], tile_nodes=100)
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, -3])
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"


def test_batch_validation_on_host(lib):
    good = (np.array([0, 1, 2]), np.array([1, 0]))
    bad = (np.array([0, 1, 1]), np.array([1]))          # asymmetric
    with pytest.raises(lib.CiaError) as e:
        lib.Plan.batch([good, bad], [[0, 0], [0, 0]])
    assert e.value.status_name == "CIA_ERR_INVALID_GRAPH"
    with pytest.raises(lib.CiaError) as e:
        lib.Plan.batch([], [])
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"
    with pytest.raises(lib.CiaError) as e:
        lib.Plan.batch([good], [[0, 0]], model="kuramoto_ho")
    assert e.value.status_name == "CIA_ERR_UNSUPPORTED"
    with pytest.raises(lib.CiaError) as e:
        lib.Plan.batch([good, (np.array([0, 1, 2]), np.array([5, 0]))], [[0, 0], [0, 0]])
    assert e.value.status_name == "CIA_ERR_INVALID_GRAPH"


def test_cucker_smale_options_on_host(lib):
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], model="cucker_smale", precision="fp64")
    assert e.value.status_name == "CIA_ERR_UNSUPPORTED"
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], np.zeros(2), model="cucker_smale", precision="fp32")
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], model="cucker_smale", precision="fp32", sigma=0.0)
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], model="cucker_smale", precision="fp32", tile_nodes=256)
    assert e.value.status_name == "CIA_ERR_INVALID_ARG"
    with pytest.raises(lib.CiaError) as e:
        _plan(lib, [0, 1, 2], [1, 0], [0, 0], model="cucker_smale", precision="fp32",
              beta=float("nan"))
    assert e.value.status_name == "CIA_ERR_NUMERIC"


def test_basis_rejects_bad_parameters_on_host(lib):
    with pytest.raises(lib.CiaError) as e:
        lib.Basis(np.full(lib.Basis.PARAMS, np.inf, dtype=np.float32))
    assert e.value.status_name == "CIA_ERR_NUMERIC"
    with pytest.raises(ValueError):
        lib.Basis(np.zeros(10, dtype=np.float32))
