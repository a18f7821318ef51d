"""Shared helpers for the parity tests (no method arithmetic here)."""
from __future__ import annotations

import numpy as np


def coupling_rel_err(got, ref, omega) -> float:
    """||(got - omega) - (ref - omega)||_inf / ||ref - omega||_inf.

    The error is measured on the coupling part of the RHS: omega can be orders
    of magnitude larger (Lorentzian frequencies) and would hide it."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    denom = np.abs(ref - omega).max()
    return float(np.abs((got - omega) - (ref - omega)).max() / max(denom, 1e-300))


def split_halves(sp):
    """The oracle's signed S as the two CSRs the library reports: -1 entries
    without the diagonal (missing) and +1 entries (inter), permuted ids."""
    n = sp.n
    miss_rp = np.zeros(n + 1, dtype=np.int64)
    inter_rp = np.zeros(n + 1, dtype=np.int64)
    miss, inter = [], []
    for m in range(n):
        cols = sp.s_col[sp.s_rowptr[m]:sp.s_rowptr[m + 1]]
        vals = sp.s_val[sp.s_rowptr[m]:sp.s_rowptr[m + 1]]
        mm = cols[(vals == -1) & (cols != m)]
        ii = cols[vals == 1]
        miss.append(mm)
        inter.append(ii)
        miss_rp[m + 1] = miss_rp[m] + len(mm)
        inter_rp[m + 1] = inter_rp[m] + len(ii)
    cat = lambda xs: np.concatenate(xs).astype(np.int32) if xs else np.zeros(0, np.int32)
    return miss_rp, cat(miss), inter_rp, cat(inter)


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
