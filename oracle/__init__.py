"""FP64 CPU oracle for the community integration algorithm (CIA).

TEST INFRASTRUCTURE ONLY: the correctness reference of the CUDA library.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the device path: its own P1 split, its
own right-hand sides (``cia_oracle.c``), its own integrators.

Contents, each following the paper (arXiv 2203.16657):

* ``split``: step P1 of Sec. 3.1 -- the permutation kappa that makes
  communities contiguous, the community sizes lambda_c, and the sparse
  remainder S of B = P A P^T = D + S (entries +1 / -1, App. A.1).
* ``kuramoto_direct`` / ``kuramoto_cia``: the plain definition of the RHS
  (eq. GeneralNetworkSystem) and the CIA steps E1/E2 (Sec. 3.2, App. A.4).
* ``ho_triadic_direct`` / ``ho_triadic_cia``: the triadic term of the
  higher-order Kuramoto model (App. A.7) on complete community hyperedges.
* ``cs_direct`` / ``cs_cia``: Cucker--Smale (App. A.6) with a separable basis.
* ``poly_direct`` / ``poly_cia``: polynomial difference coupling with a
  potential (App. A.3 and the Desai--Zwanzig model, App. A.5), the CIA by
  polynomial moments.
* ``fourier_*``: the Fourier basis of a radial pair weight (App. A.6).
* ``rk4_step`` / ``euler_step``: classical RK4 (textbook; the paper allows any
  Runge--Kutta method, Sec. 3) and explicit Euler (Sec. 4).
* ``order_parameter``: r = |sum_l e^{i theta_l}| / N (eq. KuramotoFirstOP).
* ``mlp_*``: the FP64 forward/backward of the learned separable basis.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cia_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcia_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, FP64, IEEE semantics, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        # CIA_ORACLE_LIB: a prebuilt copy of the same source (the sanitizer test builds one)
        path = os.environ.get("CIA_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        lib.ora_num_threads.restype = ctypes.c_int
        lib.ora_set_num_threads.argtypes = [ctypes.c_int]
        lib.ora_kuramoto_direct.argtypes = [I64, P, P, P, P, D, ctypes.c_int, P, P, P]
        lib.ora_kuramoto_cia.argtypes = [I64, I64, P, P, P, P, P, P, D, ctypes.c_int, P, P,
                                         P, P, P]
        lib.ora_ho_triadic_direct.argtypes = [I64, I64, P, P, D, I64, P, P]
        lib.ora_ho_triadic_cia.argtypes = [I64, I64, P, P, D, P, P, P, P, P]
        lib.ora_cs_direct.argtypes = [I64, P, P, P, D, D, D, P]
        lib.ora_cs_cia.argtypes = [I64, I64, P, P, P, P, P, P, I64, D, D, D, P, P, P]
        lib.ora_poly_direct.argtypes = [I64, P, P, P, D, ctypes.c_int, P, ctypes.c_int, P, P]
        lib.ora_poly_cia.argtypes = [I64, I64, P, P, P, P, P, D, ctypes.c_int, P, ctypes.c_int, P,
                                     P, P]
        lib.ora_polyg_direct.argtypes = [I64, P, P, P, D, ctypes.c_int, P, ctypes.c_int, P, P]
        lib.ora_polyg_cia.argtypes = [I64, I64, P, P, P, P, P, D, ctypes.c_int, P, ctypes.c_int, P,
                                      P, P]
        lib.ora_polyw_direct.argtypes = [I64, P, P, P, D, ctypes.c_int, P, ctypes.c_int, P, P, P, P]
        lib.ora_polyw_cia.argtypes = [I64, I64, P, P, P, P, P, D, ctypes.c_int, P, ctypes.c_int, P,
                                      P, P, P, P]
        lib.ora_fourierg_direct.argtypes = [I64, P, P, P, D, ctypes.c_int, D, P, P, P, P, ctypes.c_int, P, P]
        lib.ora_fourierg_cia.argtypes = [I64, I64, P, P, P, P, P, D, ctypes.c_int, D, P, P, P, P,
                                         ctypes.c_int, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return _load().ora_num_threads()


def set_num_threads(t: int) -> None:
    _load().ora_set_num_threads(int(t))


# --------------------------------------------------------------------------
# Step P1: permutation and the split B = D + S (Sec. 3.1, App. A.1)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Split:
    """Result of step P1.

    perm[m]  = original id of permuted node m (kappa(m) in Sec. 3.1)
    iperm[i] = permuted id of original node i
    off      = int64[M+1]; community c is [off[c], off[c+1]); nodes from off[M]
               to n belong to no community.
    s_rowptr/s_col/s_val: S in CSR (permuted ids), values +1 (inter-community
               link) and -1 (missing link inside a block, diagonal included).
    """

    n: int
    M: int
    perm: np.ndarray
    iperm: np.ndarray
    off: np.ndarray
    s_rowptr: np.ndarray
    s_col: np.ndarray
    s_val: np.ndarray

    def community_of(self) -> np.ndarray:
        """Community id of each permuted node (-1 for none)."""
        out = np.full(self.n, -1, dtype=np.int64)
        for c in range(self.M):
            out[self.off[c]:self.off[c + 1]] = c
        return out


def split(rowptr: np.ndarray, col: np.ndarray, labels: np.ndarray) -> Split:
    """Step P1 for given community labels (label -1 = no community).

    kappa orders nodes by (label, original id), unlabelled nodes last, so each
    community occupies consecutive permuted ids.  Row m of B = P A P^T holds
    the permuted ids of the neighbours of kappa(m).  D has a block of ones
    over each community (diagonal included), so S = B - D has +1 where B links
    outside the block and -1 where the block has no link in B.
    """
    n = len(labels)
    labels = np.asarray(labels, dtype=np.int64)
    M = int(labels.max()) + 1 if n and labels.max() >= 0 else 0
    key = np.where(labels < 0, M, labels)
    perm = np.lexsort((np.arange(n), key)).astype(np.int64)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    sizes = np.bincount(key, minlength=M + 1)[:M]
    off = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])

    comm_of_perm = np.full(n, -1, dtype=np.int64)
    for c in range(M):
        comm_of_perm[off[c]:off[c + 1]] = c

    rows_cols, rows_vals = [], []
    counts = np.zeros(n, dtype=np.int64)
    for m in range(n):
        i = perm[m]
        brow = np.sort(iperm[col[rowptr[i]:rowptr[i + 1]]])
        c = comm_of_perm[m]
        if c < 0:
            cols = brow
            vals = np.ones(len(brow), dtype=np.int8)
        else:
            lo, hi = off[c], off[c + 1]
            outside = brow[(brow < lo) | (brow >= hi)]
            inside = brow[(brow >= lo) & (brow < hi)]
            block = np.arange(lo, hi, dtype=np.int64)
            missing = np.setdiff1d(block, inside, assume_unique=True)
            cols = np.concatenate([outside, missing])
            vals = np.concatenate([np.ones(len(outside), np.int8),
                                   -np.ones(len(missing), np.int8)])
            order = np.argsort(cols, kind="stable")
            cols, vals = cols[order], vals[order]
        rows_cols.append(cols)
        rows_vals.append(vals)
        counts[m] = len(cols)
    s_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=s_rowptr[1:])
    s_col = (np.concatenate(rows_cols) if n else np.zeros(0)).astype(np.int32)
    s_val = (np.concatenate(rows_vals) if n else np.zeros(0)).astype(np.int8)
    return Split(n=n, M=M, perm=perm, iperm=iperm, off=off,
                 s_rowptr=s_rowptr, s_col=s_col, s_val=s_val)


def rebuild_b(sp: Split) -> tuple[np.ndarray, np.ndarray]:
    """B = D + S as a CSR of permuted ids (checks the split is lossless)."""
    rows = []
    comm = sp.community_of()
    for m in range(sp.n):
        s = sp.s_col[sp.s_rowptr[m]:sp.s_rowptr[m + 1]].astype(np.int64)
        v = sp.s_val[sp.s_rowptr[m]:sp.s_rowptr[m + 1]]
        entries = dict()
        c = comm[m]
        if c >= 0:
            for ell in range(sp.off[c], sp.off[c + 1]):
                entries[int(ell)] = 1
        for ell, val in zip(s.tolist(), v.tolist()):
            entries[ell] = entries.get(ell, 0) + val
        rows.append(sorted(k for k, val in entries.items() if val != 0))
        assert all(val in (0, 1) for val in entries.values())
    rowptr = np.zeros(sp.n + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=rowptr[1:])
    col = np.array([x for r in rows for x in r], dtype=np.int64)
    return rowptr, col


# --------------------------------------------------------------------------
# Right-hand sides (thin marshalling around cia_oracle.c)
# --------------------------------------------------------------------------

def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def kuramoto_direct(rowptr, col, theta, omega, K, d_sin=(1.0,), d_cos=(0.0,)) -> np.ndarray:
    """omega_m + (K/N) sum_l a_ml h(theta_l - theta_m), original node order."""
    lib = _load()
    theta, omega = _f64(theta), _f64(omega)
    rowptr, col = _i64(rowptr), _i32(col)
    ds, dc = _f64(d_sin), _f64(d_cos)
    out = np.empty_like(theta)
    lib.ora_kuramoto_direct(len(theta), _p(rowptr), _p(col), _p(theta), _p(omega), float(K),
                            len(ds), _p(ds), _p(dc), _p(out))
    return out


def kuramoto_cia(sp: Split, phi, omega_perm, K, d_sin=(1.0,), d_cos=(0.0,)) -> np.ndarray:
    """CIA RHS on the permuted state phi (steps E1 and E2)."""
    lib = _load()
    phi, omega_perm = _f64(phi), _f64(omega_perm)
    ds, dc = _f64(d_sin), _f64(d_cos)
    p = len(ds)
    qc = np.zeros(max(1, sp.M * p))
    qs = np.zeros(max(1, sp.M * p))
    out = np.empty_like(phi)
    lib.ora_kuramoto_cia(sp.n, sp.M, _p(sp.off), _p(sp.s_rowptr), _p(sp.s_col), _p(sp.s_val),
                         _p(phi), _p(omega_perm), float(K), p, _p(ds), _p(dc),
                         _p(qc), _p(qs), _p(out))
    return out


def ho_triadic_direct(sp: Split, phi, K2, nodes) -> np.ndarray:
    """Brute-force triadic term for the given permuted node ids."""
    lib = _load()
    phi = _f64(phi)
    nodes = _i64(nodes)
    out = np.zeros(len(nodes))
    lib.ora_ho_triadic_direct(sp.n, sp.M, _p(sp.off), _p(phi), float(K2), len(nodes),
                              _p(nodes), _p(out))
    return out


def ho_triadic_cia(sp: Split, phi, K2) -> np.ndarray:
    """Triadic term of every permuted node from the moments Z1, Z2."""
    lib = _load()
    phi = _f64(phi)
    z = [np.zeros(max(1, sp.M)) for _ in range(4)]
    out = np.zeros(sp.n)
    lib.ora_ho_triadic_cia(sp.n, sp.M, _p(sp.off), _p(phi), float(K2),
                           *[_p(a) for a in z], _p(out))
    return out


def cs_direct(rowptr, col, x, K=1.0, sigma=1.0, beta=0.4) -> np.ndarray:
    """Cucker--Smale RHS, x = n x 4 (s_x, s_y, v_x, v_y), original order."""
    lib = _load()
    x = _f64(x).reshape(-1, 4)
    rowptr, col = _i64(rowptr), _i32(col)
    out = np.empty_like(x)
    lib.ora_cs_direct(len(x), _p(rowptr), _p(col), _p(x), float(K), float(sigma),
                      float(beta), _p(out))
    return out


def cs_cia(sp: Split, x_perm, feat_perm, K=1.0, sigma=1.0, beta=0.4) -> np.ndarray:
    """Cucker--Smale CIA RHS with a separable basis (rows of feat_perm)."""
    lib = _load()
    x = _f64(x_perm).reshape(-1, 4)
    feat = _f64(feat_perm)
    R = feat.shape[1]
    U = np.zeros(max(1, sp.M * R))
    H = np.zeros(max(1, sp.M * R * 2))
    out = np.empty_like(x)
    lib.ora_cs_cia(sp.n, sp.M, _p(sp.off), _p(sp.s_rowptr), _p(sp.s_col), _p(sp.s_val),
                   _p(x), _p(feat), R, float(K), float(sigma), float(beta),
                   _p(U), _p(H), _p(out))
    return out


def poly_direct(rowptr, col, x, K, c, dv) -> np.ndarray:
    """x' = -V'(x_m) + (K/N) sum_l a_ml h(x_l - x_m) with h = sum_a c[a] x^a and
    V' = sum_j dv[j] x^j (polynomial difference coupling, Desai--Zwanzig)."""
    lib = _load()
    x = _f64(x)
    c, dv = _f64(c), _f64(dv)
    out = np.empty_like(x)
    lib.ora_poly_direct(len(x), _p(_i64(rowptr)), _p(_i32(col)), _p(x), float(K), len(c) - 1, _p(c),
                        len(dv) - 1, _p(dv), _p(out))
    return out


def poly_cia(sp: Split, x_perm, K, c, dv) -> np.ndarray:
    """The same right-hand side by the CIA with polynomial moments (permuted order)."""
    lib = _load()
    x = _f64(x_perm)
    c, dv = _f64(c), _f64(dv)
    w = np.zeros(max(1, sp.M * len(c)))
    out = np.empty_like(x)
    lib.ora_poly_cia(sp.n, sp.M, _p(sp.off), _p(sp.s_rowptr), _p(sp.s_col), _p(sp.s_val), _p(x),
                     float(K), len(c) - 1, _p(c), len(dv) - 1, _p(dv), _p(w), _p(out))
    return out


def _square(G) -> np.ndarray:
    G = _f64(G)
    if G.ndim != 2 or G.shape[0] != G.shape[1] or G.shape[0] < 1:
        raise ValueError("G must be a square (p+1) x (p+1) array")
    return np.ascontiguousarray(G)


def polyg_direct(rowptr, col, x, K, G, dv) -> np.ndarray:
    """x' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m) with the general polynomial
    g(u, y) = sum_{a,b} G[a, b] u^a y^b (eq. PolyApprox)."""
    lib = _load()
    x = _f64(x)
    G, dv = _square(G), _f64(dv)
    out = np.empty_like(x)
    lib.ora_polyg_direct(len(x), _p(_i64(rowptr)), _p(_i32(col)), _p(x), float(K), G.shape[0] - 1,
                         _p(G), len(dv) - 1, _p(dv), _p(out))
    return out


def polyg_cia(sp: Split, x_perm, K, G, dv) -> np.ndarray:
    """The same right-hand side by the CIA: moments w_a (eq. PolyMoments), the
    dense term sum_{a,b} G[a, b] w_a x_m^b (eq. PolyRHS), the sparse sum over S."""
    lib = _load()
    x = _f64(x_perm)
    G, dv = _square(G), _f64(dv)
    w = np.zeros(max(1, sp.M * G.shape[0]))
    out = np.empty_like(x)
    lib.ora_polyg_cia(sp.n, sp.M, _p(sp.off), _p(sp.s_rowptr), _p(sp.s_col), _p(sp.s_val), _p(x),
                      float(K), G.shape[0] - 1, _p(G), len(dv) - 1, _p(dv), _p(w), _p(out))
    return out


def polyw_direct(rowptr, col, x, K, G, dv, alpha, beta) -> np.ndarray:
    """Rank-one weighted links (eq. rank1system on a graph): x' = -V'(x_m) +
    (K/N) sum_l a_ml alpha_m beta_l g(x_l, x_m), g as in polyg_direct."""
    lib = _load()
    x = _f64(x)
    G, dv = _square(G), _f64(dv)
    alpha, beta = _f64(alpha), _f64(beta)
    if len(alpha) != len(x) or len(beta) != len(x):
        raise ValueError("alpha and beta need n entries")
    out = np.empty_like(x)
    lib.ora_polyw_direct(len(x), _p(_i64(rowptr)), _p(_i32(col)), _p(x), float(K), G.shape[0] - 1,
                         _p(G), len(dv) - 1, _p(dv), _p(alpha), _p(beta), _p(out))
    return out


def polyw_cia(sp: Split, x_perm, K, G, dv, alpha_perm, beta_perm) -> np.ndarray:
    """The same by the CIA: weighted moments r_a = (1/N) sum_{l in c} beta_l x_l^a
    (eq. rank1precompute), dense term alpha_m sum G[a, b] r_a x_m^b (eq. rank1fast),
    the sparse sum over S with the link weights (permuted order)."""
    lib = _load()
    x = _f64(x_perm)
    G, dv = _square(G), _f64(dv)
    alpha, beta = _f64(alpha_perm), _f64(beta_perm)
    w = np.zeros(max(1, sp.M * G.shape[0]))
    out = np.empty_like(x)
    lib.ora_polyw_cia(sp.n, sp.M, _p(sp.off), _p(sp.s_rowptr), _p(sp.s_col), _p(sp.s_val), _p(x),
                      float(K), G.shape[0] - 1, _p(G), len(dv) - 1, _p(dv), _p(alpha), _p(beta), _p(w),
                      _p(out))
    return out


def _fourier_blocks(C):
    C = [_square(c) for c in C]
    if len(C) != 4 or len({c.shape for c in C}) != 1:
        raise ValueError("C must be four square (p+1) x (p+1) arrays C11, C12, C21, C22")
    return C


def fourierg_direct(rowptr, col, x, K, L, C, dv) -> np.ndarray:
    """x' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m) with the real 2-D Fourier
    coupling of eq. FourierRealExpansion: C = (C11, C12, C21, C22), each
    (p+1) x (p+1), frequencies pi a / L."""
    lib = _load()
    x = _f64(x)
    C11, C12, C21, C22 = _fourier_blocks(C)
    dv = _f64(dv)
    out = np.empty_like(x)
    lib.ora_fourierg_direct(len(x), _p(_i64(rowptr)), _p(_i32(col)), _p(x), float(K), C11.shape[0] - 1,
                            float(L), _p(C11), _p(C12), _p(C21), _p(C22), len(dv) - 1, _p(dv), _p(out))
    return out


def fourierg_cia(sp: Split, x_perm, K, L, C, dv) -> np.ndarray:
    """The same by the CIA: the real generalised order parameters r^cos_a, r^sin_a
    per community (eq. RealOP), the dense term from them, the sparse sum over S."""
    lib = _load()
    x = _f64(x_perm)
    C11, C12, C21, C22 = _fourier_blocks(C)
    dv = _f64(dv)
    w = np.zeros(max(1, 2 * sp.M * C11.shape[0]))
    out = np.empty_like(x)
    lib.ora_fourierg_cia(sp.n, sp.M, _p(sp.off), _p(sp.s_rowptr), _p(sp.s_col), _p(sp.s_val), _p(x),
                         float(K), C11.shape[0] - 1, float(L), _p(C11), _p(C12), _p(C21), _p(C22),
                         len(dv) - 1, _p(dv), _p(w), _p(out))
    return out


# --------------------------------------------------------------------------
# Community detection objective (Sec. "Community Detection (P1)")
# --------------------------------------------------------------------------

def potts_hamiltonian(rowptr, col, labels, gamma, mu=0.0) -> float:
    """H = -sum_{m != l} (a_ml - gamma p) delta(c_m, c_l) + mu M with the
    Erdos-Renyi null model p = nnz(A) / (N (N - 1)); labels >= 0 name the
    communities (every label is a community, also of size one)."""
    rowptr, col = _i64(rowptr), _i32(col)
    labels = np.asarray(labels, dtype=np.int64)
    n = len(labels)
    p = len(col) / (n * (n - 1)) if n > 1 else 0.0
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    e_in = int(np.sum(labels[rows] == labels[col]))
    _, sizes = np.unique(labels, return_counts=True)
    pairs = float(np.sum(sizes.astype(np.float64) * (sizes - 1)))
    return -e_in + gamma * p * pairs + mu * len(sizes)


def best_single_move_gain(rowptr, col, labels, gamma, mu=0.0) -> float:
    """Largest decrease of H over all moves of one node to the community of a
    neighbour or to a new community of its own, each H evaluated in full by
    potts_hamiltonian (brute force, small graphs)."""
    labels = np.asarray(labels, dtype=np.int64).copy()
    h0 = potts_hamiltonian(rowptr, col, labels, gamma, mu)
    fresh = labels.max() + 1
    best = 0.0
    for m in range(len(labels)):
        own = labels[m]
        cands = set(int(labels[l]) for l in col[rowptr[m]:rowptr[m + 1]]) | {int(fresh)}
        cands.discard(int(own))
        for c in cands:
            labels[m] = c
            best = max(best, h0 - potts_hamiltonian(rowptr, col, labels, gamma, mu))
        labels[m] = own
    return best


# --------------------------------------------------------------------------
# Time stepping and observables
# --------------------------------------------------------------------------

def rk4_step(rhs, x: np.ndarray, dt: float) -> np.ndarray:
    """One classical Runge--Kutta step (nodes c = 0, 1/2, 1/2, 1; weights
    1/6, 1/3, 1/3, 1/6) of an autonomous system x' = rhs(x)."""
    k1 = rhs(x)
    k2 = rhs(x + 0.5 * dt * k1)
    k3 = rhs(x + 0.5 * dt * k2)
    k4 = rhs(x + dt * k3)
    return x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def euler_step(rhs, x: np.ndarray, dt: float) -> np.ndarray:
    """One explicit Euler step (the integrator of the paper's timings, Sec. 4)."""
    return x + dt * rhs(x)


def wrap_phase(theta: np.ndarray) -> np.ndarray:
    """Representative of theta in R / 2 pi Z closest to zero (IEEE remainder)."""
    return np.remainder(theta + np.pi, 2.0 * np.pi) - np.pi


def order_parameter(theta: np.ndarray) -> float:
    """|r_1| with r_1 = (1/N) sum_l e^{i theta_l} (eq. KuramotoFirstOP)."""
    return float(np.abs(np.exp(1j * np.asarray(theta, dtype=np.float64)).mean()))


def integrate(rhs, x0: np.ndarray, dt: float, steps: int, *, method: str = "rk4",
              wrap: bool = False, observe=None):
    """Integrate x' = rhs(x) for `steps` steps; optionally wrap phases after
    each step and record observe(x) after each step."""
    step = rk4_step if method == "rk4" else euler_step
    x = np.array(x0, dtype=np.float64)
    obs = []
    for _ in range(steps):
        x = step(rhs, x, dt)
        if wrap:
            x = wrap_phase(x)
        if observe is not None:
            obs.append(observe(x))
    return x, obs


def angle_diff(a, b) -> np.ndarray:
    """Signed difference a - b taken on the circle, in [-pi, pi)."""
    return wrap_phase(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))


from .mlp import (mlp_forward, mlp_backward, pair_loss, pair_loss_grad,  # noqa: E402
                  silu, silu_grad, cs_kernel_weight, bf16_round, unpack_params, pack_params)
from .fourier import fourier_coefficients, fourier_basis, fourier_features, radial  # noqa: E402

__all__ = [
    "build", "num_threads", "set_num_threads", "Split", "split", "rebuild_b",
    "kuramoto_direct", "kuramoto_cia", "ho_triadic_direct", "ho_triadic_cia",
    "cs_direct", "cs_cia", "poly_direct", "poly_cia", "rk4_step", "euler_step", "wrap_phase", "order_parameter",
    "integrate", "angle_diff", "mlp_forward", "mlp_backward", "pair_loss",
    "pair_loss_grad", "silu", "silu_grad", "cs_kernel_weight", "bf16_round",
    "unpack_params", "pack_params", "fourier_coefficients", "fourier_basis", "fourier_features",
    "radial",
]
