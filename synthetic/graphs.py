"""Seeded synthetic networks with planted community structure.

This module only draws random graphs, labels and initial data.  It holds none
of the community integration arithmetic: the oracle and the CUDA path both
take their inputs from here and from nowhere else.

Randomness comes from numpy's Philox counter-based bit generator, seeded per
workload, so every graph is reproducible from its seed.

Graphs are undirected, unweighted and without self loops (the setting of the
general network model, Sec. 2, where A is symmetric with entries in {0, 1}).
They are returned as a symmetric CSR in *original* node numbering: node ids are
shuffled by a random permutation so that the community detection step's
permutation (Sec. 3.1, step P1) has real work to do.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Graph:
    """Symmetric CSR adjacency plus planted community labels.

    rowptr: int64[n+1]; col: int32[nnz] (sorted ascending within each row);
    labels: int32[n], community id in [0, M) or -1 for "no community".
    sizes: int64[M], the planted community sizes (lambda_1..lambda_M).
    """

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    labels: np.ndarray
    sizes: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        return int(len(self.sizes))


def rng_for(seed: int) -> np.random.Generator:
    """Philox-backed generator for one workload seed."""
    return np.random.Generator(np.random.Philox(int(seed)))


def lognormal_sizes(n: int, m: int, mean: float, sigma: float,
                    rng: np.random.Generator, min_size: int = 2) -> np.ndarray:
    """M community sizes summing to n, lognormal with the given mean.

    Draws lambda_c ~ LogNormal(ln(mean) - sigma^2/2, sigma), scales them to sum
    to n and rounds by largest remainder; every size is at least min_size.
    """
    mu = np.log(mean) - 0.5 * sigma * sigma
    raw = rng.lognormal(mu, sigma, size=m)
    scaled = raw * (n / raw.sum())
    sizes = np.maximum(np.floor(scaled).astype(np.int64), min_size)
    rem = n - int(sizes.sum())
    frac = scaled - np.floor(scaled)
    if rem > 0:
        order = np.argsort(-frac, kind="stable")
        sizes[order[:rem]] += 1
    while rem < 0:
        # take one node from each of the largest communities until balanced
        order = np.argsort(-sizes, kind="stable")
        for c in order:
            if rem == 0:
                break
            if sizes[c] > min_size:
                sizes[c] -= 1
                rem += 1
    assert int(sizes.sum()) == n
    return sizes


def equal_sizes(n: int, m: int) -> np.ndarray:
    """M sizes differing by at most one and summing to n."""
    base = np.full(m, n // m, dtype=np.int64)
    base[: n - int(base.sum())] += 1
    return base


def _intra_block(size: int, p_in: float, rng: np.random.Generator):
    """Directed (row, col) entries of one community block, local indices.

    Each unordered pair i<j is present with probability p_in; the block is
    mirrored so the result is symmetric, rows ascending, cols ascending.
    """
    if size < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    u = rng.random((size, size)) < p_in
    blk = np.triu(u, 1)
    blk |= blk.T
    r, c = np.nonzero(blk)
    return r.astype(np.int64), c.astype(np.int64)


def _inter_pairs_degree(comm: np.ndarray, mean_degree: float,
                        rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """Uniform random inter-community pairs, n*mean_degree/2 of them, unique.

    comm is the community id of each node in block order (-1 nodes count as
    their own singleton community, so any pair with them is inter-community).
    """
    n = len(comm)
    target = int(round(n * mean_degree / 2.0))
    if target == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    keys = np.zeros(0, np.int64)
    while len(keys) < target:
        need = int((target - len(keys)) * 1.25) + 64
        i = rng.integers(0, n, size=need, dtype=np.int64)
        j = rng.integers(0, n, size=need, dtype=np.int64)
        ok = (i != j) & ((comm[i] != comm[j]) | (comm[i] < 0))
        i, j = i[ok], j[ok]
        lo, hi = np.minimum(i, j), np.maximum(i, j)
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    if len(keys) > target:
        pick = np.sort(rng.choice(len(keys), size=target, replace=False))
        keys = keys[pick]
    return keys // n, keys % n


def _inter_pairs_bernoulli(comm: np.ndarray, p_out: float,
                           rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """Every inter-community pair i<j present with probability p_out (small n)."""
    n = len(comm)
    iu, ju = np.triu_indices(n, 1)
    inter = (comm[iu] != comm[ju]) | (comm[iu] < 0)
    iu, ju = iu[inter], ju[inter]
    keep = rng.random(len(iu)) < p_out
    return iu[keep].astype(np.int64), ju[keep].astype(np.int64)


def sbm_graph(sizes, p_in: float, *, seed: int, p_out: float | None = None,
              inter_degree: float | None = None, n_free: int = 0,
              shuffle: bool = True) -> Graph:
    """Planted-partition graph: communities of the given sizes plus sparse links.

    Inside community c each pair is linked with probability p_in; between
    communities either every pair is linked with probability p_out, or
    n*inter_degree/2 distinct uniformly random inter-community pairs are
    linked.  n_free extra nodes carry label -1 ("no community", allowed for
    numerical reasons in Sec. 3.1); their links are all inter-community.
    With shuffle=True the node ids are randomly permuted.
    """
    if (p_out is None) == (inter_degree is None):
        raise ValueError("give exactly one of p_out, inter_degree")
    rng = rng_for(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    m = len(sizes)
    n = int(sizes.sum()) + int(n_free)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    comm = np.full(n, -1, dtype=np.int64)
    for c in range(m):
        comm[offsets[c]:offsets[c + 1]] = c

    # new id of each block-order node
    perm = rng.permutation(n).astype(np.int64) if shuffle else np.arange(n, dtype=np.int64)

    keys = []
    for c in range(m):
        r, cc = _intra_block(int(sizes[c]), p_in, rng)
        base = offsets[c]
        keys.append(perm[r + base] * n + perm[cc + base])
    if p_out is not None:
        i, j = _inter_pairs_bernoulli(comm, p_out, rng)
    else:
        i, j = _inter_pairs_degree(comm, inter_degree, rng)
    pi, pj = perm[i], perm[j]
    keys.append(pi * n + pj)
    keys.append(pj * n + pi)
    allk = np.concatenate(keys)
    del keys
    allk.sort()
    rows = allk // n
    col = (allk - rows * n).astype(np.int32)
    del allk
    counts = np.bincount(rows, minlength=n)
    del rows
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    labels = np.full(n, -1, dtype=np.int32)
    labels[perm] = comm.astype(np.int32)
    return Graph(n=n, rowptr=rowptr, col=col, labels=labels, sizes=sizes)


def _native():
    """The row-parallel generator (hash_sbm.c), compiled once with gcc."""
    global _NATIVE
    if _NATIVE is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "hash_sbm.c")
        out_dir = os.path.join(here, "_build")
        so = os.path.join(out_dir, "libhash_sbm.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            os.makedirs(out_dir, exist_ok=True)
            tmp = so + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, src])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        P, I64, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
        lib.syn_pair_hash.restype = U64
        lib.syn_pair_hash.argtypes = [U64, U64]
        lib.syn_hash_sbm_rowptr.restype = I64
        lib.syn_hash_sbm_rowptr.argtypes = [I64, I64, P, U64, U64, ctypes.c_int, P, P]
        lib.syn_hash_sbm_fill.restype = None
        lib.syn_hash_sbm_fill.argtypes = [I64, I64, P, U64, U64, ctypes.c_int, P, P, P, P]
        _NATIVE = lib
    return _NATIVE


_NATIVE = None


def pair_threshold(p_in: float) -> tuple[int, int]:
    """(thr, all): a pair is linked iff its hash is below thr = floor(p_in * 2^64)
    (exact: a double times a power of two), or always when all = 1 (p_in = 1)."""
    if not 0.0 <= p_in <= 1.0:
        raise ValueError("p_in must be in [0, 1]")
    return (0, 1) if p_in == 1.0 else (int(p_in * 2.0 ** 64), 0)


def hash_sbm_graph(sizes, p_in: float, *, seed: int, inter_degree: float = 0.0,
                   n_free: int = 0) -> Graph:
    """Planted-partition graph whose intra-community links are decided pair by
    pair by a counter-based hash (hash_sbm.c): each pair of one community is
    linked with probability p_in, independently; n*inter_degree/2 distinct
    uniformly random inter-community pairs are linked as in sbm_graph; n_free
    extra nodes (label -1) have inter links only.  Node ids are in block order
    (not shuffled) and the rows are generated in parallel, so communities of
    10^4 to 10^5 nodes and ensembles of thousands of networks are built in
    seconds.
    """
    import ctypes
    lib = _native()
    rng = rng_for(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    m = len(sizes)
    n = int(sizes.sum()) + int(n_free)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    comm = np.full(n, -1, dtype=np.int64)
    comm[:off[-1]] = np.repeat(np.arange(m, dtype=np.int64), sizes)
    if inter_degree > 0:
        i, j = _inter_pairs_degree(comm, inter_degree, rng)
        ik = np.concatenate([i * n + j, j * n + i])
        ik.sort()
    else:
        ik = np.zeros(0, np.int64)
    irow = ik // max(n, 1)
    inter_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(irow, minlength=n), out=inter_rowptr[1:])
    inter_col = np.ascontiguousarray((ik % max(n, 1)).astype(np.int32))
    thr, full = pair_threshold(p_in)
    hseed = int(rng.integers(0, 2 ** 63, dtype=np.int64))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    nnz = lib.syn_hash_sbm_rowptr(n, m, ptr(off), hseed, thr, full, ptr(inter_rowptr), ptr(rowptr))
    col = np.empty(nnz, dtype=np.int32)
    lib.syn_hash_sbm_fill(n, m, ptr(off), hseed, thr, full, ptr(inter_rowptr), ptr(inter_col), ptr(rowptr),
                          ptr(col))
    return Graph(n=n, rowptr=rowptr, col=col, labels=comm.astype(np.int32), sizes=sizes)


def hierarchical_sbm_graph(groups: int, subs: int, size: int, p_sub: float, p_group: float, *,
                           seed: int, inter_degree: float = 0.0) -> Graph:
    """Two-level planted partition: `groups` groups of `subs` communities of
    `size` nodes; pairs inside a community are linked with probability p_sub,
    pairs of different communities of one group with p_group, and
    n*inter_degree/2 distinct uniform pairs of different groups.  Labels are
    the small communities; node ids are in block order."""
    rng = rng_for(seed)
    g_n = subs * size
    n = groups * g_n
    sub_of = np.arange(g_n) // size
    prob = np.where(sub_of[:, None] == sub_of[None, :], p_sub, p_group)
    iu, ju = np.triu_indices(g_n, 1)
    keys = []
    for g in range(groups):
        keep = rng.random(len(iu)) < prob[iu, ju]
        i, j = iu[keep] + g * g_n, ju[keep] + g * g_n
        keys += [i * n + j, j * n + i]
    comm = np.repeat(np.arange(groups, dtype=np.int64), g_n)
    if inter_degree > 0:
        i, j = _inter_pairs_degree(comm, inter_degree, rng)
        keys += [i * n + j, j * n + i]
    allk = np.sort(np.concatenate(keys))
    rows = allk // n
    col = (allk - rows * n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    labels = (np.arange(n) // size).astype(np.int32)
    return Graph(n=n, rowptr=rowptr, col=col, labels=labels,
                 sizes=np.full(groups * subs, size, dtype=np.int64))


def complete_graph_communities(sizes, *, seed: int, shuffle: bool = True) -> Graph:
    """Disjoint complete graphs (p_in = 1, no inter-community links)."""
    return sbm_graph(sizes, 1.0, seed=seed, inter_degree=0.0, shuffle=shuffle)


def random_labels_graph(n: int, p: float, m: int, *, seed: int,
                        free_frac: float = 0.1) -> Graph:
    """Erdos-Renyi graph with arbitrary (unplanted) labels, for brute-force checks.

    Labels are drawn uniformly from [0, m), a fraction free_frac set to -1.
    The split B = D + S is then far from sparse, which is exactly what a
    brute-force comparison on a tiny graph wants to stress.
    """
    rng = rng_for(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    i, j = iu[keep].astype(np.int64), ju[keep].astype(np.int64)
    rows = np.concatenate([i, j])
    cols = np.concatenate([j, i])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    labels = rng.integers(0, m, size=n).astype(np.int32)
    labels[rng.random(n) < free_frac] = -1
    sizes = np.bincount(labels[labels >= 0], minlength=m).astype(np.int64)
    return Graph(n=n, rowptr=rowptr, col=cols.astype(np.int32), labels=labels, sizes=sizes)
