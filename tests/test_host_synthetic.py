"""The row-parallel graph generator (synthetic/hash_sbm.c) on the CPU.

Its pair hash is the SplitMix64 output function (Steele, Lea, Flood 2014): the
first outputs of the published generator for two seeds pin it.  A numpy
evaluation of the same hash rebuilds every intra-community row bit-exactly,
and the graph is checked for what every workload graph must be: symmetric,
no self loops, rows ascending, links only where the recipe allows them.
"""
import numpy as np
import pytest

from synthetic.graphs import _native, hash_sbm_graph, pair_threshold

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def test_pair_hash_is_splitmix64():
    lib = _native()
    # SplitMix64 outputs k = 1, 2, ... of state s are mix(s + k * gamma)
    assert [lib.syn_pair_hash(1234567, k) for k in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert lib.syn_pair_hash(0, 0) == 0xE220A8397B1DCDAF


def _mix_np(z):
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


@pytest.mark.parametrize("p_in", [0.0, 0.35, 0.9, 1.0])
def test_hash_sbm_rows_match_numpy_hash(p_in):
    sizes, n_free = [37, 64, 5, 1], 9
    g = hash_sbm_graph(sizes, p_in, seed=17, inter_degree=3.0, n_free=n_free)
    n = g.n
    A = np.zeros((n, n), dtype=bool)
    for i in range(n):
        row = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(row) > 0), i
        A[i, row] = True
    assert (A == A.T).all() and not A.diagonal().any()
    lab = g.labels.astype(np.int64)
    assert (lab[-n_free:] == -1).all() and np.array_equal(np.bincount(lab[lab >= 0]), sizes)
    same = (lab[:, None] == lab[None, :]) & (lab[:, None] >= 0)
    # the intra links are exactly the pairs whose hash is below the threshold
    thr, full = pair_threshold(p_in)
    from synthetic.graphs import rng_for, _inter_pairs_degree
    rng = rng_for(17)
    comm = np.where(lab >= 0, lab, -1)
    _inter_pairs_degree(comm, 3.0, rng)               # the same draws as the generator
    hseed = np.uint64(int(rng.integers(0, 2 ** 63, dtype=np.int64)))
    i, j = np.triu_indices(n, 1)
    keys = i.astype(np.uint64) * np.uint64(n) + j.astype(np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        h = _mix_np(hseed + keys * np.uint64(GAMMA))
    want = np.zeros((n, n), dtype=bool)
    want[i, j] = True if full else (h < np.uint64(thr))
    want = (want | want.T) & same
    assert np.array_equal(A & same, want)
    # inter links: the requested count, none inside a community
    assert (A & ~same).sum() == 2 * int(round(n * 3.0 / 2.0))


def test_hash_sbm_density_is_p_in():
    g = hash_sbm_graph([400, 300], 0.7, seed=2)
    lam = np.array([400, 300])
    frac = g.nnz / float((lam * (lam - 1)).sum())
    assert abs(frac - 0.7) < 0.005           # about 4 standard deviations of a 125k-pair draw
