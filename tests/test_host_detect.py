"""Community detection for step P1 (host code in libcia, no GPU): the Potts
Hamiltonian with the Erdos-Renyi null model (Sec. "Community Detection (P1)").

What is unique is checked exactly (H of the returned partition against the
oracle's definition, the entries of S against the oracle's split); the rest
by properties: no single-node move lowers H (brute force in the oracle),
planted communities are found, a charge per community reduces their number.
"""
import numpy as np
import pytest

import synthetic as S


@pytest.fixture(scope="module")
def cia():
    import paper_2203_16657_gb300 as P
    P.load()
    return P


def same_partition(a, b):
    """True if the two labelings define the same partition."""
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def density(g):
    return len(g.col) / (g.n * (g.n - 1))


@pytest.mark.parametrize("seed", range(3))
def test_planted_partition_is_recovered(cia, seed):
    g = S.sbm_graph([40, 60, 30, 50], 0.9, inter_degree=2.0, seed=200 + seed)
    labels, rep = cia.detect_communities(g.rowptr, g.col, seed=seed)
    assert rep["communities"] == 4 and rep["unlabelled"] == 0
    assert same_partition(labels, g.labels)


@pytest.mark.parametrize("gamma_p", [None, 0.5])
@pytest.mark.parametrize("seed", range(3))
def test_local_minimum_and_hamiltonian(cia, oracle_mod, seed, gamma_p):
    """No move of one node to a neighbouring or a new community lowers H,
    and the reported H is the oracle's H of the returned partition."""
    g = S.random_labels_graph(70, 0.12, 3, seed=300 + seed, free_frac=0.0)
    gamma = 1.0 if gamma_p is None else gamma_p / density(g)
    labels, rep = cia.detect_communities(g.rowptr, g.col, gamma=gamma, min_size=1, seed=seed)
    assert labels.min() >= 0
    h = oracle_mod.potts_hamiltonian(g.rowptr, g.col, labels, gamma)
    assert rep["hamiltonian"] == pytest.approx(h, abs=1e-6)
    assert oracle_mod.best_single_move_gain(g.rowptr, g.col, labels, gamma) < 1e-6


def test_entries_of_s_match_the_oracle_split(cia, oracle_mod):
    g = S.sbm_graph([30, 25, 40, 3, 2], 0.85, inter_degree=3.0, seed=7, n_free=6)
    labels, rep = cia.detect_communities(g.rowptr, g.col, min_size=4, seed=1)
    sp = oracle_mod.split(g.rowptr, g.col, labels)
    rows = np.repeat(np.arange(g.n), np.diff(sp.s_rowptr))
    diag = (sp.s_col == rows) & (sp.s_val == -1)
    assert rep["nnz_missing"] == int(np.sum((sp.s_val == -1) & ~diag))
    assert rep["nnz_inter"] == int(np.sum(sp.s_val == 1))
    assert rep["unlabelled"] == int(np.sum(labels < 0))
    sizes = np.bincount(labels[labels >= 0])
    assert sizes.min() >= 4 and len(sizes) == rep["communities"]


def test_half_density_minimises_s_on_planted_graphs(cia):
    """With gamma p = 1/2, H counts the entries of S: on clear planted graphs the
    result has no more entries of S than the planted labels."""
    from oracle import split
    for seed in range(3):
        g = S.sbm_graph([50, 35, 60], 0.8, inter_degree=3.0, seed=400 + seed)
        labels, rep = cia.detect_communities(g.rowptr, g.col, gamma=0.5 / density(g), min_size=1, seed=seed)
        planted = split(g.rowptr, g.col, g.labels)
        rows = np.repeat(np.arange(g.n), np.diff(planted.s_rowptr))
        nnz_planted = int(np.sum(planted.s_val != 0)) - int(np.sum((planted.s_val == -1) & (planted.s_col == rows)))
        assert rep["nnz_missing"] + rep["nnz_inter"] <= nnz_planted


def test_community_cost_merges_communities(cia):
    """A charge per community (the E1 cost of each community) yields fewer
    communities, never more, as it grows."""
    g = S.sbm_graph([8] * 12, 0.9, inter_degree=3.0, seed=11)
    counts = []
    for mu in (0.0, 10.0, 40.0, 200.0):
        _, rep = cia.detect_communities(g.rowptr, g.col, community_cost=mu, min_size=1, seed=2)
        counts.append(rep["communities"])
    assert counts[0] == 12
    assert all(b <= a for a, b in zip(counts, counts[1:])) and counts[-1] < counts[0]


def test_deterministic_for_a_seed(cia):
    g = S.random_labels_graph(200, 0.05, 5, seed=12, free_frac=0.0)
    a, ra = cia.detect_communities(g.rowptr, g.col, seed=5)
    b, rb = cia.detect_communities(g.rowptr, g.col, seed=5)
    assert np.array_equal(a, b) and ra == rb


def test_degenerate_graphs(cia):
    g = S.random_labels_graph(20, 0.0, 3, seed=2, free_frac=0.0)          # no links
    labels, rep = cia.detect_communities(g.rowptr, g.col)
    assert np.all(labels == -1) and rep["communities"] == 0 and rep["nnz_inter"] == 0
    g = S.complete_graph_communities([25], seed=1)
    # p = 1: with gamma = 1 every partition has H = 0; gamma p = 1/2 counts S
    labels, rep = cia.detect_communities(g.rowptr, g.col, gamma=0.5)
    assert np.all(labels == 0) and rep["nnz_missing"] == 0 and rep["nnz_inter"] == 0
    labels, rep = cia.detect_communities(np.array([0, 0]), np.zeros(0, np.int32), min_size=1)
    assert labels.tolist() == [0] and rep["communities"] == 1


def test_labels_feed_a_plan_split(cia, oracle_mod):
    """Detected labels are valid plan input; the oracle's CIA with them equals
    the direct sum (the split is lossless for any labels)."""
    g = S.sbm_graph([30, 45, 20], 0.85, inter_degree=3.0, seed=13, n_free=5)
    labels, _ = cia.detect_communities(g.rowptr, g.col, seed=3)
    sp = oracle_mod.split(g.rowptr, g.col, labels)
    theta = np.random.default_rng(1).uniform(-np.pi, np.pi, g.n)
    om = np.zeros(g.n)
    ref = oracle_mod.kuramoto_direct(g.rowptr, g.col, theta, om, 2.0)
    got = oracle_mod.kuramoto_cia(sp, theta[sp.perm], om[sp.perm], 2.0)[sp.iperm]
    assert np.abs(got - ref).max() < 1e-12


def test_rejections(cia):
    g = S.random_labels_graph(10, 0.3, 2, seed=1, free_frac=0.0)
    for kw in (dict(gamma=0.0), dict(gamma=np.inf), dict(community_cost=-1.0), dict(min_size=0),
               dict(max_levels=0)):
        with pytest.raises(cia.CiaError):
            cia.detect_communities(g.rowptr, g.col, **kw)
    bad_col = g.col.copy()
    bad_col[0] = g.n + 3
    with pytest.raises(cia.CiaError):
        cia.detect_communities(g.rowptr, bad_col)
