"""Pins of the FP64 oracle to what the paper and the mathematics fix.

None of these compares the oracle with a retyped copy of itself: each check
is a closed form, an invariant, a textbook result, a hand-evaluated fixture
(tests/golden/) or an exhaustive brute force on a tiny input, chosen so that
a dropped term, a flipped sign, a wrong index or normalisation fails one.
"""
import json
import math
import os

import numpy as np
import pytest

import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def complete_csr(n):
    rows = [[j for j in range(n) if j != i] for i in range(n)]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=rowptr[1:])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    return rowptr, col


# ---------------------------------------------------------------- integrators

def test_rk4_linear_amplification(oracle_mod):
    """One RK4 step of x' = lam x multiplies by 1 + z + z^2/2 + z^3/6 + z^4/24,
    z = lam dt (textbook stability polynomial); Euler by 1 + z."""
    for lam in (-1.0, -3.7, 0.4):
        for dt in (0.01, 0.1, 0.5):
            z = lam * dt
            x0 = np.array([1.0, -2.5, 3.25])
            x1 = oracle_mod.rk4_step(lambda x: lam * x, x0, dt)
            R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
            np.testing.assert_allclose(x1, R * x0, rtol=1e-15, atol=0)
            xe = oracle_mod.euler_step(lambda x: lam * x, x0, dt)
            np.testing.assert_allclose(xe, (1 + z) * x0, rtol=1e-15, atol=0)


def test_rk4_fourth_order_on_adler_equation(oracle_mod):
    """Two linked identical oscillators: psi = theta_2 - theta_1 obeys
    psi' = -K sin psi (N = 2, so each node gets (K/2) sin of the difference),
    solved by tan(psi/2) = tan(psi0/2) e^{-K t}; the mean phase moves at omega.
    Halving dt must shrink the RK4 error by about 2^4."""
    rowptr = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([1, 0], dtype=np.int32)
    K, omega, psi0, T = 1.5, 0.3, 2.0, 2.0
    th0 = np.array([0.1, 0.1 + psi0])
    om = np.array([omega, omega])
    rhs = lambda th: oracle_mod.kuramoto_direct(rowptr, col, th, om, K)
    exact_psi = 2 * math.atan(math.tan(psi0 / 2) * math.exp(-K * T))
    errs = []
    for steps in (40, 80):
        th, _ = oracle_mod.integrate(rhs, th0, T / steps, steps)
        errs.append(abs((th[1] - th[0]) - exact_psi))
        assert abs(th.mean() - (th0.mean() + omega * T)) < 1e-13
    assert errs[0] < 1e-6
    assert 12.0 < errs[0] / errs[1] < 20.0


def test_adler_phase_locking_sign(oracle_mod):
    """With omega_2 - omega_1 = d and |d| < K the difference locks at
    arcsin(d / K) (psi' = d - K sin psi); a sign error in h or in omega would
    lock at the mirrored angle or drift."""
    rowptr = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([1, 0], dtype=np.int32)
    K, d = 2.0, 0.8
    om = np.array([0.0, d])
    rhs = lambda th: oracle_mod.kuramoto_direct(rowptr, col, th, om, K)
    th, _ = oracle_mod.integrate(rhs, np.array([0.0, 0.0]), 0.01, 3000)
    assert abs((th[1] - th[0]) - math.asin(d / K)) < 1e-9


# ---------------------------------------------------------------- P1 split

def test_split_is_lossless_and_permutation_consistent(oracle_mod):
    for seed in range(4):
        g = S.random_labels_graph(37, 0.3, 4, seed=seed, free_frac=0.2)
        sp = oracle_mod.split(g.rowptr, g.col, g.labels)
        n = g.n
        assert np.array_equal(sp.perm[sp.iperm], np.arange(n))
        assert np.all(np.diff(sp.off) >= 0)
        assert sp.off[-1] == int((g.labels >= 0).sum())
        # communities are contiguous and ordered by label, ids ascending inside
        for c in range(sp.M):
            members = sp.perm[sp.off[c]:sp.off[c + 1]]
            assert np.all(g.labels[members] == c)
            assert np.all(np.diff(members) > 0)
        # B = D + S reproduces P A P^T exactly
        rp, cl = oracle_mod.rebuild_b(sp)
        for m in range(n):
            i = sp.perm[m]
            want = np.sort(sp.iperm[g.col[g.rowptr[i]:g.rowptr[i + 1]]])
            assert np.array_equal(cl[rp[m]:rp[m + 1]], want)
        # S holds -1 on the diagonal of every community block
        for m in range(sp.off[-1]):
            row = sp.s_col[sp.s_rowptr[m]:sp.s_rowptr[m + 1]]
            vals = sp.s_val[sp.s_rowptr[m]:sp.s_rowptr[m + 1]]
            assert vals[list(row).index(m)] == -1


# ---------------------------------------------------------------- Kuramoto

@pytest.mark.parametrize("d_sin,d_cos", [((1.0,), (0.0,)), ((0.0,), (1.0,)),
                                         ((0.7, -0.2, 0.05), (0.3, 0.1, -0.4))])
def test_cia_equals_direct_on_complete_communities(oracle_mod, d_sin, d_cos):
    """The addition theorems make E1 exact for a finite Fourier coupling
    (Sec. 3.2, App. A.4): on complete communities with no extra links, S is
    the diagonal only and the CIA equals the direct sum to rounding."""
    g = S.complete_graph_communities([7, 12, 5], seed=11)
    rng = np.random.default_rng(3)
    th = rng.uniform(0, 2 * np.pi, g.n)
    om = rng.normal(size=g.n)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    assert np.all(sp.s_val == -1) and len(sp.s_col) == g.n
    d = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 2.5, d_sin, d_cos)
    c = oracle_mod.kuramoto_cia(sp, th[sp.perm], om[sp.perm], 2.5, d_sin, d_cos)
    np.testing.assert_allclose(c, d[sp.perm], rtol=0, atol=1e-13)


def test_cosine_coupling_closed_form(oracle_mod):
    """h = cos on a complete graph with equal phases: every node gets
    omega + K (N-1)/N, since a_mm = 0 (the diagonal of the block is removed)."""
    n = 9
    rowptr, col = complete_csr(n)
    labels = np.zeros(n, dtype=np.int32)
    th = np.full(n, 0.77)
    om = np.linspace(-1, 1, n)
    sp = oracle_mod.split(rowptr, col, labels)
    for f in (lambda: oracle_mod.kuramoto_direct(rowptr, col, th, om, 3.0, (0.0,), (1.0,)),
              lambda: oracle_mod.kuramoto_cia(sp, th[sp.perm], om[sp.perm], 3.0,
                                              (0.0,), (1.0,))[sp.iperm]):
        np.testing.assert_allclose(f(), om + 3.0 * (n - 1) / n, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_cia_equals_brute_force_on_tiny_random_graphs(oracle_mod, seed):
    """Exhaustive check on <= 50 nodes: arbitrary labels (unlabelled nodes,
    empty communities, dense S) must still give the direct sum."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 51))
    g = S.random_labels_graph(n, float(rng.uniform(0.05, 0.9)), int(rng.integers(1, 6)),
                              seed=seed, free_frac=0.15)
    th = rng.uniform(-10, 10, n)
    om = rng.normal(size=n)
    ds, dc = rng.normal(size=2), rng.normal(size=2)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    d = oracle_mod.kuramoto_direct(g.rowptr, g.col, th, om, 1.3, ds, dc)
    c = oracle_mod.kuramoto_cia(sp, th[sp.perm], om[sp.perm], 1.3, ds, dc)
    np.testing.assert_allclose(c[sp.iperm], d, rtol=0, atol=1e-12)


def test_sum_of_rhs_equals_sum_of_frequencies(oracle_mod):
    """For symmetric A and odd h the coupling cancels pairwise: sum theta' =
    sum omega (direct and CIA)."""
    w = S.kuramoto_sbm_small(scale=0.25)
    g = w.graph
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    d = oracle_mod.kuramoto_direct(g.rowptr, g.col, w.theta0, w.omega, w.K, (1.0, 0.5), (0.0, 0.0))
    c = oracle_mod.kuramoto_cia(sp, w.theta0[sp.perm], w.omega[sp.perm], w.K, (1.0, 0.5), (0.0, 0.0))
    assert abs(d.sum() - w.omega.sum()) < 1e-11
    assert abs(c.sum() - w.omega.sum()) < 1e-11
    assert np.abs(d - w.omega).max() > 1e-2   # the coupling is not trivially zero


def test_identical_all_to_all_synchronises(oracle_mod):
    """Identical oscillators, all-to-all: a gradient flow of -r^2 (textbook),
    so r(t) never decreases and tends to 1."""
    n = 64
    rowptr, col = complete_csr(n)
    sp = oracle_mod.split(rowptr, col, np.zeros(n, dtype=np.int32))
    th0 = np.random.default_rng(5).uniform(0, 2 * np.pi, n)
    rhs = lambda x: oracle_mod.kuramoto_cia(sp, x, np.zeros(n), 1.0)
    _, r = oracle_mod.integrate(rhs, th0, 0.05, 800, wrap=True,
                                observe=oracle_mod.order_parameter)
    r = np.array(r)
    assert np.all(np.diff(r) > -1e-12)
    assert r[-1] > 1 - 1e-6


def test_lorentzian_self_consistency(oracle_mod):
    """All-to-all Kuramoto with Lorentzian frequencies of half-width D has the
    stationary order parameter r = sqrt(1 - 2D/K) for K > 2D (Kuramoto's
    self-consistency; textbook, not in the paper).  Deterministic quantiles of
    the Lorentzian keep the finite-N deviation small."""
    n, D, K = 1500, 0.5, 2.0
    q = (np.arange(n) + 0.5) / n
    om = D * np.tan(np.pi * (q - 0.5))
    rowptr, col = complete_csr(n)
    sp = oracle_mod.split(rowptr, col, np.zeros(n, dtype=np.int32))
    th0 = np.random.default_rng(9).uniform(0, 2 * np.pi, n)
    rhs = lambda x: oracle_mod.kuramoto_cia(sp, x, om, K)
    _, r = oracle_mod.integrate(rhs, th0, 0.05, 1200, wrap=True,
                                observe=oracle_mod.order_parameter)
    r_late = float(np.mean(r[-400:]))
    assert abs(r_late - math.sqrt(1 - 2 * D / K)) < 0.02


# ---------------------------------------------------------------- higher order

def test_triadic_hand_evaluated(oracle_mod):
    gd = json.load(open(os.path.join(GOLDEN, "triadic_three_nodes.json")))
    n = gd["N"]
    rowptr, col = complete_csr(n)
    sp = oracle_mod.split(rowptr, col, np.zeros(n, dtype=np.int32))
    phi = np.array(gd["phi"])
    d = oracle_mod.ho_triadic_direct(sp, phi, gd["K2"], np.arange(n))
    c = oracle_mod.ho_triadic_cia(sp, phi, gd["K2"])
    np.testing.assert_allclose(d, gd["expected"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(c, gd["expected"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_triadic_moments_equal_brute_force(oracle_mod, seed):
    """The moment formula with the degenerate tuples removed equals the plain
    sum over ordered pairs of distinct other members (App. A.7)."""
    rng = np.random.default_rng(seed)
    g = S.random_labels_graph(48, 0.2, 3, seed=seed, free_frac=0.1)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    phi = rng.uniform(-4, 4, g.n)
    d = oracle_mod.ho_triadic_direct(sp, phi, 2.0, np.arange(g.n))
    c = oracle_mod.ho_triadic_cia(sp, phi, 2.0)
    np.testing.assert_allclose(c, d, rtol=0, atol=1e-13)
    assert np.abs(d).max() > 1e-4


# ---------------------------------------------------------------- Cucker-Smale

def test_cs_two_agents_hand_evaluated(oracle_mod):
    gd = json.load(open(os.path.join(GOLDEN, "cucker_smale_two_agents.json")))
    rowptr = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([1, 0], dtype=np.int32)
    out = oracle_mod.cs_direct(rowptr, col, np.array(gd["x"]), 1.0, 1.0, 0.4)
    np.testing.assert_allclose(out, gd["expected"], rtol=0, atol=1e-15)


def test_cs_momentum_conservation(oracle_mod):
    """Symmetric A and an even weight: sum_m v_m' = 0."""
    g = S.sbm_graph([30, 25, 20], 0.8, inter_degree=3.0, seed=4)
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(0, 10, (g.n, 2)), rng.normal(size=(g.n, 2))], axis=1)
    out = oracle_mod.cs_direct(g.rowptr, g.col, x)
    assert np.abs(out[:, 2:].sum(axis=0)).max() < 1e-14
    assert np.abs(out[:, 2:]).max() > 1e-3


def test_cs_cia_exact_for_constant_weight(oracle_mod):
    """With beta = 0 the weight is the constant K, exactly separable with the
    single feature sqrt(K); the CIA must then equal the direct sum."""
    g = S.random_labels_graph(40, 0.4, 3, seed=8, free_frac=0.1)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(0, 10, (g.n, 2)), rng.normal(size=(g.n, 2))], axis=1)
    K = 1.7
    d = oracle_mod.cs_direct(g.rowptr, g.col, x, K, 1.0, 0.0)
    feat = np.full((g.n, 1), math.sqrt(K))
    c = oracle_mod.cs_cia(sp, x[sp.perm], feat, K, 1.0, 0.0)
    np.testing.assert_allclose(c[sp.iperm], d, rtol=0, atol=1e-13)


def _separable_weight(dx, dy, L):
    """g(d) = 1 + cos(pi d_x / L) + 0.5 cos(2 pi d_y / L): non-constant and, by
    cos(a - b) = cos a cos b + sin a sin b, exactly phi(s_l) . phi(s_m) for the
    five features of _separable_features."""
    return 1.0 + np.cos(np.pi * dx / L) + 0.5 * np.cos(2 * np.pi * dy / L)


def _separable_features(s, L):
    a, b = np.pi * s[:, 0] / L, 2 * np.pi * s[:, 1] / L
    h = math.sqrt(0.5)
    return np.stack([np.ones(len(s)), np.cos(a), np.sin(a), h * np.cos(b), h * np.sin(b)], axis=1)


@pytest.mark.parametrize("beta,seed", [(0.0, 21), (0.4, 22), (0.4, 23)])
def test_cs_cia_non_constant_separable_weight_brute_force(oracle_mod, beta, seed):
    """Eqs. Cucker_Smale_orderParams and Cucker_Smale_fast_RHS with an exactly
    separable, non-constant weight g on the community blocks D and the exact
    weight eta on the links of S (-1 missing, +1 inter).  The expected value is
    the definition summed pair by pair over a dense adjacency:

        v_m' = (1/N) [ sum_{l in c(m)} g(s_l - s_m)(v_l - v_m)
                       - sum_{l in c(m), l != m, a_ml = 0} eta (v_l - v_m)
                       + sum_{l not in c(m), a_ml = 1} eta (v_l - v_m) ].

    Every feature value differs between nodes and between features, so a
    transposed feature index, node m's feature row used for l (or the other way
    round), or another community's U/H row changes the result."""
    g = S.random_labels_graph(44, 0.45, 4, seed=seed, free_frac=0.15)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    rng = np.random.default_rng(seed)
    L = 10.0
    x = np.concatenate([rng.uniform(0, 10, (g.n, 2)), rng.normal(size=(g.n, 2))], axis=1)
    K, sigma = 1.3, 1.0
    n = g.n
    A = np.zeros((n, n))
    for i in range(n):
        A[i, g.col[g.rowptr[i]:g.rowptr[i + 1]]] = 1.0
    lab = np.asarray(g.labels)
    same = (lab[:, None] == lab[None, :]) & (lab[:, None] >= 0)
    want = np.zeros((n, 4))
    for m in range(n):
        dv = x[:, 2:] - x[m, 2:]
        dx, dy = x[:, 0] - x[m, 0], x[:, 1] - x[m, 1]
        eta = K * (sigma * sigma + dx * dx + dy * dy) ** (-beta)
        w = np.where(same[m], _separable_weight(dx, dy, L), 0.0)
        w -= np.where(same[m] & (A[m] == 0) & (np.arange(n) != m), eta, 0.0)
        w += np.where(~same[m] & (A[m] == 1), eta, 0.0)
        want[m, :2] = x[m, 2:]
        want[m, 2:] = (w[:, None] * dv).sum(axis=0) / n
    feat = _separable_features(x[:, :2], L)
    assert np.ptp(feat, axis=0)[1:].min() > 0.5            # non-constant in every feature
    got = oracle_mod.cs_cia(sp, x[sp.perm], feat[sp.perm], K, sigma, beta)[sp.iperm]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    assert np.abs(want[:, 2:]).max() > 0.05


# ---------------------------------------------------------------- learned basis

def _params(rng, H=8, R=4):
    return {"W1": rng.normal(size=(H, 2)), "b1": rng.normal(size=H),
            "W2": rng.normal(size=(R, H)) / np.sqrt(H), "b2": rng.normal(size=R) * 0.1}


def test_mlp_forward_hand_evaluated(oracle_mod):
    """H = R = 1: phi(x) = w2 act(w1 . x + b1) + b2.  sin: w1 . x + b1 = 0 and
    pi/2 give 0 and 1; SiLU: silu(0) = 0 and silu(1) = 1/(1 + e^-1)."""
    p = {"W1": np.array([[1.0, -2.0]]), "b1": np.array([0.0]),
         "W2": np.array([[3.0]]), "b2": np.array([0.25])}
    out, _ = oracle_mod.mlp_forward(p, np.array([[2.0, 1.0], [np.pi / 2, 0.0]]))
    np.testing.assert_allclose(out[:, 0], [0.25, 3.25], rtol=0, atol=1e-15)
    out, _ = oracle_mod.mlp_forward(p, np.array([[2.0, 1.0], [1.0, 0.0]]), act="silu")
    np.testing.assert_allclose(out[:, 0], [0.25, 3.0 / (1.0 + math.exp(-1.0)) + 0.25],
                               rtol=0, atol=1e-15)


def test_mlp_gradient_central_differences(oracle_mod):
    rng = np.random.default_rng(0)
    p = _params(rng)
    a, c = rng.normal(size=(16, 2)), rng.normal(size=(16, 2))
    t = oracle_mod.cs_kernel_weight(((a - c) ** 2).sum(axis=1))
    for act in ("sin", "silu"):
        _check_pair_gradient(oracle_mod, p, a, c, t, act)


def _check_pair_gradient(oracle_mod, p, a, c, t, act):
    loss, grads = oracle_mod.pair_loss_grad(p, a, c, t, act=act)
    assert abs(loss - oracle_mod.pair_loss(p, a, c, t, act=act)) < 1e-15
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = oracle_mod.pair_loss(p, a, c, t, act=act)
            flat[idx] = old - h
            lm = oracle_mod.pair_loss(p, a, c, t, act=act)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_bf16_round_ties_to_even(oracle_mod):
    """bfloat16 keeps 8 significand bits: the spacing at 1 is 2^-7.  Halfway
    cases go to the even neighbour; other values to the nearest."""
    r = oracle_mod.bf16_round
    cases = [(1.0, 1.0), (1.0 + 2.0 ** -8, 1.0), (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),
             (1.0 + 2.0 ** -7, 1.0 + 2.0 ** -7), (1.0 + 1.1 * 2.0 ** -8, 1.0 + 2.0 ** -7),
             (-3.0 - 2.0 ** -7, -3.0), (0.0, 0.0), (2.0 ** -130, 2.0 ** -130)]
    for x, want in cases:
        assert r(np.array([x]))[0] == want, (x, r(np.array([x]))[0], want)
    v = np.random.default_rng(3).normal(size=1000) * 100
    q = r(v)
    # representable: low 16 bits of the float32 pattern are zero, and within half a spacing
    assert not (q.astype(np.float32).view(np.uint32) & 0xFFFF).any()
    assert (np.abs(q - v) <= np.abs(v) * 2.0 ** -8 + 1e-300).all()


def test_param_packing_round_trip(oracle_mod):
    rng = np.random.default_rng(4)
    vec = rng.normal(size=128 * 2 + 128 + 64 * 128 + 64)
    p = oracle_mod.unpack_params(vec)
    assert p["W1"].shape == (128, 2) and p["W2"].shape == (64, 128)
    assert p["W1"][5, 1] == vec[11] and p["b1"][0] == vec[256] and p["W2"][1, 0] == vec[384 + 128]
    np.testing.assert_array_equal(oracle_mod.pack_params(p), vec)


def test_fourier_coefficients_of_a_gaussian(oracle_mod):
    """A narrow Gaussian on a wide box: the periodic coefficients are samples
    of its continuous Fourier transform, c_alpha = (2 pi s^2 / (2L)^2)
    exp(-pi^2 s^2 |alpha|^2 / (2 L^2)) (periodisation error ~ e^{-L^2/2s^2})."""
    L, sg = 10.0, 1.3
    g2 = lambda X, Y: np.exp(-(X * X + Y * Y) / (2 * sg * sg))
    alpha, c = oracle_mod.fourier_coefficients(g2, L, 128)
    want = (2 * np.pi * sg * sg / (2 * L) ** 2) * np.exp(
        -np.pi ** 2 * sg * sg * (alpha ** 2).sum(axis=1) / (2 * L * L))
    assert np.abs(c - want).max() < 1e-12


def test_fourier_features_reproduce_trigonometric_weights(oracle_mod):
    """g(d) = 1 + cos(pi d_x / L) + 0.5 cos(2 pi d_y / L) has exactly three
    mode pairs: the rank-5 basis reproduces it for any two positions."""
    L = 7.0
    g2 = lambda X, Y: 1.0 + np.cos(np.pi * X / L) + 0.5 * np.cos(2 * np.pi * Y / L)
    alpha, c = oracle_mod.fourier_basis(g2, L, rank=5, grid=64)
    got = {tuple(a): v for a, v in zip(alpha.tolist(), c)}
    assert set(got) == {(0, 0), (1, 0), (0, 2)}
    assert abs(got[(0, 0)] - 1.0) < 1e-12 and abs(got[(1, 0)] - 0.5) < 1e-12
    assert abs(got[(0, 2)] - 0.25) < 1e-12
    rng = np.random.default_rng(8)
    s1, s2 = rng.uniform(-3, 3, (50, 2)), rng.uniform(-3, 3, (50, 2))
    f1 = oracle_mod.fourier_features(s1, alpha, c, L)
    f2 = oracle_mod.fourier_features(s2, alpha, c, L)
    d = s1 - s2
    np.testing.assert_allclose((f1 * f2).sum(axis=1), g2(d[:, 0], d[:, 1]), rtol=0, atol=1e-12)


def test_fourier_basis_of_the_cs_weight_converges(oracle_mod):
    """More modes, smaller error of the separable approximation of
    (1 + r^2)^-0.4 over differences of positions in a 10 x 10 box."""
    eta = lambda d2: oracle_mod.cs_kernel_weight(d2, 1.0, 1.0, 0.4)
    rng = np.random.default_rng(9)
    s1, s2 = rng.uniform(0, 10, (2000, 2)), rng.uniform(0, 10, (2000, 2))
    ref = eta(((s1 - s2) ** 2).sum(axis=1))
    errs = []
    for rank in (9, 25, 64, 121):
        alpha, c = oracle_mod.fourier_basis(oracle_mod.radial(eta), 10.0, rank)
        f1 = oracle_mod.fourier_features(s1, alpha, c, 10.0)
        f2 = oracle_mod.fourier_features(s2, alpha, c, 10.0)
        assert f1.shape[1] <= rank
        errs.append(np.sqrt((((f1 * f2).sum(axis=1) - ref) ** 2).mean()))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_desai_zwanzig_hand_values(oracle_mod):
    """One uncoupled particle in the double well V = x^4/4 - x^2/2:
    x' = x - x^3 (0 at the minima +-1 and the maximum 0, 3/8 at x = 1/2)."""
    rowptr, col = np.zeros(2, np.int64), np.zeros(0, np.int32)
    for x, want in [(1.0, 0.0), (-1.0, 0.0), (0.0, 0.0), (0.5, 0.375)]:
        out = oracle_mod.poly_direct(rowptr, col, np.array([x]), 2.0, [0.0, 1.0], [0.0, -1.0, 0.0, 1.0])
        assert out[0] == want


def test_linear_consensus_decays_by_the_rk4_polynomial(oracle_mod):
    """V' = 0, h(x) = x on a complete graph: x' = K (xbar - x_m) exactly, so the
    mean is kept and every deviation is multiplied by R(-K dt) per RK4 step."""
    n, K, dt, steps = 12, 1.7, 0.05, 30
    rowptr, col = complete_csr(n)
    x0 = np.random.default_rng(11).normal(size=n)
    rhs = lambda y: oracle_mod.poly_direct(rowptr, col, y, K, [0.0, 1.0], [0.0])
    got, _ = oracle_mod.integrate(rhs, x0, dt, steps, wrap=False)
    z = -K * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    want = x0.mean() + (x0 - x0.mean()) * R ** steps
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_polynomial_cia_equals_direct(oracle_mod, seed):
    """The moment formula (binomial expansion of h) plus the exact sparse
    corrections reaches the direct sum on random graphs with unlabelled nodes,
    for a cubic coupling and a quartic potential."""
    import synthetic as S
    g = S.random_labels_graph(45, 0.3, 3, seed=60 + seed, free_frac=0.2)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=g.n)
    c = rng.normal(size=4)
    dv = rng.normal(size=5)
    ref = oracle_mod.poly_direct(g.rowptr, g.col, x, 1.3, c, dv)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    got = oracle_mod.poly_cia(sp, x[sp.perm], 1.3, c, dv)[sp.iperm]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------ general polynomial g(x_l, x_m)

def test_general_polynomial_linear_neighbour_term_is_a_sparse_matvec(oracle_mod):
    """g(u, y) = u: x' = (K/N) A x, checked against scipy's CSR product."""
    sp_mod = pytest.importorskip("scipy.sparse")
    import synthetic as S
    g = S.random_labels_graph(60, 0.2, 3, seed=3, free_frac=0.1)
    x = np.random.default_rng(1).normal(size=g.n)
    A = sp_mod.csr_matrix((np.ones(len(g.col)), g.col, g.rowptr), shape=(g.n, g.n))
    G = np.zeros((2, 2))
    G[1, 0] = 1.0
    got = oracle_mod.polyg_direct(g.rowptr, g.col, x, 2.0, G, [0.0])
    np.testing.assert_allclose(got, (2.0 / g.n) * (A @ x), rtol=1e-14, atol=1e-15)


def test_general_polynomial_own_term_scales_with_degree(oracle_mod):
    """g(u, y) = y^2 does not depend on the neighbour: x' = (K/N) deg(m) x_m^2."""
    import synthetic as S
    g = S.random_labels_graph(50, 0.3, 2, seed=4, free_frac=0.2)
    x = np.random.default_rng(2).normal(size=g.n)
    G = np.zeros((3, 3))
    G[0, 2] = 1.0
    got = oracle_mod.polyg_direct(g.rowptr, g.col, x, 1.5, G, [0.0])
    deg = np.diff(g.rowptr)
    np.testing.assert_allclose(got, (1.5 / g.n) * deg * x * x, rtol=1e-14, atol=0)


def test_general_polynomial_of_a_difference_matches_the_difference_form(oracle_mod):
    """h(u - y) = sum_a c_a (u - y)^a expands to G[a, b] = c_{a+b} binom(a+b, a)
    (-1)^b: the general form reaches the difference oracle (eq. PolyApprox with
    g(x, y) = h(x - y))."""
    from math import comb
    import synthetic as S
    g = S.random_labels_graph(40, 0.3, 3, seed=5, free_frac=0.2)
    rng = np.random.default_rng(3)
    c = rng.normal(size=5)
    p = len(c) - 1
    G = np.zeros((p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1 - a):
            G[a, b] = c[a + b] * comb(a + b, a) * (-1) ** b
    x = rng.uniform(-1, 1, g.n)
    dv = rng.normal(size=3)
    ref = oracle_mod.poly_direct(g.rowptr, g.col, x, 1.1, c, dv)
    got = oracle_mod.polyg_direct(g.rowptr, g.col, x, 1.1, G, dv)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_general_polynomial_brute_force_tiny(oracle_mod):
    """A 6-node graph with a dense adjacency matrix, summed in plain Python."""
    A = np.array([[0, 1, 1, 0, 0, 1], [1, 0, 1, 0, 0, 0], [1, 1, 0, 1, 0, 0],
                  [0, 0, 1, 0, 1, 1], [0, 0, 0, 1, 0, 1], [1, 0, 0, 1, 1, 0]])
    rowptr = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int64)
    col = np.concatenate([np.nonzero(r)[0] for r in A]).astype(np.int32)
    rng = np.random.default_rng(4)
    G = rng.normal(size=(3, 3))
    dv = [0.5, -1.0]
    x = rng.normal(size=6)
    K, n = 0.7, 6
    want = np.zeros(n)
    for m in range(n):
        s = 0.0
        for l in range(n):
            if A[m, l]:
                s += sum(G[a, b] * x[l] ** a * x[m] ** b for a in range(3) for b in range(3))
        want[m] = -(dv[0] + dv[1] * x[m]) + K / n * s
    got = oracle_mod.polyg_direct(rowptr, col, x, K, G, dv)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_general_polynomial_cia_equals_direct(oracle_mod, seed):
    """Moments w_a with the dense term sum G[a, b] w_a x_m^b (eq. PolyRHS) plus
    the exact sparse corrections over S reach the direct sum."""
    import synthetic as S
    g = S.random_labels_graph(45, 0.3, 3, seed=80 + seed, free_frac=0.2)
    rng = np.random.default_rng(seed)
    p = 1 + seed
    G = rng.normal(size=(p + 1, p + 1))
    dv = rng.normal(size=4)
    x = rng.normal(size=g.n)
    ref = oracle_mod.polyg_direct(g.rowptr, g.col, x, 1.3, G, dv)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    got = oracle_mod.polyg_cia(sp, x[sp.perm], 1.3, G, dv)[sp.iperm]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------ rank-one weighted links

def test_rank_one_weights_brute_force_dense_matrix(oracle_mod):
    """A 40-node graph as a dense 0/1 matrix: sum over l of A_ml alpha_m beta_l
    g(x_l, x_m) by numpy broadcasting, independent of the oracle's loops."""
    import synthetic as S
    g = S.random_labels_graph(40, 0.3, 3, seed=9, free_frac=0.2)
    A = np.zeros((g.n, g.n))
    for m in range(g.n):
        A[m, g.col[g.rowptr[m]:g.rowptr[m + 1]]] = 1.0
    rng = np.random.default_rng(21)
    x, al, be = rng.normal(size=g.n), rng.uniform(0.2, 2, g.n), rng.normal(size=g.n)
    G = rng.normal(size=(3, 3))
    U, Y = x[None, :], x[:, None]                  # U[m, l] = x_l, Y[m, l] = x_m
    gmat = sum(G[a, b] * U ** a * Y ** b for a in range(3) for b in range(3))
    want = -(0.5 * x ** 3) + 1.3 / g.n * (al[:, None] * A * be[None, :] * gmat).sum(1)
    got = oracle_mod.polyw_direct(g.rowptr, g.col, x, 1.3, G, [0, 0, 0, 0.5], al, be)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_rank_one_linear_neighbour_term_is_a_weighted_matvec(oracle_mod):
    """g(u, y) = u: x' = (K/N) diag(alpha) A diag(beta) x (scipy CSR products)."""
    sp_mod = pytest.importorskip("scipy.sparse")
    import synthetic as S
    g = S.random_labels_graph(70, 0.2, 4, seed=10, free_frac=0.1)
    A = sp_mod.csr_matrix((np.ones(len(g.col)), g.col, g.rowptr), shape=(g.n, g.n))
    rng = np.random.default_rng(22)
    x, al, be = rng.normal(size=g.n), rng.normal(size=g.n), rng.normal(size=g.n)
    G = np.zeros((2, 2))
    G[1, 0] = 1.0
    got = oracle_mod.polyw_direct(g.rowptr, g.col, x, 0.8, G, [0.0], al, be)
    want = (0.8 / g.n) * al * (A @ (be * x))
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_rank_one_cia_equals_direct(oracle_mod, seed):
    """Weighted moments (eq. rank1precompute) with alpha_m scaling (eq. rank1fast)
    plus the weighted sparse corrections reach the direct sum."""
    import synthetic as S
    g = S.random_labels_graph(50, 0.35, 3, seed=30 + seed, free_frac=0.2)
    rng = np.random.default_rng(40 + seed)
    x, al, be = rng.normal(size=g.n), rng.normal(size=g.n), rng.uniform(-1, 2, g.n)
    G = rng.normal(size=(seed + 2, seed + 2))
    dv = rng.normal(size=3)
    ref = oracle_mod.polyw_direct(g.rowptr, g.col, x, 1.1, G, dv, al, be)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    got = oracle_mod.polyw_cia(sp, x[sp.perm], 1.1, G, dv, al[sp.perm], be[sp.perm])[sp.iperm]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------ general real 2-D Fourier coupling

def _blocks(p, rng=None):
    if rng is None:
        return [np.zeros((p + 1, p + 1)) for _ in range(4)]
    return [rng.normal(size=(p + 1, p + 1)) for _ in range(4)]


def test_fourier_general_sine_of_difference_is_kuramoto(oracle_mod):
    """sin(w(u - y)) = sin(wu)cos(wy) - cos(wu)sin(wy): C21[1,1] = 1, C12[1,1] = -1
    gives the Kuramoto coupling of the phases w x (the Kuramoto oracle)."""
    import synthetic as S
    g = S.random_labels_graph(60, 0.25, 3, seed=12, free_frac=0.2)
    rng = np.random.default_rng(31)
    L = 2.5
    x = rng.uniform(-L, L, g.n)
    C = _blocks(1)
    C[2][1, 1], C[1][1, 1] = 1.0, -1.0
    got = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 1.7, L, C, [0.0])
    want = oracle_mod.kuramoto_direct(g.rowptr, g.col, np.pi * x / L, np.zeros(g.n), 1.7)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_fourier_general_constant_and_own_terms(oracle_mod):
    """C11[0,0] = 1 sums the degree; C12[0,2] = 1 gives deg(m) sin(2 w x_m)."""
    import synthetic as S
    g = S.random_labels_graph(40, 0.3, 2, seed=13, free_frac=0.1)
    x = np.random.default_rng(32).uniform(-3, 3, g.n)
    deg = np.diff(g.rowptr)
    C = _blocks(2)
    C[0][0, 0] = 1.0
    got = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 2.0, 3.0, C, [0.0])
    np.testing.assert_allclose(got, 2.0 / g.n * deg, rtol=1e-15, atol=0)
    C = _blocks(2)
    C[1][0, 2] = 1.0
    got = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 2.0, 3.0, C, [0.0])
    np.testing.assert_allclose(got, 2.0 / g.n * deg * np.sin(2 * np.pi * x / 3.0), rtol=1e-13, atol=1e-16)


def test_fourier_general_brute_force_and_periodicity(oracle_mod):
    """Dense-matrix brute force with numpy's cos/sin; shifting every state by 2L
    leaves the coupling unchanged (period of the series)."""
    import synthetic as S
    g = S.random_labels_graph(30, 0.35, 3, seed=14, free_frac=0.2)
    A = np.zeros((g.n, g.n))
    for m in range(g.n):
        A[m, g.col[g.rowptr[m]:g.rowptr[m + 1]]] = 1.0
    rng = np.random.default_rng(33)
    p, L, K = 2, 1.5, 0.9
    C = _blocks(p, rng)
    x = rng.uniform(-L, L, g.n)
    w = np.pi / L
    U, Y = x[None, :], x[:, None]
    G = sum(C[0][a, b] * np.cos(a * w * U) * np.cos(b * w * Y) + C[1][a, b] * np.cos(a * w * U) * np.sin(b * w * Y)
            + C[2][a, b] * np.sin(a * w * U) * np.cos(b * w * Y) + C[3][a, b] * np.sin(a * w * U) * np.sin(b * w * Y)
            for a in range(p + 1) for b in range(p + 1))
    want = K / g.n * (A * G).sum(1)
    got = oracle_mod.fourierg_direct(g.rowptr, g.col, x, K, L, C, [0.0])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)
    shifted = oracle_mod.fourierg_direct(g.rowptr, g.col, x + 2 * L, K, L, C, [0.0])
    np.testing.assert_allclose(shifted, got, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_fourier_general_cia_equals_direct(oracle_mod, p):
    """The real generalised order parameters (eq. RealOP) with the dense formula
    plus the exact sparse corrections reach the direct sum."""
    import synthetic as S
    g = S.random_labels_graph(50, 0.35, 3, seed=70 + p, free_frac=0.2)
    rng = np.random.default_rng(80 + p)
    C = _blocks(p, rng)
    dv = rng.normal(size=3)
    x = rng.uniform(-2, 2, g.n)
    ref = oracle_mod.fourierg_direct(g.rowptr, g.col, x, 1.2, 2.0, C, dv)
    sp = oracle_mod.split(g.rowptr, g.col, g.labels)
    got = oracle_mod.fourierg_cia(sp, x[sp.perm], 1.2, 2.0, C, dv)[sp.iperm]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------ community detection objective

def test_potts_hamiltonian_counts_s_at_half_density(oracle_mod):
    """With gamma p = 1/2 and mu = 0, H = nnz(S)/2 - |E|, nnz(S) counted from the
    oracle's own split of B = D + S (missing without the diagonal, plus inter)."""
    import synthetic as S
    for seed in range(3):
        g = S.random_labels_graph(60, 0.2, 4, seed=90 + seed, free_frac=0.0)
        n, nnz = g.n, len(g.col)
        gamma = 0.5 / (nnz / (n * (n - 1)))
        sp = oracle_mod.split(g.rowptr, g.col, g.labels)
        nnz_s = int(np.sum(sp.s_val != 0)) - int(np.sum((sp.s_val == -1) & (sp.s_col == np.repeat(
            np.arange(n), np.diff(sp.s_rowptr)))))   # without the diagonal -1 entries
        h = oracle_mod.potts_hamiltonian(g.rowptr, g.col, g.labels, gamma)
        assert abs(h - (nnz_s / 2 - nnz / 2)) < 1e-9


def test_potts_hamiltonian_special_partitions(oracle_mod):
    """Singletons: H = mu N.  One community of a complete graph (p = 1):
    H = (gamma - 1) N (N - 1) + mu."""
    import synthetic as S
    g = S.random_labels_graph(30, 0.3, 2, seed=3, free_frac=0.0)
    assert oracle_mod.potts_hamiltonian(g.rowptr, g.col, np.arange(g.n), 1.0, 0.7) == pytest.approx(0.7 * g.n)
    n = 12
    rowptr, col = complete_csr(n)
    h = oracle_mod.potts_hamiltonian(rowptr, col, np.zeros(n), 1.3, 2.0)
    assert h == pytest.approx((1.3 - 1) * n * (n - 1) + 2.0)
