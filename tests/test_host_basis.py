"""Host-side parts of the learned basis without a GPU: the Fourier
initialisation (cia_basis_params_fourier) against the oracle's Fourier basis."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2203_16657_gb300 import build
    build.build()
    import paper_2203_16657_gb300 as P
    return P


def test_fourier_parameters_reproduce_the_oracle_basis(lib, oracle_mod):
    """cia_basis_params_fourier (host code) against the oracle's Fourier basis
    of the same weight: the same truncated series up to the choice among
    modes of equal coefficient (the weight is radial, so (a, b) and (b, a)
    tie), and the same accuracy against the exact weight."""
    eta = lambda d2: oracle_mod.cs_kernel_weight(d2, 1.0, 1.0, 0.4)
    vec = lib.Basis.params_fourier(1.0, 1.0, 0.4, 10.0, seed=3)
    p = oracle_mod.unpack_params(vec.astype(np.float64))
    alpha, c = oracle_mod.fourier_basis(oracle_mod.radial(eta), 10.0, rank=64)
    rng = np.random.default_rng(10)
    s1, s2 = rng.uniform(-5, 5, (3000, 2)), rng.uniform(-5, 5, (3000, 2))
    f1, _ = oracle_mod.mlp_forward(p, s1)
    f2, _ = oracle_mod.mlp_forward(p, s2)
    g1 = oracle_mod.fourier_features(s1, alpha, c, 10.0)
    g2 = oracle_mod.fourier_features(s2, alpha, c, 10.0)
    k_lib, k_ora = (f1 * f2).sum(axis=1), (g1 * g2).sum(axis=1)
    ex = eta(((s1 - s2) ** 2).sum(axis=1))
    assert np.abs(k_lib - k_ora).max() < 0.02
    e_lib, e_ora = np.sqrt(((k_lib - ex) ** 2).mean()), np.sqrt(((k_ora - ex) ** 2).mean())
    assert abs(e_lib - e_ora) < 0.1 * e_ora, (e_lib, e_ora)
