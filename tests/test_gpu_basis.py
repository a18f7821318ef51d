"""Learned Cucker--Smale basis on the GPU (include/cia_basis.h) against the
FP64 oracle MLP (oracle/mlp.py).

Forward tolerance, derived from the arithmetic: the device rounds every
hidden activation a_j = sin(z_j) to BF16 before the second layer (relative
error at most 2^-8, the BF16 unit roundoff) after an FP32 sine whose absolute
error stays below 1e-5 for the arguments used here, so

    |phi_r(gpu) - phi_r(exact)| <= sum_j |W2_rj| (2^-8 |a_j| + 1e-5)  (+ FP32 rounding),

with the exact phi computed by the oracle in FP64 from the same weights (W2
rounded to BF16 as the device holds it).
Gradients: the backward products use BF16 operands (dPhi, W2, A1), so they are
compared by relative norm (<= 2e-2) and cosine (>= 0.999) per parameter block.
"""
import numpy as np
import pytest

from helpers import cuda_available

pytestmark = pytest.mark.gpu

H, R = 128, 64


def _params(seed, w1=0.5, b1=0.5, w2=None, b2=0.1):
    rng = np.random.default_rng(seed)
    w2 = 1.0 / np.sqrt(H) if w2 is None else w2
    p = {"W1": rng.normal(0, w1, (H, 2)), "b1": rng.normal(0, b1, H),
         "W2": rng.normal(0, w2, (R, H)), "b2": rng.normal(0, b2, R)}
    return p


def _vec(oracle_mod, p):
    return oracle_mod.pack_params(p).astype(np.float32)


def _bf16_params(oracle_mod, vec):
    """The evaluated model: W2 (the tensor-core operand) rounded to BF16, the
    first layer and the biases in FP32."""
    p = oracle_mod.unpack_params(np.asarray(vec, dtype=np.float32).astype(np.float64))
    p["W2"] = oracle_mod.bf16_round(p["W2"])
    return p


@pytest.fixture(scope="module")
def P():
    if not cuda_available():
        pytest.skip("no CUDA device")
    import paper_2203_16657_gb300 as P
    from paper_2203_16657_gb300 import build
    build.build()
    return P


@pytest.mark.parametrize("count", [1, 127, 128, 129, 1000, 40000])
def test_features_within_bf16_bound(P, oracle_mod, count):
    import torch
    vec = _vec(oracle_mod, _params(11))
    basis = P.Basis(vec)
    rng = np.random.default_rng(100 + count)
    x = rng.uniform(-6, 6, (count, 2)).astype(np.float32)
    phi = basis.features(torch.from_numpy(x).cuda())
    basis.sync()
    phi = phi.cpu().numpy().astype(np.float64)
    p = _bf16_params(oracle_mod, vec)
    ref, cache = oracle_mod.mlp_forward(p, x.astype(np.float64))
    S = np.abs(cache["a1"]) @ np.abs(p["W2"]).T
    bound = (2.0 ** -8 + 1e-5) * S + 1e-5 * np.abs(p["W2"]).sum(axis=1) + 1e-5 * (np.abs(ref) + 1.0)
    err = np.abs(phi - ref)
    assert (err <= bound).all(), float((err / bound).max())
    # with the same BF16 rounding of the hidden layer on the oracle side, the
    # two agree to FP32 rounding except where a rounding decision flipped
    ref_r, _ = oracle_mod.mlp_forward(p, x.astype(np.float64), hidden_round=oracle_mod.bf16_round)
    close = np.abs(phi - ref_r) <= 1e-5 * (S + 1.0)
    assert close.mean() > 0.95, close.mean()


def test_features_constant_map(P, oracle_mod):
    """W2 = 0: phi(x) = b2 exactly (FP32 value), for every input."""
    import torch
    p = _params(12)
    p["W2"][:] = 0.0
    vec = _vec(oracle_mod, p)
    basis = P.Basis(vec)
    x = torch.randn(300, 2, device="cuda")
    phi = basis.features(x).cpu().numpy()
    np.testing.assert_array_equal(phi, np.broadcast_to(vec[-R:], phi.shape))


def _pairs(oracle_mod, B, seed, spread=3.0):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-spread, spread, (B, 2))
    c = rng.uniform(-spread, spread, (B, 2))
    a = a.astype(np.float32).astype(np.float64)
    c = c.astype(np.float32).astype(np.float64)
    t = oracle_mod.cs_kernel_weight(((a - c) ** 2).sum(axis=1)).astype(np.float32)
    return np.concatenate([a, c, t[:, None]], axis=1).astype(np.float32)


@pytest.mark.parametrize("B", [1, 63, 64, 1000, 20000])
def test_pair_gradient_matches_oracle(P, oracle_mod, B):
    import torch
    vec = _vec(oracle_mod, _params(13))
    basis = P.Basis(vec)
    pairs = _pairs(oracle_mod, B, 200 + B)
    g, loss = basis.pair_grad(torch.from_numpy(pairs).cuda())
    basis.sync()
    g = oracle_mod.unpack_params(g.cpu().numpy().astype(np.float64))
    p = _bf16_params(oracle_mod, vec)
    pd = pairs.astype(np.float64)
    lref, gref = oracle_mod.pair_loss_grad(p, pd[:, 0:2], pd[:, 2:4], pd[:, 4],
                                           hidden_round=oracle_mod.bf16_round)
    assert abs(loss.item() - lref) <= 1e-4 * lref + 1e-9
    for k in ("W1", "b1", "W2", "b2"):
        a, b = g[k].ravel(), gref[k].ravel()
        nb = np.linalg.norm(b)
        rel = np.linalg.norm(a - b) / nb
        cos = float(a @ b / (np.linalg.norm(a) * nb))
        assert rel <= 2e-2 and cos >= 0.999, (k, rel, cos)


def test_adam_step_matches_definition(P, oracle_mod):
    """Two Adam steps (Kingma & Ba, Algorithm 1, bias-corrected) from zero moments."""
    import torch
    vec = _vec(oracle_mod, _params(14))
    basis = P.Basis(vec)
    rng = np.random.default_rng(5)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    p = vec.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in (1, 2):
        g = rng.normal(size=p.shape).astype(np.float32)
        basis.adam_step(torch.from_numpy(g).cuda(), lr=lr, beta1=b1, beta2=b2, eps=eps)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g.astype(np.float64) ** 2
        p = p - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    got = basis.params().astype(np.float64)
    np.testing.assert_allclose(got, p, rtol=0, atol=1e-5)


def test_fit_reduces_pair_loss(P, oracle_mod):
    import torch
    vec = _vec(oracle_mod, _params(15, w2=0.05, b2=0.05))
    basis = P.Basis(vec)
    pairs = torch.from_numpy(_pairs(oracle_mod, 200000, 7)).cuda()
    rep = basis.fit(pairs, batch=4096, epochs=4, lr=2e-3)
    assert rep["steps"] == 4 * ((200000 + 4095) // 4096)
    assert rep["last_epoch_loss"] < 0.1 * rep["first_loss"], rep
    # the loss the device reports is the oracle's loss of the fitted model
    vec2 = basis.params()
    p = _bf16_params(oracle_mod, vec2)
    pd = pairs.cpu().numpy().astype(np.float64)[:5000]
    lref = oracle_mod.pair_loss(p, pd[:, 0:2], pd[:, 2:4], pd[:, 4],
                                hidden_round=oracle_mod.bf16_round)
    _, lg = basis.pair_grad(pairs[:5000])
    assert abs(lg.item() - lref) <= 1e-3 * lref + 1e-9

