"""FP64 forward and backward of the learned separable Cucker--Smale basis.

TEST INFRASTRUCTURE ONLY (part of the oracle package).

The Cucker--Smale weight eta(||s_l - s_m||^2) = K (sigma^2 + ||s_l - s_m||^2)^-beta
(eq. Cucker_Smale, App. A.6) is approximated by a rank-R separable form
phi(s_l) . phi(s_m), which plays the role of the Fourier expansion of step P2
(eq. Cucker_Smale_etaExpansion): the paper only needs *some* basis that
separates the l and m parts (Sec. 3.3).  The feature map is a two-layer
perceptron

    phi(x) = W2 sin(W1 x + b1) + b2,     W1: [H, 2], W2: [R, H]

(act="silu" gives the SiLU variant z / (1 + e^-z) instead of sin.)

evaluated on positions x relative to a shift common to the community.  It is
fitted by least squares on pairs:

    L = (1/B) sum_b (eta_b - phi(a_b) . phi(c_b))^2.

Everything here is plain numpy in float64; matrix products are the only
library primitive used.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round to the nearest bfloat16 value, ties to even (the 8-bit-significand
    format the tensor cores read), returned as float64.  Values are first
    rounded to float32, as the device holds them."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack_params(vec) -> dict:
    """Split a packed parameter vector (W1 [H, 2], b1 [H], W2 [R, H], b2 [R],
    in that order, H = 128, R = 64) into arrays of float64."""
    v = np.asarray(vec, dtype=np.float64)
    H, R = 128, 64
    o1 = 2 * H
    o2 = o1 + H
    o3 = o2 + R * H
    assert v.shape == (o3 + R,)
    return {"W1": v[:o1].reshape(H, 2), "b1": v[o1:o2], "W2": v[o2:o3].reshape(R, H),
            "b2": v[o3:]}


def pack_params(p: dict) -> np.ndarray:
    return np.concatenate([p["W1"].reshape(-1), p["b1"], p["W2"].reshape(-1), p["b2"]])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def cs_kernel_weight(d2, K=1.0, sigma=1.0, beta=0.4):
    """eta(y) = K / (sigma^2 + y)^beta with y = squared distance."""
    return K * np.power(sigma * sigma + np.asarray(d2, dtype=np.float64), -beta)


ACTS = {"sin": (np.sin, np.cos)}


def mlp_forward(params: dict, x: np.ndarray, hidden_round=None, act: str = "sin"):
    """phi(x) for x of shape [B, 2]; returns (phi [B, R], cache).

    hidden_round, if given, is applied to the hidden activations before the
    second layer (a quantisation step that is part of the evaluated model).
    """
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ params["W1"].T + params["b1"]
    a1 = silu(z1) if act == "silu" else ACTS[act][0](z1)
    if hidden_round is not None:
        a1 = hidden_round(a1)
    out = a1 @ params["W2"].T + params["b2"]
    return out, {"x": x, "z1": z1, "a1": a1, "act": act}


def mlp_backward(params: dict, cache: dict, dout: np.ndarray) -> dict:
    """Gradients of sum(dout * phi) with respect to W1, b1, W2, b2."""
    a1, z1, x = cache["a1"], cache["z1"], cache["x"]
    dW2 = dout.T @ a1
    db2 = dout.sum(axis=0)
    da1 = dout @ params["W2"]
    dz1 = da1 * (silu_grad(z1) if cache["act"] == "silu" else ACTS[cache["act"]][1](z1))
    dW1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return {"W1": dW1, "b1": db1, "W2": dW2, "b2": db2}


def pair_loss(params: dict, a: np.ndarray, c: np.ndarray, target: np.ndarray,
              hidden_round=None, act: str = "sin") -> float:
    """(1/B) sum_b (target_b - phi(a_b) . phi(c_b))^2."""
    fa, _ = mlp_forward(params, a, hidden_round, act)
    fc, _ = mlp_forward(params, c, hidden_round, act)
    e = (fa * fc).sum(axis=1) - target
    return float((e * e).mean())


def pair_loss_grad(params: dict, a: np.ndarray, c: np.ndarray, target: np.ndarray,
                   hidden_round=None, act: str = "sin"):
    """Loss and its gradient (both inputs share the weights: tied features)."""
    fa, ca = mlp_forward(params, a, hidden_round, act)
    fc, cc = mlp_forward(params, c, hidden_round, act)
    B = len(target)
    e = (fa * fc).sum(axis=1) - target
    loss = float((e * e).mean())
    g = 2.0 / B * e
    ga = mlp_backward(params, ca, g[:, None] * fc)
    gc = mlp_backward(params, cc, g[:, None] * fa)
    grads = {k: ga[k] + gc[k] for k in ga}
    return loss, grads
