"""Fourier basis of a radial pair weight on a periodic box (step P2 of the
CIA with the paper's Fourier modes, App. A.6, eq. Cucker_Smale_etaExpansion).

TEST INFRASTRUCTURE ONLY (part of the oracle package).

A pair weight g(d) = eta(||d||^2) of the difference d = s_l - s_m, for d in
the box [-L, L]^2, is expanded in the modes e^{i pi <alpha, d> / L}; the
coefficients are those of the periodic extension,

    c_alpha = (2L)^-2 int_{[-L,L]^2} g(d) e^{-i pi <alpha, d> / L} dd,

approximated by the rectangle rule on a G x G grid (an FFT).  Because g is
even and real, c_alpha = c_-alpha is real and

    g(s_l - s_m) ~ sum_alpha c_alpha cos(pi <alpha, s_l - s_m> / L)
                 = sum_alpha c_alpha [cos a_l cos a_m + sin a_l sin a_m],

a_l = pi <alpha, s_l> / L: with c_alpha >= 0 the real features
sqrt(c_alpha) (cos a, sin a) separate the pair as phi(s_l) . phi(s_m).
"""
from __future__ import annotations

import numpy as np


def fourier_coefficients(g2, L: float, grid: int = 256) -> tuple[np.ndarray, np.ndarray]:
    """Coefficients of the even real function g2(d_x, d_y) on the grid:
    (alpha [G*G, 2] ints, c [G*G] real)."""
    G = int(grid)
    x = -L + 2.0 * L * np.arange(G) / G
    X, Y = np.meshgrid(x, x, indexing="ij")
    g = g2(X, Y)
    F = np.fft.fft2(g) / (G * G)
    k = np.fft.fftfreq(G, d=1.0 / G).astype(np.int64)     # 0, 1, ..., -1
    A1, A2 = np.meshgrid(k, k, indexing="ij")
    # the grid starts at -L: e^{-i pi alpha x_j / L} = (-1)^alpha e^{-2 pi i alpha j / G}
    c = (F * ((-1.0) ** (A1 + A2))).real
    alpha = np.stack([A1.ravel(), A2.ravel()], axis=1)
    return alpha, c.ravel()


def radial(eta):
    """g2(d_x, d_y) = eta(d_x^2 + d_y^2)."""
    return lambda X, Y: eta(X * X + Y * Y)


def fourier_basis(g2, L: float, rank: int, grid: int = 256):
    """The modes with the largest coefficients, one per pair +-alpha, such that
    the real feature count (2 per mode, 1 for alpha = 0) is at most `rank`.
    Returns (alpha [K, 2], c [K]) with c > 0."""
    alpha, c = fourier_coefficients(g2, L, grid)
    # one representative per +-alpha: the first nonzero component positive
    rep = (alpha[:, 0] > 0) | ((alpha[:, 0] == 0) & (alpha[:, 1] >= 0))
    a, cc = alpha[rep], c[rep]
    order = np.argsort(-cc, kind="stable")
    chosen, used = [], 0
    for i in order:
        if cc[i] <= 0:
            break
        need = 1 if (a[i] == 0).all() else 2
        if used + need > rank:
            continue
        chosen.append(i)
        used += need
    return a[chosen], cc[chosen]


def fourier_features(s: np.ndarray, alpha: np.ndarray, c: np.ndarray, L: float) -> np.ndarray:
    """phi(s) [B, R]: for each mode sqrt(c) cos a and (unless alpha = 0)
    sqrt(c) sin a with a = pi <alpha, s> / L.  For alpha != 0 the coefficient
    counts for both +alpha and -alpha, hence the factor sqrt(2 c)."""
    s = np.asarray(s, dtype=np.float64)
    cols = []
    for (a1, a2), ca in zip(alpha, c):
        arg = np.pi * (a1 * s[:, 0] + a2 * s[:, 1]) / L
        if a1 == 0 and a2 == 0:
            cols.append(np.sqrt(ca) * np.ones(len(s)))
        else:
            w = np.sqrt(2.0 * ca)
            cols.append(w * np.cos(arg))
            cols.append(w * np.sin(arg))
    return np.stack(cols, axis=1) if cols else np.zeros((len(s), 0))
