"""Trigonometric density initialisation (FP64). TEST INFRASTRUCTURE ONLY (see the package
header).

Sec. 6.2: basis T_n = {cos(2 pi k xb_i), sin(2 pi k xb_i) : 0 < k <= n, i = 0, 1, 2} at the
element centres, xb = R_q (x - b), b = (1/2, 1/2, 1/2), R_q the rotation of a normalised
quaternion q; Q_n = T_n together with the products of two members of T_n; random weights
in [-1, 1] (inputs here) weight Q_n; the sum y is projected by the rescaled sigmoid
S(y) = rho_min + V^ / (1 + exp(-k (y - mu))), k = 15, V^ = min(1.5 V, 1), with mu such
that the mean density is V.

Readings (the text leaves these open): the quaternion is scalar-first (q0 + q1 i + q2 j +
q3 k); "products of any two items" are the unordered pairs including squares, ordered
(a, b) with a <= b in the order of T_n, which is cos before sin, then k = 1..n, then axis
i = 0..2 innermost, i.e. T index = 2 (3 (k - 1) + i) + (0 for cos, 1 for sin); S is
clamped to [rho_min, 1] (rho_min + V^ exceeds 1 once V >= 2/3); mu is found by bisection.
"""
from __future__ import annotations

import numpy as np


def quaternion_rotation(q) -> np.ndarray:
    """3x3 rotation of the normalised scalar-first quaternion q."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def basis_count(nb: int) -> int:
    t = 6 * nb
    return t + t * (t + 1) // 2


def trig_basis(n: int, nb: int, q) -> np.ndarray:
    """(N, |Q_n|) basis values at the element centres (x fastest)."""
    c = (np.arange(n) + 0.5) / n
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    X = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1) - 0.5
    Xb = X @ quaternion_rotation(q).T
    T = []
    for k in range(1, nb + 1):
        for i in range(3):
            T.append(np.cos(2 * np.pi * k * Xb[:, i]))
            T.append(np.sin(2 * np.pi * k * Xb[:, i]))
    T = np.stack(T, axis=1)
    P = [T[:, a] * T[:, b] for a in range(T.shape[1]) for b in range(a, T.shape[1])]
    return np.concatenate([T, np.stack(P, axis=1)], axis=1)


def sigmoid_projection(y: np.ndarray, V: float, rho_min: float = 1e-3, k: float = 15.0):
    """(rho, mu): rho = clamp(rho_min + Vh / (1 + exp(-k (y - mu))), rho_min, 1) with mu
    bisected so that mean(rho) = V (mean decreasing in mu)."""
    Vh = min(1.5 * V, 1.0)
    y = np.asarray(y, dtype=np.float64)

    def rho_of(mu):
        return np.clip(rho_min + Vh / (1.0 + np.exp(-k * (y - mu))), rho_min, 1.0)
    lo, hi = y.min() - 60.0 / k, y.max() + 60.0 / k
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if rho_of(mid).mean() > V:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return rho_of(mu), mu


def trig_initialization(n: int, nb: int, q, weights, V: float, rho_min: float = 1e-3) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    if w.size != basis_count(nb):
        raise ValueError("one weight per member of Q_n")
    y = trig_basis(n, nb, q) @ w
    return sigmoid_projection(y, V, rho_min)[0]
