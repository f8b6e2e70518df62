"""Randomized truncated SVD and its acceptance certificate, in float64.

Test infrastructure only (see oracle/__init__.py).  Not in the paper: the
library can replace the sweep's exact truncated SVD of theta by the range
finder of Halko, Martinsson and Tropp (SIAM Rev. 53, 2011, Alg. 4.4 with q
power iterations) and accepts the result only when a bound shows it is within
a tolerance of the optimal update.  This module states that bound so tests
can check it on matrices whose SVD is known.

Bound (Ky Fan): with Q orthonormal and B = Q^+ G,
    G^+ G = B^+ B + G^+ (I - Q Q^+) G,
both terms positive semidefinite, so the sum of the k largest eigenvalues of
G^+ G (the best weight f_opt(k) of a rank-k truncation of G) is at most the
sum of the k largest of B^+ B plus the trace of the rest,
|G|_F^2 - |B|_F^2.
"""
from __future__ import annotations

import numpy as np


def range_finder(g: np.ndarray, l: int, q: int, rng: np.random.Generator) -> np.ndarray:
    """Orthonormal basis Q (m x l') of the range of G Omega after q power
    iterations with re-orthonormalisation (directions of zero weight dropped)."""
    def orth(y):
        u, s, _ = np.linalg.svd(y, full_matrices=False)
        keep = s > 1e-13 * max(s[0], 1e-300) if s.size else s.astype(bool)
        return u[:, keep]
    n = g.shape[1]
    omega = (rng.normal(size=(n, l)) + 1j * rng.normal(size=(n, l))) / np.sqrt(2.0)
    qm = orth(g @ omega)
    for _ in range(q):
        z = orth(g.conj().T @ qm)
        qm = orth(g @ z)
    return qm


def sketch_svd(g: np.ndarray, qm: np.ndarray, chi: int, rel_cut: float):
    """Truncated SVD of G from the sketch: U_k = Q W_k, s_k, with k <= chi
    values above rel_cut * s_1 of B = Q^+ G.  Returns (U_k, s_k, s_all)."""
    b = qm.conj().T @ g
    w, s, _ = np.linalg.svd(b, full_matrices=False)
    k = int(min(chi, np.sum(s > rel_cut * s[0])))
    return qm @ w[:, :k], s[:k], s


def certificate_excess(g: np.ndarray, s_all: np.ndarray, k: int, chi: int) -> float:
    """Upper bound of f_opt - f over the truncations the sweep could choose
    (at most chi values), where f = sum of the k kept s^2 of the sketch:
    |G|^2 - |B|^2 (the weight outside the sketch) plus, when k < chi, the
    sketch's dropped weight."""
    fro = float(np.sum(np.abs(g) ** 2))
    trh = float(np.sum(s_all ** 2))
    f = float(np.sum(s_all[:k] ** 2))
    return (fro - trh) + (trh - f if k < chi else 0.0)
