"""Rank model of the learned truncated SVD: plain definitions in float64.

Test infrastructure only (see oracle/__init__.py).  Nothing here is in the
paper: the paper truncates with an exact SVD.  The randomized SVD that the
learned mode drives follows Halko, Martinsson and Tropp (SIAM Rev. 53, 2011);
these functions define what the model reads and predicts and the network
itself, so the library's records, forward pass and gradients can be checked.

Parameter layout (FP32 in the library, float64 here): W1 [H][IN] row-major,
b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1].
"""
from __future__ import annotations

import numpy as np

IN = 36
HID = 128
NPARAM = HID * IN + HID + HID * HID + HID + HID + 1
LABEL_FRAC = 1.0 - 1e-6


def spectrum_summary(s_kept: np.ndarray) -> np.ndarray:
    """32 samples of log10(s_mu^2 / sum s^2) of a kept spectrum (descending),
    at mu_j = round(j (k-1) / 31) (round half to even); -30 for a zero ratio."""
    s = np.asarray(s_kept, dtype=np.float64)
    k = s.size
    tot = float(np.sum(s * s))
    out = np.empty(32)
    for j in range(32):
        mu = int(np.rint(j * (k - 1) / 31.0)) if k > 1 else 0
        q = s[mu] ** 2 / tot if tot > 0 else 0.0
        out[j] = np.log10(q) if q > 1e-30 else -30.0
    return out


def rank_label(s_kept: np.ndarray, frac: float = LABEL_FRAC) -> int:
    """Smallest r with sum_{mu<r} s_mu^2 >= frac * sum_{mu<k} s_mu^2."""
    w = np.asarray(s_kept, dtype=np.float64) ** 2
    tot = float(np.sum(w))
    run = 0.0
    for r, x in enumerate(w, start=1):
        run += x
        if run >= frac * tot:
            return r
    return w.size


def model_input(prev_kept: np.ndarray, mpo_bond: int, theta_min_side: int, visited_in_layer: bool) -> np.ndarray:
    """The 36 inputs for an update at a bond: the previous kept spectrum's
    summary, log2 of its length, log2 of the MPO bond dimension, log2 of the
    smaller side of theta, and whether the bond was updated in this layer."""
    x = np.empty(IN)
    x[:32] = spectrum_summary(prev_kept)
    x[32] = np.log2(max(len(prev_kept), 1))
    x[33] = np.log2(max(mpo_bond, 1))
    x[34] = np.log2(max(theta_min_side, 1))
    x[35] = 1.0 if visited_in_layer else 0.0
    return x


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    w1 = p[o:o + HID * IN].reshape(HID, IN); o += HID * IN
    b1 = p[o:o + HID]; o += HID
    w2 = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = p[o:o + HID]; o += HID
    w3 = p[o:o + HID]; o += HID
    b3 = p[o]
    return w1, b1, w2, b2, w3, b3


def forward(p: np.ndarray, x: np.ndarray) -> np.ndarray:
    """f(x) = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, rows of x."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    h1 = np.maximum(x @ w1.T + b1, 0.0)
    h2 = np.maximum(h1 @ w2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_grad(p: np.ndarray, x: np.ndarray, y: np.ndarray):
    """L = (1/n) sum (f(x) - y)^2 and dL/dp by the chain rule (backpropagation)."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    n = x.shape[0]
    z1 = x @ w1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0.0)
    f = h2 @ w3 + b3
    r = f - y
    loss = float(np.mean(r * r))
    df = 2.0 * r / n                      # dL/df
    g_w3 = h2.T @ df
    g_b3 = np.sum(df)
    dz2 = np.outer(df, w3) * (z2 > 0)     # dL/dz2
    g_w2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w2) * (z1 > 0)
    g_w1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    grad = np.concatenate([g_w1.ravel(), g_b1, g_w2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, grad


def expected_records(layer_results, mpo_bonds_per_layer):
    """The (input, label) records a logging run makes, from the oracle's own
    per-update spectra: one per update at a bond that was updated before (in
    this or an earlier layer), label log2 of rank_label of the kept spectrum.
    `mpo_bonds_per_layer[l][i]` is the MPO bond dimension between sites i and
    i+1 in layer l."""
    last = {}
    xs, ys = [], []
    for li, res in enumerate(layer_results):
        seen = set()
        for (pass_id, i), full, k in zip(res.bonds, res.spectra, res.kept):
            kept = np.asarray(full)[:k]
            if i in last:
                xs.append(model_input(last[i], mpo_bonds_per_layer[li][i], len(full), i in seen))
                ys.append(np.log2(max(rank_label(kept), 1)))
            last[i] = kept
            seen.add(i)
    return np.array(xs).reshape(-1, IN), np.array(ys)
