"""Layer MPO of K gate cycles, built gate by gate and compressed losslessly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper contracts the K layers of one compression step vertically and
merges one-qubit gates into neighbouring gates first (Sec. IV.B.2, "Contraction
strategy", Fig. 4).  The same object written as a matrix product operator over
the MPS sites: W_i[w, s, t, w'] with s the output (bra) index, t the input
(ket) index, and the operator O[s_1..s_N; t_1..t_N] = prod_i W_i.

Construction (plain): start from the identity MPO (bond 1); for each gate in
time order left-multiply it in.  A two-qubit gate on sites p < q is split by
an operator SVD, g = sum_k A_k (x) B_k (App. A, "splitting" a tensor by SVD);
A_k multiplies site p, B_k site q, and the bond index k passes through the
sites in between.  Finally the MPO is brought to left-canonical form (QR) and
truncated from the right by SVD at 1e-14 of the largest operator Schmidt
value at each cut, which drops only numerical zeros.

Site order: a snake along columns (down column 0, up column 1, ...), so
site -> qubit is order[site].
"""
from __future__ import annotations

import numpy as np


def snake_order(rows: int, cols: int) -> list[int]:
    """order[site] = qubit index q = r*cols + c, snake down the columns."""
    order = []
    for c in range(cols):
        rr = range(rows) if c % 2 == 0 else range(rows - 1, -1, -1)
        order += [r * cols + c for r in rr]
    return order


def chain_order(rows: int, cols: int, kind: str = "V") -> list[int]:
    """order[site] = qubit of the chain along which the MPS runs.
    V: the snake along columns (snake_order); H: the snake along rows (row 0
    left to right, row 1 right to left, ...); D: the anti-diagonals r + c = d
    in increasing d, each walked in increasing r for even d, decreasing for
    odd d.  Groups of consecutive columns, rows or diagonals (Sec. V.C,
    groupings V, H, D) are then runs of consecutive sites."""
    if kind == "V":
        return snake_order(rows, cols)
    order = []
    if kind == "H":
        for r in range(rows):
            cc = range(cols) if r % 2 == 0 else range(cols - 1, -1, -1)
            order += [r * cols + c for c in cc]
        return order
    if kind == "D":
        for d in range(rows + cols - 1):
            rr = list(range(max(0, d - cols + 1), min(rows - 1, d) + 1))
            if d % 2 == 1:
                rr.reverse()
            order += [r * cols + (d - r) for r in rr]
        return order
    raise ValueError(kind)


def identity_mpo(n: int) -> list[np.ndarray]:
    eye = np.eye(2, dtype=np.complex128).reshape(1, 2, 2, 1)
    return [eye.copy() for _ in range(n)]


def operator_split(u4: np.ndarray, rel_cut: float = 1e-14):
    """g[(s_p s_q),(t_p t_q)] = sum_k A_k[s_p,t_p] B_k[s_q,t_q] (App. A)."""
    g = np.asarray(u4, dtype=np.complex128).reshape(2, 2, 2, 2)  # s_p s_q t_p t_q
    m = g.transpose(0, 2, 1, 3).reshape(4, 4)                    # (s_p t_p),(s_q t_q)
    u, s, vh = np.linalg.svd(m)
    r = int(np.sum(s > rel_cut * s[0]))
    a = (u[:, :r] * np.sqrt(s[:r])).T.reshape(r, 2, 2)
    b = (np.sqrt(s[:r])[:, None] * vh[:r]).reshape(r, 2, 2)
    return a, b


def apply_gate_to_mpo(w: list[np.ndarray], sp: int, sq: int, u: np.ndarray) -> list[np.ndarray]:
    """Left-multiply one gate (given on sites sp, sq with sp the gate's first
    qubit) into the MPO.  Returns a new list."""
    w = list(w)
    u = np.asarray(u, dtype=np.complex128)
    if sq < 0:
        w[sp] = np.einsum("su,wutv->wstv", u, w[sp])
        return w
    if sp > sq:  # reorder the gate so that its first qubit is the left site
        u = u.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)
        sp, sq = sq, sp
    a, b = operator_split(u)
    r = a.shape[0]
    # site p: new right bond (w', k), k fastest
    t = np.einsum("ksu,wutv->wstvk", a, w[sp])
    d0, _, _, d1, _ = t.shape
    w[sp] = t.reshape(d0, 2, 2, d1 * r)
    for j in range(sp + 1, sq):
        x = w[j]
        d0, _, _, d1 = x.shape
        t = np.einsum("wstv,kl->wkstvl", x, np.eye(r))
        w[j] = t.reshape(d0 * r, 2, 2, d1 * r)
    t = np.einsum("ksu,wutv->wkstv", b, w[sq])
    d0, _, _, d1 = w[sq].shape
    w[sq] = t.reshape(d0 * r, 2, 2, d1)
    return w


def compress_mpo(w: list[np.ndarray], rel_cut: float = 1e-14) -> list[np.ndarray]:
    """Lossless compression: left-canonical QR sweep, then right-to-left SVD
    keeping operator Schmidt values above rel_cut * largest."""
    w = [x.copy() for x in w]
    n = len(w)
    for i in range(n - 1):
        d0, _, _, d1 = w[i].shape
        q, r = np.linalg.qr(w[i].reshape(d0 * 4, d1))
        k = q.shape[1]
        w[i] = q.reshape(d0, 2, 2, k)
        w[i + 1] = np.einsum("kv,vstw->kstw", r, w[i + 1])
    for i in range(n - 1, 0, -1):
        d0, _, _, d1 = w[i].shape
        u, s, vh = np.linalg.svd(w[i].reshape(d0, 4 * d1), full_matrices=False)
        k = int(np.sum(s > rel_cut * s[0]))
        w[i] = vh[:k].reshape(k, 2, 2, d1)
        w[i - 1] = np.einsum("wstv,vk->wstk", w[i - 1], u[:, :k] * s[:k])
    return w


def layer_mpo(layer, order: list[int], compress: bool = True) -> list[np.ndarray]:
    """MPO of one layer (gates in time order, qubit indices) over the sites."""
    n = len(order)
    site_of = {q: i for i, q in enumerate(order)}
    w = identity_mpo(n)
    for (q0, q1, u) in layer:
        if q1 < 0:
            w = apply_gate_to_mpo(w, site_of[q0], -1, u)
        else:
            w = apply_gate_to_mpo(w, site_of[q0], site_of[q1], u)
    return compress_mpo(w) if compress else w


def bond_dims(w: list[np.ndarray]) -> list[int]:
    return [x.shape[3] for x in w[:-1]]


def mpo_dense(w: list[np.ndarray], order: list[int]) -> np.ndarray:
    """Contract the MPO to a dense matrix in qubit order (qubit 0 MSB)."""
    n = len(w)
    t = w[0]  # [1, s, t, w]
    t = t.reshape(2, 2, -1)  # s0 t0 w
    for i in range(1, n):
        t = np.einsum("...w,wstv->...stv", t, w[i])
        t = t.reshape(t.shape[:-1] + (w[i].shape[3],))
    t = t.reshape([2, 2] * n)  # s0 t0 s1 t1 ... in site order
    s_axes = [2 * i for i in range(n)]
    t_axes = [2 * i + 1 for i in range(n)]
    # site i holds qubit order[i]; permute to qubit order
    inv = [0] * n
    for i, q in enumerate(order):
        inv[q] = i
    perm = [s_axes[inv[q]] for q in range(n)] + [t_axes[inv[q]] for q in range(n)]
    return t.transpose(perm).reshape(2 ** n, 2 ** n)
