"""Single-site circuit-DMRG compression with grouped qubits, complex128.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

This is the paper's own variant of the compression step (Sec. IV.A, IV.B.1,
V.C); the two-site variant lives in oracle/dmrg.py.

MPS (Sec. IV.A): m tensors M^(tau)[a, s, c]; tensor tau holds the r_tau qubits
of one group, consecutive sites of the chain order, and s runs over their
2^{r_tau} basis states with the group's first site the most significant bit.

Layer operator per group: W^(tau)[w, s, t, w'], the product of the per-site
MPO tensors of the group's sites (gates inside a group are absorbed into it,
Sec. IV.B.2); w, w' are the MPO bonds at the group's two ends.

One update (Sec. IV.B.1).  With every tensor but tau in orthogonal form
(left isometries before tau, right isometries after it),
  <Psi|U|Psi_Q> = Tr F^(tau) M^(tau)*                         (Eq. scalarproduct)
  F^(tau)[a, s, c] = sum L_tau[a, w, b] B^(tau)[b, t, b'] W^(tau)[w, s, t, w'] R_tau[c, w', b']
where L_tau (R_tau) contracts the conjugated new tensors, the layer operator
and the old tensors B of the groups left (right) of tau.  Under <Psi|Psi> = 1
the optimum is
  M^(tau) = F^(tau) / sqrt(f_tau),   f_tau = Tr F F*          (Eq. optimization)
and f_tau = |<Psi|U|Psi_Q>|^2 after the update, so f never decreases along a
sweep; the last f of the last sweep is f_delta (Eq. fa-sup).

Moving the orthogonality centre (Sec. IV.B.1 uses QR): after the update at
tau the sweep continues to tau +- 1 with M^(tau) replaced by an isometry
spanning the same space: moving right, the left singular vectors of
M[(a s), c]; moving left, the right singular vectors of M[a, (s c)].  Only
singular values above the numerical-zero level are kept (a direction M does
not use carries no weight, and its basis vector would be arbitrary), so a
rank-deficient M shrinks its bond.  The remaining factor is dropped: the
next update replaces the neighbouring tensor by its own F / sqrt(f).

Initial guess (Sec. V.D.1: an arbitrary random MPS): bonds
  chi_tau = min(chi, 2^{qubits left of the cut}, 2^{qubits right}, chi_old_tau * D_tau)
(D_tau the layer MPO's bond at the cut: U |Psi_Q> has no larger rank there);
entries (2u - 1) + i (2u' - 1) with u, u' consecutive SplitMix64 uniforms of
the given seed (counter-based, see random_guess); then brought to orthogonal
form with the centre on tensor 1 by LQ factorisations from the right, each
triangular factor carried into the tensor on its left (Sec. IV.B.1).

Sweeps: n_s sweeps over tau = 1..m, then m..1, alternating; every sweep
visits all m tensors (m updates per sweep, as the paper counts them).
"""
from __future__ import annotations

import numpy as np

from .dmrg import ZERO_REL, env_left, env_right

MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15


# --------------------------------------------------------------- group tensors


def group_mpo(w: list[np.ndarray], sizes: list[int]) -> list[np.ndarray]:
    """W^(tau)[w, s, t, w'] for consecutive groups of sites of the per-site
    MPO w (W_i[w, s, t, w'])."""
    assert sum(sizes) == len(w)
    out, p = [], 0
    for r in sizes:
        g = w[p]
        for j in range(1, r):
            x = w[p + j]
            d0, ds, dt, _ = g.shape
            g = np.einsum("wstv,vxyu->wsxtyu", g, x).reshape(d0, ds * 2, dt * 2, x.shape[3])
        out.append(g)
        p += r
    return out


def group_product_zero(sizes: list[int]) -> list[np.ndarray]:
    """|0...0> as group tensors [1, 2^r, 1]."""
    out = []
    for r in sizes:
        t = np.zeros((1, 2 ** r, 1), dtype=np.complex128)
        t[0, 0, 0] = 1.0
        out.append(t)
    return out


def group_dense(m: list[np.ndarray], sizes: list[int], order: list[int]) -> np.ndarray:
    """Contract the grouped MPS into the state tensor in qubit order."""
    t = np.ones((1,), dtype=np.complex128)
    for a in m:
        t = np.tensordot(t, a, axes=([t.ndim - 1], [0]))
    n = sum(sizes)
    t = t.reshape([2] * n)   # site order (s of a group: first site most significant)
    inv = [0] * n
    for i, q in enumerate(order):
        inv[q] = i
    return t.transpose([inv[q] for q in range(n)])


# ----------------------------------------------------------- random guess


def splitmix64_uniform_array(seed: int, counters: np.ndarray) -> np.ndarray:
    """splitmix64_uniform(seed, c) for an array of counters (uint64 arithmetic
    wraps modulo 2^64 as the generator requires)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (c + np.uint64(1)) * np.uint64(GOLDEN64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def random_guess(bonds: list[int], sizes: list[int], seed: int) -> list[np.ndarray]:
    """Tensors [bonds[tau], 2^r_tau, bonds[tau+1]] with entry e (row-major
    within tensor tau, after all entries of the tensors before it, counted
    as `off + e`) equal to (2u - 1) + i (2u' - 1), u = uniform(seed, 2(off+e)),
    u' = uniform(seed, 2(off+e) + 1)."""
    out, off = [], 0
    for tau, r in enumerate(sizes):
        shape = (bonds[tau], 2 ** r, bonds[tau + 1])
        cnt = int(np.prod(shape))
        e = np.arange(cnt, dtype=np.uint64) + np.uint64(off)
        re = 2.0 * splitmix64_uniform_array(seed, 2 * e) - 1.0
        im = 2.0 * splitmix64_uniform_array(seed, 2 * e + 1) - 1.0
        out.append((re + 1j * im).reshape(shape))
        off += cnt
    return out


def guess_bonds(sizes: list[int], chi: int, old_bonds: list[int], mpo_bonds: list[int]) -> list[int]:
    """chi_tau at every cut (m + 1 entries, 1 at both ends)."""
    n = sum(sizes)
    out, left = [1], 0
    for tau in range(len(sizes) - 1):
        left += sizes[tau]
        b = min(chi, 2 ** min(left, n - left), old_bonds[tau + 1] * mpo_bonds[tau + 1])
        out.append(max(1, b))
    out.append(1)
    return out


def lq_right_canonical(m: list[np.ndarray]) -> list[np.ndarray]:
    """Orthogonal form with the centre on tensor 0: for tau = m-1 .. 1,
    M^(tau)[a, (s c)] = Lo Q with orthonormal rows Q (QR of M^+), tensor tau
    becomes Q and Lo is carried into tensor tau - 1."""
    m = [t.copy() for t in m]
    for tau in range(len(m) - 1, 0, -1):
        a, s, c = m[tau].shape
        q, r = np.linalg.qr(m[tau].reshape(a, s * c).conj().T)   # M^+ = q r, M = r^+ q^+
        k = q.shape[1]
        m[tau] = q.conj().T.reshape(k, s, c)
        m[tau - 1] = np.einsum("asb,bk->ask", m[tau - 1], r.conj().T)
    return m


# ------------------------------------------------------------- contractions


def x_of(lenv: np.ndarray, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """X[a, s, w', b'] = sum L[a, w, b] B[b, t, b'] W[w, s, t, w'] (top-down,
    Sec. IV.B.2: the environment with the old tensor, then the operator)."""
    lb = np.einsum("awb,btc->awtc", lenv, b, optimize=True)
    return np.einsum("awtc,wsty->asyc", lb, w, optimize=True)


def y_of(renv: np.ndarray, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Y[s, c, w, b] = sum R[c, w', b'] B[b, t, b'] W[w, s, t, w'] (bottom-up)."""
    rb = np.einsum("cyd,btd->cybt", renv, b, optimize=True)
    return np.einsum("cybt,wsty->scwb", rb, w, optimize=True)


def f_tensor(x: np.ndarray, renv: np.ndarray) -> np.ndarray:
    """F^(tau)[a, s, c] = sum_{w', b'} X[a, s, w', b'] R[c, w', b']."""
    return np.einsum("asyd,cyd->asc", x, renv, optimize=True)


def zero_level_rank(s: np.ndarray, zero_rel: float) -> int:
    """Number of singular values above zero_rel * |s|_2 (at least 1)."""
    if s.size == 0 or s[0] == 0.0:
        return 1
    return max(1, int(np.sum(s > zero_rel * np.sqrt(np.sum(s ** 2)))))


# ------------------------------------------------------------------ the step


class SingleSiteResult:
    def __init__(self):
        self.f = []        # f_tau after every update, in order
        self.taus = []     # (sweep, tau) of every update
        self.bonds = []    # bonds of the new state at the end

    @property
    def f_delta(self) -> float:
        return self.f[-1]


def compress_layer(b: list[np.ndarray], wg: list[np.ndarray], sizes: list[int], chi: int,
                   n_sweeps: int, seed: int, zero_rel: float = ZERO_REL):
    """One compression step with single-tensor updates (Sec. IV.B.1).
    b: the old normalised grouped MPS; wg: the layer's group operators
    (group_mpo).  Returns (new tensors with the centre at the last updated
    tensor, SingleSiteResult, centre)."""
    m = len(b)
    res = SingleSiteResult()
    old_bonds = [1] + [t.shape[2] for t in b[:-1]] + [1]
    mpo_bonds = [1] + [t.shape[3] for t in wg[:-1]] + [1]
    bonds = guess_bonds(sizes, chi, old_bonds, mpo_bonds)
    a = lq_right_canonical(random_guess(bonds, sizes, seed))
    one = np.ones((1, 1, 1), dtype=np.complex128)
    lenv = [None] * (m + 1)
    renv = [None] * (m + 1)
    lenv[0], renv[m] = one, one
    for tau in range(m - 1, 0, -1):      # R_tau from the right-canonical guess
        renv[tau] = env_right(a[tau], y_of(renv[tau + 1], b[tau], wg[tau]))
    centre = 0
    for k in range(n_sweeps):
        right = k % 2 == 0
        taus = range(m) if right else range(m - 1, -1, -1)
        for tau in taus:
            x = x_of(lenv[tau], b[tau], wg[tau])
            f_t = f_tensor(x, renv[tau + 1])
            f = float(np.vdot(f_t, f_t).real)
            mt = f_t / np.sqrt(f)
            res.f.append(f)
            res.taus.append((k, tau))
            al, s, cr = mt.shape
            if right and tau < m - 1:
                u, sv, _ = np.linalg.svd(mt.reshape(al * s, cr), full_matrices=False)
                kk = zero_level_rank(sv, zero_rel)
                a[tau] = u[:, :kk].reshape(al, s, kk)
                lenv[tau + 1] = env_left(a[tau], x)
                centre = tau + 1
            elif not right and tau > 0:
                _, sv, vh = np.linalg.svd(mt.reshape(al, s * cr), full_matrices=False)
                kk = zero_level_rank(sv, zero_rel)
                a[tau] = vh[:kk].reshape(kk, s, cr)
                renv[tau] = env_right(a[tau], y_of(renv[tau + 1], b[tau], wg[tau]))
                centre = tau - 1
            else:
                a[tau] = mt
                centre = tau
    # the tensor at the centre is the last M; neighbours' stale shapes are fine
    res.bonds = [1] + [t.shape[2] for t in a[:-1]] + [1]
    return a, res, centre


def run_circuit(mpos: list[list[np.ndarray]], sizes: list[int], chi: int, n_sweeps: int, seed: int,
                **kw):
    """Open mode (Sec. IV.C) with single-site updates: layer delta uses the
    guess seed `seed + delta`.  Returns (final tensors, results, log F_tilde)."""
    mps = group_product_zero(sizes)
    results, log_ft = [], 0.0
    for d, w in enumerate(mpos):
        mps, res, _ = compress_layer(mps, group_mpo(w, sizes), sizes, chi, n_sweeps, seed + d, **kw)
        results.append(res)
        log_ft += np.log(res.f_delta)
    return mps, results, log_ft

