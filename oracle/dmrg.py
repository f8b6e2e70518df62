"""Two-site circuit-DMRG compression step, complex128, step by step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. IV.B: given the normalised MPS |Psi_Q(D)> (tensors B_i) and the layer
operator U (MPO W_i), find the normalised MPS |Psi> of bond <= chi that
maximises |<Psi|U|Psi_Q(D)>|^2, optimising a block of tensors at a time while
the rest stay fixed, and sweeping over the blocks.

With the rest of |Psi> in orthogonal form (Sec. IV.B.1), the overlap is linear
in the optimised block: <Psi|U|Psi_Q> = Tr F M* (Eq. scalarproduct), and the
constrained optimum is M = F / sqrt(f) with f = Tr F F* the partial fidelity
(Eq. optimization).  The paper optimises one grouped tensor at a time and
mentions the two-site variant (Sec. IV.B); this oracle follows the two-site
variant with one qubit per site:

* F becomes the two-site tensor theta[(a s1), (s2 c)] at bond (i, i+1),
  theta = X_i . Y_{i+1} with X_i = L_{i-1} B_i W_i and Y_{i+1} = R_{i+2} B_{i+1} W_{i+1}
  (the top-down / bottom-up contraction of Sec. IV.B.2 meeting at the bond).
* The bond-chi constraint makes the optimum the truncated SVD of theta
  (Eckart-Young): keep k = min(chi, #{s_mu > cut * s_1}) values;
  left-to-right: A_i = U_k, A_{i+1} = S_k V_k^+ / |S_k|;
  right-to-left: A_{i+1} = V_k^+, A_i = U_k S_k / |S_k|.
  Then <Psi|U|Psi_Q> = |S_k| is real and positive, which fixes the phase,
  and f = sum_{mu<=k} s_mu^2 is the partial fidelity after the update.
* f is non-decreasing along the sweep (Sec. IV.B.1), and the f of the last
  update of the last sweep is f_delta (Eq. fa-sup); F_tilde = prod f_delta
  (Eq. Ftilde-sup).

Initial guess (the paper uses a random MPS or a TEBD-like start, Sec. V.D.1):
a zip-up of W.B from both ends towards the centre site m = N // 2.  At a site
whose matrix has r <= chi rows the full row space is kept with the identity
basis (no truncation, no SVD); otherwise the top left singular vectors with
s_mu > zip_cut * s_1, at most chi, never splitting a degenerate multiplet.
The guess is therefore exact whenever chi >= 2^{max(m, N-m-1)}, i.e.
chi >= 2^{N/2}.  It depends on the gauge of the MPO bond (the remainder it
truncates against is not orthonormal), so a comparison of two implementations
must give both the same MPO up to a unitary gauge per bond.

Sweep schedule, 2(N-1) two-site updates per layer (n_s = 2 one-direction
sweeps): bonds (m-1,m) .. (0,1) right-to-left, then (0,1) .. (N-2,N-1)
left-to-right, then (N-2,N-1) .. (m,m+1) right-to-left.  The state starts and
ends with its orthogonality centre on site m; sites < m are left-canonical,
sites > m right-canonical.

Tensor layouts: MPS A_i[a, s, b]; MPO W_i[w, s, t, w']; left environment
L_i[a_new, w, b_old]; right environment R_i[c_new, w, b_old];
X_i[a, s, w', b'] ; Y_i[s, c, w, b] (w, b the bonds on the left of site i).
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------- contractions


def make_x(lenv: np.ndarray, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """X[a, s, y, c] = sum_{w,b,t} L[a,w,b] B[b,t,c] W[w,s,t,y], contracted
    top-down as in Sec. IV.B.2: the environment with the old tensor first,
    then the layer operator."""
    lb = np.einsum("awb,btc->awtc", lenv, b, optimize=True)
    return np.einsum("awtc,wsty->asyc", lb, w, optimize=True)


def make_y(renv: np.ndarray, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Y[s, c, y, a] = sum_{w,b,t} R[c,w,b] B[a,t,b] W[y,s,t,w], contracted
    bottom-up (Sec. IV.B.2): the environment with the old tensor first, then
    the layer operator."""
    rb = np.einsum("cwb,atb->cwat", renv, b, optimize=True)
    return np.einsum("cwat,ystw->scya", rb, w, optimize=True)


def theta_of(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """theta[(a s1), (s2 c)] = sum_{w,b} X[a,s1,w,b] Y[s2,c,w,b] (Eq. scalarproduct)."""
    a, s1, wd, bd = x.shape
    s2, c, _, _ = y.shape
    return x.reshape(a * s1, wd * bd) @ y.reshape(s2 * c, wd * bd).T


def env_left(a_new: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L_i[k, w, b] = sum_{a,s} conj(A[a,s,k]) X[a,s,w,b]."""
    return np.einsum("ask,aswb->kwb", a_new.conj(), x, optimize=True)


def env_right(a_new: np.ndarray, y: np.ndarray) -> np.ndarray:
    """R_i[k, w, b] = sum_{s,c} conj(A[k,s,c]) Y[s,c,w,b]."""
    return np.einsum("ksc,scwb->kwb", a_new.conj(), y, optimize=True)


def truncation_rank(s: np.ndarray, chi: int, rel_cut: float, floor: float = 0.0) -> int:
    """k = min(chi, #{s_mu > max(rel_cut * s_1, floor)}), at least 1."""
    if s.size == 0 or s[0] == 0.0:
        return 1
    return max(1, min(chi, int(np.sum(s > max(rel_cut * s[0], floor)))))


# Numerical-zero level of a singular value relative to |theta|_F in complex128
# arithmetic: directions below it carry no information and are never kept.
ZERO_REL = 1e-13


def svd_truncate(theta: np.ndarray, chi: int, rel_cut: float, zero_rel: float = ZERO_REL):
    """Truncated SVD of theta: (U_k, s_k, Vh_k), LAPACK complex128.  Keeps
    s_mu > max(rel_cut * s_1, zero_rel * |theta|_F), at most chi."""
    u, s, vh = np.linalg.svd(theta, full_matrices=False)
    k = truncation_rank(s, chi, rel_cut, zero_rel * np.sqrt(np.sum(s ** 2)))
    return u[:, :k], s[:k], vh[:k], s


# ------------------------------------------------------------------ the step


class LayerResult:
    def __init__(self):
        self.f = []          # partial fidelity after every update, in order
        self.kept = []       # kept rank k after every update
        self.bonds = []      # (pass, i) of every update
        self.spectra = []    # full singular spectrum of every theta
        self.guess_overlap = 0.0
        self.zip_ambiguous = False  # a zip-up cut fell in a multiplet reaching s_1
        self.records = {}    # optional snapshots keyed by (pass, i)

    @property
    def f_delta(self) -> float:
        return self.f[-1] if self.f else self.guess_overlap ** 2


ZIP_AMBIGUOUS: list = []   # rows of zip-up cuts that fell in a multiplet reaching s_1


def zip_matrix_basis(mat: np.ndarray, chi: int, zip_cut: float, tie_cut: float = 1e-10,
                     zero_rel: float = ZERO_REL):
    """Left basis kept by the zip-up for a matrix with r rows: the identity if
    r <= chi, else the top-k left singular vectors (s_mu > zip_cut * s_1).
    If the cut at chi falls inside a degenerate multiplet (s_k - s_{k+1} <=
    tie_cut * s_1) the whole multiplet is dropped, so that the kept subspace,
    and with it the guess, is unique."""
    r = mat.shape[0]
    if r <= chi:
        return np.eye(r, dtype=np.complex128)
    u, s, _ = np.linalg.svd(mat, full_matrices=False)
    # floor: s^2 above zero_rel times the Frobenius norm of the Gram matrix M M^+
    floor = np.sqrt(zero_rel * np.sqrt(np.sum(s ** 4)))
    k = truncation_rank(s, chi, zip_cut, floor)
    if k < s.size and s[k] > max(zip_cut * s[0], floor) and s[k - 1] - s[k] <= tie_cut * s[0]:
        kk = k
        while kk > 1 and s[kk - 1] - s[kk] <= tie_cut * s[0]:
            kk -= 1
        if kk == 1 and s[0] - s[1] <= tie_cut * s[0]:
            ZIP_AMBIGUOUS.append(r)   # the multiplet reaches s_1: cut kept at chi
        else:
            k = kk
    return u[:, :k]


def compress_layer(b: list[np.ndarray], w: list[np.ndarray], chi: int,
                   sweep_cut: float = 1e-12, zip_cut: float = 1e-5, tie_cut: float = 1e-10,
                   zero_rel: float = ZERO_REL, record: set | None = None):
    """One compression step (Sec. IV.B): returns (new MPS tensors, LayerResult)."""
    n = len(b)
    m = n // 2
    res = LayerResult()
    ZIP_AMBIGUOUS.clear()
    a = [None] * n
    xs = [None] * n   # X_i, valid for sites left of the current bond
    ys = [None] * n   # Y_i, valid for sites right of the current bond

    # --- zip-up guess, left part
    lenv = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(m):
        x = make_x(lenv, b[i], w[i])
        xs[i] = x
        al, s, wd, bd = x.shape
        mat = x.reshape(al * s, wd * bd)
        basis = zip_matrix_basis(mat, chi, zip_cut, tie_cut, zero_rel)
        a[i] = basis.reshape(al, 2, basis.shape[1])
        lenv = env_left(a[i], x)
    # --- zip-up guess, right part
    renv = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(n - 1, m, -1):
        y = make_y(renv, b[i], w[i])
        ys[i] = y
        s, cr, wd, bd = y.shape
        mat = y.reshape(s * cr, wd * bd)
        basis = zip_matrix_basis(mat, chi, zip_cut, tie_cut, zero_rel)
        a[i] = basis.T.reshape(basis.shape[1], 2, cr)
        renv = env_right(a[i], y)
    res.zip_ambiguous = len(ZIP_AMBIGUOUS) > 0
    # --- centre
    xm = make_x(lenv, b[m], w[m])
    xs[m] = xm
    centre = np.einsum("asyc,dyc->asd", xm, renv, optimize=True)
    nrm = np.linalg.norm(centre)
    res.guess_overlap = float(nrm)
    a[m] = centre / nrm
    r_right = renv  # R_{m+1}

    def update(pass_id, i, x, y, left_to_right):
        th = theta_of(x, y)
        u, s, vh, full = svd_truncate(th, chi, sweep_cut, zero_rel)
        k = s.size
        nrm_s = np.linalg.norm(s)
        al = x.shape[0]
        cr = y.shape[1]
        if left_to_right:
            a[i] = u.reshape(al, 2, k)
            a[i + 1] = ((s[:, None] * vh) / nrm_s).reshape(k, 2, cr)
        else:
            a[i + 1] = vh.reshape(k, 2, cr)
            a[i] = ((u * s[None, :]) / nrm_s).reshape(al, 2, k)
        res.f.append(float(nrm_s ** 2))
        res.kept.append(k)
        res.bonds.append((pass_id, i))
        res.spectra.append(full)
        if record is not None and (pass_id, i) in record:
            res.records[(pass_id, i)] = {"theta": th.copy(),
                                         "mps_before": None}

    # --- pass 1: (m-1, m) .. (0, 1), right to left
    renv = r_right
    for i in range(m - 1, -1, -1):
        y = make_y(renv, b[i + 1], w[i + 1])
        ys[i + 1] = y
        if record is not None and (1, i) in record:
            snap = [t.copy() if t is not None else None for t in a]
        update(1, i, xs[i], y, left_to_right=False)
        if record is not None and (1, i) in record:
            res.records[(1, i)]["mps_before"] = snap
        renv = env_right(a[i + 1], y)
    # --- pass 2: (0, 1) .. (n-2, n-1), left to right
    lenv = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(0, n - 1):
        x = make_x(lenv, b[i], w[i])
        xs[i] = x
        if record is not None and (2, i) in record:
            snap = [t.copy() if t is not None else None for t in a]
        update(2, i, x, ys[i + 1], left_to_right=True)
        if record is not None and (2, i) in record:
            res.records[(2, i)]["mps_before"] = snap
        lenv = env_left(a[i], x)
    # --- pass 3: (n-2, n-1) .. (m, m+1), right to left
    renv = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(n - 2, m - 1, -1):
        y = make_y(renv, b[i + 1], w[i + 1])
        ys[i + 1] = y
        update(3, i, xs[i], y, left_to_right=False)
        renv = env_right(a[i + 1], y)
    return a, res


# ----------------------------------------------------------- whole circuits


def product_state(n: int) -> list[np.ndarray]:
    """|0...0> as an MPS of bond 1."""
    t = np.zeros((1, 2, 1), dtype=np.complex128)
    t[0, 0, 0] = 1.0
    return [t.copy() for _ in range(n)]


def run_circuit(mpos: list[list[np.ndarray]], n: int, chi: int, **kw):
    """Open mode (Sec. IV.C): one compression step per layer.
    Returns (final MPS, list of LayerResult, log F_tilde)."""
    mps = product_state(n)
    results = []
    log_ft = 0.0
    for w in mpos:
        mps, res = compress_layer(mps, w, chi, **kw)
        results.append(res)
        log_ft += np.log(res.f_delta)
    return mps, results, log_ft


# ----------------------------------------------------------- read-outs


def mps_dense(a: list[np.ndarray], order: list[int]) -> np.ndarray:
    """Contract the MPS into a state tensor in qubit order."""
    t = a[0].reshape(2, -1)
    for i in range(1, len(a)):
        t = np.einsum("...a,asb->...sb", t, a[i])
    t = t.reshape([2] * len(a))
    inv = [0] * len(a)
    for i, q in enumerate(order):
        inv[q] = i
    return t.transpose([inv[q] for q in range(len(a))])


def amplitude(a: list[np.ndarray], order: list[int], bits_qubit_order) -> complex:
    """<x|Psi> = prod_i A_i[:, x_i, :] (the MPS definition, Sec. IV.A)."""
    v = np.ones((1,), dtype=np.complex128)
    for i, q in enumerate(order):
        v = v @ a[i][:, int(bits_qubit_order[q]), :]
    return complex(v[0])


MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15


def splitmix64_uniform(seed: int, counter: int) -> float:
    """The (counter+1)-th output of SplitMix64 seeded with `seed` (Steele, Lea,
    Flood 2014), mapped to [0, 1) with 53 bits.  Counter-based: state =
    seed + (counter+1) * golden gamma."""
    z = (seed + (counter + 1) * GOLDEN64) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    z = z ^ (z >> 31)
    return (z >> 11) * (1.0 / 9007199254740992.0)


def right_norm_matrices(a: list[np.ndarray], centre: int) -> list[np.ndarray]:
    """E_i = norm matrix of sites > i: identity for i >= centre (those sites are
    right-canonical), E_i = sum_s A_{i+1}[s] E_{i+1} A_{i+1}[s]^+ below."""
    n = len(a)
    e = [None] * n
    for i in range(n - 1, -1, -1):
        if i >= centre:
            e[i] = np.eye(a[i].shape[2], dtype=np.complex128)
        else:
            nxt = a[i + 1]
            e[i] = sum(nxt[:, s, :] @ e[i + 1] @ nxt[:, s, :].conj().T for s in range(2))
    return e


def sample(a: list[np.ndarray], order: list[int], centre: int, count: int, seed: int) -> np.ndarray:
    """Sequential conditional sampling of bitstrings from the MPS.
    p(x_i | x_<i) from v E_i v^+ with v = A_0[x_0]...A_i[x_i]; bit i of sample j
    is 0 iff u(seed, j*N + i) < p(0 | prefix).  Output in qubit order."""
    n = len(a)
    e = right_norm_matrices(a, centre)
    out = np.zeros((count, n), dtype=np.uint8)
    for j in range(count):
        v = np.ones((1,), dtype=np.complex128)
        for i in range(n):
            w0 = v @ a[i][:, 0, :]
            w1 = v @ a[i][:, 1, :]
            p0 = float(np.real(w0 @ e[i] @ w0.conj()))
            p1 = float(np.real(w1 @ e[i] @ w1.conj()))
            u = splitmix64_uniform(seed, j * n + i)
            if u < p0 / (p0 + p1):
                x, v, p = 0, w0, p0
            else:
                x, v, p = 1, w1, p1
            v = v / np.sqrt(p)
            out[j, order[i]] = x
        del v
    return out


def metropolis(amp, n: int, chains: int, steps: int, seed: int):
    """Metropolis sampling of |<x|Psi>|^2 (App. C): chain c starts at a uniform
    random string x_0 and at step t = 1..steps proposes a uniform random x',
    accepted with probability min(|<x'|Psi>|^2 / |<x|Psi>|^2, 1) (always when
    the current weight is 0), else the chain stays.  Random numbers: SplitMix64
    uniforms of `seed` at counter g (n + 1) + q for bit q (qubit order; the bit
    is 1 iff u >= 1/2) and g (n + 1) + n for the acceptance test, with
    g = c (steps + 1) + t; x' is accepted iff u p(x) < p(x').
    amp(bits [count, n]) -> amplitudes.  Returns (samples [chains, steps, n]
    uint8, qubit order: the state after each step; accepted proposals)."""
    out = np.zeros((chains, steps, n), dtype=np.uint8)
    accepted = 0
    for c in range(chains):
        def draw(t):
            g = c * (steps + 1) + t
            return np.array([1 if splitmix64_uniform(seed, g * (n + 1) + q) >= 0.5 else 0 for q in range(n)],
                            dtype=np.uint8), splitmix64_uniform(seed, g * (n + 1) + n)
        x, _ = draw(0)
        p = abs(complex(amp(x[None, :])[0])) ** 2
        for t in range(1, steps + 1):
            y, u = draw(t)
            q = abs(complex(amp(y[None, :])[0])) ** 2
            if p == 0.0 or u * p < q:
                x, p = y, q
                accepted += 1
            out[c, t - 1] = x
    return out, accepted
