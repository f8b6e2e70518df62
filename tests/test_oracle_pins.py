"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU only.  None retypes the oracle's formula: each
compares against an independent computation (statevector, closed form,
published value, invariant) chosen so that a dropped term, a wrong sign or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as om
from oracle import statevector as sv
from synthetic import circuits as sc


# ------------------------------------------------------------------ gates


def test_fsim_has_four_operator_schmidt_values():
    """Sec. V.A: the fSim gate used 'has four different singular values', read as
    operator Schmidt rank 4 (at theta=1, phi=pi/2 two of the four values
    coincide: 1.434, 0.841, 0.841, 0.727)."""
    for theta, phi in [(1.0, math.pi / 2), (math.pi / 2, math.pi / 6)]:
        a, b = om.operator_split(sc.fsim(theta, phi))
        assert a.shape[0] == 4
        m = sc.fsim(theta, phi).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
        s = np.linalg.svd(m, compute_uv=False)
        assert s[-1] > 0.5
        # Frobenius norm of a 4x4 unitary is 2, shared over the Schmidt values
        assert abs(np.sum(s ** 2) - 4.0) < 1e-12
        # the split reproduces the gate
        g = np.einsum("kab,kcd->acbd", a, b).reshape(4, 4)
        assert np.abs(g - sc.fsim(theta, phi)).max() < 1e-14
    # exp(-i g ZZ) = cos g II - i sin g ZZ has operator rank 2
    a, _ = om.operator_split(sc.zz_rotation(0.3))
    assert a.shape[0] == 2


def test_gate_identities():
    for name, p in [("X", [[0, 1], [1, 0]]), ("Y", [[0, -1j], [1j, 0]])]:
        r = sc.sqrt_pauli(name)
        assert np.allclose(r @ r, -1j * np.array(p), atol=1e-15)
    w = sc.sqrt_pauli("W")
    assert np.allclose(w @ w, -1j * (np.array([[0, 1], [1, 0]]) + np.array([[0, -1j], [1j, 0]])) / math.sqrt(2), atol=1e-15)
    for u in [sc.sqrt_pauli("X"), sc.sqrt_pauli("Y"), w, sc.fsim(0.7, 0.2), sc.zz_rotation(1.1), sc.x_rotation(0.4)]:
        assert np.allclose(u.conj().T @ u, np.eye(u.shape[0]), atol=1e-14)


def test_fsim_action_and_msb_convention():
    """fSim(pi/2, phi)|q0=0,q1=1> = -i|q0=1,q1=0>: swaps with a phase; q0 is the MSB."""
    psi = np.zeros((2, 2, 2), dtype=np.complex128)
    psi[0, 1, 0] = 1.0       # qubit0=0, qubit1=1, qubit2=0
    out = sv.apply_gate(psi, 0, 1, sc.fsim(math.pi / 2, 0.3))
    want = np.zeros_like(psi)
    want[1, 0, 0] = -1j
    assert np.allclose(out, want, atol=1e-15)
    # same gate listed as (1, 0): symmetric gate, same result
    out2 = sv.apply_gate(psi, 1, 0, sc.fsim(math.pi / 2, 0.3))
    assert np.allclose(out2, want, atol=1e-15)


def test_random_circuit_rules():
    circ = sc.random_circuit(3, 4, 8, seed=5)
    assert len(circ.layers) == 4
    prev = {}
    pats = sc.grid_edges(3, 4)
    cyc_gates = []
    for layer in circ.layers:
        cur = []
        for (q0, q1, u) in layer:
            if q1 < 0:
                cur.append(("1q", q0, u))
            else:
                cur.append(("2q", (q0, q1), u))
        cyc_gates += cur
    # split by cycles: 12 one-qubit gates followed by the pattern's pairs
    pos = 0
    for cyc in range(8):
        pat = pats[sc.PATTERN_ORDER[cyc % 8]]
        ones = cyc_gates[pos:pos + 12]
        pos += 12
        for (_, q, u) in ones:
            key = tuple(np.round(u.reshape(-1), 12))
            assert prev.get(q) != key  # never the same gate twice in a row
            prev[q] = key
        twos = cyc_gates[pos:pos + len(pat)]
        pos += len(pat)
        assert [t[1] for t in twos] == pat
    # each qubit meets at most one two-qubit gate per pattern; patterns tile the edges once
    edges = sorted(pats["A"] + pats["B"] + pats["C"] + pats["D"])
    assert edges == sc.all_edges(3, 4) and len(set(edges)) == len(edges)
    for p in "ABCD":
        qs = [q for e in pats[p] for q in e]
        assert len(qs) == len(set(qs))


# ------------------------------------------------------------ statevector


def test_qaoa_p1_closed_form():
    """p=1 QAOA MaxCut on a triangle-free graph (Wang, Hadfield, Jiang, Rieffel,
    PRA 97, 022304 (2018)): <C_uv> = 1/2 + 1/4 sin(4b) sin(g') (cos^{d_u-1} g'
    + cos^{d_v-1} g'), with U_C = exp(-i g' C), C = sum (1 - Z Z)/2, which is
    exp(-i gamma ZZ) per edge for g' = -2 gamma (up to a global phase)."""
    rows, cols = 2, 4
    circ, g, b, edges = sc.qaoa_circuit(rows, cols, 1, seed=11)
    psi = sv.run(rows * cols, circ.layers)[-1]
    p = np.abs(psi) ** 2
    idx = np.indices([2] * (rows * cols))
    deg = np.zeros(rows * cols, dtype=int)
    for (u, v) in edges:
        deg[u] += 1
        deg[v] += 1
    gp = -2 * g[0]
    for (u, v) in edges:
        zz = (1 - 2 * idx[u]) * (1 - 2 * idx[v])
        got = float(np.sum(p * (1 - zz) / 2))
        want = 0.5 + 0.25 * math.sin(4 * b[0]) * math.sin(gp) * (
            math.cos(gp) ** (deg[u] - 1) + math.cos(gp) ** (deg[v] - 1))
        assert abs(got - want) < 1e-12


def test_statevector_norm_and_unitary():
    circ = sc.random_circuit(2, 3, 4, seed=2)
    u = sv.layer_unitary(6, circ.layers[0])
    assert np.allclose(u.conj().T @ u, np.eye(64), atol=1e-13)
    for psi in sv.run(6, circ.layers):
        assert abs(np.linalg.norm(psi) - 1) < 1e-13


# ------------------------------------------------------------------- MPO


@pytest.mark.parametrize("rows,cols,seed", [(3, 4, 0), (2, 5, 1)])
def test_mpo_equals_dense_layer_unitary(rows, cols, seed):
    """The product of the W_i equals the layer unitary built by the statevector
    simulator column by column (independent of the MPO code)."""
    circ = sc.random_circuit(rows, cols, 4, seed=seed)
    order = om.snake_order(rows, cols)
    for layer in circ.layers:
        u = sv.layer_unitary(rows * cols, layer)
        for compress in (False, True):
            w = om.layer_mpo(layer, order, compress=compress)
            assert np.abs(om.mpo_dense(w, order) - u).max() < 1e-12


def test_mpo_qaoa_equals_dense():
    circ, *_ = sc.qaoa_circuit(2, 4, 2, seed=4)
    order = om.snake_order(2, 4)
    for layer in circ.layers:
        u = sv.layer_unitary(8, layer)
        w = om.layer_mpo(layer, order)
        assert np.abs(om.mpo_dense(w, order) - u).max() < 1e-12


def test_mpo_bond_equals_operator_schmidt_rank():
    """Lossless compression leaves exactly the operator Schmidt rank of U across
    each snake cut (computed from the dense unitary by SVD)."""
    rows, cols = 3, 4
    n = rows * cols
    circ = sc.random_circuit(rows, cols, 2, seed=9)
    order = om.snake_order(rows, cols)
    layer = circ.layers[0]
    u = sv.layer_unitary(n, layer).reshape([2] * (2 * n))
    w = om.layer_mpo(layer, order)
    dims = om.bond_dims(w)
    for cut in range(n - 1):
        left = order[:cut + 1]
        right = order[cut + 1:]
        perm = left + [n + q for q in left] + right + [n + q for q in right]
        m = u.transpose(perm).reshape(4 ** len(left), -1)
        s = np.linalg.svd(m, compute_uv=False)
        assert dims[cut] == int(np.sum(s > 1e-10 * s[0]))


def test_snake_order():
    assert om.snake_order(3, 4) == [0, 4, 8, 9, 5, 1, 2, 6, 10, 11, 7, 3]


# ------------------------------------------------------------- compression


def _config1(seed=0, rows=3, cols=4, cycles=8):
    circ = sc.random_circuit(rows, cols, cycles, seed=seed)
    order = om.snake_order(rows, cols)
    mpos = [om.layer_mpo(l, order) for l in circ.layers]
    return circ, order, mpos


def test_exact_at_full_bond_dimension():
    """T1 (Sec. III: chi = 2^{N/2} gives an exact simulation): every amplitude of
    every layer matches the statevector, F_tilde = 1."""
    circ, order, mpos = _config1()
    n = 12
    states = sv.run(n, circ.layers)
    mps = od.product_state(n)
    log_ft = 0.0
    for li, w in enumerate(mpos):
        mps, res = od.compress_layer(mps, w, 64)
        log_ft += math.log(res.f_delta)
        psi = od.mps_dense(mps, order)
        assert np.abs(psi - states[li]).max() < 1e-12
        assert abs(res.f_delta - 1) < 1e-12
    assert abs(log_ft) < 1e-11


def test_f_delta_is_exact_overlap_and_monotone():
    """Eq. (fa-sup): f_delta = |<Psi_Q(D+K)|U|Psi_Q(D)>|^2, checked with dense
    vectors; Sec. IV.B.1: f never decreases along the sweeps."""
    circ, order, mpos = _config1(seed=3)
    n = 12
    mps = od.product_state(n)
    for li, w in enumerate(mpos):
        old = od.mps_dense(mps, order)
        new_mps, res = od.compress_layer(mps, w, 8)
        new = od.mps_dense(new_mps, order)
        target = sv.apply_layer(old, circ.layers[li])
        ov = np.vdot(new.reshape(-1), target.reshape(-1))
        assert abs(abs(ov) ** 2 - res.f_delta) < 1e-12
        assert abs(ov.imag) < 1e-12 and ov.real > 0  # phase fixed: real positive
        f = np.array(res.f)
        assert np.all(np.diff(f) >= -1e-13)
        assert f[0] >= res.guess_overlap ** 2 - 1e-13
        assert len(res.f) == 2 * (n - 1)
        mps = new_mps


def test_canonical_form_and_norm():
    """Sec. IV.B.1: orthogonal form; <Psi|Psi> = Tr M M* on the centre."""
    circ, order, mpos = _config1(seed=4)
    mps, _, _ = od.run_circuit(mpos, 12, 16)
    m = 6
    for i, a in enumerate(mps):
        al, _, ar = a.shape
        if i < m:
            mat = a.reshape(al * 2, ar)
            assert np.allclose(mat.conj().T @ mat, np.eye(ar), atol=1e-12)
        elif i > m:
            mat = a.reshape(al, 2 * ar)
            assert np.allclose(mat @ mat.conj().T, np.eye(al), atol=1e-12)
    assert abs(np.linalg.norm(mps[m]) - 1) < 1e-12
    assert abs(np.linalg.norm(od.mps_dense(mps, order)) - 1) < 1e-12


def test_single_lossy_step_gives_exact_fidelity():
    """When every earlier step is lossless, F equals the only lossy f_delta
    (Eq. fa-sup applied to an exact previous state)."""
    circ, order, mpos = _config1(seed=6)
    n = 12
    mps = od.product_state(n)
    for w in mpos[:-1]:
        mps, _ = od.compress_layer(mps, w, 64)
    mps, res = od.compress_layer(mps, mpos[-1], 6)
    exact = sv.run(n, circ.layers)[-1]
    f = sv.fidelity(exact, od.mps_dense(mps, order))
    assert res.f_delta < 0.999
    assert abs(f - res.f_delta) < 1e-12


def test_fidelity_estimate_and_best_mps_bound():
    """T5 (Eq. FvsFtilde, 'typically less than 5%' on small systems) and
    T6 (Sec. VI.A: F cannot exceed the Schmidt weight chi keeps at any cut)."""
    for seed, chi in [(0, 8), (1, 16), (2, 12)]:
        circ, order, mpos = _config1(seed=seed)
        n = 12
        mps, res, log_ft = od.run_circuit(mpos, n, chi)
        exact = sv.run(n, circ.layers)[-1]
        f = sv.fidelity(exact, od.mps_dense(mps, order))
        assert abs(log_ft - math.log(f)) <= 0.05 * abs(math.log(f))
        bound = min(float(np.sum(sv.schmidt_values(exact, order[:c + 1])[:chi] ** 2))
                    for c in range(n - 1))
        assert f <= bound + 1e-12


def test_theta_is_projection_of_target_state():
    """Tier-S check of Eq. (scalarproduct): at a bond, theta equals the exact
    target U|Psi_old> projected on the current left basis (x) 2 (x) 2 (x) right
    basis, computed with dense vectors and no MPO."""
    circ, order, mpos = _config1(seed=7)
    n = 12
    mps = od.product_state(n)
    for w in mpos[:2]:
        mps, _ = od.compress_layer(mps, w, 16)
    old = od.mps_dense(mps, order)
    layer = circ.layers[2]
    target = sv.apply_layer(old, layer)
    # target in site order
    tgt = target.transpose(order)
    checks = [(1, 3), (2, 0), (2, 5), (2, 8)]
    _, res = od.compress_layer(mps, mpos[2], 16, record=set(checks))
    for (p, i) in checks:
        rec = res.records[(p, i)]
        snap = rec["mps_before"]
        # dense left basis from sites < i, right basis from sites > i+1
        lb = np.ones((1, 1), dtype=np.complex128)
        for j in range(i):
            lb = np.einsum("xa,asb->xsb", lb, snap[j]).reshape(-1, snap[j].shape[2])
        rb = np.ones((1, 1), dtype=np.complex128)
        for j in range(n - 1, i + 1, -1):
            rb = np.einsum("asb,by->asy", snap[j], rb).reshape(snap[j].shape[0], -1)
        t = tgt.reshape(2 ** i, 2, 2, 2 ** (n - i - 2))
        th = np.einsum("xa,xsty,cy->astc", lb.conj(), t, rb.conj())
        th = th.reshape(lb.shape[1] * 2, 2 * rb.shape[0])
        assert np.abs(th - rec["theta"]).max() < 1e-12


# ---------------------------------------------------- truncated SVD (App. B)


def _g(x):
    """g(x) = 2 cos(A^{-1}(pi x) / 2), A(t) = t - sin t (App. B.2)."""
    from scipy.optimize import brentq
    if x <= 0:
        return 2.0
    if x >= 1:
        return 0.0
    t = brentq(lambda u: u - math.sin(u) - math.pi * x, 0.0, 2 * math.pi)
    return 2 * math.cos(t / 2)


def test_truncation_captures_chaotic_optimum():
    """App. B: for a Porter-Thomas state of N qubits cut in halves, the weight
    kept by the chi largest Schmidt values is int_0^{chi/2^{N/2}} g(x)^2 dx,
    ~ 4 chi / 2^{N/2} for small chi (Eq. chaotic_opt)."""
    from scipy.integrate import quad
    rng = np.random.default_rng(1234)
    nq = 20
    n = 2 ** (nq // 2)
    sig = math.sqrt(1.0 / (2 * 2 ** nq))
    psi = rng.normal(0, sig, (n, n)) + 1j * rng.normal(0, sig, (n, n))
    for chi in (16, 64, 256, 512):
        u, s, vh, full = od.svd_truncate(psi, chi, 1e-12)
        kept = float(np.sum(s ** 2))
        want = quad(lambda x: _g(x) ** 2, 0, chi / n, limit=200)[0]
        assert s.size == chi
        assert abs(kept - want) < 0.02 * want + 2e-3
        # reconstruction of the kept part is the best rank-chi approximation
        assert abs(np.linalg.norm(psi - (u * s) @ vh) ** 2 - (np.sum(full ** 2) - kept)) < 1e-10
    # leading term of the small-chi expansion: F(chi) / (chi / 2^{N/2}) -> 4
    x = 1e-6
    assert abs(quad(lambda y: _g(y) ** 2, 0, x)[0] / x - 4) < 1e-3


def test_truncation_rank_rules():
    s = np.array([1.0, 0.5, 1e-13, 0.0])
    assert od.truncation_rank(s, 8, 1e-12) == 2
    assert od.truncation_rank(s, 1, 1e-12) == 1
    assert od.truncation_rank(np.array([2.0, 1.0, 1.0]), 2, 1e-12) == 2


# ---------------------------------------------------- amplitude and sampling


def test_splitmix64_published_vector():
    """SplitMix64 seeded with 0: outputs 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f (Steele, Lea, Flood 2014; reference implementation)."""
    for c, want in enumerate([0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]):
        assert od.splitmix64_uniform(0, c) == (want >> 11) / 9007199254740992.0
    u = np.array([od.splitmix64_uniform(42, c) for c in range(20000)])
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005


def test_amplitudes_match_statevector():
    circ, order, mpos = _config1(seed=8, rows=2, cols=4, cycles=6)
    mps, _, _ = od.run_circuit(mpos, 8, 16)
    exact = sv.run(8, circ.layers)[-1]
    bits = sc.random_bitstrings(8, 50, seed=1)
    got = np.array([od.amplitude(mps, order, b) for b in bits])
    assert np.abs(got - sv.amplitudes(exact, bits)).max() < 1e-12


def test_sampler_goodness_of_fit():
    """Samples follow |<x|Psi>|^2: chi-square test over all 2^8 bitstrings."""
    from scipy.stats import chisquare
    circ, order, mpos = _config1(seed=2, rows=2, cols=4, cycles=4)
    mps, _, _ = od.run_circuit(mpos, 8, 16)
    psi = od.mps_dense(mps, order)
    p = (np.abs(psi) ** 2).reshape(-1)
    count = 6000
    smp = od.sample(mps, order, 4, count, seed=77)
    idx = np.zeros(count, dtype=int)
    for q in range(8):
        idx = idx * 2 + smp[:, q].astype(int)
    obs = np.bincount(idx, minlength=256)
    exp = p * count
    keep = exp > 5
    stat = chisquare(obs[keep], exp[keep] * obs[keep].sum() / exp[keep].sum())
    assert stat.pvalue > 1e-4
