"""Shared test helpers: run a circuit through the oracle and through the library."""
from __future__ import annotations

import math

import numpy as np

from oracle import dmrg as od
from oracle import mpo as om
from synthetic import circuits as sc


def oracle_run(circ, chi, n_sweeps=2, compress=False, **kw):
    """The zip-up guess depends on the gauge of the MPO bond (it truncates
    against a non-orthonormal remainder), so parity runs give the oracle the
    same exact, uncompressed MPO the library builds: bond = the tuple of
    straddling gates' Schmidt legs, balanced split A = U sqrt(s), B = sqrt(s) V^+.
    The two MPOs then differ only by a unitary gauge on each bond."""
    order = om.snake_order(circ.rows, circ.cols)
    mpos = [om.layer_mpo(l, order, compress=compress) for l in circ.layers]
    mps = od.product_state(circ.n_qubits)
    results, states = [], []
    for w in mpos:
        mps, res = od.compress_layer(mps, w, chi, **kw)
        results.append(res)
        states.append([t.copy() for t in mps])
    log_ft = float(sum(math.log(r.f_delta) for r in results))
    return order, states, results, log_ft


def gpu_run(circ, chi, precision=0, n_sweeps=2, **opts):
    from paper_2207_05612_gb300 import Context
    ctx = Context(circ.rows, circ.cols, chi, precision=precision, **opts)
    per_layer = []
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(n_sweeps)
        lf, fd = ctx.fidelity()
        per_layer.append({"f_delta": fd, "log_ft": lf, "hist": ctx.history(),
                          "bonds": ctx.bond_dims()[0]})
    return ctx, per_layer


def all_bitstrings(n):
    idx = np.arange(2 ** n)
    return ((idx[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1).astype(np.uint8)


def layer_gaps(results, cut=1e-12):
    """Per layer, the smallest relative gap (s_k - s_{k+1}) / s_1 at the sweep
    truncations the oracle made by chi (inf when none)."""
    out = []
    for r in results:
        gap = np.inf
        for s, k in zip(r.spectra, r.kept):
            if k < s.size and s[k] > cut * s[0]:
                gap = min(gap, (s[k - 1] - s[k]) / s[0])
        out.append(gap)
    return out


def min_gap(results, chi):
    """Smallest relative gap at every truncation by chi the oracle made."""
    g = layer_gaps(results)
    return min(g) if g else np.inf


def compare_layers(per, results, gap_min=1e-8, tol=1e-10):
    """Compare per-update partial fidelities layer by layer, up to the first
    layer whose sweep cut falls on a (near-)degenerate spectrum or whose zip-up
    cut falls in a multiplet reaching s_1: from there on several equally valid
    results exist and the runs may differ.
    Returns the number of layers compared in full agreement."""
    gaps = layer_gaps(results)
    n = 0
    for p, r, g in zip(per, results, gaps):
        assert len(p["hist"]) == len(r.f)
        diff = np.abs(np.array(p["hist"]) - np.array(r.f)).max()
        if g <= gap_min or r.zip_ambiguous:
            # the f values of this layer are still unique up to the first tie
            return n
        assert diff < tol, (n, diff, g)
        n += 1
    return n


def mpo_overlap(new, w, prev):
    """<new| W |prev> for MPSs new, prev (A[a, s, b]) and an MPO W[w, s, t, w']
    (s the output index), contracted from the left site by site."""
    e = np.ones((1, 1, 1), dtype=np.complex128)   # [a_new, w, b_prev]
    for a, wi, b in zip(new, w, prev):
        e = np.einsum("awb,asc,wstv,btd->cvd", e, a.conj(), wi, b, optimize=True)
    return complex(e.reshape(-1)[0])


def check_step_invariants(new, centre, hist, w, prev, tol=1e-11, target=None, chi=None, order=None):
    """What a compression step guarantees whatever truncation it met
    (Sec. IV.B.1 and Eq. (fa-sup)), checked on the library's own state:
      - the partial fidelities of the step never decrease;
      - the last one is |<new|U_layer|prev>|^2 (U_layer as the oracle's MPO);
      - sites left of the centre are left isometries, right of it right
        isometries, and the state has norm 1;
      - optionally (dense target, N small) F <= the weight chi Schmidt values
        of the target keep at every cut (Sec. VI.A)."""
    h = np.asarray(hist)
    assert np.all(np.diff(h) >= -tol), np.diff(h).min()
    ov = mpo_overlap(new, w, prev)
    assert abs(abs(ov) ** 2 - h[-1]) < tol, (abs(ov) ** 2, h[-1])
    for i, a in enumerate(new):
        al, _, ar = a.shape
        if i < centre:
            m = a.reshape(al * 2, ar)
            assert np.abs(m.conj().T @ m - np.eye(ar)).max() < tol
        elif i > centre:
            m = a.reshape(al, 2 * ar)
            assert np.abs(m @ m.conj().T - np.eye(al)).max() < tol
    assert abs(np.linalg.norm(new[centre]) - 1) < tol
    if target is not None:
        from oracle import statevector as sv
        n = len(order)
        for c in range(1, n):
            s = sv.schmidt_values(target, order[:c])
            assert h[-1] <= float(np.sum(s[:chi] ** 2)) + tol


def gpu_run_checked(circ, chi, precision=0, n_sweeps=2, dense=False, tol=1e-11, **opts):
    """gpu_run with check_step_invariants after every layer (the layer MPO is
    the oracle's; dense=True also checks the Schmidt bound on the statevector)."""
    from oracle import statevector as sv
    from paper_2207_05612_gb300 import Context
    order = om.snake_order(circ.rows, circ.cols)
    ctx = Context(circ.rows, circ.cols, chi, precision=precision, **opts)
    per = []
    prev, _ = ctx.get_mps()
    prev_dense = sv.zero_state(circ.n_qubits) if dense else None
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(n_sweeps)
        lf, fd = ctx.fidelity()
        hist = ctx.history()
        new, centre = ctx.get_mps()
        w = om.layer_mpo(layer, order, compress=False)
        target = sv.apply_layer(prev_dense, layer) if dense else None
        check_step_invariants(new, centre, hist, w, prev, tol=tol, target=target, chi=chi, order=order)
        if dense:
            prev_dense = od.mps_dense(new, order)
        per.append({"f_delta": fd, "log_ft": lf, "hist": hist, "bonds": ctx.bond_dims()[0]})
        prev = new
    return ctx, per
