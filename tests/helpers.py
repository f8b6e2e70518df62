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
