"""Shared test helpers: run a circuit through the oracle and through the library."""
from __future__ import annotations

import math

import numpy as np

from oracle import dmrg as od
from oracle import mpo as om
from synthetic import circuits as sc


def oracle_run(circ, chi, n_sweeps=2, **kw):
    order = om.snake_order(circ.rows, circ.cols)
    mpos = [om.layer_mpo(l, order) for l in circ.layers]
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


def min_gap(results, chi):
    """Smallest relative gap s_k - s_{k+1} at every truncation the oracle made."""
    gap = np.inf
    for r in results:
        for s, k in zip(r.spectra, r.kept):
            if k < s.size and s[k] > 1e-12 * s[0]:
                gap = min(gap, (s[k - 1] - s[k]) / s[0])
    return gap
