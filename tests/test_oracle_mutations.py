"""Planted mistakes in the oracle (CPU only) must be caught by its pins.

Each case patches one oracle step with a plausible bug (a transposed MPO,
a dropped conjugate, a transposed one-qubit gate, a wrong index order in Y) and
checks that the exactness pin (T1) or the overlap identity (Eq. fa-sup) fails.
"""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as om
from oracle import statevector as sv
from synthetic import circuits as sc


def _exact_error(rows=2, cols=4, cycles=4, chi=16, seed=3):
    circ = sc.random_circuit(rows, cols, cycles, seed=seed)
    order = om.snake_order(rows, cols)
    mpos = [om.layer_mpo(l, order) for l in circ.layers]
    mps, res, _ = od.run_circuit(mpos, rows * cols, chi)
    exact = sv.run(rows * cols, circ.layers)[-1]
    return np.abs(od.mps_dense(mps, order) - exact).max()


def test_unpatched_oracle_is_exact():
    assert _exact_error() < 1e-12


@pytest.mark.parametrize("bug", ["mpo_transposed", "env_no_conj", "one_qubit_transposed", "y_wrong_leg"])
def test_planted_bug_is_caught(monkeypatch, bug):
    if bug == "mpo_transposed":
        orig = od.make_x
        monkeypatch.setattr(od, "make_x", lambda l, b, w: orig(l, b, w.transpose(0, 2, 1, 3)))
    elif bug == "env_no_conj":
        monkeypatch.setattr(od, "env_left",
                            lambda a, x: np.einsum("ask,aswb->kwb", a, x))
    elif bug == "one_qubit_transposed":
        orig = om.apply_gate_to_mpo

        def transposed(w, sp, sq, u):
            return orig(w, sp, sq, u.T if sq < 0 else u)
        monkeypatch.setattr(om, "apply_gate_to_mpo", transposed)
    elif bug == "y_wrong_leg":
        monkeypatch.setattr(od, "make_y", lambda r, b, w: np.einsum(
            "cwb,atb,ystw->scya", r, b, w.transpose(0, 2, 1, 3), optimize=True))
    assert _exact_error() > 1e-3
