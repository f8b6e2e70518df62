"""The oracle against the values the paper prints (tests/golden/paper_values.json,
each entry with its passage), CPU only.

Each check reaches the printed value through the oracle's own routines
(truncated SVD, Metropolis chains, statevector, operator splitting), so a
mistake in those routines moves the result away from the paper's figure:
- App. C: the mean acceptance of a uniformly proposed Metropolis move on
  Porter-Thomas amplitudes (about 70%) and the amplitudes per accepted string;
- App. B: the end points g(0) = 2, g(1) = 0 of the Schmidt-value scaling of a
  Porter-Thomas state, the chaotic slope F / (chi / 2^{N/2}) -> 4, and the
  slope 1 of a state whose Schmidt values are all equal;
- Sec. VII, Eq. (randomF): two independent random states overlap as 1 / N;
- Sec. V.A: the fSim gate splits into four operator Schmidt terms.
"""
import json
import math
import pathlib

import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as om
from oracle import statevector as sv
from synthetic import circuits as sc

GOLDEN = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_values.json").read_text())


def _printed(key):
    e = GOLDEN[key]
    return e["printed"], e["resolution"]


def _porter_thomas(n_qubits, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=2 ** n_qubits) + 1j * rng.normal(size=2 ** n_qubits)
    return psi / np.linalg.norm(psi)


def _amp_of(psi, n):
    w = 1 << np.arange(n - 1, -1, -1)
    return lambda bits: psi[(bits.astype(np.int64) * w).sum(1)]


def test_every_entry_cites_a_passage():
    for key, e in GOLDEN.items():
        if key.startswith("_"):
            continue
        assert {"printed", "resolution", "cite"} <= set(e)
        assert any(tag in e["cite"] for tag in ("Sec.", "App.", "Eq."))


def test_metropolis_first_move_acceptance_is_the_printed_70_percent():
    """Chains started at uniform strings: the fraction accepting their first
    proposal is the paper's mean acceptance.  6000 chains give a standard
    error of 0.006; the printed figure is rounded to 0.01."""
    val, res = _printed("metropolis_mean_acceptance")
    n = 12
    psi = _porter_thomas(n, 21)
    chains = 6000
    _, acc = od.metropolis(_amp_of(psi, n), n, chains, 1, 17)
    rate = acc / chains
    assert abs(rate - val) <= res + 4 * math.sqrt(rate * (1 - rate) / chains), rate
    per, res_per = _printed("metropolis_amplitudes_per_accepted_string")
    assert abs(1 / rate - per) <= res_per, 1 / rate


def _schmidt_of_porter_thomas(n_qubits, seed):
    half = 2 ** (n_qubits // 2)
    psi = _porter_thomas(n_qubits, seed).reshape(half, half)
    _, _, _, s = od.svd_truncate(psi, half, 0.0)
    return psi, s


def test_porter_thomas_schmidt_values_end_at_g0_and_g1():
    """S_mu 2^{N/4} against x = mu / 2^{N/2}: the largest value approaches
    g(0) = 2 (its finite-size shift is O(2^{-N/3})) and the smallest g(1) = 0."""
    g0, _ = _printed("porter_thomas_schmidt_scaling_g0")
    g1, _ = _printed("porter_thomas_schmidt_scaling_g1")
    nq = 20
    _, s = _schmidt_of_porter_thomas(nq, 5)
    scaled = s * 2 ** (nq / 4)
    assert abs(scaled[0] - g0) < 0.05 * g0, scaled[0]
    assert abs(scaled[-1] - g1) < 0.02, scaled[-1]
    assert np.all(np.diff(scaled) <= 0)


def test_chaotic_truncation_slope_is_four():
    """F(chi) / (chi / 2^{N/2}) for the oracle's chi-truncation of a
    Porter-Thomas state tends to the printed 4 as chi / 2^{N/2} -> 0: at
    N = 20 and chi = 8 (x = 1/128) the next term, of relative order x^{2/3},
    is below 10%."""
    slope, _ = _printed("chaotic_fidelity_slope")
    nq = 20
    psi, _ = _schmidt_of_porter_thomas(nq, 7)
    half = psi.shape[0]
    for chi, tol in ((8, 0.10), (32, 0.20)):
        _, s, _, _ = od.svd_truncate(psi, chi, 0.0)
        ratio = float(np.sum(s ** 2)) / (chi / half)
        assert abs(ratio - slope) < tol * slope, (chi, ratio)
        assert ratio < slope   # g decreases, so the finite-chi ratio lies below its limit


def test_equal_schmidt_values_give_slope_one():
    """A state U D V^T with Haar-like U, V and all Schmidt values 2^{-N/4}:
    its chi-truncation keeps exactly chi / 2^{N/2}."""
    slope, _ = _printed("equal_schmidt_values_fidelity_slope")
    rng = np.random.default_rng(3)
    half = 64
    u, _ = np.linalg.qr(rng.normal(size=(half, half)) + 1j * rng.normal(size=(half, half)))
    v, _ = np.linalg.qr(rng.normal(size=(half, half)) + 1j * rng.normal(size=(half, half)))
    psi = (u / math.sqrt(half)) @ v.T
    for chi in (1, 5, 32):
        _, s, _, _ = od.svd_truncate(psi, chi, 0.0)
        assert abs(float(np.sum(s ** 2)) / (chi / half) - slope) < 1e-10


def test_independent_random_circuit_states_overlap_as_one_over_dimension():
    """Pairs of states from independent deep random circuits (oracle
    statevector, 10 qubits, 14 cycles): the mean |<a|b>|^2 times 2^N is 1.
    The overlaps are exponentially distributed, so 300 pairs give a relative
    standard error of about 6%."""
    val, _ = _printed("random_state_overlap_times_dimension")
    rows, cols = 2, 5
    n = rows * cols
    states = [sv.run(n, sc.random_circuit(rows, cols, 14, seed=100 + i).layers)[-1] for i in range(600)]
    ov = np.array([abs(np.vdot(states[2 * i], states[2 * i + 1])) ** 2 for i in range(300)])
    mean = ov.mean() * 2 ** n
    assert abs(mean - val) < 4 * 1 / math.sqrt(300), mean


@pytest.mark.parametrize("theta,phi", [(1.0, math.pi / 2), (math.pi / 2, math.pi / 6)])
def test_fsim_splits_into_the_printed_number_of_terms(theta, phi):
    """The oracle's operator splitting of fSim (the paper's angles and the
    workload's) keeps four terms, and they rebuild the gate."""
    count, _ = _printed("fsim_operator_schmidt_values")
    a, b = om.operator_split(sc.fsim(theta, phi))
    assert a.shape[0] == count
    g = np.einsum("kab,kcd->acbd", a, b).reshape(4, 4)
    assert np.abs(g - sc.fsim(theta, phi)).max() < 1e-14
