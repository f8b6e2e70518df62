"""Pins of the Metropolis sampler of the oracle (App. C), CPU only.

- From a uniform start, the first move is accepted with probability
  E min(p'/p, 1) over two independent Porter-Thomas weights: the paper's
  integral, which equals ln 2 (~0.693, the "about 70%" of App. C).
- In the stationary chain the current string is drawn with weight p, and the
  acceptance becomes E_{p ~ p e^-p} min(p'/p, 1) = 1/2 exactly.
- The chains sample |<x|Psi>|^2: long runs match the exact distribution.
- The random numbers follow the stated SplitMix64 counter layout.
"""
import numpy as np
from scipy import integrate

from oracle import dmrg as od


def _porter_thomas_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    return psi / np.linalg.norm(psi)


def _amp_of(psi, n):
    w = 1 << np.arange(n - 1, -1, -1)
    return lambda bits: psi[(bits.astype(np.int64) * w).sum(1)]


def test_paper_integral_is_ln2():
    v, _ = integrate.dblquad(lambda y, x: min(x / y, 1.0) * np.exp(-x - y), 0, 60, 0, 60)
    assert abs(v - np.log(2)) < 1e-7


def test_first_step_acceptance_is_ln2():
    n = 12
    psi = _porter_thomas_state(n, 1)
    chains = 6000
    _, acc = od.metropolis(_amp_of(psi, n), n, chains, 1, 5)
    rate = acc / chains
    assert abs(rate - np.log(2)) < 0.025, rate


def test_stationary_acceptance_is_one_half():
    n = 12
    psi = _porter_thomas_state(n, 2)
    s, _ = od.metropolis(_amp_of(psi, n), n, 30, 700, 9)
    moves = np.any(s[:, 101:] != s[:, 100:-1], axis=2)
    rate = moves.mean()
    assert abs(rate - 0.5) < 0.02, rate


def test_chains_sample_the_exact_distribution():
    n = 5
    psi = _porter_thomas_state(n, 3)
    s, _ = od.metropolis(_amp_of(psi, n), n, 100, 400, 11)
    idx = (s[:, 50:].astype(np.int64) * (1 << np.arange(n - 1, -1, -1))).sum(2).reshape(-1)
    emp = np.bincount(idx, minlength=2 ** n) / idx.size
    tv = 0.5 * np.abs(emp - np.abs(psi) ** 2).sum()
    assert tv < 0.04, tv


def test_counter_layout():
    n, steps, seed = 4, 3, 21
    psi = _porter_thomas_state(n, 4)
    s, _ = od.metropolis(_amp_of(psi, n), n, 2, steps, seed)
    # chain 1 ends step 1 either at its start (g = 1 * 4 + 0) or at the
    # proposal of step 1 (g = 5)
    def draw(g):
        return np.array([1 if od.splitmix64_uniform(seed, g * (n + 1) + q) >= 0.5 else 0 for q in range(n)])
    x0, x1 = draw(4), draw(5)
    u = od.splitmix64_uniform(seed, 5 * (n + 1) + n)
    amp = _amp_of(psi, n)
    p0, p1 = abs(amp(x0[None])[0]) ** 2, abs(amp(x1[None])[0]) ** 2
    want = x1 if u * p0 < p1 else x0
    assert np.array_equal(s[1, 0], want)
