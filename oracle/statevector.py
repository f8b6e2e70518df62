"""Exact statevector simulation: the plain definition of the circuit output.

Eq. (perfect): |Psi(D)> = U^(D) ... U^(1) |Psi(0)>, applied gate by gate.
Eq. (F-sup): F = |<Psi_Q|Psi_P>|^2.
Sec. VI.A (best possible MPS): Schmidt spectrum of the exact state at a cut.

State layout: a complex128 tensor of shape [2]*N, axis q is qubit q (qubit
order, not MPS site order).  Gate convention: <s_q0 s_q1|U|t_q0 t_q1> with q0
the most significant bit.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros([2] * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    return psi


def apply_gate(psi: np.ndarray, q0: int, q1: int, u: np.ndarray) -> np.ndarray:
    """Apply one gate to the state tensor (returns a new tensor)."""
    u = np.asarray(u, dtype=np.complex128)
    if q1 < 0:
        out = np.tensordot(u, psi, axes=([1], [q0]))
        return np.moveaxis(out, 0, q0)
    g = u.reshape(2, 2, 2, 2)  # [s0, s1, t0, t1]
    out = np.tensordot(g, psi, axes=([2, 3], [q0, q1]))
    return np.moveaxis(out, [0, 1], [q0, q1])


def apply_layer(psi: np.ndarray, layer) -> np.ndarray:
    for (q0, q1, u) in layer:
        psi = apply_gate(psi, q0, q1, u)
    return psi


def run(n: int, layers) -> list[np.ndarray]:
    """States after each layer, starting from |0...0> (Eq. perfect)."""
    psi = zero_state(n)
    out = []
    for layer in layers:
        psi = apply_layer(psi, layer)
        out.append(psi.copy())
    return out


def layer_unitary(n: int, layer) -> np.ndarray:
    """Dense 2^N x 2^N matrix of a layer, built by applying the layer to every
    basis state (columns), qubit 0 most significant."""
    dim = 2 ** n
    cols = []
    for j in range(dim):
        e = np.zeros(dim, dtype=np.complex128)
        e[j] = 1.0
        cols.append(apply_layer(e.reshape([2] * n), layer).reshape(dim))
    return np.stack(cols, axis=1)


def fidelity(psi_p: np.ndarray, psi_q: np.ndarray) -> float:
    """Eq. (F-sup) for normalised states."""
    return float(abs(np.vdot(psi_q.reshape(-1), psi_p.reshape(-1))) ** 2)


def schmidt_values(psi: np.ndarray, left_qubits) -> np.ndarray:
    """Singular values of the state across the bipartition left | rest
    (Sec. VI.A), descending."""
    n = psi.ndim
    left = list(left_qubits)
    right = [q for q in range(n) if q not in left]
    m = np.transpose(psi, left + right).reshape(2 ** len(left), -1)
    return np.linalg.svd(m, compute_uv=False)


def amplitudes(psi: np.ndarray, bits: np.ndarray) -> np.ndarray:
    """<x|psi> for bitstrings given in qubit order, uint8 [count, N]."""
    return np.array([psi[tuple(int(b) for b in row)] for row in bits])
