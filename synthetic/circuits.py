"""Seeded synthetic circuits: the only inputs shared by the oracle and the CUDA path.

This module generates gate lists and nothing else. It holds none of the
compression method's arithmetic (no MPO, no MPS, no contraction); the gate
matrices it emits are the circuit, i.e. the input of the method.

Workload families (paper Sec. V.A "Three quantum circuits"):

* Sequence I, Sycamore-like random circuit: per cycle, a random one-qubit gate
  from {sqrt(X), sqrt(Y), sqrt(W)} on every qubit, never the same as that
  qubit's previous one, followed by fSim on the pairs of one coupler pattern;
  patterns follow the order ABCD-CDAB repeated (Sec. V.A).  The paper's
  lattice is the diagonal Sycamore chip (Fig. 1); on a rectangular rows x cols
  grid the four patterns are read as a staggered tiling:
  A = horizontal (r,c)-(r,c+1) with r+c even, B = vertical (r,c)-(r+1,c) with
  r+c even, C = horizontal with r+c odd, D = vertical with r+c odd.  Each
  qubit then meets at most one gate per cycle and the four patterns cover
  every grid edge once.
* Sequence II: the same gates with the pattern order CDBA-BACD repeated
  (Sec. V.A), which the paper found harder to simulate.
* Sequence III, QAOA MaxCut (Sec. V.A): U = prod_k U_B(beta_k) U_C(gamma_k)
  with U_C = prod_{edges} exp(-i gamma Z_m Z_n) and U_B = prod_m exp(-i beta X_m),
  here on the nearest-neighbour grid graph, started from |+>^N (Hadamards on
  |0...0> in the first layer).

Conventions: qubit q sits at (r, c) with q = r*cols + c.  A gate is a tuple
(q0, q1, U) with q1 = -1 for one-qubit gates; a two-qubit U is indexed
<s_q0 s_q1|U|t_q0 t_q1> with q0 the most significant bit.  A layer is a list of
gates in time order; K cycles are grouped into one layer (the paper's K).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT_HALF = 1.0 / math.sqrt(2.0)


def sqrt_pauli(name: str) -> np.ndarray:
    """exp(-i pi P / 4) for P in {X, Y, W=(X+Y)/sqrt 2}."""
    x = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    p = {"X": x, "Y": y, "W": (x + y) * SQRT_HALF}[name]
    return SQRT_HALF * (np.eye(2, dtype=np.complex128) - 1j * p)


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) in the basis |00>,|01>,|10>,|11>."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array(
        [[1, 0, 0, 0],
         [0, c, -1j * s, 0],
         [0, -1j * s, c, 0],
         [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def zz_rotation(gamma: float) -> np.ndarray:
    """exp(-i gamma Z x Z)."""
    e = np.exp(-1j * gamma)
    return np.diag([e, np.conj(e), np.conj(e), e]).astype(np.complex128)


def x_rotation(beta: float) -> np.ndarray:
    """exp(-i beta X)."""
    c, s = math.cos(beta), math.sin(beta)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


HADAMARD = SQRT_HALF * np.array([[1, 1], [1, -1]], dtype=np.complex128)


def grid_edges(rows: int, cols: int) -> dict[str, list[tuple[int, int]]]:
    """The four staggered coupler patterns A, B, C, D of a rows x cols grid."""
    pats: dict[str, list[tuple[int, int]]] = {"A": [], "B": [], "C": [], "D": []}
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            even = (r + c) % 2 == 0
            if c + 1 < cols:
                pats["A" if even else "C"].append((q, q + 1))
            if r + 1 < rows:
                pats["B" if even else "D"].append((q, q + cols))
    return pats


def all_edges(rows: int, cols: int) -> list[tuple[int, int]]:
    """Every nearest-neighbour edge of the grid graph, sorted."""
    p = grid_edges(rows, cols)
    return sorted(p["A"] + p["B"] + p["C"] + p["D"])


PATTERN_ORDER = "ABCDCDAB"  # Sec. V.A: ABCD-CDAB-ABCD-...
PATTERN_ORDER_II = "CDBABACD"  # Sequence II (Sec. V.A): CDBA-BACD-...


@dataclass
class Circuit:
    rows: int
    cols: int
    layers: list[list[tuple[int, int, np.ndarray]]] = field(default_factory=list)
    n_two_qubit: int = 0

    @property
    def n_qubits(self) -> int:
        return self.rows * self.cols


def random_circuit(rows: int, cols: int, cycles: int, cycles_per_layer: int = 2,
                   seed: int = 0, theta: float = math.pi / 2,
                   phi: float = math.pi / 6, pattern_order: str = PATTERN_ORDER) -> Circuit:
    """Sequence I on a rows x cols grid, grouped into layers of K cycles
    (pattern_order=PATTERN_ORDER_II gives Sequence II)."""
    if not pattern_order or set(pattern_order) - set("ABCD"):
        raise ValueError("pattern_order is a string over A, B, C, D")
    rng = np.random.default_rng(seed)
    n = rows * cols
    names = ("X", "Y", "W")
    mats = {k: sqrt_pauli(k) for k in names}
    two = fsim(theta, phi)
    pats = grid_edges(rows, cols)
    prev = [-1] * n
    circ = Circuit(rows, cols)
    layer: list = []
    for cyc in range(cycles):
        for q in range(n):
            if prev[q] < 0:
                g = int(rng.integers(3))
            else:
                others = [k for k in range(3) if k != prev[q]]
                g = others[int(rng.integers(2))]
            prev[q] = g
            layer.append((q, -1, mats[names[g]].copy()))
        for (a, b) in pats[pattern_order[cyc % len(pattern_order)]]:
            layer.append((a, b, two.copy()))
            circ.n_two_qubit += 1
        if (cyc + 1) % cycles_per_layer == 0 or cyc == cycles - 1:
            circ.layers.append(layer)
            layer = []
    return circ


def qaoa_circuit(rows: int, cols: int, p: int, seed: int = 0):
    """Sequence III on the grid graph: one layer per QAOA level.

    Returns (circuit, gammas, betas, edges).  gamma_k ~ U(0, pi),
    beta_k ~ U(0, pi/2).  The first layer starts with a Hadamard on every
    qubit so that the run starts from |0...0>.
    """
    rng = np.random.default_rng(seed)
    gammas = rng.uniform(0.0, math.pi, size=p)
    betas = rng.uniform(0.0, math.pi / 2, size=p)
    edges = all_edges(rows, cols)
    n = rows * cols
    circ = Circuit(rows, cols)
    for k in range(p):
        layer: list = []
        if k == 0:
            layer += [(q, -1, HADAMARD.copy()) for q in range(n)]
        zz = zz_rotation(float(gammas[k]))
        for (a, b) in edges:
            layer.append((a, b, zz.copy()))
            circ.n_two_qubit += 1
        xr = x_rotation(float(betas[k]))
        layer += [(q, -1, xr.copy()) for q in range(n)]
        circ.layers.append(layer)
    return circ, gammas, betas, edges


def random_bitstrings(n_qubits: int, count: int, seed: int = 0) -> np.ndarray:
    """Seeded uniform bitstrings, uint8 [count, n_qubits], qubit order."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(count, n_qubits), dtype=np.uint8)


def gates_to_records(layer) -> np.ndarray:
    """Pack a layer into the C-ABI record layout: int32 q0, int32 q1, then
    a row-major complex128 4x4 (two-qubit) or 2x2 (one-qubit, first 8 doubles)
    matrix as 32 doubles (re, im interleaved)."""
    rec = np.zeros(len(layer), dtype=[("q0", "<i4"), ("q1", "<i4"), ("mat", "<f8", (32,))])
    for i, (q0, q1, u) in enumerate(layer):
        rec[i]["q0"] = q0
        rec[i]["q1"] = q1
        flat = np.asarray(u, dtype=np.complex128).reshape(-1)
        buf = np.zeros(32)
        buf[0:2 * flat.size:2] = flat.real
        buf[1:2 * flat.size:2] = flat.imag
        rec[i]["mat"] = buf
    return rec


def grouping(rows: int, cols: int, kind: str, widths) -> list[int]:
    """Qubit groups of the single-site variant (Sec. V.C, groupings V, H, D)
    on a rows x cols grid: kind "V" groups consecutive columns, "H"
    consecutive rows, "D" consecutive anti-diagonals r + c = const; widths[g]
    is the number of such lines in group g (they must add up to all lines).
    Returns the number of qubits in each group, in the order of the lines.
    A description of the input only: which qubits share an MPS tensor."""
    if kind == "V":
        lines = [rows] * cols
    elif kind == "H":
        lines = [cols] * rows
    elif kind == "D":
        lines = [min(d + 1, rows, cols, rows + cols - 1 - d) for d in range(rows + cols - 1)]
    else:
        raise ValueError(kind)
    widths = list(widths)
    if sum(widths) != len(lines) or min(widths) < 1:
        raise ValueError(f"widths {widths} do not tile the {len(lines)} lines")
    out, p = [], 0
    for w in widths:
        out.append(sum(lines[p:p + w]))
        p += w
    return out


# Batched workload: independent random-circuit instances of uneven size, depth
# and bond dimension.  Grid for each qubit count: the nearest near-rectangular one.
BATCH_GRIDS = {16: (4, 4), 20: (4, 5), 24: (4, 6), 30: (5, 6), 36: (6, 6), 42: (6, 7), 54: (6, 9)}
BATCH_CHIS = (32, 64, 128, 256)


@dataclass
class BatchInstance:
    rows: int
    cols: int
    cycles: int
    chi: int
    seed: int
    circuit: Circuit


def batch_instances(count: int, seed: int = 0, qubits=tuple(BATCH_GRIDS), chis=BATCH_CHIS,
                    min_cycles: int = 8, max_cycles: int = 20) -> list[BatchInstance]:
    """`count` instances: N uniform over `qubits`, depth uniform in
    [min_cycles, max_cycles] cycles, chi uniform over `chis`; each instance's
    gates drawn from its own seed (Sequence I, K = 2 cycles per layer)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(qubits))
        rows, cols = BATCH_GRIDS[n]
        cycles = int(rng.integers(min_cycles, max_cycles + 1))
        chi = int(rng.choice(chis))
        s = int(rng.integers(2**31))
        out.append(BatchInstance(rows, cols, cycles, chi, s, random_circuit(rows, cols, cycles, seed=s)))
    return out


def perturb_circuit(circ: Circuit, eps: float, seed: int = 0) -> Circuit:
    """The same circuit with every gate U replaced by exp(i eps H) U, H a
    random Hermitian matrix with unit-variance entries: a unitary perturbation
    of size ~eps, used to measure how sensitive a result is to rounding-level
    changes of its input."""
    rng = np.random.default_rng(seed)
    out = Circuit(circ.rows, circ.cols)
    out.n_two_qubit = circ.n_two_qubit
    for layer in circ.layers:
        new = []
        for (a, b, u) in layer:
            h = rng.normal(size=u.shape) + 1j * rng.normal(size=u.shape)
            h = (h + h.conj().T) / 2
            w, v = np.linalg.eigh(h)
            new.append((a, b, (v * np.exp(1j * eps * w)) @ v.conj().T @ u))
        out.layers.append(new)
    return out
