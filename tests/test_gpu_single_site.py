"""The single-site variant over grouped qubits (Sec. IV.A, IV.B.1, V.C) on the
GPU against the oracle (oracle/single_site.py), through the C ABI.

The guess is the same seeded random tensor train on both sides, and an update
makes no discrete decision but the numerical-zero rank, so the whole sequence
of partial fidelities and the final state are unique: FP64 runs match the
oracle update by update and the dense states entry by entry (the state does
not depend on the gauge of the bonds, so no phase is free)."""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as om
from oracle import single_site as ss
from oracle import statevector as sv
from synthetic import circuits as sc

pytestmark = pytest.mark.gpu

SEED = 1234


def _oracle(circ, rows, cols, kind, sizes, chi, n_sweeps):
    order = om.chain_order(rows, cols, kind)
    mps = ss.group_product_zero(sizes)
    per = []
    for d, layer in enumerate(circ.layers):
        wg = ss.group_mpo(om.layer_mpo(layer, order), sizes)
        mps, res, _ = ss.compress_layer(mps, wg, sizes, chi, n_sweeps, SEED + d)
        per.append((list(res.f), [t.copy() for t in mps]))
    return order, per


def _gpu(circ, rows, cols, kind, sizes, chi, n_sweeps, precision=0):
    from paper_2207_05612_gb300 import Context
    ctx = Context(rows, cols, chi, precision=precision, order=kind, groups=sizes, seed=SEED, mpo_compress=1)
    per = []
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(n_sweeps)
        mps, centre = ctx.get_mps()
        per.append((ctx.history(), mps, centre, ctx.fidelity()))
    return ctx, per


CASES = [("V", [1, 2, 1], 4), ("V", [1, 2, 1], 64), ("H", [1, 1, 1], 5), ("D", [2, 2, 2], 6),
         ("V", [1, 1, 1, 1], 3), ("D", [1, 3, 2], 64)]


@pytest.mark.parametrize("kind,widths,chi", CASES)
def test_fp64_matches_oracle_update_by_update(kind, widths, chi):
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 6, seed=21)
    sizes = sc.grouping(rows, cols, kind, widths)
    order, want = _oracle(circ, rows, cols, kind, sizes, chi, 3)
    _, got = _gpu(circ, rows, cols, kind, sizes, chi, 3)
    for (fw, mw), (fg, mg, centre, (lf, fd)) in zip(want, got):
        assert len(fg) == 3 * len(sizes)
        assert np.abs(np.array(fg) - np.array(fw)).max() < 1e-10
        dw = ss.group_dense(mw, sizes, order)
        dg = ss.group_dense(mg, sizes, order)
        assert np.abs(dw - dg).max() < 1e-10
        assert abs(fd - fw[-1]) < 1e-12


def test_fp64_invariants_and_exactness_at_full_chi():
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 6, seed=5)
    sizes = sc.grouping(rows, cols, "V", [1, 1, 1, 1])
    _, got = _gpu(circ, rows, cols, "V", sizes, 64, 2)
    order = om.chain_order(rows, cols, "V")
    psi = sv.run(rows * cols, circ.layers)[-1]
    fg, mg, centre, (lf, _) = got[-1]
    assert abs(lf) < 1e-10
    dense = ss.group_dense(mg, sizes, order)
    assert abs(abs(np.vdot(dense.reshape(-1), psi.reshape(-1))) - 1) < 1e-10
    for tau, a in enumerate(mg):
        al, s, ar = a.shape
        if tau < centre:
            m = a.reshape(al * s, ar)
            assert np.abs(m.conj().T @ m - np.eye(ar)).max() < 1e-12
        elif tau > centre:
            m = a.reshape(al, s * ar)
            assert np.abs(m @ m.conj().T - np.eye(al)).max() < 1e-12


def test_trivial_layer_is_lossless_on_gpu():
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 4, seed=11)
    sizes = sc.grouping(rows, cols, "V", [1, 1, 1, 1])
    edges = sc.grid_edges(rows, cols)
    rng = np.random.default_rng(4)
    trivial = [(q, -1, sc.sqrt_pauli("XYW"[rng.integers(3)])) for q in range(rows * cols)]
    trivial += [(a, b, sc.fsim(np.pi / 2, np.pi / 6)) for (a, b) in edges["B"] + edges["D"]]
    from paper_2207_05612_gb300 import Context
    ctx = Context(rows, cols, 3, order="V", groups=sizes, seed=3, mpo_compress=1)
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(2)
    assert ctx.fidelity()[1] < 0.999
    ctx.apply_layer(trivial)
    ctx.sweep(2)
    assert abs(ctx.fidelity()[1] - 1) < 1e-12


@pytest.mark.parametrize("precision,tol", [(1, 2e-4), (2, 2e-4), (3, 2e-4)])
def test_mixed_precision_against_oracle_4x6(precision, tol):
    """4 x 6 grid, column groups of 4 qubits (physical dimension 16), chi = 24:
    log F~ of the complex64 modes within tol of the oracle's."""
    rows, cols = 4, 6
    circ = sc.random_circuit(rows, cols, 8, seed=2)
    sizes = sc.grouping(rows, cols, "V", [1] * cols)
    order, want = _oracle(circ, rows, cols, "V", sizes, 24, 2)
    lf_want = float(sum(np.log(f[-1]) for f, _ in want))
    _, got = _gpu(circ, rows, cols, "V", sizes, 24, 2, precision=precision)
    lf = got[-1][3][0]
    print(f"prec {precision}: log F~ {lf:.9f} oracle {lf_want:.9f} |delta| {abs(lf - lf_want):.2e}")
    assert abs(lf - lf_want) < tol
    for fg, _, _, _ in got:
        assert np.all(np.diff(fg) >= -1e-5)


def test_single_group_is_the_whole_state():
    rows, cols = 2, 3
    circ = sc.random_circuit(rows, cols, 4, seed=1)
    _, got = _gpu(circ, rows, cols, "V", [6], 4, 2)
    for fg, mg, centre, (lf, fd) in got:
        assert len(fg) == 2 and abs(fd - 1) < 1e-12 and mg[0].shape == (1, 64, 1)


def test_grouped_context_rejects_what_it_does_not_do():
    from paper_2207_05612_gb300 import Context, binding
    with pytest.raises(binding.DmrgcError):
        Context(3, 4, 8, groups=[3, 3, 3])          # does not add up to 12
    with pytest.raises(binding.DmrgcError):
        Context(3, 4, 8, groups=[12, 0])
    ctx = Context(3, 4, 8, groups=[6, 6], mpo_compress=1)
    circ = sc.random_circuit(3, 4, 2, seed=0)
    ctx.apply_layer(circ.layers[0])
    ctx.sweep(1)
    with pytest.raises(binding.DmrgcError):
        ctx.sample(4, 1)


@pytest.mark.parametrize("kind,widths,chi", [("V", [1, 2, 1], 4), ("D", [2, 2, 2], 6)])
def test_grouped_amplitudes_and_metropolis_fp64(kind, widths, chi):
    """Amplitudes of the grouped GPU state equal the oracle's state's (the
    state is unique, no phase is free), and Metropolis chains on it equal the
    oracle's chains on the oracle's amplitudes."""
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 6, seed=21)
    sizes = sc.grouping(rows, cols, kind, widths)
    order, want = _oracle(circ, rows, cols, kind, sizes, chi, 3)
    ctx, _ = _gpu(circ, rows, cols, kind, sizes, chi, 3)
    dense = ss.group_dense(want[-1][1], sizes, order)
    bits = sc.random_bitstrings(rows * cols, 300, seed=2)
    got = ctx.amplitude(bits)
    exp = sv.amplitudes(dense, bits)
    assert np.abs(got - exp).max() < 1e-10
    amp = lambda b: sv.amplitudes(dense, b)
    w_s, w_acc = od.metropolis(amp, rows * cols, 16, 20, 3)
    g_s, g_acc = ctx.metropolis(16, 20, 3)
    assert g_acc == w_acc and np.array_equal(g_s, w_s)
