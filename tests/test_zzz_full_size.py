"""The hot path at the benchmark's full size and launch configuration (6 x 9 =
54 qubits, chi = 512, K = 2 cycles per step, two sweeps, BF16x3 tensor cores,
compressed layer MPO, Gram eigensolver with Jacobi fallback), through the C
ABI, checked where the oracle can follow one output at a time and otherwise by
properties that hold at any size:

- amplitudes of sampled bit strings against the oracle's product of the
  downloaded site matrices (Sec. IV.A), one string at a time;
- the mixed-canonical form the sweep leaves: isometries left and right of
  the orthogonality centre, a unit-norm centre (Sec. IV.B.1);
- f never decreases within a step (Sec. IV.B.1), and log F~ is the sum of
  the steps' log f_delta (Eq. Ftilde-sup);
- bonds within chi and within the exact bound 2^{min(i, N - i)}.

The oracle cannot run the sweep itself at this size; the smaller parity tests
compare it update by update."""
import math

import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as om
from synthetic import circuits as sc

pytestmark = pytest.mark.gpu

ROWS, COLS, CHI, CYCLES = 6, 9, 512, 10


@pytest.fixture(scope="module")
def full_run():
    from paper_2207_05612_gb300 import Context, binding
    circ = sc.random_circuit(ROWS, COLS, CYCLES, seed=0)
    ctx = Context(ROWS, COLS, CHI, precision=binding.DMRGC_BF16X3, mpo_compress=1)
    per = []
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(2)
        lf, fd = ctx.fidelity()
        per.append({"hist": np.array(ctx.history()), "log_ft": lf, "f_delta": fd,
                    "bonds": ctx.bond_dims()[0]})
    mps, centre = ctx.get_mps()
    yield ctx, per, mps, centre
    ctx.close()


def test_reaches_the_saturated_regime(full_run):
    ctx, per, _, _ = full_run
    n = ROWS * COLS
    assert max(per[-1]["bonds"]) == CHI
    for p in per:
        for i, b in enumerate(p["bonds"]):
            assert 1 <= b <= min(CHI, 2 ** min(i + 1, n - i - 1))
    st = ctx.stats()
    assert st["eig_svds"] > 0


def test_f_monotone_within_each_step_and_log_f_tilde_is_their_sum(full_run):
    _, per, _, _ = full_run
    total = 0.0
    for p in per:
        h = p["hist"]
        assert len(h) == 2 * (ROWS * COLS - 1)
        assert np.all(np.isfinite(h)) and np.all((h > 0) & (h <= 1 + 1e-4))
        assert np.all(np.diff(h) >= -1e-3 * h[1:])
        assert p["f_delta"] == h[-1]
        total += math.log(p["f_delta"])
        assert abs(p["log_ft"] - total) <= 1e-9 * max(1.0, abs(total))


def test_mixed_canonical_form(full_run):
    """Tensors left of the centre have orthonormal columns, those right of it
    orthonormal rows, the centre unit norm: within 1e-3 for complex64 storage
    and FP32 factorisations (the kernel tests hold each factor to 1e-4 at
    these sizes)."""
    _, _, mps, centre = full_run
    assert len(mps) == ROWS * COLS
    for i, a in enumerate(mps):
        al, s, ar = a.shape
        assert s == 2
        if i < centre:
            m = a.reshape(al * s, ar)
            assert np.abs(m.conj().T @ m - np.eye(ar)).max() < 1e-3, i
        elif i > centre:
            m = a.reshape(al, s * ar)
            assert np.abs(m @ m.conj().T - np.eye(al)).max() < 1e-3, i
        else:
            assert abs(np.linalg.norm(a) - 1) < 1e-4


def test_sampled_amplitudes_against_the_oracle(full_run):
    """64 random strings: the library's batched read-out (one GEMM per site
    for the chunk) against the oracle's product of the same site matrices in
    complex128.  The read-out's products carry TF32x3 rounding, ~1e-6 of the
    row norms per site, so the bound is 1e-3 of the amplitudes' RMS."""
    ctx, _, mps, _ = full_run
    order = om.snake_order(ROWS, COLS)
    bits = sc.random_bitstrings(ROWS * COLS, 64, seed=7)
    got = ctx.amplitude(bits)
    want = np.array([od.amplitude(mps, order, b) for b in bits])
    rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
    assert rms > 0 and np.all(np.isfinite(got))
    err = float(np.abs(got - want).max())
    print(f"54 qubits, chi 512: max |amp - oracle| = {err:.3e}, rms amplitude {rms:.3e}")
    assert err <= 1e-3 * rms
