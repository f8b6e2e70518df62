"""GPU checks of the randomized and learned truncated SVD (svd_mode 1 and 2)
and of the rank model's kernels against the float64 oracle."""
import numpy as np
import pytest

from oracle import mpo as om
from oracle import rank_model as rm
from synthetic import circuits as sc
from tests.helpers import all_bitstrings, oracle_run

pytestmark = pytest.mark.gpu


def _net(seed=0, scale=0.15):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=rm.NPARAM) * scale).astype(np.float32)


def test_mlp_gradient_matches_oracle():
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(1)
    p = _net(1)
    x = rng.normal(size=(96, rm.IN)).astype(np.float32)
    y = rng.normal(size=96).astype(np.float32)
    loss, g = binding.dmrgc_mlp_loss_grad(p, x, y)
    lo, go = rm.loss_grad(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    # FP32 against float64, relative to the largest gradient entry of each block
    blocks = [(0, rm.HID * rm.IN), (rm.HID * rm.IN, rm.HID), (rm.HID * rm.IN + rm.HID, rm.HID * rm.HID),
              (rm.NPARAM - 2 * rm.HID - 1, rm.HID), (rm.NPARAM - rm.HID - 1, rm.HID), (rm.NPARAM - 1, 1)]
    for off, size in blocks:
        a, b = g[off:off + size], go[off:off + size]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), off


def test_mlp_forward_fp32_and_bf16():
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(2)
    p = _net(2)
    x = rng.normal(size=(40, rm.IN)).astype(np.float32)
    ref = rm.forward(p.astype(np.float64), x.astype(np.float64))
    y32 = binding.dmrgc_mlp_predict(p, x, bf16=False)
    y16 = binding.dmrgc_mlp_predict(p, x, bf16=True)
    scale = np.abs(ref).max()
    assert np.abs(y32 - ref).max() <= 1e-5 * scale
    assert np.abs(y16 - ref).max() <= 3e-2 * scale


def test_mlp_training_fits_a_smooth_target():
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4096, rm.IN)).astype(np.float32)
    y = (2.0 + x[:, 32] - 0.5 * x[:, 0] + 0.3 * np.tanh(x[:, 5] * x[:, 6])).astype(np.float32)
    params, loss = binding.dmrgc_mlp_train(x, y, epochs=30, batch=128, lr=2e-3, seed=7)
    assert loss[-1] < 0.05 * loss[0]
    pred = binding.dmrgc_mlp_predict(params, x[:512], bf16=False)
    assert np.mean((pred - y[:512]) ** 2) < 0.05 * np.var(y)
    # deterministic for a given seed
    params2, loss2 = binding.dmrgc_mlp_train(x, y, epochs=30, batch=128, lr=2e-3, seed=7)
    assert np.array_equal(params, params2)


def test_logged_records_match_oracle():
    """FP64 logging run on a truncating 3x4 circuit: every record's input and
    label equal those the oracle's own spectra define."""
    from paper_2207_05612_gb300 import Context
    circ = sc.random_circuit(3, 4, 8, seed=21)
    chi = 12
    order, states, results, lo = oracle_run(circ, chi)
    ctx = Context(3, 4, chi, log_rank_records=1)
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(2)
    xg, yg = ctx.rank_records()
    bonds = [[w.shape[3] for w in om.layer_mpo(l, order, compress=False)] for l in circ.layers]
    xo, yo = rm.expected_records(results, bonds)
    assert xg.shape == xo.shape and xg.shape[0] > 50
    assert np.allclose(xg[:, 32:], xo[:, 32:])
    # log10 ratios: float32 of the same spectrum (clamped at -30 for zeros)
    assert np.abs(xg[:, :32] - xo[:, :32]).max() < 1e-4
    assert np.mean(np.isclose(yg, yo, atol=1e-6)) > 0.98
    ctx.close()


def _run(circ, chi, precision, **opts):
    from paper_2207_05612_gb300 import Context
    ctx = Context(circ.rows, circ.cols, chi, precision=precision, timing=True, **opts)
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(2)
    return ctx


def test_randomized_mode_certified_against_jacobi_fp64():
    """FP64 QAOA runs where some bonds' spectra decay well inside the bond
    dimension: sketches are tried there, and every accepted one is certified
    within tol of the optimal update, so F_tilde moves by at most about tol
    per accepted sketch (2x margin) from the Jacobi run, which equals the
    oracle."""
    for rows, cols, p, chi in ((4, 4, 2, 256), (4, 6, 2, 128)):
        circ, _, _, _ = sc.qaoa_circuit(rows, cols, p, seed=5)
        order, states, results, lo = oracle_run(circ, chi)
        base = _run(circ, chi, 0)
        rnd = _run(circ, chi, 0, svd_mode=1)
        lb, _ = base.fidelity()
        lr_, _ = rnd.fidelity()
        st = rnd.stats()
        assert abs(lb - lo) < 1e-10
        assert st["rsvd_attempts"] > 0
        assert abs(lr_ - lb) <= 2 * 1e-6 * max(1, st["rsvd_accepted"]) + 1e-12, (lr_, lb, st["rsvd_accepted"])
        print(f"{rows}x{cols} p={p} chi={chi}: sketches {st['rsvd_accepted']}/{st['rsvd_attempts']}, "
              f"log F {lr_:.10f} vs {lb:.10f}")
        base.close()
        rnd.close()


def test_randomized_exact_lowrank_amplitudes():
    """Exact regime, tight tolerance: accepted sketches change no amplitude
    beyond 1e-10 (rejected ones fall back to the Jacobi SVD)."""
    circ, _, _, _ = sc.qaoa_circuit(4, 4, 2, seed=5)
    order, states, results, lo = oracle_run(circ, 256)
    ctx = _run(circ, 256, 0, svd_mode=1, rsvd_tolerance=1e-13)
    from oracle import dmrg as od
    bits = all_bitstrings(16)[::7]
    amp = ctx.amplitude(bits)
    ref = np.array([od.amplitude(states[-1], order, b) for b in bits])
    assert np.abs(amp - ref).max() < 1e-10
    assert ctx.stats()["rsvd_attempts"] > 0
    ctx.close()


def test_learned_mode_trains_on_logged_spectra_and_is_judged_by_jacobi():
    """Train the rank model on records logged from QAOA and random circuits,
    then run the learned mode on a held-out QAOA circuit: the model asks for
    sketches, and the fidelity stays that of the full Jacobi SVD (accepted
    sketches are certified)."""
    from paper_2207_05612_gb300 import binding
    xs, ys = [], []
    for seed in range(6):
        circ, _, _, _ = sc.qaoa_circuit(4, 6, 3, seed=100 + seed)
        ctx = _run(circ, 64, 2, log_rank_records=1)
        x, y = ctx.rank_records()
        xs.append(x)
        ys.append(y)
        ctx.close()
    for seed in range(2):
        circ = sc.random_circuit(4, 6, 10, seed=200 + seed)
        ctx = _run(circ, 64, 2, log_rank_records=1)
        x, y = ctx.rank_records()
        xs.append(x)
        ys.append(y)
        ctx.close()
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    assert x.shape[0] > 500
    params, loss = binding.dmrgc_mlp_train(x, y, epochs=60, batch=128, lr=2e-3, seed=1)
    assert loss[-1] < loss[0]
    circ, _, _, _ = sc.qaoa_circuit(4, 6, 3, seed=999)
    full = _run(circ, 64, 2)
    from paper_2207_05612_gb300 import Context
    ctx = Context(4, 6, 64, precision=2, timing=True, svd_mode=2)
    ctx.set_rank_model(params)
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(2)
    lf, _ = full.fidelity()
    ll, _ = ctx.fidelity()
    sf, sl = full.stats(), ctx.stats()
    assert sl["rsvd_attempts"] > 0
    assert abs(ll - lf) <= 1e-3 * max(1.0, abs(lf)), (ll, lf)
    print(f"learned: log F {ll:.6f} vs {lf:.6f}; sketches {sl['rsvd_accepted']}/{sl['rsvd_attempts']}; "
          f"svd {sl['svd_ms']:.1f} ms vs {sf['svd_ms']:.1f} ms; sweeps {sl['jacobi_sweeps']} vs {sf['jacobi_sweeps']}")
    full.close()
    ctx.close()
