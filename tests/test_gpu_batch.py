"""Batched runs (independent instances of uneven N, depth and chi on
concurrent worker streams) against one-context runs and the oracle."""
import pytest

from synthetic import circuits as sc
from tests.helpers import gpu_run, layer_gaps, oracle_run

pytestmark = pytest.mark.gpu

# (rows, cols, chi, cycles, seed): exact (chi >= 2^(N/2)) and truncating cases
CASES = [(2, 3, 8, 6, 1), (3, 4, 64, 8, 2), (3, 4, 16, 8, 3), (2, 4, 4, 6, 4),
         (3, 3, 8, 8, 5), (4, 4, 32, 8, 6), (2, 5, 8, 7, 7), (4, 5, 32, 6, 8)]


def _batch(cases, workers, precision=0):
    from paper_2207_05612_gb300 import binding
    circs = [sc.random_circuit(r, c, cyc, seed=s) for (r, c, chi, cyc, s) in cases]
    items, keep = binding.pack_batch([(r, c, chi, circ.layers, 2)
                                      for (r, c, chi, _, _), circ in zip(cases, circs)])
    opt = binding.dmrgc_default_options()
    opt.precision = precision
    wall = binding.dmrgc_batch_run(items, len(cases), workers, opt)
    return circs, [items[i] for i in range(len(cases))], wall


def test_batch_matches_single_context_and_oracle():
    circs, res, wall = _batch(CASES, workers=3)
    assert wall > 0
    for (rows, cols, chi, cyc, seed), circ, r in zip(CASES, circs, res):
        n = rows * cols
        assert r.status == 0
        assert r.updates == len(circ.layers) * 2 * (n - 1)
        assert 0 <= r.worker < 3
        ctx, per = gpu_run(circ, chi, precision=0)
        assert abs(r.log_F_tilde - per[-1]["log_ft"]) < 1e-12
        ctx.close()
        if chi >= 2 ** (n // 2):
            assert abs(r.log_F_tilde) < 1e-10
        _, _, results, lo = oracle_run(circ, chi)
        if all(g > 1e-8 for g in layer_gaps(results)) and not any(x.zip_ambiguous for x in results):
            assert abs(r.log_F_tilde - lo) < 1e-10, (rows, cols, chi)
    # more than one worker took part
    assert len({r.worker for r in res}) > 1


def test_batch_is_independent_of_worker_count():
    _, one, _ = _batch(CASES, workers=1)
    _, many, _ = _batch(CASES, workers=8)
    for a, b in zip(one, many):
        assert a.status == 0 and b.status == 0
        assert abs(a.log_F_tilde - b.log_F_tilde) < 1e-12
        assert a.updates == b.updates


def test_batch_reuse_across_sizes_and_mixed_precision():
    """One worker reuses its context for instances that grow and shrink: FP64
    results equal single-context runs; in BF16x3 the exact-regime instances
    keep F_tilde = 1 (truncated ones are compared nowhere bit for bit: the
    tensor-core split-K order is not fixed)."""
    cases = [(4, 6, 64, 8, 11), (2, 3, 4, 4, 12), (4, 6, 32, 8, 13), (3, 4, 64, 6, 14)]
    circs, res, _ = _batch(cases, workers=1, precision=0)
    for (rows, cols, chi, cyc, seed), circ, r in zip(cases, circs, res):
        assert r.status == 0
        ctx, per = gpu_run(circ, chi, precision=0)
        ctx.close()
        assert abs(r.log_F_tilde - per[-1]["log_ft"]) < 1e-12
    exact = [(3, 4, 64, 8, 15), (2, 3, 8, 6, 16), (4, 4, 256, 6, 17), (2, 4, 16, 6, 18)]
    circs, res, _ = _batch(exact, workers=2, precision=1)
    for r in res:
        assert r.status == 0
        assert abs(r.log_F_tilde) < 1e-4


def test_batch_learned_mode_equals_single_context():
    """svd_mode 2 in a batch: every worker loads the same rank model, so each
    instance equals a single-context run with that model (FP64)."""
    import numpy as np
    from paper_2207_05612_gb300 import Context, binding
    rng = np.random.default_rng(9)
    model = (rng.normal(size=binding.MLP_PARAMS) * 0.05).astype(np.float32)
    model[-1] = 3.0   # bias: predicts about 8 (2^3) kept values
    cases = [(4, 4, 32, 6, 31), (3, 4, 16, 8, 32), (4, 5, 32, 6, 33)]
    circs = [sc.random_circuit(r, c, cyc, seed=s) for (r, c, chi, cyc, s) in cases]
    items, keep = binding.pack_batch([(r, c, chi, circ.layers, 2)
                                      for (r, c, chi, _, _), circ in zip(cases, circs)])
    opt = binding.dmrgc_default_options()
    opt.svd_mode = 2
    binding.dmrgc_batch_run(items, len(cases), 2, opt, rank_model=model)
    for i, ((rows, cols, chi, cyc, seed), circ) in enumerate(zip(cases, circs)):
        r = items[i]
        assert r.status == 0
        ctx = Context(rows, cols, chi, svd_mode=2)
        ctx.set_rank_model(model)
        for layer in circ.layers:
            ctx.apply_layer(layer)
            ctx.sweep(2)
        lf, _ = ctx.fidelity()
        ctx.close()
        assert abs(r.log_F_tilde - lf) < 1e-12
