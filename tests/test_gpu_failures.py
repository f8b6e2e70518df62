"""Failure detection without a GPU fault.

Every failure here is made on the host or by a bounded wait that is told to
give up early; nothing traps, faults or hangs the GPU.  After each failure the
same process runs a correct SVD or sweep on the same device, so the CUDA
context stayed usable.
"""
import numpy as np
import pytest

from synthetic import circuits as sc

pytestmark = pytest.mark.gpu


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _svd_still_works():
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(1)
    g = _rand(rng, (96, 80))
    s, k, _ = binding.dmrgc_test_svd(3, g, 40, 2e-5)
    want = np.linalg.svd(g, compute_uv=False)
    assert k == 40 and np.abs(s[:80] - want).max() <= 3e-5 * want[0]


def test_etimeout_from_a_wait_that_runs_out():
    """The Jacobi kernels' spin waits (grid barrier, per-block round counters)
    are bounded; with a limit of one poll a CTA that must wait for another gives
    up, sets the launch's error flag, every CTA leaves at its next wait, and the
    call returns DMRGC_ETIMEOUT."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(2)
    g = _rand(rng, (512, 512))
    binding.dmrgc_set_wait_limit(1)
    try:
        with pytest.raises(binding.DmrgcError) as e:
            binding.dmrgc_test_svd(3, g, 256, 2e-5)
        assert e.value.status == binding.DMRGC_ETIMEOUT
    finally:
        binding.dmrgc_set_wait_limit(0)
    _svd_still_works()


def test_etimeout_reaches_the_sweep_and_the_context_recovers():
    from paper_2207_05612_gb300 import Context, binding
    circ = sc.random_circuit(3, 4, 8, seed=1)
    ctx = Context(3, 4, 16, precision=binding.DMRGC_FP32)
    ctx.apply_layer(circ.layers[0])
    ctx.sweep(2)
    binding.dmrgc_set_wait_limit(1)
    try:
        with pytest.raises(binding.DmrgcError) as e:
            ctx.apply_layer(circ.layers[1])
            ctx.sweep(2)
        assert e.value.status == binding.DMRGC_ETIMEOUT
    finally:
        binding.dmrgc_set_wait_limit(0)
    ctx.close()
    fresh = Context(3, 4, 16, precision=binding.DMRGC_FP32)
    for layer in circ.layers:
        fresh.apply_layer(layer)
        fresh.sweep(2)
    lf, _ = fresh.fidelity()
    assert np.isfinite(lf) and lf <= 0
    fresh.close()


def test_enoconv_when_the_sweep_cap_is_reached():
    """max_jacobi_sweeps = 1: the first SVD that still rotates after its only
    sweep reports DMRGC_ENOCONV."""
    from paper_2207_05612_gb300 import Context, binding
    circ = sc.random_circuit(3, 4, 8, seed=1)
    ctx = Context(3, 4, 16, precision=binding.DMRGC_FP32, max_jacobi_sweeps=1)
    with pytest.raises(binding.DmrgcError) as e:
        for layer in circ.layers:
            ctx.apply_layer(layer)
            ctx.sweep(2)
    assert e.value.status == binding.DMRGC_ENOCONV
    ctx.close()
    _svd_still_works()


def test_enumeric_on_a_zero_state():
    """A gate that maps the state to zero (a zero matrix passes the host's
    finiteness check) leaves nothing to keep: the truncation sees s_1 = 0 and
    the call returns DMRGC_ENUMERIC; a zero matrix given to the SVD entry point
    does the same."""
    from paper_2207_05612_gb300 import Context, binding
    ctx = Context(2, 3, 4, precision=binding.DMRGC_FP64)
    layer = sc.random_circuit(2, 3, 2, seed=3).layers[0] + [(2, -1, np.zeros((2, 2)))]
    with pytest.raises(binding.DmrgcError) as e:
        ctx.apply_layer(layer)
        ctx.sweep(2)
    assert e.value.status == binding.DMRGC_ENUMERIC
    ctx.close()
    with pytest.raises(binding.DmrgcError) as e:
        binding.dmrgc_test_svd(3, np.zeros((64, 48), dtype=complex), 8, 2e-5)
    assert e.value.status == binding.DMRGC_ENUMERIC
    _svd_still_works()


def test_nan_gates_are_rejected_on_the_host():
    from paper_2207_05612_gb300 import Context, binding
    ctx = Context(2, 2, 4)
    bad = np.eye(4, dtype=complex)
    bad[1, 1] = np.nan
    with pytest.raises(binding.DmrgcError) as e:
        ctx.apply_layer([(0, 1, bad)])
    assert e.value.status == binding.DMRGC_EINVAL
    ctx.close()
