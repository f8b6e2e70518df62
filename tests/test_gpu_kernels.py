"""Kernel-level GPU parity through the diagnostic C entry points.

The contraction engine against numpy matrix products (every operand op,
ragged sizes that are not tile multiples) and the one-sided Jacobi SVD against
LAPACK singular values.  FP64 to 1e-12 relative, FP32 to 2e-5 relative
(K up to 300 products of FP32-rounded operands).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OPS = {0: lambda x: x, 1: lambda x: x.T, 2: lambda x: x.conj().T, 3: lambda x: x.conj()}


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


# BF16x3: each operand is hi + lo with 16 significant bits (2^-17 relative),
# products ~1.5e-5 relative; TF32x3: ~2^-22 per operand.  FP32 accumulation.
GEMM_TOL = [(0, 1e-12), (3, 2e-5), (1, 5e-5), (2, 5e-6)]


@pytest.mark.parametrize("prec,tol", GEMM_TOL)
@pytest.mark.parametrize("op_a", [0, 1, 2, 3])
@pytest.mark.parametrize("op_b", [0, 1, 2, 3])
def test_gemm_ops(prec, tol, op_a, op_b):
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(10 * op_a + op_b)
    m, n, k = 67, 131, 45
    a = _rand(rng, (m, k) if op_a in (0, 3) else (k, m))
    b = _rand(rng, (k, n) if op_b in (0, 3) else (n, k))
    want = OPS[op_a](a) @ OPS[op_b](b)
    got = binding.dmrgc_test_gemm(prec, a, b, op_a, op_b, m, n, k)
    assert np.abs(got - want).max() <= tol * np.abs(want).max() * np.sqrt(k)


@pytest.mark.parametrize("prec,tol", GEMM_TOL)
@pytest.mark.parametrize("m,n,k", [(130, 70, 300), (300, 257, 1000), (8, 8, 4000)])
def test_gemm_large_k(prec, tol, m, n, k):
    """Several M/N tiles, ragged edges, and K long enough for split-K."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(3 + k)
    a = _rand(rng, (m, k))
    b = _rand(rng, (n, k))
    want = a @ b.T
    got = binding.dmrgc_test_gemm(prec, a, b, 0, 1, m, n, k)
    assert np.abs(got - want).max() <= tol * np.abs(want).max() * np.sqrt(k)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 3e-5)])
@pytest.mark.parametrize("m,n", [(40, 40), (64, 30), (30, 64), (96, 96)])
def test_jacobi_svd(prec, tol, m, n):
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(m * 7 + n)
    # graded spectrum so that the ordering and the truncation are both exercised
    u, _ = np.linalg.qr(_rand(rng, (m, m)))
    v, _ = np.linalg.qr(_rand(rng, (n, n)))
    r = min(m, n)
    sv = np.exp(-np.linspace(0, 6, r))
    g = (u[:, :r] * sv) @ v[:, :r].conj().T
    chi = r // 2
    s, k, uk = binding.dmrgc_test_svd(prec, g, chi, 1e-12 if prec == 0 else 2e-5)
    assert np.abs(s[:r] - sv).max() <= tol * sv[0]
    assert k == chi
    assert np.allclose(uk.conj().T @ uk, np.eye(k), atol=10 * tol)
    # the kept vectors span the top-k left singular subspace
    p_true = u[:, :k] @ u[:, :k].conj().T
    assert np.abs(p_true @ uk - uk).max() < 1e3 * tol


@pytest.mark.parametrize("prec", [0, 3])
def test_jacobi_rank_deficient_wide(prec):
    """More columns than rows (the right-to-left case): columns that must go to
    zero are recognised as numerically zero and the rank is found."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(5)
    m, n, r = 24, 60, 9
    g = _rand(rng, (m, r)) @ _rand(rng, (r, n))
    want = np.linalg.svd(g, compute_uv=False)
    s, k, uk = binding.dmrgc_test_svd(prec, g, 40, 1e-12 if prec == 0 else 2e-5)
    assert k == r
    tol = 1e-12 if prec == 0 else 3e-5
    assert np.abs(s[:r] - want[:r]).max() <= tol * want[0]


@pytest.mark.parametrize("m,n", [(64, 48), (200, 130), (512, 512), (1000, 700), (1024, 1024), (37, 200)])
def test_jacobi_gram_kernel_matches_lapack(m, n):
    """The Gram-block Jacobi kernel (complex64, m <= 1024): singular values
    against LAPACK, orthonormal kept vectors spanning the top subspace, ragged
    sizes (n not a multiple of 8, m not of 512) included."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(m + 3 * n)
    r = min(m, n)
    u, _ = np.linalg.qr(_rand(rng, (m, r)))
    v, _ = np.linalg.qr(_rand(rng, (n, r)))
    sv = np.exp(-np.linspace(0, 5, r))
    g = (u * sv) @ v.conj().T
    chi = max(1, r // 2)
    binding.dmrgc_set_jacobi_kernel(1)
    try:
        s, k, uk = binding.dmrgc_test_svd(3, g, chi, 2e-5)
    finally:
        binding.dmrgc_set_jacobi_kernel(0)
    tol = 2e-5
    assert np.abs(s[:r] - sv).max() <= tol * sv[0] * 10
    assert k == chi
    assert np.allclose(uk.conj().T @ uk, np.eye(k), atol=1e-4)
    p_true = u[:, :k] @ u[:, :k].conj().T
    assert np.abs(p_true @ uk - uk).max() < 1e-2
