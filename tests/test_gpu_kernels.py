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


def test_gemm_accumulation_bias():
    """Sums of positive products: the CUDA-core FP32 GEMM is unbiased, the
    tensor-core modes come out systematically small, by about 1.8e-10 K
    (BF16x3) and 4.8e-10 K (TF32x3) relative for K real terms (the FP32
    accumulation of the tensor cores rounds toward zero).  Pins the reading
    behind the TF32x3 fidelity bound of the parity tests."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(11)
    K = 8192
    a = rng.random((128, K)) + 0j
    b = rng.random((256, K)) + 0j
    want = (a @ b.T).real
    bias = {}
    for prec in (1, 2, 3):
        got = binding.dmrgc_test_gemm(prec, a, b, 0, 1, 128, 256, K).real
        bias[prec] = float(((got - want) / want).mean())
    print("mean relative error at K = 8192:", bias)
    assert abs(bias[3]) < 2e-7
    assert -5e-6 < bias[1] < 0 and -1e-5 < bias[2] < 0


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


def _check_spectrum(s, want, g, tol=3e-5):
    """Singular values above the complex64 numerical-zero level (1e-5 |G|_F,
    whose columns the Jacobi kernels never rotate and the truncation never
    keeps) within tol * s_1 of LAPACK; the rest at or below a few times that
    level."""
    r = want.size
    zl = 1e-5 * np.linalg.norm(g)
    big = want > 3 * zl
    err = np.abs(s[:r] - want)
    i = int(np.argmax(np.where(big, err, 0)))
    print(f"max error {err[big].max():.2e} at index {i} (s = {want[i]:.3e}, s_1 = {want[0]:.3e}); "
          f"{int((~big).sum())} values below 3 x zero level {zl:.2e}")
    assert err[big].max() <= tol * want[0]
    assert np.all(s[:r][~big] <= 4 * zl)


def _weight(g, u):
    """|U^+ G|_F^2: the weight a truncation onto span(U) keeps."""
    return float(np.sum(np.abs(u.conj().T @ g) ** 2))


# The sweep's complex64 Jacobi kernels by size: m <= 256 -> jacobi_wp4<8, .>,
# m <= 512 -> <16, .>, m <= 1024 -> <32, .> (VEC = 2 for even m, 1 for odd m),
# m <= 2048 -> jacobi_reg<float, 16>.  At chi = 512 every saturated update runs
# <32, 2> on a 1024 x 1024 theta, at chi = 1024 jacobi_reg on 2048 x 2048.
SWEEP_SIZES = [(1024, 1024), (1000, 700), (600, 600), (300, 280), (1001, 640), (255, 300), (2048, 2048)]


@pytest.mark.parametrize("m,n", SWEEP_SIZES)
def test_jacobi_default_kernels_at_sweep_sizes(m, n):
    """The default complex64 kernels against LAPACK on flat (Porter-Thomas-like)
    spectra, as in the saturated sweep: every singular value, the kept rank,
    orthonormal kept vectors, and the kept weight |U_k^+ G|_F^2 equal to the
    optimum sum_{j<k} s_j^2 (Eckart-Young) to 1e-5."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(m * 13 + n)
    g = _rand(rng, (m, n)) / np.sqrt(2 * m)
    want = np.linalg.svd(g, compute_uv=False)
    r = min(m, n)
    chi = r // 2
    s, k, uk = binding.dmrgc_test_svd(3, g, chi, 2e-5)
    _check_spectrum(s, want, g)
    assert k == chi
    assert np.abs(uk.conj().T @ uk - np.eye(k)).max() < 1e-4
    f_opt = float(np.sum(want[:k] ** 2))
    assert abs(_weight(g, uk) - f_opt) <= 1e-5 * f_opt


@pytest.mark.parametrize("m,n", [(1024, 1024), (2048, 2048)])
def test_jacobi_default_kernels_graded_spectrum(m, n):
    """Graded spectrum through the same kernels: the singular values to
    3e-5 s_1 and the kept vectors in the top-k left singular subspace."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(m + 7)
    r = min(m, n)
    u, _ = np.linalg.qr(_rand(rng, (m, r)))
    v, _ = np.linalg.qr(_rand(rng, (n, r)))
    sv = np.exp(-np.linspace(0, 4, r))
    g = (u * sv) @ v.conj().T
    chi = r // 2
    s, k, uk = binding.dmrgc_test_svd(3, g, chi, 2e-5)
    _check_spectrum(s, sv, g)
    assert k == chi
    assert np.abs(uk.conj().T @ uk - np.eye(k)).max() < 1e-4
    f_opt = float(np.sum(sv[:k] ** 2))
    assert abs(_weight(g, uk) - f_opt) <= 1e-5 * f_opt


# ---- the Gram eigensolver path (options.svd_path 0): H = G G^+ by the
# contraction engine, Householder tridiagonalisation, bisection, FP64 inverse
# iteration, back-transformation.  Bounds: H from TF32x3 products carries an
# absolute error of ~1e-5 lambda_1, so s_j moves by ~1e-5 s_1 at s_j ~ s_1/2;
# the kept weight moves only at second order.
GRAM_SIZES = [(1024, 1024), (2048, 2048), (1000, 700), (600, 600), (300, 280), (130, 200), (1023, 2000)]


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("m,n", GRAM_SIZES)
def test_gram_eigensolver_svd_against_lapack(prec, m, n):
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(m * 17 + n)
    g = _rand(rng, (m, n)) / np.sqrt(2 * m)
    want = np.linalg.svd(g, compute_uv=False)
    chi = min(m, n) // 2
    s, k, uk = binding.dmrgc_test_svd_gram(prec, g, chi, 2e-5)
    assert k == chi
    err = np.abs(s[:k + 1] - want[:k + 1]).max()
    print(f"{m}x{n} prec {prec}: max |s - s_lapack| {err:.2e} (s_1 {want[0]:.3f})")
    assert err <= 3e-5 * want[0]
    assert np.abs(uk.conj().T @ uk - np.eye(k)).max() < 1e-4
    f_opt = float(np.sum(want[:k] ** 2))
    assert abs(_weight(g, uk) - f_opt) <= 1e-5 * f_opt


def test_gram_eigensolver_declines_unresolved_spectra():
    """A kept spectrum reaching below 3e-3 s_1 (1e-5 of the largest Gram
    eigenvalue) is left to the Jacobi SVD: k = -1."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(3)
    m = n = 512
    u, _ = np.linalg.qr(_rand(rng, (m, m)))
    v, _ = np.linalg.qr(_rand(rng, (n, n)))
    sv = np.exp(-np.linspace(0, 12, m))
    g = (u * sv) @ v.conj().T
    _, k, uk = binding.dmrgc_test_svd_gram(2, g, 256, 2e-5)
    assert k == -1 and uk is None
    # a rank-deficient matrix whose rank is below chi: the count is set by the cut
    g2 = _rand(rng, (m, 100)) @ _rand(rng, (100, n))
    _, k2, _ = binding.dmrgc_test_svd_gram(2, g2, 256, 2e-5)
    assert k2 == -1
    # ... which is trusted when the cut lies above the resolution level (the
    # zip-up's 4e-3: cut^2 = 1.6e-5 >= 1e-5): rank 100, spectrum 1 .. 0.1
    s3 = np.linspace(1.0, 0.1, 100)
    g3 = (u[:, :100] * s3) @ v[:, :100].conj().T
    s_out, k3, u3 = binding.dmrgc_test_svd_gram(2, g3, 256, 4e-3)
    assert k3 == 100
    assert np.abs(u3.conj().T @ u3 - np.eye(100)).max() < 1e-4
    proj = np.linalg.norm(u3.conj().T @ u[:, :100], axis=0)
    assert proj.min() > 1 - 1e-4


def test_gram_eigensolver_tiny_last_off_diagonal():
    """H = G G^+ block-diagonal, its last block 2 x 2 with an off-diagonal of
    -1e-15 i: the reduction leaves that entry as the tridiagonal form's last
    off-diagonal, and the phase reflector that makes it real would have
    tau ~ 1/|x|^2, beyond FP32, which the back-transformation would spread
    into every kept vector.  The reduction drops such a column instead (a
    perturbation far below the Gram's rounding): the vectors stay finite,
    orthonormal and optimal."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(8)
    m, n = 256, 300
    g = np.zeros((m, n), dtype=np.complex128)
    g[:m - 2, :n - 2] = _rand(rng, (m - 2, n - 2)) / np.sqrt(2 * m)
    g[m - 2, n - 2] = 1.0
    g[m - 1, n - 2] = 1e-15j
    g[m - 1, n - 1] = 1.0
    want = np.linalg.svd(g, compute_uv=False)
    s, k, uk = binding.dmrgc_test_svd_gram(2, g, 128, 2e-5)
    assert k == 128
    assert np.all(np.isfinite(uk))
    assert np.abs(s[:k + 1] - want[:k + 1]).max() <= 3e-5 * want[0]
    assert np.abs(uk.conj().T @ uk - np.eye(k)).max() < 1e-4
    f_opt = float(np.sum(want[:k] ** 2))
    assert abs(_weight(g, uk) - f_opt) <= 1e-5 * f_opt


def test_gram_eigensolver_degenerate_spectrum():
    """Exactly degenerate singular values (multiplets of 4) above the cut:
    inverse iteration inside a cluster is orthogonalised, so the kept vectors
    stay orthonormal and span the top subspace."""
    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(4)
    m = n = 256
    u, _ = np.linalg.qr(_rand(rng, (m, m)))
    v, _ = np.linalg.qr(_rand(rng, (n, n)))
    sv = np.repeat(np.linspace(1.0, 0.2, m // 4), 4)
    g = (u * sv) @ v.conj().T
    s, k, uk = binding.dmrgc_test_svd_gram(2, g, 128, 2e-5)
    assert k == 128
    assert np.abs(s[:k] - sv[:k]).max() <= 3e-5
    assert np.abs(uk.conj().T @ uk - np.eye(k)).max() < 1e-4
    p_true = u[:, :k] @ u[:, :k].conj().T
    assert np.abs(p_true @ uk - uk).max() < 1e-3
