"""CPU checks that constructed inputs of the GPU tests have the structure their
docstrings rely on (so that a GPU test exercises the case it names)."""
import numpy as np
from scipy import linalg


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_block_diagonal_gram_ends_its_tridiagonal_form_with_a_tiny_coupling():
    """The input of test_gram_eigensolver_tiny_last_off_diagonal: H = G G^+ is
    block-diagonal, its last 2 x 2 block coupled by -1e-15 i.  A Householder
    reduction of H (LAPACK's, through scipy) leaves that coupling as the last
    off-diagonal, complex and of size 1e-15 relative to max H_ii, while every
    other column it reduces is of order one: the last phase reflector is the
    one whose tau (~ 1 / |x|^2) leaves FP32."""
    rng = np.random.default_rng(8)
    m, n = 256, 300
    g = np.zeros((m, n), dtype=np.complex128)
    g[:m - 2, :n - 2] = _rand(rng, (m - 2, n - 2)) / np.sqrt(2 * m)
    g[m - 2, n - 2] = 1.0
    g[m - 1, n - 2] = 1e-15j
    g[m - 1, n - 1] = 1.0
    h = g @ g.conj().T
    h /= h.diagonal().real.max()
    assert np.abs(h[:m - 2, m - 2:]).max() == 0.0
    t = linalg.hessenberg(h)
    sub = np.abs(np.diag(t, -1))
    assert 1e-17 < sub[-1] < 1e-14
    assert sub[-2] == 0.0 or sub[-2] < 1e-14      # the block boundary
    assert np.median(sub[:m - 3]) > 1e-2
    # in FP32 the phase reflector of that (imaginary) entry overflows:
    # beta = -|x|, u0 = |x| + i Im x, q = -1 / (beta |u0|^2) = 1 / (2 |x|^3)
    x = np.float32(sub[-1])
    with np.errstate(over="ignore", divide="ignore", under="ignore"):
        q = np.float32(1.0) / (x * (np.float32(2) * x * x))
    assert not np.isfinite(q)
