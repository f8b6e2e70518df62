"""Pins of the randomized-SVD certificate (CPU, float64): the Ky Fan bound
the library's acceptance test relies on, checked against exact SVDs."""
import numpy as np

from oracle import rsvd


def _matrix(rng, m, n, spectrum):
    u, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    v, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    r = len(spectrum)
    return (u[:, :r] * spectrum) @ v[:, :r].conj().T


def test_exact_low_rank_sketch_is_the_svd():
    """Rank 12 < sketch 20: the sketch spans the range, the certificate is 0
    to rounding, and the kept vectors and values are the SVD's."""
    rng = np.random.default_rng(0)
    sv = np.exp(-np.linspace(0, 3, 12))
    g = _matrix(rng, 60, 50, sv)
    q = rsvd.range_finder(g, 20, 1, rng)
    uk, sk, s_all = rsvd.sketch_svd(g, q, chi=8, rel_cut=1e-12)
    assert np.allclose(sk, sv[:8], rtol=1e-12)
    assert rsvd.certificate_excess(g, s_all, len(sk), 8) < 1e-12 * np.sum(sv ** 2)
    u_true, _, _ = np.linalg.svd(g)
    proj = u_true[:, :8] @ u_true[:, :8].conj().T
    assert np.allclose(proj @ uk, uk, atol=1e-10)


def test_bound_holds_for_any_sketch():
    """For random matrices and sketches of every size, the best rank-chi
    weight never exceeds the sketch's kept weight plus the certificate's
    excess (the Ky Fan inequality), and the excess is 0 only when the sketch
    is exact."""
    rng = np.random.default_rng(1)
    for trial in range(40):
        m, n = rng.integers(10, 40, size=2)
        r = int(min(m, n))
        sv = np.sort(rng.exponential(size=r))[::-1]
        g = _matrix(rng, m, n, sv)
        chi = int(rng.integers(1, r + 1))
        l = int(rng.integers(1, r + 1))
        q = rsvd.range_finder(g, l, int(rng.integers(0, 3)), rng)
        uk, sk, s_all = rsvd.sketch_svd(g, q, chi, rel_cut=1e-12)
        f = float(np.sum(sk ** 2))
        f_opt = float(np.sum(sv[:chi] ** 2))
        excess = rsvd.certificate_excess(g, s_all, len(sk), chi)
        assert f <= f_opt * (1 + 1e-12)
        assert f_opt <= f + excess + 1e-10 * f_opt, (trial, f_opt, f, excess)


def test_truncating_regime_fails_the_certificate():
    """A flat spectrum truncated at chi: a sketch of chi + 8 columns misses
    weight the optimum holds, and the excess exposes it (so the library falls
    back to the full SVD there)."""
    rng = np.random.default_rng(2)
    g = _matrix(rng, 64, 64, np.ones(64))
    q = rsvd.range_finder(g, 40, 1, rng)
    uk, sk, s_all = rsvd.sketch_svd(g, q, chi=32, rel_cut=1e-12)
    f = float(np.sum(sk ** 2))
    excess = rsvd.certificate_excess(g, s_all, len(sk), 32)
    assert excess > 1e-2 * f
