"""The allocation-free truncated SVD entry point against the allocating one.

Some callers cannot call cudaMalloc (their device memory is claimed by their
own allocator, or their loop must not pay the synchronisation an allocation
can cause); dmrgc_svd_noalloc serves them with scratch compiled into the
library.  Here the test is the caller: it owns the device buffers (torch) and
checks two calls in a row against dmrgc_test_svd, which allocates its own
memory, to the tolerances of the kernel tests.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _matrix(rng, m, n):
    u, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    v, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    r = min(m, n)
    s = np.exp(-np.linspace(0, 5, r))
    return (u[:, :r] * s) @ v[:, :r].conj().T


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 3e-5)])
def test_noalloc_svd_matches_allocating_entry_point(prec, tol):
    import torch

    from paper_2207_05612_gb300 import binding
    ctype = torch.complex128 if prec == 0 else torch.complex64
    rng = np.random.default_rng(2024)
    for call, (m, n, chi) in enumerate([(96, 80, 40), (64, 128, 48)]):
        g = _matrix(rng, m, n)
        s_ref, k_ref, u_ref = binding.dmrgc_test_svd(prec, g, chi, 1e-12 if prec == 0 else 2e-5)
        dev_g = torch.tensor(np.asfortranarray(g).reshape(-1, order="F"), dtype=ctype, device="cuda")
        dev_s = torch.zeros(n, dtype=torch.float64, device="cuda")
        dev_u = torch.zeros(m * min(chi, n), dtype=ctype, device="cuda")
        torch.cuda.synchronize()
        k = binding.dmrgc_svd_noalloc(prec, dev_g.data_ptr(), m, n, chi,
                                      1e-12 if prec == 0 else 2e-5, dev_s.data_ptr(),
                                      dev_u.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert k == k_ref, (call, k, k_ref)
        s = dev_s.cpu().numpy()
        assert np.abs(s - s_ref).max() <= tol * s_ref[0]
        u = dev_u[:m * k].cpu().numpy().astype(np.complex128).reshape(m, k)
        # same kept subspace (columns are defined up to phases)
        assert np.abs(u @ u.conj().T - u_ref @ u_ref.conj().T).max() < 100 * tol
        assert np.allclose(u.conj().T @ u, np.eye(k), atol=10 * tol)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2207_05612_gb300 import binding
    with pytest.raises(binding.DmrgcError) as e:
        binding.dmrgc_svd_noalloc(0, 1, 8, 4097, 4, 1e-12, 1, 1, 0)
    assert e.value.status == 1
