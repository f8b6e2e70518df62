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


def test_noalloc_svd_against_lapack_and_allocates_nothing():
    """At 1024 x 1024 (the saturated theta of chi = 512, the kernel the sweep
    runs there) the singular values match LAPACK and the kept vectors carry the
    optimal weight; after a first call has resolved the scratch address,
    further calls leave the device's free memory and torch's allocator
    untouched."""
    import torch

    from paper_2207_05612_gb300 import binding
    rng = np.random.default_rng(7)
    m = n = 1024
    chi = 512
    g = (rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))) / np.sqrt(2 * m)
    want = np.linalg.svd(g, compute_uv=False)
    stream = torch.cuda.current_stream().cuda_stream
    host_g = torch.tensor(np.asfortranarray(g).reshape(-1, order="F"), dtype=torch.complex64)
    dev_g = torch.empty_like(host_g, device="cuda")
    dev_s = torch.zeros(n, dtype=torch.float64, device="cuda")
    dev_u = torch.zeros(m * chi, dtype=torch.complex64, device="cuda")
    dev_g.copy_(host_g)
    torch.cuda.synchronize()
    binding.dmrgc_svd_noalloc(3, dev_g.data_ptr(), m, n, chi, 2e-5, dev_s.data_ptr(), dev_u.data_ptr(), stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(2):
        dev_g.copy_(host_g)
        torch.cuda.synchronize()
        k = binding.dmrgc_svd_noalloc(3, dev_g.data_ptr(), m, n, chi, 2e-5, dev_s.data_ptr(),
                                      dev_u.data_ptr(), stream)
        torch.cuda.synchronize()
        assert k == chi
        s = dev_s.cpu().numpy()
        big = want > 3e-5 * np.linalg.norm(g)   # above the complex64 numerical-zero level
        assert np.abs(s - want)[big].max() <= 3e-5 * want[0]
        u = dev_u.cpu().numpy().astype(np.complex128).reshape(m, k)
        assert np.abs(u.conj().T @ u - np.eye(k)).max() < 1e-4
        f_opt = float(np.sum(want[:k] ** 2))
        assert abs(float(np.sum(np.abs(u.conj().T @ g) ** 2)) - f_opt) <= 1e-5 * f_opt
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2207_05612_gb300 import binding
    with pytest.raises(binding.DmrgcError) as e:
        binding.dmrgc_svd_noalloc(0, 1, 8, 4097, 4, 1e-12, 1, 1, 0)
    assert e.value.status == 1
