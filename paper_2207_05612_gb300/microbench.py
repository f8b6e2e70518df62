"""Kernel micro-benchmarks through the C ABI, one kernel class at a time, on
seeded random inputs.  Also the small-case driver for profiler captures of a
single kernel.

  python -m paper_2207_05612_gb300.microbench gemm --precision bf16x3 --m 65536 --n 1024 --k 512
  python -m paper_2207_05612_gb300.microbench svd --precision fp32 --m 1024 --n 1024 [--jacobi gram]
  python -m paper_2207_05612_gb300.microbench gram --precision tf32x3 --m 1024 --n 1024
  python -m paper_2207_05612_gb300.microbench readout --precision bf16x3 --rows 6 --cols 9 --chi 512 --count 16384

gemm: C = A B through dmrgc_test_gemm (host complex128 buffers in and out, so
the wall time includes the transfers and the operand split); reports the wall
time per call and the algorithmic complex flops 8 M N K.
svd: the one-sided Jacobi, truncation and gather on a device matrix through
dmrgc_svd_noalloc, timed with CUDA events on its stream; the matrix is
re-copied from a pristine device copy before each call (the copy is outside
the events).
gram: the Gram-eigensolver truncated SVD (chi = m / 2) through
dmrgc_test_svd_gram (host buffers in and out): the Gram product, the
tridiagonalisation, bisection, inverse iteration, the cluster pass and the
back-transformation, one launch each per call; reports the wall time per call
and the largest error of the kept singular values against LAPACK.
readout: a seeded random right-canonical MPS (rows x cols qubits, bonds
min(2^i, 2^(N-i), chi)) loaded with dmrgc_set_mps, then one amplitude call
for `count` random bit strings and one sampling call for `count` samples
(one per site: a chunk GEMM V A and the select kernel); reports the wall time
of each call and the algorithmic bytes of one select launch at the largest
bond.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding

PREC = {"fp64": binding.DMRGC_FP64, "bf16x3": binding.DMRGC_BF16X3,
        "tf32x3": binding.DMRGC_TF32X3, "fp32": binding.DMRGC_FP32}


def _cplx(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)


def bench_gemm(prec: int, m: int, n: int, k: int, reps: int, seed: int) -> dict:
    rng = np.random.default_rng(seed)
    a = _cplx(rng, (m, k))
    b = _cplx(rng, (k, n))
    binding.dmrgc_test_gemm(prec, a, b, 0, 0, m, n, k)   # warm-up
    t0 = time.perf_counter()
    for _ in range(reps):
        c = binding.dmrgc_test_gemm(prec, a, b, 0, 0, m, n, k)
    dt = (time.perf_counter() - t0) / reps
    rows = rng.choice(m, size=min(m, 64), replace=False)
    ref = a[rows] @ b
    err = float(np.abs(c[rows] - ref).max() / np.abs(ref).max())
    return {"kernel": "gemm", "m": m, "n": n, "k": k, "wall_ms_per_call": dt * 1e3,
            "algorithmic_gflop": 8.0 * m * n * k / 1e9, "max_rel_err_sampled_rows": err,
            "note": "wall time includes host<->device copies and operand split"}


def bench_svd(prec: int, m: int, n: int, reps: int, seed: int) -> dict:
    import torch
    rng = np.random.default_rng(seed)
    g = _cplx(rng, (m, n)) / np.sqrt(m * n)
    cdt = torch.complex128 if prec == binding.DMRGC_FP64 else torch.complex64
    dev = torch.device("cuda")
    # column-major m x n = row-major n x m transposed
    pristine = torch.from_numpy(np.ascontiguousarray(g.T)).to(cdt).to(dev)
    work = torch.empty_like(pristine)
    s = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.empty(m * n, dtype=cdt, device=dev)
    st = torch.cuda.current_stream()
    chi = n

    def call():
        return binding.dmrgc_svd_noalloc(prec, work.data_ptr(), m, n, chi, 1e-12, s.data_ptr(),
                                         u.data_ptr(), st.cuda_stream)

    work.copy_(pristine)
    call()   # warm-up (and the first-call set-up)
    times = []
    for _ in range(reps):
        work.copy_(pristine)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        call()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ref = np.linalg.svd(g, compute_uv=False)
    err = float(np.abs(s.cpu().numpy()[:ref.size] - ref).max() / ref[0])
    return {"kernel": "svd", "m": m, "n": n, "ms_per_call": float(np.median(times)),
            "max_rel_err_s": err}


def bench_gram(prec: int, m: int, n: int, reps: int, seed: int) -> dict:
    rng = np.random.default_rng(seed)
    g = _cplx(rng, (m, n)) / np.sqrt(m)
    chi = min(m, n) // 2
    binding.dmrgc_test_svd_gram(prec, g, chi, 2e-5)   # warm-up
    t0 = time.perf_counter()
    for _ in range(reps):
        s, k, _ = binding.dmrgc_test_svd_gram(prec, g, chi, 2e-5)
    dt = (time.perf_counter() - t0) / reps
    ref = np.linalg.svd(g, compute_uv=False)
    err = float(np.abs(s[:chi] - ref[:chi]).max() / ref[0])
    return {"kernel": "gram", "m": m, "n": n, "chi": chi, "k": k, "wall_ms_per_call": dt * 1e3,
            "max_rel_err_kept_s": err, "note": "wall time includes host<->device copies"}


def random_right_canonical(n: int, chi: int, rng) -> list:
    """Tensors [chi_l][2][chi_r] whose sites 1..n-1 have orthonormal rows of
    the (chi_l, 2 chi_r) reshape and site 0 unit norm: a normalised state."""
    bonds = [min(2 ** i, 2 ** (n - i), chi) for i in range(n + 1)]
    mps = [None] * n
    for i in range(n - 1, 0, -1):
        cl, cr = bonds[i], bonds[i + 1]
        q, _ = np.linalg.qr(_cplx(rng, (cl, 2 * cr)).conj().T)
        mps[i] = q.conj().T.reshape(cl, 2, cr)
    a0 = _cplx(rng, (1, 2, bonds[1]))
    mps[0] = a0 / np.linalg.norm(a0)
    return mps


def bench_readout(prec: int, rows: int, cols: int, chi: int, count: int, seed: int) -> dict:
    rng = np.random.default_rng(seed)
    n = rows * cols
    mps = random_right_canonical(n, chi, rng)
    ctx = binding.Context(rows, cols, chi, precision=prec)
    ctx.set_mps(mps)
    bits = rng.integers(0, 2, size=(count, n), dtype=np.uint8)
    ctx.amplitude(bits[:16])   # warm-up: one launch per site
    t0 = time.perf_counter()
    amp = ctx.amplitude(bits)
    t_amp = time.perf_counter() - t0
    t0 = time.perf_counter()
    smp = ctx.sample(count, seed)
    t_smp = time.perf_counter() - t0
    ctx.close()
    esz = 16 if prec == binding.DMRGC_FP64 else 8
    bonds = [a.shape[2] for a in mps]
    # per site, W [count][2 chi_r] is the chain GEMM's output: the amplitude
    # select reads the chosen half and writes V [count][chi_r]; the sampling
    # select reads both halves (p_0, p_1) and writes V
    mb = max(bonds)
    return {"kernel": "readout", "n_qubits": n, "chi": chi, "count": count,
            "amplitude_wall_ms": t_amp * 1e3, "sample_wall_ms": t_smp * 1e3, "max_bond": mb,
            "amp_select_bytes_at_max_bond": count * 2 * mb * esz,
            "sample_select_bytes_at_max_bond": count * 3 * mb * esz,
            "amp_finite": bool(np.all(np.isfinite(amp))), "samples_shape": list(smp.shape),
            "note": "wall times include host<->device copies of bits, amplitudes and samples"}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("kernel", choices=["gemm", "svd", "gram", "readout"])
    ap.add_argument("--precision", default="bf16x3", choices=list(PREC))
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--k", type=int, default=512)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rows", type=int, default=6, help="readout: grid rows")
    ap.add_argument("--cols", type=int, default=9, help="readout: grid columns")
    ap.add_argument("--chi", type=int, default=512, help="readout: bond dimension")
    ap.add_argument("--count", type=int, default=16384, help="readout: bit strings and samples")
    ap.add_argument("--jacobi", default="wp4", choices=["wp4", "gram"],
                    help="complex64 Jacobi kernel for m <= 1024")
    a = ap.parse_args(argv)
    binding.dmrgc_set_jacobi_kernel(0 if a.jacobi == "wp4" else 1)
    prec = PREC[a.precision]
    if a.kernel == "gemm":
        out = bench_gemm(prec, a.m, a.n, a.k, a.reps, a.seed)
    elif a.kernel == "gram":
        out = bench_gram(prec, a.m, a.n, a.reps, a.seed)
    elif a.kernel == "readout":
        out = bench_readout(prec, a.rows, a.cols, a.chi, a.count, a.seed)
    else:
        out = bench_svd(prec, a.m, a.n, a.reps, a.seed)
    out["precision"] = a.precision
    out["jacobi"] = a.jacobi
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
