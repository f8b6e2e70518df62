"""CPU oracle for the circuit-DMRG compression sweep, in complex128.

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
CPU-baseline leg may import or run anything here; the product path never does.
It shares no code with the CUDA library: the two meet only through the seeded
gate lists of the `synthetic` package.

Two tiers:
* `statevector`: the plain definition, Eq. (perfect) and Eq. (F-sup): the
  exact state, exact fidelity, exact Schmidt spectra (N <= ~24).
* `mpo`, `dmrg`: the two-site compression step taken step by step
  (Sec. IV.B, Eq. (scalarproduct), Eq. (optimization), Eq. (Ftilde-sup),
  Eq. (fa-sup)) with numpy einsum and LAPACK SVD.
* `single_site`: the paper's own single-tensor update with grouped qubits
  (Sec. IV.A, IV.B.1, V.C), M = F / sqrt(f) from a seeded random guess.

Pins for every function live in tests/test_oracle_*.py.
"""
