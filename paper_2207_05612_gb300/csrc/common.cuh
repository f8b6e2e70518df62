// Shared declarations of the dmrgc CUDA library (device helpers, kernel
// launchers, the context).  Complex numbers are stored as interleaved
// (re, im) pairs: double2 in FP64 mode, float2 in the complex64 modes.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dmrgc.h"

namespace dmrgc {

// ------------------------------------------------------------------ complex

template <typename R> struct cplx;
template <> struct cplx<double> { using T = double2; };
template <> struct cplx<float> { using T = float2; };

template <typename C2>
__host__ __device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return C2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C2>
__host__ __device__ __forceinline__ C2 cconj(C2 a) { return C2{a.x, -a.y}; }
template <typename C2>
__host__ __device__ __forceinline__ C2 cadd(C2 a, C2 b) { return C2{a.x + b.x, a.y + b.y}; }

// ------------------------------------------------------------------- GEMM

// Row-major batched complex GEMM:  C[b] = alpha * op(A[b]) * op(B[b]) (+ beta*C[b])
// op(A)[m][k]: OP_N A[m*lda+k], OP_T A[k*lda+m], OP_C conj(A[k*lda+m]), OP_R conj(A[m*lda+k])
// op(B)[k][n]: OP_N B[k*ldb+n], OP_T B[n*ldb+k], OP_C conj(B[n*ldb+k]), OP_R conj(B[k*ldb+n])
// batch index b = i1*b2 + i2 with element offsets i1*s?1 + i2*s?2.
enum Op { OP_N = 0, OP_T = 1, OP_C = 2, OP_R = 3 };

struct GemmArgs {
  int M = 0, N = 0, K = 0;
  int b1 = 1, b2 = 1;
  const void* A = nullptr; long long lda = 0, sA1 = 0, sA2 = 0; int opA = OP_N;
  const void* B = nullptr; long long ldb = 0, sB1 = 0, sB2 = 0; int opB = OP_N;
  void* C = nullptr; long long ldc = 0, sC1 = 0, sC2 = 0;
  double alpha_re = 1.0, alpha_im = 0.0;
  int beta_one = 0;   // 1: accumulate into C
  int upper_only = 0; // 1 (M == N, one instance, tensor-core path): only the output tiles that
                      // touch the upper triangle are computed; C below them is left undefined
};

cudaError_t gemm_simt(const GemmArgs& g, bool fp64, cudaStream_t st);

// Tensor-core path (complex64 data): packed split operands live in TcWork.
// err_dev: device int set to DMRGC_ETIMEOUT if a bounded wait ran out.
struct TcWork {
  // 0-3: packed split operands (A hi, A lo, B hi, B lo); 4: split-K partials
  void* buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t cap[5] = {0, 0, 0, 0, 0};
  cudaError_t ensure(int i, size_t bytes);
  void release();
};
// *launches (optional): kernels launched (operand packs, C clear, the GEMM)
cudaError_t gemm_tc(const GemmArgs& g, int precision, TcWork& w, int* err_dev, cudaStream_t st,
                    int* launches = nullptr);

// --------------------------------------------------------------------- SVD

// One-sided (Hestenes) Jacobi on the columns of G (column-major, m x n,
// leading dimension m), in place: on return G = W = G0 V with mutually
// orthogonal columns.  fro2: device pointer to |G|_F^2; columns with norm
// below zero_rel*|G|_F are treated as zero.  ctl must point to device scratch
// of jacobi_ctl_bytes(n); it starts with a JacobiStatus the host may read.
struct JacobiStatus {
  int err;                        // 0, DMRGC_ETIMEOUT or DMRGC_ENOCONV
  int sweeps;                     // sweeps executed
  unsigned long long rotations;   // rotations applied
};
size_t jacobi_ctl_bytes(int n);
cudaError_t jacobi_orthogonalize(void* G, int m, int n, bool fp64, double tol, int max_sweeps,
                                 const double* fro2, double zero_rel, void* ctl, cudaStream_t st,
                                 int* launches);

// Column norms of W, sort descending, truncation rank.  Writes into res (device):
// res->k, res->f = sum_{j<k} s_j^2, res->perm[j], res->s[j] (sorted).
// squared: the column norms are s^2 (Gram input) -> s = sqrt(norm).
// tie_rel > 0: if the cut falls inside a multiplet (s_k - s_{k+1} <= tie_rel*s_1),
// k is lowered to the multiplet's upper edge so that the kept subspace is unique.
struct TruncResult {
  int k;
  int n;
  int status;     // 0 ok, 5 = numeric (NaN/zero)
  int pad;        // 1: the cut fell in a multiplet reaching s_1 (kept at chi, not unique)
  double f;       // sum of kept s^2
  double norm2;   // sum of all s^2
  int nnz;        // columns above the numerical-zero level (the rank found)
  int by_cut;     // 1: k was set by the cutoff (fewer than min(chi, n) values above it)
  double tail;    // (s_{k-1} / s_1)^2: the smallest kept Gram eigenvalue over the largest
};
size_t trunc_bytes(int n);  // TruncResult followed by double s[n], int perm[n]
// fro2 / zero_rel: the Frobenius norm^2 of the matrix given to the Jacobi kernel
// and its zero level; columns at or below that level are never kept.
cudaError_t truncate_columns(const void* W, int m, int n, bool fp64, int chi, double rel_cut,
                             bool squared, double tie_rel, const double* fro2, double zero_rel,
                             void* res, cudaStream_t st);

// Gather kept columns into MPS layouts.  mode:
//  0: out[row*k + j] = W[row + perm[j]*m] / scale_j            (U_k row-major [m][k])
//  1: out[j*m + row] = W[row + perm[j]*m] / scale_j            (U_k^T, [k][m])
//  2: out[j*m + row] = conj(W[row + perm[j]*m]) / scale_j      (V_k^+, [k][m])
// scale_j = s_j (or s_j^2 when squared: Gram input, where the column norm is s^2).
cudaError_t gather_columns(const void* W, int m, int n_total, int k, const void* res,
                           bool squared, int mode, void* out, bool fp64, cudaStream_t st);

// Truncated SVD through the Gram matrix's eigenproblem (eig_herm.cu), complex64.
// H: n x n row-major Hermitian (overwritten), 3 <= n <= 2048.  Keeps
// k = min(chi, n, #{s > cut s_1}) with the multiplet rule of tie_rel (> 0)
// and writes res (TruncResult + s[n] + perm[n], as truncate_columns) and the
// k leading eigenvectors to out: mode 0 out[r * k + v], mode 1 out[v * n + r],
// mode 2 out[v * n + r] conjugated.  res->status: 0 done; 1 not resolved
// (lambda_{k-1} < resolve * lambda_0, or the count set by a cut with
// cut^2 < resolve: use the Jacobi SVD; nothing is written to out);
// DMRGC_ENUMERIC; DMRGC_ETIMEOUT.
size_t eig_work_bytes(int n, int kk);
cudaError_t eig_truncate(void* H, int n, int chi, double cut, double tie_rel, double resolve, void* work,
                         void* res, void* out, int mode, cudaStream_t st, int* launches);
// |x|^2 (FP64 sum in a fixed order: the same bits on every run) to *out_dev;
// x /= |x| if scale.  part_dev: 256 doubles of scratch.  Two kernels of 256 CTAs.
cudaError_t norm2_scale(void* x, long long n, bool fp64, double* out_dev, double* part_dev, bool scale,
                        cudaStream_t st);

// Spectrum read-outs of a truncation result (k = kept count):
// out32[j] = log10(s_mu^2 / sum_{nu<k} s_nu^2) at mu = round(j (k-1) / 31), j < 32;
// *out = smallest r with sum_{mu<r} s_mu^2 >= frac * sum_{mu<k} s_mu^2.
cudaError_t spectrum_summary(const void* res, int k, float* out32, cudaStream_t st);
cudaError_t rank_label(const void* res, int k, double frac, int* out, cudaStream_t st);

// n complex entries of unit variance, E|z|^2 = 1: Box-Muller on SplitMix64
// uniforms at counters ctr0 + 2j, ctr0 + 2j + 1 (entry j).
cudaError_t fill_gaussian(void* dst, long long n, bool fp64, unsigned long long seed,
                          unsigned long long ctr0, cudaStream_t st);
// n complex entries (2u - 1) + i (2u' - 1), u, u' the SplitMix64 uniforms at
// counters ctr0 + 2j, ctr0 + 2j + 1 (entry j): the random guess of the
// single-site variant (Sec. V.D.1).
cudaError_t fill_unit_square(void* dst, long long n, bool fp64, unsigned long long seed,
                             unsigned long long ctr0, cudaStream_t st);

// Rank model (mlp.cu): BF16 copy of the FP32 parameters, and one inference
// from 32 device floats (the spectrum summary) + 4 host extras.
cudaError_t mlp_to_bf16(const float* params_dev, void* out_bf16, cudaStream_t st);
cudaError_t mlp_infer_one(const void* w_bf16, const float* feat32, const float* extras, float* y,
                          cudaStream_t st);

// ---------------------------------------------------------------- MPO build

struct GateDev {   // device copy of one gate, already in site order
  int p, q;        // sites, p < q; q = -1 for a one-qubit gate
  int swap;        // 1: the given matrix lists q1's index first
  int pad;
  double mat[32];
};
// Operator Schmidt split of every two-qubit gate (App. A splitting):
// U = sum_k A_k (x) B_k, k < rank; A, B stored [gate][4][2][2] complex128.
cudaError_t gate_split(const GateDev* gates, int n_gates, int* rank, double2* fa, double2* fb,
                       cudaStream_t st);

// Build W_i of one site from its plan: writes Wx[s][w_out][w_in][t] and
// Wy[s][w_in][w_out][t] in the working precision.
struct SitePlan {
  int d_in, d_out;
  int n_in, n_out, n_ops, pad;
  long long off;   // offset (ints) into the plan table of this site's records
};
cudaError_t build_site_mpo(const int* plan_tab, SitePlan sp, const GateDev* gates, const double2* fa,
                           const double2* fb, void* wx, void* wy, bool fp64, cudaStream_t st);

// ------------------------------------------------------------------- misc

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum
// (minus its static shared memory), once per kernel and thread-safely, so that
// host threads launching the same kernel with different sizes on different
// streams never lower the limit under one another.
cudaError_t allow_dyn_smem(const void* fn);

cudaError_t copy_transpose(const void* src, int rows, int cols, bool conj, void* dst, bool fp64,
                           cudaStream_t st);   // dst[c*rows + r] = op(src[r*cols + c])
cudaError_t copy_conj(const void* src, long long n, void* dst, bool fp64, cudaStream_t st);
// 4-index transpose of a complex tensor: dims are the input's, out axis k is in axis perm[k]
cudaError_t permute4(const void* src, const int* dims, const int* perm, void* dst, bool fp64, cudaStream_t st);
cudaError_t permute_phys_first(const void* src, int a, int b, void* dst, bool fp64,
                               cudaStream_t st);  // [a][2][b] -> [2][a][b]
cudaError_t set_identity(void* dst, int n, bool fp64, cudaStream_t st);  // n x n
cudaError_t set_scalar_one(void* dst, bool fp64, cudaStream_t st);
cudaError_t sum_abs2(const void* x, long long n, bool fp64, double* out_dev, cudaStream_t st);
cudaError_t scale_inplace(void* x, long long n, const double* norm2_dev, bool fp64,
                          cudaStream_t st);
cudaError_t to_complex128(const void* src, long long n, bool fp64, double2* dst, cudaStream_t st);
cudaError_t from_complex128(const double2* src, long long n, bool fp64, void* dst, cudaStream_t st);

// --------------------------------------------------------------- read-outs

// Batched read-outs (readout.cu), one site at a time, for a chunk of B strings
// whose running row vectors V[B][l] the caller multiplies by the site tensor
// (W[B][2 r] = V A_i, the contraction engine) before each call:
//  readout_start: V[b][0] = 1;
//  amp_select:    V[b][c] = W[b][x_b r + c], x_b = the bits of the tensor's g
//                 qubits (qubits[0..g), the first the most significant), W[B][2^g r];
//  sample_select: draws bit x of sample row0 + b at `site` from p_x = |W_x|^2
//                 (T = null) or Re <T_x, W_x> (T = W E, left of the centre),
//                 out[(row0 + b) * n + qubit] = x, V[b] = W_x / sqrt(p_x);
//  amp_store:     out[b] = V[b][0] as complex128.
cudaError_t readout_start(void* V, int B, bool fp64, cudaStream_t st);
cudaError_t amp_select(const void* W, int B, int r, const unsigned char* bits, int n, const int* qubits, int g,
                       void* V, bool fp64, cudaStream_t st);
cudaError_t sample_select(const void* W, const void* T, int B, int r, unsigned long long seed, long long row0, int n,
                          int site, int qubit, unsigned char* out, void* V, bool fp64, cudaStream_t st);
cudaError_t amp_store(const void* V, int B, double2* out, bool fp64, cudaStream_t st);
// Metropolis chains (App. C), step t of `steps` for C chains over n qubits:
// metro_draw writes the proposals prop[C][n] and acceptance uniforms uacc[C]
// (SplitMix64 at counters g (n + 1) + q and g (n + 1) + n, g = c (steps + 1) + t);
// metro_step, given the proposals' amplitudes, moves chain c iff t = 0, its
// weight pcur[c] is 0 or uacc[c] pcur[c] < |amp[c]|^2 (acc[c] counts moves
// at t >= 1), and for t >= 1 writes its string to out[c][t - 1][n].
cudaError_t metro_draw(unsigned char* prop, double* uacc, int C, int n, int steps, int t, unsigned long long seed,
                       cudaStream_t st);
cudaError_t metro_step(const unsigned char* prop, const double2* amp, const double* uacc, unsigned char* cur,
                       double* pcur, long long* acc, unsigned char* out, int C, int n, int steps, int t,
                       cudaStream_t st);

}  // namespace dmrgc
