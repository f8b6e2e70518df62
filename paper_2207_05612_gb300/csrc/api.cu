// C ABI and host orchestration of the compression step (Sec. IV.B).
//
// Data layout in device memory (row-major, complex interleaved):
//   MPS site i          A_i[chi_i][2][chi_{i+1}]     (new state)  B_i (previous state)
//   layer MPO site i    Wx_i[s][D_{i+1}][D_i][t]  and  Wy_i[s][D_i][D_{i+1}][t]
//   left environment    L[a_new][w][b_old],  right environment R[c_new][w][b_old]
//   X_i = L_{i-1} B_i W_i        [a][s][w'][b']   (cached per site)
//   Y_i = R_{i+1} B_i W_i        [s][c][w][b]     (cached per site)
//   theta at bond (i,i+1) = X_i Y_{i+1}^T   [(a s1)][(s2 c)]   (Eq. scalarproduct)
// Every contraction is one batched complex GEMM; the truncated SVD is the
// one-sided Jacobi kernel.  X_i computed in a left-to-right update is what the
// next right-to-left pass needs at the same bond, and Y_{i+1} likewise the
// other way round, so each update computes one of X / Y and reuses the other.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ctx.cuh"

using namespace dmrgc;

using namespace dmrgc_host;


namespace dmrgc_host {

dmrgc_status fail(dmrgc_ctx* c, dmrgc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}


dmrgc_status ensure(dmrgc_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return DMRGC_OK;
  if (b.p) {
    cudaStreamSynchronize(c->st);
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&b.p, bytes);
    want = bytes;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(c, DMRGC_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  b.cap = want;
  return DMRGC_OK;
}

// ---- timing

cudaEvent_t take_event(dmrgc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}


void flush_timing(dmrgc_ctx* c) {
  for (auto& p : c->pend) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    switch (p.cls) {
      case TC_GEMM: c->stats.gemm_ms += ms; c->stats.gemm_flops += p.flops; break;
      case TC_SVD: c->stats.svd_ms += ms; break;
      case TC_MPO: c->stats.mpo_ms += ms; break;
      default: c->stats.other_ms += ms; break;
    }
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pend.clear();
}

dmrgc_status sync(dmrgc_ctx* c) {
  CK(cudaStreamSynchronize(c->st));
  flush_timing(c);
  if (c->tcerr.p) {
    int e = 0;
    CK(cudaMemcpy(&e, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return fail(c, DMRGC_ETIMEOUT, "a tensor-core GEMM wait timed out");
  }
  return DMRGC_OK;
}

// ---- GEMM dispatch

cudaError_t run_gemm(int precision, const GemmArgs& g, TcWork* w, int* err_dev, cudaStream_t st,
                     int* launches = nullptr) {
  if (precision == DMRGC_BF16X3 || precision == DMRGC_TF32X3) return gemm_tc(g, precision, *w, err_dev, st, launches);
  if (launches) *launches = 1;
  return gemm_simt(g, precision == DMRGC_FP64, st);
}

dmrgc_status gemm(dmrgc_ctx* c, const GemmArgs& g, int precision) {
  if (precision < 0) precision = c->opt.precision;
  const bool tc = precision == DMRGC_BF16X3 || precision == DMRGC_TF32X3;
  if (tc && !c->tcerr.p) {
    TRY(ensure(c, c->tcerr, 64));
    CK(cudaMemsetAsync(c->tcerr.p, 0, 64, c->st));
  }
  const double fl = 8.0 * g.M * (double)g.N * g.K * g.b1 * g.b2;
  Span sp(c, TC_GEMM, fl);
  int launches = 0;
  CK(run_gemm(precision, g, &c->tcw, (int*)c->tcerr.p, c->st, &launches));
  c->stats.gemm_launches++;
  c->stats.kernel_launches += launches;
  return DMRGC_OK;
}

// X[a][s][w'][b'] = L[a][w][b] B[b][t][b'] W[w][s][t][w']
dmrgc_status make_x(dmrgc_ctx* c, const EnvRef& L, int site, DevBuf& out) {
  const int a = L.a, dw = L.w, b = L.b;
  const int bp = c->chiB[site + 1];
  const int dout = c->D[site + 1];
  if (dw != c->D[site] || b != c->chiB[site]) return fail(c, DMRGC_ESTATE, "make_x: shape mismatch");
  TRY(ensure(c, c->T, (size_t)a * dw * 2 * bp * c->esz));
  TRY(ensure(c, out, (size_t)a * 2 * dout * bp * c->esz));
  GemmArgs g1;
  g1.M = a * dw; g1.N = 2 * bp; g1.K = b;
  g1.A = L.p; g1.lda = b; g1.opA = OP_N;
  g1.B = c->B[site].p; g1.ldb = 2 * bp; g1.opB = OP_N;
  g1.C = c->T.p; g1.ldc = 2 * bp;
  TRY(gemm(c, g1));
  GemmArgs g2;
  g2.M = 2 * dout; g2.N = bp; g2.K = 2 * dw; g2.b1 = a;
  g2.A = c->Wx[site].p; g2.lda = 2 * dw; g2.sA1 = 0; g2.opA = OP_N;
  g2.B = c->T.p; g2.ldb = bp; g2.sB1 = (long long)dw * 2 * bp; g2.opB = OP_N;
  g2.C = out.p; g2.ldc = bp; g2.sC1 = (long long)2 * dout * bp;
  return gemm(c, g2);
}

// Y[s][c][w][b] = R[c][w''][b''] B[b][t][b''] W[w][s][t][w'']
dmrgc_status make_y(dmrgc_ctx* c, const EnvRef& R, int site, DevBuf& out) {
  const int cc = R.a, dout = R.w, bpp = R.b;
  const int bl = c->chiB[site];
  const int din = c->D[site];
  if (dout != c->D[site + 1] || bpp != c->chiB[site + 1]) return fail(c, DMRGC_ESTATE, "make_y: shape mismatch");
  TRY(ensure(c, c->bt, (size_t)2 * bl * bpp * c->esz));
  {
    Span sp(c, TC_OTHER);
    CK(permute_phys_first(c->B[site].p, bl, bpp, c->bt.p, c->fp64, c->st));
    c->stats.kernel_launches++;
  }
  TRY(ensure(c, c->T, (size_t)cc * dout * 2 * bl * c->esz));
  TRY(ensure(c, out, (size_t)2 * cc * din * bl * c->esz));
  GemmArgs g1;
  g1.M = cc * dout; g1.N = 2 * bl; g1.K = bpp;
  g1.A = R.p; g1.lda = bpp; g1.opA = OP_N;
  g1.B = c->bt.p; g1.ldb = bpp; g1.opB = OP_T;
  g1.C = c->T.p; g1.ldc = 2 * bl;
  TRY(gemm(c, g1));
  GemmArgs g2;
  g2.M = din; g2.N = bl; g2.K = 2 * dout; g2.b1 = 2; g2.b2 = cc;
  g2.A = c->Wy[site].p; g2.lda = 2 * dout; g2.sA1 = (long long)din * 2 * dout; g2.sA2 = 0; g2.opA = OP_N;
  g2.B = c->T.p; g2.ldb = bl; g2.sB1 = 0; g2.sB2 = (long long)dout * 2 * bl; g2.opB = OP_N;
  g2.C = out.p; g2.ldc = bl; g2.sC1 = (long long)cc * din * bl; g2.sC2 = (long long)din * bl;
  return gemm(c, g2);
}

double jacobi_tol(const dmrgc_ctx* c, int m) {
  const double eps = c->fp64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
  return 8.0 * eps * std::sqrt((double)std::max(m, 1));
}

// Orthogonalise the columns of jw (m x n column-major), truncate; returns k, f.
// squared: jw is a Gram matrix (its column norms are s^2); tie_rel > 0 applies
// the multiplet rule at the cut.
// W: the matrix (default jw); chi_cap: the most columns kept (default chi);
// norm2 (optional): the sum of all s^2.
dmrgc_status svd_columns(dmrgc_ctx* c, int m, int n, double rel_cut, bool squared, double tie_rel,
                         int& k, double& f, int* nnz, double* norm2, void* W, int chi_cap) {
  if (!W) W = c->jw.p;
  if (chi_cap < 0) chi_cap = c->chi;
  TRY(ensure(c, c->jctl, jacobi_ctl_bytes(n)));
  TRY(ensure(c, c->tres, trunc_bytes(n)));
  TRY(ensure(c, c->scal, 64 + 256 * sizeof(double)));
  double* fro2 = (double*)c->scal.p + 1;
  {
    Span sp(c, TC_SVD);
    int launches = 0;
    CK(sum_abs2(W, (long long)m * n, c->fp64, fro2, c->st));
    CK(jacobi_orthogonalize(W, m, n, c->fp64, jacobi_tol(c, m), c->max_jsweeps, fro2,
                            c->zero_rel, c->jctl.p, c->st, &launches));
    CK(truncate_columns(W, m, n, c->fp64, chi_cap, rel_cut, squared, tie_rel, fro2, c->zero_rel,
                        c->tres.p, c->st));
    c->stats.svd_launches += launches + 3;
    c->stats.kernel_launches += launches + 3;
  }
  JacobiStatus ctl{};
  TruncResult tr{};
  CK(cudaMemcpyAsync(&ctl, c->jctl.p, sizeof(ctl), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(&tr, c->tres.p, sizeof(tr), cudaMemcpyDeviceToHost, c->st));
  TRY(sync(c));
  if (ctl.err == DMRGC_ETIMEOUT) return fail(c, DMRGC_ETIMEOUT, "Jacobi SVD grid barrier timed out");
  if (ctl.err == DMRGC_ENOCONV)
    return fail(c, DMRGC_ENOCONV, "Jacobi SVD did not converge in " + std::to_string(c->max_jsweeps) + " sweeps");
  if (tr.status != 0 || !std::isfinite(tr.f) || !(tr.f > 0))
    return fail(c, DMRGC_ENUMERIC, "truncated SVD met a zero or non-finite spectrum");
  c->last_tr = tr;
  c->stats.jacobi_sweeps += ctl.sweeps;
  c->stats.svd_flops += (double)ctl.sweeps * 0.5 * n * (n - 1) * 16.0 * m + (double)ctl.rotations * 14.0 * m;
  k = tr.k;
  f = tr.f;
  if (nnz) *nnz = tr.nnz;
  if (norm2) *norm2 = tr.norm2;
  return DMRGC_OK;
}

// ---- truncated SVD through the Gram matrix's eigenproblem (complex64 modes)
//
// The kept singular vectors of G (rows x kdim, row-major; conj = true: G is
// conj(theta) read column-wise, i.e. the kept vectors are those of theta^+)
// are the leading eigenvectors of H = G G^+, formed by the contraction
// engine with TF32x3 split products (FP32 CUDA cores in the FP32 mode), then
// diagonalised by eig_truncate.  done = false when the kept eigenvalues are not
// all resolved above the Gram's rounding level (or the path does not apply):
// the caller then runs the Jacobi SVD.  out receives the k vectors in layout
// `mode` (see eig_truncate).
// lambda_{k-1} >= 1e-5 lambda_0 (s_{k-1} >= 3e-3 s_1): ten times the Gram
// path's absolute eigenvalue error (~1e-6 lambda_0 for a TF32x3 Gram and an
// FP32 reduction), so only directions whose weights differ by less than that
// can trade places at the cut
constexpr double kEigResolve = 1e-5;
constexpr int kEigMinN = 128;

bool eig_applies(const dmrgc_ctx* c, int rows) {
  return !c->fp64 && c->opt.svd_path == 0 && rows >= kEigMinN && rows <= 2048 && c->chi < rows;
}

// after a truncated SVD at `bond` (either path): would the eigensolver have
// resolved it?  Spectra change little between visits of a bond, so the next
// visit tries the eigensolver only if this one was resolvable, and otherwise
// goes straight to the Jacobi SVD instead of paying for a declined attempt.
void note_resolvable(dmrgc_ctx* c, int bond) {
  if (bond < 0 || bond >= (int)c->eig_ok.size()) return;
  c->eig_ok[bond] = (!c->last_tr.by_cut && c->last_tr.tail >= kEigResolve) ? 1 : 0;
}

dmrgc_status eig_try(dmrgc_ctx* c, int bond, const void* G, int rows, int kdim, bool conj_cols, double cut,
                     double tie, DevBuf& out, int mode, int& k, bool& done) {
  done = false;
  if (!eig_applies(c, rows)) return DMRGC_OK;
  if (bond >= 0 && bond < (int)c->eig_ok.size() && !c->eig_ok[bond]) {
    c->stats.eig_skipped++;
    return DMRGC_OK;
  }
  TRY(ensure(c, c->jw, (size_t)rows * rows * c->esz));
  GemmArgs g;   // H[r1][r2] = sum_x G[r1][x] conj(G[r2][x])
  g.M = rows; g.N = rows; g.K = kdim;
  if (!conj_cols) {
    g.A = G; g.lda = kdim; g.opA = OP_N;
    g.B = G; g.ldb = kdim; g.opB = OP_C;
  } else {        // G = theta^+ with theta [kdim][rows]: H = theta^+ theta
    g.A = G; g.lda = rows; g.opA = OP_C;
    g.B = G; g.ldb = rows; g.opB = OP_N;
  }
  g.C = c->jw.p; g.ldc = rows;
  g.upper_only = 1;   // Hermitian: the eigensolver mirrors the upper triangle
  const int gp = c->opt.precision == DMRGC_FP32 ? DMRGC_FP32 : DMRGC_TF32X3;
  TRY(gemm(c, g, gp));
  const int kk = std::min(c->chi + 1, rows);
  TRY(ensure(c, c->ework, eig_work_bytes(rows, kk)));
  TRY(ensure(c, c->tres, trunc_bytes(rows)));
  TRY(ensure(c, out, (size_t)rows * std::min(c->chi, rows) * c->esz));
  {
    Span sp(c, TC_SVD);
    int launches = 0;
    const cudaError_t ee = eig_truncate(c->jw.p, rows, c->chi, cut, tie, kEigResolve, c->ework.p, c->tres.p,
                                       out.p, mode, c->st, &launches);
    if (ee == cudaErrorInvalidConfiguration || ee == cudaErrorInvalidValue) {
      cudaGetLastError();   // a size or launch shape the eigensolver does not take: Jacobi SVD
      c->stats.eig_fallbacks++;
      return DMRGC_OK;
    }
    CK(ee);
    c->stats.svd_launches += launches;
    c->stats.kernel_launches += launches;
  }
  TruncResult tr{};
  CK(cudaMemcpyAsync(&tr, c->tres.p, sizeof(tr), cudaMemcpyDeviceToHost, c->st));
  TRY(sync(c));
  c->last_tr = tr;
  if (tr.status == DMRGC_ETIMEOUT) return fail(c, DMRGC_ETIMEOUT, "Gram eigensolver grid barrier timed out");
  if (tr.status == DMRGC_ENUMERIC) return fail(c, DMRGC_ENUMERIC, "Gram eigensolver met a zero or non-finite spectrum");
  if (tr.status != 0) {   // 1: not resolved, 2: a non-finite value: the Jacobi SVD decides
    c->stats.eig_fallbacks++;
    return DMRGC_OK;
  }
  k = tr.k;
  done = true;
  c->stats.eig_svds++;
  c->stats.svd_flops += 16.0 / 3.0 * (double)rows * rows * rows + 8.0 * (double)rows * rows * k;
  return DMRGC_OK;
}

// f = |A|^2 of the unnormalised block just formed, then A /= sqrt(f)
dmrgc_status normalise_block(dmrgc_ctx* c, void* A, long long elems, double& f) {
  TRY(ensure(c, c->scal, 64 + 256 * sizeof(double)));
  {
    Span sp(c, TC_OTHER);
    CK(norm2_scale(A, elems, c->fp64, (double*)c->scal.p, (double*)c->scal.p + 8, true, c->st));
    c->stats.kernel_launches += 2;
  }
  CK(cudaMemcpyAsync(&f, c->scal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  TRY(sync(c));
  if (!(f > 0) || !std::isfinite(f)) return fail(c, DMRGC_ENUMERIC, "update kept a zero or non-finite weight");
  return DMRGC_OK;
}

// theta[(a s1)][(s2 c)] = X_i Y_{i+1}^T
dmrgc_status form_theta(dmrgc_ctx* c, int i, int& mrow, int& ncol) {
  const int a = c->chiA[i], cc = c->chiA[i + 2];
  const int kdim = c->D[i + 1] * c->chiB[i + 1];
  mrow = 2 * a;
  ncol = 2 * cc;
  TRY(ensure(c, c->theta, (size_t)mrow * ncol * c->esz));
  GemmArgs g;
  g.M = mrow; g.N = ncol; g.K = kdim;
  g.A = c->XY[i].p; g.lda = kdim; g.opA = OP_N;
  g.B = c->XY[i + 1].p; g.ldb = kdim; g.opB = OP_T;
  g.C = c->theta.p; g.ldc = ncol;
  return gemm(c, g);
}

// ---- randomized truncated SVD (svd_mode 1, 2)
//
// Range finder of Halko, Martinsson and Tropp (SIAM Rev. 53, 2011): Y = G Omega
// with a Gaussian Omega of l = r + p columns, q power iterations G (G^+ Q) with
// re-orthonormalisation, B = Q^+ G, then the left singular vectors of B from the
// eigenvectors of B B^+ (one-sided Jacobi on the Hermitian l x l matrix), and
// U = Q W.  G = theta (left vectors, left-to-right update) or theta^+ (right
// vectors, right-to-left update).  Every orthonormalisation is the one-sided
// Jacobi with the numerical-zero level, so rank-deficient sketches lose their
// null directions instead of dividing by them.
//
// Acceptance (else the update falls back to the full Jacobi SVD), a
// certificate: theta^+ theta = B^+ B + (rest), both positive semidefinite, so
// by Ky Fan the best weight of k <= chi singular values of theta is at most
// that of B plus |theta|^2 - |B|^2.  With f the weight kept from B: if k = chi
// the optimum is at most f + |theta|^2 - |B|^2; if fewer were kept (the rest
// fell below the cut) at most |theta|^2.  Accept when that excess is at most
// tol * f: the result is then within tol of the optimal update.
//
// Sketch size: r + p with r the rank that held all but 1e-6 of the kept
// weight at the bond's last update (svd_mode 1), or the rank model's
// prediction of it (svd_mode 2).  The sketch is tried only when r + p is below
// half the smaller side of theta: each orthonormalisation is a Jacobi on r + p
// columns, so a larger sketch costs about as much as the full SVD.

// orthonormal basis of the columns of W (column-major rows x cols): every
// direction above the numerical-zero level, out row-major [rows][r]
// (mode 1: out column-major [rows][r])
dmrgc_status orth_columns(dmrgc_ctx* c, void* W, int rows, int cols, void* out, int& r, int mode = 0) {
  int k = 0, nnz = 0;
  double f = 0;
  TRY(svd_columns(c, rows, cols, 0.0, false, 0.0, k, f, &nnz, nullptr, W, cols));
  r = k;
  Span sp(c, TC_SVD);
  CK(gather_columns(W, rows, cols, k, c->tres.p, false, mode, out, c->fp64, c->st));
  c->stats.kernel_launches++;
  return DMRGC_OK;
}

dmrgc_status rsvd_try(dmrgc_ctx* c, int i, bool adj, int mrow, int ncol, int l, bool& accepted, int& k,
                      double& f) {
  accepted = false;
  const int mg = adj ? ncol : mrow, ng = adj ? mrow : ncol;
  const size_t es = c->esz;
  // op codes on theta (row-major [mrow][ncol]) giving G^T [ng][mg], conj(G) [mg][ng], G [mg][ng]
  const int opGT = adj ? OP_R : OP_T;
  const int opGc = adj ? OP_T : OP_R;
  const int opG = adj ? OP_C : OP_N;
  TRY(ensure(c, c->scal, 64 + 256 * sizeof(double)));
  double* fro_t = (double*)c->scal.p + 3;
  TRY(ensure(c, c->rs_om, (size_t)ng * l * es));
  TRY(ensure(c, c->rs_y, (size_t)l * std::max(mg, ng) * es));
  TRY(ensure(c, c->rs_q, (size_t)mg * l * es));
  {
    Span sp(c, TC_SVD);
    CK(sum_abs2(c->theta.p, (long long)mrow * ncol, c->fp64, fro_t, c->st));
    CK(fill_gaussian(c->rs_om.p, (long long)ng * l, c->fp64, c->opt.seed, c->rs_ctr, c->st));
    c->stats.kernel_launches += 2;
  }
  c->rs_ctr += 2ull * ng * l;
  c->stats.rsvd_attempts++;
  // Y^T = S^T G^T for a basis S [ng][cols]: [cols][mg] row-major = Y column-major
  auto sketch = [&](const void* S, int cols) -> dmrgc_status {
    GemmArgs g;
    g.M = cols; g.N = mg; g.K = ng;
    g.A = S; g.lda = cols; g.opA = OP_T;
    g.B = c->theta.p; g.ldb = ncol; g.opB = opGT;
    g.C = c->rs_y.p; g.ldc = mg;
    return gemm(c, g);
  };
  TRY(sketch(c->rs_om.p, l));
  int lq = 0;
  TRY(orth_columns(c, c->rs_y.p, mg, l, c->rs_q.p, lq));
  for (int it = 0; it < c->rs_pow; ++it) {
    GemmArgs g;   // Z^T = Q^T conj(G): [lq][ng] = (G^+ Q) column-major
    g.M = lq; g.N = ng; g.K = mg;
    g.A = c->rs_q.p; g.lda = lq; g.opA = OP_T;
    g.B = c->theta.p; g.ldb = ncol; g.opB = opGc;
    g.C = c->rs_y.p; g.ldc = ng;
    TRY(gemm(c, g));
    int lz = 0;
    TRY(orth_columns(c, c->rs_y.p, ng, lq, c->rs_om.p, lz));   // [ng][lz], in Omega's buffer
    TRY(sketch(c->rs_om.p, lz));
    TRY(orth_columns(c, c->rs_y.p, mg, lz, c->rs_q.p, lq));
  }
  TRY(ensure(c, c->rs_b, (size_t)lq * ng * es));
  {
    GemmArgs g;   // B = Q^+ G [lq][ng]
    g.M = lq; g.N = ng; g.K = mg;
    g.A = c->rs_q.p; g.lda = lq; g.opA = OP_C;
    g.B = c->theta.p; g.ldb = ncol; g.opB = opG;
    g.C = c->rs_b.p; g.ldc = ng;
    TRY(gemm(c, g));
  }
  TRY(ensure(c, c->rs_h, (size_t)lq * lq * es));
  {
    GemmArgs g;   // H = B B^+ [lq][lq]; Hermitian, so the buffer is conj(H) column-major
    g.M = lq; g.N = lq; g.K = ng;
    g.A = c->rs_b.p; g.lda = ng; g.opA = OP_N;
    g.B = c->rs_b.p; g.ldb = ng; g.opB = OP_C;
    g.C = c->rs_h.p; g.ldc = lq;
    TRY(gemm(c, g));
  }
  int kk = 0, nnz = 0;
  double ff = 0, trh = 0, fro_theta = 0;
  TRY(svd_columns(c, lq, lq, c->sweep_cut, true, 0.0, kk, ff, &nnz, &trh, c->rs_h.p, c->chi));
  CK(cudaMemcpy(&fro_theta, fro_t, sizeof(double), cudaMemcpyDeviceToHost));
  // weight the optimum could hold beyond ff: everything outside the sketch, and,
  // when fewer than chi values were kept, the sketch's own values below the cut
  const double tol = c->rs_tol;
  const double gap = (fro_theta - trh) + (kk < c->chi ? trh - ff : 0.0);
  if (!(gap <= tol * ff)) return DMRGC_OK;
  accepted = true;
  c->stats.rsvd_accepted++;
  TRY(ensure(c, c->rs_w, (size_t)lq * kk * es));
  {
    Span sp(c, TC_SVD);   // normalised eigenvectors of conj(H): conj(W) [lq][kk]
    CK(gather_columns(c->rs_h.p, lq, lq, kk, c->tres.p, true, 0, c->rs_w.p, c->fp64, c->st));
    c->stats.kernel_launches++;
  }
  GemmArgs g;
  if (!adj) {   // A_i = Q W [mrow][kk]
    TRY(ensure(c, c->A[i], (size_t)mrow * kk * es));
    g.M = mg; g.N = kk; g.K = lq;
    g.A = c->rs_q.p; g.lda = lq; g.opA = OP_N;
    g.B = c->rs_w.p; g.ldb = kk; g.opB = OP_R;
    g.C = c->A[i].p; g.ldc = kk;
  } else {      // A_{i+1} = (Q W)^+ [kk][ncol]
    TRY(ensure(c, c->A[i + 1], (size_t)kk * ncol * es));
    g.M = kk; g.N = mg; g.K = lq;
    g.A = c->rs_w.p; g.lda = kk; g.opA = OP_T;
    g.B = c->rs_q.p; g.ldb = lq; g.opB = OP_C;
    g.C = c->A[i + 1].p; g.ldc = mg;
  }
  TRY(gemm(c, g));
  k = kk;
  f = ff;
  return DMRGC_OK;
}

// Rank-model input at bond i: the summary of the spectrum at its last update
// (32 values on the device), then log2 of that kept rank, log2 of the MPO bond
// dimension there, log2 of the smaller side of theta, and 1 if the bond was
// already updated in this layer.
void model_extras(const dmrgc_ctx* c, int i, int nmin, float* e) {
  e[0] = (float)std::log2((double)std::max(c->kprev[i], 1));
  e[1] = (float)std::log2((double)std::max(c->D[i + 1], 1));
  e[2] = (float)std::log2((double)std::max(nmin, 1));
  e[3] = c->visit_layer[i] == c->layer_no ? 1.f : 0.f;
}

// Sketch size for the update at bond i, 0 = full Jacobi.
dmrgc_status sketch_size(dmrgc_ctx* c, int i, int mrow, int ncol, int& l) {
  l = 0;
  const int nmin = std::min(mrow, ncol);
  if (c->opt.svd_mode == 0 || nmin < 32) return DMRGC_OK;
  int r = 0;
  if (c->opt.svd_mode == 1) {
    if (c->kprev[i] <= 0) return DMRGC_OK;
    int lab = 0;   // the rank the last update here needed (its spectrum's label)
    CK(cudaMemcpyAsync(&lab, (const int*)c->lab.p + i, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    TRY(sync(c));
    r = lab;
  } else {
    if (!c->mlp_ready || c->kprev[i] <= 0) return DMRGC_OK;
    float e[4];
    model_extras(c, i, nmin, e);
    TRY(ensure(c, c->mlp_out, 64));
    {
      Span sp(c, TC_SVD);
      CK(mlp_infer_one(c->mlp_w.p, (const float*)c->feat.p + 32 * (size_t)i, e, (float*)c->mlp_out.p, c->st));
      c->stats.kernel_launches++;
    }
    float y = 0.f;
    CK(cudaMemcpyAsync(&y, c->mlp_out.p, sizeof(float), cudaMemcpyDeviceToHost, c->st));
    TRY(sync(c));
    if (!std::isfinite(y)) return DMRGC_OK;
    r = (int)std::ceil(std::exp2(std::min(std::max((double)y, 0.0), 20.0)));
  }
  const int want = r + c->rs_p;
  if (2 * want >= nmin) return DMRGC_OK;
  l = std::max(want, 1);
  return DMRGC_OK;
}

// Before an update at bond i: the host copy of the rank-model input the record
// logged by this update will carry.
dmrgc_status record_begin(dmrgc_ctx* c, int i, int nmin, std::vector<float>& x) {
  x.clear();
  if (!c->opt.log_rank_records || c->kprev[i] <= 0) return DMRGC_OK;
  x.resize(DMRGC_MLP_IN);
  CK(cudaMemcpyAsync(x.data(), (const float*)c->feat.p + 32 * (size_t)i, 32 * sizeof(float),
                     cudaMemcpyDeviceToHost, c->st));
  TRY(sync(c));
  model_extras(c, i, nmin, x.data() + 32);
  return DMRGC_OK;
}

// After the SVD of an update at bond i with k kept (tres holds its spectrum):
// the spectrum summary for the next visit and, for a full SVD, the record's label.
dmrgc_status record_end(dmrgc_ctx* c, int i, int k, bool full, const std::vector<float>& x) {
  if (c->opt.svd_mode == 2 || c->opt.log_rank_records) {
    TRY(ensure(c, c->feat, sizeof(float) * 32 * (size_t)c->N));
    Span sp(c, TC_SVD);
    CK(spectrum_summary(c->tres.p, k, (float*)c->feat.p + 32 * (size_t)i, c->st));
    c->stats.kernel_launches++;
  }
  if (c->opt.svd_mode != 0 || c->opt.log_rank_records) {
    // per bond: the rank holding all but 1e-6 of the kept weight
    TRY(ensure(c, c->lab, sizeof(int) * (size_t)c->N));
    CK(rank_label(c->tres.p, k, 1.0 - 1e-6, (int*)c->lab.p + i, c->st));
    c->stats.kernel_launches++;
  }
  if (full && !x.empty()) {
    int r = 0;
    CK(cudaMemcpyAsync(&r, (const int*)c->lab.p + i, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    TRY(sync(c));
    c->rec_x.insert(c->rec_x.end(), x.begin(), x.end());
    c->rec_y.push_back((float)std::log2((double)std::max(r, 1)));
  }
  c->kprev[i] = k;
  c->visit_layer[i] = c->layer_no;
  return DMRGC_OK;
}

dmrgc_status update_ltr(dmrgc_ctx* c, int i) {
  // X_i from the running left environment
  EnvRef L = c->L;
  if (i == 0) { L.p = c->one.p; L.a = 1; L.w = 1; L.b = 1; }
  TRY(make_x(c, L, i, c->XY[i]));
  c->xyk[i] = 'X';
  if (c->xyk[i + 1] != 'Y') return fail(c, DMRGC_ESTATE, "right cache missing");
  int mrow, ncol;
  TRY(form_theta(c, i, mrow, ncol));
  std::vector<float> rec;
  TRY(record_begin(c, i, std::min(mrow, ncol), rec));
  int k = 0, nnz = 0, l = 0;
  double f = 0;
  bool sketched = false;
  TRY(sketch_size(c, i, mrow, ncol, l));
  if (l > 0) TRY(rsvd_try(c, i, false, mrow, ncol, l, sketched, k, f));
  bool eig = false;
  if (sketched) {
    TRY(record_end(c, i, k, false, rec));
  } else {
    // U_k: leading eigenvectors of theta theta^+ where they are resolved, else Jacobi
    TRY(eig_try(c, i, c->theta.p, mrow, ncol, false, c->sweep_cut, 0.0, c->A[i], 0, k, eig));
    if (!eig) {
      TRY(ensure(c, c->jw, (size_t)mrow * ncol * c->esz));
      {
        Span sp(c, TC_OTHER);
        CK(copy_transpose(c->theta.p, mrow, ncol, false, c->jw.p, c->fp64, c->st));
        c->stats.kernel_launches++;
      }
      TRY(svd_columns(c, mrow, ncol, c->sweep_cut, false, 0.0, k, f, &nnz));
      TRY(ensure(c, c->A[i], (size_t)mrow * k * c->esz));
      Span sp(c, TC_SVD);
      CK(gather_columns(c->jw.p, mrow, ncol, k, c->tres.p, false, 0, c->A[i].p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    note_resolvable(c, i);
    TRY(record_end(c, i, k, true, rec));
  }
  TRY(ensure(c, c->A[i + 1], (size_t)k * ncol * c->esz));
  GemmArgs g;   // A_{i+1} = A_i^+ theta / |S_k|
  g.M = k; g.N = ncol; g.K = mrow;
  g.A = c->A[i].p; g.lda = k; g.opA = OP_C;
  g.B = c->theta.p; g.ldb = ncol; g.opB = OP_N;
  g.C = c->A[i + 1].p; g.ldc = ncol;
  // complex64 modes: f = |U_k^+ theta|^2 of the vectors as stored (the kept weight
  // of the basis actually used, exact up to one FP64 sum), then normalise; FP64
  // mode: f = sum of the kept s^2 from the SVD
  const bool renorm = eig || !c->fp64;
  g.alpha_re = renorm ? 1.0 : 1.0 / std::sqrt(f);
  TRY(gemm(c, g));
  if (renorm) TRY(normalise_block(c, c->A[i + 1].p, (long long)k * ncol, f));
  c->chiA[i + 1] = k;
  // L_i = A_i^+ X_i
  const int kdim = c->D[i + 1] * c->chiB[i + 1];
  TRY(ensure(c, c->envL, (size_t)k * kdim * c->esz));
  GemmArgs h;
  h.M = k; h.N = kdim; h.K = mrow;
  h.A = c->A[i].p; h.lda = k; h.opA = OP_C;
  h.B = c->XY[i].p; h.ldb = kdim; h.opB = OP_N;
  h.C = c->envL.p; h.ldc = kdim;
  TRY(gemm(c, h));
  c->L.p = c->envL.p; c->L.a = k; c->L.w = c->D[i + 1]; c->L.b = c->chiB[i + 1];
  c->f_cur = f;
  c->hist.push_back(f);
  c->centre = i + 1;
  c->stats.updates++;
  return DMRGC_OK;
}

dmrgc_status update_rtl(dmrgc_ctx* c, int i) {
  EnvRef R = c->R;
  if (i + 1 == c->N - 1) { R.p = c->one.p; R.a = 1; R.w = 1; R.b = 1; }
  TRY(make_y(c, R, i + 1, c->XY[i + 1]));
  c->xyk[i + 1] = 'Y';
  if (c->xyk[i] != 'X') return fail(c, DMRGC_ESTATE, "left cache missing");
  int mrow, ncol;
  TRY(form_theta(c, i, mrow, ncol));
  std::vector<float> rec;
  TRY(record_begin(c, i, std::min(mrow, ncol), rec));
  int k = 0, nnz = 0, l = 0;
  double f = 0;
  bool sketched = false;
  TRY(sketch_size(c, i, mrow, ncol, l));
  if (l > 0) TRY(rsvd_try(c, i, true, mrow, ncol, l, sketched, k, f));
  bool eig = false;
  if (sketched) {
    TRY(record_end(c, i, k, false, rec));
  } else {
    // V_k^+: leading eigenvectors of theta^+ theta (conjugated rows) where resolved, else Jacobi
    TRY(eig_try(c, i, c->theta.p, ncol, mrow, true, c->sweep_cut, 0.0, c->A[i + 1], 2, k, eig));
    if (!eig) {
      TRY(ensure(c, c->jw, (size_t)mrow * ncol * c->esz));
      {
        Span sp(c, TC_OTHER);
        CK(copy_conj(c->theta.p, (long long)mrow * ncol, c->jw.p, c->fp64, c->st));
        c->stats.kernel_launches++;
      }
      // columns of theta^+ (column-major == conj(theta) row-major): ncol rows, mrow columns
      TRY(svd_columns(c, ncol, mrow, c->sweep_cut, false, 0.0, k, f, &nnz));
      TRY(ensure(c, c->A[i + 1], (size_t)k * ncol * c->esz));
      Span sp(c, TC_SVD);
      CK(gather_columns(c->jw.p, ncol, mrow, k, c->tres.p, false, 2, c->A[i + 1].p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    note_resolvable(c, i);
    TRY(record_end(c, i, k, true, rec));
  }
  TRY(ensure(c, c->A[i], (size_t)mrow * k * c->esz));
  GemmArgs g;   // A_i = theta A_{i+1}^+ / |S_k|
  g.M = mrow; g.N = k; g.K = ncol;
  g.A = c->theta.p; g.lda = ncol; g.opA = OP_N;
  g.B = c->A[i + 1].p; g.ldb = ncol; g.opB = OP_C;
  g.C = c->A[i].p; g.ldc = k;
  const bool renorm = eig || !c->fp64;   // as in update_ltr
  g.alpha_re = renorm ? 1.0 : 1.0 / std::sqrt(f);
  TRY(gemm(c, g));
  if (renorm) TRY(normalise_block(c, c->A[i].p, (long long)mrow * k, f));
  c->chiA[i + 1] = k;
  const int kdim = c->D[i + 1] * c->chiB[i + 1];
  TRY(ensure(c, c->envR, (size_t)k * kdim * c->esz));
  GemmArgs h;   // R_{i+1} = conj(A_{i+1}) Y_{i+1}
  h.M = k; h.N = kdim; h.K = ncol;
  h.A = c->A[i + 1].p; h.lda = ncol; h.opA = OP_R;
  h.B = c->XY[i + 1].p; h.ldb = kdim; h.opB = OP_N;
  h.C = c->envR.p; h.ldc = kdim;
  TRY(gemm(c, h));
  c->R.p = c->envR.p; c->R.a = k; c->R.w = c->D[i + 1]; c->R.b = c->chiB[i + 1];
  c->f_cur = f;
  c->hist.push_back(f);
  c->centre = i;
  c->stats.updates++;
  return DMRGC_OK;
}

// Gram matrix (column-major) of the rows of M (r x K row-major): G = M M^+
dmrgc_status gram_colmajor(dmrgc_ctx* c, const void* M, int r, int kdim) {
  TRY(ensure(c, c->jw, (size_t)r * r * c->esz));
  GemmArgs g;   // buffer[r1][r2] = sum_k conj(M[r1][k]) M[r2][k] = G[r2][r1]
  g.M = r; g.N = r; g.K = kdim;
  g.A = M; g.lda = kdim; g.opA = OP_R;
  g.B = M; g.ldb = kdim; g.opB = OP_T;
  g.C = c->jw.p; g.ldc = r;
  return gemm(c, g);
}

dmrgc_status set_identity_site(dmrgc_ctx* c, DevBuf& dst, int r) {
  TRY(ensure(c, dst, (size_t)r * r * c->esz));
  Span sp(c, TC_OTHER);
  CK(set_identity(dst.p, r, c->fp64, c->st));
  c->stats.kernel_launches++;
  return DMRGC_OK;
}

// Zip-up initial guess from both ends towards the centre site m.
dmrgc_status zip_guess(dmrgc_ctx* c) {
  const int N = c->N, m = c->m;
  c->chiA.assign(N + 1, 1);
  // left part
  EnvRef L;
  L.p = c->one.p; L.a = 1; L.w = 1; L.b = 1;
  for (int i = 0; i < m; ++i) {
    TRY(make_x(c, L, i, c->XY[i]));
    c->xyk[i] = 'X';
    const int r = 2 * c->chiA[i];
    const int kdim = c->D[i + 1] * c->chiB[i + 1];
    if (r <= c->chi) {
      TRY(set_identity_site(c, c->A[i], r));
      c->chiA[i + 1] = r;
      L.p = c->XY[i].p; L.a = r; L.w = c->D[i + 1]; L.b = c->chiB[i + 1];
      continue;
    }
    int k;
    double f;
    bool eig = false;
    TRY(eig_try(c, i, c->XY[i].p, r, kdim, false, c->zip_cut, c->tie_rel, c->A[i], 0, k, eig));
    if (!eig) {
      TRY(gram_colmajor(c, c->XY[i].p, r, kdim));
      TRY(svd_columns(c, r, r, c->zip_cut, true, c->tie_rel, k, f));
      TRY(ensure(c, c->A[i], (size_t)r * k * c->esz));
      Span sp(c, TC_SVD);
      CK(gather_columns(c->jw.p, r, r, k, c->tres.p, true, 0, c->A[i].p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    c->chiA[i + 1] = k;
    TRY(ensure(c, c->envL, (size_t)k * kdim * c->esz));
    GemmArgs h;
    h.M = k; h.N = kdim; h.K = r;
    h.A = c->A[i].p; h.lda = k; h.opA = OP_C;
    h.B = c->XY[i].p; h.ldb = kdim; h.opB = OP_N;
    h.C = c->envL.p; h.ldc = kdim;
    TRY(gemm(c, h));
    L.p = c->envL.p; L.a = k; L.w = c->D[i + 1]; L.b = c->chiB[i + 1];
  }
  // right part
  EnvRef R;
  R.p = c->one.p; R.a = 1; R.w = 1; R.b = 1;
  for (int i = N - 1; i > m; --i) {
    TRY(make_y(c, R, i, c->XY[i]));
    c->xyk[i] = 'Y';
    const int r = 2 * c->chiA[i + 1];
    const int kdim = c->D[i] * c->chiB[i];
    if (r <= c->chi) {
      TRY(set_identity_site(c, c->A[i], r));
      c->chiA[i] = r;
      R.p = c->XY[i].p; R.a = r; R.w = c->D[i]; R.b = c->chiB[i];
      continue;
    }
    int k;
    double f;
    bool eig = false;
    TRY(eig_try(c, i - 1, c->XY[i].p, r, kdim, false, c->zip_cut, c->tie_rel, c->A[i], 1, k, eig));
    if (!eig) {
      TRY(gram_colmajor(c, c->XY[i].p, r, kdim));
      TRY(svd_columns(c, r, r, c->zip_cut, true, c->tie_rel, k, f));
      TRY(ensure(c, c->A[i], (size_t)k * r * c->esz));
      Span sp(c, TC_SVD);
      CK(gather_columns(c->jw.p, r, r, k, c->tres.p, true, 1, c->A[i].p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    c->chiA[i] = k;
    TRY(ensure(c, c->envR, (size_t)k * kdim * c->esz));
    GemmArgs h;
    h.M = k; h.N = kdim; h.K = r;
    h.A = c->A[i].p; h.lda = r; h.opA = OP_R;
    h.B = c->XY[i].p; h.ldb = kdim; h.opB = OP_N;
    h.C = c->envR.p; h.ldc = kdim;
    TRY(gemm(c, h));
    R.p = c->envR.p; R.a = k; R.w = c->D[i]; R.b = c->chiB[i];
  }
  // centre: C = X_m R_{m+1}^T, normalised
  TRY(make_x(c, L, m, c->XY[m]));
  c->xyk[m] = 'X';
  const int mrow = 2 * c->chiA[m], ncol = c->chiA[m + 1];
  const int kdim = c->D[m + 1] * c->chiB[m + 1];
  TRY(ensure(c, c->A[m], (size_t)mrow * ncol * c->esz));
  GemmArgs g;
  g.M = mrow; g.N = ncol; g.K = kdim;
  g.A = c->XY[m].p; g.lda = kdim; g.opA = OP_N;
  g.B = R.p; g.ldb = kdim; g.opB = OP_T;
  g.C = c->A[m].p; g.ldc = ncol;
  TRY(gemm(c, g));
  TRY(ensure(c, c->scal, 64 + 256 * sizeof(double)));
  {
    Span sp(c, TC_OTHER);
    CK(sum_abs2(c->A[m].p, (long long)mrow * ncol, c->fp64, (double*)c->scal.p, c->st));
    CK(scale_inplace(c->A[m].p, (long long)mrow * ncol, (const double*)c->scal.p, c->fp64, c->st));
    c->stats.kernel_launches += 2;
  }
  double nrm2 = 0;
  CK(cudaMemcpyAsync(&nrm2, c->scal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  TRY(sync(c));
  if (!(nrm2 > 0) || !std::isfinite(nrm2))
    return fail(c, DMRGC_ENUMERIC, "zip-up guess has zero overlap with the target state");
  c->f_cur = nrm2;
  c->L = L;
  c->R = R;
  c->centre = m;
  return DMRGC_OK;
}

// ---- layer MPO plan

// Lossless compression of the layer MPO: its bonds are reduced to the operator
// Schmidt ranks of the layer across each cut (the built bond is the product of
// the straddling gates' Schmidt ranks, which over-counts where gates share
// qubits).  Site tensors are taken as matrices, factored by the one-sided
// Jacobi SVD and cut at the sweep's relative cutoff (1e-12 in FP64, 2e-5 in
// complex64) and the numerical-zero level; the singular values themselves
// stay in the neighbouring tensor, so the product of the tensors does not
// change beyond that cut.
//  left to right:  W_i = Q R with orthonormal columns Q,  W_{i+1} <- R W_{i+1};
//  right to left:  W_i = L Q' with orthonormal rows Q',  W_{i-1} <- W_{i-1} L.
// After the first pass the left part is an isometry, so the second pass sees
// the true operator Schmidt values.  A cut at full rank is left as it is.
dmrgc_status compress_mpo(dmrgc_ctx* c) {
  const int N = c->N;
  const size_t es = c->esz;
  if ((int)c->Wc.size() < N) c->Wc.resize(N);
  for (int i = 0; i < N; ++i) {   // Wy[s][w_in][w_out][t] -> Wc[w_in][s][t][w_out]
    const int dims[4] = {2, c->D[i], c->D[i + 1], 2}, perm[4] = {1, 0, 3, 2};
    TRY(ensure(c, c->Wc[i], (size_t)4 * c->D[i] * c->D[i + 1] * es));
    Span sp(c, TC_MPO);
    CK(permute4(c->Wy[i].p, dims, perm, c->Wc[i].p, c->fp64, c->st));
    c->stats.kernel_launches++;
  }
  auto replace = [&](DevBuf& dst, const DevBuf& src, size_t bytes) -> dmrgc_status {
    TRY(ensure(c, dst, bytes));
    CK(cudaMemcpyAsync(dst.p, src.p, bytes, cudaMemcpyDeviceToDevice, c->st));
    return DMRGC_OK;
  };
  for (int i = 0; i + 1 < N; ++i) {
    const int dl = c->D[i], dr = c->D[i + 1], dr2 = c->D[i + 2], rows = 4 * dl;
    if (dr == 1) continue;
    TRY(ensure(c, c->jw, (size_t)rows * dr * es));
    {
      Span sp(c, TC_OTHER);
      CK(copy_transpose(c->Wc[i].p, rows, dr, false, c->jw.p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    int k = 0, nnz = 0;
    double f = 0;
    TRY(svd_columns(c, rows, dr, c->sweep_cut, false, 0.0, k, f, &nnz, nullptr, c->jw.p, dr));
    if (k >= dr) continue;
    TRY(ensure(c, c->T, (size_t)rows * k * es));
    {
      Span sp(c, TC_SVD);
      CK(gather_columns(c->jw.p, rows, dr, k, c->tres.p, false, 0, c->T.p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    TRY(ensure(c, c->envL, (size_t)k * dr * es));
    GemmArgs g;   // R = Q^+ W_i  [k][dr]
    g.M = k; g.N = dr; g.K = rows;
    g.A = c->T.p; g.lda = k; g.opA = OP_C;
    g.B = c->Wc[i].p; g.ldb = dr; g.opB = OP_N;
    g.C = c->envL.p; g.ldc = dr;
    TRY(gemm(c, g));
    TRY(ensure(c, c->envR, (size_t)k * 4 * dr2 * es));
    GemmArgs h;   // W_{i+1} <- R W_{i+1}  [k][4 dr2]
    h.M = k; h.N = 4 * dr2; h.K = dr;
    h.A = c->envL.p; h.lda = dr; h.opA = OP_N;
    h.B = c->Wc[i + 1].p; h.ldb = 4 * dr2; h.opB = OP_N;
    h.C = c->envR.p; h.ldc = 4 * dr2;
    TRY(gemm(c, h));
    TRY(replace(c->Wc[i + 1], c->envR, (size_t)k * 4 * dr2 * es));
    TRY(replace(c->Wc[i], c->T, (size_t)rows * k * es));
    c->D[i + 1] = k;
  }
  for (int i = N - 1; i >= 1; --i) {
    const int dl = c->D[i], dr = c->D[i + 1], dl2 = c->D[i - 1], cols = 4 * dr;
    if (dl == 1) continue;
    TRY(ensure(c, c->jw, (size_t)dl * cols * es));
    {
      Span sp(c, TC_OTHER);   // columns of W_i^+ (column-major == conj(W_i) row-major)
      CK(copy_conj(c->Wc[i].p, (long long)dl * cols, c->jw.p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    int k = 0, nnz = 0;
    double f = 0;
    TRY(svd_columns(c, cols, dl, c->sweep_cut, false, 0.0, k, f, &nnz, nullptr, c->jw.p, dl));
    if (k >= dl) continue;
    TRY(ensure(c, c->T, (size_t)k * cols * es));
    {
      Span sp(c, TC_SVD);   // Q' [k][cols], orthonormal rows spanning the row space of W_i
      CK(gather_columns(c->jw.p, cols, dl, k, c->tres.p, false, 2, c->T.p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    TRY(ensure(c, c->envL, (size_t)dl * k * es));
    GemmArgs g;   // L = W_i Q'^+  [dl][k]
    g.M = dl; g.N = k; g.K = cols;
    g.A = c->Wc[i].p; g.lda = cols; g.opA = OP_N;
    g.B = c->T.p; g.ldb = cols; g.opB = OP_C;
    g.C = c->envL.p; g.ldc = k;
    TRY(gemm(c, g));
    TRY(ensure(c, c->envR, (size_t)4 * dl2 * k * es));
    GemmArgs h;   // W_{i-1} <- W_{i-1} L  [4 dl2][k]
    h.M = 4 * dl2; h.N = k; h.K = dl;
    h.A = c->Wc[i - 1].p; h.lda = dl; h.opA = OP_N;
    h.B = c->envL.p; h.ldb = k; h.opB = OP_N;
    h.C = c->envR.p; h.ldc = k;
    TRY(gemm(c, h));
    TRY(replace(c->Wc[i - 1], c->envR, (size_t)4 * dl2 * k * es));
    TRY(replace(c->Wc[i], c->T, (size_t)k * cols * es));
    c->D[i] = k;
  }
  for (int i = 0; i < N; ++i) {   // Wc -> Wx[s][w_out][w_in][t], Wy[s][w_in][w_out][t]
    const int dims[4] = {c->D[i], 2, 2, c->D[i + 1]};
    const int px[4] = {1, 3, 0, 2}, py[4] = {1, 0, 3, 2};
    const size_t bytes = (size_t)4 * c->D[i] * c->D[i + 1] * es;
    TRY(ensure(c, c->Wx[i], bytes));
    TRY(ensure(c, c->Wy[i], bytes));
    Span sp(c, TC_MPO);
    CK(permute4(c->Wc[i].p, dims, px, c->Wx[i].p, c->fp64, c->st));
    CK(permute4(c->Wc[i].p, dims, py, c->Wy[i].p, c->fp64, c->st));
    c->stats.kernel_launches += 2;
  }
  return DMRGC_OK;
}

dmrgc_status build_mpo(dmrgc_ctx* c, const dmrgc_gate* gates, int n_gates) {
  const int N = c->N;
  std::vector<GateDev> gd(n_gates);
  for (int g = 0; g < n_gates; ++g) {
    const dmrgc_gate& x = gates[g];
    if (x.q0 < 0 || x.q0 >= N || x.q1 >= N || x.q1 < -1 || x.q1 == x.q0)
      return fail(c, DMRGC_EINVAL, "gate " + std::to_string(g) + " has invalid qubits");
    for (int j = 0; j < 32; ++j)
      if (!std::isfinite(x.mat[j])) return fail(c, DMRGC_EINVAL, "gate " + std::to_string(g) + " is not finite");
    GateDev d{};
    const int s0 = c->site_of[x.q0];
    if (x.q1 < 0) { d.p = s0; d.q = -1; d.swap = 0; }
    else {
      const int s1 = c->site_of[x.q1];
      d.p = std::min(s0, s1); d.q = std::max(s0, s1); d.swap = s0 > s1 ? 1 : 0;
    }
    std::memcpy(d.mat, x.mat, sizeof(d.mat));
    gd[g] = d;
  }
  const int ng = std::max(n_gates, 1);
  TRY(ensure(c, c->gates_d, sizeof(GateDev) * ng));
  TRY(ensure(c, c->rank_d, sizeof(int) * ng));
  TRY(ensure(c, c->fa_d, sizeof(double2) * 16 * ng));
  TRY(ensure(c, c->fb_d, sizeof(double2) * 16 * ng));
  std::vector<int> rank(ng, 0);
  if (n_gates > 0) {
    CK(cudaMemcpyAsync(c->gates_d.p, gd.data(), sizeof(GateDev) * n_gates, cudaMemcpyHostToDevice, c->st));
    {
      Span sp(c, TC_MPO);
      CK(gate_split((const GateDev*)c->gates_d.p, n_gates, (int*)c->rank_d.p, (double2*)c->fa_d.p,
                    (double2*)c->fb_d.p, c->st));
      c->stats.kernel_launches++;
    }
    CK(cudaMemcpyAsync(rank.data(), c->rank_d.p, sizeof(int) * n_gates, cudaMemcpyDeviceToHost, c->st));
    TRY(sync(c));
  }
  // legs crossing each cut (between site i-1 and i), in gate order
  std::vector<std::vector<int>> legs(N + 1);
  c->D.assign(N + 1, 1);
  for (int cut = 1; cut < N; ++cut) {
    double d = 1;
    for (int g = 0; g < n_gates; ++g)
      if (gd[g].q >= 0 && gd[g].p < cut && cut <= gd[g].q && rank[g] > 0) {
        legs[cut].push_back(g);
        d *= rank[g];
      }
    if (d > 4096 || legs[cut].size() > 24)
      return fail(c, DMRGC_EINVAL, "layer MPO bond at cut " + std::to_string(cut) + " exceeds 4096");
    c->D[cut] = (int)d;
  }
  // plan table
  std::vector<int> tab;
  std::vector<SitePlan> plans(N);
  for (int i = 0; i < N; ++i) {
    const std::vector<int>& in = legs[i];
    const std::vector<int>& out = legs[i + 1];
    SitePlan sp{};
    sp.d_in = c->D[i];
    sp.d_out = c->D[i + 1];
    sp.n_in = (int)in.size();
    sp.n_out = (int)out.size();
    sp.off = (long long)tab.size();
    for (int g : in) {
      int po = -1;
      for (size_t j = 0; j < out.size(); ++j)
        if (out[j] == g) po = (int)j;
      tab.push_back(g); tab.push_back(rank[g]); tab.push_back(po);
    }
    for (int g : out) { tab.push_back(g); tab.push_back(rank[g]); }
    int nops = 0;
    for (int g = 0; g < n_gates; ++g) {
      if (gd[g].q < 0) {
        if (gd[g].p == i) { tab.push_back(0); tab.push_back(g); tab.push_back(0); ++nops; }
      } else if (gd[g].p == i) {
        int j = (int)(std::find(out.begin(), out.end(), g) - out.begin());
        tab.push_back(1); tab.push_back(g); tab.push_back(j); ++nops;
      } else if (gd[g].q == i) {
        int j = (int)(std::find(in.begin(), in.end(), g) - in.begin());
        tab.push_back(2); tab.push_back(g); tab.push_back(j); ++nops;
      }
    }
    sp.n_ops = nops;
    plans[i] = sp;
  }
  TRY(ensure(c, c->plan_d, sizeof(int) * std::max<size_t>(tab.size(), 1)));
  if (!tab.empty())
    CK(cudaMemcpyAsync(c->plan_d.p, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, c->st));
  for (int i = 0; i < N; ++i) {
    const size_t bytes = (size_t)plans[i].d_in * 4 * plans[i].d_out * c->esz;
    TRY(ensure(c, c->Wx[i], bytes));
    TRY(ensure(c, c->Wy[i], bytes));
    Span sp(c, TC_MPO);
    CK(build_site_mpo((const int*)c->plan_d.p, plans[i], (const GateDev*)c->gates_d.p,
                      (const double2*)c->fa_d.p, (const double2*)c->fb_d.p, c->Wx[i].p, c->Wy[i].p,
                      c->fp64, c->st));
    c->stats.kernel_launches++;
  }
  if (c->opt.mpo_compress) TRY(compress_mpo(c));
  return DMRGC_OK;
}

// the next `total` updates of the bouncing schedule (Sec. IV.B), then a sync
dmrgc_status run_updates(dmrgc_ctx* c, long long total) {
  for (long long u = 0; u < total; ++u) {
    if (c->N < 2) break;
    if (c->bond < 0) { c->bond = 0; c->dir = +1; }
    const int b = c->bond;
    if (c->dir < 0) {
      TRY(update_rtl(c, b));
      if (b == 0) c->dir = +1; else c->bond = b - 1;
    } else {
      TRY(update_ltr(c, b));
      if (b == c->N - 2) c->dir = -1; else c->bond = b + 1;
    }
  }
  return sync(c);
}

}  // namespace dmrgc_host

dmrgc_ctx::~dmrgc_ctx() {
  auto fr = [](DevBuf& b) { if (b.p) cudaFree(b.p); b.p = nullptr; };
  for (auto* v : {&A, &B, &Wx, &Wy, &XY, &E, &Wc, &GL, &GR})
    for (auto& b : *v) fr(b);
  for (DevBuf* b : {&envL, &envR, &T, &theta, &jw, &bt, &one, &jctl, &tres, &scal, &gates_d, &rank_d,
                    &fa_d, &fb_d, &plan_d, &ptrs_d, &bonds_d, &order_d, &bits_d, &out_d, &stage_d, &tcerr,
                    &ovl[0], &ovl[1], &ework, &rv[0], &rv[1], &rv[2], &gx[0], &gx[1], &gf})
    fr(*b);
  tcw.release();
  for (auto& p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : pool) cudaEventDestroy(e);
}

extern "C" {

dmrgc_status dmrgc_default_options(dmrgc_options* opt) {
  if (!opt) return DMRGC_EINVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = DMRGC_FP64;
  opt->svd_mode = 0;
  opt->rsvd_oversample = 8;
  opt->rsvd_power_iters = 1;
  opt->rsvd_tolerance = 0.0;
  opt->log_rank_records = 0;
  opt->max_jacobi_sweeps = 40;
  return DMRGC_OK;
}

}  // extern "C"

namespace {

bool valid_shape(int n_qubits, const dmrgc_grid* grid, int chi) {
  return grid && n_qubits >= 1 && n_qubits <= 4096 && grid->rows >= 1 && grid->cols >= 1 &&
         grid->rows * grid->cols == n_qubits && grid->order >= 0 && grid->order <= 2 && chi >= 1 && chi <= 4096;
}

// (Re)initialise a context for a new circuit in |0...0>.  Device buffers the
// context already owns are kept (they only grow), so a context can be reused
// for a sequence of circuits without new allocations once it has seen the
// largest one.
dmrgc_status ctx_setup(dmrgc_ctx* c, int n_qubits, const dmrgc_grid* grid, int chi, const dmrgc_options& opt) {
  c->opt = opt;
  if (c->opt.precision < 0 || c->opt.precision > 3 || c->opt.svd_mode < 0 || c->opt.svd_mode > 2 ||
      c->opt.rsvd_power_iters > 8)
    return fail(c, DMRGC_EINVAL, "bad options");
  c->N = n_qubits; c->chi = chi; c->rows = grid->rows; c->cols = grid->cols; c->m = n_qubits / 2;
  c->st = reinterpret_cast<cudaStream_t>(c->opt.cuda_stream);
  const bool fp64 = c->opt.precision == DMRGC_FP64;
  // buffers are sized in bytes, so a change of element size needs no release
  c->fp64 = fp64;
  c->esz = c->fp64 ? 16 : 8;
  // numerically-zero level of a Jacobi column, relative to |theta|_F, and the
  // cutoffs above it: FP64 1e-13 / sweep 1e-12 / zip 1e-5; complex64 1e-5 / 2e-5 / 4e-3
  // (a Gram column norm is s^2, so the zip cutoff on s is the square root).
  c->zero_rel = c->fp64 ? 1e-13 : 1e-5;
  c->tie_rel = c->fp64 ? 1e-10 : 1e-5;
  c->sweep_cut = c->opt.sweep_rel_cutoff > 0 ? c->opt.sweep_rel_cutoff : (c->fp64 ? 1e-12 : 2e-5);
  c->zip_cut = c->opt.zip_rel_cutoff > 0 ? c->opt.zip_rel_cutoff : (c->fp64 ? 1e-5 : 4e-3);
  c->max_jsweeps = c->opt.max_jacobi_sweeps > 0 ? c->opt.max_jacobi_sweeps : 40;
  c->order.clear();
  if (grid->order == 0) {          // snake along the columns
    for (int col = 0; col < c->cols; ++col)
      for (int k = 0; k < c->rows; ++k) {
        const int r = (col % 2 == 0) ? k : c->rows - 1 - k;
        c->order.push_back(r * c->cols + col);
      }
  } else if (grid->order == 1) {   // snake along the rows
    for (int r = 0; r < c->rows; ++r)
      for (int k = 0; k < c->cols; ++k) {
        const int col = (r % 2 == 0) ? k : c->cols - 1 - k;
        c->order.push_back(r * c->cols + col);
      }
  } else {                         // anti-diagonals r + col = d, alternating direction
    for (int d = 0; d < c->rows + c->cols - 1; ++d) {
      const int r0 = std::max(0, d - c->cols + 1), r1 = std::min(c->rows - 1, d);
      for (int k = 0; k <= r1 - r0; ++k) {
        const int r = (d % 2 == 0) ? r0 + k : r1 - k;
        c->order.push_back(r * c->cols + (d - r));
      }
    }
  }
  c->site_of.assign(n_qubits, 0);
  for (int i = 0; i < n_qubits; ++i) c->site_of[c->order[i]] = i;
  for (auto* v : {&c->A, &c->B, &c->Wx, &c->Wy, &c->XY, &c->E, &c->Wc})
    if ((int)v->size() < n_qubits) v->resize(n_qubits);
  c->xyk.assign(n_qubits, 0);
  c->chiA.assign(n_qubits + 1, 1); c->chiB.assign(n_qubits + 1, 1); c->D.assign(n_qubits + 1, 1);
  c->L = EnvRef(); c->R = EnvRef();
  c->layer_no = 0;
  c->visit_layer.assign(n_qubits, -1);
  c->kprev.assign(n_qubits, 0);
  c->eig_ok.assign(n_qubits, 1);
  c->rs_ctr = 0;
  c->rs_p = c->opt.rsvd_oversample > 0 ? c->opt.rsvd_oversample : 8;
  c->rs_pow = c->opt.rsvd_power_iters >= 0 ? c->opt.rsvd_power_iters : 1;
  c->rs_tol = c->opt.rsvd_tolerance > 0 ? c->opt.rsvd_tolerance : (c->fp64 ? 1e-6 : 2e-5);
  c->rec_x.clear(); c->rec_y.clear();
  c->ng = 0;
  c->gsize.assign(n_qubits, 1);
  c->gstart.resize(n_qubits);
  for (int i = 0; i < n_qubits; ++i) c->gstart[i] = i;
  c->gsweep = 0;
  c->phase = 0; c->bond = 0; c->dir = -1; c->centre = 0;
  c->log_ft = 0.0; c->f_cur = 1.0;
  c->hist.clear();
  c->err.clear();
  TRY(ensure(c, c->one, 64));
  CK(set_scalar_one(c->one.p, c->fp64, c->st));
  for (int i = 0; i < n_qubits; ++i) {
    TRY(ensure(c, c->B[i], 2 * c->esz));
    CK(cudaMemsetAsync(c->B[i].p, 0, 2 * c->esz, c->st));
    CK(set_scalar_one(c->B[i].p, c->fp64, c->st));
  }
  if (c->tcerr.p) CK(cudaMemsetAsync(c->tcerr.p, 0, 64, c->st));
  return sync(c);
}

}  // namespace

extern "C" {

dmrgc_status dmrgc_create(int n_qubits, const dmrgc_grid* grid, int chi, const dmrgc_options* opt,
                          dmrgc_ctx** out) {
  if (!out || !grid) return DMRGC_EINVAL;
  *out = nullptr;
  if (!valid_shape(n_qubits, grid, chi)) return DMRGC_EINVAL;
  dmrgc_ctx* c = new (std::nothrow) dmrgc_ctx();
  if (!c) return DMRGC_ENOMEM;
  dmrgc_options o;
  if (opt) o = *opt; else dmrgc_default_options(&o);
  c->esz = 0;
  dmrgc_status s = ctx_setup(c, n_qubits, grid, chi, o);
  if (s != DMRGC_OK) { delete c; return s; }
  *out = c;
  return DMRGC_OK;
}

dmrgc_status dmrgc_create_grouped(int n_qubits, const dmrgc_grid* grid, const int* group_sizes, int n_groups,
                                  int chi, const dmrgc_options* opt, dmrgc_ctx** out) {
  if (!out || !grid || !group_sizes || n_groups < 1 || n_groups > n_qubits) return DMRGC_EINVAL;
  *out = nullptr;
  if (!valid_shape(n_qubits, grid, chi)) return DMRGC_EINVAL;
  int total = 0;
  for (int g = 0; g < n_groups; ++g) {
    if (group_sizes[g] < 1 || group_sizes[g] > 20) return DMRGC_EINVAL;
    total += group_sizes[g];
  }
  if (total != n_qubits) return DMRGC_EINVAL;
  dmrgc_ctx* c = nullptr;
  dmrgc_status s = dmrgc_create(n_qubits, grid, chi, opt, &c);
  if (s != DMRGC_OK) return s;
  c->ng = n_groups;
  c->gsize.assign(group_sizes, group_sizes + n_groups);
  c->gstart.assign(n_groups, 0);
  for (int g = 1; g < n_groups; ++g) c->gstart[g] = c->gstart[g - 1] + c->gsize[g - 1];
  c->chiA.assign(n_groups + 1, 1);
  c->chiB.assign(n_groups + 1, 1);
  for (int g = 0; g < n_groups; ++g) {   // |0...0>: entry s = 0 of each [1][2^r][1] tensor
    const size_t n = (size_t)1 << c->gsize[g];
    s = ensure(c, c->B[g], n * c->esz);
    if (s == DMRGC_OK && cudaMemsetAsync(c->B[g].p, 0, n * c->esz, c->st) != cudaSuccess) s = DMRGC_ECUDA;
    if (s == DMRGC_OK && set_scalar_one(c->B[g].p, c->fp64, c->st) != cudaSuccess) s = DMRGC_ECUDA;
    if (s != DMRGC_OK) { dmrgc_destroy(c); return s; }
  }
  s = sync(c);
  if (s != DMRGC_OK) { dmrgc_destroy(c); return s; }
  *out = c;
  return DMRGC_OK;
}

dmrgc_status dmrgc_group_sizes(const dmrgc_ctx* c, int* sizes, int* count) {
  if (!c) return DMRGC_EINVAL;
  const int nt = c->ng > 0 ? c->ng : c->N;
  if (sizes)
    for (int g = 0; g < nt; ++g) sizes[g] = c->gsize[g];
  if (count) *count = nt;
  return DMRGC_OK;
}

dmrgc_status dmrgc_set_rank_model(dmrgc_ctx* c, const float* params) {
  if (!c || !params) return DMRGC_EINVAL;
  DevBuf tmp;
  TRY(ensure(c, tmp, DMRGC_MLP_PARAMS * sizeof(float)));
  TRY(ensure(c, c->mlp_w, DMRGC_MLP_PARAMS * 2));
  cudaError_t e = cudaMemcpyAsync(tmp.p, params, DMRGC_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = mlp_to_bf16((const float*)tmp.p, c->mlp_w.p, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  cudaFree(tmp.p);
  tmp.p = nullptr;
  if (e != cudaSuccess) return fail(c, DMRGC_ECUDA, cudaGetErrorString(e));
  c->stats.kernel_launches++;
  c->mlp_ready = true;
  return DMRGC_OK;
}

dmrgc_status dmrgc_rank_records(dmrgc_ctx* c, float* features, float* labels, int max, int* count) {
  if (!c || !count || max < 0 || (max > 0 && (!features || !labels))) return DMRGC_EINVAL;
  const int n = std::min<int>(max, (int)c->rec_y.size());
  std::copy(c->rec_x.begin(), c->rec_x.begin() + (size_t)n * DMRGC_MLP_IN, features);
  std::copy(c->rec_y.begin(), c->rec_y.begin() + n, labels);
  c->rec_x.erase(c->rec_x.begin(), c->rec_x.begin() + (size_t)n * DMRGC_MLP_IN);
  c->rec_y.erase(c->rec_y.begin(), c->rec_y.begin() + n);
  *count = n;
  return DMRGC_OK;
}

dmrgc_status dmrgc_batch_run(dmrgc_batch_item* items, int count, int n_workers, const dmrgc_options* opt,
                             const float* rank_model, double* wall_seconds) {
  if (wall_seconds) *wall_seconds = 0.0;
  if (count < 0 || (count > 0 && !items) || n_workers < 1 || n_workers > 64) return DMRGC_EINVAL;
  for (int i = 0; i < count; ++i) {
    dmrgc_batch_item& it = items[i];
    if (!valid_shape(it.rows * it.cols, &it.grid_view, it.chi) || it.grid_view.rows != it.rows ||
        it.grid_view.cols != it.cols ||
        it.n_layers < 0 || (it.n_layers > 0 && (!it.gates || !it.layer_sizes)) || it.n_sweeps < 0)
      return DMRGC_EINVAL;
    for (int l = 0; l < it.n_layers; ++l)
      if (it.layer_sizes[l] < 0) return DMRGC_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    items[i].status = DMRGC_ESTATE;   // not run (yet)
    items[i].worker = -1;
    items[i].log_F_tilde = 0.0;
    items[i].seconds = 0.0;
    items[i].updates = 0;
  }
  dmrgc_options base;
  if (opt) base = *opt; else dmrgc_default_options(&base);
  if (base.precision < 0 || base.precision > 3 || base.svd_mode < 0 || base.svd_mode > 2 ||
      (base.svd_mode == 2 && !rank_model))
    return DMRGC_EINVAL;
  if (count == 0) return DMRGC_OK;
  if (n_workers > count) n_workers = count;
  std::atomic<int> next{0};
  std::vector<dmrgc_status> worker_status(n_workers, DMRGC_OK);
  const auto t0 = std::chrono::steady_clock::now();
  auto work = [&](int wid) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      worker_status[wid] = DMRGC_ECUDA;
      return;
    }
    dmrgc_ctx* c = new (std::nothrow) dmrgc_ctx();
    if (!c) { worker_status[wid] = DMRGC_ENOMEM; cudaStreamDestroy(st); return; }
    c->esz = 0;
    c->st = st;
    if (rank_model) {   // every worker's context gets its own copy of the model
      const dmrgc_status ms = dmrgc_set_rank_model(c, rank_model);
      if (ms != DMRGC_OK) {
        worker_status[wid] = ms;
        delete c;
        cudaStreamDestroy(st);
        return;
      }
    }
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      dmrgc_batch_item& it = items[i];
      const auto s0 = std::chrono::steady_clock::now();
      dmrgc_options o = base;
      o.cuda_stream = st;
      o.timing = 0;
      dmrgc_status s = ctx_setup(c, it.rows * it.cols, &it.grid_view, it.chi, o);
      const dmrgc_gate* g = it.gates;
      long long updates0 = c->stats.updates;
      for (int l = 0; l < it.n_layers && s == DMRGC_OK; ++l) {
        s = dmrgc_apply_layer(c, g, it.layer_sizes[l]);
        g += it.layer_sizes[l];
        if (s == DMRGC_OK) s = dmrgc_sweep(c, it.n_sweeps, nullptr);
      }
      double lf = 0.0;
      if (s == DMRGC_OK) s = dmrgc_fidelity(c, &lf, nullptr);
      it.status = (int)s;
      it.log_F_tilde = lf;
      it.updates = c->stats.updates - updates0;
      it.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - s0).count();
      it.worker = wid;
    }
    delete c;
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < n_workers; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
  if (wall_seconds)
    *wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (auto st : worker_status)
    if (st != DMRGC_OK) return st;
  return DMRGC_OK;
}

dmrgc_status dmrgc_apply_layer(dmrgc_ctx* c, const dmrgc_gate* gates, int n_gates) {
  Range nvtx_range("dmrgc_apply_layer");
  if (!c) return DMRGC_EINVAL;
  if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(c, DMRGC_EINVAL, "bad gate list");
  if (c->phase == 1) {   // commit the previous step: its state becomes |Psi_Q(D)>
    c->log_ft += std::log(c->f_cur);
    std::swap(c->A, c->B);
    c->chiB = c->chiA;
  }
  c->hist.clear();
  c->layer_no++;
  // a new layer changes every spectrum: the first visit of each bond tries
  // the eigensolver again
  std::fill(c->eig_ok.begin(), c->eig_ok.end(), 1);
  TRY(build_mpo(c, gates, n_gates));
  if (c->ng > 0) {   // single-site variant: random guess in orthogonal form
    TRY(grouped_guess(c));
    c->phase = 1;
    return DMRGC_OK;
  }
  std::fill(c->xyk.begin(), c->xyk.end(), 0);
  TRY(zip_guess(c));
  c->bond = c->m - 1;
  c->dir = -1;
  c->phase = 1;
  return DMRGC_OK;
}

dmrgc_status dmrgc_sweep(dmrgc_ctx* c, int n_sweeps, double* f_last) {
  Range nvtx_range("dmrgc_sweep");
  if (!c) return DMRGC_EINVAL;
  if (c->phase != 1) return fail(c, DMRGC_ESTATE, "dmrgc_sweep before dmrgc_apply_layer");
  if (n_sweeps < 0) return fail(c, DMRGC_EINVAL, "n_sweeps < 0");
  if (c->ng > 0) TRY(grouped_sweeps(c, n_sweeps));
  else TRY(run_updates(c, (long long)n_sweeps * (c->N - 1)));
  if (f_last) *f_last = c->f_cur;
  return DMRGC_OK;
}

dmrgc_status dmrgc_fidelity(dmrgc_ctx* c, double* log_F_tilde, double* f_delta_last) {
  if (!c) return DMRGC_EINVAL;
  double lf = c->log_ft;
  if (c->phase == 1) lf += std::log(c->f_cur);
  if (log_F_tilde) *log_F_tilde = lf;
  if (f_delta_last) *f_delta_last = c->phase == 1 ? c->f_cur : 1.0;
  return DMRGC_OK;
}

static std::vector<DevBuf>& current_state(dmrgc_ctx* c, std::vector<int>*& bonds) {
  if (c->phase == 1) { bonds = &c->chiA; return c->A; }
  bonds = &c->chiB;
  return c->B;
}

// ---- batched read-outs: per site one GEMM W = V A_i for a chunk of strings
// (each site tensor read once per chunk), then a select kernel per row.  The
// GEMMs run in FP64 (FP64 mode), FP32 CUDA cores (FP32 mode) or TF32x3 on the
// tensor cores (both split modes: their finer split keeps the 54-site product
// within ~1e-5 relative).
int readout_precision(const dmrgc_ctx* c) {
  if (c->fp64) return DMRGC_FP64;
  return c->opt.precision == DMRGC_FP32 ? DMRGC_FP32 : DMRGC_TF32X3;
}

// rows per chunk: W[B][phys r] stays within 256 MB (phys = 2 or 2^r_tau)
int readout_chunk(const dmrgc_ctx* c, long long count, int maxb, long long phys = 2) {
  const long long cap = (256ll << 20) / (phys * std::max(maxb, 1) * (long long)c->esz);
  return (int)std::max(1ll, std::min({count, cap, 16384ll}));
}

dmrgc_status readout_site(dmrgc_ctx* c, const void* Ai, int B, int l, int r, int phys = 2) {
  GemmArgs g;   // W[b][(x c)] = sum_a V[b][a] A_i[a][(x c)]
  g.M = B; g.N = phys * r; g.K = l;
  g.A = c->rv[0].p; g.lda = l; g.opA = OP_N;
  g.B = Ai; g.ldb = (long long)phys * r; g.opB = OP_N;
  g.C = c->rv[1].p; g.ldc = (long long)phys * r;
  return gemm(c, g, readout_precision(c));
}

}  // extern "C"

namespace dmrgc_host {

// <x|Psi> for count strings already on the device (bits_dev [count][N], qubit
// order) into out_dev[count] (complex128), chunk by chunk
dmrgc_status amplitudes_device(dmrgc_ctx* c, const unsigned char* bits_dev, long long count, double2* out_dev) {
  std::vector<int>* bonds;
  auto& st = current_state(c, bonds);
  const int N = c->N;
  const int nt = c->ng > 0 ? c->ng : N;   // tensors; tensor i holds gsize[i] sites from gstart[i]
  const int maxb = *std::max_element(bonds->begin(), bonds->begin() + nt + 1);
  const int gmax = *std::max_element(c->gsize.begin(), c->gsize.begin() + nt);
  const long long pmax = 1ll << gmax;
  const int B0 = readout_chunk(c, count, maxb, pmax);
  TRY(ensure(c, c->rv[0], (size_t)B0 * maxb * c->esz));
  TRY(ensure(c, c->rv[1], (size_t)B0 * pmax * maxb * c->esz));
  TRY(ensure(c, c->order_d, sizeof(int) * N));   // qubit of each chain site
  CK(cudaMemcpyAsync(c->order_d.p, c->order.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c->st));
  const int* od = (const int*)c->order_d.p;
  for (long long row0 = 0; row0 < count; row0 += B0) {
    const int B = (int)std::min<long long>(B0, count - row0);
    const unsigned char* bd = bits_dev + row0 * N;
    {
      Span sp(c, TC_OTHER);
      CK(readout_start(c->rv[0].p, B, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    for (int i = 0; i < nt; ++i) {
      const int l = (*bonds)[i], r = (*bonds)[i + 1], g = c->gsize[i];
      TRY(readout_site(c, st[i].p, B, l, r, 1 << g));
      Span sp(c, TC_OTHER);
      CK(amp_select(c->rv[1].p, B, r, bd, N, od + c->gstart[i], g, c->rv[0].p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    Span sp(c, TC_OTHER);
    CK(amp_store(c->rv[0].p, B, out_dev + row0, c->fp64, c->st));
    c->stats.kernel_launches++;
  }
  return DMRGC_OK;
}

}  // namespace dmrgc_host

extern "C" {

dmrgc_status dmrgc_amplitude(dmrgc_ctx* c, const unsigned char* bits, long long count, double* out_re_im) {
  Range nvtx_range("dmrgc_amplitude");
  if (!c) return DMRGC_EINVAL;
  if (count < 0 || (count > 0 && (!bits || !out_re_im))) return fail(c, DMRGC_EINVAL, "bad amplitude arguments");
  if (count == 0) return DMRGC_OK;
  if (count > 0x7fffffffLL) return fail(c, DMRGC_EINVAL, "count too large");
  for (long long j = 0; j < count * c->N; ++j)
    if (bits[j] > 1) return fail(c, DMRGC_EINVAL, "bits must be 0 or 1");
  const int N = c->N;
  TRY(ensure(c, c->bits_d, (size_t)count * N));
  TRY(ensure(c, c->out_d, (size_t)count * sizeof(double2)));
  CK(cudaMemcpyAsync(c->bits_d.p, bits, (size_t)count * N, cudaMemcpyHostToDevice, c->st));
  TRY(amplitudes_device(c, (const unsigned char*)c->bits_d.p, count, (double2*)c->out_d.p));
  CK(cudaMemcpyAsync(out_re_im, c->out_d.p, (size_t)count * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
  return sync(c);
}

dmrgc_status dmrgc_metropolis(dmrgc_ctx* c, int chains, int steps, unsigned long long seed, unsigned char* out_bits,
                              long long* accepted) {
  Range nvtx_range("dmrgc_metropolis");
  if (!c) return DMRGC_EINVAL;
  if (chains < 1 || steps < 1 || !out_bits || (long long)chains * (steps + 1) > (1ll << 40))
    return fail(c, DMRGC_EINVAL, "bad metropolis arguments");
  const int N = c->N;
  const size_t outb = (size_t)chains * steps * N;
  TRY(ensure(c, c->bits_d, (size_t)chains * N * 2));   // proposals, current strings
  TRY(ensure(c, c->out_d, (size_t)chains * (sizeof(double2) + 2 * sizeof(double) + sizeof(long long))));
  TRY(ensure(c, c->stage_d, outb));
  unsigned char* prop = (unsigned char*)c->bits_d.p;
  unsigned char* cur = prop + (size_t)chains * N;
  double2* amp = (double2*)c->out_d.p;
  double* uacc = (double*)(amp + chains);
  double* pcur = uacc + chains;
  long long* acc = (long long*)(pcur + chains);
  CK(cudaMemsetAsync(acc, 0, (size_t)chains * sizeof(long long), c->st));
  for (int t = 0; t <= steps; ++t) {
    {
      Span sp(c, TC_OTHER);
      CK(metro_draw(prop, uacc, chains, N, steps, t, seed, c->st));
      c->stats.kernel_launches++;
    }
    TRY(amplitudes_device(c, prop, chains, amp));
    Span sp(c, TC_OTHER);
    CK(metro_step(prop, amp, uacc, cur, pcur, acc, (unsigned char*)c->stage_d.p, chains, N, steps, t, c->st));
    c->stats.kernel_launches++;
  }
  CK(cudaMemcpyAsync(out_bits, c->stage_d.p, outb, cudaMemcpyDeviceToHost, c->st));
  std::vector<long long> a(chains);
  CK(cudaMemcpyAsync(a.data(), acc, (size_t)chains * sizeof(long long), cudaMemcpyDeviceToHost, c->st));
  TRY(sync(c));
  if (accepted) {
    long long tot = 0;
    for (long long v : a) tot += v;
    *accepted = tot;
  }
  return DMRGC_OK;
}

dmrgc_status dmrgc_overlap(dmrgc_ctx* a, dmrgc_ctx* b, double* out_re_im) {
  Range nvtx_range("dmrgc_overlap");
  if (!a || !b || !out_re_im) return DMRGC_EINVAL;
  dmrgc_ctx* c = a;   // errors are reported on a
  if (a->N != b->N || a->rows != b->rows || a->cols != b->cols || a->fp64 != b->fp64 || a->order != b->order)
    return fail(a, DMRGC_EINVAL, "overlap needs contexts of the same grid, order and storage precision");
  if (a->ng > 0 || b->ng > 0) return fail(a, DMRGC_EINVAL, "overlap: contexts with one qubit per tensor only");
  std::vector<int>* ba;
  std::vector<int>* bb;
  auto& sa = current_state(a, ba);
  auto& sb = current_state(b, bb);
  if (b->st != a->st) CK(cudaStreamSynchronize(b->st));   // b's tensors are read on a's stream
  const size_t es = a->esz;
  // E[alpha][beta] over the bonds of a and b, from the left: E <- A_i^+ (E B_i).
  // The ping-pong buffers are a's own overlap scratch: envL / envR hold the
  // running sweep environments (c->L, c->R point into them), which a later
  // dmrgc_sweep on a still reads.
  const void* e_in = a->one.p;
  DevBuf* bufs[2] = {&a->ovl[0], &a->ovl[1]};
  for (int i = 0; i < a->N; ++i) {
    const int la = (*ba)[i], ra = (*ba)[i + 1], lb = (*bb)[i], rb = (*bb)[i + 1];
    TRY(ensure(a, a->T, (size_t)la * 2 * rb * es));
    GemmArgs g;   // T[alpha][s][b'] = E[alpha][beta] B_i[beta][s][b']
    g.M = la; g.N = 2 * rb; g.K = lb;
    g.A = e_in; g.lda = lb; g.opA = OP_N;
    g.B = sb[i].p; g.ldb = 2 * rb; g.opB = OP_N;
    g.C = a->T.p; g.ldc = 2 * rb;
    TRY(gemm(a, g));
    DevBuf* out = bufs[i & 1];
    TRY(ensure(a, *out, (size_t)ra * rb * es));
    GemmArgs h;   // E'[a'][b'] = sum_{alpha, s} conj(A_i[alpha][s][a']) T[alpha][s][b']
    h.M = ra; h.N = rb; h.K = 2 * la;
    h.A = sa[i].p; h.lda = ra; h.opA = OP_C;
    h.B = a->T.p; h.ldb = rb; h.opB = OP_N;
    h.C = out->p; h.ldc = rb;
    TRY(gemm(a, h));
    e_in = out->p;
  }
  TRY(ensure(a, a->out_d, sizeof(double2)));
  {
    Span sp(a, TC_OTHER);
    CK(to_complex128(e_in, 1, a->fp64, (double2*)a->out_d.p, a->st));
    a->stats.kernel_launches++;
  }
  CK(cudaMemcpyAsync(out_re_im, a->out_d.p, sizeof(double2), cudaMemcpyDeviceToHost, a->st));
  return sync(a);
}

dmrgc_status dmrgc_overlap_layer(dmrgc_ctx* a, dmrgc_ctx* b, const dmrgc_gate* gates, int n_gates,
                                 double* out_re_im) {
  Range nvtx_range("dmrgc_overlap_layer");
  if (!a || !b || !out_re_im || n_gates < 0 || (n_gates > 0 && !gates)) return DMRGC_EINVAL;
  dmrgc_ctx* c = a;   // errors are reported on a
  if (a->N != b->N || a->rows != b->rows || a->cols != b->cols || a->fp64 != b->fp64 || a->order != b->order)
    return fail(a, DMRGC_EINVAL, "overlap needs contexts of the same grid, order and storage precision");
  if (a->ng > 0 || b->ng > 0) return fail(a, DMRGC_EINVAL, "overlap: contexts with one qubit per tensor only");
  // the middle section's MPO lives in a scratch context on a's stream: o keeps
  // a's cuda_stream, so m->st == a->st and every ensure(m, ...) that grows a
  // buffer synchronises the stream the GEMMs below run on
  dmrgc_options o = a->opt;
  o.mpo_compress = 0;
  o.svd_mode = 0;
  o.log_rank_records = 0;
  dmrgc_grid grid{a->rows, a->cols, 0};
  dmrgc_ctx* m = nullptr;
  dmrgc_status st = dmrgc_create(a->N, &grid, 1, &o, &m);
  if (st != DMRGC_OK) return fail(a, st, "overlap: scratch context");
  struct Guard { dmrgc_ctx* p; ~Guard() { dmrgc_destroy(p); } } guard{m};
  if (m->st != a->st) return fail(a, DMRGC_ESTATE, "overlap: scratch context on another stream");
  st = build_mpo(m, gates, n_gates);
  if (st != DMRGC_OK) return fail(a, st, std::string("overlap: ") + m->err);
  if (b->st != a->st) CK(cudaStreamSynchronize(b->st));
  CK(cudaStreamSynchronize(m->st));
  std::vector<int>* ba;
  std::vector<int>* bb;
  auto& sa = current_state(a, ba);
  auto& sb = current_state(b, bb);
  const size_t es = a->esz;
  // E[alpha][w][beta] from the left: X = E B_i W_i (as in the sweep), E <- A_i^+ X
  const void* e_in = a->one.p;
  DevBuf* bufs[2] = {&m->envL, &m->envR};
  for (int i = 0; i < a->N; ++i) {
    const int la = (*ba)[i], ra = (*ba)[i + 1], lb = (*bb)[i], rb = (*bb)[i + 1];
    const int dw = m->D[i], dout = m->D[i + 1];
    TRY(ensure(m, m->T, (size_t)la * dw * 2 * rb * es));
    GemmArgs g1;   // T[alpha][w][t][b'] = E[alpha][w][beta] B_i[beta][t][b']
    g1.M = la * dw; g1.N = 2 * rb; g1.K = lb;
    g1.A = e_in; g1.lda = lb; g1.opA = OP_N;
    g1.B = sb[i].p; g1.ldb = 2 * rb; g1.opB = OP_N;
    g1.C = m->T.p; g1.ldc = 2 * rb;
    TRY(gemm(a, g1));
    TRY(ensure(m, m->jw, (size_t)la * 2 * dout * rb * es));
    GemmArgs g2;   // X[alpha][s][w'][b'] = sum_{w,t} W[w][s][t][w'] T[alpha][w][t][b']
    g2.M = 2 * dout; g2.N = rb; g2.K = 2 * dw; g2.b1 = la;
    g2.A = m->Wx[i].p; g2.lda = 2 * dw; g2.sA1 = 0; g2.opA = OP_N;
    g2.B = m->T.p; g2.ldb = rb; g2.sB1 = (long long)dw * 2 * rb; g2.opB = OP_N;
    g2.C = m->jw.p; g2.ldc = rb; g2.sC1 = (long long)2 * dout * rb;
    TRY(gemm(a, g2));
    DevBuf* out = bufs[i & 1];
    TRY(ensure(m, *out, (size_t)ra * dout * rb * es));
    GemmArgs h;   // E'[a'][w'][b'] = sum_{alpha, s} conj(A_i[alpha][s][a']) X[alpha][s][w'][b']
    h.M = ra; h.N = dout * rb; h.K = 2 * la;
    h.A = sa[i].p; h.lda = ra; h.opA = OP_C;
    h.B = m->jw.p; h.ldb = dout * rb; h.opB = OP_N;
    h.C = out->p; h.ldc = dout * rb;
    TRY(gemm(a, h));
    e_in = out->p;
  }
  TRY(ensure(a, a->out_d, sizeof(double2)));
  {
    Span sp(a, TC_OTHER);
    CK(to_complex128(e_in, 1, a->fp64, (double2*)a->out_d.p, a->st));
    a->stats.kernel_launches++;
  }
  CK(cudaMemcpyAsync(out_re_im, a->out_d.p, sizeof(double2), cudaMemcpyDeviceToHost, a->st));
  return sync(a);
}

dmrgc_status dmrgc_sample(dmrgc_ctx* c, long long count, unsigned long long seed, unsigned char* out_bits) {
  Range nvtx_range("dmrgc_sample");
  if (!c) return DMRGC_EINVAL;
  if (c->ng > 0) return fail(c, DMRGC_EINVAL, "sample: contexts with one qubit per tensor only");
  if (count < 0 || (count > 0 && !out_bits)) return fail(c, DMRGC_EINVAL, "bad sample arguments");
  if (count == 0) return DMRGC_OK;
  if (count > 0x7fffffffLL) return fail(c, DMRGC_EINVAL, "count too large");
  std::vector<int>* bonds;
  auto& st = current_state(c, bonds);
  const int N = c->N;
  const int centre = c->phase == 1 ? c->centre : 0;   // product state: any centre works
  // norm matrices E_i of sites > i for i < centre
  std::vector<const void*> eptr(N, nullptr);
  for (int i = centre - 1; i >= 0; --i) {
    const int a = (*bonds)[i + 1], b = (*bonds)[i + 2];
    TRY(ensure(c, c->E[i], (size_t)a * a * c->esz));
    TRY(ensure(c, c->T, (size_t)a * 2 * b * c->esz));
    const void* An = st[i + 1].p;
    const void* Tsrc = An;
    if (i + 1 < centre) {   // T[(a s)][b] = A_{i+1}[(a s)][b'] E_{i+1}[b'][b]
      GemmArgs g;
      g.M = 2 * a; g.N = b; g.K = b;
      g.A = An; g.lda = b; g.opA = OP_N;
      g.B = c->E[i + 1].p; g.ldb = b; g.opB = OP_N;
      g.C = c->T.p; g.ldc = b;
      TRY(gemm(c, g, readout_precision(c)));
      Tsrc = c->T.p;
    }
    GemmArgs h;   // E_i[a][a'] = sum_{(s b)} T[a][(s b)] conj(A_{i+1}[a'][(s b)])
    h.M = a; h.N = a; h.K = 2 * b;
    h.A = Tsrc; h.lda = 2 * b; h.opA = OP_N;
    h.B = An; h.ldb = 2 * b; h.opB = OP_C;
    h.C = c->E[i].p; h.ldc = a;
    TRY(gemm(c, h, readout_precision(c)));
    eptr[i] = c->E[i].p;
  }
  const int maxb = *std::max_element(bonds->begin(), bonds->begin() + N + 1);
  const int B0 = readout_chunk(c, count, maxb);
  TRY(ensure(c, c->rv[0], (size_t)B0 * maxb * c->esz));
  TRY(ensure(c, c->rv[1], (size_t)B0 * 2 * maxb * c->esz));
  if (centre > 0) TRY(ensure(c, c->rv[2], (size_t)B0 * 2 * maxb * c->esz));
  TRY(ensure(c, c->bits_d, (size_t)count * N));
  for (long long row0 = 0; row0 < count; row0 += B0) {
    const int B = (int)std::min<long long>(B0, count - row0);
    {
      Span sp(c, TC_OTHER);
      CK(readout_start(c->rv[0].p, B, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
    for (int i = 0; i < N; ++i) {
      const int l = (*bonds)[i], r = (*bonds)[i + 1];
      TRY(readout_site(c, st[i].p, B, l, r));
      const void* T = nullptr;
      if (i < centre) {   // T[(b x)][c'] = sum_c W[(b x)][c] E_i[c][c']
        GemmArgs g;
        g.M = 2 * B; g.N = r; g.K = r;
        g.A = c->rv[1].p; g.lda = r; g.opA = OP_N;
        g.B = eptr[i]; g.ldb = r; g.opB = OP_N;
        g.C = c->rv[2].p; g.ldc = r;
        TRY(gemm(c, g, readout_precision(c)));
        T = c->rv[2].p;
      }
      Span sp(c, TC_OTHER);
      CK(sample_select(c->rv[1].p, T, B, r, seed, row0, N, i, c->order[i], (unsigned char*)c->bits_d.p,
                       c->rv[0].p, c->fp64, c->st));
      c->stats.kernel_launches++;
    }
  }
  CK(cudaMemcpyAsync(out_bits, c->bits_d.p, (size_t)count * N, cudaMemcpyDeviceToHost, c->st));
  return sync(c);
}

dmrgc_status dmrgc_xeb(dmrgc_ctx* sampled, dmrgc_ctx* reference, long long count, unsigned long long seed,
                       double* f_b, double* stderr_out) {
  Range nvtx_range("dmrgc_xeb");
  if (!sampled || !reference || !f_b || count < 2 || count > (1LL << 26)) return DMRGC_EINVAL;
  dmrgc_ctx* c = sampled;
  if (sampled->N != reference->N || sampled->rows != reference->rows || sampled->cols != reference->cols)
    return fail(c, DMRGC_EINVAL, "xeb needs two contexts on the same grid");
  if (sampled->N > 62) return fail(c, DMRGC_EINVAL, "xeb: 2^N does not fit");
  if (sampled->ng > 0 || reference->ng > 0) return fail(c, DMRGC_EINVAL, "xeb: contexts with one qubit per tensor only");
  const int N = sampled->N;
  std::vector<unsigned char> bits((size_t)count * N);
  TRY(dmrgc_sample(sampled, count, seed, bits.data()));
  std::vector<double> amp((size_t)count * 2);
  const dmrgc_status st = dmrgc_amplitude(reference, bits.data(), count, amp.data());
  if (st != DMRGC_OK) return fail(c, st, std::string("xeb: ") + reference->err);
  // F_B = 2^N <p(x)> - 1 over the samples x (Eq. FB-estim); p = |<x|reference>|^2
  const double scale = std::ldexp(1.0, N);
  double sum = 0, sum2 = 0;
  for (long long j = 0; j < count; ++j) {
    const double p = amp[2 * j] * amp[2 * j] + amp[2 * j + 1] * amp[2 * j + 1];
    sum += scale * p;
    sum2 += scale * p * scale * p;
  }
  const double mean = sum / count;
  *f_b = mean - 1.0;
  if (stderr_out) *stderr_out = std::sqrt(std::max(sum2 / count - mean * mean, 0.0) / (count - 1));
  return DMRGC_OK;
}

dmrgc_status dmrgc_bond_dims(const dmrgc_ctx* c, int* mps_bonds, int* mpo_bonds) {
  if (!c) return DMRGC_EINVAL;
  const std::vector<int>& b = c->phase == 1 ? c->chiA : c->chiB;
  const int nt = c->ng > 0 ? c->ng : c->N;
  for (int i = 0; i + 1 < nt; ++i)
    if (mps_bonds) mps_bonds[i] = b[i + 1];
  for (int i = 0; i + 1 < c->N; ++i)
    if (mpo_bonds) mpo_bonds[i] = c->D[i + 1];
  return DMRGC_OK;
}

long long dmrgc_mps_size(const dmrgc_ctx* c) {
  if (!c) return -1;
  const std::vector<int>& b = c->phase == 1 ? c->chiA : c->chiB;
  const int nt = c->ng > 0 ? c->ng : c->N;
  long long s = 0;
  for (int i = 0; i < nt; ++i) s += (1LL << c->gsize[i]) * b[i] * b[i + 1];
  return s;
}

dmrgc_status dmrgc_get_mps(const dmrgc_ctx* cc, double* out_re_im, int* centre) {
  dmrgc_ctx* c = const_cast<dmrgc_ctx*>(cc);
  if (!c || !out_re_im) return DMRGC_EINVAL;
  std::vector<int>* bonds;
  auto& st = current_state(c, bonds);
  const int nt = c->ng > 0 ? c->ng : c->N;
  long long off = 0;
  for (int i = 0; i < nt; ++i) {
    const long long n = (1LL << c->gsize[i]) * (*bonds)[i] * (*bonds)[i + 1];
    TRY(ensure(c, c->stage_d, (size_t)n * sizeof(double2)));
    CK(to_complex128(st[i].p, n, c->fp64, (double2*)c->stage_d.p, c->st));
    CK(cudaMemcpyAsync(out_re_im + 2 * off, c->stage_d.p, (size_t)n * sizeof(double2),
                       cudaMemcpyDeviceToHost, c->st));
    TRY(sync(c));
    off += n;
  }
  if (centre) *centre = c->phase == 1 ? c->centre : 0;
  return DMRGC_OK;
}

dmrgc_status dmrgc_set_mps(dmrgc_ctx* c, const double* in_re_im, const int* bonds, double log_F_tilde) {
  if (!c) return DMRGC_EINVAL;
  if (!in_re_im || !bonds) return fail(c, DMRGC_EINVAL, "set_mps: null argument");
  const int N = c->ng > 0 ? c->ng : c->N;   // tensors
  if (bonds[0] != 1 || bonds[N] != 1) return fail(c, DMRGC_EINVAL, "set_mps: outer bonds must be 1");
  for (int i = 1; i < N; ++i)
    if (bonds[i] < 1 || bonds[i] > c->chi)
      return fail(c, DMRGC_EINVAL, "set_mps: bond " + std::to_string(i) + " out of range");
  for (int i = 0; i < N; ++i)
    if ((long long)bonds[i] * bonds[i + 1] * (1ll << c->gsize[i]) > (1ll << 27))
      return fail(c, DMRGC_EINVAL, "set_mps: tensor too large");
  long long off = 0;
  for (int i = 0; i < N; ++i) {
    const long long n = (1LL << c->gsize[i]) * bonds[i] * bonds[i + 1];
    TRY(ensure(c, c->B[i], (size_t)n * c->esz));
    TRY(ensure(c, c->stage_d, (size_t)n * sizeof(double2)));
    CK(cudaMemcpyAsync(c->stage_d.p, in_re_im + 2 * off, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice,
                       c->st));
    CK(from_complex128((const double2*)c->stage_d.p, n, c->fp64, c->B[i].p, c->st));
    TRY(sync(c));
    off += n;
  }
  c->chiB.assign(bonds, bonds + N + 1);
  c->chiA = c->chiB;
  c->phase = 0;
  c->log_ft = log_F_tilde;
  c->f_cur = 1.0;
  c->hist.clear();
  c->L = EnvRef();
  c->R = EnvRef();
  c->gsweep = 0;
  std::fill(c->xyk.begin(), c->xyk.end(), 0);
  return DMRGC_OK;
}

dmrgc_status dmrgc_sweep_updates(dmrgc_ctx* c, long long n_updates, double* f_last) {
  Range nvtx_range("dmrgc_sweep_updates");
  if (!c) return DMRGC_EINVAL;
  if (c->phase != 1) return fail(c, DMRGC_ESTATE, "dmrgc_sweep_updates before dmrgc_apply_layer");
  if (n_updates < 0) return fail(c, DMRGC_EINVAL, "n_updates < 0");
  if (c->ng > 0) return fail(c, DMRGC_EINVAL, "dmrgc_sweep_updates: two-site contexts only");
  TRY(run_updates(c, n_updates));
  if (f_last) *f_last = c->f_cur;
  return DMRGC_OK;
}

dmrgc_status dmrgc_step_history(const dmrgc_ctx* c, double* f, int cap, int* count) {
  if (!c) return DMRGC_EINVAL;
  const int n = (int)c->hist.size();
  if (f)
    for (int i = 0; i < n && i < cap; ++i) f[i] = c->hist[i];
  if (count) *count = n;
  return DMRGC_OK;
}

dmrgc_status dmrgc_get_stats(const dmrgc_ctx* c, dmrgc_stats* out) {
  if (!c || !out) return DMRGC_EINVAL;
  *out = c->stats;
  return DMRGC_OK;
}

dmrgc_status dmrgc_reset_stats(dmrgc_ctx* c) {
  if (!c) return DMRGC_EINVAL;
  dmrgc_status s = sync(c);
  std::memset(&c->stats, 0, sizeof(c->stats));
  return s;
}

const char* dmrgc_last_error(const dmrgc_ctx* c) { return c ? c->err.c_str() : "null context"; }

// ---- diagnostic entry points: one kernel family on host data

namespace {
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() { for (void* p : ptrs) cudaFree(p); }
  void* get(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    ptrs.push_back(p);
    return p;
  }
};

cudaError_t upload_as(const double* host, long long n, bool fp64, Scratch& s, void** out) {
  double2* z = (double2*)s.get(sizeof(double2) * n);
  *out = s.get((fp64 ? 16 : 8) * n);
  if (!z || !*out) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpy(z, host, sizeof(double2) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return from_complex128(z, n, fp64, *out, 0);
}

cudaError_t download_from(const void* dev, long long n, bool fp64, Scratch& s, double* host) {
  double2* z = (double2*)s.get(sizeof(double2) * n);
  if (!z) return cudaErrorMemoryAllocation;
  cudaError_t e = to_complex128(dev, n, fp64, z, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host, z, sizeof(double2) * n, cudaMemcpyDeviceToHost);
  return e;
}
}  // namespace

dmrgc_status dmrgc_test_gemm(int precision, int M, int N, int K, int opA, int opB, const double* A,
                             long long a_elems, long long lda, const double* B, long long b_elems,
                             long long ldb, double* C) {
  if (precision < 0 || precision > 3 || M < 1 || N < 1 || K < 1 || opA < 0 || opA > 3 || opB < 0 ||
      opB > 3 || !A || !B || !C || a_elems < 1 || b_elems < 1)
    return DMRGC_EINVAL;
  const bool fp64 = precision == DMRGC_FP64;
  Scratch s;
  void *dA, *dB;
  if (upload_as(A, a_elems, fp64, s, &dA) != cudaSuccess) return DMRGC_ECUDA;
  if (upload_as(B, b_elems, fp64, s, &dB) != cudaSuccess) return DMRGC_ECUDA;
  void* dC = s.get((size_t)(fp64 ? 16 : 8) * M * N);
  if (!dC) return DMRGC_ENOMEM;
  GemmArgs g;
  g.M = M; g.N = N; g.K = K;
  g.A = dA; g.lda = lda; g.opA = opA;
  g.B = dB; g.ldb = ldb; g.opB = opB;
  g.C = dC; g.ldc = N;
  int* err = (int*)s.get(sizeof(int));
  if (!err || cudaMemset(err, 0, sizeof(int)) != cudaSuccess) return DMRGC_ENOMEM;
  TcWork w;
  cudaError_t e = run_gemm(precision, g, &w, err, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  w.release();
  if (e != cudaSuccess) return DMRGC_ECUDA;
  if (herr) return DMRGC_ETIMEOUT;
  if (download_from(dC, (long long)M * N, fp64, s, C) != cudaSuccess) return DMRGC_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? DMRGC_OK : DMRGC_ECUDA;
}

dmrgc_status dmrgc_test_svd_gram(int precision, int m, int n, const double* G, int chi, double rel_cut,
                                 double* s_out, int* k_out, double* U_out) {
  if (precision < 1 || precision > 3 || m < 3 || m > 2048 || n < 1 || chi < 1 || chi >= m || !G || !s_out ||
      !k_out || !U_out)
    return DMRGC_EINVAL;
  Scratch s;
  void* dG;
  if (upload_as(G, (long long)m * n, false, s, &dG) != cudaSuccess) return DMRGC_ECUDA;
  void* dH = s.get((size_t)8 * m * m);
  const int kk = std::min(chi + 1, m);
  void* work = s.get(eig_work_bytes(m, kk));
  void* res = s.get(trunc_bytes(m));
  void* dU = s.get((size_t)8 * m * chi);
  int* err = (int*)s.get(sizeof(int));
  if (!dH || !work || !res || !dU || !err || cudaMemset(err, 0, sizeof(int)) != cudaSuccess) return DMRGC_ENOMEM;
  // G column-major m x n is the row-major [n][m] matrix Gt: H[r1][r2] = sum_c Gt[c][r1] conj(Gt[c][r2])
  GemmArgs g;
  g.M = m; g.N = m; g.K = n;
  g.A = dG; g.lda = m; g.opA = OP_T;
  g.B = dG; g.ldb = m; g.opB = OP_R;
  g.C = dH; g.ldc = m;
  g.upper_only = 1;
  TcWork w;
  cudaError_t e = run_gemm(precision == DMRGC_FP32 ? DMRGC_FP32 : DMRGC_TF32X3, g, &w, err, 0);
  if (e == cudaSuccess) e = eig_truncate(dH, m, chi, rel_cut, 0.0, kEigResolve, work, res, dU, 0, 0, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  w.release();
  if (e != cudaSuccess) return DMRGC_ECUDA;
  int herr = 0;
  TruncResult tr{};
  if (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&tr, res, sizeof(tr), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DMRGC_ECUDA;
  if (herr || tr.status == DMRGC_ETIMEOUT) return DMRGC_ETIMEOUT;
  if (tr.status == DMRGC_ENUMERIC) return DMRGC_ENUMERIC;
  if (cudaMemcpy(s_out, (const char*)res + sizeof(TruncResult), sizeof(double) * m, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return DMRGC_ECUDA;
  if (tr.status != 0) {
    *k_out = -1;
    return DMRGC_OK;
  }
  *k_out = tr.k;
  if (download_from(dU, (long long)m * tr.k, false, s, U_out) != cudaSuccess) return DMRGC_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? DMRGC_OK : DMRGC_ECUDA;
}

dmrgc_status dmrgc_test_svd(int precision, int m, int n, const double* G, int chi, double rel_cut,
                            double* s_out, int* k_out, double* U_out) {
  if (precision < 0 || precision > 3 || m < 1 || n < 2 || chi < 1 || !G || !s_out || !k_out || !U_out)
    return DMRGC_EINVAL;
  const bool fp64 = precision == DMRGC_FP64;
  Scratch s;
  void* dG;
  if (upload_as(G, (long long)m * n, fp64, s, &dG) != cudaSuccess) return DMRGC_ECUDA;
  void* ctl = s.get(jacobi_ctl_bytes(n));
  void* res = s.get(trunc_bytes(n));
  double* fro2 = (double*)s.get(sizeof(double));
  void* dU = s.get((size_t)(fp64 ? 16 : 8) * m * n);
  if (!ctl || !res || !fro2 || !dU) return DMRGC_ENOMEM;
  const double eps = fp64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
  const double tol = 8.0 * eps * std::sqrt((double)m);
  int launches = 0;
  if (sum_abs2(dG, (long long)m * n, fp64, fro2, 0) != cudaSuccess) return DMRGC_ECUDA;
  if (jacobi_orthogonalize(dG, m, n, fp64, tol, 40, fro2, fp64 ? 1e-13 : 1e-5, ctl, 0, &launches) !=
      cudaSuccess)
    return DMRGC_ECUDA;
  if (truncate_columns(dG, m, n, fp64, chi, rel_cut, false, 0.0, fro2, fp64 ? 1e-13 : 1e-5, res, 0) !=
      cudaSuccess)
    return DMRGC_ECUDA;
  TruncResult tr{};
  JacobiStatus cs{};
  if (cudaMemcpy(&tr, res, sizeof(tr), cudaMemcpyDeviceToHost) != cudaSuccess) return DMRGC_ECUDA;
  if (cudaMemcpy(&cs, ctl, sizeof(cs), cudaMemcpyDeviceToHost) != cudaSuccess) return DMRGC_ECUDA;
  if (cs.err == DMRGC_ETIMEOUT) return DMRGC_ETIMEOUT;
  if (cs.err == DMRGC_ENOCONV) return DMRGC_ENOCONV;
  if (tr.status != 0) return DMRGC_ENUMERIC;
  if (cudaMemcpy(s_out, (const char*)res + sizeof(TruncResult), sizeof(double) * n,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return DMRGC_ECUDA;
  *k_out = tr.k;
  if (gather_columns(dG, m, n, tr.k, res, false, 0, dU, fp64, 0) != cudaSuccess) return DMRGC_ECUDA;
  if (download_from(dU, (long long)m * tr.k, fp64, s, U_out) != cudaSuccess) return DMRGC_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? DMRGC_OK : DMRGC_ECUDA;
}

void dmrgc_destroy(dmrgc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  delete c;
}

}  // extern "C"
