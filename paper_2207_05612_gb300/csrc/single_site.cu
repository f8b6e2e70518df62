// Single-site compression over grouped qubits (Sec. IV.A, IV.B.1, V.C).
//
// The MPS has ng tensors; tensor tau holds the gsize[tau] consecutive sites
// from gstart[tau] on, M^(tau)[a][s][c] with s the 2^r basis states of its
// sites (the first site the most significant bit).  The layer operator stays
// per site (Wx_i[(s w')][(w t)], the two-site path's layout); a group's
// operator is applied one site at a time inside the contractions below, so no
// 4^r operator tensor is ever formed.  Device layouts (row-major, complex):
//   L_tau [a][w][b]    contraction of the new tensors' conjugates, the layer
//                      operator and the old tensors B of the groups left of tau
//   R_tau [c][w][b]    the same right of tau (cut tau is left of tensor tau)
//   X     [a][s_1..s_r][w'][b']  = L_tau B^(tau) W^(tau): T0 = L B, then per
//                      site j one batched GEMM contracting (w_{j-1}, t_j)
//                      into (s_j, w_j), batch = (a, s_1..s_{j-1})
//   F     [(a s)][c]   = X R_{tau+1}^T                  (Eq. scalarproduct)
// One update: f = |F|^2, M = F / sqrt(f) (Eq. optimization); moving right,
// M[(a s)][c] is replaced by its left singular vectors, moving left M[a][(s c)]
// by its right ones (the Jacobi SVD; values at the numerical-zero level are
// dropped, which may shrink the bond), and the environment is extended over
// tensor tau: L_{tau+1} = U^+ X, or R_tau = conj(V^+) R_{tau+1} W^(tau)^T B^T
// site by site from the right.  The guess is a random tensor train (entries
// in the unit square from SplitMix64, Sec. V.D.1) brought to orthogonal form
// with its centre on tensor 0 by right-to-left factorisations that carry each
// remaining factor into the left neighbour.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ctx.cuh"

using namespace dmrgc;

namespace dmrgc_host {
namespace {

constexpr long long kMaxBatch = 65535;   // grid z of one GEMM launch

// gemm with the first batch index split into launches of at most kMaxBatch
dmrgc_status gemm_chunked(dmrgc_ctx* c, GemmArgs g) {
  const int total = g.b1;
  for (int b0 = 0; b0 < total; b0 += (int)kMaxBatch) {
    GemmArgs h = g;
    h.b1 = (int)std::min<long long>(kMaxBatch, total - b0);
    const size_t e = c->esz;
    h.A = static_cast<const char*>(g.A) + (size_t)b0 * g.sA1 * e;
    h.B = static_cast<const char*>(g.B) + (size_t)b0 * g.sB1 * e;
    h.C = static_cast<char*>(g.C) + (size_t)b0 * g.sC1 * e;
    TRY(gemm(c, h));
  }
  return DMRGC_OK;
}

int pow2cap(int bits) { return bits >= 30 ? (1 << 30) : (1 << bits); }

// largest per-site MPO bond inside group tau (its two end cuts included)
long long max_inner_bond(const dmrgc_ctx* c, int tau) {
  long long d = 1;
  for (int j = 0; j <= c->gsize[tau]; ++j) d = std::max<long long>(d, c->D[c->gstart[tau] + j]);
  return d;
}

// ping-pong buffers large enough for the X chain and the R chain of tensor tau
// (rows a of the environment side, k the new bond)
dmrgc_status chain_buffers(dmrgc_ctx* c, int tau, long long rows) {
  const long long S = 1ll << c->gsize[tau];
  const long long bmax = std::max(c->chiB[tau], c->chiB[tau + 1]);
  const size_t bytes = (size_t)(rows * S * max_inner_bond(c, tau) * bmax) * c->esz;
  TRY(ensure(c, c->gx[0], bytes));
  return ensure(c, c->gx[1], bytes);
}

// X^(tau) = L B^(tau) W^(tau) into c->gx[which]: [a][s_1..s_r][w_r][b']
dmrgc_status make_x_group(dmrgc_ctx* c, int tau, const void* L, int a, int& which) {
  const int r = c->gsize[tau], p = c->gstart[tau];
  const int b = c->chiB[tau], bp = c->chiB[tau + 1];
  const long long S = 1ll << r;
  TRY(chain_buffers(c, tau, a));
  GemmArgs g;   // T0[(a w_0)][(t b')] = L[(a w_0)][b] B[b][(t b')]
  g.M = a * c->D[p]; g.N = (int)(S * bp); g.K = b;
  g.A = L; g.lda = b; g.opA = OP_N;
  g.B = c->B[tau].p; g.ldb = S * bp; g.opB = OP_N;
  g.C = c->gx[0].p; g.ldc = S * bp;
  TRY(gemm(c, g));
  int cur = 0;
  for (int j = 1; j <= r; ++j) {   // site p + j - 1: (w_{j-1}, t_j) -> (s_j, w_j)
    const int din = c->D[p + j - 1], dout = c->D[p + j];
    const long long rest = (S >> j) * bp;
    GemmArgs h;
    h.M = 2 * dout; h.N = (int)rest; h.K = 2 * din; h.b1 = a << (j - 1);
    h.A = c->Wx[p + j - 1].p; h.lda = 2 * din; h.sA1 = 0; h.opA = OP_N;
    h.B = c->gx[cur].p; h.ldb = rest; h.sB1 = 2 * din * rest; h.opB = OP_N;
    h.C = c->gx[cur ^ 1].p; h.ldc = rest; h.sC1 = 2 * dout * rest;
    TRY(gemm_chunked(c, h));
    cur ^= 1;
  }
  which = cur;
  return DMRGC_OK;
}

// R_tau[k][w_0][b] = sum conj(A[k][s][c]) R_{tau+1}[c][w_r][b'] W^(tau) B^(tau)[b][t][b']
// (A: the right isometry of tensor tau, k rows); into GR[tau]
dmrgc_status make_r_group(dmrgc_ctx* c, int tau, int k) {
  const int r = c->gsize[tau], p = c->gstart[tau];
  const int b = c->chiB[tau], bp = c->chiB[tau + 1];
  const int cc = c->chiA[tau + 1];
  const long long S = 1ll << r;
  const int dr = c->D[p + r];
  TRY(chain_buffers(c, tau, k));
  GemmArgs g;   // P[(k s)][(w_r b')] = conj(A)[(k s)][c] R_{tau+1}[c][(w_r b')]
  g.M = (int)(k * S); g.N = dr * bp; g.K = cc;
  g.A = c->A[tau].p; g.lda = cc; g.opA = OP_R;
  g.B = c->GR[tau + 1].p; g.ldb = (long long)dr * bp; g.opB = OP_N;
  g.C = c->gx[0].p; g.ldc = (long long)dr * bp;
  TRY(gemm(c, g));
  int cur = 0;
  for (int j = r; j >= 1; --j) {   // site p + j - 1: (s_j, w_j) -> (w_{j-1}, t_j)
    const int din = c->D[p + j - 1], dout = c->D[p + j];
    const long long rest = (S >> j) * bp;
    GemmArgs h;
    h.M = 2 * din; h.N = (int)rest; h.K = 2 * dout; h.b1 = k << (j - 1);
    h.A = c->Wx[p + j - 1].p; h.lda = 2 * din; h.sA1 = 0; h.opA = OP_T;
    h.B = c->gx[cur].p; h.ldb = rest; h.sB1 = 2 * dout * rest; h.opB = OP_N;
    h.C = c->gx[cur ^ 1].p; h.ldc = rest; h.sC1 = 2 * din * rest;
    TRY(gemm_chunked(c, h));
    cur ^= 1;
  }
  const int d0 = c->D[p];
  TRY(ensure(c, c->GR[tau], (size_t)k * d0 * b * c->esz));
  GemmArgs e;   // R_tau[(k w_0)][b] = P[(k w_0)][(t b')] B[b][(t b')]^T
  e.M = k * d0; e.N = b; e.K = (int)(S * bp);
  e.A = c->gx[cur].p; e.lda = S * bp; e.opA = OP_N;
  e.B = c->B[tau].p; e.ldb = S * bp; e.opB = OP_T;
  e.C = c->GR[tau].p; e.ldc = b;
  return gemm(c, e);
}

// the isometry of the block in `src` (rows x cols, row-major): left = true:
// the left singular vectors U [rows][k]; left = false: the right ones V^+
// [k][cols]; singular values at the numerical-zero level are dropped.  The
// result goes to dst, k to *k.
dmrgc_status isometry(dmrgc_ctx* c, const void* src, long long rows, long long cols, bool left, DevBuf& dst,
                      int& k) {
  TRY(ensure(c, c->jw, (size_t)(rows * cols) * c->esz));
  {
    Span sp(c, TC_OTHER);
    if (left) CK(copy_transpose(src, (int)rows, (int)cols, false, c->jw.p, c->fp64, c->st));   // M, column-major
    else CK(copy_conj(src, rows * cols, c->jw.p, c->fp64, c->st));   // M^+, column-major
    c->stats.kernel_launches++;
  }
  const int m = (int)(left ? rows : cols), n = (int)(left ? cols : rows);
  double f = 0;
  int nnz = 0;
  TRY(svd_columns(c, m, n, 0.0, false, 0.0, k, f, &nnz, nullptr, nullptr, n));
  TRY(ensure(c, dst, (size_t)m * k * c->esz));
  Span sp(c, TC_SVD);
  CK(gather_columns(c->jw.p, m, n, k, c->tres.p, false, left ? 0 : 2, dst.p, c->fp64, c->st));
  c->stats.kernel_launches++;
  return DMRGC_OK;
}

// one update of tensor tau (Sec. IV.B.1); right: the sweep moves to tau + 1
dmrgc_status update_group(dmrgc_ctx* c, int tau, bool right) {
  const int ng = c->ng;
  const int a = c->chiA[tau], cc = c->chiA[tau + 1];
  const int r = c->gsize[tau], p = c->gstart[tau];
  const long long S = 1ll << r;
  const int dr = c->D[p + r], bp = c->chiB[tau + 1];
  int xi = 0;
  TRY(make_x_group(c, tau, c->GL[tau].p, a, xi));
  TRY(ensure(c, c->gf, (size_t)(a * S * cc) * c->esz));
  GemmArgs g;   // F[(a s)][c] = X[(a s)][(w_r b')] R_{tau+1}[c][(w_r b')]^T
  g.M = (int)(a * S); g.N = cc; g.K = dr * bp;
  g.A = c->gx[xi].p; g.lda = (long long)dr * bp; g.opA = OP_N;
  g.B = c->GR[tau + 1].p; g.ldb = (long long)dr * bp; g.opB = OP_T;
  g.C = c->gf.p; g.ldc = cc;
  TRY(gemm(c, g));
  double f = 0;
  TRY(normalise_block(c, c->gf.p, a * S * cc, f));
  c->f_cur = f;
  c->hist.push_back(f);
  c->stats.updates++;
  if (right && tau < ng - 1) {
    int k = 0;
    TRY(isometry(c, c->gf.p, a * S, cc, true, c->A[tau], k));
    c->chiA[tau + 1] = k;
    TRY(ensure(c, c->GL[tau + 1], (size_t)k * dr * bp * c->esz));
    GemmArgs h;   // L_{tau+1}[k][(w_r b')] = U^+ X
    h.M = k; h.N = dr * bp; h.K = (int)(a * S);
    h.A = c->A[tau].p; h.lda = k; h.opA = OP_C;
    h.B = c->gx[xi].p; h.ldb = (long long)dr * bp; h.opB = OP_N;
    h.C = c->GL[tau + 1].p; h.ldc = (long long)dr * bp;
    TRY(gemm(c, h));
    c->centre = tau + 1;
  } else if (!right && tau > 0) {
    int k = 0;
    TRY(isometry(c, c->gf.p, a, S * cc, false, c->A[tau], k));
    c->chiA[tau] = k;
    TRY(make_r_group(c, tau, k));
    c->centre = tau - 1;
  } else {
    TRY(ensure(c, c->A[tau], (size_t)(a * S * cc) * c->esz));
    CK(cudaMemcpyAsync(c->A[tau].p, c->gf.p, (size_t)(a * S * cc) * c->esz, cudaMemcpyDeviceToDevice, c->st));
    c->centre = tau;
  }
  return DMRGC_OK;
}

}  // namespace

// Random guess of the layer (seed opt.seed + layer number) in orthogonal form
// with its centre on tensor 0, and the right environments R_1..R_{ng-1}.
dmrgc_status grouped_guess(dmrgc_ctx* c) {
  const int ng = c->ng;
  // bonds: min(chi, 2^{sites left}, 2^{sites right}, chi_old D at the cut)
  c->chiA.assign(ng + 1, 1);
  for (int tau = 1; tau < ng; ++tau) {
    const int left = c->gstart[tau];
    const long long cap = (long long)c->chiB[tau] * c->D[left];
    c->chiA[tau] = (int)std::max<long long>(
        1, std::min<long long>({(long long)c->chi, (long long)pow2cap(std::min(left, c->N - left)), cap}));
  }
  const unsigned long long seed = c->opt.seed + (unsigned long long)(c->layer_no - 1);
  unsigned long long off = 0;
  for (int tau = 0; tau < ng; ++tau) {
    const long long n = (long long)c->chiA[tau] * (1ll << c->gsize[tau]) * c->chiA[tau + 1];
    TRY(ensure(c, c->A[tau], (size_t)n * c->esz));
    Span sp(c, TC_OTHER);
    CK(fill_unit_square(c->A[tau].p, n, c->fp64, seed, 2ull * off, c->st));
    c->stats.kernel_launches++;
    off += (unsigned long long)n;
  }
  // right-to-left: M^(tau) = Lo V^+, tensor tau <- V^+, tensor tau-1 <- tensor tau-1 Lo
  for (int tau = ng - 1; tau >= 1; --tau) {
    const int a = c->chiA[tau], cc = c->chiA[tau + 1];
    const long long S = 1ll << c->gsize[tau];
    int k = 0;
    TRY(isometry(c, c->A[tau].p, a, S * cc, false, c->gf, k));
    TRY(ensure(c, c->T, (size_t)a * k * c->esz));
    GemmArgs g;   // Lo[a][k] = M[a][(s c)] V[(s c)][k]
    g.M = a; g.N = k; g.K = (int)(S * cc);
    g.A = c->A[tau].p; g.lda = S * cc; g.opA = OP_N;
    g.B = c->gf.p; g.ldb = S * cc; g.opB = OP_C;
    g.C = c->T.p; g.ldc = k;
    TRY(gemm(c, g));
    std::swap(c->A[tau], c->gf);
    const int al = c->chiA[tau - 1];
    const long long Sl = 1ll << c->gsize[tau - 1];
    TRY(ensure(c, c->gf, (size_t)(al * Sl * k) * c->esz));
    GemmArgs h;   // M^(tau-1)[(a' s')][k] = M^(tau-1)[(a' s')][a] Lo[a][k]
    h.M = (int)(al * Sl); h.N = k; h.K = a;
    h.A = c->A[tau - 1].p; h.lda = a; h.opA = OP_N;
    h.B = c->T.p; h.ldb = k; h.opB = OP_N;
    h.C = c->gf.p; h.ldc = k;
    TRY(gemm(c, h));
    std::swap(c->A[tau - 1], c->gf);
    c->chiA[tau] = k;
  }
  if ((int)c->GL.size() < ng + 1) c->GL.resize(ng + 1);
  if ((int)c->GR.size() < ng + 1) c->GR.resize(ng + 1);
  TRY(ensure(c, c->GL[0], 64));
  TRY(ensure(c, c->GR[ng], 64));
  CK(set_scalar_one(c->GL[0].p, c->fp64, c->st));
  CK(set_scalar_one(c->GR[ng].p, c->fp64, c->st));
  for (int tau = ng - 1; tau >= 1; --tau) TRY(make_r_group(c, tau, c->chiA[tau]));
  c->gsweep = 0;
  c->centre = 0;
  return sync(c);
}

dmrgc_status grouped_sweeps(dmrgc_ctx* c, int n_sweeps) {
  for (int k = 0; k < n_sweeps; ++k) {
    const bool right = c->gsweep % 2 == 0;
    if (right)
      for (int tau = 0; tau < c->ng; ++tau) TRY(update_group(c, tau, true));
    else
      for (int tau = c->ng - 1; tau >= 0; --tau) TRY(update_group(c, tau, false));
    c->gsweep++;
  }
  return sync(c);
}

}  // namespace dmrgc_host
