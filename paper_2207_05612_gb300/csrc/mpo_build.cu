// Layer-MPO builder: K gate cycles -> W_i[D_{i}, 2, 2, D_{i+1}] over the MPS sites.
//
// The paper merges one-qubit gates into neighbouring gates and contracts the K
// layers of a compression step vertically (Sec. IV.B.2, Fig. 4).  Here every
// two-qubit gate is split by an operator SVD (App. A), U = sum_k A_k (x) B_k,
// and the layer becomes an exact MPO: the bond at a snake cut is the tuple of
// Schmidt indices of the gates that straddle the cut (mixed radix, the later
// gate fastest).  Site i's tensor is, for each value of its legs, the time-
// ordered product of the 2x2 operators acting on its qubit (one-qubit gates
// and the A_k / B_k factors of its two-qubit gates), times a Kronecker delta on
// the legs of gates that only pass over the site.  No truncation: the MPO is
// exactly the layer unitary.
#include "common.cuh"

namespace dmrgc {
namespace {

__device__ inline void gate_matrix(const GateDev& g, int sp, int sq, int tp, int tq, double2& out) {
  // <s_p s_q|U|t_p t_q>; the stored matrix lists q0 first, q0 at site p unless swapped
  int r, c;
  if (!g.swap) { r = 2 * sp + sq; c = 2 * tp + tq; }
  else { r = 2 * sq + sp; c = 2 * tq + tp; }
  out = double2{g.mat[2 * (4 * r + c)], g.mat[2 * (4 * r + c) + 1]};
}

// one thread per gate: 4x4 complex SVD by one-sided Jacobi with V accumulated
__global__ void gate_split_kernel(const GateDev* __restrict__ gates, int n, int* __restrict__ rank,
                                  double2* __restrict__ fa, double2* __restrict__ fb) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= n) return;
  const GateDev g = gates[gi];
  if (g.q < 0) { rank[gi] = 0; return; }
  double2 M[4][4], V[4][4];   // M[row][col], row = 2 s_p + t_p, col = 2 s_q + t_q
  for (int sp = 0; sp < 2; ++sp)
    for (int tp = 0; tp < 2; ++tp)
      for (int sq = 0; sq < 2; ++sq)
        for (int tq = 0; tq < 2; ++tq) gate_matrix(g, sp, sq, tp, tq, M[2 * sp + tp][2 * sq + tq]);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) V[i][j] = double2{i == j ? 1.0 : 0.0, 0.0};
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double al = 0, be = 0, gr = 0, gim = 0;
        for (int i = 0; i < 4; ++i) {
          const double2 x = M[i][a], y = M[i][b];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          gr += x.x * y.x + x.y * y.y;
          gim += x.x * y.y - x.y * y.x;
        }
        const double ga = sqrt(gr * gr + gim * gim);
        if (al < 1e-300 || be < 1e-300 || ga < 1e-300) continue;
        const double rel = ga / sqrt(al * be);
        if (rel < 1e-16) continue;
        off = fmax(off, rel);
        const double er = gr / ga, ei = -gim / ga;
        const double zeta = (al - be) / (2 * ga);
        const double sg = zeta >= 0 ? 1.0 : -1.0;
        const double t = -sg / (fabs(zeta) + sqrt(1 + zeta * zeta));
        const double c = 1 / sqrt(1 + t * t), s = c * t;
        for (int i = 0; i < 4; ++i) {
          double2 x = M[i][a], y = M[i][b];
          double2 ye{y.x * er - y.y * ei, y.x * ei + y.y * er};
          M[i][a] = double2{c * x.x - s * ye.x, c * x.y - s * ye.y};
          M[i][b] = double2{s * x.x + c * ye.x, s * x.y + c * ye.y};
          x = V[i][a]; y = V[i][b];
          ye = double2{y.x * er - y.y * ei, y.x * ei + y.y * er};
          V[i][a] = double2{c * x.x - s * ye.x, c * x.y - s * ye.y};
          V[i][b] = double2{s * x.x + c * ye.x, s * x.y + c * ye.y};
        }
      }
    if (off < 1e-16) break;
  }
  double sv[4];
  int idx[4];
  for (int j = 0; j < 4; ++j) {
    double s = 0;
    for (int i = 0; i < 4; ++i) s += M[i][j].x * M[i][j].x + M[i][j].y * M[i][j].y;
    sv[j] = sqrt(s);
    idx[j] = j;
  }
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b)
      if (sv[idx[b]] > sv[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
  int r = 0;
  for (int j = 0; j < 4; ++j)
    if (sv[idx[j]] > 1e-14 * sv[idx[0]]) ++r;
  rank[gi] = r;
  for (int k = 0; k < 4; ++k) {
    const int j = idx[k];
    const double s = sv[j];
    const double inv = (k < r && s > 0) ? 1.0 / sqrt(s) : 0.0;
    const double rs = (k < r) ? sqrt(s) : 0.0;
    for (int x = 0; x < 4; ++x) {
      // A_k[x] = W[x][j] / sqrt(s) ; B_k[y] = sqrt(s) conj(V[y][j])
      fa[(gi * 4 + k) * 4 + x] = double2{M[x][j].x * inv, M[x][j].y * inv};
      fb[(gi * 4 + k) * 4 + x] = double2{rs * V[x][j].x, -rs * V[x][j].y};
    }
  }
}

constexpr int kMaxLegs = 24;

template <typename C2>
__global__ void site_mpo_kernel(const int* __restrict__ tab, SitePlan sp, const GateDev* __restrict__ gates,
                                const double2* __restrict__ fa, const double2* __restrict__ fb,
                                C2* __restrict__ wx, C2* __restrict__ wy) {
  const long long total = (long long)sp.d_in * sp.d_out;
  const int* in_rec = tab + sp.off;                 // n_in x {gate, radix, pass_out}
  const int* out_rec = in_rec + 3 * sp.n_in;        // n_out x {gate, radix}
  const int* ops = out_rec + 2 * sp.n_out;          // n_ops x {kind, gate, leg}
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int w_out = (int)(e / sp.d_in);
    const int w_in = (int)(e % sp.d_in);
    int din[kMaxLegs], dout[kMaxLegs];
    int rem = w_in;
    for (int j = sp.n_in - 1; j >= 0; --j) { const int rad = in_rec[3 * j + 1]; din[j] = rem % rad; rem /= rad; }
    rem = w_out;
    for (int j = sp.n_out - 1; j >= 0; --j) { const int rad = out_rec[2 * j + 1]; dout[j] = rem % rad; rem /= rad; }
    bool ok = true;
    for (int j = 0; j < sp.n_in; ++j) {
      const int po = in_rec[3 * j + 2];
      if (po >= 0 && din[j] != dout[po]) ok = false;
    }
    double2 O[2][2] = {{{1, 0}, {0, 0}}, {{0, 0}, {1, 0}}};
    if (ok) {
      for (int o = 0; o < sp.n_ops; ++o) {
        const int kind = ops[3 * o], gid = ops[3 * o + 1], leg = ops[3 * o + 2];
        double2 G[2][2];
        if (kind == 0) {
          const double* m = gates[gid].mat;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) G[a][b] = double2{m[2 * (2 * a + b)], m[2 * (2 * a + b) + 1]};
        } else {
          const int k = (kind == 1) ? dout[leg] : din[leg];
          const double2* f = (kind == 1 ? fa : fb) + (gid * 4 + k) * 4;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) G[a][b] = f[2 * a + b];
        }
        double2 T[2][2];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            double2 acc{0, 0};
            for (int c = 0; c < 2; ++c) acc = cadd(acc, cmul(G[a][c], O[c][b]));
            T[a][b] = acc;
          }
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) O[a][b] = T[a][b];
      }
    }
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < 2; ++t) {
        const double2 v = ok ? O[s][t] : double2{0, 0};
        const C2 c{(decltype(C2{}.x))v.x, (decltype(C2{}.x))v.y};
        wx[(((long long)s * sp.d_out + w_out) * sp.d_in + w_in) * 2 + t] = c;
        wy[(((long long)s * sp.d_in + w_in) * sp.d_out + w_out) * 2 + t] = c;
      }
  }
}

}  // namespace

cudaError_t gate_split(const GateDev* gates, int n_gates, int* rank, double2* fa, double2* fb,
                       cudaStream_t st) {
  if (n_gates <= 0) return cudaSuccess;
  gate_split_kernel<<<(n_gates + 63) / 64, 64, 0, st>>>(gates, n_gates, rank, fa, fb);
  return cudaGetLastError();
}

cudaError_t build_site_mpo(const int* plan_tab, SitePlan sp, const GateDev* gates, const double2* fa,
                           const double2* fb, void* wx, void* wy, bool fp64, cudaStream_t st) {
  if (sp.n_in > kMaxLegs || sp.n_out > kMaxLegs) return cudaErrorInvalidValue;
  const long long total = (long long)sp.d_in * sp.d_out;
  long long blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (fp64)
    site_mpo_kernel<double2><<<(int)blocks, 256, 0, st>>>(plan_tab, sp, gates, fa, fb, (double2*)wx,
                                                           (double2*)wy);
  else
    site_mpo_kernel<float2><<<(int)blocks, 256, 0, st>>>(plan_tab, sp, gates, fa, fb, (float2*)wx,
                                                          (float2*)wy);
  return cudaGetLastError();
}

}  // namespace dmrgc
