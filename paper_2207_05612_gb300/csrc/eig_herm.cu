// Truncated SVD through the Hermitian eigenproblem of the Gram matrix.
//
// The update of Sec. IV.B keeps the chi leading singular vectors of theta on
// one side (Eq. optimization with the bond constraint).  Those are the leading
// eigenvectors of the Gram matrix H = G G^+ (G = theta for the left vectors,
// theta^+ for the right ones), formed by the contraction engine.  This file
// diagonalises H in three steps instead of the one-sided Jacobi sweeps:
//
//  1. he_tridiag_kernel: unitary Householder reduction H = Q T Q^+ with T
//     real symmetric tridiagonal (Q = P_0 P_1 ... P_{n-2}, P_j = I - tau_j u_j u_j^+).
//     One persistent cooperative kernel; rows are owned by CTAs cyclically and
//     kept in shared memory where they fit.  Step j forms column j of the
//     current matrix, the reflector, p = tau A u over the owned rows
//     (applying step j-1's rank-2 update A -= u w^+ + w u^+ in the same pass)
//     and a partial Re(conj(tau) u^+ p); one bounded grid barrier per step;
//     every CTA then forms w = p - (1/2) Re(conj(tau) u^+ p) u itself.
//     complex64 arithmetic.  The reflectors follow the LAPACK zlarfg
//     convention (complex tau, real beta), so T is real: the last one, of
//     size 1, only makes the final off-diagonal real.  A column below 1e-12
//     gets none (its tau would overflow FP32).
//  2. tri_bisect_kernel, tri_invit_kernel, tri_cluster_kernel: the leading
//     eigenvalues of T by Sturm-count multisection (FP32, one warp per
//     eigenvalue); their eigenvectors by inverse iteration in FP64 (the small
//     core), one thread per eigenvalue, then modified Gram-Schmidt inside
//     clusters of close eigenvalues and the Rayleigh quotients.
//  3. bt_wy_kernel and he_backtrans_kernel: eigenvector of H = Q z.  The
//     reflectors are grouped in blocks of WY in compact WY form
//     P_a .. P_{a+WY-1} = I - V Tb V^+ (Tb upper triangular), and each block is
//     applied to a column of z with one WY-wide reduction.
//
// H is scaled by 1/max_i H_ii first, so every entry lies in [-1, 1] whatever
// the scale of theta.  The Gram squares the condition number: eigenvalues
// carry an absolute error of about eps |H|, so singular values below ~1e-3
// s_1 are not resolved.  The caller therefore uses this path only when the
// kept eigenvalues all lie well above that level (lambda_{k-1} >= 1e-5
// lambda_0, set by the caller); otherwise, or when the eigensolver meets a
// non-finite value, the update falls back to the Jacobi SVD of theta itself.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace dmrgc {
namespace {

struct HeCtl {
  int err;            // 0 ok, DMRGC_ETIMEOUT
  unsigned count;     // grid-barrier arrivals of the tridiagonalisation (never reset in a launch)
  unsigned gen;       // (unused)
  int status;         // inverse iteration / clusters: 0 ok, 1 not resolved
  float scale;        // max(|d|, |beta|) of T, for the tridiagonal kernels
  int pad0;
  double gscale;      // max_i H_ii: H was divided by it
  int pad[8];
};
static_assert(sizeof(HeCtl) == 64, "control block layout");

constexpr unsigned long long kHeSpinLimit = 20000000ull;   // x ~64 ns, about 1.3 s

// Grid barrier: every CTA adds 1 to a counter that is never reset (zeroed
// before the launch) and waits until it reaches `target` = the number of
// arrivals of all steps so far, so no CTA has to observe a second write after
// the last arrival (bounded; on timeout or another CTA's error every thread
// of the CTA returns false).
__device__ __forceinline__ bool he_grid_barrier(HeCtl* c, unsigned target) {
  __shared__ int s_bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vcount = &c->count;
    volatile int* verr = &c->err;
    int bad = 0;
    __threadfence();
    atomicAdd(&c->count, 1u);
    unsigned long long it = 0;
    while (*vcount < target) {
      if (it > 2048) __nanosleep(32);
      if (*verr != 0) { bad = 1; break; }
      if (++it > kHeSpinLimit) {
        atomicExch(&c->err, (int)DMRGC_ETIMEOUT);
        bad = 1;
        break;
      }
    }
    __threadfence();
    s_bad = bad;
  }
  __syncthreads();
  return s_bad == 0;
}

__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ float2 f2cmul(float2 a, float2 b) {   // conj(a) b
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float2 f2conj(float2 a) { return {a.x, -a.y}; }

template <int NT>
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// block sum with one barrier: the caller alternates `red` buffers so that a
// buffer is rewritten only after a barrier has passed since its last read
template <int NT>
__device__ __forceinline__ float block_sum1(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// gscale = max_i Re H_ii (> 0 for a nonzero Gram), into ctl
__global__ void gram_scale_kernel(const float2* __restrict__ H, int n, HeCtl* ctl) {
  __shared__ float red[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, H[(long long)i * n + i].x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    ctl->gscale = (t > 0.f && isfinite(t)) ? (double)t : 1.0;
  }
}

// H <- upper triangle of H / gscale, mirrored: H[c][r] = conj(H[r][c]) for
// c > r and a real diagonal (the contraction engine computes only the tiles
// that touch the upper triangle of the Hermitian Gram)
__global__ void herm_sym_kernel(float2* __restrict__ H, int n, const HeCtl* __restrict__ ctl) {
  const float inv = (float)(1.0 / ctl->gscale);
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    if (c < r) continue;
    const float2 a = H[(long long)r * n + c];
    if (c == r) {
      H[(long long)r * n + c] = make_float2(inv * a.x, 0.f);
    } else {
      const float2 m = make_float2(inv * a.x, inv * a.y);
      H[(long long)r * n + c] = m;
      H[(long long)c * n + r] = make_float2(m.x, -m.y);
    }
  }
}

// ---------------------------------------------------------------- step 1
//
// Reflector of x = (alpha, x_2..) (the LAPACK zlarfg convention, written with
// the unscaled u): beta = -sign(Re alpha) |x| real, u = (alpha - beta, x_2..),
// tau = -1 / (beta conj(alpha - beta)); then P = I - tau u u^+ is unitary and
// P^+ x = beta e_1.  No reflection (tau = 0, beta = Re alpha) when x_2.. = 0
// and alpha is real, or when |x| < 1e-12: the scaled H has entries <= 1, so
// dropping such a column perturbs it far below its FP32 rounding, while its
// tau (~ 1 / |x|^2, formed through |x|^3) would overflow FP32 below ~1e-13.
// With P^+ A P = A - u w^+ - w u^+, p = tau A u, K = Re(conj(tau) u^+ p) / 2
// and w = p - K u.
constexpr int TD_THREADS = 256;
constexpr int TD_NQ = 8;   // columns per thread in the per-step loads: n <= 2048

__device__ __forceinline__ void reflector(float2 alpha, float rest, float2& tau, float& beta, float2& u0) {
  const float n2 = alpha.x * alpha.x + alpha.y * alpha.y + rest;
  if ((rest == 0.f && alpha.y == 0.f) || n2 < 1e-24f) {   // NaN takes the other branch
    tau = make_float2(0.f, 0.f);
    beta = alpha.x;
    u0 = alpha;
    return;
  }
  const float nrm = sqrtf(n2);
  beta = alpha.x >= 0.f ? -nrm : nrm;
  u0 = make_float2(alpha.x - beta, alpha.y);
  // tau = -1 / (beta conj(u0)) = -u0 / (beta |u0|^2)
  const float q = -1.f / (beta * (u0.x * u0.x + u0.y * u0.y));
  tau = make_float2(q * u0.x, q * u0.y);
}

// S: n x n row-major complex64, Hermitian (scaled); on return row j holds u_j
// at columns j+1..n-1.  d[n]: diagonal of T; beta[n-1]: its off-diagonal;
// tau[n-1]; pbuf: 2 n complex (p of the last two steps); rowbuf: 3 n complex
// (rows published by their owners); part: 2 gridDim.x floats.
// SMEM_ROWS: the CTA's rows (r = cta + G t) live in shared memory.
//
// Step j, in every CTA: (a) w_{j-1} = p_{j-1} - K u_{j-1} from the loads of
// the last barrier; (b) column j = conj(row j) with update j-1 (row j as its
// owner published it), the reflector; (c) the owned rows r >= j+1: update
// j-1, p_r, publication of row j+1 (and at the last step row j+2); (d) the
// barrier.
template <bool SMEM_ROWS>
__global__ void __launch_bounds__(TD_THREADS, 1)
    he_tridiag_kernel(float2* __restrict__ S, int n, double* __restrict__ d, double* __restrict__ beta,
                      float2* __restrict__ tau, float2* __restrict__ pbuf, float2* __restrict__ rowbuf,
                      float* __restrict__ part, HeCtl* ctl) {
  extern __shared__ float2 sm[];
  float2* vb0 = sm;              // u of even steps
  float2* vb1 = sm + n;          // u of odd steps
  float2* wp = sm + 2 * n;       // w of the previous step
  float2* rows = sm + 3 * n;     // owned rows (SMEM_ROWS)
  __shared__ float red[TD_THREADS / 32];
  __shared__ float red2[TD_THREADS / 32];
  __shared__ float2 s_tau;
  __shared__ float s_k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, cta = blockIdx.x;
  const int nrows = cta < n ? (n - 1 - cta) / G + 1 : 0;
  if (SMEM_ROWS) {
    for (int t = 0; t < nrows; ++t) {
      const float2* src = S + (size_t)(cta + G * t) * n;
      for (int c = tid; c < n; c += TD_THREADS) rows[(size_t)t * n + c] = src[c];
    }
  }
  for (int c = tid; c < n; c += TD_THREADS) {
    vb0[c] = make_float2(0.f, 0.f);
    vb1[c] = make_float2(0.f, 0.f);
    wp[c] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int j = 0; j + 2 < n; ++j) {
    float2* uc = (j & 1) ? vb1 : vb0;   // u_j
    float2* up = (j & 1) ? vb0 : vb1;   // u_{j-1}
    const bool pending = j > 0;
    const float2* rj = j == 0 ? S : rowbuf + (size_t)(j % 3) * n;
    const float2* Pp = pbuf + (size_t)((j - 1) & 1) * n;
    // one round of L2 loads per step: p_{j-1} and row j; thread tid owns
    // columns c = j + tid + TD_THREADS q
    float2 pv[TD_NQ], rv[TD_NQ];
#pragma unroll
    for (int q = 0; q < TD_NQ; ++q) {
      const int c = j + tid + TD_THREADS * q;
      pv[q] = (pending && c < n) ? __ldcg(Pp + c) : make_float2(0.f, 0.f);
      rv[q] = c < n ? __ldcg(rj + c) : make_float2(0.f, 0.f);
    }
    // w_{j-1} = p_{j-1} - K u_{j-1}, K = half the sum of the CTAs' partials,
    // summed by every warp (no broadcast barrier); each thread writes w for
    // its own columns and forms w_j of column j itself
    float2 wj = make_float2(0.f, 0.f);
    if (pending) {
      float v = 0.f;
      for (int g = lane; g < G; g += 32) v += __ldcg(part + (size_t)((j - 1) & 1) * G + g);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const float K = 0.5f * v;
#pragma unroll
      for (int q = 0; q < TD_NQ; ++q) {
        const int c = j + tid + TD_THREADS * q;
        if (c < n) {
          const float2 u = up[c];
          wp[c] = make_float2(pv[q].x - K * u.x, pv[q].y - K * u.y);
          if (cta == 0) S[(size_t)(j - 1) * n + c] = u;   // reflector j-1 for the back-transformation
        }
      }
      const float2 pj = tid == 0 ? pv[0] : __ldcg(Pp + j);
      wj = make_float2(pj.x - K * up[j].x, pj.y - K * up[j].y);
    }
    // column j below the diagonal = conj(row j) right of it, with update j-1
    float ss = 0.f;
    float2 djj = rv[0];   // thread 0: the diagonal element (c = j)
#pragma unroll
    for (int q = 0; q < TD_NQ; ++q) {
      const int c = j + tid + TD_THREADS * q;
      if (c <= j || c >= n) continue;
      float2 s = rv[q];
      if (pending) {
        const float2 t1 = f2mul(up[j], f2conj(wp[c]));
        const float2 t2 = f2mul(wj, f2conj(up[c]));
        s.x -= t1.x + t2.x;
        s.y -= t1.y + t2.y;
      }
      const float2 x = f2conj(s);
      uc[c] = x;
      if (c > j + 1) ss += x.x * x.x + x.y * x.y;
    }
    const float rest = block_sum1<TD_THREADS>(ss, red);   // ends after a __syncthreads
    if (tid == 0) {
      float2 t, u0;
      float b;
      reflector(uc[j + 1], rest, t, b, u0);
      uc[j + 1] = u0;
      uc[j] = make_float2(0.f, 0.f);
      s_tau = t;
      if (cta == 0) {
        if (pending) djj.x -= 2.f * f2mul(up[j], f2conj(wj)).x;
        d[j] = (double)djj.x;
        beta[j] = (double)b;
        tau[j] = t;
      }
    }
    __syncthreads();
    const float2 tj = s_tau;
    float dot = 0.f;
    float2* P = pbuf + (size_t)(j & 1) * n;
    const int t0 = j + 1 > cta ? (j + 1 - cta + G - 1) / G : 0;   // first owned row >= j+1
    for (int t = t0 + warp; t < nrows; t += TD_THREADS / 32) {
      const int r = cta + G * t;
      float2* row = SMEM_ROWS ? rows + (size_t)t * n : S + (size_t)r * n;
      const bool publish = r == j + 1 || (j + 3 == n && r == j + 2);
      float2* pub = rowbuf + (size_t)(r % 3) * n;
      const float2 ur = up[r], wr = wp[r];
      float px = 0.f, py = 0.f;
      for (int c = j + 1 + lane; c < n; c += 32) {
        float2 a = row[c];
        if (pending) {
          const float2 t1 = f2mul(ur, f2conj(wp[c]));
          const float2 t2 = f2mul(wr, f2conj(up[c]));
          a.x -= t1.x + t2.x;
          a.y -= t1.y + t2.y;
          row[c] = a;
        }
        if (publish) pub[c] = a;
        const float2 u = uc[c];
        px += a.x * u.x - a.y * u.y;
        py += a.x * u.y + a.y * u.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        px += __shfl_xor_sync(0xffffffffu, px, o);
        py += __shfl_xor_sync(0xffffffffu, py, o);
      }
      if (lane == 0) {
        const float2 p = f2mul(tj, make_float2(px, py));
        P[r] = p;
        dot += f2cmul(tj, f2cmul(uc[r], p)).x;   // Re(conj(tau) conj(u_r) p_r)
      }
    }
    const float tot = block_sum1<TD_THREADS>(dot, red2);
    if (tid == 0) part[(size_t)(j & 1) * G + cta] = tot;
    if (!he_grid_barrier(ctl, (unsigned)G * (unsigned)(j + 1))) return;
  }
  // trailing 2 x 2 block with the last pending update, and the 1 x 1 reflector
  // that makes its off-diagonal real (CTA 0)
  if (cta != 0) return;
  const int a = n - 2, jl = n - 3;
  float2* ul = (jl & 1) ? vb1 : vb0;   // u of the last step
  if (warp == 0) {
    float v = 0.f;
    for (int g = lane; g < G; g += 32) v += __ldcg(part + (size_t)(jl & 1) * G + g);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_k = 0.5f * v;
  }
  __syncthreads();
  const float K = s_k;
  const float2* P = pbuf + (size_t)(jl & 1) * n;
  for (int c = jl + 1 + tid; c < n; c += TD_THREADS) {
    const float2 p = __ldcg(P + c);
    const float2 u = ul[c];
    wp[c] = make_float2(p.x - K * u.x, p.y - K * u.y);
    S[(size_t)jl * n + c] = u;   // the last full reflector
  }
  __syncthreads();
  if (tid == 0) {
    const float2* ra = rowbuf + (size_t)(a % 3) * n;
    const float2* rb = rowbuf + (size_t)((n - 1) % 3) * n;
    float2 x00 = __ldcg(ra + a), x01 = __ldcg(ra + (n - 1)), x11 = __ldcg(rb + (n - 1));
    x00.x -= 2.f * f2mul(ul[a], f2conj(wp[a])).x;
    x11.x -= 2.f * f2mul(ul[n - 1], f2conj(wp[n - 1])).x;
    const float2 t1 = f2mul(ul[a], f2conj(wp[n - 1]));
    const float2 t2 = f2mul(wp[a], f2conj(ul[n - 1]));
    x01.x -= t1.x + t2.x;
    x01.y -= t1.y + t2.y;
    float2 t, u0;
    float b;
    reflector(f2conj(x01), 0.f, t, b, u0);   // A[n-1][n-2] = conj(A[n-2][n-1])
    d[a] = (double)x00.x;
    d[n - 1] = (double)x11.x;
    beta[a] = (double)b;
    tau[a] = t;
    S[(size_t)a * n + (n - 1)] = u0;
  }
}

// ---------------------------------------------------------------- step 2
//
// Real symmetric tridiagonal T: diagonal d, off-diagonal e (= beta).  prep:
// scale = max(|d|, |e|) (stored in ctl), the scaled diagonal and squared
// off-diagonal in FP32 for the Sturm counts.
__global__ void tri_prep_kernel(const double* __restrict__ d, const double* __restrict__ e, int n,
                                float* __restrict__ d32, float* __restrict__ e2_32, HeCtl* ctl) {
  __shared__ double red[1024];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mx = fmax(mx, fabs(d[i]));
    if (i + 1 < n) mx = fmax(mx, fabs(e[i]));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double scale = (red[0] > 0.0 && isfinite(red[0])) ? red[0] : 1.0;
  const double inv = 1.0 / scale;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d32[i] = (float)(d[i] * inv);
    if (i + 1 < n) {
      const float es = (float)(e[i] * inv);
      e2_32[i] = es * es;
    }
  }
  if (threadIdx.x == 0) ctl->scale = (float)scale;
}

// number of eigenvalues of the (scaled) T below x: negative pivots of the
// LDL^T factorisation of T - x I (Sturm sequence); approximate division
// (a couple of ulp) is ample for bisection
__device__ __forceinline__ int sturm_count(const float* __restrict__ d, const float* __restrict__ e2, int n, float x) {
  const float tiny = 1e-30f;
  int cnt = 0;
  float q = d[0] - x;
  if (fabsf(q) < tiny) q = -tiny;
  cnt += q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < tiny) q = -tiny;
    cnt += q < 0.f;
  }
  return cnt;
}

// one warp per eigenvalue (descending index i < kk): 6 rounds of 33-section
// on the Gershgorin interval; lam[i] in the scaled units of T
__global__ void tri_bisect_kernel(const float* __restrict__ d, const float* __restrict__ e2, int n, int kk,
                                  float* __restrict__ lam) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= kk) return;
  // Gershgorin bounds of the scaled matrix (entries <= 1): [-3, 3] holds every eigenvalue
  float lo = -3.0f, hi = 3.0f;
  const int target = n - 1 - warp;   // ascending index
  for (int round = 0; round < 6; ++round) {
    const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
    const int c = sturm_count(d, e2, n, x);
    const unsigned mask = __ballot_sync(0xffffffffu, c > target);
    const int f = mask ? __ffs(mask) - 1 : 32;
    const float x_hi = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
    const float x_lo = __shfl_sync(0xffffffffu, x, f > 0 ? (f < 32 ? f - 1 : 31) : 0);
    if (f == 32) lo = x_hi;            // every probe below the eigenvalue
    else {
      hi = x_hi;
      if (f > 0) lo = x_lo;
    }
  }
  if (lane == 0) lam[warp] = 0.5f * (lo + hi);
}

// Inverse iteration in FP64 for eigenvectors 0..kv-1 of T (scaled), one
// thread per eigenvalue.  Factorisation of T - sigma I by Gaussian
// elimination with partial pivoting (pivots below pivmin raised to pivmin),
// reciprocal pivots stored; INVIT_ITERS solves, each followed by a
// normalisation.  A thread keeps its factors, its row swaps and its vector in
// shared memory (5 n doubles + n bytes, blockDim.x threads per CTA, element i
// of thread lt at [i * blockDim.x + lt]).  Z: n x kk doubles (element i of
// vector v at Z[i * kk + v]).  Eigenvalues closer than the bisection's
// resolution give vectors that are not mutually orthogonal; tri_cluster_kernel
// orthonormalises each such cluster afterwards (their span is the cluster's
// invariant subspace, which is all the truncation uses) and forms the
// Rayleigh quotients.  Only vectors 0..kv-1 above the cut (lam[v] > cut2
// lam[0], cut2 = half the cut on s squared) are computed: kv is the most the
// truncation can keep, and the extra eigenvalue and those below the cut keep
// their bisection values.  A computed eigenvalue below half the resolution
// level (lam[v] < 0.5 resolve lam[0]) cannot belong to a resolved
// truncation: the thread flags the result unresolved and computes nothing
// more.
constexpr int INVIT_ITERS = 2;
constexpr int MAX_CLUSTER = 32;

// 1 / a for 1e-15 <= |a| <= 1e30: an FP32 reciprocal refined by two
// Newton-Raphson steps x <- x + x (1 - a x) in FP64 (each squares the
// relative error: ~1e-7 -> ~1e-14 -> below FP64 rounding)
__device__ __forceinline__ double recip_nr(double a) {
  double x = (double)__frcp_rn((float)a);
  double e = fma(-a, x, 1.0);
  x = fma(x, e, x);
  e = fma(-a, x, 1.0);
  return fma(x, e, x);
}

__global__ void tri_invit_kernel(const double* __restrict__ d0, const double* __restrict__ e0, int n, int kk,
                                 int kv, const float* __restrict__ lam, double cut2, double resolve,
                                 double* __restrict__ Z, double* __restrict__ lam_out, HeCtl* ctl) {
  extern __shared__ double ivs[];
  const int IV = blockDim.x, lt = threadIdx.x;
  double* IU0 = ivs;                      // 1 / pivot
  double* U1 = ivs + (size_t)n * IV;
  double* U2 = ivs + (size_t)2 * n * IV;
  double* L = ivs + (size_t)3 * n * IV;   // multipliers
  double* z = ivs + (size_t)4 * n * IV;
  unsigned char* swp = reinterpret_cast<unsigned char*>(ivs + (size_t)5 * n * IV);
  const int v = blockIdx.x * IV + lt;
  if (v >= kk) return;
  const double scale = (double)ctl->scale;
  if (v >= kv || !((double)lam[v] > cut2 * (double)lam[0])) {
    // the extra eigenvalue, or one below the cut (never kept): bisection value only
    lam_out[v] = (double)lam[v] * scale;
    return;
  }
  if (!((double)lam[v] >= 0.5 * resolve * (double)lam[0])) {
    atomicExch(&ctl->status, 1);
    return;
  }
  const double inv_scale = 1.0 / scale;
  const double pivmin = 1e-15;
#define IVX(arr, i) arr[(size_t)(i) * IV + lt]
  const double sigma = (double)lam[v];
  // factorisation (scaled entries)
  double ca = d0[0] * inv_scale - sigma;
  double cb = n > 1 ? e0[0] * inv_scale : 0.0;
  double ck = cb;   // subdiagonal of row k+1 = e_k
  for (int k = 0; k + 1 < n; ++k) {
    const double ak1 = d0[k + 1] * inv_scale - sigma;
    const double bk1 = (k + 2 < n) ? e0[k + 1] * inv_scale : 0.0;
    if (fabs(ca) >= fabs(ck)) {
      double piv = ca;
      if (fabs(piv) < pivmin) piv = piv < 0.0 ? -pivmin : pivmin;
      const double ip = recip_nr(piv);
      const double l = ck * ip;
      IVX(IU0, k) = ip; IVX(U1, k) = cb; IVX(U2, k) = 0.0; IVX(L, k) = l; IVX(swp, k) = 0;
      ca = ak1 - l * cb;
      cb = bk1;
    } else {
      const double ip = recip_nr(fabs(ck) < pivmin ? (ck < 0.0 ? -pivmin : pivmin) : ck);
      const double l = ca * ip;
      IVX(IU0, k) = ip; IVX(U1, k) = ak1; IVX(U2, k) = bk1; IVX(L, k) = l; IVX(swp, k) = 1;
      ca = cb - l * ak1;
      cb = -l * bk1;
    }
    ck = bk1;
  }
  {
    double piv = ca;
    if (fabs(piv) < pivmin) piv = piv < 0.0 ? -pivmin : pivmin;
    IVX(IU0, n - 1) = recip_nr(piv);
  }
  // start vector: a fixed pseudo-random sequence (integer hash of i, v)
  for (int i = 0; i < n; ++i) {
    unsigned h = (unsigned)i * 2654435761u ^ ((unsigned)v * 0x9E3779B9u + 0x7F4A7C15u);
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
    IVX(z, i) = 0.5 + (double)(h & 0xFFFFu) / 65536.0;
  }
  for (int it = 0; it < INVIT_ITERS; ++it) {
    // forward: the row operations of the elimination (y_k carried in a register)
    double yk = IVX(z, 0);
    for (int k = 0; k + 1 < n; ++k) {
      double yk1 = IVX(z, k + 1);
      const double l = IVX(L, k);
      if (IVX(swp, k)) { const double t = yk; yk = yk1; yk1 = t - l * yk; }
      else yk1 -= l * yk;
      IVX(z, k) = yk;
      yk = yk1;
    }
    IVX(z, n - 1) = yk;
    // back substitution (x_{k+1}, x_{k+2} carried in registers), with the norm
    double x2 = 0.0, x1 = 0.0, nrm = 0.0;
    for (int k = n - 1; k >= 0; --k) {
      double y = IVX(z, k);
      if (k + 1 < n) y -= IVX(U1, k) * x1;
      if (k + 2 < n) y -= IVX(U2, k) * x2;
      const double x = y * IVX(IU0, k);
      IVX(z, k) = x;
      nrm += x * x;
      x2 = x1;
      x1 = x;
    }
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int i = 0; i < n; ++i) IVX(z, i) *= inv;
  }
  for (int i = 0; i < n; ++i) Z[(size_t)i * kk + v] = IVX(z, i);
#undef IVX
}

// One CTA per eigenvalue index v < kv above the cut; the leader of each
// cluster (consecutive computed eigenvalues closer than clus_gap, scaled
// units) orthonormalises the
// cluster's vectors by modified Gram-Schmidt, twice, and every member gets its
// Rayleigh quotient z^T T z (units of H) in lam_out.  Clusters longer than
// MAX_CLUSTER flag the result unresolved.  256 threads.
__global__ void __launch_bounds__(256) tri_cluster_kernel(const double* __restrict__ d0,
                                                          const double* __restrict__ e0, int n, int kk, int kv,
                                                          const float* __restrict__ lam, double cut2,
                                                          double clus_gap, double* __restrict__ Z,
                                                          double* __restrict__ lam_out, HeCtl* ctl) {
  __shared__ double red[8];
  __shared__ int s_status;
  const int v0 = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) s_status = *((volatile int*)&ctl->status);
  __syncthreads();
  const double lcut = cut2 * (double)lam[0];
  if (v0 >= kv || s_status != 0 || !((double)lam[v0] > lcut)) return;   // uniform per CTA
  if (v0 > 0 && (double)lam[v0 - 1] - (double)lam[v0] <= clus_gap) return;   // not a cluster leader
  int v1 = v0 + 1;
  while (v1 < kv && (double)lam[v1] > lcut && (double)lam[v1 - 1] - (double)lam[v1] <= clus_gap) ++v1;
  if (v1 - v0 > MAX_CLUSTER) {
    if (tid == 0) atomicExch(&ctl->status, 1);
    return;
  }
  auto block_sum = [&](double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = x;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    return t;
  };
  if (v1 - v0 > 1) {
    for (int pass = 0; pass < 2; ++pass)
      for (int v = v0; v < v1; ++v) {
        for (int q = v0; q < v; ++q) {
          double dp = 0.0;
          for (int i = tid; i < n; i += 256) dp += Z[(size_t)i * kk + q] * Z[(size_t)i * kk + v];
          dp = block_sum(dp);
          for (int i = tid; i < n; i += 256) Z[(size_t)i * kk + v] -= dp * Z[(size_t)i * kk + q];
          __syncthreads();
        }
        double nr = 0.0;
        for (int i = tid; i < n; i += 256) { const double t = Z[(size_t)i * kk + v]; nr += t * t; }
        nr = block_sum(nr);
        const double inv = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
        for (int i = tid; i < n; i += 256) Z[(size_t)i * kk + v] *= inv;
        __syncthreads();
      }
  }
  for (int v = v0; v < v1; ++v) {   // Rayleigh quotient with the unscaled T
    double rq = 0.0;
    for (int i = tid; i < n; i += 256) {
      const double zi = Z[(size_t)i * kk + v];
      double tz = d0[i] * zi;
      if (i > 0) tz += e0[i - 1] * Z[(size_t)(i - 1) * kk + v];
      if (i + 1 < n) tz += e0[i] * Z[(size_t)(i + 1) * kk + v];
      rq += zi * tz;
    }
    rq = block_sum(rq);
    if (tid == 0) lam_out[v] = rq;
  }
}

// Truncation from the eigenvalues (kk = min(chi + 1, n) leading ones, in the
// units of the scaled H), in the result block of the Jacobi path
// (TruncResult, then s[n] descending and perm[n] = identity) so that the
// spectrum read-outs work unchanged: k = min(chi, n, #{s > cut s_1}); with
// tie_rel > 0 a cut inside a multiplet (s_{k-1} - s_k <= tie_rel s_1) moves
// down to the multiplet's upper edge.  status 0: every kept eigenvalue is
// resolved (lambda_{k-1} >= resolve lambda_0) and the count was not set by a
// cut below the resolution level (cut^2 < resolve: the sweep's cut, not the
// zip-up's); 1: not resolved; 2: the eigensolver met a non-finite value (both:
// the caller falls back to the Jacobi SVD); DMRGC_ETIMEOUT: a grid-barrier
// wait ran out.  One CTA of 1024.
__global__ void __launch_bounds__(1024) eig_trunc_kernel(const double* __restrict__ lam, int n, int kk, int chi,
                                                         double cut, double tie_rel, double resolve,
                                                         const double* __restrict__ d0, const float* __restrict__ lam32,
                                                         double cut2, TruncResult* res, HeCtl* ctl) {
  __shared__ double red[32];
  double* s = reinterpret_cast<double*>(res + 1);
  int* perm = reinterpret_cast<int*>(s + n);
  const int tid = threadIdx.x;
  const double gs = ctl->gscale;
  double tr = 0.0;
  int bad = 0;
  for (int i = tid; i < n; i += 1024) {
    tr += d0[i];   // trace of the scaled H
    const double l = i < kk ? lam[i] * gs : 0.0;
    if (!isfinite(l)) bad = 1;
    s[i] = l > 0.0 ? sqrt(l) : 0.0;
    perm[i] = i;
  }
  bad = __syncthreads_or(bad);
  double t = tr;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((tid & 31) == 0) red[tid >> 5] = t;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < 32; ++w) tot += red[w];
    tot *= gs;
    const int kmax = chi < n ? chi : n;
    int k = 0;
    while (k < kmax && s[k] > cut * s[0]) ++k;
    const int by_cut = k < kmax;
    if (tie_rel > 0 && k >= 1 && k < kk && s[k] > cut * s[0] && s[k - 1] - s[k] <= tie_rel * s[0]) {
      int kt = k;
      while (kt > 1 && s[kt - 1] - s[kt] <= tie_rel * s[0]) --kt;
      if (kt > 1 || s[0] - s[1] > tie_rel * s[0]) k = kt;
    }
    if (k < 1) k = 1;
    double f = 0.0;
    for (int i = 0; i < k; ++i) f += s[i] * s[i];
    // a timed-out reduction or a skipped (oversized) cluster leaves lam unset: decide on those first
    int st = 0;
    if (ctl->err != 0) st = (int)DMRGC_ETIMEOUT;
    else if (ctl->status != 0) st = 1;
    else if (bad || !isfinite(f) || !isfinite(tot)) st = 2;
    // a count set by the cut is trusted only when the cut itself (cut^2 in
    // eigenvalue units) lies at or above the resolution level
    else if ((by_cut && cut * cut < resolve) || !(lam[k - 1] >= resolve * lam[0]) || !(lam[0] > 0.0)) st = 1;
    // every kept vector must be one inverse iteration computed
    else if (k > kk || !((double)lam32[k - 1] > cut2 * (double)lam32[0])) st = 1;
    res->k = k;
    res->n = n;
    res->status = st;
    res->pad = 0;
    res->f = f;
    res->norm2 = tot;
    res->nnz = k;
    res->by_cut = by_cut;
    res->tail = s[0] > 0.0 ? (s[k - 1] / s[0]) * (s[k - 1] / s[0]) : 0.0;
  }
}

// ---------------------------------------------------------------- step 3
//
// Compact WY form of reflector blocks a = WY b .. WY b + WY - 1 (fewer in the
// last block): P_a P_{a+1} .. P_{a+m-1} = I - V Tb V^+ with V's columns the
// u_t (zero above row t+1) and Tb upper triangular:
//   Tb[i][i] = tau_i,  Tb[0..i-1][i] = -tau_i Tb[0..i-1][0..i-1] (V_{0..i-1}^+ u_i).
// One CTA per block computes the Gram V^+ V of its WY columns and Tb.
constexpr int WY = 8;

__global__ void __launch_bounds__(256) bt_wy_kernel(const float2* __restrict__ S, const float2* __restrict__ tau,
                                                    int n, float2* __restrict__ Tout) {
  __shared__ float2 g[WY][WY];
  __shared__ float2 T[WY][WY];
  const int b = blockIdx.x;
  const int a = b * WY;
  const int nref = n - 1;
  const int m = min(WY, nref - a);
  const int tid = threadIdx.x, lane = tid & 31;
  // g[i][j] = u_{a+i}^+ u_{a+j}, i < j (both nonzero only at rows > a+j)
  for (int p = tid >> 5; p < WY * WY; p += 8) {
    const int i = p / WY, j = p % WY;
    if (i >= j || j >= m) continue;
    const float2* ui = S + (size_t)(a + i) * n;
    const float2* uj = S + (size_t)(a + j) * n;
    float sx = 0.f, sy = 0.f;
    for (int r = a + j + 1 + lane; r < n; r += 32) {
      const float2 q = f2cmul(ui[r], uj[r]);
      sx += q.x;
      sy += q.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) g[i][j] = make_float2(sx, sy);
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < WY; ++i)
      for (int j = 0; j < WY; ++j) T[i][j] = make_float2(0.f, 0.f);
    for (int i = 0; i < m; ++i) {
      const float2 ti = tau[a + i];
      T[i][i] = ti;
      for (int r = 0; r < i; ++r) {
        float2 acc = make_float2(0.f, 0.f);
        for (int q = r; q < i; ++q) {
          const float2 t = f2mul(T[r][q], g[q][i]);
          acc.x += t.x;
          acc.y += t.y;
        }
        const float2 v = f2mul(ti, acc);
        T[r][i] = make_float2(-v.x, -v.y);
      }
    }
  }
  __syncthreads();
  if (tid < WY * WY) Tout[(size_t)b * WY * WY + tid] = (&T[0][0])[tid];
}

// One warp per eigenvector v < k (k = res->k): y = z_v (lane owns rows
// lane + 32 e), then for the blocks from the last to the first
// y <- (I - V Tb V^+) y: c = V^+ y (WY reductions in one pass), c <- Tb c,
// y -= V c.  The block's columns are staged in shared memory by the CTA.
// Output: mode 0: out[r * k + v] = y_r; mode 1: out[v * n + r] = y_r;
// mode 2: out[v * n + r] = conj(y_r).  A vector with a non-finite entry sets
// res->status = 2 (the caller then takes the Jacobi SVD).
constexpr int BT_WARPS = 4;

// 8-byte asynchronous global -> shared copy; src_bytes 0 writes zeros
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// DB: the WY blocks are staged in two shared buffers, the next block's copy
// in flight while the current one is applied (E <= 32: 2 x 64 KB)
template <int E, bool DB>
__global__ void __launch_bounds__(BT_WARPS * 32)
    he_backtrans_kernel(const float2* __restrict__ S, const float2* __restrict__ Tw, const double* __restrict__ Z,
                        int n, int kk, TruncResult* __restrict__ res, int mode, float2* __restrict__ out) {
  extern __shared__ float2 vsh_all[];   // (DB ? 2 : 1) x WY columns x 32 E rows
  __shared__ float2 tsh[WY * WY];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * BT_WARPS + warp;
  const int k = res->k;
  if (res->status != 0 || blockIdx.x * BT_WARPS >= k) return;   // uniform per CTA
  const bool active = v < k;
  float2 y[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = lane + 32 * e;
    y[e] = make_float2(active && r < n ? (float)Z[(size_t)r * kk + v] : 0.f, 0.f);
  }
  const int nref = n - 1;
  const int nblk = (nref + WY - 1) / WY;
  // V of block b (column i = u_{b WY + i}, zero at rows <= b WY + i) into buf
  auto stage = [&](int b, float2* buf) {
    const int a = b * WY;
    const int m = min(WY, nref - a);
    for (int p = threadIdx.x; p < WY * 32 * E; p += BT_WARPS * 32) {
      const int i = p / (32 * E), r = p % (32 * E);
      const bool ok = i < m && r > a + i && r < n;
      if (DB) cp_async8(buf + p, ok ? S + (size_t)(a + i) * n + r : S, ok ? 8 : 0);
      else buf[p] = ok ? S[(size_t)(a + i) * n + r] : make_float2(0.f, 0.f);
    }
    if (DB) cp_async_commit();
  };
  if (DB) stage(nblk - 1, vsh_all);
  for (int b = nblk - 1; b >= 0; --b) {
    const int a = b * WY;
    float2* vsh = DB ? vsh_all + (size_t)((nblk - 1 - b) & 1) * WY * 32 * E : vsh_all;
    __syncthreads();   // every warp is done with the buffer about to be refilled, and with tsh
    if (DB) {
      if (b > 0) {
        stage(b - 1, vsh_all + (size_t)((nblk - b) & 1) * WY * 32 * E);
        cp_async_wait<1>();   // block b's copy has landed (b - 1's may still be in flight)
      } else {
        cp_async_wait<0>();
      }
    } else {
      stage(b, vsh);
    }
    for (int p = threadIdx.x; p < WY * WY; p += BT_WARPS * 32) tsh[p] = Tw[(size_t)b * WY * WY + p];
    __syncthreads();
    if (!active) continue;
    float2 c[WY];
#pragma unroll
    for (int i = 0; i < WY; ++i) c[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (32 * e + 31 <= a) continue;   // rows <= a: every column of the block is zero there
      const float2 ys = make_float2(y[e].y, y[e].x);
#pragma unroll
      for (int i = 0; i < WY; ++i) {   // c_i += conj(v) y, two packed FMAs
        const float2 vv = vsh[i * 32 * E + lane + 32 * e];
        c[i] = __ffma2_rn(make_float2(vv.x, vv.x), y[e], c[i]);
        c[i] = __ffma2_rn(make_float2(vv.y, -vv.y), ys, c[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < WY; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        c[i].x += __shfl_xor_sync(0xffffffffu, c[i].x, o);
        c[i].y += __shfl_xor_sync(0xffffffffu, c[i].y, o);
      }
    }
    float2 tc[WY];
#pragma unroll
    for (int i = 0; i < WY; ++i) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = i; q < WY; ++q) {
        const float2 t = f2mul(tsh[i * WY + q], c[q]);
        acc.x += t.x;
        acc.y += t.y;
      }
      tc[i] = acc;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (32 * e + 31 <= a) continue;
#pragma unroll
      for (int i = 0; i < WY; ++i) {   // y -= v tc, two packed FMAs
        const float2 vv = vsh[i * 32 * E + lane + 32 * e];
        y[e] = __ffma2_rn(make_float2(-vv.x, -vv.x), tc[i], y[e]);
        y[e] = __ffma2_rn(make_float2(vv.y, -vv.y), make_float2(tc[i].y, tc[i].x), y[e]);
      }
    }
  }
  if (!active) return;
  bool finite = true;
#pragma unroll
  for (int e = 0; e < E; ++e) finite = finite && isfinite(y[e].x) && isfinite(y[e].y);
  if (!__all_sync(0xffffffffu, finite) && lane == 0) atomicExch(&res->status, 2);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = lane + 32 * e;
    if (r < n) {
      if (mode == 0) out[(size_t)r * k + v] = y[e];
      else if (mode == 1) out[(size_t)v * n + r] = y[e];
      else out[(size_t)v * n + r] = make_float2(y[e].x, -y[e].y);
    }
  }
}

// work-space layout of eig_truncate, parts rounded to 256 bytes
constexpr int kParts = 13;

struct EigParts {
  size_t off[kParts];
  size_t total;
};

EigParts eig_parts(int n, int kk) {
  const size_t NK = (size_t)n * kk;
  const int nblk = (n - 1 + WY - 1) / WY;
  const size_t sizes[kParts] = {sizeof(HeCtl),                            // ctl
                                (size_t)2 * n * sizeof(float2),           // pbuf
                                (size_t)3 * n * sizeof(float2),           // rowbuf
                                (size_t)2 * 1024 * sizeof(float),         // partial sums (<= 1024 CTAs)
                                (size_t)n * sizeof(double),               // d
                                (size_t)n * sizeof(double),               // e (= beta)
                                (size_t)n * sizeof(double),               // lam (Rayleigh quotients)
                                (size_t)n * sizeof(float2),               // tau
                                (size_t)n * sizeof(float),                // d32
                                (size_t)n * sizeof(float),                // e2_32
                                (size_t)n * sizeof(float),                // lam32
                                (size_t)nblk * WY * WY * sizeof(float2),  // WY blocks
                                NK * sizeof(double)};                     // Z
  EigParts p{};
  size_t o = 0;
  for (int i = 0; i < kParts; ++i) {
    p.off[i] = o;
    o += (sizes[i] + 255) & ~size_t(255);
  }
  p.total = o;
  return p;
}

}  // namespace

size_t eig_work_bytes(int n, int kk) { return eig_parts(n, kk).total; }

cudaError_t eig_truncate(void* H, int n, int chi, double cut, double tie_rel, double resolve, void* work,
                         void* res, void* out, int mode, cudaStream_t st, int* launches) {
  if (n < 3 || n > 2048 || chi < 1) return cudaErrorInvalidValue;
  const int kk = chi + 1 < n ? chi + 1 : n;
  const EigParts P = eig_parts(n, kk);
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  HeCtl* ctl = reinterpret_cast<HeCtl*>(w + P.off[0]);
  float2* pbuf = reinterpret_cast<float2*>(w + P.off[1]);
  float2* rowbuf = reinterpret_cast<float2*>(w + P.off[2]);
  float* part = reinterpret_cast<float*>(w + P.off[3]);
  double* d = reinterpret_cast<double*>(w + P.off[4]);
  double* e = reinterpret_cast<double*>(w + P.off[5]);
  double* lam = reinterpret_cast<double*>(w + P.off[6]);
  float2* tau = reinterpret_cast<float2*>(w + P.off[7]);
  float* d32 = reinterpret_cast<float*>(w + P.off[8]);
  float* e2 = reinterpret_cast<float*>(w + P.off[9]);
  float* lam32 = reinterpret_cast<float*>(w + P.off[10]);
  float2* Tw = reinterpret_cast<float2*>(w + P.off[11]);
  double* Z = reinterpret_cast<double*>(w + P.off[12]);
  cudaError_t e_ = cudaMemsetAsync(ctl, 0, sizeof(HeCtl), st);
  if (e_ != cudaSuccess) return e_;
  float2* S = reinterpret_cast<float2*>(H);
  gram_scale_kernel<<<1, 1024, 0, st>>>(S, n, ctl);
  if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  herm_sym_kernel<<<std::min(4096, (n * n + 255) / 256), 256, 0, st>>>(S, n, ctl);
  if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  // 1. tridiagonalisation (cooperative: every CTA resident).  Rows in shared
  // memory when ceil(n / G) rows and the three vectors fit in one CTA.
  int dev = 0, sms = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t static_smem = 1024;
  int G = std::min(sms, std::max(1, n / 4));
  const size_t row_bytes = (size_t)n * sizeof(float2);
  size_t dsm = (size_t)(3 + (n + G - 1) / G) * row_bytes;
  const bool smem_rows = dsm + static_smem <= (size_t)max_smem;
  const void* tfn = smem_rows ? (const void*)he_tridiag_kernel<true> : (const void*)he_tridiag_kernel<false>;
  if (!smem_rows) dsm = 3 * row_bytes;
  if ((e_ = allow_dyn_smem(tfn)) != cudaSuccess) return e_;
  int per_sm = 0;
  if ((e_ = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tfn, TD_THREADS, dsm)) != cudaSuccess) return e_;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (!smem_rows) G = std::min(sms * per_sm, std::min(1024, std::max(1, n / 8)));
  {
    int nn = n;
    void* args[] = {&S, &nn, &d, &e, &tau, &pbuf, &rowbuf, &part, &ctl};
    e_ = cudaLaunchCooperativeKernel(tfn, dim3(G), dim3(TD_THREADS), args, dsm, st);
    if (e_ != cudaSuccess) return e_;
  }
  // 2. eigenvalues and eigenvectors of T
  tri_prep_kernel<<<1, 1024, 0, st>>>(d, e, n, d32, e2, ctl);
  if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  tri_bisect_kernel<<<(kk * 32 + 255) / 256, 256, 0, st>>>(d32, e2, n, kk, lam32);
  if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  // clusters: consecutive eigenvalues (scaled units) closer than 3e-5; iv
  // threads per CTA with 5 n doubles + n bytes of shared memory each
  {
    const size_t per_thread = (size_t)n * (5 * sizeof(double) + 1);
    int iv = (int)std::min<size_t>(8, ((size_t)max_smem - static_smem) / per_thread);
    if (iv < 1) return cudaErrorInvalidConfiguration;
    while (iv > 1 && (kk + iv - 1) / iv < sms) iv /= 2;   // spread small problems over the SMs
    const size_t ism = per_thread * iv;
    if ((e_ = allow_dyn_smem((const void*)tri_invit_kernel)) != cudaSuccess) return e_;
    const int kv = kk > chi ? chi : kk;   // vectors the truncation can keep
    // vectors are computed down to half the squared cut: the truncation
    // counts with the Rayleigh quotients, which differ from the bisection
    // values by far less than that margin, so it never counts a vector that
    // was not computed (eig_trunc_kernel checks this too)
    const double cut2 = 0.5 * cut * cut;
    tri_invit_kernel<<<(kk + iv - 1) / iv, iv, ism, st>>>(d, e, n, kk, kv, lam32, cut2, resolve, Z, lam, ctl);
    if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
    tri_cluster_kernel<<<kv, 256, 0, st>>>(d, e, n, kk, kv, lam32, cut2, 3e-5, Z, lam, ctl);
    if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  }
  TruncResult* tr = reinterpret_cast<TruncResult*>(res);
  eig_trunc_kernel<<<1, 1024, 0, st>>>(lam, n, kk, chi, cut, tie_rel, resolve, d, lam32, 0.5 * cut * cut, tr, ctl);
  if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  // 3. back-transformation of the k kept eigenvectors
  const int nblk = (n - 1 + WY - 1) / WY;
  bt_wy_kernel<<<nblk, 256, 0, st>>>(S, tau, n, Tw);
  if ((e_ = cudaGetLastError()) != cudaSuccess) return e_;
  const void* fn;
  int E;
  if (n <= 32 * 8) { fn = (const void*)he_backtrans_kernel<8, true>; E = 8; }
  else if (n <= 32 * 16) { fn = (const void*)he_backtrans_kernel<16, true>; E = 16; }
  else if (n <= 32 * 32) { fn = (const void*)he_backtrans_kernel<32, true>; E = 32; }
  else { fn = (const void*)he_backtrans_kernel<64, false>; E = 64; }
  const size_t bsm = (size_t)(E <= 32 ? 2 : 1) * WY * 32 * E * sizeof(float2);
  if ((e_ = allow_dyn_smem(fn)) != cudaSuccess) return e_;
  {
    const float2* Sc = S;
    const float2* tc = Tw;
    const double* zc = Z;
    float2* o = reinterpret_cast<float2*>(out);
    int nn = n, kkk = kk, md = mode;
    TruncResult* rc = tr;
    void* args[] = {(void*)&Sc, (void*)&tc, (void*)&zc, &nn, &kkk, (void*)&rc, &md, &o};
    e_ = cudaLaunchKernel(fn, dim3((kk + BT_WARPS - 1) / BT_WARPS), dim3(BT_WARPS * 32), args, bsm, st);
    if (e_ != cudaSuccess) return e_;
  }
  if (launches) *launches += 10;
  return cudaSuccess;
}

}  // namespace dmrgc
