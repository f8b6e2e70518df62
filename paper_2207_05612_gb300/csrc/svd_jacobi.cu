// Truncated complex SVD by one-sided (Hestenes) Jacobi.
//
// theta (or a Gram matrix) is orthogonalised column-pair by column-pair:
// for a pair (u, v) with alpha = |u|^2, beta = |v|^2, gamma = u^+ v, a unitary
// 2x2 rotation zeroes gamma.  Pairs follow the round-robin (circle) order, so
// one round holds n/2 disjoint pairs that run in parallel, one warp per pair;
// n-1 rounds make a sweep.  All sweeps run in one persistent cooperative
// kernel: rounds are separated by a grid barrier whose wait is bounded (an
// exhausted wait sets an error flag and every CTA returns).  Convergence: a
// sweep whose largest |gamma|/sqrt(alpha beta) is below tol ends the loop.
//
// On return the columns of W = G V are mutually orthogonal; their norms are
// the singular values and W_j / |W_j| the left singular vectors (Eckart-Young
// truncation then keeps the k largest, Eq. optimization with the bond
// constraint).  The side computed this way is orthonormal to working
// precision, which is why callers orthogonalise theta for a left-to-right
// update and theta^+ for a right-to-left one.
#include <cooperative_groups.h>

#include <atomic>
#include <cstddef>
#include <mutex>

#include "common.cuh"

namespace dmrgc {
namespace {

struct JacobiCtl {
  int err;                // 0 ok, DMRGC_ETIMEOUT, DMRGC_ENOCONV   (JacobiStatus)
  int sweeps;             // sweeps executed                         (JacobiStatus)
  unsigned long long rotations;   // rotations applied (flop count)  (JacobiStatus)
  unsigned count;
  unsigned gen;
  unsigned off_bits[3];   // float bits of the largest relative off-diagonal of a sweep
  unsigned pad[7];
  // followed by one round counter per column block (jacobi_wp4_kernel)
};
static_assert(sizeof(JacobiCtl) == 64, "control block layout");
static_assert(offsetof(JacobiCtl, rotations) == offsetof(JacobiStatus, rotations), "status prefix");

__device__ __forceinline__ unsigned* block_rounds(JacobiCtl* c) { return reinterpret_cast<unsigned*>(c + 1); }

// Iteration limit of every spin wait in the Jacobi kernels (the grid barrier
// and the per-block round counters): 20M polls of ~64 ns, about 1.3 s.  One
// copy per device; dmrgc_set_wait_limit changes it (tests make a wait run
// out with a limit of a few polls, which ends the launch with ETIMEOUT).
constexpr unsigned long long kSpinLimitDefault = 20000000ull;
__device__ unsigned long long g_spin_limit = kSpinLimitDefault;

__device__ __forceinline__ bool grid_barrier(JacobiCtl* c, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &c->gen;
    volatile int* verr = &c->err;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&c->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&c->count, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      unsigned long long it = 0;
      const unsigned long long lim = g_spin_limit;
      while (*vgen == g) {
        if (it > 4096) __nanosleep(64);
        if (*verr != 0) break;
        if (++it > lim) {
          atomicExch(&c->err, (int)DMRGC_ETIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&c->err) == 0;
}

// Wait (thread 0 polls, bounded) until blocks I and J have each completed
// `need` rounds; then the CTA may read their columns.  false: error or timeout.
__device__ __forceinline__ bool wait_rounds(JacobiCtl* c, const unsigned* done, int I, int J, unsigned need) {
  if (threadIdx.x == 0) {
    volatile const unsigned* di = done + I;
    volatile const unsigned* dj = done + J;
    volatile int* verr = &c->err;
    unsigned long long it = 0;
    const unsigned long long lim = g_spin_limit;
    while (*di < need || *dj < need) {
      if (it > 4096) __nanosleep(64);
      if (*verr != 0) break;
      if (++it > lim) {
        atomicExch(&c->err, (int)DMRGC_ETIMEOUT);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&c->err) == 0;
}

// After the CTA stored blocks I and J: mark them `rounds` complete.
__device__ __forceinline__ void publish_rounds(unsigned* done, int I, int J, unsigned rounds) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(done + I, rounds);
    atomicExch(done + J, rounds);
  }
  __syncthreads();
}

__device__ __forceinline__ void round_robin_pair(int r, int p, int np, int& a, int& b) {
  // circle method: player 0 fixed, players 1..np-1 rotate
  auto idx = [&](int x) { return (x + r) % (np - 1) + 1; };
  if (p == 0) { a = 0; b = idx(0); }
  else { a = idx(p); b = idx(np - 1 - p); }
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__global__ void __launch_bounds__(128) jacobi_kernel(typename cplx<R>::T* __restrict__ G, int m,
                                                     int n, int np, R tol, int max_sweeps,
                                                     const double* __restrict__ fro2, R zero_rel,
                                                     JacobiCtl* ctl) {
  using C2 = typename cplx<R>::T;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned nb = gridDim.x;
  // columns whose norm is below zero_rel * |G|_F are numerically zero: their
  // direction is rounding noise, so they are never rotated (and are dropped
  // later by the truncation cutoff, which lies above zero_rel)
  const double fz = (double)zero_rel * (double)zero_rel * (*fro2);
  const R tiny = (R)fmax(fz, (sizeof(R) == 8) ? 1e-280 : 1e-30);
  int sweep = 0;
  unsigned long long rot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float local_off = 0.f;
    for (int r = 0; r < np - 1; ++r) {
      for (int p = warp; p < np / 2; p += nwarps) {
        int a, b;
        round_robin_pair(r, p, np, a, b);
        if (a >= n || b >= n) continue;
        C2* u = G + (long long)a * m;
        C2* v = G + (long long)b * m;
        R al = 0, be = 0, gr = 0, gi = 0;
        for (int i = lane; i < m; i += 32) {
          const C2 x = u[i], y = v[i];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          gr += x.x * y.x + x.y * y.y;   // conj(x) * y
          gi += x.x * y.y - x.y * y.x;
        }
        al = warp_sum(al); be = warp_sum(be); gr = warp_sum(gr); gi = warp_sum(gi);
        const R gabs = sqrt(gr * gr + gi * gi);
        if (al <= tiny || be <= tiny || gabs <= tiny) continue;
        const R rel = gabs / sqrt(al * be);
        if (!(rel > tol)) continue;
        local_off = fmaxf(local_off, (float)rel);
        ++rot;
        // phase e^{-i phi} of gamma, real rotation on (u, e^{-i phi} v)
        const R er = gr / gabs, ei = -gi / gabs;
        const R zeta = (al - be) / (2 * gabs);
        const R sg = zeta >= 0 ? R(1) : R(-1);
        const R t = -sg / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
        const R c = R(1) / sqrt(R(1) + t * t);
        const R s = c * t;
        const R mst = -s * (s / (R(1) + c));   // c - 1, accurate when c rounds to 1
        // u' = c u - s e^{-i phi} v ;  v' = s u + c e^{-i phi} v, as corrections
        // of the columns themselves (see the column-pair kernel below)
        for (int i = lane; i < m; i += 32) {
          const C2 x = u[i], y = v[i];
          const C2 ye{y.x * er - y.y * ei, y.x * ei + y.y * er};
          u[i] = C2{x.x + (mst * x.x - s * ye.x), x.y + (mst * x.y - s * ye.y)};
          v[i] = C2{ye.x + (s * x.x + mst * ye.x), ye.y + (s * x.y + mst * ye.y)};
        }
      }
      if (lane == 0 && local_off > 0.f)
        atomicMax(&ctl->off_bits[sweep & 1], __float_as_uint(local_off));
      local_off = 0.f;
      if (!grid_barrier(ctl, nb)) {
        if (lane == 0 && rot) atomicAdd(&ctl->rotations, rot);
        return;
      }
      if (r == 0 && blockIdx.x == 0 && threadIdx.x == 0) ctl->off_bits[(sweep + 1) & 1] = 0u;
    }
    const float off = __uint_as_float(*((volatile unsigned*)&ctl->off_bits[sweep & 1]));
    if (!(off > (float)tol)) { ++sweep; break; }
  }
  if (lane == 0 && rot) atomicAdd(&ctl->rotations, rot);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->sweeps = sweep;
    const float off = __uint_as_float(ctl->off_bits[(sweep - 1) & 1]);
    if (sweep >= max_sweeps && off > (float)tol && ctl->err == 0) ctl->err = (int)DMRGC_ENOCONV;
  }
}

// Register-resident variant for m <= 128*E: one CTA (128 threads) per column
// pair, each thread holding E elements of both columns, so a pair costs one
// load, one block reduction and one store.  Same rotation and stopping rule.
template <typename R, int E>
__global__ void __launch_bounds__(128) jacobi_reg_kernel(typename cplx<R>::T* __restrict__ G, int m,
                                                         int n, int np, R tol, int max_sweeps,
                                                         const double* __restrict__ fro2, R zero_rel,
                                                         JacobiCtl* ctl) {
  using C2 = typename cplx<R>::T;
  __shared__ R red[2][4][4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned nb = gridDim.x;
  const double fz = (double)zero_rel * (double)zero_rel * (*fro2);
  const R tiny = (R)fmax(fz, (sizeof(R) == 8) ? 1e-280 : 1e-30);
  int sweep = 0, buf = 0;
  unsigned long long rot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float local_off = 0.f;
    for (int r = 0; r < np - 1; ++r) {
      for (int p = blockIdx.x; p < np / 2; p += gridDim.x) {
        int a, b;
        round_robin_pair(r, p, np, a, b);
        if (a >= n || b >= n) continue;
        C2* u = G + (long long)a * m;
        C2* v = G + (long long)b * m;
        C2 x[E], y[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = tid + e * 128;
          if (i < m) { x[e] = u[i]; y[e] = v[i]; }
          else { x[e] = C2{0, 0}; y[e] = C2{0, 0}; }
        }
        R al = 0, be = 0, gr = 0, gi = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          al += x[e].x * x[e].x + x[e].y * x[e].y;
          be += y[e].x * y[e].x + y[e].y * y[e].y;
          gr += x[e].x * y[e].x + x[e].y * y[e].y;
          gi += x[e].x * y[e].y - x[e].y * y[e].x;
        }
        al = warp_sum(al); be = warp_sum(be); gr = warp_sum(gr); gi = warp_sum(gi);
        if (lane == 0) { red[buf][wid][0] = al; red[buf][wid][1] = be; red[buf][wid][2] = gr; red[buf][wid][3] = gi; }
        __syncthreads();
        al = red[buf][0][0] + red[buf][1][0] + red[buf][2][0] + red[buf][3][0];
        be = red[buf][0][1] + red[buf][1][1] + red[buf][2][1] + red[buf][3][1];
        gr = red[buf][0][2] + red[buf][1][2] + red[buf][2][2] + red[buf][3][2];
        gi = red[buf][0][3] + red[buf][1][3] + red[buf][2][3] + red[buf][3][3];
        buf ^= 1;   // the next pair reduces into the other buffer: no second barrier
        const R gabs = sqrt(gr * gr + gi * gi);
        if (al <= tiny || be <= tiny || gabs <= tiny) continue;
        const R rel = gabs / sqrt(al * be);
        if (!(rel > tol)) continue;
        local_off = fmaxf(local_off, (float)rel);
        if (tid == 0) ++rot;
        const R er = gr / gabs, ei = -gi / gabs;
        const R zeta = (al - be) / (2 * gabs);
        const R sg = zeta >= 0 ? R(1) : R(-1);
        const R t = -sg / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
        const R c = R(1) / sqrt(R(1) + t * t);
        const R sn = c * t;
        const R mst = -sn * (sn / (R(1) + c));   // c - 1, accurate when c rounds to 1
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = tid + e * 128;
          if (i < m) {
            const C2 ye{y[e].x * er - y[e].y * ei, y[e].x * ei + y[e].y * er};
            u[i] = C2{x[e].x + (mst * x[e].x - sn * ye.x), x[e].y + (mst * x[e].y - sn * ye.y)};
            v[i] = C2{ye.x + (sn * x[e].x + mst * ye.x), ye.y + (sn * x[e].y + mst * ye.y)};
          }
        }
      }
      if (tid == 0 && local_off > 0.f) atomicMax(&ctl->off_bits[sweep & 1], __float_as_uint(local_off));
      local_off = 0.f;
      if (!grid_barrier(ctl, nb)) {
        if (tid == 0 && rot) atomicAdd(&ctl->rotations, rot);
        return;
      }
      if (r == 0 && blockIdx.x == 0 && tid == 0) ctl->off_bits[(sweep + 1) & 1] = 0u;
    }
    const float off = __uint_as_float(*((volatile unsigned*)&ctl->off_bits[sweep & 1]));
    if (!(off > (float)tol)) { ++sweep; break; }
  }
  if (tid == 0 && rot) atomicAdd(&ctl->rotations, rot);
  if (blockIdx.x == 0 && tid == 0) {
    ctl->sweeps = sweep;
    const float off = __uint_as_float(ctl->off_bits[(sweep - 1) & 1]);
    if (sweep >= max_sweeps && off > (float)tol && ctl->err == 0) ctl->err = (int)DMRGC_ENOCONV;
  }
}

// Warp-pair variant with 4-column blocks (complex64, m <= 32*E): 8 warps per
// CTA, so that 128 CTAs cover n = 1024 (the 8-column version left most SMs
// idle); both columns of a pair live in registers, the column exchange is
// double buffered (one CTA barrier per sub-round), and each warp runs the code
// of its role without per-element selects.
template <int SUB>
__device__ __forceinline__ int wp4_partner(int w) {
  if (SUB < 3) {   // intra-block: (0,1)(2,3) / (0,2)(1,3) / (0,3)(1,2) in both blocks
    const int blk = w >> 2, q = w & 3;
    const int pr = SUB == 0 ? (q ^ 1) : SUB == 1 ? (q ^ 2) : (3 - q);
    return blk * 4 + pr;
  }
  const int s = SUB - 3;   // cross: slot q of block I with slot (q + s) mod 4 of block J
  return w < 4 ? 4 + ((w + s) & 3) : ((w - 4 - s) & 3);
}

// Sums of four values over the warp, the same in every lane: reduce-scatter
// over lane bits 4 and 3 (lane L keeps one of the four), sums over bits 2..0,
// then each value is read from a lane that holds it (10 shuffles, not 20).
__device__ __forceinline__ void warp_sum4(float& a, float& b, float& c, float& d) {
  const int lane = threadIdx.x & 31;
  const bool u4 = lane & 16, u3 = lane & 8;
  float k0 = u4 ? c : a, k1 = u4 ? d : b;
  const float s0 = u4 ? a : c, s1 = u4 ? b : d;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  float k = u3 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, u3 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  a = __shfl_sync(0xffffffffu, k, 0);
  b = __shfl_sync(0xffffffffu, k, 8);
  c = __shfl_sync(0xffffffffu, k, 16);
  d = __shfl_sync(0xffffffffu, k, 24);
}

template <bool FIRST, int E>
__device__ __forceinline__ void wp4_pair(float2 (&x)[E], const float2 (&y)[E], bool ok, float tiny, float tol,
                                         float& local_off, unsigned long long& rot) {
  // (u, v) = (first, second) column: the same arithmetic in both warps of the
  // pair.  Packed FP32x2 FMAs: nu = (sum ux^2, sum uy^2), nv likewise,
  // p1 = (sum ux vx, sum uy vy), p2 = (sum ux vy, sum uy vx).
  float2 nu{0.f, 0.f}, nv{0.f, 0.f}, p1{0.f, 0.f}, p2{0.f, 0.f};
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const float2 u = FIRST ? x[e] : y[e];
    const float2 v = FIRST ? y[e] : x[e];
    nu = __ffma2_rn(u, u, nu);
    nv = __ffma2_rn(v, v, nv);
    p1 = __ffma2_rn(u, v, p1);
    p2 = __ffma2_rn(u, make_float2(v.y, v.x), p2);
  }
  float al = nu.x + nu.y, be = nv.x + nv.y, gr = p1.x + p1.y, gi = p2.x - p2.y;
  warp_sum4(al, be, gr, gi);
  const float gabs = sqrtf(gr * gr + gi * gi);
  if (!ok || !(al > tiny) || !(be > tiny) || !(gabs > tiny)) return;
  const float rel = gabs / sqrtf(al * be);
  if (!(rel > tol)) return;
  if (FIRST) {
    local_off = fmaxf(local_off, rel);
    if ((threadIdx.x & 31) == 0) ++rot;
  }
  const float er = gr / gabs, ei = -gi / gabs;
  const float zeta = (al - be) / (2.f * gabs);
  const float sg = zeta >= 0.f ? 1.f : -1.f;
  const float t = -sg / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = 1.f / sqrtf(1.f + t * t);
  const float sn = c * t;
  // first: u' = c u - s e^{-i phi} v;  second: v' = s u + c e^{-i phi} v,
  // applied as corrections of the column itself with tau = s / (1 + c), since
  // c = 1 - s tau:  u' = u + (-s tau u - s e v),  v' = e v + (-s tau e v + s u)
  // (e = e^{-i phi}).  For small rotations c rounds to 1 while c^2 + s^2 = 1 + t^2
  // does not; the plain form then grows every column by t^2 / 2 per rotation,
  // a bias that thousands of late-sweep rotations turn into ~1e-4 of s_1.
  const float mst = -sn * (sn / (1.f + c));
  const float2 MST{mst, mst};
  if (FIRST) {
    const float br = -sn * er, bi = -sn * ei;
    const float2 BR{br, br}, BI{-bi, bi};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float2 u = x[e], v = y[e];
      const float2 d = __ffma2_rn(MST, u, __ffma2_rn(BR, v, __fmul2_rn(BI, make_float2(v.y, v.x))));
      x[e] = make_float2(u.x + d.x, u.y + d.y);
    }
  } else {
    const float2 ER{er, er}, EI{-ei, ei}, SN{sn, sn};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float2 u = y[e], v = x[e];
      const float2 ev = __ffma2_rn(ER, v, __fmul2_rn(EI, make_float2(v.y, v.x)));
      const float2 d = __ffma2_rn(MST, ev, __fmul2_rn(SN, u));
      x[e] = make_float2(ev.x + d.x, ev.y + d.y);
    }
  }
}

template <int SUB, int E, int VEC>
__device__ __forceinline__ void wp4_subround(float2 (&x)[E], bool valid_me, const bool* valid_all, float2* sbuf,
                                             int m, int& buf, float tiny, float tol, float& local_off,
                                             unsigned long long& rot) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = wp4_partner<SUB>(w);
  // columns are padded to 32 E rows in shared memory (rows >= m hold zeros in
  // x and rotate as zeros), so the exchange needs no bounds checks
  float2* base = sbuf + (long long)buf * 8 * 32 * E;
  float2* mine = base + (long long)w * 32 * E;
  const float2* theirs = base + (long long)p * 32 * E;
  float2 y[E];
  if constexpr (VEC == 2) {   // 16-byte accesses: elements 2h, 2h+1 of a lane side by side
    float4* mine4 = reinterpret_cast<float4*>(mine);
    const float4* theirs4 = reinterpret_cast<const float4*>(theirs);
#pragma unroll
    for (int h = 0; h < E / 2; ++h) mine4[lane + 32 * h] = make_float4(x[2 * h].x, x[2 * h].y, x[2 * h + 1].x, x[2 * h + 1].y);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < E / 2; ++h) {
      const float4 v = theirs4[lane + 32 * h];
      y[2 * h] = make_float2(v.x, v.y);
      y[2 * h + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) mine[lane + 32 * e] = x[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) y[e] = theirs[lane + 32 * e];
  }
  buf ^= 1;   // the next sub-round writes the other buffer: no second barrier
  const bool ok = valid_me && valid_all[p];
  if (w < p) wp4_pair<true, E>(x, y, ok, tiny, tol, local_off, rot);
  else wp4_pair<false, E>(x, y, ok, tiny, tol, local_off, rot);
}

// VEC = 2 (m even): a lane holds rows 64 h + 2 lane and 64 h + 2 lane + 1 as
// elements 2h, 2h+1 and moves them with 16-byte loads and stores; VEC = 1: row
// lane + 32 e as element e.
template <int E, int VEC>
__global__ void __launch_bounds__(256, 1) jacobi_wp4_kernel(float2* __restrict__ G, int m, int n, int nblk,
                                                            float tol, int max_sweeps,
                                                            const double* __restrict__ fro2, float zero_rel,
                                                            JacobiCtl* ctl) {
  extern __shared__ float2 sbuf[];          // 2 buffers x 8 columns x 32 E
  __shared__ bool valid_all[8];
  __shared__ float off_w[8];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const unsigned nb = gridDim.x;
  const double fz = (double)zero_rel * (double)zero_rel * (*fro2);
  const float tiny = (float)fmax(fz, 1e-30);
  // stop after a sweep whose largest rotation is below conv: the columns are
  // then orthogonal to about conv^2 (the sweep's rotations move the pairs
  // rotated earlier in it only at second order)
  const float conv = fmaxf(tol, 2e-3f);
  unsigned* done = block_rounds(ctl);      // rounds completed per column block
  int sweep = 0, buf = 0;
  unsigned long long rot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // slot of the sweep after next: every CTA read it at the end of sweep - 2,
    // before passing the barrier that ended sweep - 1
    if (blockIdx.x == 0 && tid == 0) ctl->off_bits[(sweep + 1) % 3] = 0u;
    float local_off = 0.f;
    for (int r = 0; r < nblk - 1; ++r) {
      const unsigned need = (unsigned)sweep * (unsigned)(nblk - 1) + (unsigned)r;
      for (int pb = blockIdx.x; pb < nblk / 2; pb += gridDim.x) {
        int I, J;
        round_robin_pair(r, pb, nblk, I, J);
        // the two blocks must have finished the previous round (point-to-point
        // instead of a grid barrier: no CTA waits for the slowest one)
        if (!wait_rounds(ctl, done, I, J, need)) {
          if (lane == 0 && rot) atomicAdd(&ctl->rotations, rot);
          return;
        }
        const int col = (w < 4 ? I : J) * 4 + (w & 3);
        const bool valid = col < n;
        if (lane == 0) valid_all[w] = valid;
        float2 x[E];
        float2* gcol = G + (long long)col * m;
        if constexpr (VEC == 2) {
#pragma unroll
          for (int h = 0; h < E / 2; ++h) {
            const int i = 64 * h + 2 * lane;   // m even: rows i, i + 1 both in range or both out
            const float4 v = (valid && i < m) ? *reinterpret_cast<const float4*>(gcol + i)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
            x[2 * h] = make_float2(v.x, v.y);
            x[2 * h + 1] = make_float2(v.z, v.w);
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int i = lane + 32 * e;
            x[e] = (valid && i < m) ? gcol[i] : float2{0.f, 0.f};
          }
        }
        if (r == 0) {
          wp4_subround<0, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
          wp4_subround<1, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
          wp4_subround<2, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
        }
        wp4_subround<3, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
        wp4_subround<4, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
        wp4_subround<5, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
        wp4_subround<6, E, VEC>(x, valid, valid_all, sbuf, m, buf, tiny, tol, local_off, rot);
        if (valid) {
          if constexpr (VEC == 2) {
#pragma unroll
            for (int h = 0; h < E / 2; ++h) {
              const int i = 64 * h + 2 * lane;
              if (i < m)
                *reinterpret_cast<float4*>(gcol + i) = make_float4(x[2 * h].x, x[2 * h].y, x[2 * h + 1].x, x[2 * h + 1].y);
            }
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int i = lane + 32 * e;
              if (i < m) gcol[i] = x[e];
            }
          }
        }
        publish_rounds(done, I, J, need + 1);   // ends with __syncthreads
      }
    }
    if (lane == 0) off_w[w] = local_off;
    __syncthreads();
    if (tid == 0) {
      float mx = 0.f;
      for (int i = 0; i < 8; ++i) mx = fmaxf(mx, off_w[i]);
      if (mx > 0.f) atomicMax(&ctl->off_bits[sweep % 3], __float_as_uint(mx));
    }
    if (!grid_barrier(ctl, nb)) {
      if (lane == 0 && rot) atomicAdd(&ctl->rotations, rot);
      return;
    }
    const float off = __uint_as_float(*((volatile unsigned*)&ctl->off_bits[sweep % 3]));
    if (!(off > conv)) { ++sweep; break; }
  }
  if (lane == 0 && rot) atomicAdd(&ctl->rotations, rot);
  if (blockIdx.x == 0 && tid == 0) {
    ctl->sweeps = sweep;
    const float off = __uint_as_float(ctl->off_bits[(sweep - 1) % 3]);
    if (sweep >= max_sweeps && off > conv && ctl->err == 0) ctl->err = (int)DMRGC_ENOCONV;
  }
}

// ---- block Jacobi on 8 x 8 Gram matrices (complex64, m <= 512 RPT)
//
// One CTA per pair of 4-column blocks (8 columns), 512 threads; thread t holds
// rows t + 512 k (k < RPT) of the 8 columns in registers, so rows are spread
// over 16 warps and no column crosses a warp boundary in the arithmetic.  Per
// round:
//  1. the 8 x 8 Gram matrix X^+ X of the block pair (8 real diagonal and 28
//     complex entries, 64 floats per thread), reduced in the warp by a
//     reduce-scatter butterfly (64 -> 2 values per lane) and over the warps
//     through shared memory;
//  2. warp 0 runs one cyclic Jacobi sweep on the Gram (7 steps of 4 disjoint
//     pairs, the round-robin order on 8 indices).  Each pair uses the column
//     kernels' rotation (same zero level, threshold and formulas); the
//     rotation is applied to the Gram on both sides and accumulated in V;
//  3. every thread replaces its rows by X V.
// Every pair of columns is rotated once per sweep, as in the column kernels.  The sweep ends, like the column
// kernels, when its largest rotated |gamma| / sqrt(alpha beta) is below the
// threshold.

// the e-th pair (i < j) of 8 indices in row order: (0,1), (0,2), ..., (6,7)
__device__ __forceinline__ void pair_index(int e, int& i, int& j) {
  i = 0;
  int rowlen = 7;
  while (e >= rowlen) { e -= rowlen; ++i; --rowlen; }
  j = i + 1 + e;
}

// Steps of the inner sweep on 8 indices (0-3: block I, 4-7: block J).  The
// four cross steps pair every column of I with every column of J; the three
// intra steps pair the columns inside each block (run in the first round of a
// sweep only, as in the column kernels).  Entry: partner * 8 + pair * 2 + first.
__constant__ unsigned char kGramStep[7][8] = {
    // cross: (i, 4 + (i + s) % 4)
    {4 * 8 + 0 * 2 + 1, 5 * 8 + 1 * 2 + 1, 6 * 8 + 2 * 2 + 1, 7 * 8 + 3 * 2 + 1,
     0 * 8 + 0 * 2 + 0, 1 * 8 + 1 * 2 + 0, 2 * 8 + 2 * 2 + 0, 3 * 8 + 3 * 2 + 0},
    {5 * 8 + 0 * 2 + 1, 6 * 8 + 1 * 2 + 1, 7 * 8 + 2 * 2 + 1, 4 * 8 + 3 * 2 + 1,
     3 * 8 + 3 * 2 + 0, 0 * 8 + 0 * 2 + 0, 1 * 8 + 1 * 2 + 0, 2 * 8 + 2 * 2 + 0},
    {6 * 8 + 0 * 2 + 1, 7 * 8 + 1 * 2 + 1, 4 * 8 + 2 * 2 + 1, 5 * 8 + 3 * 2 + 1,
     2 * 8 + 2 * 2 + 0, 3 * 8 + 3 * 2 + 0, 0 * 8 + 0 * 2 + 0, 1 * 8 + 1 * 2 + 0},
    {7 * 8 + 0 * 2 + 1, 4 * 8 + 1 * 2 + 1, 5 * 8 + 2 * 2 + 1, 6 * 8 + 3 * 2 + 1,
     1 * 8 + 1 * 2 + 0, 2 * 8 + 2 * 2 + 0, 3 * 8 + 3 * 2 + 0, 0 * 8 + 0 * 2 + 0},
    // intra: (0,1)(2,3)(4,5)(6,7); (0,2)(1,3)(4,6)(5,7); (0,3)(1,2)(4,7)(5,6)
    {1 * 8 + 0 * 2 + 1, 0 * 8 + 0 * 2 + 0, 3 * 8 + 1 * 2 + 1, 2 * 8 + 1 * 2 + 0,
     5 * 8 + 2 * 2 + 1, 4 * 8 + 2 * 2 + 0, 7 * 8 + 3 * 2 + 1, 6 * 8 + 3 * 2 + 0},
    {2 * 8 + 0 * 2 + 1, 3 * 8 + 1 * 2 + 1, 0 * 8 + 0 * 2 + 0, 1 * 8 + 1 * 2 + 0,
     6 * 8 + 2 * 2 + 1, 7 * 8 + 3 * 2 + 1, 4 * 8 + 2 * 2 + 0, 5 * 8 + 3 * 2 + 0},
    {3 * 8 + 0 * 2 + 1, 2 * 8 + 1 * 2 + 1, 1 * 8 + 1 * 2 + 0, 0 * 8 + 0 * 2 + 0,
     7 * 8 + 2 * 2 + 1, 6 * 8 + 3 * 2 + 1, 5 * 8 + 3 * 2 + 0, 4 * 8 + 2 * 2 + 0}};

__device__ __forceinline__ void step_role(int s, int x, int& partner, int& pair, bool& first) {
  const int c = kGramStep[s][x];
  partner = c >> 3;
  pair = (c >> 1) & 3;
  first = c & 1;
}

// R_{x x} (self) and R_{partner, x} (other) of the 2x2 rotation with
// parameters (c, s, e^{-i phi} = er + i ei):  first: c, -s e^{-i phi};
// second: c e^{-i phi}, s.
__device__ __forceinline__ void rot_coeffs(const float4 r, bool first, float2& self, float2& other) {
  if (first) { self = make_float2(r.x, 0.f); other = make_float2(-r.y * r.z, -r.y * r.w); }
  else { self = make_float2(r.x * r.z, r.x * r.w); other = make_float2(r.y, 0.f); }
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmulcf(float2 a, float2 b) {   // conj(a) b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

template <int RPT>
__global__ void __launch_bounds__(512, 1) jacobi_gram_kernel(float2* __restrict__ G, int m, int n, int nblk,
                                                             float tol, int max_sweeps,
                                                             const double* __restrict__ fro2, float zero_rel,
                                                             JacobiCtl* ctl) {
  __shared__ float part[16][64];
  __shared__ float2 gm[64];
  __shared__ float2 vm[64];
  __shared__ float4 rot[4];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const unsigned nb = gridDim.x;
  const double fz = (double)zero_rel * (double)zero_rel * (*fro2);
  const float tiny = (float)fmax(fz, 1e-30);
  const float conv = fmaxf(tol, 2e-4f);
  int sweep = 0;
  unsigned long long rotations = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float local_off = 0.f;
    for (int r = 0; r < nblk - 1; ++r) {
      for (int pb = blockIdx.x; pb < nblk / 2; pb += gridDim.x) {
        int I, J;
        round_robin_pair(r, pb, nblk, I, J);
        int col[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int cj = (j < 4 ? I * 4 + j : J * 4 + j - 4);
          col[j] = cj < n ? cj : -1;
        }
        // 1. Gram partials, 64 floats: |x_i|^2 (i < 8), then (re, im) of
        // conj(x_i) x_j for the 28 pairs i < j; one row slot at a time
        float v[64];
#pragma unroll
        for (int h = 0; h < 64; ++h) v[h] = 0.f;
#pragma unroll 1
        for (int k = 0; k < RPT; ++k) {
          const int row = tid + 512 * k;
          float2 x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            x[j] = (col[j] >= 0 && row < m) ? G[(long long)col[j] * m + row] : float2{0.f, 0.f};
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = fmaf(x[i].x, x[i].x, fmaf(x[i].y, x[i].y, v[i]));
          int e = 8;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = i + 1; j < 8; ++j) {
              const float2 a = x[i], b = x[j];
              v[e] = fmaf(a.x, b.x, fmaf(a.y, b.y, v[e]));
              v[e + 1] = fmaf(a.x, b.y, fmaf(-a.y, b.x, v[e + 1]));
              e += 2;
            }
          }
        }
        // reduce-scatter over the five lane bits: 64 -> 2 values per lane;
        // lane L ends with values 2 * (L reversed-bit-order position) .. + 1
#pragma unroll
        for (int bit = 4, half = 32; bit >= 0; --bit, half >>= 1) {
          const bool up = (lane >> bit) & 1;
#pragma unroll
          for (int h = 0; h < half; ++h) {
            const float send = up ? v[h] : v[half + h];
            const float keep = up ? v[half + h] : v[h];
            v[h] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << bit);
          }
        }
        {
          const int base = ((lane >> 4) & 1) * 32 + ((lane >> 3) & 1) * 16 + ((lane >> 2) & 1) * 8 +
                           ((lane >> 1) & 1) * 4 + (lane & 1) * 2;
          part[w][base] = v[0];
          part[w][base + 1] = v[1];
        }
        __syncthreads();
        if (tid < 64) {
          float sum = 0.f;
#pragma unroll
          for (int ww = 0; ww < 16; ++ww) sum += part[ww][tid];
          float* g = reinterpret_cast<float*>(gm);
          if (tid < 8) {
            g[2 * (tid * 9)] = sum;
            g[2 * (tid * 9) + 1] = 0.f;
          } else {
            int i, j;
            pair_index((tid - 8) >> 1, i, j);
            if (tid & 1) {
              g[2 * (i * 8 + j) + 1] = sum;
              g[2 * (j * 8 + i) + 1] = -sum;
            } else {
              g[2 * (i * 8 + j)] = sum;
              g[2 * (j * 8 + i)] = sum;
            }
          }
        } else if (tid >= 128 && tid < 192) {
          const int e = tid - 128;
          vm[e] = make_float2((e % 9) == 0 ? 1.f : 0.f, 0.f);
        }
        __syncthreads();
        // 2. one cyclic Jacobi sweep on the Gram (warp 0)
        if (w == 0) {
          for (int st = (r == 0 ? 0 : 3); st < 7; ++st) {
            const int sx = st < 3 ? st + 4 : st - 3;   // intra steps first in round 0
            if (lane < 4) {
              // pair `lane` of step sx: its first index p and partner q
              int p = 0;
#pragma unroll
              for (int x = 0; x < 8; ++x) {
                const int cx = kGramStep[sx][x];
                if ((cx & 1) && ((cx >> 1) & 3) == lane) p = x;
              }
              const int q = kGramStep[sx][p] >> 3;
              const float al = gm[p * 9].x, be = gm[q * 9].x;
              const float2 g = gm[p * 8 + q];
              const float gabs = sqrtf(g.x * g.x + g.y * g.y);
              float4 rr = make_float4(1.f, 0.f, 1.f, 0.f);
              if (al > tiny && be > tiny && gabs > tiny) {
                const float rel = gabs / sqrtf(al * be);
                if (rel > tol) {
                  local_off = fmaxf(local_off, rel);
                  ++rotations;
                  const float zeta = (al - be) / (2.f * gabs);
                  const float sg = zeta >= 0.f ? 1.f : -1.f;
                  const float t = -sg / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                  const float c = 1.f / sqrtf(1.f + t * t);
                  rr = make_float4(c, c * t, g.x / gabs, -g.y / gabs);
                }
              }
              rot[lane] = rr;
            }
            __syncwarp();
            float2 ng[2], nv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int e = lane + 32 * u, i = e >> 3, j = e & 7;
              int pi, pj, ki, kj;
              bool fi, fj;
              step_role(sx, i, pi, ki, fi);
              step_role(sx, j, pj, kj, fj);
              float2 ai, bi, aj, bj;
              rot_coeffs(rot[ki], fi, ai, bi);
              rot_coeffs(rot[kj], fj, aj, bj);
              // G'_ij = conj(A_i) (G_ij A_j + G_i,pj B_j) + conj(B_i) (G_pi,j A_j + G_pi,pj B_j)
              const float2 t1 = make_float2(cmulf(gm[i * 8 + j], aj).x + cmulf(gm[i * 8 + pj], bj).x,
                                            cmulf(gm[i * 8 + j], aj).y + cmulf(gm[i * 8 + pj], bj).y);
              const float2 t2 = make_float2(cmulf(gm[pi * 8 + j], aj).x + cmulf(gm[pi * 8 + pj], bj).x,
                                            cmulf(gm[pi * 8 + j], aj).y + cmulf(gm[pi * 8 + pj], bj).y);
              const float2 u1 = cmulcf(ai, t1), u2 = cmulcf(bi, t2);
              ng[u] = make_float2(u1.x + u2.x, u1.y + u2.y);
              const float2 v1 = cmulf(vm[i * 8 + j], aj), v2 = cmulf(vm[i * 8 + pj], bj);
              nv[u] = make_float2(v1.x + v2.x, v1.y + v2.y);
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              gm[lane + 32 * u] = ng[u];
              vm[lane + 32 * u] = nv[u];
            }
            __syncwarp();
          }
        }
        __syncthreads();
        // 3. X <- X V (rows re-read: they are in L1)
#pragma unroll 1
        for (int k = 0; k < RPT; ++k) {
          const int row = tid + 512 * k;
          if (row >= m) break;
          float2 x[8], y[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            x[j] = col[j] >= 0 ? G[(long long)col[j] * m + row] : float2{0.f, 0.f};
            y[j] = make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float2 vv = vm[i * 8 + j];
              y[j].x = fmaf(x[i].x, vv.x, fmaf(-x[i].y, vv.y, y[j].x));
              y[j].y = fmaf(x[i].x, vv.y, fmaf(x[i].y, vv.x, y[j].y));
            }
          }
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (col[j] >= 0) G[(long long)col[j] * m + row] = y[j];
        }
        __syncthreads();   // part, gm, vm are reused by the next pair of blocks
      }
      if (w == 0) {
        float mx = local_off;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx > 0.f) atomicMax(&ctl->off_bits[sweep & 1], __float_as_uint(mx));
      }
      local_off = 0.f;
      if (!grid_barrier(ctl, nb)) {
        if (rotations) atomicAdd(&ctl->rotations, rotations);
        return;
      }
      if (r == 0 && blockIdx.x == 0 && tid == 0) ctl->off_bits[(sweep + 1) & 1] = 0u;
    }
    const float off = __uint_as_float(*((volatile unsigned*)&ctl->off_bits[sweep & 1]));
    if (!(off > conv)) { ++sweep; break; }
  }
  if (rotations) atomicAdd(&ctl->rotations, rotations);
  if (blockIdx.x == 0 && tid == 0) {
    ctl->sweeps = sweep;
    const float off = __uint_as_float(ctl->off_bits[(sweep - 1) & 1]);
    if (sweep >= max_sweeps && off > conv && ctl->err == 0) ctl->err = (int)DMRGC_ENOCONV;
  }
}

// ---- column norms, sort, truncation rank

template <typename R>
__global__ void col_norms_kernel(const typename cplx<R>::T* __restrict__ W, int m, int n,
                                 double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= n) return;
  const auto* w = W + (long long)col * m;
  double s = 0;
  for (int i = lane; i < m; i += 32) s += (double)w[i].x * w[i].x + (double)w[i].y * w[i].y;
  s = warp_sum(s);
  if (lane == 0) out[col] = s;
}

// single CTA: bitonic sort of (value, index) descending over the next power of two
__global__ void sort_trunc_kernel(TruncResult* res, double* s, int* perm, const double* nrm2,
                                  int n, int chi, double rel_cut, int squared, double tie_rel,
                                  const double* fro2, double zero_rel) {
  extern __shared__ unsigned char smem[];
  int np = 1;
  while (np < n) np <<= 1;
  double* v = reinterpret_cast<double*>(smem);
  int* ix = reinterpret_cast<int*>(v + np);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    if (i < n) {
      const double q = nrm2[i];   // |W_i|^2
      // singular value of theta: |W_i|; of a Gram matrix: |W_i| = s^2
      v[i] = squared ? sqrt(sqrt(q)) : sqrt(q);
      ix[i] = i;
    } else {
      v[i] = -1.0;
      ix[i] = -1;
    }
  }
  __syncthreads();
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool desc = (i & k) == 0;
          const bool swap = desc ? (v[i] < v[l] || (v[i] == v[l] && ix[i] > ix[l]))
                                 : (v[i] > v[l] || (v[i] == v[l] && ix[i] < ix[l]));
          if (swap) {
            double tv = v[i]; v[i] = v[l]; v[l] = tv;
            int ti = ix[i]; ix[i] = ix[l]; ix[l] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) { s[i] = v[i]; perm[i] = ix[i]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double s1 = v[0];
    // a column the Jacobi kernel treated as zero (norm <= zero_rel |G|_F) is
    // never kept: the cut is the larger of rel_cut * s_1 and that level
    const double zthr = zero_rel * sqrt(*fro2);              // on the column norm
    const double scut = fmax(rel_cut * s1, squared ? sqrt(zthr) : zthr);
    int k = 0, nnz = 0;
    double f = 0, tot = 0;
    for (int i = 0; i < n; ++i) {
      tot += v[i] * v[i];
      if (v[i] > (squared ? sqrt(zthr) : zthr)) ++nnz;
    }
    for (int i = 0; i < n && k < chi; ++i) {
      if (v[i] > scut) ++k; else break;
    }
    // tie rule: never split a (numerically) degenerate multiplet at the cut;
    // a multiplet that reaches s_1 cannot be dropped, the cut then stays at chi
    int ambiguous = 0;
    if (tie_rel > 0 && k >= 1 && k < n && v[k] > scut && v[k - 1] - v[k] <= tie_rel * s1) {
      int kk = k;
      while (kk > 1 && v[kk - 1] - v[kk] <= tie_rel * s1) --kk;
      if (kk == 1 && v[0] - v[1] <= tie_rel * s1) ambiguous = 1;
      else k = kk;
    }
    for (int i = 0; i < k; ++i) f += v[i] * v[i];
    res->status = 0;
    res->pad = ambiguous;
    if (!(s1 > 0.0) || !isfinite(s1)) { res->status = (int)DMRGC_ENUMERIC; k = k > 0 ? k : 1; }
    if (k < 1) k = 1;
    res->k = k;
    res->n = n;
    res->f = f;
    res->norm2 = tot;
    res->nnz = nnz;
    res->by_cut = k < (chi < n ? chi : n) ? 1 : 0;
    res->tail = s1 > 0.0 ? (v[k - 1] / s1) * (v[k - 1] / s1) : 0.0;
  }
}

template <typename R>
__global__ void gather_kernel(const typename cplx<R>::T* __restrict__ W, int m, int k,
                              const double* __restrict__ s, const int* __restrict__ perm, int squared,
                              int mode, typename cplx<R>::T* __restrict__ out) {
  const long long total = (long long)m * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int row, j;
    if (mode == 0) { row = (int)(e / k); j = (int)(e % k); }
    else { j = (int)(e / m); row = (int)(e % m); }
    const double sj = s[j];
    const double scale = squared ? sj * sj : sj;
    const R inv = scale > 0 ? (R)(1.0 / scale) : (R)0;
    auto w = W[(long long)perm[j] * m + row];
    if (mode == 2) w.y = -w.y;
    w.x *= inv;
    w.y *= inv;
    if (mode == 0) out[(long long)row * k + j] = w;
    else out[(long long)j * m + row] = w;
  }
}

}  // namespace

size_t jacobi_ctl_bytes(int n) { return sizeof(JacobiCtl) + sizeof(unsigned) * (size_t)((n + 3) / 4 + 2); }

namespace {

// complex64 Jacobi kernel for m <= 1024: 0 = warp-pair columns (jacobi_wp4),
// 1 = Gram blocks (jacobi_gram); set by dmrgc_set_jacobi_kernel
std::atomic<int> g_jacobi_variant{0};
int jacobi_variant() { return g_jacobi_variant.load(std::memory_order_relaxed); }

template <typename R>
cudaError_t launch_jacobi(void* G, int m, int n, double tol, int max_sweeps, const double* fro2,
                          double zero_rel, JacobiCtl* c, cudaStream_t st) {
  using C2 = typename cplx<R>::T;
  const int np = (n + 1) & ~1;
  const int pairs = np / 2;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* fn;
  int threads = 128, blocks;
  const bool gram = sizeof(R) == 4 && m <= 512 * 2 && n >= 16 && jacobi_variant() == 1;
  const bool wide = !gram && sizeof(R) == 4 && m <= 32 * 32 && n >= 16;
  int nblk = 0;
  size_t dyn_smem = 0;
  if (gram) {
    threads = 512;
    nblk = (n + 3) / 4;
    nblk += nblk & 1;
    fn = (m <= 512) ? (void*)jacobi_gram_kernel<1> : (void*)jacobi_gram_kernel<2>;
    blocks = nblk / 2;
  } else if (wide) {
    threads = 256;
    nblk = (n + 3) / 4;
    nblk += nblk & 1;
    // 16-byte column accesses need an even m (column starts then stay 16-byte aligned)
    const bool v2 = (m % 2) == 0 && (reinterpret_cast<uintptr_t>(G) % 16) == 0;
    if (m <= 32 * 8) fn = v2 ? (void*)jacobi_wp4_kernel<8, 2> : (void*)jacobi_wp4_kernel<8, 1>;
    else if (m <= 32 * 16) fn = v2 ? (void*)jacobi_wp4_kernel<16, 2> : (void*)jacobi_wp4_kernel<16, 1>;
    else fn = v2 ? (void*)jacobi_wp4_kernel<32, 2> : (void*)jacobi_wp4_kernel<32, 1>;
    const int E = m <= 32 * 8 ? 8 : (m <= 32 * 16 ? 16 : 32);
    dyn_smem = (size_t)2 * 8 * 32 * E * sizeof(float2);
    cudaError_t ea = allow_dyn_smem(fn);
    if (ea != cudaSuccess) return ea;
    blocks = nblk / 2;
  } else if (m <= 128 * 16) {
    if (m <= 128 * 2) fn = (void*)jacobi_reg_kernel<R, 2>;
    else if (m <= 128 * 4) fn = (void*)jacobi_reg_kernel<R, 4>;
    else if (m <= 128 * 8) fn = (void*)jacobi_reg_kernel<R, 8>;
    else fn = (void*)jacobi_reg_kernel<R, 16>;
    blocks = pairs;   // one CTA per pair
  } else {
    fn = (void*)jacobi_kernel<R>;
    blocks = (pairs + threads / 32 - 1) / (threads / 32);
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, dyn_smem);
  if (e != cudaSuccess) return e;
  const int cap = sms * per_sm;   // every CTA of a cooperative launch must be resident
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  C2* g = reinterpret_cast<C2*>(G);
  R tl = (R)tol, zr = (R)zero_rel;
  int mm = m, nn = n, npp = (gram || wide) ? nblk : np, ms = max_sweeps;
  void* args[] = {&g, &mm, &nn, &npp, &tl, &ms, (void*)&fro2, &zr, &c};
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, dyn_smem, st);
}

}  // namespace

cudaError_t jacobi_orthogonalize(void* G, int m, int n, bool fp64, double tol, int max_sweeps,
                                 const double* fro2, double zero_rel, void* ctl, cudaStream_t st,
                                 int* launches) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, jacobi_ctl_bytes(n), st);
  if (e != cudaSuccess) return e;
  if (n < 2 || m < 1) return cudaSuccess;
  JacobiCtl* c = reinterpret_cast<JacobiCtl*>(ctl);
  e = fp64 ? launch_jacobi<double>(G, m, n, tol, max_sweeps, fro2, zero_rel, c, st)
           : launch_jacobi<float>(G, m, n, tol, max_sweeps, fro2, zero_rel, c, st);
  if (launches) *launches += 1;
  return e;
}

size_t trunc_bytes(int n) {
  return sizeof(TruncResult) + sizeof(double) * (size_t)n + sizeof(int) * (size_t)n + 64;
}

cudaError_t truncate_columns(const void* W, int m, int n, bool fp64, int chi, double rel_cut,
                             bool squared, double tie_rel, const double* fro2, double zero_rel,
                             void* res, cudaStream_t st) {
  TruncResult* r = reinterpret_cast<TruncResult*>(res);
  double* s = reinterpret_cast<double*>(r + 1);
  int* perm = reinterpret_cast<int*>(s + n);
  // column norms go to the s array first (then sorted in place via shared memory)
  const int threads = 256;
  const int blocks = (n * 32 + threads - 1) / threads;
  if (fp64)
    col_norms_kernel<double><<<blocks, threads, 0, st>>>(reinterpret_cast<const double2*>(W), m, n, s);
  else
    col_norms_kernel<float><<<blocks, threads, 0, st>>>(reinterpret_cast<const float2*>(W), m, n, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int np = 1;
  while (np < n) np <<= 1;
  const size_t sm = (size_t)np * (sizeof(double) + sizeof(int));
  if (sm > 48 * 1024 && (e = allow_dyn_smem((const void*)sort_trunc_kernel)) != cudaSuccess) return e;
  sort_trunc_kernel<<<1, 1024, sm, st>>>(r, s, perm, s, n, chi, rel_cut, squared ? 1 : 0, tie_rel,
                                         fro2, zero_rel);
  return cudaGetLastError();
}

namespace {

// 32 samples of log10(s_mu^2 / sum_{nu<k} s_nu^2) at mu_j = round(j (k-1) / 31)
__global__ void spectrum_summary_kernel(const TruncResult* __restrict__ r, int k, float* __restrict__ out) {
  const double* s = reinterpret_cast<const double*>(r + 1);
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < k; ++i) t += s[i] * s[i];
    tot = t;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < 32) {
    const int mu = k > 1 ? (int)lrint((double)j * (k - 1) / 31.0) : 0;
    const double q = tot > 0 ? s[mu] * s[mu] / tot : 0.0;
    out[j] = (float)(q > 1e-30 ? log10(q) : -30.0);
  }
}

// smallest r with sum_{mu<r} s_mu^2 >= frac * sum_{mu<k} s_mu^2
__global__ void rank_label_kernel(const TruncResult* __restrict__ r, int k, double frac, int* __restrict__ out) {
  const double* s = reinterpret_cast<const double*>(r + 1);
  double tot = 0;
  for (int i = 0; i < k; ++i) tot += s[i] * s[i];
  double run = 0;
  int rr = k;
  for (int i = 0; i < k; ++i) {
    run += s[i] * s[i];
    if (run >= frac * tot) { rr = i + 1; break; }
  }
  *out = rr;
}

}  // namespace

cudaError_t spectrum_summary(const void* res, int k, float* out32, cudaStream_t st) {
  spectrum_summary_kernel<<<1, 32, 0, st>>>(reinterpret_cast<const TruncResult*>(res), k, out32);
  return cudaGetLastError();
}

cudaError_t rank_label(const void* res, int k, double frac, int* out, cudaStream_t st) {
  rank_label_kernel<<<1, 1, 0, st>>>(reinterpret_cast<const TruncResult*>(res), k, frac, out);
  return cudaGetLastError();
}

cudaError_t gather_columns(const void* W, int m, int n_total, int k, const void* res,
                           bool squared, int mode, void* out, bool fp64, cudaStream_t st) {
  const TruncResult* r = reinterpret_cast<const TruncResult*>(res);
  const double* s = reinterpret_cast<const double*>(r + 1);
  const int* perm = reinterpret_cast<const int*>(s + n_total);
  const long long total = (long long)m * k;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  if (fp64)
    gather_kernel<double><<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(W), m, k, s, perm,
                                                  squared ? 1 : 0, mode,
                                                  reinterpret_cast<double2*>(out));
  else
    gather_kernel<float><<<blocks, 256, 0, st>>>(reinterpret_cast<const float2*>(W), m, k, s, perm,
                                                 squared ? 1 : 0, mode,
                                                 reinterpret_cast<float2*>(out));
  return cudaGetLastError();
}

// ---- truncated SVD that allocates nothing
//
// Same Jacobi + truncation + gather path as the sweep, but its scratch (the
// barrier/convergence block, |G|_F^2 and the sorted spectrum with its
// permutation) lives in one file-scope device array instead of memory from
// cudaMalloc.  Host code must not pass the array's name to a kernel (on the
// host it is only a stand-in symbol); it resolves the device address once per
// device with cudaGetSymbolAddress, with that device current.

namespace {

constexpr int kNoAllocMaxCols = 4096;
constexpr size_t kNoAllocBytes = 65536;   // >= 256 + trunc_bytes(kNoAllocMaxCols)
static __device__ __align__(256) unsigned char g_svd_scratch[kNoAllocBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[256] = {};

cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_svd_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = reinterpret_cast<unsigned char*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

}  // namespace dmrgc

extern "C" dmrgc_status dmrgc_svd_noalloc(int precision, int m, int n, void* G, int chi,
                                          double rel_cut, double* s_out, int* k_out, void* U_out,
                                          void* stream) {
  using namespace dmrgc;
  constexpr size_t kCtl = 4352;   // >= jacobi_ctl_bytes(kNoAllocMaxCols) = 4168
  static_assert(kCtl + 256 + sizeof(TruncResult) + (sizeof(double) + sizeof(int)) * kNoAllocMaxCols + 64 <=
                    kNoAllocBytes,
                "scratch array too small");
  if (precision < 0 || precision > 3 || m < 1 || m > (1 << 20) || n < 2 || n > kNoAllocMaxCols ||
      chi < 1 || !G || !s_out || !k_out || !U_out || !(rel_cut >= 0.0))
    return DMRGC_EINVAL;
  const bool fp64 = precision == DMRGC_FP64;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return DMRGC_ECUDA;
  if (jacobi_ctl_bytes(n) > kCtl) return DMRGC_EINVAL;
  void* ctl = base;                                   // control block, cleared by the Jacobi launcher
  double* fro2 = reinterpret_cast<double*>(base + kCtl);  // cleared by sum_abs2
  void* res = base + kCtl + 256;                      // TruncResult, s[n], perm[n]: written in full
  const double eps = fp64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
  const double tol = 8.0 * eps * std::sqrt((double)m);
  const double zero_rel = fp64 ? 1e-13 : 1e-5;
  int launches = 0;
  if (sum_abs2(G, (long long)m * n, fp64, fro2, st) != cudaSuccess) return DMRGC_ECUDA;
  if (jacobi_orthogonalize(G, m, n, fp64, tol, 40, fro2, zero_rel, ctl, st, &launches) != cudaSuccess)
    return DMRGC_ECUDA;
  if (truncate_columns(G, m, n, fp64, chi, rel_cut, false, 0.0, fro2, zero_rel, res, st) != cudaSuccess)
    return DMRGC_ECUDA;
  JacobiStatus hc{};
  TruncResult tr{};
  if (cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&tr, res, sizeof(tr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DMRGC_ECUDA;
  if (hc.err == DMRGC_ETIMEOUT) return DMRGC_ETIMEOUT;
  if (hc.err == DMRGC_ENOCONV) return DMRGC_ENOCONV;
  if (tr.status != 0) return DMRGC_ENUMERIC;
  const double* s_dev = reinterpret_cast<const double*>(reinterpret_cast<const TruncResult*>(res) + 1);
  if (cudaMemcpyAsync(s_out, s_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return DMRGC_ECUDA;
  if (gather_columns(G, m, n, tr.k, res, false, 0, U_out, fp64, st) != cudaSuccess) return DMRGC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DMRGC_ECUDA;
  *k_out = tr.k;
  return DMRGC_OK;
}

extern "C" dmrgc_status dmrgc_set_wait_limit(unsigned long long spins) {
  const unsigned long long v = spins ? spins : dmrgc::kSpinLimitDefault;
  return cudaMemcpyToSymbol(dmrgc::g_spin_limit, &v, sizeof(v)) == cudaSuccess ? DMRGC_OK : DMRGC_ECUDA;
}

extern "C" dmrgc_status dmrgc_set_jacobi_kernel(int variant) {
  if (variant < 0 || variant > 1) return DMRGC_EINVAL;
  dmrgc::g_jacobi_variant.store(variant, std::memory_order_relaxed);
  return DMRGC_OK;
}
