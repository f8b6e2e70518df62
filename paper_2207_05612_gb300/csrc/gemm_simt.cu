// Batched complex GEMM on CUDA cores (FFMA / DFMA), any operand op.
//
// This is the FP64 path's contraction engine and the FP32 reference path of
// the complex64 modes.  One CTA of 256 threads computes a 64x64 tile of C;
// every thread owns a 4x4 block of complex accumulators.  Operand tiles are
// staged in shared memory with the loads ordered along the operand's
// contiguous index so that global reads coalesce for every op.
#include "common.cuh"

namespace dmrgc {
namespace {

constexpr int BM = 64, BN = 64, TM = 4, TN = 4, NT = 256;

template <typename R> struct Tile;
template <> struct Tile<float> { static constexpr int BK = 16; };
template <> struct Tile<double> { static constexpr int BK = 8; };

template <typename R, int BK>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g) {
  using C2 = typename cplx<R>::T;
  __shared__ C2 As[BK][BM + 1];
  __shared__ C2 Bs[BK][BN + 1];

  const int bz = blockIdx.z;
  const int i1 = bz / g.b2, i2 = bz % g.b2;
  const C2* __restrict__ A = reinterpret_cast<const C2*>(g.A) + i1 * g.sA1 + i2 * g.sA2;
  const C2* __restrict__ B = reinterpret_cast<const C2*>(g.B) + i1 * g.sB1 + i2 * g.sB2;
  C2* __restrict__ C = reinterpret_cast<C2*>(g.C) + i1 * g.sC1 + i2 * g.sC2;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);

  C2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = C2{0, 0};

  const bool a_kfast = (g.opA == OP_N || g.opA == OP_R);
  const bool a_conj = (g.opA == OP_C || g.opA == OP_R);
  const bool b_nfast = (g.opB == OP_N || g.opB == OP_R);
  const bool b_conj = (g.opB == OP_C || g.opB == OP_R);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    // A tile: BM x BK
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      const int m = m0 + mm, k = k0 + kk;
      C2 v{0, 0};
      if (m < g.M && k < g.K) {
        v = a_kfast ? A[(long long)m * g.lda + k] : A[(long long)k * g.lda + m];
        if (a_conj) v.y = -v.y;
      }
      As[kk][mm] = v;
    }
    // B tile: BK x BN
    for (int e = tid; e < BN * BK; e += NT) {
      int nn, kk;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int n = n0 + nn, k = k0 + kk;
      C2 v{0, 0};
      if (n < g.N && k < g.K) {
        v = b_nfast ? B[(long long)k * g.ldb + n] : B[(long long)n * g.ldb + k];
        if (b_conj) v.y = -v.y;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C2 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  const R ar = (R)g.alpha_re, ai = (R)g.alpha_im;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + i * (BM / TM);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + j * (BN / TN);
      if (n >= g.N) continue;
      C2 v{acc[i][j].x * ar - acc[i][j].y * ai, acc[i][j].x * ai + acc[i][j].y * ar};
      C2* dst = C + (long long)m * g.ldc + n;
      if (g.beta_one) { C2 o = *dst; v.x += o.x; v.y += o.y; }
      *dst = v;
    }
  }
}

}  // namespace

cudaError_t gemm_simt(const GemmArgs& g, bool fp64, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.b1 <= 0 || g.b2 <= 0) return cudaSuccess;
  const long long batch = (long long)g.b1 * g.b2;
  if (batch > 65535) return cudaErrorInvalidConfiguration;
  const long long gy = (g.M + BM - 1) / BM;
  if (gy > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((g.N + BN - 1) / BN, (unsigned)gy, (unsigned)batch);
  if (g.K <= 0) {
    // empty contraction: C = 0 (or unchanged with beta)
    if (!g.beta_one) {
      // fall through with K=0: the kernel writes zeros
    }
  }
  if (fp64)
    gemm_kernel<double, Tile<double>::BK><<<grid, NT, 0, st>>>(g);
  else
    gemm_kernel<float, Tile<float>::BK><<<grid, NT, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace dmrgc
