// Read-outs of the MPS: amplitudes <x|Psi> and bit-string sampling.
//
// Amplitude (Sec. IV.A, the MPS definition): <x|Psi> = A_1[x_1] ... A_N[x_N],
// one CTA per bit string, the running row vector kept in shared memory.
// Sampling: sequential conditional sampling.  With the orthogonality centre on
// site c, the norm of any continuation of the prefix x_<=i is v E_i v^+ where
// v = A_1[x_1]..A_i[x_i] and E_i is the norm matrix of sites > i (identity for
// i >= c, built from the right for i < c).  Bit i of sample j is 0 iff
// u < p(0 | prefix), u from SplitMix64 (Steele, Lea, Flood 2014) evaluated at
// counter j*N + i; probabilities accumulate in double.
#include "common.cuh"

namespace dmrgc {
namespace {

__device__ __forceinline__ double splitmix64_uniform(unsigned long long seed, unsigned long long ctr) {
  unsigned long long z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

template <typename C2>
__global__ void amp_kernel(const void* const* __restrict__ sites, const int* __restrict__ bonds,
                           const int* __restrict__ order, int n, const unsigned char* __restrict__ bits,
                           long long count, double2* __restrict__ out) {
  extern __shared__ double2 sv[];   // [2][max_bond]
  const long long j = blockIdx.x;
  if (j >= count) return;
  double2* v = sv;
  const int maxb = bonds[n + 1];
  double2* w = sv + maxb;
  if (threadIdx.x == 0) v[0] = double2{1.0, 0.0};
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    const int l = bonds[i], r = bonds[i + 1];
    const int x = bits[j * n + order[i]];
    const C2* A = reinterpret_cast<const C2*>(sites[i]);
    for (int b = threadIdx.x; b < r; b += blockDim.x) {
      double2 acc{0, 0};
      for (int a = 0; a < l; ++a) {
        const C2 t = A[((long long)a * 2 + x) * r + b];
        const double2 tv{(double)t.x, (double)t.y};
        acc = cadd(acc, cmul(v[a], tv));
      }
      w[b] = acc;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < r; b += blockDim.x) v[b] = w[b];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = v[0];
}

template <typename C2>
__global__ void sample_kernel(const void* const* __restrict__ sites, const void* const* __restrict__ emat,
                              const int* __restrict__ bonds, const int* __restrict__ order, int n,
                              int centre, unsigned long long seed, long long count,
                              unsigned char* __restrict__ out) {
  extern __shared__ double2 sm[];   // v, w0, w1 [max_bond each], red[32]
  const long long j = blockIdx.x;
  if (j >= count) return;
  const int maxb = bonds[n + 1];
  double2* v = sm;
  double2* w0 = sm + maxb;
  double2* w1 = sm + 2 * maxb;
  double* red = reinterpret_cast<double*>(sm + 3 * maxb);
  if (threadIdx.x == 0) v[0] = double2{1.0, 0.0};
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    const int l = bonds[i], r = bonds[i + 1];
    const C2* A = reinterpret_cast<const C2*>(sites[i]);
    for (int b = threadIdx.x; b < r; b += blockDim.x) {
      double2 a0{0, 0}, a1{0, 0};
      for (int a = 0; a < l; ++a) {
        const C2 t0 = A[((long long)a * 2 + 0) * r + b];
        const C2 t1 = A[((long long)a * 2 + 1) * r + b];
        a0 = cadd(a0, cmul(v[a], double2{(double)t0.x, (double)t0.y}));
        a1 = cadd(a1, cmul(v[a], double2{(double)t1.x, (double)t1.y}));
      }
      w0[b] = a0;
      w1[b] = a1;
    }
    __syncthreads();
    double p0 = 0, p1 = 0;
    if (i >= centre) {
      for (int b = threadIdx.x; b < r; b += blockDim.x) {
        p0 += w0[b].x * w0[b].x + w0[b].y * w0[b].y;
        p1 += w1[b].x * w1[b].x + w1[b].y * w1[b].y;
      }
    } else {
      // p = w E w^+ = sum_b w[b] sum_b' E[b][b'] conj(w[b'])
      const C2* E = reinterpret_cast<const C2*>(emat[i]);
      for (int b = threadIdx.x; b < r; b += blockDim.x) {
        double2 e0{0, 0}, e1{0, 0};
        for (int bb = 0; bb < r; ++bb) {
          const C2 t = E[(long long)b * r + bb];
          const double2 tv{(double)t.x, (double)t.y};
          e0 = cadd(e0, cmul(tv, cconj(w0[bb])));
          e1 = cadd(e1, cmul(tv, cconj(w1[bb])));
        }
        p0 += cmul(w0[b], e0).x;
        p1 += cmul(w1[b], e1).x;
      }
    }
    p0 = block_sum(p0, red);
    p1 = block_sum(p1, red);
    const double u = splitmix64_uniform(seed, (unsigned long long)j * n + i);
    const double tot = p0 + p1;
    const int x = (tot > 0 && u < p0 / tot) ? 0 : 1;
    const double px = x == 0 ? p0 : p1;
    const double inv = px > 0 ? 1.0 / sqrt(px) : 0.0;
    const double2* src = x == 0 ? w0 : w1;
    for (int b = threadIdx.x; b < r; b += blockDim.x) v[b] = double2{src[b].x * inv, src[b].y * inv};
    if (threadIdx.x == 0) out[j * n + order[i]] = (unsigned char)x;
    __syncthreads();
  }
}

}  // namespace

cudaError_t amplitudes(const void* const* sites, const int* bonds, const int* order, int n_sites,
                       int max_bond, const unsigned char* bits, long long count, double2* out,
                       bool fp64, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (count > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t sm = 2 * (size_t)max_bond * sizeof(double2);
  const int threads = max_bond >= 256 ? 256 : 128;
  cudaError_t e;
  if (fp64) {
    e = allow_dyn_smem((const void*)amp_kernel<double2>);
    if (e != cudaSuccess) return e;
    amp_kernel<double2><<<(unsigned)count, threads, sm, st>>>(sites, bonds, order, n_sites, bits, count, out);
  } else {
    e = allow_dyn_smem((const void*)amp_kernel<float2>);
    if (e != cudaSuccess) return e;
    amp_kernel<float2><<<(unsigned)count, threads, sm, st>>>(sites, bonds, order, n_sites, bits, count, out);
  }
  return cudaGetLastError();
}

cudaError_t sample_bits(const void* const* sites, const void* const* emat, const int* bonds,
                        const int* order, int n_sites, int centre, int max_bond,
                        unsigned long long seed, long long count, unsigned char* out, bool fp64,
                        cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (count > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t sm = 3 * (size_t)max_bond * sizeof(double2) + 32 * sizeof(double);
  const int threads = 256;
  cudaError_t e;
  if (fp64) {
    e = allow_dyn_smem((const void*)sample_kernel<double2>);
    if (e != cudaSuccess) return e;
    sample_kernel<double2><<<(unsigned)count, threads, sm, st>>>(sites, emat, bonds, order, n_sites,
                                                                 centre, seed, count, out);
  } else {
    e = allow_dyn_smem((const void*)sample_kernel<float2>);
    if (e != cudaSuccess) return e;
    sample_kernel<float2><<<(unsigned)count, threads, sm, st>>>(sites, emat, bonds, order, n_sites,
                                                                centre, seed, count, out);
  }
  return cudaGetLastError();
}

}  // namespace dmrgc
