// Read-outs of the MPS: amplitudes <x|Psi> and bit-string sampling.
//
// Amplitude (Sec. IV.A, the MPS definition): <x|Psi> = A_1[x_1] ... A_N[x_N],
// for a chunk of strings at once, site by site.
// Sampling: sequential conditional sampling.  With the orthogonality centre on
// site c, the norm of any continuation of the prefix x_<=i is v E_i v^+ where
// v = A_1[x_1]..A_i[x_i] and E_i is the norm matrix of sites > i (identity for
// i >= c, built from the right for i < c).  Bit i of sample j is 0 iff
// u < p(0 | prefix), u from SplitMix64 (Steele, Lea, Flood 2014) evaluated at
// counter j*N + i; probabilities accumulate in double.
#include <algorithm>

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

// Batched read-outs.  Per site i the running row vectors of a chunk of B
// strings, V[B][l], are multiplied by the whole site tensor as one GEMM
// (W[b][x r + c] = sum_a V[b][a] A_i[a][x][c], done by the contraction engine
// before this kernel), so every site tensor is read once per chunk instead of
// once per string.  The kernels below take one row per CTA and pick x.

// amplitudes: V'[b][c] = W[b][x_b r + c], x_b the string's bit at site i
template <typename C2>
__global__ void amp_select_kernel(const C2* __restrict__ W, int r, const unsigned char* __restrict__ bits,
                                  int n, const int* __restrict__ qubits, int g, C2* __restrict__ V) {
  const int b = blockIdx.x;
  int x = 0;   // the tensor's physical index: its g qubits, the first the most significant bit
  for (int j = 0; j < g; ++j) x = (x << 1) | (bits[(long long)b * n + qubits[j]] & 1);
  const C2* src = W + (long long)b * ((long long)r << g) + (long long)x * r;
  C2* dst = V + (long long)b * r;
  for (int c = threadIdx.x; c < r; c += blockDim.x) dst[c] = src[c];
}

// sampling: p_x = |W_x|^2 (site at or right of the centre, T = null) or
// Re sum_c T[b][x r + c] conj(W[b][x r + c]) with T = W E_i (left of it);
// bit 0 iff u < p_0 / (p_0 + p_1), u = SplitMix64 at counter j N + i for
// global sample j = row0 + b; V'[b] = W_x[b] / sqrt(p_x).  The terms and the
// warp sums are in the storage precision, the sum of the warp sums in FP64
// by thread 0 alone: FP64 arithmetic in every thread would bound the
// complex64 kernel by GB300's FP64 rate (1/64 of FP32) instead of by HBM.
// (In the FP64 mode this is the plain FP64 sum in the same order.)
template <typename C2>
__global__ void sample_select_kernel(const C2* __restrict__ W, const C2* __restrict__ T, int r,
                                     unsigned long long seed, long long row0, int n, int site, int qubit,
                                     unsigned char* __restrict__ out, C2* __restrict__ V) {
  __shared__ double red[32];
  __shared__ int s_x;
  __shared__ double s_inv;
  const int b = blockIdx.x;
  const C2* w = W + (long long)b * 2 * r;
  const C2* t = T ? T + (long long)b * 2 * r : nullptr;
  using R = decltype(w->x);
  R q0 = 0, q1 = 0;
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    const C2 a0 = w[c], a1 = w[r + c];
    if (t) {
      const C2 e0 = t[c], e1 = t[r + c];
      q0 += e0.x * a0.x + e0.y * a0.y;
      q1 += e1.x * a1.x + e1.y * a1.y;
    } else {
      q0 += a0.x * a0.x + a0.y * a0.y;
      q1 += a1.x * a1.x + a1.y * a1.y;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    q0 += __shfl_xor_sync(0xffffffffu, q0, o);
    q1 += __shfl_xor_sync(0xffffffffu, q1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = (double)q0;
    red[16 + (threadIdx.x >> 5)] = (double)q1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double p0 = 0, p1 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      p0 += red[i];
      p1 += red[16 + i];
    }
    const long long j = row0 + b;
    const double u = splitmix64_uniform(seed, (unsigned long long)j * n + site);
    const double tot = p0 + p1;
    const int x = (tot > 0 && u < p0 / tot) ? 0 : 1;
    const double px = x == 0 ? p0 : p1;
    s_x = x;
    s_inv = px > 0 ? 1.0 / sqrt(px) : 0.0;
    out[j * n + qubit] = (unsigned char)x;
  }
  __syncthreads();
  const int x = s_x;
  const double inv = s_inv;
  const C2* src = w + (long long)x * r;
  C2* dst = V + (long long)b * r;
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    const C2 a = src[c];
    dst[c] = C2{(decltype(a.x))(a.x * inv), (decltype(a.x))(a.y * inv)};
  }
}

template <typename C2>
__global__ void amp_store_kernel(const C2* __restrict__ V, int B, double2* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) out[b] = double2{(double)V[b].x, (double)V[b].y};
}

template <typename C2>
__global__ void ones_kernel(C2* __restrict__ V, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) V[b] = C2{1, 0};
}

// Metropolis chains (App. C): counters g (n + 1) + q (bit q, qubit order,
// 1 iff u >= 1/2) and g (n + 1) + n (acceptance), g = chain (steps + 1) + t.
__global__ void metro_draw_kernel(unsigned char* __restrict__ prop, double* __restrict__ uacc, int C, int n,
                                  int steps, int t, unsigned long long seed) {
  const long long total = (long long)C * (n + 1);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(k / (n + 1)), q = (int)(k % (n + 1));
    const unsigned long long g = (unsigned long long)c * (steps + 1) + t;
    const double u = splitmix64_uniform(seed, g * (n + 1) + q);
    if (q < n) prop[(size_t)c * n + q] = u >= 0.5 ? 1 : 0;
    else uacc[c] = u;
  }
}

// t = 0: the chain takes its draw; t >= 1: it moves to the proposal iff
// u p(x) < p(x') (p(x) = 0 always moves); the chain's string after step t is
// written to out[c][t - 1].
__global__ void metro_step_kernel(const unsigned char* __restrict__ prop, const double2* __restrict__ amp,
                                  const double* __restrict__ uacc, unsigned char* __restrict__ cur,
                                  double* __restrict__ pcur, long long* __restrict__ acc,
                                  unsigned char* __restrict__ out, int C, int n, int steps, int t) {
  const int c = blockIdx.x;
  if (c >= C) return;
  __shared__ int move;
  if (threadIdx.x == 0) {
    const double q = amp[c].x * amp[c].x + amp[c].y * amp[c].y;
    move = t == 0 || pcur[c] == 0.0 || uacc[c] * pcur[c] < q;
    if (move) {
      pcur[c] = q;
      if (t > 0) acc[c] += 1;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    if (move) cur[(size_t)c * n + q] = prop[(size_t)c * n + q];
    if (t > 0) out[((size_t)c * steps + (t - 1)) * n + q] = cur[(size_t)c * n + q];
  }
}

}  // namespace

cudaError_t readout_start(void* V, int B, bool fp64, cudaStream_t st) {
  if (fp64) ones_kernel<<<(B + 255) / 256, 256, 0, st>>>(reinterpret_cast<double2*>(V), B);
  else ones_kernel<<<(B + 255) / 256, 256, 0, st>>>(reinterpret_cast<float2*>(V), B);
  return cudaGetLastError();
}

cudaError_t amp_select(const void* W, int B, int r, const unsigned char* bits, int n, const int* qubits, int g,
                       void* V, bool fp64, cudaStream_t st) {
  const int threads = r >= 256 ? 256 : (r >= 64 ? 64 : 32);
  if (fp64)
    amp_select_kernel<<<B, threads, 0, st>>>(reinterpret_cast<const double2*>(W), r, bits, n, qubits, g,
                                             reinterpret_cast<double2*>(V));
  else
    amp_select_kernel<<<B, threads, 0, st>>>(reinterpret_cast<const float2*>(W), r, bits, n, qubits, g,
                                             reinterpret_cast<float2*>(V));
  return cudaGetLastError();
}

cudaError_t sample_select(const void* W, const void* T, int B, int r, unsigned long long seed, long long row0, int n,
                          int site, int qubit, unsigned char* out, void* V, bool fp64, cudaStream_t st) {
  const int threads = r >= 256 ? 256 : (r >= 64 ? 64 : 32);
  if (fp64)
    sample_select_kernel<<<B, threads, 0, st>>>(reinterpret_cast<const double2*>(W),
                                                reinterpret_cast<const double2*>(T), r, seed, row0, n, site, qubit,
                                                out, reinterpret_cast<double2*>(V));
  else
    sample_select_kernel<<<B, threads, 0, st>>>(reinterpret_cast<const float2*>(W),
                                                reinterpret_cast<const float2*>(T), r, seed, row0, n, site, qubit,
                                                out, reinterpret_cast<float2*>(V));
  return cudaGetLastError();
}

cudaError_t amp_store(const void* V, int B, double2* out, bool fp64, cudaStream_t st) {
  if (fp64) amp_store_kernel<<<(B + 255) / 256, 256, 0, st>>>(reinterpret_cast<const double2*>(V), B, out);
  else amp_store_kernel<<<(B + 255) / 256, 256, 0, st>>>(reinterpret_cast<const float2*>(V), B, out);
  return cudaGetLastError();
}

}  // namespace dmrgc

namespace dmrgc {

cudaError_t metro_draw(unsigned char* prop, double* uacc, int C, int n, int steps, int t, unsigned long long seed,
                       cudaStream_t st) {
  const long long total = (long long)C * (n + 1);
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  metro_draw_kernel<<<blocks, 256, 0, st>>>(prop, uacc, C, n, steps, t, seed);
  return cudaGetLastError();
}

cudaError_t metro_step(const unsigned char* prop, const double2* amp, const double* uacc, unsigned char* cur,
                       double* pcur, long long* acc, unsigned char* out, int C, int n, int steps, int t,
                       cudaStream_t st) {
  metro_step_kernel<<<C, 64, 0, st>>>(prop, amp, uacc, cur, pcur, acc, out, C, n, steps, t);
  return cudaGetLastError();
}

}  // namespace dmrgc
