// Small layout and reduction kernels: transposed / conjugated copies, the
// physical-index-first permutation of MPS tensors, identities, norms, scaling.
#include "common.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace dmrgc {
namespace {

inline int blocks_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b > 65536) b = 65536;
  return b < 1 ? 1 : (int)b;
}

template <typename C2>
__global__ void transpose_kernel(const C2* __restrict__ src, int rows, int cols, int conj,
                                 C2* __restrict__ dst) {
  __shared__ C2 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = src[(long long)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = bx + j, r = by + threadIdx.x;
    if (r < rows && c < cols) {
      C2 v = tile[threadIdx.x][j];
      if (conj) v.y = -v.y;
      dst[(long long)c * rows + r] = v;
    }
  }
}

template <typename C2>
__global__ void conj_kernel(const C2* __restrict__ src, long long n, C2* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    C2 v = src[i];
    v.y = -v.y;
    dst[i] = v;
  }
}

template <typename C2>
__global__ void phys_first_kernel(const C2* __restrict__ src, int a, int b, C2* __restrict__ dst) {
  const long long n = 2LL * a * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long ia = e / (2LL * b);
    const long long rem = e % (2LL * b);
    const long long s = rem / b, ib = rem % b;
    dst[s * a * b + ia * b + ib] = src[e];
  }
}

template <typename C2>
__global__ void identity_kernel(C2* __restrict__ dst, int n) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, c = e % n;
    dst[e] = C2{(decltype(C2{}.x))(r == c ? 1 : 0), (decltype(C2{}.x))0};
  }
}

template <typename C2>
__global__ void sum_abs2_kernel(const C2* __restrict__ x, long long n, double* out) {
  double s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += (double)x[i].x * x[i].x + (double)x[i].y * x[i].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) atomicAdd(out, t);
  }
}

// |x|^2 in FP64 in a fixed order: CTA b sums the chunk [b chunk, (b+1) chunk)
// (thread, warp and CTA trees fixed), then every CTA of the second kernel adds
// the kNormParts partials in the same fixed order, so every CTA and every run
// sees the same bits.
constexpr int kNormParts = 256;

__device__ __forceinline__ double block256_sum(double s, double* red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += red[w];
  return t;
}

template <typename C2>
__global__ void __launch_bounds__(256) norm2_part_kernel(const C2* __restrict__ x, long long n, long long chunk,
                                                         double* __restrict__ part) {
  __shared__ double red[8];
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += 256) s += (double)x[i].x * x[i].x + (double)x[i].y * x[i].y;
  s = block256_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename C2>
__global__ void __launch_bounds__(256) norm2_finish_kernel(C2* __restrict__ x, long long n, long long chunk,
                                                           const double* __restrict__ part, double* __restrict__ out,
                                                           int scale) {
  __shared__ double red[8];
  const double tot = block256_sum(part[threadIdx.x], red);   // blockDim == kNormParts
  if (blockIdx.x == 0 && threadIdx.x == 0) *out = tot;
  if (!scale) return;
  const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  for (long long i = lo + threadIdx.x; i < hi; i += 256) {
    C2 v = x[i];
    v.x = (decltype(v.x))(v.x * inv);
    v.y = (decltype(v.y))(v.y * inv);
    x[i] = v;
  }
}

template <typename C2>
__global__ void scale_kernel(C2* __restrict__ x, long long n, const double* norm2) {
  const double nrm = sqrt(*norm2);
  const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    C2 v = x[i];
    v.x = (decltype(v.x))(v.x * inv);
    v.y = (decltype(v.y))(v.y * inv);
    x[i] = v;
  }
}

template <typename C2>
__global__ void to_z_kernel(const C2* __restrict__ x, long long n, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = double2{(double)x[i].x, (double)x[i].y};
}

template <typename C2>
__global__ void from_z_kernel(const double2* __restrict__ x, long long n, C2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = C2{(decltype(C2{}.x))x[i].x, (decltype(C2{}.x))x[i].y};
}

}  // namespace

cudaError_t allow_dyn_smem(const void* fn) {
  static std::mutex mu;
  static std::vector<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first == dev && d.second == fn) return cudaSuccess;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
  const int dyn = optin - (int)fa.sharedSizeBytes;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
  done.emplace_back(dev, fn);
  return cudaSuccess;
}

namespace {

__device__ __forceinline__ double mix_uniform(unsigned long long seed, unsigned long long ctr) {
  // SplitMix64 (Steele, Lea, Flood 2014) at counter ctr, top 53 bits -> [0, 1)
  unsigned long long z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

template <typename C2>
__global__ void gaussian_kernel(C2* __restrict__ out, long long n, unsigned long long seed,
                                unsigned long long ctr0) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const double u1 = mix_uniform(seed, ctr0 + 2ull * j);
    const double u2 = mix_uniform(seed, ctr0 + 2ull * j + 1ull);
    const double rad = sqrt(-log1p(-u1));   // |z|^2 ~ Exp(1): E|z|^2 = 1
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[j].x = rad * cs;
    out[j].y = rad * sn;
  }
}

template <typename C2>
__global__ void unit_square_kernel(C2* __restrict__ out, long long n, unsigned long long seed,
                                   unsigned long long ctr0) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    out[j].x = 2.0 * mix_uniform(seed, ctr0 + 2ull * j) - 1.0;
    out[j].y = 2.0 * mix_uniform(seed, ctr0 + 2ull * j + 1ull) - 1.0;
  }
}

}  // namespace

cudaError_t fill_unit_square(void* dst, long long n, bool fp64, unsigned long long seed,
                             unsigned long long ctr0, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  if (fp64) unit_square_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<double2*>(dst), n, seed, ctr0);
  else unit_square_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<float2*>(dst), n, seed, ctr0);
  return cudaGetLastError();
}

cudaError_t fill_gaussian(void* dst, long long n, bool fp64, unsigned long long seed,
                          unsigned long long ctr0, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  if (fp64) gaussian_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<double2*>(dst), n, seed, ctr0);
  else gaussian_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<float2*>(dst), n, seed, ctr0);
  return cudaGetLastError();
}

cudaError_t from_complex128(const double2* src, long long n, bool fp64, void* dst, cudaStream_t st) {
  if (fp64) from_z_kernel<<<blocks_for(n), 256, 0, st>>>(src, n, (double2*)dst);
  else from_z_kernel<<<blocks_for(n), 256, 0, st>>>(src, n, (float2*)dst);
  return cudaGetLastError();
}

cudaError_t copy_transpose(const void* src, int rows, int cols, bool conj, void* dst, bool fp64,
                           cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  if (fp64)
    transpose_kernel<<<grid, block, 0, st>>>((const double2*)src, rows, cols, conj ? 1 : 0, (double2*)dst);
  else
    transpose_kernel<<<grid, block, 0, st>>>((const float2*)src, rows, cols, conj ? 1 : 0, (float2*)dst);
  return cudaGetLastError();
}

namespace {

// out[o0][o1][o2][o3] = in[...], out axis k = in axis p[k]
template <typename C2>
__global__ void permute4_kernel(const C2* __restrict__ in, int4 dims, int4 perm, C2* __restrict__ out, long long n) {
  const int d[4] = {dims.x, dims.y, dims.z, dims.w};
  const int p[4] = {perm.x, perm.y, perm.z, perm.w};
  long long stride_in[4];
  stride_in[3] = 1;
  for (int k = 2; k >= 0; --k) stride_in[k] = stride_in[k + 1] * d[k + 1];
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    long long rem = o, src = 0;
    for (int k = 3; k >= 0; --k) {
      const int dk = d[p[k]];
      src += (rem % dk) * stride_in[p[k]];
      rem /= dk;
    }
    out[o] = in[src];
  }
}

}  // namespace

cudaError_t permute4(const void* src, const int* dims, const int* perm, void* dst, bool fp64, cudaStream_t st) {
  const long long n = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (n <= 0) return cudaSuccess;
  const int4 d = make_int4(dims[0], dims[1], dims[2], dims[3]);
  const int4 p = make_int4(perm[0], perm[1], perm[2], perm[3]);
  if (fp64) permute4_kernel<<<blocks_for(n), 256, 0, st>>>((const double2*)src, d, p, (double2*)dst, n);
  else permute4_kernel<<<blocks_for(n), 256, 0, st>>>((const float2*)src, d, p, (float2*)dst, n);
  return cudaGetLastError();
}

cudaError_t copy_conj(const void* src, long long n, void* dst, bool fp64, cudaStream_t st) {
  if (fp64) conj_kernel<<<blocks_for(n), 256, 0, st>>>((const double2*)src, n, (double2*)dst);
  else conj_kernel<<<blocks_for(n), 256, 0, st>>>((const float2*)src, n, (float2*)dst);
  return cudaGetLastError();
}

cudaError_t permute_phys_first(const void* src, int a, int b, void* dst, bool fp64, cudaStream_t st) {
  const long long n = 2LL * a * b;
  if (fp64) phys_first_kernel<<<blocks_for(n), 256, 0, st>>>((const double2*)src, a, b, (double2*)dst);
  else phys_first_kernel<<<blocks_for(n), 256, 0, st>>>((const float2*)src, a, b, (float2*)dst);
  return cudaGetLastError();
}

cudaError_t set_identity(void* dst, int n, bool fp64, cudaStream_t st) {
  const long long t = (long long)n * n;
  if (fp64) identity_kernel<<<blocks_for(t), 256, 0, st>>>((double2*)dst, n);
  else identity_kernel<<<blocks_for(t), 256, 0, st>>>((float2*)dst, n);
  return cudaGetLastError();
}

cudaError_t set_scalar_one(void* dst, bool fp64, cudaStream_t st) { return set_identity(dst, 1, fp64, st); }

cudaError_t sum_abs2(const void* x, long long n, bool fp64, double* out_dev, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int b = blocks_for(n);
  if (b > 1024) b = 1024;
  if (fp64) sum_abs2_kernel<<<b, 256, 0, st>>>((const double2*)x, n, out_dev);
  else sum_abs2_kernel<<<b, 256, 0, st>>>((const float2*)x, n, out_dev);
  return cudaGetLastError();
}

cudaError_t norm2_scale(void* x, long long n, bool fp64, double* out_dev, double* part_dev, bool scale,
                        cudaStream_t st) {
  const long long chunk = (n + kNormParts - 1) / kNormParts;
  if (fp64) {
    norm2_part_kernel<<<kNormParts, 256, 0, st>>>((const double2*)x, n, chunk, part_dev);
    norm2_finish_kernel<<<kNormParts, 256, 0, st>>>((double2*)x, n, chunk, part_dev, out_dev, scale ? 1 : 0);
  } else {
    norm2_part_kernel<<<kNormParts, 256, 0, st>>>((const float2*)x, n, chunk, part_dev);
    norm2_finish_kernel<<<kNormParts, 256, 0, st>>>((float2*)x, n, chunk, part_dev, out_dev, scale ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t scale_inplace(void* x, long long n, const double* norm2_dev, bool fp64, cudaStream_t st) {
  if (fp64) scale_kernel<<<blocks_for(n), 256, 0, st>>>((double2*)x, n, norm2_dev);
  else scale_kernel<<<blocks_for(n), 256, 0, st>>>((float2*)x, n, norm2_dev);
  return cudaGetLastError();
}

cudaError_t to_complex128(const void* src, long long n, bool fp64, double2* dst, cudaStream_t st) {
  if (fp64) to_z_kernel<<<blocks_for(n), 256, 0, st>>>((const double2*)src, n, dst);
  else to_z_kernel<<<blocks_for(n), 256, 0, st>>>((const float2*)src, n, dst);
  return cudaGetLastError();
}

}  // namespace dmrgc
