// Complex GEMM on the 5th-generation tensor cores (tcgen05, TMEM, TMA) with
// split-precision operands: BF16x3 (kind::f16) or TF32x3 (kind::tf32), FP32
// accumulation.
//
// Complex product as one real GEMM.  With A'[m][2k+0] = Re A, A'[m][2k+1] = Im A
// and the N-side operand expanded to
//   B'[2n  ][2k] = Re B,  B'[2n  ][2k+1] = -Im B,
//   B'[2n+1][2k] = Im B,  B'[2n+1][2k+1] =  Re B,
// C' = A' B'^T gives C'[m][2n] = Re C and C'[m][2n+1] = Im C, i.e. C' is the
// complex output already interleaved.  Each real operand x is split into
// hi = round(x) and lo = round(x - hi) in the narrow format, and
// A'B'^T ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T (the lo*lo term is below the
// FP32 accumulation error).
//
// Kernel: persistent, one CTA of 6 warps per SM looping over 128 x 256 tiles
// of C' (128 x 128 complex).  Warp 0 (one thread) streams the K blocks of
// A_hi, A_lo, B_hi, B_lo with TMA (128-byte swizzle, K-major) into a 2-stage
// ring; warp 1 (one thread) issues 3 x (BK / MMA_K) MMAs per stage into one of
// two accumulators of 256 TMEM columns and frees the stage with
// tcgen05.commit; warps 2-5 read the other accumulator (32 lanes x 32 columns
// per load, each warp its quarter of the TMEM lanes) and write complex C, so
// a tile's epilogue overlaps the next tile's main loop.  With split-K each
// split writes its partial product to a workspace and one more kernel sums the
// partials in a fixed order (no atomics), so every product is reproducible.
// Every mbarrier wait is bounded by the global timer; an exhausted wait sets
// an error flag, stops issuing, drains what is in flight (bounded), frees TMEM
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace dmrgc {
namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_THREADS = 192, TC_STAGES = 2, TC_ACC = 2;
constexpr int TC_ROW_BYTES = 128;                        // one swizzle row of K per stage
constexpr int TC_A_BYTES = TC_BM * TC_ROW_BYTES;         // 16 KiB
constexpr int TC_B_BYTES = TC_BN * TC_ROW_BYTES;         // 32 KiB
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // 2 s per wait

struct TcArgs {
  int M, N;            // complex output rows / cols
  int tiles_n, tiles_m;   // tile grid of one instance and split; tiles run in the order (z, m, n)
  long long total;        // tiles_n * tiles_m * batches * split
  int ktiles;          // K blocks of BK real elements
  int split;           // split-K factor
  int per;             // K blocks per split
  int b1, b2;
  int a_m1, a_m2, b_m1, b_m2;   // packed-instance index multipliers
  float2* C;
  long long ldc, sC1, sC2;
  float alpha_re, alpha_im;
  int mode;            // 0 store, 1 add to C (beta = 1), 2 split-K partial into P
  int upper;           // 1: skip the tiles strictly below the diagonal (square C)
  float2* P;           // split-K partials [split][batch][M][N] (mode 2)
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on a phase; false when the time limit or an abort ends it
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > TC_WAIT_NS) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 128-byte swizzle: 8 rows x 128 B per 1024-B atom
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

template <int ESZ>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (ESZ == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// instruction descriptor: D = F32, A/B = BF16 (ESZ 2) or TF32 (ESZ 4), both K-major
template <int ESZ>
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | ((ESZ == 2 ? 1u : 2u) << 7) | ((ESZ == 2 ? 1u : 2u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int ESZ>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                   const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                   TcArgs g) {
  constexpr int BK = TC_ROW_BYTES / ESZ;      // real K elements per stage
  constexpr int MMA_K = 32 / ESZ;             // K per MMA: 16 (bf16), 8 (tf32)
  constexpr int KSTEPS = BK / MMA_K;          // 4
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accf = empty + TC_STAGES;      // accumulator a holds a finished tile (MMA -> epilogue)
  uint64_t* acce = accf + TC_ACC;          // accumulator a has been read out (epilogue -> MMA)
  uint64_t* drain = acce + TC_ACC;         // every issued MMA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* s_issued = reinterpret_cast<int*>(tmem_slot + 2);   // loads issued / stages consumed (teardown)
  int* s_consumed = s_issued + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long per_z = (long long)g.tiles_n * g.tiles_m;
  // tile t -> (z = batch * split + ks, m tile, n tile); a Hermitian product
  // enumerates only the tiles on or above the diagonal (bx >= by), row by row
  auto decode = [&](long long t, int& bx, int& by, int& z) {
    if (g.upper) {
      const long long per_u = (long long)g.tiles_m * (g.tiles_m + 1) / 2;
      z = (int)(t / per_u);
      int r = (int)(t % per_u);
      by = 0;
      while (r >= g.tiles_m - by) { r -= g.tiles_m - by; ++by; }
      bx = by + r;
      return;
    }
    z = (int)(t / per_z);
    const long long r = t % per_z;
    by = (int)(r / g.tiles_n);
    bx = (int)(r % g.tiles_n);
  };
  auto kblocks = [&](int ks) {
    int nk = g.ktiles - ks * g.per;
    if (nk > g.per) nk = g.per;
    return nk < 0 ? 0 : nk;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < TC_ACC; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], 4); }
    mbar_init(drain, 1);
    *abort_flag = 0;
    *s_issued = 0;
    *s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_ACC * 256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int it = 0;
    for (long long t = blockIdx.x; t < g.total && !*abort_flag; t += gridDim.x) {
      int bx, by, z;
      decode(t, bx, by, z);
      const int batch = z / g.split, ks = z % g.split;
      const int i1 = batch / g.b2, i2 = batch % g.b2;
      const int instA = i1 * g.a_m1 + i2 * g.a_m2, instB = i1 * g.b_m1 + i2 * g.b_m2;
      const int nk = kblocks(ks), kt0 = ks * g.per;
      for (int k = 0; k < nk; ++k, ++it) {
        const int s = it % TC_STAGES;
        const uint32_t ph = (uint32_t)((it / TC_STAGES) & 1);
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) { *abort_flag = 1; break; }
        uint8_t* st = smem + s * TC_STAGE_BYTES;
        mbar_expect_tx(&full[s], TC_STAGE_BYTES);
        const int kx = (kt0 + k) * BK;
        tma_load_3d(st, &tA_hi, kx, by * TC_BM, instA, &full[s]);
        tma_load_3d(st + TC_A_BYTES, &tA_lo, kx, by * TC_BM, instA, &full[s]);
        tma_load_3d(st + 2 * TC_A_BYTES, &tB_hi, kx, bx * TC_BN, instB, &full[s]);
        tma_load_3d(st + 2 * TC_A_BYTES + TC_B_BYTES, &tB_lo, kx, bx * TC_BN, instB, &full[s]);
        *s_issued = it + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t ID = idesc<ESZ>(TC_BM, TC_BN);
    int it = 0, lt = 0;
    for (long long t = blockIdx.x; t < g.total && !*abort_flag; t += gridDim.x) {
      int bx, by, z;
      decode(t, bx, by, z);
      const int nk = kblocks(z % g.split);
      const int a = lt & 1;
      if (!mbar_wait(&acce[a], (uint32_t)(((lt >> 1) & 1) ^ 1), abort_flag)) { *abort_flag = 1; break; }
      tc_fence_after();
      const uint32_t acc_tmem = tmem + (uint32_t)(a * 256);
      bool ok = true;
      for (int k = 0; k < nk; ++k, ++it) {
        const int s = it % TC_STAGES;
        const uint32_t ph = (uint32_t)((it / TC_STAGES) & 1);
        if (!mbar_wait(&full[s], ph, abort_flag)) { *abort_flag = 1; ok = false; break; }
        tc_fence_after();
        const uint32_t base = smem_u32(smem + s * TC_STAGE_BYTES);
        const uint64_t a_hi = sdesc_sw128(base), a_lo = sdesc_sw128(base + TC_A_BYTES);
        const uint64_t b_hi = sdesc_sw128(base + 2 * TC_A_BYTES);
        const uint64_t b_lo = sdesc_sw128(base + 2 * TC_A_BYTES + TC_B_BYTES);
#pragma unroll
        for (int kk = 0; kk < KSTEPS; ++kk) {
          const uint64_t off = (uint64_t)((kk * MMA_K * ESZ) >> 4);   // 32 B per K step
          umma<ESZ>(acc_tmem, a_hi + off, b_hi + off, ID, (k | kk) ? 1u : 0u);
          umma<ESZ>(acc_tmem, a_hi + off, b_lo + off, ID, 1u);
          umma<ESZ>(acc_tmem, a_lo + off, b_hi + off, ID, 1u);
        }
        umma_commit(&empty[s]);
        *s_consumed = it + 1;
      }
      if (!ok) break;
      umma_commit(&accf[a]);   // arrives once the tile's MMAs have completed
      ++lt;
    }
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile)
    const int q = warp & 3;
    int lt = 0;
    for (long long t = blockIdx.x; t < g.total && !*abort_flag; t += gridDim.x) {
      int bx, by, z;
      decode(t, bx, by, z);
      const int a = lt & 1;
      if (!mbar_wait(&accf[a], (uint32_t)((lt >> 1) & 1), abort_flag)) { *abort_flag = 1; break; }
      tc_fence_after();
      const int batch = z / g.split, ks = z % g.split;
      const int i1 = batch / g.b2, i2 = batch % g.b2;
      const int row = by * TC_BM + q * 32 + lane;
      const int n0 = bx * TC_BN;
      float2* Cb = g.C + (long long)i1 * g.sC1 + (long long)i2 * g.sC2;
#pragma unroll 1
      for (int c = 0; c < TC_BN / 32; ++c) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 256 + c * 32), r);
        if (row < g.M) {
          const int ncol0 = (n0 + c * 32) >> 1;
          float2* dst = Cb + (long long)row * g.ldc + ncol0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (ncol0 + j < g.N) {
              const float re = __uint_as_float(r[2 * j]), im = __uint_as_float(r[2 * j + 1]);
              const float vr = re * g.alpha_re - im * g.alpha_im;
              const float vi = re * g.alpha_im + im * g.alpha_re;
              if (g.mode == 2) {
                float2* pd = g.P + ((long long)ks * (g.b1 * g.b2) + batch) * ((long long)g.M * g.N) +
                             (long long)row * g.N + ncol0;
                pd[j] = make_float2(vr, vi);
              } else if (g.mode == 1) {
                float2 o = dst[j];
                dst[j] = make_float2(o.x + vr, o.y + vi);
              } else {
                dst[j] = make_float2(vr, vi);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[a])) : "memory");
      ++lt;
    }
  }
  __syncwarp();
  // ---- teardown: nothing may still write smem or TMEM when the CTA leaves
  __syncthreads();
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    umma_commit(drain);
    mbar_wait(drain, 0, &never);   // every issued MMA has completed (bounded)
  }
  if (*abort_flag && warp == 0 && lane == 0) {
    // TMA loads the MMA thread never consumed (bounded waits)
    volatile int never = 0;
    for (int it = *s_consumed; it < *s_issued; ++it)
      mbar_wait(&full[it % TC_STAGES], (uint32_t)((it / TC_STAGES) & 1), &never);
  }
  if (*abort_flag && threadIdx.x == 0) atomicExch(g.err, (int)DMRGC_ETIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_ACC * 256) : "memory");
  }
}

// ---- operand packing: complex -> split real operands, K-major, row stride kp

__device__ __forceinline__ void split2(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ float tf32_rne(float x) {
  uint32_t b = __float_as_uint(x);
  if ((b & 0x7F800000u) == 0x7F800000u) return x;   // inf / nan unchanged
  b += 0xFFFu + ((b >> 13) & 1u);
  return __uint_as_float(b & 0xFFFFE000u);
}

__device__ __forceinline__ void split4(float x, float& hi, float& lo) {
  hi = tf32_rne(x);
  lo = tf32_rne(x - hi);
}

// one 32 x 32 tile of (row = m or n, col = k) complex values via shared memory
// so that both the source (either index contiguous) and the destination
// (k contiguous) are read / written in order.  expand = 1: the N-side 2x2 form.
template <int ESZ>
__global__ void pack_kernel(const float2* __restrict__ src, long long ld, long long s1, long long s2,
                            int src_kfast, int conj, int rows, int K, int kp, int expand, int inst_b1_stride,
                            int n_inst1, int n_inst2, void* __restrict__ hi_out, void* __restrict__ lo_out) {
  __shared__ float2 tile[32][33];
  const int inst = blockIdx.z;
  const int j1 = inst / n_inst2, j2 = inst % n_inst2;
  const float2* S = src + j1 * s1 + j2 * s2;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  (void)inst_b1_stride;
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    // t indexes the slow index of the source read, threadIdx.x the fast one
    int r, k;
    if (src_kfast) { r = r0 + t; k = k0 + threadIdx.x; } else { k = k0 + t; r = r0 + threadIdx.x; }
    float2 v = make_float2(0.f, 0.f);
    if (r < rows && k < K) v = src_kfast ? S[(long long)r * ld + k] : S[(long long)k * ld + r];
    if (conj) v.y = -v.y;
    if (src_kfast) tile[t][threadIdx.x] = v; else tile[threadIdx.x][t] = v;
  }
  __syncthreads();
  const int out_rows = expand ? 2 * rows : rows;
  const long long inst_elems = (long long)out_rows * kp;
  // write: each (row, 2 reals of one k); 32 rows x 64 reals
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int r = r0 + t;
    if (r >= rows) continue;
    for (int q = threadIdx.x; q < 64; q += 32) {
      const int kk = 2 * k0 + q;          // real column
      if (kk >= kp) continue;
      const int k = kk >> 1, part = kk & 1;
      float2 v = (k < K) ? tile[t][k - k0] : make_float2(0.f, 0.f);
      float a, b;
      if (!expand) {
        a = part ? v.y : v.x;
        b = 0.f;
      } else {   // rows 2r (Re, -Im) and 2r+1 (Im, Re)
        a = part ? -v.y : v.x;
        b = part ? v.x : v.y;
      }
      const long long o0 = inst * inst_elems + (long long)(expand ? 2 * r : r) * kp + kk;
      if constexpr (ESZ == 2) {
        __nv_bfloat16 h, l;
        split2(a, h, l);
        reinterpret_cast<__nv_bfloat16*>(hi_out)[o0] = h;
        reinterpret_cast<__nv_bfloat16*>(lo_out)[o0] = l;
        if (expand) {
          split2(b, h, l);
          reinterpret_cast<__nv_bfloat16*>(hi_out)[o0 + kp] = h;
          reinterpret_cast<__nv_bfloat16*>(lo_out)[o0 + kp] = l;
        }
      } else {
        float h, l;
        split4(a, h, l);
        reinterpret_cast<float*>(hi_out)[o0] = h;
        reinterpret_cast<float*>(lo_out)[o0] = l;
        if (expand) {
          split4(b, h, l);
          reinterpret_cast<float*>(hi_out)[o0 + kp] = h;
          reinterpret_cast<float*>(lo_out)[o0 + kp] = l;
        }
      }
    }
  }
}

// split-K reduction in a fixed order (partial 0 first), so that a product is
// the same bit for bit from run to run: C (+)= sum_s P[s][batch]
__global__ void splitk_reduce_kernel(const float2* __restrict__ P, int split, int nbatch, float2* C, int M, int N,
                                     long long ldc, long long s1, long long s2, int b2, int beta_one) {
  const int batch = blockIdx.z;
  float2* Cb = C + (long long)(batch / b2) * s1 + (long long)(batch % b2) * s2;
  const long long mn = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn;
       e += (long long)gridDim.x * blockDim.x) {
    float2 acc = P[(long long)batch * mn + e];
    for (int s = 1; s < split; ++s) {
      const float2 v = P[((long long)s * nbatch + batch) * mn + e];
      acc.x += v.x;
      acc.y += v.y;
    }
    float2* dst = Cb + (e / N) * ldc + (e % N);
    if (beta_one) {
      const float2 o = *dst;
      acc.x = o.x + acc.x;
      acc.y = o.y + acc.y;
    }
    *dst = acc;
  }
}

// ---- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* tm, int esz, void* base, int kp, int rows, int inst, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)inst};
  cuuint64_t strides[2] = {(cuuint64_t)kp * esz, (cuuint64_t)kp * esz * rows};
  cuuint32_t box[3] = {(cuuint32_t)(TC_ROW_BYTES / esz), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(tm, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

template <int ESZ>
cudaError_t run_tc(const GemmArgs& g, TcWork& w, int* err_dev, cudaStream_t st, int* launches) {
  const int esz = ESZ;
  const int align = 16 / esz;
  const int kp = ((2 * g.K + align - 1) / align) * align;
  // distinct operand instances along the two batch dimensions
  const int a1 = g.sA1 ? g.b1 : 1, a2 = g.sA2 ? g.b2 : 1;
  const int bb1 = g.sB1 ? g.b1 : 1, bb2 = g.sB2 ? g.b2 : 1;
  const long long instA = (long long)a1 * a2, instB = (long long)bb1 * bb2;
  if (instA > 65535 || instB > 65535) return cudaErrorInvalidValue;
  const size_t a_bytes = (size_t)instA * g.M * kp * esz;
  const size_t b_bytes = (size_t)instB * 2 * g.N * kp * esz;
  cudaError_t e;
  if ((e = w.ensure(0, a_bytes)) != cudaSuccess) return e;
  if ((e = w.ensure(1, a_bytes)) != cudaSuccess) return e;
  if ((e = w.ensure(2, b_bytes)) != cudaSuccess) return e;
  if ((e = w.ensure(3, b_bytes)) != cudaSuccess) return e;
  // pack A: rows m, K; source k-contiguous for op N / R
  {
    const bool kfast = (g.opA == OP_N || g.opA == OP_R);
    const bool cj = (g.opA == OP_C || g.opA == OP_R);
    dim3 grid((kp / 2 + 31) / 32, (g.M + 31) / 32, (unsigned)instA);
    pack_kernel<ESZ><<<grid, dim3(32, 8), 0, st>>>((const float2*)g.A, g.lda, g.sA1, g.sA2, kfast, cj, g.M, g.K, kp, 0,
                                                   0, a1, a2, w.buf[0], w.buf[1]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // pack B (expanded): rows n, K; source k-contiguous for op T / C
  {
    const bool kfast = (g.opB == OP_T || g.opB == OP_C);
    const bool cj = (g.opB == OP_C || g.opB == OP_R);
    dim3 grid((kp / 2 + 31) / 32, (g.N + 31) / 32, (unsigned)instB);
    pack_kernel<ESZ><<<grid, dim3(32, 8), 0, st>>>((const float2*)g.B, g.ldb, g.sB1, g.sB2, kfast, cj, g.N, g.K, kp, 1,
                                                   0, bb1, bb2, w.buf[2], w.buf[3]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  CUtensorMap tAh, tAl, tBh, tBl;
  if (!make_map(&tAh, esz, w.buf[0], kp, g.M, (int)instA, TC_BM) ||
      !make_map(&tAl, esz, w.buf[1], kp, g.M, (int)instA, TC_BM) ||
      !make_map(&tBh, esz, w.buf[2], kp, 2 * g.N, (int)instB, TC_BN) ||
      !make_map(&tBl, esz, w.buf[3], kp, 2 * g.N, (int)instB, TC_BN))
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = g.M; a.N = g.N;
  a.ktiles = (kp + (TC_ROW_BYTES / esz) - 1) / (TC_ROW_BYTES / esz);
  a.b1 = g.b1; a.b2 = g.b2;
  a.a_m1 = g.sA1 ? (g.sA2 ? g.b2 : 1) : 0; a.a_m2 = g.sA2 ? 1 : 0;
  a.b_m1 = g.sB1 ? (g.sB2 ? g.b2 : 1) : 0; a.b_m2 = g.sB2 ? 1 : 0;
  a.C = (float2*)g.C; a.ldc = g.ldc; a.sC1 = g.sC1; a.sC2 = g.sC2;
  a.alpha_re = (float)g.alpha_re; a.alpha_im = (float)g.alpha_im;
  a.err = err_dev;
  long long tiles = (long long)((2 * g.N + TC_BN - 1) / TC_BN) * ((g.M + TC_BM - 1) / TC_BM) * g.b1 * g.b2;
  const bool upper = g.upper_only && g.M == g.N && g.b1 * g.b2 == 1 && !g.beta_one;
  if (upper) {   // tiles on or above the diagonal only
    const long long tm = (g.M + TC_BM - 1) / TC_BM;
    tiles = tm * (tm + 1) / 2;
  }
  // split-K for grids of a few waves: one CTA per SM is resident (the ring
  // takes 192 KB of shared memory), so a grid of T tiles split s ways runs
  // ceil(T s / SMs) waves of K / s blocks each; take the s (<= 32, >= 4 K
  // blocks per split) with the fewest wave-blocks, preferring the smaller s
  // within 3% (each split adds a partial product to write and sum)
  int split = 1;
  const long long sms = sm_count();
  if (tiles < 4 * sms && a.ktiles >= 8) {
    double best = 1e300;
    const int smax = std::min(32, a.ktiles / 4);
    for (int sp = 1; sp <= smax; ++sp) {
      const long long waves = (tiles * sp + sms - 1) / sms;
      const double cost = (double)waves * (double)((a.ktiles + sp - 1) / sp);
      if (cost < 0.97 * best) { best = cost; split = sp; }
    }
  }
  if ((long long)g.b1 * g.b2 * split > 65535) split = 1;
  a.per = (a.ktiles + split - 1) / split;
  split = (a.ktiles + a.per - 1) / a.per;   // every split owns at least one K block
  a.split = split;
  a.mode = split > 1 ? 2 : (g.beta_one ? 1 : 0);
  a.upper = upper ? 1 : 0;
  const int nbatch = g.b1 * g.b2;
  if (split > 1) {
    if ((e = w.ensure(4, (size_t)split * nbatch * g.M * g.N * sizeof(float2))) != cudaSuccess) return e;
    a.P = (float2*)w.buf[4];
  }
  if (launches) *launches = 3 + (split > 1 ? 1 : 0);
  if ((e = allow_dyn_smem((const void*)tc_gemm_kernel<ESZ>)) != cudaSuccess) return e;
  a.tiles_n = (2 * g.N + TC_BN - 1) / TC_BN;
  a.tiles_m = (g.M + TC_BM - 1) / TC_BM;
  a.total = (upper ? (long long)a.tiles_m * (a.tiles_m + 1) / 2 : (long long)a.tiles_n * a.tiles_m) *
            nbatch * split;
  const long long ctas = std::min<long long>(a.total, (long long)sm_count());
  tc_gemm_kernel<ESZ><<<(unsigned)ctas, TC_THREADS, TC_SMEM_BYTES, st>>>(tAh, tAl, tBh, tBl, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (split > 1) {
    const long long mn = (long long)g.M * g.N;
    int bx = (int)std::min<long long>((mn + 255) / 256, 1024);
    dim3 rg(bx < 1 ? 1 : bx, 1, (unsigned)nbatch);
    splitk_reduce_kernel<<<rg, 256, 0, st>>>(a.P, split, nbatch, (float2*)g.C, g.M, g.N, g.ldc, g.sC1, g.sC2, g.b2,
                                             g.beta_one);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

cudaError_t TcWork::ensure(int i, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (cap[i] >= bytes) return cudaSuccess;
  if (buf[i]) {
    cudaDeviceSynchronize();
    cudaFree(buf[i]);
    buf[i] = nullptr;
    cap[i] = 0;
  }
  cudaError_t e = cudaMalloc(&buf[i], bytes + bytes / 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    buf[i] = nullptr;
    return e;
  }
  cap[i] = bytes + bytes / 8;
  return cudaSuccess;
}

void TcWork::release() {
  for (int i = 0; i < 5; ++i) {
    if (buf[i]) cudaFree(buf[i]);
    buf[i] = nullptr;
    cap[i] = 0;
  }
}

cudaError_t gemm_tc(const GemmArgs& g, int precision, TcWork& w, int* err_dev, cudaStream_t st, int* launches) {
  if (launches) *launches = 0;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.b1 <= 0 || g.b2 <= 0) return cudaSuccess;
  if (precision == DMRGC_BF16X3) return run_tc<2>(g, w, err_dev, st, launches);
  if (precision == DMRGC_TF32X3) return run_tc<4>(g, w, err_dev, st, launches);
  return cudaErrorInvalidValue;
}

}  // namespace dmrgc
