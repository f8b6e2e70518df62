// Rank model: a three-layer perceptron x (36) -> 128 -> 128 -> 1 with ReLU,
// trained on the GPU with hand-written FP32 kernels (forward, backward, Adam)
// and evaluated with BF16 weights and FP32 accumulation inside the sweep.
//
// Not part of the paper's method: it predicts the sketch rank of the
// randomized SVD (svd_mode 2).  Every reduction is a fixed-order loop (no
// atomics), so training is deterministic for a given seed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dmrgc {
namespace {

constexpr int IN = DMRGC_MLP_IN, HID = DMRGC_MLP_HIDDEN, NPAR = DMRGC_MLP_PARAMS;
constexpr int O_W1 = 0, O_B1 = O_W1 + HID * IN, O_W2 = O_B1 + HID, O_B2 = O_W2 + HID * HID,
              O_W3 = O_B2 + HID, O_B3 = O_W3 + HID;
static_assert(O_B3 + 1 == NPAR, "parameter layout");

// Y[b][o] = act(bias[o] + sum_i W[o][i] X[row(b)][i]); one CTA per row, `out` threads
__global__ void dense_fwd_kernel(const float* __restrict__ X, const int* __restrict__ rows, int in,
                                 const float* __restrict__ W, const float* __restrict__ bias, int out,
                                 float* __restrict__ Y, int relu) {
  __shared__ float x[HID];
  const int b = blockIdx.x;
  const long long r = rows ? rows[b] : b;
  for (int i = threadIdx.x; i < in; i += blockDim.x) x[i] = X[r * in + i];
  __syncthreads();
  const int o = threadIdx.x;
  if (o < out) {
    float acc = bias[o];
    const float* w = W + (size_t)o * in;
    for (int i = 0; i < in; ++i) acc = fmaf(w[i], x[i], acc);
    Y[(size_t)b * out + o] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

// y[b] = w3 . H[b] + b3; with targets: dy[b] = 2 (y - t) / B and sq[b] = (y - t)^2
__global__ void out_fwd_kernel(const float* __restrict__ H, const float* __restrict__ w3,
                               const float* __restrict__ b3, const float* __restrict__ T,
                               const int* __restrict__ rows, int B, float* __restrict__ y,
                               float* __restrict__ dy, float* __restrict__ sq) {
  const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  float acc = 0.f;
  for (int o = lane; o < HID; o += 32) acc = fmaf(w3[o], H[(size_t)b * HID + o], acc);
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) {
    const float v = acc + *b3;
    y[b] = v;
    if (T) {
      const float t = T[rows ? rows[b] : b];
      dy[b] = 2.f * (v - t) / (float)B;
      sq[b] = (v - t) * (v - t);
    }
  }
}

// dIn[b][i] = [Hin[b][i] > 0] * sum_o dOut[b][o] W[o][i]; one CTA per row
__global__ void dense_bwd_input_kernel(const float* __restrict__ dOut, int out, const float* __restrict__ W,
                                       int in, const float* __restrict__ Hin, float* __restrict__ dIn) {
  __shared__ float d[HID];
  const int b = blockIdx.x;
  for (int o = threadIdx.x; o < out; o += blockDim.x) d[o] = dOut[(size_t)b * out + o];
  __syncthreads();
  const int i = threadIdx.x;
  if (i < in) {
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc = fmaf(d[o], W[(size_t)o * in + i], acc);
    dIn[(size_t)b * in + i] = Hin[(size_t)b * in + i] > 0.f ? acc : 0.f;
  }
}

// dW[o][i] = sum_b dOut[b][o] X[row(b)][i], db[o] = sum_b dOut[b][o]; one CTA per o
__global__ void dense_bwd_weight_kernel(const float* __restrict__ dOut, int out, const float* __restrict__ X,
                                        const int* __restrict__ rows, int in, int B, float* __restrict__ dW,
                                        float* __restrict__ db) {
  const int o = blockIdx.x;
  const int i = threadIdx.x;
  float acc = 0.f, accb = 0.f;
  for (int b = 0; b < B; ++b) {
    const float g = dOut[(size_t)b * out + o];
    const long long r = rows ? rows[b] : b;
    if (i < in) acc = fmaf(g, X[r * in + i], acc);
    accb += g;
  }
  if (i < in) dW[(size_t)o * in + i] = acc;
  if (i == 0) db[o] = accb;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float beta1, float beta2, float eps,
                            float bc1, float bc2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float gj = g[j];
  const float mj = beta1 * m[j] + (1.f - beta1) * gj;
  const float vj = beta2 * v[j] + (1.f - beta2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  p[j] -= lr * (mj / bc1) / (sqrtf(vj / bc2) + eps);
}

// acc[slot] += sum_b sq[b] / B (one thread, fixed order)
__global__ void loss_accum_kernel(const float* __restrict__ sq, int B, double* __restrict__ acc, int slot) {
  double s = 0;
  for (int b = 0; b < B; ++b) s += sq[b];
  acc[slot] += s / B;
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ out, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = __float2bfloat16_rn(w[j]);
}

// Inference with BF16 parameters, FP32 accumulation; one CTA (HID threads) per row.
// x: rows of IN floats, or (one row) 32 device floats + 4 extras.
__global__ void infer_bf16_kernel(const __nv_bfloat16* __restrict__ w, const float* __restrict__ X,
                                  float4 extra, int use_extra, float* __restrict__ y) {
  __shared__ float x[IN];
  __shared__ float h1[HID];
  __shared__ float part[HID / 32];
  const int b = blockIdx.x, t = threadIdx.x;
  if (use_extra) {
    if (t < 32) x[t] = X[t];
    if (t == 32) x[32] = extra.x;
    if (t == 33) x[33] = extra.y;
    if (t == 34) x[34] = extra.z;
    if (t == 35) x[35] = extra.w;
  } else if (t < IN) {
    x[t] = X[(size_t)b * IN + t];
  }
  __syncthreads();
  float a = __bfloat162float(w[O_B1 + t]);
  for (int i = 0; i < IN; ++i) a = fmaf(__bfloat162float(w[O_W1 + t * IN + i]), x[i], a);
  h1[t] = fmaxf(a, 0.f);
  __syncthreads();
  a = __bfloat162float(w[O_B2 + t]);
  for (int i = 0; i < HID; ++i) a = fmaf(__bfloat162float(w[O_W2 + t * HID + i]), h1[i], a);
  float v = fmaxf(a, 0.f) * __bfloat162float(w[O_W3 + t]);
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  if ((t & 31) == 0) part[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    float s = __bfloat162float(w[O_B3]);
    for (int k = 0; k < HID / 32; ++k) s += part[k];
    y[b] = s;
  }
}

struct Dev {
  std::vector<void*> ptrs;
  ~Dev() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

// SplitMix64 (Steele, Lea, Flood 2014)
unsigned long long mix64(unsigned long long& state) {
  unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double mix_unit(unsigned long long& state) { return (double)(mix64(state) >> 11) * (1.0 / 9007199254740992.0); }

// Forward and backward of one batch of B rows (row indices `rows`, or the first
// B rows); gradients into g.  Returns the first CUDA error.
cudaError_t fwd_bwd(const float* par, const float* X, const float* T, const int* rows, int B, float* H1,
                    float* H2, float* y, float* dy, float* sq, float* dH2, float* dH1, float* g, cudaStream_t st) {
  dense_fwd_kernel<<<B, HID, 0, st>>>(X, rows, IN, par + O_W1, par + O_B1, HID, H1, 1);
  dense_fwd_kernel<<<B, HID, 0, st>>>(H1, nullptr, HID, par + O_W2, par + O_B2, HID, H2, 1);
  out_fwd_kernel<<<(B + 7) / 8, 256, 0, st>>>(H2, par + O_W3, par + O_B3, T, rows, B, y, dy, sq);
  dense_bwd_weight_kernel<<<1, HID, 0, st>>>(dy, 1, H2, nullptr, HID, B, g + O_W3, g + O_B3);
  dense_bwd_input_kernel<<<B, HID, 0, st>>>(dy, 1, par + O_W3, HID, H2, dH2);
  dense_bwd_weight_kernel<<<HID, HID, 0, st>>>(dH2, HID, H1, nullptr, HID, B, g + O_W2, g + O_B2);
  dense_bwd_input_kernel<<<B, HID, 0, st>>>(dH2, HID, par + O_W2, HID, H1, dH1);
  dense_bwd_weight_kernel<<<HID, HID, 0, st>>>(dH1, HID, X, rows, IN, B, g + O_W1, g + O_B1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_to_bf16(const float* params_dev, void* out_bf16, cudaStream_t st) {
  to_bf16_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(params_dev, static_cast<__nv_bfloat16*>(out_bf16), NPAR);
  return cudaGetLastError();
}

cudaError_t mlp_infer_one(const void* w_bf16, const float* feat32, const float* extras, float* y,
                          cudaStream_t st) {
  const float4 e = make_float4(extras[0], extras[1], extras[2], extras[3]);
  infer_bf16_kernel<<<1, HID, 0, st>>>(static_cast<const __nv_bfloat16*>(w_bf16), feat32, e, 1, y);
  return cudaGetLastError();
}

}  // namespace dmrgc

using namespace dmrgc;

extern "C" {

dmrgc_status dmrgc_mlp_loss_grad(const float* params, const float* x, const float* y, int n, float* loss,
                                 float* grad) {
  if (!params || !x || !y || !loss || !grad || n < 1 || n > (1 << 24)) return DMRGC_EINVAL;
  Dev d;
  float *par = d.get<float>(NPAR), *X = d.get<float>((size_t)n * IN), *T = d.get<float>(n);
  float *H1 = d.get<float>((size_t)n * HID), *H2 = d.get<float>((size_t)n * HID), *yy = d.get<float>(n);
  float *dy = d.get<float>(n), *sq = d.get<float>(n), *dH2 = d.get<float>((size_t)n * HID);
  float *dH1 = d.get<float>((size_t)n * HID), *g = d.get<float>(NPAR);
  double* acc = d.get<double>(1);
  if (!par || !X || !T || !H1 || !H2 || !yy || !dy || !sq || !dH2 || !dH1 || !g || !acc) return DMRGC_ENOMEM;
  cudaError_t e = cudaMemcpy(par, params, NPAR * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(X, x, (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(T, y, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(acc, 0, sizeof(double));
  if (e == cudaSuccess) e = fwd_bwd(par, X, T, nullptr, n, H1, H2, yy, dy, sq, dH2, dH1, g, 0);
  if (e == cudaSuccess) {
    loss_accum_kernel<<<1, 1, 0, 0>>>(sq, n, acc, 0);
    e = cudaGetLastError();
  }
  double l = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&l, acc, sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(grad, g, NPAR * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return DMRGC_ECUDA;
  *loss = (float)l;
  return DMRGC_OK;
}

dmrgc_status dmrgc_mlp_predict(const float* params, const float* x, int n, int bf16, float* y_out) {
  if (!params || !x || !y_out || n < 1 || n > (1 << 24)) return DMRGC_EINVAL;
  Dev d;
  float *par = d.get<float>(NPAR), *X = d.get<float>((size_t)n * IN), *yy = d.get<float>(n);
  float *H1 = d.get<float>((size_t)n * HID), *H2 = d.get<float>((size_t)n * HID);
  __nv_bfloat16* wb = d.get<__nv_bfloat16>(NPAR);
  if (!par || !X || !yy || !H1 || !H2 || !wb) return DMRGC_ENOMEM;
  cudaError_t e = cudaMemcpy(par, params, NPAR * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(X, x, (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (bf16) {
      e = mlp_to_bf16(par, wb, 0);
      if (e == cudaSuccess) {
        infer_bf16_kernel<<<n, HID, 0, 0>>>(wb, X, make_float4(0, 0, 0, 0), 0, yy);
        e = cudaGetLastError();
      }
    } else {
      dense_fwd_kernel<<<n, HID, 0, 0>>>(X, nullptr, IN, par + O_W1, par + O_B1, HID, H1, 1);
      dense_fwd_kernel<<<n, HID, 0, 0>>>(H1, nullptr, HID, par + O_W2, par + O_B2, HID, H2, 1);
      out_fwd_kernel<<<(n + 7) / 8, 256, 0, 0>>>(H2, par + O_W3, par + O_B3, nullptr, nullptr, n, yy,
                                                 nullptr, nullptr);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(y_out, yy, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DMRGC_OK : DMRGC_ECUDA;
}

dmrgc_status dmrgc_mlp_train(const float* x, const float* y, int n, int epochs, int batch, float lr,
                             unsigned long long seed, float* params_out, float* epoch_loss) {
  if (!x || !y || !params_out || n < 2 || n > (1 << 24) || epochs < 1 || epochs > 100000 || batch < 1 ||
      batch > 4096 || !(lr > 0.f))
    return DMRGC_EINVAL;
  // standardise inputs and labels (folded back into the first and last layers)
  std::vector<double> mu(IN, 0.0), sd(IN, 0.0);
  double my = 0, sy = 0;
  for (int r = 0; r < n; ++r) {
    for (int i = 0; i < IN; ++i) mu[i] += x[(size_t)r * IN + i];
    my += y[r];
  }
  for (int i = 0; i < IN; ++i) mu[i] /= n;
  my /= n;
  for (int r = 0; r < n; ++r) {
    for (int i = 0; i < IN; ++i) {
      const double v = x[(size_t)r * IN + i] - mu[i];
      sd[i] += v * v;
    }
    sy += (y[r] - my) * (y[r] - my);
  }
  for (int i = 0; i < IN; ++i) sd[i] = std::max(std::sqrt(sd[i] / n), 1e-3);
  sy = std::max(std::sqrt(sy / n), 1e-3);
  std::vector<float> xs((size_t)n * IN), ys(n);
  for (int r = 0; r < n; ++r) {
    for (int i = 0; i < IN; ++i) xs[(size_t)r * IN + i] = (float)((x[(size_t)r * IN + i] - mu[i]) / sd[i]);
    ys[r] = (float)((y[r] - my) / sy);
  }
  // He-uniform initialisation, zero biases
  std::vector<float> p0(NPAR, 0.f);
  unsigned long long rs = seed;
  auto init = [&](int off, int rows, int fan_in) {
    const double a = std::sqrt(6.0 / fan_in);
    for (int j = 0; j < rows * fan_in; ++j) p0[off + j] = (float)((2.0 * mix_unit(rs) - 1.0) * a);
  };
  init(O_W1, HID, IN);
  init(O_W2, HID, HID);
  init(O_W3, 1, HID);
  const int B = std::min(batch, n);
  Dev d;
  float *par = d.get<float>(NPAR), *X = d.get<float>((size_t)n * IN), *T = d.get<float>(n);
  float *H1 = d.get<float>((size_t)B * HID), *H2 = d.get<float>((size_t)B * HID), *yy = d.get<float>(B);
  float *dy = d.get<float>(B), *sq = d.get<float>(B), *dH2 = d.get<float>((size_t)B * HID);
  float *dH1 = d.get<float>((size_t)B * HID), *g = d.get<float>(NPAR), *m = d.get<float>(NPAR);
  float* v = d.get<float>(NPAR);
  int* idx = d.get<int>(n);
  double* acc = d.get<double>(epochs);
  if (!par || !X || !T || !H1 || !H2 || !yy || !dy || !sq || !dH2 || !dH1 || !g || !m || !v || !idx || !acc)
    return DMRGC_ENOMEM;
  cudaError_t e = cudaMemcpy(par, p0.data(), NPAR * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(X, xs.data(), (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(T, ys.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m, 0, NPAR * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(v, 0, NPAR * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(acc, 0, epochs * sizeof(double));
  std::vector<int> perm(n);
  const int nb = (n + B - 1) / B;
  long long step = 0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int r = 0; r < n; ++r) perm[r] = r;
    for (int r = n - 1; r > 0; --r) {   // Fisher-Yates
      const int j = (int)(mix64(rs) % (unsigned long long)(r + 1));
      std::swap(perm[r], perm[j]);
    }
    e = cudaMemcpy(idx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice);
    for (int bi = 0; bi < nb && e == cudaSuccess; ++bi) {
      const int b0 = bi * B, bb = std::min(B, n - b0);
      e = fwd_bwd(par, X, T, idx + b0, bb, H1, H2, yy, dy, sq, dH2, dH1, g, 0);
      if (e != cudaSuccess) break;
      loss_accum_kernel<<<1, 1, 0, 0>>>(sq, bb, acc, ep);
      ++step;
      const float bc1 = 1.f - (float)std::pow(0.9, (double)step);
      const float bc2 = 1.f - (float)std::pow(0.999, (double)step);
      adam_kernel<<<(NPAR + 255) / 256, 256, 0, 0>>>(par, g, m, v, NPAR, lr, 0.9f, 0.999f, 1e-8f, bc1, bc2);
      e = cudaGetLastError();
    }
  }
  std::vector<float> p(NPAR);
  std::vector<double> el(epochs);
  if (e == cudaSuccess) e = cudaMemcpy(p.data(), par, NPAR * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(el.data(), acc, epochs * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return DMRGC_ECUDA;
  if (epoch_loss)
    for (int ep = 0; ep < epochs; ++ep) epoch_loss[ep] = (float)(el[ep] / nb);
  // fold the standardisation: W1' = W1 / sd, b1' = b1 - W1' mu; w3' = sy w3, b3' = sy b3 + my
  for (int o = 0; o < HID; ++o) {
    double shift = 0;
    for (int i = 0; i < IN; ++i) {
      const double w = p[O_W1 + o * IN + i] / sd[i];
      p[O_W1 + o * IN + i] = (float)w;
      shift += w * mu[i];
    }
    p[O_B1 + o] = (float)(p[O_B1 + o] - shift);
    p[O_W3 + o] = (float)(p[O_W3 + o] * sy);
  }
  p[O_B3] = (float)(p[O_B3] * sy + my);
  std::copy(p.begin(), p.end(), params_out);
  return DMRGC_OK;
}

}  // extern "C"
