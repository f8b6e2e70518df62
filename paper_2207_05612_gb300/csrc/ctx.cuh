// Host-side context of the compression step and the helpers shared by the
// translation units that orchestrate it (api.cu: the two-site sweep, the
// read-outs and the C ABI; single_site.cu: the single-site sweep over
// grouped qubits, Sec. IV.B.1).
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace dmrgc_host {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct EnvRef {
  const void* p = nullptr;
  int a = 1, w = 1, b = 1;   // [a][w][b]
};

enum TimeClass { TC_GEMM = 0, TC_SVD = 1, TC_MPO = 2, TC_OTHER = 3 };

}  // namespace dmrgc_host

using dmrgc::GemmArgs;
using dmrgc::TcWork;
using dmrgc::TruncResult;
using dmrgc_host::DevBuf;
using dmrgc_host::EnvRef;

struct dmrgc_ctx {
  int N = 0, chi = 0, rows = 0, cols = 0, m = 0;
  dmrgc_options opt{};
  cudaStream_t st = nullptr;
  bool fp64 = true;
  size_t esz = 16;
  double sweep_cut = 1e-12, zip_cut = 1e-5, zero_rel = 1e-13, tie_rel = 1e-10;
  int max_jsweeps = 40;
  std::vector<int> order, site_of;
  std::vector<DevBuf> A, B, Wx, Wy, XY, E;
  std::vector<DevBuf> Wc;   // layer MPO in [w_in][s][t][w_out] while it is compressed
  std::vector<int> chiA, chiB, D;     // N+1 entries each
  std::vector<char> xyk;
  DevBuf envL, envR, T, theta, jw, bt, one, jctl, tres, scal, gates_d, rank_d, fa_d, fb_d, plan_d;
  DevBuf ptrs_d, bonds_d, order_d, bits_d, out_d, stage_d, tcerr;
  DevBuf ovl[2];   // ping-pong environments of dmrgc_overlap (never the sweep's envL / envR)
  DevBuf ework;    // work space of the Gram eigensolver path (eig_truncate)
  TruncResult last_tr{};          // result of the last truncated SVD (either path)
  std::vector<char> eig_ok;       // per bond: the last SVD there was resolvable by the eigensolver
  DevBuf rv[3];    // read-outs: running rows V, site products W = V A_i, T = W E_i
  TcWork tcw;
  // randomized SVD and the rank model (svd_mode 1, 2)
  DevBuf rs_om, rs_y, rs_q, rs_b, rs_h, rs_w, feat, mlp_w, mlp_out, lab;
  int layer_no = 0;
  std::vector<int> visit_layer;   // per bond: layer of the last update there (-1 none)
  std::vector<int> kprev;         // per bond: kept rank at the last update (0 = none)
  unsigned long long rs_ctr = 0;  // counter of the sketch random stream
  double rs_tol = 1e-6;
  int rs_p = 8, rs_pow = 1;
  bool mlp_ready = false;
  std::vector<float> rec_x, rec_y;   // logged (features, label) records
  EnvRef L, R;
  int phase = 0;           // 0 created, 1 guess ready / sweeping
  int bond = 0, dir = -1;  // next update (bond, bond+1), dir -1 = right-to-left
  int centre = 0;
  double log_ft = 0.0, f_cur = 1.0;
  std::vector<double> hist;
  std::string err;
  dmrgc_stats stats{};
  struct Pend { int cls; cudaEvent_t a, b; double flops; };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> pool;
  // single-site variant over grouped qubits (ng > 0; Sec. IV.A, IV.B.1):
  // tensor tau holds the gsize[tau] sites from gstart[tau] on; A, B, chiA,
  // chiB then index tensors and cuts between them (ng + 1 cuts)
  int ng = 0;
  std::vector<int> gsize, gstart;
  std::vector<DevBuf> GL, GR;     // environments at every cut: L_tau [a][w][b], R_tau [c][w][b]
  DevBuf gx[2], gf;               // X / R-chain ping-pong buffers, F (then M) of the update
  int gsweep = 0, gtau = 0;       // sweeps finished in this layer, next tensor
  ~dmrgc_ctx();
};

namespace dmrgc_host {

dmrgc_status fail(dmrgc_ctx* c, dmrgc_status s, const std::string& msg);
dmrgc_status ensure(dmrgc_ctx* c, DevBuf& b, size_t bytes);
cudaEvent_t take_event(dmrgc_ctx* c);
dmrgc_status sync(dmrgc_ctx* c);
// one (batched) complex GEMM on the context's stream; precision < 0: the context's
dmrgc_status gemm(dmrgc_ctx* c, const GemmArgs& g, int precision = -1);
// f = |A|^2 of a block just formed, then A /= sqrt(f)
dmrgc_status normalise_block(dmrgc_ctx* c, void* A, long long elems, double& f);
// Jacobi SVD of the columns of c->jw (or W): m x n column-major; k kept, f their weight
dmrgc_status svd_columns(dmrgc_ctx* c, int m, int n, double rel_cut, bool squared, double tie_rel, int& k,
                         double& f, int* nnz = nullptr, double* norm2 = nullptr, void* W = nullptr,
                         int chi_cap = -1);

// timing span of one class of device work (CUDA events on the context's stream)
// NVTX range for the span of a host call (named in profilers and ncu's
// --nvtx filters; without an attached tool the push and pop do nothing)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

struct Span {
  dmrgc_ctx* c;
  int cls;
  double flops;
  cudaEvent_t a = nullptr;
  Span(dmrgc_ctx* c_, int cls_, double flops_ = 0) : c(c_), cls(cls_), flops(flops_) {
    static const char* const kName[] = {"contraction", "truncated SVD", "layer MPO", "other"};
    nvtxRangePushA(kName[cls & 3]);
    if (c->opt.timing) {
      a = take_event(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~Span() {
    if (c->opt.timing) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->st);
      c->pend.push_back({cls, a, b, flops});
    }
    nvtxRangePop();
  }
  Span(const Span&) = delete;
  Span& operator=(const Span&) = delete;
};

// single_site.cu: the random guess of a layer in orthogonal form, and sweeps
dmrgc_status grouped_guess(dmrgc_ctx* c);
dmrgc_status grouped_sweeps(dmrgc_ctx* c, int n_sweeps);

}  // namespace dmrgc_host

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess)                                                             \
      return dmrgc_host::fail(c, DMRGC_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)                          \
  do {                                  \
    dmrgc_status s_ = (x);              \
    if (s_ != DMRGC_OK) return s_;      \
  } while (0)
