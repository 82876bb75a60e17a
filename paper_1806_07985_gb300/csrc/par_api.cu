// Par-NNCP (Alg. 2; Sec. IV-C): the per-processor side of NNCP over a
// P_1 x ... x P_N processor grid.  This file is the local computation of one
// grid position -- its block of the tensor, its rows of the factors, the
// redundant Grams and lambda -- between the collectives, which the caller runs
// (Reduce-Scatter of M(n) and All-Gather of H(n) over the mode-n processor
// slice, All-Reduce of the Gram and <M, W> partials over every processor).
//
// Data distribution (Sec. IV-C "Data Distribution"): mode n is cut into P_n
// contiguous blocks, block k = [floor(k I_n / P_n), floor((k+1) I_n / P_n));
// processor p holds the tensor block of its coordinates, and the block p_n of
// every factor redundantly with the rest of its mode-n slice.  Within that
// block the rows are cut again into P / P_n contiguous pieces, one per slice
// member in the order of its other coordinates (mode 1 fastest): the rows it
// owns, updates and contributes to the Gram.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/nncp.h"
#include "nncp_internal.cuh"

using namespace nncp;

struct nncp_par {
  int N = 0, R = 0, P = 1;
  int64_t dims[kMaxModes] = {};
  int grid[kMaxModes] = {};
  int coords[kMaxModes] = {};
  int64_t block_lo[kMaxModes] = {}, block_rows[kMaxModes] = {};
  int64_t owned_lo[kMaxModes] = {}, owned_rows[kMaxModes] = {};
  int slice_index[kMaxModes] = {}, slice_size[kMaxModes] = {};
  int precision = NNCP_FP32_SIMT;
  nncp_ctx* ctx = nullptr;  // the local tensor block and its dimension tree
  cudaStream_t stream = nullptr;
  // device scratch (in the caller's workspace after the context's)
  char* ws = nullptr;
  size_t ctx_bytes = 0, total = 0;
  float* S32 = nullptr;      // R x R
  double* lam_dev = nullptr; // R
  double* gram = nullptr;    // blocks x (R*R + 1)
  int* flags = nullptr;      // 16, zero
  float* inv = nullptr;      // R
  double* red = nullptr;     // kRedParts + 1: partial sums of ||X_p||^2, then the total
  int max_blocks = 0;
  double* host_part = nullptr;  // pinned, blocks x (R*R + 1)
  float* host_small = nullptr;  // pinned, R*R + R floats
  // redundant float64 state
  std::vector<double> G;    // N x R x R
  std::vector<double> lam;  // R
  std::vector<double> fits;
  double alpha = 0.0, tol = 0.0;
  bool begun = false, stop = false;
  std::string err;
};

namespace {

nncp_status pfail(nncp_par* p, nncp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (p) p->err = buf;
  record_global_error(buf);
  return s;
}

#define PCK(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return pfail(p, NNCP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

constexpr int kRedParts = 1024;

// S = Hadamard of every Gram but mode n's (Alg. 2, Hadamard line), float64
void hadamard_except(const nncp_par* p, int n, double* S) {
  const int R2 = p->R * p->R;
  for (int e = 0; e < R2; ++e) S[e] = 1.0;
  for (int k = 0; k < p->N; ++k)
    if (k != n)
      for (int e = 0; e < R2; ++e) S[e] *= p->G[(size_t)k * R2 + e];
}

}  // namespace

extern "C" {

nncp_status nncp_par_create(int N, const int64_t* dims, const int* grid, const int* coords, int R,
                            nncp_precision precision, nncp_par** out) {
  if (!out) return pfail(nullptr, NNCP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 2 || N > kMaxModes || !dims || !grid || !coords)
    return pfail(nullptr, NNCP_ERR_INVALID_ARG, "N=%d not in [2,8] or a null array", N);
  if (R < 1 || R > kMaxRank) return pfail(nullptr, NNCP_ERR_INVALID_ARG, "R=%d not in [1,128]", R);
  nncp_par* p = new (std::nothrow) nncp_par();
  if (!p) return pfail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "host allocation failed");
  p->N = N;
  p->R = R;
  p->precision = precision;
  int64_t P = 1;
  for (int n = 0; n < N; ++n) {
    if (grid[n] < 1 || coords[n] < 0 || coords[n] >= grid[n] || dims[n] < grid[n]) {
      delete p;
      return pfail(nullptr, NNCP_ERR_INVALID_ARG,
                   "mode %d: need 1 <= P_n <= I_n and 0 <= p_n < P_n (I=%lld P=%d p=%d)", n + 1,
                   (long long)dims[n], grid[n], coords[n]);
    }
    p->dims[n] = dims[n];
    p->grid[n] = grid[n];
    p->coords[n] = coords[n];
    P *= grid[n];
  }
  if (P > (1 << 20)) {
    delete p;
    return pfail(nullptr, NNCP_ERR_INVALID_ARG, "more than 2^20 processors");
  }
  p->P = (int)P;
  int64_t local[kMaxModes];
  for (int n = 0; n < N; ++n) {
    const int64_t I = dims[n];
    p->block_lo[n] = coords[n] * I / grid[n];
    p->block_rows[n] = (coords[n] + 1) * I / grid[n] - p->block_lo[n];
    local[n] = p->block_rows[n];
    // position within the mode-n slice: the other coordinates, mode 1 fastest
    int q = 0, Q = 1;
    for (int k = 0; k < N; ++k)
      if (k != n) {
        q += coords[k] * Q;
        Q *= grid[k];
      }
    p->slice_index[n] = q;
    p->slice_size[n] = Q;
    const int64_t L = p->block_rows[n];
    p->owned_lo[n] = p->block_lo[n] + q * L / Q;
    p->owned_rows[n] = (q + 1) * L / Q - q * L / Q;
  }
  nncp_status s = nncp_create(N, local, R, &p->ctx);
  if (s == NNCP_OK) s = nncp_set_options(p->ctx, precision, 0, nullptr);
  if (s != NNCP_OK) {
    p->err = nncp_last_error(p->ctx);
    nncp_destroy(p->ctx);
    delete p;
    return s;
  }
  size_t cb = 0;
  nncp_workspace_size(p->ctx, &cb);
  int64_t maxo = 1;
  for (int n = 0; n < N; ++n) maxo = std::max(maxo, p->owned_rows[n]);
  p->max_blocks = hals_gram_blocks(maxo);
  const int R2 = R * R;
  p->ctx_bytes = al256(cb);
  p->total = p->ctx_bytes + al256((size_t)R2 * 4) + al256((size_t)R * 8) +
             al256((size_t)p->max_blocks * (R2 + 1) * 8) + al256(16 * 4) + al256((size_t)R * 4) +
             al256((kRedParts + 1) * 8);
  if (cudaMallocHost(reinterpret_cast<void**>(&p->host_part),
                     (size_t)p->max_blocks * (R2 + 1) * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&p->host_small), (size_t)(R2 + R) * sizeof(float)) !=
          cudaSuccess) {
    nncp_destroy(p->ctx);
    if (p->host_part) cudaFreeHost(p->host_part);
    delete p;
    return pfail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "pinned host buffers");
  }
  p->G.assign((size_t)N * R2, 0.0);
  p->lam.assign(R, 1.0);
  *out = p;
  return NNCP_OK;
}

nncp_status nncp_par_layout(const nncp_par* p, int mode, int64_t* block_lo, int64_t* block_rows,
                            int64_t* owned_lo, int64_t* owned_rows, int* slice_index,
                            int* slice_size) {
  if (!p || mode < 1 || mode > p->N)
    return pfail(const_cast<nncp_par*>(p), NNCP_ERR_INVALID_ARG, "null par or mode out of range");
  const int n = mode - 1;
  if (block_lo) *block_lo = p->block_lo[n];
  if (block_rows) *block_rows = p->block_rows[n];
  if (owned_lo) *owned_lo = p->owned_lo[n];
  if (owned_rows) *owned_rows = p->owned_rows[n];
  if (slice_index) *slice_index = p->slice_index[n];
  if (slice_size) *slice_size = p->slice_size[n];
  return NNCP_OK;
}

nncp_status nncp_par_workspace_size(const nncp_par* p, size_t* bytes) {
  if (!p || !bytes) return pfail(nullptr, NNCP_ERR_INVALID_ARG, "null argument");
  *bytes = p->total;
  return NNCP_OK;
}

nncp_status nncp_par_set_workspace(nncp_par* p, void* dev_ptr, size_t bytes, void* stream) {
  if (!p) return pfail(nullptr, NNCP_ERR_INVALID_ARG, "null par");
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255) || bytes < p->total)
    return pfail(p, NNCP_ERR_INVALID_ARG, "workspace: 256-byte aligned, at least %zu bytes",
                 p->total);
  p->stream = static_cast<cudaStream_t>(stream);
  nncp_status s = nncp_set_options(p->ctx, p->precision, 0, stream);
  if (s == NNCP_OK) s = nncp_set_workspace(p->ctx, dev_ptr, p->ctx_bytes);
  if (s != NNCP_OK) return pfail(p, s, "%s", nncp_last_error(p->ctx));
  const int R = p->R, R2 = R * R;
  char* w = static_cast<char*>(dev_ptr) + p->ctx_bytes;
  p->S32 = reinterpret_cast<float*>(w);
  w += al256((size_t)R2 * 4);
  p->lam_dev = reinterpret_cast<double*>(w);
  w += al256((size_t)R * 8);
  p->gram = reinterpret_cast<double*>(w);
  w += al256((size_t)p->max_blocks * (R2 + 1) * 8);
  p->flags = reinterpret_cast<int*>(w);
  w += al256(16 * 4);
  p->inv = reinterpret_cast<float*>(w);
  w += al256((size_t)R * 4);
  p->red = reinterpret_cast<double*>(w);
  PCK(cudaMemsetAsync(p->flags, 0, 16 * sizeof(int), p->stream));
  p->ws = static_cast<char*>(dev_ptr);
  return NNCP_OK;
}

nncp_status nncp_par_set_data(nncp_par* p, const float* X_local, float* const* H_block) {
  if (!p || !X_local || !H_block) return pfail(p, NNCP_ERR_INVALID_ARG, "null argument");
  if (!p->ws) return pfail(p, NNCP_ERR_INVALID_ARG, "workspace not set");
  nncp_status s = nncp_set_tensor(p->ctx, X_local);
  if (s == NNCP_OK) s = nncp_set_factors(p->ctx, H_block);
  if (s != NNCP_OK) return pfail(p, s, "%s", nncp_last_error(p->ctx));
  p->begun = false;
  return NNCP_OK;
}

nncp_status nncp_par_alpha_local(nncp_par* p, const float* X_local, double* local) {
  if (!p || !X_local || !local) return pfail(p, NNCP_ERR_INVALID_ARG, "null argument");
  if (!p->ws) return pfail(p, NNCP_ERR_INVALID_ARG, "workspace not set");
  int64_t n = 1;
  for (int k = 0; k < p->N; ++k) n *= p->block_rows[k];
  PCK(launch_sumsq(X_local, 0, n, p->red, kRedParts, p->red + kRedParts, nullptr, p->stream));
  PCK(cudaMemcpyAsync(p->host_part, p->red + kRedParts, sizeof(double), cudaMemcpyDeviceToHost,
                      p->stream));
  PCK(cudaStreamSynchronize(p->stream));
  *local = p->host_part[0];
  return NNCP_OK;
}

nncp_status nncp_par_begin(nncp_par* p, double alpha, double tol) {
  if (!p) return pfail(nullptr, NNCP_ERR_INVALID_ARG, "null par");
  if (!(alpha > 0.0) || !(tol >= 0.0))
    return pfail(p, NNCP_ERR_INVALID_ARG, "alpha must be > 0 and tol >= 0");
  p->alpha = alpha;
  p->tol = tol;
  std::fill(p->lam.begin(), p->lam.end(), 1.0);
  std::fill(p->G.begin(), p->G.end(), 0.0);
  p->fits.clear();
  p->stop = false;
  p->begun = true;
  return NNCP_OK;
}

nncp_status nncp_par_mttkrp(nncp_par* p, int mode, float* M_block) {
  if (!p || mode < 1 || mode > p->N || !M_block)
    return pfail(p, NNCP_ERR_INVALID_ARG, "null par or output, or mode out of range");
  const nncp_status s = nncp_mttkrp_cached(p->ctx, mode, M_block);
  if (s != NNCP_OK) return pfail(p, s, "%s", nncp_last_error(p->ctx));
  return NNCP_OK;
}

nncp_status nncp_par_update(nncp_par* p, int mode, const float* M_owned, float* H_owned,
                            double* partial) {
  if (!p || mode < 1 || mode > p->N || !partial)
    return pfail(p, NNCP_ERR_INVALID_ARG, "null par or partial, or mode out of range");
  if (!p->begun) return pfail(p, NNCP_ERR_INVALID_ARG, "call nncp_par_begin first");
  const int n = mode - 1, R = p->R, R2 = R * R;
  const int64_t rows = p->owned_rows[n];
  for (int e = 0; e <= R2; ++e) partial[e] = 0.0;
  if (rows == 0) return NNCP_OK;
  if (!H_owned) return pfail(p, NNCP_ERR_INVALID_ARG, "H_owned is NULL");
  SolveState st;
  memset(&st, 0, sizeof st);
  st.S32 = p->S32;
  st.lam = p->lam_dev;
  st.gram_part = p->gram;
  st.flags = p->flags;
  if (M_owned) {
    // S(n) (float64, redundant) in float32 for the row arithmetic, and lambda
    std::vector<double> S((size_t)R2);
    hadamard_except(p, n, S.data());
    for (int e = 0; e < R2; ++e) p->host_small[e] = (float)S[e];
    PCK(cudaMemcpyAsync(p->S32, p->host_small, (size_t)R2 * sizeof(float), cudaMemcpyHostToDevice,
                        p->stream));
    PCK(cudaMemcpyAsync(p->lam_dev, p->lam.data(), (size_t)R * sizeof(double),
                        cudaMemcpyHostToDevice, p->stream));
    PCK(launch_hals_gram(H_owned, M_owned, rows, R, st, p->stream));
  } else {
    PCK(launch_gram_only(H_owned, rows, R, st, p->stream));
  }
  const int nb = hals_gram_blocks(rows);
  PCK(cudaMemcpyAsync(p->host_part, p->gram, (size_t)nb * (R2 + 1) * sizeof(double),
                      cudaMemcpyDeviceToHost, p->stream));
  PCK(cudaStreamSynchronize(p->stream));
  for (int b = 0; b < nb; ++b)
    for (int e = 0; e <= R2; ++e) partial[e] += p->host_part[(size_t)b * (R2 + 1) + e];
  return NNCP_OK;
}

nncp_status nncp_par_normalize(nncp_par* p, int mode, const double* sum, float* H_owned, int init,
                               double* fit_out, int* stop_out) {
  if (!p || mode < 1 || mode > p->N || !sum)
    return pfail(p, NNCP_ERR_INVALID_ARG, "null par or sums, or mode out of range");
  if (!p->begun) return pfail(p, NNCP_ERR_INVALID_ARG, "call nncp_par_begin first");
  const int n = mode - 1, R = p->R, R2 = R * R;
  // lambda = column 2-norms of W over every processor's rows (Alg. 3
  // Col-Norms), H = W diag(lambda)^-1, G(n) = H^T H, all from the summed W^T W
  std::vector<double> c((size_t)R);
  for (int r = 0; r < R; ++r) c[r] = sqrt(std::max(0.0, sum[r * R + r]));
  for (int r = 0; r < R; ++r) p->lam[r] = init ? p->lam[r] * c[r] : c[r];
  double* Gn = p->G.data() + (size_t)n * R2;
  for (int a = 0; a < R; ++a)
    for (int b = 0; b < R; ++b)
      Gn[a * R + b] = (c[a] > 0.0 && c[b] > 0.0) ? sum[a * R + b] / (c[a] * c[b]) : 0.0;
  const int64_t rows = p->owned_rows[n];
  if (rows > 0) {
    if (!H_owned) return pfail(p, NNCP_ERR_INVALID_ARG, "H_owned is NULL");
    for (int r = 0; r < R; ++r) p->host_small[r] = c[r] > 0.0 ? (float)(1.0 / c[r]) : 0.0f;
    PCK(cudaMemcpyAsync(p->inv, p->host_small, (size_t)R * sizeof(float), cudaMemcpyHostToDevice,
                        p->stream));
    PCK(launch_scale_columns(H_owned, rows, R, p->inv, p->stream));
    PCK(cudaStreamSynchronize(p->stream));
  }
  // the tree nodes that contracted the old factor n are recomputed at their
  // next use (after the caller's All-Gather has refreshed the block)
  nncp_factor_changed(p->ctx, mode);
  if (!init && n == p->N - 1) {
    // fit = 1 - eps, eps^2 = (alpha - 2 beta + gamma) / alpha (Sec. IV-B), with
    // beta = <M, W> and gamma = sum_ab S_ab (W^T W)_ab summed over processors
    std::vector<double> S((size_t)R2);
    hadamard_except(p, n, S.data());
    double gamma = 0.0;
    for (int e = 0; e < R2; ++e) gamma += S[e] * sum[e];
    const double beta = sum[R2];
    const double eps = sqrt(std::max(0.0, p->alpha - 2.0 * beta + gamma) / p->alpha);
    const double fit = 1.0 - eps;
    const bool stop = !std::isfinite(fit) ||
                      (!p->fits.empty() && fabs(fit - p->fits.back()) < p->tol);
    p->fits.push_back(fit);
    p->stop = stop;
    if (fit_out) *fit_out = fit;
    if (stop_out) *stop_out = stop ? 1 : 0;
    if (!std::isfinite(fit)) return pfail(p, NNCP_ERR_NUMERIC, "non-finite fit");
  } else {
    if (fit_out) *fit_out = p->fits.empty() ? 0.0 : p->fits.back();
    if (stop_out) *stop_out = 0;
  }
  return NNCP_OK;
}

nncp_status nncp_par_result(const nncp_par* p, double* lambda_out, double* fits, int max_fits,
                            int* iters_out) {
  if (!p) return pfail(nullptr, NNCP_ERR_INVALID_ARG, "null par");
  if (lambda_out) memcpy(lambda_out, p->lam.data(), (size_t)p->R * sizeof(double));
  const int n = (int)p->fits.size();
  if (fits)
    for (int i = 0; i < std::min(n, max_fits); ++i) fits[i] = p->fits[i];
  if (iters_out) *iters_out = n;
  return NNCP_OK;
}

const char* nncp_par_last_error(const nncp_par* p) {
  return p ? p->err.c_str() : nncp_global_error();
}

void nncp_par_destroy(nncp_par* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  nncp_destroy(p->ctx);
  if (p->host_part) cudaFreeHost(p->host_part);
  if (p->host_small) cudaFreeHost(p->host_small);
  delete p;
}

}  // extern "C"
