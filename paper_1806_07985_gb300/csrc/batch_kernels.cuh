// Batched NNCP-HALS kernels (many independent tensors of one order N).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nncp_internal.cuh"

namespace nncp {

constexpr int kBatchMaxI = 256;     // longest mode of a batched tensor
constexpr int kBatchMaxRank = 64;   // largest rank of a batched tensor
constexpr long long kAlphaChunk = 65536;

// One tensor of a batch: shapes, caller buffers, and its slice of the workspace.
struct BTensor {
  int N, R;
  int64_t dims[kMaxModes];
  int64_t I;            // elements
  const float* X;       // mode-1 fastest
  float* H[kMaxModes];  // I_n x R row-major
  float* node[kMaxModes];  // node {d..N} (0-based d = 1..N-2); node[1] = M when N = 2
  float* M;             // max_n I_n x R
  float* part;          // root -> {1} partials: nchunk x I_1 x R
  long long jchunk;     // columns of X_(1) per partial chunk
  int nchunk;
  int fit_cap;          // fit history slots
  int max_iters;
  double* G;            // N x R x R
  double* S;            // R x R
  float* S32;           // R x R
  double* lam;          // R
  double* fits;         // fit_cap
  double* scal;         // [0] alpha, [1] tol
  int* flags;           // [0] done, [1] iterations, [2] non-finite fit
};

cudaError_t batch_attributes_init();
cudaError_t launch_b_init(BTensor* ts, int count, const int2* alpha_items, int n_alpha_items,
                          double* alpha_part, const int* alpha_first, double tol, int max_iters,
                          cudaStream_t st);
cudaError_t launch_b_pm_right(int rmax, const BTensor* ts, const int2* items, int n_items,
                              int count, cudaStream_t st);
cudaError_t launch_b_pm_left(int rmax, const BTensor* ts, const int2* items, int n_items,
                             cudaStream_t st);
cudaError_t launch_b_mttv_leaf(const BTensor* ts, int count, int a, cudaStream_t st);
cudaError_t launch_b_mttv_first(const BTensor* ts, int count, int a, cudaStream_t st);
cudaError_t launch_b_update(int rmax, BTensor* ts, int count, int n, int* done_count,
                            cudaStream_t st);
// per tensor: iterations, last fit, lambda into contiguous arrays
cudaError_t launch_b_gather(const BTensor* ts, int count, int* iters, double* fits,
                            double* lam, const int* lam_off, int* nonfinite, cudaStream_t st);

}  // namespace nncp
