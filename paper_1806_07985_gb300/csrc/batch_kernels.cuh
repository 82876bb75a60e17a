// Batched NNCP-HALS kernels (many independent tensors of one order N).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nncp_internal.cuh"

namespace nncp {

constexpr int kBatchMaxI = 256;     // longest mode of a batched tensor
constexpr int kBatchMaxRank = 64;   // largest rank of a batched tensor
constexpr long long kAlphaChunk = 65536;
constexpr long long kBatchMaxElems = (1LL << 31) - 1;  // per tensor (32-bit indices)

// Tiles of the two root partial MTTKRPs.  X_(1) of a tensor is read as rows j
// of I_1 contiguous floats; a tile is a run of whole rows (a multiple of four
// rows, so every tile starts 16-byte aligned), at most kTileFloats floats.
constexpr int kTileFloats = 8192;
constexpr int kWsFloats = 4096;       // Khatri-Rao tile (rows x padded rank)
constexpr int kLeftMaxRows = 2048;    // padded X tile <= kTileFloats + kLeftMaxRows
constexpr int kRightTileTarget = 32768;  // elements per root -> {1} chunk
constexpr int kLeftItemTiles = 4;        // tiles per root -> {2..N} item
// rank groups of four, rounded up to a power of two (1 .. 16), and the padded rank
__host__ __device__ inline int b_rq(int R) {
  int q = 1;
  while (4 * q < R) q *= 2;
  return q;
}
__host__ __device__ inline int b_rank_pad(int R) { return 4 * b_rq(R); }
__host__ __device__ inline int b_rows_right(int I1, int R) {
  const int a = kTileFloats / I1, b = kWsFloats / b_rank_pad(R);
  return (a < b ? a : b) & ~3;
}
__host__ __device__ inline int b_rows_left(int I1) {
  const int a = kTileFloats / I1;
  return (a < kLeftMaxRows ? a : kLeftMaxRows) & ~3;
}
// rank groups per thread of the root -> {2..N} kernel: the largest power of two
// that still leaves 256 (row, rank block) pairs per tile, at least 1
__host__ __device__ inline int b_rqb_left(int I1, int R) {
  const int rq = b_rq(R);
  const int v = rq * b_rows_left(I1) / 256;
  int q = 1;
  while (2 * q <= v && 2 * q <= rq) q *= 2;
  return q;
}

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
  long long jchunk;     // columns of X_(1) per partial chunk (multiple of rows_r)
  int nchunk;
  int rows_r, rows_l;   // tile rows of the root -> {1} / root -> {2..N} kernels
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
                             int hs_floats, cudaStream_t st);
cudaError_t launch_b_mttv_leaf(const BTensor* ts, int count, int a, cudaStream_t st);
cudaError_t launch_b_mttv_first(const BTensor* ts, int count, int a, cudaStream_t st);
cudaError_t launch_b_update(int rmax, BTensor* ts, int count, int n, int* done_count,
                            cudaStream_t st);
// per tensor: iterations, last fit, lambda into contiguous arrays
cudaError_t launch_b_gather(const BTensor* ts, int count, int* iters, double* fits,
                            double* lam, const int* lam_off, int* nonfinite, cudaStream_t st);

}  // namespace nncp
