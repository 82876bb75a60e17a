// Batched NNCP-HALS kernels (many independent tensors of one order N).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "nncp_internal.cuh"

namespace nncp {

constexpr int kBatchMaxI = 256;     // longest mode of a batched tensor
constexpr int kBatchMaxRank = 64;   // largest rank of a batched tensor
constexpr long long kAlphaChunk = 65536;
constexpr long long kBatchMaxElems = (1LL << 31) - 1;  // per tensor (32-bit indices)

// Tiles of the two root partial MTTKRPs.  X_(1) of a tensor is read as rows j
// of I_1 contiguous floats; a tile is a run of whole rows (a multiple of four
// rows, so every tile starts 16-byte aligned), at most kTileFloats floats,
// double-buffered in shared memory.
constexpr int kTileFloats = 4096;
constexpr int kWsFloats = 2048;       // Khatri-Rao tile (rows x padded rank)
constexpr int kLeftMaxRows = 512;     // padded X tile <= kTileFloats + kLeftMaxRows
constexpr int kRightTileTarget = 32768;  // elements per root -> {1} chunk
constexpr int kLeftItemTiles = 16;       // tiles per root -> {2..N} item
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

// Other phases: elements of a tensor (or of a dimension-tree node) per work item.
constexpr int kItemElems = 65536;
constexpr int kMaxChunks = 256;       // partial-sum chunks per tensor and phase
constexpr int kLeafTileK = 64;        // rows k per Khatri-Rao tile of a leaf multi-TTV
constexpr int kLeafBlock = 1024;      // outputs (i, r) per leaf item
constexpr int kReduceBlock = 256;     // outputs per reduction item

// One tensor of a batch: shapes, caller buffers, and its slice of the workspace.
// Everything below `X` is laid out by b_tensor_layout from the shape alone.
struct BTensor {
  int N, R;
  int64_t dims[kMaxModes];
  int64_t I;            // elements
  const float* X;       // mode-1 fastest
  float* H[kMaxModes];  // I_n x R row-major
  float* node[kMaxModes];  // node {d..N} (0-based d = 1..N-2); node[1] = M when N = 2
  float* M;             // max_n I_n x R
  float* part;          // root -> {1} partials: nchunk x I_1 x R
  float* lpart;         // leaf partials: leaf_nkc[a] x I_a x R
  long long jchunk;     // columns of X_(1) per partial chunk (multiple of rows_r)
  int nchunk;
  int rows_r, rows_l;   // tile rows of the root -> {1} / root -> {2..N} kernels
  int leaf_kc[kMaxModes];   // rows k per leaf chunk of node {a..N}
  int leaf_nkc[kMaxModes];  // leaf chunks of node {a..N}
  int first_jb[kMaxModes];  // rows j per item of node {a..N} -> node {a+1..N}
  int fit_cap;          // fit history slots
  int max_iters;        // stopping rule (set by the host before init)
  double tol;
  double* G;            // N x R x R
  double* S;            // R x R
  float* S32;           // R x R
  double* lam;          // R
  double* fits;         // fit_cap
  double* scal;         // [0] alpha, [1] tol
  int* flags;           // [0] done, [1] iterations, [2] non-finite fit
};

// Work lists of one batch composition: every phase of the iteration is one
// launch over a contiguous range of (tensor, y, z, 0) items.
struct BPhase {
  int off = 0, count = 0;
};
struct BPlan {
  int count = 0, N = 0, rmax = 16, hs_floats = 0;
  int max_rows = 1;  // longest mode of any tensor of the batch
  std::vector<int4> items;
  BPhase alpha, pmr, pmr_red, pml;
  BPhase leaf[kMaxModes], leaf_red[kMaxModes], first[kMaxModes];
  std::vector<int> alpha_first;  // per tensor, into the alpha phase (count + 1 entries)
  std::vector<int> lam_off;      // per tensor, into a packed lambda array
  size_t lam_total = 0;
};

// Lays out one tensor's slice (node buffers, M, partials, state) at `base`
// (sizes only when base is NULL) and fills the shape-derived fields of *d.
size_t b_tensor_layout(int N, const int64_t* dims, int R, int fit_cap, BTensor* d, char* base);
void b_build_plan(const BTensor* ts, int count, int N, BPlan* p);

cudaError_t batch_attributes_init();
// alpha, normalisation, Grams and S of every tensor of the plan
cudaError_t b_launch_init(const BPlan& p, BTensor* ts, const int4* items, double* alpha_part,
                          const int* alpha_first, cudaStream_t st);
// How the two root phases run: 0 = one CTA per work item (scheduled by the
// hardware), 1 = one wave of persistent CTAs taking items from a counter,
// 2 = one wave of persistent CTAs with the work split by warp role: a
// scheduler warp takes items from a counter, a loader warp streams dense
// tiles through a ring of shared-memory stages, builder warps form the
// Khatri-Rao rows (root -> {1}) or restride the tile and stage H_1
// (root -> {2..N}), and the remaining warps contract.  A tensor's bits are
// the same under every schedule.
struct BSchedule {
  int pm_right = 0, pm_left = 0;
  long long wait_cycles = 0;  // bounded-wait limit of the streamed kernels (0: about 2 s)
};
constexpr int kRightSchedules = 3, kLeftSchedules = 3;
// The root phases alone (no state changes but their outputs, which every
// iteration recomputes): what the schedule tuner times.  queue: a device
// counter set to 0 before the launch (unused by schedule 0); err: a device
// int that a streamed launch sets to 1 when one of its bounded waits expires.
cudaError_t launch_pm_right(const BPlan& p, const BTensor* ts, const int4* items, int mode,
                            int* queue, int* err, cudaStream_t st, long long wait_cycles = 0);
cudaError_t launch_pm_left(const BPlan& p, const BTensor* ts, const int4* items, int mode,
                           int* queue, int* err, cudaStream_t st, long long wait_cycles = 0);
// one outer iteration (Alg. 1 over the Fig. 1 tree with root split 1);
// queues: three device ints (the two root phases' counters and the error
// word of the streamed schedule), or NULL for schedule 0 everywhere
cudaError_t b_launch_iteration(const BPlan& p, BTensor* ts, const int4* items, int* done_count,
                               cudaStream_t st, const BSchedule& sch, int* queues);
// per tensor: iterations, last fit, lambda into contiguous arrays, and a state
// word (bit 0: non-finite fit, bit 1: stopped)
cudaError_t launch_b_gather(const BTensor* ts, int count, int* iters, double* fits,
                            double* lam, const int* lam_off, int* nonfinite, cudaStream_t st);

}  // namespace nncp
