// Internal declarations shared by the CUDA translation units of the NNCP library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace nncp {

// ---- programmatic dependent launch --------------------------------------------
// The kernels of one outer iteration are captured into a CUDA graph with
// programmatic stream serialization, so a kernel may be scheduled while its
// predecessor in the iteration is still running.  Every kernel launched that way
// calls pdl_wait() before its first access to memory that an earlier kernel
// writes, or that a later one writes while an earlier one may still read it.  pdl_wait() returns
// once every predecessor grid has completed and its writes are visible, so the
// chain stays ordered transitively.  Small kernels then call pdl_trigger(), which
// lets their successor be scheduled on the SMs they leave free; large grids do
// not, so their successor is scheduled as their CTAs exit.  Outside such a
// launch both return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches k(args...) on st: with programmatic stream serialization while st is
// being captured into a graph, as an ordinary launch otherwise.  Only kernels
// that follow the pdl_wait() rule above are launched through this.
// cluster_x > 0 launches the grid as thread-block clusters of cluster_x CTAs.
template <typename... P, typename... A>
cudaError_t launch_kernel_cluster(void (*k)(P...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t st, int cluster_x, A&&... args) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute at[2];
  unsigned na = 0;
  if (cluster_x > 0) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cluster_x;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  if (cs == cudaStreamCaptureStatusActive) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

template <typename... P, typename... A>
cudaError_t launch_kernel(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          A&&... args) {
  return launch_kernel_cluster(k, grid, block, smem, st, 0, std::forward<A>(args)...);
}

constexpr int kMaxModes = 8;
constexpr int kMaxRank = 128;
constexpr int kFitCapacity = 1 << 16;  // fit history slots on the device

// Khatri-Rao product of a list of factor matrices, formed on the fly.
// Row k of the product over modes m_0 (fastest), m_1, ... is the Hadamard
// product of rows k_0, k_1, ... of the factors, k = k_0 + dim_0*(k_1 + ...).
// Factors are row-major dim x R.  nm = 0 means the all-ones row.
struct KrpDesc {
  int nm;
  int64_t dim[kMaxModes];
  const float* H[kMaxModes];
};

// Per-solve device state (lives in the caller's workspace).
struct SolveState {
  double* G;        // N x R x R, Gram of each normalised factor (float64)
  double* S;        // N x R x R: S for mode m (the Hadamard of every Gram but
                    // G_m, float64) at S + m R^2; an update of mode n reads
                    // its own and writes next_mode's, so the two never alias
  float* S32;       // R x R, float32 copy of the S of the mode updated next,
                    // read by the per-row NLS arithmetic
  double* lam;      // R
  double* gram_part;  // blocks x (R*R + 1): per-block W^T W and <M, W>
  double* scalars;  // [0] alpha = ||X||^2, [1] beta, [2] gamma, [3] eps, [4] tol,
                    // [5] the last recorded fit, [8..9] explicit residual and ||X||^2
  double* fits;     // kFitCapacity
  int* flags;       // [0] done, [1] status, [2] iteration count, [3] nonfinite, [8] CTA ticket
};

// ---- launchers (return cudaSuccess or the launch error) ----------------------

// out(i, r) = sum_{l < L, q < Q} X[l + L*(i + I*q)] * KL(l, r) * KQ(q, r)
// for i < I, r < R: the generic (direct or partial) MTTKRP on CUDA cores.
// X is float32.  When the contraction is split across CTAs the per-chunk
// results go to `partials` (capacity `part_cap` floats) and are summed in a
// fixed order, so results are bitwise reproducible.
cudaError_t launch_simt_mttkrp(const float* X, int64_t L, int64_t I, int64_t Q,
                               const KrpDesc& KL, const KrpDesc& KQ, int R, float* out,
                               float* partials, size_t part_cap, int num_sms,
                               cudaStream_t st);
size_t simt_mttkrp_partials(int64_t L, int64_t I, int64_t Q, int R, int num_sms);
cudaError_t launch_simt_mttkrp_capped(const float* X, int64_t L, int64_t I, int64_t Q,
                                      const KrpDesc& KL, const KrpDesc& KQ, int R, float* out,
                                      float* partials, size_t part_cap, int num_sms,
                                      cudaStream_t st);

// Records a message for nncp_global_error().
void record_global_error(const char* msg);

}  // namespace nncp

struct nncp_ctx;

namespace nncp {

// Serving hooks on a plain context: initialise a solve with stopping
// tolerance tol (as nncp_solve does) without running it, and the device
// addresses of its state: flags[4] = {done, -, iterations, non-finite},
// lambda (R), the fit history, and the tensor-core error word (NULL when the
// context has no tensor-core scratch).
int ctx_solve_begin_tol(nncp_ctx* c, double tol);
// Mode-1 length to store a host tensor with so that a tensor-core precision
// can run it: when I_1...I_s times the element size is not a multiple of 16
// bytes for the split in use, I_1 rounded up to a multiple of 16 bytes' worth
// of elements (zero slices, with zero rows in H_1).  dims[0] otherwise, or
// when padding does not make the shape supported.
int64_t tc_padded_mode1(int precision, int N, const int64_t* dims, int R, int root_split);
void ctx_device_state(const nncp_ctx* c, const int** flags, const double** lam,
                      const double** fits, const int** tc_error);

// out[e] = sum_{c < C} part[c * E + e] in chunk order (deterministic).
cudaError_t launch_reduce_chunks(const float* part, int64_t E, int C, float* out, int num_sms,
                                 cudaStream_t st);

// Multi-TTV leaf: out(i, r) = sum_{k < K} T[((i + I*k) * R) + r] * KK(k, r).
cudaError_t launch_mttv_leaf(const float* T, int64_t I, int64_t K, const KrpDesc& KK,
                             int R, float* out, float* partials, size_t part_cap,
                             int num_sms, cudaStream_t st);
size_t mttv_leaf_partials(int64_t I, int64_t K, int R, int num_sms);

// Multi-TTV to the child node: out(j, r) = sum_{i < I} T[((i + I*j) * R) + r] * H(i, r).
cudaError_t launch_mttv_first(const float* T, int64_t I, int64_t J, const float* H, int R,
                              float* out, cudaStream_t st);

// sum of squares of n float32 (or bf16) values into *out (float64), deterministic.
cudaError_t launch_sumsq(const void* X, int bf16, int64_t n, double* partials, int nparts,
                         double* out, const int* flags, cudaStream_t st);

// float32 -> bf16 (round to nearest even).
cudaError_t launch_to_bf16(const float* X, uint16_t* Y, int64_t n, cudaStream_t st);

// ---- factor update kernels (update_kernels.cu) -----------------------------

// Shared-memory opt-ins of every kernel that needs them; once per process and
// device, before any launch or capture.
cudaError_t kernel_attributes_init();
cudaError_t tc_attributes_init();

// HALS sweep on W = H diag(lam) for every row, in place in H, followed by the
// per-block partials of W^T W and <M, W> into st.gram_part.
cudaError_t launch_hals_gram(float* H, const float* M, int64_t In, int R, SolveState st,
                             cudaStream_t stream);
int hals_gram_blocks(int64_t In);

// Whole mode update (HALS, Gram, normalisation, fit, next S) in one launch over
// CTAs of up to 512 rows (R <= 32) or 128 rows (R <= 64), used when
// multi_update_ok(In, R); `part` is device scratch of multi_update_scratch(In, R)
// floats.
bool multi_update_ok(int64_t In, int R);
size_t multi_update_scratch(int64_t In, int R);
// The same update on one thread-block cluster (cluster_update_ok(In, R):
// I_n <= 1024, R <= 64), preferred where it applies; needs no scratch.
// sweep = 0: H holds W already (written by the kernel just before), no HALS
// sweep; the rest of the update as above.  U (non-null with sweep = 0): the
// rows' ADMM duals, divided by the new lambda along with H.
bool cluster_update_ok(int64_t In, int R);
cudaError_t launch_update_cluster(float* H, const float* M, int64_t In, int R, int N, int n,
                                  int next_mode, int is_last, SolveState st, cudaStream_t stream,
                                  int sweep = 1, float* U = nullptr);
cudaError_t launch_update_multi(float* H, const float* M, int64_t In, int R, int N, int n,
                                int next_mode, int is_last, SolveState st, float* part,
                                cudaStream_t stream);

// Block principal pivoting NLS update (R <= 32): W = argmin_{W >= 0} of the
// row-wise least squares with S = st.S and M, written to H unnormalised,
// followed by the Gram partials and <M, W> into st.gram_part (then
// launch_finalize, as after launch_hals_gram).
cudaError_t launch_bpp_update(float* H, const float* M, int64_t In, int R, SolveState st,
                              int num_sms, cudaStream_t stream);
// The row solves alone (W into H, unnormalised), for launch_update_cluster(sweep = 0).
cudaError_t launch_bpp_rows(float* H, const float* M, int64_t In, int R, SolveState st,
                            int num_sms, cudaStream_t stream);

// AO-ADMM NLS update (R <= 32): `iters` ADMM iterations on every row from
// z = H diag(lam), u = U diag(lam); z into H (unnormalised W), u into U.  The
// _update form adds the Gram partials and <M, W> (then launch_finalize with
// U); the _rows form is for launch_update_cluster(sweep = 0, U).
cudaError_t launch_admm_rows(float* H, float* U, const float* M, int64_t In, int R, int iters,
                            SolveState st, cudaStream_t stream);
cudaError_t launch_admm_update(float* H, float* U, const float* M, int64_t In, int R, int iters,
                               SolveState st, cudaStream_t stream);

// Accelerated projected gradient NLS update (R <= 32): `iters` FISTA steps on
// every row from W = H diag(lam), W into H (unnormalised).  The _update form
// adds the Gram partials and <M, W> (then launch_finalize); the _rows form is
// for launch_update_cluster(sweep = 0).
cudaError_t launch_apg_rows(float* H, const float* M, int64_t In, int R, int iters,
                           SolveState st, cudaStream_t stream);
cudaError_t launch_apg_update(float* H, const float* M, int64_t In, int R, int iters,
                              SolveState st, cudaStream_t stream);

// H(i, r) *= inv(r) over `rows` rows (inv: R floats, device).
cudaError_t launch_scale_columns(float* H, int64_t rows, int R, const float* inv,
                                 cudaStream_t stream);

// Gram partials of H as given (initialisation: W = H).
cudaError_t launch_gram_only(const float* H, int64_t In, int R, SolveState st,
                             cudaStream_t stream);

// Single-CTA finalise of a mode update:
//   W^T W = sum of the partials; lam = sqrt(diag); G_n = D^-1 W^T W D^-1;
//   H_n = W / lam (in place); if is_last: fit from the Sec. IV-B identity;
//   S for mode next_mode.  init = 1: lam *= column norms instead of replacing.
//   U non-null: the rows' ADMM duals, divided by the new lambda along with H.
cudaError_t launch_finalize(float* H, int64_t In, int R, int N, int n, int next_mode,
                            int nblocks, int is_last, int init, double tol, SolveState st,
                            cudaStream_t stream, float* U = nullptr);

// lambda = 1, flags and fit counter cleared, tolerance stored (before initialisation).
cudaError_t launch_solve_reset(SolveState st, int R, double tol, cudaStream_t stream);

// S = Hadamard of every Gram but mode's, in float64 (st.S + mode R^2) and as
// the float32 copy st.S32.
cudaError_t launch_compute_S(SolveState st, int N, int R, int mode, cudaStream_t stream);

// Explicit residual ||X - [[lam; H]]||^2 accumulated in float64 into out[0];
// out[1] = ||X||^2.
cudaError_t launch_explicit_residual(const float* X, int N, const int64_t* dims, int R,
                                     float* const* H, const double* lam, double* partials,
                                     int nparts, double* out, cudaStream_t stream);

}  // namespace nncp
