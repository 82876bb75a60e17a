/*
 * nncp.h -- C ABI of the GB300 NNCP-HALS library (dimension-tree MTTKRP).
 *
 * Problem (Eq. 1 of "Parallel Nonnegative CP Decomposition of Dense Tensors",
 * Ballard, Hayashi, Kannan, arXiv:1806.07985):
 *     min_{H_n >= 0} || X - sum_r H_1(:,r) o ... o H_N(:,r) ||^2
 * solved by block coordinate descent over whole factor matrices (Alg. 1, with
 * the normalisation and error steps of Alg. 3), MTTKRPs through a dimension
 * tree (Sec. IV-A), one HALS column sweep per block update (Sec. II-B), and the
 * relative error from the identity of Sec. IV-B.
 *
 * Conventions shared by every call:
 *   - Tensor X: dense, N-way, I_1 x ... x I_N, stored mode-1 fastest (the
 *     layout of Sec. IV-C "Data Distribution": linear index
 *     i_1 + I_1*(i_2 + I_2*(...)), 0-based).  float32, or bfloat16 in the
 *     NNCP_BF16_STORED precision mode.  Device memory, 16-byte aligned.
 *   - Factor H_n: I_n x R float32, ROW-major (the R entries of a row are
 *     contiguous), device memory, 16-byte aligned.  (The paper's Armadillo
 *     matrices are column-major; rows are what the HALS update and the
 *     on-the-fly Khatri-Rao product read, so rows are contiguous here.)
 *   - Modes are numbered 1..N at this boundary.
 *   - Ownership: the caller owns X, the factors, outputs and the workspace;
 *     the library never frees caller memory.  A context holds only pointers.
 *   - Streams are passed as void* (a cudaStream_t); NULL is the legacy
 *     default stream.
 *   - Errors: every call returns an nncp_status; nothing aborts or throws
 *     across the ABI.  On NNCP_ERR_INVALID_ARG the context is unchanged.
 *     nncp_last_error() returns a message for the last failing call.
 *   - Thread safety: a context may be used by one host thread at a time.
 */
#ifndef NNCP_H
#define NNCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nncp_ctx nncp_ctx;

typedef int nncp_status;
#define NNCP_OK                 0
#define NNCP_ERR_INVALID_ARG    1
#define NNCP_ERR_OUT_OF_MEMORY  2
#define NNCP_ERR_CUDA           3
#define NNCP_ERR_NUMERIC        4   /* non-finite fit */
#define NNCP_ERR_TIMEOUT        5
#define NNCP_ERR_NOT_READY      6
#define NNCP_ERR_UNSUPPORTED    7

/* How the partial MTTKRPs (the two root branches of the dimension tree)
 * contract the tensor.  All accumulate in float32. */
typedef int nncp_precision;
#define NNCP_FP32_SIMT     0   /* CUDA-core FFMA */
#define NNCP_TF32          1   /* tcgen05 kind::tf32 on the float32 tensor */
#define NNCP_SPLIT_BF16X3  2   /* tcgen05 kind::f16: x = hi + lo (bf16), hi*hi + hi*lo + lo*hi */
#define NNCP_BF16_STORED   3   /* tensor stored as bf16; factors split hi + lo */

/* Library version string and whether tcgen05 kernels were compiled in. */
const char* nncp_version(void);

/* Create a context for an N-way tensor with mode lengths dims[0..N-1] and
 * rank R.  2 <= N <= 8, dims[n] >= 1, 1 <= R <= 128.  Defaults: precision
 * NNCP_FP32_SIMT, root split chosen by nncp_default_split, stream NULL.
 * The context owns no device memory until nncp_set_workspace. */
nncp_status nncp_create(int N, const int64_t* dims, int R, nncp_ctx** out);

/* Root split s of the dimension tree: modes 1..s versus s+1..N (Sec. IV-A,
 * Fig. 1).  Returns the s in [1, N-1] that makes the products of the two
 * halves' lengths closest (Sec. IV-C "Memory"), the smaller s on ties. */
int nncp_default_split(int N, const int64_t* dims);

/* precision: one of NNCP_*; root_split: 0 = default, else s in [1, N-1];
 * stream: cudaStream_t the context launches on.  Invalidates captured graphs. */
nncp_status nncp_set_options(nncp_ctx* ctx, nncp_precision precision, int root_split,
                             void* stream);

/* Solve with or without the dimension tree (enabled = 1, the default).
 * Without it every outer iteration computes each M(n) by a full MTTKRP over
 * the whole tensor (N passes per iteration instead of two) -- the
 * implementation without the optimization that Sec. V-C benchmarks (results
 * in Sec. V-D) and the third line of the cost table in Sec. IV-C.  FP32 SIMT only:
 * NNCP_ERR_UNSUPPORTED for a tensor-core precision.  Takes effect at the
 * next solve or iteration. */
nncp_status nncp_set_dimtree(nncp_ctx* ctx, int enabled);

/* Fuse the first multi-TTV out of the right root node into that node's
 * partial MTTKRP (enabled = 1, the default; Sec. IV-A, Fig. 2b): the leaf of
 * the node's first mode is accumulated from the tensor-core kernel's
 * accumulators while the node is written, instead of by a separate pass over
 * the node.  Applies to the tensor-core precisions when the node has two or
 * more modes, its first mode is a multiple of 128, its rows fill the GPU (no
 * split contraction) and R <= 32; otherwise, and with enabled = 0, the leaf is
 * a separate multi-TTV.  Results agree to rounding (a different summation
 * order).  Takes effect at the next solve or iteration. */
nncp_status nncp_set_leaf_fusion(nncp_ctx* ctx, int enabled);

/* NLS-Update of Alg. 1 (Sec. II-B): NNCP_NLS_HALS (the default) makes one
 * HALS sweep from W = H_n diag(lambda); NNCP_NLS_BPP solves each row's
 * nonnegative least squares exactly by block principal pivoting (the solver
 * the paper benchmarks), whatever the starting W, then normalises as HALS
 * does; NNCP_NLS_ADMM runs a fixed number of ADMM iterations on every row
 * (AO-ADMM, one of the alternatives Sec. II-B names; rho = trace(S) / R),
 * from z = H_n diag(lambda) and the scaled dual its previous update of the
 * mode left (zero at the start of a solve), and takes z as the new W;
 * NNCP_NLS_APG runs a fixed number of Nesterov accelerated projected
 * gradient steps (FISTA form, step 1/L with L the largest absolute row sum
 * of S) from W = H_n diag(lambda).  BPP, ADMM and APG support R <= 32
 * (NNCP_ERR_UNSUPPORTED above) and any precision of the MTTKRPs.  Takes
 * effect at the next solve or iteration. */
#define NNCP_NLS_HALS 0
#define NNCP_NLS_BPP  1
#define NNCP_NLS_ADMM 2
#define NNCP_NLS_APG  3
nncp_status nncp_set_nls(nncp_ctx* ctx, int nls);
/* Inner iterations per mode update of the iterative NLS updates
 * (NNCP_NLS_ADMM, NNCP_NLS_APG): 1 <= iters <= 10000 (NNCP_ERR_INVALID_ARG
 * otherwise); default 5. */
nncp_status nncp_set_nls_iters(nncp_ctx* ctx, int iters);
/* Bytes of device scratch the context needs for its current options
 * (dimension-tree node temporaries, split-K partials, Gram/S/lambda state,
 * and I_n x R floats per mode for the ADMM duals). */
nncp_status nncp_workspace_size(const nncp_ctx* ctx, size_t* bytes);

/* Hand the context a caller-allocated device buffer of at least
 * nncp_workspace_size bytes, 256-byte aligned.  The caller keeps it alive
 * until nncp_destroy or the next nncp_set_workspace. */
nncp_status nncp_set_workspace(nncp_ctx* ctx, void* dev_ptr, size_t bytes);

/* Point the context at the tensor (device, layout above).  The data must stay
 * unchanged while the context uses it. */
nncp_status nncp_set_tensor(nncp_ctx* ctx, const void* X_dev);

/* Point the context at the N factor matrices (device, I_n x R row-major).
 * nncp_solve_bound reads the initial values there and leaves the result there. */
nncp_status nncp_set_factors(nncp_ctx* ctx, float* const* H_dev);

/* M_mode = X_(mode) (H_N (.) ... (.) H_{mode+1} (.) H_{mode-1} (.) ... (.) H_1)
 * (Sec. II-A), for the current factors, into M_dev (I_mode x R row-major,
 * device).  use_dimtree = 0: one direct pass over the tensor; 1: the root
 * partial MTTKRP of the half holding `mode` followed by multi-TTVs down the
 * tree (Sec. IV-A).  Asynchronous on the context's stream. */
nncp_status nncp_mttkrp(nncp_ctx* ctx, int mode, int use_dimtree, float* M_dev);

/* One root partial MTTKRP of the dimension tree (Sec. IV-A, Fig. 2a) for the
 * current factors, in the context's precision mode:
 *   side 0: T_L = X_(1:s) (H_N (.) ... (.) H_{s+1}),  (I_1...I_s) x R
 *   side 1: T_R = X_(1:s)^T (H_s (.) ... (.) H_1),    (I_{s+1}...I_N) x R
 * X_(1:s) is the column-major matricization with modes 1..s on the rows,
 * which is the tensor's memory as it lies.  Rows of T run over the node's
 * modes with the lowest fastest; T_dev is row-major (R contiguous), device.
 * Asynchronous on the context's stream. */
nncp_status nncp_partial_mttkrp(nncp_ctx* ctx, int side, float* T_dev);

/* M_mode through the dimension tree (Sec. IV-A, Fig. 1) for the current
 * factors, reusing the tree nodes that earlier calls left and whose factors
 * have not changed since: a node {a..b} holds the tensor contracted with
 * every factor outside modes a..b, and is recomputed only when one of those
 * was reported changed by nncp_factor_changed.  Called in BCD order (modes
 * 1..N, each factor reported changed right after its update) this reads the
 * tensor twice per sweep -- the local MTTKRP of Alg. 2, whose factor updates
 * happen outside the library.  M_dev: I_mode x R row-major, device.
 * Asynchronous on the context's stream.  Any other call that computes
 * (nncp_mttkrp, nncp_partial_mttkrp, a solve) or rebinds data forgets the
 * cached nodes. */
nncp_status nncp_mttkrp_cached(nncp_ctx* ctx, int mode, float* M_dev);

/* Reports that the caller has changed factor `mode` (1..N) in place: tree
 * nodes computed from it are recomputed at their next use. */
nncp_status nncp_factor_changed(nncp_ctx* ctx, int mode);

/* Full NNCP-HALS solve of min_{H_n >= 0} ||X - [[lambda; H_1..H_N]]||
 * (Eq. 1) for the tensor X_dev and the factors H_dev (N device pointers,
 * I_n x R row-major: in, the initial factors; out, the result), with the
 * outputs of Alg. 3 (column-normalised factors, lambda, the error).
 * X_dev / H_dev may be NULL to keep what nncp_set_tensor / nncp_set_factors
 * bound; passing the pointers already bound keeps the captured graphs.
 * Initialisation normalises the given factors (2-norm columns) and folds the
 * norms into lambda; each outer iteration updates modes 1..N in order (BCD,
 * Alg. 1) with MTTKRPs through the dimension tree and the NLS update (one HALS
 * sweep by default, Sec. II-B), then computes fit = 1 - eps with eps from the
 * Sec. IV-B identity.  Stops when |fit_k - fit_{k-1}| < tol (k >= 2) or
 * k = max_iters (1 <= max_iters <= 65536).
 * On return the factors hold H_1..H_N with unit-norm columns, lambda_out
 * (host, R doubles, may be NULL) the weights, *iters_out the outer
 * iterations run and *fit_out the last fit (either pointer may be NULL).
 * Blocks until done.  NNCP_ERR_NUMERIC if the fit became non-finite,
 * NNCP_ERR_TIMEOUT if a tensor-core kernel gave up waiting. */
nncp_status nncp_solve(nncp_ctx* ctx, const void* X_dev, float* const* H_dev, double* lambda_out,
                       int max_iters, double tol, int* iters_out, double* fit_out);

/* nncp_solve on the tensor and factors already bound (nncp_set_tensor,
 * nncp_set_factors); same behaviour and outputs. */
nncp_status nncp_solve_bound(nncp_ctx* ctx, int max_iters, double tol, double* lambda_out,
                             int* iters_out, double* fit_out);

/* Per-iteration fit history of the last nncp_solve (host array of at least
 * max_iters doubles); *count receives the number of iterations. */
nncp_status nncp_fit_history(const nncp_ctx* ctx, double* fits, int max_count, int* count);

/* Fit of the current model [[lambda; H]].  exact = 0: the identity value from
 * the last solve iteration; exact = 1: a full pass reconstructing every entry
 * (float64 accumulation) to compute 1 - ||X - model|| / ||X||. */
nncp_status nncp_fit(nncp_ctx* ctx, int exact, double* fit_out);

/* Run exactly `iters` outer iterations on the device state left by a previous
 * nncp_solve (or nncp_solve_begin), without host synchronisation: the unit
 * that the benchmark times.  Launches captured CUDA graphs of four iterations
 * (whole batches of four) and of one (the rest). */
nncp_status nncp_solve_begin(nncp_ctx* ctx);
nncp_status nncp_iterate(nncp_ctx* ctx, int iters);

/* Number of kernels one captured outer iteration launches (*count). */
nncp_status nncp_iteration_kernels(nncp_ctx* ctx, int* count);

/* Convert a float32 tensor to the bfloat16 copy NNCP_BF16_STORED contracts
 * (round to nearest even).  n elements, device pointers. */
nncp_status nncp_tensor_to_bf16(const float* X_dev, uint16_t* Xb_dev, int64_t n, void* stream);

/* One-call solve from HOST buffers: allocates device memory, copies the
 * tensor and initial factors in, solves, copies factors, lambda and fit back.
 * X_host: float32, mode-1 fastest; H_host[n]: I_n x R row-major (in: initial
 * factors, out: normalised result).  A tensor-core precision on a shape it
 * cannot tile (I_1...I_s times the element size not a multiple of 16 bytes)
 * runs with mode 1 stored padded by zero slices to a multiple of 4 (8 for
 * NNCP_BF16_STORED) and H_1 given matching zero rows: a HALS row update with
 * m = 0 and w = 0 yields 0, so those rows stay zero, add nothing to the Grams,
 * lambda or the fit, and the iteration is that of the unpadded problem up to
 * rounding (Sec. II-B update rule).  Only the first I_1 rows are returned.
 * The call keeps one plan per process -- the context, its captured graphs and
 * the device buffers of the last (stored shape, R, precision, root_split,
 * device) -- and reuses it when the next call matches, so repeated solves of
 * one shape allocate nothing and capture nothing; a call made while another
 * thread holds the plan runs without it.  The plan's device memory stays
 * allocated until nncp_solve_host_release or process exit. */
nncp_status nncp_solve_host(int N, const int64_t* dims, int R, const float* X_host,
                            float* const* H_host, nncp_precision precision, int root_split,
                            int max_iters, double tol, double* lambda_out, int* iters_out,
                            double* fit_out);

/* Frees the plan nncp_solve_host keeps (a no-op if there is none). */
void nncp_solve_host_release(void);

/* ---- Batched solver: many independent problems of one order N ----------
 * `count` tensors, tensor t with mode lengths dims[t*N .. t*N+N-1] (each in
 * [1, 256], at most 2^31 - 1 elements) and rank R[t] (in [1, 64]), all solved
 * by the NNCP-HALS iteration
 * of nncp_solve (Alg. 1 with the normalisation and error steps of Alg. 3,
 * Sec. II-B HALS, Sec. IV-B fit) with root split 1 for every tensor, so one
 * outer iteration is the same sequence of launches for the whole batch
 * (captured once as a CUDA graph).  Each tensor stops on its own
 * |fit_k - fit_{k-1}| < tol or at max_iters; a tensor's results are the same
 * bits whatever else is in the batch.  Same layouts as above: X_t float32
 * mode-1 fastest, H_t,n I_n x R_t row-major, device memory, caller-owned.
 * max_iters at create sizes the per-tensor fit history. */
typedef struct nncp_batch nncp_batch;
nncp_status nncp_batch_create(int count, int N, const int64_t* dims, const int* R, int max_iters,
                              nncp_batch** out);
nncp_status nncp_batch_workspace_size(const nncp_batch* b, size_t* bytes);
/* Caller-allocated device buffer (256-byte aligned) of nncp_batch_workspace_size bytes. */
nncp_status nncp_batch_set_workspace(nncp_batch* b, void* dev_ptr, size_t bytes);
/* X_dev[t] for t < count; H_dev[t*N + n] for factor n of tensor t; every
 * pointer 16-byte aligned (NNCP_ERR_INVALID_ARG otherwise). */
nncp_status nncp_batch_set_data(nncp_batch* b, const float* const* X_dev, float* const* H_dev);
/* Solve all tensors; factors are overwritten with the normalised results.
 * iters_out[t], fits_out[t] (host, count entries) and lambda_out (host, sum of
 * R_t doubles, tensor after tensor) may each be NULL.  Blocks until done. */
nncp_status nncp_batch_run(nncp_batch* b, int max_iters, double tol, int* iters_out,
                           double* fits_out, double* lambda_out, void* stream);

/* One call for `count` independent problems of any orders (the Eq. 1 problem
 * for each, with the Alg. 3 outputs): tensor t has order N[t] (2..8), mode
 * lengths dims[t][0..N[t]-1], rank R[t], tensor X_dev[t] and factors
 * H_dev[t][0..N[t]-1] (device, layouts as above, within the limits of
 * nncp_batch_create).  The tensors of each order are solved together as one
 * batch (nncp_batch_create / _run, so the same bits as that path), each
 * stopping on its own rule.  Outputs: factors overwritten in place, lambda[t]
 * (host, R[t] doubles; the array or an entry may be NULL), iters[t] and
 * fits[t] (host, count entries, may be NULL).  Allocates each batch's
 * workspace with cudaMalloc and frees it before returning; blocks until done.
 * On an error no further order is started; nncp_global_error says why. */
nncp_status nncp_batch_solve(int count, const int* N, const int64_t* const* dims, const int* R,
                             const void* const* X_dev, float* const* const* H_dev,
                             double* const* lambda, int max_iters, double tol, int* iters,
                             double* fits, void* stream);
/* Schedule of the two root partial MTTKRP phases (the paper has no
 * counterpart; a launch-shape choice): 0 = one CTA per work item, scheduled by
 * the hardware; 1 = one wave of persistent CTAs taking items from a counter;
 * 2 = one wave of persistent CTAs taking items from a counter, each
 * streaming its tiles through rings of shared-memory stages (a scheduler
 * warp, a loader warp, builder warps that form Khatri-Rao rows for pm_right
 * or restride the tile and stage H_1 for pm_left, contraction warps);
 * -1 (the default) = chosen at the next nncp_batch_run by timing every
 * schedule on this batch, cached per class of batch (order, largest rank,
 * magnitudes of the tensor count and element total) for the process.  An
 * output is computed the same way under each, so the results are the same
 * bits.  Both in -1..2, else NNCP_ERR_INVALID_ARG.  A run whose streamed
 * kernel gave up waiting on its pipeline (bounded waits, about two seconds)
 * returns NNCP_ERR_TIMEOUT. */
nncp_status nncp_batch_set_schedule(nncp_batch* b, int pm_right, int pm_left);
/* Test hook for the failure path: the limit, in SM clock cycles, of every
 * bounded wait of the streamed schedule's kernel (0, the default, is about
 * two seconds).  A tiny limit makes waits that are merely not yet satisfied
 * expire, so a run returns NNCP_ERR_TIMEOUT without any fault or hang; the
 * batch stays usable.  cycles < 0: NNCP_ERR_INVALID_ARG. */
nncp_status nncp_batch_set_wait_limit(nncp_batch* b, long long cycles);
/* The schedule the last run used (NNCP_ERR_NOT_READY before the first). */
nncp_status nncp_batch_get_schedule(const nncp_batch* b, int* pm_right, int* pm_left);
const char* nncp_batch_last_error(const nncp_batch* b);
void nncp_batch_destroy(nncp_batch* b);

/* Direct MTTKRP of one mode that allocates nothing (the paper has no
 * counterpart; this is a deployment convenience).
 *
 * For callers that must not allocate device memory: a host whose caching
 * allocator has already reserved the free device memory (so a cudaMalloc would
 * fail or fragment its pool), a plugin or UDF host that only hands in buffers
 * it allocated itself, or a latency-critical serving loop in which cudaMalloc
 * would synchronise the device and stall every other stream.
 *
 * Computes the same M_mode as nncp_mttkrp(ctx, mode, 0, M_dev) -- one direct
 * float32 pass over X with the Khatri-Rao rows formed on the fly -- from the
 * caller's X_dev (float32, mode-1 fastest), H_dev[0..N-1] (I_n x R row-major)
 * and M_dev (I_mode x R row-major), all device pointers, 16-byte aligned.
 * No context, no workspace: the split-K partial sums live in a file-scope
 * __device__ array of NNCP_NOALLOC_SCRATCH_FLOATS floats (8 MiB) that every
 * GPU which loads the library holds until the process exits.
 *   - Sizes: I_mode * R must be at most NNCP_NOALLOC_SCRATCH_FLOATS / 2;
 *     larger requests return NNCP_ERR_INVALID_ARG (nncp_global_error says
 *     why) and launch nothing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - Every call on a device shares the one array.  Each call overwrites the
 *     partials it reads, so nothing needs clearing, but calls whose kernels
 *     overlap on the GPU (different streams, or different host threads) race
 *     on it: serialise them.
 *   - Asynchronous on `stream` (cudaStream_t, NULL = legacy default). */
#define NNCP_NOALLOC_SCRATCH_FLOATS (1 << 21)
nncp_status nncp_mttkrp_noalloc(int N, const int64_t* dims, int R, const float* X_dev,
                                const float* const* H_dev, int mode, float* M_dev,
                                void* stream);

/* ---- Par-NNCP: one processor of a P_1 x ... x P_N grid (Alg. 2) ---------
 * The tensor is block-partitioned (Sec. IV-C "Data Distribution"): mode n is
 * cut into P_n contiguous blocks, block k = [floor(k I_n / P_n),
 * floor((k+1) I_n / P_n)), and processor p = (p_1..p_N) holds the block of its
 * coordinates, stored mode-1 fastest.  Every processor of the mode-n slice
 * (same p_n) holds the rows of factor n in block p_n; within that block each
 * slice member owns a contiguous piece of the rows, cut in P / P_n parts in
 * the order of the members' other coordinates (mode 1 fastest).  The object
 * does one processor's local computation; the caller runs the collectives
 * between the calls, per inner iteration n (Alg. 2):
 *   nncp_par_mttkrp    local MTTKRP of the block through a local dimension
 *                      tree (nncp_mttkrp_cached): block-rows x R;
 *   [Reduce-Scatter of it over the mode-n slice: the owned rows of M(n)]
 *   nncp_par_update    HALS sweep (Sec. II-B) on the owned rows of
 *                      W = H_n diag(lambda) with S = the Hadamard of the other
 *                      Grams, and this processor's W^T W and <M, W>;
 *   [All-Reduce of those R*R + 1 doubles over every processor]
 *   nncp_par_normalize lambda = column norms (float64), H_n = W / lambda on
 *                      the owned rows, G_n, and at n = N the fit (Sec. IV-B)
 *                      and the stopping test;
 *   [All-Gather of the owned rows over the mode-n slice into the block.]
 * Initialisation (Alg. 2, first loop): nncp_par_alpha_local +
 * [All-Reduce] + nncp_par_begin, then for every mode nncp_par_update with
 * M_owned = NULL (the Gram of the rows as given), [All-Reduce],
 * nncp_par_normalize with init = 1 (norms folded into lambda), [All-Gather].
 * Device buffers are the caller's: the local tensor block (float32), the N
 * factor blocks (block-rows x R, row-major, bound by nncp_par_set_data; the
 * owned rows of mode n start at row owned_lo - block_lo), M blocks and owned
 * rows.  The Grams, lambda, alpha and the fits are float64 host state held
 * redundantly by every processor. */
typedef struct nncp_par nncp_par;
/* dims: global mode lengths; grid: P_1..P_N (1 <= P_n <= I_n); coords: this
 * processor's p_1..p_N (0-based); precision of the local partial MTTKRPs
 * (NNCP_ERR_UNSUPPORTED if the local block cannot use it). */
nncp_status nncp_par_create(int N, const int64_t* dims, const int* grid, const int* coords, int R,
                            nncp_precision precision, nncp_par** out);
/* Layout of mode `mode` (1..N): factor block [block_lo, block_lo + block_rows),
 * owned rows [owned_lo, owned_lo + owned_rows) (global row indices), and this
 * processor's index and the member count of its mode-n slice.  Any output
 * may be NULL. */
nncp_status nncp_par_layout(const nncp_par* p, int mode, int64_t* block_lo, int64_t* block_rows,
                            int64_t* owned_lo, int64_t* owned_rows, int* slice_index,
                            int* slice_size);
nncp_status nncp_par_workspace_size(const nncp_par* p, size_t* bytes);
/* Caller-allocated device workspace (256-byte aligned); `stream` is the
 * stream every call of this object runs on. */
nncp_status nncp_par_set_workspace(nncp_par* p, void* dev_ptr, size_t bytes, void* stream);
nncp_status nncp_par_set_data(nncp_par* p, const float* X_local, float* const* H_block);
/* ||X_p||^2 of the local block (float64), for the All-Reduce giving alpha. */
nncp_status nncp_par_alpha_local(nncp_par* p, const float* X_local, double* local);
/* Starts a solve: alpha = ||X||^2 (the All-Reduce of the local values), the
 * stopping tolerance on |fit_k - fit_{k-1}|; lambda = 1, no fits yet. */
nncp_status nncp_par_begin(nncp_par* p, double alpha, double tol);
/* Local MTTKRP of mode `mode` into M_block (block-rows x R, device). */
nncp_status nncp_par_mttkrp(nncp_par* p, int mode, float* M_block);
/* HALS sweep on the owned rows (H_owned, device, in place: W) against
 * M_owned (device, the owned rows after the Reduce-Scatter), or, with
 * M_owned = NULL, no sweep (initialisation).  partial (host, R*R + 1
 * doubles): this processor's W^T W and <M, W>.  Blocks until done. */
nncp_status nncp_par_update(nncp_par* p, int mode, const float* M_owned, float* H_owned,
                            double* partial);
/* From the All-Reduced sums (host, R*R + 1 doubles): lambda (init = 1:
 * multiplied into lambda), H_owned = W / lambda, G_n; at mode N (init = 0)
 * the fit of the iteration (*fit_out) and *stop_out = 1 when
 * |fit_k - fit_{k-1}| < tol or the fit is not finite (NNCP_ERR_NUMERIC).
 * Blocks until done. */
nncp_status nncp_par_normalize(nncp_par* p, int mode, const double* sums, float* H_owned, int init,
                               double* fit_out, int* stop_out);
/* lambda (host, R doubles), the fits of the iterations so far (host, up to
 * max_fits) and their count; any output may be NULL. */
nncp_status nncp_par_result(const nncp_par* p, double* lambda_out, double* fits, int max_fits,
                            int* iters_out);
const char* nncp_par_last_error(const nncp_par* p);
void nncp_par_destroy(nncp_par* p);

/* Throughput probe (a measurement utility; the paper has no counterpart): one
 * launch on `stream` of a kernel that runs at the device's peak rate of
 *   kind 0: float32 FFMA on the CUDA cores (8 independent chains per thread,
 *           2048 threads per SM), the bound of NNCP_FP32_SIMT;
 *   kind 1: dense tcgen05 MMAs, kind::tf32, M = 128, N = 256, operands in
 *           shared memory, one CTA per SM (the bound of NNCP_TF32);
 *   kind 2: the same with kind::f16 bf16 operands;
 *   kind 3: packed float32 pairs (fma.rn.f32x2, two FMAs per instruction).
 * reps (1..2^24) scales the work; *flops_out receives the floating-point
 * operations the launch performs (2 per multiply-add).  sink_dev: 16 bytes
 * of device memory, 16-byte aligned, that the kernels may write (the MMA
 * probe sets its first int to 1 if its bounded wait expired).  The caller
 * times the launch with events on the stream. */
nncp_status nncp_peak_probe(int kind, int reps, void* sink_dev, void* stream, double* flops_out);

/* ---- Server: continuous batching of independent solve requests ----------
 * Each request is one NNCP-HALS problem (Alg. 1 with the normalisation and
 * error steps of Alg. 3, Sec. II-B HALS, Sec. IV-B fit; the paper has no
 * serving counterpart) within the batched limits: order 2..8, modes of
 * 1..256, rank 1..64, at most 2^31 - 1 elements.  A worker thread owns one
 * device pool of hbm_budget_bytes, taken with cudaMalloc at create on the
 * device current then.  Requests wait in submission order; the one at the
 * head is admitted when its footprint (nncp_server_footprint: tensor,
 * factors, dimension-tree nodes, partial sums, solver state) fits in the
 * pool and fewer than max_slots requests are active; admission copies its
 * tensor and initial factors to the device.  Between two sweeps the active
 * set may change; one sweep advances every active request by one outer
 * iteration; a request leaves when its own stopping rule holds
 * (|fit_k - fit_{k-1}| < tol, or max_iters), its factors and lambda are
 * copied back and its pool space is freed.  A request's results are the same
 * bits whatever else is active.
 * Two lanes, each admitted in submission order: requests of fewer than
 * NNCP_SERVER_SOLO_ELEMS elements (or the threshold given to
 * nncp_server_create_ex) share
 * the batched FP32 iteration of their order (root split 1, the same bits as
 * nncp_batch_run); larger ones, which fill the GPU alone, each run the
 * single-problem solver of nncp_solve_bound on their own stream -- root split by
 * nncp_default_split, the request's precision (mode 1 padded as in
 * nncp_solve_host where that lets the tensor-core path tile the shape, FP32
 * SIMT where nothing does), the same bits as nncp_solve_host with that
 * precision and root_split 0 -- launched in chunks of 4, 8, then 16
 * iterations and polled without blocking the batched lane.  At most
 * NNCP_SERVER_MAX_SOLO of those run at once (two: one's latency-bound mode
 * updates overlap the other's bandwidth-bound partial MTTKRPs, and neither
 * is slowed much), while small requests keep being admitted beside them.
 * No call blocks without a bound: submit copies the request (or borrows the
 * tensor, borrow_x) and returns, wait gives up after timeout_ms. */
#define NNCP_SERVER_SOLO_ELEMS (1LL << 22)
#define NNCP_SERVER_MAX_SOLO 2
typedef struct nncp_server nncp_server;
typedef struct {
  int N;                            /* order */
  const int64_t* dims;              /* N mode lengths */
  int R;                            /* rank */
  const float* X_host;              /* I_1...I_N floats, mode-1 fastest; copied by submit
                                       unless borrow_x */
  const float* const* H_init_host;  /* N pointers, I_n x R row-major; copied by submit */
  int max_iters;                    /* 1..65536 */
  double tol;                       /* stop when |fit_k - fit_{k-1}| < tol */
  nncp_precision precision;         /* solo lane: NNCP_FP32_SIMT, NNCP_TF32 or NNCP_SPLIT_BF16X3 */
  int borrow_x;                     /* 0: submit copies X_host.  1: the server keeps the pointer
                                       and uploads from it at admission; the caller keeps it
                                       valid and unchanged until the request is done (poll or
                                       wait returned its result).  From page-locked memory the
                                       upload is an asynchronous copy with no host-side copy. */
} nncp_request;
typedef struct {
  nncp_status status;       /* NNCP_OK, NNCP_ERR_NUMERIC (non-finite fit) or NNCP_ERR_CUDA */
  int iters;                /* outer iterations run */
  double fit;               /* 1 - eps of the last iteration (Sec. IV-B identity) */
  const double* lambda;     /* R weights, server-owned until nncp_server_release */
  const float* const* H;    /* N column-normalised factors, I_n x R row-major, server-owned */
  double t_submit, t_admit, t_done;  /* seconds on the server clock */
} nncp_result;
typedef struct {
  uint64_t submitted, completed, sweeps;
  int active, queued, peak_active;
  size_t budget, bytes_in_use, peak_bytes_in_use;
} nncp_server_stats;
/* max_slots >= 1: most requests active at once. */
nncp_status nncp_server_create(size_t hbm_budget_bytes, int max_slots, nncp_server** out);
/* As nncp_server_create, with the lane settings: requests of at least
 * solo_elems elements (>= 1) take the solo lane, and at most max_solo (>= 1)
 * of them run at once (the others wait in submission order; small requests
 * are admitted meanwhile). */
nncp_status nncp_server_create_ex(size_t hbm_budget_bytes, int max_slots, int64_t solo_elems,
                                  int max_solo, nncp_server** out);
/* Device bytes a request takes from the pool (NNCP_ERR_INVALID_ARG if its
 * shape is outside the limits). */
nncp_status nncp_server_footprint(const nncp_server* s, int N, const int64_t* dims, int R,
                                  int max_iters, nncp_precision precision, size_t* bytes);
/* Copies the request; *ticket identifies it.  NNCP_ERR_INVALID_ARG if the
 * shape is outside the limits or the footprint exceeds the budget. */
nncp_status nncp_server_submit(nncp_server* s, const nncp_request* req, uint64_t* ticket);
/* NNCP_ERR_NOT_READY until the request is done; then fills *res. */
nncp_status nncp_server_poll(nncp_server* s, uint64_t ticket, nncp_result* res);
/* Waits at most timeout_ms (>= 0): NNCP_ERR_TIMEOUT if still not done. */
nncp_status nncp_server_wait(nncp_server* s, uint64_t ticket, int timeout_ms, nncp_result* res);
/* Frees a done request's results (its pointers in nncp_result die). */
nncp_status nncp_server_release(nncp_server* s, uint64_t ticket);
nncp_status nncp_server_get_stats(nncp_server* s, nncp_server_stats* st);
/* Seconds since create on the clock of the t_* fields. */
double nncp_server_clock(const nncp_server* s);
const char* nncp_server_last_error(const nncp_server* s);
/* Stops the worker after its current sweep; pending requests are dropped. */
void nncp_server_destroy(nncp_server* s);

const char* nncp_last_error(const nncp_ctx* ctx);
/* Message of the last failure of a call that had no context to record it in. */
const char* nncp_global_error(void);
void nncp_destroy(nncp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NNCP_H */
