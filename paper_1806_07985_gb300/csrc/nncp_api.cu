// C-ABI entry points, dimension-tree planning and the BCD driver.
//
// The driver issues, per outer iteration, the dimension-tree schedule of
// Sec. IV-A (Fig. 1 shape): the root is split after mode s; the node of each
// half is produced by one partial MTTKRP from the tensor, and every node
// {a..b} yields the leaf M(a) by a multi-TTV over modes a+1..b and its child
// {a+1..b} by a multi-TTV over mode a with the freshly updated H(a).  Each
// leaf is followed by the factor update of Alg. 1/Alg. 3 (HALS sweep,
// normalisation, Gram), and the fit of Sec. IV-B closes the iteration.  The
// right node's first leaf comes out of its partial MTTKRP's epilogue where the
// tensor-core kernel can fuse it.  The outer iteration is captured into CUDA
// graphs of one and of four iterations (programmatic dependent launches inside)
// and relaunched.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nncp.h"
#include "nncp_internal.cuh"
#include "tc_kernels.cuh"

using namespace nncp;

namespace {

thread_local std::string g_error;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct nncp_ctx {
  int N = 0, R = 0;
  int64_t dims[kMaxModes] = {};
  int64_t I = 1;
  int precision = NNCP_FP32_SIMT;
  int split = 1;
  int dimtree = 1;  // 0: every M(n) by a direct MTTKRP (N tensor passes per iteration)
  cudaStream_t user_stream = nullptr;
  cudaStream_t work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int device = 0, num_sms = 148;

  char* ws = nullptr;
  size_t ws_bytes = 0;
  const void* X = nullptr;
  float* H[kMaxModes] = {};

  // workspace views
  float* node[2][kMaxModes] = {};  // [half][depth] node temporaries (>= 2 modes)
  float* Mbuf = nullptr;
  float* upd_part = nullptr;  // multi-CTA update partials
  float* partials = nullptr;
  size_t part_cap = 0;
  double* red_part = nullptr;
  int red_nparts = 0;
  SolveState st = {};
  TcScratch tc = {};

  bool fuse_leaf = true;              // fuse first leaf multi-TTVs into partial MTTKRPs
  int nls = NNCP_NLS_HALS;            // NLS-Update: HALS, block principal pivoting, ADMM, APG
  int nls_iters = 5;                  // inner iterations of the ADMM and APG updates
  float* U[kMaxModes] = {};           // ADMM duals, I_n x R, normalised frame (workspace)
  cudaGraphExec_t graph = nullptr;   // one outer iteration
  cudaGraphExec_t graph4 = nullptr;  // kGraphIters outer iterations, back to back
  int graph_kernels = 0;
  int* host_flags = nullptr;  // pinned
  double* host_dbl = nullptr; // pinned
  bool initialised = false;   // nncp_solve_begin ran on the current state
  // nncp_mttkrp_cached: versions of the factors (bumped by nncp_factor_changed)
  // and, per tree node [half][depth], whether it holds a result and the
  // factor versions it was computed from
  uint64_t fver[kMaxModes] = {};
  bool node_ok[2][kMaxModes] = {};
  uint64_t node_ver[2][kMaxModes][kMaxModes] = {};
  std::string err;
};

namespace {

nncp_status fail(nncp_ctx* c, nncp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_error = buf;
  return s;
}

nncp_status cuda_fail(nncp_ctx* c, cudaError_t e, const char* where) {
  return fail(c, NNCP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

int64_t prod(const int64_t* d, int a, int b) {  // inclusive range, 1 if empty
  int64_t p = 1;
  for (int m = a; m <= b; ++m) p *= d[m];
  return p;
}

KrpDesc krp(const nncp_ctx* c, int first, int last) {
  KrpDesc k;
  memset(&k, 0, sizeof k);
  k.nm = 0;
  for (int m = first; m <= last; ++m) {
    k.dim[k.nm] = c->dims[m];
    k.H[k.nm] = c->H[m];
    ++k.nm;
  }
  return k;
}

struct Plan {
  size_t node_off[2][kMaxModes];
  size_t node_bytes[2][kMaxModes];
  size_t M_off, upd_off, part_off, part_cap, gram_off, G_off, S_off, S32_off, lam_off, scal_off,
      fits_off, flags_off, red_off;
  size_t dual_off[kMaxModes];
  int red_nparts;
  size_t tc_off, tc_bytes;
  size_t total;
};

// Node {a..b} of the left chain is depth a (a = 0..s-2), of the right chain
// depth a - s (a = s..N-2).  Single-mode nodes are leaves and use Mbuf.
Plan make_plan(const nncp_ctx* c) {
  Plan p;
  memset(&p, 0, sizeof p);
  const int N = c->N, R = c->R, s = c->split;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  for (int a = 0; a + 1 < s; ++a) {
    p.node_bytes[0][a] = (size_t)prod(c->dims, a, s - 1) * R * sizeof(float);
    p.node_off[0][a] = take(p.node_bytes[0][a]);
  }
  for (int a = s; a + 1 < N; ++a) {
    p.node_bytes[1][a - s] = (size_t)prod(c->dims, a, N - 1) * R * sizeof(float);
    p.node_off[1][a - s] = take(p.node_bytes[1][a - s]);
  }
  int64_t maxIn = 0;
  for (int n = 0; n < N; ++n) maxIn = std::max(maxIn, c->dims[n]);
  p.M_off = take((size_t)maxIn * R * sizeof(float));
  size_t upd = 4;
  for (int n = 0; n < N; ++n)
    if (multi_update_ok(c->dims[n], R)) upd = std::max(upd, multi_update_scratch(c->dims[n], R));
  p.upd_off = take(upd * sizeof(float));

  // split-K partial capacity: max over every MTTKRP this context may launch
  size_t cap = 0;
  const int64_t IL = prod(c->dims, 0, s - 1), IR = prod(c->dims, s, N - 1);
  cap = std::max(cap, simt_mttkrp_partials(1, IL, IR, R, c->num_sms));
  cap = std::max(cap, simt_mttkrp_partials(IL, IR, 1, R, c->num_sms));
  for (int n = 0; n < N; ++n)
    cap = std::max(cap, simt_mttkrp_partials(prod(c->dims, 0, n - 1), c->dims[n],
                                             prod(c->dims, n + 1, N - 1), R, c->num_sms));
  for (int a = 0; a + 1 < s; ++a)
    cap = std::max(cap, mttv_leaf_partials(c->dims[a], prod(c->dims, a + 1, s - 1), R,
                                           c->num_sms));
  for (int a = s; a + 1 < N; ++a)
    cap = std::max(cap, mttv_leaf_partials(c->dims[a], prod(c->dims, a + 1, N - 1), R,
                                           c->num_sms));
  // read-only tree walks (nncp_mttkrp with use_dimtree) contract down to any leaf
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b)
      cap = std::max(cap, mttv_leaf_partials(c->dims[a], prod(c->dims, a + 1, b), R,
                                             c->num_sms));
  p.part_cap = cap;
  p.part_off = take(std::max<size_t>(cap, 1) * sizeof(float));

  int maxblocks = 0;
  for (int n = 0; n < N; ++n) maxblocks = std::max(maxblocks, hals_gram_blocks(c->dims[n]));
  p.gram_off = take((size_t)maxblocks * (R * R + 1) * sizeof(double));
  p.G_off = take((size_t)N * R * R * sizeof(double));
  p.S_off = take((size_t)N * R * R * sizeof(double));
  p.S32_off = take((size_t)R * R * sizeof(float));
  p.lam_off = take((size_t)R * sizeof(double));
  p.scal_off = take(16 * sizeof(double));
  p.fits_off = take((size_t)kFitCapacity * sizeof(double));
  p.flags_off = take(16 * sizeof(int));
  p.red_nparts = 4 * c->num_sms;
  p.red_off = take((size_t)2 * p.red_nparts * sizeof(double));
  p.tc_bytes = tc_scratch_bytes(c->N, c->dims, c->R, c->split, c->precision, c->num_sms);
  p.tc_off = take(std::max<size_t>(p.tc_bytes, 1));
  for (int n = 0; n < N; ++n) p.dual_off[n] = take((size_t)c->dims[n] * R * sizeof(float));
  p.total = off;
  return p;
}

void bind_workspace(nncp_ctx* c) {
  Plan p = make_plan(c);
  char* w = c->ws;
  for (int h = 0; h < 2; ++h)
    for (int d = 0; d < kMaxModes; ++d)
      c->node[h][d] = p.node_bytes[h][d] ? reinterpret_cast<float*>(w + p.node_off[h][d]) : nullptr;
  c->Mbuf = reinterpret_cast<float*>(w + p.M_off);
  c->upd_part = reinterpret_cast<float*>(w + p.upd_off);
  c->partials = reinterpret_cast<float*>(w + p.part_off);
  c->part_cap = p.part_cap;
  c->st.gram_part = reinterpret_cast<double*>(w + p.gram_off);
  c->st.G = reinterpret_cast<double*>(w + p.G_off);
  c->st.S = reinterpret_cast<double*>(w + p.S_off);
  c->st.S32 = reinterpret_cast<float*>(w + p.S32_off);
  c->st.lam = reinterpret_cast<double*>(w + p.lam_off);
  c->st.scalars = reinterpret_cast<double*>(w + p.scal_off);
  c->st.fits = reinterpret_cast<double*>(w + p.fits_off);
  c->st.flags = reinterpret_cast<int*>(w + p.flags_off);
  c->red_part = reinterpret_cast<double*>(w + p.red_off);
  c->red_nparts = p.red_nparts;
  for (int n = 0; n < kMaxModes; ++n)
    c->U[n] = n < c->N ? reinterpret_cast<float*>(w + p.dual_off[n]) : nullptr;
  c->tc.base = w + p.tc_off;
  c->tc.bytes = p.tc_bytes;
}

// Forget every cached tree node (their buffers are shared with the solver and
// the read-only tree walk, and the bound tensor, factors or layout may change).
void tree_cache_clear(nncp_ctx* c) {
  for (int h = 0; h < 2; ++h)
    for (int d = 0; d < kMaxModes; ++d) c->node_ok[h][d] = false;
}

void drop_graph(nncp_ctx* c) {
  tree_cache_clear(c);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph4) cudaGraphExecDestroy(c->graph4);
  c->graph = nullptr;
  c->graph4 = nullptr;
}

// ---- one partial MTTKRP from the root (precision-dependent) ----------------

cudaError_t pm_right(nncp_ctx* c, float* out, cudaStream_t st, const TcLeaf* leaf = nullptr) {
  const int s = c->split, N = c->N;
  const int64_t IL = prod(c->dims, 0, s - 1), IR = prod(c->dims, s, N - 1);
  KrpDesc none;
  memset(&none, 0, sizeof none);
  KrpDesc KQ = krp(c, s, N - 1);
  if (c->precision != NNCP_FP32_SIMT)
    return tc_partial_mttkrp(c->precision, /*contract_fast=*/0, c->X, IL, IR, KQ, c->R, out,
                             c->tc, c->num_sms, st, leaf);
  return launch_simt_mttkrp(static_cast<const float*>(c->X), 1, IL, IR, none, KQ, c->R, out,
                            c->partials, c->part_cap, c->num_sms, st);
}

cudaError_t pm_left(nncp_ctx* c, float* out, cudaStream_t st, const TcLeaf* leaf = nullptr) {
  const int s = c->split, N = c->N;
  const int64_t IL = prod(c->dims, 0, s - 1), IR = prod(c->dims, s, N - 1);
  KrpDesc none;
  memset(&none, 0, sizeof none);
  KrpDesc KL = krp(c, 0, s - 1);
  if (c->precision != NNCP_FP32_SIMT)
    return tc_partial_mttkrp(c->precision, /*contract_fast=*/1, c->X, IL, IR, KL, c->R, out,
                             c->tc, c->num_sms, st, leaf);
  return launch_simt_mttkrp(static_cast<const float*>(c->X), IL, IR, 1, KL, none, c->R, out,
                            c->partials, c->part_cap, c->num_sms, st);
}

cudaError_t update_mode(nncp_ctx* c, int n, cudaStream_t st) {
  if (c->nls == NNCP_NLS_APG) {
    if (cluster_update_ok(c->dims[n], c->R)) {
      cudaError_t e = launch_apg_rows(c->H[n], c->Mbuf, c->dims[n], c->R, c->nls_iters, c->st, st);
      if (e != cudaSuccess) return e;
      return launch_update_cluster(c->H[n], c->Mbuf, c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                                   n == c->N - 1, c->st, st, 0);
    }
    cudaError_t e = launch_apg_update(c->H[n], c->Mbuf, c->dims[n], c->R, c->nls_iters, c->st, st);
    if (e != cudaSuccess) return e;
    return launch_finalize(c->H[n], c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                           hals_gram_blocks(c->dims[n]), n == c->N - 1, 0, 0.0, c->st, st);
  }
  if (c->nls == NNCP_NLS_ADMM) {
    if (cluster_update_ok(c->dims[n], c->R)) {
      cudaError_t e = launch_admm_rows(c->H[n], c->U[n], c->Mbuf, c->dims[n], c->R,
                                       c->nls_iters, c->st, st);
      if (e != cudaSuccess) return e;
      return launch_update_cluster(c->H[n], c->Mbuf, c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                                   n == c->N - 1, c->st, st, 0, c->U[n]);
    }
    cudaError_t e = launch_admm_update(c->H[n], c->U[n], c->Mbuf, c->dims[n], c->R,
                                       c->nls_iters, c->st, st);
    if (e != cudaSuccess) return e;
    return launch_finalize(c->H[n], c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                           hals_gram_blocks(c->dims[n]), n == c->N - 1, 0, 0.0, c->st, st,
                           c->U[n]);
  }
  if (c->nls == NNCP_NLS_BPP) {
    if (cluster_update_ok(c->dims[n], c->R)) {
      cudaError_t e = launch_bpp_rows(c->H[n], c->Mbuf, c->dims[n], c->R, c->st, c->num_sms, st);
      if (e != cudaSuccess) return e;
      return launch_update_cluster(c->H[n], c->Mbuf, c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                                   n == c->N - 1, c->st, st, 0);
    }
    cudaError_t e = launch_bpp_update(c->H[n], c->Mbuf, c->dims[n], c->R, c->st, c->num_sms, st);
    if (e != cudaSuccess) return e;
    return launch_finalize(c->H[n], c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                           hals_gram_blocks(c->dims[n]), n == c->N - 1, 0, 0.0, c->st, st);
  }
  if (cluster_update_ok(c->dims[n], c->R))
    return launch_update_cluster(c->H[n], c->Mbuf, c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                                 n == c->N - 1, c->st, st);
  if (multi_update_ok(c->dims[n], c->R))
    return launch_update_multi(c->H[n], c->Mbuf, c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                               n == c->N - 1, c->st, c->upd_part, st);
  cudaError_t e = launch_hals_gram(c->H[n], c->Mbuf, c->dims[n], c->R, c->st, st);
  if (e != cudaSuccess) return e;
  return launch_finalize(c->H[n], c->dims[n], c->R, c->N, n, (n + 1) % c->N,
                         hals_gram_blocks(c->dims[n]), n == c->N - 1, 0, 0.0, c->st, st);
}

// Node {a..last} held in T (half h, depth d): leaf M(a), update, child node.
// leaf_done: M(a) is in Mbuf already (fused into the partial MTTKRP).
cudaError_t visit(nncp_ctx* c, const float* T, int a, int last, int h, int base,
                  cudaStream_t st, bool leaf_done = false) {
  const int R = c->R;
  cudaError_t e;
  if (a == last) return update_mode(c, a, st);  // T is Mbuf already
  KrpDesc rest = krp(c, a + 1, last);
  if (!leaf_done) {
    e = launch_mttv_leaf(T, c->dims[a], prod(c->dims, a + 1, last), rest, R, c->Mbuf,
                         c->partials, c->part_cap, c->num_sms, st);
    if (e != cudaSuccess) return e;
  }
  e = update_mode(c, a, st);
  if (e != cudaSuccess) return e;
  float* child = (a + 1 == last) ? c->Mbuf : c->node[h][a + 1 - base];
  e = launch_mttv_first(T, c->dims[a], prod(c->dims, a + 1, last), c->H[a], R, child, st);
  if (e != cudaSuccess) return e;
  return visit(c, child, a + 1, last, h, base, st);
}

// Node {a..last} of half h at depth d = a - first depends on every factor
// outside {a..last}.
bool node_current(const nncp_ctx* c, int h, int d, int a, int last) {
  if (!c->node_ok[h][d]) return false;
  for (int k = 0; k < c->N; ++k)
    if ((k < a || k > last) && c->node_ver[h][d][k] != c->fver[k]) return false;
  return true;
}

void node_stamp(nncp_ctx* c, int h, int d) {
  c->node_ok[h][d] = true;
  for (int k = 0; k < c->N; ++k) c->node_ver[h][d][k] = c->fver[k];
}

cudaError_t run_iteration(nncp_ctx* c, cudaStream_t st) {
  const int s = c->split, N = c->N;
  if (!c->dimtree) {
    // without the tree: a full MTTKRP per mode, each over the whole tensor
    for (int n = 0; n < N; ++n) {
      KrpDesc KL = krp(c, 0, n - 1), KQ = krp(c, n + 1, N - 1);
      cudaError_t e = launch_simt_mttkrp(static_cast<const float*>(c->X), prod(c->dims, 0, n - 1),
                                         c->dims[n], prod(c->dims, n + 1, N - 1), KL, KQ, c->R,
                                         c->Mbuf, c->partials, c->part_cap, c->num_sms, st);
      if (e == cudaSuccess) e = update_mode(c, n, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // a node of two or more modes gets its first leaf M(a) from the partial
  // MTTKRP's epilogue when the tensor-core kernel can fuse it
  const int64_t IL = prod(c->dims, 0, s - 1), IR = prod(c->dims, s, N - 1);
  TcLeaf lf{c->dims[0], krp(c, 1, s - 1), c->Mbuf};
  TcLeaf rf{c->dims[s], krp(c, s + 1, N - 1), c->Mbuf};
  const bool fuse_l = c->fuse_leaf && s >= 2 &&
                      tc_leaf_ok(c->precision, 0, IL, IR, c->R, lf.I, c->num_sms);
  const bool fuse_r = c->fuse_leaf && N - s >= 2 &&
                      tc_leaf_ok(c->precision, 1, IL, IR, c->R, rf.I, c->num_sms);
  float* TL = (s == 1) ? c->Mbuf : c->node[0][0];
  cudaError_t e = pm_right(c, TL, st, fuse_l ? &lf : nullptr);
  if (e != cudaSuccess) return e;
  e = visit(c, TL, 0, s - 1, 0, 0, st, fuse_l);
  if (e != cudaSuccess) return e;
  float* TR = (N - s == 1) ? c->Mbuf : c->node[1][0];
  e = pm_left(c, TR, st, fuse_r ? &rf : nullptr);
  if (e != cudaSuccess) return e;
  return visit(c, TR, s, N - 1, 1, s, st, fuse_r);
}

nncp_status check_ready(nncp_ctx* c) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (!c->ws) return fail(c, NNCP_ERR_INVALID_ARG, "workspace not set");
  if (!c->X) return fail(c, NNCP_ERR_INVALID_ARG, "tensor not set");
  for (int n = 0; n < c->N; ++n)
    if (!c->H[n]) return fail(c, NNCP_ERR_INVALID_ARG, "factor %d not set", n + 1);
  return NNCP_OK;
}

nncp_status begin_on_work(nncp_ctx* c) {
  CK(cudaEventRecord(c->ev_in, c->user_stream));
  CK(cudaStreamWaitEvent(c->work, c->ev_in, 0));
  return NNCP_OK;
}

nncp_status end_on_work(nncp_ctx* c) {
  CK(cudaEventRecord(c->ev_out, c->work));
  CK(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
  return NNCP_OK;
}

nncp_status solve_init(nncp_ctx* c, double tol) {
  cudaStream_t st = c->work;
  const int R = c->R, N = c->N;
  CK(launch_solve_reset(c->st, R, tol, st));
  for (int n = 0; n < N; ++n)
    CK(cudaMemsetAsync(c->U[n], 0, (size_t)c->dims[n] * R * sizeof(float), st));
  CK(launch_sumsq(c->X, c->precision == NNCP_BF16_STORED, c->I, c->red_part, c->red_nparts,
                  c->st.scalars, nullptr, st));
  for (int n = 0; n < N; ++n) {
    CK(launch_gram_only(c->H[n], c->dims[n], R, c->st, st));
    CK(launch_finalize(c->H[n], c->dims[n], R, N, n, -1, hals_gram_blocks(c->dims[n]), 0, 1,
                       0.0, c->st, st));
  }
  CK(launch_compute_S(c->st, N, R, 0, st));
  c->initialised = true;
  return NNCP_OK;
}

// Captures the outer iteration into a graph, once as one iteration and once as
// kGraphIters iterations back to back.  Inside a graph the kernels are launched
// with programmatic serialization, so a kernel can start (and, for the partial
// MTTKRP, stream tensor tiles) while its predecessor finishes; between two
// graph launches the dependency is a full one, so longer graphs leave fewer
// such boundaries.  Iterations after the stop flag is set do no work.
constexpr int kGraphIters = 4;

nncp_status capture_iterations(nncp_ctx* c, int iters, cudaGraphExec_t* out, int* kernels) {
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(c->work, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < iters && e == cudaSuccess; ++k) e = run_iteration(c, c->work);
  cudaError_t e2 = cudaStreamEndCapture(c->work, &g);
  if (e != cudaSuccess) {
    if (e2 == cudaSuccess) cudaGraphDestroy(g);
    return cuda_fail(c, e, "capturing the outer iteration");
  }
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
  if (kernels) {
    size_t nn = 0;
    *kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++*kernels;
        }
    }
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  return NNCP_OK;
}

nncp_status ensure_graph(nncp_ctx* c) {
  if (c->graph && c->graph4) return NNCP_OK;
  nncp_status s = NNCP_OK;
  if (!c->graph) s = capture_iterations(c, 1, &c->graph, &c->graph_kernels);
  if (s == NNCP_OK && !c->graph4) s = capture_iterations(c, kGraphIters, &c->graph4, nullptr);
  return s;
}

// `iters` outer iterations on the work stream
cudaError_t launch_iterations(nncp_ctx* c, int iters) {
  cudaError_t e = cudaSuccess;
  for (; iters >= kGraphIters && e == cudaSuccess; iters -= kGraphIters)
    e = cudaGraphLaunch(c->graph4, c->work);
  for (; iters > 0 && e == cudaSuccess; --iters) e = cudaGraphLaunch(c->graph, c->work);
  return e;
}

}  // namespace

namespace nncp {
void record_global_error(const char* msg) { g_error = msg; }
}  // namespace nncp

// =============================== C ABI ======================================

namespace nncp {

int ctx_solve_begin_tol(nncp_ctx* c, double tol) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  if ((s = begin_on_work(c)) != NNCP_OK) return s;
  if ((s = solve_init(c, tol)) != NNCP_OK) return s;
  if ((s = ensure_graph(c)) != NNCP_OK) return s;
  return end_on_work(c);
}

int64_t tc_padded_mode1(int precision, int N, const int64_t* dims, int R, int root_split) {
  if (precision != NNCP_TF32 && precision != NNCP_SPLIT_BF16X3 && precision != NNCP_BF16_STORED)
    return dims[0];
  if (N < 2 || N > kMaxModes) return dims[0];
  const int s0 = root_split ? root_split : nncp_default_split(N, dims);
  if (!tc_unsupported_reason(precision, N, dims, R, s0)) return dims[0];
  const int64_t q = precision == NNCP_BF16_STORED ? 8 : 4;
  int64_t pd[kMaxModes];
  for (int n = 0; n < N; ++n) pd[n] = dims[n];
  pd[0] = (dims[0] + q - 1) / q * q;
  const int s1 = root_split ? root_split : nncp_default_split(N, pd);
  return tc_unsupported_reason(precision, N, pd, R, s1) ? dims[0] : pd[0];
}

void ctx_device_state(const nncp_ctx* c, const int** flags, const double** lam,
                      const double** fits, const int** tc_error) {
  *flags = c->st.flags;
  *lam = c->st.lam;
  *fits = c->st.fits;
  *tc_error = c->tc.bytes ? tc_error_word(c->tc) : nullptr;
}

}  // namespace nncp

extern "C" {

const char* nncp_version(void) {
  return tc_available() ? "nncp-gb300 0.1 (sm_103a, tcgen05)" : "nncp-gb300 0.1 (sm_103a)";
}

int nncp_default_split(int N, const int64_t* dims) {
  if (N < 2 || !dims) return 1;
  double best = -1.0;
  int best_s = 1;
  for (int s = 1; s < N; ++s) {
    double l = 0.0, r = 0.0;
    for (int m = 0; m < s; ++m) l += log((double)dims[m]);
    for (int m = s; m < N; ++m) r += log((double)dims[m]);
    double score = fabs(l - r);
    if (best < 0.0 || score < best - 1e-12) {
      best = score;
      best_s = s;
    }
  }
  return best_s;
}

nncp_status nncp_create(int N, const int64_t* dims, int R, nncp_ctx** out) {
  if (!out) return fail(nullptr, NNCP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 2 || N > kMaxModes) return fail(nullptr, NNCP_ERR_INVALID_ARG, "N=%d not in [2,8]", N);
  if (R < 1 || R > kMaxRank) return fail(nullptr, NNCP_ERR_INVALID_ARG, "R=%d not in [1,128]", R);
  if (!dims) return fail(nullptr, NNCP_ERR_INVALID_ARG, "dims is NULL");
  int64_t I = 1;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1) return fail(nullptr, NNCP_ERR_INVALID_ARG, "dims[%d]=%lld < 1", n, (long long)dims[n]);
    if (dims[n] * (int64_t)R >= (1LL << 31))
      return fail(nullptr, NNCP_ERR_INVALID_ARG, "dims[%d]*R too large", n);
    I *= dims[n];
    if (I > (1LL << 40)) return fail(nullptr, NNCP_ERR_INVALID_ARG, "tensor too large");
  }
  nncp_ctx* c = new (std::nothrow) nncp_ctx();
  if (!c) return fail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "host allocation failed");
  c->N = N;
  c->R = R;
  for (int n = 0; n < N; ++n) c->dims[n] = dims[n];
  c->I = I;
  c->split = nncp_default_split(N, dims);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_flags, 16 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_dbl, 16 * sizeof(double));
  if (e == cudaSuccess) e = kernel_attributes_init();
  if (e != cudaSuccess) {
    nncp_status s = cuda_fail(nullptr, e, "nncp_create");
    nncp_destroy(c);
    return s;
  }
  *out = c;
  return NNCP_OK;
}

nncp_status nncp_set_dimtree(nncp_ctx* c, int enabled) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (!enabled && c->precision != NNCP_FP32_SIMT)
    return fail(c, NNCP_ERR_UNSUPPORTED, "the solve without the dimension tree is FP32 SIMT only");
  c->dimtree = enabled ? 1 : 0;
  drop_graph(c);
  return NNCP_OK;
}

nncp_status nncp_set_nls(nncp_ctx* c, int nls) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (nls != NNCP_NLS_HALS && nls != NNCP_NLS_BPP && nls != NNCP_NLS_ADMM && nls != NNCP_NLS_APG)
    return fail(c, NNCP_ERR_INVALID_ARG, "unknown NLS update %d", nls);
  if (nls == NNCP_NLS_BPP && c->R > 32)
    return fail(c, NNCP_ERR_UNSUPPORTED, "block principal pivoting supports R <= 32");
  if (nls == NNCP_NLS_ADMM && c->R > 32)
    return fail(c, NNCP_ERR_UNSUPPORTED, "the ADMM update supports R <= 32");
  if (nls == NNCP_NLS_APG && c->R > 32)
    return fail(c, NNCP_ERR_UNSUPPORTED, "the accelerated gradient update supports R <= 32");
  c->nls = nls;
  drop_graph(c);
  return NNCP_OK;
}

nncp_status nncp_set_nls_iters(nncp_ctx* c, int iters) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (iters < 1 || iters > 10000)
    return fail(c, NNCP_ERR_INVALID_ARG, "NLS inner iterations %d outside 1..10000", iters);
  c->nls_iters = iters;
  drop_graph(c);
  return NNCP_OK;
}

nncp_status nncp_set_leaf_fusion(nncp_ctx* c, int enabled) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  c->fuse_leaf = enabled != 0;
  drop_graph(c);
  return NNCP_OK;
}

nncp_status nncp_set_options(nncp_ctx* c, nncp_precision precision, int root_split, void* stream) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (precision < NNCP_FP32_SIMT || precision > NNCP_BF16_STORED)
    return fail(c, NNCP_ERR_INVALID_ARG, "unknown precision %d", precision);
  if (root_split < 0 || root_split >= c->N)
    return fail(c, NNCP_ERR_INVALID_ARG, "root_split %d not in [0, N-1]", root_split);
  if (precision != NNCP_FP32_SIMT && !tc_available())
    return fail(c, NNCP_ERR_UNSUPPORTED, "tensor-core kernels not compiled in");
  if (precision != NNCP_FP32_SIMT && !c->dimtree)
    return fail(c, NNCP_ERR_UNSUPPORTED, "the solve without the dimension tree is FP32 SIMT only");
  const int split = root_split ? root_split : nncp_default_split(c->N, c->dims);
  if (precision != NNCP_FP32_SIMT) {
    const char* why = tc_unsupported_reason(precision, c->N, c->dims, c->R, split);
    if (why) return fail(c, NNCP_ERR_UNSUPPORTED, "%s", why);
  }
  const bool relayout = (split != c->split) || (precision != c->precision);
  c->precision = precision;
  c->split = split;
  c->user_stream = static_cast<cudaStream_t>(stream);
  drop_graph(c);
  if (relayout && c->ws) {
    c->ws = nullptr;  // the caller must size and set a new workspace
    c->ws_bytes = 0;
  }
  c->initialised = false;
  return NNCP_OK;
}

nncp_status nncp_workspace_size(const nncp_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null argument");
  *bytes = make_plan(c).total;
  return NNCP_OK;
}

nncp_status nncp_set_workspace(nncp_ctx* c, void* dev_ptr, size_t bytes) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
    return fail(c, NNCP_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  size_t need = make_plan(c).total;
  if (bytes < need)
    return fail(c, NNCP_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", bytes, need);
  c->ws = static_cast<char*>(dev_ptr);
  c->ws_bytes = bytes;
  bind_workspace(c);
  drop_graph(c);
  if (c->tc.bytes) {
    CK(cudaMemsetAsync(c->tc.base, 0, 256, c->work));
    CK(cudaStreamSynchronize(c->work));
  }
  c->initialised = false;
  return NNCP_OK;
}

nncp_status nncp_set_tensor(nncp_ctx* c, const void* X_dev) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (!X_dev || (reinterpret_cast<uintptr_t>(X_dev) & 15))
    return fail(c, NNCP_ERR_INVALID_ARG, "tensor must be a 16-byte aligned device pointer");
  c->X = X_dev;
  drop_graph(c);
  c->initialised = false;
  return NNCP_OK;
}

nncp_status nncp_set_factors(nncp_ctx* c, float* const* H_dev) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (!H_dev) return fail(c, NNCP_ERR_INVALID_ARG, "factor array is NULL");
  for (int n = 0; n < c->N; ++n)
    if (!H_dev[n] || (reinterpret_cast<uintptr_t>(H_dev[n]) & 15))
      return fail(c, NNCP_ERR_INVALID_ARG, "factor %d must be a 16-byte aligned device pointer", n + 1);
  for (int n = 0; n < c->N; ++n) c->H[n] = H_dev[n];
  drop_graph(c);
  c->initialised = false;
  return NNCP_OK;
}

nncp_status nncp_mttkrp(nncp_ctx* c, int mode, int use_dimtree, float* M_dev) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  tree_cache_clear(c);
  if (mode < 1 || mode > c->N) return fail(c, NNCP_ERR_INVALID_ARG, "mode %d not in [1, N]", mode);
  if (!M_dev) return fail(c, NNCP_ERR_INVALID_ARG, "output is NULL");
  const int n = mode - 1, N = c->N, R = c->R, sp = c->split;
  cudaStream_t st = c->user_stream;
  KrpDesc none;
  memset(&none, 0, sizeof none);
  if (!use_dimtree) {
    if (c->precision == NNCP_BF16_STORED)
      return fail(c, NNCP_ERR_UNSUPPORTED, "the direct MTTKRP reads a float32 tensor");
    KrpDesc KL = krp(c, 0, n - 1), KQ = krp(c, n + 1, N - 1);
    CK(launch_simt_mttkrp(static_cast<const float*>(c->X), prod(c->dims, 0, n - 1), c->dims[n],
                          prod(c->dims, n + 1, N - 1), KL, KQ, R, M_dev, c->partials,
                          c->part_cap, c->num_sms, st));
    return NNCP_OK;
  }
  // read-only walk down the tree to leaf n
  const bool left = n < sp;
  const int first = left ? 0 : sp, last = left ? sp - 1 : N - 1;
  const int h = left ? 0 : 1;
  float* T = (first == last) ? M_dev : c->node[h][0];
  CK(left ? pm_right(c, T, st) : pm_left(c, T, st));
  for (int a = first; a < n; ++a) {
    // contract mode a: node {a..last} -> {a+1..last}
    float* child = (a + 1 == last) ? M_dev : c->node[h][a + 1 - first];
    CK(launch_mttv_first(T, c->dims[a], prod(c->dims, a + 1, last), c->H[a], R, child, st));
    T = child;
  }
  if (n < last) {
    KrpDesc rest = krp(c, n + 1, last);
    CK(launch_mttv_leaf(T, c->dims[n], prod(c->dims, n + 1, last), rest, R, M_dev, c->partials,
                        c->part_cap, c->num_sms, st));
  }
  return NNCP_OK;
}

nncp_status nncp_partial_mttkrp(nncp_ctx* c, int side, float* T_dev) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  if (side != 0 && side != 1) return fail(c, NNCP_ERR_INVALID_ARG, "side must be 0 or 1");
  if (!T_dev) return fail(c, NNCP_ERR_INVALID_ARG, "output is NULL");
  CK(side == 0 ? pm_right(c, T_dev, c->user_stream) : pm_left(c, T_dev, c->user_stream));
  return NNCP_OK;
}

nncp_status nncp_factor_changed(nncp_ctx* c, int mode) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  if (mode < 1 || mode > c->N) return fail(c, NNCP_ERR_INVALID_ARG, "mode %d not in [1, N]", mode);
  ++c->fver[mode - 1];
  return NNCP_OK;
}

nncp_status nncp_mttkrp_cached(nncp_ctx* c, int mode, float* M_dev) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  if (mode < 1 || mode > c->N) return fail(c, NNCP_ERR_INVALID_ARG, "mode %d not in [1, N]", mode);
  if (!M_dev) return fail(c, NNCP_ERR_INVALID_ARG, "output is NULL");
  const int n = mode - 1, N = c->N, R = c->R, sp = c->split;
  cudaStream_t st = c->user_stream;
  const bool left = n < sp;
  const int h = left ? 0 : 1, first = left ? 0 : sp, last = left ? sp - 1 : N - 1;
  if (first == last) {
    // a one-mode half: its partial MTTKRP is M(n) itself
    CK(left ? pm_right(c, M_dev, st) : pm_left(c, M_dev, st));
    return NNCP_OK;
  }
  float* T = c->node[h][0];
  if (!node_current(c, h, 0, first, last)) {
    CK(left ? pm_right(c, T, st) : pm_left(c, T, st));
    node_stamp(c, h, 0);
  }
  for (int a = first; a < n; ++a) {
    const int d = a + 1 - first;  // depth of the child node {a+1..last}
    if (a + 1 == last) {
      // the child is the one-mode node {last} = M(last)
      CK(launch_mttv_first(T, c->dims[a], prod(c->dims, a + 1, last), c->H[a], R, M_dev, st));
      return NNCP_OK;
    }
    float* child = c->node[h][d];
    if (!node_current(c, h, d, a + 1, last)) {
      CK(launch_mttv_first(T, c->dims[a], prod(c->dims, a + 1, last), c->H[a], R, child, st));
      node_stamp(c, h, d);
    }
    T = child;
  }
  KrpDesc rest = krp(c, n + 1, last);
  CK(launch_mttv_leaf(T, c->dims[n], prod(c->dims, n + 1, last), rest, R, M_dev, c->partials,
                      c->part_cap, c->num_sms, st));
  return NNCP_OK;
}

nncp_status nncp_iteration_kernels(nncp_ctx* c, int* count) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  if (!count) return fail(c, NNCP_ERR_INVALID_ARG, "count is NULL");
  if ((s = ensure_graph(c)) != NNCP_OK) return s;
  *count = c->graph_kernels;
  return NNCP_OK;
}

nncp_status nncp_solve_begin(nncp_ctx* c) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  tree_cache_clear(c);
  if ((s = begin_on_work(c)) != NNCP_OK) return s;
  if ((s = solve_init(c, 0.0)) != NNCP_OK) return s;
  if ((s = ensure_graph(c)) != NNCP_OK) return s;
  return end_on_work(c);
}

nncp_status nncp_iterate(nncp_ctx* c, int iters) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  if (!c->initialised) return fail(c, NNCP_ERR_INVALID_ARG, "call nncp_solve_begin first");
  tree_cache_clear(c);
  if ((s = ensure_graph(c)) != NNCP_OK) return s;
  if ((s = begin_on_work(c)) != NNCP_OK) return s;
  CK(launch_iterations(c, iters));
  return end_on_work(c);
}

nncp_status nncp_solve_bound(nncp_ctx* c, int max_iters, double tol, double* lambda_out,
                             int* iters_out, double* fit_out) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  tree_cache_clear(c);
  if (max_iters < 1) return fail(c, NNCP_ERR_INVALID_ARG, "max_iters < 1");
  if (max_iters > kFitCapacity) return fail(c, NNCP_ERR_INVALID_ARG, "max_iters > %d", kFitCapacity);
  if ((s = begin_on_work(c)) != NNCP_OK) return s;
  if ((s = solve_init(c, tol)) != NNCP_OK) return s;
  if ((s = ensure_graph(c)) != NNCP_OK) return s;
  int launched = 0, check_every = 4;
  while (launched < max_iters) {
    int batch = std::min(check_every, max_iters - launched);
    CK(launch_iterations(c, batch));
    launched += batch;
    CK(cudaMemcpyAsync(c->host_flags, c->st.flags, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                       c->work));
    CK(cudaStreamSynchronize(c->work));
    if (c->host_flags[0]) break;
    check_every = std::min(check_every * 2, 32);
  }
  CK(cudaMemcpyAsync(c->host_flags, c->st.flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->work));
  CK(cudaStreamSynchronize(c->work));
  const int iters = c->host_flags[2];
  if (lambda_out)
    CK(cudaMemcpy(lambda_out, c->st.lam, c->R * sizeof(double), cudaMemcpyDeviceToHost));
  double fit = 0.0;
  if (iters > 0)
    CK(cudaMemcpy(&fit, c->st.fits + (iters - 1), sizeof(double), cudaMemcpyDeviceToHost));
  if (iters_out) *iters_out = iters;
  if (fit_out) *fit_out = fit;
  if ((s = end_on_work(c)) != NNCP_OK) return s;
  if (c->tc.bytes) {
    int tc_err = 0;
    CK(cudaMemcpy(&tc_err, tc_error_word(c->tc), sizeof(int), cudaMemcpyDeviceToHost));
    if (tc_err)
      return fail(c, NNCP_ERR_TIMEOUT, "a tensor-core kernel gave up waiting (error word set)");
  }
  if (c->host_flags[3]) return fail(c, NNCP_ERR_NUMERIC, "non-finite fit at iteration %d", iters);
  return NNCP_OK;
}

nncp_status nncp_solve(nncp_ctx* c, const void* X_dev, float* const* H_dev, double* lambda_out,
                       int max_iters, double tol, int* iters_out, double* fit_out) {
  if (!c) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null context");
  nncp_status s;
  // rebinding only what changed keeps the captured iteration graphs
  if (X_dev && X_dev != c->X && (s = nncp_set_tensor(c, X_dev)) != NNCP_OK) return s;
  if (H_dev) {
    bool same = true;
    for (int n = 0; n < c->N; ++n) same = same && H_dev[n] == c->H[n];
    if (!same && (s = nncp_set_factors(c, H_dev)) != NNCP_OK) return s;
  }
  return nncp_solve_bound(c, max_iters, tol, lambda_out, iters_out, fit_out);
}

nncp_status nncp_fit_history(const nncp_ctx* cc, double* fits, int max_count, int* count) {
  nncp_ctx* c = const_cast<nncp_ctx*>(cc);
  if (!c || !fits || !count) return fail(c, NNCP_ERR_INVALID_ARG, "null argument");
  if (!c->ws) return fail(c, NNCP_ERR_INVALID_ARG, "workspace not set");
  CK(cudaStreamSynchronize(c->work));
  int flags[4];
  CK(cudaMemcpy(flags, c->st.flags, sizeof flags, cudaMemcpyDeviceToHost));
  int n = std::min(std::min(flags[2], max_count), kFitCapacity);
  if (n > 0) CK(cudaMemcpy(fits, c->st.fits, n * sizeof(double), cudaMemcpyDeviceToHost));
  *count = n;
  return NNCP_OK;
}

nncp_status nncp_fit(nncp_ctx* c, int exact, double* fit_out) {
  nncp_status s = check_ready(c);
  if (s != NNCP_OK) return s;
  if (!fit_out) return fail(c, NNCP_ERR_INVALID_ARG, "fit_out is NULL");
  if (!exact) {
    double f[1];
    int n = 0;
    double hist[1];
    (void)hist;
    int flags[4];
    CK(cudaStreamSynchronize(c->work));
    CK(cudaMemcpy(flags, c->st.flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[2] < 1) return fail(c, NNCP_ERR_NOT_READY, "no solve iteration has run");
    n = std::min(flags[2], kFitCapacity);
    CK(cudaMemcpy(f, c->st.fits + (n - 1), sizeof(double), cudaMemcpyDeviceToHost));
    *fit_out = f[0];
    return NNCP_OK;
  }
  if (c->precision == NNCP_BF16_STORED)
    return fail(c, NNCP_ERR_UNSUPPORTED, "the explicit residual reads a float32 tensor");
  if (!c->initialised) return fail(c, NNCP_ERR_NOT_READY, "no solve has run (lambda unset)");
  if ((s = begin_on_work(c)) != NNCP_OK) return s;
  CK(launch_explicit_residual(static_cast<const float*>(c->X), c->N, c->dims, c->R, c->H,
                              c->st.lam, c->red_part, c->red_nparts, c->st.scalars + 8, c->work));
  CK(cudaMemcpyAsync(c->host_dbl, c->st.scalars + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                     c->work));
  CK(cudaStreamSynchronize(c->work));
  *fit_out = 1.0 - sqrt(c->host_dbl[0] / c->host_dbl[1]);
  return end_on_work(c);
}

nncp_status nncp_tensor_to_bf16(const float* X_dev, uint16_t* Xb_dev, int64_t n, void* stream) {
  if (!X_dev || !Xb_dev || n < 0) return fail(nullptr, NNCP_ERR_INVALID_ARG, "bad argument");
  nncp_ctx* c = nullptr;
  CK(launch_to_bf16(X_dev, Xb_dev, n, static_cast<cudaStream_t>(stream)));
  return NNCP_OK;
}

static nncp_status solve_host_uncached(int N, const int64_t* dims, int R, const float* X_host,
                            float* const* H_host, nncp_precision precision, int root_split,
                            int max_iters, double tol, double* lambda_out, int* iters_out,
                            double* fit_out) {
  if (!X_host || !H_host) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null host buffer");
  if (N < 2 || N > kMaxModes || !dims) return fail(nullptr, NNCP_ERR_INVALID_ARG, "N=%d not in [2,8]", N);
  // a tensor-core precision on a shape it cannot tile: store mode 1 padded
  // with zero slices (H_1 with zero rows, which HALS keeps zero)
  int64_t pd[kMaxModes];
  for (int n = 0; n < N; ++n) pd[n] = dims[n];
  if (dims[0] >= 1 && R >= 1) pd[0] = tc_padded_mode1(precision, N, dims, R, root_split);
  const bool padded = pd[0] != dims[0];
  nncp_ctx* c = nullptr;
  nncp_status s = nncp_create(N, pd, R, &c);
  if (s != NNCP_OK) return s;
  void* dX = nullptr;
  void* dXb = nullptr;
  float* dH[kMaxModes] = {};
  void* dws = nullptr;
  size_t wsb = 0;
  cudaStream_t st = c->work;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(dX);
    cudaFree(dXb);
    for (int n = 0; n < N; ++n) cudaFree(dH[n]);
    cudaFree(dws);
    nncp_destroy(c);
  };
#define CKH(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      s = cuda_fail(nullptr, e_, #call);                 \
      cleanup();                                         \
      return s;                                          \
    }                                                    \
  } while (0)
  s = nncp_set_options(c, precision, root_split, st);
  if (s != NNCP_OK) {
    g_error = c->err;
    cleanup();
    return s;
  }
  CKH(cudaMalloc(&dX, (size_t)c->I * sizeof(float)));
  if (padded) {
    const size_t rows = (size_t)(c->I / pd[0]);
    CKH(cudaMemsetAsync(dX, 0, (size_t)c->I * sizeof(float), st));
    CKH(cudaMemcpy2DAsync(dX, (size_t)pd[0] * sizeof(float), X_host, (size_t)dims[0] * sizeof(float),
                          (size_t)dims[0] * sizeof(float), rows, cudaMemcpyHostToDevice, st));
  } else {
    CKH(cudaMemcpyAsync(dX, X_host, (size_t)c->I * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  const void* Xuse = dX;
  if (precision == NNCP_BF16_STORED) {
    CKH(cudaMalloc(&dXb, (size_t)c->I * 2));
    CKH(launch_to_bf16(static_cast<float*>(dX), static_cast<uint16_t*>(dXb), c->I, st));
    Xuse = dXb;
  }
  for (int n = 0; n < N; ++n) {
    CKH(cudaMalloc(&dH[n], (size_t)pd[n] * R * sizeof(float)));
    if (pd[n] != dims[n]) CKH(cudaMemsetAsync(dH[n], 0, (size_t)pd[n] * R * sizeof(float), st));
    CKH(cudaMemcpyAsync(dH[n], H_host[n], (size_t)dims[n] * R * sizeof(float),
                        cudaMemcpyHostToDevice, st));
  }
  nncp_workspace_size(c, &wsb);
  CKH(cudaMalloc(&dws, wsb));
  if ((s = nncp_set_workspace(c, dws, wsb)) != NNCP_OK ||
      (s = nncp_set_tensor(c, Xuse)) != NNCP_OK || (s = nncp_set_factors(c, dH)) != NNCP_OK ||
      (s = nncp_solve_bound(c, max_iters, tol, lambda_out, iters_out, fit_out)) != NNCP_OK) {
    g_error = c->err;
    cleanup();
    return s;
  }
  for (int n = 0; n < N; ++n)
    CKH(cudaMemcpyAsync(H_host[n], dH[n], (size_t)dims[n] * R * sizeof(float),
                        cudaMemcpyDeviceToHost, st));
  CKH(cudaStreamSynchronize(st));
  cleanup();
  return NNCP_OK;
#undef CKH
}

namespace {
// The plan nncp_solve_host keeps between calls: the context of the last shape
// solved (with its captured graphs) and its device buffers.  A call with the
// same stored shape, rank, precision and split on the same device reuses them:
// no allocation, no graph capture -- the graphs stay valid because the
// buffers do not move.  Held on the heap and never destroyed at exit (the
// driver reclaims it); nncp_solve_host_release frees it earlier.
struct HostPlan {
  std::mutex mu;
  int device = -1, N = 0, R = 0, precision = -1, split = -1;
  int64_t dims[nncp::kMaxModes] = {};
  nncp_ctx* c = nullptr;
  void* dX = nullptr;
  void* dXb = nullptr;
  float* dH[nncp::kMaxModes] = {};
  void* dws = nullptr;
  bool matches(int dev, int n, const int64_t* d, int r, int prec, int sp) const {
    if (!c || dev != device || n != N || r != R || prec != precision || sp != split) return false;
    for (int k = 0; k < n; ++k)
      if (d[k] != dims[k]) return false;
    return true;
  }
  void release() {
    if (c && c->work) cudaStreamSynchronize(c->work);
    cudaFree(dX);
    cudaFree(dXb);
    for (int k = 0; k < nncp::kMaxModes; ++k) cudaFree(dH[k]);
    cudaFree(dws);
    nncp_destroy(c);
    c = nullptr;
    dX = dXb = dws = nullptr;
    for (int k = 0; k < nncp::kMaxModes; ++k) dH[k] = nullptr;
    device = -1;
  }
};
HostPlan* g_host_plan = new HostPlan;
}  // namespace

nncp_status nncp_solve_host(int N, const int64_t* dims, int R, const float* X_host,
                            float* const* H_host, nncp_precision precision, int root_split,
                            int max_iters, double tol, double* lambda_out, int* iters_out,
                            double* fit_out) {
  if (!X_host || !H_host) return fail(nullptr, NNCP_ERR_INVALID_ARG, "null host buffer");
  if (N < 2 || N > kMaxModes || !dims) return fail(nullptr, NNCP_ERR_INVALID_ARG, "N=%d not in [2,8]", N);
  for (int n = 0; n < N; ++n)
    if (dims[n] < 1 || !H_host[n]) return fail(nullptr, NNCP_ERR_INVALID_ARG, "invalid mode %d", n + 1);
  if (R < 1) return fail(nullptr, NNCP_ERR_INVALID_ARG, "R=%d", R);
  std::unique_lock<std::mutex> lk(g_host_plan->mu, std::try_to_lock);
  if (!lk.owns_lock())  // another thread holds the plan: solve without it
    return solve_host_uncached(N, dims, R, X_host, H_host, precision, root_split, max_iters, tol,
                               lambda_out, iters_out, fit_out);
  HostPlan& P = *g_host_plan;
  int64_t pd[kMaxModes];
  for (int n = 0; n < N; ++n) pd[n] = dims[n];
  pd[0] = tc_padded_mode1(precision, N, dims, R, root_split);
  const bool padded = pd[0] != dims[0];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, NNCP_ERR_CUDA, "cudaGetDevice");
  nncp_status s = NNCP_OK;
#define CKP(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      s = cuda_fail(nullptr, e_, #call);                 \
      P.release();                                       \
      return s;                                          \
    }                                                    \
  } while (0)
  if (!P.matches(dev, N, pd, R, precision, root_split)) {
    P.release();
    if ((s = nncp_create(N, pd, R, &P.c)) != NNCP_OK) return s;
    if ((s = nncp_set_options(P.c, precision, root_split, P.c->work)) != NNCP_OK) {
      g_error = P.c->err;
      P.release();
      return s;
    }
    const size_t I = (size_t)P.c->I;
    CKP(cudaMalloc(&P.dX, I * sizeof(float)));
    if (padded) CKP(cudaMemsetAsync(P.dX, 0, I * sizeof(float), P.c->work));  // zero slices stay zero
    if (precision == NNCP_BF16_STORED) CKP(cudaMalloc(&P.dXb, I * 2));
    for (int n = 0; n < N; ++n) CKP(cudaMalloc(&P.dH[n], (size_t)pd[n] * R * sizeof(float)));
    size_t wsb = 0;
    nncp_workspace_size(P.c, &wsb);
    CKP(cudaMalloc(&P.dws, wsb));
    if ((s = nncp_set_workspace(P.c, P.dws, wsb)) != NNCP_OK ||
        (s = nncp_set_tensor(P.c, P.dXb ? P.dXb : P.dX)) != NNCP_OK ||
        (s = nncp_set_factors(P.c, P.dH)) != NNCP_OK) {
      g_error = P.c->err;
      P.release();
      return s;
    }
    P.device = dev;
    P.N = N;
    P.R = R;
    P.precision = precision;
    P.split = root_split;
    for (int n = 0; n < N; ++n) P.dims[n] = pd[n];
  }
  cudaStream_t st = P.c->work;
  const size_t rows = (size_t)(P.c->I / pd[0]);
  if (padded)
    CKP(cudaMemcpy2DAsync(P.dX, (size_t)pd[0] * sizeof(float), X_host, (size_t)dims[0] * sizeof(float),
                          (size_t)dims[0] * sizeof(float), rows, cudaMemcpyHostToDevice, st));
  else
    CKP(cudaMemcpyAsync(P.dX, X_host, (size_t)P.c->I * sizeof(float), cudaMemcpyHostToDevice, st));
  if (P.dXb)
    CKP(launch_to_bf16(static_cast<float*>(P.dX), static_cast<uint16_t*>(P.dXb), P.c->I, st));
  for (int n = 0; n < N; ++n) {
    if (pd[n] != dims[n]) CKP(cudaMemsetAsync(P.dH[n], 0, (size_t)pd[n] * R * sizeof(float), st));
    CKP(cudaMemcpyAsync(P.dH[n], H_host[n], (size_t)dims[n] * R * sizeof(float),
                        cudaMemcpyHostToDevice, st));
  }
  if ((s = nncp_solve_bound(P.c, max_iters, tol, lambda_out, iters_out, fit_out)) != NNCP_OK) {
    g_error = P.c->err;
    P.release();
    return s;
  }
  for (int n = 0; n < N; ++n)
    CKP(cudaMemcpyAsync(H_host[n], P.dH[n], (size_t)dims[n] * R * sizeof(float),
                        cudaMemcpyDeviceToHost, st));
  CKP(cudaStreamSynchronize(st));
  return NNCP_OK;
#undef CKP
}

void nncp_solve_host_release(void) {
  std::lock_guard<std::mutex> lk(g_host_plan->mu);
  g_host_plan->release();
}

const char* nncp_last_error(const nncp_ctx* c) { return c ? c->err.c_str() : g_error.c_str(); }

const char* nncp_global_error(void) { return g_error.c_str(); }

void nncp_destroy(nncp_ctx* c) {
  if (!c) return;
  if (c->work) cudaStreamSynchronize(c->work);
  drop_graph(c);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->work) cudaStreamDestroy(c->work);
  if (c->host_flags) cudaFreeHost(c->host_flags);
  if (c->host_dbl) cudaFreeHost(c->host_dbl);
  delete c;
}

}  // extern "C"
