// C ABI of the batched solver: many independent NNCP-HALS problems of one
// order N advanced together, one graph-captured outer iteration at a time.
// Also the host side shared with the server: per-tensor layout and the work
// lists of a batch composition.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <map>
#include <string>
#include <vector>

#include "../../include/nncp.h"
#include "batch_kernels.cuh"

namespace nncp {

namespace {
size_t al(size_t v) { return (v + 255) / 256 * 256; }
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
}  // namespace

size_t b_tensor_layout(int N, const int64_t* dm, int R, int fit_cap, BTensor* d, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = al(off + bytes);
    return base ? base + o : nullptr;
  };
  int64_t maxI = 0, I = 1;
  for (int n = 0; n < N; ++n) {
    maxI = std::max(maxI, dm[n]);
    I *= dm[n];
  }
  // root -> {1}: chunks of whole tiles, about kRightTileTarget elements, at most kMaxChunks
  const int64_t J = I / dm[0];
  const int rows_r = b_rows_right((int)dm[0], R);
  int64_t tiles = std::max<int64_t>(1, kRightTileTarget / ((int64_t)rows_r * dm[0]));
  tiles = std::max<int64_t>(tiles, cdiv(J, (int64_t)kMaxChunks * rows_r));
  const int64_t jchunk = tiles * rows_r;
  const int nchunk = (int)cdiv(J, jchunk);
  // node {a..N} phases: leaf chunks (at most kMaxChunks) and child row blocks
  int leaf_kc[kMaxModes] = {0}, leaf_nkc[kMaxModes] = {0}, first_jb[kMaxModes] = {0};
  int64_t lpart_floats = 1;
  for (int a = 1; a + 1 < N; ++a) {
    int64_t K = 1;
    for (int m = a + 1; m < N; ++m) K *= dm[m];
    const int64_t E = dm[a] * R;
    int64_t kc = std::max<int64_t>(1, kItemElems / std::min<int64_t>(E, kLeafBlock));
    kc = std::max<int64_t>(kc, cdiv(K, kMaxChunks));
    leaf_kc[a] = (int)kc;
    leaf_nkc[a] = (int)cdiv(K, kc);
    lpart_floats = std::max<int64_t>(lpart_floats, leaf_nkc[a] * E);
    first_jb[a] = (int)std::max<int64_t>(1, kItemElems / E);
  }
  if (d) {
    memset(d, 0, sizeof *d);
    d->N = N;
    d->R = R;
    for (int n = 0; n < N; ++n) d->dims[n] = dm[n];
    d->I = I;
    d->jchunk = jchunk;
    d->nchunk = nchunk;
    d->rows_r = rows_r;
    d->rows_l = b_rows_left((int)dm[0]);
    for (int a = 0; a < kMaxModes; ++a) {
      d->leaf_kc[a] = leaf_kc[a];
      d->leaf_nkc[a] = leaf_nkc[a];
      d->first_jb[a] = first_jb[a];
    }
    d->fit_cap = fit_cap;
    d->max_iters = fit_cap;
  }
  for (int a = 1; a + 1 < N; ++a) {
    int64_t sz = 1;
    for (int m = a; m < N; ++m) sz *= dm[m];
    char* p = take((size_t)sz * R * sizeof(float));
    if (d) d->node[a] = reinterpret_cast<float*>(p);
  }
  char* pM = take((size_t)maxI * R * sizeof(float));
  char* pP = take((size_t)nchunk * dm[0] * R * sizeof(float));
  char* pLP = take((size_t)lpart_floats * sizeof(float));
  char* pG = take((size_t)N * R * R * sizeof(double));
  char* pS = take((size_t)R * R * sizeof(double));
  char* pS32 = take((size_t)R * R * sizeof(float));
  char* pL = take((size_t)R * sizeof(double));
  char* pF = take((size_t)fit_cap * sizeof(double));
  char* pSc = take(4 * sizeof(double));
  char* pFl = take(4 * sizeof(int));
  if (d) {
    d->M = reinterpret_cast<float*>(pM);
    if (N == 2) d->node[1] = d->M;
    d->part = reinterpret_cast<float*>(pP);
    d->lpart = reinterpret_cast<float*>(pLP);
    d->G = reinterpret_cast<double*>(pG);
    d->S = reinterpret_cast<double*>(pS);
    d->S32 = reinterpret_cast<float*>(pS32);
    d->lam = reinterpret_cast<double*>(pL);
    d->fits = reinterpret_cast<double*>(pF);
    d->scal = reinterpret_cast<double*>(pSc);
    d->flags = reinterpret_cast<int*>(pFl);
  }
  return off;
}

void b_build_plan(const BTensor* ts, int C, int N, BPlan* p) {
  p->count = C;
  p->N = N;
  p->items.clear();
  p->alpha_first.assign(C + 1, 0);
  p->lam_off.assign(C, 0);
  p->lam_total = 0;
  int rmax = 1;
  p->hs_floats = 0;
  p->max_rows = 1;
  for (int t = 0; t < C; ++t) {
    rmax = std::max(rmax, ts[t].R);
    p->hs_floats = std::max(p->hs_floats, (int)ts[t].dims[0] * b_rank_pad(ts[t].R));
    for (int n = 0; n < N; ++n) p->max_rows = std::max(p->max_rows, (int)ts[t].dims[n]);
    p->lam_off[t] = (int)p->lam_total;
    p->lam_total += ts[t].R;
  }
  p->rmax = rmax <= 16 ? 16 : (rmax <= 32 ? 32 : 64);
  auto begin = [&](BPhase& ph) { ph.off = (int)p->items.size(); };
  auto end = [&](BPhase& ph) { ph.count = (int)p->items.size() - ph.off; };
  auto push = [&](int t, int64_t y, int64_t z) {
    p->items.push_back(make_int4(t, (int)y, (int)z, 0));
  };
  begin(p->alpha);
  for (int t = 0; t < C; ++t) {
    p->alpha_first[t] = (int)p->items.size() - p->alpha.off;
    for (int64_t c = 0; c * kAlphaChunk < ts[t].I; ++c) push(t, c, 0);
  }
  end(p->alpha);
  p->alpha_first[C] = p->alpha.count;
  begin(p->pmr);
  for (int t = 0; t < C; ++t)
    for (int c = 0; c < ts[t].nchunk; ++c) push(t, c, 0);
  end(p->pmr);
  begin(p->pmr_red);
  for (int t = 0; t < C; ++t)
    for (int64_t b = 0; b < cdiv(ts[t].dims[0] * ts[t].R, kReduceBlock); ++b) push(t, b, 0);
  end(p->pmr_red);
  begin(p->pml);
  for (int t = 0; t < C; ++t) {
    const int64_t J = ts[t].I / ts[t].dims[0];
    const int64_t rows = (int64_t)ts[t].rows_l * kLeftItemTiles;
    for (int64_t b = 0; b < cdiv(J, rows); ++b) push(t, b, 0);
  }
  end(p->pml);
  for (int a = 0; a < kMaxModes; ++a) p->leaf[a] = p->leaf_red[a] = p->first[a] = BPhase();
  for (int a = 1; a + 1 < N; ++a) {
    begin(p->leaf[a]);
    for (int t = 0; t < C; ++t) {
      const int64_t E = ts[t].dims[a] * ts[t].R;
      for (int c = 0; c < ts[t].leaf_nkc[a]; ++c)
        for (int64_t b = 0; b < cdiv(E, kLeafBlock); ++b) push(t, c, b);
    }
    end(p->leaf[a]);
    begin(p->leaf_red[a]);
    for (int t = 0; t < C; ++t)
      for (int64_t b = 0; b < cdiv(ts[t].dims[a] * ts[t].R, kReduceBlock); ++b) push(t, b, a);
    end(p->leaf_red[a]);
    begin(p->first[a]);
    for (int t = 0; t < C; ++t) {
      int64_t K = 1;
      for (int m = a + 1; m < N; ++m) K *= ts[t].dims[m];
      for (int64_t b = 0; b < cdiv(K, ts[t].first_jb[a]); ++b) push(t, b, 0);
    }
    end(p->first[a]);
  }
}

}  // namespace nncp

using namespace nncp;

struct nncp_batch {
  int count = 0, N = 0, fit_cap = 0;
  std::vector<int64_t> dims;  // count x N
  std::vector<int> R;
  std::vector<BTensor> ts;    // host copy of the descriptors
  BPlan plan;
  // workspace layout (byte offsets)
  size_t off_ts = 0, off_items = 0, off_alpha_first = 0, off_alpha_part = 0, off_done = 0,
         off_out_iters = 0, off_out_fits = 0, off_out_lam = 0, off_lam_off = 0, off_nonfinite = 0,
         off_tensors = 0, total = 0;
  std::vector<size_t> t_off;  // per-tensor slice offsets
  char* ws = nullptr;
  cudaStream_t work = nullptr;
  cudaGraphExec_t graph = nullptr;
  int* host_done = nullptr;
  bool have_data = false;
  // schedule of the two root phases: -1 = chosen by the tuner at the next run
  int want_right = -1, want_left = -1;
  long long wait_cycles = 0;  // bounded-wait limit of the streamed kernel (0: default)
  BSchedule sched;
  bool sched_set = false;
  size_t off_queues = 0;
  std::string err;
};

namespace {

nncp_status bfail(nncp_batch* b, nncp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  record_global_error(buf);
  return s;
}

#define BCK(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return bfail(b, NNCP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void plan(nncp_batch* b) {
  const int C = b->count;
  b->ts.assign(C, BTensor());
  b->t_off.assign(C, 0);
  for (int t = 0; t < C; ++t)
    b_tensor_layout(b->N, &b->dims[(size_t)t * b->N], b->R[t], b->fit_cap, &b->ts[t], nullptr);
  b_build_plan(b->ts.data(), C, b->N, &b->plan);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = al(off + bytes);
    return o;
  };
  b->off_ts = take(C * sizeof(BTensor));
  b->off_items = take(std::max<size_t>(1, b->plan.items.size()) * sizeof(int4));
  b->off_alpha_first = take((C + 1) * sizeof(int));
  b->off_alpha_part = take(std::max(1, b->plan.alpha.count) * sizeof(double));
  b->off_done = take(sizeof(int) * 4);
  b->off_queues = take(sizeof(int) * 4);  // root-phase counters, error word
  b->off_out_iters = take(C * sizeof(int));
  b->off_out_fits = take(C * sizeof(double));
  b->off_out_lam = take(std::max<size_t>(1, b->plan.lam_total) * sizeof(double));
  b->off_lam_off = take(C * sizeof(int));
  b->off_nonfinite = take(C * sizeof(int));
  b->off_tensors = off;
  for (int t = 0; t < C; ++t) {
    b->t_off[t] = off;
    off += al(b_tensor_layout(b->N, &b->dims[(size_t)t * b->N], b->R[t], b->fit_cap, nullptr, nullptr));
  }
  b->total = off;
}

template <typename T>
T* at(nncp_batch* b, size_t off) {
  return reinterpret_cast<T*>(b->ws + off);
}

}  // namespace

// ---- schedule tuner ----------------------------------------------------------
// The root phases' schedule (one CTA per item, or persistent CTAs taking items
// from a counter) changes which CTA computes an item, never how: a tensor's
// bits are the same under every schedule, so it can be chosen by timing.
// Key: the batch's order, largest rank and the binary magnitudes of its tensor
// count and element total (compositions of one class share the choice); the
// choice is cached for the process.
struct SchedKey {
  int N, rmax, count_log2, elems_log2;
  bool operator<(const SchedKey& o) const {
    if (N != o.N) return N < o.N;
    if (rmax != o.rmax) return rmax < o.rmax;
    if (count_log2 != o.count_log2) return count_log2 < o.count_log2;
    return elems_log2 < o.elems_log2;
  }
};
std::mutex g_sched_mu;
std::map<SchedKey, BSchedule> g_sched_cache;

int ilog2(long long v) {
  int l = 0;
  while (v > 1) {
    v >>= 1;
    ++l;
  }
  return l;
}

SchedKey sched_key(const nncp_batch* b) {
  long long elems = 0;
  for (const BTensor& t : b->ts) elems += t.I;
  return SchedKey{b->N, b->plan.rmax, ilog2(b->count), ilog2(elems)};
}

// Median of three timed launches of one root phase under schedule `mode`.
nncp_status time_phase(nncp_batch* b, int right, int mode, float* ms) {
  BTensor* d_ts = at<BTensor>(b, b->off_ts);
  const int4* d_items = at<int4>(b, b->off_items);
  int* q = at<int>(b, b->off_queues);
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  float t[4];
  for (int r = 0; r < 4; ++r) {
    BCK(cudaEventRecord(e0, b->work));
    if (mode) BCK(cudaMemsetAsync(q, 0, sizeof(int), b->work));
    BCK(right ? launch_pm_right(b->plan, d_ts, d_items, mode, q, q + 2, b->work, b->wait_cycles)
              : launch_pm_left(b->plan, d_ts, d_items, mode, q, q + 2, b->work, b->wait_cycles));
    BCK(cudaEventRecord(e1, b->work));
    BCK(cudaEventSynchronize(e1));
    BCK(cudaEventElapsedTime(&t[r], e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(t + 1, t + 4);  // the first launch is a warm-up
  *ms = t[2];
  return NNCP_OK;
}

// Chooses b->sched: a fixed request as given, else the cached choice for the
// batch's class, else the faster schedule of each root phase, timed here
// (after initialisation, before the iteration graph is captured).
nncp_status choose_schedule(nncp_batch* b) {
  const SchedKey key = sched_key(b);
  BSchedule sch;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_sched_mu);
    auto it = g_sched_cache.find(key);
    if (it != g_sched_cache.end()) {
      sch = it->second;
      cached = true;
    }
  }
  if (!cached && (b->want_right < 0 || b->want_left < 0)) {
    for (int right = 0; right < 2; ++right) {
      float best = 0.0f;
      int pick = 0;
      for (int mode = 0; mode < (right ? kRightSchedules : kLeftSchedules); ++mode) {
        float ms = 0.0f;
        nncp_status st = time_phase(b, right, mode, &ms);
        if (st != NNCP_OK) return st;
        if (mode == 0 || ms < best) {
          best = ms;
          pick = mode;
        }
      }
      (right ? sch.pm_right : sch.pm_left) = pick;
    }
    std::lock_guard<std::mutex> lock(g_sched_mu);
    g_sched_cache[key] = sch;
  }
  if (b->want_right >= 0) sch.pm_right = b->want_right;
  if (b->want_left >= 0) sch.pm_left = b->want_left;
  sch.wait_cycles = b->wait_cycles;
  if (!b->sched_set || sch.pm_right != b->sched.pm_right || sch.pm_left != b->sched.pm_left ||
      sch.wait_cycles != b->sched.wait_cycles) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->sched = sch;
  b->sched_set = true;
  return NNCP_OK;
}

extern "C" {

nncp_status nncp_batch_create(int count, int N, const int64_t* dims, const int* R, int max_iters,
                              nncp_batch** out) {
  if (!out) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !dims || !R) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "empty batch");
  if (N < 2 || N > kMaxModes) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "N=%d not in [2,8]", N);
  if (max_iters < 1 || max_iters > 65536)
    return bfail(nullptr, NNCP_ERR_INVALID_ARG, "max_iters %d not in [1, 65536]", max_iters);
  for (int t = 0; t < count; ++t) {
    if (R[t] < 1 || R[t] > kBatchMaxRank)
      return bfail(nullptr, NNCP_ERR_INVALID_ARG, "tensor %d: R=%d not in [1,%d]", t, R[t], kBatchMaxRank);
    int64_t I = 1;
    for (int n = 0; n < N; ++n) {
      const int64_t d = dims[(size_t)t * N + n];
      if (d < 1 || d > kBatchMaxI)
        return bfail(nullptr, NNCP_ERR_INVALID_ARG, "tensor %d: dims[%d]=%lld not in [1,%d]", t, n,
                     (long long)d, kBatchMaxI);
      I *= d;
      if (I > kBatchMaxElems)
        return bfail(nullptr, NNCP_ERR_INVALID_ARG, "tensor %d: more than %lld elements", t,
                     (long long)kBatchMaxElems);
    }
  }
  nncp_batch* b = new (std::nothrow) nncp_batch();
  if (!b) return bfail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "host allocation failed");
  b->count = count;
  b->N = N;
  b->fit_cap = max_iters;
  b->dims.assign(dims, dims + (size_t)count * N);
  b->R.assign(R, R + count);
  cudaError_t e = cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&b->host_done, 4 * sizeof(int));
  if (e == cudaSuccess) e = batch_attributes_init();
  if (e != cudaSuccess) {
    nncp_status s = bfail(nullptr, NNCP_ERR_CUDA, "nncp_batch_create: %s", cudaGetErrorString(e));
    nncp_batch_destroy(b);
    return s;
  }
  plan(b);
  *out = b;
  return NNCP_OK;
}

nncp_status nncp_batch_workspace_size(const nncp_batch* b, size_t* bytes) {
  if (!b || !bytes) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null argument");
  *bytes = b->total;
  return NNCP_OK;
}

nncp_status nncp_batch_set_workspace(nncp_batch* b, void* dev_ptr, size_t bytes) {
  if (!b) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null batch");
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
    return bfail(b, NNCP_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  if (bytes < b->total) return bfail(b, NNCP_ERR_INVALID_ARG, "workspace %zu < %zu bytes", bytes, b->total);
  b->ws = static_cast<char*>(dev_ptr);
  for (int t = 0; t < b->count; ++t) {
    const float* X = b->ts[t].X;
    float* H[kMaxModes];
    for (int n = 0; n < kMaxModes; ++n) H[n] = b->ts[t].H[n];
    b_tensor_layout(b->N, &b->dims[(size_t)t * b->N], b->R[t], b->fit_cap, &b->ts[t],
                    b->ws + b->t_off[t]);
    b->ts[t].X = X;
    for (int n = 0; n < kMaxModes; ++n) b->ts[t].H[n] = H[n];
  }
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  const BPlan& p = b->plan;
  BCK(cudaMemcpyAsync(b->ws + b->off_items, p.items.data(), p.items.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, b->work));
  BCK(cudaMemcpyAsync(b->ws + b->off_alpha_first, p.alpha_first.data(),
                      p.alpha_first.size() * sizeof(int), cudaMemcpyHostToDevice, b->work));
  BCK(cudaMemcpyAsync(b->ws + b->off_lam_off, p.lam_off.data(), p.lam_off.size() * sizeof(int),
                      cudaMemcpyHostToDevice, b->work));
  BCK(cudaStreamSynchronize(b->work));
  return NNCP_OK;
}

nncp_status nncp_batch_set_data(nncp_batch* b, const float* const* X_dev, float* const* H_dev) {
  if (!b || !X_dev || !H_dev) return bfail(b, NNCP_ERR_INVALID_ARG, "null argument");
  if (!b->ws) return bfail(b, NNCP_ERR_INVALID_ARG, "workspace not set");
  for (int t = 0; t < b->count; ++t) {
    if (!X_dev[t] || (reinterpret_cast<uintptr_t>(X_dev[t]) & 15))
      return bfail(b, NNCP_ERR_INVALID_ARG, "tensor %d is NULL or not 16-byte aligned", t);
    for (int n = 0; n < b->N; ++n) {
      float* h = H_dev[(size_t)t * b->N + n];
      if (!h || (reinterpret_cast<uintptr_t>(h) & 15))
        return bfail(b, NNCP_ERR_INVALID_ARG, "factor %d of tensor %d is NULL or not 16-byte aligned",
                     n + 1, t);
    }
  }
  for (int t = 0; t < b->count; ++t) {
    b->ts[t].X = X_dev[t];
    for (int n = 0; n < b->N; ++n) b->ts[t].H[n] = H_dev[(size_t)t * b->N + n];
  }
  b->have_data = true;
  return NNCP_OK;
}

nncp_status nncp_batch_run(nncp_batch* b, int max_iters, double tol, int* iters_out,
                           double* fits_out, double* lambda_out, void* stream) {
  if (!b) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null batch");
  if (!b->have_data) return bfail(b, NNCP_ERR_INVALID_ARG, "data not set");
  if (max_iters < 1 || max_iters > b->fit_cap)
    return bfail(b, NNCP_ERR_INVALID_ARG, "max_iters %d not in [1, %d]", max_iters, b->fit_cap);
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  for (int t = 0; t < b->count; ++t) {
    b->ts[t].max_iters = max_iters;
    b->ts[t].tol = tol;
  }
  BTensor* d_ts = at<BTensor>(b, b->off_ts);
  const int4* d_items = at<int4>(b, b->off_items);
  cudaEvent_t ev;
  BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  BCK(cudaEventRecord(ev, user));
  BCK(cudaStreamWaitEvent(b->work, ev, 0));
  BCK(cudaMemcpyAsync(d_ts, b->ts.data(), b->ts.size() * sizeof(BTensor), cudaMemcpyHostToDevice,
                      b->work));
  int* done = at<int>(b, b->off_done);
  BCK(cudaMemsetAsync(done, 0, sizeof(int), b->work));
  int* d_err = at<int>(b, b->off_queues) + 2;
  BCK(cudaMemsetAsync(d_err, 0, sizeof(int), b->work));
  BCK(b_launch_init(b->plan, d_ts, d_items, at<double>(b, b->off_alpha_part),
                    at<int>(b, b->off_alpha_first), b->work));
  {
    const nncp_status st = choose_schedule(b);
    if (st != NNCP_OK) return st;
  }
  if (!b->graph) {
    cudaGraph_t g;
    BCK(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = b_launch_iteration(b->plan, d_ts, d_items, done, b->work, b->sched,
                                       at<int>(b, b->off_queues));
    cudaError_t e2 = cudaStreamEndCapture(b->work, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(g);
      return bfail(b, NNCP_ERR_CUDA, "capturing the batched iteration: %s",
                   cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, NNCP_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
  }
  int launched = 0, every = 4;
  while (launched < max_iters) {
    const int n = std::min(every, max_iters - launched);
    for (int k = 0; k < n; ++k) BCK(cudaGraphLaunch(b->graph, b->work));
    launched += n;
    BCK(cudaMemcpyAsync(b->host_done, done, sizeof(int), cudaMemcpyDeviceToHost, b->work));
    BCK(cudaStreamSynchronize(b->work));
    if (b->host_done[0] >= b->count) break;
    every = std::min(every * 2, 16);
  }
  int* d_iters = at<int>(b, b->off_out_iters);
  double* d_fits = at<double>(b, b->off_out_fits);
  double* d_lam = at<double>(b, b->off_out_lam);
  int* d_nf = at<int>(b, b->off_nonfinite);
  BCK(launch_b_gather(d_ts, b->count, d_iters, d_fits, lambda_out ? d_lam : nullptr,
                      at<int>(b, b->off_lam_off), d_nf, b->work));
  std::vector<int> nf(b->count);
  if (iters_out)
    BCK(cudaMemcpyAsync(iters_out, d_iters, b->count * sizeof(int), cudaMemcpyDeviceToHost, b->work));
  if (fits_out)
    BCK(cudaMemcpyAsync(fits_out, d_fits, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->work));
  if (lambda_out)
    BCK(cudaMemcpyAsync(lambda_out, d_lam, b->plan.lam_total * sizeof(double),
                        cudaMemcpyDeviceToHost, b->work));
  BCK(cudaMemcpyAsync(nf.data(), d_nf, b->count * sizeof(int), cudaMemcpyDeviceToHost, b->work));
  BCK(cudaMemcpyAsync(b->host_done + 1, d_err, sizeof(int), cudaMemcpyDeviceToHost, b->work));
  BCK(cudaStreamSynchronize(b->work));
  BCK(cudaEventRecord(ev, b->work));
  BCK(cudaStreamWaitEvent(user, ev, 0));
  cudaEventDestroy(ev);
  if (b->host_done[1])
    return bfail(b, NNCP_ERR_TIMEOUT,
                 "a streamed root kernel gave up waiting on its pipeline (wait site %d)",
                 b->host_done[1] - 1);
  for (int t = 0; t < b->count; ++t)
    if (nf[t] & 1) return bfail(b, NNCP_ERR_NUMERIC, "tensor %d: non-finite fit", t);
  return NNCP_OK;
}

nncp_status nncp_batch_solve(int count, const int* N, const int64_t* const* dims, const int* R,
                             const void* const* X_dev, float* const* const* H_dev,
                             double* const* lambda, int max_iters, double tol, int* iters,
                             double* fits, void* stream) {
  if (count < 1 || !N || !dims || !R || !X_dev || !H_dev)
    return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null argument or empty batch");
  for (int t = 0; t < count; ++t)
    if (N[t] < 2 || N[t] > kMaxModes || !dims[t] || !H_dev[t])
      return bfail(nullptr, NNCP_ERR_INVALID_ARG, "tensor %d: N=%d not in [2,8] or null shape/factors",
                   t, N[t]);
  // one batch per order, tensors in their given order within it
  for (int order = 2; order <= kMaxModes; ++order) {
    std::vector<int> idx;
    for (int t = 0; t < count; ++t)
      if (N[t] == order) idx.push_back(t);
    if (idx.empty()) continue;
    const int c = (int)idx.size();
    std::vector<int64_t> dm((size_t)c * order);
    std::vector<int> rk(c);
    std::vector<const float*> xs(c);
    std::vector<float*> hs((size_t)c * order);
    for (int i = 0; i < c; ++i) {
      const int t = idx[i];
      for (int n = 0; n < order; ++n) {
        dm[(size_t)i * order + n] = dims[t][n];
        hs[(size_t)i * order + n] = H_dev[t][n];
      }
      rk[i] = R[t];
      xs[i] = static_cast<const float*>(X_dev[t]);
    }
    nncp_batch* b = nullptr;
    nncp_status st = nncp_batch_create(c, order, dm.data(), rk.data(), max_iters, &b);
    if (st != NNCP_OK) return st;  // the message is in nncp_global_error
    void* ws = nullptr;
    const cudaError_t e = cudaMalloc(&ws, std::max<size_t>(b->total, 256));
    if (e != cudaSuccess) {
      nncp_batch_destroy(b);
      return bfail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "workspace of %zu bytes: %s", b->total,
                   cudaGetErrorString(e));
    }
    std::vector<int> it(c);
    std::vector<double> ft(c);
    std::vector<double> lam(b->plan.lam_total > 0 ? b->plan.lam_total : 1);
    st = nncp_batch_set_workspace(b, ws, std::max<size_t>(b->total, 256));
    if (st == NNCP_OK) st = nncp_batch_set_data(b, xs.data(), hs.data());
    if (st == NNCP_OK) st = nncp_batch_run(b, max_iters, tol, it.data(), ft.data(), lam.data(), stream);
    cudaFree(ws);
    nncp_batch_destroy(b);
    if (st != NNCP_OK) return st;
    size_t o = 0;
    for (int i = 0; i < c; ++i) {
      const int t = idx[i];
      if (iters) iters[t] = it[i];
      if (fits) fits[t] = ft[i];
      if (lambda && lambda[t]) memcpy(lambda[t], lam.data() + o, (size_t)rk[i] * sizeof(double));
      o += (size_t)rk[i];
    }
  }
  return NNCP_OK;
}

nncp_status nncp_batch_set_schedule(nncp_batch* b, int pm_right, int pm_left) {
  if (!b) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null batch");
  if (pm_right < -1 || pm_right >= kRightSchedules || pm_left < -1 || pm_left >= kLeftSchedules)
    return bfail(b, NNCP_ERR_INVALID_ARG,
                 "schedules are -1 (tuned), 0..%d (root -> {1}) and 0..%d (root -> {2..N})",
                 kRightSchedules - 1, kLeftSchedules - 1);
  b->want_right = pm_right;
  b->want_left = pm_left;
  return NNCP_OK;
}

nncp_status nncp_batch_set_wait_limit(nncp_batch* b, long long cycles) {
  if (!b) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null batch");
  if (cycles < 0) return bfail(b, NNCP_ERR_INVALID_ARG, "wait limit %lld < 0", cycles);
  b->wait_cycles = cycles;
  return NNCP_OK;
}

nncp_status nncp_batch_get_schedule(const nncp_batch* b, int* pm_right, int* pm_left) {
  if (!b || !pm_right || !pm_left) return bfail(nullptr, NNCP_ERR_INVALID_ARG, "null argument");
  if (!b->sched_set) return bfail(const_cast<nncp_batch*>(b), NNCP_ERR_NOT_READY, "no run yet");
  *pm_right = b->sched.pm_right;
  *pm_left = b->sched.pm_left;
  return NNCP_OK;
}

const char* nncp_batch_last_error(const nncp_batch* b) { return b ? b->err.c_str() : nncp_global_error(); }

void nncp_batch_destroy(nncp_batch* b) {
  if (!b) return;
  if (b->work) cudaStreamSynchronize(b->work);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->work) cudaStreamDestroy(b->work);
  if (b->host_done) cudaFreeHost(b->host_done);
  delete b;
}

}  // extern "C"
