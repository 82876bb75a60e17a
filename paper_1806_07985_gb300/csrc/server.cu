// Serving loop: continuous batching of independent NNCP-HALS requests on one
// GPU.  A worker thread admits requests from a FIFO into a device pool
// (first-fit, coalescing free list), groups the active ones by order N, and
// runs sweeps: one outer iteration of every active request (the batched
// launches over a plan rebuilt whenever a group's membership changed), then
// retires the requests whose stopping rule fired.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/nncp.h"
#include "batch_kernels.cuh"

using namespace nncp;

namespace {

size_t al(size_t v) { return (v + 255) / 256 * 256; }

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Pool {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;  // offset -> length
  size_t used_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  int N = 0, R = 0, max_iters = 0;
  int64_t dims[kMaxModes] = {0};
  int64_t I = 0;
  double tol = 0.0;
  std::vector<float> X;               // host copy until admission (empty when borrowed)
  const float* Xb = nullptr;          // the caller's tensor when borrowed (borrow_x)
  const float* x_host() const { return Xb ? Xb : X.data(); }
  std::vector<std::vector<float>> H;  // initial factors, then the results
  std::vector<const float*> Hp;
  std::vector<double> lam;
  size_t bytes = 0, off = 0;          // pool block
  BTensor desc;                       // batched lane
  nncp_ctx* ctx = nullptr;            // solo lane: a single-problem context
  size_t ws_bytes = 0;
  int64_t I1p = 0;                    // solo lane: stored mode-1 length (padded)
  bool ctx_was_solo = false;          // took the solo lane (ctx is gone once retired)
  int* h_flags = nullptr;             // solo lane: pinned copy of the context's flags
  cudaStream_t sst = nullptr;         // solo lane: the request's own stream
  cudaEvent_t sev = nullptr;          //   marks the end of its launched chunk
  int launched = 0, chunk = 4;        //   iterations launched, next chunk size
  bool inflight = false;
  bool done = false;
  nncp_status status = NNCP_OK;
  int iters = 0;
  double fit = 0.0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

// Active requests of one order N and the device copy of their plan.
struct Group {
  std::vector<Request*> members;
  std::vector<BTensor> ts;
  BPlan plan;
  bool dirty = false;
  BTensor* d_ts = nullptr;
  int4* d_items = nullptr;
  int* d_state = nullptr;  // gather outputs: iterations, fits, state words
  int* d_iters = nullptr;
  double* d_fits = nullptr;
  size_t cap_ts = 0, cap_items = 0, cap_iters = 0, cap_fits = 0, cap_state = 0;
  std::vector<int> h_iters, h_state;
  std::vector<double> h_fits;
};

bool valid_precision(int p) {
  return p == NNCP_FP32_SIMT || p == NNCP_TF32 || p == NNCP_SPLIT_BF16X3;
}

bool valid_shape(int N, const int64_t* dims, int R, int max_iters) {
  if (N < 2 || N > kMaxModes || !dims || R < 1 || R > kBatchMaxRank) return false;
  if (max_iters < 1 || max_iters > 65536) return false;
  int64_t I = 1;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1 || dims[n] > kBatchMaxI) return false;
    I *= dims[n];
    if (I > kBatchMaxElems) return false;
  }
  return true;
}

int64_t elems(int N, const int64_t* dims) {
  int64_t I = 1;
  for (int n = 0; n < N; ++n) I *= dims[n];
  return I;
}

bool solo_lane(int N, const int64_t* dims, int64_t solo_elems) { return elems(N, dims) >= solo_elems; }

// tensor and factors, then the lane's workspace (ws_bytes for the solo lane)
size_t footprint(int N, const int64_t* dims, int R, int max_iters, bool solo, size_t ws_bytes,
                 int64_t I1p) {
  const int64_t I1 = solo ? I1p : dims[0];
  size_t b = al((size_t)(elems(N, dims) / dims[0] * I1) * sizeof(float));
  b += al((size_t)I1 * R * sizeof(float));
  for (int n = 1; n < N; ++n) b += al((size_t)dims[n] * R * sizeof(float));
  if (solo) return b + al(ws_bytes);
  return b + al(b_tensor_layout(N, dims, R, max_iters, nullptr, nullptr));
}

// Solo lane: a context with the requested precision and the automatic root
// split, on mode 1 padded as nncp_solve_host pads it (*I1p), or FP32 SIMT on
// the unpadded shape where the tensor-core path refuses it anyway.
nncp_status make_solo_ctx(int N, const int64_t* dims, int R, int precision, cudaStream_t st,
                          nncp_ctx** out, size_t* ws, int64_t* I1p) {
  int64_t pd[kMaxModes];
  for (int n = 0; n < N; ++n) pd[n] = dims[n];
  pd[0] = tc_padded_mode1(precision, N, dims, R, 0);
  nncp_ctx* c = nullptr;
  nncp_status e = nncp_create(N, pd, R, &c);
  if (e != NNCP_OK) return e;
  e = nncp_set_options(c, precision, 0, st);
  if (e == NNCP_ERR_UNSUPPORTED && precision != NNCP_FP32_SIMT) {
    nncp_destroy(c);
    c = nullptr;
    pd[0] = dims[0];
    e = nncp_create(N, pd, R, &c);
    if (e != NNCP_OK) return e;
    e = nncp_set_options(c, NNCP_FP32_SIMT, 0, st);
  }
  if (e == NNCP_OK) e = nncp_workspace_size(c, ws);
  if (e != NNCP_OK) {
    nncp_destroy(c);
    return e;
  }
  *out = c;
  *I1p = pd[0];
  return NNCP_OK;
}

}  // namespace

struct nncp_server {
  size_t budget = 0;
  int64_t solo_elems = NNCP_SERVER_SOLO_ELEMS;
  int max_slots = 1, device = 0;
  char* pool_base = nullptr;
  Pool pool;
  cudaStream_t st = nullptr;   // batched lane (each solo-lane request has its own stream)
  std::vector<Request*> solo;  // active solo-lane requests
  // scratch for admissions (init) and the done counter the update kernel bumps
  BTensor* d_init_ts = nullptr;
  int4* d_init_items = nullptr;
  double* d_alpha_part = nullptr;
  int* d_alpha_first = nullptr;
  int* d_done = nullptr;
  size_t cap_init_ts = 0, cap_init_items = 0, cap_alpha = 0, cap_alpha_first = 0;
  Group groups[kMaxModes + 1];

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue_b, queue_s;  // waiting requests of the batched / solo lane
  int max_solo = NNCP_SERVER_MAX_SOLO, solo_active = 0;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  int active = 0;
  uint64_t next_ticket = 1;
  bool stop = false, broken = false;
  nncp_server_stats stats{};
  std::string err;
  std::chrono::steady_clock::time_point t0;
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

nncp_status sfail(nncp_server* s, nncp_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) {
    std::lock_guard<std::mutex> g(s->mu);
    s->err = buf;
  }
  record_global_error(buf);
  return code;
}

template <typename T>
cudaError_t ensure(T** p, size_t* cap, size_t n) {
  if (n <= *cap && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t want = std::max<size_t>(n, 16) * 3 / 2;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), want * sizeof(T));
  if (e == cudaSuccess) *cap = want;
  return e;
}

// Admission: lay out the request in its pool block, copy tensor and factors.
cudaError_t admit_one(nncp_server* s, Request* r) {
  char* base = s->pool_base + r->off;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base + o;
    o += al(bytes);
    return p;
  };
  const int64_t I1 = r->ctx ? r->I1p : r->dims[0];
  const int64_t rows = r->I / r->dims[0];
  float* X = reinterpret_cast<float*>(take((size_t)(rows * I1) * sizeof(float)));
  float* H[kMaxModes];
  H[0] = reinterpret_cast<float*>(take((size_t)I1 * r->R * sizeof(float)));
  for (int n = 1; n < r->N; ++n) H[n] = reinterpret_cast<float*>(take((size_t)r->dims[n] * r->R * sizeof(float)));
  if (r->ctx) {
    char* ws = take(0);
    cudaStream_t st = r->sst;
    cudaError_t e = cudaSuccess;
    if (I1 != r->dims[0]) {  // zero slices of mode 1 and zero rows of H_1
      e = cudaMemsetAsync(X, 0, (size_t)(rows * I1) * sizeof(float), st);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(X, (size_t)I1 * sizeof(float), r->x_host(), (size_t)r->dims[0] * sizeof(float),
                              (size_t)r->dims[0] * sizeof(float), (size_t)rows, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(H[0], 0, (size_t)I1 * r->R * sizeof(float), st);
    } else {
      e = cudaMemcpyAsync(X, r->x_host(), (size_t)r->I * sizeof(float), cudaMemcpyHostToDevice, st);
    }
    for (int n = 0; n < r->N && e == cudaSuccess; ++n)
      e = cudaMemcpyAsync(H[n], r->H[n].data(), r->H[n].size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMallocHost(&r->h_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->sev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    for (int n = 0; n < r->N; ++n) r->desc.H[n] = H[n];
    if (nncp_set_workspace(r->ctx, ws, r->ws_bytes) != NNCP_OK || nncp_set_tensor(r->ctx, X) != NNCP_OK ||
        nncp_set_factors(r->ctx, H) != NNCP_OK || ctx_solve_begin_tol(r->ctx, r->tol) != NNCP_OK)
      return cudaErrorUnknown;
    return cudaSuccess;
  }
  b_tensor_layout(r->N, r->dims, r->R, r->max_iters, &r->desc, take(0));
  r->desc.X = X;
  for (int n = 0; n < r->N; ++n) r->desc.H[n] = H[n];
  r->desc.max_iters = r->max_iters;
  r->desc.tol = r->tol;
  cudaError_t e = cudaMemcpyAsync(X, r->x_host(), (size_t)r->I * sizeof(float), cudaMemcpyHostToDevice, s->st);
  for (int n = 0; n < r->N && e == cudaSuccess; ++n)
    e = cudaMemcpyAsync(H[n], r->H[n].data(), r->H[n].size() * sizeof(float), cudaMemcpyHostToDevice, s->st);
  return e;
}

// alpha, normalisation, Grams and S of the newly admitted requests (any orders)
cudaError_t init_new(nncp_server* s, const std::vector<Request*>& fresh) {
  if (fresh.empty()) return cudaSuccess;
  std::vector<BTensor> ts;
  BPlan p;
  p.count = (int)fresh.size();
  p.alpha.off = 0;
  p.alpha_first.assign(fresh.size() + 1, 0);
  for (size_t t = 0; t < fresh.size(); ++t) {
    ts.push_back(fresh[t]->desc);
    p.alpha_first[t] = (int)p.items.size();
    for (int64_t c = 0; c * kAlphaChunk < fresh[t]->I; ++c)
      p.items.push_back(make_int4((int)t, (int)c, 0, 0));
  }
  p.alpha.count = (int)p.items.size();
  p.alpha_first[fresh.size()] = p.alpha.count;
  cudaError_t e = ensure(&s->d_init_ts, &s->cap_init_ts, ts.size());
  if (e == cudaSuccess) e = ensure(&s->d_init_items, &s->cap_init_items, p.items.size());
  if (e == cudaSuccess) e = ensure(&s->d_alpha_part, &s->cap_alpha, p.items.size());
  if (e == cudaSuccess) e = ensure(&s->d_alpha_first, &s->cap_alpha_first, p.alpha_first.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_init_ts, ts.data(), ts.size() * sizeof(BTensor), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_init_items, p.items.data(), p.items.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_alpha_first, p.alpha_first.data(), p.alpha_first.size() * sizeof(int),
                        cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = b_launch_init(p, s->d_init_ts, s->d_init_items, s->d_alpha_part, s->d_alpha_first, s->st);
  return e;
}

cudaError_t upload_group(nncp_server* s, Group& g, int N) {
  g.ts.clear();
  for (Request* r : g.members) g.ts.push_back(r->desc);
  b_build_plan(g.ts.data(), (int)g.ts.size(), N, &g.plan);
  const size_t C = g.ts.size();
  cudaError_t e = ensure(&g.d_ts, &g.cap_ts, C);
  if (e == cudaSuccess) e = ensure(&g.d_items, &g.cap_items, std::max<size_t>(1, g.plan.items.size()));
  if (e == cudaSuccess) e = ensure(&g.d_iters, &g.cap_iters, C);
  if (e == cudaSuccess) e = ensure(&g.d_fits, &g.cap_fits, C);
  if (e == cudaSuccess) e = ensure(&g.d_state, &g.cap_state, C);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.d_ts, g.ts.data(), C * sizeof(BTensor), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.d_items, g.plan.items.data(), g.plan.items.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, s->st);
  g.h_iters.resize(C);
  g.h_fits.resize(C);
  g.h_state.resize(C);
  g.dirty = false;
  return e;
}

// Copies a finished request's results back and frees its pool block.
cudaError_t retire(nncp_server* s, Request* r, int iters, double fit, int state) {
  cudaError_t e = cudaSuccess;
  for (int n = 0; n < r->N && e == cudaSuccess; ++n)
    e = cudaMemcpyAsync(r->H[n].data(), r->desc.H[n], r->H[n].size() * sizeof(float),
                        cudaMemcpyDeviceToHost, s->st);
  r->lam.resize(r->R);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->lam.data(), r->desc.lam, r->R * sizeof(double), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  r->iters = iters;
  r->fit = fit;
  r->status = (state & 1) ? NNCP_ERR_NUMERIC : NNCP_OK;
  return e;
}

// Frees a solo-lane request's context, stream, event and pinned flags.
void release_solo(Request* r) {
  if (r->ctx) nncp_destroy(r->ctx);
  r->ctx = nullptr;
  if (r->sev) cudaEventDestroy(r->sev);
  r->sev = nullptr;
  if (r->sst) cudaStreamDestroy(r->sst);
  r->sst = nullptr;
  if (r->h_flags) cudaFreeHost(r->h_flags);
  r->h_flags = nullptr;
}

// Solo lane: its flags {done, -, iterations, non-finite} were read back.
cudaError_t retire_solo(nncp_server* s, Request* r) {
  const int* dflags;
  const double *dlam, *dfits;
  const int* dtc;
  ctx_device_state(r->ctx, &dflags, &dlam, &dfits, &dtc);
  const int iters = r->h_flags[2];
  cudaStream_t st = r->sst;
  cudaError_t e = cudaSuccess;
  for (int n = 0; n < r->N && e == cudaSuccess; ++n)
    e = cudaMemcpyAsync(r->H[n].data(), r->desc.H[n], r->H[n].size() * sizeof(float),
                        cudaMemcpyDeviceToHost, st);
  r->lam.resize(r->R);
  double fit = 0.0;
  int tc_err = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->lam.data(), dlam, r->R * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && iters > 0)
    e = cudaMemcpyAsync(&fit, dfits + (iters - 1), sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && dtc) e = cudaMemcpyAsync(&tc_err, dtc, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  r->iters = iters;
  r->fit = fit;
  r->status = tc_err ? NNCP_ERR_TIMEOUT : (r->h_flags[3] ? NNCP_ERR_NUMERIC : NNCP_OK);
  release_solo(r);
  return e;
}

// Solo lane, without waiting: a request whose chunk has completed is retired
// if its rule fired (device flags: done, iterations, non-finite) and gets its
// next chunk otherwise (4, 8, then 16 iterations, never past max_iters; the
// device flag makes iterations launched after convergence no-ops, as in
// nncp_solve).  Finished requests are appended to `finished`.
cudaError_t solo_step(nncp_server* s, std::vector<Request*>* finished) {
  cudaError_t e = cudaSuccess;
  std::vector<Request*> keep;
  for (Request* r : s->solo) {
    if (e != cudaSuccess) {
      keep.push_back(r);
      continue;
    }
    if (r->inflight) {
      const cudaError_t q = cudaEventQuery(r->sev);
      if (q == cudaErrorNotReady) {
        keep.push_back(r);
        continue;
      }
      if (q != cudaSuccess) {
        e = q;
        keep.push_back(r);
        continue;
      }
      r->inflight = false;
      if (r->h_flags[0] || r->h_flags[3] || r->h_flags[2] >= r->max_iters) {
        e = retire_solo(s, r);
        finished->push_back(r);
        continue;
      }
    }
    const int n = std::min(r->chunk, r->max_iters - r->launched);
    const int* dflags;
    const double *dlam, *dfits;
    const int* dtc;
    ctx_device_state(r->ctx, &dflags, &dlam, &dfits, &dtc);
    if (n > 0 && nncp_iterate(r->ctx, n) != NNCP_OK) e = cudaErrorUnknown;
    r->launched += std::max(n, 0);
    r->chunk = std::min(2 * r->chunk, 16);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->h_flags, dflags, 4 * sizeof(int), cudaMemcpyDeviceToHost, r->sst);
    if (e == cudaSuccess) e = cudaEventRecord(r->sev, r->sst);
    r->inflight = true;
    keep.push_back(r);
  }
  s->solo.swap(keep);
  return e;
}

void fail_all(nncp_server* s, const char* what, cudaError_t e) {
  std::lock_guard<std::mutex> g(s->mu);
  char buf[512];
  snprintf(buf, sizeof buf, "server worker: %s: %s", what, cudaGetErrorString(e));
  s->err = buf;
  record_global_error(buf);
  s->broken = true;
  const double t = s->now();
  for (auto& kv : s->reqs) {
    Request* r = kv.second.get();
    if (!r->done) {
      r->done = true;
      r->status = NNCP_ERR_CUDA;
      r->t_done = t;
    }
  }
  s->queue_b.clear();
  s->queue_s.clear();
  s->solo_active = 0;
  for (auto& grp : s->groups) grp.members.clear();
  s->solo.clear();
  s->active = 0;
  s->cv_done.notify_all();
}

void worker_main(nncp_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> fresh;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return s->stop || s->active > 0 || !s->queue_b.empty() || !s->queue_s.empty();
      });
      if (s->stop) return;
      // admission in submission order within each lane while the head fits;
      // at most max_solo solo-lane requests run at once
      for (bool progress = true; progress;) {
        progress = false;
        std::deque<Request*>* lanes[2] = {&s->queue_b, &s->queue_s};
        for (std::deque<Request*>* q : lanes) {
          if (q->empty() || s->active + (int)fresh.size() >= s->max_slots) continue;
          if (q == &s->queue_s && s->solo_active >= s->max_solo) continue;
          Request* r = q->front();
          size_t off = 0;
          if (!s->pool.alloc(r->bytes, &off)) continue;
          r->off = off;
          r->t_admit = s->now();
          q->pop_front();
          fresh.push_back(r);
          if (r->ctx) ++s->solo_active;
          progress = true;
        }
      }
      s->stats.bytes_in_use = s->pool.used();
      s->stats.peak_bytes_in_use = std::max(s->stats.peak_bytes_in_use, s->pool.used());
      if (s->active == 0 && fresh.empty()) {
        // the head does not fit an empty pool: cannot happen (submit checks the budget)
        s->cv_work.wait_for(lk, std::chrono::milliseconds(10));
        continue;
      }
    }
    cudaError_t e = cudaSuccess;
    std::vector<Request*> fresh_batched;
    for (Request* r : fresh) {
      if (e == cudaSuccess) e = admit_one(s, r);
      if (!r->ctx) fresh_batched.push_back(r);
    }
    if (e == cudaSuccess) e = init_new(s, fresh_batched);
    if (e != cudaSuccess) {
      fail_all(s, "admission", e);
      return;
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      for (Request* r : fresh) {
        r->X.clear();
        r->X.shrink_to_fit();
        if (r->ctx) {
          s->solo.push_back(r);
        } else {
          s->groups[r->N].members.push_back(r);
          s->groups[r->N].dirty = true;
        }
      }
      s->active += (int)fresh.size();
      s->stats.active = s->active;
      s->stats.queued = (int)(s->queue_b.size() + s->queue_s.size());
      s->stats.peak_active = std::max(s->stats.peak_active, s->active);
    }
    // solo lane: retire finished chunks' requests, launch the next chunks
    std::vector<Request*> finished;
    if (e == cudaSuccess) e = solo_step(s, &finished);
    // batched lane: one sweep, an outer iteration of every active request
    bool swept = false;
    for (int N = 2; N <= kMaxModes && e == cudaSuccess; ++N) {
      Group& g = s->groups[N];
      if (g.members.empty()) continue;
      swept = true;
      if (g.dirty) e = upload_group(s, g, N);
      if (e == cudaSuccess) e = b_launch_iteration(g.plan, g.d_ts, g.d_items, s->d_done, s->st, BSchedule(), nullptr);
      if (e == cudaSuccess)
        e = launch_b_gather(g.d_ts, (int)g.members.size(), g.d_iters, g.d_fits, nullptr, nullptr,
                            g.d_state, s->st);
      const size_t C = g.members.size();
      if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_iters.data(), g.d_iters, C * sizeof(int), cudaMemcpyDeviceToHost, s->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_fits.data(), g.d_fits, C * sizeof(double), cudaMemcpyDeviceToHost, s->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_state.data(), g.d_state, C * sizeof(int), cudaMemcpyDeviceToHost, s->st);
    }
    if (e == cudaSuccess && swept) e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess && !swept && finished.empty() && !s->solo.empty()) {
      // only solo chunks in flight: block on one of them rather than spin
      for (Request* r : s->solo)
        if (r->inflight) {
          e = cudaEventSynchronize(r->sev);
          break;
        }
    }
    if (e != cudaSuccess) {
      fail_all(s, "sweep", e);
      return;
    }
    // retire the batched requests that stopped
    for (int N = 2; N <= kMaxModes && e == cudaSuccess && swept; ++N) {
      Group& g = s->groups[N];
      if (g.members.empty()) continue;
      std::vector<Request*> keep;
      for (size_t t = 0; t < g.members.size(); ++t) {
        Request* r = g.members[t];
        if (g.h_state[t] & 2) {
          e = retire(s, r, g.h_iters[t], g.h_fits[t], g.h_state[t]);
          if (e != cudaSuccess) break;
          finished.push_back(r);
        } else {
          keep.push_back(r);
        }
      }
      if (keep.size() != g.members.size()) {
        g.members.swap(keep);
        g.dirty = true;
      }
    }
    if (e != cudaSuccess) {
      fail_all(s, "retire", e);
      return;
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      const double t = s->now();
      for (Request* r : finished) {
        s->pool.release(r->off, r->bytes);
        r->done = true;
        r->t_done = t;
        if (r->ctx_was_solo) --s->solo_active;
      }
      s->active -= (int)finished.size();
      s->stats.completed += finished.size();
      s->stats.sweeps += swept ? 1 : 0;
      s->stats.active = s->active;
      s->stats.bytes_in_use = s->pool.used();
    }
    if (!finished.empty()) s->cv_done.notify_all();
  }
}

void fill_result(Request* r, nncp_result* res) {
  r->Hp.resize(r->N);
  for (int n = 0; n < r->N; ++n) r->Hp[n] = r->H[n].data();
  res->status = r->status;
  res->iters = r->iters;
  res->fit = r->fit;
  res->lambda = r->lam.empty() ? nullptr : r->lam.data();
  res->H = r->Hp.data();
  res->t_submit = r->t_submit;
  res->t_admit = r->t_admit;
  res->t_done = r->t_done;
}

}  // namespace

extern "C" {

nncp_status nncp_server_footprint(const nncp_server* s, int N, const int64_t* dims, int R,
                                  int max_iters, nncp_precision precision, size_t* bytes) {
  if (!s || !bytes || !valid_shape(N, dims, R, max_iters) || !valid_precision(precision))
    return sfail(nullptr, NNCP_ERR_INVALID_ARG, "request outside the server's limits");
  size_t ws = 0;
  int64_t I1p = dims[0];
  const bool solo = solo_lane(N, dims, s->solo_elems);
  if (solo) {
    nncp_ctx* c = nullptr;
    nncp_status e = make_solo_ctx(N, dims, R, precision, nullptr, &c, &ws, &I1p);
    if (e != NNCP_OK) return e;
    nncp_destroy(c);
  }
  *bytes = footprint(N, dims, R, max_iters, solo, ws, I1p);
  return NNCP_OK;
}

nncp_status nncp_server_create(size_t hbm_budget_bytes, int max_slots, nncp_server** out) {
  return nncp_server_create_ex(hbm_budget_bytes, max_slots, NNCP_SERVER_SOLO_ELEMS,
                               NNCP_SERVER_MAX_SOLO, out);
}

nncp_status nncp_server_create_ex(size_t hbm_budget_bytes, int max_slots, int64_t solo_elems,
                                  int max_solo, nncp_server** out) {
  if (!out) return sfail(nullptr, NNCP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < 4096 || max_slots < 1 || solo_elems < 1 || max_solo < 1)
    return sfail(nullptr, NNCP_ERR_INVALID_ARG,
                 "budget below 4 KiB, or max_slots, solo_elems or max_solo below 1");
  std::unique_ptr<nncp_server> s(new (std::nothrow) nncp_server());
  if (!s) return sfail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->solo_elems = solo_elems;
  s->max_solo = max_solo;
  s->budget = al(hbm_budget_bytes - 255);
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = batch_attributes_init();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_done, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->d_done, 0, sizeof(int));
  if (e == cudaSuccess) {
    e = cudaMalloc(&s->pool_base, s->budget);
    if (e != cudaSuccess) {
      s->pool_base = nullptr;
      cudaGetLastError();
      if (s->st) cudaStreamDestroy(s->st);
      if (s->d_done) cudaFree(s->d_done);
      return sfail(nullptr, NNCP_ERR_OUT_OF_MEMORY, "pool of %zu bytes: %s", s->budget,
                   cudaGetErrorString(e));
    }
  }
  if (e != cudaSuccess) {
    if (s->st) cudaStreamDestroy(s->st);
    if (s->d_done) cudaFree(s->d_done);
    return sfail(nullptr, NNCP_ERR_CUDA, "nncp_server_create: %s", cudaGetErrorString(e));
  }
  s->pool.reset(s->budget);
  s->stats.budget = s->budget;
  nncp_server* raw = s.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return NNCP_OK;
}

nncp_status nncp_server_submit(nncp_server* s, const nncp_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return sfail(s, NNCP_ERR_INVALID_ARG, "null argument");
  if (!valid_shape(q->N, q->dims, q->R, q->max_iters) || !valid_precision(q->precision))
    return sfail(s, NNCP_ERR_INVALID_ARG, "request outside the server's limits");
  if (!q->X_host || !q->H_init_host) return sfail(s, NNCP_ERR_INVALID_ARG, "null tensor or factors");
  for (int n = 0; n < q->N; ++n)
    if (!q->H_init_host[n]) return sfail(s, NNCP_ERR_INVALID_ARG, "factor %d is NULL", n + 1);
  const double t_submit = s->now();
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return sfail(s, NNCP_ERR_OUT_OF_MEMORY, "host allocation failed");
  const bool solo = solo_lane(q->N, q->dims, s->solo_elems);
  if (solo) {
    if (cudaStreamCreateWithFlags(&r->sst, cudaStreamNonBlocking) != cudaSuccess)
      return sfail(s, NNCP_ERR_CUDA, "solo-lane stream");
    nncp_status e = make_solo_ctx(q->N, q->dims, q->R, q->precision, r->sst, &r->ctx, &r->ws_bytes,
                                  &r->I1p);
    if (e != NNCP_OK) {
      release_solo(r.get());
      return sfail(s, e, "solo-lane context: %s", nncp_global_error());
    }
  }
  const size_t bytes = footprint(q->N, q->dims, q->R, q->max_iters, solo, r->ws_bytes, r->I1p);
  if (bytes > s->budget) {
    release_solo(r.get());
    return sfail(s, NNCP_ERR_INVALID_ARG, "request needs %zu bytes, budget is %zu", bytes, s->budget);
  }
  r->N = q->N;
  r->R = q->R;
  r->max_iters = q->max_iters;
  r->tol = q->tol;
  r->I = 1;
  for (int n = 0; n < q->N; ++n) {
    r->dims[n] = q->dims[n];
    r->I *= q->dims[n];
  }
  r->bytes = bytes;
  try {
    if (q->borrow_x)
      r->Xb = q->X_host;
    else
      r->X.assign(q->X_host, q->X_host + r->I);
    r->H.resize(q->N);
    for (int n = 0; n < q->N; ++n)
      r->H[n].assign(q->H_init_host[n], q->H_init_host[n] + r->dims[n] * r->R);
  } catch (...) {
    release_solo(r.get());
    return sfail(s, NNCP_ERR_OUT_OF_MEMORY, "host copy of the request failed");
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->broken) {
      release_solo(r.get());
      return NNCP_ERR_CUDA;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = t_submit;
    *ticket = r->ticket;
    r->ctx_was_solo = r->ctx != nullptr;
    (r->ctx ? s->queue_s : s->queue_b).push_back(r.get());
    s->reqs.emplace(r->ticket, std::move(r));
    s->stats.submitted += 1;
    s->stats.queued = (int)(s->queue_b.size() + s->queue_s.size());
  }
  s->cv_work.notify_one();
  return NNCP_OK;
}

nncp_status nncp_server_poll(nncp_server* s, uint64_t ticket, nncp_result* res) {
  if (!s || !res) return sfail(s, NNCP_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return NNCP_ERR_INVALID_ARG;
  if (!it->second->done) return NNCP_ERR_NOT_READY;
  fill_result(it->second.get(), res);
  return NNCP_OK;
}

nncp_status nncp_server_wait(nncp_server* s, uint64_t ticket, int timeout_ms, nncp_result* res) {
  if (!s || !res || timeout_ms < 0) return sfail(s, NNCP_ERR_INVALID_ARG, "null argument or negative timeout");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return NNCP_ERR_INVALID_ARG;
  Request* r = it->second.get();
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
    return NNCP_ERR_TIMEOUT;
  fill_result(r, res);
  return NNCP_OK;
}

nncp_status nncp_server_release(nncp_server* s, uint64_t ticket) {
  if (!s) return sfail(nullptr, NNCP_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || !it->second->done) return NNCP_ERR_INVALID_ARG;
  s->reqs.erase(it);
  return NNCP_OK;
}

nncp_status nncp_server_get_stats(nncp_server* s, nncp_server_stats* st) {
  if (!s || !st) return sfail(s, NNCP_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  *st = s->stats;
  return NNCP_OK;
}

double nncp_server_clock(const nncp_server* s) { return s ? s->now() : 0.0; }

const char* nncp_server_last_error(const nncp_server* s) {
  return s ? s->err.c_str() : nncp_global_error();
}

void nncp_server_destroy(nncp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->st) cudaStreamSynchronize(s->st);
  for (auto& kv : s->reqs) {
    Request* r = kv.second.get();
    if (r->sst) cudaStreamSynchronize(r->sst);
    release_solo(r);
  }
  for (auto& g : s->groups) {
    if (g.d_ts) cudaFree(g.d_ts);
    if (g.d_items) cudaFree(g.d_items);
    if (g.d_iters) cudaFree(g.d_iters);
    if (g.d_fits) cudaFree(g.d_fits);
    if (g.d_state) cudaFree(g.d_state);
  }
  if (s->d_init_ts) cudaFree(s->d_init_ts);
  if (s->d_init_items) cudaFree(s->d_init_items);
  if (s->d_alpha_part) cudaFree(s->d_alpha_part);
  if (s->d_alpha_first) cudaFree(s->d_alpha_first);
  if (s->d_done) cudaFree(s->d_done);
  if (s->pool_base) cudaFree(s->pool_base);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
}

}  // extern "C"
