// Batched NNCP-HALS: many independent tensors of the same order N, each with
// its own mode lengths and rank, solved together.  Every tensor uses root
// split 1 (node {1} and node {2..N}, Fig. 1 shape below it), so the
// dimension-tree schedule of one outer iteration (Sec. IV-A; Alg. 1) is the
// same sequence of operations for all of them, and each operation is one
// launch over a device work list of (tensor, chunk) items.  Tensors whose fit
// has converged are skipped by every item.  Reductions across chunks are
// summed in chunk order, so a tensor's result does not depend on the batch.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "batch_kernels.cuh"

namespace nncp {

namespace {

__device__ __forceinline__ bool tensor_done(const BTensor& t) { return t.flags[0] != 0; }

// ---------------------------------------------------------------- init --

// alpha partials: item (tensor, chunk of kAlphaChunk elements) -> alpha_part[item];
// squares summed four at a time in FP32, the rest in FP64 (fixed order)
__global__ void __launch_bounds__(256) k_b_sumsq(const BTensor* __restrict__ ts,
                                                 const int4* __restrict__ items,
                                                 double* __restrict__ alpha_part) {
  const int4 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  const long long e0 = (long long)it.y * kAlphaChunk;
  const int n = (int)min(kAlphaChunk, t.I - e0);
  const float* x = t.X + e0;
  const int n4 = n >> 2;
  double acc = 0.0;
#pragma unroll 4
  for (int v = threadIdx.x; v < n4; v += blockDim.x) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(x) + v);
    acc += (double)(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
  }
  if ((int)threadIdx.x < n - 4 * n4) {
    const float v = x[4 * n4 + threadIdx.x];
    acc += (double)(v * v);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    alpha_part[blockIdx.x] = s;
  }
}

// per tensor: alpha = sum of its partials (in order), normalise every factor
// (lambda = product of the column norms), G_n = H_n^T H_n, S for mode 1,
// flags and fit history cleared (Alg. 3 initialisation).
__global__ void k_b_init(BTensor* __restrict__ ts, const double* __restrict__ alpha_part,
                         const int* __restrict__ alpha_first) {
  BTensor& t = ts[blockIdx.x];
  const int R = t.R, N = t.N, R2 = R * R;
  __shared__ double lam[kBatchMaxRank];
  __shared__ double cn[kBatchMaxRank];
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int c = alpha_first[blockIdx.x]; c < alpha_first[blockIdx.x + 1]; ++c) a += alpha_part[c];
    t.scal[0] = a;
    t.scal[1] = t.tol;
    t.flags[0] = 0;
    t.flags[1] = 0;
    t.flags[2] = 0;
  }
  for (int r = threadIdx.x; r < R; r += blockDim.x) lam[r] = 1.0;
  __syncthreads();
  for (int n = 0; n < N; ++n) {
    float* Hn = t.H[n];
    const int In = (int)t.dims[n];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < In; ++i) s += (double)Hn[i * R + r] * Hn[i * R + r];
      cn[r] = sqrt(s);
      lam[r] *= cn[r];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < In * R; e += blockDim.x) {
      const double c = cn[e % R];
      Hn[e] = c > 0.0 ? (float)((double)Hn[e] / c) : 0.0f;
    }
    __syncthreads();
    double* Gn = t.G + (long long)n * R2;
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
      const int a = e / R, b = e % R;
      double s = 0.0;
      for (int i = 0; i < In; ++i) s += (double)Hn[i * R + a] * Hn[i * R + b];
      Gn[e] = s;
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < R; r += blockDim.x) t.lam[r] = lam[r];
  for (int e = threadIdx.x; e < R2; e += blockDim.x) {
    double s = 1.0;
    for (int k = 1; k < N; ++k) s *= t.G[(long long)k * R2 + e];
    t.S[e] = s;
    t.S32[e] = (float)s;
  }
}

// ------------------------------------------------ partial MTTKRPs (root) --
//
// Both root contractions stream X_(1)^T (rows j of I_1 contiguous floats) in
// tiles of whole rows.  A tile is fetched into registers (eight float4 per
// thread, every load issued before any is used) one tile ahead of the
// compute, then stored to shared memory; the thread mapping is sized from
// the tensor's own rank, and when one tile holds too few (row, rank-group)
// pairs for 256 threads the contraction range is split over thread groups
// whose partial sums are added in group order.

constexpr int kThreads = 256;
// Split groups are sized for kGroupThreads whatever the block size, so the
// summation order of an output depends only on its tensor's shape.
constexpr int kGroupThreads = 256;

// Tiles are copied global -> shared with cp.async (no registers held while
// in flight) into a two-stage ring, so tile k+1 streams in while tile k is
// formed and contracted; X is read once per pass.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NPENDING) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// floats [0, L) of src (16-byte aligned) to Xs[0, L)
__device__ __forceinline__ void tile_copy_dense(float* Xs, const float* __restrict__ src, int L) {
  const int L4 = L & ~3;
  for (int e = 4 * (int)threadIdx.x; e < L4; e += 4 * kThreads) cp_async16(Xs + e, src + e);
  const int tail = L4 + (int)threadIdx.x;
  if (tail < L) cp_async4(Xs + tail, src + tail);
}

// rows of I1 floats to an odd stride S (threads reading one column of
// consecutive rows hit distinct banks): Xs[row * S + col] = src[row * I1 + col]
__device__ __forceinline__ void tile_copy_rows(float* Xs, const float* __restrict__ src, int L,
                                               int I1, int S) {
  if (S == I1) {
    tile_copy_dense(Xs, src, L);
    return;
  }
  int e = threadIdx.x;
  int row = e / I1, col = e - row * I1;
  const int drow = kThreads / I1, dcol = kThreads - drow * I1;
  for (; e < L; e += kThreads) {
    cp_async4(Xs + row * S + col, src + e);
    row += drow;
    col += dcol;
    if (col >= I1) {
      col -= I1;
      ++row;
    }
  }
}

// ranks r0 .. r0 + 3 of a factor row (zero beyond R); vector load when R % 4 == 0
__device__ __forceinline__ float4 ld_rank4(const float* __restrict__ row, int r0, int R) {
  if ((R & 3) == 0) {
    if (r0 >= R) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    return __ldg(reinterpret_cast<const float4*>(row + r0));
  }
  float4 h;
  h.x = r0 < R ? __ldg(row + r0) : 0.0f;
  h.y = r0 + 1 < R ? __ldg(row + r0 + 1) : 0.0f;
  h.z = r0 + 2 < R ? __ldg(row + r0 + 2) : 0.0f;
  h.w = r0 + 3 < R ? __ldg(row + r0 + 3) : 0.0f;
  return h;
}

__device__ __forceinline__ void fma4(float (&a)[4], float x, const float4& w) {
  a[0] = fmaf(x, w.x, a[0]);
  a[1] = fmaf(x, w.y, a[1]);
  a[2] = fmaf(x, w.z, a[2]);
  a[3] = fmaf(x, w.w, a[3]);
}

// root -> node {1}: part[c](i, r) = sum_{j in chunk c} X[i + I1 j] K(j, r),
// K = H_N (.) ... (.) H_2 (rows formed per tile, never stored whole).
// Item (tensor, chunk).  Thread = row i with all RQB = b_rq(R) rank groups;
// 256 / I1 column groups split each tile's rows (j = g, g + G, ...) and are
// added in group order at the end of the chunk.
template <int RQB>
__device__ __forceinline__ void pm_right_item(const BTensor& t, int chunk, float* smem) {
  constexpr int WU = kWsFloats / 4 / kThreads;
  float* Xbuf[2] = {smem, smem + kTileFloats};
  float* Ws = smem + 2 * kTileFloats;  // kWsFloats: rows x padded rank
  const int tid = threadIdx.x;
  const int R = t.R, N = t.N;
  const int I1 = (int)t.dims[0];
  const int nj = t.rows_r;
  const int J = (int)(t.I / I1);
  const int j0 = chunk * (int)t.jchunk;
  const int j1 = min(J, j0 + (int)t.jchunk);
  const int G = kGroupThreads / I1;
  const int g = tid / I1, i = tid - g * I1;
  const bool act = g < G;
  float acc[RQB][4];
#pragma unroll
  for (int u = 0; u < RQB; ++u)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[u][b] = 0.0f;
  const int ntile = (j1 - j0 + nj - 1) / nj;
  const float4* W4 = reinterpret_cast<const float4*>(Ws);
  tile_copy_dense(Xbuf[0], t.X + (long long)j0 * I1, min(nj, j1 - j0) * I1);
  cp_async_commit();
  for (int k = 0; k < ntile; ++k) {
    const int jt = j0 + k * nj, njk = min(nj, j1 - jt);
    if (k + 1 < ntile) {
      const int jn = jt + nj;
      tile_copy_dense(Xbuf[(k + 1) & 1], t.X + (long long)jn * I1, min(nj, j1 - jn) * I1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    // Khatri-Rao rows of the tile: float4 entries (row, rank group), nj * RQB <= kWsFloats / 4
    {
      float4 w[WU];
      int rem[WU];
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        rem[u] = jt + (tid + kThreads * u) / RQB;
        w[u] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
      }
      for (int m = 1; m < N; ++m) {
        const int dm = (int)t.dims[m];
        const float* Hm = t.H[m];
#pragma unroll
        for (int u = 0; u < WU; ++u) {
          const int e = tid + kThreads * u;
          if (e / RQB < njk) {
            const int jm = rem[u] % dm;
            rem[u] /= dm;
            const float4 h = ld_rank4(Hm + jm * R, 4 * (e % RQB), R);
            w[u].x *= h.x;
            w[u].y *= h.y;
            w[u].z *= h.z;
            w[u].w *= h.w;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        const int e = tid + kThreads * u;
        if (e / RQB < njk) reinterpret_cast<float4*>(Ws)[e] = w[u];
      }
    }
    __syncthreads();
    if (act) {
      const float* xp = Xbuf[k & 1] + i;
#pragma unroll 2
      for (int jj = g; jj < njk; jj += G) {
        const float x = xp[jj * I1];
#pragma unroll
        for (int u = 0; u < RQB; ++u) fma4(acc[u], x, W4[jj * RQB + u]);
      }
    }
    __syncthreads();
  }
  float* out = t.part + (long long)chunk * I1 * R;
  if (G > 1) {
    float4* red = reinterpret_cast<float4*>(Xbuf[0]);  // G * I1 <= 256 float4
#pragma unroll
    for (int u = 0; u < RQB; ++u) {
      if (act) red[tid] = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
      __syncthreads();
      if (tid < I1) {
        float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int gg = 0; gg < G; ++gg) {
          const float4 v = red[gg * I1 + tid];
          s4[0] += v.x;
          s4[1] += v.y;
          s4[2] += v.z;
          s4[3] += v.w;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (4 * u + b < R) out[tid * R + 4 * u + b] = s4[b];
      }
      __syncthreads();
    }
  } else if (act) {
#pragma unroll
    for (int u = 0; u < RQB; ++u)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * u + b < R) out[i * R + 4 * u + b] = acc[u][b];
  }
}

// Work item w of a phase for this CTA: with queue == NULL the CTA's own
// index (one CTA per item, the hardware schedules them); otherwise the next
// item taken from the phase's counter by a persistent CTA (-1: none left).
// Either way an item is computed the same way, so the choice changes no bits.
__device__ __forceinline__ int next_item(int* queue, int n_items, int* slot, bool first) {
  if (!queue) return first ? (int)blockIdx.x : -1;
  __syncthreads();  // every thread has read the previous item
  if (threadIdx.x == 0) *slot = atomicAdd(queue, 1);
  __syncthreads();
  return *slot < n_items ? *slot : -1;
}

template <int RMAX>
__global__ void __launch_bounds__(kThreads, RMAX <= 16 ? 4 : (RMAX <= 32 ? 3 : 2))
k_b_pm_right(const BTensor* __restrict__ ts, const int4* __restrict__ items, int n_items,
             int* queue) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int slot;
  for (int w = next_item(queue, n_items, &slot, true); w >= 0;
       w = next_item(queue, n_items, &slot, false)) {
    const int4 it = items[w];
    const BTensor& t = ts[it.x];
    if (tensor_done(t)) continue;
    switch (b_rq(t.R)) {
      case 1: pm_right_item<1>(t, it.y, smem); break;
      case 2: pm_right_item<2>(t, it.y, smem); break;
      case 4: pm_right_item<4>(t, it.y, smem); break;
      case 8: if constexpr (RMAX >= 32) pm_right_item<8>(t, it.y, smem); break;
      default: if constexpr (RMAX >= 64) pm_right_item<16>(t, it.y, smem); break;
    }
  }
}

// ------------------------------------- streamed root -> {1} (schedule 2) --
//
// The arithmetic of pm_right_item (every output's products and sums in the
// same order, so the same bits) with its jobs split over the warps of a
// persistent CTA, the tiles passing through a ring of shared-memory stages:
//   warp 0, scheduler: takes items from the counter (several at a time while
//                      it meets converged tensors), skips those, and writes
//                      each item's descriptor into a ring of item slots;
//   warp 1, loader:    copies an item's descriptor into the header of every
//                      stage of it and the stage's rows of X_(1)^T into the
//                      stage (cp.async, L2 evict-first), arriving on the
//                      stage's full barrier as the copies land;
//   warps 2-4, builders: take stages in turn and form a stage's Khatri-Rao
//                      rows;
//   warps 5-12, consumers (the 256 threads of pm_right_item): contract each
//                      tile and free its stage; at the end of an item they
//                      add the column groups in group order through the last
//                      stage's tile area, then free it.
// The scheduler runs ahead of the loader and the loader ahead of the rest, so
// tiles stream in across item boundaries.  Every wait is on an mbarrier and
// bounded (about two seconds): on expiry a thread records the error word and
// leaves, and the waits of the other roles then expire in turn.

constexpr int kWsBuildWarps = 3, kWsConsWarps = 8;
constexpr int kWsConsFirstWarp = 2 + kWsBuildWarps;
constexpr int kWsThreads = 32 * (kWsConsFirstWarp + kWsConsWarps);
constexpr int kWsStageFloats = kTileFloats + kWsFloats;
constexpr int kWsItemSlots = 4;
// Khatri-Rao entries (row, rank group) per builder lane and pass: a tile has at most kWsFloats / 4
constexpr int kWsBuildPer = 4;
constexpr int kWsBuildPasses = (kWsFloats / 4 + 32 * kWsBuildPer - 1) / (32 * kWsBuildPer);
constexpr long long kWsWaitCycles = 4000000000LL;

// One item as the builders and consumers need it (w < 0: no more items);
// seq: the item's position in this CTA's sequence; dims[m - 1] and H[m - 1]
// are I_{m+1} and factor m + 1 (root -> {1}); for root -> {2..N}, H[0] is H_1.
struct WsDesc {
  int w, I1, R, N, nj, j0, j1, ntile;
  int seq;
  int dims[kMaxModes - 1];
  float* out;
  const float* H[kMaxModes - 1];
};
struct WsHeader {
  WsDesc d;
  int k;  // tile within the item
  int pad[3];
};
struct WsSlot {
  WsDesc d;
  const float* X;
};
static_assert(sizeof(WsDesc) % 8 == 0 && sizeof(WsHeader) % 16 == 0 && sizeof(WsSlot) % 8 == 0,
              "descriptor layout");
constexpr int kWsDescWords = (int)(sizeof(WsDesc) / 4);
static_assert(kWsDescWords <= 32, "one descriptor word per lane");

__device__ __forceinline__ void mb_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// arrives once every cp.async this thread has issued so far has landed
__device__ __forceinline__ void mb_arrive_cp_async(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mb_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of a whole warp (all 32 lanes call it, converged): every lane
// polls (and so acquires the phase), the warp decides together, so a warp
// never splits over an expired wait (the lanes read one clock).  On expiry
// the first wait site to give up is recorded in *err (1 + site).  `limit`:
// clock64 cycles (kWsWaitCycles unless a test shortens it).
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity, long long limit, int* err,
                                        int site) {
  if (__all_sync(0xffffffffu, mb_test(bar, parity))) return true;
  const long long t0 = clock64();
  while (!__all_sync(0xffffffffu, mb_test(bar, parity))) {
    if (clock64() - t0 > limit) {
      if ((threadIdx.x & 31) == 0) atomicCAS(err, 0, 1 + site);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16_hint(float* dst, const float* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)),
               "l"(src), "l"(pol)
               : "memory");
}

// Shared memory of the streamed kernel: S stages (X tile, Khatri-Rao tile),
// their headers, the item slots and the barriers.
struct WsSmem {
  float* stage0;
  WsHeader* hdr;
  WsSlot* slot;
  uint32_t bar0;
  int S;
  long long wait;  // bounded-wait limit, clock64 cycles
  __device__ float* xs(int s) const { return stage0 + (size_t)s * kWsStageFloats; }
  __device__ uint32_t full(int s) const { return bar0 + 8u * s; }
  __device__ uint32_t empty(int s) const { return bar0 + 8u * (S + s); }
  __device__ uint32_t hfull(int s) const { return bar0 + 8u * (2 * S + s); }
  __device__ uint32_t islot_full(int i) const { return bar0 + 8u * (3 * S + i); }
  __device__ uint32_t islot_empty(int i) const { return bar0 + 8u * (3 * S + kWsItemSlots + i); }
  __device__ uint32_t red_full() const { return bar0 + 8u * (3 * S + 2 * kWsItemSlots); }
  __device__ uint32_t red_empty() const { return bar0 + 8u * (3 * S + 2 * kWsItemSlots + 1); }
  __device__ uint32_t cons_sync() const { return bar0 + 8u * (3 * S + 2 * kWsItemSlots + 2); }
};

__host__ __device__ constexpr size_t ws_smem_bytes(int S) {
  return (size_t)S * kWsStageFloats * sizeof(float) + (size_t)S * sizeof(WsHeader) +
         (size_t)kWsItemSlots * sizeof(WsSlot) +
         (size_t)(3 * S + 2 * kWsItemSlots + 3) * sizeof(uint64_t);
}

template <bool LEFT, typename SM>
__device__ void ws_scheduler(const BTensor* __restrict__ ts, const int4* __restrict__ items,
                             int n_items, int* queue, const SM& sm, int* err) {
  const int lane = threadIdx.x & 31;
  int m = 0;      // item slots filled
  int grab = 1;   // candidates taken per round: doubles while they are all converged
  bool more = true;
  while (more) {
    const int c = lane < grab ? atomicAdd(queue, 1) : n_items;
    const bool live = c < n_items;
    const bool active = live && !tensor_done(ts[items[c].x]);
    unsigned act = __ballot_sync(0xffffffffu, active);
    more = __ballot_sync(0xffffffffu, live) == (grab >= 32 ? 0xffffffffu : (1u << grab) - 1u);
    grab = act ? 1 : min(32, 2 * grab);
    while (act) {
      const int src = __ffs(act) - 1;
      act &= act - 1;
      const int w = __shfl_sync(0xffffffffu, c, src);
      const int sl = m % kWsItemSlots;
      if (!mb_wait(sm.islot_empty(sl), ((m / kWsItemSlots) & 1) ^ 1, sm.wait, err, 1)) return;
      if (lane == 0) {
        const int4 it = items[w];
        const BTensor& t = ts[it.x];
        WsSlot q;
        WsDesc& d = q.d;
        d.w = w;
        d.I1 = (int)t.dims[0];
        d.R = t.R;
        d.N = t.N;
        d.seq = m;
        const int J = (int)(t.I / d.I1);
        if (LEFT) {  // rows [j0, j1) of X_(1)^T in tiles of rows_l, H_1, T = node {2..N}
          d.nj = t.rows_l;
          d.j0 = it.y * d.nj * kLeftItemTiles;
          d.j1 = min(J, d.j0 + d.nj * kLeftItemTiles);
          for (int n = 1; n < kMaxModes; ++n) {
            d.dims[n - 1] = 0;
            d.H[n - 1] = nullptr;
          }
          d.H[0] = t.H[0];
          d.out = t.node[1];
        } else {     // chunk it.y of the columns, Khatri-Rao factors 2..N, a partial of M(1)
          d.nj = t.rows_r;
          d.j0 = it.y * (int)t.jchunk;
          d.j1 = min(J, d.j0 + (int)t.jchunk);
          for (int n = 1; n < kMaxModes; ++n) {
            d.dims[n - 1] = n < d.N ? (int)t.dims[n] : 0;
            d.H[n - 1] = n < d.N ? t.H[n] : nullptr;
          }
          d.out = t.part + (long long)it.y * d.I1 * d.R;
        }
        d.ntile = (d.j1 - d.j0 + d.nj - 1) / d.nj;
        q.X = t.X;
        sm.slot[sl] = q;
      }
      __syncwarp();
      if (lane == 0) mb_arrive(sm.islot_full(sl));
      ++m;
    }
  }
  // no more items
  const int sl = m % kWsItemSlots;
  if (!mb_wait(sm.islot_empty(sl), ((m / kWsItemSlots) & 1) ^ 1, sm.wait, err, 2)) return;
  if (lane == 0) sm.slot[sl].d.w = -1;
  __syncwarp();
  if (lane == 0) mb_arrive(sm.islot_full(sl));
}

// the loader of both streamed kernels: stage headers and dense tiles of
// rows of X_(1)^T; the last item is followed by one stop stage per builder warp
template <typename SM>
__device__ void ws_loader(const SM& sm, int* err) {
  const int lane = threadIdx.x & 31;
  const uint64_t pol = l2_evict_first_policy();
  int n = 0;  // stages posted
  for (int m = 0;; ++m) {
    const int sl = m % kWsItemSlots;
    if (!mb_wait(sm.islot_full(sl), (m / kWsItemSlots) & 1, sm.wait, err, 3)) break;
    const WsDesc& d = sm.slot[sl].d;
    const int w = d.w, I1 = d.I1, nj = d.nj, j0 = d.j0, j1 = d.j1;
    const int ntile = w >= 0 ? d.ntile : kWsBuildWarps;
    const float* X = sm.slot[sl].X;
    const uint32_t word = lane < kWsDescWords ? reinterpret_cast<const uint32_t*>(&d)[lane] : 0u;
    __syncwarp();
    if (lane == 0) mb_arrive(sm.islot_empty(sl));
    bool ok = true;
    for (int k = 0; k < ntile; ++k, ++n) {
      const int s = n % sm.S;
      if (!mb_wait(sm.empty(s), ((n / sm.S) & 1) ^ 1, sm.wait, err, 4)) {
        ok = false;
        break;
      }
      if (lane < kWsDescWords) reinterpret_cast<uint32_t*>(&sm.hdr[s].d)[lane] = word;
      if (lane == 0) sm.hdr[s].k = k;
      if (w >= 0) {
        const int jt = j0 + k * nj, L = min(nj, j1 - jt) * I1;
        const float* src = X + (long long)jt * I1;
        float* dst = sm.xs(s);
        const int L4 = L & ~3;
        for (int e = 4 * lane; e < L4; e += 128) cp_async16_hint(dst + e, src + e, pol);
        if (L4 + lane < L) cp_async4(dst + L4 + lane, src + L4 + lane);
      }
      mb_arrive_cp_async(sm.full(s));
      __syncwarp();
      if (lane == 0) mb_arrive(sm.hfull(s));
    }
    if (!ok || w < 0) break;
  }
  cp_async_wait_all();
}

// Builder warp b forms the Khatri-Rao tiles of stages b, b + 3, b + 6, ...
__device__ void ws_builder(const WsSmem& sm, int* err) {
  const int lane = threadIdx.x & 31;
  const int b = (threadIdx.x >> 5) - 2;
  for (int n = b;; n += kWsBuildWarps) {
    const int s = n % sm.S;
    if (!mb_wait(sm.hfull(s), (n / sm.S) & 1, sm.wait, err, 5)) return;
    const WsHeader& h = sm.hdr[s];
    const int w = h.d.w;
    if (w >= 0) {
      const int R = h.d.R, N = h.d.N, RQB = b_rq(R), lg = __ffs(RQB) - 1;
      const int jt = h.d.j0 + h.k * h.d.nj, njk = min(h.d.nj, h.d.j1 - jt);
      const int ne = njk * RQB;
      float4* W = reinterpret_cast<float4*>(sm.xs(s) + kTileFloats);
      for (int rd = 0; rd < kWsBuildPasses; ++rd) {
        const int e0 = lane + 32 * kWsBuildPer * rd;
        if (e0 >= ne) break;
        // every entry of this pass at once, so that the factor-row loads of
        // all of them are in flight together
        float4 v[kWsBuildPer];
        int rem[kWsBuildPer];
#pragma unroll
        for (int u = 0; u < kWsBuildPer; ++u) {
          rem[u] = jt + ((e0 + 32 * u) >> lg);
          v[u] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
        }
        for (int m = 1; m < N; ++m) {
          const int dm = h.d.dims[m - 1];
          const float* Hm = h.d.H[m - 1];
#pragma unroll
          for (int u = 0; u < kWsBuildPer; ++u) {
            const int e = e0 + 32 * u;
            if (e < ne) {
              const int jm = rem[u] % dm;
              rem[u] /= dm;
              const float4 hv = ld_rank4(Hm + jm * R, 4 * (e & (RQB - 1)), R);
              v[u].x *= hv.x;
              v[u].y *= hv.y;
              v[u].z *= hv.z;
              v[u].w *= hv.w;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kWsBuildPer; ++u) {
          const int e = e0 + 32 * u;
          if (e < ne) W[e] = v[u];
        }
      }
    }
    __syncwarp();
    if (lane == 0) mb_arrive(sm.full(s));
    if (w < 0) return;
  }
}

// One item's tiles (the first already waited for), then its group sum.
// false: a wait expired.
template <int RQB>
__device__ bool ws_consume(const WsDesc& d, int& n, int& nred, int& nsync, const WsSmem& sm,
                           int* err) {
  const int ct = threadIdx.x - 32 * kWsConsFirstWarp;  // 0 .. 255
  const int lane = threadIdx.x & 31;
  const int R = d.R, I1 = d.I1, nj = d.nj, j0 = d.j0, j1 = d.j1, ntile = d.ntile;
  float* out = d.out;
  const int G = kGroupThreads / I1;
  const int g = ct / I1, i = ct - g * I1;
  const bool act = g < G;
  float acc[RQB][4];
#pragma unroll
  for (int u = 0; u < RQB; ++u)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[u][b] = 0.0f;
  int s = 0;
  for (int k = 0; k < ntile; ++k, ++n) {
    s = n % sm.S;
    if (k > 0 && !mb_wait(sm.full(s), (n / sm.S) & 1, sm.wait, err, 6)) return false;
    const int jt = j0 + k * nj, njk = min(nj, j1 - jt);
    if (act) {
      const float* xp = sm.xs(s) + i;
      const float4* W4 = reinterpret_cast<const float4*>(sm.xs(s) + kTileFloats);
#pragma unroll 2
      for (int jj = g; jj < njk; jj += G) {
        const float x = xp[jj * I1];
#pragma unroll
        for (int u = 0; u < RQB; ++u) fma4(acc[u], x, W4[jj * RQB + u]);
      }
    }
    if (k + 1 < ntile || G == 1) {
      __syncwarp();
      if (lane == 0) mb_arrive(sm.empty(s));
    }
  }
  if (G > 1) {
    // column groups added in group order, through the last stage's tile area
    // (still held), up to 4 rank groups at a time, once every consumer warp
    // is done reading that tile
    __syncwarp();
    if (lane == 0) mb_arrive(sm.cons_sync());
    if (!mb_wait(sm.cons_sync(), nsync & 1, sm.wait, err, 7)) return false;
    ++nsync;
    float4* red = reinterpret_cast<float4*>(sm.xs(s));
#pragma unroll
    for (int u0 = 0; u0 < RQB; u0 += 4) {
      const uint32_t par = nred & 1;
      ++nred;
      if (u0 > 0 && !mb_wait(sm.red_empty(), par ^ 1, sm.wait, err, 8)) return false;
      if (act) {
#pragma unroll
        for (int u = u0; u < u0 + 4 && u < RQB; ++u)
          red[(u - u0) * kThreads + ct] = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
      }
      __syncwarp();
      if (lane == 0) mb_arrive(sm.red_full());
      if ((ct & ~31) < I1 && !mb_wait(sm.red_full(), par, sm.wait, err, 9)) return false;  // warps with readers
      if (ct < I1) {
#pragma unroll
        for (int u = u0; u < u0 + 4 && u < RQB; ++u) {
          float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          for (int gg = 0; gg < G; ++gg) {
            const float4 v = red[(u - u0) * kThreads + gg * I1 + ct];
            s4[0] += v.x;
            s4[1] += v.y;
            s4[2] += v.z;
            s4[3] += v.w;
          }
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (4 * u + b < R) out[ct * R + 4 * u + b] = s4[b];
        }
      }
      __syncwarp();
      if (lane == 0) mb_arrive(sm.red_empty());
    }
    __syncwarp();
    if (lane == 0) mb_arrive(sm.empty(s));
  } else if (act) {
#pragma unroll
    for (int u = 0; u < RQB; ++u)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * u + b < R) out[i * R + 4 * u + b] = acc[u][b];
  }
  return true;
}

template <int RMAX>
__device__ void ws_consumer(const WsSmem& sm, int* err) {
  int nred = 0, nsync = 0;
  for (int n = 0;;) {
    const int s = n % sm.S;
    if (!mb_wait(sm.full(s), (n / sm.S) & 1, sm.wait, err, 10)) return;
    const WsDesc& d = sm.hdr[s].d;
    if (d.w < 0) return;
    bool ok = true;
    switch (b_rq(d.R)) {
      case 1: ok = ws_consume<1>(d, n, nred, nsync, sm, err); break;
      case 2: ok = ws_consume<2>(d, n, nred, nsync, sm, err); break;
      case 4: ok = ws_consume<4>(d, n, nred, nsync, sm, err); break;
      case 8: if constexpr (RMAX >= 32) ok = ws_consume<8>(d, n, nred, nsync, sm, err); break;
      default: if constexpr (RMAX >= 64) ok = ws_consume<16>(d, n, nred, nsync, sm, err); break;
    }
    if (!ok) return;
  }
}

template <int RMAX>
__global__ void __launch_bounds__(kWsThreads, RMAX <= 16 ? 2 : 1)
k_b_pm_right_ws(const BTensor* __restrict__ ts, const int4* __restrict__ items, int n_items,
                int* queue, int S, int* err, long long wait_cycles) {
  extern __shared__ __align__(16) float smem[];
  WsSmem sm;
  sm.S = S;
  sm.wait = wait_cycles > 0 ? wait_cycles : kWsWaitCycles;
  sm.stage0 = smem;
  sm.hdr = reinterpret_cast<WsHeader*>(smem + (size_t)S * kWsStageFloats);
  sm.slot = reinterpret_cast<WsSlot*>(sm.hdr + S);
  sm.bar0 = smem_u32(sm.slot + kWsItemSlots);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(sm.full(s), 32 + 1);  // the loader lanes' copies + the stage's builder warp
      mb_init(sm.empty(s), kWsConsWarps);
      mb_init(sm.hfull(s), 1);
    }
    for (int i = 0; i < kWsItemSlots; ++i) {
      mb_init(sm.islot_full(i), 1);
      mb_init(sm.islot_empty(i), 1);
    }
    mb_init(sm.red_full(), kWsConsWarps);
    mb_init(sm.red_empty(), kWsConsWarps);
    mb_init(sm.cons_sync(), kWsConsWarps);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  if (warp == 0)
    ws_scheduler<false>(ts, items, n_items, queue, sm, err);
  else if (warp == 1)
    ws_loader(sm, err);
  else if (warp < kWsConsFirstWarp)
    ws_builder(sm, err);
  else
    ws_consumer<RMAX>(sm, err);
}

// M = sum of a phase's partial chunks in chunk order.  Item (tensor, block of
// kReduceBlock outputs, a): a = 0 sums the root -> {1} partials (M(1)),
// a >= 1 the leaf partials of node {a..N} (M(a)).
__global__ void __launch_bounds__(kReduceBlock) k_b_reduce(const BTensor* __restrict__ ts,
                                                           const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  if (tensor_done(t)) return;
  const int a = it.z;
  const int E = (int)t.dims[a] * t.R;
  const int nparts = a == 0 ? t.nchunk : t.leaf_nkc[a];
  const float* src = a == 0 ? t.part : t.lpart;
  const int e = it.y * kReduceBlock + threadIdx.x;
  if (e < E) {
    float s = 0.0f;
#pragma unroll 4
    for (int c = 0; c < nparts; ++c) s += src[(long long)c * E + e];
    t.M[e] = s;
  }
}

constexpr int kLeftRedFloats = 4 * kThreads;
constexpr int kLeftStageFloats = kTileFloats + kLeftMaxRows;  // rows at odd stride

__host__ __device__ constexpr int left_fixed_floats() {
  return 2 * kLeftStageFloats + kLeftRedFloats;
}

// root -> node {2..N}: T(j, r) = sum_i X[i + I1 j] H_1(i, r).  Item (tensor,
// kLeftItemTiles tiles of rows j); H_1 (rank padded to b_rank_pad(R) with
// zeros) sits in shared memory.  Thread = (row j, block of RQB rank groups);
// when a tile has fewer than 256 such pairs (then RQB = 1) the i range is
// split over groups added in group order.
template <int RQB>
__device__ __forceinline__ void pm_left_item(const BTensor& t, int item, float* smem) {
  float* Xbuf[2] = {smem, smem + kLeftStageFloats};
  float* red = smem + 2 * kLeftStageFloats;  // kLeftRedFloats
  float* Hs = red + kLeftRedFloats;          // I1 x padded rank
  const int tid = threadIdx.x;
  const int R = t.R, Rq = b_rq(R), Rp = 4 * Rq;
  const int I1 = (int)t.dims[0], S = I1 | 1;
  const int nj = t.rows_l;
  const int J = (int)(t.I / I1);
  const int jb0 = item * nj * kLeftItemTiles;
  const int jb1 = min(J, jb0 + nj * kLeftItemTiles);
  const int NB = Rq / RQB;  // rank blocks per row
  const int P = nj * NB;
  const int G = P >= kGroupThreads ? 1 : kGroupThreads / P;
  const int npass = (P + kThreads - 1) / kThreads;
  const int g = G > 1 ? tid / P : 0;
  const int ia = g * I1 / G, ib = (g + 1) * I1 / G;
  tile_copy_rows(Xbuf[0], t.X + (long long)jb0 * I1, min(nj, jb1 - jb0) * I1, I1, S);
  cp_async_commit();
  {
    const float* H1 = t.H[0];
    if (R == Rp) {
      const int n4 = I1 * Rq;
      for (int v0 = tid; v0 < n4; v0 += 4 * kThreads) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * kThreads;
          if (v < n4) h[u] = __ldg(reinterpret_cast<const float4*>(H1) + v);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * kThreads;
          if (v < n4) reinterpret_cast<float4*>(Hs)[v] = h[u];
        }
      }
    } else {
      for (int e = tid; e < I1 * Rp; e += kThreads) {
        const int i = e / Rp, r = e - i * Rp;
        Hs[e] = r < R ? __ldg(H1 + i * R + r) : 0.0f;
      }
    }
  }
  const float4* H4 = reinterpret_cast<const float4*>(Hs);
  float* T = t.node[1];
  const int ntile = (jb1 - jb0 + nj - 1) / nj;
  for (int k = 0; k < ntile; ++k) {
    const int jt = jb0 + k * nj, njk = min(nj, jb1 - jt);
    if (k + 1 < ntile) {
      const int jn = jt + nj;
      tile_copy_rows(Xbuf[(k + 1) & 1], t.X + (long long)jn * I1, min(nj, jb1 - jn) * I1, I1, S);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* Xs = Xbuf[k & 1];
    for (int p = 0; p < npass; ++p) {
      const int pair = G > 1 ? tid - g * P : tid + kThreads * p;
      const int jl = pair / NB, qb = pair - jl * NB;
      const bool v = g < G && pair < P && jl < njk;
      float a[RQB][4];
#pragma unroll
      for (int u = 0; u < RQB; ++u)
#pragma unroll
        for (int b = 0; b < 4; ++b) a[u][b] = 0.0f;
      if (v) {
        const float* xp = Xs + jl * S;
        const float4* hp = H4 + qb * RQB;
#pragma unroll 4
        for (int i = ia; i < ib; ++i) {
          const float x = xp[i];
#pragma unroll
          for (int u = 0; u < RQB; ++u) fma4(a[u], x, hp[i * Rq + u]);
        }
      }
      if (G > 1) {  // RQB == 1 here
        if (g < G) reinterpret_cast<float4*>(red)[tid] = make_float4(a[0][0], a[0][1], a[0][2], a[0][3]);
        __syncthreads();
        if (tid < P) {
          const int jl0 = tid / NB, q0 = tid - jl0 * NB;
          if (jl0 < njk) {
            float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int gg = 0; gg < G; ++gg) {
              const float4 w = reinterpret_cast<const float4*>(red)[gg * P + tid];
              s4[0] += w.x;
              s4[1] += w.y;
              s4[2] += w.z;
              s4[3] += w.w;
            }
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (4 * q0 + b < R) T[(long long)(jt + jl0) * R + 4 * q0 + b] = s4[b];
          }
        }
        __syncthreads();
      } else if (v) {
#pragma unroll
        for (int u = 0; u < RQB; ++u)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = 4 * (qb * RQB + u) + b;
            if (r < R) T[(long long)(jt + jl) * R + r] = a[u][b];
          }
      }
    }
    __syncthreads();
  }
}

template <int RMAX>
__global__ void __launch_bounds__(kThreads, RMAX <= 16 ? 4 : 2)
k_b_pm_left(const BTensor* __restrict__ ts, const int4* __restrict__ items, int n_items,
            int* queue) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int slot;
  for (int w = next_item(queue, n_items, &slot, true); w >= 0;
       w = next_item(queue, n_items, &slot, false)) {
    const int4 it = items[w];
    const BTensor& t = ts[it.x];
    if (tensor_done(t)) continue;
    switch (b_rqb_left((int)t.dims[0], t.R)) {
      case 1: pm_left_item<1>(t, it.y, smem); break;
      case 2: pm_left_item<2>(t, it.y, smem); break;
      case 4: pm_left_item<4>(t, it.y, smem); break;
      case 8: if constexpr (RMAX >= 32) pm_left_item<8>(t, it.y, smem); break;
      default: if constexpr (RMAX >= 64) pm_left_item<16>(t, it.y, smem); break;
    }
  }
}

// ------------------------------------ streamed root -> {2..N} (schedule 2) --
//
// The arithmetic of pm_left_item (same sums in the same order, so the same
// bits) with its jobs split over the warps of a persistent CTA, built from
// the parts of the streamed root -> {1} kernel:
//   warp 0, scheduler and warp 1, loader: as there (ws_scheduler<true>,
//                      ws_loader): dense tiles of rows of X_(1)^T into a ring
//                      of SD stages;
//   warps 2-4, builders: take the dense stages in turn; at an item's first
//                      tile stage H_1 (rank padded with zeros) into one of two
//                      H slots; copy the tile to the odd row stride S = I_1 | 1
//                      (conflict-free column reads) into a ring of SO stages,
//                      with the header; free the dense stage;
//   warps 5-12, consumers (the 256 threads of pm_left_item): the (row, rank
//                      block) passes over each odd-stride tile, group sums
//                      through a small buffer, rows of T written out; an odd
//                      stage is freed after its tile, an H slot after its item.
// Waits: mbarriers, warp-uniform and bounded, an error word.

struct WlHeader {
  WsDesc d;
  int k;      // tile within the item
  int hslot;  // H slot of the item
  int pad[2];
};
static_assert(sizeof(WlHeader) % 16 == 0, "header layout");

// Shared-memory counter helpers: a consumer warp's release of an odd stage,
// and the builder's bounded, warp-uniform wait for a number of releases
// (an exact count: builders fill the odd ring out of order, so a parity wait
// could pass on a phase two laps old).
__device__ __forceinline__ void smem_add_release(const unsigned* p, unsigned v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned smem_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ bool count_wait(const unsigned* p, unsigned target, long long limit,
                                           int* err, int site) {
  if (__all_sync(0xffffffffu, smem_ld_acquire(p) >= target)) return true;
  const long long t0 = clock64();
  while (!__all_sync(0xffffffffu, smem_ld_acquire(p) >= target)) {
    if (clock64() - t0 > limit) {
      if ((threadIdx.x & 31) == 0) atomicCAS(err, 0, 1 + site);
      return false;
    }
  }
  return true;
}

struct WlSmem {
  float* stage0;  // SD dense stages of kTileFloats
  float* odd0;    // SO odd-stride stages of kLeftStageFloats
  float* hs0;     // two H slots of hs_floats
  float4* red;    // kThreads
  WsHeader* hdr;  // SD (dense, written by the loader)
  WlHeader* ohdr; // SO (odd, written by the builders)
  WsSlot* slot;
  unsigned* ocons;  // SO: consumer-warp releases of each odd stage so far
  uint32_t bar0;
  int S, SO, hs_floats;
  long long wait;
  __device__ float* xs(int s) const { return stage0 + (size_t)s * kTileFloats; }
  __device__ float* os(int o) const { return odd0 + (size_t)o * kLeftStageFloats; }
  __device__ float* hs(int h) const { return hs0 + (size_t)h * hs_floats; }
  __device__ uint32_t full(int s) const { return bar0 + 8u * s; }
  __device__ uint32_t empty(int s) const { return bar0 + 8u * (S + s); }
  __device__ uint32_t hfull(int s) const { return bar0 + 8u * (2 * S + s); }
  __device__ uint32_t ofull(int o) const { return bar0 + 8u * (3 * S + o); }
  __device__ uint32_t islot_full(int i) const { return bar0 + 8u * (3 * S + SO + i); }
  __device__ uint32_t islot_empty(int i) const { return bar0 + 8u * (3 * S + SO + kWsItemSlots + i); }
  __device__ uint32_t hslot_empty(int h) const {
    return bar0 + 8u * (3 * S + SO + 2 * kWsItemSlots + h);
  }
  __device__ uint32_t red_full() const { return bar0 + 8u * (3 * S + SO + 2 * kWsItemSlots + 2); }
  __device__ uint32_t red_empty() const { return bar0 + 8u * (3 * S + SO + 2 * kWsItemSlots + 3); }
  __host__ __device__ static constexpr int bars(int S, int SO) { return 3 * S + SO + 2 * kWsItemSlots + 4; }
};

__host__ __device__ constexpr size_t wl_smem_bytes(int S, int SO, int hs_floats) {
  return (size_t)S * kTileFloats * sizeof(float) + (size_t)SO * kLeftStageFloats * sizeof(float) +
         2 * (size_t)hs_floats * sizeof(float) + (size_t)kThreads * sizeof(float4) +
         (size_t)S * sizeof(WsHeader) + (size_t)SO * sizeof(WlHeader) +
         (size_t)kWsItemSlots * sizeof(WsSlot) + (size_t)WlSmem::bars(S, SO) * sizeof(uint64_t) +
         (size_t)((SO + 1) / 2) * sizeof(uint64_t);
}

// Builder warp b handles dense stages b, b + 3, b + 6, ...; dense stage n
// becomes odd stage n % SO.
__device__ void wl_builder(const WlSmem& sm, int* err) {
  const int lane = threadIdx.x & 31;
  const int b = (threadIdx.x >> 5) - 2;
  for (int n = b;; n += kWsBuildWarps) {
    const int s = n % sm.S, o = n % sm.SO;
    if (!mb_wait(sm.hfull(s), (n / sm.S) & 1, sm.wait, err, 20)) return;
    const WsHeader& h = sm.hdr[s];
    const int w = h.d.w, k = h.k;
    if (w < 0) {
      if (k == 0) {  // the first stop stage ends the odd ring too
        if (!count_wait(sm.ocons + o, kWsConsWarps * (unsigned)(n / sm.SO), sm.wait, err, 21)) return;
        if (lane == 0) sm.ohdr[o].d.w = -1;
        __syncwarp();
        if (lane == 0) mb_arrive(sm.ofull(o));
      }
      return;
    }
    const int I1 = h.d.I1, R = h.d.R, seq = h.d.seq;
    const int jt = h.d.j0 + k * h.d.nj, njk = min(h.d.nj, h.d.j1 - jt);
    const float* H1 = h.d.H[0];
    const uint32_t word = reinterpret_cast<const uint32_t*>(&h.d)[lane];
    if (!mb_wait(sm.full(s), (n / sm.S) & 1, sm.wait, err, 22)) return;
    if (!count_wait(sm.ocons + o, kWsConsWarps * (unsigned)(n / sm.SO), sm.wait, err, 23)) return;
    const int hslot = seq & 1;
    if (k == 0) {  // H_1 of the item, rank padded to Rp with zeros
      if (!mb_wait(sm.hslot_empty(hslot), ((seq >> 1) & 1) ^ 1, sm.wait, err, 24)) return;
      float* hd = sm.hs(hslot);
      const int Rp = b_rank_pad(R);
      for (int e = lane; e < I1 * Rp; e += 32) {
        const int i = e / Rp, r = e - i * Rp;
        hd[e] = r < R ? __ldg(H1 + i * R + r) : 0.0f;
      }
    }
    // the tile at odd row stride: four consecutive elements per lane and step
    const float* src = sm.xs(s);
    float* dst = sm.os(o);
    const int ST = I1 | 1, L = njk * I1, L4 = L & ~3;
    int row = (4 * lane) / I1, col = 4 * lane - row * I1;
    const int drow = 128 / I1, dcol = 128 - drow * I1;
    for (int e = 4 * lane; e < L4; e += 128) {
      const float4 v = *reinterpret_cast<const float4*>(src + e);
      int r = row, c = col;
      dst[r * ST + c] = v.x;
      if (++c == I1) c = 0, ++r;
      dst[r * ST + c] = v.y;
      if (++c == I1) c = 0, ++r;
      dst[r * ST + c] = v.z;
      if (++c == I1) c = 0, ++r;
      dst[r * ST + c] = v.w;
      row += drow;
      col += dcol;
      if (col >= I1) {
        col -= I1;
        ++row;
      }
    }
    if (L4 + lane < L) {
      const int e = L4 + lane, r = e / I1;
      dst[r * ST + (e - r * I1)] = src[e];
    }
    reinterpret_cast<uint32_t*>(&sm.ohdr[o].d)[lane] = word;
    if (lane == 0) {
      sm.ohdr[o].k = k;
      sm.ohdr[o].hslot = hslot;
    }
    __syncwarp();
    if (lane == 0) {
      mb_arrive(sm.empty(s));  // the dense stage has been read
      mb_arrive(sm.ofull(o));  // the odd stage, its header and the H slot are written
    }
  }
}

// One item of root -> {2..N} (its first odd stage already waited for).
template <int RQB>
__device__ bool wl_consume(const WlHeader& h0, int& n, int& nred, const WlSmem& sm, int* err) {
  const int ct = threadIdx.x - 32 * kWsConsFirstWarp;  // 0 .. 255
  const int lane = threadIdx.x & 31;
  const WsDesc& d = h0.d;
  const int R = d.R, I1 = d.I1, nj = d.nj, jb0 = d.j0, jb1 = d.j1, ntile = d.ntile;
  const int hslot = h0.hslot;
  float* T = d.out;
  const int Rq = b_rq(R), ST = I1 | 1;
  const int NB = Rq / RQB;
  const int P = nj * NB;
  const int G = P >= kGroupThreads ? 1 : kGroupThreads / P;
  const int npass = (P + kThreads - 1) / kThreads;
  const int g = G > 1 ? ct / P : 0;
  const int ia = g * I1 / G, ib = (g + 1) * I1 / G;
  const float4* H4 = reinterpret_cast<const float4*>(sm.hs(hslot));
  for (int k = 0; k < ntile; ++k, ++n) {
    const int o = n % sm.SO;
    if (k > 0 && !mb_wait(sm.ofull(o), (n / sm.SO) & 1, sm.wait, err, 25)) return false;
    const int jt = jb0 + k * nj, njk = min(nj, jb1 - jt);
    const float* Xs = sm.os(o);
    for (int p = 0; p < npass; ++p) {
      const int pair = G > 1 ? ct - g * P : ct + kThreads * p;
      const int jl = pair / NB, qb = pair - jl * NB;
      const bool v = g < G && pair < P && jl < njk;
      float a[RQB][4];
#pragma unroll
      for (int u = 0; u < RQB; ++u)
#pragma unroll
        for (int b = 0; b < 4; ++b) a[u][b] = 0.0f;
      if (v) {
        const float* xp = Xs + jl * ST;
        const float4* hp = H4 + qb * RQB;
#pragma unroll 4
        for (int i = ia; i < ib; ++i) {
          const float x = xp[i];
#pragma unroll
          for (int u = 0; u < RQB; ++u) fma4(a[u], x, hp[i * Rq + u]);
        }
      }
      if (G > 1) {  // RQB == 1 here
        const uint32_t par = nred & 1;
        ++nred;
        if (!mb_wait(sm.red_empty(), par ^ 1, sm.wait, err, 26)) return false;
        if (g < G) sm.red[ct] = make_float4(a[0][0], a[0][1], a[0][2], a[0][3]);
        __syncwarp();
        if (lane == 0) mb_arrive(sm.red_full());
        if ((ct & ~31) < P && !mb_wait(sm.red_full(), par, sm.wait, err, 27)) return false;
        if (ct < P) {
          const int jl0 = ct / NB, q0 = ct - jl0 * NB;
          if (jl0 < njk) {
            float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int gg = 0; gg < G; ++gg) {
              const float4 wv = sm.red[gg * P + ct];
              s4[0] += wv.x;
              s4[1] += wv.y;
              s4[2] += wv.z;
              s4[3] += wv.w;
            }
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (4 * q0 + b < R) T[(long long)(jt + jl0) * R + 4 * q0 + b] = s4[b];
          }
        }
        __syncwarp();
        if (lane == 0) mb_arrive(sm.red_empty());
      } else if (v) {
#pragma unroll
        for (int u = 0; u < RQB; ++u)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = 4 * (qb * RQB + u) + b;
            if (r < R) T[(long long)(jt + jl) * R + r] = a[u][b];
          }
      }
    }
    __syncwarp();
    if (lane == 0) smem_add_release(sm.ocons + o, 1u);
  }
  __syncwarp();
  if (lane == 0) mb_arrive(sm.hslot_empty(hslot));
  return true;
}

template <int RMAX>
__device__ void wl_consumer(const WlSmem& sm, int* err) {
  int nred = 0;
  for (int n = 0;;) {
    const int o = n % sm.SO;
    if (!mb_wait(sm.ofull(o), (n / sm.SO) & 1, sm.wait, err, 28)) return;
    const WlHeader& h = sm.ohdr[o];
    if (h.d.w < 0) return;
    bool ok = true;
    switch (b_rqb_left(h.d.I1, h.d.R)) {
      case 1: ok = wl_consume<1>(h, n, nred, sm, err); break;
      case 2: ok = wl_consume<2>(h, n, nred, sm, err); break;
      case 4: ok = wl_consume<4>(h, n, nred, sm, err); break;
      case 8: if constexpr (RMAX >= 32) ok = wl_consume<8>(h, n, nred, sm, err); break;
      default: if constexpr (RMAX >= 64) ok = wl_consume<16>(h, n, nred, sm, err); break;
    }
    if (!ok) return;
  }
}

template <int RMAX>
__global__ void __launch_bounds__(kWsThreads, RMAX <= 16 ? 2 : 1)
k_b_pm_left_ws(const BTensor* __restrict__ ts, const int4* __restrict__ items, int n_items,
               int* queue, int S, int SO, int hs_floats, int* err, long long wait_cycles) {
  extern __shared__ __align__(16) float smem[];
  WlSmem sm;
  sm.S = S;
  sm.SO = SO;
  sm.hs_floats = hs_floats;
  sm.wait = wait_cycles > 0 ? wait_cycles : kWsWaitCycles;
  sm.stage0 = smem;
  sm.odd0 = smem + (size_t)S * kTileFloats;
  sm.hs0 = sm.odd0 + (size_t)SO * kLeftStageFloats;
  sm.red = reinterpret_cast<float4*>(sm.hs0 + 2 * (size_t)hs_floats);
  sm.hdr = reinterpret_cast<WsHeader*>(sm.red + kThreads);
  sm.ohdr = reinterpret_cast<WlHeader*>(sm.hdr + S);
  sm.slot = reinterpret_cast<WsSlot*>(sm.ohdr + SO);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm.slot + kWsItemSlots);
  sm.bar0 = smem_u32(bars);
  sm.ocons = reinterpret_cast<unsigned*>(bars + WlSmem::bars(S, SO));
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mb_init(sm.full(s), 32);  // the loader lanes' copies
      mb_init(sm.empty(s), 1);  // the builder warp of the stage
      mb_init(sm.hfull(s), 1);  // the loader's header
    }
    for (int o = 0; o < SO; ++o) {
      mb_init(sm.ofull(o), 1);  // the builder warp of the stage
      sm.ocons[o] = 0u;
    }
    for (int i = 0; i < kWsItemSlots; ++i) {
      mb_init(sm.islot_full(i), 1);
      mb_init(sm.islot_empty(i), 1);
    }
    mb_init(sm.hslot_empty(0), kWsConsWarps);
    mb_init(sm.hslot_empty(1), kWsConsWarps);
    mb_init(sm.red_full(), kWsConsWarps);
    mb_init(sm.red_empty(), kWsConsWarps);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  if (warp == 0)
    ws_scheduler<true>(ts, items, n_items, queue, sm, err);
  else if (warp == 1)
    ws_loader(sm, err);
  else if (warp < kWsConsFirstWarp)
    wl_builder(sm, err);
  else
    wl_consumer<RMAX>(sm, err);
}

// ---------------------------------------------------------- multi-TTVs --

// leaf M(a) from node {a..N} (Fig. 1): M(i, r) = sum_k T[(i + I_a k) R + r] KK(k, r),
// KK = H_N (.) ... (.) H_{a+1}.  Item (tensor, chunk c of leaf_kc[a] rows k,
// block of kLeafBlock outputs).  For each k the node slice of all (i, r) is
// contiguous, so thread = output e = i R + r reads it coalesced; KK rows are
// formed per tile of kLeafTileK rows in shared memory.  Writes lpart[c].
__global__ void __launch_bounds__(256) k_b_mttv_leaf(const BTensor* __restrict__ ts,
                                                     const int4* __restrict__ items, int a) {
  const int4 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  if (tensor_done(t)) return;
  __shared__ float KKs[kLeafTileK * kBatchMaxRank];
  const int tid = threadIdx.x;
  const int R = t.R, N = t.N;
  const int E = (int)t.dims[a] * R;
  int K = 1;
  for (int m = a + 1; m < N; ++m) K *= (int)t.dims[m];
  const int kc = t.leaf_kc[a];
  const int k0 = it.y * kc, k1 = min(K, k0 + kc);
  int ep[4], rp[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ep[q] = it.z * kLeafBlock + tid + 256 * q;
    rp[q] = ep[q] % R;
  }
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float* T = t.node[a];
  for (int kt = k0; kt < k1; kt += kLeafTileK) {
    const int nk = min(kLeafTileK, k1 - kt);
    __syncthreads();
    // KK rows of the tile: entries x = kk R + r < nk R <= 4096, four per thread at a time
    for (int x0 = tid; x0 < nk * R; x0 += 4 * 256) {
      float w[4];
      int rem[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        rem[u] = kt + (x0 + 256 * u) / R;
        w[u] = 1.0f;
      }
      for (int m = a + 1; m < N; ++m) {
        const int dm = (int)t.dims[m];
        const float* Hm = t.H[m];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int x = x0 + 256 * u;
          if (x < nk * R) {
            const int jm = rem[u] % dm;
            rem[u] /= dm;
            w[u] *= __ldg(Hm + jm * R + x % R);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int x = x0 + 256 * u;
        if (x < nk * R) KKs[x] = w[u];
      }
    }
    __syncthreads();
    const float* Tb = T + (long long)kt * E;
#pragma unroll 4
    for (int kk = 0; kk < nk; ++kk) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ep[q] < E) acc[q] = fmaf(Tb[(long long)kk * E + ep[q]], KKs[kk * R + rp[q]], acc[q]);
    }
  }
  float* out = t.lpart + (long long)it.y * E;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (ep[q] < E) out[ep[q]] = acc[q];
}

// child node {a+1..N} from node {a..N}: out(j, r) = sum_i T[(i + I_a j) R + r] H_a(i, r)
// with the updated H_a; the output is M when the child is a leaf.  Item
// (tensor, block of first_jb[a] rows j); warp per row j (two rows at a time,
// for more loads in flight): lanes = (i phase, rank) read the row's I_a x R
// block coalesced, then add their i phases in a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_b_mttv_first(const BTensor* __restrict__ ts,
                                                      const int4* __restrict__ items, int a) {
  const int4 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  if (tensor_done(t)) return;
  const int R = t.R, N = t.N;
  const int Ia = (int)t.dims[a];
  const int E = Ia * R;
  int K = 1;
  for (int m = a + 1; m < N; ++m) K *= (int)t.dims[m];
  const int jb = t.first_jb[a];
  const int j0 = it.y * jb, j1 = min(K, j0 + jb);
  const float* T = t.node[a];
  float* out = (a + 1 == N - 1) ? t.M : t.node[a + 1];
  const float* Ha = t.H[a];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int rb = 0; rb < R; rb += 32) {
    const int Rb = min(32, R - rb), S = 32 / Rb;
    const int sub = lane / Rb, r = rb + lane - sub * Rb;
    const bool act = sub < S;
    for (int j = j0 + warp; j < j1; j += 2 * nwarp) {
      const int j2 = j + nwarp;
      const bool two = j2 < j1;
      const float* Tj = T + (long long)j * E;
      const float* Tk = T + (long long)(two ? j2 : j) * E;
      float acc = 0.0f, acc2 = 0.0f;
      if (act) {
#pragma unroll 8
        for (int i = sub; i < Ia; i += S) {
          const float h = __ldg(Ha + i * R + r);
          acc = fmaf(Tj[i * R + r], h, acc);
          acc2 = fmaf(Tk[i * R + r], h, acc2);
        }
      }
      for (int o = 1; o < S; o <<= 1) {
        const float v = __shfl_down_sync(0xffffffffu, acc, o * Rb);
        const float v2 = __shfl_down_sync(0xffffffffu, acc2, o * Rb);
        if (act && (sub & (2 * o - 1)) == 0 && sub + o < S) {
          acc += v;
          acc2 += v2;
        }
      }
      if (act && sub == 0) {
        out[(long long)j * R + r] = acc;
        if (two) out[(long long)j2 * R + r] = acc2;
      }
    }
  }
}

// ---------------------------------------------------------- mode update --

// One CTA per tensor (I_n <= kBatchMaxI rows, R <= RMAX): HALS sweep
// (Sec. II-B, row per thread, row in registers), W^T W, lambda, G_n,
// H_n = W / lambda, the fit at n = N (Sec. IV-B) with the stopping test, and
// S for the next mode -- all in shared memory.
template <int RMAX>
__global__ void __launch_bounds__(256)
k_b_update(BTensor* __restrict__ ts, int n, int* __restrict__ done_count, int rows) {
  BTensor& t = ts[blockIdx.x];
  if (tensor_done(t)) return;
  constexpr int RP = RMAX + 1;
  const int R = t.R, N = t.N, R2 = R * R;
  const int In = (int)t.dims[n];
  const int tid = threadIdx.x;
  extern __shared__ __align__(16) float bsm[];
  // rows: the longest mode of the batch, so that small tensors leave room for
  // more CTAs per SM
  float* St = bsm;                 // RMAX x RMAX, St[r][c] = S[c][r], zero padded
  float* Ws = St + RMAX * RMAX;    // rows x RP (W, then H)
  float* Ms = Ws + rows * RP;      // rows x RP (M)
  __shared__ float lamf[RMAX], sinv[RMAX];
  __shared__ double GW[RMAX * RMAX];
  __shared__ double cinv[RMAX];
  __shared__ double red[8];
  float* Hn = t.H[n];
  // staging with the global loads of a loop issued in batches
#pragma unroll 4
  for (int e = tid; e < RMAX * RMAX; e += blockDim.x) {
    const int r = e / RMAX, c = e % RMAX;
    St[e] = (r < R && c < R) ? t.S32[c * R + r] : 0.0f;
  }
  for (int r = tid; r < RMAX; r += blockDim.x) {
    lamf[r] = r < R ? (float)t.lam[r] : 0.0f;
    const float srr = r < R ? t.S32[r * R + r] : 0.0f;
    sinv[r] = srr != 0.0f ? 1.0f / srr : 0.0f;
  }
  __syncthreads();
#pragma unroll 4
  for (int e = tid; e < In * R; e += blockDim.x) {
    const int i = e / R, c = e - i * R;
    Ws[i * RP + c] = Hn[e] * lamf[c];
    Ms[i * RP + c] = t.M[e];
  }
  for (int i = tid; i < In; i += blockDim.x)
    for (int c = R; c < RMAX; ++c) Ws[i * RP + c] = 0.0f;
  __syncthreads();
  double bp = 0.0;
  for (int i = tid; i < In; i += blockDim.x) {
    // row W(i, :) updated in place in shared memory (odd stride: one bank per
    // thread); rolled column loop, unrolled dot product (see the HALS sweep
    // of the single-problem update)
    float* wrow = Ws + i * RP;
    const float* mrow = Ms + i * RP;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      const float si = sinv[r];
      const float mr = mrow[r];
      float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
      for (int c = 0; c < RMAX; c += 2) {
        d0 = fmaf(wrow[c], St[r * RMAX + c], d0);
        d1 = fmaf(wrow[c + 1], St[r * RMAX + c + 1], d1);
      }
      const float wr = wrow[r];
      const float upd = fmaxf(0.0f, wr + (mr - (d0 + d1)) * si);
      wrow[r] = si != 0.0f ? upd : wr;
    }
    float b = 0.0f;
    for (int c = 0; c < R; ++c) b = fmaf(mrow[c], wrow[c], b);
    bp += (double)b;
  }
  for (int o = 16; o > 0; o >>= 1) bp += __shfl_xor_sync(0xffffffffu, bp, o);
  if ((tid & 31) == 0) red[tid >> 5] = bp;
  __syncthreads();
  for (int e = tid; e < R2; e += blockDim.x) {
    const int a = e / R, b = e % R;
    float s0 = 0.0f, s1 = 0.0f;
    int i = 0;
    for (; i + 1 < In; i += 2) {
      s0 = fmaf(Ws[i * RP + a], Ws[i * RP + b], s0);
      s1 = fmaf(Ws[(i + 1) * RP + a], Ws[(i + 1) * RP + b], s1);
    }
    if (i < In) s0 = fmaf(Ws[i * RP + a], Ws[i * RP + b], s0);
    GW[e] = (double)(s0 + s1);
  }
  __syncthreads();
  for (int r = tid; r < R; r += blockDim.x) {
    const double v = sqrt(GW[r * R + r]);
    t.lam[r] = v;
    cinv[r] = v > 0.0 ? 1.0 / v : 0.0;
    lamf[r] = v > 0.0 ? (float)(1.0 / v) : 0.0f;
  }
  __syncthreads();
  double* Gn = t.G + (long long)n * R2;
  for (int e = tid; e < R2; e += blockDim.x) Gn[e] = GW[e] * cinv[e / R] * cinv[e % R];
  for (int e = tid; e < In * R; e += blockDim.x) Hn[e] = Ws[(e / R) * RP + e % R] * lamf[e % R];
  if (n == N - 1) {
    double g = 0.0;
    for (int e = tid; e < R2; e += blockDim.x) g += t.S[e] * GW[e];
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    __syncthreads();
    __shared__ double red2[8];
    if ((tid & 31) == 0) red2[tid >> 5] = g;
    __syncthreads();
    if (tid == 0) {
      double beta = 0.0, gamma = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        beta += red[w];
        gamma += red2[w];
      }
      const double alpha = t.scal[0];
      const double eps = sqrt(fmax(0.0, alpha - 2.0 * beta + gamma) / alpha);
      const double fit = 1.0 - eps;
      const int k = t.flags[1];
      if (k < t.fit_cap) t.fits[k] = fit;
      t.flags[1] = k + 1;
      bool stop = !isfinite(fit) || (k + 1 >= t.max_iters);
      if (!isfinite(fit)) t.flags[2] = 1;
      if (k >= 1 && k - 1 < t.fit_cap && fabs(fit - t.fits[k - 1]) < t.scal[1]) stop = true;
      if (stop) {
        t.flags[0] = 1;
        atomicAdd(done_count, 1);
      }
    }
  }
  __syncthreads();
  const int next = (n + 1) % N;
  for (int e = tid; e < R2; e += blockDim.x) {
    double s = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != next) s *= (k == n) ? Gn[e] : t.G[(long long)k * R2 + e];
    t.S[e] = s;
    t.S32[e] = (float)s;
  }
}

__global__ void k_b_gather(const BTensor* __restrict__ ts, int count, int* iters, double* fits,
                           double* lam, const int* lam_off, int* nonfinite) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
    const BTensor& t = ts[b];
    const int k = t.flags[1];
    iters[b] = k;
    fits[b] = (k >= 1 && k <= t.fit_cap) ? t.fits[k - 1] : 0.0;
    nonfinite[b] = (t.flags[2] ? 1 : 0) | (t.flags[0] ? 2 : 0);  // bit 0 non-finite, bit 1 done
    if (lam)
      for (int r = 0; r < t.R; ++r) lam[lam_off[b] + r] = t.lam[r];
  }
}

template <int RMAX>
size_t update_smem(int rows = kBatchMaxI) {
  return (size_t)(RMAX * RMAX + 2 * rows * (RMAX + 1)) * sizeof(float);
}

}  // namespace

cudaError_t batch_attributes_init() {
  cudaError_t e = cudaFuncSetAttribute(k_b_update<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)update_smem<16>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_b_update<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_smem<32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_b_update<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_smem<64>());
  const int right = (2 * kTileFloats + kWsFloats) * (int)sizeof(float);
  const int left = (left_fixed_floats() + kBatchMaxI * kBatchMaxRank) * (int)sizeof(float);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_right<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, right);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_right<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, right);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_right<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, right);
  int dev = 0, optin = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_right_ws<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_right_ws<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_right_ws<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_left_ws<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_left_ws<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_left_ws<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_left<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, left);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_left<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, left);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_pm_left<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, left);
  return e;
}

namespace {

// Grid of a root phase: one CTA per item (queue NULL), or one wave of
// persistent CTAs (every CTA that fits at once at this shared-memory size)
// taking items from the counter `queue`.
template <typename K>
int phase_grid(K kernel, size_t smem, int n_items, const int* queue) {
  if (!queue) return n_items;
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return std::max(1, std::min(n_items, sms * per_sm));
}

}  // namespace

namespace {

// Streamed root -> {1}: as many ring stages (at most 8) as fit at two CTAs per
// SM (RMAX 16) or one, and one wave of CTAs.
template <int RMAX>
cudaError_t launch_pm_right_ws(const BTensor* ts, const int4* it, int n, int* queue, int* err,
                               long long wait_cycles, cudaStream_t st) {
  int dev = 0, sms = 1, smem_sm = 0, reserved = 0, optin = 0, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int want = RMAX <= 16 ? 2 : 1;
  const size_t budget = std::min<size_t>((size_t)optin, (size_t)(smem_sm / want - reserved));
  int S = 8;
  while (S > kWsBuildWarps + 1 && ws_smem_bytes(S) > budget) --S;
  const size_t bytes = ws_smem_bytes(S);
  if (bytes > (size_t)optin) return cudaErrorInvalidConfiguration;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_pm_right_ws<RMAX>, kWsThreads,
                                                    bytes) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int grid = std::max(1, std::min(n, sms * per_sm));
  k_b_pm_right_ws<RMAX><<<grid, kWsThreads, bytes, st>>>(ts, it, n, queue, S, err, wait_cycles);
  return cudaGetLastError();
}

// Streamed root -> {2..N}: the largest dense / odd-stride rings (at least
// three dense stages, one per builder's stop stage) that fit beside the two
// H_1 slots at two CTAs per SM (RMAX 16, when they fit) or one.
template <int RMAX>
cudaError_t launch_pm_left_ws(const BTensor* ts, const int4* it, int n, int* queue, int hs_floats,
                              int* err, long long wait_cycles, cudaStream_t st) {
  int dev = 0, sms = 1, smem_sm = 0, reserved = 0, optin = 0, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  static const int cand[][2] = {{4, 3}, {4, 2}, {3, 3}, {3, 2}};
  int S = 0, SO = 0;
  // two CTAs per SM at ranks <= 16 when the H_1 slots leave room, else one
  for (int want = RMAX <= 16 ? 2 : 1; want >= 1 && S == 0; --want) {
    const size_t budget = std::min<size_t>((size_t)optin, (size_t)(smem_sm / want - reserved));
    for (const auto& c : cand)
      if (wl_smem_bytes(c[0], c[1], hs_floats) <= budget) {
        S = c[0];
        SO = c[1];
        break;
      }
  }
  if (S == 0) return cudaErrorInvalidConfiguration;
  const size_t bytes = wl_smem_bytes(S, SO, hs_floats);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_pm_left_ws<RMAX>, kWsThreads,
                                                    bytes) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int grid = std::max(1, std::min(n, sms * per_sm));
  k_b_pm_left_ws<RMAX><<<grid, kWsThreads, bytes, st>>>(ts, it, n, queue, S, SO, hs_floats, err,
                                                        wait_cycles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pm_right(const BPlan& p, const BTensor* ts, const int4* items, int mode,
                            int* queue, int* err, cudaStream_t st, long long wait_cycles) {
  const size_t sm = (size_t)(2 * kTileFloats + kWsFloats) * sizeof(float);
  const int n = p.pmr.count;
  const int4* it = items + p.pmr.off;
  if (mode == 0 || !queue) queue = nullptr;
  if (n > 0 && mode == 2 && queue && err) {
    cudaError_t e = p.rmax <= 16   ? launch_pm_right_ws<16>(ts, it, n, queue, err, wait_cycles, st)
                    : p.rmax <= 32 ? launch_pm_right_ws<32>(ts, it, n, queue, err, wait_cycles, st)
                                   : launch_pm_right_ws<64>(ts, it, n, queue, err, wait_cycles, st);
    if (e != cudaSuccess) return e;
  } else if (n > 0) {
    if (p.rmax <= 16)
      k_b_pm_right<16><<<phase_grid(k_b_pm_right<16>, sm, n, queue), kThreads, sm, st>>>(ts, it, n, queue);
    else if (p.rmax <= 32)
      k_b_pm_right<32><<<phase_grid(k_b_pm_right<32>, sm, n, queue), kThreads, sm, st>>>(ts, it, n, queue);
    else
      k_b_pm_right<64><<<phase_grid(k_b_pm_right<64>, sm, n, queue), kThreads, sm, st>>>(ts, it, n, queue);
  }
  if (p.pmr_red.count > 0)
    k_b_reduce<<<p.pmr_red.count, kReduceBlock, 0, st>>>(ts, items + p.pmr_red.off);
  return cudaGetLastError();
}

cudaError_t launch_pm_left(const BPlan& p, const BTensor* ts, const int4* items, int mode,
                           int* queue, int* err, cudaStream_t st, long long wait_cycles) {
  if (mode == 0 || !queue) queue = nullptr;
  const int n = p.pml.count;
  if (n == 0) return cudaSuccess;
  const int4* it = items + p.pml.off;
  if (mode == 2 && queue && err)
    return p.rmax <= 16   ? launch_pm_left_ws<16>(ts, it, n, queue, p.hs_floats, err, wait_cycles, st)
           : p.rmax <= 32 ? launch_pm_left_ws<32>(ts, it, n, queue, p.hs_floats, err, wait_cycles, st)
                          : launch_pm_left_ws<64>(ts, it, n, queue, p.hs_floats, err, wait_cycles, st);
  const size_t sm = (size_t)(left_fixed_floats() + p.hs_floats) * sizeof(float);
  if (p.rmax <= 16)
    k_b_pm_left<16><<<phase_grid(k_b_pm_left<16>, sm, n, queue), kThreads, sm, st>>>(ts, it, n, queue);
  else if (p.rmax <= 32)
    k_b_pm_left<32><<<phase_grid(k_b_pm_left<32>, sm, n, queue), kThreads, sm, st>>>(ts, it, n, queue);
  else
    k_b_pm_left<64><<<phase_grid(k_b_pm_left<64>, sm, n, queue), kThreads, sm, st>>>(ts, it, n, queue);
  return cudaGetLastError();
}

namespace {

cudaError_t launch_update(const BPlan& p, BTensor* ts, int n, int* done_count, cudaStream_t st) {
  const int rows = p.max_rows;
  if (p.rmax <= 16)
    k_b_update<16><<<p.count, 256, update_smem<16>(rows), st>>>(ts, n, done_count, rows);
  else if (p.rmax <= 32)
    k_b_update<32><<<p.count, 256, update_smem<32>(rows), st>>>(ts, n, done_count, rows);
  else
    k_b_update<64><<<p.count, 256, update_smem<64>(rows), st>>>(ts, n, done_count, rows);
  return cudaGetLastError();
}

}  // namespace

cudaError_t b_launch_init(const BPlan& p, BTensor* ts, const int4* items, double* alpha_part,
                          const int* alpha_first, cudaStream_t st) {
  if (p.count == 0) return cudaSuccess;
  if (p.alpha.count > 0)
    k_b_sumsq<<<p.alpha.count, 256, 0, st>>>(ts, items + p.alpha.off, alpha_part);
  k_b_init<<<p.count, 256, 0, st>>>(ts, alpha_part, alpha_first);
  return cudaGetLastError();
}

cudaError_t b_launch_iteration(const BPlan& p, BTensor* ts, const int4* items, int* done_count,
                               cudaStream_t st, const BSchedule& sch, int* queues) {
  if (p.count == 0) return cudaSuccess;
  const int N = p.N;
  cudaError_t e = cudaSuccess;
  const bool counters = queues && (sch.pm_right || sch.pm_left);
  if (counters) e = cudaMemsetAsync(queues, 0, 2 * sizeof(int), st);
  int* err = queues ? queues + 2 : nullptr;
  if (e == cudaSuccess)
    e = launch_pm_right(p, ts, items, counters ? sch.pm_right : 0, queues, err, st, sch.wait_cycles);
  if (e == cudaSuccess) e = launch_update(p, ts, 0, done_count, st);
  if (e == cudaSuccess)
    e = launch_pm_left(p, ts, items, counters ? sch.pm_left : 0, queues ? queues + 1 : nullptr, err, st,
                       sch.wait_cycles);
  // node {2..N} walk (Fig. 1 shape): leaf M(a), update, child node
  for (int a = 1; a < N && e == cudaSuccess; ++a) {
    if (a == N - 1) {
      e = launch_update(p, ts, a, done_count, st);
      break;
    }
    if (p.leaf[a].count > 0)
      k_b_mttv_leaf<<<p.leaf[a].count, 256, 0, st>>>(ts, items + p.leaf[a].off, a);
    if (p.leaf_red[a].count > 0)
      k_b_reduce<<<p.leaf_red[a].count, kReduceBlock, 0, st>>>(ts, items + p.leaf_red[a].off);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_update(p, ts, a, done_count, st);
    if (e == cudaSuccess && p.first[a].count > 0) {
      k_b_mttv_first<<<p.first[a].count, 256, 0, st>>>(ts, items + p.first[a].off, a);
      e = cudaGetLastError();
    }
  }
  return e;
}

cudaError_t launch_b_gather(const BTensor* ts, int count, int* iters, double* fits,
                            double* lam, const int* lam_off, int* nonfinite, cudaStream_t st) {
  k_b_gather<<<(count + 255) / 256, 256, 0, st>>>(ts, count, iters, fits, lam, lam_off, nonfinite);
  return cudaGetLastError();
}

}  // namespace nncp
