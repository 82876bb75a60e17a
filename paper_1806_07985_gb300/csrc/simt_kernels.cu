// CUDA-core kernels: generic MTTKRP over a (L, I, Q) view of the tensor,
// multi-TTVs on dimension-tree nodes, sums of squares, bf16 conversion.
//
// The (L, I, Q) view: mode set split as [modes before] x [output modes] x
// [modes after], so X[l + L*(i + I*q)] holds the entry with left index l,
// output index i and right index q (mode-1-fastest layout, Sec. IV-C).
//   * direct MTTKRP of mode n (Sec. II-A): L = I_1..I_{n-1}, I = I_n,
//     Q = I_{n+1}..I_N;
//   * partial MTTKRP root -> {1..s} (Sec. IV-A, Fig. 2a): L = 1,
//     I = I_1..I_s, Q = I_{s+1}..I_N (contracts the slow modes);
//   * partial MTTKRP root -> {s+1..N}: L = I_1..I_s, I = I_{s+1}..I_N, Q = 1
//     (contracts the fast modes).
// The Khatri-Rao rows are formed on the fly in shared memory from factor rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "nncp_internal.cuh"

namespace nncp {

namespace {

constexpr int kBI = 128;  // output rows per CTA
constexpr int kBK = 32;   // contraction tile
constexpr int kRT = 32;   // rank columns per CTA
constexpr int kThreads = 256;

// Per-tile row offsets of the Khatri-Rao factors: for contraction index k,
// off[m] = (row of mode m) * R, so KRP(k, r) = prod_m H_m[off[m] + r].
struct TileRows {
  int off[2 * kMaxModes];
  long long xbase;  // X offset of (i = 0, k)
  int valid;
};

__device__ __forceinline__ void decompose(const KrpDesc& d, long long k, int R, int* off) {
  for (int m = 0; m < d.nm; ++m) {
    long long dm = d.dim[m];
    long long km = k % dm;
    k /= dm;
    off[m] = (int)(km * R);
  }
}

__device__ __forceinline__ float krp_value(const KrpDesc& d, const int* off, int r) {
  float v = 1.0f;
  for (int m = 0; m < d.nm; ++m) v *= __ldg(d.H[m] + off[m] + r);
  return v;
}

// X elements each thread stages per contraction tile
constexpr int kXPer = kBK * kBI / kThreads;

template <bool kSlow>
__global__ void __launch_bounds__(kThreads, 4)
k_simt_mttkrp(const float* __restrict__ X, long long L, long long I, long long Q, KrpDesc KL,
              KrpDesc KQ, int R, long long kchunk, float* __restrict__ out,
              long long out_chunk_stride) {
  pdl_wait();  // no early trigger: a large grid; its successor spreads as CTAs exit
  __shared__ __align__(16) float Xs[kBK][kBI + 4];
  __shared__ __align__(16) float Ws[kBK][kRT];
  __shared__ TileRows rows[2][kBK];  // this tile's and the next one's

  const long long Ktot = L * Q;
  const long long i0 = (long long)blockIdx.x * kBI;
  const int r0 = blockIdx.z * kRT;
  const long long kbeg = (long long)blockIdx.y * kchunk;
  const long long kend = min(Ktot, kbeg + kchunk);
  const int tid = threadIdx.x;
  const int tx = tid & 7;   // rank group: r0 + 4*tx .. +3
  const int ty = tid >> 3;  // row group:  i0 + 4*ty .. +3

  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;

  // row metadata of the tile at k0 into rows[buf] (threads < kBK)
  auto tile_rows = [&](long long k0, int buf) {
    if (tid < kBK) {
      long long k = k0 + tid;
      TileRows tr;
      tr.valid = k < kend;
      if (tr.valid) {
        long long l = k % L, q = k / L;
        decompose(KL, l, R, tr.off);
        decompose(KQ, q, R, tr.off + kMaxModes);
        tr.xbase = l + L * I * q;
      } else {
        tr.xbase = 0;
      }
      rows[buf][tid] = tr;
    }
  };
  // this thread's X elements of the tile described by rows[buf]: element
  // (i, k) at xbase(k) + L*i, read along whichever of i and k is contiguous
  float xr[kXPer];
  // L == 1 with I % 4 == 0 and X 16-byte aligned: every tile row is four-float
  // aligned, so thread tid reads four consecutive i of rows tid / 32 + 8 v.
  // L % 32 == 0 (and X aligned): a tile's 32 k share q and have consecutive l,
  // and chunks and totals are multiples of 32, so a tile is wholly valid or
  // not; thread tid reads four consecutive k of row i = (tid + 256 v) / 8.
  const bool aligned = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  const bool vec = kSlow && (I & 3) == 0 && aligned;
  const bool veck = !kSlow && (L & 31) == 0 && aligned;
  auto load_x = [&](int buf) {
    if (veck) {
#pragma unroll
      for (int v = 0; v < kXPer / 4; ++v) {
        const int id = tid + kThreads * v, ii = id >> 3, kk = 4 * (id & 7);
        const long long i = i0 + ii;
        float4 x4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (rows[buf][kk].valid && i < I)
          x4 = __ldg(reinterpret_cast<const float4*>(X + rows[buf][kk].xbase + L * i));
        xr[4 * v] = x4.x;
        xr[4 * v + 1] = x4.y;
        xr[4 * v + 2] = x4.z;
        xr[4 * v + 3] = x4.w;
      }
      return;
    }
    if (vec) {
      const int ii = 4 * (tid & 31);
#pragma unroll
      for (int v = 0; v < kXPer / 4; ++v) {
        const int kk = (tid >> 5) + 8 * v;
        const long long i = i0 + ii;
        float4 x4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (rows[buf][kk].valid && i < I)  // i < I covers i .. i + 3 (I % 4 == 0)
          x4 = __ldg(reinterpret_cast<const float4*>(X + rows[buf][kk].xbase + i));
        xr[4 * v] = x4.x;
        xr[4 * v + 1] = x4.y;
        xr[4 * v + 2] = x4.z;
        xr[4 * v + 3] = x4.w;
      }
      return;
    }
#pragma unroll
    for (int u = 0; u < kXPer; ++u) {
      const int e = tid + kThreads * u;
      int kk, ii;
      if (kSlow) { kk = e / kBI; ii = e % kBI; }   // L == 1: rows contiguous in i
      else       { kk = e % kBK; ii = e / kBK; }   // contiguous in k (l fastest)
      const long long i = i0 + ii;
      xr[u] = (rows[buf][kk].valid && i < I) ? __ldg(X + rows[buf][kk].xbase + L * i) : 0.0f;
    }
  };

  int cur = 0;
  if (kbeg < kend) {
    tile_rows(kbeg, 0);
    __syncthreads();
    load_x(0);
  }
  for (long long k0 = kbeg; k0 < kend; k0 += kBK, cur ^= 1) {
    const bool more = k0 + kBK < kend;
    for (int e = tid; e < kBK * kRT; e += kThreads) {
      int kk = e / kRT, rr = e % kRT;
      int r = r0 + rr;
      float w = 0.0f;
      if (rows[cur][kk].valid && r < R)
        w = krp_value(KL, rows[cur][kk].off, r) * krp_value(KQ, rows[cur][kk].off + kMaxModes, r);
      Ws[kk][rr] = w;
    }
    if (veck) {
#pragma unroll
      for (int v = 0; v < kXPer / 4; ++v) {
        const int id = tid + kThreads * v, ii = id >> 3, kk = 4 * (id & 7);
#pragma unroll
        for (int j = 0; j < 4; ++j) Xs[kk + j][ii] = xr[4 * v + j];
      }
    } else if (vec) {
#pragma unroll
      for (int v = 0; v < kXPer / 4; ++v)
        *reinterpret_cast<float4*>(&Xs[(tid >> 5) + 8 * v][4 * (tid & 31)]) =
            make_float4(xr[4 * v], xr[4 * v + 1], xr[4 * v + 2], xr[4 * v + 3]);
    } else {
#pragma unroll
      for (int u = 0; u < kXPer; ++u) {
        const int e = tid + kThreads * u;
        int kk, ii;
        if (kSlow) { kk = e / kBI; ii = e % kBI; }
        else       { kk = e % kBK; ii = e / kBK; }
        Xs[kk][ii] = xr[u];
      }
    }
    if (more) tile_rows(k0 + kBK, cur ^ 1);
    __syncthreads();
    if (more) load_x(cur ^ 1);  // the next tile's tensor values stream in during this tile
#pragma unroll 8
    for (int kk = 0; kk < kBK; ++kk) {
      float4 xv = *reinterpret_cast<const float4*>(&Xs[kk][ty * 4]);
      float4 wv = *reinterpret_cast<const float4*>(&Ws[kk][tx * 4]);
      float xa[4] = {xv.x, xv.y, xv.z, xv.w};
      float wa[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], wa[b], acc[a][b]);
    }
    __syncthreads();
  }

  float* o = out + (long long)blockIdx.y * out_chunk_stride;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    long long i = i0 + ty * 4 + a;
    if (i >= I) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int r = r0 + tx * 4 + b;
      if (r < R) o[i * R + r] = acc[a][b];
    }
  }
}

// out[e] = sum_{c < C} part[c * E + e] (deterministic: four interleaved partial
// sums over c = 0, 4, 8, ... / 1, 5, 9, ... combined in a fixed order).  The
// loads of eight chunks are issued before any is added; V = 4 sums four
// consecutive elements per thread with 16-byte loads (large E only).
template <int V>
__global__ void k_reduce_chunks(const float* __restrict__ part, long long E, int C,
                                float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  using VT = typename std::conditional<V == 4, float4, float>::type;
  const VT* pv = reinterpret_cast<const VT*>(part);
  VT* ov = reinterpret_cast<VT*>(out);
  const long long Ev = E / V;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < Ev;
       e += (long long)gridDim.x * blockDim.x) {
    float s[4][V];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < V; ++i) s[q][i] = 0.0f;
    int c = 0;
    for (; c + 8 <= C; c += 8) {
      VT v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = __ldg(pv + (long long)(c + q) * Ev + e);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float* f = reinterpret_cast<const float*>(&v[q]);
#pragma unroll
        for (int i = 0; i < V; ++i) s[q & 3][i] += f[i];
      }
    }
    for (; c + 4 <= C; c += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const VT v = __ldg(pv + (long long)(c + q) * Ev + e);
        const float* f = reinterpret_cast<const float*>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) s[q][i] += f[i];
      }
    }
    for (; c < C; ++c) {
      const VT v = __ldg(pv + (long long)c * Ev + e);
      const float* f = reinterpret_cast<const float*>(&v);
#pragma unroll
      for (int i = 0; i < V; ++i) s[0][i] += f[i];
    }
    VT r;
    float* rf = reinterpret_cast<float*>(&r);
#pragma unroll
    for (int i = 0; i < V; ++i) rf[i] = (s[0][i] + s[1][i]) + (s[2][i] + s[3][i]);
    ov[e] = r;
  }
}

// The sums of k_reduce_chunks<1> (chunk c into accumulator c mod 4, the chunks
// past the last multiple of four into accumulator 0, then (a0 + a1) + (a2 + a3),
// so the same bits) with one accumulator per lane of a quad: four times the
// threads, each with a quarter of the dependent loads.
__global__ void k_reduce_chunks_quad(const float* __restrict__ part, long long E, int C,
                                     float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 2;
  const int q = threadIdx.x & 3;
  const int C4 = C & ~3;
  float s = 0.0f;
  if (e < E) {
#pragma unroll 4
    for (int c = q; c < C4; c += 4) s += __ldg(part + (long long)c * E + e);
    if (q == 0)
      for (int c = C4; c < C; ++c) s += __ldg(part + (long long)c * E + e);
  }
  const float u = s + __shfl_down_sync(0xffffffffu, s, 1);  // q = 0: a0 + a1, q = 2: a2 + a3
  const float v = u + __shfl_down_sync(0xffffffffu, u, 2);  // q = 0: (a0 + a1) + (a2 + a3)
  if (q == 0 && e < E) out[e] = v;
}

// Multi-TTV leaf: out(i, r) = sum_k T[(i + I*k)*R + r] * KK(k, r).
// Threads cover consecutive flattened (i, r) positions (V per thread, V = 4
// when R % 4 == 0), so every k step reads one contiguous run of the node
// temporary; the k loop is unrolled to keep several loads in flight.
template <int V>
__global__ void __launch_bounds__(kThreads)
k_mttv_leaf(const float* __restrict__ T, long long I, long long K, KrpDesc KK, int R,
            long long kchunk, float* __restrict__ out, long long out_chunk_stride) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float smem[];
  float* Ws = smem;  // kBK x R
  __shared__ int offs[kBK][kMaxModes];
  const long long E = I * R;
  const long long e = ((long long)blockIdx.x * kThreads + threadIdx.x) * V;
  const int r = (int)(e % R);
  const long long kbeg = (long long)blockIdx.y * kchunk;
  const long long kend = min(K, kbeg + kchunk);
  float acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.0f;
  for (long long k0 = kbeg; k0 < kend; k0 += kBK) {
    if (threadIdx.x < kBK) {
      long long k = k0 + threadIdx.x;
      if (k < kend) decompose(KK, k, R, offs[threadIdx.x]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kBK * R; t += kThreads) {
      int kk = t / R, rr = t % R;
      Ws[t] = (k0 + kk < kend) ? krp_value(KK, offs[kk], rr) : 0.0f;
    }
    __syncthreads();
    if (e < E) {
      const int kn = (int)min((long long)kBK, kend - k0);
      const float* Tp = T + (I * k0) * R + e;
      if (V == 4) {
        // eight node rows in flight, then their products in k order
        int kk = 0;
        for (; kk + 8 <= kn; kk += 8) {
          float4 tv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            tv[q] = __ldg(reinterpret_cast<const float4*>(Tp + I * R * (kk + q)));
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 wv = *reinterpret_cast<const float4*>(Ws + (kk + q) * R + r);
            acc[0] = fmaf(tv[q].x, wv.x, acc[0]);
            acc[V > 1 ? 1 : 0] = fmaf(tv[q].y, wv.y, acc[V > 1 ? 1 : 0]);
            acc[V > 2 ? 2 : 0] = fmaf(tv[q].z, wv.z, acc[V > 2 ? 2 : 0]);
            acc[V > 3 ? 3 : 0] = fmaf(tv[q].w, wv.w, acc[V > 3 ? 3 : 0]);
          }
        }
#pragma unroll 4
        for (; kk < kn; ++kk) {
          const float4 tv = __ldg(reinterpret_cast<const float4*>(Tp + I * R * kk));
          const float4 wv = *reinterpret_cast<const float4*>(Ws + kk * R + r);
          acc[0] = fmaf(tv.x, wv.x, acc[0]);
          acc[V > 1 ? 1 : 0] = fmaf(tv.y, wv.y, acc[V > 1 ? 1 : 0]);
          acc[V > 2 ? 2 : 0] = fmaf(tv.z, wv.z, acc[V > 2 ? 2 : 0]);
          acc[V > 3 ? 3 : 0] = fmaf(tv.w, wv.w, acc[V > 3 ? 3 : 0]);
        }
      } else {
#pragma unroll 4
        for (int kk = 0; kk < kn; ++kk) acc[0] = fmaf(__ldg(Tp + I * R * kk), Ws[kk * R + r], acc[0]);
      }
    }
    __syncthreads();
  }
  if (e < E) {
    float* o = out + (long long)blockIdx.y * out_chunk_stride + e;
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = acc[v];
  }
}

// Multi-TTV to the child node: out(j, r) = sum_i T[(i + I*j)*R + r] * H(i, r).
// One CTA per j; thread (g, r-group) strides over i (V = 4 consecutive ranks
// per thread when R % 4 == 0); a fixed-order reduction over g.
template <int V>
__global__ void k_mttv_first(const float* __restrict__ T, long long I, const float* __restrict__ H,
                             int R, int G, float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float red[];  // G x R
  const long long j = blockIdx.x;
  const int RV = R / V;
  const int rv = threadIdx.x % RV;
  const int g = threadIdx.x / RV;
  if (g < G) {
    const float* Tj = T + I * j * R;
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.0f;
    if (V == 4) {
#pragma unroll 4
      for (long long i = g; i < I; i += G) {
        const float4 tv = __ldg(reinterpret_cast<const float4*>(Tj + i * R) + rv);
        const float4 hv = __ldg(reinterpret_cast<const float4*>(H + i * R) + rv);
        acc[0] = fmaf(tv.x, hv.x, acc[0]);
        acc[V > 1 ? 1 : 0] = fmaf(tv.y, hv.y, acc[V > 1 ? 1 : 0]);
        acc[V > 2 ? 2 : 0] = fmaf(tv.z, hv.z, acc[V > 2 ? 2 : 0]);
        acc[V > 3 ? 3 : 0] = fmaf(tv.w, hv.w, acc[V > 3 ? 3 : 0]);
      }
    } else {
#pragma unroll 4
      for (long long i = g; i < I; i += G)
        acc[0] = fmaf(__ldg(Tj + i * R + rv), __ldg(H + i * R + rv), acc[0]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) red[g * R + rv * V + v] = acc[v];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < R; t += blockDim.x) {
    float sum = 0.0f;
    for (int gg = 0; gg < G; ++gg) sum += red[gg * R + t];
    out[j * R + t] = sum;
  }
}

__device__ __forceinline__ double block_sum_double(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;  // valid in thread 0
}

__global__ void k_sumsq_partial(const void* __restrict__ Xv, int bf16, long long n,
                                double* __restrict__ partials, const int* flags) {
  if (flags && flags[0]) return;
  __shared__ double sh[32];
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!bf16) {
    const float* X = static_cast<const float*>(Xv);
    const long long n4 = n / 4;
    const float4* X4 = reinterpret_cast<const float4*>(X);
    for (long long t = t0; t < n4; t += stride) {
      float4 v = __ldg(X4 + t);
      float s = v.x * v.x;
      s = fmaf(v.y, v.y, s);
      s = fmaf(v.z, v.z, s);
      s = fmaf(v.w, v.w, s);
      acc += (double)s;
    }
    for (long long t = n4 * 4 + t0; t < n; t += stride) acc += (double)X[t] * X[t];
  } else {
    const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(Xv);
    for (long long t = t0; t < n; t += stride) {
      float v = __bfloat162float(X[t]);
      acc += (double)(v * v);
    }
  }
  double tot = block_sum_double(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* out,
                               const int* flags) {
  if (flags && flags[0]) return;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partials[i];
    out[0] = s;
  }
}

__global__ void k_to_bf16(const float* __restrict__ X, __nv_bfloat16* __restrict__ Y, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    Y[t] = __float2bfloat16_rn(X[t]);
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Split of the contraction across CTAs: enough CTAs for ~4 per SM, each
// chunk at least `min_chunk` contraction elements.
int choose_chunks(long long ctas_other, long long Ktot, int num_sms, long long min_chunk = 8LL * kBK) {
  long long target = 4LL * num_sms;
  if (ctas_other >= target) return 1;
  long long C = ceil_div(target, ctas_other);
  long long max_c = max(1LL, ceil_div(Ktot, min_chunk));
  return (int)min(C, max_c);
}

// Multi-TTV chunks: one contraction element is a whole I*R block of the node,
// so chunks of 8 elements already stream enough bytes.
constexpr long long kMttvMinChunk = 8;

}  // namespace

size_t simt_mttkrp_partials(int64_t L, int64_t I, int64_t Q, int R, int num_sms) {
  long long gx = ceil_div(I, kBI), gz = ceil_div(R, kRT);
  int C = choose_chunks(gx * gz, (long long)L * Q, num_sms);
  return C > 1 ? (size_t)C * I * R : 0;
}

cudaError_t launch_simt_mttkrp(const float* X, int64_t L, int64_t I, int64_t Q,
                               const KrpDesc& KL, const KrpDesc& KQ, int R, float* out,
                               float* partials, size_t part_cap, int num_sms,
                               cudaStream_t st) {
  long long Ktot = (long long)L * Q;
  long long gx = ceil_div(I, kBI), gz = ceil_div(R, kRT);
  int C = choose_chunks(gx * gz, Ktot, num_sms);
  long long kchunk = ceil_div(ceil_div(Ktot, C), kBK) * kBK;
  C = (int)ceil_div(Ktot, kchunk);
  float* dst = out;
  if (C > 1) {
    if ((size_t)C * I * R > part_cap || partials == nullptr) return cudaErrorInvalidValue;
    dst = partials;
  }
  dim3 grid((unsigned)gx, (unsigned)C, (unsigned)gz);
  cudaError_t e = launch_kernel(L == 1 ? k_simt_mttkrp<true> : k_simt_mttkrp<false>, grid,
                                dim3(kThreads), 0, st, X, (long long)L, (long long)I,
                                (long long)Q, KL, KQ, R, kchunk, dst, (long long)I * R);
  if (e != cudaSuccess || C == 1) return e;
  return launch_reduce_chunks(partials, (long long)I * R, C, out, num_sms, st);
}

// Same MTTKRP with the split-K chunk count capped so the partials fit in
// `part_cap` floats (used by the entry point that allocates nothing).
cudaError_t launch_simt_mttkrp_capped(const float* X, int64_t L, int64_t I, int64_t Q,
                                      const KrpDesc& KL, const KrpDesc& KQ, int R, float* out,
                                      float* partials, size_t part_cap, int num_sms,
                                      cudaStream_t st) {
  long long Ktot = (long long)L * Q;
  long long gx = ceil_div(I, kBI), gz = ceil_div(R, kRT);
  long long fit = (long long)(part_cap / ((size_t)I * R));
  int C = (int)max(1LL, min((long long)choose_chunks(gx * gz, Ktot, num_sms), fit));
  long long kchunk = ceil_div(ceil_div(Ktot, C), kBK) * kBK;
  C = (int)ceil_div(Ktot, kchunk);
  float* dst = out;
  if (C > 1) {
    if ((size_t)C * I * R > part_cap || partials == nullptr) return cudaErrorInvalidValue;
    dst = partials;
  }
  dim3 grid((unsigned)gx, (unsigned)C, (unsigned)gz);
  cudaError_t e = launch_kernel(L == 1 ? k_simt_mttkrp<true> : k_simt_mttkrp<false>, grid,
                                dim3(kThreads), 0, st, X, (long long)L, (long long)I,
                                (long long)Q, KL, KQ, R, kchunk, dst, (long long)I * R);
  if (e != cudaSuccess || C == 1) return e;
  return launch_reduce_chunks(partials, (long long)I * R, C, out, num_sms, st);
}

cudaError_t launch_reduce_chunks(const float* part, int64_t E, int C, float* out, int num_sms,
                                 cudaStream_t st) {
  // four elements per thread only when that still leaves a full wave of CTAs:
  // the reduction is bound by how many SMs pull the partials
  const bool v4 = E % 4 == 0 && E / 4 >= (int64_t)num_sms * 8 * 256 &&
                  reinterpret_cast<uintptr_t>(part) % 16 == 0 &&
                  reinterpret_cast<uintptr_t>(out) % 16 == 0;
  if (!v4)  // small outputs: a quad of threads per output (same sums)
    return launch_kernel(k_reduce_chunks_quad, dim3((unsigned)ceil_div(4 * (long long)E, 256)),
                         dim3(256), 0, st, part, (long long)E, C, out);
  const long long Ev = E / 4;
  int blocks = (int)min(ceil_div(Ev, 256), (long long)num_sms * 8);
  if (blocks < 1) blocks = 1;
  return launch_kernel(k_reduce_chunks<4>, dim3(blocks), dim3(256), 0, st, part, (long long)E, C,
                       out);
}

size_t mttv_leaf_partials(int64_t I, int64_t K, int R, int num_sms) {
  const int V = (R % 4 == 0) ? 4 : 1;
  long long gx = ceil_div(ceil_div((long long)I * R, V), kThreads);
  int C = choose_chunks(gx, K, num_sms, kMttvMinChunk);
  return C > 1 ? (size_t)C * I * R : 0;
}

cudaError_t launch_mttv_leaf(const float* T, int64_t I, int64_t K, const KrpDesc& KK, int R,
                             float* out, float* partials, size_t part_cap, int num_sms,
                             cudaStream_t st) {
  const int V = (R % 4 == 0) ? 4 : 1;
  long long E = (long long)I * R;
  long long gx = ceil_div(ceil_div(E, V), kThreads);
  int C = choose_chunks(gx, K, num_sms, kMttvMinChunk);
  long long kchunk = ceil_div(K, C);
  C = (int)ceil_div(K, kchunk);
  float* dst = out;
  if (C > 1) {
    if ((size_t)C * E > part_cap || partials == nullptr) return cudaErrorInvalidValue;
    dst = partials;
  }
  size_t smem = (size_t)kBK * R * sizeof(float);
  cudaError_t e = launch_kernel(V == 4 ? k_mttv_leaf<4> : k_mttv_leaf<1>,
                                dim3((unsigned)gx, (unsigned)C), dim3(kThreads), smem, st, T,
                                (long long)I, (long long)K, KK, R, kchunk, dst, E);
  if (e != cudaSuccess || C == 1) return e;
  return launch_reduce_chunks(partials, E, C, out, num_sms, st);
}

cudaError_t launch_mttv_first(const float* T, int64_t I, int64_t J, const float* H, int R,
                              float* out, cudaStream_t st) {
  const int V = (R % 4 == 0) ? 4 : 1;
  const int RV = R / V;
  int G = std::max(1, 256 / RV);
  if (G > I) G = (int)I;
  const int threads = G * RV;
  size_t smem = (size_t)G * R * sizeof(float);
  return launch_kernel(V == 4 ? k_mttv_first<4> : k_mttv_first<1>, dim3((unsigned)J),
                       dim3(threads), smem, st, T, (long long)I, H, R, G, out);
}

cudaError_t launch_sumsq(const void* X, int bf16, int64_t n, double* partials, int nparts,
                         double* out, const int* flags, cudaStream_t st) {
  k_sumsq_partial<<<nparts, 256, 0, st>>>(X, bf16, n, partials, flags);
  k_sum_partials<<<1, 32, 0, st>>>(partials, nparts, out, flags);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* X, uint16_t* Y, int64_t n, cudaStream_t st) {
  int blocks = (int)min(ceil_div(n, 256), 152LL * 16);
  if (blocks < 1) blocks = 1;
  k_to_bf16<<<blocks, 256, 0, st>>>(X, reinterpret_cast<__nv_bfloat16*>(Y), n);
  return cudaGetLastError();
}

}  // namespace nncp
