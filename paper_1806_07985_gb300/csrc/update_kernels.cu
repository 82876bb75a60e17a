// Factor-update kernels of one BCD inner iteration (Alg. 1 / Alg. 3): the
// HALS sweep (Sec. II-B) on W = H_n diag(lambda), row-parallel; W^T W and
// <M, W>; lambda = column norms, G_n = H_n^T H_n, H_n = W diag(lambda)^-1,
// the fit from the Sec. IV-B identity at n = N, and S = Hadamard of the other
// Grams for the next mode.  Three forms by mode length:
//   k_update_cluster  I_n <= 1024: one launch on a thread-block cluster that
//                     exchanges its partials through distributed shared memory;
//   k_update_multi    I_n <= 16384: CTAs of 128 rows, the last CTA (atomic
//                     ticket) finishes;
//   k_hals_gram + k_finalize  otherwise (and for the solve's initialisation).
// The factors, the HALS arithmetic, the Grams and S are float32.  The sums the
// fit needs to more than float32 precision (<M, W> and lambda^T (S * G) lambda)
// are float-float (unevaluated hi + lo pairs added with the error-free TwoSum),
// and only the fit's last few scalar steps are float64: float64 issues about
// 60x slower than float32 on this GPU, so it is kept off every per-element path.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "nncp_internal.cuh"

namespace nncp {

namespace {

constexpr int kRowsPerBlock = 64;
constexpr int kHalsThreads = 256;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1 / sqrt(g) and sqrt(g) in float64 for a float32 g: a float32 estimate
// refined by two steps of Newton's iteration for the reciprocal square root,
// r <- r (3 - g r^2) / 2, each of which squares the relative error (~2^-22
// -> ~2^-43 -> below float64 rounding).  A few dependent multiply-adds
// instead of a float64 square root and a float64 division, which on this
// GPU's float64 pipe cost about a microsecond per mode update.  g = 0 gives
// 0 and 0; a non-finite g takes the plain functions, so NaN propagates.
__device__ __forceinline__ void rsqrt_sqrt_f64(float g32, double* rinv, double* root) {
  if (g32 > 0.0f && g32 < INFINITY) {
    const double g = g32;
    double r = (double)rsqrtf(g32);
    r = r * (1.5 - 0.5 * g * r * r);
    r = r * (1.5 - 0.5 * g * r * r);
    *rinv = r;
    *root = g * r;
  } else {
    *root = sqrt((double)g32);
    *rinv = g32 > 0.0f ? 1.0 / *root : 0.0;
  }
}

// Butterfly sum: every lane ends with the same bits (each step adds the same
// two values in the same order on both partners).
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One HALS sweep per row, one warp per row; lane holds columns lane + 32*j.
// Then the block's partial W^T W (float32 over <= 64 rows, stored as double)
// and partial <M, W>.
__global__ void __launch_bounds__(kHalsThreads)
k_hals_gram(float* __restrict__ H, const float* __restrict__ M, long long In, int R,
            const float* __restrict__ S, const double* __restrict__ lam,
            double* __restrict__ gram_part, const int* __restrict__ flags, int do_hals) {
  // do_hals: 1 = HALS sweep on W = H diag(lam), then the partials; 0 = the
  // partials of W = H alone (no <M, W>); 2 = W given in H (the block
  // principal pivoting update): the partials and <M, W>, no sweep
  pdl_wait();
  pdl_trigger();
  if (flags && flags[0]) return;
  extern __shared__ float sm[];
  float* Ss = sm;                        // R x R
  float* Ws = Ss + R * R;                // kRowsPerBlock x (R + 1)
  __shared__ double wbeta[kHalsThreads / 32];
  const int RP = R + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long row0 = (long long)blockIdx.x * kRowsPerBlock;
  const int nrows = (int)min((long long)kRowsPerBlock, In - row0);

  if (do_hals)
    for (int t = threadIdx.x; t < R * R; t += blockDim.x) Ss[t] = S[t];
  __syncthreads();

  double beta_acc = 0.0;
  for (int rr = warp; rr < nrows; rr += kHalsThreads / 32) {
    const long long i = row0 + rr;
    float w[4], m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = lane + 32 * j;
      w[j] = 0.0f;
      m[j] = 0.0f;
      if (c < R) {
        w[j] = H[i * R + c];
        if (do_hals) {
          if (do_hals == 1) w[j] = w[j] * (float)lam[c];
          m[j] = M[i * R + c];
        }
      }
    }
    if (do_hals == 1) {
      for (int r = 0; r < R; ++r) {
        const float srr = Ss[r * R + r];
        if (srr == 0.0f) continue;  // warp-uniform
        float part = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int c = lane + 32 * j;
          if (c < R) part = fmaf(w[j], Ss[c * R + r], part);
        }
        const float dot = warp_sum(part);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (lane + 32 * j == r) w[j] = fmaxf(0.0f, w[j] + (m[j] - dot) / srr);
      }
    }
    if (do_hals) {
      float bp = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) bp = fmaf(m[j], w[j], bp);
      beta_acc += (double)warp_sum(bp);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = lane + 32 * j;
      if (c < R) {
        if (do_hals == 1) H[i * R + c] = w[j];
        Ws[rr * RP + c] = w[j];
      }
    }
  }
  if (lane == 0) wbeta[warp] = beta_acc;
  __syncthreads();
  double* gp = gram_part + (long long)blockIdx.x * (R * R + 1);
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    const int a = t / R, b = t % R;
    float s = 0.0f;
    for (int rr = 0; rr < nrows; ++rr) s = fmaf(Ws[rr * RP + a], Ws[rr * RP + b], s);
    gp[t] = (double)s;
  }
  if (threadIdx.x == 0) {
    double bsum = 0.0;
    for (int w = 0; w < kHalsThreads / 32; ++w) bsum += wbeta[w];
    gp[R * R] = bsum;
  }
}

// fit = 1 - eps, eps^2 = (alpha - 2 beta + gamma) / alpha clamped at 0 (Sec. IV-B);
// appends to the fit history and sets the stop flag on |delta fit| < tol.
__device__ void record_fit(SolveState st, double beta, double gamma) {
  const double alpha = st.scalars[0];
  const double eps = sqrt(fmax(0.0, alpha - 2.0 * beta + gamma) / alpha);
  const double fit = 1.0 - eps;
  st.scalars[1] = beta;
  st.scalars[2] = gamma;
  st.scalars[3] = eps;
  const int it = st.flags[2];
  const double prev = st.scalars[5];
  if (it < kFitCapacity) st.fits[it] = fit;
  st.flags[2] = it + 1;
  st.scalars[5] = fit;
  const double tol = st.scalars[4];
  if (!isfinite(fit)) {
    st.flags[3] = 1;
    st.flags[0] = 1;
  } else if (it >= 1 && fabs(fit - prev) < tol) {
    st.flags[0] = 1;
  }
}


// Single CTA (1024 threads).  Shared: GW (R*R doubles) + c (R doubles).
__global__ void __launch_bounds__(1024)
k_finalize(float* __restrict__ H, long long In, int R, int N, int n, int next_mode,
           int nblocks, int is_last, int init, SolveState st, float* __restrict__ U) {
  pdl_wait();
  pdl_trigger();
  if (st.flags[0]) return;
  extern __shared__ double dsm[];
  double* GW = dsm;          // R x R
  double* c = GW + R * R;    // R
  __shared__ double red[32];
  const int R2 = R * R;
  const int tid = threadIdx.x;

  for (int t = tid; t < R2; t += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += st.gram_part[(long long)b * (R2 + 1) + t];
    GW[t] = s;
  }
  __syncthreads();
  for (int r = tid; r < R; r += blockDim.x) {
    double v = sqrt(GW[r * R + r]);
    c[r] = v;
    if (init) st.lam[r] *= v;
    else st.lam[r] = v;
  }
  __syncthreads();
  __shared__ double cinv[kMaxRank];
  for (int r = tid; r < R; r += blockDim.x) cinv[r] = c[r] > 0.0 ? 1.0 / c[r] : 0.0;
  __syncthreads();
  double* Gn = st.G + (long long)n * R2;
  for (int t = tid; t < R2; t += blockDim.x) {
    const int a = t / R, b = t % R;
    Gn[t] = GW[t] * cinv[a] * cinv[b];
  }
  for (long long t = tid; t < In * R; t += blockDim.x) {
    const int r = (int)(t % R);
    H[t] = c[r] > 0.0 ? H[t] / (float)c[r] : 0.0f;
    if (U) U[t] = c[r] > 0.0 ? U[t] / (float)c[r] : 0.0f;  // ADMM dual, same frame as H
  }
  if (is_last) {
    // gamma = lam^T (S * G_N) lam = sum_ab S_ab (W^T W)_ab
    const double* Sn = st.S + (long long)n * R2;
    double g = 0.0;
    for (int t = tid; t < R2; t += blockDim.x) g += Sn[t] * GW[t];
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if ((tid & 31) == 0) red[tid >> 5] = g;
    __syncthreads();
    if (tid == 0) {
      double gamma = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gamma += red[w];
      double beta = 0.0;
      for (int b = 0; b < nblocks; ++b) beta += st.gram_part[(long long)b * (R2 + 1) + R2];
      record_fit(st, beta, gamma);
    }
  }
  __syncthreads();
  // S for the next mode: Hadamard of every Gram but next_mode's (float64)
  if (next_mode >= 0) {
    for (int t = tid; t < R2; t += blockDim.x) {
      double s = 1.0;
      for (int k = 0; k < N; ++k)
        if (k != next_mode) s *= st.G[(long long)k * R2 + t];
      st.S[(long long)next_mode * R2 + t] = s;
      st.S32[t] = (float)s;
    }
  }
}

__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// float-float: the unevaluated sum hi + lo of two float32 values.  ff_add is
// the TwoSum-based addition (Knuth): the rounding error of hi_a + hi_b is
// recovered exactly and carried in lo, so a sum of float32 terms keeps about
// 44 bits.  Its result does not depend on the operand order, so butterfly
// reductions leave the same bits in every lane.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float t = e + (a.lo + b.lo);
  const float hi = s + t;
  return {hi, t - (hi - s)};
}

__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff_add(v, FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

// Mode update spread over CTAs of MultiCfg<RMAX>::ROWS rows (I_n <= kMultiMaxRows, R <= 64):
//   every CTA stages its rows of H and M in shared memory (coalesced), runs the
//   HALS sweep (Sec. II-B) with one thread per row, and forms its partial W^T W
//   and <M, W>.  A single CTA finishes on its own from shared memory;
//   otherwise every CTA writes W and its partials and the last CTA to finish
//   (atomic ticket) sums the partials in CTA order and scales H by 1 / lambda.
//   The finishing CTA forms lambda, G_n, the fit at n = N and S for the next
//   mode.  Results do not depend on arrival order.
constexpr int kMultiThreads = 512;
constexpr int kGpreDoubles = 3072;  // other modes' Grams staged for the next S (24 KB)
constexpr int kMultiMaxRows = 16384;

template <int RMAX>
struct MultiCfg {
  static constexpr int T = kMultiThreads;
  // rows per CTA, one HALS thread each (a mode of up to ROWS rows is updated
  // by one CTA without a global round trip)
  static constexpr int ROWS = 128;
  static constexpr int RP = RMAX + 4;        // padded row stride (16-byte multiple) in shared memory
  static constexpr int NB = RMAX / 4;
  static constexpr int GROUPS = T / (NB * NB);  // Gram row groups
};

int multi_rows(int R) { return R <= 32 ? MultiCfg<32>::ROWS : MultiCfg<64>::ROWS; }  // all 128

template <int RMAX>
__global__ void __launch_bounds__(kMultiThreads, 1)
k_update_multi(float* __restrict__ H, const float* __restrict__ M, int In, int R, int N, int n,
               int next_mode, int is_last, SolveState st, float* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  if (st.flags[0]) return;
  using C = MultiCfg<RMAX>;
  constexpr int T = C::T, ROWS = C::ROWS, RP = C::RP, GROUPS = C::GROUPS;
  constexpr int EPT = (RMAX * RMAX + T - 1) / T;  // R x R elements per thread
  extern __shared__ __align__(16) float usm[];
  float* St = usm;                      // RMAX x RMAX, St[r][c] = S[c][r], zero padded
  float* Hs = St + RMAX * RMAX;         // ROWS x RP: H, then W
  float* Ms = Hs + ROWS * RP;           // ROWS x RP
  float* gpart = Ms + ROWS * RP;        // GROUPS x R x R, then W^T W
  // R x R: the new G_n (float64; the float offsets above are multiples of 4)
  double* Gn = reinterpret_cast<double*>(gpart + GROUPS * RMAX * RMAX);
  double* Gpre = Gn + RMAX * RMAX;      // the other modes' Grams for the next S
  __shared__ __align__(16) float lamf[RMAX];
  __shared__ double linv[RMAX];
  __shared__ float sinv[RMAX];
  __shared__ FF red[T / 32];
  __shared__ double redd[T / 32];
  __shared__ FF beta_sh;
  __shared__ double scal_sh[3];  // alpha, previous fit, tol
  __shared__ int last_sh, it_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R2 = R * R;
  const int row0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, In - row0);
  const bool single = gridDim.x == 1;

  // ---- staging: every load the update needs is issued here, in one batch
#pragma unroll
  for (int e = tid; e < RMAX * RMAX; e += T) {
    const int r = e / RMAX, c = e % RMAX;
    St[e] = (r < R && c < R) ? st.S32[c * R + r] : 0.0f;
  }
  for (int r = tid; r < RMAX; r += T) {
    lamf[r] = r < R ? (float)st.lam[r] : 0.0f;
    const float srr = r < R ? st.S32[r * R + r] : 0.0f;
    sinv[r] = srr != 0.0f ? 1.0f / srr : 0.0f;
  }
  const float* Hg = H + (long long)row0 * R;
  const float* Mg = M + (long long)row0 * R;
  if ((R & 3) == 0) {
    // 16-byte asynchronous copies straight into the padded rows (R % 4 == 0:
    // every source row and destination row starts on a 16-byte boundary)
    const int n4 = nrows * R / 4;
    for (int v = tid; v < n4; v += T) {
      const int rr = 4 * v / R, c = 4 * v - rr * R;
      cp_async16(Hs + rr * RP + c, Hg + 4 * v);
      cp_async16(Ms + rr * RP + c, Mg + 4 * v);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  } else {
#pragma unroll 4
    for (int e = tid; e < nrows * R; e += T) {
      const int rr = e / R, c = e % R;
      Hs[rr * RP + c] = Hg[e];
      Ms[rr * RP + c] = Mg[e];
    }
  }
  // the other modes' Grams for the next S, when they fit (slots in mode order)
  const int ng = N - (next_mode == n ? 1 : 2);
  const bool gpre = ng > 0 && ng * R2 <= kGpreDoubles;
  if (gpre) {
    for (int k = 0, slot = 0; k < N; ++k) {
      if (k == n || k == next_mode) continue;
      for (int e = tid; e < R2; e += T) Gpre[slot * R2 + e] = st.G[(long long)k * R2 + e];
      ++slot;
    }
  }
  if (tid == 0) {
    it_sh = st.flags[2];
    scal_sh[0] = st.scalars[0];
    scal_sh[1] = st.scalars[5];
    scal_sh[2] = st.scalars[4];
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();

  // ---- HALS sweep (Sec. II-B): thread = row, columns in order.  Up to 32
  // columns the row lives in registers (fully unrolled sweep); at 64 that
  // straight-line code is too long to fetch once per warp, so the row is
  // updated in place in its shared-memory row by a rolled column loop.  Both
  // form each dot product in the same order, so they give the same bits.
  FF bp{0.0f, 0.0f};
  if (tid < nrows) {
    float b = 0.0f;
    if constexpr (RMAX <= 32) {
      float w[RMAX];
#pragma unroll
      for (int c = 0; c < RMAX; ++c) w[c] = c < R ? Hs[tid * RP + c] * lamf[c] : 0.0f;
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        const float si = sinv[r];
        const float mr = Ms[tid * RP + r];
        const float4* col = reinterpret_cast<const float4*>(St + r * RMAX);
        float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
#pragma unroll
        for (int c = 0; c < RMAX; c += 4) {
          const float4 sv = col[c >> 2];
          d0 = fmaf(w[c], sv.x, d0);
          d1 = fmaf(w[c + 1], sv.y, d1);
          d2 = fmaf(w[c + 2], sv.z, d2);
          d3 = fmaf(w[c + 3], sv.w, d3);
        }
        const float dot = (d0 + d1) + (d2 + d3);
        const float upd = fmaxf(0.0f, w[r] + (mr - dot) * si);
        w[r] = si != 0.0f ? upd : w[r];  // S_rr = 0: column left as it is
      }
#pragma unroll
      for (int c = 0; c < RMAX; ++c) {
        if (c < R) {
          b = fmaf(Ms[tid * RP + c], w[c], b);
          Hs[tid * RP + c] = w[c];
        }
      }
    } else {
      float* wrow = Hs + tid * RP;
#pragma unroll
      for (int c = 0; c < RMAX; ++c) wrow[c] = c < R ? wrow[c] * lamf[c] : 0.0f;
      const float4* wv = reinterpret_cast<const float4*>(wrow);
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const float si = sinv[r];
        const float mr = Ms[tid * RP + r];
        const float4* col = reinterpret_cast<const float4*>(St + r * RMAX);
        float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
#pragma unroll
        for (int c = 0; c < RMAX / 4; ++c) {
          const float4 sv = col[c];
          const float4 w4 = wv[c];
          d0 = fmaf(w4.x, sv.x, d0);
          d1 = fmaf(w4.y, sv.y, d1);
          d2 = fmaf(w4.z, sv.z, d2);
          d3 = fmaf(w4.w, sv.w, d3);
        }
        const float dot = (d0 + d1) + (d2 + d3);
        const float wr = wrow[r];
        const float upd = fmaxf(0.0f, wr + (mr - dot) * si);
        wrow[r] = si != 0.0f ? upd : wr;
      }
      for (int c = 0; c < R; ++c) b = fmaf(Ms[tid * RP + c], wrow[c], b);
    }
    bp.hi = b;
  }
  // <M, W> of this CTA: float-float over the rows (warp, then warps in order)
  if (warp * 32 < nrows) bp = ff_warp_sum(bp);
  if (lane == 0) red[warp] = bp;
  __syncthreads();
  if (tid == 0) {
    FF s{0.0f, 0.0f};
    for (int k = 0; k < T / 32; ++k) s = ff_add(s, red[k]);
    beta_sh = s;
  }
  if (!single) {
    float* Hw = H + (long long)row0 * R;
    for (int e = tid; e < nrows * R; e += T) Hw[e] = Hs[(e / R) * RP + e % R];
  }

  // ---- partial W^T W: thread = (4x4 tile, row group), register tiles
  const int nb4 = (R + 3) / 4;
  const int tiles = nb4 * nb4;
  const int groups = min(GROUPS, max(1, T / tiles));
  if (tid < tiles * groups) {
    const int tile = tid % tiles, g = tid / tiles;
    const int a0 = (tile / nb4) * 4, b0 = (tile % nb4) * 4;
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
    for (int rr = g; rr < nrows; rr += groups) {
      const float4 qa = *reinterpret_cast<const float4*>(Hs + rr * RP + a0);
      const float4 qb = *reinterpret_cast<const float4*>(Hs + rr * RP + b0);
      const float va[4] = {qa.x, qa.y, qa.z, qa.w};
      const float vb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(va[x], vb[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (a0 + x < R && b0 + y < R) gpart[(g * R + a0 + x) * R + b0 + y] = acc[x][y];
  }
  __syncthreads();
  // W^T W summed over the row groups (group order)
  float gsum[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * T;
    gsum[q] = 0.0f;
    if (e < R2)
      for (int g = 0; g < groups; ++g) gsum[q] += gpart[g * R2 + e];
  }
  float* GW = gpart;  // R x R, after the group sums are read
  if (single) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * T;
      if (e < R2) GW[e] = gsum[q];
    }
  } else {
    float* pb = part + (long long)blockIdx.x * (R2 + 2);
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * T;
      if (e < R2) pb[e] = gsum[q];
    }
    if (tid == 0) {
      pb[R2] = beta_sh.hi;
      pb[R2 + 1] = beta_sh.lo;
    }
    // ---- the last CTA finishes the update
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int ticket = atomicAdd(&st.flags[8], 1);
      last_sh = ticket == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
    const int nbk = gridDim.x;
#pragma unroll 4
    for (int e = tid; e < R2; e += T) {
      float v[8];
      float sum = 0.0f;
      int b = 0;
      for (; b + 8 <= nbk; b += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = part[(long long)(b + q) * (R2 + 2) + e];
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += v[q];
      }
      for (; b < nbk; ++b) sum += part[(long long)b * (R2 + 2) + e];
      GW[e] = sum;
    }
    if (tid == 0) {
      FF s{0.0f, 0.0f};
      for (int k = 0; k < nbk; ++k)
        s = ff_add(s, FF{part[(long long)k * (R2 + 2) + R2], part[(long long)k * (R2 + 2) + R2 + 1]});
      beta_sh = s;
      st.flags[8] = 0;  // ticket reset for the next launch
    }
  }
  __syncthreads();
  // lambda = column norms of W in float64; from here on lamf holds 1 / lambda
  // (float32, for the row scaling) and linv the float64 reciprocal
  for (int r = tid; r < R; r += T) {
    double l, li;
    rsqrt_sqrt_f64(GW[r * R + r], &li, &l);
    st.lam[r] = l;
    linv[r] = li;
    lamf[r] = (float)li;
  }
  __syncthreads();
  double* Gng = st.G + (long long)n * R2;
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * T;
    if (e < R2) {
      const double v = (double)GW[e] * linv[e / R] * linv[e % R];
      Gn[e] = v;
      Gng[e] = v;
    }
  }
  // H = W / lambda (multiplication by the float32 reciprocal)
  if (single && (R & 3) == 0) {
    const float4* l4 = reinterpret_cast<const float4*>(lamf);
    for (int v = tid; v < nrows * R / 4; v += T) {
      const int e = 4 * v, rr = e / R, c = e - rr * R;
      const float4 w = *reinterpret_cast<const float4*>(Hs + rr * RP + c);
      const float4 l = l4[c >> 2];
      reinterpret_cast<float4*>(H)[v] = make_float4(w.x * l.x, w.y * l.y, w.z * l.z, w.w * l.w);
    }
  } else if (single) {
    for (int e = tid; e < nrows * R; e += T) H[e] = Hs[(e / R) * RP + e % R] * lamf[e % R];
  } else if ((R & 3) == 0) {
    const int tot4 = In * R / 4;
    const float4* l4 = reinterpret_cast<const float4*>(lamf);
    float4* H4 = reinterpret_cast<float4*>(H);
    for (int v0 = tid; v0 < tot4; v0 += 8 * T) {
      float4 w[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int v = v0 + q * T;
        if (v < tot4) w[q] = H4[v];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int v = v0 + q * T;
        if (v < tot4) {
          const float4 l = l4[(4 * v % R) >> 2];
          H4[v] = make_float4(w[q].x * l.x, w[q].y * l.y, w[q].z * l.z, w[q].w * l.w);
        }
      }
    }
  } else {
    const int tot = In * R;  // <= kMultiMaxRows * 64: 32-bit index arithmetic
    for (int e0 = tid; e0 < tot; e0 += 16 * T) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = e0 + q * T;
        v[q] = e < tot ? H[e] : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = e0 + q * T;
        if (e < tot) H[e] = v[q] * lamf[e % R];
      }
    }
  }
  if (is_last) {
    // gamma = lambda^T (S * G_N) lambda = sum_ab S_ab (W^T W)_ab (Sec. IV-B),
    // float64 (S of this mode, written by an earlier update) over the
    // thread's terms, the warp, then the warps in order
    const double* Sn = st.S + (long long)n * R2;
    double g = 0.0;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * T;
      if (e < R2) g = fma(Sn[e], (double)GW[e], g);
    }
    g = warp_sum_d(g);
    __syncthreads();
    if (lane == 0) redd[warp] = g;
    __syncthreads();
    if (tid == 0) {
      double gamma = 0.0;
      for (int k = 0; k < T / 32; ++k) gamma += redd[k];
      const double beta = (double)beta_sh.hi + (double)beta_sh.lo;
      const double alpha = scal_sh[0], prev = scal_sh[1], tol = scal_sh[2];
      const double eps = sqrt(fmax(0.0, alpha - 2.0 * beta + gamma) / alpha);
      const double fit = 1.0 - eps;
      const int it = it_sh;
      st.scalars[1] = beta;
      st.scalars[2] = gamma;
      st.scalars[3] = eps;
      st.scalars[5] = fit;
      if (it < kFitCapacity) st.fits[it] = fit;
      st.flags[2] = it + 1;
      if (!isfinite(fit)) {
        st.flags[3] = 1;
        st.flags[0] = 1;
      } else if (it >= 1 && fabs(fit - prev) < tol) {
        st.flags[0] = 1;
      }
    }
  }
  __syncthreads();
  // S for the next mode: Hadamard of every Gram but next_mode's, in mode order
  // (mode n's is the new one)
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * T;
    if (e < R2) {
      double s = 1.0;
      for (int k = 0, slot = 0; k < N; ++k) {
        if (k == next_mode) continue;
        if (k == n) {
          s *= Gn[e];
        } else {
          s *= gpre ? Gpre[slot * R2 + e] : st.G[(long long)k * R2 + e];
          ++slot;
        }
      }
      st.S[(long long)next_mode * R2 + e] = s;
      st.S32[e] = (float)s;
    }
  }
}

template <int RMAX>
size_t multi_smem() {
  using C = MultiCfg<RMAX>;
  return (size_t)(RMAX * RMAX + 2 * C::ROWS * C::RP + C::GROUPS * RMAX * RMAX) * sizeof(float) +
         (size_t)(RMAX * RMAX + kGpreDoubles) * sizeof(double);
}

// ---- thread-block cluster helpers (distributed shared memory) ---------------
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// address of `p` (this CTA's shared memory) in the shared memory of CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(const void* p, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_cluster(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ float4 ld_cluster4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}
// every thread of every CTA of the cluster arrives; wait returns once all have
// (release / acquire: shared-memory writes before the arrive are visible after the wait)
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Mode update on one thread-block cluster (I_n <= kClusterMaxRows, R <= 64):
// CTA k of the cluster owns rows [k * rows, (k + 1) * rows).  Every CTA stages
// its rows of H and M, runs the HALS sweep (Sec. II-B) with one thread per row,
// and forms its partial W^T W and <M, W> in its own shared memory.  After a
// cluster barrier each CTA reads every CTA's partials through distributed
// shared memory, in CTA order, so all of them hold the same W^T W bits, forms
// lambda and writes its own rows of H = W / lambda and its slice of G_n and of
// S for the next mode; CTA 0 also writes lambda and the fit at n = N.  No global round trip
// between the phases, no atomics; the hardware schedules the cluster's CTAs
// together, so the barrier needs no co-residency assumption.
//
// Launched in the iteration graph with programmatic serialization, the kernel
// may start while its predecessor runs.  Everything it reads except M (H_n, S,
// G, lambda, the scalars and flags) is written two or more kernels earlier and
// never by the kernel just before an update (a partial MTTKRP, a multi-TTV or a
// reduction), and every kernel of the iteration lets its successor start only
// after its own pdl_wait(): those loads are issued before pdl_wait(), M after.
// With sweep = 0 the kernel just before wrote W into H (an exact NLS solve of
// the rows), so H is staged after pdl_wait() as well and taken as W as it is.
constexpr int kClusterThreads = 256;
constexpr int kClusterMax = 8;      // portable cluster size
constexpr int kClusterRowsMax = 128;
constexpr int kClusterMaxRows = kClusterMax * kClusterRowsMax;

template <int RMAX>
struct ClusterCfg {
  static constexpr int T = kClusterThreads;
  static constexpr int RP = RMAX + 4;   // padded row stride (16-byte multiple)
  static constexpr int NB = RMAX / 4;
  static constexpr int GROUPS = T / (NB * NB) > 0 ? T / (NB * NB) : 1;  // Gram row groups
};

// rows per CTA: I_n spread over at most kClusterMax CTAs, a multiple of 32
int cluster_rows(int64_t In) {
  int r = (int)((In + kClusterMax - 1) / kClusterMax);
  r = (r + 31) / 32 * 32;
  return std::max(32, r);
}

template <int RMAX>
__global__ void __launch_bounds__(kClusterThreads, 1)
k_update_cluster(float* __restrict__ H, const float* __restrict__ M, int In, int R, int N, int n,
                 int next_mode, int is_last, int rows, int sweep, SolveState st,
                 float* __restrict__ U) {
  using C = ClusterCfg<RMAX>;
  constexpr int T = C::T, RP = C::RP, GROUPS = C::GROUPS;
  extern __shared__ __align__(16) float csm[];
  // Srot[j][c] = S[(4 floor(j / 4) + c) mod RMAX][j], zero outside R x R: row j
  // holds column j of S in the rotated order in which the HALS sweep keeps W
  float* Srot = csm;
  float* Hs = Srot + RMAX * RMAX;              // rows x RP: H, then W
  float* Ms = Hs + kClusterRowsMax * RP;       // rows x RP
  float* gpart = Ms + kClusterRowsMax * RP;    // GROUPS x R x R
  float* Gown = gpart + GROUPS * RMAX * RMAX;  // this CTA's W^T W (read by the cluster)
  float* GW = Gown + RMAX * RMAX;              // the cluster's W^T W
  // float64 from here (the float offsets above are multiples of 4)
  double* Gpre = reinterpret_cast<double*>(GW + RMAX * RMAX);  // the other modes' Grams, this CTA's slice
  double* Sd = Gpre + kGpreDoubles;            // S of this mode (float64), for gamma
  __shared__ __align__(16) float lamf[RMAX];
  __shared__ __align__(8) double lamd[RMAX];
  __shared__ float sinv[RMAX];
  __shared__ FF red[T / 32];
  __shared__ double redd[T / 32];
  __shared__ FF beta_own, beta_sh;
  __shared__ __align__(8) double scal_sh[4];  // alpha, tol, previous fit
  __shared__ int flag_sh[2];                  // stop flag, iteration count
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned rank = cluster_rank(), nrank = cluster_size();
  const bool lead = rank == 0;
  const int R2 = R * R;
  const int row0 = (int)rank * rows;
  const int nrows = min(rows, In - row0);
  const bool vec = (R & 3) == 0;

  // ---- staging: asynchronous copies, one round trip.  First everything an
  // earlier kernel than the predecessor wrote ...
#pragma unroll 1
  for (int e = tid; e < RMAX * RMAX; e += T) {
    const int j = e / RMAX, c = e % RMAX;
    const int a = ((j & ~3) + c) & (RMAX - 1);
    if (j < R && a < R) cp_async4(Srot + e, st.S32 + a * R + j);
    else Srot[e] = 0.0f;
  }
  if (lead && is_last) {
#pragma unroll 1
    for (int e = tid; e < R2; e += T) cp_async8(Sd + e, st.S + (long long)n * R2 + e);
  }
  for (int r = tid; r < R; r += T) cp_async8(lamd + r, st.lam + r);
  const float* Hg = H + (long long)row0 * R;
  const float* Mg = M + (long long)row0 * R;
  // rows x R from global into a padded tile
  auto stage_rows = [&](float* dst, const float* src) {
    if (vec) {
#pragma unroll 1
      for (int v = tid; v < nrows * R / 4; v += T) {
        const int rr = 4 * v / R, c = 4 * v - rr * R;
        cp_async16(dst + rr * RP + c, src + 4 * v);
      }
    } else {
#pragma unroll 1
      for (int e = tid; e < nrows * R; e += T) cp_async4(dst + (e / R) * RP + e % R, src + e);
    }
  };
  // without the sweep H holds W, which the predecessor writes
  if (sweep) stage_rows(Hs, Hg);
  // this CTA's slice [s0, s0 + ssz) of the R x R outputs G_n and the next S
  const int ssz = (R2 + (int)nrank - 1) / (int)nrank;
  const int s0 = min(R2, (int)rank * ssz), s1 = min(R2, s0 + ssz);
  const int ng = N - (next_mode == n ? 1 : 2);
  const bool gpre = ng > 0 && ng * ssz <= kGpreDoubles;
  if (gpre) {
#pragma unroll 1
    for (int k = 0, slot = 0; k < N; ++k) {
      if (k == n || k == next_mode) continue;
#pragma unroll 1
      for (int e = s0 + tid; e < s1; e += T)
        cp_async8(Gpre + slot * ssz + (e - s0), st.G + (long long)k * R2 + e);
      ++slot;
    }
  }
  if (tid == 0) {
    cp_async4(reinterpret_cast<float*>(flag_sh), reinterpret_cast<const float*>(st.flags));
    cp_async4(reinterpret_cast<float*>(flag_sh + 1), reinterpret_cast<const float*>(st.flags + 2));
    cp_async8(scal_sh, st.scalars);
    cp_async8(scal_sh + 1, st.scalars + 4);
    cp_async8(scal_sh + 2, st.scalars + 5);
  }
  // ... then M, which the predecessor writes
  pdl_wait();
  pdl_trigger();
  if (!sweep) stage_rows(Hs, Hg);
  stage_rows(Ms, Mg);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // the stop flag is the same for every CTA (written by an earlier kernel only):
  // every CTA of the cluster leaves here, before any cluster barrier
  if (flag_sh[0]) return;
  for (int r = tid; r < RMAX; r += T) {
    lamf[r] = r < R ? (float)lamd[r] : 0.0f;
    const float srr = r < R ? Srot[r * RMAX + (r & 3)] : 0.0f;  // S_rr
    sinv[r] = srr != 0.0f ? 1.0f / srr : 0.0f;
  }
  __syncthreads();

  // ---- HALS sweep (Sec. II-B): thread = row, columns in order.  The row of
  // W sits in registers, rotated so that column j is w[j mod 4] while columns
  // 4 floor(j / 4) .. + 3 are swept; the sweep is a rolled loop over those
  // blocks (a 4-column body, then a rotation by 4), which keeps the code small
  // enough to stay in the instruction cache.  Columns R .. R rounded up to 4
  // are zero padding (S_rr = 0 leaves them as they are).
  FF bp{0.0f, 0.0f};
  if (tid < nrows && !sweep) {
    // W given (an exact NLS solve wrote it): only <M, W>
    const float* wrow = Hs + tid * RP;
    const float* mrow = Ms + tid * RP;
    float b = 0.0f;
    for (int c = 0; c < R; ++c) b = fmaf(mrow[c], wrow[c], b);
    bp.hi = b;
  } else if (tid < nrows) {
    const float* hrow = Hs + tid * RP;
    const float* mrow = Ms + tid * RP;
    float w[RMAX];
#pragma unroll
    for (int c = 0; c < RMAX; ++c) w[c] = c < R ? hrow[c] * lamf[c] : 0.0f;
    const int Rpad = (R + 3) & ~3;
#pragma unroll 1
    for (int j0 = 0; j0 < Rpad; j0 += 4) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = j0 + t;
        // the column swept last (rotated index p) enters the dot product last,
        // so the other terms do not wait for its update
        const int p = t == 0 ? RMAX - 1 : t - 1;
        const float* srow = Srot + j * RMAX;
        float d[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c4 = 0; c4 < RMAX / 4; ++c4) {
          const float4 sv = reinterpret_cast<const float4*>(srow)[c4];
          const float sa[4] = {sv.x, sv.y, sv.z, sv.w};
          const int h = 4 * (c4 & 1);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (4 * c4 + k != p) d[h + k] = fmaf(w[4 * c4 + k], sa[k], d[h + k]);
        }
        float dot = ((d[0] + d[4]) + (d[1] + d[5])) + ((d[2] + d[6]) + (d[3] + d[7]));
        dot = fmaf(w[p], srow[p], dot);
        const float si = sinv[j];
        const float upd = fmaxf(0.0f, w[t] + (mrow[j] - dot) * si);
        w[t] = si != 0.0f ? upd : w[t];  // S_jj = 0: column left as it is
      }
      const float r0 = w[0], r1 = w[1], r2 = w[2], r3 = w[3];
#pragma unroll
      for (int c = 0; c < RMAX - 4; ++c) w[c] = w[c + 4];
      w[RMAX - 4] = r0;
      w[RMAX - 3] = r1;
      w[RMAX - 2] = r2;
      w[RMAX - 1] = r3;
    }
    // w[c] is now column (Rpad + c) mod RMAX
    float b = 0.0f;
    float* wrow = Hs + tid * RP;
#pragma unroll
    for (int c = 0; c < RMAX; ++c) {
      const int col = (Rpad + c) & (RMAX - 1);
      if (col < R) {
        b = fmaf(mrow[col], w[c], b);
        wrow[col] = w[c];
      }
    }
    bp.hi = b;
  }
  // <M, W> of this CTA: float-float over its rows (warp, then warps in order)
  if (warp * 32 < nrows) bp = ff_warp_sum(bp);
  if (lane == 0) red[warp] = bp;
  __syncthreads();
  if (tid == 0) {
    FF s{0.0f, 0.0f};
    for (int k = 0; k < T / 32; ++k) s = ff_add(s, red[k]);
    beta_own = s;
  }

  // ---- partial W^T W: thread = (4x4 tile, row group), register tiles
  const int nb4 = (R + 3) / 4;
  const int tiles = nb4 * nb4;
  const int groups = min(GROUPS, max(1, T / tiles));
#pragma unroll 1
  for (int t0 = tid; t0 < tiles * groups; t0 += T) {
    const int tile = t0 % tiles, g = t0 / tiles;
    const int a0 = (tile / nb4) * 4, b0 = (tile % nb4) * 4;
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
#pragma unroll 4
    for (int rr = g; rr < nrows; rr += groups) {
      const float4 qa = *reinterpret_cast<const float4*>(Hs + rr * RP + a0);
      const float4 qb = *reinterpret_cast<const float4*>(Hs + rr * RP + b0);
      const float va[4] = {qa.x, qa.y, qa.z, qa.w};
      const float vb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(va[x], vb[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (a0 + x < R && b0 + y < R) gpart[(g * R + a0 + x) * R + b0 + y] = acc[x][y];
  }
  __syncthreads();
#pragma unroll 1
  for (int e = tid; e < R2; e += T) {
    float s = 0.0f;
    for (int g = 0; g < groups; ++g) s += gpart[g * R2 + e];
    Gown[e] = s;
  }
  cluster_arrive();
  cluster_wait();

  // ---- the cluster's W^T W and <M, W>, summed in CTA order (same bits in
  // every CTA); four elements per remote load, every CTA's loads in flight at once
#pragma unroll 1
  for (int e4 = tid; e4 < (R2 + 3) / 4; e4 += T) {
    const int e = 4 * e4;
    float4 v[kClusterMax];
    if (e + 4 <= R2) {
#pragma unroll
      for (int k = 0; k < kClusterMax; ++k)
        if (k < (int)nrank) v[k] = ld_cluster4(cluster_addr(Gown + e, k));
    } else {
#pragma unroll
      for (int k = 0; k < kClusterMax; ++k)
        if (k < (int)nrank) {
          v[k].x = ld_cluster(cluster_addr(Gown + e, k));
          v[k].y = e + 1 < R2 ? ld_cluster(cluster_addr(Gown + e + 1, k)) : 0.0f;
          v[k].z = e + 2 < R2 ? ld_cluster(cluster_addr(Gown + e + 2, k)) : 0.0f;
          v[k].w = 0.0f;
        }
    }
    float4 sum = v[0];
#pragma unroll
    for (int k = 1; k < kClusterMax; ++k)
      if (k < (int)nrank) {
        sum.x += v[k].x;
        sum.y += v[k].y;
        sum.z += v[k].z;
        sum.w += v[k].w;
      }
    const float sv[4] = {sum.x, sum.y, sum.z, sum.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (e + i < R2) GW[e + i] = sv[i];
  }
  if (warp == 0) {
    // lane k fetches CTA k's <M, W>; lane 0 adds them in CTA order
    FF bk{0.0f, 0.0f};
    if (lane < (int)nrank)
      bk = FF{ld_cluster(cluster_addr(&beta_own.hi, lane)), ld_cluster(cluster_addr(&beta_own.lo, lane))};
    FF s{0.0f, 0.0f};
    for (int k = 0; k < (int)nrank; ++k)
      s = ff_add(s, FF{__shfl_sync(0xffffffffu, bk.hi, k), __shfl_sync(0xffffffffu, bk.lo, k)});
    if (lane == 0) beta_sh = s;
  }
  // done reading the other CTAs' shared memory; they may leave once all have
  cluster_arrive();
  __syncthreads();

  // ---- lambda = column norms of W in float64; from here on lamd holds
  // 1 / lambda and lamf its float32 value (for the row scaling)
  for (int r = tid; r < R; r += T) {
    double l, li;
    rsqrt_sqrt_f64(GW[r * R + r], &li, &l);
    if (lead) st.lam[r] = l;
    lamd[r] = li;
    lamf[r] = (float)li;
  }
  __syncthreads();
  // this CTA's rows of H = W / lambda (multiplication by the float32 reciprocal)
  float* Hw = H + (long long)row0 * R;
  if (vec) {
    const float4* l4 = reinterpret_cast<const float4*>(lamf);
#pragma unroll 1
    for (int v = tid; v < nrows * R / 4; v += T) {
      const int e = 4 * v, rr = e / R, c = e - rr * R;
      const float4 w = *reinterpret_cast<const float4*>(Hs + rr * RP + c);
      const float4 l = l4[c >> 2];
      reinterpret_cast<float4*>(Hw)[v] = make_float4(w.x * l.x, w.y * l.y, w.z * l.z, w.w * l.w);
    }
  } else {
#pragma unroll 1
    for (int e = tid; e < nrows * R; e += T) Hw[e] = Hs[(e / R) * RP + e % R] * lamf[e % R];
  }
  if (U) {
    // the ADMM dual of these rows (written by the kernel just before) into
    // the frame of the normalised factor
    float* Uw = U + (long long)row0 * R;
#pragma unroll 1
    for (int e = tid; e < nrows * R; e += T) Uw[e] *= lamf[e % R];
  }
  // this CTA's slice of G_n and of S for the next mode: Hadamard of every Gram
  // but next_mode's, in mode order (mode n's is the new one)
  double* Gng = st.G + (long long)n * R2;
#pragma unroll 1
  for (int e = s0 + tid; e < s1; e += T) {
    const double gn = (double)GW[e] * lamd[e / R] * lamd[e % R];
    Gng[e] = gn;
    double s = 1.0;
    for (int k = 0, slot = 0; k < N; ++k) {
      if (k == next_mode) continue;
      if (k == n) {
        s *= gn;
      } else {
        s *= gpre ? Gpre[slot * ssz + (e - s0)] : st.G[(long long)k * R2 + e];
        ++slot;
      }
    }
    st.S[(long long)next_mode * R2 + e] = s;
    st.S32[e] = (float)s;
  }
  if (lead && is_last) {
    // gamma = lambda^T (S * G_N) lambda = sum_ab S_ab (W^T W)_ab (Sec. IV-B),
    // float64 over the thread's terms, the warp, then the warps in order
    double g0 = 0.0, g1 = 0.0;  // two chains, joined in a fixed order
#pragma unroll 1
    for (int e = tid; e < R2; e += 2 * T) {
      g0 = fma(Sd[e], (double)GW[e], g0);
      if (e + T < R2) g1 = fma(Sd[e + T], (double)GW[e + T], g1);
    }
    double g = warp_sum_d(g0 + g1);
    if (lane == 0) redd[warp] = g;
    __syncthreads();
    if (tid == 0) {
      // the eight warps' sums as a fixed tree
      static_assert(T / 32 == 8, "gamma tree over eight warps");
      const double gamma = ((redd[0] + redd[1]) + (redd[2] + redd[3])) +
                           ((redd[4] + redd[5]) + (redd[6] + redd[7]));
      const double beta = (double)beta_sh.hi + (double)beta_sh.lo;
      const double alpha = scal_sh[0], tol = scal_sh[1], prev = scal_sh[2];
      const double eps = sqrt(fmax(0.0, alpha - 2.0 * beta + gamma) / alpha);
      const double fit = 1.0 - eps;
      const int it = flag_sh[1];
      st.scalars[1] = beta;
      st.scalars[2] = gamma;
      st.scalars[3] = eps;
      st.scalars[5] = fit;
      if (it < kFitCapacity) st.fits[it] = fit;
      st.flags[2] = it + 1;
      if (!isfinite(fit)) {
        st.flags[3] = 1;
        st.flags[0] = 1;
      } else if (it >= 1 && fabs(fit - prev) < tol) {
        st.flags[0] = 1;
      }
    }
  }
  // the other CTAs have read this CTA's partials before it leaves
  cluster_wait();
}

template <int RMAX>
size_t cluster_smem() {
  using C = ClusterCfg<RMAX>;
  return (size_t)(RMAX * RMAX + 2 * kClusterRowsMax * C::RP + C::GROUPS * RMAX * RMAX +
                  2 * RMAX * RMAX) * sizeof(float) +
         (size_t)(kGpreDoubles + RMAX * RMAX) * sizeof(double);
}

// ---- warp Cholesky ------------------------------------------------------------
// A = L L^T for a 32 x 32 symmetric positive definite A held one row per lane
// (a[j] = A(lane, j)); on return a[k] = L(lane, k) for k <= lane and
// dinv = 1 / L(lane, lane).  Right-looking: column k is scaled by the
// reciprocal square root of its pivot and broadcast by shuffles, and the
// trailing rows take its rank-one update.  Every register index is static.
// Called by all 32 lanes of a warp.
__device__ __forceinline__ void warp_cholesky32(float (&a)[32], float& dinv) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  dinv = 1.0f;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float dkk = __shfl_sync(full, a[k], k);
    const float inv = rsqrtf(dkk);
    const float l = a[k] * inv;
    if (lane == k) {
      a[k] = dkk * inv;
      dinv = inv;
    } else if (lane > k) {
      a[k] = l;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j > k) {
        const float ljk = __shfl_sync(full, l, j);
        if (lane >= j) a[j] = fmaf(-l, ljk, a[j]);
      }
    }
  }
}

// ---- block principal pivoting NLS update -----------------------------------
// Alg. 1's NLS-Update solved exactly, one warp per row of W (R <= 32): lane j
// owns variable j.  For the row's m (its row of M) it finds x >= 0 with
// y = S x - m >= 0 and x_j y_j = 0 by block principal pivoting.  The passive
// set F is a lane bit, started from the support of the row's previous value
// in H (the solution is unique for positive definite S, so the start changes
// only the number of steps; near convergence the first solve is feasible).
// Each step solves S_FF x_F = m_F with a Cholesky factor of S whose rows and
// columns outside F are replaced by the identity (x stays 0 there): lane i
// holds row i of the factor in registers, columns broadcast by shuffles; the
// forward substitution runs on the rows, the backward one on L^T read back
// from a transpose in the warp's tile of shared memory.  Then every
// infeasible index (x_j < 0 in F, y_j < 0 outside it: a warp ballot) changes
// sides at once while their count falls, up to three more times otherwise,
// then only the largest one (the backup rule).  Columns with S_jj = 0 stay at
// 0.  At most 50 R + 50 solves, as in the FP64 oracle.  W is written to H,
// unnormalised.  An index that the single-index rule would flip straight back
// (possible only through rounding, see below) is left as it is, and x is
// clamped at 0 on exit.
constexpr int kBppWarps = 4;

__global__ void __launch_bounds__(kBppWarps * 32)
k_bpp_rows(float* __restrict__ W, const float* __restrict__ M, int In, int R,
           const float* __restrict__ S, const int* __restrict__ flags) {
  pdl_wait();
  pdl_trigger();
  if (flags[0]) return;
  __shared__ float Ss[32][33];
  __shared__ float Lt[kBppWarps][32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int a = e >> 5, b = e & 31;
    Ss[a][b] = (a < R && b < R) ? S[a * R + b] : 0.0f;
  }
  __syncthreads();
  float(*T)[33] = Lt[warp];
  const bool usable = lane < R && Ss[lane][lane] > 0.0f;
  for (int row = blockIdx.x * kBppWarps + warp; row < In; row += gridDim.x * kBppWarps) {
    const long long off = (long long)row * R + lane;
    const float m = lane < R ? M[off] : 0.0f;
    bool inF = usable && W[off] > 0.0f;
    float x = 0.0f;
    int best = R + 1, backups = 3, last = -1;
#pragma unroll 1
    for (int step = 0; step < 50 * R + 50; ++step) {
      const unsigned Fm = __ballot_sync(full, inF);
      // a = row `lane` of S_FF, identity outside F
      float a[32];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        a[j] = (inF && ((Fm >> j) & 1u)) ? Ss[lane][j] : (lane == j ? 1.0f : 0.0f);
      float dinv;
      warp_cholesky32(a, dinv);
      // L z = b (b = m on F, 0 elsewhere)
      float z = inF ? m : 0.0f;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float zk = __shfl_sync(full, z * dinv, k);
        if (lane == k) z = zk;
        else if (lane > k) z = fmaf(-a[k], zk, z);
      }
      // L^T x = z, column k of L^T (row k of L) from the transpose
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j <= lane) T[lane][j] = a[j];
      __syncwarp();
#pragma unroll
      for (int k = 31; k >= 0; --k) {
        const float xk = __shfl_sync(full, z * dinv, k);
        if (lane == k) z = xk;
        else if (lane < k) z = fmaf(-T[k][lane], xk, z);
      }
      __syncwarp();
      x = inF ? z : 0.0f;
      // y = S x - m outside F
      float y = -m;
#pragma unroll
      for (int k = 0; k < 32; ++k) y = fmaf(Ss[lane][k], __shfl_sync(full, x, k), y);
      if (inF || !usable) y = 0.0f;
      const unsigned V = __ballot_sync(full, usable && (inF ? x < 0.0f : y < 0.0f));
      if (V == 0u) break;
      const int count = __popc(V);
      unsigned flip;
      if (count < best) {
        best = count;
        backups = 3;
        flip = V;
        last = -1;
      } else if (backups > 0) {
        --backups;
        flip = V;
        last = -1;
      } else {
        // a single pivot on a positive definite S reverses the sign of its
        // variable, so the index flipped just before is infeasible again only
        // by rounding: it is left as it is
        const unsigned Vb = last >= 0 ? V & ~(1u << last) : V;
        if (Vb == 0u) break;
        last = 31 - __clz(Vb);
        flip = 1u << last;
      }
      if ((flip >> lane) & 1u) inF = !inF;
    }
    if (lane < R) W[off] = fmaxf(x, 0.0f);
  }
}

// ---- AO-ADMM NLS update ----------------------------------------------------
// `iters` iterations of ADMM (scaled form) on every row's NNLS, R <= RMAX <= 32:
// rho = trace(S) / R; x = (S + rho I)^-1 (m + rho (z - u)); z = max(0, x + u);
// u = u + x - z, starting from z = H diag(lam) and u = U diag(lam) (the dual
// this mode's previous update left, in the normalised frame).  Every row
// shares S + rho I: warp 0 of each CTA factors it (warp_cholesky32, identity
// outside R), inverts the factor in registers (Z = L^-1) and forms
// P = Z^T Z through a copy of Z in shared memory.  Then kAdmmSplit threads
// share a row, each keeping z, u, m and x of its RMAX / kAdmmSplit columns in
// registers; the right-hand side is gathered across the row's lanes by
// shuffles and x accumulates the owned part of the columns of P.  Rows are
// staged in and written back through padded shared-memory tiles (coalesced).
// z goes to H (unnormalised W), u to U; the update's tail divides both by the
// new lambda.
// trace(S) = 0 gives z = u = 0.  Everything but M is staged, and the inverse
// formed, before griddepcontrol.wait (see the kernel).
constexpr int kAdmmSplit = 4;                    // threads per row
constexpr int kAdmmThreads = 64;
constexpr int kAdmmRows = kAdmmThreads / kAdmmSplit;  // rows per CTA

template <int RMAX>
__global__ void __launch_bounds__(kAdmmThreads)
k_admm_rows(float* __restrict__ W, float* __restrict__ U, const float* __restrict__ M, int In,
            int R, const float* __restrict__ S, const double* __restrict__ lam, int iters,
            const int* __restrict__ flags) {
  __shared__ __align__(16) float P[RMAX][RMAX];
  __shared__ __align__(16) float Zt[32][36];  // rows of L^-1 (row stride 16-byte aligned)
  __shared__ float Zs[kAdmmRows][RMAX + 1], Us[kAdmmRows][RMAX + 1], Ms[kAdmmRows][RMAX + 1];
  __shared__ float lamf[RMAX];
  __shared__ float rho_s;
  const int tid = threadIdx.x, lane = tid & 31;
  const unsigned full = 0xffffffffu;
  const long long row0 = (long long)blockIdx.x * kAdmmRows;
  const int nrows = (int)min((long long)kAdmmRows, (long long)In - row0);
  // H, U, S and lambda are written two or more kernels earlier (this mode's
  // previous update, the previous mode's): staged, and the inverse formed,
  // before griddepcontrol.wait, overlapping the predecessor; M after it
#pragma unroll 1
  for (int e = tid; e < nrows * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    cp_async4(&Zs[r][c], W + row0 * R + e);
    cp_async4(&Us[r][c], U + row0 * R + e);
  }
  if (tid < RMAX) lamf[tid] = tid < R ? (float)lam[tid] : 0.0f;
  if (tid < 32) {
    const float sll = lane < R ? S[lane * R + lane] : 0.0f;
    float tr = sll;
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(full, tr, o);
    const float rho = __shfl_sync(full, tr, 0) / (float)R;
    if (lane == 0) rho_s = rho;
    if (rho > 0.0f) {
      float a[32];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        a[j] = (lane < R && j < R) ? S[lane * R + j] + (j == lane ? rho : 0.0f)
                                   : (j == lane ? 1.0f : 0.0f);
      float dinv;
      warp_cholesky32(a, dinv);
      // Z = L^-1, lane i holding row i: right-looking forward substitution on
      // all 32 right-hand sides at once; row k is final once scaled and is
      // broadcast by shuffles to the rows below it
      float z[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = j == lane ? 1.0f : 0.0f;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (lane == k) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j <= k) z[j] *= dinv;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j <= k) {
            const float zkj = __shfl_sync(full, z[j], k);
            if (lane > k) z[j] = fmaf(-a[k], zkj, z[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) Zt[lane][j] = j <= lane ? z[j] : 0.0f;
      __syncwarp();
      // P = Z^T Z: lane i accumulates row i, P(i, j) = sum_k Z(k, i) Z(k, j),
      // from broadcasts of the rows of Z, and writes it as column i (so the
      // column reads of the update loop get P's columns as computed)
      float pr[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) pr[j] = 0.0f;
#pragma unroll 1
      for (int k = 0; k < 32; ++k) {
        const float zki = Zt[k][lane];
        const float4* zr = reinterpret_cast<const float4*>(&Zt[k][0]);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          const float4 v = zr[j4];
          pr[4 * j4] = fmaf(zki, v.x, pr[4 * j4]);
          pr[4 * j4 + 1] = fmaf(zki, v.y, pr[4 * j4 + 1]);
          pr[4 * j4 + 2] = fmaf(zki, v.z, pr[4 * j4 + 2]);
          pr[4 * j4 + 3] = fmaf(zki, v.w, pr[4 * j4 + 3]);
        }
      }
#pragma unroll
      for (int j = 0; j < RMAX; ++j)
        if (lane < RMAX) P[j][lane] = (j < R && lane < R) ? pr[j] : 0.0f;
    }
  }
  pdl_wait();
  pdl_trigger();
  if (flags[0]) {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
#pragma unroll 1
  for (int e = tid; e < nrows * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    cp_async4(&Ms[r][c], M + row0 * R + e);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const float rho = rho_s;
  // thread q of a row's group of kAdmmSplit consecutive lanes owns columns
  // [q * OWN, (q + 1) * OWN); every lane takes part in the shuffles (rows past
  // I_n on zeros) and only rows below I_n are written
  constexpr int OWN = RMAX / kAdmmSplit;
  const int row = tid / kAdmmSplit, q = tid % kAdmmSplit, c0 = q * OWN;
  const int src0 = lane & ~(kAdmmSplit - 1);
  const bool live = row < nrows && rho > 0.0f;
  float z[OWN], u[OWN], m[OWN];
#pragma unroll
  for (int k = 0; k < OWN; ++k) {
    const int c = c0 + k;
    const bool v = live && c < R;
    z[k] = v ? Zs[row][c] * lamf[c] : 0.0f;
    u[k] = v ? Us[row][c] * lamf[c] : 0.0f;
    m[k] = v ? Ms[row][c] : 0.0f;
  }
  if (rho > 0.0f) {
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
      // P is reread every iteration rather than held in registers
      asm volatile("" ::: "memory");
      float bown[OWN], x[OWN];
#pragma unroll
      for (int k = 0; k < OWN; ++k) {
        bown[k] = fmaf(rho, z[k] - u[k], m[k]);
        x[k] = 0.0f;
      }
      // x = P b over the owned columns: column j of P (read as row j, P being
      // symmetric) times b_j, b_j fetched from the lane that owns column j
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        const float bj = __shfl_sync(full, bown[j % OWN], src0 | (j / OWN));
        if constexpr (OWN % 4 == 0) {
          const float4* Pj = reinterpret_cast<const float4*>(&P[j][c0]);
#pragma unroll
          for (int k4 = 0; k4 < OWN / 4; ++k4) {
            const float4 pv = Pj[k4];
            x[4 * k4] = fmaf(pv.x, bj, x[4 * k4]);
            x[4 * k4 + 1] = fmaf(pv.y, bj, x[4 * k4 + 1]);
            x[4 * k4 + 2] = fmaf(pv.z, bj, x[4 * k4 + 2]);
            x[4 * k4 + 3] = fmaf(pv.w, bj, x[4 * k4 + 3]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < OWN; ++k) x[k] = fmaf(P[j][c0 + k], bj, x[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < OWN; ++k) {
        const float zn = fmaxf(0.0f, x[k] + u[k]);
        u[k] = u[k] + (x[k] - zn);
        z[k] = zn;
      }
    }
  }
  if (row < nrows) {
#pragma unroll
    for (int k = 0; k < OWN; ++k) {
      const int c = c0 + k;
      if (c < R) {
        Zs[row][c] = z[k];
        Us[row][c] = u[k];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < nrows * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    const long long g = row0 * R + e;
    W[g] = Zs[r][c];
    U[g] = Us[r][c];
  }
}

// ---- accelerated projected gradient NLS update -------------------------------
// `iters` steps of Nesterov's accelerated projected gradient (FISTA form) on
// every row's NNLS, R <= RMAX <= 32: with L = max_i sum_j |S_ij| (a bound on
// the largest eigenvalue of S), x_k = max(0, y_k - (S y_k - m) / L),
// t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, y_{k+1} = x_k + ((t_k - 1) / t_{k+1})
// (x_k - x_{k-1}), from x_0 = y_1 = H diag(lam).  One thread per row keeps x,
// y and the gradient in registers; the gradient accumulates the columns of S
// (read as rows, S being symmetric) from shared-memory broadcasts.  S, H and
// lambda are written two or more kernels earlier and staged before
// griddepcontrol.wait; M after it.  x goes to H (unnormalised W).  L = 0
// leaves W = H diag(lam).
constexpr int kApgRows = 64;

template <int RMAX>
__global__ void __launch_bounds__(kApgRows)
k_apg_rows(float* __restrict__ W, const float* __restrict__ M, int In, int R,
           const float* __restrict__ S, const double* __restrict__ lam, int iters,
           const int* __restrict__ flags) {
  __shared__ __align__(16) float Ss[RMAX][RMAX];
  __shared__ float Xs[kApgRows][RMAX + 1], Ms[kApgRows][RMAX + 1];
  __shared__ float lamf[RMAX];
  __shared__ float linv_s;
  const int tid = threadIdx.x, lane = tid & 31;
  const unsigned full = 0xffffffffu;
  const long long row0 = (long long)blockIdx.x * kApgRows;
  const int nrows = (int)min((long long)kApgRows, (long long)In - row0);
#pragma unroll 1
  for (int e = tid; e < nrows * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    cp_async4(&Xs[r][c], W + row0 * R + e);
  }
  for (int e = tid; e < RMAX * RMAX; e += blockDim.x) {
    const int a = e / RMAX, b = e - a * RMAX;
    Ss[a][b] = (a < R && b < R) ? S[a * R + b] : 0.0f;
  }
  if (tid < RMAX) lamf[tid] = tid < R ? (float)lam[tid] : 0.0f;
  if (tid < 32) {
    // L: largest absolute row sum, lane r summing row r
    float rs = 0.0f;
    if (lane < R)
      for (int j = 0; j < R; ++j) rs += fabsf(S[lane * R + j]);
    for (int o = 16; o > 0; o >>= 1) rs = fmaxf(rs, __shfl_xor_sync(full, rs, o));
    if (lane == 0) linv_s = rs > 0.0f ? 1.0f / rs : 0.0f;
  }
  pdl_wait();
  pdl_trigger();
  if (flags[0]) {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
#pragma unroll 1
  for (int e = tid; e < nrows * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    cp_async4(&Ms[r][c], M + row0 * R + e);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const float linv = linv_s;
  if (tid < nrows) {
    float x[RMAX], y[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      x[j] = j < R ? Xs[tid][j] * lamf[j] : 0.0f;
      y[j] = x[j];
    }
    if (linv > 0.0f) {
      float t = 1.0f;
#pragma unroll 1
      for (int it = 0; it < iters; ++it) {
        // S is reread every step rather than held in registers
        asm volatile("" ::: "memory");
        float g[RMAX];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) g[j] = j < R ? -Ms[tid][j] : 0.0f;
#pragma unroll
        for (int j = 0; j < RMAX; ++j) {
          const float4* Sj = reinterpret_cast<const float4*>(&Ss[j][0]);
#pragma unroll
          for (int i4 = 0; i4 < RMAX / 4; ++i4) {
            const float4 sv = Sj[i4];
            g[4 * i4] = fmaf(sv.x, y[j], g[4 * i4]);
            g[4 * i4 + 1] = fmaf(sv.y, y[j], g[4 * i4 + 1]);
            g[4 * i4 + 2] = fmaf(sv.z, y[j], g[4 * i4 + 2]);
            g[4 * i4 + 3] = fmaf(sv.w, y[j], g[4 * i4 + 3]);
          }
        }
        const float tn = 0.5f * (1.0f + sqrtf(fmaf(4.0f * t, t, 1.0f)));
        const float beta = (t - 1.0f) / tn;
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
          const float xn = fmaxf(0.0f, fmaf(-g[i], linv, y[i]));
          y[i] = fmaf(beta, xn - x[i], xn);
          x[i] = xn;
        }
        t = tn;
      }
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j)
      if (j < R) Xs[tid][j] = x[j];
  }
  __syncthreads();
  for (int e = tid; e < nrows * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    W[row0 * R + e] = Xs[r][c];
  }
}

__global__ void k_solve_reset(SolveState st, int R, double tol) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) st.lam[r] = 1.0;
  if (threadIdx.x == 0) {
    st.flags[0] = 0;
    st.flags[1] = 0;
    st.flags[2] = 0;
    st.flags[3] = 0;
    st.flags[8] = 0;
    st.scalars[4] = tol;
    st.scalars[5] = 0.0;
  }
}

__global__ void k_compute_S(SolveState st, int N, int R, int mode) {
  const int R2 = R * R;
  for (int t = threadIdx.x; t < R2; t += blockDim.x) {
    double s = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != mode) s *= st.G[(long long)k * R2 + t];
    st.S[(long long)mode * R2 + t] = s;
    st.S32[t] = (float)s;
  }
}

struct ResidualArgs {
  int N;
  long long dims[kMaxModes];
  const float* H[kMaxModes];
};

// ||X - [[lam; H]]||^2 and ||X||^2: CTA per mode-1 fibre (grid-stride over
// fibres), coefficient c_r = lam_r * prod_{n>=2} H_n(i_n, r) in shared memory.
__global__ void k_explicit_residual(const float* __restrict__ X, ResidualArgs a, int R,
                                    const double* __restrict__ lam, long long nfib,
                                    double* __restrict__ partials) {
  __shared__ float coef[kMaxRank];
  __shared__ double sh[64];
  const long long I1 = a.dims[0];
  double acc = 0.0, accx = 0.0;
  for (long long f = blockIdx.x; f < nfib; f += gridDim.x) {
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double v = lam[r];
      long long rem = f;
      for (int m = 1; m < a.N; ++m) {
        long long im = rem % a.dims[m];
        rem /= a.dims[m];
        v *= (double)a.H[m][im * R + r];
      }
      coef[r] = (float)v;
    }
    __syncthreads();
    for (long long i = threadIdx.x; i < I1; i += blockDim.x) {
      float mv = 0.0f;
      for (int r = 0; r < R; ++r) mv = fmaf(a.H[0][i * R + r], coef[r], mv);
      const float xv = X[f * I1 + i];
      const double d = (double)xv - (double)mv;
      acc += d * d;
      accx += (double)xv * xv;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    accx += __shfl_xor_sync(0xffffffffu, accx, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[w] = acc;
    sh[32 + w] = accx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, sx = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s += sh[k];
      sx += sh[32 + k];
    }
    partials[2 * blockIdx.x] = s;
    partials[2 * blockIdx.x + 1] = sx;
  }
}

__global__ void k_sum_pairs(const double* __restrict__ partials, int n, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0, sx = 0.0;
    for (int i = 0; i < n; ++i) {
      s += partials[2 * i];
      sx += partials[2 * i + 1];
    }
    out[0] = s;
    out[1] = sx;
  }
}

size_t hals_smem(int R) {
  return (size_t)R * R * sizeof(float) + (size_t)kRowsPerBlock * (R + 1) * sizeof(float);
}

}  // namespace

cudaError_t kernel_attributes_init() {
  cudaError_t e = cudaFuncSetAttribute(k_hals_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_multi<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)multi_smem<16>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_multi<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)multi_smem<32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_multi<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)multi_smem<64>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_cluster<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cluster_smem<16>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_cluster<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cluster_smem<32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_cluster<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cluster_smem<64>());
  if (e == cudaSuccess) e = tc_attributes_init();
  return e;
}

int hals_gram_blocks(int64_t In) { return (int)((In + kRowsPerBlock - 1) / kRowsPerBlock); }

cudaError_t launch_hals_gram(float* H, const float* M, int64_t In, int R, SolveState st,
                             cudaStream_t stream) {
  size_t smem = hals_smem(R);
  return launch_kernel(k_hals_gram, dim3(hals_gram_blocks(In)), dim3(kHalsThreads), smem, stream,
                       H, M, (long long)In, R, st.S32, (const double*)st.lam,
                       st.gram_part, (const int*)st.flags, 1);
}

cudaError_t launch_bpp_rows(float* H, const float* M, int64_t In, int R, SolveState st,
                            int num_sms, cudaStream_t stream) {
  if (R > 32) return cudaErrorInvalidValue;
  const long long ctas = (In + kBppWarps - 1) / kBppWarps;
  const int grid = (int)std::max(1LL, std::min(ctas, (long long)num_sms * 4));
  return launch_kernel(k_bpp_rows, dim3(grid), dim3(kBppWarps * 32), 0, stream, H, M, (int)In, R,
                       st.S32, (const int*)st.flags);
}

cudaError_t launch_bpp_update(float* H, const float* M, int64_t In, int R, SolveState st,
                              int num_sms, cudaStream_t stream) {
  cudaError_t e = launch_bpp_rows(H, M, In, R, st, num_sms, stream);
  if (e != cudaSuccess) return e;
  // Gram partials and <M, W> of the new W (no sweep)
  return launch_kernel(k_hals_gram, dim3(hals_gram_blocks(In)), dim3(kHalsThreads), hals_smem(R),
                       stream, H, M, (long long)In, R, st.S32, (const double*)st.lam,
                       st.gram_part, (const int*)st.flags, 2);
}

cudaError_t launch_admm_rows(float* H, float* U, const float* M, int64_t In, int R, int iters,
                            SolveState st, cudaStream_t stream) {
  if (R > 32 || In > INT32_MAX) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((In + kAdmmRows - 1) / kAdmmRows)), block(kAdmmThreads);
  const int rmax = R <= 8 ? 8 : (R <= 16 ? 16 : 32);
  auto k = rmax == 8 ? k_admm_rows<8> : (rmax == 16 ? k_admm_rows<16> : k_admm_rows<32>);
  return launch_kernel(k, grid, block, 0, stream, H, U, M, (int)In, R, st.S32,
                       (const double*)st.lam, iters, (const int*)st.flags);
}

cudaError_t launch_admm_update(float* H, float* U, const float* M, int64_t In, int R, int iters,
                               SolveState st, cudaStream_t stream) {
  cudaError_t e = launch_admm_rows(H, U, M, In, R, iters, st, stream);
  if (e != cudaSuccess) return e;
  return launch_kernel(k_hals_gram, dim3(hals_gram_blocks(In)), dim3(kHalsThreads), hals_smem(R),
                       stream, H, M, (long long)In, R, st.S32, (const double*)st.lam,
                       st.gram_part, (const int*)st.flags, 2);
}

cudaError_t launch_apg_rows(float* H, const float* M, int64_t In, int R, int iters,
                           SolveState st, cudaStream_t stream) {
  if (R > 32 || In > INT32_MAX) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((In + kApgRows - 1) / kApgRows)), block(kApgRows);
  const int rmax = R <= 8 ? 8 : (R <= 16 ? 16 : 32);
  auto k = rmax == 8 ? k_apg_rows<8> : (rmax == 16 ? k_apg_rows<16> : k_apg_rows<32>);
  return launch_kernel(k, grid, block, 0, stream, H, M, (int)In, R, st.S32,
                       (const double*)st.lam, iters, (const int*)st.flags);
}

cudaError_t launch_apg_update(float* H, const float* M, int64_t In, int R, int iters,
                              SolveState st, cudaStream_t stream) {
  cudaError_t e = launch_apg_rows(H, M, In, R, iters, st, stream);
  if (e != cudaSuccess) return e;
  return launch_kernel(k_hals_gram, dim3(hals_gram_blocks(In)), dim3(kHalsThreads), hals_smem(R),
                       stream, H, M, (long long)In, R, st.S32, (const double*)st.lam,
                       st.gram_part, (const int*)st.flags, 2);
}

cudaError_t launch_gram_only(const float* H, int64_t In, int R, SolveState st,
                             cudaStream_t stream) {
  size_t smem = hals_smem(R);
  k_hals_gram<<<hals_gram_blocks(In), kHalsThreads, smem, stream>>>(
      const_cast<float*>(H), nullptr, In, R, st.S32, st.lam, st.gram_part, st.flags, 0);
  return cudaGetLastError();
}

// H(i, r) *= inv(r) for `rows` rows of R columns (row-major).
__global__ void k_scale_columns(float* __restrict__ H, long long n, int R,
                                const float* __restrict__ inv) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    H[e] *= inv[e % R];
}

cudaError_t launch_scale_columns(float* H, int64_t rows, int R, const float* inv,
                                 cudaStream_t stream) {
  const long long n = (long long)rows * R;
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  k_scale_columns<<<blocks, 256, 0, stream>>>(H, n, R, inv);
  return cudaGetLastError();
}

bool multi_update_ok(int64_t In, int R) { return In <= kMultiMaxRows && R <= 64; }

// partial scratch needed by the multi-CTA update (floats)
size_t multi_update_scratch(int64_t In, int R) {
  const int64_t nb = (In + multi_rows(R) - 1) / multi_rows(R);
  return (size_t)(nb + 1) * (R * R + 2) + 2 * (size_t)R * R + 4;
}

cudaError_t launch_update_multi(float* H, const float* M, int64_t In, int R, int N, int n,
                                int next_mode, int is_last, SolveState st, float* part,
                                cudaStream_t stream) {
  const int nb = (int)((In + multi_rows(R) - 1) / multi_rows(R));
  const int rmax = R <= 16 ? 16 : (R <= 32 ? 32 : 64);
  switch (rmax) {
    case 16:
      return launch_kernel(k_update_multi<16>, dim3(nb), dim3(MultiCfg<16>::T), multi_smem<16>(),
                           stream, H, M, (int)In, R, N, n, next_mode, is_last, st, part);
    case 32:
      return launch_kernel(k_update_multi<32>, dim3(nb), dim3(MultiCfg<32>::T), multi_smem<32>(),
                           stream, H, M, (int)In, R, N, n, next_mode, is_last, st, part);
    default:
      return launch_kernel(k_update_multi<64>, dim3(nb), dim3(MultiCfg<64>::T), multi_smem<64>(),
                           stream, H, M, (int)In, R, N, n, next_mode, is_last, st, part);
  }
}

bool cluster_update_ok(int64_t In, int R) { return In >= 1 && In <= kClusterMaxRows && R <= 64; }

cudaError_t launch_update_cluster(float* H, const float* M, int64_t In, int R, int N, int n,
                                  int next_mode, int is_last, SolveState st, cudaStream_t stream,
                                  int sweep, float* U) {
  const int rows = cluster_rows(In);
  const int nb = (int)((In + rows - 1) / rows);
  const int rmax = R <= 16 ? 16 : (R <= 32 ? 32 : 64);
  switch (rmax) {
    case 16:
      return launch_kernel_cluster(k_update_cluster<16>, dim3(nb), dim3(kClusterThreads),
                                   cluster_smem<16>(), stream, nb, H, M, (int)In, R, N, n,
                                   next_mode, is_last, rows, sweep, st, U);
    case 32:
      return launch_kernel_cluster(k_update_cluster<32>, dim3(nb), dim3(kClusterThreads),
                                   cluster_smem<32>(), stream, nb, H, M, (int)In, R, N, n,
                                   next_mode, is_last, rows, sweep, st, U);
    default:
      return launch_kernel_cluster(k_update_cluster<64>, dim3(nb), dim3(kClusterThreads),
                                   cluster_smem<64>(), stream, nb, H, M, (int)In, R, N, n,
                                   next_mode, is_last, rows, sweep, st, U);
  }
}

cudaError_t launch_finalize(float* H, int64_t In, int R, int N, int n, int next_mode,
                            int nblocks, int is_last, int init, double tol, SolveState st,
                            cudaStream_t stream, float* U) {
  (void)tol;
  size_t smem = ((size_t)R * R + R) * sizeof(double);
  return launch_kernel(k_finalize, dim3(1), dim3(1024), smem, stream, H, (long long)In, R, N, n,
                       next_mode, nblocks, is_last, init, st, U);
}

cudaError_t launch_solve_reset(SolveState st, int R, double tol, cudaStream_t stream) {
  k_solve_reset<<<1, 128, 0, stream>>>(st, R, tol);
  return cudaGetLastError();
}

cudaError_t launch_compute_S(SolveState st, int N, int R, int mode, cudaStream_t stream) {
  k_compute_S<<<1, 1024, 0, stream>>>(st, N, R, mode);
  return cudaGetLastError();
}

cudaError_t launch_explicit_residual(const float* X, int N, const int64_t* dims, int R,
                                     float* const* H, const double* lam, double* partials,
                                     int nparts, double* out, cudaStream_t stream) {
  ResidualArgs a;
  a.N = N;
  long long nfib = 1;
  for (int m = 0; m < kMaxModes; ++m) {
    a.dims[m] = m < N ? dims[m] : 1;
    a.H[m] = m < N ? H[m] : nullptr;
    if (m >= 1 && m < N) nfib *= dims[m];
  }
  int blocks = (int)min((long long)nparts, nfib);
  k_explicit_residual<<<blocks, 256, 0, stream>>>(X, a, R, lam, nfib, partials);
  k_sum_pairs<<<1, 32, 0, stream>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace nncp
