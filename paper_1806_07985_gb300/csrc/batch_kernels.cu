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

#include "batch_kernels.cuh"

namespace nncp {

namespace {

constexpr int kTileJ = 32;  // contraction tile of the batched partial MTTKRPs

__device__ __forceinline__ bool tensor_done(const BTensor& t) { return t.flags[0] != 0; }

// KRP row offsets of element k over modes [m0, m1) of tensor t: off[m - m0] = k_m * R
__device__ __forceinline__ void krp_offsets(const BTensor& t, int m0, int m1, long long k, int* off) {
  for (int m = m0; m < m1; ++m) {
    const long long dm = t.dims[m];
    off[m - m0] = (int)((k % dm) * t.R);
    k /= dm;
  }
}

// ---------------------------------------------------------------- init --

// alpha partials: item (tensor, chunk of kAlphaChunk elements) -> alpha_part[item]
__global__ void k_b_sumsq(const BTensor* __restrict__ ts, const int2* __restrict__ items,
                          double* __restrict__ alpha_part) {
  const int2 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  const long long e0 = (long long)it.y * kAlphaChunk;
  const long long e1 = min((long long)t.I, e0 + kAlphaChunk);
  double acc = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const float v = t.X[e];
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
                         const int* __restrict__ alpha_first, double tol, int max_iters) {
  BTensor& t = ts[blockIdx.x];
  const int R = t.R, N = t.N, R2 = R * R;
  __shared__ double lam[kBatchMaxRank];
  __shared__ double cn[kBatchMaxRank];
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int c = alpha_first[blockIdx.x]; c < alpha_first[blockIdx.x + 1]; ++c) a += alpha_part[c];
    t.scal[0] = a;
    t.scal[1] = tol;
    t.max_iters = max_iters;
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

// root -> node {1}: part[c](i, r) = sum_{j in chunk c} X[i + I1 j] K(j, r),
// K = H_N (.) ... (.) H_2.  Item (tensor, chunk); thread = row i (I1 <= 256).
template <int RMAX>
__global__ void __launch_bounds__(256)
k_b_pm_right(const BTensor* __restrict__ ts, const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  if (tensor_done(t)) return;
  const int R = t.R, N = t.N;
  const int I1 = (int)t.dims[0];
  const long long J = t.I / I1;
  const long long j0 = (long long)it.y * t.jchunk;
  const long long j1 = min(J, j0 + t.jchunk);
  __shared__ float Xs[kTileJ][kBatchMaxI + 1];
  __shared__ __align__(16) float Ws[kTileJ][RMAX];
  __shared__ int offs[kTileJ][kMaxModes];
  const int tid = threadIdx.x;
  float acc[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) acc[r] = 0.0f;
  for (long long jt = j0; jt < j1; jt += kTileJ) {
    const int nj = (int)min((long long)kTileJ, j1 - jt);
    if (tid < kTileJ && tid < nj) krp_offsets(t, 1, N, jt + tid, offs[tid]);
    // the tile's columns are contiguous: nj * I1 floats
    const float* xb = t.X + jt * I1;
    for (int e = tid; e < nj * I1; e += blockDim.x) Xs[e / I1][e % I1] = xb[e];
    __syncthreads();
    for (int e = tid; e < kTileJ * RMAX; e += blockDim.x) {
      const int jj = e / RMAX, r = e % RMAX;
      float w = 0.0f;
      if (jj < nj && r < R) {
        w = 1.0f;
        for (int m = 1; m < N; ++m) w *= t.H[m][offs[jj][m - 1] + r];
      }
      Ws[jj][r] = w;
    }
    __syncthreads();
    if (tid < I1) {
      for (int jj = 0; jj < nj; ++jj) {
        const float x = Xs[jj][tid];
#pragma unroll
        for (int r = 0; r < RMAX; r += 4) {
          const float4 w = *reinterpret_cast<const float4*>(&Ws[jj][r]);
          acc[r] = fmaf(x, w.x, acc[r]);
          acc[r + 1] = fmaf(x, w.y, acc[r + 1]);
          acc[r + 2] = fmaf(x, w.z, acc[r + 2]);
          acc[r + 3] = fmaf(x, w.w, acc[r + 3]);
        }
      }
    }
    __syncthreads();
  }
  if (tid < I1) {
    float* out = t.part + ((long long)it.y * I1 + tid) * R;
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < R) out[r] = acc[r];
  }
}

// M(1) = sum of the chunks' partials in chunk order; CTA per tensor
__global__ void k_b_reduce_m(const BTensor* __restrict__ ts) {
  const BTensor& t = ts[blockIdx.x];
  if (tensor_done(t)) return;
  const int E = (int)t.dims[0] * t.R;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < t.nchunk; ++c) s += t.part[(long long)c * E + e];
    t.M[e] = s;
  }
}

// root -> node {2..N}: T(j, r) = sum_i X[i + I1 j] H_1(i, r).  Item (tensor,
// block of 128 rows j); thread = row j; contraction in tiles of 32 i.
template <int RMAX>
__global__ void __launch_bounds__(128)
k_b_pm_left(const BTensor* __restrict__ ts, const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const BTensor& t = ts[it.x];
  if (tensor_done(t)) return;
  const int R = t.R;
  const int I1 = (int)t.dims[0];
  const long long J = t.I / I1;
  const long long jb = (long long)it.y * 128;
  const int nj = (int)min(128LL, J - jb);
  __shared__ float Xs[128][33];
  __shared__ __align__(16) float Hs[32][RMAX];
  const int tid = threadIdx.x;
  float acc[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) acc[r] = 0.0f;
  const float* H1 = t.H[0];
  for (int i0 = 0; i0 < I1; i0 += 32) {
    const int ni = min(32, I1 - i0);
    for (int e = tid; e < 128 * 32; e += 128) {
      const int jj = e >> 5, ii = e & 31;
      Xs[jj][ii] = (jj < nj && ii < ni) ? t.X[(jb + jj) * I1 + i0 + ii] : 0.0f;
    }
    for (int e = tid; e < 32 * RMAX; e += 128) {
      const int ii = e / RMAX, r = e % RMAX;
      Hs[ii][r] = (ii < ni && r < R) ? H1[(i0 + ii) * R + r] : 0.0f;
    }
    __syncthreads();
    for (int ii = 0; ii < ni; ++ii) {
      const float x = Xs[tid][ii];
#pragma unroll
      for (int r = 0; r < RMAX; r += 4) {
        const float4 h = *reinterpret_cast<const float4*>(&Hs[ii][r]);
        acc[r] = fmaf(x, h.x, acc[r]);
        acc[r + 1] = fmaf(x, h.y, acc[r + 1]);
        acc[r + 2] = fmaf(x, h.z, acc[r + 2]);
        acc[r + 3] = fmaf(x, h.w, acc[r + 3]);
      }
    }
    __syncthreads();
  }
  if (tid < nj) {
    float* out = t.node[1] + (jb + tid) * R;
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < R) out[r] = acc[r];
  }
}

// ---------------------------------------------------------- multi-TTVs --

// leaf M(a) from node {a..N}: M(i, r) = sum_k T[(i + I_a k) R + r] KK(k, r),
// KK = H_N (.) ... (.) H_{a+1}; CTA per tensor, threads over (i, r).
__global__ void k_b_mttv_leaf(const BTensor* __restrict__ ts, int a) {
  const BTensor& t = ts[blockIdx.x];
  if (tensor_done(t)) return;
  const int R = t.R, N = t.N;
  const int Ia = (int)t.dims[a];
  long long K = 1;
  for (int m = a + 1; m < N; ++m) K *= t.dims[m];
  const float* T = t.node[a];
  __shared__ int offs[kTileJ][kMaxModes];
  __shared__ float Ws[kTileJ][kBatchMaxRank];
  const int E = Ia * R;
  for (int eb = 0; eb < E; eb += 4 * (int)blockDim.x) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // outputs eb + threadIdx.x + q * blockDim
    for (long long k0 = 0; k0 < K; k0 += kTileJ) {
      const int nk = (int)min((long long)kTileJ, K - k0);
      if (threadIdx.x < nk) krp_offsets(t, a + 1, N, k0 + threadIdx.x, offs[threadIdx.x]);
      __syncthreads();
      for (int e = threadIdx.x; e < kTileJ * R; e += blockDim.x) {
        const int kk = e / R, r = e % R;
        float w = 0.0f;
        if (kk < nk) {
          w = 1.0f;
          for (int m = a + 1; m < N; ++m) w *= t.H[m][offs[kk][m - a - 1] + r];
        }
        Ws[kk][r] = w;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = eb + threadIdx.x + q * blockDim.x;
        if (e < E) {
          const int r = e % R;
          const float* tp = T + k0 * (long long)E + e;
          float s = acc[q];
          for (int kk = 0; kk < nk; ++kk) s = fmaf(tp[(long long)kk * E], Ws[kk][r], s);
          acc[q] = s;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = eb + threadIdx.x + q * blockDim.x;
      if (e < E) t.M[e] = acc[q];
    }
  }
}

// child node {a+1..N} from node {a..N}: out(j, r) = sum_i T[(i + I_a j) R + r] H_a(i, r)
// (the updated H_a); output is M when the child is a leaf.  CTA per tensor.
__global__ void k_b_mttv_first(const BTensor* __restrict__ ts, int a) {
  const BTensor& t = ts[blockIdx.x];
  if (tensor_done(t)) return;
  const int R = t.R, N = t.N;
  const int Ia = (int)t.dims[a];
  long long Jn = 1;
  for (int m = a + 1; m < N; ++m) Jn *= t.dims[m];
  const float* T = t.node[a];
  float* out = (a + 1 == N - 1) ? t.M : t.node[a + 1];
  const float* Ha = t.H[a];
  const long long E = Jn * R;
  for (long long e = threadIdx.x; e < E; e += blockDim.x) {
    const long long j = e / R;
    const int r = (int)(e % R);
    const float* tp = T + (j * Ia) * R + r;
    float s = 0.0f;
    for (int i = 0; i < Ia; ++i) s = fmaf(tp[(long long)i * R], Ha[i * R + r], s);
    out[e] = s;
  }
}

// ---------------------------------------------------------- mode update --

// One CTA per tensor (I_n <= kBatchMaxI rows, R <= RMAX): HALS sweep
// (Sec. II-B, row per thread, row in registers), W^T W, lambda, G_n,
// H_n = W / lambda, the fit at n = N (Sec. IV-B) with the stopping test, and
// S for the next mode -- all in shared memory.
template <int RMAX>
__global__ void __launch_bounds__(256)
k_b_update(BTensor* __restrict__ ts, int n, int* __restrict__ done_count) {
  BTensor& t = ts[blockIdx.x];
  if (tensor_done(t)) return;
  constexpr int RP = RMAX + 1;
  const int R = t.R, N = t.N, R2 = R * R;
  const int In = (int)t.dims[n];
  const int tid = threadIdx.x;
  extern __shared__ __align__(16) float bsm[];
  float* St = bsm;                 // RMAX x RMAX, St[r][c] = S[c][r], zero padded
  float* Ws = St + RMAX * RMAX;    // kBatchMaxI x RP (W, then H)
  __shared__ float lamf[RMAX], sinv[RMAX];
  __shared__ double GW[kBatchMaxRank * kBatchMaxRank];
  __shared__ double cinv[kBatchMaxRank];
  __shared__ double red[8];
  float* Hn = t.H[n];
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
  double bp = 0.0;
  for (int i = tid; i < In; i += blockDim.x) {
    float w[RMAX];
#pragma unroll
    for (int c = 0; c < RMAX; ++c) w[c] = c < R ? Hn[i * R + c] * lamf[c] : 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const float si = sinv[r];
      const float mr = r < R ? t.M[i * R + r] : 0.0f;
      float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
      for (int c = 0; c < RMAX; c += 2) {
        d0 = fmaf(w[c], St[r * RMAX + c], d0);
        d1 = fmaf(w[c + 1], St[r * RMAX + c + 1], d1);
      }
      const float upd = fmaxf(0.0f, w[r] + (mr - (d0 + d1)) * si);
      w[r] = si != 0.0f ? upd : w[r];
    }
    float b = 0.0f;
#pragma unroll
    for (int c = 0; c < RMAX; ++c) {
      if (c < R) b = fmaf(t.M[i * R + c], w[c], b);
      Ws[i * RP + c] = w[c];
    }
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
    nonfinite[b] = t.flags[2];
    if (lam)
      for (int r = 0; r < t.R; ++r) lam[lam_off[b] + r] = t.lam[r];
  }
}

template <int RMAX>
size_t update_smem() {
  return (size_t)(RMAX * RMAX + kBatchMaxI * (RMAX + 1)) * sizeof(float);
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
  return e;
}

cudaError_t launch_b_init(BTensor* ts, int count, const int2* alpha_items, int n_alpha_items,
                          double* alpha_part, const int* alpha_first, double tol, int max_iters,
                          cudaStream_t st) {
  if (n_alpha_items > 0) k_b_sumsq<<<n_alpha_items, 256, 0, st>>>(ts, alpha_items, alpha_part);
  k_b_init<<<count, 256, 0, st>>>(ts, alpha_part, alpha_first, tol, max_iters);
  return cudaGetLastError();
}

cudaError_t launch_b_pm_right(int rmax, const BTensor* ts, const int2* items, int n_items,
                              int count, cudaStream_t st) {
  if (n_items > 0) {
    if (rmax <= 16) k_b_pm_right<16><<<n_items, 256, 0, st>>>(ts, items);
    else if (rmax <= 32) k_b_pm_right<32><<<n_items, 256, 0, st>>>(ts, items);
    else k_b_pm_right<64><<<n_items, 256, 0, st>>>(ts, items);
  }
  k_b_reduce_m<<<count, 256, 0, st>>>(ts);
  return cudaGetLastError();
}

cudaError_t launch_b_pm_left(int rmax, const BTensor* ts, const int2* items, int n_items,
                             cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  if (rmax <= 16) k_b_pm_left<16><<<n_items, 128, 0, st>>>(ts, items);
  else if (rmax <= 32) k_b_pm_left<32><<<n_items, 128, 0, st>>>(ts, items);
  else k_b_pm_left<64><<<n_items, 128, 0, st>>>(ts, items);
  return cudaGetLastError();
}

cudaError_t launch_b_mttv_leaf(const BTensor* ts, int count, int a, cudaStream_t st) {
  k_b_mttv_leaf<<<count, 256, 0, st>>>(ts, a);
  return cudaGetLastError();
}

cudaError_t launch_b_mttv_first(const BTensor* ts, int count, int a, cudaStream_t st) {
  k_b_mttv_first<<<count, 256, 0, st>>>(ts, a);
  return cudaGetLastError();
}

cudaError_t launch_b_gather(const BTensor* ts, int count, int* iters, double* fits,
                            double* lam, const int* lam_off, int* nonfinite, cudaStream_t st) {
  k_b_gather<<<(count + 255) / 256, 256, 0, st>>>(ts, count, iters, fits, lam, lam_off, nonfinite);
  return cudaGetLastError();
}

cudaError_t launch_b_update(int rmax, BTensor* ts, int count, int n, int* done_count,
                            cudaStream_t st) {
  if (rmax <= 16) k_b_update<16><<<count, 256, update_smem<16>(), st>>>(ts, n, done_count);
  else if (rmax <= 32) k_b_update<32><<<count, 256, update_smem<32>(), st>>>(ts, n, done_count);
  else k_b_update<64><<<count, 256, update_smem<64>(), st>>>(ts, n, done_count);
  return cudaGetLastError();
}

}  // namespace nncp
