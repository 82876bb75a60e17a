// Factor-update kernels of one BCD inner iteration (Alg. 1 / Alg. 3):
//   HALS sweep (Sec. II-B) on W = H_n diag(lambda), row-parallel;
//   per-block partials of W^T W and <M, W>;
//   a single-CTA finalise: lambda = column norms, G_n = H_n^T H_n,
//   H_n = W diag(lambda)^-1, the fit from the Sec. IV-B identity at n = N,
//   and S = Hadamard of the other Grams for the next mode.
// FP64 is used for S, lambda, the Gram sums and the fit; the HALS arithmetic
// and the factors are float32.
#include <cuda_runtime.h>
#include <math.h>

#include "nncp_internal.cuh"

namespace nncp {

namespace {

constexpr int kRowsPerBlock = 64;
constexpr int kHalsThreads = 256;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One HALS sweep per row, one warp per row; lane holds columns lane + 32*j.
// Then the block's partial W^T W (float32 over <= 64 rows, stored as double)
// and partial <M, W>.
__global__ void __launch_bounds__(kHalsThreads)
k_hals_gram(float* __restrict__ H, const float* __restrict__ M, long long In, int R,
            const float* __restrict__ S32, const double* __restrict__ lam,
            double* __restrict__ gram_part, const int* __restrict__ flags, int do_hals) {
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
    for (int t = threadIdx.x; t < R * R; t += blockDim.x) Ss[t] = S32[t];
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
          w[j] = w[j] * (float)lam[c];
          m[j] = M[i * R + c];
        }
      }
    }
    if (do_hals) {
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
      float bp = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) bp = fmaf(m[j], w[j], bp);
      beta_acc += (double)warp_sum(bp);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = lane + 32 * j;
      if (c < R) {
        if (do_hals) H[i * R + c] = w[j];
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

// Single CTA (1024 threads).  Shared: GW (R*R doubles) + c (R doubles).
__global__ void __launch_bounds__(1024)
k_finalize(float* __restrict__ H, long long In, int R, int N, int n, int next_mode,
           int nblocks, int is_last, int init, SolveState st) {
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
  double* Gn = st.G + (long long)n * R2;
  for (int t = tid; t < R2; t += blockDim.x) {
    const int a = t / R, b = t % R;
    Gn[t] = (c[a] > 0.0 && c[b] > 0.0) ? GW[t] / (c[a] * c[b]) : 0.0;
  }
  for (long long t = tid; t < In * R; t += blockDim.x) {
    const int r = (int)(t % R);
    H[t] = c[r] > 0.0 ? H[t] / (float)c[r] : 0.0f;
  }
  if (is_last) {
    // gamma = lam^T (S * G_N) lam = sum_ab S_ab (W^T W)_ab
    double g = 0.0;
    for (int t = tid; t < R2; t += blockDim.x) g += st.S[t] * GW[t];
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if ((tid & 31) == 0) red[tid >> 5] = g;
    __syncthreads();
    if (tid == 0) {
      double gamma = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gamma += red[w];
      double beta = 0.0;
      for (int b = 0; b < nblocks; ++b) beta += st.gram_part[(long long)b * (R2 + 1) + R2];
      const double alpha = st.scalars[0];
      const double eps = sqrt(fmax(0.0, alpha - 2.0 * beta + gamma) / alpha);
      const double fit = 1.0 - eps;
      st.scalars[1] = beta;
      st.scalars[2] = gamma;
      st.scalars[3] = eps;
      const int it = st.flags[2];
      if (it < kFitCapacity) st.fits[it] = fit;
      st.flags[2] = it + 1;
      const double tol = st.scalars[4];
      if (!isfinite(fit)) {
        st.flags[3] = 1;
        st.flags[0] = 1;
      } else if (it >= 1 && it < kFitCapacity && fabs(fit - st.fits[it - 1]) < tol) {
        st.flags[0] = 1;
      }
    }
  }
  __syncthreads();
  // S for the next mode: Hadamard of every Gram but next_mode's
  if (next_mode >= 0) {
    for (int t = tid; t < R2; t += blockDim.x) {
      double s = 1.0;
      for (int k = 0; k < N; ++k)
        if (k != next_mode) s *= st.G[(long long)k * R2 + t];
      st.S[t] = s;
      st.S32[t] = (float)s;
    }
  }
}

__global__ void k_solve_reset(SolveState st, int R, double tol) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) st.lam[r] = 1.0;
  if (threadIdx.x == 0) {
    st.flags[0] = 0;
    st.flags[1] = 0;
    st.flags[2] = 0;
    st.flags[3] = 0;
    st.scalars[4] = tol;
  }
}

__global__ void k_compute_S(SolveState st, int N, int R, int mode) {
  const int R2 = R * R;
  for (int t = threadIdx.x; t < R2; t += blockDim.x) {
    double s = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != mode) s *= st.G[(long long)k * R2 + t];
    st.S[t] = s;
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
  if (e == cudaSuccess) e = tc_attributes_init();
  return e;
}

int hals_gram_blocks(int64_t In) { return (int)((In + kRowsPerBlock - 1) / kRowsPerBlock); }

cudaError_t launch_hals_gram(float* H, const float* M, int64_t In, int R, SolveState st,
                             cudaStream_t stream) {
  size_t smem = hals_smem(R);
  k_hals_gram<<<hals_gram_blocks(In), kHalsThreads, smem, stream>>>(
      H, M, In, R, st.S32, st.lam, st.gram_part, st.flags, 1);
  return cudaGetLastError();
}

cudaError_t launch_gram_only(const float* H, int64_t In, int R, SolveState st,
                             cudaStream_t stream) {
  size_t smem = hals_smem(R);
  k_hals_gram<<<hals_gram_blocks(In), kHalsThreads, smem, stream>>>(
      const_cast<float*>(H), nullptr, In, R, st.S32, st.lam, st.gram_part, st.flags, 0);
  return cudaGetLastError();
}

cudaError_t launch_finalize(float* H, int64_t In, int R, int N, int n, int next_mode,
                            int nblocks, int is_last, int init, double tol, SolveState st,
                            cudaStream_t stream) {
  (void)tol;
  size_t smem = ((size_t)R * R + R) * sizeof(double);
  k_finalize<<<1, 1024, smem, stream>>>(H, In, R, N, n, next_mode, nblocks, is_last, init, st);
  return cudaGetLastError();
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
