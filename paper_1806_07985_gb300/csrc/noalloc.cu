// nncp_mttkrp_noalloc: the direct MTTKRP with its split-K scratch in a
// file-scope __device__ array, for callers that cannot allocate device memory.
// Nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/nncp.h"
#include "nncp_internal.cuh"

using namespace nncp;

namespace {

constexpr size_t kScratchFloats = NNCP_NOALLOC_SCRATCH_FLOATS;  // 8 MiB of float32
constexpr int kMaxDevices = 64;

// Split-K partial sums of every nncp_mttkrp_noalloc call on this device.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

struct DeviceSlot {
  float* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
};
std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

nncp_status reject(nncp_status s, const char* fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, a, b);
  record_global_error(buf);
  return s;
}

// Set-up, once per device, with that device current: the host-side name of
// the array is only a stand-in, so its device address is looked up here.
nncp_status device_slot(DeviceSlot* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(NNCP_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return reject(NNCP_ERR_UNSUPPORTED, "device %lld out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSlot& s = g_slots[dev];
  if (!s.scratch) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return reject(NNCP_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return reject(NNCP_ERR_CUDA, "cudaDeviceGetAttribute failed");
    s.num_sms = sms;
    s.scratch = static_cast<float*>(p);
  }
  *out = s;
  return NNCP_OK;
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

extern "C" nncp_status nncp_mttkrp_noalloc(int N, const int64_t* dims, int R, const float* X_dev,
                                           const float* const* H_dev, int mode, float* M_dev,
                                           void* stream) {
  if (N < 2 || N > kMaxModes || !dims) return reject(NNCP_ERR_INVALID_ARG, "N=%lld not in [2,8]", N);
  if (R < 1 || R > kMaxRank) return reject(NNCP_ERR_INVALID_ARG, "R=%lld not in [1,128]", R);
  if (mode < 1 || mode > N) return reject(NNCP_ERR_INVALID_ARG, "mode %lld not in [1,N]", mode);
  if (!aligned16(X_dev) || !aligned16(M_dev) || !H_dev)
    return reject(NNCP_ERR_INVALID_ARG, "X, M and H must be 16-byte aligned device pointers");
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1) return reject(NNCP_ERR_INVALID_ARG, "dims[%lld] < 1", n);
    if (!aligned16(H_dev[n])) return reject(NNCP_ERR_INVALID_ARG, "factor %lld is not aligned", n + 1);
  }
  const int n = mode - 1;
  const long long rows = dims[n];
  if ((size_t)rows * R * 2 > kScratchFloats)
    return reject(NNCP_ERR_INVALID_ARG,
                  "I_mode*R = %lld exceeds the no-alloc limit of %lld (NNCP_NOALLOC_SCRATCH_FLOATS/2)",
                  rows * R, (long long)(kScratchFloats / 2));
  DeviceSlot slot;
  nncp_status s = device_slot(&slot);
  if (s != NNCP_OK) return s;

  KrpDesc KL, KQ;
  memset(&KL, 0, sizeof KL);
  memset(&KQ, 0, sizeof KQ);
  int64_t L = 1, Q = 1;
  for (int m = 0; m < n; ++m) {
    KL.dim[KL.nm] = dims[m];
    KL.H[KL.nm++] = H_dev[m];
    L *= dims[m];
  }
  for (int m = n + 1; m < N; ++m) {
    KQ.dim[KQ.nm] = dims[m];
    KQ.H[KQ.nm++] = H_dev[m];
    Q *= dims[m];
  }
  cudaError_t e = launch_simt_mttkrp_capped(X_dev, L, rows, Q, KL, KQ, R, M_dev, slot.scratch,
                                            kScratchFloats, slot.num_sms,
                                            static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    record_global_error(cudaGetErrorString(e));
    return NNCP_ERR_CUDA;
  }
  return NNCP_OK;
}
