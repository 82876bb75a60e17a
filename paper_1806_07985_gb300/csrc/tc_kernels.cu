#include "tc_kernels.cuh"

namespace nncp {

bool tc_available() { return false; }

const char* tc_unsupported_reason(int, int, const int64_t*, int, int) {
  return "tensor-core partial MTTKRP not built";
}

size_t tc_scratch_bytes(int, const int64_t*, int, int, int, int) { return 0; }

cudaError_t tc_partial_mttkrp(int, int, const void*, int64_t, int64_t, const KrpDesc&, int,
                              float*, const TcScratch&, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t tc_attributes_init() { return cudaSuccess; }

}  // namespace nncp
