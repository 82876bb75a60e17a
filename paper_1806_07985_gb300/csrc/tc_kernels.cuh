// Tensor-core (tcgen05 / TMEM / TMA) partial MTTKRP kernels for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nncp_internal.cuh"

namespace nncp {

// Device scratch owned by the caller's workspace (split-K partials, packed
// Khatri-Rao operands).
struct TcScratch {
  void* base;
  size_t bytes;
};

// True when the tcgen05 kernels are compiled in.
bool tc_available();

// NULL when `precision` can run the root partial MTTKRPs of this shape with
// tensor cores; otherwise a reason.
const char* tc_unsupported_reason(int precision, int N, const int64_t* dims, int R, int split);

// Device word the tensor-core kernels set to 1 when a bounded wait expired.
int* tc_error_word(const TcScratch& s);

size_t tc_scratch_bytes(int N, const int64_t* dims, int R, int split, int precision, int num_sms);

// The first multi-TTV out of the output node, fused into the partial MTTKRP
// (Sec. IV-A, Fig. 2b): the node's rows are (I = size of its first mode,
// fastest) x (its other modes); out_leaf(i, r) = sum_rest node(i + I*rest, r) *
// rest_krp(rest, r), the same contraction as the leaf multi-TTV, whose factors
// are final before the partial MTTKRP runs.
struct TcLeaf {
  int64_t I;
  KrpDesc rest;
  float* out;  // I x R
};

// True when tc_partial_mttkrp can fuse a leaf with first-mode size leaf_I
// (a multiple of 128; no split contraction; tensor-memory columns free).
bool tc_leaf_ok(int precision, int contract_fast, int64_t IL, int64_t IR, int R, int64_t leaf_I,
                int num_sms);

// Root partial MTTKRP on tensor cores.  X viewed as the column-major
// IL x IR matrix X_(1:s) (no reordering, Sec. IV-A):
//   contract_fast = 1:  out(j, r) = sum_i X[i + IL*j] * K(i, r)   (root -> right node)
//   contract_fast = 0:  out(i, r) = sum_j X[i + IL*j] * K(j, r)   (root -> left node)
// K is the Khatri-Rao product described by `K` (formed on the fly).  With
// `leaf` (tc_leaf_ok), leaf->out receives the fused first multi-TTV as well.
cudaError_t tc_partial_mttkrp(int precision, int contract_fast, const void* X, int64_t IL,
                              int64_t IR, const KrpDesc& K, int R, float* out,
                              const TcScratch& scratch, int num_sms, cudaStream_t st,
                              const TcLeaf* leaf = nullptr);

}  // namespace nncp
