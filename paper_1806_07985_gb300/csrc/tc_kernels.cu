// Root partial MTTKRPs of the dimension tree (Sec. IV-A, Fig. 2a) on the
// 5th-generation tensor cores of sm_103a: tcgen05.mma with TMEM accumulators,
// tensor operands staged by TMA, Khatri-Rao rows formed on the fly in shared
// memory (never written to HBM).
//
// The tensor is viewed as the column-major IL x IR matrix X_(1:s) that its
// memory already is.  Two contractions:
//   contract_fast: out(j, r) = sum_i X[i + IL*j] K(i, r)   (M = IR rows, K = IL)
//   contract_slow: out(i, r) = sum_j X[i + IL*j] K(j, r)   (M = IL rows, K = IR)
// contract_fast tiles (128 output rows x 64 contraction elements per stage)
// arrive K-major from TMA with the 128-byte swizzle; contract_slow tiles arrive
// MN-major (no swizzle).  SPLIT_BF16X3 converter threads read one row of A each
// and write its bf16 hi and lo parts into a ring of A stages in tensor memory
// (tcgen05.st, one TMEM lane per row), from which the MMA takes A; the TMA stage
// is released as soon as it has been read.  The other modes hand A to the MMA
// from shared memory, K-major with the 128-byte swizzle: TF32 K-major tiles
// directly, everything else converted in place (the converted tile has the size
// of its source, so each converter thread reads its share into registers, a
// named barrier separates the reads from the writes, and the result overwrites
// the TMA stage).  Precision modes:
//   TF32         kind::tf32 on the float32 tensor (direct when K-major);
//   SPLIT_BF16X3 x = hi + lo in bf16, K = Khi + Klo: D = [hi*Khi | hi*Klo +
//                lo*Khi] (three products in two float32 TMEM accumulators,
//                added in the epilogue; the large product hi*Khi alone in the
//                first, so fewer additions meet it);
//   BF16_STORED  the tensor is bf16 in HBM: D = X*[Khi|Klo].
//
// Warp roles (16 warps, one CTA per SM, persistent over work units):
//   warp 0      TMA producer          warp 1      TMEM owner + MMA issuer
//   warps 2-7   Khatri-Rao B builders, two per B stage slot (each half of the
//               stage's 64 contraction elements), so three stages are formed
//               concurrently (their factor-row loads are L2 latency)
//   warps 8-15  converters (hi/lo split, transposes); warps 8-11 (8-15 above
//               32 rank columns) also run the epilogue (tcgen05.ld TMEM ->
//               registers -> global); an accumulator is read after the next
//               one's conversions, TMEM holding two.
// Split-BF16x3 accumulates at most kSegStages stages in one TMEM accumulator
// and adds these segments in float32 registers: the tensor core's own
// accumulation does not round to nearest, and over a long chain of
// nonnegative products its bias exceeded the float32-level bound.
// A work unit is one 128-row output tile over one contraction range; when the
// output has fewer tiles than SMs the contraction is split and the per-range
// partials are summed afterwards in a fixed order.
//
// Every mbarrier wait is bounded (about two seconds of clock64): on expiry
// the kernel records an error word, stops issuing work, waits (bounded) for
// its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "../../include/nncp.h"
#include "tc_kernels.cuh"

namespace nncp {

namespace {

constexpr int kKC = 64;  // contraction elements per stage
constexpr int kMaxSF = 8;  // A (TMA) stages: sized at launch from the shared memory left
constexpr int kSB = 3;     // B (Khatri-Rao) stages
constexpr int kThreads = 512;
constexpr int kWarpTMA = 0, kWarpMMA = 1, kWarpB = 2, kWarpConv = 8;
constexpr int kConvThreads = 256;  // two converter threads per row (one per contraction half)
constexpr int kMaxRp = 64;
constexpr long long kWaitCycles = 4000000000LL;

constexpr int kOffsBytes = kSB * kKC * (kMaxModes + 1) * 4;  // B builder row offsets
// barriers: raw full/empty/converted per A stage, B full/empty, acc full/empty x2, drain
// A stages in tensor memory (split-BF16x3), 64 columns each: at most kSA, and
// no more than fit beside the two accumulators (4 Rp columns) in the 512
// columns.  Their full barriers are the conv_full slots, initialised for every
// A stage even where there are fewer TMA stages.  (Six stages, which fit for
// R <= 32, measured slower on the 512^3 root -> left contraction.)
constexpr int kSA = 4;
// split-BF16x3: stages (of kKC contraction elements, four MMAs of hi*Khi
// into the first accumulator each) per tensor-memory accumulation chain;
// see TcParams::seg
#ifndef NNCP_TC_SEG_STAGES
#define NNCP_TC_SEG_STAGES 16
#endif
constexpr int kSegStages = NNCP_TC_SEG_STAGES;
static_assert(kSA <= kMaxSF, "A stages use conv_full barrier slots");
constexpr int kNumBars = 3 * kMaxSF + 2 * kSB + 4 + kSA + 1;
constexpr int kMiscBytes = kNumBars * 8 + 256;
constexpr int kSmemMax = 232448;  // 227 KB per CTA on sm_103a

// Shared-memory carve-up, decided on the host per launch (all offsets 1024-aligned).
struct SmemPlan {
  int raw_bytes, nsf, b_bytes, b_tiles;  // b_tiles: B tiles held (3 ring slots, or all stages)
  int off_raw, off_b, off_offs, off_bar, off_misc, total;
};

struct TcParams {
  int mode;
  int contract_fast;
  int direct;  // MMA reads the TMA stage (no converter)
  int bf16x;   // tensor stored as bf16
  int b_resident;  // every unit spans the whole contraction: B formed once per CTA
  // Stages accumulated in one tensor-memory accumulator before it is added into
  // float32 registers (split-BF16x3; one segment per unit otherwise).  The
  // tensor core adds each MMA's products into the accumulator without
  // rounding to nearest, which biases a long chain of nonnegative terms
  // (measured 2.5e-5 relative over 108 stages of exactly split operands;
  // 1.7e-6 with chains of 16 stages);
  // bounding the chain bounds that bias, and the segments are summed with
  // ordinary float32 adds.
  int seg;
  long long M, K;
  int R, Rp;
  long long n_mt, nsplit, kper, n_units;
  SmemPlan sm;
  KrpDesc krp;
  float* out;
  int* err;
  // Fused first multi-TTV of the output node (leaf_I > 0; Sec. IV-A, Fig. 2b):
  // output rows are node rows (the node's first mode fastest, then its other
  // modes), so tile mt holds rows i_lead in [128 (mt mod nblk), +128) of slice
  // rest = mt / nblk, nblk = leaf_I / 128.  The epilogue adds
  // row(r) * q(rest, r), q the Khatri-Rao row of the node's other modes, into
  // the CTA's partial leaf kept in tensor memory (a CTA's tiles share
  // mt mod nblk because the grid is a multiple of nblk); at the end every CTA
  // writes its partial to leaf_part[blockIdx / nblk][i_lead][r].
  long long leaf_I;
  KrpDesc leaf_krp;
  float* leaf_part;
};

// ------------------------------------------------------------ PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
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

// Bounded wait: false (and the abort flag set) when the wait expires or
// another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicExch(err, 1);
      return false;
    }
  }
}

// OR of `pred` over the `nthreads` threads of named barrier `id` (also a barrier).
__device__ __forceinline__ int bar_red_or(int id, int nthreads, int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(id), "r"(nthreads)
      : "memory");
  return r;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// `policy` is an L2 cache policy (createpolicy): the tensor is read once per
// partial MTTKRP, so its lines are marked evict-first and the streamed half
// gigabyte does not flush what the other kernels of the iteration keep in L2
// (their code, the factors, M, the node temporaries).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); LBO unused for this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // LBO (16 B, ignored)
  d |= (uint64_t)(1024 >> 4) << 32;       // SBO
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor: D float32, A/B type `ab` (1 = bf16 under kind::f16,
// 2 = tf32 under kind::tf32), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab, uint32_t n) {
  return (1u << 4) | (ab << 7) | (ab << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// A operand in tensor memory (lane = row of A, 32-bit column = two bf16
// contraction elements, the lower one in the low half), B in shared memory.
__device__ __forceinline__ void mma_f16_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_st16f(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
               : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                       uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

__device__ __forceinline__ float lds32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t lds16(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
  return v;
}

// Byte address of 16-byte chunk `chunk` of row `row` in a K-major SW128 tile.
__device__ __forceinline__ uint32_t sw128_chunk(uint32_t base, int row, int chunk) {
  return base + row * 128 + (((chunk ^ row) & 7) << 4);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<uint32_t*>(&h);
}

// hi = bf16(x), lo = bf16(x - hi) for 8 values, packed in pairs (x - hi is
// exact in float32, so hi + lo carries about 16 significant bits of x)
__device__ __forceinline__ void split8(const float* x, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
    hi[i] = *reinterpret_cast<const uint32_t*>(&h);
    lo[i] = *reinterpret_cast<const uint32_t*>(&l);
  }
}

struct Unit {
  long long mt, kbeg, kend;
  int nk;
};

__device__ __forceinline__ Unit get_unit(const TcParams& p, long long u) {
  Unit w;
  w.mt = u % p.n_mt;
  const long long kc = u / p.n_mt;
  w.kbeg = kc * p.kper;
  w.kend = min(p.K, w.kbeg + p.kper);
  w.nk = (int)((w.kend - w.kbeg + kKC - 1) / kKC);
  return w;
}

// ------------------------------------------------------------------ kernel --

// LEAF: the fused first multi-TTV (TcParams::leaf_I > 0), a separate
// instantiation so that the plain kernel carries none of its code.  SPLIT:
// the split-BF16x3 precision (A in tensor memory, segmented accumulation),
// separate so that neither form carries the other's registers.
template <bool LEAF, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_partial_mttkrp(const __grid_constant__ CUtensorMap tmap, TcParams p) {
  // Launched in a graph with programmatic serialization, the kernel may start
  // while its predecessor runs: only the B builders (factor rows) and the
  // epilogue (output) touch memory that other kernels of the iteration write or
  // read, so only they wait for it (pdl_wait); the producer streams the tensor,
  // which nothing in the iteration writes, and the converters fill the tensor-
  // memory A stages from it in the meantime.  The kernel does not trigger its
  // successor early: that one is scheduled as CTAs exit, and CTAs placed on the
  // first SMs to free up would crowd there instead of spreading over the GPU.
  extern __shared__ uint8_t smem_dyn[];
  const uint32_t sbase_raw = smem_u32(smem_dyn);
  const uint32_t sbase = (sbase_raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_dyn + (sbase - sbase_raw);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  const int kSF = p.sm.nsf;
  const int kRawBytes = p.sm.raw_bytes;
  const int kBBytes = p.sm.b_bytes;
  const uint32_t raw0 = sbase + p.sm.off_raw;
  const uint32_t b0 = sbase + p.sm.off_b;
  int* offs = reinterpret_cast<int*>(gbase + p.sm.off_offs);  // [kSB][kKC][kMaxModes + 1]
  const uint32_t bar0 = sbase + p.sm.off_bar;
  auto raw_full = [&](int i) { return bar0 + 8u * i; };
  auto raw_empty = [&](int i) { return bar0 + 8u * (kMaxSF + i); };
  auto conv_full = [&](int i) { return bar0 + 8u * (2 * kMaxSF + i); };
  auto b_full = [&](int i) { return bar0 + 8u * (3 * kMaxSF + i); };
  auto b_empty = [&](int i) { return bar0 + 8u * (3 * kMaxSF + kSB + i); };
  auto acc_full = [&](int i) { return bar0 + 8u * (3 * kMaxSF + 2 * kSB + i); };
  auto acc_empty = [&](int i) { return bar0 + 8u * (3 * kMaxSF + 2 * kSB + 2 + i); };
  // split-BF16x3: the converters write A (hi and lo) to tensor memory; conv_full(i)
  // then marks A stage i written, a_empty(i) its MMAs done
  auto a_empty = [&](int i) { return bar0 + 8u * (3 * kMaxSF + 2 * kSB + 4 + i); };
  constexpr bool a_tmem = SPLIT;
  const uint32_t drain_bar = bar0 + 8u * (kNumBars - 1);
  uint8_t* misc = gbase + p.sm.off_bar + kNumBars * 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 8);
  // Khatri-Rao factor descriptors, copied to shared memory for the builders
  const float** kH = reinterpret_cast<const float**>(misc + 64);   // [kMaxModes]
  uint32_t* kdim = reinterpret_cast<uint32_t*>(misc + 128);        // [kMaxModes]

  const int Rp = p.Rp;
  const uint32_t acc_cols = 2u * Rp;  // per accumulator buffer
  const uint32_t a_col0 = 2u * acc_cols;  // A stages (split-BF16x3) after the accumulators
  uint32_t tmem_cols = 32;
  const int nsa = min(kSA, (int)(512u - a_col0) / 64);  // A stages (a_tmem)
  while (tmem_cols < a_col0 + (a_tmem ? 64u * nsa : 0u)) tmem_cols <<= 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kSF; ++i) {
      mbar_init(raw_full(i), 1);
      // split-BF16x3: every converter warp releases the stage once it has read it
      mbar_init(raw_empty(i), a_tmem ? kConvThreads / 32 : 1);
      mbar_init(conv_full(i), kConvThreads / 32);
    }
    // a_tmem: conv_full(i) marks A stage i written (i < nsa), which may exceed kSF
    for (int i = kSF; i < nsa; ++i) mbar_init(conv_full(i), kConvThreads / 32);
    for (int i = 0; i < nsa; ++i) mbar_init(a_empty(i), 1);
    for (int i = 0; i < kSB; ++i) {
      mbar_init(b_full(i), (p.b_resident && i == 0) ? 2 * kSB : 2);
      mbar_init(b_empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(acc_full(i), 1);
      // the epilogue warps (warps 8-11, or 8-15 above 32 rank columns), and
      // with the fused leaf its four warps too
      mbar_init(acc_empty(i), (p.Rp > 32 ? 8 : 4) + (LEAF ? 4 : 0));
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    for (int m = 0; m < kMaxModes; ++m) {
      kH[m] = m < p.krp.nm ? p.krp.H[m] : nullptr;
      kdim[m] = m < p.krp.nm ? (uint32_t)p.krp.dim[m] : 1u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kWarpMMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const long long n_units = p.n_units;
  const int R = p.R;

  if (warp == kWarpTMA) {
    // ---------------------------------------------------------- producer --
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
      int sf = 0;
      uint32_t ph = 0;
      int issued[kMaxSF] = {0, 0, 0, 0, 0, 0, 0, 0};
      const uint32_t tx = p.bf16x ? 16384u : 32768u;
      const uint64_t pol = l2_evict_first_policy();
      bool ok = true;
      for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const Unit w = get_unit(p, u);
        for (int s = 0; s < w.nk; ++s) {
          if (!mbar_wait(raw_empty(sf), ph ^ 1u, abort_flag, p.err)) { ok = false; break; }
          mbar_arrive_tx(raw_full(sf), tx);
          const int k0 = (int)(w.kbeg + (long long)s * kKC);
          const int m0 = (int)(w.mt * 128);
          const uint32_t dst = raw0 + sf * kRawBytes;
          if (p.contract_fast) {
            if (p.bf16x) {
              tma_load_2d(dst, &tmap, k0, m0, raw_full(sf), pol);
            } else {
              tma_load_2d(dst, &tmap, k0, m0, raw_full(sf), pol);
              tma_load_2d(dst + 16384, &tmap, k0 + 32, m0, raw_full(sf), pol);
            }
          } else {
            tma_load_2d(dst, &tmap, m0, k0, raw_full(sf), pol);
          }
          ++issued[sf];
          if (++sf == kSF) { sf = 0; ph ^= 1u; }
        }
      }
      // wait for every copy this thread issued before the CTA can exit
      for (int i = 0; i < kSF; ++i) {
        if (issued[i] == 0) continue;
        const uint32_t par = (uint32_t)((issued[i] - 1) & 1);
        const long long t0 = clock64();
        while (!mbar_test(raw_full(i), par) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == kWarpMMA) {
    // --------------------------------------------------------- MMA issue --
    if (lane == 0) {
      int sa = 0, sb = 0;
      uint32_t pha = 0, phb = 0;
      const int nA = kSF;
      bool ok = true;
      const bool split = p.mode == NNCP_SPLIT_BF16X3;
      const bool tf32 = p.mode == NNCP_TF32;
      const uint32_t idesc_full = tf32 ? make_idesc(2, Rp) : make_idesc(1, 2 * Rp);
      const uint32_t idesc_hi = make_idesc(1, Rp);
      if (p.b_resident && n_units > blockIdx.x && !mbar_wait(b_full(0), 0, abort_flag, p.err))
        ok = false;
      // accumulator segment g (over this CTA's units) uses buffer g & 1
      const int P = SPLIT ? p.seg : (1 << 30);
      long long g = 0;
      for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const Unit w = get_unit(p, u);
        int bsel = 0;
        uint32_t d = tmem_base;
        for (int s = 0, sp = 0; s < w.nk; ++s, sp = (sp + 1 == P) ? 0 : sp + 1) {
          if (sp == 0) {
            bsel = (int)(g & 1);
            if (!mbar_wait(acc_empty(bsel), (uint32_t)(((g >> 1) & 1) ^ 1), abort_flag, p.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d = tmem_base + bsel * acc_cols;
          }
          if constexpr (SPLIT) {
            // A (hi, lo) in tensor memory stage sa, B in shared memory
            if (!mbar_wait(conv_full(sa), pha, abort_flag, p.err) ||
                (!p.b_resident && !mbar_wait(b_full(sb), phb, abort_flag, p.err))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ahi = tmem_base + a_col0 + 64u * sa;
            const uint32_t b = b0 + (p.b_resident ? s : sb) * kBBytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t bd = sw128_desc(b + kk * 32);
              mma_f16_ta(d, ahi + kk * 8, bd, idesc_full, (sp > 0 || kk > 0) ? 1u : 0u);
              mma_f16_ta(d + Rp, ahi + 32 + kk * 8, bd, idesc_hi, 1u);
            }
            mma_commit(a_empty(sa));
            if (!p.b_resident) mma_commit(b_empty(sb));
            if (++sa == nsa) { sa = 0; pha ^= 1u; }
            if (++sb == kSB) { sb = 0; phb ^= 1u; }
          } else {
            const uint32_t afull = p.direct ? raw_full(sa) : conv_full(sa);
            const uint32_t aempty = raw_empty(sa);
            if (!mbar_wait(afull, pha, abort_flag, p.err) ||
                (!p.b_resident && !mbar_wait(b_full(sb), phb, abort_flag, p.err))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a = raw0 + sa * kRawBytes;
            const uint32_t b = b0 + (p.b_resident ? s : sb) * kBBytes;
            if (tf32) {
              // two fp32 sub-tiles of 32 contraction elements, K = 8 per MMA
#pragma unroll
              for (int kk = 0; kk < 8; ++kk) {
                const uint32_t t = kk >> 2, o = (kk & 3) * 32;
                mma_tf32(d, sw128_desc(a + t * 16384 + o), sw128_desc(b + t * Rp * 128 + o),
                         idesc_full, (sp > 0 || kk > 0) ? 1u : 0u);
              }
            } else {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t o = kk * 32;
                mma_f16(d, sw128_desc(a + o), sw128_desc(b + o), idesc_full,
                        (sp > 0 || kk > 0) ? 1u : 0u);
                if (split) mma_f16(d, sw128_desc(a + 16384 + o), sw128_desc(b + o), idesc_hi, 1u);
              }
            }
            mma_commit(aempty);
            if (!p.b_resident) mma_commit(b_empty(sb));
            if (++sa == nA) { sa = 0; pha ^= 1u; }
            if (++sb == kSB) { sb = 0; phb ^= 1u; }
          }
          if (sp == P - 1 || s + 1 == w.nk) {
            mma_commit(acc_full(bsel));
            ++g;
          }
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(drain_bar);
      const long long t0 = clock64();
      while (!mbar_test(drain_bar, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp < kWarpConv) {
    // ---------------------------------------------- Khatri-Rao B builders --
    pdl_wait();
    // Builder warps 2w and 2w+1 form, for every stage t with t % kSB == w,
    // contraction elements [32 h, 32 h + 32) of B slot w (h = warp parity).
    const int bw = (warp - kWarpB) >> 1;
    const int half = (warp - kWarpB) & 1;
    const int nm = p.krp.nm;
    const bool tf32 = p.mode == NNCP_TF32;
    int* so = offs + bw * kKC * (kMaxModes + 1);  // this slot's offsets [kKC][kMaxModes + 1]
    uint32_t bt_base = b0 + bw * kBBytes;
    // the first Khatri-Rao mode spans whole 64-element stages: the other modes'
    // rows are the same for every element of a stage
    const bool lead_aligned = (kdim[0] % kKC) == 0;
    // write rank row rr, elements [32 half, 32 half + 32) of the B tile
    auto store_b_rows = [&](const float* v, int rr) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const float* x8 = v + 8 * g;
        const int kk0 = half * 32 + 8 * g;
        if (tf32) {
          const uint32_t sub = bt_base + (kk0 >> 5) * Rp * 128;
          const int c0 = (kk0 & 31) >> 2;
          sts128(sw128_chunk(sub, rr, c0), __float_as_uint(x8[0]), __float_as_uint(x8[1]),
                 __float_as_uint(x8[2]), __float_as_uint(x8[3]));
          sts128(sw128_chunk(sub, rr, c0 + 1), __float_as_uint(x8[4]), __float_as_uint(x8[5]),
                 __float_as_uint(x8[6]), __float_as_uint(x8[7]));
        } else {
          uint32_t hi[4], lo[4];
          split8(x8, hi, lo);
          const int c = kk0 >> 3;
          sts128(sw128_chunk(bt_base, rr, c), hi[0], hi[1], hi[2], hi[3]);
          sts128(sw128_chunk(bt_base, Rp + rr, c), lo[0], lo[1], lo[2], lo[3]);
        }
      }
    };
    long long t = 0;  // stage counter over this CTA's units
    bool ok = true;
    // resident B: one pass over the whole contraction, tile s into slot s
    const long long n_pass = p.b_resident ? (blockIdx.x < n_units ? 1 : 0) : n_units;
    const uint32_t kd0 = kdim[0];
    for (long long u = blockIdx.x, pass = 0; pass < n_pass && ok; u += gridDim.x, ++pass) {
      Unit w = get_unit(p, p.b_resident ? 0 : u);
      if (p.b_resident) {
        w.kbeg = 0;
        w.kend = p.K;
        w.nk = (int)((p.K + kKC - 1) / kKC);
      }
      if (!p.b_resident && u >= n_units) break;
      // lead-aligned position of this half's first element, kept incrementally:
      // k = kbeg + 64 s + 32 half = lq * kd0 + lk (one 64-bit division per unit)
      const long long kb = w.kbeg + half * 32;
      long long lq = kb / kd0;
      uint32_t lk = (uint32_t)(kb - lq * kd0);
      int ls = 0;                 // stage the position refers to
      long long cst_q = -1;       // slow index the cached constant belongs to
      float cst = 1.0f;
      for (int s = 0; s < w.nk; ++s, ++t) {
        if ((int)(t % kSB) != bw) continue;
        if (p.b_resident) bt_base = b0 + s * kBBytes;
        const long long kst = w.kbeg + (long long)s * kKC + half * 32;  // first element of this half
        // The factor loads of a stage do not depend on the B slot being free, only
        // the stores do: issue the loads, then wait for the slot, then store.
        bool slot_ok = true, waited = p.b_resident;
        auto wait_slot = [&]() {
          if (waited) return;
          waited = true;
          const uint32_t use = (uint32_t)(t / kSB);
          const bool got = mbar_wait(b_empty(bw), (use & 1u) ^ 1u, abort_flag, p.err);
          slot_ok = __all_sync(0xffffffffu, got);
        };
        if (!lead_aligned) {
          // row offsets of the contraction element this lane owns
          const int kk = half * 32 + lane;
          const long long k = kst + lane;
          int* o = so + kk * (kMaxModes + 1);
          const int valid = k < w.kend;
          o[kMaxModes] = valid;
          uint32_t rem = valid ? (uint32_t)k : 0u;
#pragma unroll
          for (int m = 0; m < kMaxModes; ++m) {
            if (m < nm) {
              const uint32_t dm = kdim[m];
              o[m] = (int)((rem % dm) * (uint32_t)R);
              rem /= dm;
            }
          }
          __syncwarp();
        }
        const int iters = (Rp + 31) >> 5;
        for (int it = 0; it < iters; ++it) {
          const int rr = lane + 32 * it;           // rank row of this lane
          const int rs = rr < R ? rr : 0;
          float v[32];
          if (lead_aligned) {
            // modes after the first are constant over the stage:
            // v(e) = H_0(k0 + e, r) * prod_{m>=1} H_m(k_m, r)
            if (it == 0) {
              // advance the position to stage s (64 elements per stage)
              lk += (uint32_t)(s - ls) * kKC;
              ls = s;
              while (lk >= kd0) {
                lk -= kd0;
                ++lq;
              }
            }
            const float* h0 = kH[0] + (long long)lk * R + rs;
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = __ldg(h0 + e * R);
            if (lq != cst_q || iters > 1) {
              long long rem = lq;
              cst = 1.0f;
              for (int m = 1; m < nm; ++m) {
                const uint32_t dm = kdim[m];
                const long long q = rem / dm;
                cst *= __ldg(kH[m] + (uint32_t)(rem - q * dm) * (uint32_t)R + rs);
                rem = q;
              }
              cst_q = lq;
            }
            if (rr < R && kst + 32 <= w.kend) {
#pragma unroll
              for (int e = 0; e < 32; ++e) v[e] *= cst;
            } else {
#pragma unroll
              for (int e = 0; e < 32; ++e)
                v[e] = (rr < R && kst + e < w.kend) ? v[e] * cst : 0.0f;
            }
          } else {
#pragma unroll
            for (int m = 0; m < kMaxModes; ++m) {
              if (m < nm) {
                const float* hb = kH[m] + rs;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                  const float x = __ldg(hb + so[(half * 32 + e) * (kMaxModes + 1) + m]);
                  v[e] = m == 0 ? x : v[e] * x;
                }
              }
            }
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (!(so[(half * 32 + e) * (kMaxModes + 1) + kMaxModes] && rr < R)) v[e] = 0.0f;
          }
          wait_slot();
          if (!slot_ok) break;
          if (rr < Rp) store_b_rows(v, rr);
        }
        if (!slot_ok) {
          ok = false;
          break;
        }
        if (!p.b_resident) {
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(b_full(bw));
        }
      }
    }
    if (p.b_resident && n_pass > 0) {
      // every builder warp has written its tiles: one arrival each on b_full(0)
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_full(0));
    }
    if constexpr (LEAF) {
      if (warp >= 4) {
        // ---------------------------------------- fused leaf multi-TTV --
        // Warps 4-7 (TMEM lane quarters 0-3; idle once the resident B is
        // built) read every unit's accumulator beside the epilogue warps and
        // add row(r) * q(rest, r) into the CTA's partial leaf, one row per
        // thread, in registers; q (the Khatri-Rao row of the tile's slice of
        // the node's other modes, lane l holding column l) is loaded before
        // the accumulator wait.
        const int lq = warp & 3;
        const uint32_t nblk = (uint32_t)(p.leaf_I >> 7);
        float lacc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) lacc[i] = 0.0f;
        // accumulator segments in the order the MMA warp fills them
        const int P = SPLIT ? p.seg : (1 << 30);
        long long g = 0;
        for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
          const Unit w = get_unit(p, u);
          uint32_t rest = (uint32_t)w.mt / nblk;  // the host fuses only below 2^31 tiles
          float qv = lane < R ? 1.0f : 0.0f;
          for (int m = 0; m < p.leaf_krp.nm; ++m) {
            const uint32_t dm = (uint32_t)p.leaf_krp.dim[m];
            const uint32_t qm = rest / dm;
            if (lane < R) qv *= __ldg(p.leaf_krp.H[m] + (size_t)(rest - qm * dm) * R + lane);
            rest = qm;
          }
          const int nseg = (w.nk + P - 1) / P;
          for (int sg = 0; sg < nseg; ++sg, ++g) {
            const int bsel = (int)(g & 1);
            const bool got = mbar_wait(acc_full(bsel), (uint32_t)((g >> 1) & 1), abort_flag, p.err);
            if (!__all_sync(0xffffffffu, got)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(lq * 32) << 16) + bsel * acc_cols;
#pragma unroll
            for (int c = 0; c < 32; c += 16) {
              if (c < Rp) {
                float v[16], v2[16];
                tmem_ld16(tbase + c, v);
                if (p.mode != NNCP_TF32) tmem_ld16(tbase + Rp + c, v2);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const float x = p.mode != NNCP_TF32 ? v[i] + v2[i] : v[i];
                  lacc[c + i] = fmaf(x, __shfl_sync(0xffffffffu, qv, c + i), lacc[c + i]);
                }
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(bsel));
          }
        }
        // this CTA's partial of the leaf: rows [128 (blockIdx mod nblk), +128)
        const long long i_lead = (long long)(blockIdx.x % nblk) * 128 + lq * 32 + lane;
        float* dst = p.leaf_part + ((long long)(blockIdx.x / nblk) * p.leaf_I + i_lead) * R;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < R) dst[i] = lacc[i];
      }
    }
  } else {
    // ---------------------------------------- converters + epilogue --
    const int ct = threadIdx.x - kWarpConv * 32;  // 0..255
    // row m and contraction half kh (elements 32 kh .. 32 kh + 31).  K-major
    // sources: the two halves of a row in lanes l and l + 16 of one warp, eight
    // consecutive rows per quarter-warp (conflict-free 16-byte reads).  MN-major
    // sources: 32 consecutive rows per warp (conflict-free 4-byte reads).
    // (split-BF16x3 writes A to tensor memory: row m must sit in this warp's lane
    // quarter, so 32 consecutive rows per warp for both sources)
    const int m = (p.contract_fast && !a_tmem) ? ((ct >> 5) * 16 + (ct & 15)) : (ct & 127);
    const int kh = (p.contract_fast && !a_tmem) ? ((ct >> 4) & 1) : (ct >> 7);
    const int q = warp & 3;                       // TMEM lane quarter of this warp
    const bool two = p.mode != NNCP_TF32;
    int sf = 0;
    uint32_t phf = 0;
    bool ok = true;
    // Epilogue: warps 8-11 read the rows in their lane quarter (above 32 rank
    // columns warps 12-15 take the second half of the 16-column chunks).  A
    // unit's accumulator arrives in segments of
    // at most P stages (buffer g & 1 for segment g over this CTA's units);
    // each segment is added into float32 registers, and the unit's last one
    // writes the row to global memory.  Segment g is taken once the
    // conversions of segment g + 1 are done (the accumulators being double
    // buffered, the MMAs of g + 1 run meanwhile).
    const int P = SPLIT ? p.seg : (1 << 30);
    const int nch = Rp >> 4;
    const int cgrp = (warp - kWarpConv) >> 2;
    // up to 32 rank columns warps 8-11 hold whole rows and warps 12-15 keep
    // converting meanwhile; above, the two groups share the columns
    const bool epi_all = Rp > 32;
    const bool epi = epi_all || cgrp == 0;
    const int c_lo = (epi_all && cgrp == 1) ? (nch + 1) >> 1 : 0;
    const int c_n = epi_all ? (cgrp == 0 ? (nch + 1) >> 1 : nch >> 1)
                            : (cgrp == 0 ? nch : 0);  // chunks held, at most 2
    float acc[32];
    struct Seg {
      long long mt, kbeg, g;
      int first, last;
    };
    Seg pend;
    pend.g = -1;
    long long gseg = 0;
    auto consume = [&](const Seg& sg) -> bool {
      if (!epi) return true;
      pdl_wait();
      const int bsel = (int)(sg.g & 1);
      const bool got = mbar_wait(acc_full(bsel), (uint32_t)((sg.g >> 1) & 1), abort_flag, p.err);
      if (!__all_sync(0xffffffffu, got)) return false;
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + bsel * acc_cols;
      const long long row = sg.mt * 128 + q * 32 + lane;
      const long long kc = sg.kbeg / p.kper;
      float* dst = p.out + (p.nsplit > 1 ? kc * p.M * R : 0) + row * R;
      const bool store = (!SPLIT || sg.last) && row < p.M;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (j < c_n) {
          const int c = (c_lo + j) * 16;
          float v[16], v2[16];
          tmem_ld16(tbase + c, v);
          if (two) tmem_ld16(tbase + Rp + c, v2);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float x = two ? v[i] + v2[i] : v[i];
            acc[16 * j + i] = (!SPLIT || sg.first) ? x : acc[16 * j + i] + x;
          }
          if (store) {
            if ((R & 3) == 0 && c + 16 <= R) {
              float4* d4 = reinterpret_cast<float4*>(dst + c);
#pragma unroll
              for (int i = 0; i < 4; ++i)
                d4[i] = make_float4(acc[16 * j + 4 * i], acc[16 * j + 4 * i + 1],
                                    acc[16 * j + 4 * i + 2], acc[16 * j + 4 * i + 3]);
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (c + i < R) dst[c + i] = acc[16 * j + i];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(bsel));
      return true;
    };
    int sa = 0;
    uint32_t pha = 0;
    for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const Unit w = get_unit(p, u);
      for (int s = 0, sp = 0; s < w.nk && SPLIT; ++s, ++sp) {
        // wait for the TMA stage and the tensor-memory A stage, then, eight
        // elements of row m (half kh) at a time, read, split into hi + lo and
        // write both to A stage sa; release the TMA stage after the last read
        bool got = mbar_wait(raw_full(sf), phf, abort_flag, p.err);
        got = got && mbar_wait(a_empty(sa), pha ^ 1u, abort_flag, p.err);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = raw0 + sf * kRawBytes;
        const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + a_col0 + 64u * sa + 16u * kh;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          float x[8];
          if (p.contract_fast) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const float4 a = lds128(sw128_chunk(st + kh * 16384, m, 2 * g + c));
              x[4 * c] = a.x; x[4 * c + 1] = a.y; x[4 * c + 2] = a.z; x[4 * c + 3] = a.w;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = lds32(st + (32 * kh + 8 * g + e) * 512 + m * 4);
          }
          uint32_t hi[4], lo[4];
          split8(x, hi, lo);
          tmem_st4(ta + 4 * g, hi);
          tmem_st4(ta + 32 + 4 * g, lo);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(raw_empty(sf));
        if (++sf == kSF) { sf = 0; phf ^= 1u; }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(conv_full(sa));
        if (++sa == nsa) { sa = 0; pha ^= 1u; }
        if (sp + 1 == P || s + 1 == w.nk) {
          if (pend.g >= 0 && !consume(pend)) {
            ok = false;
            break;
          }
          pend = Seg{w.mt, w.kbeg, gseg++, s < P, s + 1 == w.nk};
          sp = -1;
        }
      }
      for (int s = 0; s < w.nk && !p.direct && !SPLIT; ++s) {
        const bool got = mbar_wait(raw_full(sf), phf, abort_flag, p.err);
        const uint32_t st = raw0 + sf * kRawBytes;
        // read phase: this thread's 32 source elements of row m, half kh
        float x[32];
        if (got) {
          if (p.mode == NNCP_BF16_STORED) {
            // MN-major bf16 source: row j holds 128 consecutive i (256 B)
#pragma unroll
            for (int e = 0; e < 32; ++e)
              x[e] = __uint_as_float(lds16(st + (32 * kh + e) * 256 + m * 2));
          } else if (p.contract_fast) {
            // K-major fp32 source: sub-tile kh, row m, its 8 chunks
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const float4 a = lds128(sw128_chunk(st + kh * 16384, m, c));
              x[4 * c] = a.x; x[4 * c + 1] = a.y; x[4 * c + 2] = a.z; x[4 * c + 3] = a.w;
            }
          } else {
            // MN-major fp32 source: row j holds 128 consecutive i (512 B)
#pragma unroll
            for (int e = 0; e < 32; ++e) x[e] = lds32(st + (32 * kh + e) * 512 + m * 4);
          }
        }
        // In place: every element is read before any is overwritten.  A K-major
        // source row m is overwritten only by row m's own output, whose two halves
        // sit in this warp; an MN-major source row is spread over all output rows,
        // so the whole converter group must have read first.
        if (p.contract_fast) {
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
        } else if (bar_red_or(2, kConvThreads, !got)) {
          ok = false;
          break;
        }
        if (p.mode == NNCP_SPLIT_BF16X3) {
          // hi tile at +0, lo tile at +16 KB; chunks 4 kh .. 4 kh + 3 of row m
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            uint32_t hi[4], lo[4];
            split8(x + 8 * g, hi, lo);
            sts128(sw128_chunk(st, m, 4 * kh + g), hi[0], hi[1], hi[2], hi[3]);
            sts128(sw128_chunk(st + 16384, m, 4 * kh + g), lo[0], lo[1], lo[2], lo[3]);
          }
        } else if (p.mode == NNCP_TF32) {
          // K-major fp32: sub-tile kh, chunks 0..7 of row m
#pragma unroll
          for (int c = 0; c < 8; ++c)
            sts128(sw128_chunk(st + kh * 16384, m, c), __float_as_uint(x[4 * c]),
                   __float_as_uint(x[4 * c + 1]), __float_as_uint(x[4 * c + 2]),
                   __float_as_uint(x[4 * c + 3]));
        } else {
          // K-major bf16: chunks 4 kh .. 4 kh + 3 of row m
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            uint32_t w4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              w4[e] = (__float_as_uint(x[8 * g + 2 * e]) & 0xFFFFu) |
                      (__float_as_uint(x[8 * g + 2 * e + 1]) << 16);
            sts128(sw128_chunk(st, m, 4 * kh + g), w4[0], w4[1], w4[2], w4[3]);
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(conv_full(sf));
        if (++sf == kSF) { sf = 0; phf ^= 1u; }
      }
      if (!SPLIT && ok) {
        // one segment per unit
        if (pend.g >= 0 && !consume(pend)) ok = false;
        pend = Seg{w.mt, w.kbeg, gseg++, 1, 1};
      }
      // every converter warp reaches this barrier once per unit, whether or not
      // its stage loop ended early, so all of them take the same exit decision
      if (bar_red_or(2, kConvThreads, !ok)) { ok = false; break; }
    }
    if (ok && pend.g >= 0) consume(pend);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kWarpMMA) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ----------------------------------------------------------------- host --

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool load_encode() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

struct Plan {
  long long M, K, n_mt, nsplit, kper, n_units;
  int Rp;
};

Plan plan_for(int contract_fast, int64_t IL, int64_t IR, int R, int num_sms) {
  Plan pl;
  pl.M = contract_fast ? IR : IL;
  pl.K = contract_fast ? IL : IR;
  pl.Rp = ((R + 15) / 16) * 16;
  pl.n_mt = (pl.M + 127) / 128;
  const long long kchunks = (pl.K + kKC - 1) / kKC;
  long long ns = 1;
  if (pl.n_mt < num_sms) ns = std::max(1LL, std::min(kchunks, (long long)num_sms / pl.n_mt));
  pl.kper = ((kchunks + ns - 1) / ns) * kKC;
  pl.nsplit = (pl.K + pl.kper - 1) / pl.kper;
  pl.n_units = pl.n_mt * pl.nsplit;
  return pl;
}

int align1k(int v) { return (v + 1023) & ~1023; }

// B tiles resident when every unit spans the whole contraction and they fit
// beside at least kMinSFResident TMA stages.
constexpr int kMinSFResident = 4;

SmemPlan plan_smem(int precision, int contract_fast, int direct, int bf16x, int Rp,
                   long long K, long long nsplit, int* b_resident) {
  SmemPlan sm;
  sm.raw_bytes = bf16x ? 16384 : 32768;
  sm.b_bytes = align1k(2 * Rp * 128);
  const int fixed = 1024 /* alignment slack */ + align1k(kOffsBytes) + align1k(kMiscBytes);
  const long long nk_total = (K + kKC - 1) / kKC;
  const bool res = nsplit == 1 &&
                   nk_total * sm.b_bytes + (long long)kMinSFResident * sm.raw_bytes + fixed <= kSmemMax;
  *b_resident = res;
  sm.b_tiles = res ? (int)nk_total : kSB;
  const int avail = kSmemMax - fixed - sm.b_tiles * sm.b_bytes;
  sm.nsf = std::min(kMaxSF, avail / sm.raw_bytes);
  sm.off_raw = 0;
  sm.off_b = sm.off_raw + sm.nsf * sm.raw_bytes;
  sm.off_offs = sm.off_b + sm.b_tiles * sm.b_bytes;
  sm.off_bar = sm.off_offs + align1k(kOffsBytes);
  sm.off_misc = sm.off_bar;
  sm.total = sm.off_bar + align1k(kMiscBytes) + 1024;
  (void)contract_fast;
  (void)direct;
  (void)precision;
  return sm;
}

int64_t prod_range(const int64_t* d, int a, int b) {
  int64_t p = 1;
  for (int m = a; m <= b; ++m) p *= d[m];
  return p;
}

}  // namespace

bool tc_available() { return true; }

const char* tc_unsupported_reason(int precision, int N, const int64_t* dims, int R, int split) {
  if (precision != NNCP_TF32 && precision != NNCP_SPLIT_BF16X3 && precision != NNCP_BF16_STORED)
    return "not a tensor-core precision";
  if (R > kMaxRp) return "tensor-core partial MTTKRP supports R <= 64";
  const int64_t IL = prod_range(dims, 0, split - 1);
  const int64_t esz = precision == NNCP_BF16_STORED ? 2 : 4;
  if ((IL * esz) % 16 != 0)
    return "tensor-core partial MTTKRP needs I_1*...*I_s * element size to be a multiple of 16 bytes";
  const int64_t IR = prod_range(dims, split, N - 1);
  if (IL >= (1LL << 31) || IR >= (1LL << 31)) return "matricization too large for TMA coordinates";
  return nullptr;
}

size_t tc_scratch_bytes(int N, const int64_t* dims, int R, int split, int precision, int num_sms) {
  if (precision == NNCP_FP32_SIMT) return 0;
  const int64_t IL = prod_range(dims, 0, split - 1), IR = prod_range(dims, split, N - 1);
  size_t need = 0;
  for (int cf = 0; cf < 2; ++cf) {
    Plan pl = plan_for(cf, IL, IR, R, num_sms);
    if (pl.nsplit > 1) need = std::max<size_t>(need, (size_t)pl.nsplit * pl.M * R * sizeof(float));
  }
  // fused leaf partials: 128 rows per CTA
  need = std::max<size_t>(need, (size_t)num_sms * 128 * R * sizeof(float));
  return 256 + need;
}

// grid of a fused-leaf launch: a multiple of the leaf's 128-row blocks
static int leaf_grid(const Plan& pl, int64_t leaf_I, int num_sms) {
  const int nblk = (int)(leaf_I / 128);
  const int g = num_sms - num_sms % nblk;
  return (int)std::min<long long>(g, pl.n_units);
}

bool tc_leaf_ok(int precision, int contract_fast, int64_t IL, int64_t IR, int R, int64_t leaf_I,
                int num_sms) {
  // the leaf runs on builder warps that are idle once a resident B is built:
  // the contract-fast (root -> right) kernel, up to 32 rank columns
  if (precision == NNCP_FP32_SIMT || !contract_fast || leaf_I <= 0 || leaf_I % 128 != 0 || R > 32)
    return false;
  const Plan pl = plan_for(contract_fast, IL, IR, R, num_sms);
  if (pl.nsplit != 1 || pl.M % leaf_I != 0 || leaf_I / 128 > num_sms || pl.n_mt >= (1LL << 31))
    return false;
  const bool bf16x = precision == NNCP_BF16_STORED;
  const bool direct = precision != NNCP_SPLIT_BF16X3;
  int resident = 0;
  plan_smem(precision, contract_fast, direct, bf16x, pl.Rp, pl.K, pl.nsplit, &resident);
  if (!resident) return false;
  const int g = leaf_grid(pl, leaf_I, num_sms);
  return g >= 1 && g % (leaf_I / 128) == 0;
}

int* tc_error_word(const TcScratch& s) { return static_cast<int*>(s.base); }

cudaError_t tc_attributes_init() {
  void (*const ks[4])(CUtensorMap, TcParams) = {
      k_tc_partial_mttkrp<false, false>, k_tc_partial_mttkrp<false, true>,
      k_tc_partial_mttkrp<true, false>, k_tc_partial_mttkrp<true, true>};
  for (auto k : ks) {
    const cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t tc_partial_mttkrp(int precision, int contract_fast, const void* X, int64_t IL,
                              int64_t IR, const KrpDesc& K, int R, float* out,
                              const TcScratch& scratch, int num_sms, cudaStream_t st,
                              const TcLeaf* leaf) {
  if (!load_encode()) return cudaErrorNotSupported;
  if (R > kMaxRp || !scratch.base) return cudaErrorInvalidValue;
  const bool bf16x = precision == NNCP_BF16_STORED;
  const int esz = bf16x ? 2 : 4;
  if ((IL * esz) % 16 != 0) return cudaErrorInvalidValue;
  Plan pl = plan_for(contract_fast, IL, IR, R, num_sms);

  CUtensorMap map;
  memset(&map, 0, sizeof map);
  cuuint64_t gdim[2] = {(cuuint64_t)IL, (cuuint64_t)IR};
  cuuint64_t gstride[1] = {(cuuint64_t)IL * esz};
  cuuint32_t box[2];
  CUtensorMapSwizzle swz;
  if (contract_fast) {
    box[0] = bf16x ? 64 : 32;  // 128 bytes of contraction elements
    box[1] = 128;              // output rows
    swz = CU_TENSOR_MAP_SWIZZLE_128B;
  } else {
    box[0] = 128;              // output rows (contiguous)
    box[1] = kKC;              // contraction elements
    swz = CU_TENSOR_MAP_SWIZZLE_NONE;
  }
  cuuint32_t estride[2] = {1, 1};
  CUresult r = g_encode(&map, bf16x ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        2, const_cast<void*>(X), gdim, gstride, box, estride,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;

  TcParams p;
  memset(&p, 0, sizeof p);
  p.mode = precision;
  p.contract_fast = contract_fast;
  p.bf16x = bf16x;
  p.direct = contract_fast && precision != NNCP_SPLIT_BF16X3;
  p.seg = precision == NNCP_SPLIT_BF16X3 ? kSegStages : (1 << 30);
  p.M = pl.M;
  p.K = pl.K;
  p.R = R;
  p.Rp = pl.Rp;
  p.n_mt = pl.n_mt;
  p.nsplit = pl.nsplit;
  p.kper = pl.kper;
  p.n_units = pl.n_units;
  p.krp = K;
  p.err = tc_error_word(scratch);
  float* partials = reinterpret_cast<float*>(static_cast<char*>(scratch.base) + 256);
  p.out = pl.nsplit > 1 ? partials : out;
  if (pl.nsplit > 1 && 256 + (size_t)pl.nsplit * pl.M * R * sizeof(float) > scratch.bytes)
    return cudaErrorInvalidValue;

  p.sm = plan_smem(precision, contract_fast, p.direct, bf16x, pl.Rp, pl.K, pl.nsplit, &p.b_resident);
  if (p.sm.nsf < 2) return cudaErrorInvalidValue;
  int grid = (int)std::min<long long>(pl.n_units, num_sms);
  if (leaf) {
    if (!tc_leaf_ok(precision, contract_fast, IL, IR, R, leaf->I, num_sms) || !leaf->out)
      return cudaErrorInvalidValue;
    grid = leaf_grid(pl, leaf->I, num_sms);
    p.leaf_I = leaf->I;
    p.leaf_krp = leaf->rest;
    p.leaf_part = partials;
    if (256 + (size_t)grid * 128 * R * sizeof(float) > scratch.bytes) return cudaErrorInvalidValue;
  }
  const bool split = precision == NNCP_SPLIT_BF16X3;
  void (*const kern)(CUtensorMap, TcParams) =
      leaf ? (split ? k_tc_partial_mttkrp<true, true> : k_tc_partial_mttkrp<true, false>)
           : (split ? k_tc_partial_mttkrp<false, true> : k_tc_partial_mttkrp<false, false>);
  cudaError_t e = launch_kernel(kern, dim3(grid), dim3(kThreads), p.sm.total, st, map, p);
  if (e != cudaSuccess) return e;
  if (leaf) {
    // the CTAs' partial leaves, summed in CTA order
    const int nblk = (int)(leaf->I / 128);
    return launch_reduce_chunks(partials, leaf->I * R, grid / nblk, leaf->out, num_sms, st);
  }
  if (pl.nsplit == 1) return e;
  return launch_reduce_chunks(partials, pl.M * R, (int)pl.nsplit, out, num_sms, st);
}

}  // namespace nncp

// ------------------------------------------------------------ peak probes --
// Throughput probes that give the roofline fractions of the compute-bound
// paths a measured denominator: float32 FFMA on the CUDA cores, and dense
// tcgen05 MMAs (kind::tf32 and kind::f16 bf16, M = 128, N = 256, operands in
// shared memory, accumulator in tensor memory), one CTA per SM.  The caller
// times the launch with events on the stream.

namespace nncp {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads)
k_probe_ffma(int reps, float seed, float* sink) {
  float a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.999999f, b = 1e-7f;
#pragma unroll 1
  for (int i = 0; i < reps; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) a[c] = fmaf(a[c], m, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += a[c];
  if (s == 12345.678f) sink[0] = s;  // keeps the chains live
}

// The same with packed pairs: fma.rn.f32x2 performs two float32 FMAs (each
// rounded to nearest, as fmaf) per instruction.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__global__ void __launch_bounds__(kProbeThreads)
k_probe_ffma2(int reps, float seed, float* sink) {
  unsigned long long a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) {
    const float2 v = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
    a[c] = *reinterpret_cast<const unsigned long long*>(&v);
  }
  const float2 mv = make_float2(0.999999f, 0.999998f), bv = make_float2(1e-7f, 2e-7f);
  const unsigned long long m = *reinterpret_cast<const unsigned long long*>(&mv);
  const unsigned long long b = *reinterpret_cast<const unsigned long long*>(&bv);
#pragma unroll 1
  for (int i = 0; i < reps; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) a[c] = ffma2(a[c], m, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) {
    const float2 v = *reinterpret_cast<const float2*>(&a[c]);
    s += v.x + v.y;
  }
  if (s == 12345.678f) sink[0] = s;  // keeps the chains live
}

// One elected thread issues `reps` x 4 MMAs of M = 128, N = 256 into one
// tensor-memory accumulator from zero-filled shared-memory operands.
template <bool TF32>
__global__ void __launch_bounds__(128, 1) k_probe_mma(int reps, int* err) {
  extern __shared__ uint8_t psm[];
  const uint32_t raw = smem_u32(psm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* g = psm + (base - raw);
  const uint32_t a0 = base, b0 = base + 16384;           // A 128 x 128 B, B 256 x 128 B
  const uint32_t bar = base + 16384 + 32768;
  uint32_t* slot = reinterpret_cast<uint32_t*>(g + 16384 + 32768 + 64);
  for (int i = threadIdx.x; i < (16384 + 32768) / 16; i += blockDim.x)
    sts128(base + 16 * i, 0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, 256u);
    for (int i = 0; i < reps; ++i) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = sw128_desc(a0 + kk * 32), bd = sw128_desc(b0 + kk * 32);
        if (TF32)
          mma_tf32(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        else
          mma_f16(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      }
    }
    mma_commit(bar);
    const long long t0 = clock64();
    bool done = false;
    while (!(done = mbar_test(bar, 0)) && clock64() - t0 < kWaitCycles) {
    }
    if (!done) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                 : "memory");
  }
}

}  // namespace
}  // namespace nncp

extern "C" nncp_status nncp_peak_probe(int kind, int reps, void* sink_dev, void* stream,
                                       double* flops_out) {
  using namespace nncp;
  if (reps < 1 || reps > (1 << 24) || !flops_out || !sink_dev ||
      (reinterpret_cast<uintptr_t>(sink_dev) & 15)) {
    record_global_error("nncp_peak_probe: reps in [1, 2^24], flops_out and a 16-byte aligned sink");
    return NNCP_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    record_global_error("nncp_peak_probe: no device");
    return NNCP_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (kind == 0) {
    const int blocks = sms * 8;  // 2048 threads per SM
    e = launch_kernel(k_probe_ffma, dim3(blocks), dim3(kProbeThreads), 0, st, reps, 1.0f,
                      static_cast<float*>(sink_dev));
    *flops_out = 2.0 * kProbeChains * 16 * (double)reps * blocks * kProbeThreads;
  } else if (kind == 3) {
    const int blocks = sms * 8;
    e = launch_kernel(k_probe_ffma2, dim3(blocks), dim3(kProbeThreads), 0, st, reps, 1.0f,
                      static_cast<float*>(sink_dev));
    *flops_out = 4.0 * kProbeChains * 16 * (double)reps * blocks * kProbeThreads;
  } else if (kind == 1 || kind == 2) {
    const int smem = 1024 + 16384 + 32768 + 128;
    auto k = kind == 1 ? k_probe_mma<true> : k_probe_mma<false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = launch_kernel(k, dim3(sms), dim3(128), smem, st, reps, static_cast<int*>(sink_dev));
    // K per MMA: 8 (tf32) or 16 (bf16) elements of a 32-byte step
    *flops_out = 2.0 * 128 * 256 * (kind == 1 ? 8 : 16) * 4.0 * reps * sms;
  } else {
    record_global_error("nncp_peak_probe: kind must be 0 (FFMA), 1 (TF32 MMA), 2 (BF16 MMA) or 3 (packed FFMA2)");
    return NNCP_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) {
    record_global_error(cudaGetErrorString(e));
    return NNCP_ERR_CUDA;
  }
  return NNCP_OK;
}
