// a6-a7 on the 5th-generation tensor cores: one network layer as a persistent GEMM,
//   out[r, c] = act(scale[c] * sum_k A[r, k] W[c, k] + bias[c]),
// with A (activations, K-major) and W (weights [N x K], K-major) streamed into shared memory
// by TMA (128-byte swizzle), multiplied by tcgen05.mma (kind::f16 for BF16, kind::f8f6f4 for
// FP8 e4m3) into FP32 accumulators in tensor memory, and read back by tcgen05.ld for a fused
// epilogue (per-channel scale, bias, tanh-GELU of Sec. 3.3.2, quantisation of the next
// layer's input). The paper's double buffering of batch k against batch k+1 (Sec. 3.3.3)
// becomes a multi-stage TMA ring and two TMEM accumulators, so the epilogue of one tile
// overlaps the MMAs of the next.
//
// Warp roles (64 + 128 E threads for E epilogue warps per TMEM lane quarter: 704 with E = 5 on
// single-CTA layers with an activation, 448 with E = 3 otherwise; one CTA per SM):
//   warp 0      TMA producer (one lane)
//   warp 1      TMEM allocator and MMA issuer (one lane)
//   warps 2..   epilogue; warp w reads TMEM lanes 32*(w%4) .. 32*(w%4)+31 and every E-th
//               32-column chunk; results go through swizzled shared-memory staging and leave
//               by TMA tensor stores
// A layer may instead run on CTA pairs (clusters of two, cta_group::2): 256-row tiles whose
// MMAs the even CTA issues over both CTAs' operands (see "CTA pairs" below).
// Every mbarrier wait is bounded by a clock budget; on expiry the CTA sets the error word,
// drains its own copies and MMAs, frees its TMEM and returns. The budget of the pipeline waits
// is a launch argument (default ~1 s); the drains on the way out always allow the full ~1 s,
// so copies and MMAs in flight land before the CTA frees its tensor memory and exits.
#include "dfgb_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <string.h>
#include <stdio.h>

#include <type_traits>

namespace dfgb {
namespace {

constexpr int BM = 128;
constexpr int kRowBytes = 128;                 // K bytes per stage row (one swizzle span)
__host__ __device__ constexpr int threads_for(int epq) { return 64 + 128 * epq; }
constexpr long long kWaitBudget = 2000000000LL;  // ~1 s of SM clocks per wait
constexpr int kSmemLimit = 232448;             // opt-in dynamic shared memory per block
constexpr uint32_t kSuspendNs = 200000;        // try_wait may park the thread this long

struct TcArgs {
  RowMap rows;
  int N, K;
  const float* bias;
  const float* col_scale;
  void* out;
  int64_t ldo;
  int out_kind;
  int gelu;
  float out_scale;
  int* err;
  void* gbuf;      // GELU'(z): written (kModeStoreG) or read as the row-group scale (kModeRowG)
  int64_t ldg;
  int ntan;        // rows per group for kModeRowG
  const float4* gtab;  // tabulated GELU, or NULL for the tanh form
  int ksplit;      // split-K: partial products over ksplit ranges of k-blocks
  int64_t split_rows;  // output row offset between the partial products of two splits
  long long budget;    // clock budget of each pipeline wait (kWaitBudget by default)
  uint32_t suspend;    // try_wait suspend-time hint, ns (short when the budget is short)
};

// Epilogue modes: plain layer; layer that also stores GELU'(z) (forward pass of the Jacobian);
// tangent layer out[r, c] = acc[r, c] * G[r / ntan, c] (no bias, no activation).
constexpr int kModePlain = 0, kModeStoreG = 1, kModeRowG = 2;

// Epilogue activation: none (read-out, tangent and gradient GEMMs), the tanh form with the
// hardware tanh, or the paper's table (compiled for BF16 hidden layers only).
constexpr int kActNone = 0, kActTanh = 1, kActTable = 2;

// Epilogue warps per TMEM lane quarter. Single-CTA layers with an activation (the
// epilogue-bound layers of one k-block among them) take five, each loading one 32-column chunk
// from tensor memory at a time; pair tiles, the read-out and the layers that also store GELU'
// (whose second store per chunk needs the registers that more warps would not leave) take
// three, each loading the next chunk while it stores the current one. Measured on 2^20 rows of
// the 32 -> 1600 layer: 0.83 ms with three per quarter (192-wide tiles), 0.61 ms with four
// (256-wide), 0.60 ms with five (160-wide, one chunk per warp); on the CTA-pair 1600 -> 800
// layer four were 2 % slower than three.
__host__ __device__ constexpr int epi_per_quarter(bool pair, int act, int mode = 0) {
  return !pair && act != kActNone && mode != kModeStoreG ? 5 : 3;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity,
                                         uint32_t suspend = kSuspendNs) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(suspend)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase of the given parity completed; false after the clock
// budget or once another role of the CTA has given up (*abort set).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          int* err, long long budget, uint32_t suspend) {
  if (mbar_try(bar, parity, suspend)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity, suspend)) return true;
    if (*abort) return false;
    if (clock64() - t0 > budget) {
      atomicOr(err, kErrTimeout);
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B
// apart (stride byte offset), leading byte offset unused for this layout, version 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128 (256 for a CTA pair),
// N = BN (N / 8 in bits 17..22; BN = 0 leaves the field for a width chosen at run time).
template <bool FP8, int BN, int MROWS = BM>
__device__ constexpr uint32_t idesc() {
  return (1u << 4) | (FP8 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(MROWS >> 4) << 24);
}

template <bool FP8>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id,
                                          uint32_t accum) {
  if (FP8) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// ---- CTA pairs (cta_group::2) ----
// Two CTAs of a cluster compute one 256-row tile: each holds its own 128 rows of A and half of
// the tile's BN rows of W in shared memory, the even CTA issues M = 256 MMAs that read both
// CTAs' operands and write each CTA's 128 accumulator rows into that CTA's tensor memory. Each
// SM then streams 128 + BN/2 operand rows per k-block for BN columns of MMA work instead of
// 128 + BN.

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

// Arrival on a barrier of the peer CTA (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity,
                                                 uint32_t suspend = kSuspendNs) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(suspend)
      : "memory");
  return ok != 0;
}

// Bounded wait on a barrier that also receives arrivals from the peer CTA.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity,
                                                  volatile int* abort, int* err, long long budget,
                                                  uint32_t suspend) {
  if (mbar_try_cluster(bar, parity, suspend)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_cluster(bar, parity, suspend)) return true;
    if (*abort) return false;
    if (clock64() - t0 > budget) {
      atomicOr(err, kErrTimeout);
      *abort = 1;
      return false;
    }
  }
}

// TMA load into this CTA's shared memory whose completion is counted on a barrier of either
// CTA of the pair (bar_cluster: a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}

template <bool FP8>
__device__ __forceinline__ void mma_issue_pair(uint32_t dtmem, uint64_t a, uint64_t b,
                                               uint32_t id, uint32_t accum) {
  if (FP8) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accum)
        : "memory");
  }
}

// Arrives on the barrier at this offset in both CTAs of the pair once the MMAs issued so far
// have completed.
__device__ __forceinline__ void mma_commit_pair_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"((uint16_t)3)
      : "memory");
}

__device__ __forceinline__ void mma_commit_pair_local(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Starts loading 32 consecutive FP32 columns of this thread's TMEM lane into r; the values
// are valid only after tmem_wait(r).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Waits for this thread's outstanding TMEM loads; r is passed through so no use of it can be
// scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
        "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
        "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]),
        "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]),
        "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]),
        "+r"(r[31])
      :
      : "memory");
}

// tanh-form GELU (Sec. 3.3.2), 0.5 x (1 + tanh(c (x + a x^3))), evaluated as
// u = x (c + a c x^2), t = tanh(u), y = 0.5 x + 0.5 x t: two multiplies, two FMAs, one MUFU
// tanh and one multiply per element.
constexpr float kGeluC = 0.7978845608028654f;        // sqrt(2 / pi)
constexpr float kGeluAC = 0.044715f * 0.7978845608028654f;

__device__ __forceinline__ float tanh_fast(float u) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return t;
}

__device__ __forceinline__ float gelu_fast(float x) {
  const float t = tanh_fast(x * fmaf(x * x, kGeluAC, kGeluC));
  const float hx = 0.5f * x;
  return fmaf(hx, t, hx);
}

// The same on two values with the packed FP32x2 instructions (one issue per pair).
__device__ __forceinline__ float2 gelu_fast2(float2 x) {
  const float2 p = __ffma2_rn(__fmul2_rn(x, x), make_float2(kGeluAC, kGeluAC),
                              make_float2(kGeluC, kGeluC));
  const float2 u = __fmul2_rn(x, p);
  const float2 t = make_float2(tanh_fast(u.x), tanh_fast(u.y));
  const float2 hx = __fmul2_rn(x, make_float2(0.5f, 0.5f));
  return __ffma2_rn(hx, t, hx);
}

constexpr int out_bytes(int outk) { return outk == kXF32 ? 4 : (outk == kXBF16 ? 2 : 1); }

template <int BN, int OUTK, bool PAIR = false, int EPQ = 3>
struct Cfg {
  static constexpr int kEpq = EPQ;               // epilogue warps per TMEM lane quarter
  static constexpr int kEpiWarps = 4 * EPQ;
  static constexpr int kThreads = threads_for(EPQ);
  // Per warp: staging buffers of 32 rows x 32 columns (the GELU' of kModeStoreG is BF16, no
  // wider than the output). Two let a warp fill one while the other's store still reads it.
  // A pair tile streams several k-blocks per accumulator, so its epilogue has time to spare,
  // and the operand ring is what sets its pace: with one buffer per warp the ring gains a stage.
  static constexpr int kStgBufs = PAIR ? 1 : 2;
  static constexpr int kStageOut = kStgBufs * 32 * 32 * out_bytes(OUTK);
  static constexpr int kBRows = PAIR ? BN / 2 : BN;   // rows of W this CTA holds per stage
  static constexpr int kStageBytes = (BM + kBRows) * kRowBytes;
  static constexpr int kStages0 = (kSmemLimit - 2048 - kEpiWarps * kStageOut) / kStageBytes;
  static constexpr int kStages = kStages0 > 8 ? 8 : kStages0;
  static constexpr int kAccStride = (BN + 31) / 32 * 32;
  static constexpr int kTmemCols = (2 * kAccStride <= 32) ? 32 : (2 * kAccStride <= 64) ? 64
                                   : (2 * kAccStride <= 128) ? 128 : (2 * kAccStride <= 256) ? 256 : 512;
  static constexpr int kSmemBytes =
      kStages * kStageBytes + kEpiWarps * kStageOut + 1024 /*align*/ + 1024 /*barriers*/;
};

// d/dx of the tanh-form GELU: 0.5 (1 + t) + 0.5 x (1 - t^2) c (1 + 3 a x^2).
__device__ __forceinline__ float gelu_grad_fast(float x) {
  const float x2 = x * x;
  const float t = tanh_fast(x * fmaf(x2, kGeluAC, kGeluC));
  const float hx = 0.5f * x;
  return fmaf(hx * fmaf(-t, t, 1.0f), fmaf(x2, 3.0f * kGeluAC, kGeluC), fmaf(0.5f, t, 0.5f));
}

__device__ __forceinline__ float2 gelu_grad_fast2(float2 x) {
  const float2 x2 = __fmul2_rn(x, x);
  const float2 u = __fmul2_rn(x, __ffma2_rn(x2, make_float2(kGeluAC, kGeluAC),
                                            make_float2(kGeluC, kGeluC)));
  const float2 t = make_float2(tanh_fast(u.x), tanh_fast(u.y));
  const float2 hx = __fmul2_rn(x, make_float2(0.5f, 0.5f));
  const float2 omt2 = __ffma2_rn(make_float2(-t.x, -t.y), t, make_float2(1.0f, 1.0f));
  const float2 dp = __ffma2_rn(x2, make_float2(3.0f * kGeluAC, 3.0f * kGeluAC),
                               make_float2(kGeluC, kGeluC));
  const float2 a = __ffma2_rn(make_float2(0.5f, 0.5f), t, make_float2(0.5f, 0.5f));
  return __ffma2_rn(__fmul2_rn(hx, omt2), dp, a);
}

// Unit position in a staging row of RB bytes under the tensor map's swizzle: the 16-byte unit u
// of row r sits at u ^ swz(r), swz = (r >> 2) & 1 for 32-byte rows (32B swizzle), (r >> 1) & 3
// for 64-byte rows (64B swizzle), r & 7 for 128-byte rows (128B swizzle). Rows of eight
// consecutive lanes then cover all 32 banks.
template <int RB>
__device__ __forceinline__ int swz(int r) {
  return RB == 128 ? (r & 7) : (RB == 64 ? ((r >> 1) & 3) : ((r >> 2) & 1));
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"((uint64_t)map), "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until at most one bulk store group of this thread is still reading shared memory.
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// Waits until no bulk store group of this thread is still reading shared memory.
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Quantises 32 values of row `lane` to OUTK, writes them into one of the warp's NBUF staging
// buffers (32 rows x 32 columns, swizzled) and has lane 0 issue a TMA tensor store of the box
// at (col0, m0); the tensor map clips rows and columns outside the output. A buffer is reused
// only after the store issued from it NBUF calls earlier has finished reading it.
template <int OUTK, int NBUF = 2>
__device__ __forceinline__ void store_chunk(const float (&v)[32], const CUtensorMap* map,
                                            float out_scale, int64_t m0, int col0, uint8_t* stg2,
                                            int& buf, int lane) {
  constexpr int esz = OUTK == kXF32 ? 4 : (OUTK == kXBF16 ? 2 : 1);
  constexpr int U = 2 * esz;     // 16-byte units per 32-column row segment
  constexpr int RB = 32 * esz;   // bytes per row segment
  uint4 w[U];
  if (OUTK == kXF32) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      w[u] = make_uint4(__float_as_uint(v[4 * u]), __float_as_uint(v[4 * u + 1]),
                        __float_as_uint(v[4 * u + 2]), __float_as_uint(v[4 * u + 3]));
  } else if (OUTK == kXBF16) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * u], v[8 * u + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * u + 2], v[8 * u + 3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * u + 4], v[8 * u + 5]);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * u + 6], v[8 * u + 7]);
      memcpy(&w[u].x, &h0, 4); memcpy(&w[u].y, &h1, 4);
      memcpy(&w[u].z, &h2, 4); memcpy(&w[u].w, &h3, 4);
    }
  } else {
    const float sc = out_scale;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uint32_t wd[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_fp8x4_e4m3 f(make_float4(v[16 * u + 4 * e] * sc, v[16 * u + 4 * e + 1] * sc,
                                            v[16 * u + 4 * e + 2] * sc, v[16 * u + 4 * e + 3] * sc));
        wd[e] = f.__x;
      }
      w[u] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
  }
  uint8_t* stg = stg2 + buf * (32 * RB);
  if (lane == 0) {
    if constexpr (NBUF == 1) bulk_wait_read0();
    else bulk_wait_read1();
  }
  __syncwarp();
  const int sw = swz<RB>(lane);
#pragma unroll
  for (int u = 0; u < U; ++u)
    *reinterpret_cast<uint4*>(stg + lane * RB + ((u ^ sw) * 16)) = w[u];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    tma_store_2d(map, smem_u32(stg), col0, (int)m0);
    bulk_commit();
  }
  if constexpr (NBUF == 2) buf ^= 1;
}

// One 32-column chunk of the epilogue: per-channel scale, bias, GELU (or the row-group scale
// of a tangent layer), then quantise and store; kModeStoreG also stores GELU'(z). With
// SMEM_BIAS the bias pointer addresses shared memory (a plain load instead of ld.global.nc).
template <int OUTK, int ACT, bool SCALE, int MODE, bool SMEM_BIAS = false, int NBUF = 2>
__device__ __forceinline__ void epilogue_chunk(const uint32_t (&r)[32], const TcArgs& g,
                                               const CUtensorMap* tmO, const CUtensorMap* tmG,
                                               int64_t M, int64_t m0, int col0, uint8_t* stg,
                                               int& buf, int lane) {
  float v[32];
  if (MODE == kModeRowG) {
    // tangent row m0 + lane belongs to cell (m0 + lane) / ntan; G is BF16 [cells x ldg]
    const int64_t row = m0 + lane;
    const int64_t cell = (row < M ? row : M - 1) / g.ntan;
    const uint4* gp = reinterpret_cast<const uint4*>((const __nv_bfloat16*)g.gbuf + cell * g.ldg + col0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint4 q = __ldg(gp + u);
      const uint32_t qs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 h2;
        memcpy(&h2, &qs[e], 4);
        const float2 f = __bfloat1622float2(h2);
        v[8 * u + 2 * e] = __uint_as_float(r[8 * u + 2 * e]) * f.x;
        v[8 * u + 2 * e + 1] = __uint_as_float(r[8 * u + 2 * e + 1]) * f.y;
      }
    }
    store_chunk<OUTK, NBUF>(v, tmO, g.out_scale, m0, col0, stg, buf, lane);
    return;
  }
  const float4* b4 = reinterpret_cast<const float4*>(g.bias + col0);  // zero padded to 32
  const float4* s4 = reinterpret_cast<const float4*>(g.col_scale + col0);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const float4 b = SMEM_BIAS ? b4[u] : __ldg(b4 + u);
    float2 z0 = make_float2(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1]));
    float2 z1 = make_float2(__uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3]));
    if (SCALE) {
      const float4 sc = __ldg(s4 + u);
      z0 = __ffma2_rn(z0, make_float2(sc.x, sc.y), make_float2(b.x, b.y));
      z1 = __ffma2_rn(z1, make_float2(sc.z, sc.w), make_float2(b.z, b.w));
    } else {
      z0 = __fadd2_rn(z0, make_float2(b.x, b.y));
      z1 = __fadd2_rn(z1, make_float2(b.z, b.w));
    }
    if constexpr (ACT == kActTanh) {
      z0 = gelu_fast2(z0);
      z1 = gelu_fast2(z1);
    } else if constexpr (ACT == kActTable) {
      z0 = make_float2(gelu_from_table(z0.x, g.gtab), gelu_from_table(z0.y, g.gtab));
      z1 = make_float2(gelu_from_table(z1.x, g.gtab), gelu_from_table(z1.y, g.gtab));
    }
    v[4 * u] = z0.x; v[4 * u + 1] = z0.y; v[4 * u + 2] = z1.x; v[4 * u + 3] = z1.y;
  }
  store_chunk<OUTK, NBUF>(v, tmO, g.out_scale, m0, col0, stg, buf, lane);
  if (MODE == kModeStoreG) {
    // second pass over the same accumulators: GELU'(z), so only one 32-value array is live
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 b = __ldg(b4 + u);
      const float2 g0 = gelu_grad_fast2(__fadd2_rn(
          make_float2(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1])), make_float2(b.x, b.y)));
      const float2 g1 = gelu_grad_fast2(__fadd2_rn(
          make_float2(__uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3])), make_float2(b.z, b.w)));
      v[4 * u] = g0.x; v[4 * u + 1] = g0.y; v[4 * u + 2] = g1.x; v[4 * u + 3] = g1.y;
    }
    store_chunk<kXBF16, NBUF>(v, tmG, 1.0f, m0, col0, stg, buf, lane);
  }
}

// The grid stride of the work items in whole m units (q), n positions (r) and q mod tiles_n
// (rot). One copy per CTA, in shared memory: the epilogue warps have no registers to spare.
struct WalkStep {
  uint32_t q;
  int r, rot;
};

// Walks the work items t = first, first + step, ... of one CTA (or CTA pair). Item t lies in
// split t / (units_m tiles_n), m unit mu = (t mod units_m tiles_n) / tiles_n and n position
// r = t mod tiles_n; its n tile is r rotated by the m unit, (r + mu) mod tiles_n, so that the
// items one CTA visits a grid stride apart cycle through the n tiles (whose MMA widths differ
// when the last one is narrowed). The position advances by additions and compares: divisions
// per item cost the layers with short k loops a few per cent. Item counts fit in 32 bits (the
// launch checks).
struct ItemWalk {
  uint32_t mu;          // m unit within the split
  int split, r, rot;    // split, n position in the m unit, mu mod tiles_n
  __device__ __forceinline__ ItemWalk(uint32_t first, uint32_t units_m, int tiles_n) {
    if (units_m == 0) {
      mu = 0;
      split = 0x7FFFFFFF;   // no items
      r = rot = 0;
    } else {
      const uint32_t tiles_mn = units_m * (uint32_t)tiles_n;
      split = (int)(first / tiles_mn);
      const uint32_t rem = first - (uint32_t)split * tiles_mn;
      mu = rem / (uint32_t)tiles_n;
      r = (int)(rem - mu * (uint32_t)tiles_n);
      rot = (int)(mu % (uint32_t)tiles_n);
    }
  }
  __device__ __forceinline__ int nt(int tiles_n) const {
    const int x = r + rot;
    return x < tiles_n ? x : x - tiles_n;
  }
  __device__ __forceinline__ void next(const WalkStep& st, uint32_t units_m, int tiles_n) {
    mu += st.q;
    r += st.r;
    rot += st.rot;
    if (rot >= tiles_n) rot -= tiles_n;
    if (r >= tiles_n) {
      r -= tiles_n;
      ++mu;
      if (++rot == tiles_n) rot = 0;
    }
    if (mu >= units_m) {   // into a later split
      split += (int)(mu / units_m);
      mu %= units_m;
      rot = (int)(mu % (uint32_t)tiles_n);
    }
  }
};

template <bool FP8, int BN, int OUTK, int ACT, bool SCALE, int MODE, bool PAIR>
__global__ void __launch_bounds__(threads_for(epi_per_quarter(PAIR, ACT, MODE)), 1) tc_gemm_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmG, TcArgs g) {
  using C = Cfg<BN, OUTK, PAIR, epi_per_quarter(PAIR, ACT, MODE)>;
  constexpr int kEpiWarps = C::kEpiWarps;
  // a 32-column epilogue chunk is stored as one TMA box, so chunks must not straddle tiles
  static_assert(BN % 32 == 0, "tile width must be a multiple of 32");
  // each CTA of a pair holds whole 8-row swizzle atoms of W
  static_assert(!PAIR || (BN / 2) % 8 == 0, "paired tile width must split into 8-row groups");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                                   // kStages x 16 KB
  uint8_t* sB = smem + C::kStages * BM * kRowBytes;     // kStages x kBRows*128 B
  uint8_t* sOut = smem + C::kStages * C::kStageBytes;  // kEpiWarps x kStageOut
  uint64_t* bars = (uint64_t*)(sOut + kEpiWarps * C::kStageOut);
  // bars: full[S], empty[S], tfull[2], tempty[2], drain
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ WalkStep walk_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * C::kStages;
  const uint32_t tfull0 = empty0 + 8 * C::kStages, tempty0 = tfull0 + 16;
  const uint32_t drain = tempty0 + 16;
  // In a pair, the even CTA (rank 0) owns the full and accumulator-empty barriers the MMAs
  // wait on: both CTAs' loads complete on its full barriers, both CTAs' epilogues arrive on
  // its tempty barriers. Each CTA's empty and tfull barriers receive the MMA commits.
  const uint32_t rank = PAIR ? cluster_rank() : 0;

  if (threadIdx.x == 0) {
    abort_sh = 0;
    const uint32_t step = PAIR ? (gridDim.x >> 1) : gridDim.x, tn = (uint32_t)((g.N + BN - 1) / BN);
    walk_sh.q = step / tn;
    walk_sh.r = (int)(step - walk_sh.q * tn);
    walk_sh.rot = (int)(walk_sh.q % tn);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, PAIR ? 2 * kEpiWarps : kEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&tmem_base_sh)),
                   "r"((uint32_t)C::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&tmem_base_sh)),
                   "r"((uint32_t)C::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // the peer's barriers are initialised before any use
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort = &abort_sh;

  const int64_t M = valid_rows(g.rows);
  const int64_t tiles_m = (M + BM - 1) / BM;
  // work items: (split, m tile, n tile), or for a pair (split, pair of m tiles, n tile)
  const int64_t units_m = PAIR ? (tiles_m + 1) / 2 : tiles_m;
  const int tiles_n = (g.N + BN - 1) / BN;
  const uint32_t units_m32 = (uint32_t)units_m;
  const int kblocks = (g.K * (FP8 ? 1 : 2) + kRowBytes - 1) / kRowBytes;
  const int kelems = kRowBytes / (FP8 ? 1 : 2);
  const int kbs = (kblocks + g.ksplit - 1) / g.ksplit;   // k-blocks per split (host: none empty)
  const uint32_t t_first = PAIR ? (blockIdx.x >> 1) : blockIdx.x;
  // first row of this CTA's part of a work item in m unit mu
  auto tile_m0 = [&](int64_t mu) -> int64_t { return PAIR ? (mu * 2 + rank) * BM : mu * BM; };
  // MMA width of n tile nt: the last tile covers only the columns left, rounded up to 16 (the N
  // granule at M = 128 and M = 256); its columns past N are clipped by the output tensor map
  auto tile_w = [&](int nt) -> int { return min(BN, (g.N - nt * BN + 15) & ~15); };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    uint32_t it = 0;
    bool ok = true;
    for (ItemWalk w(t_first, units_m32, tiles_n); w.split < g.ksplit && ok;
         w.next(walk_sh, units_m32, tiles_n)) {
      const int kb0 = w.split * kbs, kb1 = min(kblocks, kb0 + kbs);
      const int m0 = (int)tile_m0(w.mu);
      // a pair splits the tile's MMA width between its CTAs: each holds half of the W rows
      const int nt = w.nt(tiles_n);
      const int n0 = nt * BN + (PAIR ? (int)rank * (tile_w(nt) >> 1) : 0);
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it % C::kStages;
        const uint32_t ph = (it / C::kStages) & 1;
        if (!mbar_wait(empty0 + 8 * s, ph ^ 1, abort, g.err, g.budget, g.suspend)) {
          ok = false;
          break;
        }
        const uint32_t dA = smem_u32(sA + s * BM * kRowBytes);
        const uint32_t dB = smem_u32(sB + s * C::kBRows * kRowBytes);
        if constexpr (PAIR) {
          const uint32_t full_leader = map_shared(full0 + 8 * s, 0);
          if (rank == 0) mbar_arrive_expect_tx(full0 + 8 * s, 2 * C::kStageBytes);
          tma_load_2d_pair(dA, &tmA, full_leader, kb * kelems, m0);
          tma_load_2d_pair(dB, &tmB, full_leader, kb * kelems, n0);
        } else {
          mbar_arrive_expect_tx(full0 + 8 * s, C::kStageBytes);
          tma_load_2d(dA, &tmA, full0 + 8 * s, kb * kelems, m0);
          tma_load_2d(dB, &tmB, full0 + 8 * s, kb * kelems, n0);
        }
      }
    }
    const uint32_t issued = it;
    const uint32_t first = issued > (uint32_t)C::kStages ? issued - C::kStages : 0;
    if (!PAIR || rank == 0) {
      // Drain: the last issued load of every stage must have landed before the CTA exits (a
      // pair's full barriers, on the even CTA, count the odd CTA's loads too).
      for (uint32_t j = first; j < issued; ++j) {
        const int s = j % C::kStages;
        const uint32_t ph = (j / C::kStages) & 1;
        const long long t0 = clock64();
        while (!mbar_try(full0 + 8 * s, ph) && clock64() - t0 < kWaitBudget) {
        }
      }
    }
    if constexpr (PAIR) {
      // Producer tail: the MMA commits that free the last stages arrive on this CTA's empty
      // barriers from the even CTA; they must have arrived before this CTA exits.
      for (uint32_t j = first; j < issued; ++j) {
        const int s = j % C::kStages;
        const uint32_t ph = (j / C::kStages) & 1;
        const long long t0 = clock64();
        while (!mbar_try_cluster(empty0 + 8 * s, ph) && clock64() - t0 < kWaitBudget) {
        }
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t id0 = idesc<FP8, 0, PAIR ? 2 * BM : BM>();
    uint32_t it = 0, j = 0;
    bool ok = true;
    for (ItemWalk w(t_first, units_m32, tiles_n); w.split < g.ksplit && ok;
         w.next(walk_sh, units_m32, tiles_n), ++j) {
      const int kb0 = w.split * kbs, kb1 = min(kblocks, kb0 + kbs);
      const uint32_t id = id0 | ((uint32_t)(tile_w(w.nt(tiles_n)) >> 3) << 17);
      const int a = j & 1;
      const uint32_t aph = (j >> 1) & 1;
      if (PAIR ? !mbar_wait_cluster(tempty0 + 8 * a, aph ^ 1, abort, g.err, g.budget, g.suspend)
               : !mbar_wait(tempty0 + 8 * a, aph ^ 1, abort, g.err, g.budget, g.suspend))
        break;
      tc_fence_after();
      const uint32_t dt = tmem + a * C::kAccStride;
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it % C::kStages;
        const uint32_t ph = (it / C::kStages) & 1;
        if (!mbar_wait(full0 + 8 * s, ph, abort, g.err, g.budget, g.suspend)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t da = desc_sw128(smem_u32(sA + s * BM * kRowBytes));
        const uint64_t db = desc_sw128(smem_u32(sB + s * C::kBRows * kRowBytes));
#pragma unroll
        for (int kk = 0; kk < kRowBytes / 32; ++kk) {  // 32 bytes of K per instruction
          if constexpr (PAIR)
            mma_issue_pair<FP8>(dt, da + 2 * kk, db + 2 * kk, id, (kb != kb0 || kk) ? 1u : 0u);
          else
            mma_issue<FP8>(dt, da + 2 * kk, db + 2 * kk, id, (kb != kb0 || kk) ? 1u : 0u);
        }
        // frees the stage (in both CTAs of a pair) when these MMAs have read it
        if constexpr (PAIR) mma_commit_pair_both(empty0 + 8 * s);
        else mma_commit(empty0 + 8 * s);
      }
      if (ok) {
        if constexpr (PAIR) mma_commit_pair_both(tfull0 + 8 * a);
        else mma_commit(tfull0 + 8 * a);
      }
    }
    // Drain: every MMA issued by this thread completes before TMEM is released.
    if constexpr (PAIR) mma_commit_pair_local(drain);
    else mma_commit(drain);
    const long long t0 = clock64();
    while (!mbar_try(drain, 0) && clock64() - t0 < kWaitBudget) {
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                   // TMEM lane quarter this warp may access
    const int slot = (warp - 2) >> 2;         // which of the quarter's interleaved chunks
    constexpr int kChunkStride = 32 * C::kEpq;
    uint8_t* stg = sOut + (warp - 2) * C::kStageOut;
    int buf = 0;
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmO) : "memory");
    }
    uint32_t j = 0;
    for (ItemWalk w(t_first, units_m32, tiles_n); w.split < g.ksplit;
         w.next(walk_sh, units_m32, tiles_n), ++j) {
      const int a = j & 1;
      const uint32_t aph = (j >> 1) & 1;
      if (!mbar_wait(tfull0 + 8 * a, aph, abort, g.err, g.budget, g.suspend)) break;
      tc_fence_after();
      const int64_t mt = tile_m0(w.mu);
      // row of the output: the tile's rows, shifted to this split's partial product
      const int64_t m0 = mt + q * 32 + w.split * g.split_rows;
      const int n0 = w.nt(tiles_n) * BN;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + a * C::kAccStride;
      // chunks c = 32 slot + kChunkStride i; with three warps per quarter TMEM loads run one
      // chunk ahead of the math, except in kModeStoreG, whose two stores per chunk leave no
      // registers for a second chunk in flight; with five, the quarter's other warps cover the
      // load. The odd CTA of a pair whose m tile lies past the rows stores nothing.
      uint32_t r0[32], r1[32];
      int c0 = (PAIR && mt >= M) ? BN : 32 * slot;
      if constexpr (MODE == kModeStoreG || C::kEpq >= 4) {
        for (; c0 < BN; c0 += kChunkStride) {
          tmem_ld32(tbase + c0, r0);
          tmem_wait(r0);
          if (n0 + c0 < g.N)
            epilogue_chunk<OUTK, ACT, SCALE, MODE, false, C::kStgBufs>(r0, g, &tmO, &tmG, M, m0,
                                                                       n0 + c0, stg, buf, lane);
        }
        c0 = BN;
      }
      if (c0 < BN) tmem_ld32(tbase + c0, r0);
      for (; c0 < BN; c0 += 2 * kChunkStride) {
        tmem_wait(r0);
        const int c1 = c0 + kChunkStride;
        if (c1 < BN) tmem_ld32(tbase + c1, r1);
        if (n0 + c0 < g.N)
          epilogue_chunk<OUTK, ACT, SCALE, MODE, false, C::kStgBufs>(r0, g, &tmO, &tmG, M, m0,
                                                                     n0 + c0, stg, buf, lane);
        if (c1 >= BN) break;
        tmem_wait(r1);
        if (c1 + kChunkStride < BN) tmem_ld32(tbase + c1 + kChunkStride, r0);
        if (n0 + c1 < g.N)
          epilogue_chunk<OUTK, ACT, SCALE, MODE, false, C::kStgBufs>(r1, g, &tmO, &tmG, M, m0,
                                                                     n0 + c1, stg, buf, lane);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR && rank != 0) mbar_arrive_cluster(map_shared(tempty0 + 8 * a, 0));
        else mbar_arrive(tempty0 + 8 * a);
      }
    }
    // the tensor stores must have read shared memory (and be complete) before the CTA exits
    if (lane == 0) bulk_wait_all();
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  // a pair frees its tensor memory together, once neither CTA reads or writes it any more
  if constexpr (PAIR) cluster_sync();
  tc_fence_after();
  if (warp == 1) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"((uint32_t)C::kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"((uint32_t)C::kTmemCols)
                   : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Opts the kernel instance into its dynamic shared memory, once per device.
template <bool FP8, int BN, int OUTK, int ACT, int MODE, bool PAIR>
cudaError_t tc_attr(int* max_clusters) {
  static bool attr_done[64] = {false};
  static int clusters[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    using C = Cfg<BN, OUTK, PAIR, epi_per_quarter(PAIR, ACT, MODE)>;
    auto kern = tc_gemm_kernel<FP8, BN, OUTK, ACT, FP8, MODE, PAIR>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (PAIR) {
      // how many CTA pairs fit on the GPU at once: a persistent grid of more would leave the
      // excess pairs to a second wave
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2, 1, 1);
      cfg.blockDim = dim3(C::kThreads, 1, 1);
      cfg.dynamicSmemBytes = C::kSmemBytes;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      e = cudaOccupancyMaxActiveClusters(&n, (const void*)kern, &cfg);
      if (e != cudaSuccess) return e;
      if (n <= 0) return cudaErrorInvalidConfiguration;
      clusters[dev] = n;
    }
    attr_done[dev] = true;
  }
  if (max_clusters) *max_clusters = clusters[dev];
  return cudaSuccess;
}

template <bool FP8, int BN, int OUTK, int ACT, int MODE = kModePlain, bool PAIR = false>
cudaError_t launch_bn(const TcLayer& L, const TcArgs& a, int num_sms, cudaStream_t st) {
  using C = Cfg<BN, OUTK, PAIR, epi_per_quarter(PAIR, ACT, MODE)>;
  constexpr bool SCALE = FP8;
  auto kern = tc_gemm_kernel<FP8, BN, OUTK, ACT, SCALE, MODE, PAIR>;
  int max_clusters = 0;
  cudaError_t e0 = tc_attr<FP8, BN, OUTK, ACT, MODE, PAIR>(&max_clusters);
  if (e0 != cudaSuccess) return e0;
  if (num_sms <= 0) return cudaSuccess;  // attribute set-up only
  const CUtensorMap& tmG = L.mode == kModeStoreG ? L.tmG : L.tmO;
  const int64_t tiles_n = (L.N + BN - 1) / BN;
  // the kernel walks its work items with 32-bit counts
  const int64_t items = (PAIR ? (a.rows.nmax + 2 * BM - 1) / (2 * BM) : (a.rows.nmax + BM - 1) / BM) *
                        tiles_n * a.ksplit;
  if (items > 0x7FFFFFFF) return cudaErrorInvalidValue;
  if constexpr (PAIR) {
    const int64_t units = items;
    const int64_t cap = std::min<int64_t>(max_clusters, num_sms / 2);
    const int64_t nc = std::max<int64_t>(1, std::min<int64_t>(units, cap));
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * nc), 1, 1);
    cfg.blockDim = dim3(C::kThreads, 1, 1);
    cfg.dynamicSmemBytes = C::kSmemBytes;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, L.tmA, L.tmB, L.tmO, tmG, a);
  } else {
    const int64_t tiles = items;
    const unsigned grid = (unsigned)(tiles < num_sms ? (tiles > 0 ? tiles : 1) : num_sms);
    kern<<<grid, C::kThreads, C::kSmemBytes, st>>>(L.tmA, L.tmB, L.tmO, tmG, a);
    return cudaGetLastError();
  }
}

// Hidden layers: GELU, output in the input precision. Last layer: linear, FP32 output.
// The Jacobian's BF16 passes add a hidden layer that also stores GELU'(z) and a tangent layer
// scaled per row group by it.
template <bool FP8>
cudaError_t launch_fmt(const TcLayer& L, const TcArgs& a, int num_sms, cudaStream_t st) {
  constexpr int HID = FP8 ? kXFP8 : kXBF16;
  if (L.mode != kModePlain) {
    if (FP8 || L.out_kind != kXBF16) return cudaErrorInvalidValue;
    if (L.pair) {
      if (L.mode == kModeStoreG) {
        switch (L.BN) {
          case 160: return launch_bn<false, 160, kXBF16, kActTanh, kModeStoreG, true>(L, a, num_sms, st);
          case 224: return launch_bn<false, 224, kXBF16, kActTanh, kModeStoreG, true>(L, a, num_sms, st);
          case 256: return launch_bn<false, 256, kXBF16, kActTanh, kModeStoreG, true>(L, a, num_sms, st);
          default: return cudaErrorInvalidValue;
        }
      }
      switch (L.BN) {
        case 160: return launch_bn<false, 160, kXBF16, kActNone, kModeRowG, true>(L, a, num_sms, st);
        case 224: return launch_bn<false, 224, kXBF16, kActNone, kModeRowG, true>(L, a, num_sms, st);
        case 256: return launch_bn<false, 256, kXBF16, kActNone, kModeRowG, true>(L, a, num_sms, st);
        default: return cudaErrorInvalidValue;
      }
    }
    if (L.mode == kModeStoreG) {
      switch (L.BN) {
        case 64: return launch_bn<false, 64, kXBF16, kActTanh, kModeStoreG>(L, a, num_sms, st);
        case 128: return launch_bn<false, 128, kXBF16, kActTanh, kModeStoreG>(L, a, num_sms, st);
        case 160: return launch_bn<false, 160, kXBF16, kActTanh, kModeStoreG>(L, a, num_sms, st);
        case 192: return launch_bn<false, 192, kXBF16, kActTanh, kModeStoreG>(L, a, num_sms, st);
        case 224: return launch_bn<false, 224, kXBF16, kActTanh, kModeStoreG>(L, a, num_sms, st);
        case 256: return launch_bn<false, 256, kXBF16, kActTanh, kModeStoreG>(L, a, num_sms, st);
        default: return cudaErrorInvalidValue;
      }
    }
    switch (L.BN) {
      case 64: return launch_bn<false, 64, kXBF16, kActNone, kModeRowG>(L, a, num_sms, st);
      case 128: return launch_bn<false, 128, kXBF16, kActNone, kModeRowG>(L, a, num_sms, st);
      case 160: return launch_bn<false, 160, kXBF16, kActNone, kModeRowG>(L, a, num_sms, st);
      case 192: return launch_bn<false, 192, kXBF16, kActNone, kModeRowG>(L, a, num_sms, st);
      case 224: return launch_bn<false, 224, kXBF16, kActNone, kModeRowG>(L, a, num_sms, st);
      case 256: return launch_bn<false, 256, kXBF16, kActNone, kModeRowG>(L, a, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (L.pair) {
    // CTA pairs: hidden layers with more than one k-block, and the FP32 weight-gradient GEMMs
    // (no activation, split-K over the batch) of training
    if (!L.gelu) {
      if (FP8 || L.gtab || L.out_kind != kXF32) return cudaErrorInvalidValue;
      switch (L.BN) {
        case 128: return launch_bn<false, 128, kXF32, kActNone, kModePlain, true>(L, a, num_sms, st);
        case 256: return launch_bn<false, 256, kXF32, kActNone, kModePlain, true>(L, a, num_sms, st);
        default: return cudaErrorInvalidValue;
      }
    }
    if (L.gtab) {
      if (FP8 || L.out_kind != kXBF16) return cudaErrorInvalidValue;
      switch (L.BN) {
        case 160: return launch_bn<false, 160, kXBF16, kActTable, kModePlain, true>(L, a, num_sms, st);
        case 224: return launch_bn<false, 224, kXBF16, kActTable, kModePlain, true>(L, a, num_sms, st);
        case 256: return launch_bn<false, 256, kXBF16, kActTable, kModePlain, true>(L, a, num_sms, st);
        default: return cudaErrorInvalidValue;
      }
    }
    if (L.out_kind != HID) return cudaErrorInvalidValue;
    switch (L.BN) {
      case 160: return launch_bn<FP8, 160, HID, kActTanh, kModePlain, true>(L, a, num_sms, st);
      case 224: return launch_bn<FP8, 224, HID, kActTanh, kModePlain, true>(L, a, num_sms, st);
      case 256: return launch_bn<FP8, 256, HID, kActTanh, kModePlain, true>(L, a, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (L.gelu && L.gtab) {
    if (FP8 || L.out_kind != kXBF16) return cudaErrorInvalidValue;
    switch (L.BN) {
      case 64: return launch_bn<false, 64, kXBF16, kActTable>(L, a, num_sms, st);
      case 128: return launch_bn<false, 128, kXBF16, kActTable>(L, a, num_sms, st);
      case 160: return launch_bn<false, 160, kXBF16, kActTable>(L, a, num_sms, st);
      case 192: return launch_bn<false, 192, kXBF16, kActTable>(L, a, num_sms, st);
      case 224: return launch_bn<false, 224, kXBF16, kActTable>(L, a, num_sms, st);
      case 256: return launch_bn<false, 256, kXBF16, kActTable>(L, a, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (L.gelu) {
    if (L.out_kind != HID) return cudaErrorInvalidValue;
    switch (L.BN) {
      case 64: return launch_bn<FP8, 64, HID, kActTanh>(L, a, num_sms, st);
      case 128: return launch_bn<FP8, 128, HID, kActTanh>(L, a, num_sms, st);
      case 160: return launch_bn<FP8, 160, HID, kActTanh>(L, a, num_sms, st);
      case 192: return launch_bn<FP8, 192, HID, kActTanh>(L, a, num_sms, st);
      case 224: return launch_bn<FP8, 224, HID, kActTanh>(L, a, num_sms, st);
      case 256: return launch_bn<FP8, 256, HID, kActTanh>(L, a, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (L.out_kind != kXF32) return cudaErrorInvalidValue;
  switch (L.BN) {
    case 32: return launch_bn<FP8, 32, kXF32, kActNone>(L, a, num_sms, st);
    case 64: return launch_bn<FP8, 64, kXF32, kActNone>(L, a, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}


// ---- layers 0 and 1 fused ----
// H1 = GELU(GELU(x W0^T + b0) W1^T + b1) without the layer-0 activation leaving the SM. A CTA
// owns 128 rows and 416 output columns of layer 1 (two MMAs per K step, N = 224 and N = 192,
// into tensor-memory columns 0..415). Layer 1's K dimension (layer 0's outputs) is walked in
// blocks of 64: for block kb the CTA first computes x W0[64 kb ..]^T (M = 128, N = 64, K <= 64)
// into a 64-column tensor-memory buffer (columns 448..511), eight warps add the bias, apply the
// tanh-form GELU, round to BF16 and write the 128 x 64 tile straight into a shared-memory stage
// in the 128-byte-swizzled K-major layout the MMA reads; then layer 1's MMAs of block kb consume
// that stage. The layer-0 block is recomputed for each of the row tile's two column tiles of
// layer 1 (a tenth of layer 1's work); in return the 3.2 KB per row of layer-0 activations is
// neither written to nor read back from HBM, and layer 1's A operand is not streamed from L2.
// Layer 0's MMA of block kb + 1 is issued before layer 1's MMA of block kb, so the tensor pipe
// works on the next block while the warps convert the current one. Single CTAs, not pairs: every
// hand-over between the MMA issuer and the converting warps stays inside the CTA (a pair would
// need a cluster-scope release per block, measured at 500-2000 clocks).
//
// Warp roles (448 threads): warp 0 TMA producer (x tiles, W0 slices, W1 stages); warp 1 tensor
// memory and the MMAs; warps 2..9 layer-0 conversion (two per tensor-memory lane quarter, 32 of
// the 64 columns each: the conversion of a block lies on the tensor pipe's critical path, so it
// gets the most warps); warps 10..13 layer-1 epilogue (one per quarter; TMA tensor stores). Both
// bias vectors are copied to shared memory first. All waits are bounded as in tc_gemm_kernel;
// the drains on the way out allow the full default budget.
constexpr int kF01Threads = 448;
constexpr int kF01Cols = 416;            // layer-1 columns per tile
constexpr int kF01N1a = 224, kF01N1b = 192;
constexpr int kF01Acc0 = 448;            // tensor-memory column of the layer-0 block
constexpr int kF01StX = 2, kF01StW0 = 2, kF01StA = 2, kF01StB = 2;
constexpr int kF01XBytes = BM * kRowBytes;                      // 16 KB
constexpr int kF01W0Bytes = 64 * kRowBytes;                     // the 64 W0 rows of a block
constexpr int kF01ABytes = BM * kRowBytes;                      // 16 KB
constexpr int kF01BBytes = kF01Cols * kRowBytes;                // 416 rows of W1 (52 KB)
constexpr int kF01StageOut = 2 * 32 * 32 * 2;                   // per epilogue warp, BF16
constexpr int kF01MaxN0 = 2048, kF01MaxN1 = 2 * kF01Cols;       // bias entries in shared memory
constexpr int kF01Smem = kF01StX * kF01XBytes + kF01StW0 * kF01W0Bytes + kF01StA * kF01ABytes +
                         kF01StB * kF01BBytes + 4 * kF01StageOut +
                         4 * (kF01MaxN0 + kF01MaxN1) + 1024 + 1024;

struct F01Args {
  RowMap rows;
  int N0, N1, K0;            // layer-0 outputs (= layer-1 inputs), layer-1 outputs, layer-0 inputs
  const float* b0;           // [N0]
  const float* b1;           // [N1] (zero padded to 32)
  int* err;
  long long budget;
  uint32_t suspend;
};

__global__ void __launch_bounds__(kF01Threads, 1) fused01_kernel(
    const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW0,
    const __grid_constant__ CUtensorMap tmW1a, const __grid_constant__ CUtensorMap tmW1b,
    const __grid_constant__ CUtensorMap tmO, F01Args g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sX = smem;
  uint8_t* sW0 = sX + kF01StX * kF01XBytes;
  uint8_t* sA = sW0 + kF01StW0 * kF01W0Bytes;
  uint8_t* sB = sA + kF01StA * kF01ABytes;
  uint8_t* sOut = sB + kF01StB * kF01BBytes;
  float* sb0 = reinterpret_cast<float*>(sOut + 4 * kF01StageOut);
  float* sb1 = sb0 + kF01MaxN0;
  uint64_t* bars = (uint64_t*)(sb1 + kF01MaxN1);
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b0a = smem_u32(bars);
  // barriers: x full/empty, w0 full/empty, b full/empty, a full/empty, acc0 full/empty,
  // acc1 full/empty, drain
  const uint32_t xfull = b0a, xempty = xfull + 8 * kF01StX;
  const uint32_t wfull = xempty + 8 * kF01StX, wempty = wfull + 8 * kF01StW0;
  const uint32_t bfull = wempty + 8 * kF01StW0, bempty = bfull + 8 * kF01StB;
  const uint32_t afull = bempty + 8 * kF01StB, aempty = afull + 8 * kF01StA;
  const uint32_t c0full = aempty + 8 * kF01StA, c0empty = c0full + 8;
  const uint32_t c1full = c0empty + 8, c1empty = c1full + 8, drain = c1empty + 8;

  if (threadIdx.x == 0) {
    abort_sh = 0;
    for (int s = 0; s < kF01StX; ++s) { mbar_init(xfull + 8 * s, 1); mbar_init(xempty + 8 * s, 1); }
    for (int s = 0; s < kF01StW0; ++s) { mbar_init(wfull + 8 * s, 1); mbar_init(wempty + 8 * s, 1); }
    for (int s = 0; s < kF01StB; ++s) { mbar_init(bfull + 8 * s, 1); mbar_init(bempty + 8 * s, 1); }
    for (int s = 0; s < kF01StA; ++s) { mbar_init(afull + 8 * s, 8); mbar_init(aempty + 8 * s, 1); }
    mbar_init(c0full, 1);
    mbar_init(c0empty, 8);
    mbar_init(c1full, 1);
    mbar_init(c1empty, 4);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)), "r"(512u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // biases (zero padded to whole 64- and 32-column blocks)
  for (int i = threadIdx.x; i < kF01MaxN0; i += blockDim.x)
    sb0[i] = i < ((g.N0 + 63) & ~63) ? g.b0[i] : 0.0f;
  for (int i = threadIdx.x; i < kF01MaxN1; i += blockDim.x)
    sb1[i] = i < ((g.N1 + 31) & ~31) ? g.b1[i] : 0.0f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort = &abort_sh;

  const int64_t M = valid_rows(g.rows);
  const int64_t tiles_m = (M + BM - 1) / BM;
  const int tiles_n = (g.N1 + kF01Cols - 1) / kF01Cols;
  const int64_t ntiles = tiles_m * tiles_n;
  const int KB = (g.N0 + 63) / 64;              // layer-1 k-blocks = layer-0 column blocks
  auto tile_m0 = [&](int64_t t) -> int64_t { return (t / tiles_n) * BM; };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmX) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmW0) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmW1a) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmW1b) : "memory");
    uint32_t ix = 0, iw = 0, ib = 0;   // loads issued: x tiles, W0 slices, W1 stages
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int m0 = (int)tile_m0(t);
      const int n0 = (int)(t % tiles_n) * kF01Cols;
      const int sx = ix % kF01StX;
      if (!mbar_wait(xempty + 8 * sx, ((ix / kF01StX) & 1) ^ 1, abort, g.err, g.budget, g.suspend))
        break;
      mbar_arrive_expect_tx(xfull + 8 * sx, kF01XBytes);
      tma_load_2d(smem_u32(sX + sx * kF01XBytes), &tmX, xfull + 8 * sx, 0, m0);
      ++ix;
      for (int kb = 0; kb < KB; ++kb) {
        const int sw = iw % kF01StW0;
        if (!mbar_wait(wempty + 8 * sw, ((iw / kF01StW0) & 1) ^ 1, abort, g.err, g.budget, g.suspend)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(wfull + 8 * sw, kF01W0Bytes);
        tma_load_2d(smem_u32(sW0 + sw * kF01W0Bytes), &tmW0, wfull + 8 * sw, 0, 64 * kb);
        ++iw;
        const int sb = ib % kF01StB;
        if (!mbar_wait(bempty + 8 * sb, ((ib / kF01StB) & 1) ^ 1, abort, g.err, g.budget, g.suspend)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(bfull + 8 * sb, kF01BBytes);
        const uint32_t dB = smem_u32(sB + sb * kF01BBytes);
        tma_load_2d(dB, &tmW1a, bfull + 8 * sb, 64 * kb, n0);
        tma_load_2d(dB + kF01N1a * kRowBytes, &tmW1b, bfull + 8 * sb, 64 * kb, n0 + kF01N1a);
        ++ib;
      }
    }
    // Drain: every issued load lands before the CTA exits.
    auto drain_ring = [&](uint32_t full, int stages, uint32_t issued) {
      const uint32_t first = issued > (uint32_t)stages ? issued - stages : 0;
      for (uint32_t j = first; j < issued; ++j) {
        const long long t0 = clock64();
        while (!mbar_try(full + 8 * (j % stages), (j / stages) & 1) && clock64() - t0 < kWaitBudget) {
        }
      }
    };
    drain_ring(xfull, kF01StX, ix);
    drain_ring(wfull, kF01StW0, iw);
    drain_ring(bfull, kF01StB, ib);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t id0 = idesc<false, 64, BM>();
    constexpr uint32_t id1a = idesc<false, kF01N1a, BM>();
    constexpr uint32_t id1b = idesc<false, kF01N1b, BM>();
    const int kk0 = (g.K0 * 2 + 31) / 32;       // K = 16 steps of layer 0 (K0 <= 64)
    uint32_t ix = 0, iw = 0, ia = 0, ib = 0, j0 = 0, jt = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++ix, ++jt) {
      const int sx = ix % kF01StX;
      if (!mbar_wait(xfull + 8 * sx, (ix / kF01StX) & 1, abort, g.err, g.budget, g.suspend)) break;
      tc_fence_after();
      const uint64_t dx = desc_sw128(smem_u32(sX + sx * kF01XBytes));
      // one layer-0 block: acc0 = x W0[64 kb ..]^T
      auto mma0 = [&](int kb) -> bool {
        const int sw = iw % kF01StW0;
        if (!mbar_wait(wfull + 8 * sw, (iw / kF01StW0) & 1, abort, g.err, g.budget, g.suspend))
          return false;
        if (!mbar_wait(c0empty, (j0 & 1) ^ 1, abort, g.err, g.budget, g.suspend)) return false;
        tc_fence_after();
        const uint64_t dw = desc_sw128(smem_u32(sW0 + sw * kF01W0Bytes));
        for (int kk = 0; kk < kk0; ++kk)
          mma_issue<false>(tmem + kF01Acc0, dx + 2 * kk, dw + 2 * kk, id0, kk ? 1u : 0u);
        mma_commit(wempty + 8 * sw);
        mma_commit(c0full);
        if (kb == KB - 1) mma_commit(xempty + 8 * sx);
        ++iw;
        ++j0;
        return true;
      };
      // one layer-1 block: acc1 += H0[:, 64 kb ..] W1[n0 .., 64 kb ..]^T
      auto mma1 = [&](int kb) -> bool {
        if (kb == 0 && !mbar_wait(c1empty, (jt & 1) ^ 1, abort, g.err, g.budget, g.suspend))
          return false;
        const int sa = ia % kF01StA;
        if (!mbar_wait(afull + 8 * sa, (ia / kF01StA) & 1, abort, g.err, g.budget, g.suspend))
          return false;
        const int sb = ib % kF01StB;
        if (!mbar_wait(bfull + 8 * sb, (ib / kF01StB) & 1, abort, g.err, g.budget, g.suspend))
          return false;
        tc_fence_after();
        const uint64_t da = desc_sw128(smem_u32(sA + sa * kF01ABytes));
        const uint64_t db = desc_sw128(smem_u32(sB + sb * kF01BBytes));
        const uint64_t db2 = desc_sw128(smem_u32(sB + sb * kF01BBytes + kF01N1a * kRowBytes));
#pragma unroll
        for (int kk = 0; kk < kRowBytes / 32; ++kk) {
          const uint32_t acc = (kb != 0 || kk) ? 1u : 0u;
          mma_issue<false>(tmem, da + 2 * kk, db + 2 * kk, id1a, acc);
          mma_issue<false>(tmem + kF01N1a, da + 2 * kk, db2 + 2 * kk, id1b, acc);
        }
        mma_commit(aempty + 8 * sa);
        mma_commit(bempty + 8 * sb);
        ++ia;
        ++ib;
        return true;
      };
      if (!mma0(0)) break;
      for (int kb = 1; kb < KB && ok; ++kb) ok = mma0(kb) && mma1(kb - 1);
      if (ok) ok = mma1(KB - 1);
      if (ok) mma_commit(c1full);
    }
    mma_commit(drain);
    const long long t0 = clock64();
    while (!mbar_try(drain, 0) && clock64() - t0 < kWaitBudget) {
    }
  } else if (warp >= 2 && warp < 10) {
    // ---------------- layer-0 conversion: acc0 -> GELU -> BF16 A stage ----------------
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + kF01Acc0 + 32 * half;
    const int row = q * 32 + lane;              // row of the CTA's 128-row tile
    uint32_t j0 = 0, ia = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int kb = 0; kb < KB; ++kb, ++j0, ++ia) {
        if (!mbar_wait(c0full, j0 & 1, abort, g.err, g.budget, g.suspend)) { ok = false; break; }
        tc_fence_after();
        uint32_t r[32];
        tmem_ld32(tb, r);
        tmem_wait(r);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(c0empty);
        const float4* b4 = reinterpret_cast<const float4*>(sb0 + 64 * kb + 32 * half);
        uint32_t w[16];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 b = b4[u];
          const float2 z0 = gelu_fast2(__fadd2_rn(
              make_float2(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1])), make_float2(b.x, b.y)));
          const float2 z1 = gelu_fast2(__fadd2_rn(
              make_float2(__uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3])), make_float2(b.z, b.w)));
          const __nv_bfloat162 h0 = __floats2bfloat162_rn(z0.x, z0.y);
          const __nv_bfloat162 h1 = __floats2bfloat162_rn(z1.x, z1.y);
          memcpy(&w[2 * u], &h0, 4);
          memcpy(&w[2 * u + 1], &h1, 4);
        }
        const int sa = ia % kF01StA;
        if (!mbar_wait(aempty + 8 * sa, ((ia / kF01StA) & 1) ^ 1, abort, g.err, g.budget, g.suspend)) {
          ok = false;
          break;
        }
        // the 128-byte K-major row of the stage: 16-byte unit u sits at u ^ (row mod 8); this
        // warp's 32 columns are units 4 half .. 4 half + 3
        uint8_t* rowp = sA + sa * kF01ABytes + row * kRowBytes;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          *reinterpret_cast<uint4*>(rowp + (((4 * half + u) ^ (row & 7)) * 16)) =
              make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(afull + 8 * sa);
      }
    }
  } else if (warp >= 10) {
    // ---------------- layer-1 epilogue: acc1 -> GELU -> BF16 -> TMA store ----------------
    const int q = warp & 3;
    uint8_t* stg = sOut + (warp - 10) * kF01StageOut;
    int buf = 0;
    if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmO) : "memory");
    TcArgs ea{};
    ea.bias = sb1;                                // indexed by the output column
    ea.out_scale = 1.0f;
    uint32_t jt = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++jt) {
      if (!mbar_wait(c1full, jt & 1, abort, g.err, g.budget, g.suspend)) break;
      tc_fence_after();
      const int64_t m0 = tile_m0(t) + q * 32;
      const int n0 = (int)(t % tiles_n) * kF01Cols;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
      uint32_t r0[32], r1[32];
      int c = 0;
      tmem_ld32(tbase + c, r0);
      for (; c < kF01Cols; c += 64) {
        tmem_wait(r0);
        const int c1 = c + 32;
        if (c1 < kF01Cols) tmem_ld32(tbase + c1, r1);
        if (n0 + c < g.N1)
          epilogue_chunk<kXBF16, kActTanh, false, kModePlain, true>(r0, ea, &tmO, &tmO, M, m0, n0 + c, stg, buf, lane);
        if (c1 >= kF01Cols) break;
        tmem_wait(r1);
        if (c1 + 32 < kF01Cols) tmem_ld32(tbase + c1 + 32, r0);
        if (n0 + c1 < g.N1)
          epilogue_chunk<kXBF16, kActTanh, false, kModePlain, true>(r1, ea, &tmO, &tmO, M, m0, n0 + c1, stg, buf, lane);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(c1empty);
    }
    if (lane == 0) bulk_wait_all();
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
}

}  // namespace

bool tc_encode_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner,
                  uint64_t outer, uint64_t row_pitch_bytes, uint32_t box_inner,
                  uint32_t box_outer, char* err, size_t errlen) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled is not available from the driver");
    return false;
  }
  if (((uintptr_t)base & 15) || (row_pitch_bytes & 15) || box_inner * elem_bytes != kRowBytes) {
    snprintf(err, errlen, "tensor map: base/pitch not 16-byte aligned or box not 128 B");
    return false;
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return false;
  }
  return true;
}

namespace {
bool encode_store(CUtensorMap* map, const void* base, int out_kind, uint64_t cols, uint64_t rows,
                  uint64_t ld_elems, char* err, size_t errlen) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled is not available from the driver");
    return false;
  }
  const int esz = out_bytes(out_kind);
  if (((uintptr_t)base & 15) || ((ld_elems * esz) & 15)) {
    snprintf(err, errlen, "output tensor map: base/pitch not 16-byte aligned");
    return false;
  }
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld_elems * esz};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = out_kind == kXF32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : out_kind == kXBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const CUtensorMapSwizzle sw = esz == 4 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : esz == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled (output) failed (%d)", (int)r);
    return false;
  }
  return true;
}
}  // namespace

bool tc_encode_out(TcLayer& L, uint64_t rows, char* err, size_t errlen) {
  if (!encode_store(&L.tmO, L.out, L.out_kind, (uint64_t)L.N, rows, (uint64_t)L.ldo, err, errlen))
    return false;
  if (L.mode == kModeStoreG)
    return encode_store(&L.tmG, L.gbuf, kXBF16, (uint64_t)L.N, rows, (uint64_t)L.ldg, err, errlen);
  L.tmG = L.tmO;
  return true;
}

int tc_stages(int BN, int out_kind, bool pair) {
  auto pick = [&](auto bn) -> int {
    constexpr int B = decltype(bn)::value;
    if (pair)
      return out_kind == kXF32 ? Cfg<B, kXF32, true>::kStages
             : out_kind == kXBF16 ? Cfg<B, kXBF16, true>::kStages : Cfg<B, kXFP8, true>::kStages;
    // single CTAs: FP32 out is the read-out (no activation), the others hidden layers
    return out_kind == kXF32 ? Cfg<B, kXF32>::kStages
           : out_kind == kXBF16 ? Cfg<B, kXBF16, false, epi_per_quarter(false, kActTanh)>::kStages
                                : Cfg<B, kXFP8, false, epi_per_quarter(false, kActTanh)>::kStages;
  };
  switch (BN) {
    case 32: return pick(std::integral_constant<int, 32>{});
    case 64: return pick(std::integral_constant<int, 64>{});
    case 128: return pick(std::integral_constant<int, 128>{});
    case 160: return pick(std::integral_constant<int, 160>{});
    case 192: return pick(std::integral_constant<int, 192>{});
    case 224: return pick(std::integral_constant<int, 224>{});
    case 256: return pick(std::integral_constant<int, 256>{});
    default: return 0;
  }
}

int tc_epi_warps_per_quarter() { return epi_per_quarter(false, kActTanh); }

cudaError_t prepare_tc(const TcLayer& L) {
  TcArgs a{};
  return L.elem_bytes == 1 ? launch_fmt<true>(L, a, 0, nullptr) : launch_fmt<false>(L, a, 0, nullptr);
}

cudaError_t launch_tc_gemm(const TcLayer& L, const RowMap& rows, int num_sms, int* err,
                           cudaStream_t st) {
  if (rows.nmax <= 0) return cudaSuccess;
  TcArgs a;
  a.rows = rows;
  a.N = L.N;
  a.K = L.K;
  a.bias = L.bias;
  a.col_scale = L.col_scale;
  a.out = L.out;
  a.ldo = L.ldo;
  a.out_kind = L.out_kind;
  a.gelu = L.gelu ? 1 : 0;
  a.out_scale = L.out_scale;
  a.err = err;
  a.gbuf = L.gbuf;
  a.ldg = L.ldg;
  a.ntan = L.ntan > 0 ? L.ntan : 1;
  a.gtab = L.gtab;
  a.ksplit = L.ksplit > 0 ? L.ksplit : 1;
  a.split_rows = L.split_rows;
  a.budget = L.wait_budget > 0 ? L.wait_budget : kWaitBudget;
  // a short budget needs a short suspend hint, or one try_wait could outlast it
  a.suspend = a.budget < kWaitBudget ? 32u : kSuspendNs;
  return L.elem_bytes == 1 ? launch_fmt<true>(L, a, num_sms, st)
                           : launch_fmt<false>(L, a, num_sms, st);
}

// ---- fused layers 0 and 1 (host side) ----
// Two 416-column tiles cover layer 1 with little padding only for 768..832 outputs; layer 0 must
// fit one 64-element k-block and give whole 64-column blocks.
bool f01_supported(int K0, int N0, int N1) {
  return K0 >= 1 && K0 <= 64 && N0 >= 64 && N0 % 64 == 0 && N0 <= kF01MaxN0 && N1 >= 768 &&
         N1 <= 2 * kF01Cols;
}

bool f01_encode(F01Layer& F, const void* W0, int64_t ldw0, const void* W1, int64_t ldw1, char* err,
                size_t errlen) {
  return tc_encode_2d(&F.tmW0, W0, 2, (uint64_t)F.K0, (uint64_t)F.N0, (uint64_t)ldw0 * 2, 64, 64,
                      err, errlen) &&
         tc_encode_2d(&F.tmW1a, W1, 2, (uint64_t)F.N0, (uint64_t)F.N1, (uint64_t)ldw1 * 2, 64,
                      kF01N1a, err, errlen) &&
         tc_encode_2d(&F.tmW1b, W1, 2, (uint64_t)F.N0, (uint64_t)F.N1, (uint64_t)ldw1 * 2, 64,
                      kF01N1b, err, errlen);
}

namespace {
// the kernel's dynamic shared memory, once per device
cudaError_t f01_attr() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!done[dev]) {
    e = cudaFuncSetAttribute(fused01_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kF01Smem);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t prepare_f01() { return f01_attr(); }

cudaError_t launch_f01(const F01Layer& F, const RowMap& rows, int num_sms, int* err, cudaStream_t st) {
  if (rows.nmax <= 0) return cudaSuccess;
  cudaError_t e = f01_attr();
  if (e != cudaSuccess) return e;
  F01Args a;
  a.rows = rows;
  a.N0 = F.N0;
  a.N1 = F.N1;
  a.K0 = F.K0;
  a.b0 = F.b0;
  a.b1 = F.b1;
  a.err = err;
  a.budget = F.wait_budget > 0 ? F.wait_budget : kWaitBudget;
  a.suspend = a.budget < kWaitBudget ? 32u : kSuspendNs;
  const int64_t tiles = ((rows.nmax + BM - 1) / BM) * ((F.N1 + kF01Cols - 1) / kF01Cols);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms));
  fused01_kernel<<<grid, kF01Threads, kF01Smem, st>>>(F.tmX, F.tmW0, F.tmW1a, F.tmW1b, F.tmO, a);
  return cudaGetLastError();
}

}  // namespace dfgb
