// Sparse-solver kernels of the many-core PDE solver (Sec. 3.2) on one GB300: the block-sparse
// matrix (Sec. 3.2.2) and its LDU conversion, SpMV and block Gauss-Seidel (Sec. 3.2.3), and
// the conflict-free face-to-cell assembly (Sec. 3.2.4).
//
// Layout in HBM (rows in the solver's numbering; block row I = rows part[I] .. part[I+1]-1):
//   dg, rd      [n]      diagonal and its reciprocal (FP64)
//   lrp         [n+1]    start of each row's in-block entries LEFT of the diagonal (the
//   lc, lv      [nnzL]   Gauss-Seidel "lower" part), ascending column: 16-bit column local to
//                        the block row, FP64 value; a block row's lower entries are contiguous
//   urp, uc, uv          the same for the in-block entries RIGHT of the diagonal
//   orp         [n+1]    start of each row's off-block entries
//   oc, oh, ov  [nnzO]   off-block entries: global column, slot of that column in the halo
//                        list, FP64 value
//   lmap, umap, omap     position of every entry in the LDU arrays: 2 f + 1 for upper[f],
//                        2 f for lower[f] (the precomputed map of Sec. 3.2.2)
//   ch_ptr, ch_row       Gauss-Seidel schedule: block row I is swept as chunks
//                        ch_ptr[I] .. ch_ptr[I+1]-1; chunk k is rows ch_row[k] .. ch_row[k+1]-1,
//                        at most 32 consecutive rows none of which has a lower entry inside
//                        the chunk (a piece of a "run", a maximal range with that property)
//   halo_ptr, halo       cells some other block row reads, ascending (so grouped by block row)
//   cf_ptr, cf           faces of every cell, ascending (the assembly's gather lists)
//   order       [n]      the rows of each block row (16-bit local index) by descending number
//                        of entries: the row order in which SpMV and Gauss-Seidel part 1 hand
//                        rows to threads, so that a warp's rows have similar lengths and its
//                        FP64 instructions run with few idle lanes (results do not depend on it)
//
// SpMV gives one CTA to a block row. A Gauss-Seidel sweep is split where its dependencies are:
// the part of every row that uses only values from before the sweep (upper and off-block
// entries) is a streaming kernel like SpMV, and the dependent part (lower entries) gives one
// warp to a block row, chunk by chunk, the GPU form of the paper's one-thread-per-block-row
// sweep; with only the block row's new x in shared memory, tens of such warps share an SM and
// hide each other's latency. Everything a CTA or warp writes belongs to its own block row, so
// no two of them write one value and every result is deterministic.
#include "state.cuh"
#include "ddfloat.cuh"
#include "../../include/df_solver.h"

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <string>
#include <vector>

namespace {

constexpr int kThreads = 256;     // SpMV, Gauss-Seidel part 1, conversion, assembly

struct SolverDev {
  const int32_t* part = nullptr;
  const int32_t* lrp = nullptr;
  const uint16_t* lc = nullptr;
  double* lv = nullptr;
  const int32_t* lmap = nullptr;
  const int32_t* urp = nullptr;
  const uint16_t* uc = nullptr;
  double* uv = nullptr;
  const int32_t* umap = nullptr;
  const int32_t* orp = nullptr;
  const int32_t* oc = nullptr;
  const int32_t* oh = nullptr;
  double* ov = nullptr;
  const int32_t* omap = nullptr;
  double* dg = nullptr;
  double* rd = nullptr;
  const int32_t* ch_ptr = nullptr;
  const int32_t* ch_row = nullptr;
  const int32_t* halo_ptr = nullptr;
  const int32_t* halo = nullptr;
  const int32_t* cf_ptr = nullptr;
  const int32_t* cf = nullptr;
  const uint16_t* order = nullptr;   // per block row: local rows by descending entry count
  int64_t n = 0, nf = 0, nnzL = 0, nnzU = 0, nnzO = 0, nh = 0;
  int t = 0;
};

// Double-float helpers (arithmetic DF_SOLVER_DOUBLE_FLOAT): a value is a pair of FP32 numbers
// held as float2 in memory, so that shared-memory and global accesses are single 8-byte ones.
__device__ __forceinline__ f2 ld2(const float2* p) {
  const float2 v = *p;
  return f2{v.x, v.y};
}
__device__ __forceinline__ void st2(float2* p, f2 a) { *p = make_float2(a.h, a.l); }

// ---------------------------------------------------------------------------------------
// Sec. 3.2.2: values of the block matrix from the LDU arrays through the position maps.
__device__ __forceinline__ double ldu_value(int32_t m, const double* lower, const double* upper) {
  return (m & 1) ? upper[m >> 1] : lower[m >> 1];
}

__global__ void convert_kernel(SolverDev d, const double* __restrict__ lower,
                               const double* __restrict__ diag, const double* __restrict__ upper) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t e = i0; e < d.nnzL; e += stride) d.lv[e] = ldu_value(d.lmap[e], lower, upper);
  for (int64_t e = i0; e < d.nnzU; e += stride) d.uv[e] = ldu_value(d.umap[e], lower, upper);
  for (int64_t e = i0; e < d.nnzO; e += stride) d.ov[e] = ldu_value(d.omap[e], lower, upper);
  for (int64_t r = i0; r < d.n; r += stride) {
    const double a = diag[r];
    d.dg[r] = a;
    d.rd[r] = 1.0 / a;
  }
}

// ---------------------------------------------------------------------------------------
// Sec. 3.2.3: y = A x (RESID: y = b - A x). One CTA per block row, one thread per row; the row
// is summed as diagonal, lower, upper, off-block entries. FP64: FP64 fused multiply-adds.
// F2: the block row's x is split once into double-float pairs in shared memory, every product
// and sum is double-float on the FP32 pipes, and each row is rounded back to FP64 at the end.
// (Measured on this GPU: with rows of 4-13 entries, one thread per row beats a warp-wide
// coalesced walk of the entries with a shared-memory segmented sum, in both arithmetics.)
template <bool RESID, bool F2>
__global__ void __launch_bounds__(kThreads) spmv_kernel(SolverDev d, const double* __restrict__ x,
                                                        const double* __restrict__ b,
                                                        double* __restrict__ y) {
  const int I = blockIdx.x;
  const int r0 = d.part[I], r1 = d.part[I + 1];
  if constexpr (!F2) {
    const double* __restrict__ xI = x + r0;
    for (int j = threadIdx.x; j < r1 - r0; j += kThreads) {
      const int r = r0 + d.order[r0 + j];
      double s = d.dg[r] * x[r];
      const int l1 = d.lrp[r + 1];
      for (int e = d.lrp[r]; e < l1; ++e) s = fma(d.lv[e], xI[d.lc[e]], s);
      const int u1 = d.urp[r + 1];
      for (int e = d.urp[r]; e < u1; ++e) s = fma(d.uv[e], xI[d.uc[e]], s);
      const int o1 = d.orp[r + 1];
      for (int e = d.orp[r]; e < o1; ++e) s = fma(d.ov[e], x[d.oc[e]], s);
      y[r] = RESID ? b[r] - s : s;
    }
  } else {
    extern __shared__ __align__(16) unsigned char spmv_smem[];
    float2* xs = reinterpret_cast<float2*>(spmv_smem);
    for (int i = threadIdx.x; i < r1 - r0; i += kThreads) st2(xs + i, f2_from(x[r0 + i]));
    __syncthreads();
    for (int j = threadIdx.x; j < r1 - r0; j += kThreads) {
      const int r = r0 + d.order[r0 + j];
      f2 s = f2_mul(f2_from(d.dg[r]), ld2(xs + (r - r0)));
      const int l1 = d.lrp[r + 1];
      for (int e = d.lrp[r]; e < l1; ++e) acc_fma(s, f2_from(d.lv[e]), ld2(xs + d.lc[e]));
      const int u1 = d.urp[r + 1];
      for (int e = d.urp[r]; e < u1; ++e) acc_fma(s, f2_from(d.uv[e]), ld2(xs + d.uc[e]));
      const int o1 = d.orp[r + 1];
      for (int e = d.orp[r]; e < o1; ++e) acc_fma(s, f2_from(d.ov[e]), f2_from(x[d.oc[e]]));
      s = f2_fin(s);
      if (RESID) s = f2_fin(f2_add(f2_from(b[r]), f2_neg(s)));
      y[r] = f2_to_int(s);
    }
  }
}

// Halo values of x before the first sweep (FP64, or double-float pairs for F2).
template <bool F2>
__global__ void halo_gather_kernel(SolverDev d, const double* __restrict__ x, void* __restrict__ h) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.nh; k += stride) {
    if constexpr (F2) st2(static_cast<float2*>(h) + k, f2_from(x[d.halo[k]]));
    else static_cast<double*>(h)[k] = x[d.halo[k]];
  }
}

// Sec. 3.2.3, Gauss-Seidel part 1: the part of every row that uses only values from before the
// sweep, p_r = b_r - sum over upper entries of a_rc x_c - sum over off-block entries of a_rc h_c
// (x_c of the block row before the sweep, h_c the halo value of another block's cell). No row
// depends on another: one CTA per block row, one thread per row, like SpMV. p is FP64, or a
// double-float pair for F2.
template <bool F2>
__global__ void __launch_bounds__(kThreads) gs_rhs_kernel(SolverDev d, const double* __restrict__ b,
                                                          const double* __restrict__ x,
                                                          const void* __restrict__ hold,
                                                          void* __restrict__ p) {
  const int I = blockIdx.x;
  const int r0 = d.part[I], r1 = d.part[I + 1];
  const double* __restrict__ xI = x + r0;
  for (int j = threadIdx.x; j < r1 - r0; j += kThreads) {
    const int r = r0 + d.order[r0 + j];
    const int u1 = d.urp[r + 1], o1 = d.orp[r + 1];
    if constexpr (F2) {
      const float2* h2 = static_cast<const float2*>(hold);
      f2 s = f2_from(b[r]);
      for (int e = d.urp[r]; e < u1; ++e) acc_fma(s, f2_neg(f2_from(d.uv[e])), f2_from(xI[d.uc[e]]));
      for (int e = d.orp[r]; e < o1; ++e) acc_fma(s, f2_neg(f2_from(d.ov[e])), ld2(h2 + d.oh[e]));
      st2(static_cast<float2*>(p) + r, f2_fin(s));
    } else {
      const double* h64 = static_cast<const double*>(hold);
      double s = b[r];
      for (int e = d.urp[r]; e < u1; ++e) s = fma(-d.uv[e], xI[d.uc[e]], s);
      for (int e = d.orp[r]; e < o1; ++e) s = fma(-d.ov[e], h64[d.oh[e]], s);
      static_cast<double*>(p)[r] = s;
    }
  }
}

// Asynchronous L2 prefetch of the byte range [p, p + bytes) widened to 16-byte bounds
// (cp.async.bulk.prefetch). Used only on the solver's own arrays, which are allocated with 16
// bytes of slack at the end.
__device__ __forceinline__ void prefetch_l2(const void* p, int64_t bytes) {
  if (bytes <= 0) return;
  const uint64_t a = (uint64_t)p & ~uint64_t(15);
  const uint64_t z = ((uint64_t)p + (uint64_t)bytes + 15) & ~uint64_t(15);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(z - a)) : "memory");
}

constexpr int kPrefetchChunks = 4;   // chunks whose data is fetched into L2 ahead of the sweep

// Shared memory of one sweeping warp, in bytes: the block row's new x (8 per cell), its row
// offsets into its lower entries (4 per cell + 4) and its chunk bounds (2 per chunk + 2).
struct SweepSmem {
  int lrp, ch, per_warp;
};

inline SweepSmem sweep_smem(int max_part, int max_chunks) {
  auto up16 = [](int v) { return (v + 15) & ~15; };
  SweepSmem L;
  L.lrp = up16(8 * max_part);
  L.ch = L.lrp + up16(4 * (max_part + 1));
  L.per_warp = L.ch + up16(2 * (max_chunks + 1));
  return L;
}

// Everything chunk k of the sweep reads from global memory, prefetched into L2 by lanes 0-4.
__device__ __forceinline__ void prefetch_chunk(const SolverDev& d, const void* p, int k, int lane) {
  const int rs = d.ch_row[k], re = d.ch_row[k + 1];
  switch (lane) {
    case 0: {
      const int e0 = d.lrp[rs], e1 = d.lrp[re];
      prefetch_l2(d.lv + e0, 8 * (int64_t)(e1 - e0));
      break;
    }
    case 1: {
      const int e0 = d.lrp[rs], e1 = d.lrp[re];
      prefetch_l2(d.lc + e0, 2 * (int64_t)(e1 - e0));
      break;
    }
    case 2: prefetch_l2(static_cast<const double*>(p) + rs, 8 * (int64_t)(re - rs)); break;
    case 3: prefetch_l2(d.rd + rs, 8 * (int64_t)(re - rs)); break;
    case 4: prefetch_l2(d.lrp + rs, 4 * (int64_t)(re - rs + 1)); break;
    default: break;
  }
}

// Row data of one chunk for one lane of the sweep: the row's p and 1/a_rr and its first
// kLowerRegs lower entries, loaded into registers one chunk ahead of their use. Rows with more
// lower entries read the rest from global memory when they are swept.
constexpr int kLowerRegs = 6;

template <bool F2>
struct SweepRow {
  int i = 0, cnt = -1, e0 = 0;            // local row, lower entries (-1: no row), first entry
  double pv = 0.0, rdv = 0.0;             // p (or its double-float pair, as bits) and 1/a_rr
  double lvv[kLowerRegs];
  int lcv[kLowerRegs];
};

template <bool F2>
__device__ __forceinline__ void sweep_load(const SolverDev& d, const void* p, int r0, int a0,
                                           const uint16_t* chs, const int32_t* lrps, int k,
                                           int lane, SweepRow<F2>& q) {
  const int i = chs[k] + lane;
  q.cnt = -1;
  if (i < chs[k + 1]) {
    q.i = i;
    q.e0 = a0 + lrps[i];
    q.cnt = lrps[i + 1] - lrps[i];
    q.pv = static_cast<const double*>(p)[r0 + i];   // FP64, or the bits of a float2 pair
    q.rdv = d.rd[r0 + i];
#pragma unroll
    for (int j = 0; j < kLowerRegs; ++j) {
      if (j >= q.cnt) break;
      q.lvv[j] = d.lv[q.e0 + j];
      q.lcv[j] = d.lc[q.e0 + j];
    }
  }
}

// Sec. 3.2.3, Gauss-Seidel part 2: the dependent part of the sweep, one warp per block row. In
// ascending order, x_r = (p_r - sum over lower entries of a_rc x_c) * (1/a_rr): lane j takes row
// j of chunk k (rows of a chunk do not depend on each other; __syncwarp orders the chunks).
// Only lower entries are read and their rows were updated earlier in this sweep, so the block
// row's new x is built in shared memory without loading the old one. The chunk bounds and row
// offsets of the block row are staged in shared memory first; each chunk's row data is loaded
// into registers while the previous chunk is swept, and fetched into L2 further ahead, so the
// dependency chain holds only shared-memory reads and arithmetic. At the end x is written
// back, and the block row's halo cells go to hnew for the next sweep.
template <bool F2>
__global__ void __launch_bounds__(128) gs_sweep_kernel(SolverDev d, const void* __restrict__ p,
                                                       double* __restrict__ x,
                                                       void* __restrict__ hnew, SweepSmem L) {
  extern __shared__ __align__(16) unsigned char gs_smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int I = blockIdx.x * (blockDim.x >> 5) + warp;
  if (I >= d.t) return;                 // no block-wide barrier below: whole warps leave
  unsigned char* base = gs_smem_raw + (size_t)warp * L.per_warp;
  double* xs = reinterpret_cast<double*>(base);
  float2* xs2 = reinterpret_cast<float2*>(base);
  int32_t* lrps = reinterpret_cast<int32_t*>(base + L.lrp);
  uint16_t* chs = reinterpret_cast<uint16_t*>(base + L.ch);
  const int r0 = d.part[I], m = d.part[I + 1] - r0;
  const int k0 = d.ch_ptr[I], nk = d.ch_ptr[I + 1] - k0;
  const int a0 = d.lrp[r0];
  for (int k = k0; k < k0 + nk && k < k0 + kPrefetchChunks; ++k) prefetch_chunk(d, p, k, lane);
  for (int j = lane; j <= nk; j += 32) chs[j] = (uint16_t)(d.ch_row[k0 + j] - r0);
  for (int i = lane; i <= m; i += 32) lrps[i] = d.lrp[r0 + i] - a0;
  __syncwarp();
  SweepRow<F2> cur, nxt;
  if (nk > 0) sweep_load<F2>(d, p, r0, a0, chs, lrps, 0, lane, cur);
  for (int k = 0; k < nk; ++k) {
    if (k + 1 < nk) sweep_load<F2>(d, p, r0, a0, chs, lrps, k + 1, lane, nxt);
    if (k + kPrefetchChunks < nk) prefetch_chunk(d, p, k0 + k + kPrefetchChunks, lane);
    if (cur.cnt >= 0) {
      if constexpr (F2) {
        f2 s = f2{__int_as_float(__double2loint(cur.pv)), __int_as_float(__double2hiint(cur.pv))};
#pragma unroll
        for (int j = 0; j < kLowerRegs; ++j) {
          if (j >= cur.cnt) break;
          acc_fma(s, f2_neg(f2_from(cur.lvv[j])), ld2(xs2 + cur.lcv[j]));
        }
        for (int j = kLowerRegs; j < cur.cnt; ++j)
          acc_fma(s, f2_neg(f2_from(d.lv[cur.e0 + j])), ld2(xs2 + d.lc[cur.e0 + j]));
        st2(xs2 + cur.i, f2_mul(f2_fin(s), f2_from(cur.rdv)));
      } else {
        double s = cur.pv;
#pragma unroll
        for (int j = 0; j < kLowerRegs; ++j) {
          if (j >= cur.cnt) break;
          s = fma(-cur.lvv[j], xs[cur.lcv[j]], s);
        }
        for (int j = kLowerRegs; j < cur.cnt; ++j) s = fma(-d.lv[cur.e0 + j], xs[d.lc[cur.e0 + j]], s);
        xs[cur.i] = s * cur.rdv;
      }
    }
    __syncwarp();
    cur = nxt;
  }
  for (int i = lane; i < m; i += 32) {
    if constexpr (F2) x[r0 + i] = f2_to_int(ld2(xs2 + i));
    else x[r0 + i] = xs[i];
  }
  if (hnew) {
    for (int k = d.halo_ptr[I] + lane; k < d.halo_ptr[I + 1]; k += 32) {
      if constexpr (F2) static_cast<float2*>(hnew)[k] = xs2[d.halo[k] - r0];
      else static_cast<double*>(hnew)[k] = xs[d.halo[k] - r0];
    }
  }
}

// Warps (block rows) per sweep CTA: as many as fit 192 KB of shared memory, at most 4.
int sweep_warps(const SweepSmem& L) { return std::max(1, std::min(4, 196608 / L.per_warp)); }

// ---------------------------------------------------------------------------------------
// Sec. 3.2.4: the face-to-cell Laplacian. Face coefficients are written by one thread per
// face, each diagonal by one thread per cell gathering its faces in ascending order.
__global__ void laplacian_kernel(SolverDev d, const double* __restrict__ g,
                                 const double* __restrict__ s, double* __restrict__ lower,
                                 double* __restrict__ diag, double* __restrict__ upper) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t f = i0; f < d.nf; f += stride) {
    const double v = -g[f];
    lower[f] = v;
    upper[f] = v;
  }
  for (int64_t c = i0; c < d.n; c += stride) {
    double a = s[c];
    const int k1 = d.cf_ptr[c + 1];
    for (int k = d.cf_ptr[c]; k < k1; ++k) a += g[d.cf[k]];
    diag[c] = a;
  }
}

int grid_for(int64_t work, int num_sms) {
  const int64_t blocks = (work + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * 8));
}

}  // namespace

struct df_solver {
  int device = 0;
  int num_sms = 0;
  int64_t n = 0, nf = 0;
  int t = 0;
  int max_part = 0, max_runs = 0, max_chunks = 0;
  int64_t nruns = 0, nchunks = 0;
  int arith = DF_SOLVER_FP64;
  bool converted = false;
  size_t bytes = 0;
  std::string err;
  SolverDev d;
  double* hbuf[2] = {nullptr, nullptr};
  double* pbuf = nullptr;                // Gauss-Seidel part-1 sums p [n]
  std::vector<void*> allocs;
  // host copies of the structure, for df_solver_export_csr
  std::vector<int32_t> h_part, h_lrp, h_urp, h_orp, h_oc;
  std::vector<uint16_t> h_lc, h_uc;
};

namespace {

df_status sfail(const df_solver* s, df_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) const_cast<df_solver*>(s)->err = buf;
  else dfgb::fail(nullptr, code, "%s", buf);
  return code;
}

// Device arrays carry 16 bytes of slack past their end, so that a bulk L2 prefetch of a range
// widened to 16-byte bounds never leaves the allocation.
constexpr size_t kSlack = 16;

template <typename T>
cudaError_t upload(df_solver* s, const T** dst, const std::vector<T>& src) {
  T* p = nullptr;
  const size_t bytes = sizeof(T) * src.size() + kSlack;
  cudaError_t e = cudaMalloc((void**)&p, bytes);
  if (e != cudaSuccess) return e;
  s->allocs.push_back(p);
  s->bytes += bytes;
  if (!src.empty()) e = cudaMemcpy(p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
  *dst = p;
  return e;
}

template <typename T>
cudaError_t alloc(df_solver* s, T** dst, size_t count) {
  T* p = nullptr;
  const size_t bytes = sizeof(T) * count + kSlack;
  cudaError_t e = cudaMalloc((void**)&p, bytes);
  if (e != cudaSuccess) return e;
  s->allocs.push_back(p);
  s->bytes += bytes;
  *dst = p;
  return cudaSuccess;
}

void release(df_solver* s) {
  if (!s) return;
  DeviceGuard g(s->device);
  for (void* p : s->allocs) cudaFree(p);
  s->allocs.clear();
}

df_status check_ready(df_solver* s) {
  if (!s) return sfail(nullptr, DF_ERR_INVALID_ARG, "solver is NULL");
  if (!s->converted) return sfail(s, DF_ERR_INVALID_ARG, "no matrix yet: call df_solver_convert first");
  return DF_OK;
}

}  // namespace

extern "C" {

df_status df_solver_create(int64_t n_cells, int64_t n_faces, const int32_t* owner,
                           const int32_t* neighbour, int32_t n_parts, const int64_t* part_ptr,
                           int32_t device, df_solver** out) {
  if (!out) return sfail(nullptr, DF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_cells <= 0 || n_cells >= (int64_t(1) << 31) || n_faces < 0 || n_faces >= (int64_t(1) << 30))
    return sfail(nullptr, DF_ERR_INVALID_ARG, "n_cells must be in 1..2^31-1, n_faces in 0..2^30-1");
  if (n_faces > 0 && (!owner || !neighbour)) return sfail(nullptr, DF_ERR_INVALID_ARG, "NULL face array");
  if (!part_ptr || n_parts < 1 || n_parts > n_cells)
    return sfail(nullptr, DF_ERR_INVALID_ARG, "bad block rows");
  if (part_ptr[0] != 0 || part_ptr[n_parts] != n_cells)
    return sfail(nullptr, DF_ERR_INVALID_ARG, "part_ptr must run from 0 to n_cells");
  int max_part = 0;
  for (int p = 0; p < n_parts; ++p) {
    const int64_t sz = part_ptr[p + 1] - part_ptr[p];
    if (sz < 1 || sz > DF_SOLVER_MAX_PART)
      return sfail(nullptr, DF_ERR_INVALID_ARG, "block row %d has %lld cells (1..%d allowed)", p,
                   (long long)sz, DF_SOLVER_MAX_PART);
    max_part = std::max(max_part, (int)sz);
  }
  for (int64_t f = 0; f < n_faces; ++f) {
    if (owner[f] < 0 || owner[f] >= neighbour[f] || neighbour[f] >= n_cells)
      return sfail(nullptr, DF_ERR_INVALID_ARG, "face %lld: need 0 <= owner < neighbour < n_cells",
                   (long long)f);
  }
  const int64_t n = n_cells;
  std::vector<int32_t> part_of(n);
  std::vector<int32_t> hpart(n_parts + 1);
  for (int p = 0; p < n_parts; ++p) {
    hpart[p] = (int32_t)part_ptr[p];
    for (int64_t r = part_ptr[p]; r < part_ptr[p + 1]; ++r) part_of[r] = p;
  }
  hpart[n_parts] = (int32_t)n;

  // every row's entries: (column, LDU position), split lower / upper in-block and off-block
  std::vector<int32_t> deg(n + 1, 0);
  for (int64_t f = 0; f < n_faces; ++f) {
    ++deg[owner[f] + 1];
    ++deg[neighbour[f] + 1];
  }
  std::vector<int64_t> rp(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) rp[r + 1] = rp[r] + deg[r + 1];
  std::vector<int32_t> col(2 * n_faces), pos(2 * n_faces);
  {
    std::vector<int64_t> w(rp.begin(), rp.end() - 1);
    for (int64_t f = 0; f < n_faces; ++f) {
      const int32_t a = owner[f], b = neighbour[f];
      col[w[a]] = b; pos[w[a]++] = (int32_t)(2 * f + 1);   // A[a][b] = upper[f]
      col[w[b]] = a; pos[w[b]++] = (int32_t)(2 * f);       // A[b][a] = lower[f]
    }
  }
  std::vector<int32_t> lrp(n + 1, 0), urp(n + 1, 0), orp(n + 1, 0);
  std::vector<uint16_t> lc, uc;
  std::vector<int32_t> lmap, umap, oc, omap;
  lc.reserve(n_faces);
  uc.reserve(n_faces);
  lmap.reserve(n_faces);
  umap.reserve(n_faces);
  std::vector<std::pair<int32_t, int32_t>> ent;
  for (int64_t r = 0; r < n; ++r) {
    ent.clear();
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) ent.emplace_back(col[k], pos[k]);
    std::sort(ent.begin(), ent.end());
    for (size_t k = 1; k < ent.size(); ++k)
      if (ent[k].first == ent[k - 1].first)
        return sfail(nullptr, DF_ERR_INVALID_ARG, "cells %lld and %d share more than one face",
                     (long long)r, ent[k].first);
    const int p = part_of[r];
    const int32_t base = hpart[p];
    for (auto& e : ent) {
      if (part_of[e.first] != p) {
        oc.push_back(e.first);
        omap.push_back(e.second);
      } else if (e.first < r) {
        lc.push_back((uint16_t)(e.first - base));
        lmap.push_back(e.second);
      } else {
        uc.push_back((uint16_t)(e.first - base));
        umap.push_back(e.second);
      }
    }
    lrp[r + 1] = (int32_t)lc.size();
    urp[r + 1] = (int32_t)uc.size();
    orp[r + 1] = (int32_t)oc.size();
  }
  col.clear(); col.shrink_to_fit();
  pos.clear(); pos.shrink_to_fit();

  // Gauss-Seidel schedule: runs (a new run starts where a row depends on a row of the current
  // run), cut into chunks of at most 32 rows
  std::vector<int32_t> ch_ptr(n_parts + 1, 0), ch_row;
  int max_runs = 0, max_chunks = 0;
  int64_t nruns = 0;
  for (int p = 0; p < n_parts; ++p) {
    const int32_t base = hpart[p];
    int32_t run_start = base, chunk_start = base;
    int runs_here = 1;
    ch_row.push_back(base);
    for (int32_t r = base + 1; r < hpart[p + 1]; ++r) {
      const bool new_run = lrp[r + 1] > lrp[r] && base + lc[lrp[r + 1] - 1] >= run_start;
      if (new_run) {
        run_start = r;
        ++runs_here;
      }
      if (new_run || r - chunk_start == 32) {
        ch_row.push_back(r);
        chunk_start = r;
      }
    }
    ch_ptr[p + 1] = (int32_t)ch_row.size();
    max_chunks = std::max(max_chunks, ch_ptr[p + 1] - ch_ptr[p]);
    max_runs = std::max(max_runs, runs_here);
    nruns += runs_here;
  }
  ch_row.push_back((int32_t)n);

  // row order for the thread-per-row kernels: within each block row, by descending number of
  // (lower + upper + off-block) entries, ties in ascending row order
  std::vector<uint16_t> order(n);
  for (int p = 0; p < n_parts; ++p) {
    const int32_t base = hpart[p], m = hpart[p + 1] - base;
    std::vector<std::pair<int, int>> key(m);
    for (int i = 0; i < m; ++i) {
      const int32_t r = base + i;
      const int len = (lrp[r + 1] - lrp[r]) + (urp[r + 1] - urp[r]) + (orp[r + 1] - orp[r]);
      key[i] = {-len, i};
    }
    std::sort(key.begin(), key.end());
    for (int i = 0; i < m; ++i) order[base + i] = (uint16_t)key[i].second;
  }

  // halo: cells read through off-block entries, ascending; each entry's slot in it
  std::vector<int32_t> halo(oc.begin(), oc.end());
  std::sort(halo.begin(), halo.end());
  halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
  std::vector<int32_t> oh(oc.size());
  for (size_t k = 0; k < oc.size(); ++k)
    oh[k] = (int32_t)(std::lower_bound(halo.begin(), halo.end(), oc[k]) - halo.begin());
  std::vector<int32_t> halo_ptr(n_parts + 1, 0);
  for (int p = 0; p <= n_parts; ++p)
    halo_ptr[p] = (int32_t)(std::lower_bound(halo.begin(), halo.end(), hpart[p]) - halo.begin());

  // faces of every cell, ascending (assembly gather lists)
  std::vector<int32_t> cf_ptr(n + 1, 0), cf(2 * n_faces);
  for (int64_t r = 0; r < n; ++r) cf_ptr[r + 1] = cf_ptr[r] + deg[r + 1];
  {
    std::vector<int32_t> w(cf_ptr.begin(), cf_ptr.end() - 1);
    for (int64_t f = 0; f < n_faces; ++f) {
      cf[w[owner[f]]++] = (int32_t)f;
      cf[w[neighbour[f]]++] = (int32_t)f;
    }
  }

  df_solver* s = new df_solver();
  s->device = device;
  s->n = n;
  s->nf = n_faces;
  s->t = n_parts;
  s->max_part = max_part;
  s->max_runs = max_runs;
  s->max_chunks = max_chunks;
  s->nruns = nruns;
  s->nchunks = (int64_t)ch_row.size() - 1;
  DeviceGuard guard(device);
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (s->num_sms <= 0) s->num_sms = 1;
  SolverDev& d = s->d;
  d.n = n;
  d.nf = n_faces;
  d.nnzL = (int64_t)lc.size();
  d.nnzU = (int64_t)uc.size();
  d.nnzO = (int64_t)oc.size();
  d.nh = (int64_t)halo.size();
  d.t = n_parts;
  cudaError_t e = cudaSuccess;
  auto up = [&](auto** dst, const auto& v) {
    if (e == cudaSuccess) e = upload(s, dst, v);
  };
  up(&d.part, hpart);
  up(&d.lrp, lrp);
  up(&d.lc, lc);
  up(&d.lmap, lmap);
  up(&d.urp, urp);
  up(&d.uc, uc);
  up(&d.umap, umap);
  up(&d.orp, orp);
  up(&d.oc, oc);
  up(&d.oh, oh);
  up(&d.omap, omap);
  up(&d.ch_ptr, ch_ptr);
  up(&d.ch_row, ch_row);
  up(&d.halo_ptr, halo_ptr);
  up(&d.halo, halo);
  up(&d.cf_ptr, cf_ptr);
  up(&d.cf, cf);
  up(&d.order, order);
  if (e == cudaSuccess) e = alloc(s, &d.lv, lc.size());
  if (e == cudaSuccess) e = alloc(s, &d.uv, uc.size());
  if (e == cudaSuccess) e = alloc(s, &d.ov, oc.size());
  if (e == cudaSuccess) e = alloc(s, &d.dg, n);
  if (e == cudaSuccess) e = alloc(s, &d.rd, n);
  if (e == cudaSuccess) e = alloc(s, &s->hbuf[0], halo.size());
  if (e == cudaSuccess) e = alloc(s, &s->hbuf[1], halo.size());
  if (e == cudaSuccess) e = alloc(s, &s->pbuf, n);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gs_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 196608);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gs_sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 196608);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spmv_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             8 * DF_SOLVER_MAX_PART);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spmv_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             8 * DF_SOLVER_MAX_PART);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    release(s);
    delete s;
    return sfail(nullptr, e == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA,
                 "df_solver_create: %s", cudaGetErrorString(e));
  }
  s->h_part = std::move(hpart);
  s->h_lrp = std::move(lrp);
  s->h_urp = std::move(urp);
  s->h_orp = std::move(orp);
  s->h_oc = std::move(oc);
  s->h_lc = std::move(lc);
  s->h_uc = std::move(uc);
  *out = s;
  return DF_OK;
}

void df_solver_destroy(df_solver* s) {
  if (!s) return;
  release(s);
  delete s;
}

df_status df_solver_get_info(const df_solver* s, df_solver_info* info) {
  if (!s || !info) return sfail(s, DF_ERR_INVALID_ARG, "NULL argument");
  info->n_cells = s->n;
  info->n_faces = s->nf;
  info->n_parts = s->t;
  info->nnz = s->n + 2 * s->nf;
  info->nnz_offblock = s->d.nnzO;
  info->n_halo = s->d.nh;
  info->n_runs = s->nruns;
  info->max_part = s->max_part;
  info->max_runs = s->max_runs;
  info->device_bytes = (int64_t)s->bytes;
  info->n_chunks = s->nchunks;
  return DF_OK;
}

df_status df_solver_set_arithmetic(df_solver* s, int32_t arithmetic) {
  if (!s) return sfail(nullptr, DF_ERR_INVALID_ARG, "solver is NULL");
  if (arithmetic != DF_SOLVER_FP64 && arithmetic != DF_SOLVER_DOUBLE_FLOAT)
    return sfail(s, DF_ERR_INVALID_ARG, "unknown arithmetic %d", arithmetic);
  s->arith = arithmetic;
  return DF_OK;
}

df_status df_solver_convert(df_solver* s, const double* lower, const double* diag,
                            const double* upper, void* stream) {
  if (!s) return sfail(nullptr, DF_ERR_INVALID_ARG, "solver is NULL");
  if (!diag || (s->nf > 0 && (!lower || !upper))) return sfail(s, DF_ERR_INVALID_ARG, "NULL array");
  DeviceGuard g(s->device);
  const int64_t work = std::max(std::max(s->d.nnzL, s->d.nnzU), std::max(s->d.nnzO, s->n));
  convert_kernel<<<grid_for(work, s->num_sms), kThreads, 0, (cudaStream_t)stream>>>(s->d, lower, diag,
                                                                                    upper);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sfail(s, DF_ERR_CUDA, "convert launch: %s", cudaGetErrorString(e));
  s->converted = true;
  return DF_OK;
}

df_status df_solver_spmv(df_solver* s, const double* x, double* y, void* stream) {
  if (df_status st = check_ready(s)) return st;
  if (!x || !y || x == y) return sfail(s, DF_ERR_INVALID_ARG, "x and y must be distinct device arrays");
  DeviceGuard g(s->device);
  const cudaStream_t st = (cudaStream_t)stream;
  if (s->arith == DF_SOLVER_DOUBLE_FLOAT)
    spmv_kernel<false, true><<<s->t, kThreads, 8 * (size_t)s->max_part, st>>>(s->d, x, nullptr, y);
  else
    spmv_kernel<false, false><<<s->t, kThreads, 0, st>>>(s->d, x, nullptr, y);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DF_OK : sfail(s, DF_ERR_CUDA, "spmv launch: %s", cudaGetErrorString(e));
}

df_status df_solver_residual(df_solver* s, const double* b, const double* x, double* r, void* stream) {
  if (df_status st = check_ready(s)) return st;
  if (!b || !x || !r || r == x || r == b)
    return sfail(s, DF_ERR_INVALID_ARG, "r must be a device array distinct from b and x");
  DeviceGuard g(s->device);
  const cudaStream_t st = (cudaStream_t)stream;
  if (s->arith == DF_SOLVER_DOUBLE_FLOAT)
    spmv_kernel<true, true><<<s->t, kThreads, 8 * (size_t)s->max_part, st>>>(s->d, x, b, r);
  else
    spmv_kernel<true, false><<<s->t, kThreads, 0, st>>>(s->d, x, b, r);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DF_OK : sfail(s, DF_ERR_CUDA, "residual launch: %s", cudaGetErrorString(e));
}

df_status df_solver_gauss_seidel(df_solver* s, const double* b, double* x, int32_t sweeps,
                                 void* stream) {
  if (df_status st = check_ready(s)) return st;
  if (!b || !x || b == x) return sfail(s, DF_ERR_INVALID_ARG, "b and x must be distinct device arrays");
  if (sweeps < 0) return sfail(s, DF_ERR_INVALID_ARG, "sweeps < 0");
  if (sweeps == 0) return DF_OK;
  DeviceGuard g(s->device);
  const cudaStream_t st = (cudaStream_t)stream;
  const bool f2 = s->arith == DF_SOLVER_DOUBLE_FLOAT;
  if (s->d.nh > 0) {
    const int hg = grid_for(s->d.nh, s->num_sms);
    if (f2) halo_gather_kernel<true><<<hg, kThreads, 0, st>>>(s->d, x, s->hbuf[0]);
    else halo_gather_kernel<false><<<hg, kThreads, 0, st>>>(s->d, x, s->hbuf[0]);
  }
  const SweepSmem L = sweep_smem(s->max_part, s->max_chunks);
  const int w = sweep_warps(L);
  const size_t smem = (size_t)w * L.per_warp;
  const int grid = (s->t + w - 1) / w;
  for (int k = 0; k < sweeps; ++k) {
    const double* hold = s->hbuf[k & 1];
    double* hnew = (k + 1 < sweeps && s->d.nh > 0) ? s->hbuf[(k + 1) & 1] : nullptr;
    if (f2) {
      gs_rhs_kernel<true><<<s->t, kThreads, 0, st>>>(s->d, b, x, hold, s->pbuf);
      gs_sweep_kernel<true><<<grid, 32 * w, smem, st>>>(s->d, s->pbuf, x, hnew, L);
    } else {
      gs_rhs_kernel<false><<<s->t, kThreads, 0, st>>>(s->d, b, x, hold, s->pbuf);
      gs_sweep_kernel<false><<<grid, 32 * w, smem, st>>>(s->d, s->pbuf, x, hnew, L);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DF_OK : sfail(s, DF_ERR_CUDA, "Gauss-Seidel launch: %s", cudaGetErrorString(e));
}

df_status df_fv_laplacian(df_solver* s, const double* face_coeff, const double* cell_source,
                          double* lower, double* diag, double* upper, void* stream) {
  if (!s) return sfail(nullptr, DF_ERR_INVALID_ARG, "solver is NULL");
  if (!cell_source || !diag || (s->nf > 0 && (!face_coeff || !lower || !upper)))
    return sfail(s, DF_ERR_INVALID_ARG, "NULL array");
  DeviceGuard g(s->device);
  const int64_t work = std::max(s->nf, s->n);
  laplacian_kernel<<<grid_for(work, s->num_sms), kThreads, 0, (cudaStream_t)stream>>>(
      s->d, face_coeff, cell_source, lower, diag, upper);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DF_OK : sfail(s, DF_ERR_CUDA, "laplacian launch: %s", cudaGetErrorString(e));
}

df_status df_solver_export_csr(df_solver* s, int64_t* row_ptr, int32_t* col, double* val) {
  if (df_status st = check_ready(s)) return st;
  if (!row_ptr || !col || !val) return sfail(s, DF_ERR_INVALID_ARG, "NULL output array");
  DeviceGuard g(s->device);
  std::vector<double> lv(s->d.nnzL), uv(s->d.nnzU), ov(s->d.nnzO), dg(s->n);
  cudaError_t e = cudaDeviceSynchronize();
  auto get = [&](std::vector<double>& h, const double* dptr) {
    if (e == cudaSuccess && !h.empty())
      e = cudaMemcpy(h.data(), dptr, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
  };
  get(lv, s->d.lv);
  get(uv, s->d.uv);
  get(ov, s->d.ov);
  get(dg, s->d.dg);
  if (e != cudaSuccess) return sfail(s, DF_ERR_CUDA, "export: %s", cudaGetErrorString(e));
  int64_t k = 0;
  int p = 0;
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t r = 0; r < s->n; ++r) {
    while (s->h_part[p + 1] <= r) ++p;
    const int32_t base = s->h_part[p];
    row.clear();
    row.emplace_back((int32_t)r, dg[r]);
    for (int32_t j = s->h_lrp[r]; j < s->h_lrp[r + 1]; ++j) row.emplace_back(base + s->h_lc[j], lv[j]);
    for (int32_t j = s->h_urp[r]; j < s->h_urp[r + 1]; ++j) row.emplace_back(base + s->h_uc[j], uv[j]);
    for (int32_t j = s->h_orp[r]; j < s->h_orp[r + 1]; ++j) row.emplace_back(s->h_oc[j], ov[j]);
    std::sort(row.begin(), row.end(),
              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                return a.first < b.first;
              });
    row_ptr[r] = k;
    for (auto& c : row) {
      col[k] = c.first;
      val[k] = c.second;
      ++k;
    }
  }
  row_ptr[s->n] = k;
  return DF_OK;
}

const char* df_solver_get_last_error(const df_solver* s) {
  return s ? s->err.c_str() : df_get_last_error(nullptr);
}

}  // extern "C"
