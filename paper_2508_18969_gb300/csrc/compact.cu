// a0: stable compaction of the reacting cells (T > T_react) into an ascending index list.
// Three launches, no inter-block waiting: per-chunk counts (warp ballot + popc), one-block
// exclusive scan of the chunk counts, then a scatter that ranks each reacting cell inside
// its chunk with ballot/popc prefix sums. Both chunk passes load all of a thread's cells
// before testing any, so a chunk costs one memory latency. Cells are visited in the same
// order by the count and the scatter pass, so the list is in ascending cell order.
#include "dfgb_internal.cuh"

namespace dfgb {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                         // cells per thread per chunk
constexpr int kChunk = kCompactChunk;              // 4096 cells per block
constexpr int kWarps = kThreads / 32;
constexpr int kCellNonfinite = 4;

__device__ __forceinline__ bool reacts(double t, double thr) { return t > thr; }

__global__ void __launch_bounds__(kThreads) count_kernel(int64_t n, double thr,
    const double* __restrict__ T, int32_t* __restrict__ status, int64_t* __restrict__ counts) {
  __shared__ int warp_tot[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // all of the thread's cells are loaded before any is tested: one memory latency per chunk
  double t[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
    t[j] = i < n ? T[i] : 0.0;
  }
  int mine = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
    const bool a = i < n && reacts(t[j], thr);
    if (status && i < n) status[i] = isfinite(t[j]) ? 0 : kCellNonfinite;
    mine += __popc(__ballot_sync(0xffffffffu, a)) * (lane == 0);
  }
  if (lane == 0) warp_tot[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int w = 0; w < kWarps; ++w) s += warp_tot[w];
    counts[blockIdx.x] = s;
  }
}

// Exclusive scan of nb chunk counts by one block; offsets[b] and the total into *count.
__global__ void __launch_bounds__(1024) scan_kernel(int64_t nb, const int64_t* __restrict__ counts,
                                                    int64_t* __restrict__ offsets,
                                                    int64_t* __restrict__ count) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b0 = t * per, b1 = (b0 + per < nb) ? b0 + per : nb;
  int64_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += counts[b];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {  // Hillis-Steele inclusive scan of the 1024 partials
    int64_t v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = (t > 0) ? part[t - 1] : 0;
  for (int64_t b = b0; b < b1; ++b) {
    offsets[b] = run;
    run += counts[b];
  }
  if (t == 1023) *count = part[1023];
}

__global__ void __launch_bounds__(kThreads) scatter_kernel(int64_t n, double thr,
    const double* __restrict__ T, const int64_t* __restrict__ offsets, int32_t* __restrict__ idx) {
  // reacting cells per (pass j, warp w) of the chunk; the chunk's cells are visited pass by
  // pass, warp by warp, lane by lane, the order of the count pass
  __shared__ int warp_tot[kItems][kWarps];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double t[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
    t[j] = i < n ? T[i] : 0.0;
  }
  unsigned m[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
    m[j] = __ballot_sync(0xffffffffu, i < n && reacts(t[j], thr));
    if (lane == 0) warp_tot[j][warp] = __popc(m[j]);
  }
  __syncthreads();
  int64_t run = offsets[blockIdx.x];
  const unsigned below = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int c = warp_tot[j][w];
      before += (w < warp) ? c : 0;
      total += c;
    }
    if ((m[j] >> lane) & 1u)
      idx[run + before + __popc(m[j] & below)] = (int32_t)(base + (int64_t)j * kThreads + threadIdx.x);
    run += total;
  }
}

}  // namespace

int64_t compact_scratch_words(int64_t n) {
  const int64_t nb = (n + kChunk - 1) / kChunk;
  return 2 * (nb > 0 ? nb : 1);
}

cudaError_t launch_compact(int64_t n, double T_react, const double* T, int32_t* idx,
                           int64_t* count, int32_t* status, int64_t* scratch, cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(count, 0, sizeof(int64_t), st);
  const int64_t nb = (n + kChunk - 1) / kChunk;
  int64_t* counts = scratch;
  int64_t* offsets = scratch + nb;
  count_kernel<<<(unsigned)nb, kThreads, 0, st>>>(n, T_react, T, status, counts);
  scan_kernel<<<1, 1024, 0, st>>>(nb, counts, offsets, count);
  scatter_kernel<<<(unsigned)nb, kThreads, 0, st>>>(n, T_react, T, offsets, idx);
  return cudaGetLastError();
}

}  // namespace dfgb

// ---- allocation-free variant -------------------------------------------------------
// Some callers cannot allocate device memory: a flow solver that has handed the whole
// device to its own pool allocator, or a caller on a path where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable. df_active_compact_static serves
// them: the chunk counts and offsets live in the file-scope array below (256 KB, resident on
// every device that loads this library until the process exits), so the call allocates
// nothing. Every call shares this one array; the count pass writes every entry the scan
// and scatter passes read, so nothing needs clearing, but calls that overlap on the GPU
// (other streams, other host threads) race on it.
#include "../../include/df.h"

#include <mutex>

namespace {

constexpr int64_t kStaticMaxCells = DF_COMPACT_STATIC_MAX_CELLS;
constexpr int64_t kStaticWords = 2 * ((kStaticMaxCells + dfgb::kCompactChunk - 1) / dfgb::kCompactChunk);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int64_t g_compact_scratch[kStaticWords];

std::mutex g_static_mu;

// The address of a __device__ variable belongs to a CUDA context, so it is cached per context:
// a caller that binds its own driver-API context, or one that resets the device and so gets a
// new primary context, is given the address in the context that is current at the call.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
struct ScratchSlot {
  CUcontext ctx;
  int64_t* ptr;
};
constexpr int kMaxSlots = 4 * kMaxDevices;
ScratchSlot g_slots[kMaxSlots] = {};
int g_nslots = 0;

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  }
  return fn;
}

// Device address of g_compact_scratch in the current context, looked up at the first call in
// that context (with its device current). The name is only a host-side handle; the kernel
// must be given this address.
cudaError_t static_scratch(int64_t** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return cudaErrorInitializationError;
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
  for (int i = 0; ctx && i < g_nslots; ++i)
    if (g_slots[i].ctx == ctx) {
      *out = g_slots[i].ptr;
      return cudaSuccess;
    }
  // first call in this context (the lookup also makes the device's primary context current
  // when no context was yet)
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_compact_scratch);
  if (e != cudaSuccess) return e;
  if (get(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorInitializationError;
  ScratchSlot& slot = g_slots[g_nslots < kMaxSlots ? g_nslots++ : kMaxSlots - 1];
  slot.ctx = ctx;
  slot.ptr = static_cast<int64_t*>(p);
  *out = slot.ptr;
  return cudaSuccess;
}

}  // namespace

namespace dfgb {
void set_global_error(const char* msg);  // state.cu
}

extern "C" df_status df_active_compact_static(int64_t n_cells, double T_react, const double* T,
                                              int32_t* idx, int64_t* count, void* stream) {
  if (n_cells < 0 || !count || (n_cells > 0 && (!T || !idx))) {
    dfgb::set_global_error("df_active_compact_static: bad arguments");
    return DF_ERR_INVALID_ARG;
  }
  if (n_cells > kStaticMaxCells) {
    dfgb::set_global_error("df_active_compact_static: n_cells exceeds DF_COMPACT_STATIC_MAX_CELLS");
    return DF_ERR_INVALID_ARG;
  }
  int64_t* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e == cudaSuccess)
    e = dfgb::launch_compact(n_cells, T_react, T, idx, count, nullptr, scratch,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) {
    dfgb::set_global_error(cudaGetErrorString(e));
    return DF_ERR_CUDA;
  }
  return DF_OK;
}
