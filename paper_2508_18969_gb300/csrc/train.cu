// Training of the chemistry network: targets, loss, the element-wise parts of the backward
// pass and the Adam update. The GEMMs of the backward pass (weight gradients dZ^T H and input
// gradients dZ W, the latter scaled by GELU'(z) in its epilogue) run on the same tcgen05 /
// SIMT kernels as the forward pass; these kernels prepare their operands.
#include "dfgb_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace dfgb {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = kTrainScratchFloats;   // element-wise grids, one loss partial each

// BC(yt) - BC(y) for the Box-Cox transform BC(x) = (x^l - 1) / l. When both are positive
// it is formed as y^l expm1(l ln(yt / y)) / l: the difference yt - y in FP64 (no cancellation
// of two nearly equal values), its ratio to y as a correctly rounded FP32 division, the rest in
// FP32. That keeps the difference itself to ~2e-7 relative; GB300's FP64 division would cost
// more than the rest of the kernel.
__device__ __forceinline__ float dboxcox(double y, double yt, float lam) {
  if (y > 0.0 && yt > 0.0) {
    const float yf = (float)y;
    const float q = __fdiv_rn((float)(yt - y), yf);
    const float lr = (q > -0.5f && q < 1.0f) ? log1pf(q) : logf(__fdiv_rn((float)yt, yf));
    return powf(yf, lam) * expm1f(lam * lr) / lam;
  }
  const float a = yt > 0.0 ? powf((float)yt, lam) : 0.0f;
  const float b = y > 0.0 ? powf((float)y, lam) : 0.0f;
  return (a - b) / lam;
}

// Ohat[b][k] = (BC(Yt) - BC(Y) - out_mean_k) / out_std_k, FP32 [B x ldh], zero pad. A thread
// per state: the FP64 reads of Y and Yt are coalesced across the batch, and each thread writes
// its row in 16-byte groups (ldh a multiple of 4).
__global__ void targets_kernel(EosParams P, int64_t B, const double* __restrict__ Y,
                               const double* __restrict__ Yt, int64_t ldY,
                               const double* __restrict__ norm, float* __restrict__ Oh,
                               int64_t ldh) {
  const int n = P.n, K0 = P.K0;
  const float lam = (float)P.lambda;
  __shared__ float mean_f[64], std_f[64];
  for (int k = threadIdx.x; k < n && k < 64; k += blockDim.x) {
    mean_f[k] = (float)norm[2 * K0 + k];
    std_f[k] = (float)norm[2 * K0 + n + k];
  }
  __syncthreads();
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    float* orow = Oh + b * ldh;
    for (int k0 = 0; k0 < ldh; k0 += 4) {
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + j;
        v[j] = 0.0f;
        if (k < n) {
          const float du = dboxcox(Y[k * ldY + b], Yt[k * ldY + b], lam);
          v[j] = (du - mean_f[k]) / std_f[k];
        }
      }
      *reinterpret_cast<float4*>(orow + k0) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// dO = 2 (O - Ohat) / B (columns >= n zero); part[block] = this block's share of
// sum (O - Ohat)^2 / B (summed in a fixed order by sum_parts_warp_kernel, so the loss is
// reproducible run to run).
template <typename GT>
__global__ void loss_grad_kernel(int64_t B, int n, const float* __restrict__ O, int64_t ldo,
                                 const float* __restrict__ Oh, int64_t ldh, GT* __restrict__ dO,
                                 int64_t ldd, float invB, float* __restrict__ part) {
  __shared__ float red[kThreads / 32];
  float acc = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < B * ldd;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ldd;
    const int k = (int)(e % ldd);
    float g = 0.0f;
    if (k < n) {
      const float r = O[b * ldo + k] - Oh[b * ldh + k];
      acc = fmaf(r * r, invB, acc);
      g = 2.0f * r * invB;
    }
    dO[e] = (GT)g;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// Two adjacent elements of a row: the unit of every global access of transpose_kernel.
template <typename T> struct Pair;
template <> struct Pair<__nv_bfloat16> {
  using V = __nv_bfloat162;
  static __device__ __forceinline__ float lo(V v) { return __low2float(v); }
  static __device__ __forceinline__ float hi(V v) { return __high2float(v); }
  static __device__ __forceinline__ V make(__nv_bfloat16 a, __nv_bfloat16 b) { return __halves2bfloat162(a, b); }
  static __device__ __forceinline__ V zero() { return __float2bfloat162_rn(0.0f); }
  static __device__ __forceinline__ __nv_bfloat16 first(V v) { return __low2bfloat16(v); }
  static __device__ __forceinline__ __nv_bfloat16 second(V v) { return __high2bfloat16(v); }
};
template <> struct Pair<float> {
  using V = float2;
  static __device__ __forceinline__ float lo(V v) { return v.x; }
  static __device__ __forceinline__ float hi(V v) { return v.y; }
  static __device__ __forceinline__ V make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V zero() { return make_float2(0.0f, 0.0f); }
  static __device__ __forceinline__ float first(V v) { return v.x; }
  static __device__ __forceinline__ float second(V v) { return v.y; }
};

constexpr int kTp = 64;   // transpose tile: 64 rows x 64 columns, 256 threads

// out[c][r] = in[r][c] for c < C, r < Rpad (zero for R <= r < Rpad). Block (x, y) takes the
// 64-column strip x and the row tiles y, y + gridDim.y, ...; every global access moves two
// adjacent elements of a row, 128 (BF16) or 256 (FP32) contiguous bytes per warp. The loads of
// the next tile are issued before the stores of the current one, so that each SM keeps enough
// bytes in flight to cover the DRAM latency of this scattered pattern. With part, the block also
// stores the FP32 column sums of its rows, part[y * C + c], summed in a fixed order (the bias
// gradient of the dZ transpose).
template <typename T>
__global__ void __launch_bounds__(256, 6) transpose_kernel(int64_t R, int64_t C,
                                                           const T* __restrict__ in, int64_t ldi,
                                                           T* __restrict__ out, int64_t ldo,
                                                           int64_t Rpad, float* __restrict__ part) {
  using P = Pair<T>;
  using V = typename P::V;
  __shared__ T tile[kTp][kTp + 2];
  __shared__ float red[8][kTp];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kTp;
  const int64_t c = c0 + 2 * lane;   // this thread's two columns c, c + 1 (load phase)
  const bool col_ok = c < C, pad_hi = c + 1 >= C;
  const int64_t ntiles = Rpad / kTp;
  // c < C: both elements lie inside the row's pitch (ldi and c even); a pad is zeroed at use
  const T* src = in + c;
  V v[kTp / 8];
  auto load = [&](int64_t tt) {
#pragma unroll
    for (int j = 0; j < kTp / 8; ++j) {
      const int64_t r = tt * kTp + w + 8 * j;
      v[j] = (r < R && col_ok) ? *reinterpret_cast<const V*>(src + r * ldi) : P::zero();
    }
  };
  float s0 = 0.0f, s1 = 0.0f;
  int64_t t = blockIdx.y;
  if (t < ntiles) load(t);
  for (; t < ntiles; t += gridDim.y) {
#pragma unroll
    for (int j = 0; j < kTp / 8; ++j) {
      V x = v[j];
      if (pad_hi) x = P::make(P::first(x), P::first(P::zero()));
      s0 += P::lo(x);
      s1 += P::hi(x);
      tile[w + 8 * j][2 * lane] = P::first(x);
      tile[w + 8 * j][2 * lane + 1] = P::second(x);
    }
    __syncthreads();
    const int64_t r0 = t * kTp;
    if (t + gridDim.y < ntiles) load(t + gridDim.y);
#pragma unroll
    for (int j = 0; j < kTp / 8; ++j) {
      const int cl = w + 8 * j;
      if (c0 + cl < C)
        *reinterpret_cast<V*>(out + (c0 + cl) * ldo + r0 + 2 * lane) =
            P::make(tile[2 * lane][cl], tile[2 * lane + 1][cl]);
    }
    __syncthreads();
  }
  if (!part) return;
  red[w][2 * lane] = s0;
  red[w][2 * lane + 1] = s1;
  __syncthreads();
  if (threadIdx.x < kTp && c0 + threadIdx.x < C) {
    float s = 0.0f;
    for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
    part[(int64_t)blockIdx.y * C + c0 + threadIdx.x] = s;
  }
}

// out[i] = sum_{s < splits} part[s * stride + i], in order of s.
__global__ void split_sum_kernel(int splits, int64_t count, int64_t stride,
                                 const float* __restrict__ part, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[k * stride + i];
    out[i] = s;
  }
}

// out[c] = sum_{j < parts} part[j * C + c] with one warp per c: lane l sums parts l, l + 32, ...
// in order, then the lanes combine in a fixed butterfly, so the result is the same every run.
__global__ void sum_parts_warp_kernel(int parts, int C, const float* __restrict__ part,
                                      float* __restrict__ out) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  float s = 0.0f;
  for (int j = lane; j < parts; j += 32) s += part[(int64_t)j * C + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}

// Adam (Kingma & Ba 2015) on one parameter array: m, v moving averages of g and g^2, bias
// corrections c1 = 1 - b1^t, c2 = 1 - b2^t, w -= lr (m / c1) / (sqrt(v / c2) + eps).
__global__ void adam_kernel(int64_t count, float* __restrict__ w, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Working copies of a master weight matrix Wm [N x ldm]: FP32 [N x ld32] (SIMT), BF16
// [N x ldb] (tensor cores), and the transposed copy [K x ldt] (FP32 or BF16) for the input
// gradient GEMM. Any destination may be NULL. Pads stay as allocated (zero).
__global__ void publish_kernel(int N, int K, const float* __restrict__ Wm, int64_t ldm, float* W32,
                               int64_t ld32, __nv_bfloat16* Wb, int64_t ldb, void* WT, int64_t ldt,
                               int WT_bf16) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / K), c = (int)(e % K);
    const float w = Wm[(int64_t)r * ldm + c];
    if (W32) W32[(int64_t)r * ld32 + c] = w;
    if (Wb) Wb[(int64_t)r * ldb + c] = __float2bfloat16_rn(w);
    if (WT) {
      if (WT_bf16) ((__nv_bfloat16*)WT)[(int64_t)c * ldt + r] = __float2bfloat16_rn(w);
      else ((float*)WT)[(int64_t)c * ldt + r] = w;
    }
  }
}

int blocks_for(int64_t work) {
  int64_t b = (work + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  return (int)(b < kMaxBlocks ? b : kMaxBlocks);
}

}  // namespace

cudaError_t launch_train_targets(const EosParams& P, int64_t B, const double* Y, const double* Yt,
                                 int64_t ldY, float* Oh, int64_t ldh, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  if ((ldh & 3) || P.n > 64) return cudaErrorInvalidValue;
  targets_kernel<<<blocks_for(B), kThreads, 0, st>>>(P, B, Y, Yt, ldY, P.norm, Oh, ldh);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(int64_t B, int n, const float* O, int64_t ldo, const float* Oh,
                             int64_t ldh, void* dO, int64_t ldd, bool bf16, float* loss,
                             float* scratch, cudaStream_t st) {
  if (B <= 0) return cudaMemsetAsync(loss, 0, sizeof(float), st);
  const float invB = 1.0f / (float)B;
  const int g = blocks_for(B * ldd);
  if (bf16)
    loss_grad_kernel<__nv_bfloat16><<<g, kThreads, 0, st>>>(B, n, O, ldo, Oh, ldh,
                                                            (__nv_bfloat16*)dO, ldd, invB, scratch);
  else
    loss_grad_kernel<float><<<g, kThreads, 0, st>>>(B, n, O, ldo, Oh, ldh, (float*)dO, ldd, invB,
                                                    scratch);
  sum_parts_warp_kernel<<<1, 32, 0, st>>>(g, 1, scratch, loss);
  return cudaGetLastError();
}

cudaError_t launch_transpose(int64_t R, int64_t C, const void* in, int64_t ldi, void* out,
                             int64_t ldo, int64_t Rpad, bool bf16, int num_sms, cudaStream_t st,
                             float* colsum, float* scratch, int64_t scratch_floats) {
  if (C <= 0) return cudaSuccess;
  if (Rpad <= 0 || (Rpad % kTp) || (ldi & 1) || (ldo & 1)) {
    if (colsum && Rpad <= 0) return cudaMemsetAsync(colsum, 0, sizeof(float) * C, st);
    return Rpad <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  }
  const int64_t strips = (C + kTp - 1) / kTp, ntiles = Rpad / kTp;
  // about six blocks per SM (its resident count); with the sums, as many row groups as the
  // scratch holds
  int64_t groups = std::max<int64_t>(1, (6LL * std::max(num_sms, 1) + strips - 1) / strips);
  groups = std::min(groups, ntiles);
  if (colsum) {
    if (!scratch || scratch_floats < C) return cudaErrorInvalidValue;
    groups = std::min<int64_t>(groups, scratch_floats / C);
  }
  const dim3 grid((unsigned)strips, (unsigned)groups);
  float* part = colsum ? scratch : nullptr;
  if (bf16)
    transpose_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(
        R, C, (const __nv_bfloat16*)in, ldi, (__nv_bfloat16*)out, ldo, Rpad, part);
  else
    transpose_kernel<float><<<grid, 256, 0, st>>>(R, C, (const float*)in, ldi, (float*)out, ldo,
                                                  Rpad, part);
  if (colsum)
    sum_parts_warp_kernel<<<(unsigned)((C + 7) / 8), 256, 0, st>>>((int)groups, (int)C, scratch, colsum);
  return cudaGetLastError();
}

cudaError_t launch_sum_splits(int splits, int64_t count, int64_t stride, const float* part,
                              float* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  split_sum_kernel<<<blocks_for(count), kThreads, 0, st>>>(splits, count, stride, part, out);
  return cudaGetLastError();
}

cudaError_t launch_adam(int64_t count, float* w, float* m, float* v, const float* g, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  adam_kernel<<<blocks_for(count), kThreads, 0, st>>>(count, w, m, v, g, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_publish(int N, int K, const float* Wm, int64_t ldm, float* W32, int64_t ld32,
                           void* Wb, int64_t ldb, void* WT, int64_t ldt, bool WT_bf16,
                           cudaStream_t st) {
  publish_kernel<<<blocks_for((int64_t)N * K), kThreads, 0, st>>>(
      N, K, Wm, ldm, W32, ld32, (__nv_bfloat16*)Wb, ldb, WT, ldt, WT_bf16 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace dfgb
