// a6-a7 in plain FP32 on the CUDA cores (no tensor cores): the "plain FP32 step" the
// tensor-core paths are measured against. Register-tiled SGEMM, 128x128 block tile, BK = 8,
// 256 threads each owning an 8x8 sub-tile, double-buffered shared memory, persistent over
// the tiles of the (device-counted) valid rows, with bias + tanh-GELU (Sec. 3.3.2) fused
// into the epilogue. GELU uses the accurate tanhf here, since this path's error budget is
// the FP32 one.
#include "dfgb_internal.cuh"

namespace dfgb {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, kThreads = 256;

__device__ __forceinline__ float gelu_accurate(float x) {
  const float u = 0.7978845608028654f * fmaf(0.044715f * x * x, x, x);
  return 0.5f * x * (1.0f + tanhf(u));
}

__device__ __forceinline__ float gelu_grad_accurate(float x) {
  const float c = 0.7978845608028654f;
  const float t = tanhf(c * fmaf(0.044715f * x * x, x, x));
  return fmaf(0.5f * x * (1.0f - t * t), c * fmaf(3.0f * 0.044715f, x * x, 1.0f), 0.5f * (1.0f + t));
}

// MODE 0: C = act(A W^T + b); 1: also G = GELU'(A W^T + b); 2: C = (A W^T) * G[row / ntan, col]
template <bool GELU, int MODE>
__global__ void __launch_bounds__(kThreads, 2) sgemm_kernel(RowMap rows, int N, int K,
    const float* __restrict__ A, int64_t lda, const float* __restrict__ W, int64_t ldw,
    const float* __restrict__ bias, float* __restrict__ C, int64_t ldc, float* __restrict__ G,
    int64_t ldg, int ntan, const float4* __restrict__ gtab) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Ws[2][BK][BN];
  const int64_t M = valid_rows(rows);
  const int64_t tiles_m = (M + BM - 1) / BM;
  const int tiles_n = (N + BN - 1) / BN;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int lrow = tid / 2, lk = (tid % 2) * 4;   // loader: one float4 of A and of W
  for (int64_t tile = blockIdx.x; tile < tiles_m * tiles_n; tile += gridDim.x) {
    const int64_t m0 = (tile / tiles_n) * BM;
    const int n0 = (int)(tile % tiles_n) * BN;
    const bool arow_ok = m0 + lrow < M;
    const bool wrow_ok = n0 + lrow < N;
    const float* Ap = A + (m0 + lrow) * lda + lk;
    const float* Wp = W + (int64_t)(n0 + lrow) * ldw + lk;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    float4 a4 = arow_ok ? *reinterpret_cast<const float4*>(Ap) : make_float4(0, 0, 0, 0);
    float4 w4 = wrow_ok ? *reinterpret_cast<const float4*>(Wp) : make_float4(0, 0, 0, 0);
    int buf = 0;
    As[0][lk + 0][lrow] = a4.x; As[0][lk + 1][lrow] = a4.y;
    As[0][lk + 2][lrow] = a4.z; As[0][lk + 3][lrow] = a4.w;
    Ws[0][lk + 0][lrow] = w4.x; Ws[0][lk + 1][lrow] = w4.y;
    Ws[0][lk + 2][lrow] = w4.z; Ws[0][lk + 3][lrow] = w4.w;
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += BK) {
      const bool more = k0 + BK < K;
      if (more) {
        a4 = arow_ok ? *reinterpret_cast<const float4*>(Ap + k0 + BK) : make_float4(0, 0, 0, 0);
        w4 = wrow_ok ? *reinterpret_cast<const float4*>(Wp + k0 + BK) : make_float4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Ws[buf][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Ws[buf][k][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (more) {
        const int nb = buf ^ 1;
        As[nb][lk + 0][lrow] = a4.x; As[nb][lk + 1][lrow] = a4.y;
        As[nb][lk + 2][lrow] = a4.z; As[nb][lk + 3][lrow] = a4.w;
        Ws[nb][lk + 0][lrow] = w4.x; Ws[nb][lk + 1][lrow] = w4.y;
        Ws[nb][lk + 2][lrow] = w4.z; Ws[nb][lk + 3][lrow] = w4.w;
        __syncthreads();
        buf = nb;
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (r >= M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (col < N) {
          if (MODE == 2) {
            C[r * ldc + col] = acc[i][j] * G[(r / ntan) * ldg + col];
          } else {
            const float z = acc[i][j] + bias[col];
            C[r * ldc + col] = GELU ? (gtab ? gelu_from_table(z, gtab) : gelu_accurate(z)) : z;
            if (MODE == 1) G[r * ldg + col] = gelu_grad_accurate(z);
          }
        }
      }
    }
    __syncthreads();  // the next tile overwrites buffer 0
  }
}

}  // namespace

cudaError_t launch_sgemm_bias_act(const RowMap& rows, int N, int K, const float* A, int64_t lda,
                                  const float* W, int64_t ldw, const float* bias, float* C,
                                  int64_t ldc, bool gelu, int num_sms, cudaStream_t st,
                                  int mode, float* G, int64_t ldg, int ntan,
                                  const float4* gtab) {
  if (rows.nmax <= 0) return cudaSuccess;
  if (K % BK != 0 || lda % 4 != 0 || ldw % 4 != 0) return cudaErrorInvalidValue;
  const int64_t tiles = ((rows.nmax + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int64_t cap = (int64_t)num_sms * 2;
  const unsigned g = (unsigned)(tiles < cap ? tiles : cap);
  if (ntan < 1) ntan = 1;
  if (mode == 2)
    sgemm_kernel<false, 2><<<g, kThreads, 0, st>>>(rows, N, K, A, lda, W, ldw, bias, C, ldc, G, ldg, ntan, gtab);
  else if (mode == 1)
    sgemm_kernel<true, 1><<<g, kThreads, 0, st>>>(rows, N, K, A, lda, W, ldw, bias, C, ldc, G, ldg, ntan, gtab);
  else if (gelu)
    sgemm_kernel<true, 0><<<g, kThreads, 0, st>>>(rows, N, K, A, lda, W, ldw, bias, C, ldc, G, ldg, ntan, gtab);
  else
    sgemm_kernel<false, 0><<<g, kThreads, 0, st>>>(rows, N, K, A, lda, W, ldw, bias, C, ldc, G, ldg, ntan, gtab);
  return cudaGetLastError();
}

}  // namespace dfgb
