// Kernels of the real-fluid property network (PRNet-style surrogate, Sec. 2): the network reads
// a cell's conserved enthalpy, pressure and composition and yields its properties (here the
// density and the temperature). Input rows, normalised training targets and de-normalised
// outputs; the network layers themselves are the tcgen05 / SIMT GEMMs of the reaction step.
//
// Normalisation (the layout of the state's norm array, K0 = n + 2 inputs, m outputs):
//   norm[c] = input mean, norm[K0 + c] = 1 / input spread        (c < K0)
//   norm[2 K0 + k] = output mean, norm[2 K0 + m + k] = output spread (k < m)
// Inputs are (h, p, BC(Y_1), ..., BC(Y_n)) Z-scored (Sec. 3.3.1), BC(y) = (y^lambda - 1) /
// lambda with negative y read as 0 (Box & Cox 1964), the same composition coordinates as the
// chemistry network; outputs are O * spread + mean.
#include "dfgb_internal.cuh"
#include "ddfloat.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace dfgb {
namespace {

constexpr int kPropThreads = 256;

// Box-Cox coordinate of a mass fraction in FP32: its input feeds a BF16 or FP32 GEMM, whose
// rounding (2^-8 or 2^-24 relative) exceeds that of exp2f / log2f and of the truncating FP64 ->
// FP32 conversion. The sign test and the conversion use integer operations (the FP64 pipe of this
// GPU runs at 1/64 of the FP32 rate).
__device__ __forceinline__ float boxcox_f32(double y, float lambda) {
  const float v = d_pos(y) ? d_to_f_trunc(y) : 0.0f;
  const float t = v > 0.0f ? exp2f(lambda * log2f(v)) : 0.0f;
  return (t - 1.0f) / lambda;
}

// One input row per thread, written in 16-byte groups (8 BF16 or 4 FP32 values) over the padded
// row width ldx (a multiple of 16 BF16 / 8 FP32 elements, so every group is aligned); the
// padding columns are written as zero.
__global__ void prop_inputs_kernel(const double* __restrict__ norm, int n, float lambda,
                                   int64_t rows, const double* __restrict__ h,
                                   const double* __restrict__ p, const double* __restrict__ Y,
                                   int64_t ldY, void* __restrict__ x, int64_t ldx, int xkind) {
  const int K0 = n + 2;
  __shared__ float mean_f[kMaxSpecies + 2], inv_f[kMaxSpecies + 2];   // FP32 normalisation
  for (int c = threadIdx.x; c < K0; c += blockDim.x) {
    mean_f[c] = (float)norm[c];
    inv_f[c] = (float)norm[K0 + c];
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    auto value = [&](int c) -> float {
      if (c == 0) return d_to_f_trunc((h[r] - norm[0]) * norm[K0]);
      if (c == 1) return d_to_f_trunc((p[r] - norm[1]) * norm[K0 + 1]);
      if (c >= K0) return 0.0f;
      const float bc = boxcox_f32(Y[(int64_t)(c - 2) * ldY + r], lambda);
      return (bc - mean_f[c]) * inv_f[c];
    };
    if (xkind == kXBF16) {
      uint4* row = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(x) + r * ldx);
      for (int g = 0; g < (int)(ldx / 8); ++g) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const __nv_bfloat162 v = __floats2bfloat162_rn(value(8 * g + 2 * q), value(8 * g + 2 * q + 1));
          w[q] = *reinterpret_cast<const uint32_t*>(&v);
        }
        row[g] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    } else {
      float4* row = reinterpret_cast<float4*>(static_cast<float*>(x) + r * ldx);
      for (int g = 0; g < (int)(ldx / 4); ++g)
        row[g] = make_float4(value(4 * g), value(4 * g + 1), value(4 * g + 2), value(4 * g + 3));
    }
  }
}

// Normalised targets of the training loss: Oh[r][k] = (target_k[r] - mean_k) / spread_k.
__global__ void prop_targets_kernel(const double* __restrict__ norm, int K0, int m, int64_t rows,
                                    const double* __restrict__ t, int64_t ldt,
                                    float* __restrict__ Oh, int64_t ldo) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride)
    for (int k = 0; k < m; ++k)
      Oh[r * ldo + k] = (float)((t[(int64_t)k * ldt + r] - norm[2 * K0 + k]) / norm[2 * K0 + m + k]);
}

// Properties from the network outputs: out_k[r] = mean_k + spread_k O[r][k] (FP64).
__global__ void prop_outputs_kernel(const double* __restrict__ norm, int K0, int m, int64_t rows,
                                    const float* __restrict__ O, int64_t ldo,
                                    double* __restrict__ out, int64_t ldout) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride)
    for (int k = 0; k < m; ++k)
      out[(int64_t)k * ldout + r] = norm[2 * K0 + k] + norm[2 * K0 + m + k] * (double)O[r * ldo + k];
}

unsigned grid_of(int64_t rows, int num_sms) {
  const int64_t g = (rows + kPropThreads - 1) / kPropThreads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms * 8));
}

}  // namespace

cudaError_t launch_prop_inputs(const double* norm, int n, double lambda, int64_t rows,
                               const double* h, const double* p, const double* Y, int64_t ldY,
                               void* x, int64_t ldx, int xkind, int num_sms, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  prop_inputs_kernel<<<grid_of(rows, num_sms), kPropThreads, 0, st>>>(norm, n, (float)lambda, rows, h,
                                                                      p, Y, ldY, x, ldx, xkind);
  return cudaGetLastError();
}

cudaError_t launch_prop_targets(const double* norm, int K0, int m, int64_t rows, const double* t,
                                int64_t ldt, float* Oh, int64_t ldo, int num_sms, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  prop_targets_kernel<<<grid_of(rows, num_sms), kPropThreads, 0, st>>>(norm, K0, m, rows, t, ldt, Oh,
                                                                       ldo);
  return cudaGetLastError();
}

cudaError_t launch_prop_outputs(const double* norm, int K0, int m, int64_t rows, const float* O,
                                int64_t ldo, double* out, int64_t ldout, int num_sms,
                                cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  prop_outputs_kernel<<<grid_of(rows, num_sms), kPropThreads, 0, st>>>(norm, K0, m, rows, O, ldo,
                                                                       out, ldout);
  return cudaGetLastError();
}

}  // namespace dfgb
