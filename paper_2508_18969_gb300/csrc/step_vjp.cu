// Reverse-mode product of the reaction step (the adjoint of the step's Jacobian): per cell,
//   g_v = gT' dT'/dv + sum_k gY'_k dY'_k/dv,   v = (T, Y_1..Y_n),
// from the columns df_chem_jacobian assembles, J[k][t] = d(Y'_k - Y_k)/dv_t (so dY'_k/dv_t =
// J[k][t] + [t = k + 1]) and dTn[t] = dT'/dv_t. A warp per cell and a lane per direction t; the
// sum over k runs in ascending order in FP64, and for each k the lanes read one contiguous row
// of J. Cells that do not react (T <= T_react, or a non-finite T) are left as they were by the
// step, so their cotangents are copied through; reacting cells the step flags have NaN columns
// and get NaN.

#include "dfgb_internal.cuh"

namespace dfgb {
namespace {

__global__ void __launch_bounds__(256) step_vjp_kernel(int n, int64_t ncell, double T_react,
    const double* __restrict__ T, const float* __restrict__ J, const double* __restrict__ dTn,
    const double* __restrict__ gT, const double* __restrict__ gY, int64_t ldg,
    double* __restrict__ oT, double* __restrict__ oY, int64_t ldo) {
  const int ntan = n + 1;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < ncell;
       r += warps) {
    const double gt = gT[r];
    if (!(T[r] > T_react)) {
      if (lane == 0) oT[r] = gt;
      for (int k = lane; k < n; k += 32) oY[(int64_t)k * ldo + r] = gY[(int64_t)k * ldg + r];
      continue;
    }
    const float* Jc = J + r * (int64_t)n * ntan;
    const double* dTc = dTn + r * (int64_t)ntan;
    for (int t = lane; t < ntan; t += 32) {
      double acc = gt * dTc[t];
      if (t > 0) acc += gY[(int64_t)(t - 1) * ldg + r];
      for (int k = 0; k < n; ++k) acc = fma(gY[(int64_t)k * ldg + r], (double)Jc[k * ntan + t], acc);
      if (t == 0)
        oT[r] = acc;
      else
        oY[(int64_t)(t - 1) * ldo + r] = acc;
    }
  }
}

}  // namespace

cudaError_t launch_step_vjp(int n, int64_t ncell, double T_react, const double* T, const float* J,
                            const double* dTn, const double* gT, const double* gY, int64_t ldg,
                            double* oT, double* oY, int64_t ldo, cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  const int64_t blocks = (ncell + 7) / 8;  // eight cells (warps) per block
  const unsigned g = (unsigned)(blocks < (1 << 20) ? blocks : (1 << 20));
  step_vjp_kernel<<<g, 256, 0, st>>>(n, ncell, T_react, T, J, dTn, gT, gY, ldg, oT, oY, ldo);
  return cudaGetLastError();
}

}  // namespace dfgb
