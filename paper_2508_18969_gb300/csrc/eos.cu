// Equation-of-state kernels of the reaction step: a1-a5 (eos_pre), a8-a10 (eos_post) and
// the real-fluid property evaluation. One thread per cell; species-major (SoA) field reads
// are coalesced across the threads of a warp. FP64 throughout except the Box-Cox features
// that feed the network (quantised to the network's precision anyway) and the FP32
// closed-form seed of the cubic roots, which FP64 Newton steps then polish.
//
// Peng-Robinson (Sec. 2 names the EoS; equations from Peng & Robinson 1976):
//   sqrt(a_k(T)) = sqrt(a_c,k) [1 + kappa_k (1 - sqrt(T / Tc_k))] = s_k - r_k sqrt(T),
//   a_m = sum_ij X_i X_j sqrt(a_i a_j) (1 - k_ij) = A0 - 2 A1 sqrt(T) + A2 T
// where A0, A1, A2 are three quadratic forms of the composition. They are computed once
// per composition, so every Newton iteration of the T-from-h solve is O(1) in the species
// count.
#include "dfgb_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace dfgb {
namespace {

constexpr double kSQ2 = 1.41421356237309504880;
constexpr int kThreads = 128;
constexpr int kCellNotConverged = 1;
constexpr int kCellNoRoot = 2;
constexpr int kCellNonfinite = 4;
constexpr double kTLo = 50.0, kTHi = 5000.0;

struct Mixture {
  double inv;        // sum_k Y_k / W_k = 1 / W_mix
  double e[6];       // ideal-gas mass-specific enthalpy: h_ig(T) = sum_j e_j T^j, J/kg
  double A0, A1, A2; // a_m(T) = A0 - 2 A1 sqrt(T) + A2 T
  double bm;
};

struct SharedConsts {
  const double* spc;   // [n * kSpcStride]
  const double* K;     // [n * n]
  const double* norm;  // [2 K0 + 2 n]
};

__device__ SharedConsts load_consts(const EosParams& P, double* sm) {
  const int nspc = P.n * kSpcStride, nk = P.n * P.n, nn = 2 * P.K0 + 2 * P.n;
  for (int i = threadIdx.x; i < nspc; i += blockDim.x) sm[i] = P.spc[i];
  for (int i = threadIdx.x; i < nk; i += blockDim.x) sm[nspc + i] = P.Kmat[i];
  for (int i = threadIdx.x; i < nn; i += blockDim.x) sm[nspc + nk + i] = P.norm[i];
  __syncthreads();
  return SharedConsts{sm, sm + nspc, sm + nspc + nk};
}

// Mixture coefficients of one composition (a1, a2 and the ideal-gas part of a4).
template <int NM>
__device__ void mixture(const double (&Y)[NM], int n, const SharedConsts& c, Mixture& m) {
  double ys[NM], yr[NM];
  double inv = 0.0, bsum = 0.0;
  double e0 = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0, e4 = 0.0, e5 = 0.0;
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    ys[k] = 0.0;
    yr[k] = 0.0;
    if (k < n) {
      const double* q = c.spc + k * kSpcStride;
      const double y = Y[k] * q[0];
      inv += y;
      ys[k] = y * q[1];
      yr[k] = y * q[2];
      bsum = fma(y, q[3], bsum);
      e0 = fma(y, q[4], e0);
      e1 = fma(y, q[5], e1);
      e2 = fma(y, q[6], e2);
      e3 = fma(y, q[7], e3);
      e4 = fma(y, q[8], e4);
      e5 = fma(y, q[9], e5);
    }
  }
  // Symmetric quadratic forms with K_ii = 1:
  //   F0 = sum_ij K_ij ys_i ys_j, F1 = sum_ij K_ij ys_i yr_j, F2 = sum_ij K_ij yr_i yr_j.
  double F0 = 0.0, F1 = 0.0, F2 = 0.0;
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    if (i < n) {
      double Pi = 0.0, Qi = 0.0;
      const double* Krow = c.K + i * n;
#pragma unroll
      for (int j = i + 1; j < NM; ++j) {
        if (j < n) {
          const double K = Krow[j];
          Pi = fma(K, ys[j], Pi);
          Qi = fma(K, yr[j], Qi);
        }
      }
      F0 = fma(ys[i], fma(2.0, Pi, ys[i]), F0);
      F1 = fma(ys[i], yr[i] + Qi, fma(yr[i], Pi, F1));
      F2 = fma(yr[i], fma(2.0, Qi, yr[i]), F2);
    }
  }
  const double Wm = 1.0 / inv;
  const double W2 = Wm * Wm;
  m.inv = inv;
  m.e[0] = e0; m.e[1] = e1; m.e[2] = e2; m.e[3] = e3; m.e[4] = e4; m.e[5] = e5;
  m.A0 = W2 * F0;
  m.A1 = W2 * F1;
  m.A2 = W2 * F2;
  m.bm = Wm * bsum;
}

__device__ __forceinline__ double h_ig(const Mixture& m, double T) {
  return fma(fma(fma(fma(fma(m.e[5], T, m.e[4]), T, m.e[3]), T, m.e[2]), T, m.e[1]), T, m.e[0]);
}

__device__ __forceinline__ double cp_ig(const Mixture& m, double T) {
  return fma(fma(fma(fma(5.0 * m.e[5], T, 4.0 * m.e[4]), T, 3.0 * m.e[3]), T, 2.0 * m.e[2]), T,
             m.e[1]);
}

__device__ __forceinline__ double cubic_polish(double Z, double c2, double c1, double c0) {
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const double f = fma(fma(Z + c2, Z, c1), Z, c0);
    const double fp = fma(fma(3.0, Z, 2.0 * c2), Z, c1);
    if (fp != 0.0) Z -= f / fp;
  }
  return Z;
}

__device__ __forceinline__ double log_ratio(double Z, double B) {
  return log((Z + (1.0 + kSQ2) * B) / (Z + (1.0 - kSQ2) * B));
}

__device__ __forceinline__ double g_dep(double Z, double A, double B) {
  return Z - 1.0 - log(Z - B) - A / (2.0 * kSQ2 * B) * log_ratio(Z, B);
}

// Compressibility (a3): the real root of
//   Z^3 - (1 - B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0
// above B with least departure Gibbs energy (ties within 1e-12 keep the larger root).
// Seeds come from the FP32 closed form (Cardano for one real root, the trigonometric form
// for three), each then polished by three FP64 Newton steps on the cubic.
__device__ double select_Z(double A, double B, int& status) {
  const double c2 = B - 1.0;
  const double c1 = A - 3.0 * B * B - 2.0 * B;
  const double c0 = B * B + B * B * B - A * B;
  const double P = c1 - c2 * c2 * (1.0 / 3.0);
  const double Q = 2.0 * c2 * c2 * c2 * (1.0 / 27.0) - c2 * c1 * (1.0 / 3.0) + c0;
  const double disc = 0.25 * Q * Q + P * P * P * (1.0 / 27.0);
  if (disc > 0.0) {
    const float qf = (float)Q, pf = (float)P;
    const float sq = sqrtf((float)disc);
    const float u = cbrtf(-0.5f * qf - copysignf(sq, qf));
    const float t = (u != 0.0f) ? u - pf / (3.0f * u) : 0.0f;
    const double Z = cubic_polish((double)t - c2 * (1.0 / 3.0), c2, c1, c0);
    if (!(Z > B)) status |= kCellNoRoot;
    return Z;
  }
  const float pf = (float)P;
  const float m = (pf < 0.0f) ? 2.0f * sqrtf(-pf / 3.0f) : 0.0f;
  float cphi = (pf < 0.0f) ? (3.0f * (float)Q / (2.0f * pf)) * sqrtf(-3.0f / pf) : 0.0f;
  cphi = fminf(fmaxf(cphi, -1.0f), 1.0f);
  const float phi = acosf(cphi) * (1.0f / 3.0f);
  double best = __longlong_as_double(0x7ff8000000000000LL);
  double gbest = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // k = 0, 1, 2 give descending seeds
    const float tk = m * cosf(phi - 2.0943951023931955f * (float)k);
    const double Z = cubic_polish((double)tk - c2 * (1.0 / 3.0), c2, c1, c0);
    if (Z > B) {
      const double g = g_dep(Z, A, B);
      if (g < gbest - 1e-12) {
        gbest = g;
        best = Z;
      }
    }
  }
  if (!(best > B)) status |= kCellNoRoot;
  return best;
}

struct PRPoint {
  double Z, h_dep, cp_dep;  // molar departure enthalpy and its T-derivative at fixed p
};

// Real-fluid state at (T, p) of a composition (a2-a4), with the departure cp if asked.
__device__ PRPoint pr_point(const Mixture& m, double T, double p, bool want_cp, int& status) {
  const double t = sqrt(T);
  const double am = fma(-2.0 * m.A1, t, fma(m.A2, T, m.A0));
  const double dam = m.A2 - m.A1 / t;
  const double RT = kR * T;
  const double A = am * p / (RT * RT);
  const double B = m.bm * p / RT;
  PRPoint r;
  r.Z = select_Z(A, B, status);
  const double Zp = r.Z + (1.0 + kSQ2) * B;
  const double Zm = r.Z + (1.0 - kSQ2) * B;
  const double L = log(Zp / Zm);
  const double k = 1.0 / (2.0 * kSQ2 * m.bm);
  r.h_dep = RT * (r.Z - 1.0) + (T * dam - am) * k * L;
  r.cp_dep = 0.0;
  if (want_cp) {
    const double d2am = m.A1 / (2.0 * T * t);
    const double dB = -B / T;
    const double dA = A * (dam / am - 2.0 / T);
    const double Z = r.Z;
    const double FZ = fma(3.0 * Z, Z, -2.0 * (1.0 - B) * Z) + (A - 3.0 * B * B - 2.0 * B);
    const double FA = Z - B;
    const double FB = Z * Z - (6.0 * B + 2.0) * Z - (A - 2.0 * B - 3.0 * B * B);
    const double dZ = -(FA * dA + FB * dB) / FZ;
    const double dL = (dZ + (1.0 + kSQ2) * dB) / Zp - (dZ + (1.0 - kSQ2) * dB) / Zm;
    r.cp_dep = kR * (Z - 1.0) + RT * dZ + k * T * d2am * L + k * (T * dam - am) * dL;
  }
  return r;
}

template <typename XT>
__device__ __forceinline__ XT to_x(float v, float scale);
template <>
__device__ __forceinline__ float to_x<float>(float v, float) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_x<__nv_bfloat16>(float v, float) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __nv_fp8_e4m3 to_x<__nv_fp8_e4m3>(float v, float scale) {
  return __nv_fp8_e4m3(v * scale);
}

// a1-a5 for the valid rows of a batch.
template <int NM, typename XT>
__global__ void __launch_bounds__(kThreads) eos_pre_kernel(EosParams P, RowMap rows,
    const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,
    int64_t ldY, double* __restrict__ h0, double* __restrict__ Zout, XT* __restrict__ x,
    int64_t ldx, float x_scale, int32_t* __restrict__ status) {
  extern __shared__ double sm[];
  const SharedConsts c = load_consts(P, sm);
  const int64_t nrow = valid_rows(rows);
  const int n = P.n, K0 = P.K0;
  const double* in_mean = c.norm;
  const double* in_is = c.norm + K0;
  const float lam = (float)P.lambda;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = row_cell(rows, r);
    const double Tc = T[cell], pc = p[cell];
    double Yk[NM];
    bool finite = isfinite(Tc) && isfinite(pc) && pc > 0.0 && Tc > 0.0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      Yk[k] = (k < n) ? Y[k * ldY + cell] : 0.0;
      finite = finite && isfinite(Yk[k]);
    }
    int st = 0;
    double h = __longlong_as_double(0x7ff8000000000000LL), Z = h;
    if (finite) {
      Mixture m;
      mixture<NM>(Yk, n, c, m);
      const PRPoint q = pr_point(m, Tc, pc, false, st);
      Z = q.Z;
      h = h_ig(m, Tc) + q.h_dep * m.inv;
      if (!isfinite(h)) st |= kCellNonfinite;
    } else {
      st = kCellNonfinite;
    }
    if (h0) h0[r] = h;
    if (Zout) Zout[r] = Z;
    if (status) status[r] = st;
    if (x) {
      XT* xr = x + r * ldx;
      xr[0] = to_x<XT>(finite ? (float)((Tc - in_mean[0]) * in_is[0]) : 0.0f, x_scale);
      xr[1] = to_x<XT>(finite ? (float)((pc - in_mean[1]) * in_is[1]) : 0.0f, x_scale);
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        if (k < n) {
          const float y = fmaxf((float)Yk[k], 0.0f);
          const float bc = (y > 0.0f) ? (exp2f(lam * log2f(y)) - 1.0f) / lam : -1.0f / lam;
          const float v = (float)(((double)bc - in_mean[2 + k]) * in_is[2 + k]);
          xr[2 + k] = to_x<XT>(finite ? v : 0.0f, x_scale);
        }
      }
      for (int k = K0; k < ldx; ++k) xr[k] = to_x<XT>(0.0f, x_scale);
    }
  }
}

__device__ __forceinline__ double ipow(double b, int m) {
  double r = 1.0;
  while (m) {
    if (m & 1) r *= b;
    b *= b;
    m >>= 1;
  }
  return r;
}

// a8-a10 for the valid rows of a batch.
template <int NM>
__global__ void __launch_bounds__(kThreads) eos_post_kernel(EosParams P, RowMap rows,
    const float* __restrict__ O, int64_t ldo, const double* __restrict__ h0,
    double* __restrict__ T, const double* __restrict__ p, double* __restrict__ Y, int64_t ldY,
    const int32_t* __restrict__ pre_status, int32_t* __restrict__ cell_status) {
  extern __shared__ double sm[];
  const SharedConsts c = load_consts(P, sm);
  const int64_t nrow = valid_rows(rows);
  const int n = P.n, K0 = P.K0;
  const double* out_mean = c.norm + 2 * K0;
  const double* out_std = c.norm + 2 * K0 + n;
  const double lam = P.lambda;
  const int mpow = P.inv_lambda;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = row_cell(rows, r);
    const double Told = T[cell], pc = p[cell], h0c = h0[r];
    int st = pre_status ? pre_status[r] : 0;  // flags eos_pre raised for this row
    double Yn[NM];
    bool finite = isfinite(Told) && isfinite(pc) && pc > 0.0 && isfinite(h0c);
    double S = 0.0;
    const float* Or = O + r * ldo;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      Yn[k] = 0.0;
      if (k < n) {
        const double y = Y[k * ldY + cell];
        finite = finite && isfinite(y);
        const double ldu = lam * fma(out_std[k], (double)Or[k], out_mean[k]);  // lambda du
        double yn;
        if (y >= 1e-30) {
          // Y' = (Y^lambda + lambda du)^(1/lambda) = Y (1 + eps)^m, eps = lambda du Y^-lambda;
          // Y^-lambda only scales the small increment, so FP32 suffices for it.
          const double eps = ldu * (double)exp2f(-(float)lam * log2f((float)y));
          yn = (eps > -1.0) ? y * ipow(1.0 + eps, mpow) : 0.0;
        } else {
          const double base = ((y > 0.0) ? pow(y, lam) : 0.0) + ldu;
          yn = (base > 0.0) ? ipow(base, mpow) : 0.0;
        }
        Yn[k] = yn;
        S += yn;
      }
    }
    if (!finite || !(S > 0.0)) st |= kCellNonfinite;
    double Tn = Told;
    int iters = 0;
    if (st == 0) {
      const double iS = 1.0 / S;
#pragma unroll
      for (int k = 0; k < NM; ++k) Yn[k] *= iS;
      Mixture m;
      mixture<NM>(Yn, n, c, m);
      double lo = kTLo, hi = kTHi;
      Tn = fmin(fmax(Told, lo), hi);
      bool conv = false;
      for (int it = 0; it < P.newton_max_iter; ++it) {
        ++iters;
        int s2 = 0;
        const PRPoint q = pr_point(m, Tn, pc, true, s2);
        if (s2) {
          st |= s2;
          break;
        }
        const double f = h_ig(m, Tn) + q.h_dep * m.inv - h0c;
        const double cp = cp_ig(m, Tn) + q.cp_dep * m.inv;
        if (f > 0.0) hi = fmin(hi, Tn); else lo = fmax(lo, Tn);
        double Tx = Tn - f / cp;
        // a step within tolerance has converged; only a longer step that leaves the
        // bracket (or is not finite) is replaced by bisection
        const bool done = fabs(Tx - Tn) <= P.newton_tol * Tn;
        if (!done && !(Tx > lo && Tx < hi)) Tx = 0.5 * (lo + hi);
        Tn = Tx;
        if (done) {
          conv = true;
          break;
        }
      }
      if (!conv && st == 0) st |= kCellNotConverged;
      if (!isfinite(Tn)) st |= kCellNonfinite;
    }
    if (st == 0) {
      T[cell] = Tn;
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) Y[k * ldY + cell] = Yn[k];
    }
    if (cell_status) cell_status[cell] = st;
    if (st && P.flagged) atomicAdd((unsigned long long*)P.flagged, 1ull);
    if (P.newton_iters) {  // one atomic per warp
      const unsigned mask = __activemask();
      const int tot = __reduce_add_sync(mask, iters);
      if ((threadIdx.x & 31) == __ffs(mask) - 1)
        atomicAdd((unsigned long long*)P.newton_iters, (unsigned long long)tot);
    }
  }
}

template <int NM>
__global__ void __launch_bounds__(kThreads) props_kernel(EosParams P, int64_t ncell,
    const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,
    int64_t ldY, double* rho, double* h, double* cp, double* Zo) {
  extern __shared__ double sm[];
  const SharedConsts c = load_consts(P, sm);
  const int n = P.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Tc = T[i], pc = p[i];
    double Yk[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) Yk[k] = (k < n) ? Y[k * ldY + i] : 0.0;
    Mixture m;
    mixture<NM>(Yk, n, c, m);
    int st = 0;
    const PRPoint q = pr_point(m, Tc, pc, cp != nullptr, st);
    if (rho) rho[i] = pc / (m.inv * q.Z * kR * Tc);
    if (h) h[i] = h_ig(m, Tc) + q.h_dep * m.inv;
    if (cp) cp[i] = cp_ig(m, Tc) + q.cp_dep * m.inv;
    if (Zo) Zo[i] = q.Z;
  }
}

size_t consts_smem(const EosParams& P) {
  return sizeof(double) * (size_t)(P.n * kSpcStride + P.n * P.n + 2 * P.K0 + 2 * P.n);
}

int grid_for(int64_t nmax) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t need = (nmax + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sms * 8;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

template <int NM>
cudaError_t pre_nm(const EosParams& P, const RowMap& rows, const double* T, const double* p,
                   const double* Y, int64_t ldY, double* h0, double* Z, void* x, int xkind,
                   int64_t ldx, float xs, int32_t* status, cudaStream_t st) {
  const size_t smem = consts_smem(P);
  const int g = grid_for(rows.nmax);
  switch (xkind) {
    case kXBF16:
      eos_pre_kernel<NM, __nv_bfloat16><<<g, kThreads, smem, st>>>(
          P, rows, T, p, Y, ldY, h0, Z, (__nv_bfloat16*)x, ldx, xs, status);
      break;
    case kXFP8:
      eos_pre_kernel<NM, __nv_fp8_e4m3><<<g, kThreads, smem, st>>>(
          P, rows, T, p, Y, ldY, h0, Z, (__nv_fp8_e4m3*)x, ldx, xs, status);
      break;
    default:
      eos_pre_kernel<NM, float><<<g, kThreads, smem, st>>>(P, rows, T, p, Y, ldY, h0, Z,
                                                            (float*)x, ldx, xs, status);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eos_pre(const EosParams& P, const RowMap& rows, const double* T,
                           const double* p, const double* Y, int64_t ldY, double* h0,
                           double* Z, void* x, int xkind, int64_t ldx, float x_scale,
                           int32_t* status, cudaStream_t st) {
  if (rows.nmax <= 0) return cudaSuccess;
  if (P.n <= 16)
    return pre_nm<16>(P, rows, T, p, Y, ldY, h0, Z, x, xkind, ldx, x_scale, status, st);
  return pre_nm<32>(P, rows, T, p, Y, ldY, h0, Z, x, xkind, ldx, x_scale, status, st);
}

cudaError_t launch_eos_post(const EosParams& P, const RowMap& rows, const float* O, int64_t ldo,
                            const double* h0, double* T, const double* p, double* Y,
                            int64_t ldY, const int32_t* pre_status, int32_t* cell_status,
                            cudaStream_t st) {
  if (rows.nmax <= 0) return cudaSuccess;
  const size_t smem = consts_smem(P);
  const int g = grid_for(rows.nmax);
  if (P.n <= 16)
    eos_post_kernel<16><<<g, kThreads, smem, st>>>(P, rows, O, ldo, h0, T, p, Y, ldY,
                                                   pre_status, cell_status);
  else
    eos_post_kernel<32><<<g, kThreads, smem, st>>>(P, rows, O, ldo, h0, T, p, Y, ldY,
                                                   pre_status, cell_status);
  return cudaGetLastError();
}

cudaError_t launch_props(const EosParams& P, int64_t n, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* rho, double* h, double* cp,
                         double* Z, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = consts_smem(P);
  const int g = grid_for(n);
  if (P.n <= 16)
    props_kernel<16><<<g, kThreads, smem, st>>>(P, n, T, p, Y, ldY, rho, h, cp, Z);
  else
    props_kernel<32><<<g, kThreads, smem, st>>>(P, n, T, p, Y, ldY, rho, h, cp, Z);
  return cudaGetLastError();
}

}  // namespace dfgb
