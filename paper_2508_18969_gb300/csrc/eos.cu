// Equation-of-state kernels of the reaction step: a1-a5 (eos_pre), a8-a10 (eos_post) and
// the real-fluid property evaluation. One thread per cell; species-major (SoA) field reads
// are coalesced across the threads of a warp.
//
// Peng-Robinson (Sec. 2 names the EoS; equations from Peng & Robinson 1976):
//   sqrt(a_k(T)) = sqrt(a_c,k) [1 + kappa_k (1 - sqrt(T / Tc_k))] = s_k - r_k sqrt(T),
//   a_m = sum_ij X_i X_j sqrt(a_i a_j) (1 - k_ij) = A0 - 2 A1 sqrt(T) + A2 T
// with three quadratic forms A0, A1, A2 of the composition, computed once per composition,
// so each Newton iteration of the T-from-h solve is O(1) in the species count.
//
// Precision plan (FP64 runs at 1/64 of the FP32 rate on this GPU, so FP64 instructions --
// arithmetic, compares and conversions alike -- are the scarce resource):
//   * every sum over species and species pairs (W_mix, b_m, the three forms, the mixture
//     NASA-7 coefficients) is accumulated in double-float on the FP32 pipes (~1e-14), from a
//     per-thread shared-memory column of the mass fractions in double-float;
//   * Y' = Y (1 + delta), its sum and the renormalisation are double-float too; delta itself
//     is FP32 (it only scales Y' - Y);
//   * finiteness and threshold tests look at the bits of the FP64 values, and the FP32 <-> FP64
//     conversions are integer operations (ddfloat.cuh);
//   * the cubic root, departure enthalpy, c_p and the Newton update are FP64; reciprocals and
//     square roots start from FP32 values and take FP64 Newton refinements;
//   * the Box-Cox features that feed the network are FP32 (they are quantised anyway).
#include "dfgb_internal.cuh"
#include "ddfloat.cuh"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace dfgb {
namespace {

constexpr double kSQ2 = 1.41421356237309504880;
constexpr double kInvR = 1.0 / kR;
// The step's EoS kernels run blocks of 256 threads, three per SM (80 registers): the constant
// tables in shared memory are then shared by more threads than with five blocks of 128, and the
// SM holds 24 warps instead of 20 (eos_pre 0.71 -> 0.66 ms, eos_post 0.69 -> 0.66 ms on the
// 2^20-cell step).
constexpr int kThreads = 256;
constexpr int kJacThreads = 64;  // the Jacobian's EoS kernel
constexpr int kPreBlocks = 3;    // resident blocks per SM the register budget is sized for
constexpr int kPostBlocks = 3;
constexpr int kPropThreads = 128;  // the property and transport kernels
constexpr int kPropBlocks = 5;
constexpr int kCellNotConverged = 1;
constexpr int kCellNoRoot = 2;
constexpr int kCellNonfinite = 4;
constexpr double kTLo = 50.0, kTHi = 5000.0;

struct Mixture {
  double inv;        // sum_k Y_k / W_k = 1 / W_mix
  double e[6];       // ideal-gas mass-specific enthalpy: h_ig(T) = sum_j e_j T^j, J/kg
  double A0, A1, A2; // a_m(T) = A0 - 2 A1 sqrt(T) + A2 T
  double bm;
  double kb;         // 1 / (2 sqrt2 b_m)
};

// The same coefficients in double-float, for the kernels that evaluate the state in double-float.
struct MixDF {
  f2 inv;
  f2 e[6];
  f2 A0, A1, A2;
  f2 bm;
  f2 kb;
};

// The raw double-float sums of one composition (before the 1/W_mix scalings).
struct MixSums {
  f2 inv, bs, e[6], F0, F1, F2;
};

struct SharedConsts {
  const f2* spcw;      // [n * kSpcStride] double-float species constants over W
  const float4* K4;    // pairs j > i, row by row: (Ks, Kr) double-float, (1 - k_ij) s_j / W_j,
                       // (1 - k_ij) r_j / W_j
  const float* kcol;   // [2 n] max_i |Ks_ij|, then max_i |Kr_ij| (rounded up)
  const float2* kf2;   // pairs j > i: (k_ij s_j / W_j, k_ij r_j / W_j) in FP32 (T-from-h only)
  const double* lnt;   // [256] log table (ln c_j, then 1 / c_j); FP64 kernels only
  const f2* lt2;       // the same table in double-float, in the same words; DF kernels only
  const double* norm;  // [2 K0 + 2 n]
  const float* normf;  // the same in FP32 (for the FP32 feature and increment arithmetic)
  const float* smax;   // [kSpcStride] EosParams::spcmax (T-from-h kernel only)
};

// 8-byte words of shared memory the constants take: FP64 normalisation, then the
// double-float tables (one f2 per word), then the FP32 normalisation.
__host__ __device__ inline int consts_words(const EosParams& P) {
  return 256 + 2 * P.K0 + 2 * P.n + P.n * kSpcStride + P.n * (P.n - 1) + 2 + P.n + (P.K0 + P.n + 1);
}

// DF: the first 256 words hold the double-float log table (the kernels that evaluate the state
// in double-float) instead of the FP64 one.
template <bool DF = false>
__device__ SharedConsts load_consts(const EosParams& P, double* sm0) {
  const int nspc = P.n * kSpcStride, nk = P.n * P.n, nn = 2 * P.K0 + 2 * P.n;
  if (DF) {
    float* t = reinterpret_cast<float*>(sm0);
    for (int i = threadIdx.x; i < 512; i += blockDim.x) t[i] = P.lntab2[i];
  } else {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sm0[i] = P.lntab[i];
  }
  double* sm = sm0 + 256;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) sm[i] = P.norm[i];
  // fs is 16-byte aligned (256 + nn doubles; nn is even) and so is the pair table after
  // the 8 n kSpcStride bytes of the species table
  float* fs = reinterpret_cast<float*>(sm + nn);
  for (int i = threadIdx.x; i < 2 * nspc; i += blockDim.x) fs[i] = P.spcw2[i];
  const int nk4 = 2 * P.n * (P.n - 1) + 4;   // the triangle's floats, padded to 16 bytes
  for (int i = threadIdx.x; i < nk4; i += blockDim.x) fs[2 * nspc + i] = P.K4[i];
  for (int i = threadIdx.x; i < 2 * P.n; i += blockDim.x) fs[2 * nspc + nk4 + i] = P.kcol[i];
  float* nf = fs + 2 * nspc + nk4 + 2 * P.n;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) nf[i] = (float)P.norm[i];
  __syncthreads();
  return SharedConsts{reinterpret_cast<const f2*>(fs),
                      reinterpret_cast<const float4*>(fs + 2 * nspc), fs + 2 * nspc + nk4,
                      nullptr, DF ? nullptr : sm0,
                      DF ? reinterpret_cast<const f2*>(sm0) : nullptr, sm, nf};
}

// The layout of the T-from-h kernel: double-float log table, FP64 normalisation, double-float
// species table, the FP32 k_ij pair table, FP32 normalisation (no double-float pair tables).
__host__ __device__ inline int consts_words_post(const EosParams& P) {
  return 256 + 2 * P.K0 + 2 * P.n + P.n * kSpcStride + P.n * (P.n - 1) / 2 + 1 +
         (P.K0 + P.n + 1) + kSpcStride / 2;
}

__device__ SharedConsts load_consts_post(const EosParams& P, double* sm0) {
  const int nspc = P.n * kSpcStride, nn = 2 * P.K0 + 2 * P.n;
  float* t = reinterpret_cast<float*>(sm0);
  for (int i = threadIdx.x; i < 512; i += blockDim.x) t[i] = P.lntab2[i];
  double* sm = sm0 + 256;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) sm[i] = P.norm[i];
  float* fs = reinterpret_cast<float*>(sm + nn);
  for (int i = threadIdx.x; i < 2 * nspc; i += blockDim.x) fs[i] = P.spcw2[i];
  float* ks = fs + 2 * nspc;   // 8-byte aligned (8 n kSpcStride bytes after fs)
  const int nkf = P.n * (P.n - 1) + 2;
  for (int i = threadIdx.x; i < nkf; i += blockDim.x) ks[i] = P.kf2[i];
  float* nf = ks + nkf;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) nf[i] = (float)P.norm[i];
  float* mx = nf + nn + 2;   // the FP32 normalisation takes K0 + n + 1 words
  for (int i = threadIdx.x; i < kSpcStride; i += blockDim.x) mx[i] = P.spcmax[i];
  __syncthreads();
  return SharedConsts{reinterpret_cast<const f2*>(fs), nullptr, nullptr,
                      reinterpret_cast<const float2*>(ks), nullptr,
                      reinterpret_cast<const f2*>(sm0), sm, nf, mx};
}

// FP64 reciprocal: FP32 seed, two FP64 Newton steps (relative error ~1 ulp).
__device__ __forceinline__ double drcp(double x) {
  double r = f_to_d(__frcp_rn(d_to_f_trunc(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Mixture coefficients of one composition (a1, a2 and the ideal-gas part of a4), all sums in
// double-float. ycol is this thread's column of mass fractions (entry k at ycol[k * STRIDE], STRIDE
// the block's threads).
// Symmetric quadratic forms with K_ii = 1, ys_i = Y_i s_i / W_i, yr_i = Y_i r_i / W_i:
//   F0 = sum_ij K_ij ys_i ys_j = sum_i ys_i (ys_i + 2 P_i),  P_i = sum_{j>i} Ks_ij Y_j,
//   F1 = sum_ij K_ij ys_i yr_j = sum_i ys_i (yr_i + Q_i) + yr_i P_i,  Q_i = sum_{j>i} Kr_ij Y_j,
//   F2 = sum_ij K_ij yr_i yr_j = sum_i yr_i (yr_i + 2 Q_i).
// The O(n^2) sums P_i and Q_i use offset accumulators (acc_off_fma) with one offset for all
// rows: B = sum_j |Y_j| max_l |Ks_lj| (summed rounding up) bounds every partial sum of every
// P_i (likewise for Q_i), and the offset is the power of two above B, or above 4 B when some
// Y_j is negative. A row's error is then a few units of 2^-48 B rather than of its own suffix
// bound, which the forms F weigh by ys_i <= B: the forms stay within ~2^-42 B^2, far inside the
// 1e-10 the state is held to, for 16 fewer operations per row than per-row offsets.
// Species i's terms of the O(n) sums (species-table columns 0 and 3..9) and its weighted mass
// fractions ys_i = Y_i s_i / W_i, yr_i = Y_i r_i / W_i.
__device__ __forceinline__ void species_row(const SharedConsts& c, int i, f2 y, float (&hq)[8],
                                            float (&lq)[8], f2& ys, f2& yr) {
  const float4* q4 = reinterpret_cast<const float4*>(c.spcw + i * kSpcStride);
  const float4 a = q4[0], b = q4[1], d = q4[2], e = q4[3], g = q4[4];
  acc_off_fma(hq[0], lq[0], y, f2{a.x, a.y});
  acc_off_fma(hq[1], lq[1], y, f2{b.z, b.w});
  acc_off_fma(hq[2], lq[2], y, f2{d.x, d.y});
  acc_off_fma(hq[3], lq[3], y, f2{d.z, d.w});
  acc_off_fma(hq[4], lq[4], y, f2{e.x, e.y});
  acc_off_fma(hq[5], lq[5], y, f2{e.z, e.w});
  acc_off_fma(hq[6], lq[6], y, f2{g.x, g.y});
  acc_off_fma(hq[7], lq[7], y, f2{g.z, g.w});
  ys = f2_mul(y, f2{a.z, a.w});
  yr = f2_mul(y, f2{b.x, b.y});
}

// Species i's terms of the three forms: F0 += ys ys + ys (2 P), F1 += ys yr + ys Q + yr P,
// F2 += yr yr + yr (2 Q).
__device__ __forceinline__ void forms_row(f2 ys, f2 yr, f2 P, f2 Q, float& F0h, float& F0l,
                                          float& F1h, float& F1l, float& F2h, float& F2l) {
  acc_off_fma(F0h, F0l, ys, ys);
  acc_off_fma(F0h, F0l, ys, f2_scale2(P));
  acc_off_fma(F1h, F1l, ys, yr);
  acc_off_fma(F1h, F1l, ys, Q);
  acc_off_fma(F1h, F1l, yr, P);
  acc_off_fma(F2h, F2l, yr, yr);
  acc_off_fma(F2h, F2l, yr, f2_scale2(Q));
}

template <int STRIDE>
__device__ void mixture_sums(const f2* ycol, int n, const SharedConsts& c, MixSums& ms) {
  constexpr int stride = STRIDE;   // threads per block: the column's entries are that far apart
  // The O(n) sums (1/W, b/W and the six enthalpy coefficients, species-table columns 0 and 3..9)
  // take offset accumulators too, with bounds Bq = sum_j |Y_j| |q_j| from the same pass.
  float Bs = 0.f, Br = 0.f, Bq[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) Bq[k] = 0.f;
  unsigned neg = 0u;
#pragma unroll 2
  for (int j = 0; j < n; ++j) {
    const float yh = ycol[j * stride].h, y = fabsf(yh);
    neg |= __float_as_uint(yh);
    const float4* q4 = reinterpret_cast<const float4*>(c.spcw + j * kSpcStride);
    const float4 a = q4[0], b = q4[1], d = q4[2], e = q4[3], g = q4[4];
    Bs = __fmaf_ru(y, c.kcol[j], Bs);
    Br = __fmaf_ru(y, c.kcol[n + j], Br);
    Bq[0] = __fmaf_ru(y, fabsf(a.x), Bq[0]);
    Bq[1] = __fmaf_ru(y, fabsf(b.z), Bq[1]);
    Bq[2] = __fmaf_ru(y, fabsf(d.x), Bq[2]);
    Bq[3] = __fmaf_ru(y, fabsf(d.z), Bq[3]);
    Bq[4] = __fmaf_ru(y, fabsf(e.x), Bq[4]);
    Bq[5] = __fmaf_ru(y, fabsf(e.z), Bq[5]);
    Bq[6] = __fmaf_ru(y, fabsf(g.x), Bq[6]);
    Bq[7] = __fmaf_ru(y, fabsf(g.z), Bq[7]);
  }
  // the bounds are rounded up throughout; |Y_j| <= |hi| (1 + 2^-23) is inside kcol's margin,
  // and the 2^-10 margin of the O(n) offsets covers the low parts of Y and of the table. The
  // terms are non-negative for Y >= 0 except in the enthalpy columns, whose coefficients have
  // either sign: those take the offset for terms of both signs.
  const float sgf = (neg >> 31) ? 4.0f : 1.0f;
  float sq[8], hq[8], lq[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    sq[k] = pow2_up(__fmul_ru((k < 2 ? sgf : 4.0f) * Bq[k], 1.0009765625f));
    hq[k] = sq[k];
    lq[k] = 0.f;
  }
  // The forms themselves: F0 += ys_i ys_i + ys_i (2 P_i), F1 += ys_i yr_i + ys_i Q_i + yr_i P_i,
  // F2 += yr_i yr_i + yr_i (2 Q_i), each into an offset accumulator. The absolute values of the
  // terms of F0 sum to sum_ij |K_ij| |ys_i| |ys_j| <= S_s Bs <= Bs^2, since S_s = sum_i |ys_i|
  // <= Bs (K_jj = 1) and sum_j |K_ij| |ys_j| <= Bs for every i; likewise Bs Br bounds F1 and
  // Br^2 bounds F2.
  const float sF0 = pow2_up(__fmul_ru(sgf, __fmul_ru(Bs, Bs)));
  const float sF1 = pow2_up(__fmul_ru(sgf, __fmul_ru(Bs, Br)));
  const float sF2 = pow2_up(__fmul_ru(sgf, __fmul_ru(Br, Br)));
  float F0h = sF0, F0l = 0.f, F1h = sF1, F1l = 0.f, F2h = sF2, F2l = 0.f;
  const float sgs = pow2_up(sgf * Bs), sgr = pow2_up(sgf * Br);   // the rows' common offsets
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const f2 y = ycol[i * stride];
    f2 ys, yr;
    species_row(c, i, y, hq, lq, ys, yr);
    float ph = sgs, pl = 0.f, qh = sgr, ql = 0.f;
    const float4* Kr4 = c.K4 + (i * n - i * (i + 1) / 2) - (i + 1);   // Kr4[j], j > i
#pragma unroll 4
    for (int j = i + 1; j < n; ++j) {
      const f2 yj = ycol[j * stride];
      const float4 k = Kr4[j];
      acc_off_fma(ph, pl, f2{k.x, k.y}, yj);
      acc_off_fma(qh, ql, f2{k.z, k.w}, yj);
    }
    forms_row(ys, yr, f2_norm(__fsub_rn(ph, sgs), pl), f2_norm(__fsub_rn(qh, sgr), ql),
              F0h, F0l, F1h, F1l, F2h, F2l);
    if ((i & 3) == 3) {  // every fourth species: keep the low parts small
#pragma unroll
      for (int k = 0; k < 8; ++k) acc_renorm(hq[k], lq[k]);
      acc_renorm(F0h, F0l);
      acc_renorm(F1h, F1l);
      acc_renorm(F2h, F2l);
    }
  }
  const f2 F0 = f2_norm(__fsub_rn(F0h, sF0), F0l);
  const f2 F1 = f2_norm(__fsub_rn(F1h, sF1), F1l);
  const f2 F2 = f2_norm(__fsub_rn(F2h, sF2), F2l);
  ms.inv = f2_norm(__fsub_rn(hq[0], sq[0]), lq[0]);
  ms.bs = f2_norm(__fsub_rn(hq[1], sq[1]), lq[1]);
#pragma unroll
  for (int k = 0; k < 6; ++k) ms.e[k] = f2_norm(__fsub_rn(hq[k + 2], sq[k + 2]), lq[k + 2]);
  ms.F0 = F0;
  ms.F1 = F1;
  ms.F2 = F2;
}

template <int STRIDE>
__device__ void mixture(const f2* ycol, int n, const SharedConsts& c, Mixture& m) {
  MixSums s;
  mixture_sums<STRIDE>(ycol, n, c, s);
  const double invd = f2_to(s.inv);
  const double Wm = drcp(invd);
  const double W2 = Wm * Wm;
  m.inv = invd;
#pragma unroll
  for (int k = 0; k < 6; ++k) m.e[k] = f2_to(s.e[k]);
  m.A0 = W2 * f2_to(s.F0);
  m.A1 = W2 * f2_to(s.F1);
  m.A2 = W2 * f2_to(s.F2);
  m.bm = Wm * f2_to(s.bs);
  m.kb = drcp(2.0 * kSQ2 * m.bm);
}

// Double-float constants (hi, lo) of the state evaluation.
constexpr float kRh = (float)kR, kRl = (float)(kR - (double)(float)kR);
constexpr float kIRh = (float)(1.0 / kR), kIRl = (float)(1.0 / kR - (double)(float)(1.0 / kR));
constexpr float kS2h = (float)(2.0 * kSQ2), kS2l = (float)(2.0 * kSQ2 - (double)(float)(2.0 * kSQ2));
constexpr float kSPh = (float)(1.0 + kSQ2), kSPl = (float)(1.0 + kSQ2 - (double)(float)(1.0 + kSQ2));
constexpr float kSMh = (float)(1.0 - kSQ2), kSMl = (float)(1.0 - kSQ2 - (double)(float)(1.0 - kSQ2));
constexpr float k3h = (float)(1.0 / 3.0), k3l = (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0));
constexpr float kL2h = (float)0.69314718055994530942,
                kL2l = (float)(0.69314718055994530942 - (double)(float)0.69314718055994530942);

// W_mix scalings of the sums, in double-float.
__device__ __forceinline__ void mix_df_final(const MixSums& s, MixDF& m) {
  const f2 Wm = f2_rcp(s.inv);
  const f2 W2 = f2_mul(Wm, Wm);
  m.inv = s.inv;
#pragma unroll
  for (int k = 0; k < 6; ++k) m.e[k] = s.e[k];
  m.A0 = f2_mul(W2, s.F0);
  m.A1 = f2_mul(W2, s.F1);
  m.A2 = f2_mul(W2, s.F2);
  m.bm = f2_mul(Wm, s.bs);
  m.kb = f2_rcp(f2_mul(m.bm, f2{kS2h, kS2l}));
}

template <int STRIDE>
__device__ void mixture_df(const f2* ycol, int n, const SharedConsts& c, MixDF& m) {
  MixSums s;
  mixture_sums<STRIDE>(ycol, n, c, s);
  mix_df_final(s, m);
}

// ln(x) for a positive normal x from the shared table: x = 2^e m, m in [1, 2); with c the
// midpoint of m's 1/128 interval, ln x = e ln2 + ln c + ln(1 + r), r = m / c - 1, |r| < 2^-8,
// ln(1 + r) by its series to r^5 (truncation below 4e-16). Other x take the library log.
__device__ __forceinline__ double dlog_tab(double x, const double* lnt) {
  const int hi = __double2hiint(x);
  const int be = (hi >> 20) & 0x7FF;
  if (hi <= 0 || be == 0 || be == 0x7FF) return log(x);
  const int j = (hi >> 13) & 127;
  const double m = __hiloint2double((hi & 0x000FFFFF) | 0x3FF00000, __double2loint(x));
  const double r = fma(m, lnt[128 + j], -1.0);
  const double poly = r * fma(r, fma(r, fma(r, fma(r, 0.2, -0.25), 1.0 / 3.0), -0.5), 1.0);
  const double e = f_to_d((float)(be - 1023));
  constexpr double kLn2Hi = 6.93147180369123816490e-01, kLn2Lo = 1.90821492927058770002e-10;
  return fma(e, kLn2Hi, lnt[j] + fma(e, kLn2Lo, poly));
}

// 1/x from the FP32 reciprocal and one FP64 Newton step (relative error ~2^-46).
__device__ __forceinline__ double drcp1(double x) {
  const double r = f_to_d(__frcp_rn(d_to_f_trunc(x)));
  return fma(r, fma(-x, r, 1.0), r);
}

// sqrt(x) for a positive normal x: t0 = x rsqrt_32(x), then one Newton step
// t = t0 + (x - t0^2) r / 2 with the FP32 r = rsqrt_32(x) (relative error ~2^-44).
__device__ __forceinline__ double dsqrt_pos(double x) {
  const float r = rsqrtf(d_to_f_trunc(x));
  const double rd = f_to_d(r);
  const double t0 = x * rd;
  return fma(fma(-t0, t0, x), 0.5 * rd, t0);
}

// mixture() for the T-from-h solve, where h(T) needs ~1e-8 relative accuracy (T' to ~1e-6 K):
// with K = 1 - k the forms split into squares of O(n) sums, kept in double-float, and k_ij
// corrections (k <= 0.1 of the squares) summed in FP32,
//   F0 = S_s^2 - 2 sum_i ys_i Pk_i,  F1 = S_s S_r - sum_i (ys_i Qk_i + yr_i Pk_i),
//   F2 = S_r^2 - 2 sum_i yr_i Qk_i,  Pk_i = sum_{j>i} k_ij ys_j,  Qk_i = sum_{j>i} k_ij yr_j.
// Species i's terms of mixture_post's ten O(n) sums; q1, q2 return s_i / W_i and r_i / W_i.
__device__ __forceinline__ void species_row_post(const SharedConsts& c, int i, f2 y,
                                                 float (&hq)[kSpcStride], float (&lq)[kSpcStride],
                                                 float& q1, float& q2) {
  const float4* q4 = reinterpret_cast<const float4*>(c.spcw + i * kSpcStride);
#pragma unroll
  for (int k = 0; k < kSpcStride / 2; ++k) {
    const float4 a = q4[k];
    acc_off_fma(hq[2 * k], lq[2 * k], y, f2{a.x, a.y});
    acc_off_fma(hq[2 * k + 1], lq[2 * k + 1], y, f2{a.z, a.w});
    if (k == 0) q1 = a.z;
    if (k == 1) q2 = a.x;
  }
}

template <int STRIDE>
__device__ void mixture_post(const f2* ycol, int n, const SharedConsts& c, MixDF& m) {
  constexpr int stride = STRIDE;
  // the ten O(n) sums over the species table take offset accumulators, as in mixture(), here
  // with the looser bounds (sum_j |Y_j|) max_j |q_j|: h(T) is needed to ~1e-8 only, and the
  // bounds then cost one addition per species instead of ten
  float S = 0.f;
  unsigned neg = 0u;
#pragma unroll 2
  for (int j = 0; j < n; ++j) {
    const float yh = ycol[j * stride].h;
    neg |= __float_as_uint(yh);
    S = __fadd_ru(S, fabsf(yh));
  }
  float Bq[kSpcStride];
#pragma unroll
  for (int k = 0; k < kSpcStride; ++k) Bq[k] = __fmul_ru(S, c.smax[k]);
  // columns 0..3 (1/W, s/W, r/W, b/W) are non-negative; the enthalpy columns have either sign
  const float sgf = (neg >> 31) ? 4.0f : 1.0f;
  float sq[kSpcStride], hq[kSpcStride], lq[kSpcStride];
#pragma unroll
  for (int k = 0; k < kSpcStride; ++k) {
    sq[k] = pow2_up(__fmul_ru((k < 4 ? sgf : 4.0f) * Bq[k], 1.0009765625f));
    hq[k] = sq[k];
    lq[k] = 0.f;
  }
  float C0 = 0.f, C1 = 0.f, C2 = 0.f;
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const f2 y = ycol[i * stride];
    float q1h, q2h;
    species_row_post(c, i, y, hq, lq, q1h, q2h);
    float Pk = 0.f, Qk = 0.f;
    const float2* R = c.kf2 + (i * n - i * (i + 1) / 2) - (i + 1);   // R[j], j > i
#pragma unroll 4
    for (int j = i + 1; j < n; ++j) {
      const float yj = ycol[j * stride].h;
      const float2 k = R[j];
      Pk = fmaf(k.x, yj, Pk);
      Qk = fmaf(k.y, yj, Qk);
    }
    if ((i & 3) == 3) {  // every fourth species: keep the low parts small
#pragma unroll
      for (int k = 0; k < kSpcStride; ++k) acc_renorm(hq[k], lq[k]);
    }
    const float ysi = y.h * q1h, yri = y.h * q2h;
    C0 = fmaf(ysi, Pk, C0);
    C1 = fmaf(ysi, Qk, fmaf(yri, Pk, C1));
    C2 = fmaf(yri, Qk, C2);
  }
  f2 r[kSpcStride];
#pragma unroll
  for (int k = 0; k < kSpcStride; ++k) r[k] = f2_norm(__fsub_rn(hq[k], sq[k]), lq[k]);
  const f2 inv = r[0], Ss = r[1], Sr = r[2], bs = r[3];
  const f2 Wm = f2_rcp(inv);
  const f2 W2 = f2_mul(Wm, Wm);
  m.inv = inv;
#pragma unroll
  for (int k = 0; k < 6; ++k) m.e[k] = r[4 + k];
  m.A0 = f2_mul(W2, f2_addf(f2_mul(Ss, Ss), -2.0f * C0));
  m.A1 = f2_mul(W2, f2_addf(f2_mul(Ss, Sr), -C1));
  m.A2 = f2_mul(W2, f2_addf(f2_mul(Sr, Sr), -2.0f * C2));
  m.bm = f2_mul(Wm, bs);
  m.kb = f2_rcp(f2_mul(m.bm, f2{kS2h, kS2l}));
}

__device__ __forceinline__ double h_ig(const Mixture& m, double T) {
  return fma(fma(fma(fma(fma(m.e[5], T, m.e[4]), T, m.e[3]), T, m.e[2]), T, m.e[1]), T, m.e[0]);
}

__device__ __forceinline__ double cp_ig(const Mixture& m, double T) {
  return fma(fma(fma(fma(5.0 * m.e[5], T, 4.0 * m.e[4]), T, 3.0 * m.e[3]), T, 2.0 * m.e[2]), T,
             m.e[1]);
}

// One Newton step on the cubic. The step uses an FP32 reciprocal of f'(Z): that scales the
// correction by (1 + O(1e-7)), so a step from an FP32-accurate seed still gains ~7 digits.
__device__ __forceinline__ double cubic_step(double Z, double c2, double c1, double c0) {
  const double f = fma(fma(Z + c2, Z, c1), Z, c0);
  const double fp = fma(fma(3.0, Z, 2.0 * c2), Z, c1);
  const float fpf = d_to_f_trunc(fp);
  return fpf != 0.0f ? fma(-f, f_to_d(__frcp_rn(fpf)), Z) : Z;
}

__device__ __forceinline__ double cubic_polish(double Z, double c2, double c1, double c0) {
  return cubic_step(cubic_step(Z, c2, c1, c0), c2, c1, c0);
}

__device__ __forceinline__ double g_dep(double Z, double A, double B, const double* lnt) {
  return Z - 1.0 - dlog_tab(Z - B, lnt) -
         A * drcp(2.0 * kSQ2 * B) * dlog_tab((Z + (1.0 + kSQ2) * B) * drcp(Z + (1.0 - kSQ2) * B), lnt);
}

// Compressibility (a3): the real root of
//   Z^3 - (1 - B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0
// above B with least departure Gibbs energy (ties within 1e-12 keep the larger root).
// Seeds come from the FP32 closed form (Cardano for one real root, the trigonometric form
// for three), each polished by FP64 Newton steps on the cubic: two, or with FAST one, plus a
// second where the first moved the seed by more than 1e-6 relative (a poor seed).
// The three-real-root case of select_Z: seeds from the trigonometric form, each polished, the
// root above B with least departure Gibbs energy kept. Out of line: it is the rarer branch,
// and keeping it out of the Newton loop's body keeps that loop's code small.
__device__ __noinline__ double select_Z3(double A, double B, double c2, double c1, double c0,
                                         double P, double Q, const double* lnt, int& status);

template <bool FAST>
__device__ double select_Z(double A, double B, const double* lnt, int& status) {
  const double c2 = B - 1.0;
  const double c1 = A - 3.0 * B * B - 2.0 * B;
  const double c0 = B * B + B * B * B - A * B;
  const double P = c1 - c2 * c2 * (1.0 / 3.0);
  const double Q = 2.0 * c2 * c2 * c2 * (1.0 / 27.0) - c2 * c1 * (1.0 / 3.0) + c0;
  const double disc = 0.25 * Q * Q + P * P * P * (1.0 / 27.0);
  if (disc > 0.0) {
    const float qf = d_to_f_trunc(Q), pf = d_to_f_trunc(P);
    const float sq = sqrtf(d_to_f_trunc(disc));
    const float u = cbrtf(-0.5f * qf - copysignf(sq, qf));
    const float t = (u != 0.0f) ? u - pf / (3.0f * u) : 0.0f;
    const double Z0 = f_to_d(t) - c2 * (1.0 / 3.0);
    double Z = cubic_step(Z0, c2, c1, c0);
    if (!FAST || fabsf(d_to_f_trunc(Z - Z0)) > 1e-6f * fabsf(d_to_f_trunc(Z)))
      Z = cubic_step(Z, c2, c1, c0);
    if (!(Z > B)) status |= kCellNoRoot;
    return Z;
  }
  return select_Z3(A, B, c2, c1, c0, P, Q, lnt, status);
}

__device__ __noinline__ double select_Z3(double A, double B, double c2, double c1, double c0,
                                         double P, double Q, const double* lnt, int& status) {
  const float pf = d_to_f_trunc(P);
  const float m = (pf < 0.0f) ? 2.0f * sqrtf(-pf / 3.0f) : 0.0f;
  float cphi = (pf < 0.0f) ? (3.0f * d_to_f_trunc(Q) / (2.0f * pf)) * sqrtf(-3.0f / pf) : 0.0f;
  cphi = fminf(fmaxf(cphi, -1.0f), 1.0f);
  const float phi = acosf(cphi) * (1.0f / 3.0f);
  double best = __longlong_as_double(0x7ff8000000000000LL);
  double gbest = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // k = 0, 1, 2 give descending seeds
    const float tk = m * cosf(phi - 2.0943951023931955f * (float)k);
    const double Z = cubic_polish(cubic_polish(f_to_d(tk) - c2 * (1.0 / 3.0), c2, c1, c0), c2,
                                  c1, c0);
    if (Z > B) {
      const double g = g_dep(Z, A, B, lnt);
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

// Real-fluid state at (T, p) of a composition (a2-a4), with the departure cp if asked. With
// FAST (the T-from-h solve, whose cp only sets the chord slope) cp is evaluated in FP32 and
// the cubic gets one polishing step.
template <bool FAST>
__device__ PRPoint pr_point(const Mixture& m, double T, double p, bool want_cp, const double* lnt,
                            int& status) {
  const double iT = FAST ? drcp1(T) : drcp(T);
  const double t = dsqrt_pos(T);
  const double it = t * iT;                       // 1 / sqrt(T)
  const double am = fma(-2.0 * m.A1, t, fma(m.A2, T, m.A0));
  const double dam = fma(-m.A1, it, m.A2);
  const double RT = kR * T;
  const double iRT = iT * kInvR;
  const double A = am * p * iRT * iRT;
  const double B = m.bm * p * iRT;
  PRPoint r;
  r.Z = select_Z<FAST>(A, B, lnt, status);
  const double Zp = r.Z + (1.0 + kSQ2) * B;
  const double Zm = r.Z + (1.0 - kSQ2) * B;
  const double iZm = FAST ? drcp1(Zm) : drcp(Zm);
  const double L = dlog_tab(Zp * iZm, lnt);
  const double tdam_am = fma(T, dam, -am);
  r.h_dep = fma(RT, r.Z - 1.0, tdam_am * m.kb * L);
  r.cp_dep = 0.0;
  if (FAST && want_cp) {
    // FP32: dA/dT = p (dam - 2 am / T) / (RT)^2 needs no division by am
    const float Tf = d_to_f_trunc(T), iTf = __frcp_rn(Tf), itf = rsqrtf(Tf);
    const float Z = d_to_f_trunc(r.Z), Af = d_to_f_trunc(A), Bf = d_to_f_trunc(B);
    const float pf = d_to_f_trunc(p), iRTf = iTf * (float)kInvR;
    const float d2am = 0.5f * d_to_f_trunc(m.A1) * itf * iTf;
    const float dB = -Bf * iTf;
    const float dA = pf * iRTf * iRTf * (d_to_f_trunc(dam) - 2.0f * d_to_f_trunc(am) * iTf);
    const float FZ = fmaf(3.0f * Z, Z, -2.0f * (1.0f - Bf) * Z) + (Af - 3.0f * Bf * Bf - 2.0f * Bf);
    const float FA = Z - Bf;
    const float FB = Z * Z - (6.0f * Bf + 2.0f) * Z - (Af - 2.0f * Bf - 3.0f * Bf * Bf);
    const float dZ = -(FA * dA + FB * dB) / FZ;
    const float s2 = (float)kSQ2;
    const float dL = (dZ + (1.0f + s2) * dB) / d_to_f_trunc(Zp) - (dZ + (1.0f - s2) * dB) / d_to_f_trunc(Zm);
    r.cp_dep = f_to_d((float)kR * (Z - 1.0f) + (float)kR * Tf * dZ +
                      d_to_f_trunc(m.kb) * (Tf * d2am * d_to_f_trunc(L) + d_to_f_trunc(tdam_am) * dL));
  } else if (want_cp) {
    const double d2am = 0.5 * m.A1 * it * iT;
    const double dB = -B * iT;
    const double dA = A * fma(dam, drcp(am), -2.0 * iT);
    const double Z = r.Z;
    const double FZ = fma(3.0 * Z, Z, -2.0 * (1.0 - B) * Z) + (A - 3.0 * B * B - 2.0 * B);
    const double FA = Z - B;
    const double FB = Z * Z - (6.0 * B + 2.0) * Z - (A - 2.0 * B - 3.0 * B * B);
    const double dZ = -(FA * dA + FB * dB) / FZ;
    const double dL = (dZ + (1.0 + kSQ2) * dB) * drcp(Zp) - (dZ + (1.0 - kSQ2) * dB) * iZm;
    r.cp_dep = kR * (Z - 1.0) + RT * dZ + m.kb * (T * d2am * L + tdam_am * dL);
  }
  return r;
}

// a9: T from h(T, p, Y') = h0 for the composition of m, safeguarded Newton inside a bracket
// that starts at [50, 5000] K and shrinks with the sign of h - h0. Adds flags to st and the
// iteration count to iters; returns the last iterate.
template <bool FAST>
__device__ double solve_T(const Mixture& m, double pc, double h0c, double Told, const EosParams& P,
                          const double* lnt, int& iters, int& st) {
  double lo = kTLo, hi = kTHi;
  double Tn = fmin(fmax(Told, lo), hi);
  bool conv = false, need_cp = true;
  double icp = 0.0;
  const float tolf = (float)P.newton_tol;
  for (int it = 0; it < P.newton_max_iter; ++it) {
    ++iters;
    int s2 = 0;
    const PRPoint q = pr_point<FAST>(m, Tn, pc, need_cp, lnt, s2);
    if (s2) {
      st |= s2;
      break;
    }
    const double f = h_ig(m, Tn) + q.h_dep * m.inv - h0c;
    // Chord steps: the slope of the first iteration is reused while the iterates stay
    // close (each step contracts the error by ~|1 - cp(T)/cp(T0)| ~ 1e-5 there); an FP32
    // reciprocal of cp scales the step by 1 + O(1e-7) on top.
    if (need_cp) icp = f_to_d(__frcp_rn(d_to_f_trunc(cp_ig(m, Tn) + q.cp_dep * m.inv)));
    // Tn lies inside [lo, hi] (the start is clamped, later iterates are inside by
    // construction), so the bracket update needs no min/max; the sign test reads the bit
    if (__double2hiint(f) >= 0) hi = Tn; else lo = Tn;
    const double step = -f * icp;
    double Tx = Tn + step;
    // a step within tolerance has converged (the test is a threshold, FP32 is enough); only
    // a longer step that leaves the bracket (or is not finite) is replaced by bisection,
    // after which the slope is evaluated afresh
    const bool done = fabsf(d_to_f_trunc(step)) <= tolf * d_to_f_trunc(Tn);
    need_cp = false;
    if (!done && !(Tx > lo && Tx < hi)) {
      Tx = 0.5 * (lo + hi);
      need_cp = true;
    }
    Tn = Tx;
    if (done) {
      conv = true;
      break;
    }
  }
  if (!conv && st == 0) st |= kCellNotConverged;
  if (!d_finite(Tn)) st |= kCellNonfinite;
  return Tn;
}

// ---------------------------------------------------------------- double-float state
// The real-fluid point of eos_pre and every Newton iteration of eos_post in double-float on
// the FP32 pipes (~2^-46 relative per operation). On this GPU one FP64 instruction costs the
// issue time of ~30 FP32 instructions (measured in the T-from-h kernel), and a double-float
// operation takes 4 to 15. The steps are those of pr_point / solve_T above.

// ln x for a positive normal double-float x from the double-float table lt (ln c_j, then
// 1 / c_j): x = 2^e m, m in [1, 2); r = m / c_j - 1 (|r| < 2^-8) formed exactly to first order;
// ln(1 + r) = r - r^2/2 in double-float plus r^3 (1/3 - r/4 + r^2/5) in FP32 (below 2^-25).
__device__ __noinline__ f2 f2_log_slow(f2 x) { return f2_from(log(f2_to(x))); }

__device__ __forceinline__ f2 f2_log_tab(f2 x, const f2* lt) {
  const unsigned u = __float_as_uint(x.h);
  const int be = (int)((u >> 23) & 0xFFu);
  if ((int)u <= 0 || be == 0 || be >= 254) return f2_log_slow(x);
  const int j = (int)((u >> 16) & 127u);
  const float sc = __uint_as_float((unsigned)(254 - be) << 23);   // 2^-(be - 127), exact
  const float mh = __fmul_rn(x.h, sc), ml = __fmul_rn(x.l, sc);
  const f2 ic = lt[128 + j];
  const float p = __fmul_rn(mh, ic.h);
  const float pe = __fmaf_rn(mh, ic.h, -p);
  const f2 r = f2_norm(__fsub_rn(p, 1.0f), __fmaf_rn(mh, ic.l, __fmaf_rn(ml, ic.h, pe)));
  const float r2 = __fmul_rn(r.h, r.h);
  const float r2e = __fmaf_rn(2.0f * r.h, r.l, __fmaf_rn(r.h, r.h, -r2));
  const float tail =
      __fmul_rn(__fmul_rn(r2, r.h), __fmaf_rn(r.h, __fmaf_rn(r.h, 0.2f, -0.25f), 0.33333334f));
  const f2 l1p = f2_addf(f2_add(r, f2{-0.5f * r2, -0.5f * r2e}), tail);
  const float E = (float)(be - 127);
  const float q = __fmul_rn(E, kL2h);
  const f2 el2 = f2_norm(q, __fmaf_rn(E, kL2l, __fmaf_rn(E, kL2h, -q)));
  return f2_add(f2_add(el2, lt[j]), l1p);
}

// x^(1/3) in FP32 for a seed: 2^(log2|x| / 3) with the sign of x, then one Newton step
// t <- t - (t^3 - x) / (3 t^2) (~1 ulp).
__device__ __forceinline__ float cbrt_seed(float x) {
  if (x == 0.0f) return 0.0f;
  const float t = copysignf(exp2f(log2f(fabsf(x)) * (1.0f / 3.0f)), x);
  return t - (t - __fdividef(x, t * t)) * (1.0f / 3.0f);
}

// One Newton step on the cubic, f(Z) and f'(Z) in double-float, the step with an approximate
// FP32 reciprocal of f'(Z) (it scales the correction by 1 + O(1e-7)).
__device__ __forceinline__ f2 cubic_step_df(f2 Z, f2 c2, f2 c1, f2 c0) {
  const f2 f = f2_fma(f2_fma(f2_add(Z, c2), Z, c1), Z, c0);
  const f2 fp = f2_fma(f2_add(f2_mulf(Z, 3.0f), f2_scale2(c2)), Z, c1);
  return fp.h != 0.0f ? f2_add(Z, f2_mulf(f, -__fdividef(1.0f, fp.h))) : Z;
}

__device__ __forceinline__ f2 g_dep_df(f2 Z, f2 A, f2 B, const f2* lt) {
  const f2 Zp = f2_fma(B, f2{kSPh, kSPl}, Z), Zm = f2_fma(B, f2{kSMh, kSMl}, Z);
  const f2 L = f2_log_tab(f2_mul(Zp, f2_rcp(Zm)), lt);
  const f2 a = f2_mul(A, f2_rcp(f2_mul(B, f2{kS2h, kS2l})));
  return f2_sub(f2_sub(f2_addf(Z, -1.0f), f2_log_tab(f2_sub(Z, B), lt)), f2_mul(a, L));
}

// Departure Gibbs energy in FP32 (for choosing among the three roots when the choice is clear).
__device__ __forceinline__ float g_dep_f(float Z, float A, float B) {
  const float s2 = 1.41421356f;
  return Z - 1.0f - __logf(Z - B) -
         __fdividef(A, 2.0f * s2 * B) * __logf(__fdividef(Z + (1.0f + s2) * B, Z + (1.0f - s2) * B));
}

// Three real roots (select_Z3 in double-float). Out of line, as there. The roots above B are
// first ranked by their FP32 seeds and FP32 departure Gibbs energies; when one root is lower
// by more than 1e-4 (FP32 errors are ~1e-6 there) and no seed lies within 1e-5 of B, only
// that root is polished. Otherwise every root is polished and compared in double-float.
__device__ __noinline__ f2 select_Z3_df(f2 A, f2 B, f2 c2, f2 c1, f2 c0, f2 c23, float Pf,
                                        float Qf, const f2* lt, int& status) {
  const float m = (Pf < 0.0f) ? 2.0f * sqrtf(-Pf / 3.0f) : 0.0f;
  float cphi = (Pf < 0.0f) ? (3.0f * Qf / (2.0f * Pf)) * sqrtf(-3.0f / Pf) : 0.0f;
  cphi = fminf(fmaxf(cphi, -1.0f), 1.0f);
  const float phi = acosf(cphi) * (1.0f / 3.0f);
  {
    float tbest = 0.0f, g1 = __int_as_float(0x7f800000), g2 = g1;
    bool clear = true;
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const float tk = m * cosf(phi - 2.0943951023931955f * (float)k);
      const float zk = tk - c23.h;
      if (fabsf(zk - B.h) <= 1e-5f * fabsf(B.h)) clear = false;
      if (zk > B.h) {
        const float g = g_dep_f(zk, A.h, B.h);
        if (!(g == g)) clear = false;
        if (g < g1) {
          g2 = g1;
          g1 = g;
          tbest = tk;
        } else if (g < g2) {
          g2 = g;
        }
      }
    }
    if (clear && g1 < g2 - 1e-4f) {
      f2 Z = f2_sub(f2{tbest, 0.0f}, c23);
#pragma unroll 1
      for (int q = 0; q < 4; ++q) Z = cubic_step_df(Z, c2, c1, c0);
      if (!f2_gt(Z, B)) status |= kCellNoRoot;
      return Z;
    }
  }
  f2 best = f2{__int_as_float(0x7fc00000), 0.0f};
  f2 gbest = f2{__int_as_float(0x7f800000), 0.0f};
  bool have = false;
#pragma unroll 1
  for (int k = 0; k < 3; ++k) {  // k = 0, 1, 2 give descending seeds
    const float tk = m * cosf(phi - 2.0943951023931955f * (float)k);
    f2 Z = f2_sub(f2{tk, 0.0f}, c23);
#pragma unroll 1
    for (int q = 0; q < 4; ++q) Z = cubic_step_df(Z, c2, c1, c0);
    if (f2_gt(Z, B)) {
      const f2 g = g_dep_df(Z, A, B, lt);
      if (!have || f2_lt(g, f2_addf(gbest, -1e-12f))) {
        gbest = g;
        best = Z;
        have = true;
      }
    }
  }
  if (!have) status |= kCellNoRoot;
  return best;
}

// select_Z in double-float: the coefficients, P, Q and the discriminant in double-float, the
// seeds in FP32, one or two double-float Newton polishes as in select_Z.
template <bool FAST>
__device__ __forceinline__ f2 select_Z_df(f2 A, f2 B, const f2* lt, int& status) {
  const f2 c2 = f2_addf(B, -1.0f);
  const f2 c1 = f2_sub(A, f2_mul(B, f2_addf(f2_mulf(B, 3.0f), 2.0f)));  // A - 3B^2 - 2B
  const f2 c0 = f2_mul(B, f2_sub(f2_fma(B, B, B), A));                 // B^2 + B^3 - AB
  const f2 c23 = f2_mul(c2, f2{k3h, k3l});                              // c2 / 3
  const f2 P = f2_sub(c1, f2_mul(c2, c23));                             // c1 - c2^2 / 3
  // Q = 2 c2^3 / 27 - c2 c1 / 3 + c0 = 2 (c2/3)^3 - (c2/3) c1 + c0
  const f2 Q = f2_add(f2_sub(f2_scale2(f2_mul(c23, f2_mul(c23, c23))), f2_mul(c23, c1)), c0);
  const f2 P3 = f2_mul(P, f2{k3h, k3l});
  const f2 Qh = f2{0.5f * Q.h, 0.5f * Q.l};
  const f2 disc = f2_fma(Qh, Qh, f2_mul(P3, f2_mul(P3, P3)));          // Q^2/4 + P^3/27
  if (disc.h > 0.0f) {
    const float qf = Q.h, pf = P.h;
    const float sq = sqrtf(disc.h);
    const float u = cbrt_seed(-0.5f * qf - copysignf(sq, qf));
    const float t = (u != 0.0f) ? u - __fdividef(pf, 3.0f * u) : 0.0f;
    const f2 Z0 = f2_sub(f2{t, 0.0f}, c23);
    f2 Z = cubic_step_df(Z0, c2, c1, c0);
    if (!FAST || fabsf(Z.h - Z0.h) > 1e-6f * fabsf(Z.h)) Z = cubic_step_df(Z, c2, c1, c0);
    if (!f2_gt(Z, B)) status |= kCellNoRoot;
    return Z;
  }
  return select_Z3_df(A, B, c2, c1, c0, c23, P.h, Q.h, lt, status);
}

struct PRPointDF {
  f2 Z, h_dep;    // compressibility, molar departure enthalpy
  float cp_dep;   // its T-derivative in FP32 (FAST with want_cp only)
};

// pr_point in double-float; with FAST the departure cp (the chord slope of the T-from-h
// solve) in FP32 as there.
template <bool FAST>
__device__ PRPointDF pr_point_df(const MixDF& m, f2 T, f2 p, bool want_cp, const f2* lt,
                                 int& status) {
  const f2 iT = f2_rcp(T);
  const f2 t = f2_sqrt_pos(T);
  const f2 it = f2_mul(t, iT);                                   // 1 / sqrt(T)
  const f2 am = f2_fma(m.A1, f2{-2.0f * t.h, -2.0f * t.l}, f2_fma(m.A2, T, m.A0));
  const f2 dam = f2_fma(f2_neg(m.A1), it, m.A2);
  const f2 RT = f2_mul(T, f2{kRh, kRl});
  const f2 iRT = f2_mul(iT, f2{kIRh, kIRl});
  const f2 piRT = f2_mul(p, iRT);
  const f2 A = f2_mul(f2_mul(am, piRT), iRT);
  const f2 B = f2_mul(m.bm, piRT);
  PRPointDF r;
  r.Z = select_Z_df<FAST>(A, B, lt, status);
  const f2 Zp = f2_fma(B, f2{kSPh, kSPl}, r.Z), Zm = f2_fma(B, f2{kSMh, kSMl}, r.Z);
  const f2 L = f2_log_tab(f2_mul(Zp, f2_rcp(Zm)), lt);
  const f2 tdam_am = f2_fma(T, dam, f2_neg(am));
  r.h_dep = f2_fma(RT, f2_addf(r.Z, -1.0f), f2_mul(f2_mul(tdam_am, m.kb), L));
  r.cp_dep = 0.0f;
  if (FAST && want_cp) {
    // FP32: dA/dT = p (dam - 2 am / T) / (RT)^2 needs no division by am
    const float Tf = T.h, iTf = __fdividef(1.0f, Tf), itf = rsqrtf(Tf);
    const float Z = r.Z.h, Af = A.h, Bf = B.h;
    const float pf = p.h, iRTf = iTf * (float)kInvR;
    const float d2am = 0.5f * m.A1.h * itf * iTf;
    const float dB = -Bf * iTf;
    const float dA = pf * iRTf * iRTf * (dam.h - 2.0f * am.h * iTf);
    const float FZ = fmaf(3.0f * Z, Z, -2.0f * (1.0f - Bf) * Z) + (Af - 3.0f * Bf * Bf - 2.0f * Bf);
    const float FA = Z - Bf;
    const float FB = Z * Z - (6.0f * Bf + 2.0f) * Z - (Af - 2.0f * Bf - 3.0f * Bf * Bf);
    // (a chord slope: approximate FP32 divisions suffice)
    const float dZ = -__fdividef(FA * dA + FB * dB, FZ);
    const float s2 = (float)kSQ2;
    const float dL = __fdividef(dZ + (1.0f + s2) * dB, Zp.h) - __fdividef(dZ + (1.0f - s2) * dB, Zm.h);
    r.cp_dep = (float)kR * (Z - 1.0f) + (float)kR * Tf * dZ +
               m.kb.h * (Tf * d2am * L.h + tdam_am.h * dL);
  }
  return r;
}

__device__ __forceinline__ f2 h_ig_df(const MixDF& m, f2 T) {
  f2 a = m.e[5];
#pragma unroll
  for (int k = 4; k >= 0; --k) a = f2_fma(a, T, m.e[k]);
  return a;
}

__device__ __forceinline__ float cp_ig_f(const MixDF& m, float T) {
  return fmaf(fmaf(fmaf(fmaf(5.0f * m.e[5].h, T, 4.0f * m.e[4].h), T, 3.0f * m.e[3].h), T,
                   2.0f * m.e[2].h), T, m.e[1].h);
}

// solve_T in double-float (a9): the same safeguarded chord-Newton iteration inside the bracket
// [50, 5000] K, the residual h(T) - h0 and the iterates in double-float.
__device__ f2 solve_T_df(const MixDF& m, f2 p, f2 h0, double Told, const EosParams& P,
                         const f2* lt, int& iters, int& st) {
  f2 lo = f2{(float)kTLo, 0.0f}, hi = f2{(float)kTHi, 0.0f};
  f2 Tn = f2_from(Told);
  if (f2_lt(Tn, lo)) Tn = lo;
  if (f2_gt(Tn, hi)) Tn = hi;
  bool conv = false, need_cp = true;
  float icp = 0.0f;
  const float tolf = (float)P.newton_tol;
  for (int it = 0; it < P.newton_max_iter; ++it) {
    ++iters;
    int s2 = 0;
    const PRPointDF q = pr_point_df<true>(m, Tn, p, need_cp, lt, s2);
    if (s2) {
      st |= s2;
      break;
    }
    const f2 f = f2_sub(f2_fma(q.h_dep, m.inv, h_ig_df(m, Tn)), h0);
    // chord steps with an FP32 reciprocal slope, as in solve_T
    if (need_cp) icp = __fdividef(1.0f, fmaf(q.cp_dep, m.inv.h, cp_ig_f(m, Tn.h)));
    if (__float_as_int(f.h) >= 0) hi = Tn; else lo = Tn;
    const f2 step = f2_mulf(f, -icp);
    f2 Tx = f2_add(Tn, step);
    const bool done = fabsf(step.h) <= tolf * Tn.h;
    need_cp = false;
    if (!done && !(f2_gt(Tx, lo) && f2_lt(Tx, hi))) {
      const f2 mid = f2_add(lo, hi);
      Tx = f2{0.5f * mid.h, 0.5f * mid.l};
      need_cp = true;
    }
    Tn = Tx;
    if (done) {
      conv = true;
      break;
    }
  }
  if (!conv && st == 0) st |= kCellNotConverged;
  if (!isfinite(Tn.h)) st |= kCellNonfinite;
  return Tn;
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

// Raw bits of a network-input element, for packing a row into 16-byte stores.
__device__ __forceinline__ uint32_t x_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t x_bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
__device__ __forceinline__ uint32_t x_bits(__nv_fp8_e4m3 v) { return v.__x; }

template <typename XT, int RW>
__device__ __forceinline__ void x_put(uint32_t (&w)[RW], int e, XT v) {
  constexpr int EPW = 4 / (int)sizeof(XT);
  w[e / EPW] |= x_bits(v) << (8 * (int)sizeof(XT) * (e % EPW));
}

// Y^lambda of a Box-Cox feature. Features rounded to BF16 or FP8 (8 or 4 significant bits)
// take the hardware approximations of log2 and exp2 (a relative error of a few 1e-7, far below
// that rounding); FP32 features take the library's accurate functions.
template <typename XT>
__device__ __forceinline__ float boxcox_pow(float y, float lam) {
  if constexpr (sizeof(XT) < 4) return __powf(y, lam);
  else return exp2f(lam * log2f(y));
}

// Species whose mass fractions a thread loads before using any (NM is a multiple of it).
constexpr int kLoadBatch = 16;

// a1-a5 for the valid rows of a batch.
template <int NM, typename XT>
__global__ void __launch_bounds__(kThreads, kPreBlocks) eos_pre_kernel(EosParams P, RowMap rows,
    const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,
    int64_t ldY, double* __restrict__ h0, double* __restrict__ Zout, XT* __restrict__ x,
    int64_t ldx, float x_scale, int32_t* __restrict__ status, double* __restrict__ rho) {
  extern __shared__ __align__(16) double sm[];
  const SharedConsts c = load_consts<true>(P, sm);
  f2* ycol = reinterpret_cast<f2*>(sm + consts_words(P)) + threadIdx.x;
  const int64_t nrow = valid_rows(rows);
  const int n = P.n, K0 = P.K0;
  const float lam = (float)P.lambda;
  const float ilam = 1.0f / lam;
  const float* mf = c.normf;        // in_mean
  const float* isf = c.normf + K0;  // 1 / in_std
  // Network-input rows go out as 16-byte stores from registers when the row pitch allows:
  // RW words hold the NM + 2 entries a row can have, EPC elements make one 16-byte chunk.
  constexpr int EPC = 16 / (int)sizeof(XT);
  constexpr int RW = ((NM + 2 + EPC - 1) / EPC) * 4;
  const int64_t row_bytes = ldx * (int64_t)sizeof(XT);
  const bool xvec = x && (row_bytes & 15) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  const int nch = (int)(row_bytes >> 4);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = row_cell(rows, r);
    const double Tc = T[cell], pc = p[cell];
    bool finite = d_finite(Tc) && d_finite(pc) && d_pos(pc) && d_pos(Tc);
    XT* xr = x ? x + r * ldx : nullptr;
    // the double-float column of Y (and, without packed rows, the a5 features), sixteen
    // species at a time with all their loads issued first: one memory latency per batch
#pragma unroll
    for (int k0 = 0; k0 < NM; k0 += kLoadBatch) {
      double yv[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) yv[u] = k0 + u < n ? Y[(k0 + u) * ldY + cell] : 0.0;
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int k = k0 + u;
        if (k < n) {
          const double yd = yv[u];
          finite = finite && d_finite(yd);
          ycol[k * kThreads] = f2_from(yd);
          if (xr && !xvec) {
            const float y = fmaxf(d_to_f_trunc(yd), 0.0f);
            const float bc = (y > 0.0f) ? (boxcox_pow<XT>(y, lam) - 1.0f) * ilam : -ilam;
            xr[2 + k] = to_x<XT>((bc - mf[2 + k]) * isf[2 + k], x_scale);
          }
        }
      }
    }
    if (xr && !xvec) {
      xr[0] = to_x<XT>(finite ? (d_to_f_trunc(Tc) - mf[0]) * isf[0] : 0.0f, x_scale);
      xr[1] = to_x<XT>(finite ? (d_to_f_trunc(pc) - mf[1]) * isf[1] : 0.0f, x_scale);
      if (!finite)
        for (int k = 0; k < n; ++k) xr[2 + k] = to_x<XT>(0.0f, x_scale);
      for (int k = K0; k < ldx; ++k) xr[k] = to_x<XT>(0.0f, x_scale);
    }
    int st = 0;
    double h = __longlong_as_double(0x7ff8000000000000LL), Z = h;
    if (finite) {
      MixDF m;
      mixture_df<kThreads>(ycol, n, c, m);
      const f2 Td = f2_from(Tc), pd = f2_from(pc);
      const PRPointDF q = pr_point_df<false>(m, Td, pd, false, c.lt2, st);
      Z = f2_to_int(q.Z);
      const f2 hd = f2_fma(q.h_dep, m.inv, h_ig_df(m, Td));
      h = f2_to_int(hd);
      if (!isfinite(hd.h)) st |= kCellNonfinite;
      // rho = p W_mix / (Z R T)
      if (rho) rho[r] = f2_to_int(f2_mul(pd, f2_rcp(f2_mul(f2_mul(m.inv, q.Z), f2_mul(Td, f2{kRh, kRl})))));
    } else {
      st = kCellNonfinite;
    }
    if (xvec) {
      // a5 features from the column (its high parts are Y rounded to FP32), packed into
      // registers and written as 16-byte stores: a row of RW words covers any n <= NM
      uint32_t w[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) w[q] = 0u;
      if (finite) {
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          if (k < n) {
            const float y = fmaxf(ycol[k * kThreads].h, 0.0f);
            const float bc = (y > 0.0f) ? (boxcox_pow<XT>(y, lam) - 1.0f) * ilam : -ilam;
            x_put(w, 2 + k, to_x<XT>((bc - mf[2 + k]) * isf[2 + k], x_scale));
          }
        }
      }
      x_put(w, 0, to_x<XT>(finite ? (d_to_f_trunc(Tc) - mf[0]) * isf[0] : 0.0f, x_scale));
      x_put(w, 1, to_x<XT>(finite ? (d_to_f_trunc(pc) - mf[1]) * isf[1] : 0.0f, x_scale));
      uint4* xo = reinterpret_cast<uint4*>(xr);
#pragma unroll
      for (int q = 0; q < RW / 4; ++q)
        if (q < nch) xo[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      for (int q = RW / 4; q < nch; ++q) xo[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (h0) h0[r] = h;
    if (Zout) Zout[r] = Z;
    if (status) status[r] = st;
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

// Y' = Y (1 + eps)^m for a growth (1 + eps)^m beyond e^80, in FP64. Out of line (rare).
__device__ __noinline__ f2 yprime_large(double y, float eps, int mpow) {
  return f2_from(y * ipow(1.0 + f_to_d(eps), mpow));
}

// Y' = Y (1 + eps)^m by log1p and expm1, for |eps| > 1/16 or 1/lambda > 16 (out of line: the
// common case takes the binomial sum).
__device__ __noinline__ f2 yprime_log(double y, float eps, float mf, int mpow) {
  const f2 yf = f2_from(y);
  const float lg = mf * log1pf(eps);
  return (lg < 80.0f) ? f2_add(yf, f2_mulf(yf, expm1f(lg))) : yprime_large(y, eps, mpow);
}

// Y' for Y below 1e-30 (or not positive): the closed form (Y^lambda + lambda du)^(1/lambda).
// Y^lambda (< 1e-30^lambda) in FP32, lambda du is FP32 already, the power in double-float: an
// absolute error of ~1e-7 Y^lambda in the base moves Y' by less than m 1e-7 Y^lambda base^(m-1).
__device__ __forceinline__ f2 yprime_small(double y, float lamf, float ldu, int mpow) {
  const float yf = d_to_f_trunc(y);
  const float base = ((yf > 0.0f) ? exp2f(lamf * log2f(yf)) : 0.0f) + ldu;
  if (!(base > 0.0f)) return f2{0.f, 0.f};
  f2 r = f2{1.0f, 0.0f}, b = f2{base, 0.0f};
  for (int m = mpow; m; m >>= 1) {
    if (m & 1) r = f2_mul(r, b);
    b = f2_mul(b, b);
  }
  return r;
}

// a8-a10 for the valid rows of a batch. Y' lives in this thread's shared-memory column (double-
// float) from the increment to the write-back, which happens only once the Newton solve for T
// has succeeded.
template <int NM>
__global__ void __launch_bounds__(kThreads, kPostBlocks) eos_post_kernel(EosParams P, RowMap rows,
    const float* __restrict__ O, int64_t ldo, const double* __restrict__ h0,
    double* __restrict__ T, const double* __restrict__ p, double* __restrict__ Y, int64_t ldY,
    const int32_t* __restrict__ pre_status, int32_t* __restrict__ cell_status, Source src) {
  extern __shared__ __align__(16) double sm[];
  const SharedConsts c = load_consts_post(P, sm);
  f2* ycol = reinterpret_cast<f2*>(sm + consts_words_post(P)) + threadIdx.x;
  constexpr int stride = kThreads;
  const int64_t nrow = valid_rows(rows);
  const int n = P.n, K0 = P.K0;
  const float* out_mean = c.normf + 2 * K0;
  const float* out_std = c.normf + 2 * K0 + n;
  const float lamf = (float)P.lambda;
  const int mpow = P.inv_lambda;
  const float mf = (float)P.inv_lambda;
  const bool binom = P.binom[0] != 0.0f;
  const bool ovec = (ldo & 3) == 0 && (reinterpret_cast<uintptr_t>(O) & 15) == 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = row_cell(rows, r);
    const double Told = T[cell], pc = p[cell], h0c = h0[r];
    int st = pre_status ? pre_status[r] : 0;  // flags eos_pre raised for this row
    bool finite = d_finite(Told) && d_finite(pc) && d_pos(pc) && d_finite(h0c);
    f2 S = {0.f, 0.f};
    const float* Or = O + r * ldo;
    // Y's column into this thread's column slots as FP64 bit patterns, sixteen loads in flight
    // at a time; each slot is overwritten by Y'_k below
#pragma unroll
    for (int k0 = 0; k0 < NM; k0 += kLoadBatch) {
      double yv[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) yv[u] = k0 + u < n ? Y[(k0 + u) * ldY + cell] : 0.0;
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u)
        if (k0 + u < n)
          ycol[(k0 + u) * stride] = f2{__int_as_float(__double2loint(yv[u])),
                                       __int_as_float(__double2hiint(yv[u]))};
    }
    // the row's outputs four at a time (one 16-byte load when the row pitch allows, the next
    // group's load issued before this group's arithmetic)
    float4 onext = ovec ? *reinterpret_cast<const float4*>(Or) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += 4) {
      float o4[4];
      if (ovec) {
        const float4 v = onext;
        if (k0 + 4 < n) onext = *reinterpret_cast<const float4*>(Or + k0 + 4);
        o4[0] = v.x;
        o4[1] = v.y;
        o4[2] = v.z;
        o4[3] = v.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) o4[q] = (k0 + q < n) ? Or[k0 + q] : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        if (k >= n) break;
        const f2 yraw = ycol[k * stride];
        const double y = __hiloint2double(__float_as_int(yraw.l), __float_as_int(yraw.h));
        finite = finite && d_finite(y);
        const float ldu = lamf * fmaf(out_std[k], o4[q], out_mean[k]);  // lambda du
        f2 yn = {0.f, 0.f};
        if (d_ge_pos(y, 1e-30)) {
          // Y' = (Y^lambda + lambda du)^(1/lambda) = Y (1 + eps)^m, eps = lambda du Y^-lambda;
          // the increment delta = (1 + eps)^m - 1 only scales Y' - Y, so FP32 suffices.
          const f2 yf = f2_from(y);
          const float eps = ldu * exp2f(-lamf * log2f(yf.h));
          if (binom && fabsf(eps) <= 0.0625f) {
            // delta = sum_{j=1..m} C(m, j) eps^j by Horner; for |eps| <= 1/16 the terms fall
            // off at least like (m eps)^j / j!, so the FP32 sum is good to a few ulp
            float b = 1.0f;
#pragma unroll 4
            for (int j = mpow - 1; j >= 1; --j) b = fmaf(b, eps, P.binom[j]);
            yn = f2_add(yf, f2_mulf(yf, b * eps));
          } else if (eps > -1.0f) {
            yn = yprime_log(y, eps, mf, mpow);
          }
        } else if (d_finite(y)) {
          yn = yprime_small(y, lamf, ldu, mpow);
        }
        ycol[k * stride] = yn;
        acc_add(S, yn);
      }
    }
    S = f2_fin(S);
    if (!finite || !(S.h > 0.0f) || !isfinite(S.h)) st |= kCellNonfinite;
    double Tn = Told;
    int iters = 0;
    if (st == 0) {
      const f2 iS = f2_rcp(S);
      for (int k = 0; k < n; ++k) ycol[k * stride] = f2_mul(ycol[k * stride], iS);
      MixDF m;
      mixture_post<kThreads>(ycol, n, c, m);
      Tn = f2_to_int(solve_T_df(m, f2_from(pc), f2_from(h0c), Told, P, c.lt2, iters, st));
    }
    if (st == 0 && src.omega) {
      // source terms rho (Y' - Y) / dt; Y' - Y in double-float
      const f2 sc = f2_from(src.rho[r] * src.inv_dt);
#pragma unroll 2
      for (int k = 0; k < n; ++k) {
        const f2 d = f2_add(ycol[k * stride], f2_from(-Y[k * ldY + cell]));
        src.omega[k * src.ldw + cell] = f2_to_int(f2_mul(d, sc));
      }
      if (src.T_new) src.T_new[cell] = Tn;
    } else if (st == 0) {
      T[cell] = Tn;
#pragma unroll 2
      for (int k = 0; k < n; ++k) Y[k * ldY + cell] = f2_to_int(ycol[k * stride]);
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
__global__ void __launch_bounds__(kPropThreads, kPropBlocks) props_kernel(EosParams P, int64_t ncell,
    const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,
    int64_t ldY, double* rho, double* h, double* cp, double* Zo) {
  extern __shared__ __align__(16) double sm[];
  const SharedConsts c = load_consts(P, sm);
  f2* ycol = reinterpret_cast<f2*>(sm + consts_words(P)) + threadIdx.x;
  const int n = P.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Tc = T[i], pc = p[i];
    for (int k = 0; k < n; ++k) ycol[k * kPropThreads] = f2_from(Y[k * ldY + i]);
    Mixture m;
    mixture<kPropThreads>(ycol, n, c, m);
    int st = 0;
    const PRPoint q = pr_point<false>(m, Tc, pc, cp != nullptr, c.lnt, st);
    if (rho) rho[i] = pc / (m.inv * q.Z * kR * Tc);
    if (h) h[i] = h_ig(m, Tc) + q.h_dep * m.inv;
    if (cp) cp[i] = cp_ig(m, Tc) + q.cp_dep * m.inv;
    if (Zo) Zo[i] = q.Z;
  }
}


// ---------------------------------------------------------------- transport properties
// Chung, Ajlan, Lee & Starling (1988), the high-pressure viscosity and thermal conductivity of
// a mixture from its pseudo-critical constants (Chung's mixing rules over the mole fractions)
// and its molar density, here the Peng-Robinson density; the ideal-gas Cv and the real-fluid c_p
// come from the same NASA-7 / Peng-Robinson state. The correlation is accurate to a few percent,
// so it is evaluated in FP32 (the PR state and the outer mixing sums stay FP64).

// Chung's coefficients E_i = a_i + b_i omega (viscosity) and B_i (conductivity), nonpolar,
// non-associating species
__constant__ float kChungE[10][2] = {
    {6.324f, 50.412f}, {1.210e-3f, -1.154e-3f}, {5.283f, 254.209f}, {6.623f, 38.096f},
    {19.745f, 7.630f}, {-1.900f, -12.537f}, {24.275f, 3.450f}, {0.7972f, 1.117f},
    {-0.2382f, 0.06770f}, {0.06863f, 0.3479f}};
__constant__ float kChungB[7][2] = {
    {2.4166f, 0.74824f}, {-0.50924f, -1.5094f}, {6.6107f, 5.6207f}, {14.543f, -8.9139f},
    {0.79274f, 0.82019f}, {-5.8634f, 12.801f}, {91.089f, 128.73f}};

// Chung's G2 with coefficients C1..C5 at reduced density y (G1 the Carnahan-Starling contact
// value); (1 - exp(-C4 y)) / y by expm1 so that dilute cells keep their digits
__device__ __forceinline__ float chung_g2(const float (&C)[10], float y, float G1) {
  const float t = y > 0.0f ? -expm1f(-C[3] * y) / y : C[3];
  return (C[0] * t + C[1] * G1 * __expf(C[4] * y) + C[2] * G1) / (C[0] * C[3] + C[1] + C[2]);
}

// mu (Pa s) and lambda (W/(m K)) of a pseudo-pure fluid (Tc K, Vc cm^3/mol, omega, M g/mol) at
// temperature T, molar density rho (mol/cm^3) and ideal-gas molar Cv (J/(mol K))
__device__ void chung(float T, float rho, float Tc, float Vc, float om, float M, float cv,
                      float& mu, float& lam) {
  const float Ts = 1.2593f * T / Tc;
  // collision integral of Neufeld, Janzen & Aziz (1972)
  const float Om = 1.16145f * __powf(Ts, -0.14874f) + 0.52487f * __expf(-0.77320f * Ts) +
                   2.16178f * __expf(-2.43787f * Ts);
  const float y = rho * Vc * (1.0f / 6.0f);
  const float omy = 1.0f - y;
  const float G1 = (1.0f - 0.5f * y) / (omy * omy * omy);
  float E[10], B[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) E[i] = kChungE[i][0] + kChungE[i][1] * om;
#pragma unroll
  for (int i = 0; i < 7; ++i) B[i] = kChungB[i][0] + kChungB[i][1] * om;
  const float G2 = chung_g2(E, y, G1);
  const float Fc = 1.0f - 0.2756f * om;
  const float c = cbrtf(Vc);
  const float vc23 = c * c;
  const float eta_k = sqrtf(Ts) / Om * Fc * (1.0f / G2 + E[5] * y);
  const float eta_p = E[6] * y * y * G2 * __expf(E[7] + E[8] / Ts + E[9] / (Ts * Ts));
  mu = (eta_k + eta_p) * 36.344f * sqrtf(M * Tc) / vc23 * 1e-7f;
  // thermal conductivity: dilute viscosity (Pa s), Cv correction Psi, dense terms
  const float Mk = M * 1e-3f;
  const float eta0 = 40.785f * Fc * sqrtf(M * T) / (vc23 * Om) * 1e-7f;
  const float a = cv * (float)kInvR - 1.5f;
  const float b = 0.7862f - 0.7109f * om + 1.3168f * om * om;
  const float Tr = T / Tc;
  const float Zp = 2.0f + 10.5f * Tr * Tr;
  const float psi = 1.0f + a * (0.215f + 0.28288f * a - 1.061f * b + 0.26665f * Zp) /
                               (0.6366f + b * Zp + 1.061f * a * b);
  const float H2 = chung_g2(B, y, G1);
  const float q = 3.586e-3f * sqrtf(Tc / Mk) / vc23;
  lam = 31.2f * eta0 * psi / Mk * (1.0f / H2 + B[5] * y) + q * B[6] * y * y * sqrtf(Tr) * H2;
}

template <int NM>
__global__ void __launch_bounds__(kPropThreads, kPropBlocks) transport_kernel(EosParams P, int64_t ncell,
    const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,
    int64_t ldY, double* mu, double* lam, double* alpha) {
  extern __shared__ __align__(16) double sm[];
  const SharedConsts c = load_consts(P, sm);
  f2* ycol = reinterpret_cast<f2*>(sm + consts_words(P)) + threadIdx.x;
  const int n = P.n, nn = P.n * P.n;
  constexpr int stride = kPropThreads;
  const float* __restrict__ tp = P.tpair;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Tk = T[i], pk = p[i];
    bool finite = d_finite(Tk) && d_finite(pk) && d_pos(pk) && d_pos(Tk);
    for (int k = 0; k < n; ++k) {
      const double yk = Y[k * ldY + i];
      finite = finite && d_finite(yk);
      ycol[k * stride] = f2_from(yk);
    }
    double m_out = __longlong_as_double(0x7ff8000000000000LL), l_out = m_out, a_out = m_out;
    if (finite) {
      Mixture m;
      mixture<kPropThreads>(ycol, n, c, m);
      int st = 0;
      const PRPoint q = pr_point<false>(m, Tk, pk, true, c.lnt, st);
      const double rho = pk / (m.inv * q.Z * kR * Tk);            // kg/m^3
      const double cpm = cp_ig(m, Tk) + q.cp_dep * m.inv;           // J/(kg K)
      const double Wm = 1.0 / m.inv;
      // mole fractions x_k = (Y_k / W_k) W_mix, kept in the column's high words
      const float Wmf = (float)Wm;
      for (int k = 0; k < n; ++k) ycol[k * stride].h = ycol[k * stride].h * c.spcw[k * kSpcStride].h * Wmf;
      // Chung's mixing sums, symmetric: sum_ij x_i x_j A_ij = sum_i x_i (A_ii x_i + 2 sum_{j>i} A_ij x_j)
      double S[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
      for (int a = 0; a < n; ++a) {
        const float xa = ycol[a * stride].h;
        float R4[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) R4[qq] = 0.5f * __ldg(tp + qq * nn + a * n + a) * xa;
        for (int b = a + 1; b < n; ++b) {
          const float xb = ycol[b * stride].h;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) R4[qq] = fmaf(__ldg(tp + qq * nn + a * n + b), xb, R4[qq]);
        }
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) S[qq] = fma(2.0 * (double)xa, (double)R4[qq], S[qq]);
      }
      const double eps_m = S[1] / S[0];
      const double sig2 = cbrt(S[0] * S[0]);                        // sigma_m^2
      const double Mr = S[3] / (eps_m * sig2);
      const float Tcm = (float)(1.2593 * eps_m);
      const float Vcm = (float)(S[0] / (0.809 * 0.809 * 0.809));
      const float omm = (float)(S[2] / S[0]);
      const float cv = (float)(cp_ig(m, Tk) * Wm - kR);             // ideal-gas molar Cv
      float muf, lamf;
      chung((float)Tk, (float)(rho * m.inv * 1e-6), Tcm, Vcm, omm, (float)(Mr * Mr), cv, muf, lamf);
      if (st == 0) {
        m_out = (double)muf;
        l_out = (double)lamf;
        a_out = (double)lamf / (rho * cpm);
      }
    }
    if (mu) mu[i] = m_out;
    if (lam) lam[i] = l_out;
    if (alpha) alpha[i] = a_out;
  }
}


// ---------------------------------------------------------------- Jacobian of the step

// dh/dY_k of the mass-specific real-fluid enthalpy at fixed T, p (FP64), for the composition in
// the per-thread column ycol (entry k at ycol[k * stride]). u_k = y_k sqrt(a_k), yr_k = y_k r_k,
// v = K u, w = K yr use the columns ucol, rcol, vcol, wcol. With sigma = sum y, W = 1/sigma:
//   a = W^2 u.Ku,  a' = -(W^2 / sqrt T) yr.Ku,  b = W sum y_k b_k,
//   da/dy_k = 2 W^2 sqrt(a_k) v_k - 2 W a,  da'/dy_k = -2 W a' - (W^2 / sqrt T)(r_k v_k + sqrt(a_k) w_k),
//   db/dy_k = W (b_k - b),  dZ from the implicit cubic, h = sum y_k h_k(T) + sigma h_dep,
//   dh/dY_k = (h_k(T) + h_dep + sigma dh_dep/dy_k) / W_k.
__device__ void h_grad(const EosParams& P, int n, int64_t ystride, const double* ycol, double T,
                       double p, int stride, double* ucol, double* rcol, int vstride,
                       double* vcol, double* wcol, double* out, int out_stride, int& st) {
  const double* spc = P.spc;
  const double* K = P.Kmat;
  const double t = sqrt(T);
  double sig = 0.0, bs = 0.0;
  for (int k = 0; k < n; ++k) {
    const double* q = spc + k * kSpcStride;
    const double y = ycol[k * ystride] * q[0];
    sig += y;
    bs += y * q[3];
    ucol[k * stride] = y * (q[1] - q[2] * t);
    rcol[k * stride] = y * q[2];
  }
  double G = 0.0, dGs = 0.0;
  for (int k = 0; k < n; ++k) {
    double v = 0.0, w = 0.0;
    for (int j = 0; j < n; ++j) {
      v = fma(K[k * n + j], ucol[j * stride], v);
      w = fma(K[k * n + j], rcol[j * stride], w);
    }
    vcol[k * vstride] = v;
    wcol[k * vstride] = w;
    G = fma(ucol[k * stride], v, G);
    dGs = fma(rcol[k * stride], v, dGs);
  }
  const double W = 1.0 / sig;
  const double a = W * W * G;
  const double da = -W * W * dGs / t;
  const double b = W * bs;
  const double RT = kR * T;
  const double A = a * p / (RT * RT);
  const double B = b * p / RT;
  const double Z = select_Z<false>(A, B, P.lntab, st);
  const double c1 = 1.0 + kSQ2, c2 = 1.0 - kSQ2;
  const double Zp = Z + c1 * B, Zm = Z + c2 * B;
  const double L = log(Zp / Zm);
  const double kb = 1.0 / (2.0 * kSQ2 * b);
  const double tda = T * da - a;
  const double hdep = RT * (Z - 1.0) + tda * kb * L;
  const double FZ = 3.0 * Z * Z - 2.0 * (1.0 - B) * Z + (A - 3.0 * B * B - 2.0 * B);
  const double FA = Z - B;
  const double FB = Z * Z - (6.0 * B + 2.0) * Z - (A - 2.0 * B - 3.0 * B * B);
  for (int k = 0; k < n; ++k) {
    const double* q = spc + k * kSpcStride;
    const double sak = q[1] - q[2] * t;
    const double vk = vcol[k * vstride], wk = wcol[k * vstride];
    const double dak = 2.0 * W * W * sak * vk - 2.0 * W * a;
    const double ddak = -2.0 * W * da - W * W * (q[2] * vk + sak * wk) / t;
    const double dbk = W * (q[3] - b);
    const double dAk = dak * p / (RT * RT);
    const double dBk = dbk * p / RT;
    const double dZk = -(FA * dAk + FB * dBk) / FZ;
    const double dLk = (dZk + c1 * dBk) / Zp - (dZk + c2 * dBk) / Zm;
    const double dkbk = -kb * dbk / b;
    const double dhdep = RT * dZk + (T * ddak - dak) * kb * L + tda * (dkbk * L + kb * dLk);
    const double hk = fma(fma(fma(fma(fma(q[9], T, q[8]), T, q[7]), T, q[6]), T, q[5]), T, q[4]);
    out[k * out_stride] = q[0] * (hk + hdep + sig * dhdep);
  }
}

// Input scales of the tangent directions (T, Y_1..Y_n): dx_0/dT = 1/std_T and
// dx_{2+j}/dY_j = BC'(Y_j) / std_{2+j}, BC'(y) = max(y, 1e-12)^(lambda - 1).
__global__ void jac_scale_kernel(EosParams P, int64_t ncell, const double* __restrict__ Y,
                                 int64_t ldY, const double* __restrict__ norm,
                                 float* __restrict__ sc) {
  const int ntan = P.n + 1, K0 = P.K0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncell * ntan;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / ntan;
    const int t = (int)(e % ntan);
    double v;
    if (t == 0) {
      v = norm[K0];
    } else {
      const double y = fmax(Y[(int64_t)(t - 1) * ldY + c], 1e-12);
      v = pow(y, P.lambda - 1.0) * norm[K0 + 1 + t];
    }
    sc[e] = (float)v;
  }
}

// Layer-1 tangents: dH1[c ntan + t, j] = sc[c, t] * W1[j, col(t)] * G1[c, j], col(0) = 0 (T),
// col(t) = t + 1 (Y_{t-1}); W1T is W1 transposed [K0 x N1]. A block takes kTanCells cells at a
// time; each thread holds eight G1 values of each of them, reads eight weights of a direction
// once (two 16-byte loads when N1 is a multiple of four) and writes the scaled products into
// the cells' tangent rows as 16-byte (BF16) or 32-byte (FP32) groups. Pitches ldg and ldh are
// multiples of eight elements.
constexpr int kTanCells = 4;
template <typename OT, typename GT>
__global__ void jac_tangent0_kernel(int64_t ncell, int ntan, int N1, const float* __restrict__ sc,
                                    const float* __restrict__ W1T, const GT* __restrict__ G1,
                                    int64_t ldg, OT* __restrict__ dH, int64_t ldh) {
  const int groups = (N1 + 7) / 8;
  const bool vec_w = (N1 & 3) == 0;
  for (int64_t c0 = (int64_t)blockIdx.x * kTanCells; c0 < ncell;
       c0 += (int64_t)gridDim.x * kTanCells) {
    const int nc = (int)(ncell - c0 < kTanCells ? ncell - c0 : kTanCells);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
      const int j0 = 8 * g;
      const int m = min(8, N1 - j0);
      float gv[kTanCells][8];
#pragma unroll
      for (int q = 0; q < kTanCells; ++q) {
        const GT* gp = G1 + (c0 + q) * ldg + j0;
#pragma unroll
        for (int e = 0; e < 8; ++e) gv[q][e] = (q < nc && e < m) ? (float)gp[e] : 0.0f;
      }
      for (int t = 0; t < ntan; ++t) {
        const int col = t == 0 ? 0 : t + 1;
        const float* wp = W1T + (int64_t)col * N1 + j0;
        float w[8];
        if (vec_w && m == 8) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(wp));
          const float4 b = __ldg(reinterpret_cast<const float4*>(wp) + 1);
          w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
          w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) w[e] = e < m ? __ldg(wp + e) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < kTanCells; ++q) {
          if (q >= nc) break;
          const int64_t row = (c0 + q) * ntan + t;
          const float s = sc[row];
          OT o[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) o[e] = (OT)(s * w[e] * gv[q][e]);
          OT* dst = dH + row * ldh + j0;
          if (m == 8) {
            // 8 elements at an offset that is a multiple of 8: 16 or 32 aligned bytes
            if constexpr (sizeof(OT) == 2) {
              *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(o);
            } else {
              reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(o)[0];
              reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(o)[1];
            }
          } else {
            for (int e = 0; e < m; ++e) dst[e] = o[e];
          }
        }
      }
    }
  }
}

// Jacobian of the step of every cell (treated as reacting): J[c][k][t] = d(Y'_k - Y_k)/dv_t and
// dTn[c][t] = dT'/dv_t, v = (T, Y_1..Y_n), from the network output O, its tangents dO
// ([c ntan + t][k] = dO_k/dv_t) and the implicit function h(T', p, Y') = h0(T, p, Y).
// Two kernels: jac_post_kernel, a thread per cell, takes the cell's equation-of-state part
// (Y', T' by Newton, dh/dY and c_p at both states) and leaves per cell in scr
// [dZ_k/du_k (n), Y'_k (n), dh/dY'_k (n), 1/S, c_p(T', Y'), two O(n) work columns (2n)] and
// its status in cst;
// jac_assemble_kernel, a warp per cell and a lane per direction t, forms the columns.
template <int NM>
__global__ void __launch_bounds__(kJacThreads) jac_post_kernel(EosParams P, int64_t ncell, int64_t cell0,
    const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,
    int64_t ldY, const float* __restrict__ O, int64_t ldo, const double* __restrict__ h0,
    double* __restrict__ dTn, double* __restrict__ scr, int32_t* __restrict__ cst) {
  extern __shared__ __align__(16) double sm[];
  const SharedConsts c = load_consts(P, sm);
  constexpr int stride = kJacThreads;
  // shared memory holds the per-thread columns read in O(n^2) loops (the double-float
  // composition of the mixing sums, the two weighted columns of h_grad); the O(n) ones live
  // in the cell's scratch row, which is also how they reach jac_assemble_kernel
  f2* ws = reinterpret_cast<f2*>(sm + consts_words(P)) + threadIdx.x;
  double* uc = sm + consts_words(P) + NM * stride + threadIdx.x;
  double* rc = uc + NM * stride;
  const int n = P.n, K0 = P.K0, ntan = n + 1;
  const float* out_mean = c.normf + 2 * K0;
  const float* out_std = c.normf + 2 * K0 + n;
  const float lamf = (float)P.lambda;
  const double lam = P.lambda;
  const int mpow = P.inv_lambda;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ncell;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = cell0 + r;
    const double Tc = T[cell], pc = p[cell], h0c = h0[r];
    // scratch row: dZ_k/du_k, Y'_k, dh/dY'_k, 1/S, c_p', then h_grad's v and w columns
    double* q = scr + r * (int64_t)(5 * n + 2);
    double* zlc = q;
    double* Ypc = q + n;
    double* hgc = q + 2 * n;
    double* vc = q + 3 * n + 2;
    double* wc = q + 4 * n + 2;
    double Yk[NM];
    bool finite = isfinite(Tc) && isfinite(pc) && pc > 0.0 && isfinite(h0c);
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      Yk[k] = (k < n) ? Y[k * ldY + cell] : 0.0;
      finite = finite && isfinite(Yk[k]);
    }
    int st = finite ? 0 : kCellNonfinite;
    double* dTc = dTn ? dTn + cell * (int64_t)ntan : nullptr;
    double cp1 = 1.0;
    if (st == 0) {
      // (T, Y): cp and dh/dY, parked in dTn (its entries are final after the column loop)
      Mixture m0;
      for (int k = 0; k < n; ++k) ws[k * stride] = f2_from(Yk[k]);
      mixture<kJacThreads>(ws, n, c, m0);
      const PRPoint q0 = pr_point<false>(m0, Tc, pc, true, c.lnt, st);
      if (dTc) {
        dTc[0] = cp_ig(m0, Tc) + q0.cp_dep * m0.inv;
        h_grad(P, n, ldY, Y + cell, Tc, pc, stride, uc, rc, 1, vc, wc, dTc + 1, 1, st);
      }
      // Y' and dZ_k/du_k = Z_k^(1 - lambda) = Z_k / (Y_k^lambda + lambda du_k)
      double S = 0.0;
      const float* Or = O + r * ldo;
      for (int k = 0; k < n; ++k) {
        const double y = Yk[k];
        const float ldu = lamf * fmaf(out_std[k], Or[k], out_mean[k]);
        const double base = ((y > 0.0) ? pow(y, lam) : 0.0) + (double)ldu;
        const double z = (base > 0.0) ? ipow(base, mpow) : 0.0;
        Ypc[k] = z;
        zlc[k] = (base > 0.0) ? z / base : 0.0;
        S += z;
      }
      if (!(S > 0.0)) st |= kCellNonfinite;
      if (st == 0) {
        const double iS = 1.0 / S;
        double Yn[NM];
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          Yn[k] = (k < n) ? Ypc[k] * iS : 0.0;
          if (k < n) Ypc[k] = Yn[k];
        }
        Mixture m1;
        for (int k = 0; k < n; ++k) ws[k * stride] = f2_from(Yn[k]);
        mixture<kJacThreads>(ws, n, c, m1);
        int iters = 0;
        const double Tn = solve_T<false>(m1, pc, h0c, Tc, P, c.lnt, iters, st);
        if (st == 0) {
          const PRPoint q1 = pr_point<false>(m1, Tn, pc, true, c.lnt, st);
          cp1 = cp_ig(m1, Tn) + q1.cp_dep * m1.inv;
          if (dTc) h_grad(P, n, 1, Ypc, Tn, pc, stride, uc, rc, 1, vc, wc, hgc, 1, st);
        }
        if (st == 0) {
          if (!dTc)
            for (int k = 0; k < n; ++k) hgc[k] = 0.0;
          q[3 * n] = iS;
          q[3 * n + 1] = cp1;
        }
      }
    }
    cst[r] = st;
  }
}


// Columns of the Jacobian from jac_post_kernel's per-cell results: a warp per cell, lane t takes
// direction t (T, then Y_1..Y_n), in the arithmetic and order of the per-cell formulas:
// ju_k = out_std_k dO_k/dv_t + [t = k + 1] BC'(Y_k), jy_k = (dZ_k/du_k ju_k - Y'_k sum_j dZ_j/du_j
// ju_j) / S, J[k][t] = jy_k - [t = k + 1], dT'/dv_t = (dh/dv_t - sum_k dh/dY'_k jy_k) / c_p.
// Cells whose status is not 0 get NaN.
template <int NM>
__global__ void __launch_bounds__(256) jac_assemble_kernel(EosParams P, int64_t ncell,
    int64_t cell0, const double* __restrict__ Y, int64_t ldY, const float* __restrict__ dO,
    int64_t lddo, const double* __restrict__ scr, const int32_t* __restrict__ cst,
    float* __restrict__ J, double* __restrict__ dTn) {
  const int n = P.n, K0 = P.K0, ntan = n + 1;
  // the FP32 output spreads as FP64 (exact), once per block, and the FP32 -> FP64 conversions
  // of dO on the integer pipes
  __shared__ double sdd[NM];
  for (int k = threadIdx.x; k < n; k += blockDim.x) sdd[k] = f_to_d((float)P.norm[2 * K0 + n + k]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const double lam = P.lambda;
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < ncell;
       r += warps) {
    const int64_t cell = cell0 + r;
    float* Jc = J + cell * (int64_t)n * ntan;
    double* dTc = dTn ? dTn + cell * (int64_t)ntan : nullptr;
    if (cst[r] != 0) {
      const float nanf = __int_as_float(0x7fc00000);
      for (int e = lane; e < n * ntan; e += 32) Jc[e] = nanf;
      if (dTc)
        for (int t = lane; t < ntan; t += 32) dTc[t] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    const double* q = scr + r * (int64_t)(5 * n + 2);
    const double* zl = q;
    const double* Yp = q + n;
    const double* hg = q + 2 * n;
    const double iS = q[3 * n], cp1 = q[3 * n + 1];
    for (int t = lane; t < ntan; t += 32) {
      const float* dOr = dO + (r * ntan + t) * lddo;
      double bcp = 0.0;
      if (t > 0) bcp = pow(fmax(Y[(int64_t)(t - 1) * ldY + cell], 1e-12), lam - 1.0);
      double sumjz = 0.0;
#pragma unroll 4
      for (int k = 0; k < n; ++k) {
        const double ju = sdd[k] * f_to_d(dOr[k]) + ((t == k + 1) ? bcp : 0.0);
        sumjz += zl[k] * ju;
      }
      double acc = 0.0;
#pragma unroll 4
      for (int k = 0; k < n; ++k) {
        const double ju = sdd[k] * f_to_d(dOr[k]) + ((t == k + 1) ? bcp : 0.0);
        const double jy = (zl[k] * ju - Yp[k] * sumjz) * iS;
        Jc[k * ntan + t] = (float)(jy - ((t == k + 1) ? 1.0 : 0.0));
        if (dTc) acc = fma(hg[k], jy, acc);
      }
      if (dTc) dTc[t] = (dTc[t] - acc) / cp1;
    }
  }
}

// Dynamic shared memory of an EoS block of `threads` threads: constants and the per-thread
// double-float column of mass fractions (n words per thread).
size_t eos_smem(const EosParams& P, int threads = kThreads) {
  return sizeof(double) * ((size_t)consts_words(P) + (size_t)P.n * threads);
}

size_t eos_smem_post(const EosParams& P) {
  return sizeof(double) * ((size_t)consts_words_post(P) + (size_t)P.n * kThreads);
}

// Opts a kernel into more than 48 KB of dynamic shared memory, once per device.
template <auto Kern>
cudaError_t smem_optin() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!done[dev]) {
    e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    // these kernels are bound by their shared-memory columns: ask for the largest carveout
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(Kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

// Grid of a grid-stride kernel: one wave of the blocks that fit on the device at once (the
// occupancy of Kern at kThreads threads and smem bytes), fewer when there is less work.
template <auto Kern>
int grid_resident(int64_t nmax, size_t smem) {
  static int per_sm[64] = {0};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int nb = (dev >= 0 && dev < 64) ? per_sm[dev] : 0;
  if (nb <= 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, Kern, kThreads, smem) != cudaSuccess ||
        nb <= 0) {
      cudaGetLastError();
      nb = 4;
    }
    if (dev >= 0 && dev < 64) per_sm[dev] = nb;
  }
  int64_t need = (nmax + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sms * nb;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

int grid_for(int64_t nmax, int threads = kThreads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t need = (nmax + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 8;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

template <int NM, typename XT>
cudaError_t pre_launch(const EosParams& P, const RowMap& rows, const double* T, const double* p,
                       const double* Y, int64_t ldY, double* h0, double* Z, XT* x, int64_t ldx,
                       float xs, int32_t* status, cudaStream_t st, double* rho) {
  cudaError_t e = smem_optin<eos_pre_kernel<NM, XT>>();
  if (e != cudaSuccess) return e;
  eos_pre_kernel<NM, XT><<<grid_resident<eos_pre_kernel<NM, XT>>(rows.nmax, eos_smem(P)), kThreads,
                           eos_smem(P), st>>>(
      P, rows, T, p, Y, ldY, h0, Z, x, ldx, xs, status, rho);
  return cudaGetLastError();
}

template <int NM>
cudaError_t pre_nm(const EosParams& P, const RowMap& rows, const double* T, const double* p,
                   const double* Y, int64_t ldY, double* h0, double* Z, void* x, int xkind,
                   int64_t ldx, float xs, int32_t* status, cudaStream_t st, double* rho) {
  switch (xkind) {
    case kXBF16:
      return pre_launch<NM>(P, rows, T, p, Y, ldY, h0, Z, (__nv_bfloat16*)x, ldx, xs, status, st, rho);
    case kXFP8:
      return pre_launch<NM>(P, rows, T, p, Y, ldY, h0, Z, (__nv_fp8_e4m3*)x, ldx, xs, status, st, rho);
    default:
      return pre_launch<NM>(P, rows, T, p, Y, ldY, h0, Z, (float*)x, ldx, xs, status, st, rho);
  }
}

template <int NM>
cudaError_t post_nm(const EosParams& P, const RowMap& rows, const float* O, int64_t ldo,
                    const double* h0, double* T, const double* p, double* Y, int64_t ldY,
                    const int32_t* pre_status, int32_t* cell_status, cudaStream_t st,
                    const Source& src) {
  cudaError_t e = smem_optin<eos_post_kernel<NM>>();
  if (e != cudaSuccess) return e;
  eos_post_kernel<NM><<<grid_resident<eos_post_kernel<NM>>(rows.nmax, eos_smem_post(P)), kThreads,
                        eos_smem_post(P), st>>>(
      P, rows, O, ldo, h0, T, p, Y, ldY, pre_status, cell_status, src);
  return cudaGetLastError();
}

template <int NM>
cudaError_t transport_nm(const EosParams& P, int64_t n, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* mu, double* lam, double* alpha,
                         cudaStream_t st) {
  cudaError_t e = smem_optin<transport_kernel<NM>>();
  if (e != cudaSuccess) return e;
  transport_kernel<NM><<<grid_for(n, kPropThreads), kPropThreads, eos_smem(P, kPropThreads), st>>>(
      P, n, T, p, Y, ldY, mu, lam, alpha);
  return cudaGetLastError();
}

template <int NM>
cudaError_t props_nm(const EosParams& P, int64_t n, const double* T, const double* p,
                     const double* Y, int64_t ldY, double* rho, double* h, double* cp, double* Z,
                     cudaStream_t st) {
  cudaError_t e = smem_optin<props_kernel<NM>>();
  if (e != cudaSuccess) return e;
  props_kernel<NM><<<grid_for(n, kPropThreads), kPropThreads, eos_smem(P, kPropThreads), st>>>(
      P, n, T, p, Y, ldY, rho, h, cp, Z);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eos_pre(const EosParams& P, const RowMap& rows, const double* T,
                           const double* p, const double* Y, int64_t ldY, double* h0,
                           double* Z, void* x, int xkind, int64_t ldx, float x_scale,
                           int32_t* status, cudaStream_t st, double* rho) {
  if (rows.nmax <= 0) return cudaSuccess;
  if (P.n <= 16)
    return pre_nm<16>(P, rows, T, p, Y, ldY, h0, Z, x, xkind, ldx, x_scale, status, st, rho);
  return pre_nm<32>(P, rows, T, p, Y, ldY, h0, Z, x, xkind, ldx, x_scale, status, st, rho);
}

template <int NM>
cudaError_t prepare_nm(int xkind) {
  cudaError_t e = xkind == kXBF16  ? smem_optin<eos_pre_kernel<NM, __nv_bfloat16>>()
                  : xkind == kXFP8 ? smem_optin<eos_pre_kernel<NM, __nv_fp8_e4m3>>()
                                   : smem_optin<eos_pre_kernel<NM, float>>();
  if (e == cudaSuccess) e = smem_optin<eos_pre_kernel<NM, float>>();  // stage entry point
  if (e == cudaSuccess) e = smem_optin<eos_post_kernel<NM>>();
  if (e == cudaSuccess) e = smem_optin<props_kernel<NM>>();
  if (e == cudaSuccess) e = smem_optin<transport_kernel<NM>>();
  return e;
}

cudaError_t prepare_eos(const EosParams& P, int xkind) {
  cudaError_t e = P.n <= 16 ? prepare_nm<16>(xkind) : prepare_nm<32>(xkind);
  if (e == cudaSuccess) e = P.n <= 16 ? smem_optin<jac_post_kernel<16>>() : smem_optin<jac_post_kernel<32>>();
  return e;
}

cudaError_t launch_jac_scale(const EosParams& P, int64_t ncell, const double* Y, int64_t ldY,
                             float* sc, cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  jac_scale_kernel<<<grid_for(ncell * (P.n + 1)), kThreads, 0, st>>>(P, ncell, Y, ldY, P.norm, sc);
  return cudaGetLastError();
}

cudaError_t launch_jac_tangent0(int64_t ncell, int ntan, int N1, const float* sc, const float* W1T,
                                const void* G1, int64_t ldg, bool bf16, void* dH, int64_t ldh,
                                cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  if ((ldg & 7) || (ldh & 7)) return cudaErrorInvalidValue;
  // kTanCells cells per block at a time, a thread per group of eight columns
  const int groups = (N1 + 7) / 8;
  const int threads = std::min(256, (groups + 31) / 32 * 32);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int g = (int)std::min<int64_t>((ncell + kTanCells - 1) / kTanCells,
                                       (int64_t)sms * (2048 / threads));
  if (bf16)
    jac_tangent0_kernel<__nv_bfloat16, __nv_bfloat16><<<g, threads, 0, st>>>(
        ncell, ntan, N1, sc, W1T, (const __nv_bfloat16*)G1, ldg, (__nv_bfloat16*)dH, ldh);
  else
    jac_tangent0_kernel<float, float><<<g, threads, 0, st>>>(ncell, ntan, N1, sc, W1T,
                                                             (const float*)G1, ldg, (float*)dH, ldh);
  return cudaGetLastError();
}

cudaError_t launch_jac_post(const EosParams& P, int64_t ncell, int64_t cell0, const double* T,
                            const double* p, const double* Y, int64_t ldY, const float* O,
                            int64_t ldo, const float* dO, int64_t lddo, const double* h0, float* J,
                            double* dTn, double* scr, int32_t* cst, cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  constexpr int kJT = kJacThreads;
  const int64_t blocks = (ncell + kJT - 1) / kJT;
  const int g = (int)(blocks < 4096 ? blocks : 4096);
  if (P.n <= 16) {
    const size_t smem = sizeof(double) * ((size_t)consts_words(P) + (size_t)(3 * 16) * kJT);
    jac_post_kernel<16><<<g, kJT, smem, st>>>(P, ncell, cell0, T, p, Y, ldY, O, ldo, h0, dTn, scr, cst);
  } else {
    const size_t smem = sizeof(double) * ((size_t)consts_words(P) + (size_t)(3 * 32) * kJT);
    jac_post_kernel<32><<<g, kJT, smem, st>>>(P, ncell, cell0, T, p, Y, ldY, O, ldo, h0, dTn, scr, cst);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ablocks = (ncell + 7) / 8;   // eight cells (warps) per block
  const unsigned ag = (unsigned)std::min<int64_t>(ablocks, 1 << 20);
  if (P.n <= 16)
    jac_assemble_kernel<16><<<ag, 256, 0, st>>>(P, ncell, cell0, Y, ldY, dO, lddo, scr, cst, J, dTn);
  else
    jac_assemble_kernel<32><<<ag, 256, 0, st>>>(P, ncell, cell0, Y, ldY, dO, lddo, scr, cst, J, dTn);
  return cudaGetLastError();
}

cudaError_t launch_eos_post(const EosParams& P, const RowMap& rows, const float* O, int64_t ldo,
                            const double* h0, double* T, const double* p, double* Y,
                            int64_t ldY, const int32_t* pre_status, int32_t* cell_status,
                            cudaStream_t st, const Source* src) {
  if (rows.nmax <= 0) return cudaSuccess;
  const Source s = src ? *src : Source{nullptr, 0, nullptr, 0.0, nullptr};
  if (P.n <= 16)
    return post_nm<16>(P, rows, O, ldo, h0, T, p, Y, ldY, pre_status, cell_status, st, s);
  return post_nm<32>(P, rows, O, ldo, h0, T, p, Y, ldY, pre_status, cell_status, st, s);
}

cudaError_t launch_props(const EosParams& P, int64_t n, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* rho, double* h, double* cp,
                         double* Z, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (P.n <= 16) return props_nm<16>(P, n, T, p, Y, ldY, rho, h, cp, Z, st);
  return props_nm<32>(P, n, T, p, Y, ldY, rho, h, cp, Z, st);
}

cudaError_t launch_transport(const EosParams& P, int64_t n, const double* T, const double* p,
                             const double* Y, int64_t ldY, double* mu, double* lam, double* alpha,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (P.n <= 16) return transport_nm<16>(P, n, T, p, Y, ldY, mu, lam, alpha, st);
  return transport_nm<32>(P, n, T, p, Y, ldY, mu, lam, alpha, st);
}

// Cells the step's eos_pre launch covers in one pass of its resident blocks (SMs x blocks per
// SM x threads); 0 if the occupancy query fails.
int64_t eos_wave_cells(const EosParams& P, int xkind) {
  const size_t smem = eos_smem(P);
  auto wave = [&](auto kern) -> int64_t {
    int nb = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return (int64_t)sms * nb * kThreads;
  };
  if (P.n <= 16)
    return xkind == kXBF16 ? wave(eos_pre_kernel<16, __nv_bfloat16>)
           : xkind == kXFP8 ? wave(eos_pre_kernel<16, __nv_fp8_e4m3>) : wave(eos_pre_kernel<16, float>);
  return xkind == kXBF16 ? wave(eos_pre_kernel<32, __nv_bfloat16>)
         : xkind == kXFP8 ? wave(eos_pre_kernel<32, __nv_fp8_e4m3>) : wave(eos_pre_kernel<32, float>);
}

}  // namespace dfgb
