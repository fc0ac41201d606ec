// Internal declarations of libdfgb: device-side parameter blocks and host launchers.
// Not part of the public ABI (include/df.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <stdint.h>

namespace dfgb {

constexpr double kR = 8.31446261815324;   // J/(mol K)
constexpr int kMaxSpecies = 32;           // register-resident species arrays
constexpr int kSpcStride = 10;            // doubles per species in EosParams::spc

// Error bits a kernel ORs into the state's device error word.
constexpr int kErrTimeout = 1;            // a bounded wait gave up

// Which rows of a batch a kernel handles. Row r of the batch is reacting-list position
// row0 + r, i.e. cell idx[row0 + r] (cell row0 + r when idx is NULL). The number of valid
// rows is min(nmax, *count - row0) when count is given, else nmax.
struct RowMap {
  const int32_t* idx;
  const int64_t* count;
  int64_t row0;
  int64_t nmax;
};

__host__ __device__ inline int64_t clamp_rows(int64_t c, int64_t row0, int64_t nmax) {
  int64_t v = c - row0;
  return v < 0 ? 0 : (v > nmax ? nmax : v);
}

#ifdef __CUDACC__
__device__ inline int64_t valid_rows(const RowMap& m) {
  return m.count ? clamp_rows(*m.count, m.row0, m.nmax) : m.nmax;
}
__device__ inline int64_t row_cell(const RowMap& m, int64_t r) {
  return m.idx ? (int64_t)m.idx[m.row0 + r] : m.row0 + r;
}
#endif

// Constants of the equation-of-state steps, in device memory.
//   spc[k * kSpcStride + j]: j = 0 1/W_k, 1 s_k, 2 r_k, 3 b_k, 4..9 enthalpy coefficients
//   hc_0..hc_5 with h_k(T) = hc_0 + hc_1 T + hc_2 T^2 + ... + hc_5 T^5 (J/mol), where
//   sqrt(a_k(T)) = s_k - r_k sqrt(T) (Peng-Robinson alpha function expanded in sqrt(T)).
//   Kmat[i * n + j] = 1 - k_ij.
//   norm: in_mean[K0], in_inv_std[K0], out_mean[n], out_std[n].
struct EosParams {
  int n;                 // species
  int K0;                // n + 2 network inputs
  int inv_lambda;        // Box-Cox 1/lambda (integer)
  // binomial coefficients C(m, k), k = 0..m, of m = inv_lambda when m <= 16 (exact in FP32),
  // for (1 + eps)^m - 1 by its expansion; binom[0] = 0 marks m > 16
  float binom[17];
  double lambda;
  double T_react;
  double newton_tol;
  int newton_max_iter;
  const double* spc;
  const double* Kmat;
  const double* norm;
  // Double-float (hi, lo) tables of the mixing sums, with 1/W folded in:
  //   spcw2[k][j]: j = 0 1/W_k, 1 s_k/W_k, 2 r_k/W_k, 3 b_k/W_k, 4..9 hc_j/W_k;
  //   K4 = (Ks hi, Ks lo, Kr hi, Kr lo) for the pairs j > i, row by row (row i from entry
  //   i n - i (i + 1) / 2), with Ks_ij = (1 - k_ij) s_j / W_j, Kr_ij = (1 - k_ij) r_j / W_j;
  //   kcol[j] = max_i |Ks_ij|, kcol[n + j] = max_i |Kr_ij| (rounded up by 2^-10: bounds for the
  //   pair sums' accumulator offsets).
  const float* spcw2;    // [n * kSpcStride * 2]
  const float* K4;       // [2 n (n - 1)] (+ 4 floats of padding)
  const float* kcol;     // [2 * n]
  // FP32 pair corrections of the T-from-h solve, (k_ij s_j / W_j, k_ij r_j / W_j) for the
  // pairs j > i, row by row (row i from pair i n - i (i + 1) / 2)
  const float* kf2;      // [n (n - 1)] (+ 2 floats of padding)
  // max_k |column j of the species table over W| (the hi parts of spcw2, rounded up): with the
  // sum of |Y| they bound the T-from-h solve's species sums
  float spcmax[kSpcStride];
  // natural-log table: ln(c_j) for j < 128, then 1 / c_j, c_j = 1 + (j + 1/2) / 128
  const double* lntab;   // [256]
  const float* lntab2;   // [512] the same table as double-float (hi, lo) pairs
  // Chung's mixing rules (transport properties): per species tsp[k] = (Tc, Vc [cm^3/mol],
  // omega, M [g/mol]); per pair tpair[q][i][j], q = 0 sigma_ij^3, 1 eps_ij sigma_ij^3,
  // 2 omega_ij sigma_ij^3, 3 eps_ij sigma_ij^2 M_ij^(1/2) (sigma in Angstrom, eps/k in K)
  const double* tsp;     // [n * 4]
  const float* tpair;    // [4 * n * n]
  int* err;              // device error word
  int64_t* flagged;      // device count of cells flagged by eos_post (may be NULL)
  int64_t* newton_iters; // device sum of Newton iterations (may be NULL)
};

enum XKind { kXF32 = 0, kXBF16 = 1, kXFP8 = 2 };

// ---- launchers (eos.cu) ----
// status (row-indexed, may be NULL) receives the per-row flags.
// rho (row-indexed, may be NULL) receives the real-fluid density.
int64_t eos_wave_cells(const EosParams& P, int xkind);
cudaError_t launch_eos_pre(const EosParams& P, const RowMap& rows, const double* T,
                           const double* p, const double* Y, int64_t ldY, double* h0,
                           double* Z, void* x, int xkind, int64_t ldx, float x_scale,
                           int32_t* status, cudaStream_t st, double* rho = nullptr);
// pre_status (row-indexed, may be NULL) carries eos_pre's flags; cell_status (cell-indexed,
// may be NULL) receives the final flags. With a Source (omega non-NULL) T and Y are left alone:
// cell columns of omega [n x ldw] receive rho (Y' - Y) / dt and T_new (may be NULL) T'.
struct Source {
  double* omega;
  int64_t ldw;
  const double* rho;     // row-indexed, from eos_pre
  double inv_dt;
  double* T_new;
};
cudaError_t launch_eos_post(const EosParams& P, const RowMap& rows, const float* O, int64_t ldo,
                            const double* h0, double* T, const double* p, double* Y,
                            int64_t ldY, const int32_t* pre_status, int32_t* cell_status,
                            cudaStream_t st, const Source* src = nullptr);
// Transport properties (Chung et al. 1988 at the Peng-Robinson density); outputs may be NULL.
cudaError_t launch_transport(const EosParams& P, int64_t n, const double* T, const double* p,
                             const double* Y, int64_t ldY, double* mu, double* lam, double* alpha,
                             cudaStream_t st);
cudaError_t launch_props(const EosParams& P, int64_t n, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* rho, double* h, double* cp,
                         double* Z, cudaStream_t st);
// Sets, on the current device, the kernel attributes the EoS launches of this configuration
// need (done once per device; later launches and graph captures then set none).
cudaError_t prepare_eos(const EosParams& P, int xkind);
// Jacobian pieces: input scales sc [ncell x (n+1)], layer-1 tangents, post-processing.
cudaError_t launch_jac_scale(const EosParams& P, int64_t ncell, const double* Y, int64_t ldY,
                             float* sc, cudaStream_t st);
cudaError_t launch_jac_tangent0(int64_t ncell, int ntan, int N1, const float* sc, const float* W1T,
                                const void* G1, int64_t ldg, bool bf16, void* dH, int64_t ldh,
                                cudaStream_t st);
// scr: ncell x (5n + 2) doubles, cst: ncell int32 (per-cell results between the two kernels).
cudaError_t launch_jac_post(const EosParams& P, int64_t ncell, int64_t cell0, const double* T,
                            const double* p, const double* Y, int64_t ldY, const float* O,
                            int64_t ldo, const float* dO, int64_t lddo, const double* h0, float* J,
                            double* dTn, double* scr, int32_t* cst, cudaStream_t st);

// ---- launcher (step_vjp.cu) ----
// Per cell of a batch: g_v = gT dT'/dv + sum_k gY_k dY'_k/dv from the batch's Jacobian J
// [ncell][n][n+1] FP32 and dTn [ncell][n+1] FP64 (cell-local); non-reacting cells copy the
// cotangents. gY / oY are species-major with leading dimensions ldg / ldo.
cudaError_t launch_step_vjp(int n, int64_t ncell, double T_react, const double* T, const float* J,
                            const double* dTn, const double* gT, const double* gY, int64_t ldg,
                            double* oT, double* oY, int64_t ldo, cudaStream_t st);

// ---- launchers (train.cu) ----
// Ohat [B x ldh] FP32 (zero pads) = (BC(Yt) - BC(Y) - out_mean) / out_std of cells 0..B-1.
cudaError_t launch_train_targets(const EosParams& P, int64_t B, const double* Y, const double* Yt,
                                 int64_t ldY, float* Oh, int64_t ldh, cudaStream_t st);
// Reductions of the training kernels are summed in a fixed order through a scratch buffer
// of kTrainScratchFloats (>= kColsumChunks x widest layer for column sums), so losses and
// gradients are reproducible run to run.
constexpr int kTrainScratchFloats = 4096;
constexpr int kColsumChunks = 64;
// dO [B x ldd] (BF16 or FP32, zero pads) = 2 (O - Ohat) / B; *loss = sum (O - Ohat)^2 / B.
// Property network (propnet.cu): input rows from (h, p, Y), normalised targets, outputs.
cudaError_t launch_prop_inputs(const double* norm, int n, double lambda, int64_t rows,
                               const double* h, const double* p, const double* Y, int64_t ldY,
                               void* x, int64_t ldx, int xkind, int num_sms, cudaStream_t st);
cudaError_t launch_prop_targets(const double* norm, int K0, int m, int64_t rows, const double* t,
                                int64_t ldt, float* Oh, int64_t ldo, int num_sms, cudaStream_t st);
cudaError_t launch_prop_outputs(const double* norm, int K0, int m, int64_t rows, const float* O,
                                int64_t ldo, double* out, int64_t ldout, int num_sms,
                                cudaStream_t st);
cudaError_t launch_loss_grad(int64_t B, int n, const float* O, int64_t ldo, const float* Oh,
                             int64_t ldh, void* dO, int64_t ldd, bool bf16, float* loss,
                             float* scratch, cudaStream_t st);
// out [C x ldo] = in^T for in [R x ldi]; rows R..Rpad-1 of the transpose are zero. Rpad a
// multiple of 64, ldi and ldo even. With colsum (and scratch of scratch_floats >= C floats),
// also colsum[c] = sum_r in[r][c], FP32, in a fixed order.
cudaError_t launch_transpose(int64_t R, int64_t C, const void* in, int64_t ldi, void* out,
                             int64_t ldo, int64_t Rpad, bool bf16, int num_sms, cudaStream_t st,
                             float* colsum = nullptr, float* scratch = nullptr,
                             int64_t scratch_floats = 0);
// out[i] = sum_{s < splits} part[s * stride + i] (fixed order), i < count.
cudaError_t launch_sum_splits(int splits, int64_t count, int64_t stride, const float* part,
                              float* out, cudaStream_t st);
cudaError_t launch_adam(int64_t count, float* w, float* m, float* v, const float* g, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t launch_publish(int N, int K, const float* Wm, int64_t ldm, float* W32, int64_t ld32,
                           void* Wb, int64_t ldb, void* WT, int64_t ldt, bool WT_bf16,
                           cudaStream_t st);

// ---- launchers (compact.cu) ----
constexpr int64_t kCompactChunk = 4096;   // cells per block of the compaction kernels
// Stable list of cells with T > T_react. Needs scratch of compact_scratch_words(n) int64.
int64_t compact_scratch_words(int64_t n);
cudaError_t launch_compact(int64_t n, double T_react, const double* T, int32_t* idx,
                           int64_t* count, int32_t* status, int64_t* scratch, cudaStream_t st);

// ---- launchers (mlp_simt.cu) ----
// C[r, c] = act(sum_k A[r, k] W[c, k] + bias[c]) for valid rows r < rows(map), c < N.
// A is [rows x lda] FP32, W is [N x ldw] FP32 with K a multiple of 8 (zero padded).
// mode 1 also writes G = GELU'(z) [rows x ldg]; mode 2 computes C = (A W^T) * G[row / ntan].
cudaError_t launch_sgemm_bias_act(const RowMap& rows, int N, int K, const float* A, int64_t lda,
                                  const float* W, int64_t ldw, const float* bias, float* C,
                                  int64_t ldc, bool gelu, int num_sms, cudaStream_t st,
                                  int mode = 0, float* G = nullptr, int64_t ldg = 0, int ntan = 1,
                                  const float4* gelu_table = nullptr);

// The tabulated GELU (DF_GELU_TABLE): 601 nodes x_i = -3 + 0.01 i, each {GELU, GELU',
// GELU''/2, 0} of the tanh form in FP32; 0 below -3, x above 3.
constexpr int kGeluTableNodes = 601;
__host__ __device__ inline float gelu_from_table(float x, const float4* tab) {
#ifdef __CUDA_ARCH__
  if (x <= -3.0f) return 0.0f;
  if (x >= 3.0f) return x;
  const float tt = (x + 3.0f) * 100.0f;
  const int i = min((int)tt, kGeluTableNodes - 2);
  const float d = x - fmaf(0.01f, (float)i, -3.0f);
  const float4 c = __ldg(tab + i);
  return fmaf(d, fmaf(d, c.z, c.y), c.x);
#else
  (void)x; (void)tab;
  return 0.0f;
#endif
}

// ---- tcgen05 GEMM (mlp_tc.cu) ----
struct TcLayer {
  CUtensorMap tmA;       // activations in, box {64 (K), 128 (M)}
  CUtensorMap tmB;       // weights [N x K], box {64, BN}
  CUtensorMap tmO;       // output [rows x ldo], box {32, 32}, swizzled (tc_encode_out)
  CUtensorMap tmG;       // GELU'(z) [rows x ldg] BF16 of kModeStoreG, same boxes
  int N, K, BN;
  const float* bias;     // [N]
  const float* col_scale;// [N] per-output-channel dequant scale (FP8) or NULL
  void* out;             // [rows x ldo] BF16 / FP8 activations, or FP32 for the last layer
  int64_t ldo;
  int out_kind;          // XKind; kXF32 for the last layer
  bool gelu;
  float out_scale;       // multiply before quantising the output (FP8 activations)
  int elem_bytes;        // 2 (BF16) or 1 (FP8)
  int mode;              // 0 plain, 1 also store GELU'(z) to gbuf, 2 scale rows by gbuf
  void* gbuf;            // BF16 [cells x ldg] GELU'(z) of the forward pass
  int64_t ldg;
  int ntan;              // tangent rows per cell (mode 2)
  const float4* gtab = nullptr;  // tabulated GELU (DF_GELU_TABLE) or NULL for the tanh form
  int ksplit = 1;        // split-K (plain mode): split s covers k-blocks [s kbs, (s+1) kbs) and
  int64_t split_rows = 0;  // stores its partial product at output rows + s * split_rows
  bool pair = false;     // computed by CTA pairs (cta_group::2): 256-row tiles, tmB box BN/2
  long long wait_budget = 0;  // clocks a pipeline wait may take before the kernel gives up
                              // (<= 0: the default, ~1 s)
};
// Network layers 0 and 1 fused in one kernel (BF16, tanh GELU on both): x [rows x K0] ->
// H1 [rows x N1], the layer-0 activations kept on chip (mlp_tc.cu: fused01_kernel).
struct F01Layer {
  CUtensorMap tmX;       // network input, as layer 0's tmA (box {64, 128})
  CUtensorMap tmW0;      // W0 [N0 x K0], box {64, 64}
  CUtensorMap tmW1a;     // W1 [N1 x N0], box {64, 224}
  CUtensorMap tmW1b;     // W1, box {64, 192}
  CUtensorMap tmO;       // H1 output, as layer 1's tmO
  int N0, N1, K0;
  const float* b0;
  const float* b1;
  long long wait_budget = 0;  // as TcLayer::wait_budget
};
bool f01_supported(int K0, int N0, int N1);
bool f01_encode(F01Layer& F, const void* W0, int64_t ldw0, const void* W1, int64_t ldw1, char* err,
                size_t errlen);
cudaError_t prepare_f01();
cudaError_t launch_f01(const F01Layer& F, const RowMap& rows, int num_sms, int* err, cudaStream_t st);
bool tc_encode_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner,
                  uint64_t outer, uint64_t row_pitch_bytes, uint32_t box_inner,
                  uint32_t box_outer, char* err, size_t errlen);
// Encodes L.tmO (and L.tmG for mode 1) for an output buffer of `rows` rows: columns 0..N-1
// of L.out (row pitch L.ldo elements of L.out_kind), boxes of 32 x 32. Rows of a tile beyond
// the valid rows of a launch are written too (up to `rows`): outputs are scratch buffers.
bool tc_encode_out(TcLayer& L, uint64_t rows, char* err, size_t errlen);
cudaError_t launch_tc_gemm(const TcLayer& L, const RowMap& rows, int num_sms, int* err,
                           cudaStream_t st);
cudaError_t prepare_tc(const TcLayer& L);
// Pipeline stages of the kernel instance with this tile width and output kind, and the
// number of epilogue warps per TMEM lane quarter (for the host's choice of tile width).
int tc_stages(int BN, int out_kind, bool pair = false);
int tc_epi_warps_per_quarter();

}  // namespace dfgb
