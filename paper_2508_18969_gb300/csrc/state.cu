// C ABI of libdfgb (include/df.h): state creation, the fused reaction step and the stage
// entry points. Host code only orchestrates; every step of the path runs in the kernels
// of eos.cu, compact.cu, mlp_simt.cu and mlp_tc.cu.
#include "state.cuh"
#include "../../include/df_propnet.h"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>


namespace dfgb {

thread_local std::string g_create_err;
const char* kVersion = "dfgb 0.1.0 (sm_103a)";

df_status fail(df_state* s, df_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) s->err = buf; else g_create_err = buf;
  return code;
}

df_status cuda_fail(df_state* s, cudaError_t e, const char* where) {
  return fail(s, e == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

// Tile of a tensor-core layer: BN output columns per CTA from {64, 128, 160, 192, 224, 256} for
// hidden layers and {32, 64} for the read-out; hidden layers of more than one k-block may also
// run on CTA pairs (BN from {160, 224, 256} | DF_TILE_PAIR: 256-row tiles, each CTA holding
// half of the tile's weight rows). Cost per layer, fitted to measured tcgen05 times on this GPU:
//   * one k-block (K <= 64 BF16, 128 FP8): the epilogue is the work; each tile costs the
//     32-column chunks its busiest epilogue warp handles, plus half a chunk of fixed cost (the
//     last tile only the chunks of the columns left);
//   * longer K: a tile costs the larger of its MMA work (0.97 BN) and the operand rows an SM
//     streams per k-block (128 + BN/2 on a pair; 0.8 (128 + BN) on a single CTA, whose loads
//     stream faster per row), x1.25 when the tile leaves the TMA ring fewer than four stages.
//     On the 1600 -> 800 layer of 2^20 rows this orders the measured times of single 160, 224
//     and pair 160, 224, 256 tiles (2.15, 1.91, 1.82, 1.73, 1.75 ms) within 7 %.
int pick_tile(int N, int K, bool hidden, int out_kind, bool allow_pair) {
  static const int hid[] = {256, 224, 192, 160, 128, 64};
  static const int last[] = {64, 32};
  static const int paired[] = {256, 224, 160};
  const int* cand = hidden ? hid : last;
  const int nc = hidden ? 6 : 2;
  const bool one_kblock = K * (out_kind == kXFP8 ? 1 : 2) <= 128;
  const int epq = tc_epi_warps_per_quarter();
  int best = cand[nc - 1];
  double best_cost = 1e300;
  auto consider = [&](int bn, bool pair) {
    const double tiles = (double)((N + bn - 1) / bn);
    double cost;
    if (one_kblock) {
      auto busiest = [&](int cols) { return (double)(((cols + 31) / 32 + epq - 1) / epq) + 0.5; };
      const int full = N / bn, rest = N - full * bn;
      cost = full * busiest(bn) + (rest > 0 ? busiest(rest) : 0.0);
    } else {
      const double rows = pair ? 128.0 + bn / 2 : 0.8 * (128.0 + bn);
      cost = tiles * std::max<double>(0.97 * bn, rows) *
             (tc_stages(bn, out_kind, pair) < 4 ? 1.25 : 1.0);
    }
    if (cost < best_cost) {
      best_cost = cost;
      best = pair ? (bn | DF_TILE_PAIR) : bn;
    }
  };
  for (int i = 0; i < nc; ++i) consider(cand[i], false);
  if (hidden && allow_pair && !one_kblock)
    for (int bn : paired) consider(bn, true);
  return best;
}


__global__ void cast_rows_kernel(int64_t rows, int K, const float* __restrict__ in,
                                 int64_t ldi, void* out, int64_t ldo, int kind, float scale) {
  const int64_t total = rows * ldo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldo;
    const int k = (int)(e % ldo);
    const float v = (k < K) ? in[r * ldi + k] : 0.0f;
    if (kind == kXF32) ((float*)out)[e] = v;
    else if (kind == kXBF16) ((__nv_bfloat16*)out)[e] = __float2bfloat16_rn(v);
    else ((__nv_fp8_e4m3*)out)[e] = __nv_fp8_e4m3(v * scale);
  }
}

cudaError_t launch_cast_rows(int64_t rows, int K, const float* in, int64_t ldi, void* out,
                             int64_t ldo, int kind, float scale, int num_sms, cudaStream_t st) {
  const int64_t total = rows * ldo;
  if (total <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 16);
  cast_rows_kernel<<<g, 256, 0, st>>>(rows, K, in, ldi, out, ldo, kind, scale);
  return cudaGetLastError();
}

int xkind_of(int precision) {
  return precision == DF_BF16 ? kXBF16 : precision == DF_FP8_E4M3 ? kXFP8 : kXF32;
}

size_t elem_of(int precision) {
  return precision == DF_BF16 ? 2 : precision == DF_FP8_E4M3 ? 1 : 4;
}

void free_jac(Jac* j) {
  if (!j) return;
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(j->x); f(j->act[0]); f(j->act[1]); f(j->tan[0]); f(j->tan[1]);
  for (auto p : j->G) f(p);
  f(j->O); f(j->dO); f(j->h0); f(j->sc); f(j->jscr); f(j->jst); f(j->W1T); f(j->zero_bias);
  for (auto p : j->Wb) f(p);
  delete j;
}

void free_state(df_state* s) {
  auto f = [](void* p) { if (p) cudaFree(p); };
  free_jac(s->jac);
  s->jac = nullptr;
  free_trn(s->trn);
  s->trn = nullptr;
  f(s->d_spc); f(s->d_K); f(s->d_norm); f(s->d_spc2); f(s->d_K4); f(s->d_kcol); f(s->d_kf2); f(s->d_lntab); f(s->d_lntab2); f(s->d_tsp); f(s->d_tpair); f(s->d_gtab); f(s->d_err); f(s->d_count); f(s->d_flagged); f(s->d_iters);
  for (auto p : s->W32) f(p);
  for (auto p : s->bias) f(p);
  for (auto p : s->Wlp) f(p);
  for (auto p : s->col_scale) f(p);
  f(s->x); f(s->act[0]); f(s->act[1]); f(s->O); f(s->h0); f(s->rho_row); f(s->rstat);
  f(s->idx); f(s->cscr); f(s->vjpJ); f(s->vjpT);
  for (int b = 0; b < 2; ++b) {
    f(s->hp.T[b]); f(s->hp.p[b]); f(s->hp.Y[b]); f(s->hp.st[b]);
    if (s->hp.ev_in[b]) cudaEventDestroy(s->hp.ev_in[b]);
    if (s->hp.ev_done[b]) cudaEventDestroy(s->hp.ev_done[b]);
    if (s->hp.ev_out[b]) cudaEventDestroy(s->hp.ev_out[b]);
  }
  f(s->hp.total);
  if (s->hp.ev_start) cudaEventDestroy(s->hp.ev_start);
  if (s->hp.in) cudaStreamDestroy(s->hp.in);
  if (s->hp.out) cudaStreamDestroy(s->hp.out);
}

cudaEvent_t prof_event(df_state* s) {
  if (!s->prof_pool.empty()) {
    cudaEvent_t e = s->prof_pool.back();
    s->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_family(df_state* s, const char* name) {
  for (size_t i = 0; i < s->prof_names.size(); ++i)
    if (s->prof_names[i] == name) return (int)i;
  s->prof_names.push_back(name);
  s->prof_launches.push_back(0);
  s->prof_ms.push_back(0.0);
  return (int)s->prof_names.size() - 1;
}

// The network layers a6-a7 on rows of the batch buffers: x -> act -> ... -> O.
df_status run_mlp(df_state* s, const RowMap& rm, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  static const char* kLayer[8] = {"layer0", "layer1", "layer2", "layer3",
                                  "layer4", "layer5", "layer6", "layer7"};
  int l0 = 0;
  if (s->fuse01) {
    ProfScope ps(s, "layer0+1", st);
    e = launch_f01(s->f01, rm, s->num_sms, s->d_err, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "fused layers 0 and 1");
    l0 = 2;
  }
  for (int l = l0; l < s->L; ++l) {
    const bool last = l == s->L - 1;
    ProfScope ps(s, kLayer[l], st);
    if (s->precision == DF_FP32) {
      const float* A = (l == 0) ? (const float*)s->x : (const float*)s->act[(l - 1) & 1];
      const int64_t lda = (l == 0) ? s->ldx : s->act_ld[(l - 1) & 1];
      float* Cout = last ? s->O : (float*)s->act[l & 1];
      const int64_t ldc = last ? s->ldo : s->act_ld[l & 1];
      e = launch_sgemm_bias_act(rm, s->widths[l + 1], s->Kp8[l], A, lda, s->W32[l], s->Kp8[l],
                                s->bias[l], Cout, ldc, !last, s->num_sms, st, 0, nullptr, 0, 1,
                                last ? nullptr : s->d_gtab);
    } else {
      e = launch_tc_gemm(s->tcl[l], rm, s->num_sms, s->d_err, st);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "network layer launch");
  }
  return DF_OK;
}

df_status check_fields(df_state* s, int64_t n, const void* a, const void* b, const void* Y,
                       int64_t ldY) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (s->netonly)
    return fail(s, DF_ERR_UNSUPPORTED, "the state holds a network only (df_network_create)");
  if (n < 0) return fail(s, DF_ERR_INVALID_ARG, "n_cells < 0");
  if (n == 0) return DF_OK;
  if (!a || !b || !Y) return fail(s, DF_ERR_INVALID_ARG, "NULL field pointer");
  if (ldY < n) return fail(s, DF_ERR_INVALID_ARG, "ldY (%lld) < n_cells (%lld)", (long long)ldY,
                           (long long)n);
  return DF_OK;
}

df_status ensure_compact(df_state* s, int64_t n) {
  if (n > s->idx_cap) {
    if (s->idx) cudaFree(s->idx);
    s->idx = nullptr;
    s->idx_cap = 0;
    cudaError_t e = dalloc(&s->idx, (size_t)n);
    if (e != cudaSuccess) return cuda_fail(s, e, "reacting-cell list");
    s->idx_cap = n;
  }
  const int64_t w = compact_scratch_words(n);
  if (w > s->cscr_words) {
    if (s->cscr) cudaFree(s->cscr);
    s->cscr = nullptr;
    s->cscr_words = 0;
    cudaError_t e = dalloc(&s->cscr, (size_t)w);
    if (e != cudaSuccess) return cuda_fail(s, e, "compaction scratch");
    s->cscr_words = w;
  }
  return DF_OK;
}

// Error text of entry points that take no state (read with df_get_last_error(NULL)).
void set_global_error(const char* msg) { g_create_err = msg; }
}  // namespace dfgb

extern "C" {

const char* df_version(void) { return kVersion; }

const char* df_get_last_error(df_state* s) { return s ? s->err.c_str() : g_create_err.c_str(); }

// A state with the mechanism (mech != NULL: the reaction step) or with a network only
// (mech == NULL: df_network_create; n = widths[0] - 2 composition inputs, any output width).
static df_status create_state(const df_mech_desc* mech, const df_mlp_desc* mlp,
                              const df_options* opt, df_state** out) {
  if (!out) return fail(nullptr, DF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!mlp || !opt) return fail(nullptr, DF_ERR_INVALID_ARG, "NULL descriptor");
  const int L = mlp->n_layers;
  if (L < 1 || L > 8 || !mlp->widths || !mlp->W || !mlp->b)
    return fail(nullptr, DF_ERR_INVALID_ARG, "bad network description");
  const bool netonly = mech == nullptr;
  const int n = netonly ? mlp->widths[0] - 2 : mech->n_species;
  if (n < 1 || n > kMaxSpecies)
    return fail(nullptr, DF_ERR_UNSUPPORTED, "n_species must be in 1..%d", kMaxSpecies);
  if (!netonly && (!mech->W || !mech->Tc || !mech->pc || !mech->omega || !mech->kij || !mech->nasa))
    return fail(nullptr, DF_ERR_INVALID_ARG, "NULL mechanism array");
  if (!netonly && (mlp->widths[0] != n + 2 || mlp->widths[L] != n))
    return fail(nullptr, DF_ERR_INVALID_ARG, "network must map n+2 inputs to n outputs");
  const int nout = mlp->widths[L];
  for (int l = 0; l <= L; ++l)
    if (mlp->widths[l] < 1 || mlp->widths[l] > 8192)
      return fail(nullptr, DF_ERR_INVALID_ARG, "layer width out of range");
  if (!mlp->in_mean || !mlp->in_std || !mlp->out_mean || !mlp->out_std)
    return fail(nullptr, DF_ERR_INVALID_ARG, "NULL normalisation array");
  if (!(mlp->lambda > 0.0)) return fail(nullptr, DF_ERR_INVALID_ARG, "lambda must be > 0");
  const double inv_l = 1.0 / mlp->lambda;
  const int m = (int)std::lround(inv_l);
  if (m < 1 || m > 64 || std::fabs(inv_l - m) > 1e-9 * inv_l)
    return fail(nullptr, DF_ERR_UNSUPPORTED, "1/lambda must be an integer in 1..64");
  if (!netonly && !(mlp->dt > 0.0)) return fail(nullptr, DF_ERR_INVALID_ARG, "dt must be > 0");
  if (netonly && opt->precision == DF_FP8_E4M3)
    return fail(nullptr, DF_ERR_UNSUPPORTED, "network-only states run in FP32 or BF16");
  if (opt->precision < DF_FP32 || opt->precision > DF_FP8_E4M3)
    return fail(nullptr, DF_ERR_INVALID_ARG, "unknown precision");
  if (opt->gelu_mode != DF_GELU_TANH && opt->gelu_mode != DF_GELU_TABLE)
    return fail(nullptr, DF_ERR_INVALID_ARG, "unknown gelu_mode");
  if (opt->gelu_mode == DF_GELU_TABLE && opt->precision == DF_FP8_E4M3)
    return fail(nullptr, DF_ERR_UNSUPPORTED, "the tabulated GELU runs on FP32 and BF16 networks");
  for (int k = 0; !netonly && k < n; ++k)
    if (!(mech->W[k] > 0) || !(mech->Tc[k] > 0) || !(mech->pc[k] > 0))
      return fail(nullptr, DF_ERR_INVALID_ARG, "W, Tc, pc must be positive");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
    return fail(nullptr, DF_ERR_CUDA, "no CUDA device");
  if (opt->device < 0 || opt->device >= ndev)
    return fail(nullptr, DF_ERR_INVALID_ARG, "device ordinal out of range");
  DeviceGuard guard(opt->device);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, opt->device);
  if (opt->precision != DF_FP32 && prop.major * 10 + prop.minor < 100)
    return fail(nullptr, DF_ERR_UNSUPPORTED, "tensor-core precisions need sm_100 or newer");

  df_state* s = new df_state();
  s->device = opt->device;
  s->num_sms = prop.multiProcessorCount;
  s->n = n;
  s->K0 = n + 2;
  s->nout = nout;
  s->netonly = netonly;
  s->L = L;
  s->widths.assign(mlp->widths, mlp->widths + L + 1);
  s->precision = opt->precision;
  s->gelu_mode = opt->gelu_mode;
  s->T_react = opt->T_react;
  s->lambda = mlp->lambda;
  s->dt = mlp->dt;
  s->cap = opt->batch_cells > 0 ? round_up(opt->batch_cells, 128) : (int64_t)1 << 20;
  cudaError_t e;
#define CK(expr, what)                          \
  do {                                          \
    e = (expr);                                 \
    if (e != cudaSuccess) {                     \
      df_status rc = cuda_fail(nullptr, e, what); \
      free_state(s);                            \
      delete s;                                 \
      return rc;                                \
    }                                           \
  } while (0)

  // ---- equation-of-state constants (Peng & Robinson 1976, NASA-7) ----
  std::vector<double> spc((size_t)n * kSpcStride), K((size_t)n * n);
  for (int k = 0; !netonly && k < n; ++k) {   // (a network-only state keeps zero tables)
    const double Tc = mech->Tc[k], pc = mech->pc[k], w = mech->omega[k];
    const double ac = 0.45724 * kR * kR * Tc * Tc / pc;
    const double b = 0.07780 * kR * Tc / pc;
    const double kap = 0.37464 + 1.54226 * w - 0.26992 * w * w;
    const double sac = std::sqrt(ac);
    double* q = &spc[(size_t)k * kSpcStride];
    const double* a = mech->nasa + 7 * k;
    q[0] = 1.0 / mech->W[k];
    q[1] = sac * (1.0 + kap);
    q[2] = sac * kap / std::sqrt(Tc);
    q[3] = b;
    q[4] = kR * a[5];
    q[5] = kR * a[0];
    q[6] = kR * a[1] / 2.0;
    q[7] = kR * a[2] / 3.0;
    q[8] = kR * a[3] / 4.0;
    q[9] = kR * a[4] / 5.0;
  }
  for (int i = 0; !netonly && i < n; ++i)
    for (int j = 0; j < n; ++j) K[(size_t)i * n + j] = (i == j) ? 1.0 : 1.0 - mech->kij[i * n + j];
  std::vector<double> norm((size_t)2 * s->K0 + 2 * nout);
  for (int k = 0; k < s->K0; ++k) {
    if (!(mlp->in_std[k] != 0.0)) {
      delete s;
      return fail(nullptr, DF_ERR_INVALID_ARG, "in_std must be non-zero");
    }
    norm[k] = mlp->in_mean[k];
    norm[s->K0 + k] = 1.0 / mlp->in_std[k];
  }
  for (int k = 0; k < nout; ++k) {
    norm[2 * s->K0 + k] = mlp->out_mean[k];
    norm[2 * s->K0 + nout + k] = mlp->out_std[k];
  }
  CK(dalloc(&s->d_spc, spc.size()), "constants");
  CK(dalloc(&s->d_K, K.size()), "constants");
  CK(dalloc(&s->d_norm, norm.size()), "constants");
  CK(cudaMemcpy(s->d_spc, spc.data(), sizeof(double) * spc.size(), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(s->d_K, K.data(), sizeof(double) * K.size(), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(s->d_norm, norm.data(), sizeof(double) * norm.size(), cudaMemcpyHostToDevice), "copy");
  // double-float (hi, lo) copies: x = hi + lo with hi = fl32(x), lo = fl32(x - hi)
  auto split = [](const std::vector<double>& v) {
    std::vector<float> o(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float h = (float)v[i];
      o[2 * i] = h;
      o[2 * i + 1] = (float)(v[i] - (double)h);
    }
    return o;
  };
  // mixing-sum tables with 1/W folded in (computed in FP64, then split)
  std::vector<double> spcw(spc.size()), Ks((size_t)n * n), Kr((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    const double iW = spc[(size_t)k * kSpcStride];
    spcw[(size_t)k * kSpcStride] = iW;
    for (int j = 1; j < kSpcStride; ++j)
      spcw[(size_t)k * kSpcStride + j] = spc[(size_t)k * kSpcStride + j] * iW;
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double* q = &spc[(size_t)j * kSpcStride];
      Ks[(size_t)i * n + j] = K[(size_t)i * n + j] * q[1] * q[0];
      Kr[(size_t)i * n + j] = K[(size_t)i * n + j] * q[2] * q[0];
    }
  const std::vector<float> spcw2 = split(spcw), Ks2 = split(Ks), Kr2 = split(Kr);
  // the pair tables interleaved per (i, j): (Ks hi, Ks lo, Kr hi, Kr lo), one 16-byte load,
  // the strict upper triangle j > i only, row by row (row i starts at i n - i (i + 1) / 2);
  // then the column maxima max_i |Ks_ij| and max_i |Kr_ij|, rounded up, for the accumulator
  // offsets of the pair sums
  std::vector<float> K4((size_t)2 * n * (n - 1) + 4), kcol((size_t)2 * n, 0.0f);
  for (int i = 0, t = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j, ++t) {
      const size_t o = (size_t)i * n + j;
      K4[4 * (size_t)t] = Ks2[2 * o];
      K4[4 * (size_t)t + 1] = Ks2[2 * o + 1];
      K4[4 * (size_t)t + 2] = Kr2[2 * o];
      K4[4 * (size_t)t + 3] = Kr2[2 * o + 1];
    }
  // (a negative entry, k_ij > 1, makes terms of both signs even for Y >= 0: the maxima are
  // scaled by four, which is what the offset needs for terms of both signs)
  bool kneg = false;
  for (size_t o = 0; o < (size_t)n * n; ++o) kneg = kneg || Ks[o] < 0.0 || Kr[o] < 0.0;
  for (int j = 0; j < n; ++j) {
    double ms = 0.0, mr = 0.0;
    for (int i = 0; i < n; ++i) {
      ms = std::max(ms, std::fabs(Ks[(size_t)i * n + j]));
      mr = std::max(mr, std::fabs(Kr[(size_t)i * n + j]));
    }
    const double f = (kneg ? 4.0 : 1.0) * (1.0 + 1.0 / 1024.0);
    kcol[j] = (float)(ms * f);
    kcol[n + j] = (float)(mr * f);
  }
  // FP32 pair corrections of the T-from-h solve, interleaved (k_ij s_j / W_j, k_ij r_j / W_j)
  // for the pairs j > i, row by row (row i from pair i n - i (i + 1) / 2)
  std::vector<float> kf2((size_t)n * (n - 1) + 2);
  for (int i = 0, t = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j, ++t) {
      const double k = 1.0 - K[(size_t)i * n + j];
      const double* q = &spc[(size_t)j * kSpcStride];
      kf2[2 * (size_t)t] = (float)(k * q[1] * q[0]);
      kf2[2 * (size_t)t + 1] = (float)(k * q[2] * q[0]);
    }
  if (s->gelu_mode == DF_GELU_TABLE) {
    // value, slope and half curvature of the tanh-form GELU at x_i = -3 + 0.01 i
    std::vector<float4> gt(kGeluTableNodes);
    const double c = 0.79788456080286535588, a = 0.044715;  // sqrt(2 / pi)
    for (int i = 0; i < kGeluTableNodes; ++i) {
      const double x = -3.0 + 0.01 * i;
      const double u = c * (x + a * x * x * x), th = std::tanh(u);
      const double up = c * (1.0 + 3.0 * a * x * x), upp = 6.0 * a * c * x;
      const double g0 = 0.5 * x * (1.0 + th);
      const double g1 = 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * up;
      const double g2 = (1.0 - th * th) * (up - x * th * up * up + 0.5 * x * upp);
      gt[i] = make_float4((float)g0, (float)g1, (float)(0.5 * g2), 0.0f);
    }
    CK(dalloc(&s->d_gtab, gt.size()), "gelu table");
    CK(cudaMemcpy(s->d_gtab, gt.data(), sizeof(float4) * gt.size(), cudaMemcpyHostToDevice), "copy");
  }
  std::vector<double> lntab(256);
  for (int j = 0; j < 128; ++j) {
    const double c = 1.0 + (j + 0.5) / 128.0;
    lntab[j] = std::log(c);
    lntab[128 + j] = 1.0 / c;
  }
  CK(dalloc(&s->d_lntab, lntab.size()), "constants");
  CK(cudaMemcpy(s->d_lntab, lntab.data(), sizeof(double) * 256, cudaMemcpyHostToDevice), "copy");
  // the same table in double-float pairs (hi, lo) for the double-float state evaluation
  const std::vector<float> lntab2 = split(lntab);
  CK(dalloc(&s->d_lntab2, lntab2.size()), "constants");
  CK(cudaMemcpy(s->d_lntab2, lntab2.data(), sizeof(float) * lntab2.size(), cudaMemcpyHostToDevice),
     "copy");
  // Chung's mixing-rule tables (transport properties): sigma_i = 0.809 Vc_i^(1/3) Angstrom,
  // eps_i / k = Tc_i / 1.2593, Vc_i = Zc R Tc_i / pc_i with the Peng-Robinson critical
  // compressibility Zc = 0.307401, binary factors 1
  std::vector<double> tsp((size_t)n * 4);
  std::vector<float> tpair((size_t)4 * n * n);
  for (int k = 0; !netonly && k < n; ++k) {
    tsp[4 * k] = mech->Tc[k];
    tsp[4 * k + 1] = 0.307401 * kR * mech->Tc[k] / mech->pc[k] * 1e6;
    tsp[4 * k + 2] = mech->omega[k];
    tsp[4 * k + 3] = mech->W[k] * 1e3;
  }
  for (int i = 0; !netonly && i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double si = 0.809 * std::cbrt(tsp[4 * i + 1]), sj = 0.809 * std::cbrt(tsp[4 * j + 1]);
      const double eij = std::sqrt(tsp[4 * i] * tsp[4 * j]) / 1.2593;
      const double s2 = si * sj, s3 = s2 * std::sqrt(s2);
      const double Mi = tsp[4 * i + 3], Mj = tsp[4 * j + 3];
      const size_t o = (size_t)i * n + j, nn = (size_t)n * n;
      tpair[o] = (float)s3;
      tpair[nn + o] = (float)(eij * s3);
      tpair[2 * nn + o] = (float)(0.5 * (tsp[4 * i + 2] + tsp[4 * j + 2]) * s3);
      tpair[3 * nn + o] = (float)(eij * s2 * std::sqrt(2.0 * Mi * Mj / (Mi + Mj)));
    }
  CK(dalloc(&s->d_tsp, tsp.size()), "constants");
  CK(dalloc(&s->d_tpair, tpair.size()), "constants");
  CK(cudaMemcpy(s->d_tsp, tsp.data(), sizeof(double) * tsp.size(), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(s->d_tpair, tpair.data(), sizeof(float) * tpair.size(), cudaMemcpyHostToDevice), "copy");
  CK(dalloc(&s->d_kf2, kf2.size()), "constants");
  CK(cudaMemcpy(s->d_kf2, kf2.data(), sizeof(float) * kf2.size(), cudaMemcpyHostToDevice), "copy");
  CK(dalloc(&s->d_spc2, spcw2.size()), "constants");
  CK(dalloc(&s->d_K4, K4.size()), "constants");
  CK(dalloc(&s->d_kcol, kcol.size()), "constants");
  CK(cudaMemcpy(s->d_spc2, spcw2.data(), sizeof(float) * spcw2.size(), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(s->d_K4, K4.data(), sizeof(float) * K4.size(), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(s->d_kcol, kcol.data(), sizeof(float) * kcol.size(), cudaMemcpyHostToDevice), "copy");
  CK(dalloc(&s->d_err, 1), "error word");
  CK(cudaMemset(s->d_err, 0, sizeof(int)), "memset");
  CK(dalloc(&s->d_count, 1), "counters");
  CK(dalloc(&s->d_flagged, 1), "counters");
  CK(dalloc(&s->d_iters, 1), "counters");
  CK(cudaMemset(s->d_iters, 0, sizeof(int64_t)), "memset");
  CK(cudaMemset(s->d_count, 0, sizeof(int64_t)), "memset");
  CK(cudaMemset(s->d_flagged, 0, sizeof(int64_t)), "memset");
  EosParams& P = s->P;
  P.n = n;
  P.K0 = s->K0;
  P.inv_lambda = m;
  for (int k = 0; k <= 16; ++k) P.binom[k] = 0.0f;
  if (m >= 1 && m <= 16) {
    double c = 1.0;
    for (int k = 0; k <= m; ++k) {
      P.binom[k] = (float)c;
      c = c * (m - k) / (k + 1);
    }
  }
  P.lambda = mlp->lambda;
  P.T_react = opt->T_react;
  P.newton_tol = opt->newton_tol > 0 ? opt->newton_tol : 1e-8;
  P.newton_max_iter = opt->newton_max_iter > 0 ? opt->newton_max_iter : 50;
  P.spc = s->d_spc;
  P.Kmat = s->d_K;
  P.norm = s->d_norm;
  P.spcw2 = s->d_spc2;
  P.K4 = s->d_K4;
  P.kcol = s->d_kcol;
  P.kf2 = s->d_kf2;
  for (int j = 0; j < kSpcStride; ++j) {
    float mx = 0.0f;
    for (int k = 0; k < n; ++k)
      mx = std::max(mx, std::fabs(spcw2[2 * ((size_t)k * kSpcStride + j)]));
    P.spcmax[j] = std::nextafter(mx, INFINITY);
  }
  P.lntab = s->d_lntab;
  P.lntab2 = s->d_lntab2;
  P.tsp = s->d_tsp;
  P.tpair = s->d_tpair;
  P.err = s->d_err;
  P.flagged = s->d_flagged;
  P.newton_iters = s->d_iters;

  // ---- network weights ----
  const bool lp = s->precision != DF_FP32;
  const size_t eb = elem_of(s->precision);
  for (int l = 0; l < L; ++l) {
    const int Kl = s->widths[l], Nl = s->widths[l + 1];
    if (!mlp->W[l] || !mlp->b[l]) {
      free_state(s);
      delete s;
      return fail(nullptr, DF_ERR_INVALID_ARG, "NULL layer array");
    }
    s->Wh.emplace_back(mlp->W[l], mlp->W[l] + (size_t)Nl * Kl);
    // bias and scales are zero padded to a multiple of 32 so the epilogue loads whole chunks
    const int64_t Npad = round_up(Nl, 32);
    float* b = nullptr;
    CK(dalloc(&b, Npad), "bias");
    s->bias.push_back(b);
    CK(cudaMemset(b, 0, sizeof(float) * Npad), "memset");
    CK(cudaMemcpy(b, mlp->b[l], sizeof(float) * Nl, cudaMemcpyHostToDevice), "copy");
    if (!lp) {
      const int kp = (int)round_up(Kl, 8);
      std::vector<float> w((size_t)Nl * kp, 0.0f);
      for (int r = 0; r < Nl; ++r)
        for (int c = 0; c < Kl; ++c) w[(size_t)r * kp + c] = mlp->W[l][(size_t)r * Kl + c];
      float* d = nullptr;
      CK(dalloc(&d, w.size()), "weights");
      CK(cudaMemcpy(d, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice), "copy");
      s->W32.push_back(d);
      s->Kp8.push_back(kp);
    } else {
      const int kp = (int)round_up(Kl, 16);
      void* d = nullptr;
      CK(cudaMalloc(&d, eb * (size_t)Nl * kp), "weights");
      float* cs = nullptr;
      if (s->precision == DF_BF16) {
        std::vector<__nv_bfloat16> w((size_t)Nl * kp, __float2bfloat16_rn(0.0f));
        for (int r = 0; r < Nl; ++r)
          for (int c = 0; c < Kl; ++c)
            w[(size_t)r * kp + c] = __float2bfloat16_rn(mlp->W[l][(size_t)r * Kl + c]);
        CK(cudaMemcpy(d, w.data(), eb * w.size(), cudaMemcpyHostToDevice), "copy");
      } else {
        // per-output-channel scale: row max |W| maps to the e4m3 maximum 448
        std::vector<uint8_t> w((size_t)Nl * kp, 0);
        std::vector<float> sc(Nl);
        for (int r = 0; r < Nl; ++r) {
          float amax = 0.0f;
          for (int c = 0; c < Kl; ++c) amax = std::max(amax, std::fabs(mlp->W[l][(size_t)r * Kl + c]));
          const float ws = amax > 0 ? amax / 448.0f : 1.0f;
          sc[r] = ws;
          for (int c = 0; c < Kl; ++c)
            w[(size_t)r * kp + c] = __nv_fp8_e4m3(mlp->W[l][(size_t)r * Kl + c] / ws).__x;
        }
        CK(cudaMemcpy(d, w.data(), w.size(), cudaMemcpyHostToDevice), "copy");
        // dequantisation = weight scale / input activation scale
        const float in_scale = kFp8ActScale;
        for (auto& v : sc) v /= in_scale;
        CK(dalloc(&cs, Npad), "scales");
        CK(cudaMemset(cs, 0, sizeof(float) * Npad), "memset");
        CK(cudaMemcpy(cs, sc.data(), sizeof(float) * Nl, cudaMemcpyHostToDevice), "copy");
        s->act_scale.push_back(in_scale);
      }
      s->Wlp.push_back(d);
      s->col_scale.push_back(cs);
      s->Kp8.push_back(kp);
    }
  }

  // ---- batch scratch ----
  const int xk = xkind_of(s->precision);
  s->ldx = round_up(s->K0, lp ? 16 : 8);
  CK(cudaMalloc(&s->x, eb * (size_t)s->cap * s->ldx), "network input");
  int64_t wmax[2] = {8, 8};
  for (int l = 0; l + 1 < L; ++l)
    wmax[l & 1] = std::max<int64_t>(wmax[l & 1], round_up(s->widths[l + 1], lp ? 16 : 8));
  for (int b = 0; b < 2; ++b) {
    s->act_ld[b] = wmax[b];
    CK(cudaMalloc(&s->act[b], eb * (size_t)s->cap * wmax[b]), "activations");
    CK(cudaMemset(s->act[b], 0, eb * (size_t)s->cap * wmax[b]), "memset");
  }
  s->ldo = round_up(nout, 8);
  CK(dalloc(&s->O, (size_t)s->cap * s->ldo), "network output");
  CK(dalloc(&s->h0, (size_t)s->cap), "h0");
  CK(dalloc(&s->rho_row, (size_t)s->cap), "rho");
  CK(dalloc(&s->rstat, (size_t)s->cap), "row status");

  if (lp) {
    char emsg[256];
    for (int l = 0; l < L; ++l) {
      const bool last = l == L - 1;
      TcLayer T{};
      T.N = s->widths[l + 1];
      T.K = s->widths[l];
      const int tile = pick_tile(T.N, T.K, !last, last ? kXF32 : xk, true);
      T.BN = tile & ~DF_TILE_PAIR;
      T.pair = (tile & DF_TILE_PAIR) != 0;
      if (const char* env = getenv("DFGB_BN")) {  // hidden-layer tile-width override (sweeps)
        const int v = atoi(env);
        if (!last && (v == 64 || v == 128 || v == 160 || v == 192 || v == 224 || v == 256)) {
          T.BN = v;
          T.pair = false;
        }
      }
      T.bias = s->bias[l];
      T.col_scale = s->col_scale[l];
      T.out = last ? (void*)s->O : s->act[l & 1];
      T.ldo = last ? s->ldo : s->act_ld[l & 1];
      T.out_kind = last ? kXF32 : xk;
      T.gelu = !last;
      T.gtab = last ? nullptr : s->d_gtab;
      T.out_scale = (s->precision == DF_FP8_E4M3 && !last) ? s->act_scale[l + 1] : 1.0f;
      T.elem_bytes = (int)eb;
      const void* Abase = (l == 0) ? s->x : s->act[(l - 1) & 1];
      const int64_t lda = (l == 0) ? s->ldx : s->act_ld[(l - 1) & 1];
      const uint32_t boxk = 128 / (uint32_t)eb;
      if (!tc_encode_2d(&T.tmA, Abase, (int)eb, (uint64_t)T.K, (uint64_t)s->cap,
                        (uint64_t)lda * eb, boxk, 128, emsg, sizeof emsg) ||
          !tc_encode_2d(&T.tmB, s->Wlp[l], (int)eb, (uint64_t)T.K, (uint64_t)T.N,
                        (uint64_t)s->Kp8[l] * eb, boxk, (uint32_t)(T.pair ? T.BN / 2 : T.BN),
                        emsg, sizeof emsg) ||
          !tc_encode_out(T, (uint64_t)s->cap, emsg, sizeof emsg)) {
        free_state(s);
        delete s;
        return fail(nullptr, DF_ERR_CUDA, "%s", emsg);
      }
      s->tcl.push_back(T);
    }
    // Layers 0 and 1 of a BF16 tanh-GELU network as one kernel (the layer-0 activations never
    // leave the SM), on request only (DFGB_FUSE01=1): on GB300 the fused kernel measured slower
    // than the two layers apart (3.40 against 2.64 ms per 2^20 rows), because single-CTA MMAs
    // run well below the CTA-pair rate and the layer-1 accumulator cannot be double-buffered
    // beside the layer-0 block in tensor memory.
    const char* fenv = getenv("DFGB_FUSE01");
    if (s->precision == DF_BF16 && s->gelu_mode == DF_GELU_TANH && L >= 3 &&
        f01_supported(s->widths[0], s->widths[1], s->widths[2]) && fenv && atoi(fenv) == 1) {
      F01Layer& F = s->f01;
      F.tmX = s->tcl[0].tmA;
      F.tmO = s->tcl[1].tmO;
      F.K0 = s->widths[0];
      F.N0 = s->widths[1];
      F.N1 = s->widths[2];
      F.b0 = s->bias[0];
      F.b1 = s->bias[1];
      if (!f01_encode(F, s->Wlp[0], s->Kp8[0], s->Wlp[1], s->Kp8[1], emsg, sizeof emsg)) {
        free_state(s);
        delete s;
        return fail(nullptr, DF_ERR_CUDA, "%s", emsg);
      }
      s->fuse01 = true;
    }
  }
  // one-time per-device kernel attributes, so that no later call (or graph capture) sets any
  CK(prepare_eos(s->P, xk), "kernel attributes");
  for (const TcLayer& T : s->tcl) CK(prepare_tc(T), "kernel attributes");
  if (s->fuse01) CK(prepare_f01(), "kernel attributes");
#undef CK
  *out = s;
  return DF_OK;
}

df_status df_state_create(const df_mech_desc* mech, const df_mlp_desc* mlp,
                          const df_options* opt, df_state** out) {
  if (!mech) {
    if (out) *out = nullptr;
    return fail(nullptr, DF_ERR_INVALID_ARG, "NULL descriptor");
  }
  return create_state(mech, mlp, opt, out);
}

df_status df_network_create(const df_mlp_desc* mlp, const df_options* opt, df_state** out) {
  return create_state(nullptr, mlp, opt, out);
}

void df_state_destroy(df_state* s) {
  if (!s) return;
  DeviceGuard guard(s->device);
  cudaDeviceSynchronize();
  for (auto& r : s->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : s->prof_pool) cudaEventDestroy(e);
  free_state(s);
  delete s;
}

df_status df_real_fluid_props(df_state* s, int64_t n_cells, const double* T, const double* p,
                              const double* Y, int64_t ldY, double* rho, double* h, double* cp,
                              double* Z, void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  DeviceGuard guard(s->device);
  cudaError_t e = launch_props(s->P, n_cells, T, p, Y, ldY, rho, h, cp, Z, (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "real-fluid properties");
}

df_status df_transport_props(df_state* s, int64_t n_cells, const double* T, const double* p,
                             const double* Y, int64_t ldY, double* mu, double* lam, double* alpha,
                             void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  DeviceGuard guard(s->device);
  cudaError_t e = launch_transport(s->P, n_cells, T, p, Y, ldY, mu, lam, alpha, (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "transport properties");
}

}  // extern "C"

namespace {

// The reaction step a0-a10 in batches of the state's capacity. With src (source terms) the
// kernels leave T and Y untouched and write omega / T_new instead.
// Reacting cells of a chunk added to the running total of df_chem_step_host.
__global__ void add_count_kernel(const int64_t* __restrict__ c, int64_t* __restrict__ total,
                                 int first) {
  *total = (first ? 0 : *total) + *c;
}

typedef CUresult (*PointerGetAttributeFn)(void*, CUpointer_attribute, CUdeviceptr);

// Device address of `bytes` bytes of host memory at `ptr` when the whole range lies in one
// page-locked allocation mapped into the device's address space; false otherwise.
template <class P>
bool host_mapped(P* ptr, size_t bytes, P** dev) {
  static PointerGetAttributeFn get_attr = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    return (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
               ? (PointerGetAttributeFn)f
               : nullptr;
  }();
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || !get_attr) return false;
  CUdeviceptr start = 0;
  size_t size = 0;
  const CUdeviceptr dp = (CUdeviceptr)(uintptr_t)a.devicePointer;
  if (get_attr(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS ||
      get_attr(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS)
    return false;
  if (dp < start || dp + bytes > start + size) return false;
  *dev = (P*)a.devicePointer;
  return true;
}

df_status run_step(df_state* s, int64_t n_cells, double dt, double* T, const double* p, double* Y,
                   int64_t ldY, int32_t* cell_status, int64_t* n_active_out, cudaStream_t st,
                   const Source* src, bool keep_counters = false) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK) return rc;
  if (!(std::fabs(dt - s->dt) <= 1e-12 * std::fabs(s->dt)))
    return fail(s, DF_ERR_DT_MISMATCH, "dt %.17g differs from the network's %.17g", dt, s->dt);
  DeviceGuard guard(s->device);
  if ((rc = ensure_compact(s, n_cells)) != DF_OK) return rc;
  cudaError_t e = cudaSuccess;
  if (!keep_counters) {
    e = cudaMemsetAsync(s->d_flagged, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_iters, 0, sizeof(int64_t), st);
  }
  if (e == cudaSuccess) {
    ProfScope ps(s, "compact", st);
    e = launch_compact(n_cells, s->T_react, T, s->idx, s->d_count, cell_status, s->cscr, st);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "reacting-cell compaction");
  const int xk = xkind_of(s->precision);
  const float xs = s->precision == DF_FP8_E4M3 ? s->act_scale[0] : 1.0f;
  for (int64_t row0 = 0; row0 < n_cells; row0 += s->cap) {
    const RowMap rm{s->idx, s->d_count, row0, std::min<int64_t>(s->cap, n_cells - row0)};
    {
      ProfScope ps(s, "eos_pre", st);
      e = launch_eos_pre(s->P, rm, T, p, Y, ldY, s->h0, nullptr, s->x, xk, s->ldx, xs, s->rstat, st,
                         src ? s->rho_row : nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "eos_pre launch");
    if ((rc = run_mlp(s, rm, st)) != DF_OK) return rc;
    {
      ProfScope ps(s, "eos_post", st);
      e = launch_eos_post(s->P, rm, s->O, s->ldo, s->h0, T, p, Y, ldY, s->rstat, cell_status, st,
                          src);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "eos_post launch");
  }
  if (n_active_out) {
    e = cudaMemcpyAsync(n_active_out, s->d_count, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "n_active copy");
  }
  return DF_OK;
}

}  // namespace

extern "C" {

df_status df_chem_step(df_state* s, int64_t n_cells, double dt, double* T, const double* p,
                       double* Y, int64_t ldY, int32_t* cell_status, int64_t* n_active_out,
                       void* stream) {
  return run_step(s, n_cells, dt, T, p, Y, ldY, cell_status, n_active_out, (cudaStream_t)stream,
                  nullptr);
}

df_status df_chem_step_host(df_state* s, int64_t n_cells, double dt, double* T, const double* p,
                            double* Y, int64_t ldY, int32_t* cell_status, int64_t chunk_cells,
                            void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  if (chunk_cells < 0 && chunk_cells != DF_HOST_DIRECT)
    return fail(s, DF_ERR_INVALID_ARG, "chunk_cells < 0");
  if (!(std::fabs(dt - s->dt) <= 1e-12 * std::fabs(s->dt)))
    return fail(s, DF_ERR_DT_MISMATCH, "dt %.17g differs from the network's %.17g", dt, s->dt);
  DeviceGuard guard(s->device);
  const int n = s->n;
  if (chunk_cells == DF_HOST_DIRECT) {
    // the kernels read and write the host arrays in place, over the host link
    double *dT = nullptr, *dY = nullptr;
    const double* dp = nullptr;
    int32_t* dst = nullptr;
    const bool mapped =
        host_mapped(T, sizeof(double) * n_cells, &dT) && host_mapped(p, sizeof(double) * n_cells, &dp) &&
        host_mapped(Y, sizeof(double) * ((size_t)(n - 1) * ldY + n_cells), &dY) &&
        (!cell_status || host_mapped(cell_status, sizeof(int32_t) * n_cells, &dst));
    if (!mapped)
      return fail(s, DF_ERR_INVALID_ARG,
                  "DF_HOST_DIRECT needs T, p, Y and cell_status in page-locked, mapped host memory");
    return run_step(s, n_cells, dt, dT, dp, dY, ldY, dst, nullptr, (cudaStream_t)stream, nullptr);
  }
  // Chunk plan. As asked: equal chunks of chunk_cells. Automatic: a short first and last chunk
  // (1/32 of the cells, at least 32768), so that only a small upload and a small download are
  // not hidden behind a step; then ramp chunks of about 3/16 of the cells, whose steps are long
  // enough to hide the upload of the chunk after them (and, at the end, the download of the
  // chunk before them), the copies running at about a quarter of the step's cells/s; and the
  // cells between them in as few chunks as the batch allows, at the long-batch rate.
  std::vector<int64_t> plan;
  if (chunk_cells > 0) {
    const int64_t c = std::min(chunk_cells, s->cap);
    for (int64_t c0 = 0; c0 < n_cells; c0 += c) plan.push_back(std::min(c, n_cells - c0));
  } else {
    const int64_t edge = std::min(s->cap, std::max<int64_t>(32768, round_up((n_cells + 31) / 32, 128)));
    const int64_t ramp = std::min(s->cap, std::max<int64_t>(32768, round_up((3 * n_cells + 15) / 16, 128)));
    if (n_cells <= 2 * edge + 3 * ramp) {
      const int64_t c = std::min(s->cap, std::max<int64_t>(32768, round_up((n_cells + 3) / 4, 128)));
      for (int64_t c0 = 0; c0 < n_cells; c0 += c) plan.push_back(std::min(c, n_cells - c0));
    } else {
      int64_t mid = n_cells - 2 * edge - 2 * ramp;
      const int64_t k = (mid + s->cap - 1) / s->cap;
      int64_t ramp1 = ramp, ramp2 = ramp;
      // A single middle chunk is cut to whole passes of the EoS kernels' resident blocks, the
      // rest going to the ramps: otherwise its last, partial pass runs a few blocks alone,
      // latency-bound, in each EoS kernel.
      const int64_t wave = k == 1 ? eos_wave_cells(s->P, xkind_of(s->precision)) : 0;
      if (wave > 0 && mid > wave) {
        const int64_t extra = mid - mid / wave * wave;
        if (ramp + extra <= s->cap) {
          ramp1 += extra / 2;
          ramp2 += extra - extra / 2;
          mid -= extra;
        }
      }
      const int64_t m = round_up((mid + k - 1) / k, 128);
      plan.push_back(edge);
      plan.push_back(ramp1);
      for (int64_t c0 = 0; c0 < mid; c0 += m) plan.push_back(std::min(m, mid - c0));
      plan.push_back(ramp2);
      plan.push_back(edge);
    }
  }
  int64_t chunk = 0;
  for (int64_t c : plan) chunk = std::max(chunk, c);
  df_state::HostPipe& hp = s->hp;
  cudaError_t e = cudaSuccess;
  if (hp.chunk < chunk) {
    e = cudaDeviceSynchronize();
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      cudaFree(hp.T[b]); cudaFree(hp.p[b]); cudaFree(hp.Y[b]); cudaFree(hp.st[b]);
      hp.T[b] = hp.p[b] = hp.Y[b] = nullptr;
      hp.st[b] = nullptr;
      e = dalloc(&hp.T[b], chunk);
      if (e == cudaSuccess) e = dalloc(&hp.p[b], chunk);
      if (e == cudaSuccess) e = dalloc(&hp.Y[b], (size_t)n * chunk);
      if (e == cudaSuccess) e = dalloc(&hp.st[b], chunk);
    }
    if (e == cudaSuccess && !hp.total) e = dalloc(&hp.total, 1);
    if (e == cudaSuccess && !hp.in) e = cudaStreamCreateWithFlags(&hp.in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !hp.out) e = cudaStreamCreateWithFlags(&hp.out, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      if (!hp.ev_in[b]) e = cudaEventCreateWithFlags(&hp.ev_in[b], cudaEventDisableTiming);
      if (e == cudaSuccess && !hp.ev_done[b])
        e = cudaEventCreateWithFlags(&hp.ev_done[b], cudaEventDisableTiming);
      if (e == cudaSuccess && !hp.ev_out[b])
        e = cudaEventCreateWithFlags(&hp.ev_out[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !hp.ev_start) e = cudaEventCreateWithFlags(&hp.ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      hp.chunk = 0;
      return cuda_fail(s, e, "host-step buffers");
    }
    hp.chunk = chunk;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t ld = hp.chunk;
  // the copies start behind the work already on the caller's stream
  e = cudaEventRecord(hp.ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.in, hp.ev_start, 0);
  int64_t nchunks = 0;
  for (int64_t c0 = 0; nchunks < (int64_t)plan.size() && e == cudaSuccess;
       c0 += plan[nchunks], ++nchunks) {
    const int b = (int)(nchunks & 1);
    const int64_t len = plan[nchunks];
    // upload into buffer b once its previous download has finished
    e = cudaStreamWaitEvent(hp.in, hp.ev_out[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.T[b], T + c0, sizeof(double) * len, cudaMemcpyHostToDevice, hp.in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.p[b], p + c0, sizeof(double) * len, cudaMemcpyHostToDevice, hp.in);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(hp.Y[b], sizeof(double) * ld, Y + c0, sizeof(double) * ldY,
                            sizeof(double) * len, (size_t)n, cudaMemcpyHostToDevice, hp.in);
    if (e == cudaSuccess) e = cudaEventRecord(hp.ev_in[b], hp.in);
    // the step on the caller's stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, hp.ev_in[b], 0);
    if (e != cudaSuccess) break;
    rc = run_step(s, len, dt, hp.T[b], hp.p[b], hp.Y[b], ld, hp.st[b], nullptr, st, nullptr,
                  nchunks > 0);
    if (rc != DF_OK) return rc;
    add_count_kernel<<<1, 1, 0, st>>>(s->d_count, hp.total, nchunks == 0 ? 1 : 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(hp.ev_done[b], st);
    // download once the step is done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.out, hp.ev_done[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T + c0, hp.T[b], sizeof(double) * len, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Y + c0, sizeof(double) * ldY, hp.Y[b], sizeof(double) * ld,
                            sizeof(double) * len, (size_t)n, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess && cell_status)
      e = cudaMemcpyAsync(cell_status + c0, hp.st[b], sizeof(int32_t) * len, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess) e = cudaEventRecord(hp.ev_out[b], hp.out);
  }
  // the caller's stream continues after the last download; the summary covers all chunks
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, hp.ev_out[(nchunks - 1) & 1], 0);
  if (e == cudaSuccess && nchunks > 1) e = cudaStreamWaitEvent(st, hp.ev_out[nchunks & 1], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_count, hp.total, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "host step");
}

df_status df_chem_source(df_state* s, int64_t n_cells, double dt, const double* T,
                         const double* p, const double* Y, int64_t ldY, double* omega, int64_t ldw,
                         double* T_new, int32_t* cell_status, int64_t* n_active_out, void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK) return rc;
  if (n_cells > 0 && !omega) return fail(s, DF_ERR_INVALID_ARG, "omega is NULL");
  if (n_cells > 0 && ldw < n_cells) return fail(s, DF_ERR_INVALID_ARG, "ldw < n_cells");
  if (!(std::fabs(dt - s->dt) <= 1e-12 * std::fabs(s->dt)))
    return fail(s, DF_ERR_DT_MISMATCH, "dt %.17g differs from the network's %.17g", dt, s->dt);
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  // cells that do not react (or get flagged) keep omega = 0 and T' = T
  cudaError_t e = cudaSuccess;
  if (n_cells > 0) {
    e = cudaMemset2DAsync(omega, sizeof(double) * ldw, 0, sizeof(double) * n_cells, (size_t)s->n, st);
    if (e == cudaSuccess && T_new)
      e = cudaMemcpyAsync(T_new, T, sizeof(double) * n_cells, cudaMemcpyDeviceToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "source-term initialisation");
  const Source src{omega, ldw, s->rho_row, 1.0 / dt, T_new};
  return run_step(s, n_cells, dt, const_cast<double*>(T), p, const_cast<double*>(Y), ldY,
                  cell_status, n_active_out, st, &src);
}

// Builds the Jacobian context: buffers for B cells, BF16 weights and tensor maps when the
// state's network runs on tensor cores.
df_status build_jac(df_state* s) {
  Jac* j = new Jac();
  const int L = s->L, n = s->n, ntan = n + 1;
  j->bf16 = s->precision != DF_FP32;
  j->eb = j->bf16 ? 2 : 4;
  j->B = std::min<int64_t>(s->cap, 65536);
  const int64_t B = j->B, R = B * ntan;
  const int64_t al = j->bf16 ? 16 : 8;
  cudaError_t e = cudaSuccess;
  auto al_ok = [&](void** p, size_t bytes, bool zero) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess && zero) e = cudaMemset(*p, 0, bytes ? bytes : 1);
  };
  j->ldx = round_up(s->K0, al);
  al_ok(&j->x, j->eb * B * j->ldx, true);
  int64_t wmax[2] = {al, al}, tmax = al;
  for (int l = 0; l + 1 < L; ++l) {
    wmax[l & 1] = std::max<int64_t>(wmax[l & 1], round_up(s->widths[l + 1], al));
    tmax = std::max<int64_t>(tmax, round_up(s->widths[l + 1], al));
  }
  for (int b = 0; b < 2; ++b) {
    j->act_ld[b] = wmax[b];
    al_ok(&j->act[b], j->eb * B * wmax[b], true);
    j->tan_ld[b] = tmax;
    al_ok(&j->tan[b], j->eb * R * tmax, true);
  }
  for (int l = 0; l + 1 < L; ++l) {
    void* g = nullptr;
    const int64_t ld = round_up(s->widths[l + 1], 32);
    al_ok(&g, j->eb * B * ld, true);
    j->G.push_back(g);
    j->ldg.push_back(ld);
  }
  j->ldo = s->ldo;
  al_ok((void**)&j->O, sizeof(float) * B * j->ldo, true);
  al_ok((void**)&j->dO, sizeof(float) * R * j->ldo, true);
  al_ok((void**)&j->h0, sizeof(double) * B, false);
  al_ok((void**)&j->sc, sizeof(float) * R, false);
  al_ok((void**)&j->jscr, sizeof(double) * B * (5 * n + 2), false);
  al_ok((void**)&j->jst, sizeof(int32_t) * B, false);
  int64_t zmax = 32;
  for (int l = 0; l < L; ++l) zmax = std::max<int64_t>(zmax, round_up(s->widths[l + 1], 32));
  al_ok((void**)&j->zero_bias, sizeof(float) * zmax, true);
  // layer-1 weights as the Jacobian's network holds them, transposed [K0 x N1]
  const int N1 = s->widths[1], K0 = s->K0;
  std::vector<float> w1t((size_t)K0 * N1);
  for (int r = 0; r < N1; ++r)
    for (int c = 0; c < K0; ++c) {
      float v = s->Wh[0][(size_t)r * K0 + c];
      if (j->bf16) v = __bfloat162float(__float2bfloat16_rn(v));
      w1t[(size_t)c * N1 + r] = v;
    }
  al_ok((void**)&j->W1T, sizeof(float) * w1t.size(), false);
  if (e == cudaSuccess)
    e = cudaMemcpy(j->W1T, w1t.data(), sizeof(float) * w1t.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_jac(j);
    return cuda_fail(s, e, "Jacobian buffers");
  }
  if (!j->bf16) {
    j->W32 = s->W32;
    j->Kp = s->Kp8;
  } else {
    // BF16 weights: the state's own for a BF16 network, fresh copies for an FP8 one
    for (int l = 0; l < L; ++l) {
      const int Kl = s->widths[l], Nl = s->widths[l + 1];
      const int kp = (int)round_up(Kl, 16);
      j->Kp.push_back(kp);
      if (s->precision == DF_BF16) {
        j->Wb.push_back(nullptr);
        continue;
      }
      std::vector<__nv_bfloat16> w((size_t)Nl * kp, __float2bfloat16_rn(0.0f));
      for (int r = 0; r < Nl; ++r)
        for (int c = 0; c < Kl; ++c) w[(size_t)r * kp + c] = __float2bfloat16_rn(s->Wh[l][(size_t)r * Kl + c]);
      void* d = nullptr;
      al_ok(&d, 2 * w.size(), false);
      if (e == cudaSuccess) e = cudaMemcpy(d, w.data(), 2 * w.size(), cudaMemcpyHostToDevice);
      j->Wb.push_back(d);
      if (e != cudaSuccess) {
        free_jac(j);
        return cuda_fail(s, e, "Jacobian weights");
      }
    }
    char emsg[256];
    for (int l = 0; l < L; ++l) {
      const bool last = l == L - 1;
      const void* Wl = s->precision == DF_BF16 ? s->Wlp[l] : j->Wb[l];
      // forward pass: hidden layers also store GELU'(z); the read-out is plain
      TcLayer F{};
      F.N = s->widths[l + 1];
      F.K = s->widths[l];
      const int tile = pick_tile(F.N, F.K, !last, last ? kXF32 : kXBF16, true);
      F.BN = tile & ~DF_TILE_PAIR;
      F.pair = (tile & DF_TILE_PAIR) != 0;
      F.bias = s->bias[l];
      F.out = last ? (void*)j->O : j->act[l & 1];
      F.ldo = last ? j->ldo : j->act_ld[l & 1];
      F.out_kind = last ? kXF32 : kXBF16;
      F.gelu = !last;
      F.out_scale = 1.0f;
      F.elem_bytes = 2;
      F.mode = last ? 0 : 1;
      F.gbuf = last ? nullptr : j->G[l];
      F.ldg = last ? 0 : j->ldg[l];
      F.ntan = 1;
      const void* Af = (l == 0) ? j->x : j->act[(l - 1) & 1];
      const int64_t ldaf = (l == 0) ? j->ldx : j->act_ld[(l - 1) & 1];
      bool ok = tc_encode_2d(&F.tmA, Af, 2, (uint64_t)F.K, (uint64_t)B, (uint64_t)ldaf * 2, 64, 128,
                             emsg, sizeof emsg) &&
                tc_encode_2d(&F.tmB, Wl, 2, (uint64_t)F.K, (uint64_t)F.N, (uint64_t)j->Kp[l] * 2, 64,
                             (uint32_t)(F.pair ? F.BN / 2 : F.BN), emsg, sizeof emsg) &&
                tc_encode_out(F, (uint64_t)B, emsg, sizeof emsg);
      // tangent pass of layers 1.. (layer 0's tangents come from jac_tangent0)
      TcLayer Tg = F;
      Tg.bias = j->zero_bias;
      Tg.out = last ? (void*)j->dO : j->tan[l & 1];
      Tg.ldo = last ? j->ldo : j->tan_ld[l & 1];
      Tg.gelu = false;
      Tg.mode = last ? 0 : 2;
      Tg.ntan = ntan;
      if (ok && l > 0)
        ok = tc_encode_2d(&Tg.tmA, j->tan[(l - 1) & 1], 2, (uint64_t)Tg.K, (uint64_t)R,
                          (uint64_t)j->tan_ld[(l - 1) & 1] * 2, 64, 128, emsg, sizeof emsg);
      if (ok) ok = tc_encode_out(Tg, (uint64_t)R, emsg, sizeof emsg);
      if (!ok) {
        free_jac(j);
        return fail(s, DF_ERR_CUDA, "%s", emsg);
      }
      j->fwd.push_back(F);
      j->tng.push_back(Tg);
      if ((e = prepare_tc(F)) != cudaSuccess || (e = prepare_tc(Tg)) != cudaSuccess) {
        free_jac(j);
        return cuda_fail(s, e, "kernel attributes");
      }
    }
  }
  s->jac = j;
  return DF_OK;
}

struct df_graph {
  df_state* s = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

df_status df_graph_create(df_state* s, int64_t n_cells, double dt, double* T, const double* p,
                          double* Y, int64_t ldY, int32_t* cell_status, int64_t* n_active_out,
                          df_graph** out) {
  if (!out) return fail(s, DF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK) return rc;
  DeviceGuard guard(s->device);
  // everything that may allocate or set function attributes happens outside the capture
  if ((rc = ensure_compact(s, n_cells)) != DF_OK) return rc;
  const bool prof = s->prof_on;
  s->prof_on = false;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    s->prof_on = prof;
    return cuda_fail(s, e, "capture stream");
  }
  // kernel attributes were set by df_state_create, so the capture records launches only
  df_graph* g = new df_graph();
  g->s = s;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = df_chem_step(s, n_cells, dt, T, p, Y, ldY, cell_status, n_active_out, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
    if (rc == DF_OK && e2 != cudaSuccess) rc = cuda_fail(s, e2, "end capture");
  } else {
    rc = cuda_fail(s, e, "begin capture");
  }
  if (rc == DF_OK) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(s, e, "graph instantiate");
  }
  cudaStreamDestroy(cs);
  s->prof_on = prof;
  if (rc != DF_OK) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return rc;
  }
  *out = g;
  return DF_OK;
}

df_status df_graph_launch(df_graph* g, void* stream) {
  if (!g) return fail(nullptr, DF_ERR_INVALID_ARG, "graph is NULL");
  DeviceGuard guard(g->s->device);
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(g->s, e, "graph launch");
}

void df_graph_destroy(df_graph* g) {
  if (!g) return;
  DeviceGuard guard(g->s->device);
  cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

df_status df_chem_jacobian(df_state* s, int64_t n_cells, const double* T, const double* p,
                           const double* Y, int64_t ldY, float* J_dY, double* dTnew, void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  if (!J_dY) return fail(s, DF_ERR_INVALID_ARG, "J_dY is NULL");
  if (s->L < 2) return fail(s, DF_ERR_UNSUPPORTED, "the Jacobian needs at least one hidden layer");
  if (s->gelu_mode != DF_GELU_TANH)
    return fail(s, DF_ERR_UNSUPPORTED, "the Jacobian needs the tanh-form GELU (DF_GELU_TANH)");
  DeviceGuard guard(s->device);
  if (s->jac && s->jac->wver != s->wver) {  // training changed the weights
    cudaDeviceSynchronize();
    free_jac(s->jac);
    s->jac = nullptr;
  }
  if (!s->jac) {
    if ((rc = sync_host_weights(s)) != DF_OK || (rc = build_jac(s)) != DF_OK) return rc;
    s->jac->wver = s->wver;
  }
  Jac* j = s->jac;
  cudaStream_t st = (cudaStream_t)stream;
  const int L = s->L, ntan = s->n + 1;
  cudaError_t e = cudaSuccess;
  for (int64_t c0 = 0; c0 < n_cells && e == cudaSuccess; c0 += j->B) {
    const int64_t nb = std::min<int64_t>(j->B, n_cells - c0);
    const RowMap cells{nullptr, nullptr, c0, nb};
    const RowMap rows{nullptr, nullptr, 0, nb};
    const RowMap trows{nullptr, nullptr, 0, nb * ntan};
    e = launch_eos_pre(s->P, cells, T, p, Y, ldY, j->h0, nullptr, j->x, j->bf16 ? kXBF16 : kXF32,
                       j->ldx, 1.0f, nullptr, st);
    // forward pass with GELU' of every hidden layer
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
      const bool last = l == L - 1;
      if (j->bf16) {
        e = launch_tc_gemm(j->fwd[l], rows, s->num_sms, s->d_err, st);
      } else {
        const float* A = (l == 0) ? (const float*)j->x : (const float*)j->act[(l - 1) & 1];
        const int64_t lda = (l == 0) ? j->ldx : j->act_ld[(l - 1) & 1];
        e = launch_sgemm_bias_act(rows, s->widths[l + 1], j->Kp[l], A, lda, j->W32[l], j->Kp[l],
                                  s->bias[l], last ? j->O : (float*)j->act[l & 1],
                                  last ? j->ldo : j->act_ld[l & 1], !last, s->num_sms, st,
                                  last ? 0 : 1, last ? nullptr : (float*)j->G[l],
                                  last ? 0 : j->ldg[l], 1);
      }
    }
    // tangents: layer 0 directly, then GEMMs scaled by GELU' per cell
    if (e == cudaSuccess) e = launch_jac_scale(s->P, nb, Y + c0, ldY, j->sc, st);
    if (e == cudaSuccess)
      e = launch_jac_tangent0(nb, ntan, s->widths[1], j->sc, j->W1T, j->G[0], j->ldg[0], j->bf16,
                              L > 1 ? j->tan[0] : (void*)j->dO, j->tan_ld[0], st);
    for (int l = 1; l < L && e == cudaSuccess; ++l) {
      const bool last = l == L - 1;
      if (j->bf16) {
        e = launch_tc_gemm(j->tng[l], trows, s->num_sms, s->d_err, st);
      } else {
        e = launch_sgemm_bias_act(trows, s->widths[l + 1], j->Kp[l], (const float*)j->tan[(l - 1) & 1],
                                  j->tan_ld[(l - 1) & 1], j->W32[l], j->Kp[l], j->zero_bias,
                                  last ? j->dO : (float*)j->tan[l & 1], last ? j->ldo : j->tan_ld[l & 1],
                                  false, s->num_sms, st, last ? 0 : 2,
                                  last ? nullptr : (float*)j->G[l], last ? 0 : j->ldg[l], ntan);
      }
    }
    if (e == cudaSuccess)
      e = launch_jac_post(s->P, nb, c0, T, p, Y, ldY, j->O, j->ldo, j->dO, j->ldo, j->h0, J_dY,
                          dTnew, j->jscr, j->jst, st);
  }
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "Jacobian");
}

df_status df_chem_step_vjp(df_state* s, int64_t n_cells, const double* T, const double* p,
                           const double* Y, int64_t ldY, const double* gT, const double* gY,
                           int64_t ldg, double* out_gT, double* out_gY, int64_t ldo,
                           void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  if (!gT || !gY || !out_gT || !out_gY) return fail(s, DF_ERR_INVALID_ARG, "NULL cotangent pointer");
  if (ldg < n_cells || ldo < n_cells)
    return fail(s, DF_ERR_INVALID_ARG, "ldg (%lld) or ldo (%lld) < n_cells (%lld)", (long long)ldg,
                (long long)ldo, (long long)n_cells);
  DeviceGuard guard(s->device);
  const int n = s->n, ntan = n + 1;
  // batches of the Jacobian's own batch size, so that each Jacobian call below is one batch
  const int64_t B = std::min<int64_t>(s->cap, 65536);
  if (s->vjp_cap < B) {
    cudaDeviceSynchronize();
    if (s->vjpJ) cudaFree(s->vjpJ);
    if (s->vjpT) cudaFree(s->vjpT);
    s->vjpJ = nullptr;
    s->vjpT = nullptr;
    s->vjp_cap = 0;
    cudaError_t e = cudaMalloc(&s->vjpJ, sizeof(float) * (size_t)B * n * ntan);
    if (e == cudaSuccess) e = cudaMalloc(&s->vjpT, sizeof(double) * (size_t)B * ntan);
    if (e != cudaSuccess) {
      if (s->vjpJ) cudaFree(s->vjpJ);
      s->vjpJ = nullptr;
      s->vjpT = nullptr;
      cudaGetLastError();
      return fail(s, DF_ERR_OOM, "Jacobian columns of one batch (%lld cells)", (long long)B);
    }
    s->vjp_cap = B;
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int64_t c0 = 0; c0 < n_cells; c0 += B) {
    const int64_t nb = std::min<int64_t>(B, n_cells - c0);
    rc = df_chem_jacobian(s, nb, T + c0, p + c0, Y + c0, ldY, s->vjpJ, s->vjpT, stream);
    if (rc != DF_OK) return rc;
    const cudaError_t e = launch_step_vjp(n, nb, s->T_react, T + c0, s->vjpJ, s->vjpT, gT + c0,
                                          gY + c0, ldg, out_gT + c0, out_gY + c0, ldo, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "reverse-mode product of the step");
  }
  return DF_OK;
}

// ---- tile-width autotuning ----

}  // extern "C"

namespace {

// Re-encodes layer l's weight map for tile `tile` (BN, | DF_TILE_PAIR for CTA pairs: the only
// part of a layer that depends on it) and sets the kernel instance's attributes.
df_status retile(df_state* s, int l, int tile) {
  TcLayer& T = s->tcl[l];
  const size_t eb = elem_of(s->precision);
  const int bn = tile & ~DF_TILE_PAIR;
  const bool pair = (tile & DF_TILE_PAIR) != 0;
  char emsg[256];
  if (!tc_encode_2d(&T.tmB, s->Wlp[l], (int)eb, (uint64_t)T.K, (uint64_t)T.N,
                    (uint64_t)s->Kp8[l] * eb, 128 / (uint32_t)eb, (uint32_t)(pair ? bn / 2 : bn),
                    emsg, sizeof emsg))
    return fail(s, DF_ERR_CUDA, "%s", emsg);
  T.BN = bn;
  T.pair = pair;
  cudaError_t e = prepare_tc(T);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "kernel attributes");
}

std::string tile_key(const df_state* s, int l, const char* dev) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s %d %d %d %d", dev, s->precision, s->widths[l], s->widths[l + 1],
           l == s->L - 1 ? 1 : 0);
  return buf;
}

}  // namespace

extern "C" {

df_status df_autotune(df_state* s, int64_t n_rows, const char* cache_path, void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (n_rows < 0) return fail(s, DF_ERR_INVALID_ARG, "n_rows < 0");
  if (s->precision == DF_FP32) return DF_OK;  // the SIMT layers have a single tiling
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, s->device);
  std::string dev = prop.name;
  for (char& ch : dev)
    if (ch == ' ' || ch == '\t') ch = '_';
  // cache: one line per layer shape, "<device> <precision> <K> <N> <last> <BN>"
  std::vector<std::pair<std::string, int>> cache;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[600];
      while (std::fgets(line, sizeof line, f)) {
        char d[512];
        int prec, K, N, last, bn;
        if (std::sscanf(line, "%511s %d %d %d %d %d", d, &prec, &K, &N, &last, &bn) == 6) {
          char key[600];
          snprintf(key, sizeof key, "%s %d %d %d %d", d, prec, K, N, last);
          cache.emplace_back(key, bn);
        }
      }
      std::fclose(f);
    }
  }
  const int64_t rows = std::max<int64_t>(128, std::min<int64_t>(n_rows > 0 ? n_rows : s->cap, s->cap));
  const RowMap rm{nullptr, nullptr, 0, rows};
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  df_status rc = DF_OK;
  bool dirty = false;
  for (int l = 0; l < s->L && rc == DF_OK && e == cudaSuccess; ++l) {
    const bool last = l == s->L - 1;
    const std::string key = tile_key(s, l, dev.c_str());
    int chosen = 0;
    for (auto& kv : cache)
      if (kv.first == key) chosen = kv.second;
    static const int hid[] = {64, 128, 160, 192, 224, 256, 160 | DF_TILE_PAIR,
                              224 | DF_TILE_PAIR, 256 | DF_TILE_PAIR};
    static const int rd[] = {32, 64};
    const bool one_kblock = s->tcl[l].K * (int)elem_of(s->precision) <= 128;
    const int* cand = last ? rd : hid;
    const int nc = last ? 2 : (one_kblock ? 6 : 9);
    bool known = false;
    for (int i = 0; i < nc; ++i) known = known || cand[i] == chosen;
    if (!known) {
      float best = 1e30f;
      for (int i = 0; i < nc && rc == DF_OK && e == cudaSuccess; ++i) {
        if ((rc = retile(s, l, cand[i])) != DF_OK) break;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_tc_gemm(s->tcl[l], rm, s->num_sms, s->d_err, st);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch_tc_gemm(s->tcl[l], rm, s->num_sms, s->d_err, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms < best) {
          best = ms;
          chosen = cand[i];
        }
      }
      cache.emplace_back(key, chosen);
      dirty = true;
    }
    if (rc == DF_OK && e == cudaSuccess) rc = retile(s, l, chosen);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(s, e, "autotune");
  if (rc != DF_OK) return rc;
  if (dirty && cache_path) {
    FILE* f = std::fopen(cache_path, "w");
    if (!f) return fail(s, DF_ERR_INVALID_ARG, "cannot write %s", cache_path);
    for (auto& kv : cache) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    std::fclose(f);
  }
  return DF_OK;
}

df_status df_get_tiles(df_state* s, int32_t* bn, int32_t max_layers, int32_t* n_layers) {
  if (!s || !n_layers || (max_layers > 0 && !bn)) return fail(s, DF_ERR_INVALID_ARG, "bad arguments");
  *n_layers = s->L;
  for (int l = 0; l < s->L && l < max_layers; ++l)
    bn[l] = s->tcl.empty() ? 0 : (s->tcl[l].BN | (s->tcl[l].pair ? DF_TILE_PAIR : 0));
  return DF_OK;
}

df_status df_set_wait_limit(df_state* s, int64_t clocks) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (s->tcl.empty()) return fail(s, DF_ERR_UNSUPPORTED, "the state has no tensor-core layers");
  for (TcLayer& L : s->tcl) L.wait_budget = clocks > 0 ? (long long)clocks : 0;
  s->f01.wait_budget = clocks > 0 ? (long long)clocks : 0;
  return DF_OK;
}

df_status df_get_step_summary(df_state* s, void* stream, df_step_stats* stats) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  DeviceGuard guard(s->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  int64_t c = 0, f = 0, it = 0;
  int err = 0;
  if ((e = cudaMemcpy(&c, s->d_count, sizeof c, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&f, s->d_flagged, sizeof f, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&it, s->d_iters, sizeof it, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&err, s->d_err, sizeof err, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(s, e, "summary read");
  if (stats) {
    stats->n_active = c;
    stats->n_flagged = f;
    stats->newton_iterations = it;
  }
  if (err & kErrTimeout) {
    cudaMemset(s->d_err, 0, sizeof(int));
    return fail(s, DF_ERR_TIMEOUT, "a kernel wait hit its time limit");
  }
  if (f > 0) return fail(s, DF_ERR_NOT_CONVERGED, "%lld cells were flagged", (long long)f);
  return DF_OK;
}

df_status df_active_compact(df_state* s, int64_t n_cells, const double* T, int32_t* idx,
                            int64_t* count, void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (n_cells < 0 || !count || (n_cells > 0 && (!T || !idx)))
    return fail(s, DF_ERR_INVALID_ARG, "bad arguments");
  if (n_cells > (int64_t)INT32_MAX)
    return fail(s, DF_ERR_INVALID_ARG, "n_cells exceeds INT32_MAX (the cell indices are int32)");
  DeviceGuard guard(s->device);
  df_status rc = ensure_compact(s, n_cells);
  if (rc != DF_OK) return rc;
  cudaError_t e = launch_compact(n_cells, s->T_react, T, idx, count, nullptr, s->cscr,
                                 (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "compaction");
}

df_status df_eos_pre(df_state* s, int64_t n_cells, const double* T, const double* p,
                     const double* Y, int64_t ldY, double* h0, double* Z, float* x,
                     int32_t* status, void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  DeviceGuard guard(s->device);
  const RowMap rm{nullptr, nullptr, 0, n_cells};
  cudaError_t e = launch_eos_pre(s->P, rm, T, p, Y, ldY, h0, Z, x, kXF32, s->K0, 1.0f, status,
                                 (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "eos_pre");
}

df_status df_mlp_forward(df_state* s, int64_t n_rows, const float* x, float* O, void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (n_rows < 0 || (n_rows > 0 && (!x || !O))) return fail(s, DF_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int xk = xkind_of(s->precision);
  const float xs = s->precision == DF_FP8_E4M3 ? s->act_scale[0] : 1.0f;
  for (int64_t r0 = 0; r0 < n_rows; r0 += s->cap) {
    const int64_t rows = std::min<int64_t>(s->cap, n_rows - r0);
    const int64_t total = rows * s->ldx;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)s->num_sms * 16);
    cast_rows_kernel<<<g, 256, 0, st>>>(rows, s->K0, x + r0 * s->K0, s->K0, s->x, s->ldx, xk, xs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "input cast");
    const RowMap rm{nullptr, nullptr, 0, rows};
    df_status rc = run_mlp(s, rm, st);
    if (rc != DF_OK) return rc;
    e = cudaMemcpy2DAsync(O + r0 * s->nout, sizeof(float) * s->nout, s->O, sizeof(float) * s->ldo,
                          sizeof(float) * s->nout, (size_t)rows, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "output copy");
  }
  return DF_OK;
}

df_status df_propnet_infer(df_state* s, int64_t n_cells, const double* h, const double* p,
                           const double* Y, int64_t ldY, double* out, int64_t ldout,
                           void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (!s->netonly) return fail(s, DF_ERR_UNSUPPORTED, "not a network-only state (df_network_create)");
  if (n_cells < 0) return fail(s, DF_ERR_INVALID_ARG, "n_cells < 0");
  if (n_cells == 0) return DF_OK;
  if (!h || !p || !Y || !out) return fail(s, DF_ERR_INVALID_ARG, "NULL array");
  if (ldY < n_cells || ldout < n_cells) return fail(s, DF_ERR_INVALID_ARG, "ldY or ldout < n_cells");
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int xk = xkind_of(s->precision);
  for (int64_t r0 = 0; r0 < n_cells; r0 += s->cap) {
    const int64_t rows = std::min<int64_t>(s->cap, n_cells - r0);
    cudaError_t e;
    {
      ProfScope ps(s, "prop_inputs", st);
      e = launch_prop_inputs(s->d_norm, s->n, s->lambda, rows, h + r0, p + r0, Y + r0, ldY, s->x,
                             s->ldx, xk, s->num_sms, st);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "property-network inputs");
    const RowMap rm{nullptr, nullptr, 0, rows};
    df_status rc = run_mlp(s, rm, st);
    if (rc != DF_OK) return rc;
    {
      ProfScope ps(s, "prop_outputs", st);
      e = launch_prop_outputs(s->d_norm, s->K0, s->nout, rows, s->O, s->ldo, out + r0, ldout,
                              s->num_sms, st);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "property-network outputs");
  }
  return DF_OK;
}

df_status df_eos_post(df_state* s, int64_t n_cells, const float* O, const double* h0,
                      double* T, const double* p, double* Y, int64_t ldY, int32_t* status,
                      void* stream) {
  df_status rc = check_fields(s, n_cells, T, p, Y, ldY);
  if (rc != DF_OK || n_cells == 0) return rc;
  if (!O || !h0) return fail(s, DF_ERR_INVALID_ARG, "NULL O or h0");
  DeviceGuard guard(s->device);
  const RowMap rm{nullptr, nullptr, 0, n_cells};
  cudaError_t e = launch_eos_post(s->P, rm, O, s->n, h0, T, p, Y, ldY, nullptr, status,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "eos_post");
}

df_status df_profile_enable(df_state* s, int32_t enable) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  s->prof_on = enable != 0;
  return DF_OK;
}

df_status df_profile_read(df_state* s, int32_t max_entries, char* names, int64_t* launches,
                          double* total_ms, int32_t* n_entries) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (max_entries < 0 || (max_entries > 0 && (!names || !launches || !total_ms)) || !n_entries)
    return fail(s, DF_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(s->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(s, e, "device synchronize");
  for (auto& r : s->prof_recs) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      s->prof_launches[r.fam] += 1;
      s->prof_ms[r.fam] += ms;
    }
    s->prof_pool.push_back(r.a);
    s->prof_pool.push_back(r.b);
  }
  s->prof_recs.clear();
  const int n = (int)std::min<size_t>(s->prof_names.size(), (size_t)max_entries);
  for (int i = 0; i < n; ++i) {
    snprintf(names + 32 * i, 32, "%s", s->prof_names[i].c_str());
    launches[i] = s->prof_launches[i];
    total_ms[i] = s->prof_ms[i];
  }
  *n_entries = n;
  std::fill(s->prof_launches.begin(), s->prof_launches.end(), 0);
  std::fill(s->prof_ms.begin(), s->prof_ms.end(), 0.0);
  return DF_OK;
}

}  // extern "C"
