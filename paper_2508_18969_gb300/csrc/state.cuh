// Host-side internals of libdfgb shared by the entry-point files (state.cu, train_api.cu):
// the opaque df_state, its Jacobian and training contexts, and small helpers.
#pragma once

#include "dfgb_internal.cuh"
#include "../../include/df.h"

#include <string>
#include <vector>

using namespace dfgb;

struct Trn;   // training context (train_api.cu)

struct Jac {
  int64_t B = 0;                         // cells per Jacobian batch
  bool bf16 = false;                     // BF16 tensor-core passes (else FP32 SIMT)
  size_t eb = 4;
  void* x = nullptr;
  int64_t ldx = 0;
  void* act[2] = {nullptr, nullptr};
  int64_t act_ld[2] = {0, 0};
  std::vector<void*> G;                  // GELU'(z) of each hidden layer [B x ldg]
  std::vector<int64_t> ldg;
  void* tan[2] = {nullptr, nullptr};     // tangent activations [B (n+1) x tan_ld]
  int64_t tan_ld[2] = {0, 0};
  float* O = nullptr;
  int64_t ldo = 0;
  float* dO = nullptr;
  double* h0 = nullptr;
  float* sc = nullptr;
  double* jscr = nullptr;                // per-cell results between the two post kernels
  int32_t* jst = nullptr;                // [B (5n + 2)] and [B]
  float* W1T = nullptr;
  float* zero_bias = nullptr;
  std::vector<void*> Wb;                 // BF16 weights owned here (FP8 states)
  std::vector<float*> W32;               // FP32 weights (SIMT), shared with the state
  std::vector<int> Kp;
  std::vector<TcLayer> fwd, tng;
  int64_t wver = 0;                      // weight version the context was built from
};

struct df_state {
  int device = 0;
  int num_sms = 0;
  int n = 0, K0 = 0, L = 0;
  int nout = 0;                          // network outputs (n for the chemistry network)
  bool netonly = false;                  // created by df_network_create: no mechanism
  std::vector<int> widths;
  int precision = DF_FP32;
  double T_react = 0, lambda = 0.1, dt = 0;
  int64_t cap = 0;                       // rows per batch
  EosParams P{};
  double* d_spc = nullptr;
  double* d_K = nullptr;
  double* d_norm = nullptr;
  float* d_spc2 = nullptr;               // double-float mixing-sum tables (EosParams)
  float* d_K4 = nullptr;
  float* d_kcol = nullptr;
  float* d_kf2 = nullptr;                // FP32 k_ij pair table (EosParams)
  double* d_lntab = nullptr;             // log table (EosParams)
  float* d_lntab2 = nullptr;             // the log table in double-float pairs
  double* d_tsp = nullptr;               // transport species constants (EosParams)
  float* d_tpair = nullptr;              // transport pair tables (EosParams)
  int gelu_mode = 0;                     // DF_GELU_TANH or DF_GELU_TABLE
  float4* d_gtab = nullptr;              // tabulated GELU (DF_GELU_TABLE)
  int* d_err = nullptr;                  // kernel error word
  int64_t* d_count = nullptr;            // reacting cells of the last step
  // df_chem_step_host: device buffers of two chunks, copy streams and their events
  struct HostPipe {
    int64_t chunk = 0;
    double* T[2] = {nullptr, nullptr};
    double* p[2] = {nullptr, nullptr};
    double* Y[2] = {nullptr, nullptr};
    int32_t* st[2] = {nullptr, nullptr};
    int64_t* total = nullptr;            // reacting cells summed over the chunks
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_out[2] = {nullptr, nullptr}, ev_start = nullptr;
  } hp;
  int64_t* d_flagged = nullptr;          // flagged cells of the last step
  int64_t* d_iters = nullptr;            // Newton iterations of the last step
  std::vector<float*> W32;               // FP32 weights, [N x Kp8] zero padded (SIMT)
  std::vector<int> Kp8;
  std::vector<float*> bias;
  std::vector<void*> Wlp;                // BF16 / FP8 weights [N x Kp16]
  std::vector<float*> col_scale;         // FP8 dequantisation scale per output channel
  std::vector<float> act_scale;          // FP8 quantisation scale of each layer's input
  // batch scratch
  void* x = nullptr;
  int64_t ldx = 0;
  void* act[2] = {nullptr, nullptr};
  int64_t act_ld[2] = {0, 0};
  float* O = nullptr;
  int64_t ldo = 0;
  double* h0 = nullptr;
  double* rho_row = nullptr;             // density of each row (source terms)
  int32_t* rstat = nullptr;
  // compaction scratch, grown on demand
  int32_t* idx = nullptr;
  int64_t idx_cap = 0;
  int64_t* cscr = nullptr;
  int64_t cscr_words = 0;
  std::vector<TcLayer> tcl;
  bool fuse01 = false;                   // layers 0 and 1 run as one fused kernel (f01)
  F01Layer f01;
  std::vector<std::vector<float>> Wh;    // host copies of the FP32 weights (Jacobian set-up)
  struct Jac* jac = nullptr;             // Jacobian context, built at the first Jacobian call
  // one batch of Jacobian columns for df_chem_step_vjp, allocated at its first call
  float* vjpJ = nullptr;                 // [vjp_cap][n][n+1]
  double* vjpT = nullptr;                // [vjp_cap][n+1]
  int64_t vjp_cap = 0;
  Trn* trn = nullptr;                    // training context, built at the first training call
  int64_t wver = 0;                      // bumped whenever training changes the weights
  std::string err;
  // kernel timing (df_profile_enable / df_profile_read)
  bool prof_on = false;
  struct Rec { int fam; cudaEvent_t a, b; };
  std::vector<Rec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<std::string> prof_names;
  std::vector<int64_t> prof_launches;
  std::vector<double> prof_ms;
};


namespace dfgb {

// FP8 activations (network input and hidden layers) are stored as e4m3(v * 32): the inputs are
// Z-scores and the hidden activations GELU outputs, both O(1-10), so x32 keeps them between
// e4m3's smallest normal (2^-6) and its maximum (448).
constexpr float kFp8ActScale = 32.0f;

df_status fail(df_state* s, df_status code, const char* fmt, ...);
df_status cuda_fail(df_state* s, cudaError_t e, const char* where);
int xkind_of(int precision);
size_t elem_of(int precision);
cudaEvent_t prof_event(df_state* s);
int prof_family(df_state* s, const char* name);
df_status check_fields(df_state* s, int64_t n, const void* a, const void* b, const void* Y,
                       int64_t ldY);
// x (state precision, [rows x ldo]) = cast of the FP32 rows in [rows x ldi] (FP8: times scale)
cudaError_t launch_cast_rows(int64_t rows, int K, const float* in, int64_t ldi, void* out,
                             int64_t ldo, int kind, float scale, int num_sms, cudaStream_t st);
void free_jac(Jac* j);
void free_trn(Trn* t);
// Refreshes the host weight copies from the training masters when training changed them.
df_status sync_host_weights(df_state* s);
// Tile of a tensor-core layer of N outputs and K inputs: its width, | DF_TILE_PAIR when CTA
// pairs are allowed and cheaper.
int pick_tile(int N, int K, bool hidden, int out_kind, bool allow_pair);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

template <typename T>
inline cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

// Tile width of a layer: hidden layers from the compiled set {64, 128, 160, 224, 256}, the

// Brackets the launches made during its lifetime with events on `st` when timing is on.
struct ProfScope {
  df_state* s;
  cudaStream_t st;
  df_state::Rec r{};
  ProfScope(df_state* s_, const char* name, cudaStream_t st_) : s(s_), st(st_) {
    if (!s->prof_on) return;
    r.fam = prof_family(s, name);
    r.a = prof_event(s);
    r.b = prof_event(s);
    cudaEventRecord(r.a, st);
  }
  ~ProfScope() {
    if (!s->prof_on || !r.a) return;
    cudaEventRecord(r.b, st);
    s->prof_recs.push_back(r);
  }
};


}  // namespace dfgb
