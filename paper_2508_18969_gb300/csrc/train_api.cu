// C ABI of network training (include/df.h, "training"): the loss of the normalised network
// outputs against targets from a stiff integration, its gradients by a layer-by-layer
// backward pass and Adam updates of FP32 master weights, whose working copies (FP32 for the
// SIMT path, BF16 for the tensor-core path) the reaction step reads in place.
//
// Backward pass of layer l (Z_l = H_{l-1} W_l^T + b_l, H_l = GELU(Z_l), linear read-out):
//   dW_l = dZ_l^T H_{l-1}   (GEMM over the batch: both operands transposed first, so the
//                            batch becomes the contiguous reduction dimension)
//   db_l = column sums of dZ_l
//   dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})   (GEMM against the transposed weight copy, the
//                                             GELU' factor applied in its epilogue)
// Every step runs in the kernels of train.cu, mlp_simt.cu and mlp_tc.cu.
#include "state.cuh"
#include "../../include/df_propnet.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

struct Trn {
  // parameters and optimiser state, kept across batch-size changes
  std::vector<int64_t> ldw;              // row pitch of the [N_l x K_l] FP32 matrices
  std::vector<float*> Wm, mW, vW, dW;    // master weights, Adam moments, gradients
  std::vector<float*> mb, vb, db;        // bias moments and gradients (master = state bias)
  std::vector<void*> WT;                 // transposed working weights [K_l x ldt_l]
  std::vector<int64_t> ldt;
  int64_t t = 0;                         // Adam steps taken
  int64_t host_wver = 0;                 // weight version of the state's host copies
  float* loss = nullptr;                 // device loss of the last step
  float* scratch = nullptr;              // fixed-order reduction partials
  int64_t scratch_floats = 0;
  float* zero_bias = nullptr;
  // batch buffers for up to B rows
  int64_t B = 0, Bp = 0;                 // Bp = B rounded up to 64 (transposed length)
  int64_t ldT = 0;                       // pitch of the transposes: Bp + 64, so that rows of a
                                         // transpose are not a power of two apart in memory
  void* x = nullptr;
  int64_t ldx = 0;
  std::vector<void*> H, G, dZ;           // hidden outputs, GELU'(Z), output gradients
  std::vector<int64_t> ldh, ldg, ldz;
  float* O = nullptr;
  float* Oh = nullptr;
  int64_t ldo = 0;
  void* ZT = nullptr;                    // dZ_l^T [N_l x Bp]
  void* HT = nullptr;                    // H_{l-1}^T [K_l x Bp]
  float* dX = nullptr;                   // input gradient [B x lddx]
  float* dWp = nullptr;                  // split-K partial weight gradients [kMaxSplit x N x ldw]
  int64_t lddx = 0;
  double* h0 = nullptr;
  int32_t* rstat = nullptr;
  std::vector<TcLayer> fwd, dgrad, wgrad;  // tensor-core layers (BF16 states)
  int64_t rows = -1;                     // rows of the last training forward pass
};

namespace dfgb {

void free_trn(Trn* t) {
  if (!t) return;
  auto f = [](void* p) { if (p) cudaFree(p); };
  for (auto v : {&t->Wm, &t->mW, &t->vW, &t->dW, &t->mb, &t->vb, &t->db})
    for (float* p : *v) f(p);
  for (void* p : t->WT) f(p);
  f(t->loss); f(t->scratch); f(t->zero_bias);
  f(t->x); f(t->O); f(t->Oh); f(t->ZT); f(t->HT); f(t->dX); f(t->dWp); f(t->h0); f(t->rstat);
  for (auto v : {&t->H, &t->G, &t->dZ})
    for (void* p : *v) f(p);
  delete t;
}

}  // namespace dfgb

namespace {

bool trains(const df_state* s) {
  return (s->precision == DF_FP32 || s->precision == DF_BF16) && s->gelu_mode == DF_GELU_TANH;
}

constexpr int kMaxSplit = 16;   // split-K of the weight-gradient GEMMs

// Splits of a weight-gradient GEMM over the batch: about two waves of tiles on the GPU, no
// split empty (an empty split would store an uninitialised accumulator).
int wgrad_splits(int64_t tiles, int kblocks, int num_sms) {
  int S = (int)std::min<int64_t>(kMaxSplit, std::max<int64_t>(1, (2 * num_sms + tiles - 1) / tiles));
  S = std::min(S, std::max(1, kblocks / 8));
  while (S > 1 && (int64_t)(S - 1) * ((kblocks + S - 1) / S) >= kblocks) --S;
  return S;
}

void free_batch(Trn* t) {
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(t->x); f(t->O); f(t->Oh); f(t->ZT); f(t->HT); f(t->dX); f(t->dWp); f(t->h0); f(t->rstat);
  for (auto v : {&t->H, &t->G, &t->dZ})
    for (void* p : *v) f(p);
  t->x = t->ZT = t->HT = nullptr;
  t->O = t->Oh = t->dX = t->dWp = nullptr;
  t->h0 = nullptr;
  t->rstat = nullptr;
  t->H.clear(); t->G.clear(); t->dZ.clear();
  t->ldh.clear(); t->ldg.clear(); t->ldz.clear();
  t->fwd.clear(); t->dgrad.clear(); t->wgrad.clear();
  t->B = t->Bp = t->ldT = 0;
  t->rows = -1;
}

// Writes the working copies (state FP32 or BF16 weights, transposed copies) from the masters.
cudaError_t publish_all(df_state* s, cudaStream_t st) {
  Trn* t = s->trn;
  const bool bf16 = s->precision == DF_BF16;
  for (int l = 0; l < s->L; ++l) {
    cudaError_t e = launch_publish(s->widths[l + 1], s->widths[l], t->Wm[l], t->ldw[l],
                                   bf16 ? nullptr : s->W32[l], s->Kp8[l],
                                   bf16 ? s->Wlp[l] : nullptr, s->Kp8[l], t->WT[l], t->ldt[l],
                                   bf16, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Masters from the state's host weights, zero moments, transposed working copies.
df_status ensure_params(df_state* s) {
  if (s->trn) return DF_OK;
  if (!trains(s)) return fail(s, DF_ERR_UNSUPPORTED, "training needs a DF_FP32 or DF_BF16 state with DF_GELU_TANH");
  Trn* t = new Trn();
  s->trn = t;
  const bool bf16 = s->precision == DF_BF16;
  const size_t eb = bf16 ? 2 : 4;
  const int64_t al = bf16 ? 16 : 8;
  cudaError_t e = cudaSuccess;
  auto zalloc = [&](void** p, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes ? bytes : 1);
  };
  int64_t wmax = 32;
  for (int l = 0; l <= s->L; ++l) wmax = std::max<int64_t>(wmax, round_up(s->widths[l], 32));
  zalloc((void**)&t->loss, sizeof(float));
  t->scratch_floats = std::max<int64_t>(kTrainScratchFloats, kColsumChunks * wmax);
  zalloc((void**)&t->scratch, sizeof(float) * t->scratch_floats);
  zalloc((void**)&t->zero_bias, sizeof(float) * wmax);
  for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
    const int N = s->widths[l + 1], K = s->widths[l];
    const int64_t ld = round_up(K, 8);
    t->ldw.push_back(ld);
    float *Wm = nullptr, *mW = nullptr, *vW = nullptr, *dW = nullptr;
    float *mb = nullptr, *vb = nullptr, *db = nullptr;
    zalloc((void**)&Wm, sizeof(float) * N * ld);
    zalloc((void**)&mW, sizeof(float) * N * ld);
    zalloc((void**)&vW, sizeof(float) * N * ld);
    zalloc((void**)&dW, sizeof(float) * N * ld);
    zalloc((void**)&mb, sizeof(float) * N);
    zalloc((void**)&vb, sizeof(float) * N);
    zalloc((void**)&db, sizeof(float) * N);
    t->Wm.push_back(Wm); t->mW.push_back(mW); t->vW.push_back(vW); t->dW.push_back(dW);
    t->mb.push_back(mb); t->vb.push_back(vb); t->db.push_back(db);
    const int64_t ldt = round_up(N, al);
    void* WT = nullptr;
    zalloc(&WT, eb * K * ldt);
    t->WT.push_back(WT);
    t->ldt.push_back(ldt);
    if (e == cudaSuccess)
      e = cudaMemcpy2D(Wm, sizeof(float) * ld, s->Wh[l].data(), sizeof(float) * K,
                       sizeof(float) * K, N, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = publish_all(s, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_trn(t);
    s->trn = nullptr;
    return cuda_fail(s, e, "training parameters");
  }
  t->host_wver = s->wver;
  return DF_OK;
}

bool encode(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch_elems,
            uint32_t box_outer, char* emsg, size_t len) {
  return tc_encode_2d(m, base, 2, inner, outer, pitch_elems * 2, 64, box_outer, emsg, len);
}

// Batch buffers (and tensor maps) for at least B rows.
df_status ensure_batch(df_state* s, int64_t B) {
  Trn* t = s->trn;
  if (B <= t->B) return DF_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(s, e, "device synchronize");
  free_batch(t);
  B = round_up(B, 128);
  const int L = s->L, K0 = s->K0;
  const bool bf16 = s->precision == DF_BF16;
  const size_t eb = bf16 ? 2 : 4;
  const int64_t al = bf16 ? 16 : 8;
  const int64_t Bp = round_up(B, 64);
  const int64_t ldT = Bp + 64;
  auto zalloc = [&](void** p, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes ? bytes : 1);
  };
  t->ldx = round_up(K0, al);
  zalloc(&t->x, eb * B * t->ldx);
  int64_t nmax = 8, kmax = 8;
  for (int l = 0; l < L; ++l) {
    const int N = s->widths[l + 1];
    nmax = std::max<int64_t>(nmax, N);
    kmax = std::max<int64_t>(kmax, s->widths[l]);
    void *H = nullptr, *G = nullptr, *dZ = nullptr;
    const int64_t ldh = round_up(N, al), ldg = round_up(N, 32), ldz = round_up(N, al);
    if (l < L - 1) {
      zalloc(&H, eb * B * ldh);
      zalloc(&G, eb * B * ldg);
    }
    zalloc(&dZ, eb * B * ldz);
    t->H.push_back(H); t->G.push_back(G); t->dZ.push_back(dZ);
    t->ldh.push_back(ldh); t->ldg.push_back(ldg); t->ldz.push_back(ldz);
  }
  t->ldo = round_up(s->nout, 8);
  zalloc((void**)&t->O, sizeof(float) * B * t->ldo);
  zalloc((void**)&t->Oh, sizeof(float) * B * t->ldo);
  zalloc(&t->ZT, eb * nmax * ldT);
  zalloc(&t->HT, eb * kmax * ldT);
  t->lddx = round_up(K0, 4);
  zalloc((void**)&t->dX, sizeof(float) * B * t->lddx);
  if (bf16) {
    int64_t wmaxp = 0;
    for (int l = 0; l < L; ++l)
      wmaxp = std::max<int64_t>(wmaxp, round_up(s->widths[l + 1], 128) * t->ldw[l]);
    zalloc((void**)&t->dWp, sizeof(float) * kMaxSplit * wmaxp);
  }
  zalloc((void**)&t->h0, sizeof(double) * B);
  zalloc((void**)&t->rstat, sizeof(int32_t) * B);
  if (e != cudaSuccess) {
    free_batch(t);
    return cuda_fail(s, e, "training buffers");
  }
  t->B = B;
  t->Bp = Bp;
  t->ldT = ldT;
  if (bf16) {
    char emsg[256];
    bool ok = true;
    for (int l = 0; l < L && ok; ++l) {
      const bool last = l == L - 1;
      const int N = s->widths[l + 1], K = s->widths[l];
      // forward: hidden layers also store GELU'(Z); the read-out is linear, FP32
      TcLayer F{};
      F.N = N;
      F.K = K;
      const int ftile = pick_tile(N, K, !last, last ? kXF32 : kXBF16, true);
      F.BN = ftile & ~DF_TILE_PAIR;
      F.pair = (ftile & DF_TILE_PAIR) != 0;
      F.bias = s->bias[l];
      F.out = last ? (void*)t->O : t->H[l];
      F.ldo = last ? t->ldo : t->ldh[l];
      F.out_kind = last ? kXF32 : kXBF16;
      F.gelu = !last;
      F.out_scale = 1.0f;
      F.elem_bytes = 2;
      F.mode = last ? 0 : 1;
      F.gbuf = last ? nullptr : t->G[l];
      F.ldg = last ? 0 : t->ldg[l];
      F.ntan = 1;
      ok = encode(&F.tmA, l == 0 ? t->x : t->H[l - 1], K, B, l == 0 ? t->ldx : t->ldh[l - 1], 128,
                  emsg, sizeof emsg) &&
           encode(&F.tmB, s->Wlp[l], K, N, s->Kp8[l], F.pair ? F.BN / 2 : F.BN, emsg, sizeof emsg) &&
           tc_encode_out(F, (uint64_t)B, emsg, sizeof emsg);
      // input gradient: dZ_l [B x N] times W_l, i.e. against W_l^T [K x N]; layer 0's result
      // is the FP32 gradient of the network input, the others are scaled by GELU'(Z_{l-1})
      TcLayer D{};
      D.N = K;
      D.K = N;
      const int dtile = pick_tile(K, N, l > 0, l > 0 ? kXBF16 : kXF32, true);
      D.BN = dtile & ~DF_TILE_PAIR;
      D.pair = (dtile & DF_TILE_PAIR) != 0;
      D.bias = t->zero_bias;
      D.out = l > 0 ? t->dZ[l - 1] : (void*)t->dX;
      D.ldo = l > 0 ? t->ldz[l - 1] : t->lddx;
      D.out_kind = l > 0 ? kXBF16 : kXF32;
      D.gelu = false;
      D.out_scale = 1.0f;
      D.elem_bytes = 2;
      D.mode = l > 0 ? 2 : 0;
      D.gbuf = l > 0 ? t->G[l - 1] : nullptr;
      D.ldg = l > 0 ? t->ldg[l - 1] : 0;
      D.ntan = 1;
      if (ok)
        ok = encode(&D.tmA, t->dZ[l], N, B, t->ldz[l], 128, emsg, sizeof emsg) &&
             encode(&D.tmB, t->WT[l], N, K, t->ldt[l], D.pair ? D.BN / 2 : D.BN, emsg, sizeof emsg) &&
             tc_encode_out(D, (uint64_t)B, emsg, sizeof emsg);
      // weight gradient: dZ_l^T [N x Bp] times (H_{l-1}^T [K x Bp])^T, FP32 out
      TcLayer Wg{};
      Wg.N = K;
      Wg.K = (int)Bp;
      // CTA pairs (256-row tiles, each CTA streaming half of the B tile) once dW has more
      // than one 128-row tile and 128 columns; the narrow cases on single CTAs
      Wg.pair = N > 128 && K >= 128;
      if (Wg.pair) {
        const int64_t c128 = (K + 127) / 128 * 192, c256 = (K + 255) / 256 * 256;
        Wg.BN = c256 <= c128 ? 256 : 128;
      } else {
        Wg.BN = K <= 32 ? 32 : 64;
      }
      Wg.bias = t->zero_bias;
      Wg.out = t->dWp;        // split-K partials, summed into dW afterwards
      Wg.ldo = t->ldw[l];
      Wg.out_kind = kXF32;
      Wg.gelu = false;
      Wg.out_scale = 1.0f;
      Wg.elem_bytes = 2;
      Wg.mode = 0;
      Wg.ntan = 1;
      if (ok)
        ok = encode(&Wg.tmA, t->ZT, Bp, N, ldT, 128, emsg, sizeof emsg) &&
             encode(&Wg.tmB, t->HT, Bp, K, ldT, Wg.pair ? Wg.BN / 2 : Wg.BN, emsg, sizeof emsg) &&
             tc_encode_out(Wg, (uint64_t)kMaxSplit * round_up(N, 128), emsg, sizeof emsg);
      if (!ok) break;
      t->fwd.push_back(F);
      t->dgrad.push_back(D);
      t->wgrad.push_back(Wg);
      if ((e = prepare_tc(F)) != cudaSuccess || (e = prepare_tc(D)) != cudaSuccess ||
          (e = prepare_tc(Wg)) != cudaSuccess) {
        free_batch(t);
        return cuda_fail(s, e, "kernel attributes");
      }
    }
    if (!ok) {
      free_batch(t);
      return fail(s, DF_ERR_CUDA, "%s", emsg);
    }
  }
  return DF_OK;
}

df_status ensure_train(df_state* s, int64_t B) {
  df_status rc = ensure_params(s);
  if (rc != DF_OK) return rc;
  return ensure_batch(s, B);
}

// Forward pass over R rows of t->x, keeping H_l and GELU'(Z_l) of every hidden layer.
cudaError_t forward(df_state* s, int64_t R, cudaStream_t st) {
  Trn* t = s->trn;
  const RowMap rows{nullptr, nullptr, 0, R};
  for (int l = 0; l < s->L; ++l) {
    const bool last = l == s->L - 1;
    cudaError_t e;
    if (s->precision == DF_BF16) {
      e = launch_tc_gemm(t->fwd[l], rows, s->num_sms, s->d_err, st);
    } else {
      const float* A = l == 0 ? (const float*)t->x : (const float*)t->H[l - 1];
      const int64_t lda = l == 0 ? t->ldx : t->ldh[l - 1];
      e = launch_sgemm_bias_act(rows, s->widths[l + 1], s->Kp8[l], A, lda, s->W32[l], s->Kp8[l],
                                s->bias[l], last ? t->O : (float*)t->H[l],
                                last ? t->ldo : t->ldh[l], !last, s->num_sms, st, last ? 0 : 1,
                                last ? nullptr : (float*)t->G[l], last ? 0 : t->ldg[l], 1);
    }
    if (e != cudaSuccess) return e;
  }
  t->rows = R;
  return cudaSuccess;
}

// Backward pass over R rows from dZ_{L-1} (already in t->dZ[L-1]); fills dW, db and, when
// want_dx, the FP32 input gradient t->dX.
cudaError_t backward(df_state* s, int64_t R, bool want_dx, cudaStream_t st) {
  Trn* t = s->trn;
  const bool bf16 = s->precision == DF_BF16;
  const int64_t Rp = round_up(R, 64);
  const RowMap rows{nullptr, nullptr, 0, R};
  cudaError_t e = cudaSuccess;
  for (int l = s->L - 1; l >= 0 && e == cudaSuccess; --l) {
    const int N = s->widths[l + 1], K = s->widths[l];
    const void* Hin = l == 0 ? t->x : t->H[l - 1];
    const int64_t ldin = l == 0 ? t->ldx : t->ldh[l - 1];
    // dZ_l^T, with db_l = column sums of dZ_l from the same pass
    e = launch_transpose(R, N, t->dZ[l], t->ldz[l], t->ZT, t->ldT, Rp, bf16, s->num_sms, st,
                         t->db[l], t->scratch, t->scratch_floats);
    if (e == cudaSuccess)
      e = launch_transpose(R, K, Hin, ldin, t->HT, t->ldT, Rp, bf16, s->num_sms, st);
    const RowMap wrows{nullptr, nullptr, 0, N};
    if (e == cudaSuccess) {
      if (bf16) {
        TcLayer Wg = t->wgrad[l];
        Wg.K = (int)Rp;
        // work items: 128-row tiles, or 256-row tiles on the GPU's CTA pairs
        const int64_t rows_per = Wg.pair ? 256 : 128;
        const int64_t tiles = ((N + rows_per - 1) / rows_per) * ((K + Wg.BN - 1) / Wg.BN);
        Wg.ksplit = wgrad_splits(tiles, (int)(Rp / 64), Wg.pair ? s->num_sms / 2 : s->num_sms);
        // each split owns whole 128-row tiles (a tile's store covers all its rows)
        Wg.split_rows = round_up(N, 128);
        e = launch_tc_gemm(Wg, wrows, s->num_sms, s->d_err, st);
        if (e == cudaSuccess)
          e = launch_sum_splits(Wg.ksplit, (int64_t)N * t->ldw[l], Wg.split_rows * t->ldw[l],
                                t->dWp, t->dW[l], st);
      } else {
        e = launch_sgemm_bias_act(wrows, K, (int)Rp, (const float*)t->ZT, t->ldT,
                                  (const float*)t->HT, t->ldT, t->zero_bias, t->dW[l], t->ldw[l],
                                  false, s->num_sms, st);
      }
    }
    if (e != cudaSuccess || (l == 0 && !want_dx)) continue;
    if (bf16) {
      e = launch_tc_gemm(t->dgrad[l], rows, s->num_sms, s->d_err, st);
    } else if (l > 0) {
      e = launch_sgemm_bias_act(rows, K, (int)t->ldt[l], (const float*)t->dZ[l], t->ldz[l],
                                (const float*)t->WT[l], t->ldt[l], t->zero_bias,
                                (float*)t->dZ[l - 1], t->ldz[l - 1], false, s->num_sms, st, 2,
                                (float*)t->G[l - 1], t->ldg[l - 1], 1);
    } else {
      e = launch_sgemm_bias_act(rows, K, (int)t->ldt[0], (const float*)t->dZ[0], t->ldz[0],
                                (const float*)t->WT[0], t->ldt[0], t->zero_bias, t->dX, t->lddx,
                                false, s->num_sms, st);
    }
  }
  return e;
}

df_status check_adam(df_state* s, const df_adam* hp) {
  if (!hp) return fail(s, DF_ERR_INVALID_ARG, "hyper-parameters are NULL");
  if (!(hp->lr > 0) || !(hp->beta1 >= 0 && hp->beta1 < 1) || !(hp->beta2 >= 0 && hp->beta2 < 1) ||
      !(hp->eps > 0))
    return fail(s, DF_ERR_INVALID_ARG, "need lr > 0, 0 <= beta1, beta2 < 1, eps > 0");
  return DF_OK;
}

cudaError_t adam(df_state* s, const df_adam* hp, cudaStream_t st) {
  Trn* t = s->trn;
  t->t += 1;
  const float c1 = (float)(1.0 - std::pow(hp->beta1, (double)t->t));
  const float c2 = (float)(1.0 - std::pow(hp->beta2, (double)t->t));
  const float lr = (float)hp->lr, b1 = (float)hp->beta1, b2 = (float)hp->beta2,
              eps = (float)hp->eps;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
    const int N = s->widths[l + 1];
    e = launch_adam((int64_t)N * t->ldw[l], t->Wm[l], t->mW[l], t->vW[l], t->dW[l], lr, b1, b2, eps,
                    c1, c2, st);
    if (e == cudaSuccess)
      e = launch_adam(N, s->bias[l], t->mb[l], t->vb[l], t->db[l], lr, b1, b2, eps, c1, c2, st);
  }
  if (e == cudaSuccess) e = publish_all(s, st);
  s->wver += 1;
  return e;
}

}  // namespace

namespace dfgb {

// Brings the state's host weight copies (used to build the Jacobian context) up to date with
// the training masters.
df_status sync_host_weights(df_state* s) {
  Trn* t = s->trn;
  if (!t || t->host_wver == s->wver) return DF_OK;
  cudaError_t e = cudaDeviceSynchronize();
  for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
    const int N = s->widths[l + 1], K = s->widths[l];
    e = cudaMemcpy2D(s->Wh[l].data(), sizeof(float) * K, t->Wm[l], sizeof(float) * t->ldw[l],
                     sizeof(float) * K, N, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "weight download");
  t->host_wver = s->wver;
  return DF_OK;
}

}  // namespace dfgb

extern "C" {

df_status df_train_step(df_state* s, int64_t batch, const double* T, const double* p,
                        const double* Y, const double* Y_target, int64_t ld, const df_adam* hp,
                        float* loss_out, void* stream) {
  df_status rc = check_fields(s, batch, T, p, Y, ld);
  if (rc != DF_OK) return rc;
  if (batch > 0 && !Y_target) return fail(s, DF_ERR_INVALID_ARG, "Y_target is NULL");
  if ((rc = check_adam(s, hp)) != DF_OK) return rc;
  DeviceGuard guard(s->device);
  if ((rc = ensure_train(s, std::max<int64_t>(batch, 1))) != DF_OK) return rc;
  Trn* t = s->trn;
  cudaStream_t st = (cudaStream_t)stream;
  const bool bf16 = s->precision == DF_BF16;
  cudaError_t e = batch > 0 ? cudaSuccess : cudaMemsetAsync(t->loss, 0, sizeof(float), st);
  if (batch > 0) {
    const RowMap cells{nullptr, nullptr, 0, batch};
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_inputs", st);
      e = launch_eos_pre(s->P, cells, T, p, Y, ld, t->h0, nullptr, t->x, bf16 ? kXBF16 : kXF32,
                         t->ldx, 1.0f, t->rstat, st);
      if (e == cudaSuccess) e = launch_train_targets(s->P, batch, Y, Y_target, ld, t->Oh, t->ldo, st);
    }
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_forward", st);
      e = forward(s, batch, st);
    }
    if (e == cudaSuccess)
      e = launch_loss_grad(batch, s->n, t->O, t->ldo, t->Oh, t->ldo, t->dZ[s->L - 1],
                           t->ldz[s->L - 1], bf16, t->loss, t->scratch, st);
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_backward", st);
      e = backward(s, batch, false, st);
    }
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_adam", st);
      e = adam(s, hp, st);
    }
  }
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpyAsync(loss_out, t->loss, sizeof(float), cudaMemcpyDefault, st);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "training step");
}

df_status df_propnet_train_step(df_state* s, int64_t batch, const double* h, const double* p,
                                const double* Y, int64_t ldY, const double* target, int64_t ldt,
                                const df_adam* hp, float* loss_out, void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (!s->netonly) return fail(s, DF_ERR_UNSUPPORTED, "not a network-only state (df_network_create)");
  if (batch < 0) return fail(s, DF_ERR_INVALID_ARG, "batch < 0");
  if (batch > 0 && (!h || !p || !Y || !target)) return fail(s, DF_ERR_INVALID_ARG, "NULL array");
  if (batch > 0 && (ldY < batch || ldt < batch))
    return fail(s, DF_ERR_INVALID_ARG, "ldY or ldt < batch");
  df_status rc = check_adam(s, hp);
  if (rc != DF_OK) return rc;
  DeviceGuard guard(s->device);
  if ((rc = ensure_train(s, std::max<int64_t>(batch, 1))) != DF_OK) return rc;
  Trn* t = s->trn;
  cudaStream_t st = (cudaStream_t)stream;
  const bool bf16 = s->precision == DF_BF16;
  cudaError_t e = batch > 0 ? cudaSuccess : cudaMemsetAsync(t->loss, 0, sizeof(float), st);
  if (batch > 0) {
    {
      ProfScope ps(s, "train_inputs", st);
      e = launch_prop_inputs(s->d_norm, s->n, s->lambda, batch, h, p, Y, ldY, t->x, t->ldx,
                             bf16 ? kXBF16 : kXF32, s->num_sms, st);
      if (e == cudaSuccess)
        e = launch_prop_targets(s->d_norm, s->K0, s->nout, batch, target, ldt, t->Oh, t->ldo,
                                s->num_sms, st);
    }
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_forward", st);
      e = forward(s, batch, st);
    }
    if (e == cudaSuccess)
      e = launch_loss_grad(batch, s->nout, t->O, t->ldo, t->Oh, t->ldo, t->dZ[s->L - 1],
                           t->ldz[s->L - 1], bf16, t->loss, t->scratch, st);
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_backward", st);
      e = backward(s, batch, false, st);
    }
    if (e == cudaSuccess) {
      ProfScope ps(s, "train_adam", st);
      e = adam(s, hp, st);
    }
  }
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpyAsync(loss_out, t->loss, sizeof(float), cudaMemcpyDefault, st);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "property-network training step");
}

df_status df_mlp_forward_train(df_state* s, int64_t n_rows, const float* x, float* O,
                               void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (n_rows < 0 || (n_rows > 0 && (!x || !O))) return fail(s, DF_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(s->device);
  df_status rc = ensure_train(s, std::max<int64_t>(n_rows, 1));
  if (rc != DF_OK) return rc;
  Trn* t = s->trn;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_rows == 0) {
    t->rows = 0;
    return DF_OK;
  }
  cudaError_t e = launch_cast_rows(n_rows, s->K0, x, s->K0, t->x, t->ldx,
                                   s->precision == DF_BF16 ? kXBF16 : kXF32, 1.0f, s->num_sms, st);
  if (e == cudaSuccess) e = forward(s, n_rows, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(O, sizeof(float) * s->nout, t->O, sizeof(float) * t->ldo,
                          sizeof(float) * s->nout, (size_t)n_rows, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "training forward pass");
}

df_status df_mlp_backward(df_state* s, int64_t n_rows, const float* dO, float* dX, void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (!s->trn || s->trn->rows < 0)
    return fail(s, DF_ERR_INVALID_ARG, "df_mlp_backward needs a df_mlp_forward_train first");
  if (n_rows != s->trn->rows)
    return fail(s, DF_ERR_INVALID_ARG, "n_rows (%lld) differs from the forward pass (%lld)",
                (long long)n_rows, (long long)s->trn->rows);
  if (n_rows > 0 && !dO) return fail(s, DF_ERR_INVALID_ARG, "dO is NULL");
  DeviceGuard guard(s->device);
  Trn* t = s->trn;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_rows == 0) {
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
      e = cudaMemsetAsync(t->dW[l], 0, sizeof(float) * s->widths[l + 1] * t->ldw[l], st);
      if (e == cudaSuccess) e = cudaMemsetAsync(t->db[l], 0, sizeof(float) * s->widths[l + 1], st);
    }
    return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "gradient reset");
  }
  const int L = s->L;
  cudaError_t e = launch_cast_rows(n_rows, s->nout, dO, s->nout, t->dZ[L - 1], t->ldz[L - 1],
                                   s->precision == DF_BF16 ? kXBF16 : kXF32, 1.0f, s->num_sms, st);
  if (e == cudaSuccess) e = backward(s, n_rows, dX != nullptr, st);
  if (e == cudaSuccess && dX)
    e = cudaMemcpy2DAsync(dX, sizeof(float) * s->K0, t->dX, sizeof(float) * t->lddx,
                          sizeof(float) * s->K0, (size_t)n_rows, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "training backward pass");
}

df_status df_adam_step(df_state* s, const df_adam* hp, void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  df_status rc = check_adam(s, hp);
  if (rc != DF_OK) return rc;
  if (!s->trn) return fail(s, DF_ERR_INVALID_ARG, "no gradients: run a backward pass first");
  DeviceGuard guard(s->device);
  cudaError_t e = adam(s, hp, (cudaStream_t)stream);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "Adam step");
}

df_status df_get_params(df_state* s, int32_t layer, int32_t which, float* W, float* b,
                        void* stream) {
  if (!s) return fail(nullptr, DF_ERR_INVALID_ARG, "state is NULL");
  if (layer < 0 || layer >= s->L) return fail(s, DF_ERR_INVALID_ARG, "layer out of range");
  if (which < DF_PARAM_WEIGHTS || which > DF_PARAM_ADAM_V)
    return fail(s, DF_ERR_INVALID_ARG, "unknown parameter set");
  DeviceGuard guard(s->device);
  df_status rc = ensure_params(s);
  if (rc != DF_OK) return rc;
  Trn* t = s->trn;
  const float* srcW = which == DF_PARAM_WEIGHTS ? t->Wm[layer] : which == DF_PARAM_GRADS ? t->dW[layer]
                      : which == DF_PARAM_ADAM_M ? t->mW[layer] : t->vW[layer];
  const float* srcb = which == DF_PARAM_WEIGHTS ? s->bias[layer] : which == DF_PARAM_GRADS ? t->db[layer]
                      : which == DF_PARAM_ADAM_M ? t->mb[layer] : t->vb[layer];
  const int N = s->widths[layer + 1], K = s->widths[layer];
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (W)
    e = cudaMemcpy2DAsync(W, sizeof(float) * K, srcW, sizeof(float) * t->ldw[layer],
                          sizeof(float) * K, N, cudaMemcpyDefault, st);
  if (e == cudaSuccess && b) e = cudaMemcpyAsync(b, srcb, sizeof(float) * N, cudaMemcpyDefault, st);
  return e == cudaSuccess ? DF_OK : cuda_fail(s, e, "parameter copy");
}

// File layout (little-endian): "DFGBTRN1", int32 L, int32 widths[L+1], int64 Adam step, then
// per layer W, b, m_W, v_W, m_b, v_b as FP32 (W and moments [N x K] row-major).
df_status df_state_save(df_state* s, const char* path) {
  if (!s || !path) return fail(s, DF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(s->device);
  df_status rc = ensure_params(s);
  if (rc != DF_OK) return rc;
  Trn* t = s->trn;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(s, e, "device synchronize");
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(s, DF_ERR_INVALID_ARG, "cannot open %s for writing", path);
  bool ok = std::fwrite("DFGBTRN1", 1, 8, f) == 8;
  const int32_t L = s->L;
  ok = ok && std::fwrite(&L, 4, 1, f) == 1;
  std::vector<int32_t> w(s->widths.begin(), s->widths.end());
  ok = ok && std::fwrite(w.data(), 4, w.size(), f) == w.size();
  ok = ok && std::fwrite(&t->t, 8, 1, f) == 1;
  for (int l = 0; l < L && ok; ++l) {
    const int N = s->widths[l + 1], K = s->widths[l];
    std::vector<float> buf((size_t)N * K);
    const float* mats[3] = {t->Wm[l], t->mW[l], t->vW[l]};
    const float* vecs[3] = {s->bias[l], t->mb[l], t->vb[l]};
    auto put_mat = [&](const float* d) {
      if (!ok) return;
      e = cudaMemcpy2D(buf.data(), sizeof(float) * K, d, sizeof(float) * t->ldw[l],
                       sizeof(float) * K, N, cudaMemcpyDeviceToHost);
      ok = e == cudaSuccess && std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    };
    auto put_vec = [&](const float* d) {
      if (!ok) return;
      e = cudaMemcpy(buf.data(), d, sizeof(float) * N, cudaMemcpyDeviceToHost);
      ok = e == cudaSuccess && std::fwrite(buf.data(), 4, N, f) == (size_t)N;
    };
    put_mat(mats[0]);
    put_vec(vecs[0]);
    put_mat(mats[1]);
    put_mat(mats[2]);
    put_vec(vecs[1]);
    put_vec(vecs[2]);
  }
  ok = (std::fclose(f) == 0) && ok;
  if (e != cudaSuccess) return cuda_fail(s, e, "parameter download");
  return ok ? DF_OK : fail(s, DF_ERR_INVALID_ARG, "write to %s failed", path);
}

df_status df_state_load(df_state* s, const char* path) {
  if (!s || !path) return fail(s, DF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(s->device);
  df_status rc = ensure_params(s);
  if (rc != DF_OK) return rc;
  Trn* t = s->trn;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(s, DF_ERR_INVALID_ARG, "cannot open %s", path);
  char magic[8];
  int32_t L = 0;
  int64_t steps = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "DFGBTRN1", 8) == 0 &&
            std::fread(&L, 4, 1, f) == 1 && L == s->L;
  std::vector<int32_t> w(s->L + 1);
  ok = ok && std::fread(w.data(), 4, w.size(), f) == w.size() &&
       std::equal(w.begin(), w.end(), s->widths.begin());
  ok = ok && std::fread(&steps, 8, 1, f) == 1 && steps >= 0;
  if (!ok) {
    std::fclose(f);
    return fail(s, DF_ERR_INVALID_ARG, "%s is not a parameter file of this network", path);
  }
  // read everything before touching the device state, so a short file changes nothing
  std::vector<std::vector<float>> blobs;
  for (int l = 0; l < s->L && ok; ++l) {
    const size_t N = s->widths[l + 1], K = s->widths[l];
    const size_t sizes[6] = {N * K, N, N * K, N * K, N, N};
    for (size_t sz : sizes) {
      blobs.emplace_back(sz);
      ok = ok && std::fread(blobs.back().data(), 4, sz, f) == sz;
    }
  }
  std::fclose(f);
  if (!ok) return fail(s, DF_ERR_INVALID_ARG, "%s is truncated", path);
  cudaError_t e = cudaDeviceSynchronize();
  for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
    const int N = s->widths[l + 1], K = s->widths[l];
    const std::vector<float>* bl = &blobs[6 * l];
    float* mats[3] = {t->Wm[l], t->mW[l], t->vW[l]};
    const int mi[3] = {0, 2, 3};
    for (int j = 0; j < 3 && e == cudaSuccess; ++j)
      e = cudaMemcpy2D(mats[j], sizeof(float) * t->ldw[l], bl[mi[j]].data(), sizeof(float) * K,
                       sizeof(float) * K, N, cudaMemcpyHostToDevice);
    float* vecs[3] = {s->bias[l], t->mb[l], t->vb[l]};
    const int vi[3] = {1, 4, 5};
    for (int j = 0; j < 3 && e == cudaSuccess; ++j)
      e = cudaMemcpy(vecs[j], bl[vi[j]].data(), sizeof(float) * N, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = publish_all(s, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(s, e, "parameter upload");
  t->t = steps;
  s->wver += 1;
  return DF_OK;
}

df_status df_train_get_step(df_state* s, int64_t* steps) {
  if (!s || !steps) return fail(s, DF_ERR_INVALID_ARG, "NULL argument");
  *steps = s->trn ? s->trn->t : 0;
  return DF_OK;
}

}  // extern "C"
