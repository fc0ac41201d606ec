/*
 * df_propnet.h -- C ABI of the real-fluid property network of libdfgb.so: a PRNet-style
 * surrogate (Sec. 2) of the equation of state.
 *
 * The paper's supercritical runs replace the real-fluid property evaluation by a second network,
 * PRNet, which reads a cell's conserved energy, pressure and composition and yields its density,
 * temperature and transport properties (Sec. 2; sizes (3,1024,512,256,1) for density and
 * (3,2048,1024,512,4) for temperature and transport, Sec. 4.1). The reaction step of this
 * library evaluates the Peng-Robinson state explicitly and recovers T by Newton (df.h, a2-a9);
 * the calls below build, train and run the surrogate of that evaluation so that the two can be
 * compared on accuracy and cost. Inputs are the cell's conserved mass-specific enthalpy h (the
 * quantity the reaction step conserves), p and Y_1..Y_n; outputs are any m properties, e.g.
 * density alone, or temperature with the logarithms of viscosity, thermal conductivity and
 * thermal diffusivity (the paper's 4-output temperature-and-transport network), trained on the
 * explicit evaluation (df_real_fluid_props, df_transport_props of df.h).
 *
 * A property network lives in a network-only df_state (df_network_create). On it the generic
 * network calls of df.h work (df_mlp_forward, df_mlp_forward_train, df_mlp_backward,
 * df_adam_step, df_get_params, df_train_get_step, df_state_save / df_state_load, df_autotune,
 * df_get_tiles, df_profile_*); the reaction-step calls return DF_ERR_UNSUPPORTED.
 * Conventions are those of df.h: DEVICE pointers, FP64 fields, species-major Y[k * ldY + i],
 * work enqueued on `stream` without synchronising.
 */
#ifndef DF_PROPNET_H
#define DF_PROPNET_H

#include <stdint.h>

#include "df.h"

#ifdef __cplusplus
extern "C" {
#endif

/* A state holding only the network `mlp`:
 *   widths[0] = n + 2 inputs, read as (h, p, BC(Y_1), ..., BC(Y_n)) with the Box-Cox transform
 *     BC(y) = (y^lambda - 1) / lambda of df.h (1/lambda an integer in 1..64), n in 1..32;
 *   widths[L] = m outputs, any m >= 1; hidden layers GELU, read-out linear (as df.h a6-a7);
 *   in_mean / in_std [n + 2] Z-score the inputs, out_mean / out_std [m] de-normalise the
 *     outputs: property_k = out_mean_k + out_std_k * O_k;
 *   dt is not used. opt->precision DF_FP32 or DF_BF16 (DF_FP8_E4M3: DF_ERR_UNSUPPORTED);
 *   T_react, newton_tol and newton_max_iter are not used.
 * Errors as df_state_create. */
df_status df_network_create(const df_mlp_desc* mlp, const df_options* opt, df_state** out);

/* Properties of n_cells cells: out[k * ldout + i] = property k of cell i (k < m), FP64,
 * device, ldout >= n_cells. h, p [n_cells], Y [n * ldY], ldY >= n_cells. The input rows are
 * formed in FP32 (the Box-Cox power by exp2/log2), the network runs in the state's precision,
 * the outputs are de-normalised in FP64. DF_ERR_UNSUPPORTED on a reaction-step state. */
df_status df_propnet_infer(df_state* s, int64_t n_cells, const double* h, const double* p,
                           const double* Y, int64_t ldY, double* out, int64_t ldout,
                           void* stream);

/* One Adam step of the property network on a batch of `batch` cells with target properties
 * target[k * ldt + i] (FP64, device, ldt >= batch): the loss is the mean over the batch of the
 * squared error of the normalised outputs, L = (1/B) sum_i sum_k (O_ik - (t_ik - out_mean_k) /
 * out_std_k)^2 (the regression reading of PRNet's training, which the paper does not print),
 * the backward pass and Adam are those of df_train_step. loss_out (FP32, device or host, may be
 * NULL) receives L before the step. Deterministic. */
df_status df_propnet_train_step(df_state* s, int64_t batch, const double* h, const double* p,
                                const double* Y, int64_t ldY, const double* target, int64_t ldt,
                                const df_adam* hp, float* loss_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DF_PROPNET_H */
