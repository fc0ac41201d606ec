/*
 * df.h -- C ABI of the GB300 reaction-step library (libdfgb.so).
 *
 * The library advances the chemistry of every cell of a real-fluid flame by one time step,
 * the pointwise data-parallel step of the DeepFlame method (Sec. 2, "Deep learning
 * approaches": a network maps the thermochemical state (T, p, Y_i) of a cell to its chemical
 * change; real-fluid properties follow the Peng-Robinson EoS). One step of one cell:
 *   a0  the cell reacts if T > T_react; reacting cells are listed in ascending index order;
 *   a1  W_mix = 1 / sum_k Y_k / W_k,  X_k = Y_k W_mix / W_k;
 *   a2  Peng-Robinson a_m(T), b_m with van der Waals mixing and k_ij;
 *   a3  compressibility Z: real root of the PR cubic above B of least departure Gibbs energy;
 *   a4  conserved mass-specific enthalpy h0 = h_ig(T, Y) + h_dep / W_mix;
 *   a5  network input (T, p, BC(Y_k)) Z-scored (Sec. 3.3.1), BC = Box-Cox;
 *   a6  hidden layers h = GELU(h W^T + b), tanh-form GELU (Sec. 3.3.2);
 *   a7  linear output layer;
 *   a8  Y'_k = inverse Box-Cox of BC(Y_k) + (std_k O_k + mean_k), renormalised;
 *   a9  T' from h(T', p, Y') = h0 by safeguarded Newton;
 *   a10 T, Y of reacting cells overwritten with T', Y'.
 *
 * Conventions shared by every entry point:
 *   - Field arrays are DEVICE pointers owned by the caller, FP64, one value per cell:
 *     T[i], p[i]; mass fractions are species-major, Y[k * ldY + i] (ldY >= n_cells).
 *   - Work is enqueued on the CUDA stream `stream` (a cudaStream_t, NULL = legacy default
 *     stream) and returns without synchronising, unless the entry point says otherwise.
 *   - Every entry point returns a df_status; on error nothing has been enqueued unless
 *     the code is DF_ERR_CUDA, and df_get_last_error() describes the cause.
 *   - A df_state is used by one host thread at a time.
 */
#ifndef DF_H
#define DF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct df_state df_state;
typedef int32_t df_status;

#define DF_OK 0
#define DF_ERR_INVALID_ARG 1      /* bad pointer, size, stride or option */
#define DF_ERR_CUDA 2             /* a CUDA call failed; see df_get_last_error */
#define DF_ERR_NOT_CONVERGED 3    /* reported by df_get_step_summary only */
#define DF_ERR_NONFINITE_INPUT 4  /* reported by df_get_step_summary only */
#define DF_ERR_DT_MISMATCH 5      /* dt differs from the network's time step */
#define DF_ERR_UNSUPPORTED 6      /* valid but not implemented (e.g. 1/lambda not integral) */
#define DF_ERR_OOM 7              /* device allocation failed */
#define DF_ERR_TIMEOUT 8          /* a kernel wait hit its limit and the kernel gave up */

/* Per-cell status bits written by df_chem_step (0 = advanced normally). A flagged cell
 * keeps its old T and Y. */
#define DF_CELL_NOT_CONVERGED 1   /* Newton on h(T) did not meet the tolerance */
#define DF_CELL_NO_ROOT 2         /* the PR cubic has no real root above B */
#define DF_CELL_NONFINITE 4       /* non-finite T, p or Y, p <= 0, or non-finite result */

/* Arithmetic of the network layers (a5-a7). The equation of state, Box-Cox, renormalisation
 * and Newton steps are FP64 in every mode (Sec. 3.3.1 keeps all non-network work double). */
typedef enum {
  DF_FP32 = 0,      /* SIMT FP32 GEMMs, accurate tanh: the plain FP32 step */
  DF_BF16 = 1,      /* tcgen05 BF16 GEMMs, FP32 accumulation, BF16 activations */
  DF_FP8_E4M3 = 2   /* tcgen05 FP8 e4m3 GEMMs, FP32 accumulation; weights e4m3(W/s_c) with
                       per-output-channel s_c = max|W_c|/448, activations e4m3(32 v) */
} df_precision;

/* Mechanism constants (host pointers, deep-copied by df_state_create). */
typedef struct {
  int32_t n_species;          /* n, 1..32 */
  const double* W;            /* [n] molar masses, kg/mol */
  const double* Tc;           /* [n] critical temperatures, K */
  const double* pc;           /* [n] critical pressures, Pa */
  const double* omega;        /* [n] acentric factors */
  const double* kij;          /* [n*n] binary interaction parameters, row-major, symmetric */
  const double* nasa;         /* [n*7] NASA-7 coefficients a1..a7 per species, row-major */
} df_mech_desc;

/* Chemistry network (host pointers, deep-copied by df_state_create). */
typedef struct {
  int32_t n_layers;           /* linear layers L, 1..8 */
  const int32_t* widths;      /* [L+1]; widths[0] = n + 2 (T, p, Y), widths[L] = n */
  const float* const* W;      /* [L] layer l is widths[l+1] x widths[l], row-major (out, in) */
  const float* const* b;      /* [L] layer l is widths[l+1] */
  double lambda;              /* Box-Cox exponent; 1/lambda must be an integer in 1..64 */
  const double* in_mean;      /* [n+2] Z-score of the inputs (T, p, BC(Y_1..n)) */
  const double* in_std;       /* [n+2] */
  const double* out_mean;     /* [n] de-normalisation of the outputs */
  const double* out_std;      /* [n] */
  double dt;                  /* time step the network advances, s */
} df_mlp_desc;

typedef struct {
  int32_t precision;          /* df_precision */
  double T_react;             /* cells with T > T_react react (K); 0 lets every cell through */
  double newton_tol;          /* stop when the Newton step |dT| <= newton_tol * T; <= 0 selects
                                 1e-8 (the accepted step leaves an error of O(dT^2)) */
  int32_t newton_max_iter;    /* <= 0 selects 50 */
  int32_t device;             /* CUDA device ordinal the state lives on */
  int64_t batch_cells;        /* reacting cells per internal batch; <= 0 selects 2^20 */
  int32_t gelu_mode;          /* DF_GELU_TANH (0) or DF_GELU_TABLE (1), below */
} df_options;

/* Hidden-layer activation of the network (a6). Both are the tanh form of Sec. 3.3.2:
 *   DF_GELU_TANH   0.5 x (1 + tanh(c (x + 0.044715 x^3))), c = sqrt(2/pi), with the hardware
 *                  tanh approximation on tensor-core paths and tanhf on the FP32 path;
 *   DF_GELU_TABLE  the paper's tabulation: 0 for x <= -3, x for x >= 3, and in between the
 *                  second-order expansion about the table node at or below x (nodes every 0.01,
 *                  value, slope and half curvature in FP32). FP32 and BF16 networks, inference
 *                  entry points only: df_state_create refuses it for DF_FP8_E4M3, and
 *                  df_chem_jacobian and the training calls return DF_ERR_UNSUPPORTED. */
#define DF_GELU_TANH 0
#define DF_GELU_TABLE 1

/* Creates a state on opt->device: copies the mechanism and network, derives the per-species
 * EoS constants and the low-precision weight copies, allocates scratch for one batch.
 * On success *out is the new state; on error *out is NULL. Thread-safe.
 * Paper: Sec. 2 (the chemistry network reads (T, p, Y_i); properties from the Peng-Robinson
 * EoS), Sec. 3.3.1 (Z-scored inputs; FP16 weights and activations, here BF16 or FP8 e4m3, all
 * other arithmetic double). */
df_status df_state_create(const df_mech_desc* mech, const df_mlp_desc* mlp,
                          const df_options* opt, df_state** out);

/* Frees the state and its device memory (synchronises the device first). NULL is a no-op.
 * Paper: no counterpart (resource management of df_state_create). */
void df_state_destroy(df_state* s);

/* One reaction step (a0-a10) of cells held in HOST memory: T [n_cells] and Y [n * ldY] are
 * updated in place, p is read, cell_status (HOST, [n_cells], may be NULL) receives the DF_CELL_*
 * bits. The cells go through the device in chunks with two device buffers: the upload of one
 * chunk and the download of another overlap the step of a third (copies on two internal
 * streams, the steps on `stream`), the GPU form of the paper's double buffering of data
 * movement against computation (Sec. 3.3.3). Chunks of chunk_cells cells (at most the state's
 * batch), or with chunk_cells = 0 a short first and last chunk of 1/16 of the cells (at least
 * 32,768) around as few middle chunks as the batch allows (at least two): only a short upload
 * and a short download are left outside the steps, and the long chunks step at the long-batch
 * rate. Page-locked host memory lets the copies run asynchronously; with
 * pageable memory CUDA stages them and they do not overlap.
 * Stream-ordered: the work starts behind the work already on `stream`, and `stream` reaches the
 * end of this call once every result is in host memory; synchronise it before reading T, Y or
 * cell_status, and keep the host arrays alive until then. df_get_step_summary afterwards covers
 * all chunks. Errors as df_chem_step.
 * chunk_cells = DF_HOST_DIRECT: no device copies; the step's kernels read and write the host
 * arrays in place over the host link (NVLink-C2C on Grace). Every array must lie in one
 * page-locked allocation mapped into the device's address space (cudaHostAlloc,
 * cudaHostRegister), else DF_ERR_INVALID_ARG. The results are bit-identical to the chunked
 * form and to df_chem_step.
 * Paper: Sec. 2 (the step), Sec. 3.3.3 (batches whose data movement overlaps the computation
 * of other batches). */
#define DF_HOST_DIRECT (-1)
df_status df_chem_step_host(df_state* s, int64_t n_cells, double dt, double* T, const double* p,
                            double* Y, int64_t ldY, int32_t* cell_status, int64_t chunk_cells,
                            void* stream);

/* Real-fluid properties (a1-a4 without the network): rho [kg/m^3], h [J/kg], cp [J/(kg K)]
 * and Z of every cell. Any output pointer may be NULL and is then not written.
 * Paper: Sec. 2 (supercritical mixture properties from the Peng-Robinson EoS; the equations are
 * Peng & Robinson 1976 with van der Waals one-fluid mixing, which the paper names but does not
 * print). Evaluated explicitly in FP64, as Sec. 3.3.1 keeps all non-network work double. */
df_status df_real_fluid_props(df_state* s, int64_t n_cells, const double* T, const double* p,
                              const double* Y, int64_t ldY, double* rho, double* h, double* cp,
                              double* Z, void* stream);

/* Transport properties of every cell at its real-fluid state: dynamic viscosity mu [Pa s],
 * thermal conductivity lam [W/(m K)] and thermal diffusivity alpha = lam / (rho c_p) [m^2/s]
 * (device [n_cells] FP64 each, any may be NULL). The method of Chung, Ajlan, Lee & Starling
 * (1988) for dense fluids and mixtures -- Chung's mixing rules over the mole fractions, critical
 * volumes from the Peng-Robinson critical compressibility (Vc = 0.307401 R Tc / pc), nonpolar
 * species -- evaluated at the Peng-Robinson molar density, with the ideal-gas Cv and the
 * real-fluid c_p of the same state. The Peng-Robinson state and the outer mixing sums are FP64;
 * the inner pair sums and the correlation itself (accurate to a few percent) are FP32, which
 * leaves up to about 1e-5 relative against an FP64 evaluation.
 * Cells whose state is not finite or has no PR root get NaN.
 * Paper: Sec. 2 (PRNet yields density, temperature and transport properties such as viscosity
 * and thermal diffusivity of the supercritical mixture, based on the Peng-Robinson EoS); the
 * paper names no transport model, Chung's method is this library's reading. */
df_status df_transport_props(df_state* s, int64_t n_cells, const double* T, const double* p,
                             const double* Y, int64_t ldY, double* mu, double* lam, double* alpha,
                             void* stream);

/* One reaction step (a0-a10) of n_cells cells, in place on T and Y; p is read only.
 * dt must equal the network's dt to 1e-12 relative, else DF_ERR_DT_MISMATCH.
 * cell_status (device, [n_cells], may be NULL) receives the DF_CELL_* bits (0 for cells that
 * do not react). n_active_out (device, may be NULL) receives the number of reacting cells.
 * Asynchronous: problems inside kernels are reported by df_get_step_summary.
 * Paper: Sec. 2 (the network maps a cell's (T, p, Y_i) to its chemical change over the flow
 * step; real-fluid state from the Peng-Robinson EoS), Sec. 3.3.1 (Z-scored inputs, reduced-
 * precision network, everything else double), Sec. 3.3.2 (tanh-form GELU). */
df_status df_chem_step(df_state* s, int64_t n_cells, double dt, double* T, const double* p,
                       double* Y, int64_t ldY, int32_t* cell_status, int64_t* n_active_out,
                       void* stream);

/* Chemical source terms for a flow solver: the same step as df_chem_step (Sec. 2: the network
 * supplies each cell's chemical change), but T and Y are read only and the result is returned
 * as rates:
 *   omega (device, [n][ldw] species-major FP64, ldw >= n_cells): omega_k = rho (Y'_k - Y_k) / dt
 *     in kg/(m^3 s), rho the real-fluid (Peng-Robinson) density at the cell's (T, p, Y);
 *   T_new (device [n_cells], may be NULL): T' from h(T', p, Y') = h0.
 * Cells that do not react, and flagged cells, get omega = 0 and T' = T. cell_status and
 * n_active_out as in df_chem_step. Asynchronous.
 * Paper: Sec. 2 (the chemistry network yields the chemical source terms omega-dot that the
 * transport equations of the flow solver consume). */
df_status df_chem_source(df_state* s, int64_t n_cells, double dt, const double* T,
                         const double* p, const double* Y, int64_t ldY, double* omega, int64_t ldw,
                         double* T_new, int32_t* cell_status, int64_t* n_active_out, void* stream);

/* Jacobian of the reaction step of each cell (every cell treated as reacting), with p fixed
 * and the inputs (T, Y_1..Y_n) taken as independent (no renormalisation of the input):
 *   J_dY  (device, [n_cells][n][n+1] row-major FP32): d(Y'_k - Y_k) / d(T, Y_1..Y_n);
 *   dTnew (device, [n_cells][n+1] FP64, may be NULL): dT'/d(T, Y_1..Y_n).
 * Forward-mode tangents through the network (Sec. 2's chemistry network; GELU of Sec. 3.3.2)
 * -- FP32 on the CUDA cores for a DF_FP32 state, BF16 tcgen05 GEMMs otherwise -- then the
 * chain through de-normalisation, renormalisation and the implicit function
 * h(T', p, Y') = h0(T, p, Y). The Box-Cox slope is taken at max(Y_j, 1e-12). Cells whose step
 * would be flagged get NaN entries. Allocates its buffers at the first call on a state: it runs
 * in batches of min(batch_cells, 65,536) cells, whose tangent activations take about
 * 2 x batch x (n + 1) x (widest hidden layer) elements (13 GB in BF16 for 30 species and a
 * 1600-wide layer). Uses the state's scratch, so it must not overlap other calls on the same
 * state.
 * Paper: Sec. 2 (the step whose derivative this is); the paper prints no Jacobian, which is
 * this library's extension for implicit coupling and training. */
df_status df_chem_jacobian(df_state* s, int64_t n_cells, const double* T, const double* p,
                           const double* Y, int64_t ldY, float* J_dY, double* dTnew, void* stream);

/* Reverse-mode product of the reaction step, the adjoint of df_chem_jacobian: it lets a model
 * that contains the step (Sec. 2's network followed by the real-fluid T-from-h solve) be
 * trained by back-propagation, e.g. through a torch.autograd.Function. Given cotangents of the
 * step's outputs (T', Y'),
 *   gT    (device [n_cells] FP64) and gY (device, [n][ldg] species-major FP64, ldg >= n_cells),
 * it writes the cotangents of the inputs (T, Y) with p fixed and the Y_j independent:
 *   out_gT[c]    = gT[c] dT'/dT   + sum_k gY[k][c] dY'_k/dT,
 *   out_gY[j][c] = gT[c] dT'/dY_j + sum_k gY[k][c] dY'_k/dY_j     ([n][ldo], ldo >= n_cells),
 * Y'_k = Y_k + (Y'_k - Y_k) with the Jacobian columns of df_chem_jacobian (same precision and
 * Box-Cox floor). Cells that do not react (T <= T_react, or a non-finite T) are left as they
 * were by the step, so their cotangents are copied through; reacting cells that the step would
 * flag get NaN. The outputs must not overlap the inputs. Runs in batches of
 * min(batch_cells, 65,536) cells: the Jacobian of a batch, then its contraction (a warp per
 * cell, FP64 sums in a fixed order, so results repeat bit for bit). Allocates the Jacobian
 * columns of one batch (batch x n x (n+1) FP32 and batch x (n+1) FP64) at its first call, on
 * top of df_chem_jacobian's buffers, and shares that call's restrictions: DF_ERR_UNSUPPORTED
 * for DF_GELU_TABLE, and no overlap with other calls on the same state. Asynchronous.
 * Paper: Sec. 2 (the step); the paper prints no derivative of it (library extension). */
df_status df_chem_step_vjp(df_state* s, int64_t n_cells, const double* T, const double* p,
                           const double* Y, int64_t ldY, const double* gT, const double* gY,
                           int64_t ldg, double* out_gT, double* out_gY, int64_t ldo, void* stream);

/* ---- training of the chemistry network ----
 * The paper trains its network offline and prints no loss; the library's reading: the network
 * is taught the change of the Box-Cox coordinates that a stiff integration of the cell
 * chemistry produces over dt, with the loss
 *   L = (1/B) sum_b sum_k (O_bk - Ohat_bk)^2,  Ohat_k = (BC(Y_target,k) - BC(Y_k) - out_mean_k)
 *                                                       / out_std_k,
 * O the network output for the cell's normalised input (a5). Gradients by a layer-by-layer
 * backward pass through the tanh-form GELU (Sec. 3.3.2); Adam (Kingma & Ba 2015) with bias
 * correction updates FP32 master weights and biases, after which the working copies the
 * reaction step reads (FP32 for a DF_FP32 state, BF16 for a DF_BF16 state) are rewritten in
 * place, so CUDA graphs of the step stay valid. DF_FP8_E4M3 states return DF_ERR_UNSUPPORTED.
 * The first training call on a state allocates the masters, Adam moments and batch buffers
 * (synchronising the device); a later call with a larger batch reallocates the batch buffers.
 * Training calls use the state's training buffers and must not overlap one another.
 * Paper: Sec. 2 (a pre-trained network stands in for the stiff ODE integration of the
 * chemistry), Sec. 3.3.2 (the activation); the training itself is offline in the paper. */
typedef struct {
  double lr;                  /* step size, > 0 */
  double beta1;               /* first-moment decay, 0 <= beta1 < 1 */
  double beta2;               /* second-moment decay, 0 <= beta2 < 1 */
  double eps;                 /* denominator guard, > 0 */
} df_adam;

/* One Adam step on `batch` states: network input from (T, p, Y) (a1-a5, FP64), targets from
 * Y and Y_target (device, species-major like Y, same ld), forward pass, loss, backward pass,
 * update. loss_out (device or host, may be NULL) receives L as FP32 on `stream`. The states
 * must be valid (finite, p > 0, the PR cubic solvable): a flagged state poisons the step.
 * Paper: Sec. 2 and Sec. 3.3.1 (inputs as for the step); loss and optimiser as stated above. */
df_status df_train_step(df_state* s, int64_t batch, const double* T, const double* p,
                        const double* Y, const double* Y_target, int64_t ld, const df_adam* hp,
                        float* loss_out, void* stream);

/* The building blocks of df_train_step, for a caller that forms its own loss (e.g. a
 * torch.autograd.Function). df_mlp_forward_train is df_mlp_forward (x [n_rows * (n+2)] and
 * O [n_rows * n] row-major FP32, device) that also keeps the activations the backward pass
 * needs. df_mlp_backward takes dL/dO (device [n_rows * n] FP32) for the rows of the last
 * df_mlp_forward_train (n_rows must match) and leaves dL/dW, dL/db in the state (overwriting
 * the previous gradients); dX (device [n_rows * (n+2)] FP32, may be NULL) receives dL/dx.
 * df_adam_step applies the stored gradients.
 * Paper: Sec. 2, Sec. 3.3.2 (the network and its activation, differentiated layer by layer). */
df_status df_mlp_forward_train(df_state* s, int64_t n_rows, const float* x, float* O,
                               void* stream);
df_status df_mlp_backward(df_state* s, int64_t n_rows, const float* dO, float* dX, void* stream);
df_status df_adam_step(df_state* s, const df_adam* hp, void* stream);

/* Copies one layer's FP32 parameters out (W [widths[l+1] * widths[l]] row-major and
 * b [widths[l+1]], device or host pointers, either may be NULL), asynchronously on `stream`:
 * the master weights, the last gradients, or Adam's first or second moments.
 * Paper: no counterpart (inspection of the training state). */
#define DF_PARAM_WEIGHTS 0
#define DF_PARAM_GRADS 1
#define DF_PARAM_ADAM_M 2
#define DF_PARAM_ADAM_V 3
df_status df_get_params(df_state* s, int32_t layer, int32_t which, float* W, float* b,
                        void* stream);
/* Number of Adam steps taken on the state (0 before training). Paper: no counterpart. */
df_status df_train_get_step(df_state* s, int64_t* steps);

/* Saves the master weights, biases, Adam moments and step count to a file; df_state_load
 * restores them into a state of the same network shape (any mechanism) and rewrites the
 * working copies. Both synchronise the device. Paper: no counterpart (checkpointing). */
df_status df_state_save(df_state* s, const char* path);
df_status df_state_load(df_state* s, const char* path);

/* ---- CUDA-graph execution of the step ----
 * A df_graph is one df_chem_step with fixed arguments (sizes, dt and the device buffers T, p,
 * Y, cell_status, n_active_out) captured into an executable CUDA graph, so a time loop replays
 * the whole step (compaction, EoS, every network layer, Newton) with one launch. The state and
 * the buffers must outlive the graph; the graph reads and writes whatever the buffers hold
 * when it runs. df_graph_create runs no kernel: it first makes sure the state's scratch fits
 * n_cells (allocating if needed), then captures on an internal stream.
 * Paper: Sec. 2 (the step, replayed once per flow time step); graphs are this library's means
 * of cutting per-launch cost, with no counterpart in the paper. */
typedef struct df_graph df_graph;
df_status df_graph_create(df_state* s, int64_t n_cells, double dt, double* T, const double* p,
                          double* Y, int64_t ldY, int32_t* cell_status, int64_t* n_active_out,
                          df_graph** out);
/* Enqueues one replay of the captured step on `stream`. Paper: as df_graph_create. */
df_status df_graph_launch(df_graph* g, void* stream);
/* Destroys the graph (synchronising with its last replay). NULL is a no-op.
 * Paper: no counterpart. */
void df_graph_destroy(df_graph* g);

/* ---- tile-width autotuning of the tensor-core layers ----
 * df_autotune times every compiled tile (64, 128, 160, 192, 224, 256 output columns per CTA for
 * hidden layers, and 160, 224, 256 on CTA pairs for hidden layers of more than one k-block of
 * 64 BF16 / 128 FP8 inputs; 32 and 64 for the read-out) of each network layer on n_rows rows of the
 * state's own buffers (<= 0 or above the batch capacity: the capacity), keeps the fastest and
 * re-encodes the layer. cache_path (may be NULL) names a text file of earlier choices, one line
 * per (device, precision, layer shape); known shapes are taken from it without timing and new
 * ones are appended. Synchronises `stream`. A no-op for DF_FP32 states. The tiling changes
 * neither the arithmetic nor its order, so results are bit-identical before and after; call
 * it before capturing graphs (a graph keeps the launch parameters it recorded).
 * df_get_tiles reports the tile of each layer (0 for SIMT layers) in bn[0..max_layers): its
 * width, | DF_TILE_PAIR when the layer runs on CTA pairs (two CTAs of a cluster share one
 * 256-row tile through cta_group::2 MMAs, each holding half of the tile's weight rows), and
 * the number of layers in *n_layers.
 * Paper: Sec. 3.3.3 (the network's matrix products tiled for the memory hierarchy of the
 * target processor); the timing-based choice of tiles has no counterpart in the paper. */
#define DF_TILE_PAIR 0x1000
df_status df_autotune(df_state* s, int64_t n_rows, const char* cache_path, void* stream);
df_status df_get_tiles(df_state* s, int32_t* bn, int32_t max_layers, int32_t* n_layers);

/* Clock budget of every pipeline wait (TMA stage, MMA completion, accumulator hand-over) in the
 * tensor-core kernels of the state's reaction-step network layers: clocks > 0 sets it, clocks
 * <= 0 restores the default (about one second of SM clocks). A wait that outlasts its budget
 * makes the kernel give up: it sets the state's timeout flag, lets the copies and MMAs it has
 * in flight finish (those drains always allow the full default), frees its tensor memory and
 * returns; the step's later kernels still run on whatever the network left, and
 * df_get_step_summary reports DF_ERR_TIMEOUT once. A budget of a few hundred clocks makes
 * waits give up on purpose, which is how the timeout path is tested without a fault. Applies
 * to launches made after the call (a captured graph keeps the budget it was captured with).
 * DF_ERR_UNSUPPORTED for DF_FP32 states (no tensor-core layers). Paper: no counterpart
 * (failure handling). */
df_status df_set_wait_limit(df_state* s, int64_t clocks);

/* Statistics of the last df_chem_step on a state. Paper: no counterpart (diagnostics). */
typedef struct {
  int64_t n_active;           /* reacting cells */
  int64_t n_flagged;          /* reacting cells that received a DF_CELL_* flag */
  int64_t newton_iterations;  /* T-from-h Newton iterations summed over reacting cells */
} df_step_stats;

/* Synchronises `stream`, fills *stats (may be NULL) for the last df_chem_step, and returns
 * DF_OK, DF_ERR_NOT_CONVERGED if any reacting cell was flagged, or DF_ERR_TIMEOUT if a
 * kernel wait gave up since the previous call. Paper: no counterpart (diagnostics). */
df_status df_get_step_summary(df_state* s, void* stream, df_step_stats* stats);

/* ---- stage entry points: the steps of df_chem_step one at a time (same kernels) ---- */

/* a0: idx (device, [n_cells] int32) receives the ascending indices of cells with
 * T > T_react, count (device, one int64) their number. n_cells above INT32_MAX is rejected
 * with DF_ERR_INVALID_ARG (the indices are int32).
 * Paper: Sec. 2 (the chemistry load varies from cell to cell, the motivation for treating only
 * reacting cells) and Sec. 3.3.3 (the network runs on batches). */
df_status df_active_compact(df_state* s, int64_t n_cells, const double* T, int32_t* idx,
                            int64_t* count, void* stream);

/* a1-a5 for n_cells cells: h0 (device [n_cells], may be NULL) the conserved enthalpy,
 * Z (device, may be NULL), x (device [n_cells * (n+2)] row-major FP32, may be NULL) the
 * normalised network input, status (device int32, may be NULL).
 * Paper: Sec. 2 (inputs T, p, Y_i; Peng-Robinson state), Sec. 3.3.1 (Z-scored inputs, FP64). */
df_status df_eos_pre(df_state* s, int64_t n_cells, const double* T, const double* p,
                     const double* Y, int64_t ldY, double* h0, double* Z, float* x,
                     int32_t* status, void* stream);

/* a6-a7: network output O (device [n_rows * n] row-major FP32) from input x (device
 * [n_rows * (n+2)] row-major FP32), computed in the state's precision.
 * Paper: Sec. 2 (the chemistry network), Sec. 3.3.1 (reduced precision), Sec. 3.3.2 (GELU),
 * Sec. 3.3.3 (batched products with the next batch's data fetched during the current one). */
df_status df_mlp_forward(df_state* s, int64_t n_rows, const float* x, float* O, void* stream);

/* a8-a10 given the network output O [n_cells * n] and h0 [n_cells]: writes Y' into Y and
 * T' into T (device, in place), status (device int32, may be NULL).
 * Paper: Sec. 2 (the chemical change applied to the cell; T from the conserved energy through
 * the real-fluid EoS), Sec. 3.3.1 (FP64). */
df_status df_eos_post(df_state* s, int64_t n_cells, const float* O, const double* h0,
                      double* T, const double* p, double* Y, int64_t ldY, int32_t* status,
                      void* stream);

/* ---- allocation-free compaction ----
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory, e.g. a flow solver whose pool allocator owns the whole device, or
 * a caller on a path where cudaMalloc's implicit device-wide synchronisation is not
 * acceptable. It does what df_active_compact does (a0: idx receives the ascending indices of
 * cells with T > T_react, count their number; device pointers, async on `stream`) without a
 * df_state and without allocating: its scratch is a 256 KB array in the library's device
 * image, resident on every device that loads the library until the process exits.
 *   - n_cells above DF_COMPACT_STATIC_MAX_CELLS is rejected with DF_ERR_INVALID_ARG; the
 *     reason is available from df_get_last_error(NULL).
 *   - The first call in a CUDA context looks up the array's device address in that context
 *     (once per context, with the device current; a driver-API context of the caller's own, or
 *     the new primary context after cudaDeviceReset, gets its own lookup); make that first call
 *     before any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU (different streams or host
 *     threads) race and must be serialised by the caller. */
#define DF_COMPACT_STATIC_MAX_CELLS ((int64_t)1 << 26)
df_status df_active_compact_static(int64_t n_cells, double T_react, const double* T,
                                   int32_t* idx, int64_t* count, void* stream);

/* ---- kernel timing ---- */

/* When enabled, df_chem_step records a pair of CUDA events on its stream around each of its
 * kernel launches, grouped into families ("compact", "eos_pre", "layer0".."layer7",
 * "eos_post"). Costs two event records per launch; off by default. Paper: no counterpart. */
df_status df_profile_enable(df_state* s, int32_t enable);

/* Synchronises the device and reports, for up to max_entries families in first-launch order,
 * names (max_entries x 32 chars, NUL-terminated), launches and total device time in ms
 * since the last read or enable; then resets the counters. *n_entries receives the count.
 * Paper: no counterpart. */
df_status df_profile_read(df_state* s, int32_t max_entries, char* names, int64_t* launches,
                          double* total_ms, int32_t* n_entries);

/* Description of the most recent error on this state (or of the last failed create when
 * s is NULL). Valid until the next call on the same state. Paper: no counterpart. */
const char* df_get_last_error(df_state* s);

/* Library version string. Paper: no counterpart. */
const char* df_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DF_H */
