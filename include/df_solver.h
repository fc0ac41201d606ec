/*
 * df_solver.h -- C ABI of the sparse-solver kernels of libdfgb.so: the many-core PDE solver of
 * the DeepFlame method (Sec. 3.2), re-designed for one GB300.
 *
 * The transport equations are discretised by finite volumes on an unstructured mesh into sparse
 * systems in LDU form (Sec. 3.2, OpenFOAM's addressing): face f joins cells owner[f] <
 * neighbour[f]; A[owner][neighbour] = upper[f], A[neighbour][owner] = lower[f], A[c][c] = diag[c].
 * The paper's solver module, and where each part lives here:
 *   - Sec. 3.2.1: decompose the mesh into t subdomains by recursive graph bisection and number
 *     each subdomain's cells contiguously in Cuthill-McKee order           -> df_mesh_decompose,
 *                                                                            df_mesh_renumber;
 *   - Sec. 3.2.2: hold the matrix as t x t blocks (block row I = the rows of subdomain I), each
 *     block CSR, and refresh its values from LDU through positions computed once, because only
 *     the values change between time steps                                -> df_solver_create,
 *                                                                            df_solver_convert;
 *   - Sec. 3.2.3: SpMV, and Gauss-Seidel in which every worker smooths its own block row and
 *     the couplings through off-diagonal blocks are not waited for        -> df_solver_spmv,
 *                                                                            df_solver_residual,
 *                                                                            df_solver_gauss_seidel;
 *   - Sec. 3.2.4: face-to-cell matrix assembly without write conflicts    -> df_fv_laplacian.
 * On the GPU a block row is the work of one CTA (SpMV, and the part of a Gauss-Seidel sweep that
 * uses values from before the sweep) or one warp (the dependent part of the sweep, with the
 * block row's new x in shared memory); in-block columns are 16-bit local indices, and the
 * dependencies inside a block row follow a precomputed schedule of chunks of independent rows.
 *
 * Conventions (in addition to those of df.h):
 *   - Arrays are DEVICE pointers, FP64 values, unless an argument says HOST.
 *   - Vectors are indexed by cell in the numbering the solver was created with; matrices are
 *     given in LDU form over that numbering (see df_mesh_renumber to get there).
 *   - Kernels are enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and return
 *     without synchronising. A df_solver is used by one host thread and one stream at a time
 *     (Gauss-Seidel keeps its halo buffers in the solver).
 *   - Errors: a df_status code; df_solver_get_last_error(s) (or df_get_last_error(NULL) for
 *     the host helpers and df_solver_create) describes it; nothing is enqueued on error unless
 *     the code is DF_ERR_CUDA.
 */
#ifndef DF_SOLVER_H
#define DF_SOLVER_H

#include <stdint.h>

#include "df.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct df_solver df_solver;

/* Largest block row, in cells: in-block columns are 16-bit and a block row's x lives in the
 * shared memory of one warp during a Gauss-Seidel sweep. Sweeps run best with a few hundred to
 * a thousand cells per block row (tens of block rows resident per SM). */
#define DF_SOLVER_MAX_PART 8192

/* Arithmetic of SpMV, residual and Gauss-Seidel (df_solver_set_arithmetic). Storage is FP64 in
 * both; the FP64 pipe of this GPU runs at 1/64 of the FP32 rate. */
#define DF_SOLVER_FP64 0          /* FP64 fused multiply-adds: the default */
#define DF_SOLVER_DOUBLE_FLOAT 1  /* products and sums as unevaluated pairs of FP32 numbers on the
                                     FP32 pipes (Dekker / Knuth), rounded to FP64 per row: each row
                                     within about 2^-44 of sum_c |a_rc x_c| */

/* Sec. 3.2.1, on the HOST. Partitions the cell graph (cells = nodes, faces = edges) into
 * n_parts subdomains by recursive bisection along breadth-first level structures grown from
 * pseudo-peripheral cells (George & Liu), splitting the cell counts in proportion to the parts
 * on each side, so subdomain sizes differ by at most one cell per bisection level. Then numbers
 * the cells of each subdomain contiguously: Cuthill-McKee (breadth-first from a
 * pseudo-peripheral cell, neighbours in ascending degree), followed by a stable sort on each
 * cell's level in the dependency order that numbering induces (level = 1 + the highest level
 * among its earlier-numbered neighbours in the subdomain). The sort keeps the relative order of
 * every pair of neighbours, so a Gauss-Seidel sweep in this numbering is the sweep in
 * Cuthill-McKee order, and cells of one level are consecutive.
 *   owner, neighbour: HOST [n_faces], cells of each face, 0 <= . < n_cells, distinct; any order.
 *   n_parts: 1 .. n_cells.
 *   new_of_old: HOST out [n_cells], the new number of each cell.
 *   part_ptr: HOST out [n_parts + 1], subdomain I = new cells part_ptr[I] .. part_ptr[I+1]-1.
 * DF_ERR_INVALID_ARG on bad sizes or indices. Multi-threaded on the host; deterministic. */
df_status df_mesh_decompose(int64_t n_cells, int64_t n_faces, const int32_t* owner,
                            const int32_t* neighbour, int32_t n_parts, int32_t* new_of_old,
                            int64_t* part_ptr);

/* On the HOST: the mesh in a new cell numbering, in LDU face order. Face k of the output joins
 * owner_out[k] < neighbour_out[k] (new numbers), faces sorted by (owner, neighbour). face_old[k]
 * is the input face it came from; face_flip[k] = 1 where the orientation was reversed, i.e.
 * where the new face's lower coefficient is the old face's upper one (face_flip may be NULL).
 * All arrays HOST, [n_faces] except new_of_old [n_cells], which must be a permutation. */
df_status df_mesh_renumber(int64_t n_cells, int64_t n_faces, const int32_t* owner,
                           const int32_t* neighbour, const int32_t* new_of_old,
                           int32_t* owner_out, int32_t* neighbour_out, int64_t* face_old,
                           uint8_t* face_flip);

/* Sec. 3.2.2. Builds, on the HOST, the block-sparse structure of the mesh's matrices and the
 * positions that map LDU coefficients onto it, plus the Gauss-Seidel schedule (maximal runs of
 * consecutive rows of a block row with no dependency among them), the halo (cells read by
 * another block row) and the cell-to-face lists of the assembly; uploads them to `device`.
 *   owner, neighbour: HOST [n_faces], owner[f] < neighbour[f] < n_cells, no repeated pair, any
 *     face order; this face order is the order of the LDU arrays of the other calls.
 *   part_ptr: HOST [n_parts + 1], 0 = part_ptr[0] < ... < part_ptr[n_parts] = n_cells, each
 *     block row at most DF_SOLVER_MAX_PART cells. Any numbering is accepted; one from
 *     df_mesh_decompose gives few, wide Gauss-Seidel runs and few off-block entries.
 * Limits: n_cells < 2^31, n_faces < 2^30, at most 255 earlier-numbered in-block neighbours per
 * cell (DF_ERR_UNSUPPORTED beyond). Synchronous; *out receives the solver. */
df_status df_solver_create(int64_t n_cells, int64_t n_faces, const int32_t* owner,
                           const int32_t* neighbour, int32_t n_parts, const int64_t* part_ptr,
                           int32_t device, df_solver** out);

void df_solver_destroy(df_solver* s);

typedef struct {
  int64_t n_cells, n_faces, n_parts;
  int64_t nnz;              /* n_cells + 2 n_faces */
  int64_t nnz_offblock;     /* entries in off-diagonal blocks */
  int64_t n_halo;           /* cells read by another block row */
  int64_t n_runs;           /* Gauss-Seidel row runs over all block rows */
  int32_t max_part;         /* cells in the largest block row */
  int32_t max_runs;         /* most runs in one block row */
  int64_t device_bytes;     /* device memory held by the solver */
  int64_t n_chunks;         /* Gauss-Seidel chunks (runs cut to at most 32 rows) */
} df_solver_info;

df_status df_solver_get_info(const df_solver* s, df_solver_info* info);

/* Selects the arithmetic of the following spmv / residual / gauss_seidel calls (DF_SOLVER_FP64
 * or DF_SOLVER_DOUBLE_FLOAT); host-side only, takes effect for later launches. */
df_status df_solver_set_arithmetic(df_solver* s, int32_t arithmetic);

/* Sec. 3.2.2: refreshes the block matrix from LDU coefficients (DEVICE, lower/upper [n_faces]
 * in the creation face order, diag [n_cells]). Entries are copied exactly; the reciprocal of
 * the diagonal used by Gauss-Seidel is formed here (a zero diagonal gives non-finite sweeps).
 * Must precede the first spmv / residual / gauss_seidel (DF_ERR_INVALID_ARG otherwise). */
df_status df_solver_convert(df_solver* s, const double* lower, const double* diag,
                            const double* upper, void* stream);

/* Sec. 3.2.3: y = A x, x and y [n_cells], x != y. */
df_status df_solver_spmv(df_solver* s, const double* x, double* y, void* stream);

/* r = b - A x, r distinct from b and x. */
df_status df_solver_residual(df_solver* s, const double* b, const double* x, double* r,
                             void* stream);

/* Sec. 3.2.3: `sweeps` block Gauss-Seidel sweeps on x in place (b distinct from x). One sweep:
 * in each block row, rows in ascending order take x_r = (b_r - sum_{c != r} A_rc x_c) / A_rr
 * with the values of the block's earlier rows already updated in this sweep and the values of
 * other blocks' cells as they were before the sweep. Deterministic. sweeps >= 0. */
df_status df_solver_gauss_seidel(df_solver* s, const double* b, double* x, int32_t sweeps,
                                 void* stream);

/* Sec. 3.2.4: LDU coefficients of the finite-volume operator
 *   (A x)_c = s_c x_c + sum over faces f of c of g_f (x_c - x_other(f)),
 * i.e. lower[f] = upper[f] = -g_f and diag[c] = s_c + sum over faces of c of g_f, summed in
 * ascending face order by one thread per cell (no two threads write one value).
 * face_coeff [n_faces], cell_source [n_cells] in; lower, upper [n_faces], diag [n_cells] out. */
df_status df_fv_laplacian(df_solver* s, const double* face_coeff, const double* cell_source,
                          double* lower, double* diag, double* upper, void* stream);

/* The converted matrix as plain CSR with ascending columns, into HOST arrays row_ptr
 * [n_cells + 1], col [nnz], val [nnz] (nnz from df_solver_get_info). Synchronises the device.
 * For checking the block format against a reference. */
df_status df_solver_export_csr(df_solver* s, int64_t* row_ptr, int32_t* col, double* val);

const char* df_solver_get_last_error(const df_solver* s);

#ifdef __cplusplus
}
#endif

#endif /* DF_SOLVER_H */
