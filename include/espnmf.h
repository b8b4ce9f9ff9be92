/*
 * espnmf.h -- C ABI of the GB300 (sm_103a) library for enforced-sparsity
 * alternating-least-squares non-negative matrix factorisation
 * (Gavin, Gadepally, Kepner, arXiv:1510.05237).
 *
 * The problem (Eq. 1, Eq. 2): a non-negative data matrix A (n terms x m
 * documents) is approximated by U V^T with U (n x k) >= 0 and V (m x k) >= 0.
 * Alg. 2 alternates two half-steps, each a sparse product, a k x k Gram
 * solve, a projection onto U, V >= 0 and an enforcement step that keeps
 * only the t largest entries (per column by default, Sec. 4; or over the
 * whole matrix as Alg. 2 prints it; or none, which is Alg. 1).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an espnmf_status; nothing throws across the ABI.
 *     After a failure, espnmf_last_error(ctx) holds a one-line message.
 *   - Sizes are int64_t; row/column indices are int32_t; CSR row pointers
 *     are int64_t.  Dense matrices are row-major and contiguous (ld = cols).
 *   - A context owns all device memory it allocates and copies every input
 *     it is given, so the caller may free its buffers once a call returns.
 *   - A context is used by one host thread at a time.  All device work is
 *     enqueued on the context's stream (the caller's, or its own if the
 *     caller passed NULL).  Calls that return host values synchronise that
 *     stream; the others are asynchronous.
 *   - The device that is current at espnmf_init is used for the context's
 *     lifetime; every call makes it current again.
 *   - There is no CPU fallback: without a usable CUDA device the calls
 *     return ESPNMF_ERR_CUDA.
 */
#ifndef ESPNMF_H
#define ESPNMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ESPNMF_OK = 0,
    ESPNMF_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range */
    ESPNMF_ERR_BAD_MATRIX = 2,    /* A is not a valid non-negative CSR matrix (Eq. 1: A >= 0) */
    ESPNMF_ERR_SINGULAR = 3,      /* a Gram matrix (U^T U or V^T V) is singular beyond its zero columns */
    ESPNMF_ERR_NONFINITE = 4,     /* a NaN or Inf appeared in an input or an iterate */
    ESPNMF_ERR_OOM = 5,           /* device or host allocation failed */
    ESPNMF_ERR_CUDA = 6,          /* a CUDA call failed (no device, launch error, ...) */
    ESPNMF_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
    ESPNMF_ERR_UNSUPPORTED = 8    /* a valid request the library does not implement */
} espnmf_status;

/* Arithmetic of a context (or the element type of a buffer).
 * ESPNMF_F64: everything in FP64 (the plain form).
 * ESPNMF_F32: A's values, the factors, the sparse products and the k x k
 *   solve applied to each row in FP32; the Gram matrices, their inverses
 *   and the residual/error reductions in FP64. */
typedef enum { ESPNMF_F64 = 0, ESPNMF_F32 = 1, ESPNMF_BF16 = 2 } espnmf_dtype;

/* Enforcement step of Alg. 2 (steps 2 and 4).
 * COLUMN: keep the t largest positive entries of every column (Sec. 4).
 * MATRIX: keep the t largest positive entries of the whole factor (Alg. 2).
 * NONE:   keep every positive entry (Alg. 1, projected ALS).
 * In every mode exactly min(t, #positive) entries survive; among equal
 * values the lower row index (COLUMN) or the lower row-major index i*k+c
 * (MATRIX) wins; zeros are never kept. */
typedef enum {
    ESPNMF_TOPT_COLUMN = 0,
    ESPNMF_TOPT_MATRIX = 1,
    ESPNMF_TOPT_NONE = 2
} espnmf_topt_mode;

typedef enum { ESPNMF_U = 0, ESPNMF_V = 1 } espnmf_which;

typedef enum {
    ESPNMF_DENSE_ROWMAJOR = 0,   /* rows x k values, zeros included */
    ESPNMF_CSC = 1,              /* ptr[k+1], idx[nnz] = row (ascending), val[nnz] */
    ESPNMF_CSR = 2               /* ptr[rows+1], idx[nnz] = column (ascending), val[nnz] */
} espnmf_layout;

/* The data matrix A (n x m, Eq. 1), compressed sparse rows over terms.
 * rowptr[n+1] non-decreasing from 0 to nnz; colidx[nnz] in [0, m),
 * strictly increasing within each row; values[nnz] finite and >= 0, of
 * type vdtype (F64 or F32).  on_device = 1 means all three arrays live in
 * device memory of the current device, 0 means host memory. */
typedef struct {
    int64_t n;
    int64_t m;
    int64_t nnz;
    const int64_t *rowptr;
    const int32_t *colidx;
    const void *values;
    espnmf_dtype vdtype;
    int32_t on_device;
} espnmf_csr;

typedef struct espnmf_ctx espnmf_ctx;

/* ------------------------------------------------------------------------ */
/* Set-up and tear-down                                                     */

/* espnmf_init -- Alg. 2 "START": validate and copy A, set U = U0.
 *   out      receives the new context (NULL on failure).
 *   A        the data matrix (see espnmf_csr); validated: monotone rowptr,
 *            sorted in-range column indices, finite non-negative values.
 *   k        rank, 1 <= k <= min(n, m) and k <= 128.
 *   t_u,t_v  maximum nonzeros kept in U and V (Alg. 2 input): per column in
 *            COLUMN mode (values above the column length behave as the
 *            column length), in total in MATRIX mode; ignored for NONE.
 *            Must be >= 0.
 *   mode     enforcement mode (see espnmf_topt_mode).
 *   compute  ESPNMF_F64 or ESPNMF_F32 (ESPNMF_BF16 returns UNSUPPORTED).
 *            A's values (A->vdtype) and U0 may be F64, F32 or BF16; BF16
 *            inputs are widened exactly (the BF16 bits are the high half of
 *            an FP32 word) and computed on in the compute type.
 *   U0       initial guess, n x k row-major of type U0_dtype (F64, F32 or BF16),
 *            host (U0_on_device = 0) or device memory; entries must be
 *            finite and >= 0.  U0 is not enforced (Alg. 2 starts from it
 *            as given).
 *   stream   a cudaStream_t for all of the context's work, or NULL to let
 *            the context create its own.
 * A is brought to the host (copied back first when it is on the device),
 * validated there, and laid out by host code: its transpose, the two
 * sliced-ELLPACK layouts (rows of A and rows of A^T) with their
 * frequent-row parts; the layouts are then uploaded.  In the FP32 form,
 * FP32 values are read in place and the layouts hold every value rounded
 * to FP32; the FP64 form keeps them in FP64.  U0 is placed in the
 * row-packed sparse factor layout and its FP64 Gram U0^T U0 formed on the
 * device.  The call synchronises; its cost grows with nnz (host work). */
espnmf_status espnmf_init(espnmf_ctx **out, const espnmf_csr *A, int32_t k,
                          int64_t t_u, int64_t t_v, espnmf_topt_mode mode,
                          espnmf_dtype compute, const void *U0,
                          espnmf_dtype U0_dtype, int32_t U0_on_device,
                          void *stream);

/* espnmf_destroy -- frees everything the context owns (NULL is a no-op).
 * Waits for the context's outstanding work first. */
espnmf_status espnmf_destroy(espnmf_ctx *ctx);

/* One-line description of the last failure on ctx ("" if none).  The
 * pointer stays valid until the next call on ctx.  ctx may be NULL, which
 * returns the message of the last failed espnmf_init on this thread. */
const char *espnmf_last_error(const espnmf_ctx *ctx);

/* Name of a status code. */
const char *espnmf_status_string(espnmf_status st);

/* ------------------------------------------------------------------------ */
/* The alternating update (Alg. 2)                                          */

/* espnmf_als_update_V -- Alg. 2 steps 1-2:
 *   V = A^T U (U^T U)^-1, negative entries set to zero, then only the t_v
 *   largest nonzeros kept (mode of the context).
 * Also forms V^T V in FP64; its inverse is taken at the start of the next
 * U update, beside that update's sparse product.
 * Asynchronous.  Errors found on the device (a non-finite value, a singular
 * V^T V) are reported by the next synchronising call. */
espnmf_status espnmf_als_update_V(espnmf_ctx *ctx);

/* espnmf_als_update_U -- Alg. 2 steps 3-4:
 *   U = A V (V^T V)^-1, negative entries set to zero, then only the t_u
 *   largest nonzeros kept.
 * Also computes, on the device and without forming U V^T, the relative
 * residual R = ||U_new - U_old||_F / ||U_new||_F and the relative error
 * E = ||A - U V^T||_F / ||A||_F (Sec. 3.1), and U^T U in FP64 for the next
 * V update.  Asynchronous. */
espnmf_status espnmf_als_update_U(espnmf_ctx *ctx);

/* espnmf_iterate -- `iters` sweeps of Alg. 2 (each: update_V then
 * update_U).  R_out and E_out are host arrays of `iters` doubles receiving
 * R and E after each sweep, or NULL.  Synchronises once at the end (only
 * if R_out or E_out is non-NULL; otherwise it stays asynchronous).
 * The sweep is replayed from a captured CUDA graph unless graphs were
 * switched off with espnmf_set_option. */
espnmf_status espnmf_iterate(espnmf_ctx *ctx, int32_t iters, double *R_out,
                             double *E_out);

/* espnmf_enforce_topt -- applies the enforcement rule (Alg. 2 step 2 or 4,
 * per the context's mode) with a new limit t to the current U or V in
 * place, then refreshes that factor's Gram matrix.  The context's own t_u /
 * t_v are unchanged. */
espnmf_status espnmf_enforce_topt(espnmf_ctx *ctx, espnmf_which which,
                                  int64_t t);

/* espnmf_set_factor -- replaces U or V with a dense rows x k row-major
 * matrix (F64, F32 or BF16, host or device), finite and >= 0, without
 * enforcement; refreshes its Gram matrix.  Used to start a step from a
 * chosen iterate. */
espnmf_status espnmf_set_factor(espnmf_ctx *ctx, espnmf_which which,
                                const void *F, espnmf_dtype dtype,
                                int32_t on_device);

/* ------------------------------------------------------------------------ */
/* Checkpoints (the paper has no counterpart: this is run management)       */

/* espnmf_save -- writes the context's state to the file `path` (replaced
 * atomically through `path`.tmp): format version, n, m, k, t_u, t_v, mode,
 * arithmetic, the number of completed sweeps, the caller's 64-bit `tag`
 * (e.g. the seed of the initial guess), U and V dense row-major in the
 * context's arithmetic, the FP64 Gram matrices U^T U and V^T V, each
 * factor's last selection thresholds (the FP32 form's selector starts
 * from them, and they decide how it groups the Gram diagonal's partial
 * sums), and a checksum.  A is not saved.  Synchronises. */
espnmf_status espnmf_save(espnmf_ctx *ctx, const char *path, uint64_t tag);

/* espnmf_load -- restores a state written by espnmf_save into a context
 * made by espnmf_init from the same A with the same k, t_u, t_v, mode and
 * arithmetic (any U0 of the right shape): U, V, their Gram matrices, the
 * selection thresholds and the sweep count.  The sweeps that follow repeat, bit for bit, those of the
 * context that saved the state.  tag and sweeps (may be NULL) receive the
 * saved tag and sweep count.  A file of another shape, mode, t or
 * arithmetic, a truncated file or a checksum mismatch gives
 * ESPNMF_ERR_INVALID_ARG and leaves the context unchanged.  Synchronises. */
espnmf_status espnmf_load(espnmf_ctx *ctx, const char *path, uint64_t *tag, int64_t *sweeps);

/* espnmf_topic_accuracy -- the document-clustering accuracy of every topic
 * (Sec. 3.2, Eq. 3-4) from the current factor (usually V: its rows are the
 * documents), on the device.  Row i belongs to topic c when entry (i, c) is
 * nonzero; labels[i] in [0, n_classes) is row i's class (device memory when
 * on_device != 0, else host); acc receives k doubles on the host:
 * (P - alpha) / (beta - alpha) with P the member pairs sharing a class,
 * alpha that count for the most even spread over the classes, beta all
 * pairs; 1 for topics of at most one member or when beta == alpha.  A
 * member row's label outside the range gives ESPNMF_ERR_INVALID_ARG.
 * Synchronises. */
espnmf_status espnmf_topic_accuracy(espnmf_ctx *ctx, espnmf_which which, const int32_t *labels,
                                    int32_t n_classes, int32_t on_device, double *acc);

/* espnmf_sweeps_done -- completed sweeps (U updates) since espnmf_init, or
 * since the state restored by espnmf_load counting its saved sweeps. */
espnmf_status espnmf_sweeps_done(espnmf_ctx *ctx, int64_t *sweeps);

/* ------------------------------------------------------------------------ */
/* Measures (Sec. 3.1)                                                      */

/* espnmf_residual -- R = ||U_i - U_{i-1}||_F / ||U_i||_F of the last
 * espnmf_als_update_U (U_{i-1} being U before that update).  R = 0 when
 * both are zero, +inf when only U_i is zero.  Returns INVALID_ARG if no U
 * update has run.  Synchronises. */
espnmf_status espnmf_residual(espnmf_ctx *ctx, double *R);

/* espnmf_error -- E = ||A - U V^T||_F / ||A||_F for the current U and V,
 * through ||A||^2 - 2 <U, A V> + <U^T U, V^T V> (clamped at 0 before the
 * square root; UV^T is never formed).  Reuses the last update's A V when V
 * has not changed since, otherwise runs one sparse product.  E = 0 when
 * ||A|| = 0.  Synchronises. */
espnmf_status espnmf_error(espnmf_ctx *ctx, double *E);

/* ------------------------------------------------------------------------ */
/* Squared objective, its gradient, projected-gradient polish               */

/* espnmf_loss -- f = ||A - U V^T||_F^2 (the squared objective of Sec. 4,
 * Eq. 6) for the current U and V, through the same identity as
 * espnmf_error: f = ||A||^2 - 2 <U, A V> + <U^T U, V^T V> (FP64 sums; U V^T
 * is never formed).  Not clamped at 0, so rounding may leave it slightly
 * negative when the factorisation is exact.  Synchronises. */
espnmf_status espnmf_loss(espnmf_ctx *ctx, double *f);

/* espnmf_grad -- the dense gradient of f with respect to one factor at the
 * current U and V:
 *   which = ESPNMF_U:  grad_U = 2 (U V^T V - A V)    (n x k)
 *   which = ESPNMF_V:  grad_V = 2 (V U^T U - A^T U)  (m x k)
 * out: row-major rows x k (leading dimension k), element type `dtype`
 * (ESPNMF_F64 or ESPNMF_F32), device memory when on_device != 0, else host
 * memory (the call then allocates a device staging buffer for the copy).
 * The product F G_O runs in FP64 over F's nonzeros; A V or A^T U comes
 * from the context's SpMM in its arithmetic.  Synchronises when out is on
 * the host; ESPNMF_ERR_INVALID_ARG when U or V has no value. */
espnmf_status espnmf_grad(espnmf_ctx *ctx, espnmf_which which, void *out,
                          espnmf_dtype dtype, int32_t on_device);

/* espnmf_pg_step -- one projected-gradient step on a factor's current
 * support S (an optional polish between sweeps; the paper has no such
 * step):  F <- P_S(F - eta grad_F f), where P_S clamps to >= 0 and keeps
 * only the entries of S (entries that reach 0 leave the support).
 * eta > 0 is used as given; eta <= 0 takes eta = 1 / (2 lambda_max(G_O)),
 * G_O the other factor's Gram, lambda_max from 20 FP64 power-iteration
 * steps from the normalised all-ones vector (eta = 0, no change, when
 * G_O = 0).  eta_used (host, may be NULL) receives the step.  The factor's
 * Gram is refreshed; R and E are not (espnmf_error recomputes E).
 * Synchronises. */
espnmf_status espnmf_pg_step(espnmf_ctx *ctx, espnmf_which which, double eta,
                             double *eta_used);

/* ------------------------------------------------------------------------ */
/* Factors out                                                              */

/* espnmf_factor_nnz -- number of nonzeros of U or V.  Synchronises. */
espnmf_status espnmf_factor_nnz(espnmf_ctx *ctx, espnmf_which which,
                                int64_t *nnz);

/* espnmf_get_factor -- copies U (n x k) or V (m x k) out in `layout`.
 *   DENSE_ROWMAJOR: val[rows*k]; ptr and idx unused (may be NULL).
 *   CSC: ptr int64[k+1], idx int32[nnz] rows ascending per column, val[nnz].
 *   CSR: ptr int64[rows+1], idx int32[nnz] columns ascending per row, val[nnz].
 * nnz from espnmf_factor_nnz sizes the buffers.  Values are written as
 * `dtype` (F64 or F32).  All buffers are host (on_device = 0) or device
 * memory.  Synchronises. */
espnmf_status espnmf_get_factor(espnmf_ctx *ctx, espnmf_which which,
                                espnmf_layout layout, int64_t *ptr,
                                int32_t *idx, void *val, espnmf_dtype dtype,
                                int32_t on_device);

/* ------------------------------------------------------------------------ */
/* Options and instrumentation                                              */

typedef enum {
    ESPNMF_OPT_USE_GRAPH = 0,     /* 1 (default): espnmf_iterate replays a CUDA graph */
    ESPNMF_OPT_PROFILE = 1,       /* 1: time every kernel launch with CUDA events (eager launches) */
    ESPNMF_OPT_WAIT_LIMIT = 2,    /* iteration limit of bounded device waits (default 1<<26) */
    /* Launch shape of the FP32 sparse products (results are bitwise the same
     * for every shape):
     *   ESPNMF_OPT_SPMM_TUNE 1 (default): before its first captured sweep,
     *     espnmf_iterate times the candidate shapes on the current factors
     *     and keeps the fastest for each product (A V and A^T U); the picks
     *     are remembered for the process by shape class (factor width, log2
     *     of the output rows and of the entries per row, frequent part or
     *     not), and later contexts of the same class reuse them without
     *     timing; 0: fixed.
     *   ESPNMF_OPT_SPMM_SPLIT: 1, 2 or 4 warps share a slice's output
     *     columns (k >= 13 for more than 1); sets both products and turns
     *     tuning off.
     *   ESPNMF_OPT_SPMM_CARVEOUT: preferred shared-memory carveout in percent
     *     (-1: the driver's choice); also turns tuning off.
     *   ESPNMF_OPT_SPMM_MASK: how entries that gather an all-zero factor row
     *     are skipped: 0 not skipped (their record is read), 1 by the
     *     nonzero-row bitmask read from global memory, 2 by the bitmask
     *     staged in shared memory (factors of at most 131072 rows; larger
     *     ones fall back to 1); also turns tuning off. */
    ESPNMF_OPT_SPMM_TUNE = 3,
    ESPNMF_OPT_SPMM_SPLIT = 4,
    ESPNMF_OPT_SPMM_CARVEOUT = 5,
    ESPNMF_OPT_SPMM_MASK = 6,
    /* FP32 form, k <= 64: 1 adds one step of iterative refinement to every
     * row solve X = Y G^-1: the residual R = Y - X G (G as an FP32 pair of
     * about 48 bits, products split exactly, compensated sums) is solved
     * with the same Cholesky factor and added before the projection, which
     * brings X to the FP64 solution of the FP32 system rounded to FP32
     * (within an ulp or two while cond(G) is well below 2^12).  0 (default):
     * no refinement. */
    ESPNMF_OPT_REFINE = 8
} espnmf_option;

espnmf_status espnmf_set_option(espnmf_ctx *ctx, espnmf_option opt,
                                int64_t value);

/* espnmf_spmm_config -- the launch shape in use for a sparse product
 * (product 0: A V of the U update, 1: A^T U of the V update): split = warps
 * per slice, carveout in percent (-1: the driver's choice), mask = how zero
 * factor rows are skipped (ESPNMF_OPT_SPMM_MASK).  Reflects the tuner's pick
 * once espnmf_iterate ran.  Any output may be NULL. */
espnmf_status espnmf_spmm_config(espnmf_ctx *ctx, int32_t product, int32_t *split,
                                 int32_t *carveout, int32_t *mask);

/* espnmf_sequential -- Alg. 3 (sequential ALS, Sec. 4): k = eta * k2
 * topics found k2 at a time.  Block b (columns b*k2 .. b*k2 + k2 - 1) starts
 * from U2 = U0 (the same n x k2 initial guess for every block) and, with the
 * converged topics U1 = U[:, :b*k2], V1 = V[:, :b*k2], runs `iters` times
 *   V2 = (A^T U2 - V1 (U1^T U2)) (U2^T U2)^-1   (Eq. 7), projected, top-t_v
 *                                                per column,
 *   U2 = (A V2 - U1 (V1^T V2)) (V2^T V2)^-1     (Eq. 8), projected, top-t_u
 *                                                per column;
 * then U[:, block] = U2, V[:, block] = V2.  The first block (no converged
 * topics) is Alg. 2 with k2 topics from U0, the START of Alg. 3.  k2 = 1
 * gives rank-1 topics, the case the paper times, where the k2 x k2 solve is
 * a division.  The sparse products, the solve, the projection and the top-t
 * rule are those of Alg. 2 with k = k2 (a k = k2 context built from A, FP32
 * or FP64 form); the deflation term runs in FP64 sums.  Each block's sweeps
 * after its first are replayed from captured CUDA graphs, as
 * espnmf_iterate runs them.  A: as for
 * espnmf_init (copied).  U0: n x k2 row-major (dtype u0_dtype, host or
 * device).  U_out (n x k) and V_out (m x k): row-major DEVICE buffers of the
 * compute dtype, written when the call returns ESPNMF_OK (it synchronises).
 * seconds_out (may be NULL): the stream time from the end of the context's
 * set-up to the last block's append (CUDA events on the call's stream): the
 * ALS iterations of all blocks, without building A's layouts.
 * Errors: espnmf_last_error(NULL).  Requires 1 <= k2, k a multiple of k2,
 * k <= min(n, m), iters >= 1; a singular k2 x k2 Gram (other than zero
 * columns, which give zero output columns) returns ESPNMF_ERR_SINGULAR. */
espnmf_status espnmf_sequential(const espnmf_csr *A, int32_t k, int32_t k2, int64_t t_u,
                                int64_t t_v, int32_t iters, espnmf_dtype compute, const void *U0,
                                espnmf_dtype u0_dtype, int32_t u0_on_device, void *U_out,
                                void *V_out, double *seconds_out, void *stream);

/* espnmf_select_stats -- how the column selections of this context's
 * enforcement steps (FP32 form, column mode) found their thresholds since
 * espnmf_init: warm = columns whose search started from the previous
 * threshold of that column and found the new one in the three histogram
 * bins around it (one pass over the column); full = columns searched from
 * scratch (first sweeps, a threshold that moved by more than about an
 * eighth of a binade, or a crowded window).  Both 0 for FP64 contexts.
 * Synchronises the context's stream.  The paper has no counterpart: this
 * reports on how the rule after Alg. 2 is evaluated, not on what it keeps. */
espnmf_status espnmf_select_stats(espnmf_ctx *ctx, int64_t *warm, int64_t *full);

/* espnmf_spmm_frequent -- the frequent part of a sparse product (product 0:
 * A V, 1: A^T U; FP32 contexts only): h = number of gathered factor rows
 * read densely (0: the product has no frequent part) and hnnz = the
 * entries of A routed to them.  The rows are chosen once by espnmf_init:
 * the gathered rows referenced by the most entries of A (the frequent
 * terms, for A^T U), kept when they carry at least a tenth of the entries.
 * As many as fit a 200 KB table are staged in shared memory; in column
 * mode the part takes up to t of them (at most t rows of the gathered
 * factor can be nonzero in every column), and when that adds at least 256
 * rows beyond the shared-memory table, the extra rows are read from the
 * factor's table in global memory (a second launch).  The paper has no
 * counterpart: this is a layout choice of the sparse product of Alg. 2
 * steps 1 and 3. */
espnmf_status espnmf_spmm_frequent(espnmf_ctx *ctx, int32_t product, int32_t *h,
                                   int64_t *hnnz);

/* Kernel statistics gathered while ESPNMF_OPT_PROFILE is on.
 * espnmf_kernel_stat_count gives the number of kernel kinds; for index i,
 * espnmf_kernel_stat returns its name, launch count, summed event time (ms)
 * and the algorithmic bytes it moved in total.  espnmf_kernel_stats_reset
 * clears them.  Synchronises. */
espnmf_status espnmf_kernel_stat_count(espnmf_ctx *ctx, int32_t *count);
espnmf_status espnmf_kernel_stat(espnmf_ctx *ctx, int32_t i,
                                 const char **name, int64_t *launches,
                                 double *total_ms, double *bytes);
espnmf_status espnmf_kernel_stats_reset(espnmf_ctx *ctx);

/* Number of kernel launches one sweep (update_V + update_U) enqueues. */
espnmf_status espnmf_launches_per_sweep(espnmf_ctx *ctx, int32_t *count);

/* espnmf_checked_flags -- in a library compiled with -DESPNMF_CHECKED (the
 * checked build: build(checked=True), loaded by the binding when the
 * environment sets ESPNMF_CHECKED=1), the union of the bounds checks that
 * failed in any kernel since the last call, then cleared: bit 0 a gathered
 * factor row beyond the factor, bit 1 a pair's column beyond the row width,
 * bit 2 a row's pair count beyond its capacity, bit 3 a frequent-part entry
 * whose table row lies beyond its table, bit 4 an output or partial row out of range, bit 5 a
 * candidate or survivor row beyond the column.  A failed check skips its
 * access.  0: every checked access was in range.  Any other build: *flags
 * = 0 and ESPNMF_ERR_UNSUPPORTED.  Reads device memory (synchronises with
 * the device). */
espnmf_status espnmf_checked_flags(uint32_t *flags);

/* espnmf_sync -- waits for the context's stream; reports device errors. */
espnmf_status espnmf_sync(espnmf_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Stand-alone solve                                                        */

/* espnmf_solve_gram -- the k x k solve of Alg. 2 steps 1 and 3 on a caller's
 * buffers: X = Y G^-1 row by row, unprojected, as the FP32 form computes it
 * (FP64 Cholesky factor of G, FP32 substitutions), with one step of
 * iterative refinement when refine != 0 (see ESPNMF_OPT_REFINE).
 *   Y  rows x k FP32 row-major device matrix (leading dimension ldy >= k).
 *   G  k x k FP64 row-major device matrix, symmetric positive semi-definite;
 *      an index j with G_jj = 0 is dropped (column j of X is 0), any other
 *      pivot at or below 64 eps max G_jj gives ESPNMF_ERR_SINGULAR.
 *   X  rows x k FP32 row-major device output (leading dimension ldx >= k).
 * 1 <= k <= 64.  Scratch comes from the stream-ordered allocator and is
 * freed before the call returns.  Enqueued on `stream` (NULL: legacy
 * default stream); synchronises it; failures are described by
 * espnmf_last_error(NULL). */
espnmf_status espnmf_solve_gram(const void *Y, int64_t rows, int32_t k, int64_t ldy,
                                const double *G, void *X, int64_t ldx, int32_t refine,
                                void *stream);

/* ------------------------------------------------------------------------ */
/* Stand-alone selector                                                     */

/* espnmf_enforce_topt_buffer -- projection plus enforcement (Alg. 2 steps
 * 1-2 after the solve) on a caller's device buffer, in place:
 *   X        rows x k row-major device matrix with leading dimension ld
 *            (ld >= k), element type dtype (F64 or F32).
 *   t, mode  as for the context (t >= 0).
 * Every entry that is not > 0 becomes +0; of the positive entries only
 * min(t, #positive) per column (COLUMN) or in total (MATRIX) survive.
 * If X holds a NaN or an infinity the call returns ESPNMF_ERR_NONFINITE and
 * leaves X unchanged.
 * Scratch memory is allocated from the stream-ordered allocator and freed
 * before the call returns.  Enqueued on `stream` (NULL: legacy default
 * stream); synchronises that stream to report errors. */
espnmf_status espnmf_enforce_topt_buffer(void *X, int64_t rows, int32_t k,
                                         int64_t ld, espnmf_dtype dtype,
                                         int64_t t, espnmf_topt_mode mode,
                                         void *stream);

/* ------------------------------------------------------------------------ */
/* Stand-alone selector that allocates nothing                              */

/* Largest rows * ld(k) (and largest rows) that
 * espnmf_enforce_topt_buffer_noalloc accepts, where ld(k) is k rounded up
 * to a multiple of 4 (k <= 64) or of 16 (k > 64). */
#define ESPNMF_NOALLOC_MAX_ELEMS 262144

/* espnmf_enforce_topt_buffer_noalloc -- the paper has no counterpart: this
 * is espnmf_enforce_topt_buffer (same arguments, same result) for callers
 * that must not allocate device memory while it runs, for instance a
 * service whose device memory is budgeted once at start-up, or a host
 * program that hands all device memory to its own pool.  It calls no
 * cudaMalloc, cudaFree or stream-ordered allocator; its scratch memory is a
 * fixed array compiled into the library (about 2.1 MB, held on every GPU
 * that loads the library until the process exits).
 *   - X larger than ESPNMF_NOALLOC_MAX_ELEMS (rows * ld(k) or rows) is
 *     rejected with ESPNMF_ERR_INVALID_ARG; nothing is modified.
 *   - X holding a NaN or an infinity gives ESPNMF_ERR_NONFINITE and X is
 *     left unchanged.
 *   - Every call looks up the array's device address on the current device
 *     (no cached address survives a device reset); the first call on a
 *     device may load the library's device code there, so make it before
 *     any stream capture.
 *   - All calls share the array: calls whose work overlaps on the GPU
 *     (other streams, other host threads on the same device) race on it and
 *     must be serialised by the caller.
 *   - Synchronises `stream` (NULL: the legacy default stream); failures are
 *     described by espnmf_last_error(NULL). */
espnmf_status espnmf_enforce_topt_buffer_noalloc(void *X, int64_t rows,
                                                 int32_t k, int64_t ld,
                                                 espnmf_dtype dtype, int64_t t,
                                                 espnmf_topt_mode mode,
                                                 void *stream);

/* ------------------------------------------------------------------------ */
/* Batched sweeps of independent problems                                   */

/* Many independent factorisations (uneven n, m, k, t), each a full context,
 * advanced together: espnmf_batch_iterate runs Alg. 2 sweeps of every
 * problem, and from the second sweep on replays one captured CUDA graph per
 * sweep that holds all problems' kernels, spread over a pool of streams so
 * that small problems overlap.  The paper factorises one matrix at a time;
 * batching adds no arithmetic (every problem's results are bitwise those of
 * its own context run alone). */
typedef struct espnmf_batch espnmf_batch;

/* espnmf_batch_init -- one context per problem, as espnmf_init would make
 * it: As[i], ks[i], t_us[i], t_vs[i] and U0s[i] (n_i x k_i row-major,
 * U0_dtype, all on the device or all on the host) for i < nprob; mode and
 * compute are shared.  streams: size of the stream pool (<= 0: 16).  On
 * failure nothing is kept and espnmf_last_error(NULL) names the problem. */
espnmf_status espnmf_batch_init(espnmf_batch **out, int32_t nprob,
                                const espnmf_csr *As, const int32_t *ks,
                                const int64_t *t_us, const int64_t *t_vs,
                                espnmf_topt_mode mode, espnmf_dtype compute,
                                const void *const *U0s, espnmf_dtype U0_dtype,
                                int32_t U0_on_device, int32_t streams);

/* espnmf_batch_destroy -- destroys every problem's context (NULL: no-op). */
espnmf_status espnmf_batch_destroy(espnmf_batch *b);

/* espnmf_batch_ctx -- the context of problem i, owned by the batch (use it
 * for espnmf_get_factor, espnmf_error, ...; do not destroy it).  A call that
 * changes one problem's factors (set_factor, enforce_topt, single updates)
 * makes the next batch sweep run without the graph until the problems are
 * back in step. */
espnmf_status espnmf_batch_ctx(espnmf_batch *b, int32_t i, espnmf_ctx **out);

/* espnmf_batch_set_option -- ESPNMF_OPT_USE_GRAPH only (1: default). */
espnmf_status espnmf_batch_set_option(espnmf_batch *b, espnmf_option opt,
                                      int64_t value);

/* espnmf_batch_iterate -- `iters` sweeps of every problem.  status_out
 * (nprob entries, may be NULL) receives each problem's status (a singular
 * or non-finite problem does not stop the others); R_out and E_out (host,
 * nprob x iters row-major, may be NULL) the per-sweep measures.  Returns the
 * first failing problem's status, or ESPNMF_OK.  Synchronises. */
espnmf_status espnmf_batch_iterate(espnmf_batch *b, int32_t iters,
                                   espnmf_status *status_out, double *R_out,
                                   double *E_out);

#ifdef __cplusplus
}
#endif

#endif /* ESPNMF_H */
