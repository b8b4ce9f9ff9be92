/*
 * espnmf_oracle.c -- plain, slow, FP64 CPU oracle for enforced-sparsity
 * ALS non-negative matrix factorisation (Gavin, Gadepally, Kepner,
 * "Enforced Sparse Non-Negative Matrix Factorization", arXiv:1510.05237).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product (the CUDA
 * library and its Python binding) never calls it, and the two share no code,
 * header, table or helper.
 *
 * Everything is FP64 and written as the paper states it; the file is built
 * single-threaded, and the benchmark's all-cores baseline builds the same
 * source with OpenMP: the loops it parallelises split work between threads
 * without changing any sum's order (each output element is still summed by
 * one thread, in the order below), so both builds give bitwise equal
 * results.  The pragmas are ignored by the single-threaded build.  It
 * covers:
 *   - Alg. 2 (Enforced Sparsity ALS), steps 1-4: V = A^T U (U^T U)^-1,
 *     clamp negatives, keep the t_v largest; U = A V (V^T V)^-1, clamp,
 *     keep the t_u largest.  With enforcement off it is Alg. 1.
 *   - Sec. 2 (after Alg. 2): the top-t rule keeps the entries at or above
 *     the t-th largest magnitude; Sec. 4 (first paragraph) gives the
 *     column-by-column variant.
 *   - Sec. 3.1: R = ||U_i - U_{i-1}|| / ||U_i||, E = ||A - U V^T|| / ||A||.
 *   - Sec. 4, Eq. 6 (the squared objective) gives the loss used by the
 *     gradient helpers.
 *   - Sec. 3.2, Eq. 3-4: the document-clustering accuracy of each topic.
 *
 * Readings where the paper is silent (all norms Frobenius; exactly
 * min(t, #positive) entries kept, ties to the lower index; zero Gram
 * columns dropped and their output set to 0; other Cholesky breakdowns
 * reported as singular) are listed in the design notes and in the comments
 * of the functions below.
 *
 * Matrix A is n x m (terms x documents) in CSR over rows: rowptr[n+1],
 * colidx[nnz], val[nnz].  Factors are dense row-major: U is n x k, V is m x k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Status codes (same meanings as the library's, defined independently). */
enum {
    OR_OK = 0,
    OR_ERR_INVALID_ARG = 1,
    OR_ERR_BAD_MATRIX = 2,
    OR_ERR_SINGULAR = 3,
    OR_ERR_NONFINITE = 4,
    OR_ERR_OOM = 5
};

/* Enforcement modes. */
enum { OR_TOPT_COLUMN = 0, OR_TOPT_MATRIX = 1, OR_TOPT_NONE = 2 };

/* ------------------------------------------------------------------------ */
/* Sparse products, Alg. 2 steps 1 and 3: the "A^T U" and "A V" factors.    */

/* B (m x k) = A^T U.  Loops over A's rows; for every stored a_ij adds
 * a_ij * U[i,:] to B[j,:].  For each B[j,c] the additions therefore come in
 * increasing row index i. */
void or_spmm_At(int64_t n, int64_t m, const int64_t *rowptr,
                const int32_t *colidx, const double *val, int32_t k,
                const double *U, double *B)
{
    memset(B, 0, sizeof(double) * (size_t)m * (size_t)k);
#ifdef _OPENMP
    /* threads own columns of B; every B[j,c] still receives its additions
     * in increasing row index i */
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < k; ++c)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                B[(int64_t)colidx[p] * k + c] += val[p] * U[i * k + c];
#else
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = colidx[p];
            double a = val[p];
            for (int32_t c = 0; c < k; ++c)
                B[j * k + c] += a * U[i * k + c];
        }
#endif
}

/* B (n x k) = A V. */
void or_spmm_A(int64_t n, int64_t m, const int64_t *rowptr,
               const int32_t *colidx, const double *val, int32_t k,
               const double *V, double *B)
{
    (void)m;
    memset(B, 0, sizeof(double) * (size_t)n * (size_t)k);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = colidx[p];
            double a = val[p];
            for (int32_t c = 0; c < k; ++c)
                B[i * k + c] += a * V[j * k + c];
        }
}

/* G (k x k) = F^T F for a rows x k factor F: the "U^T U" / "V^T V" of
 * Alg. 2 steps 1 and 3. */
void or_gram(int64_t rows, int32_t k, const double *F, double *G)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t c = 0; c < k; ++c)
        for (int32_t d = 0; d < k; ++d) {
            double s = 0.0;
            for (int64_t i = 0; i < rows; ++i)
                s += F[i * k + c] * F[i * k + d];
            G[c * k + d] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* The k x k solve of Alg. 2 steps 1 and 3: X = B G^-1 row by row, i.e.
 * x G = b for every row b of B (G symmetric, so G x^T = b^T).
 *
 * Reading (the paper is silent on a singular Gram): an index j with
 * G_jj == 0 belongs to an all-zero factor column; it is dropped, the reduced
 * system is solved, and output column j is 0 (the minimum-norm solution).
 * Any other Cholesky pivot <= 64 * eps * max_j G_jj is reported as
 * OR_ERR_SINGULAR. */
int or_cholesky(int32_t k, const double *G, double *L, int32_t *active)
{
    double maxdiag = 0.0;
    for (int32_t j = 0; j < k; ++j) {
        double d = G[j * k + j];
        if (!isfinite(d)) return OR_ERR_NONFINITE;
        active[j] = d != 0.0;
        if (d > maxdiag) maxdiag = d;
    }
    memset(L, 0, sizeof(double) * (size_t)k * (size_t)k);
    double tol = 64.0 * 2.220446049250313e-16 * maxdiag;
    for (int32_t j = 0; j < k; ++j) {
        if (!active[j]) continue;
        double s = G[j * k + j];
        for (int32_t e = 0; e < j; ++e)
            if (active[e]) s -= L[j * k + e] * L[j * k + e];
        if (!(s > tol)) return OR_ERR_SINGULAR;
        double ljj = sqrt(s);
        L[j * k + j] = ljj;
        for (int32_t i = j + 1; i < k; ++i) {
            if (!active[i]) continue;
            double t = G[i * k + j];
            for (int32_t e = 0; e < j; ++e)
                if (active[e]) t -= L[i * k + e] * L[j * k + e];
            L[i * k + j] = t / ljj;
        }
    }
    return OR_OK;
}

/* Solves x (L L^T) = b for every row: forward substitution L z = b, then
 * back substitution L^T x = z, on the active indices only. */
void or_solve_rows(int64_t rows, int32_t k, const double *L,
                   const int32_t *active, const double *B, double *X)
{
#pragma omp parallel
    {
    double *z = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
#pragma omp for schedule(static)
    for (int64_t r = 0; r < rows; ++r) {
        const double *b = B + r * k;
        double *x = X + r * k;
        for (int32_t j = 0; j < k; ++j) {
            if (!active[j]) { z[j] = 0.0; continue; }
            double s = b[j];
            for (int32_t e = 0; e < j; ++e)
                if (active[e]) s -= L[j * k + e] * z[e];
            z[j] = s / L[j * k + j];
        }
        for (int32_t j = k - 1; j >= 0; --j) {
            if (!active[j]) { x[j] = 0.0; continue; }
            double s = z[j];
            for (int32_t e = j + 1; e < k; ++e)
                if (active[e]) s -= L[e * k + j] * x[e];
            x[j] = s / L[j * k + j];
        }
    }
    free(z);
    }
}

/* X = B G^-1 (the least-squares step before projection). */
int or_ls_solve(int64_t rows, int32_t k, const double *B, const double *G,
                double *X)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)k + 8);
    if (!L || !act) { free(L); free(act); return OR_ERR_OOM; }
    int st = or_cholesky(k, G, L, act);
    if (st == OR_OK) or_solve_rows(rows, k, L, act, B, X);
    free(L);
    free(act);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Projection, Alg. 2 steps 1 and 3: negative entries become zero.
 * Non-finite values are an error, never clamped away.  Everything that is
 * not > 0 (including -0.0) becomes +0.0. */
int or_project(double *X, int64_t count)
{
    for (int64_t q = 0; q < count; ++q)
        if (!isfinite(X[q])) return OR_ERR_NONFINITE;
    for (int64_t q = 0; q < count; ++q)
        X[q] = X[q] > 0.0 ? X[q] : 0.0;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Enforcement, Alg. 2 steps 2 and 4 with the rule stated after Alg. 2:
 * order the entries that are nonzero (after the projection: positive) by
 * size and zero all but the t biggest.  Readings: exactly min(t, #positive) entries are kept; among
 * equal values the lower index wins (row index in column mode, row-major
 * linear index i*k+c in matrix mode); zeros are never kept.
 * OR_TOPT_COLUMN applies the rule to each column separately (Sec. 4),
 * OR_TOPT_MATRIX to the whole matrix (Alg. 2 as printed), OR_TOPT_NONE
 * keeps everything (Alg. 1). */
typedef struct { double v; int64_t idx; } or_entry;

static int or_entry_cmp(const void *a, const void *b)
{
    const or_entry *x = (const or_entry *)a, *y = (const or_entry *)b;
    if (x->v > y->v) return -1;
    if (x->v < y->v) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

int or_topt(double *X, int64_t rows, int32_t k, int64_t t, int mode)
{
    if (t < 0) return OR_ERR_INVALID_ARG;
    if (mode == OR_TOPT_NONE) return OR_OK;
    if (mode == OR_TOPT_COLUMN) {
        int st = OR_OK;
#pragma omp parallel
        {
        or_entry *e = (or_entry *)malloc(sizeof(or_entry) * (size_t)(rows > 0 ? rows : 1));
        if (!e) st = OR_ERR_OOM;
#pragma omp for schedule(dynamic, 1)
        for (int32_t c = 0; c < k; ++c) {
            if (!e) continue;
            int64_t cnt = 0;
            for (int64_t i = 0; i < rows; ++i)
                if (X[i * k + c] > 0.0) { e[cnt].v = X[i * k + c]; e[cnt].idx = i; ++cnt; }
            if (cnt <= t) continue;
            qsort(e, (size_t)cnt, sizeof(or_entry), or_entry_cmp);
            for (int64_t q = t; q < cnt; ++q) X[e[q].idx * k + c] = 0.0;
        }
        free(e);
        }
        return st;
    }
    if (mode == OR_TOPT_MATRIX) {
        int64_t total = rows * (int64_t)k;
        or_entry *e = (or_entry *)malloc(sizeof(or_entry) * (size_t)(total > 0 ? total : 1));
        if (!e) return OR_ERR_OOM;
        int64_t cnt = 0;
        for (int64_t q = 0; q < total; ++q)
            if (X[q] > 0.0) { e[cnt].v = X[q]; e[cnt].idx = q; ++cnt; }
        if (cnt > t) {
            qsort(e, (size_t)cnt, sizeof(or_entry), or_entry_cmp);
            for (int64_t q = t; q < cnt; ++q) X[e[q].idx] = 0.0;
        }
        free(e);
        return OR_OK;
    }
    return OR_ERR_INVALID_ARG;
}

/* ------------------------------------------------------------------------ */
/* One half-step of Alg. 2.
 * or_update_V: steps 1-2 -- V = A^T U (U^T U)^-1, clamp, keep t_v largest.
 * or_update_U: steps 3-4 -- U = A V (V^T V)^-1, clamp, keep t_u largest.
 * If `pre` is non-NULL it receives the least-squares step before the
 * projection. */
int or_update_V(int64_t n, int64_t m, const int64_t *rowptr,
                const int32_t *colidx, const double *val, int32_t k,
                const double *U, int64_t t_v, int mode, double *V, double *pre)
{
    double *B = (double *)malloc(sizeof(double) * (size_t)m * (size_t)k + 8);
    double *G = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    if (!B || !G) { free(B); free(G); return OR_ERR_OOM; }
    or_spmm_At(n, m, rowptr, colidx, val, k, U, B);
    or_gram(n, k, U, G);
    int st = or_ls_solve(m, k, B, G, V);
    if (st == OR_OK && pre) memcpy(pre, V, sizeof(double) * (size_t)m * (size_t)k);
    if (st == OR_OK) st = or_project(V, m * (int64_t)k);
    if (st == OR_OK) st = or_topt(V, m, k, t_v, mode);
    free(B);
    free(G);
    return st;
}

int or_update_U(int64_t n, int64_t m, const int64_t *rowptr,
                const int32_t *colidx, const double *val, int32_t k,
                const double *V, int64_t t_u, int mode, double *U, double *pre)
{
    double *B = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k + 8);
    double *G = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    if (!B || !G) { free(B); free(G); return OR_ERR_OOM; }
    or_spmm_A(n, m, rowptr, colidx, val, k, V, B);
    or_gram(m, k, V, G);
    int st = or_ls_solve(n, k, B, G, U);
    if (st == OR_OK && pre) memcpy(pre, U, sizeof(double) * (size_t)n * (size_t)k);
    if (st == OR_OK) st = or_project(U, n * (int64_t)k);
    if (st == OR_OK) st = or_topt(U, n, k, t_u, mode);
    free(B);
    free(G);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 measures.
 * R = ||U_new - U_old||_F / ||U_new||_F.  Reading for ||U_new|| = 0:
 * R = 0 if U_old is also 0, else +inf. */
double or_residual(int64_t rows, int32_t k, const double *Unew,
                   const double *Uold)
{
    double num = 0.0, den = 0.0, old = 0.0;
    for (int64_t q = 0; q < rows * (int64_t)k; ++q) {
        double d = Unew[q] - Uold[q];
        num += d * d;
        den += Unew[q] * Unew[q];
        old += Uold[q] * Uold[q];
    }
    if (den == 0.0) return old == 0.0 ? 0.0 : INFINITY;
    return sqrt(num) / sqrt(den);
}

/* ||A||_F^2 */
double or_norm2_A(int64_t nnz, const double *val)
{
    double s = 0.0;
    for (int64_t p = 0; p < nnz; ++p) s += val[p] * val[p];
    return s;
}

/* f = ||A - U V^T||_F^2 without forming U V^T:
 *   ||A||^2 - 2 <U, A V> + <U^T U, V^T V>.
 * The middle term is sum_ij U_ic (A V)_ic; the last is trace(U^TU V^TV). */
double or_loss(int64_t n, int64_t m, const int64_t *rowptr,
               const int32_t *colidx, const double *val, int32_t k,
               const double *U, const double *V)
{
    double *AV = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k + 8);
    double *GU = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    double *GV = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    or_spmm_A(n, m, rowptr, colidx, val, k, V, AV);
    or_gram(n, k, U, GU);
    or_gram(m, k, V, GV);
    double a2 = or_norm2_A(rowptr[n], val);
    double cross = 0.0;
    for (int64_t q = 0; q < n * (int64_t)k; ++q) cross += U[q] * AV[q];
    double tr = 0.0;
    for (int32_t q = 0; q < k * k; ++q) tr += GU[q] * GV[q];
    free(AV);
    free(GU);
    free(GV);
    return a2 - 2.0 * cross + tr;
}

/* E = ||A - U V^T||_F / ||A||_F through the identity above, clamped at 0
 * before the square root.  E = 0 when ||A|| = 0. */
double or_error_identity(int64_t n, int64_t m, const int64_t *rowptr,
                         const int32_t *colidx, const double *val, int32_t k,
                         const double *U, const double *V)
{
    double a2 = or_norm2_A(rowptr[n], val);
    if (a2 == 0.0) return 0.0;
    double f = or_loss(n, m, rowptr, colidx, val, k, U, V);
    return sqrt(f > 0.0 ? f : 0.0) / sqrt(a2);
}

/* E from the dense reconstruction A - U V^T (tiny inputs only). */
double or_error_direct(int64_t n, int64_t m, const int64_t *rowptr,
                       const int32_t *colidx, const double *val, int32_t k,
                       const double *U, const double *V)
{
    double *D = (double *)calloc((size_t)n * (size_t)m + 1, sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            D[i * m + colidx[p]] = val[p];
    double num = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j) {
            double s = 0.0;
            for (int32_t c = 0; c < k; ++c) s += U[i * k + c] * V[j * k + c];
            double d = D[i * m + j] - s;
            num += d * d;
        }
    free(D);
    double a2 = or_norm2_A(rowptr[n], val);
    if (a2 == 0.0) return 0.0;
    return sqrt(num) / sqrt(a2);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 driver: U = U0 (not enforced); every sweep runs steps 1-4, then
 * R (against the U of the previous sweep, U0 for the first) and E with the
 * current U and V.  R_out / E_out may be NULL. */
int or_iterate(int64_t n, int64_t m, const int64_t *rowptr,
               const int32_t *colidx, const double *val, int32_t k,
               const double *U0, int64_t t_u, int64_t t_v, int mode,
               int32_t iters, double *R_out, double *E_out, double *U_out,
               double *V_out)
{
    double *Uprev = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k + 8);
    if (!Uprev) return OR_ERR_OOM;
    memcpy(U_out, U0, sizeof(double) * (size_t)n * (size_t)k);
    memcpy(Uprev, U0, sizeof(double) * (size_t)n * (size_t)k);
    int st = OR_OK;
    for (int32_t it = 0; it < iters && st == OR_OK; ++it) {
        st = or_update_V(n, m, rowptr, colidx, val, k, U_out, t_v, mode, V_out, NULL);
        if (st != OR_OK) break;
        st = or_update_U(n, m, rowptr, colidx, val, k, V_out, t_u, mode, U_out, NULL);
        if (st != OR_OK) break;
        if (R_out) R_out[it] = or_residual(n, k, U_out, Uprev);
        if (E_out) E_out[it] = or_error_identity(n, m, rowptr, colidx, val, k, U_out, V_out);
        memcpy(Uprev, U_out, sizeof(double) * (size_t)n * (size_t)k);
    }
    free(Uprev);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Gradients of f(U, V) = ||A - U V^T||_F^2 (the squared objective, Eq. 6):
 *   grad_U = 2 (U V^T V - A V),   grad_V = 2 (V U^T U - A^T U). */
void or_grad_U(int64_t n, int64_t m, const int64_t *rowptr,
               const int32_t *colidx, const double *val, int32_t k,
               const double *U, const double *V, double *gU)
{
    double *AV = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k + 8);
    double *GV = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    or_spmm_A(n, m, rowptr, colidx, val, k, V, AV);
    or_gram(m, k, V, GV);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t c = 0; c < k; ++c) {
            double s = 0.0;
            for (int32_t d = 0; d < k; ++d) s += U[i * k + d] * GV[d * k + c];
            gU[i * k + c] = 2.0 * (s - AV[i * k + c]);
        }
    free(AV);
    free(GV);
}

void or_grad_V(int64_t n, int64_t m, const int64_t *rowptr,
               const int32_t *colidx, const double *val, int32_t k,
               const double *U, const double *V, double *gV)
{
    double *AtU = (double *)malloc(sizeof(double) * (size_t)m * (size_t)k + 8);
    double *GU = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    or_spmm_At(n, m, rowptr, colidx, val, k, U, AtU);
    or_gram(n, k, U, GU);
    for (int64_t j = 0; j < m; ++j)
        for (int32_t c = 0; c < k; ++c) {
            double s = 0.0;
            for (int32_t d = 0; d < k; ++d) s += V[j * k + d] * GU[d * k + c];
            gV[j * k + c] = 2.0 * (s - AtU[j * k + c]);
        }
    free(AtU);
    free(GU);
}

/* Largest eigenvalue of a k x k symmetric non-negative matrix by 20 steps
 * of power iteration from the normalised all-ones vector. */
double or_lambda_max(int32_t k, const double *G)
{
    double *x = (double *)malloc(sizeof(double) * (size_t)k + 8);
    double *y = (double *)malloc(sizeof(double) * (size_t)k + 8);
    for (int32_t c = 0; c < k; ++c) x[c] = 1.0 / sqrt((double)k);
    double lam = 0.0;
    for (int it = 0; it < 20; ++it) {
        double nrm = 0.0;
        for (int32_t c = 0; c < k; ++c) {
            double s = 0.0;
            for (int32_t d = 0; d < k; ++d) s += G[c * k + d] * x[d];
            y[c] = s;
            nrm += s * s;
        }
        lam = sqrt(nrm);
        if (lam == 0.0) break;
        for (int32_t c = 0; c < k; ++c) x[c] = y[c] / lam;
    }
    free(x);
    free(y);
    return lam;
}

/* Projected-gradient polish on a fixed support (not in the paper; an
 * addition on top of Alg. 2): U <- P_S(U - eta grad_U f) with
 * eta = 1 / (2 lambda_max(V^T V)), where P_S clamps to >= 0 and zeroes
 * every entry outside the current support S = {U != 0}.  which = 0 polishes
 * U (V fixed), which = 1 polishes V (U fixed). */
int or_pg_step(int64_t n, int64_t m, const int64_t *rowptr,
               const int32_t *colidx, const double *val, int32_t k,
               double *U, double *V, int which)
{
    int64_t rows = which == 0 ? n : m;
    double *g = (double *)malloc(sizeof(double) * (size_t)rows * (size_t)k + 8);
    double *G = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k + 8);
    if (!g || !G) { free(g); free(G); return OR_ERR_OOM; }
    double *F = which == 0 ? U : V;
    if (which == 0) {
        or_grad_U(n, m, rowptr, colidx, val, k, U, V, g);
        or_gram(m, k, V, G);
    } else {
        or_grad_V(n, m, rowptr, colidx, val, k, U, V, g);
        or_gram(n, k, U, G);
    }
    double lam = or_lambda_max(k, G);
    if (lam > 0.0) {
        double eta = 1.0 / (2.0 * lam);
        for (int64_t q = 0; q < rows * (int64_t)k; ++q) {
            if (F[q] == 0.0) continue;
            double x = F[q] - eta * g[q];
            F[q] = x > 0.0 ? x : 0.0;
        }
    }
    free(g);
    free(G);
    return OR_OK;
}

/*
 * Sec. 3.2, Eq. 3 and Eq. 4: the document-clustering accuracy of each topic
 * (column c of V, rows = documents).  A document belongs to topic c when
 * V[i][c] != 0; n_D is the number of such documents and n_J the number of
 * classes (journals in the paper; planted topics here), with labels[i] in
 * [0, n_J).  Acc = (P - alpha) / (beta - alpha), P = the number of pairs
 * i < k of the topic's documents with the same label (counted pair by
 * pair), alpha = q (n_J (q - 1) / 2 + r) with q = floor(n_D / n_J),
 * r = n_D mod n_J (the pairs of an even spread), beta = n_D (n_D - 1) / 2.
 * Acc = 1 when n_D <= 1 (as the paper sets it) and, a reading, when
 * beta == alpha (then every spread is as good as any: n_J == 1).  Writes
 * acc[c] for the k topics; returns OR_ERR_INVALID_ARG on a label outside
 * [0, n_J) of a member document.
 */
int or_topic_accuracy(int64_t m, int32_t k, const double *V, const int32_t *labels,
                      int32_t n_J, double *acc)
{
    if (n_J < 1) return OR_ERR_INVALID_ARG;
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    if (!members) return OR_ERR_OOM;
    for (int32_t c = 0; c < k; ++c) {
        int64_t nD = 0;
        for (int64_t i = 0; i < m; ++i) {
            if (V[i * k + c] != 0.0) {
                if (labels[i] < 0 || labels[i] >= n_J) {
                    free(members);
                    return OR_ERR_INVALID_ARG;
                }
                members[nD++] = i;
            }
        }
        if (nD <= 1) {
            acc[c] = 1.0;
            continue;
        }
        double same = 0.0;
        for (int64_t a = 0; a + 1 < nD; ++a)
            for (int64_t b = a + 1; b < nD; ++b)
                if (labels[members[a]] == labels[members[b]]) same += 1.0;
        const double q = (double)(nD / n_J), r = (double)(nD % n_J);
        const double alpha = q * ((double)n_J * (q - 1.0) / 2.0 + r);
        const double beta = (double)nD * (double)(nD - 1) / 2.0;
        acc[c] = beta == alpha ? 1.0 : (same - alpha) / (beta - alpha);
    }
    free(members);
    return OR_OK;
}

/*
 * Sec. 4, Alg. 3 (sequential ALS): the k = eta * k2 topics are found k2 at a
 * time.  Eq. 5 splits U V^T = U1 V1^T + U2 V2^T, with U1, V1 the topics
 * converged so far (the first k1 = b * k2 columns of U, V when block b is
 * found) and U2 (n x k2), V2 (m x k2) the new block.
 *   START (b = 0): U2, V2 from Alg. 2 with k2 topics and U0 as the initial
 *          guess (or_update_V / or_update_U, iters sweeps).
 *   NEXT  (b = 1 .. eta - 1): U2 = U0 (the same initial guess for every
 *          block, a reading), then iters times
 *            V2 = (A^T U2 - V1 (U1^T U2)) (U2^T U2)^-1   (Eq. 7),
 *                 projected, t_v largest kept per column;
 *            U2 = (A V2 - U1 (V1^T V2)) (V2^T V2)^-1     (Eq. 8),
 *                 projected, t_u largest kept per column.
 *   Append: U[:, k1 : k1 + k2] = U2, V[:, k1 : k1 + k2] = V2.
 * The k2 x k2 solves are those of Alg. 2 (or_ls_solve: a zero Gram column
 * gives a zero output column).  For k2 = 1 the solve is the division by
 * u^T u (v^T v) the paper mentions.  U0: n x k2 row-major.  If vpre/upre
 * are non-NULL they receive the last block's last V2 (m x k2) and U2
 * (n x k2) before the projection.  U (n x k), V (m x k) row-major outputs.
 */
int or_sequential(int64_t n, int64_t m, const int64_t *rowptr, const int32_t *colidx,
                  const double *val, int32_t k, int32_t k2, const double *U0, int64_t t_u,
                  int64_t t_v, int32_t iters, double *U, double *V, double *vpre, double *upre)
{
    if (k < 1 || k2 < 1 || k % k2 != 0 || iters < 1 || t_u < 0 || t_v < 0)
        return OR_ERR_INVALID_ARG;
    const int32_t eta = k / k2;
    const size_t nk2 = (size_t)n * (size_t)k2, mk2 = (size_t)m * (size_t)k2;
    double *U2 = (double *)malloc(sizeof(double) * nk2 + 8);
    double *V2 = (double *)malloc(sizeof(double) * mk2 + 8);
    double *Y = (double *)malloc(sizeof(double) * (nk2 > mk2 ? nk2 : mk2) + 8);
    double *G = (double *)malloc(sizeof(double) * (size_t)k2 * (size_t)k2 + 8);
    double *g = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k2 + 8);
    if (!U2 || !V2 || !Y || !G || !g) {
        free(U2); free(V2); free(Y); free(G); free(g);
        return OR_ERR_OOM;
    }
    memset(U, 0, sizeof(double) * (size_t)n * (size_t)k);
    memset(V, 0, sizeof(double) * (size_t)m * (size_t)k);
    int st = OR_OK;
    for (int32_t b = 0; b < eta && st == OR_OK; ++b) {
        const int32_t k1 = b * k2;
        const int last = b == eta - 1;
        memcpy(U2, U0, sizeof(double) * nk2);
        for (int32_t it = 0; it < iters && st == OR_OK; ++it) {
            double *vp = last && it == iters - 1 ? vpre : NULL;
            double *up = last && it == iters - 1 ? upre : NULL;
            if (b == 0) {
                /* START: Alg. 2 steps 1-4 with k2 topics */
                st = or_update_V(n, m, rowptr, colidx, val, k2, U2, t_v, OR_TOPT_COLUMN, V2, vp);
                if (st == OR_OK)
                    st = or_update_U(n, m, rowptr, colidx, val, k2, V2, t_u, OR_TOPT_COLUMN, U2, up);
                continue;
            }
            /* Eq. 7: Y = A^T U2 - V1 (U1^T U2), then V2 = Y (U2^T U2)^-1 */
            or_spmm_At(n, m, rowptr, colidx, val, k2, U2, Y);
            for (int32_t c = 0; c < k1; ++c)
                for (int32_t j = 0; j < k2; ++j) {
                    double s = 0.0;
                    for (int64_t i = 0; i < n; ++i) s += U[i * k + c] * U2[i * k2 + j];
                    g[c * k2 + j] = s;
                }
            for (int64_t i = 0; i < m; ++i)
                for (int32_t j = 0; j < k2; ++j) {
                    double d = 0.0;
                    for (int32_t c = 0; c < k1; ++c) d += V[i * k + c] * g[c * k2 + j];
                    Y[i * k2 + j] -= d;
                }
            or_gram(n, k2, U2, G);
            st = or_ls_solve(m, k2, Y, G, V2);
            if (st == OR_OK && vp) memcpy(vp, V2, sizeof(double) * mk2);
            if (st == OR_OK) st = or_project(V2, (int64_t)mk2);
            if (st == OR_OK) st = or_topt(V2, m, k2, t_v, OR_TOPT_COLUMN);
            if (st != OR_OK) break;
            /* Eq. 8: Y = A V2 - U1 (V1^T V2), then U2 = Y (V2^T V2)^-1 */
            or_spmm_A(n, m, rowptr, colidx, val, k2, V2, Y);
            for (int32_t c = 0; c < k1; ++c)
                for (int32_t j = 0; j < k2; ++j) {
                    double s = 0.0;
                    for (int64_t i = 0; i < m; ++i) s += V[i * k + c] * V2[i * k2 + j];
                    g[c * k2 + j] = s;
                }
            for (int64_t i = 0; i < n; ++i)
                for (int32_t j = 0; j < k2; ++j) {
                    double d = 0.0;
                    for (int32_t c = 0; c < k1; ++c) d += U[i * k + c] * g[c * k2 + j];
                    Y[i * k2 + j] -= d;
                }
            or_gram(m, k2, V2, G);
            st = or_ls_solve(n, k2, Y, G, U2);
            if (st == OR_OK && up) memcpy(up, U2, sizeof(double) * nk2);
            if (st == OR_OK) st = or_project(U2, (int64_t)nk2);
            if (st == OR_OK) st = or_topt(U2, n, k2, t_u, OR_TOPT_COLUMN);
        }
        for (int64_t i = 0; i < n; ++i)
            for (int32_t j = 0; j < k2; ++j) U[i * k + k1 + j] = U2[i * k2 + j];
        for (int64_t i = 0; i < m; ++i)
            for (int32_t j = 0; j < k2; ++j) V[i * k + k1 + j] = V2[i * k2 + j];
    }
    free(U2); free(V2); free(Y); free(G); free(g);
    return st;
}

/* Threads of the OpenMP build (no effect on the single-threaded build). */
void or_set_threads(int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}
