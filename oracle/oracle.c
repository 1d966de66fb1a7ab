/*
 * Oracle: plain, slow, FP64 CPU reference for the three structured solves.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * The problems (the paper's case studies, Fig. 2 caption, and the annotated
 * input "X^T X = A" of the "Generator structure" paragraph):
 *   (a) X_u^T X_u = A,        A symmetric positive definite, X_u upper triangular;
 *   (b) L X_s + X_s L^T = S,  L lower triangular, S and X_s symmetric;
 *   (c) L X + X U = C,        L lower triangular, U upper triangular.
 * All matrices are n x n, double precision (the paper's "Preliminary
 * performance results" paragraph).  (c) is also given for a rectangular X
 * (L m x m, U n x n), a generalisation the paper does not state, and (a)
 * is used to solve A X = B (oracle_posv_upper).
 *
 * Each routine is the textbook unblocked recurrence obtained by writing the
 * defining equation out entry by entry and solving for one unknown at a time.
 * No blocking, no reordering, no fusion.  Storage is column-major: element
 * (i, j) of a matrix with leading dimension ld sits at p[i + j * ld].
 *
 * Readings taken where the paper is silent:
 *   - the Cholesky factor has a positive diagonal (this makes it unique);
 *   - the Cholesky routine reads only the upper triangle of A and writes only
 *     the upper triangle of X;
 *   - the Lyapunov routine reads only the lower triangle of S and writes only
 *     the lower triangle of X (X is symmetric);
 *   - sums run left to right in plain FP64 (built with -ffp-contract=off);
 *   - the Sylvester and Lyapunov right-hand sides carry no minus sign: the
 *     equations are taken literally as printed.
 *
 * Return codes (the same convention as the library's per-instance info):
 *   0      success;
 *   j + 1  (Cholesky) the pivot of column j (0-based) was not positive or was NaN;
 *   1      (Sylvester / Lyapunov) some divisor l_ii + u_jj had magnitude at or below
 *          delta = n * DBL_EPSILON * max_i,j(|l_ii|, |u_jj|), or was NaN.
 */
#include <math.h>
#include <float.h>
#include <stddef.h>

#define AT(p, ld, i, j) ((p)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

/*
 * Upper Cholesky, problem (a).  Entry (i, j), i <= j, of X^T X is
 *   sum_{k <= i} x_ki x_kj,
 * so for i < j:  x_ij = (a_ij - sum_{k < i} x_ki x_kj) / x_ii
 * and           x_jj = sqrt(a_jj - sum_{k < j} x_kj^2).
 * Columns are produced left to right; inside a column, rows top to bottom.
 */
int oracle_potrf_upper(int n, const double *A, int lda, double *X, int ldx)
{
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < j; ++i) {
            double s = AT(A, lda, i, j);
            for (int k = 0; k < i; ++k)
                s = s - AT(X, ldx, k, i) * AT(X, ldx, k, j);
            AT(X, ldx, i, j) = s / AT(X, ldx, i, i);
        }
        double d = AT(A, lda, j, j);
        for (int k = 0; k < j; ++k)
            d = d - AT(X, ldx, k, j) * AT(X, ldx, k, j);
        if (!(d > 0.0))
            return j + 1;
        AT(X, ldx, j, j) = sqrt(d);
    }
    return 0;
}

/*
 * SPD solve A X = B (A n x n symmetric positive definite, B and X n x k)
 * through the Cholesky factor: R = the upper factor of A (R^T R = A, the
 * routine above, written to R), then the two triangular systems
 *   R^T Y = B:  y_ij = (b_ij - sum_{l < i} r_li y_lj) / r_ii,   i ascending,
 *   R X = Y:    x_ij = (y_ij - sum_{l > i} r_il x_lj) / r_ii,   i descending,
 * column by column; Y is held in X.  The paper names the factorisation as a
 * building block for solving linear systems; this is that use of it.  Returns
 * the Cholesky info; X is not written when it is nonzero.
 */
int oracle_posv_upper(int n, int k, const double *A, int lda, double *R, int ldr,
                      const double *B, int ldb, double *X, int ldx)
{
    const int info = oracle_potrf_upper(n, A, lda, R, ldr);
    if (info != 0)
        return info;
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = AT(B, ldb, i, j);
            for (int l = 0; l < i; ++l)
                s = s - AT(R, ldr, l, i) * AT(X, ldx, l, j);
            AT(X, ldx, i, j) = s / AT(R, ldr, i, i);
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = AT(X, ldx, i, j);
            for (int l = i + 1; l < n; ++l)
                s = s - AT(R, ldr, i, l) * AT(X, ldx, l, j);
            AT(X, ldx, i, j) = s / AT(R, ldr, i, i);
        }
    }
    return 0;
}

static double divisor_threshold(int n, double maxdiag)
{
    return (double)n * DBL_EPSILON * maxdiag;
}

/*
 * Triangular Sylvester, problem (c).  Entry (i, j) of L X + X U is
 *   sum_{k <= i} l_ik x_kj + sum_{k <= j} x_ik u_kj,
 * so  x_ij = (c_ij - sum_{k < i} l_ik x_kj - sum_{k < j} x_ik u_kj) / (l_ii + u_jj).
 * Rows top to bottom, columns left to right: every x on the right is known.
 */
int oracle_trsyl_lu(int n, const double *L, int ldl, const double *U, int ldu,
                    const double *C, int ldc, double *X, int ldx)
{
    double maxdiag = 0.0;
    for (int i = 0; i < n; ++i) {
        if (fabs(AT(L, ldl, i, i)) > maxdiag) maxdiag = fabs(AT(L, ldl, i, i));
        if (fabs(AT(U, ldu, i, i)) > maxdiag) maxdiag = fabs(AT(U, ldu, i, i));
    }
    const double delta = divisor_threshold(n, maxdiag);
    int info = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double s = AT(C, ldc, i, j);
            for (int k = 0; k < i; ++k)
                s = s - AT(L, ldl, i, k) * AT(X, ldx, k, j);
            for (int k = 0; k < j; ++k)
                s = s - AT(X, ldx, i, k) * AT(U, ldu, k, j);
            double d = AT(L, ldl, i, i) + AT(U, ldu, j, j);
            if (!(fabs(d) > delta))
                info = 1;
            AT(X, ldx, i, j) = s / d;
        }
    }
    return info;
}

/*
 * Rectangular triangular Sylvester: L X + X U = C with L (m x m) lower
 * triangular, U (n x n) upper triangular, C and X m x n.  The paper states
 * the Sylvester problem for n x n matrices (Fig. 2 caption); nothing in the
 * equation needs m = n, and the recurrence is the square one with rows
 * i = 0..m-1 and columns j = 0..n-1, both ascending:
 *   x_ij = (c_ij - sum_{k < i} l_ik x_kj - sum_{k < j} x_ik u_kj) / (l_ii + u_jj).
 * info = 1 if some |l_ii + u_jj| <= max(m, n) * DBL_EPSILON * max(max_i |l_ii|,
 * max_j |u_jj|) or is NaN (the square threshold with max(m, n) for n).
 */
int oracle_trsyl_rect(int m, int n, const double *L, int ldl, const double *U, int ldu,
                      const double *C, int ldc, double *X, int ldx)
{
    double maxdiag = 0.0;
    for (int i = 0; i < m; ++i)
        if (fabs(AT(L, ldl, i, i)) > maxdiag) maxdiag = fabs(AT(L, ldl, i, i));
    for (int j = 0; j < n; ++j)
        if (fabs(AT(U, ldu, j, j)) > maxdiag) maxdiag = fabs(AT(U, ldu, j, j));
    const double delta = divisor_threshold(m > n ? m : n, maxdiag);
    int info = 0;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
            double s = AT(C, ldc, i, j);
            for (int k = 0; k < i; ++k)
                s = s - AT(L, ldl, i, k) * AT(X, ldx, k, j);
            for (int k = 0; k < j; ++k)
                s = s - AT(X, ldx, i, k) * AT(U, ldu, k, j);
            double d = AT(L, ldl, i, i) + AT(U, ldu, j, j);
            if (!(fabs(d) > delta))
                info = 1;
            AT(X, ldx, i, j) = s / d;
        }
    }
    return info;
}

/* Read element (r, c) of the symmetric X from its stored lower triangle. */
static double sym_lower(const double *X, int ldx, int r, int c)
{
    return r >= c ? AT(X, ldx, r, c) : AT(X, ldx, c, r);
}

/*
 * Triangular Lyapunov, problem (b): the Sylvester equation with U = L^T, so
 * u_kj = l_jk.  Only i >= j is computed; an unknown x_kj with k < j is the
 * stored x_jk (symmetry of X):
 *   x_ij = (s_ij - sum_{k < i} l_ik x_kj - sum_{k < j} x_ik l_jk) / (l_ii + l_jj).
 */
int oracle_trlyap_l(int n, const double *L, int ldl, const double *S, int lds,
                    double *X, int ldx)
{
    double maxdiag = 0.0;
    for (int i = 0; i < n; ++i)
        if (fabs(AT(L, ldl, i, i)) > maxdiag) maxdiag = fabs(AT(L, ldl, i, i));
    const double delta = divisor_threshold(n, maxdiag);
    int info = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = AT(S, lds, i, j);
            for (int k = 0; k < i; ++k)
                s = s - AT(L, ldl, i, k) * sym_lower(X, ldx, k, j);
            for (int k = 0; k < j; ++k)
                s = s - sym_lower(X, ldx, i, k) * AT(L, ldl, j, k);
            double d = AT(L, ldl, i, i) + AT(L, ldl, j, j);
            if (!(fabs(d) > delta))
                info = 1;
            AT(X, ldx, i, j) = s / d;
        }
    }
    return info;
}

/*
 * Batched drivers over a packed buffer: instance b has order n[b] and starts
 * at element offset off[b] of every operand buffer; its leading dimension is
 * n[b].  info[b] receives the routine's return code.  Loops over instances in
 * order; thread-level parallelism, when wanted, is the caller's (the routines
 * keep no state).
 */
void oracle_potrf_upper_batch(int batch, const int *n, const long long *off,
                              const double *A, double *X, int *info)
{
    for (int b = 0; b < batch; ++b)
        info[b] = oracle_potrf_upper(n[b], A + off[b], n[b], X + off[b], n[b]);
}

void oracle_trsyl_lu_batch(int batch, const int *n, const long long *off,
                           const double *L, const double *U, const double *C,
                           double *X, int *info)
{
    for (int b = 0; b < batch; ++b)
        info[b] = oracle_trsyl_lu(n[b], L + off[b], n[b], U + off[b], n[b],
                                  C + off[b], n[b], X + off[b], n[b]);
}

void oracle_trlyap_l_batch(int batch, const int *n, const long long *off,
                           const double *L, const double *S, double *X, int *info)
{
    for (int b = 0; b < batch; ++b)
        info[b] = oracle_trlyap_l(n[b], L + off[b], n[b], S + off[b], n[b],
                                  X + off[b], n[b]);
}

/* Rectangular Sylvester batch: instance b has L at offL[b] (ld m[b]), U at
   offU[b] (ld n[b]), C and X at offC[b] (ld m[b]). */
void oracle_trsyl_rect_batch(int batch, const int *m, const int *n, const long long *offL,
                             const long long *offU, const long long *offC, const double *L,
                             const double *U, const double *C, double *X, int *info)
{
    for (int b = 0; b < batch; ++b) {
        const int mm = m[b] > 0 ? m[b] : 1, nn = n[b] > 0 ? n[b] : 1;
        info[b] = oracle_trsyl_rect(m[b], n[b], L + offL[b], mm, U + offU[b], nn,
                                    C + offC[b], mm, X + offC[b], mm);
    }
}

/* SPD solve batch: instance b has A and R at offA[b] (n x n, ld n), B and X at
   offB[b] (n x k, ld n). */
void oracle_posv_upper_batch(int batch, const int *n, const int *k, const long long *offA,
                             const long long *offB, const double *A, double *R,
                             const double *B, double *X, int *info)
{
    for (int b = 0; b < batch; ++b) {
        const int ld = n[b] > 0 ? n[b] : 1;
        info[b] = oracle_posv_upper(n[b], k[b], A + offA[b], ld, R + offA[b], ld,
                                    B + offB[b], ld, X + offB[b], ld);
    }
}
