/*
 * Plain FP64 CPU oracle for dense LU / Cholesky / triangular substitution.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library. The product
 * path (paper_1511_07174_gb300) never calls it and shares no code with it.
 *
 * Everything is written out from the textbook definitions the paper points to
 * (section 2: A = LU with unit lower L and upper U, A = L L^t for SPD
 * matrices, then L y = b and U x = y by forward / back substitution; the LU
 * "with partial pivoting" of Golub & Van Loan). No blocking, no fusion, no
 * reordering beyond those definitions. Storage is column-major with a leading
 * dimension, 0-based indices inside, LAPACK 1-based pivots outside.
 * Compiled with -ffp-contract=off: every multiply and add rounds separately.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define AT(M, ld, i, j) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

/*
 * LU with partial pivoting, outer-product (right-looking, unblocked) form
 * (paper section 2, "standard LU factorization algorithm with partial
 * pivoting"). Runs the first `ksteps` elimination steps only (ksteps = n is
 * the full factorisation; a smaller value is a bounded sample of the same
 * work).
 *
 * Step j: p = first row i >= j with the largest |a_ij| (ties -> lowest i);
 * ipiv[j] = p + 1; if a_pj != 0 swap rows j and p across all n columns and
 * divide the multipliers a_ij (i > j) by a_jj; otherwise record info = j + 1
 * (first one only) and leave the column as it is; then a_ik -= a_ij * a_jk
 * for all i, k > j.
 */
int oracle_getrf_steps(int n, double *A, int lda, int *ipiv, int *info, int ksteps)
{
    if (n < 0 || lda < (n > 1 ? n : 1) || ksteps < 0) return -1;
    if (ksteps > n) ksteps = n;
    *info = 0;
    for (int j = 0; j < ksteps; ++j) {
        int p = j;
        double best = fabs(AT(A, lda, j, j));
        for (int i = j + 1; i < n; ++i) {
            double v = fabs(AT(A, lda, i, j));
            if (v > best) { best = v; p = i; }
        }
        ipiv[j] = p + 1;
        if (AT(A, lda, p, j) != 0.0) {
            if (p != j) {
                for (int k = 0; k < n; ++k) {
                    double t = AT(A, lda, j, k);
                    AT(A, lda, j, k) = AT(A, lda, p, k);
                    AT(A, lda, p, k) = t;
                }
            }
            double piv = AT(A, lda, j, j);
            for (int i = j + 1; i < n; ++i) AT(A, lda, i, j) = AT(A, lda, i, j) / piv;
        } else if (*info == 0) {
            *info = j + 1;
        }
        for (int k = j + 1; k < n; ++k) {
            double u = AT(A, lda, j, k);
            for (int i = j + 1; i < n; ++i) {
                double prod = AT(A, lda, i, j) * u;
                AT(A, lda, i, k) = AT(A, lda, i, k) - prod;
            }
        }
    }
    return 0;
}

int oracle_getrf(int n, double *A, int lda, int *ipiv, int *info)
{
    return oracle_getrf_steps(n, A, lda, ipiv, info, n);
}

/*
 * Cholesky A = L L^t of an SPD matrix (paper section 2), lower triangle, column
 * by column: d = a_jj - sum_{k<j} l_jk^2; d <= 0 (or NaN) -> info = j + 1 and
 * stop; l_jj = sqrt(d); l_ij = (a_ij - sum_{k<j} l_ik l_jk) / l_jj for i > j.
 * Reads and writes the lower triangle only; the strict upper triangle is not
 * touched.
 */
int oracle_potrf(int n, double *A, int lda, int *info)
{
    if (n < 0 || lda < (n > 1 ? n : 1)) return -1;
    *info = 0;
    for (int j = 0; j < n; ++j) {
        double d = AT(A, lda, j, j);
        for (int k = 0; k < j; ++k) {
            double l = AT(A, lda, j, k);
            d = d - l * l;
        }
        if (!(d > 0.0)) { *info = j + 1; return 0; }
        double ljj = sqrt(d);
        AT(A, lda, j, j) = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = AT(A, lda, i, j);
            for (int k = 0; k < j; ++k) {
                double prod = AT(A, lda, i, k) * AT(A, lda, j, k);
                s = s - prod;
            }
            AT(A, lda, i, j) = s / ljj;
        }
    }
    return 0;
}

/*
 * Solve A X = B from P A = L U (paper section 2, second step): apply the row
 * interchanges ipiv[0..n) to B in order, then L y = Pb by forward substitution
 * with unit diagonal, then U x = y by back substitution.
 */
int oracle_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv,
                 double *B, int ldb)
{
    if (n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return -1;
    for (int c = 0; c < nrhs; ++c) {
        double *b = B + (size_t)c * ldb;
        for (int j = 0; j < n; ++j) {
            int p = ipiv[j] - 1;
            if (p != j) { double t = b[j]; b[j] = b[p]; b[p] = t; }
        }
        for (int j = 0; j < n; ++j) {
            double bj = b[j];
            for (int i = j + 1; i < n; ++i) b[i] = b[i] - AT(LU, lda, i, j) * bj;
        }
        for (int j = n - 1; j >= 0; --j) {
            b[j] = b[j] / AT(LU, lda, j, j);
            double bj = b[j];
            for (int i = 0; i < j; ++i) b[i] = b[i] - AT(LU, lda, i, j) * bj;
        }
    }
    return 0;
}

/*
 * Solve A X = B from A = L L^t: L y = b (forward substitution), then
 * L^t x = y (back substitution with the transpose of L).
 */
int oracle_potrs(int n, int nrhs, const double *L, int lda, double *B, int ldb)
{
    if (n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return -1;
    for (int c = 0; c < nrhs; ++c) {
        double *b = B + (size_t)c * ldb;
        for (int j = 0; j < n; ++j) {
            b[j] = b[j] / AT(L, lda, j, j);
            double bj = b[j];
            for (int i = j + 1; i < n; ++i) b[i] = b[i] - AT(L, lda, i, j) * bj;
        }
        for (int j = n - 1; j >= 0; --j) {
            double s = b[j];
            for (int i = j + 1; i < n; ++i) s = s - AT(L, lda, i, j) * b[i];
            b[j] = s / AT(L, lda, j, j);
        }
    }
    return 0;
}

/*
 * Normwise backward error of each column x of X for A x = b:
 *   beta = ||b - A x||_inf / (||A||_inf * ||x||_inf),
 * with ||A||_inf the largest absolute row sum. r = b - A x is accumulated in
 * plain FP64, one row at a time. beta[c] is written for every column c.
 */
int oracle_backward_error(int n, int nrhs, const double *A, int lda,
                          const double *X, int ldx, const double *B, int ldb,
                          double *beta)
{
    if (n < 0 || nrhs < 0) return -1;
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = s + fabs(AT(A, lda, i, j));
        if (s > anorm) anorm = s;
    }
    for (int c = 0; c < nrhs; ++c) {
        const double *x = X + (size_t)c * ldx;
        const double *b = B + (size_t)c * ldb;
        double rmax = 0.0, xmax = 0.0;
        for (int i = 0; i < n; ++i) {
            double r = b[i];
            for (int j = 0; j < n; ++j) r = r - AT(A, lda, i, j) * x[j];
            if (fabs(r) > rmax) rmax = fabs(r);
        }
        for (int i = 0; i < n; ++i)
            if (fabs(x[i]) > xmax) xmax = fabs(x[i]);
        double den = anorm * xmax;
        beta[c] = den > 0.0 ? rmax / den : (rmax > 0.0 ? INFINITY : 0.0);
    }
    return 0;
}

/*
 * Gradient of x = A^{-1} b for an upstream gradient G = dL/dx:
 *   gB = A^{-t} G,   gA = -gB X^t.
 * A^t is factored on its own (its own pivots) with oracle_getrf and solved
 * with oracle_getrs, so this shares nothing with a transposed solve that
 * reuses the factors of A. gA is n x n (leading dimension n), gB n x nrhs.
 * Returns the info of the factorisation of A^t (0 when nonsingular).
 */
int oracle_solve_grad(int n, int nrhs, const double *A, int lda,
                      const double *X, int ldx, const double *G, int ldg,
                      double *gA, double *gB)
{
    if (n < 0 || nrhs < 0) return -1;
    double *At = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
    int *piv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!At || !piv) { free(At); free(piv); return -2; }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) AT(At, n, i, j) = AT(A, lda, j, i);
    int info = 0;
    oracle_getrf(n, At, n, piv, &info);
    for (int c = 0; c < nrhs; ++c)
        for (int i = 0; i < n; ++i) AT(gB, n, i, c) = AT(G, ldg, i, c);
    oracle_getrs(n, nrhs, At, n, piv, gB, n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int c = 0; c < nrhs; ++c) s = s + AT(gB, n, i, c) * AT(X, ldx, j, c);
            AT(gA, n, i, j) = -s;
        }
    free(At);
    free(piv);
    return info;
}

/*
 * Smallest relative gap, over the first `ksteps` elimination steps, between
 * the largest and the second-largest |candidate| of the pivot search:
 * (|a_p| - |a_second|) / |a_p|. Runs its own unblocked elimination on a copy
 * (same arithmetic as oracle_getrf_steps). Inputs whose gap is tiny can have
 * more than one valid pivot sequence under rounding, so pivot-vector
 * comparisons use only inputs with a clear gap. Returns 1.0 when every
 * column has a single candidate.
 */
double oracle_min_pivot_gap(int n, const double *A, int lda, int ksteps)
{
    if (n <= 0) return 1.0;
    if (ksteps > n) ksteps = n;
    double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!W) return -1.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) AT(W, n, i, j) = AT(A, lda, i, j);
    double gap = 1.0;
    for (int j = 0; j < ksteps; ++j) {
        int p = j;
        double best = fabs(AT(W, n, j, j)), second = -1.0;
        for (int i = j + 1; i < n; ++i) {
            double v = fabs(AT(W, n, i, j));
            if (v > best) { second = best; best = v; p = i; }
            else if (v > second) second = v;
        }
        if (second >= 0.0 && best > 0.0) {
            double g = (best - second) / best;
            if (g < gap) gap = g;
        }
        if (AT(W, n, p, j) != 0.0) {
            if (p != j)
                for (int k = 0; k < n; ++k) {
                    double t = AT(W, n, j, k);
                    AT(W, n, j, k) = AT(W, n, p, k);
                    AT(W, n, p, k) = t;
                }
            double piv = AT(W, n, j, j);
            for (int i = j + 1; i < n; ++i) AT(W, n, i, j) = AT(W, n, i, j) / piv;
        }
        for (int k = j + 1; k < n; ++k) {
            double u = AT(W, n, j, k);
            for (int i = j + 1; i < n; ++i) {
                double prod = AT(W, n, i, j) * u;
                AT(W, n, i, k) = AT(W, n, i, k) - prod;
            }
        }
    }
    free(W);
    return gap;
}
