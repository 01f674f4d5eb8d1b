/*
 * Plain FP64 CPU oracle for the inversion of a symmetric positive definite
 * matrix (Agullo et al., "Towards an Efficient Tile Matrix Inversion of
 * Symmetric Positive Definite Matrices on Multicore Architectures").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * What it computes (Sec. 2, Algorithm 1 and the text after it): the three
 * steps of the inversion, each as the plain unblocked definition that the
 * paper's tile algorithm reaches up to rounding order.  The paper states that
 * Algorithm 1 follows the LAPACK 3.2.1 variants, so each step below is the
 * corresponding unblocked LAPACK operation written out as its formula:
 *
 *   Step 1 (Cholesky, A = L L^T, lower):
 *       L_jj = sqrt(A_jj - sum_{k<j} L_jk^2)
 *       L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj          (i > j)
 *   Step 2 (triangular inversion, X = L^{-1}, lower, non-unit), from X L = I:
 *       X_jj = 1 / L_jj
 *       X_ij = -(sum_{k=j+1..i} X_ik L_kj) * X_jj             (i > j)
 *   Step 3 (product A^{-1} = X^T X, lower triangle):
 *       (X^T X)_ij = sum_{k>=i} X_ki X_kj                      (i >= j)
 *
 * Storage: column-major with leading dimension lda >= n; only the lower
 * triangle (i >= j) is read or written, the strictly upper part is left as is.
 *
 * Error behaviour (LAPACK convention):
 *   oracle_potf2 returns j+1 for the first column j whose pivot
 *   A_jj - sum L_jk^2 is not > 0 (this includes NaN), 0 on success; the
 *   columns before j hold the factor, the rest is partially updated.
 *   oracle_trti2 returns j+1 for the first exactly-zero diagonal entry and then
 *   leaves the matrix untouched.
 *
 * Parallelism: OpenMP over the independent entries of one column (Step 1,
 * Step 2) or one row (Step 3).  The algorithm stays unblocked; the
 * summation order of each entry is fixed, so the result does not depend on
 * the thread count.  Build with -ffp-contract=off so no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(M, i, j) (M)[(int64_t)(i) + (int64_t)(j) * lda]

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Step 1: unblocked Cholesky, lower (LAPACK potf2 semantics). */
int oracle_potf2(int64_t n, double* A, int64_t lda) {
    for (int64_t j = 0; j < n; ++j) {
        double d = AT(A, j, j);
        for (int64_t k = 0; k < j; ++k) d -= AT(A, j, k) * AT(A, j, k);
        if (!(d > 0.0)) return (int)(j + 1); /* non-positive or NaN pivot */
        const double ljj = sqrt(d);
        AT(A, j, j) = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double s = AT(A, i, j);
            for (int64_t k = 0; k < j; ++k) s -= AT(A, i, k) * AT(A, j, k);
            AT(A, i, j) = s / ljj;
        }
    }
    return 0;
}

/* Step 2: inverse of a lower non-unit triangular matrix (LAPACK trti2). */
int oracle_trti2(int64_t n, double* A, int64_t lda) {
    for (int64_t j = 0; j < n; ++j)
        if (AT(A, j, j) == 0.0) return (int)(j + 1);
    double* col = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!col) return -1;
    for (int64_t j = n - 1; j >= 0; --j) {
        const double xjj = 1.0 / AT(A, j, j);
        /* columns k > j already hold X; column j below the diagonal holds L */
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int64_t k = j + 1; k <= i; ++k) s += AT(A, i, k) * AT(A, k, j);
            col[i] = -s * xjj;
        }
        for (int64_t i = j + 1; i < n; ++i) AT(A, i, j) = col[i];
        AT(A, j, j) = xjj;
    }
    free(col);
    return 0;
}

/* Step 3: lower triangle of X^T X for lower triangular X (LAPACK lauu2). */
int oracle_lauu2(int64_t n, double* A, int64_t lda) {
    double* row = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!row) return -1;
    for (int64_t i = 0; i < n; ++i) {
        /* row i of the result reads only rows k >= i of X, none written yet */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int64_t k = i; k < n; ++k) s += AT(A, k, i) * AT(A, k, j);
            row[j] = s;
        }
        for (int64_t j = 0; j <= i; ++j) AT(A, i, j) = row[j];
    }
    free(row);
    return 0;
}

/* All three steps in order: A -> lower triangle of A^{-1} (Algorithm 1). */
int oracle_potri(int64_t n, double* A, int64_t lda) {
    int info = oracle_potf2(n, A, lda);
    if (info != 0) return info;
    info = oracle_trti2(n, A, lda);
    if (info != 0) return info;
    return oracle_lauu2(n, A, lda);
}
