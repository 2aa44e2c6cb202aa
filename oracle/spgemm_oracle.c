/*
 * Plain CPU oracle for the column-wise sparse product C = A x B (CSC).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * loads this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against an obviously
 * correct, slow implementation written from the paper (arXiv 2303.02471).
 *
 * Storage (Section 2.1): a CSC matrix is values[nnz], row_indices[nnz] and
 * column_pointers[ncols + 1] with column_pointers[0] = 0 and
 * column_pointers[ncols] = nnz.  Row order inside a column does not matter
 * on input.  Row indices are int32, column pointers int64, values double
 * (single-precision inputs are widened by the caller).
 *
 * Functions and the passages they follow:
 *   oracle_op_counts       Op_j = sum over stored B_kj of Z^A_k (Section 3.1).
 *   oracle_spgemm_count    nnz of each C column: the SPA counter of Algorithm 1.
 *   oracle_spgemm_fill     C values with the dense accumulator of Algorithm 1,
 *                          each column emitted in ascending row order, plus
 *                          the per-entry sum of |A_ik * B_kj| (error scale).
 *   oracle_spgemm_backward gradients of the stored values: for the product
 *                          C = A B, dA = (dC B^T) sampled on pattern(A) and
 *                          dB = (A^T dC) sampled on pattern(B).  The paper has
 *                          no backward; these are the textbook derivatives of
 *                          C_ij = sum_k A_ik B_kj.
 *
 * Pinned by the CPU tests against the worked example of Fig. 1, dense brute
 * force, the boolean product, A x I = A, the closed form of the squared
 * 5-point Laplacian, (A B) x = A (B x), and (backward) dense brute force,
 * adjoint identities and finite differences.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  With
 * -ffp-contract=off every product is rounded before it is added, in B storage
 * order then A storage order, so the result does not depend on the thread
 * count (threads split whole columns).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Section 3.1: the operation count of column j of B. */
int64_t oracle_op_counts(int64_t nB, const int64_t *Bcp, const int32_t *Brow,
                         const int64_t *Acp, int64_t *op)
{
    int64_t total = 0;
    for (int64_t j = 0; j < nB; ++j) {
        int64_t s = 0;
        for (int64_t p = Bcp[j]; p < Bcp[j + 1]; ++p) {
            int32_t k = Brow[p];
            s += Acp[k + 1] - Acp[k];
        }
        op[j] = s;
        total += s;
    }
    return total;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Algorithm 1 without values: SPA_flags and the counter give nnz(C[:, j]). */
int oracle_spgemm_count(int64_t mA, int64_t nB,
                        const int64_t *Acp, const int32_t *Arow,
                        const int64_t *Bcp, const int32_t *Brow,
                        int64_t *cnt, int nthreads)
{
    int err = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        unsigned char *flag = (unsigned char *)calloc((size_t)(mA > 0 ? mA : 1), 1);
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mA > 0 ? mA : 1));
        if (!flag || !list) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < nB; ++j) {
            if (!flag || !list) continue;
            int64_t counter = 0;
            for (int64_t p = Bcp[j]; p < Bcp[j + 1]; ++p) {
                int32_t k = Brow[p];
                for (int64_t q = Acp[k]; q < Acp[k + 1]; ++q) {
                    int32_t i = Arow[q];
                    if (!flag[i]) {
                        flag[i] = 1;
                        list[counter++] = i;
                    }
                }
            }
            for (int64_t c = 0; c < counter; ++c) flag[list[c]] = 0;
            cnt[j] = counter;
        }
        free(flag);
        free(list);
    }
    return err;
}

/*
 * Algorithm 1 with values.  SPA_values[i] accumulates A_ik * B_kj for every
 * stored B_kj of column j (B storage order) and stored A_ik of column k (A
 * storage order); SPA_flags marks the first touch of row i, which appends i
 * to SPA_indices.  The touched rows are then sorted ascending (the paper
 * emits them in first-touch order; the sorted order is this library's
 * canonical form) and written at Ccp[j].  Cabs receives sum |A_ik * B_kj|
 * for every emitted entry.  Returns 1 if a column's count disagrees with Ccp.
 */
int oracle_spgemm_fill(int64_t mA, int64_t nB,
                       const int64_t *Acp, const int32_t *Arow, const double *Aval,
                       const int64_t *Bcp, const int32_t *Brow, const double *Bval,
                       const int64_t *Ccp, int32_t *Crow, double *Cval, double *Cabs,
                       int nthreads)
{
    int err = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
        size_t m = (size_t)(mA > 0 ? mA : 1);
        double *spa_values = (double *)calloc(m, sizeof(double));
        double *spa_abs = (double *)calloc(m, sizeof(double));
        unsigned char *spa_flags = (unsigned char *)calloc(m, 1);
        int32_t *spa_indices = (int32_t *)malloc(sizeof(int32_t) * m);
        int ok = spa_values && spa_abs && spa_flags && spa_indices;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < nB; ++j) {
            if (!ok) continue;
            int64_t counter = 0;
            for (int64_t p = Bcp[j]; p < Bcp[j + 1]; ++p) {
                int32_t k = Brow[p];
                double b = Bval[p];
                for (int64_t q = Acp[k]; q < Acp[k + 1]; ++q) {
                    int32_t i = Arow[q];
                    double tmp_val = Aval[q] * b;
                    spa_values[i] += tmp_val;
                    spa_abs[i] += fabs(tmp_val);
                    if (spa_flags[i] == 0) {
                        spa_flags[i] = 1;
                        spa_indices[counter] = i;
                        counter++;
                    }
                }
            }
            qsort(spa_indices, (size_t)counter, sizeof(int32_t), cmp_i32);
            if (Ccp[j] + counter != Ccp[j + 1]) {
#pragma omp atomic write
                err = 1;
            } else {
                for (int64_t c = 0; c < counter; ++c) {
                    int32_t i = spa_indices[c];
                    Crow[Ccp[j] + c] = i;
                    Cval[Ccp[j] + c] = spa_values[i];
                    Cabs[Ccp[j] + c] = spa_abs[i];
                }
            }
            for (int64_t c = 0; c < counter; ++c) {
                int32_t i = spa_indices[c];
                spa_values[i] = 0.0;
                spa_abs[i] = 0.0;
                spa_flags[i] = 0;
            }
        }
        free(spa_values);
        free(spa_abs);
        free(spa_flags);
        free(spa_indices);
    }
    return err;
}

/*
 * Gradients of the stored values for C = A B given dC on pattern(C):
 *   dB_kj = sum_i A_ik dC_ij           for each stored (k, j) of B,
 *   dA_ik = sum_{j : B_kj stored} dC_ij B_kj   for each stored (i, k) of A.
 * Column j of dC is scattered into a dense vector; every stored A_ik B_kj has
 * (i, j) in pattern(C), so each lookup lands on a stored dC entry.
 * Returns 1 if a looked-up row is missing from column j of C.
 */
int oracle_spgemm_backward(int64_t mA, int64_t nA, int64_t nB,
                           const int64_t *Acp, const int32_t *Arow, const double *Aval,
                           const int64_t *Bcp, const int32_t *Brow, const double *Bval,
                           const int64_t *Ccp, const int32_t *Crow, const double *dCval,
                           double *dAval, double *dBval)
{
    size_t m = (size_t)(mA > 0 ? mA : 1);
    double *d = (double *)calloc(m, sizeof(double));
    unsigned char *present = (unsigned char *)calloc(m, 1);
    int err = 0;
    if (!d || !present) {
        free(d);
        free(present);
        return 2;
    }
    if (dAval) memset(dAval, 0, sizeof(double) * (size_t)(Acp[nA] > 0 ? Acp[nA] : 0));
    for (int64_t j = 0; j < nB; ++j) {
        for (int64_t c = Ccp[j]; c < Ccp[j + 1]; ++c) {
            d[Crow[c]] = dCval[c];
            present[Crow[c]] = 1;
        }
        for (int64_t p = Bcp[j]; p < Bcp[j + 1]; ++p) {
            int32_t k = Brow[p];
            double s = 0.0;
            for (int64_t q = Acp[k]; q < Acp[k + 1]; ++q) {
                int32_t i = Arow[q];
                if (!present[i]) err = 1;
                s += Aval[q] * d[i];
                if (dAval) dAval[q] += d[i] * Bval[p];
            }
            if (dBval) dBval[p] = s;
        }
        for (int64_t c = Ccp[j]; c < Ccp[j + 1]; ++c) {
            d[Crow[c]] = 0.0;
            present[Crow[c]] = 0;
        }
    }
    free(d);
    free(present);
    return err;
}

/* Number of OpenMP threads the oracle would use for a request (for reports). */
int oracle_threads(int requested)
{
#ifdef _OPENMP
    int n = 0;
#pragma omp parallel num_threads(requested > 0 ? requested : 1)
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    (void)requested;
    return 1;
#endif
}
