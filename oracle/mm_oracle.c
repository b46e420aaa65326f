/*
 * mm_oracle.c -- CPU reference for the dense product C = A*B (TEST INFRASTRUCTURE).
 *
 * This file is the oracle that the GPU library is checked against. Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the library itself never calls it and shares no code with it.
 *
 * What it computes follows the paper's definition of the matrix product
 * (Sec. III, the defining equation for C[i][j] and the row-by-column dot
 * product spelled out below it): every C[i][j] is the dot product of row i
 * of A with column j of B. Storage is row-major, as the paper's C program uses
 * (Sec. III, paragraph on row-major order), with leading dimensions.
 *
 * Reading of the paper: it does not print its loop order; the product is
 * taken as the i-j-k triple loop with k ascending (Sec. V describes the timed
 * program as the unoptimised textbook product). Every product and every
 * sum is an IEEE-754 double operation rounded to nearest-even; the build
 * passes -ffp-contract=off so no fused multiply-add is formed.
 *
 * The threaded variant is the paper's OpenMP scheme (Sec. III-A-1, one
 * parallel-for pragma above the loop nest), parallel over rows of C. It
 * computes the same values in the same order per element.
 */
#include <stdint.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* C[i][j] = sum_{k ascending} A[i][k]*B[k][j] for rows i in [r0, r1).
 * Cr points at the output row of i = r0 (row i goes to Cr + (i-r0)*ldc). */
static void gemm_rows(int64_t r0, int64_t r1, int64_t n, int64_t k,
                      const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *Cr, int64_t ldc)
{
    for (int64_t i = r0; i < r1; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double prod = A[i * lda + p] * B[p * ldb + j];
                acc = acc + prod;
            }
            Cr[(i - r0) * ldc + j] = acc;
        }
    }
}

/* Serial triple loop over all of C (Sec. V, the serial experiment). */
void oracle_gemm(int64_t m, int64_t n, int64_t k,
                 const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc)
{
    gemm_rows(0, m, n, k, A, lda, B, ldb, C, ldc);
}

/* Rows [r0, r1) only (Cr receives row r0 first): used to check sampled rows
 * of very large products. */
void oracle_gemm_rows(int64_t r0, int64_t r1, int64_t n, int64_t k,
                      const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc)
{
    gemm_rows(r0, r1, n, k, A, lda, B, ldb, C, ldc);
}

/* One element C[i][j] (Sec. III: the dot product of row i and column j). */
double oracle_dot(int64_t i, int64_t j, int64_t k,
                  const double *A, int64_t lda, const double *B, int64_t ldb)
{
    double acc = 0.0;
    for (int64_t p = 0; p < k; ++p) {
        double prod = A[i * lda + p] * B[p * ldb + j];
        acc = acc + prod;
    }
    return acc;
}

/* OpenMP parallel-for over rows [r0, r1) of C (Sec. III-A-1, Threads); C
 * receives row r0 first. Returns the number of threads that ran. */
int oracle_gemm_omp(int64_t r0, int64_t r1, int64_t n, int64_t k,
                    const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(static)
        for (int64_t i = r0; i < r1; ++i)
            gemm_rows(i, i + 1, n, k, A, lda, B, ldb, C + (i - r0) * ldc, ldc);
    }
#else
    (void)nthreads;
    gemm_rows(r0, r1, n, k, A, lda, B, ldb, C, ldc);
#endif
    return used;
}

/* |A|*|B| (elementwise absolute values), the scale of the componentwise
 * error bound |C - C_ref| <= gamma * (|A||B|). Same loop as the product. */
void oracle_absprod(int64_t m, int64_t n, int64_t k,
                    const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *D, int64_t ldd)
{
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double prod = fabs(A[i * lda + p]) * fabs(B[p * ldb + j]);
                acc = acc + prod;
            }
            D[i * ldd + j] = acc;
        }
    }
}

/* |A|*|B| for rows [r0, r1); D receives row r0 first. */
void oracle_absprod_rows(int64_t r0, int64_t r1, int64_t n, int64_t k,
                         const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *D, int64_t ldd)
{
    D -= r0 * ldd;
    for (int64_t i = r0; i < r1; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double prod = fabs(A[i * lda + p]) * fabs(B[p * ldb + j]);
                acc = acc + prod;
            }
            D[i * ldd + j] = acc;
        }
    }
}

/* |A|*|B| for rows [r0, r1) with the same OpenMP parallel-for over rows as
 * oracle_gemm_omp; every element is the serial loop's. Returns the threads. */
int oracle_absprod_omp(int64_t r0, int64_t r1, int64_t n, int64_t k,
                       const double *A, int64_t lda, const double *B, int64_t ldb,
                       double *D, int64_t ldd, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(static)
        for (int64_t i = r0; i < r1; ++i)
            oracle_absprod_rows(i, i + 1, n, k, A, lda, B, ldb, D + (i - r0) * ldd, ldd);
    }
#else
    (void)nthreads;
    oracle_absprod_rows(r0, r1, n, k, A, lda, B, ldb, D, ldd);
#endif
    return used;
}
