/*
 * cpu_variants.c -- the paper's two CPU optimisations of the triple loop, as
 * extra CPU-baseline rows (TEST INFRASTRUCTURE, like the rest of oracle/).
 *
 * Sec. III discusses column prefetching (copying a column of B into a
 * contiguous array before the dot products that use it) and cache tiling
 * (working on blocks of the matrices so the data stay in cache). Both are
 * written here with the OpenMP parallel-for over rows of Sec. III-A. Each
 * element of C is still summed over k in ascending order, with every product
 * and every addition an IEEE double operation rounded to nearest (built with
 * -ffp-contract=off), so both return exactly the oracle's values; the tests
 * check that bit for bit. Only the benchmark's CPU leg times them.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Column prefetching: for each column j, copy B[:, j] into a contiguous
 * buffer, then form C[i][j] for this thread's rows. Rows [r0, r1); C receives
 * row r0 first. Returns the number of threads that ran (0 on allocation
 * failure). */
int cpu_gemm_colprefetch(int64_t r0, int64_t r1, int64_t n, int64_t k,
                         const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *C, int64_t ldc, int nthreads)
{
    int used = 1, failed = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *col = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        int64_t lo = r0, hi = r1;
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
        {
            /* this thread's rows: the static partition of [r0, r1) */
            int64_t t = omp_get_thread_num(), T = omp_get_num_threads(), rows = r1 - r0;
            lo = r0 + rows * t / T;
            hi = r0 + rows * (t + 1) / T;
        }
#endif
        if (!col) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        } else {
            for (int64_t j = 0; j < n; ++j) {
                for (int64_t p = 0; p < k; ++p) col[p] = B[p * ldb + j];
                for (int64_t i = lo; i < hi; ++i) {
                    const double *a = A + i * lda;
                    double acc = 0.0;
                    for (int64_t p = 0; p < k; ++p) {
                        double prod = a[p] * col[p];
                        acc = acc + prod;
                    }
                    C[(i - r0) * ldc + j] = acc;
                }
            }
            free(col);
        }
    }
    return failed ? 0 : used;
}

/* Cache tiling: blocks of TI rows x TJ columns x TK of the inner dimension;
 * inside a block the loops run i, p, j so the row of B and the row of C are
 * contiguous, and each C[i][j] still takes its products in ascending p. Rows
 * [r0, r1); C receives row r0 first. Returns the number of threads that ran. */
int cpu_gemm_tiled(int64_t r0, int64_t r1, int64_t n, int64_t k,
                   const double *A, int64_t lda, const double *B, int64_t ldb,
                   double *C, int64_t ldc, int nthreads)
{
    enum { TI = 32, TJ = 256, TK = 128 };
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(static)
#endif
        for (int64_t ib = r0; ib < r1; ib += TI) {
            const int64_t ie = ib + TI < r1 ? ib + TI : r1;
            for (int64_t jb = 0; jb < n; jb += TJ) {
                const int64_t je = jb + TJ < n ? jb + TJ : n;
                for (int64_t i = ib; i < ie; ++i)
                    for (int64_t j = jb; j < je; ++j) C[(i - r0) * ldc + j] = 0.0;
                for (int64_t pb = 0; pb < k; pb += TK) {
                    const int64_t pe = pb + TK < k ? pb + TK : k;
                    for (int64_t i = ib; i < ie; ++i) {
                        double *c = C + (i - r0) * ldc;
                        for (int64_t p = pb; p < pe; ++p) {
                            const double a = A[i * lda + p];
                            const double *b = B + p * ldb;
                            for (int64_t j = jb; j < je; ++j) {
                                double prod = a * b[j];
                                c[j] = c[j] + prod;
                            }
                        }
                    }
                }
            }
        }
#ifdef _OPENMP
    }
#else
    (void)nthreads;
#endif
    return used;
}
