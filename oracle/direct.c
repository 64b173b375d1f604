/*
 * O1 row sums in plain C: (W x)_j = sum_{i != j} exp(-||v_j - v_i||^2 / sigma^2) x_i
 * for selected rows j, each over all n sources (Sec. 2, eq. (W_gaussian)).
 *
 * Test infrastructure (the oracle): only tests/, the smoke check and the
 * CPU-baseline leg of bench.py may load this library.  Plain loops in FP64,
 * no reordering of the definition; rows are split across OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* v: n x d row-major; x: n x nrhs column-major with leading dimension ldx;
 * rows: nrows indices; out: nrows x nrhs column-major (leading dim nrows). */
int oracle_gauss_rows(const double *v, int64_t n, int d, double sigma,
                      const double *x, int64_t nrhs, int64_t ldx,
                      const int64_t *rows, int64_t nrows, double *out,
                      int nthreads) {
    if (n < 0 || d < 1 || sigma <= 0.0 || nrhs < 1 || ldx < n) return 1;
    for (int64_t k = 0; k < nrows; ++k)
        if (rows[k] < 0 || rows[k] >= n) return 1;
    const double inv_s2 = 1.0 / (sigma * sigma);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t j = rows[k];
        for (int64_t r = 0; r < nrhs; ++r) out[k + r * nrows] = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (i == j) continue;
            double dist2 = 0.0;
            for (int a = 0; a < d; ++a) {
                const double diff = v[j * d + a] - v[i * d + a];
                dist2 += diff * diff;
            }
            const double w = exp(-dist2 * inv_s2);
            for (int64_t r = 0; r < nrhs; ++r) out[k + r * nrows] += w * x[i + r * ldx];
        }
    }
    return 0;
}
