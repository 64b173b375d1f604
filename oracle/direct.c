/*
 * O1 row sums in plain C: (W x)_j = sum_{i != j} K(v_j - v_i) x_i for selected
 * rows j, each over all n sources, with the kernels of Sec. 2: kind 0 the
 * Gaussian exp(-r^2/sigma^2) (eq. (W_gaussian)), 1 the Laplacian RBF
 * exp(-r/sigma), 2 the multiquadric (r^2 + c^2)^{1/2}, 3 the inverse
 * multiquadric (r^2 + c^2)^{-1/2}, 4 the sigma-derivative of the Gaussian
 * (2 r^2 / sigma^3) exp(-r^2/sigma^2); r = ||v_j - v_i||, c passed as sigma.
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
static double kernel_of(int kind, double dist2, double sigma) {
    switch (kind) {
        case 0: return exp(-dist2 / (sigma * sigma));
        case 1: return exp(-sqrt(dist2) / sigma);
        case 2: return sqrt(dist2 + sigma * sigma);
        case 3: return 1.0 / sqrt(dist2 + sigma * sigma);
        default: return 2.0 * dist2 / (sigma * sigma * sigma) * exp(-dist2 / (sigma * sigma));
    }
}

int oracle_kernel_rows(const double *v, int64_t n, int d, int kind, double sigma,
                       const double *x, int64_t nrhs, int64_t ldx,
                       const int64_t *rows, int64_t nrows, double *out,
                       int nthreads) {
    if (n < 0 || d < 1 || kind < 0 || kind > 4 || sigma <= 0.0 || nrhs < 1 || ldx < n) return 1;
    for (int64_t k = 0; k < nrows; ++k)
        if (rows[k] < 0 || rows[k] >= n) return 1;
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
            const double w = kernel_of(kind, dist2, sigma);
            for (int64_t r = 0; r < nrhs; ++r) out[k + r * nrows] += w * x[i + r * ldx];
        }
    }
    return 0;
}
