// Krylov solvers on top of the fast products, all vector work in FP64 on
// the device.
//
// Lanczos (Sec. 4): q_1 = r / ||r||, and for j = 1, 2, ...
//   w = A q_j,  alpha_j = q_j^T w,  w -= alpha_j q_j + beta_j q_{j-1},
//   full reorthogonalization w -= Q_j (Q_j^T w), done twice (classical
//   Gram-Schmidt twice, DGKS), beta_{j+1} = ||w||, q_{j+1} = w / beta_{j+1},
// so that A Q_k = Q_k T_k + beta_{k+1} q_{k+1} e_k^T (eq. (krylov1)).
// Ritz pairs (theta, Q_k s) of T_k have residual |beta_{k+1} s_k| (Sec. 4);
// the k largest theta of A give the k smallest eigenvalues 1 - theta of L_s.
// T_k is diagonalised on the device by implicit QL with Wilkinson shifts.
//
// CG (Sec. 6.2.2, eq. (ssl::system)): conjugate gradients on the SPD
// operator u -> beta L_s u + diag(s) u, stopping at ||r|| <= tol ||f||.
//
// Refined CG: mixed-precision iterative refinement around it.  Sec. 4 notes
// that Krylov methods tolerate inexact products (the relaxation results of
// Simoncini and Szyld); here the inexact products are the mixed form's
// (FP32 arithmetic, error ~3e-7 relative) and the outer loop restores FP64
// accuracy: r_k = f - (beta L_s + S) u_k with the FP64 plan's products,
// (beta L_s~ + S) c_k = r_k by CG with the mixed plan's products to a
// relative residual inner_tol, u_{k+1} = u_k + c_k.  Each outer step shrinks
// the FP64 residual by about max(inner_tol, kappa * eps_mixed), so a few
// steps, each one FP64 product, reach FP64 accuracy while nearly all
// products run in the mixed form.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.h"

namespace nfl {

static constexpr int kRedBlocks = 512;

// ---------------------------------------------------------- vector kernels
__global__ void dot_partials(const double *a, const double *b, int64_t n, double *part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i] * b[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// c[t] = sum_i Q[i + t n] w[i] for t < ncol: grid (kRedBlocks, ncol) of partials.
__global__ void multidot_partials(const double *Q, int64_t n, const double *w, double *part) {
    __shared__ double red[256];
    const int t = blockIdx.y;
    const double *q = Q + (int64_t)t * n;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += q[i] * w[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)t * gridDim.x + blockIdx.x] = red[0];
}

// out[t] = sum of the nblk partials of column t, in a fixed order.
__global__ void sum_partials(const double *part, int nblk, int ncol, double *out) {
    __shared__ double red[256];
    for (int t = blockIdx.x; t < ncol; t += gridDim.x) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[(int64_t)t * nblk + i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[t] = red[0];
        __syncthreads();
    }
}

// w[i] -= sum_t Q[i + t n] c[t]
__global__ void sub_Qc(const double *Q, int64_t n, int ncol, const double *c, double *w) {
    extern __shared__ double cs[];
    for (int t = threadIdx.x; t < ncol; t += blockDim.x) cs[t] = c[t];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < ncol; ++t) acc += Q[i + (int64_t)t * n] * cs[t];
        w[i] -= acc;
    }
}

// y[i] = sum_t Q[i + t n] S[t]  (a Ritz vector)
__global__ void gemv_Qs(const double *Q, int64_t n, int ncol, const double *S, double *y) {
    extern __shared__ double cs[];
    for (int t = threadIdx.x; t < ncol; t += blockDim.x) cs[t] = S[t];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < ncol; ++t) acc += Q[i + (int64_t)t * n] * cs[t];
        y[i] = acc;
    }
}

// w = w - alpha q - beta qprev  (qprev may be null)
__global__ void three_term(double *w, const double *q, const double *qprev, int64_t n, double alpha, double beta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = w[i] - alpha * q[i];
        if (qprev) v -= beta * qprev[i];
        w[i] = v;
    }
}

__global__ void scale_copy(const double *src, double *dst, int64_t n, double s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * s;
}

// splitmix64 counter hash -> two uniforms -> one standard normal (Box-Muller)
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void random_normal(double *x, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h1 = splitmix64(seed * 0x632be59bd9b4e019ull + 2 * (uint64_t)i);
        const uint64_t h2 = splitmix64(seed * 0x632be59bd9b4e019ull + 2 * (uint64_t)i + 1);
        const double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);   // (0, 1]
        const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);            // [0, 1)
        x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// CG helpers
__global__ void cg_operator(const double *Lp, const double *p, const double *shift, int64_t n, double beta, double *q) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = beta * Lp[i] + (shift ? shift[i] : 1.0) * p[i];
}

__global__ void sub_into(const double *f, const double *q, int64_t n, double *r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = f[i] - q[i];
}

__global__ void cg_update(double *u, double *r, const double *p, const double *q, int64_t n, double alpha) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

__global__ void axpy(double *y, const double *x, int64_t n, double a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void cg_direction(double *p, const double *r, int64_t n, double gamma) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + gamma * p[i];
}

// --------------------------------------------- tridiagonal eigensolver (QL)
// Symmetric tridiagonal T (diag d[0..k), off-diagonal e[0..k-1)) -> eigenvalues
// in d and orthonormal eigenvectors in the columns of Z (row-major k x k).
// Implicit QL sweeps with a Wilkinson-type shift; each sweep's Givens
// rotations are computed by one thread and then applied to all rows of Z by
// the whole block (rows are independent).  info[0] = 0 on success, 1 if an
// eigenvalue needed more than 64 sweeps.
__global__ void tridiag_ql(double *d, double *e_in, int k, double *Z, int *info) {
    extern __shared__ double sh[];
    double *cs = sh;           // cosines of the current sweep
    double *sn = sh + k;       // sines
    __shared__ int sweep_lo, sweep_hi, done_flag, fail;
    double *e = e_in;          // length k (e[k-1] = 0 used as sentinel)
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) Z[i] = (i / k == i % k) ? 1.0 : 0.0;
    if (threadIdx.x == 0) { fail = 0; e[k - 1] = 0.0; }
    __syncthreads();
    for (int l = 0; l < k; ++l) {
        int iter = 0;
        while (true) {
            if (threadIdx.x == 0) {
                int m = l;
                for (; m < k - 1; ++m) {
                    const double dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= 2.220446049250313e-16 * dd) break;
                }
                done_flag = (m == l);
                sweep_lo = l;
                sweep_hi = m;
                if (!done_flag) {
                    if (++iter > 64) { fail = 1; done_flag = 1; }
                }
                if (!done_flag) {
                    // shift from the leading 2x2 block
                    double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                    double r = hypot(g, 1.0);
                    g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
                    double s = 1.0, c = 1.0, p = 0.0;
                    int i = m - 1;
                    bool underflow = false;
                    for (; i >= l; --i) {
                        const double f = s * e[i];
                        const double b = c * e[i];
                        r = hypot(f, g);
                        e[i + 1] = r;
                        if (r == 0.0) {
                            d[i + 1] -= p;
                            e[m] = 0.0;
                            underflow = true;
                            break;
                        }
                        s = f / r;
                        c = g / r;
                        g = d[i + 1] - p;
                        r = (d[i] - g) * s + 2.0 * c * b;
                        p = s * r;
                        d[i + 1] = g + p;
                        g = c * r - b;
                        cs[i] = c;
                        sn[i] = s;
                    }
                    sweep_lo = underflow ? i + 1 : l;   // rotations recorded for [sweep_lo, m)
                    if (!underflow) {
                        d[l] -= p;
                        e[l] = g;
                        e[m] = 0.0;
                    }
                }
            }
            __syncthreads();
            if (done_flag) break;
            // apply the recorded rotations (i = m-1 down to sweep_lo) to every row of Z
            const int lo = sweep_lo, hi = sweep_hi;
            for (int row = threadIdx.x; row < k; row += blockDim.x) {
                double *z = Z + (int64_t)row * k;
                for (int i = hi - 1; i >= lo; --i) {
                    const double f = z[i + 1];
                    z[i + 1] = sn[i] * z[i] + cs[i] * f;
                    z[i] = cs[i] * z[i] - sn[i] * f;
                }
            }
            __syncthreads();
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) info[0] = fail;
}

// ----------------------------------------------------------------- helpers
struct Dev {
    double *buf = nullptr;
    ~Dev() { cudaFree(buf); }
};

static cudaError_t dot(Plan &P, const double *a, const double *b, double *part, double *dres, double *hres) {
    dot_partials<<<kRedBlocks, 256, 0, P.stream>>>(a, b, P.n, part);
    sum_partials<<<1, 256, 0, P.stream>>>(part, kRedBlocks, 1, dres);
    NFL_CUDA_TRY(cudaMemcpyAsync(hres, dres, sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    return cudaStreamSynchronize(P.stream);
}

static int vec_blocks(const Plan &P) { return std::max(1, P.num_sms * 8); }

// Work vectors of one CG solve (n each) and its reduction space.
struct CgWork {
    double *r, *p, *q, *lp, *part, *sc;
};

// Conjugate gradients on u -> beta L_s u + diag(s) u with P's products (Sec. 6.2.2):
// u holds the initial guess (zero_start: u is set to 0 and r = f without a product),
// stops at ||r|| <= tol ||f||.  *iters, *relres: steps taken, final ||r|| / ||f||.
static nfl_status cg_core(Plan &P, double beta, const double *shift, const double *f, double *u, bool zero_start,
                          double tol, int maxit, const CgWork &w, int *iters, double *relres) {
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    const int vb = vec_blocks(P);
    double *r = w.r, *p = w.p, *q = w.q, *lp = w.lp;
    double fn2 = 0.0;
    *iters = 0;
    if (dot(P, f, f, w.part, w.sc, &fn2) != cudaSuccess) return NFL_ERR_CUDA;
    const double fn = std::sqrt(fn2);
    if (zero_start) {
        if (cudaMemsetAsync(u, 0, n * 8, s) != cudaSuccess ||
            cudaMemcpyAsync(r, f, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return NFL_ERR_CUDA;
    } else {
        // r = f - op(u)
        const nfl_status st = run_column(P, OP_LS, u, lp);
        if (st != NFL_OK) return st;
        cg_operator<<<vb, 256, 0, s>>>(lp, u, shift, n, beta, q);
        sub_into<<<vb, 256, 0, s>>>(f, q, n, r);
    }
    if (cudaMemcpyAsync(p, r, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return NFL_ERR_CUDA;
    double rr = 0.0;
    if (dot(P, r, r, w.part, w.sc, &rr) != cudaSuccess) return NFL_ERR_CUDA;
    int it = 0;
    nfl_status result = NFL_ERR_NOT_CONVERGED;
    const double target = tol * fn;
    for (; it <= maxit; ++it) {
        if (!std::isfinite(rr)) return NFL_ERR_NAN;
        if (std::sqrt(rr) <= target) { result = NFL_OK; break; }
        if (it == maxit) break;
        const nfl_status st = run_column(P, OP_LS, p, lp);
        if (st != NFL_OK) return st;
        cg_operator<<<vb, 256, 0, s>>>(lp, p, shift, n, beta, q);
        double pq = 0.0;
        if (dot(P, p, q, w.part, w.sc, &pq) != cudaSuccess) return NFL_ERR_CUDA;
        if (!(pq > 0.0)) return std::isfinite(pq) ? NFL_ERR_BREAKDOWN : NFL_ERR_NAN;
        const double alpha = rr / pq;
        cg_update<<<vb, 256, 0, s>>>(u, r, p, q, n, alpha);
        double rr_new = 0.0;
        if (dot(P, r, r, w.part, w.sc, &rr_new) != cudaSuccess) return NFL_ERR_CUDA;
        cg_direction<<<vb, 256, 0, s>>>(p, r, n, rr_new / rr);
        rr = rr_new;
    }
    *iters = it;
    *relres = fn > 0.0 ? std::sqrt(rr) / fn : std::sqrt(rr);
    if (cudaStreamSynchronize(s) != cudaSuccess) return NFL_ERR_CUDA;
    return result;
}

}  // namespace nfl

using nfl::Plan;

extern "C" {

nfl_status nfl_lanczos_k_smallest(nfl_plan *plan, int k, double tol, int maxit, uint64_t seed,
                                  double *evals, double *evecs, int *iters) {
    using namespace nfl;
    if (!plan || !evals || k < 1 || !(tol > 0.0)) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (k >= P.n || maxit <= k || maxit > P.n || maxit > 4096) return NFL_ERR_INVALID_ARG;
    if (!P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    const int64_t n = P.n;
    const int kmax = maxit;
    const cudaStream_t s = P.stream;
    Dev Qm, W, part, sc, Tm;
    // Q: n x (kmax + 1); part: kRedBlocks x (kmax + 1); sc: (kmax+1) scalars + 2; Tm: d, e, Z, S
    if (cudaMalloc(&Qm.buf, (size_t)n * (kmax + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&W.buf, (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&part.buf, (size_t)kRedBlocks * (kmax + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&sc.buf, (size_t)(kmax + 4) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Tm.buf, (size_t)(2 * (kmax + 1) + (size_t)kmax * kmax + 2) * sizeof(double)) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    double *Q = Qm.buf, *w = W.buf;
    double *td = Tm.buf, *te = td + (kmax + 1), *Z = te + (kmax + 1);
    int *info = reinterpret_cast<int *>(Z + (size_t)kmax * kmax);
    const int vb = vec_blocks(P);
    std::vector<double> alpha, beta;   // beta[j] couples q_j and q_{j+1}
    double h = 0.0;

    random_normal<<<vb, 256, 0, s>>>(Q, n, seed);
    if (dot(P, Q, Q, part.buf, sc.buf, &h) != cudaSuccess) return NFL_ERR_CUDA;
    if (!(h > 0.0)) return NFL_ERR_NAN;
    scale_copy<<<vb, 256, 0, s>>>(Q, Q, n, 1.0 / std::sqrt(h));

    std::vector<double> hd, he, hZ, theta;
    std::vector<int> order;
    int steps = 0;
    nfl_status result = NFL_ERR_NOT_CONVERGED;
    auto ritz = [&](int j) -> nfl_status {
        // eigen-decompose T_j on the device
        if (cudaMemcpyAsync(td, alpha.data(), j * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) return NFL_ERR_CUDA;
        std::vector<double> eh(j, 0.0);
        for (int i = 0; i + 1 < j; ++i) eh[i] = beta[i];
        if (cudaMemcpyAsync(te, eh.data(), j * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) return NFL_ERR_CUDA;
        tridiag_ql<<<1, 256, 2 * j * sizeof(double), s>>>(td, te, j, Z, info);
        hd.resize(j);
        hZ.resize((size_t)j * j);
        int hinfo = 0;
        if (cudaMemcpyAsync(hd.data(), td, j * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hZ.data(), Z, (size_t)j * j * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return NFL_ERR_CUDA;
        if (hinfo) return NFL_ERR_NOT_CONVERGED;
        order.resize(j);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int b) { return hd[a] > hd[b]; });
        return NFL_OK;
    };

    for (int j = 0; j < kmax; ++j) {
        double *qj = Q + (int64_t)j * n;
        nfl_status st = run_column(P, OP_A, qj, w);                     // w = A q_j
        if (st != NFL_OK) return st;
        double a = 0.0;
        if (dot(P, qj, w, part.buf, sc.buf, &a) != cudaSuccess) return NFL_ERR_CUDA;
        if (!std::isfinite(a)) return NFL_ERR_NAN;
        three_term<<<vb, 256, 0, s>>>(w, qj, j > 0 ? qj - n : nullptr, n, a, j > 0 ? beta[j - 1] : 0.0);
        for (int pass = 0; pass < 2; ++pass) {                           // DGKS
            dim3 g(kRedBlocks, j + 1);
            multidot_partials<<<g, 256, 0, s>>>(Q, n, w, part.buf);
            sum_partials<<<std::min(j + 1, 1024), 256, 0, s>>>(part.buf, kRedBlocks, j + 1, sc.buf);
            sub_Qc<<<vb, 256, (j + 1) * sizeof(double), s>>>(Q, n, j + 1, sc.buf, w);
        }
        double bb = 0.0;
        if (dot(P, w, w, part.buf, sc.buf, &bb) != cudaSuccess) return NFL_ERR_CUDA;
        if (!std::isfinite(bb)) return NFL_ERR_NAN;
        const double b = std::sqrt(bb);
        alpha.push_back(a);
        beta.push_back(b);
        steps = j + 1;
        const bool breakdown = b <= 1e-14 * std::max(1.0, std::fabs(a));
        if (steps >= k && (steps % 5 == 0 || breakdown || steps == kmax)) {
            st = ritz(steps);
            if (st == NFL_ERR_CUDA) return st;
            if (st == NFL_OK) {
                bool conv = true;
                for (int t = 0; t < k; ++t) {
                    const int c = order[t];
                    const double resid = std::fabs(b * hZ[(size_t)(steps - 1) * steps + c]);
                    if (resid > tol) conv = false;
                }
                if (conv || breakdown) {
                    result = NFL_OK;
                    break;
                }
            }
        }
        if (breakdown) {
            result = steps >= k ? NFL_OK : NFL_ERR_BREAKDOWN;
            break;
        }
        scale_copy<<<vb, 256, 0, s>>>(w, Q + (int64_t)(j + 1) * n, n, 1.0 / b);
    }
    if (steps < k) return result == NFL_OK ? NFL_ERR_BREAKDOWN : result;
    if (order.size() != (size_t)steps) {
        nfl_status st = ritz(steps);
        if (st != NFL_OK) return st;
    }
    // eigenvalues of L_s ascending = 1 - theta for theta descending
    for (int t = 0; t < k; ++t) evals[t] = 1.0 - hd[order[t]];
    if (evecs) {
        std::vector<double> col(steps);
        double *dcol = sc.buf;
        for (int t = 0; t < k; ++t) {
            for (int i = 0; i < steps; ++i) col[i] = hZ[(size_t)i * steps + order[t]];
            if (cudaMemcpyAsync(dcol, col.data(), steps * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return NFL_ERR_CUDA;
            gemv_Qs<<<vb, 256, steps * sizeof(double), s>>>(Q, n, steps, dcol, evecs + (int64_t)t * n);
            if (cudaStreamSynchronize(s) != cudaSuccess) return NFL_ERR_CUDA;
        }
    }
    if (iters) *iters = steps;
    if (cudaStreamSynchronize(s) != cudaSuccess) return NFL_ERR_CUDA;
    return result;
}

nfl_status nfl_cg_solve(nfl_plan *plan, double beta, const double *shift, const double *f, double *u, double tol,
                        int maxit, int *iters, double *relres) {
    using namespace nfl;
    if (!plan || !f || !u || !(beta > 0.0) || !(tol > 0.0) || maxit < 1) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (!P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    const int64_t n = P.n;
    Dev W, part, sc;
    if (cudaMalloc(&W.buf, 4 * n * 8) != cudaSuccess || cudaMalloc(&part.buf, kRedBlocks * 8) != cudaSuccess ||
        cudaMalloc(&sc.buf, 8 * 8) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    const CgWork w{W.buf, W.buf + n, W.buf + 2 * n, W.buf + 3 * n, part.buf, sc.buf};
    int it = 0;
    double rel = 0.0;
    const nfl_status st = cg_core(P, beta, shift, f, u, false, tol, maxit, w, &it, &rel);
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return st;
}

/*
 * Mixed-precision iterative refinement of the CG solve: residuals with the
 * outer plan's products (FP64), corrections by CG with the inner plan's
 * products (FP32C).
 */
nfl_status nfl_cg_solve_refined(nfl_plan *plan, nfl_plan *inner, double beta, const double *shift, const double *f,
                                double *u, double tol, double inner_tol, int maxit, int max_outer, int *iters,
                                int *outer, double *relres) {
    using namespace nfl;
    if (!plan || !inner || plan == inner || !f || !u || !(beta > 0.0) || !(tol > 0.0) || !(inner_tol > 0.0) ||
        !(inner_tol < 1.0) || maxit < 1 || max_outer < 1)
        return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    Plan &Q = *reinterpret_cast<Plan *>(inner);
    if (Q.n != P.n || Q.d != P.d || Q.kernel != P.kernel || Q.sigma != P.sigma) return NFL_ERR_INVALID_ARG;
    for (int a = 0; a < P.d; ++a)
        if (Q.center[a] != P.center[a]) return NFL_ERR_INVALID_ARG;     // other nodes
    if (!P.degree_ok || !Q.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    const int vb = vec_blocks(P);
    Dev W, part, sc;
    if (cudaMalloc(&W.buf, 6 * n * 8) != cudaSuccess || cudaMalloc(&part.buf, kRedBlocks * 8) != cudaSuccess ||
        cudaMalloc(&sc.buf, 8 * 8) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    // inner CG work (4 n), the outer residual r and the correction c
    const CgWork w{W.buf, W.buf + n, W.buf + 2 * n, W.buf + 3 * n, part.buf, sc.buf};
    double *r = W.buf + 4 * n, *c = W.buf + 5 * n;
    // the inner plan works on this plan's stream for the call
    const cudaStream_t qs = Q.stream;
    Q.stream = s;
    double fn2 = 0.0, rr = 0.0;
    int total = 0, k = 0;
    nfl_status result = NFL_ERR_NOT_CONVERGED;
    nfl_status st = dot(P, f, f, part.buf, sc.buf, &fn2) == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
    const double fn = std::sqrt(fn2);
    for (; st == NFL_OK; ++k) {
        // r = f - (beta L_s + S) u with the outer (FP64) products
        st = run_column(P, OP_LS, u, w.lp);
        if (st != NFL_OK) break;
        cg_operator<<<vb, 256, 0, s>>>(w.lp, u, shift, n, beta, w.q);
        sub_into<<<vb, 256, 0, s>>>(f, w.q, n, r);
        if (dot(P, r, r, part.buf, sc.buf, &rr) != cudaSuccess) { st = NFL_ERR_CUDA; break; }
        if (!std::isfinite(rr)) { st = NFL_ERR_NAN; break; }
        if (std::sqrt(rr) <= tol * fn) { result = NFL_OK; break; }
        if (k == max_outer) break;
        // (beta L_s + S) c = r with the inner products, from c = 0, to inner_tol ||r||
        int it = 0;
        double rel = 0.0;
        const nfl_status ist = cg_core(Q, beta, shift, r, c, true, inner_tol, maxit, w, &it, &rel);
        total += it;
        if (ist != NFL_OK && ist != NFL_ERR_NOT_CONVERGED) { st = ist; break; }
        axpy<<<vb, 256, 0, s>>>(u, c, n, 1.0);
    }
    Q.stream = qs;
    if (iters) *iters = total;
    if (outer) *outer = k;
    if (relres) *relres = fn > 0.0 ? std::sqrt(rr) / fn : std::sqrt(rr);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == NFL_OK) st = NFL_ERR_CUDA;
    return st != NFL_OK ? st : result;
}

}  // extern "C"

// ------------------------------------------------------- gradients through CG
namespace nfl {

// out_i = -lambda_i u_i
__global__ void neg_product(const double *lam, const double *u, int64_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = -lam[i] * u[i];
}

// a~ = a / sqrt(d), b~ = b / sqrt(d)
__global__ void scale_by_degree(const double *a, const double *b, const double *d, int64_t n, double *at,
                                double *bt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = 1.0 / sqrt(d[i]);
        at[i] = a[i] * s;
        bt[i] = b[i] * s;
    }
}

// per-block partial sums of -a~_i (W_s b~)_i + (delta_i / d_i) (a~_i (W b~)_i + (W a~)_i b~_i) / 2
__global__ void dsigma_form_partials(const double *at, const double *bt, const double *Wsb, const double *Wb,
                                     const double *Wa, const double *delta, const double *d, int64_t n,
                                     double *part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += -at[i] * Wsb[i] + 0.5 * delta[i] / d[i] * (at[i] * Wb[i] + Wa[i] * bt[i]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace nfl

extern "C" {

nfl_status nfl_cg_solve_backward(nfl_plan *plan, nfl_plan *dplan, double beta, const double *shift,
                                 const double *u, const double *g, double tol, int maxit, double *grad_f,
                                 double *grad_shift, double *grad_beta, double *grad_sigma, int *iters,
                                 double *relres) {
    using namespace nfl;
    if (!plan || !u || !g || !grad_f) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (grad_sigma && !dplan) return NFL_ERR_INVALID_ARG;
    if (dplan) {
        const Plan &D = *reinterpret_cast<const Plan *>(dplan);
        if (D.n != P.n || D.d != P.d || D.kernel != NFL_KERNEL_GAUSSIAN_DSIGMA || P.kernel != NFL_KERNEL_GAUSSIAN ||
            D.sigma != P.sigma || D.N != P.N || D.m != P.m || D.p != P.p || D.eps_B != P.eps_B)
            return NFL_ERR_INVALID_ARG;
    }
    // lambda = (beta L_s + diag(s))^{-1} g: the operator is symmetric
    nfl_status st = nfl_cg_solve(plan, beta, shift, g, grad_f, tol, maxit, iters, relres);
    if (st != NFL_OK) return st;
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    const int vb = vec_blocks(P);
    const double *lam = grad_f;
    if (grad_shift) neg_product<<<vb, 256, 0, s>>>(lam, u, n, grad_shift);
    if (!grad_beta && !grad_sigma) return cudaStreamSynchronize(s) == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
    Dev part, sc, T0, T1, T2, T3, T4;
    if (cudaMalloc(&part.buf, kRedBlocks * 8) != cudaSuccess || cudaMalloc(&sc.buf, 8 * 8) != cudaSuccess ||
        cudaMalloc(&T0.buf, n * 8) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    if (grad_beta) {
        // dl/dbeta = -lambda^T L_s u
        st = run_column(P, OP_LS, u, T0.buf);
        if (st != NFL_OK) return st;
        double v = 0.0;
        if (dot(P, lam, T0.buf, part.buf, sc.buf, &v) != cudaSuccess) return NFL_ERR_CUDA;
        *grad_beta = -v;
    }
    if (grad_sigma) {
        Plan &D = *reinterpret_cast<Plan *>(dplan);
        if (cudaMalloc(&T1.buf, n * 8) != cudaSuccess || cudaMalloc(&T2.buf, n * 8) != cudaSuccess ||
            cudaMalloc(&T3.buf, n * 8) != cudaSuccess || cudaMalloc(&T4.buf, n * 8) != cudaSuccess)
            return NFL_ERR_OUT_OF_MEMORY;
        double *at = T0.buf, *bt = T1.buf, *Wb = T2.buf, *Wa = T3.buf, *Wsb = T4.buf;
        scale_by_degree<<<vb, 256, 0, s>>>(lam, u, P.degree, n, at, bt);
        st = run_column(P, OP_W, bt, Wb);
        if (st == NFL_OK) st = run_column(P, OP_W, at, Wa);
        if (st != NFL_OK) return st;
        // the derivative plan runs on this plan's stream for the call
        const cudaStream_t ds = D.stream;
        D.stream = s;
        st = run_column(D, OP_W, bt, Wsb);
        D.stream = ds;
        if (st != NFL_OK) return st;
        dsigma_form_partials<<<kRedBlocks, 256, 0, s>>>(at, bt, Wsb, Wb, Wa, D.degree, P.degree, n, part.buf);
        sum_partials<<<1, 256, 0, s>>>(part.buf, kRedBlocks, 1, sc.buf);
        double form = 0.0;
        if (cudaMemcpyAsync(&form, sc.buf, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return NFL_ERR_CUDA;
        *grad_sigma = -beta * form;                       // form = lambda^T (dL_s/dsigma) u
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

}  // extern "C"

// ------------------------------------- gradient of a~^T W b~ in the node coordinates
namespace nfl {

// c = (a~ (W b~) + b~ (W a~)) / d
__global__ void form_c(const double *at, const double *bt, const double *Wa, const double *Wb, const double *d,
                       int64_t n, double *c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = (at[i] * Wb[i] + bt[i] * Wa[i]) / d[i];
}

// S0 = a~ (W b~) + b~ (W a~) - c d / 2 - (W c) / 2
__global__ void form_s0(const double *at, const double *bt, const double *Wa, const double *Wb, const double *c,
                        const double *d, const double *Wc, int64_t n, double *S0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        S0[i] = at[i] * Wb[i] + bt[i] * Wa[i] - 0.5 * c[i] * d[i] - 0.5 * Wc[i];
}

// columns (b~ y, a~ y, y, c y) of X (n x 4, column-major) for y = v_alpha - center_alpha
__global__ void form_columns(const double *v, int dim, int alpha, double center, const double *at, const double *bt,
                             const double *c, int64_t n, double *X) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double y = v[i * dim + alpha] - center;
        X[i] = bt[i] * y;
        X[i + n] = at[i] * y;
        X[i + 2 * n] = y;
        X[i + 3 * n] = c[i] * y;
    }
}

// grad[i, alpha] = scale (y_i S0_i - (a~_i Y0_i + b~_i Y1_i - c_i Y2_i / 2 - Y3_i / 2))
__global__ void form_grad_axis(const double *v, int dim, int alpha, double center, const double *S0,
                               const double *at, const double *bt, const double *c, const double *Y, int64_t n,
                               double scale, double *grad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double y = v[i * dim + alpha] - center;
        const double s1 = at[i] * Y[i] + bt[i] * Y[i + n] - 0.5 * c[i] * Y[i + 2 * n] - 0.5 * Y[i + 3 * n];
        grad[i * dim + alpha] = scale * (y * S0[i] - s1);
    }
}

}  // namespace nfl

extern "C" {

nfl_status nfl_form_grad_nodes(nfl_plan *plan, const double *v, const double *a, const double *b, double *grad) {
    using namespace nfl;
    if (!plan || !v || !a || !b || !grad) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (P.kernel != NFL_KERNEL_GAUSSIAN) return NFL_ERR_INVALID_ARG;
    if (!P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    const int vb = vec_blocks(P);
    Dev at, bt, Wa, Wb, c, Wc, S0, X, Y;
    for (Dev *t : {&at, &bt, &Wa, &Wb, &c, &Wc, &S0})
        if (cudaMalloc(&t->buf, n * 8) != cudaSuccess) return NFL_ERR_OUT_OF_MEMORY;
    if (cudaMalloc(&X.buf, 4 * n * 8) != cudaSuccess || cudaMalloc(&Y.buf, 4 * n * 8) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    scale_by_degree<<<vb, 256, 0, s>>>(a, b, P.degree, n, at.buf, bt.buf);
    nfl_status st = run_column(P, OP_W, at.buf, Wa.buf);
    if (st == NFL_OK) st = run_column(P, OP_W, bt.buf, Wb.buf);
    if (st != NFL_OK) return st;
    form_c<<<vb, 256, 0, s>>>(at.buf, bt.buf, Wa.buf, Wb.buf, P.degree, n, c.buf);
    st = run_column(P, OP_W, c.buf, Wc.buf);
    if (st != NFL_OK) return st;
    form_s0<<<vb, 256, 0, s>>>(at.buf, bt.buf, Wa.buf, Wb.buf, c.buf, P.degree, Wc.buf, n, S0.buf);
    // grad K(y) = -(2 / sigma^2) y K(y) for the Gaussian
    const double scale = -2.0 / (P.sigma * P.sigma);
    for (int alpha = 0; alpha < P.d; ++alpha) {
        form_columns<<<vb, 256, 0, s>>>(v, P.d, alpha, P.center[alpha], at.buf, bt.buf, c.buf, n, X.buf);
        for (int col = 0; col < 4 && st == NFL_OK; ++col) st = run_column(P, OP_W, X.buf + col * n, Y.buf + col * n);
        if (st != NFL_OK) return st;
        form_grad_axis<<<vb, 256, 0, s>>>(v, P.d, alpha, P.center[alpha], S0.buf, at.buf, bt.buf, c.buf, Y.buf, n,
                                          scale, grad);
    }
    if (cudaGetLastError() != cudaSuccess) return NFL_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

}  // extern "C"

// ------------------------------------------------ Alg. 3: Nystrom-Gaussian-NFFT
namespace nfl {

// Pair t of round r of the round-robin ordering on cp players (cp even): every
// pair of players meets once in the cp - 1 rounds, and the pairs of a round are
// disjoint.
__device__ __forceinline__ void rr_pair(int r, int t, int cp, int *p, int *q) {
    if (t == 0) {
        *p = r % (cp - 1);
        *q = cp - 1;
    } else {
        *p = (r + t) % (cp - 1);
        *q = (r - t + cp - 1) % (cp - 1);
    }
}

// Eigen-decomposition of a symmetric c x c matrix A (column-major, overwritten),
// one CTA: cyclic Jacobi sweeps in the parallel ordering (each round rotates the
// c/2 disjoint pairs of the round-robin schedule at once, A <- J^T A J with J the
// product of the round's plane rotations, each chosen to zero its A_pq), until the
// off-diagonal part is below 1e-30 of A in the squared Frobenius norm (60 sweeps
// at most).  Then the eigenvalues are ranked in descending order and the first
// `keep` are written to vals with their eigenvectors as the columns of vecs
// (c x keep, column-major).  V is c x c workspace.  info[0] = 1 when the sweeps
// did not converge, info[1] = 1 when a kept eigenvalue is not positive (with
// require_positive), info[2] = 1 when A held a NaN or Inf.
__global__ void __launch_bounds__(1024) jacobi_eig_kernel(double *A, int c, double *V, int keep, int require_positive,
                                                          double *vals, double *vecs, int *info) {
    extern __shared__ double sh[];
    const int cp = c + (c & 1), np = cp / 2;
    double *cs = sh, *sn = sh + np;
    __shared__ double red_off[1024], red_tot[1024];
    __shared__ int stop;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < c * c; e += nt) V[e] = (e % c == e / c) ? 1.0 : 0.0;
    __syncthreads();
    int sweep = 0;
    for (; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < c * c; e += nt) {
            const double a2 = A[e] * A[e];
            tot += a2;
            if (e % c != e / c) off += a2;
        }
        red_off[tid] = off;
        red_tot[tid] = tot;
        __syncthreads();
        for (int h = nt / 2; h > 0; h >>= 1) {
            if (tid < h) {
                red_off[tid] += red_off[tid + h];
                red_tot[tid] += red_tot[tid + h];
            }
            __syncthreads();
        }
        if (tid == 0) {
            const double o = red_off[0], t = red_tot[0];
            stop = !isfinite(t) ? 2 : ((o <= 1e-30 * t || o == 0.0) ? 1 : 0);
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < cp - 1; ++r) {
            for (int t = tid; t < np; t += nt) {
                int p, q;
                rr_pair(r, t, cp, &p, &q);
                double cv = 1.0, sv = 0.0;
                if (p < c && q < c) {
                    const double apq = A[p + (int64_t)q * c];
                    if (apq != 0.0) {
                        const double theta = (A[q + (int64_t)q * c] - A[p + (int64_t)p * c]) / (2.0 * apq);
                        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        cv = 1.0 / sqrt(tt * tt + 1.0);
                        sv = tt * cv;
                    }
                }
                cs[t] = cv;
                sn[t] = sv;
            }
            __syncthreads();
            // rows p, q of A (A <- J^T A)
            for (int e = tid; e < np * c; e += nt) {
                const int t = e / c, k = e - t * c;
                int p, q;
                rr_pair(r, t, cp, &p, &q);
                if (p >= c || q >= c) continue;
                const double apk = A[p + (int64_t)k * c], aqk = A[q + (int64_t)k * c];
                A[p + (int64_t)k * c] = cs[t] * apk - sn[t] * aqk;
                A[q + (int64_t)k * c] = sn[t] * apk + cs[t] * aqk;
            }
            __syncthreads();
            // columns p, q of A and V (A <- A J, V <- V J)
            for (int e = tid; e < np * c; e += nt) {
                const int t = e / c, k = e - t * c;
                int p, q;
                rr_pair(r, t, cp, &p, &q);
                if (p >= c || q >= c) continue;
                const double akp = A[k + (int64_t)p * c], akq = A[k + (int64_t)q * c];
                A[k + (int64_t)p * c] = cs[t] * akp - sn[t] * akq;
                A[k + (int64_t)q * c] = sn[t] * akp + cs[t] * akq;
                const double vkp = V[k + (int64_t)p * c], vkq = V[k + (int64_t)q * c];
                V[k + (int64_t)p * c] = cs[t] * vkp - sn[t] * vkq;
                V[k + (int64_t)q * c] = sn[t] * vkp + cs[t] * vkq;
            }
            __syncthreads();
        }
    }
    // rank of eigenvalue i in descending order (ties by index), keep the first `keep`
    for (int i = tid; i < c; i += nt) {
        const double li = A[i + (int64_t)i * c];
        int rank = 0;
        for (int j = 0; j < c; ++j) {
            const double lj = A[j + (int64_t)j * c];
            rank += (lj > li || (lj == li && j < i)) ? 1 : 0;
        }
        if (rank < keep) {
            vals[rank] = li;
            for (int k = 0; k < c; ++k) vecs[k + (int64_t)rank * c] = V[k + (int64_t)i * c];
            if (require_positive && !(li > 0.0)) atomicExch(&info[1], 1);
        }
    }
    if (tid == 0) {
        if (stop == 2) info[2] = 1;
        else if (!stop) info[0] = 1;
    }
}

// B = (B + B^T) / 2 for a c x c matrix (column-major).
__global__ void symmetrize(double *B, int c) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
        const int i = e % c, j = e / c;
        if (i < j) {
            const double a = 0.5 * (B[i + (int64_t)j * c] + B[j + (int64_t)i * c]);
            B[i + (int64_t)j * c] = a;
            B[j + (int64_t)i * c] = a;
        }
    }
}

// R[0..j) of column j += coef[0..j)  (Gram-Schmidt coefficients)
__global__ void add_coef(double *Rj, const double *coef, int j) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) Rj[i] += coef[i];
}

// Column j's norm: R_jj = ||x_j|| unless it fell below 1e-13 of its norm before
// orthogonalization (n0), in which case the column is dependent (R_jj = 0, and
// the column is zeroed); scale[0] receives the factor applied to x_j.
__global__ void gs_norm(double *Rjj, const double *n0, const double *nn, double *scale, int *info) {
    const double nrm = sqrt(*nn);
    if (!isfinite(*n0) || !isfinite(*nn)) info[2] = 1;
    const bool dependent = !(nrm > 1e-13 * sqrt(*n0));
    *Rjj = dependent ? 0.0 : nrm;
    *scale = dependent ? 0.0 : 1.0 / nrm;
}

__global__ void scale_by(double *x, int64_t n, const double *s) {
    const double f = *s;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

// T = R diag(1 / sig) R^T, R M x M column-major.
__global__ void form_T(const double *R, const double *sig, int M, double *T) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += gridDim.x * blockDim.x) {
        const int i = e % M, j = e / M;
        double acc = 0.0;
        for (int t = 0; t < M; ++t) acc += R[i + (int64_t)t * M] * R[j + (int64_t)t * M] / sig[t];
        T[e] = acc;
    }
}

// Orthonormalize the c columns of X (n x c, column-major, in place) by Gram-Schmidt
// with one reorthogonalization (DGKS), all on the device: R (device, c x c,
// column-major, upper triangular) receives X_in = X_out R; a column that falls
// below 1e-13 of its norm is dependent and becomes zero (R_jj = 0).  sc holds
// c + 4 doubles of workspace.
static cudaError_t gs_qr(Plan &P, double *X, int c, double *part, double *sc, double *R, int *info) {
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    const int vb = vec_blocks(P);
    double *n0 = sc + c, *nn = sc + c + 1, *scale = sc + c + 2;
    NFL_CUDA_TRY(cudaMemsetAsync(R, 0, (size_t)c * c * sizeof(double), s));
    for (int j = 0; j < c; ++j) {
        double *xj = X + (int64_t)j * n;
        dot_partials<<<kRedBlocks, 256, 0, s>>>(xj, xj, n, part);
        sum_partials<<<1, 256, 0, s>>>(part, kRedBlocks, 1, n0);
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            dim3 g(kRedBlocks, j);
            multidot_partials<<<g, 256, 0, s>>>(X, n, xj, part);
            sum_partials<<<std::min(j, 1024), 256, 0, s>>>(part, kRedBlocks, j, sc);
            sub_Qc<<<vb, 256, j * sizeof(double), s>>>(X, n, j, sc, xj);
            add_coef<<<1, 256, 0, s>>>(R + (int64_t)j * c, sc, j);
        }
        dot_partials<<<kRedBlocks, 256, 0, s>>>(xj, xj, n, part);
        sum_partials<<<1, 256, 0, s>>>(part, kRedBlocks, 1, nn);
        gs_norm<<<1, 1, 0, s>>>(R + (int64_t)j * c + j, n0, nn, scale, info);
        scale_by<<<vb, 256, 0, s>>>(xj, n, scale);
    }
    return cudaGetLastError();
}

// Y[:, j] = X S[:, j] for j < ncol, X n x c and S c x ncol (column-major), both on the device.
static cudaError_t times_small(Plan &P, const double *X, int c, const double *S, int ncol, double *Y) {
    for (int j = 0; j < ncol; ++j)
        gemv_Qs<<<vec_blocks(P), 256, c * sizeof(double), P.stream>>>(X, P.n, c, S + (int64_t)j * c,
                                                                       Y + (int64_t)j * P.n);
    return cudaGetLastError();
}

static cudaError_t jacobi(Plan &P, double *A, int c, double *V, int keep, bool positive, double *vals, double *vecs,
                          int *info) {
    const int np = (c + 1) / 2;
    jacobi_eig_kernel<<<1, 1024, 2 * np * sizeof(double), P.stream>>>(A, c, V, keep, positive ? 1 : 0, vals, vecs,
                                                                      info);
    return cudaGetLastError();
}

}  // namespace nfl

extern "C" {

nfl_status nfl_nystrom_k_largest(nfl_plan *plan, int k, int L, int M, const double *G, uint64_t seed,
                                 double *evals, double *evecs) {
    using namespace nfl;
    if (!plan || !evals || k < 1 || M < k || L < M) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (L > P.n || L > 512) return NFL_ERR_INVALID_ARG;
    if (!P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;               // step 2 (degrees of the plan)
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    // device: Y, B1 (n x L), C (n x M); the small matrices B2, V (L x L), U_M (L x M),
    // sig (L), R (L x L), T, Uh (M x M), lam (M), U_k (M x k); status flags
    Dev Yb, Bb, Cb, part, sc, small, flags;
    const size_t nsmall = (size_t)4 * L * L + 2 * L + 2 * (size_t)M * M + M + (size_t)M * k + 8;
    if (cudaMalloc(&Yb.buf, (size_t)n * L * 8) != cudaSuccess || cudaMalloc(&Bb.buf, (size_t)n * L * 8) != cudaSuccess ||
        cudaMalloc(&Cb.buf, (size_t)n * M * 8) != cudaSuccess ||
        cudaMalloc(&part.buf, (size_t)kRedBlocks * L * 8) != cudaSuccess ||
        cudaMalloc(&sc.buf, (size_t)(L + 8) * 8) != cudaSuccess || cudaMalloc(&small.buf, nsmall * 8) != cudaSuccess ||
        cudaMalloc(&flags.buf, 8 * sizeof(int)) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    double *Y = Yb.buf, *B1 = Bb.buf, *C = Cb.buf;
    double *B2 = small.buf, *V = B2 + (size_t)L * L, *UM = V + (size_t)L * L, *sig = UM + (size_t)L * L;
    double *R = sig + L, *T = R + (size_t)L * L, *Uh = T + (size_t)M * M, *lam = Uh + (size_t)M * M;
    double *Uk = lam + M;
    int *info = reinterpret_cast<int *>(flags.buf);
    NFL_STATUS_TRY(cudaMemsetAsync(info, 0, 8 * sizeof(int), s));
    // step 3: Y = A G column by column, Q = orth(Y) (in place)
    if (G) {
        if (cudaMemcpyAsync(B1, G, (size_t)n * L * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return NFL_ERR_CUDA;
    } else {
        random_normal<<<vec_blocks(P), 256, 0, s>>>(B1, n * L, seed);
    }
    for (int j = 0; j < L; ++j) {
        nfl_status st = run_column(P, OP_A, B1 + (int64_t)j * n, Y + (int64_t)j * n);
        if (st != NFL_OK) return st;
    }
    NFL_STATUS_TRY(gs_qr(P, Y, L, part.buf, sc.buf, R, info));
    // step 4: B1 = A Q, B2 = Q^T B1 (symmetrized)
    for (int j = 0; j < L; ++j) {
        nfl_status st = run_column(P, OP_A, Y + (int64_t)j * n, B1 + (int64_t)j * n);
        if (st != NFL_OK) return st;
    }
    for (int j = 0; j < L; ++j) {
        dim3 g(kRedBlocks, L);
        multidot_partials<<<g, 256, 0, s>>>(Y, n, B1 + (int64_t)j * n, part.buf);
        sum_partials<<<std::min(L, 1024), 256, 0, s>>>(part.buf, kRedBlocks, L, B2 + (int64_t)j * L);
    }
    symmetrize<<<std::max(1, (L * L + 255) / 256), 256, 0, s>>>(B2, L);
    // step 5: the M largest eigenvalues of B2 (all positive) and their eigenvectors U_M (L x M)
    NFL_STATUS_TRY(jacobi(P, B2, L, V, M, true, sig, UM, info));
    // step 6: Qh Rh = B1 U_M
    NFL_STATUS_TRY(times_small(P, B1, L, UM, M, C));
    NFL_STATUS_TRY(gs_qr(P, C, M, part.buf, sc.buf, R, info));
    // step 7: eig of T = Rh Sigma_M^{-1} Rh^T; V_M = Qh Uh
    form_T<<<std::max(1, (M * M + 255) / 256), 256, 0, s>>>(R, sig, M, T);
    NFL_STATUS_TRY(jacobi(P, T, M, Uh, k, false, lam, Uk, info));
    // step 8: the k largest
    int h_info[8] = {0};
    NFL_STATUS_TRY(cudaMemcpyAsync(h_info, info, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NFL_STATUS_TRY(cudaMemcpyAsync(evals, lam, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    NFL_STATUS_TRY(cudaStreamSynchronize(s));
    if (h_info[2]) return NFL_ERR_NAN;
    if (h_info[0]) return NFL_ERR_NOT_CONVERGED;
    if (h_info[1]) return NFL_ERR_BREAKDOWN;
    if (evecs) NFL_STATUS_TRY(times_small(P, C, M, Uk, k, evecs));
    return cudaStreamSynchronize(s) == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

}  // extern "C"
