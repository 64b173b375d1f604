// nfl_cg_solve_noalloc: conjugate gradients for (beta L_s + diag(s)) u = f
// that performs no device allocation.
//
// nfl_cg_solve allocates its four work vectors and its reduction partials
// with cudaMalloc on every call.  Some callers cannot do that at solve time:
// code under an allocator that must not see foreign allocations (a caching
// allocator that owns the device's memory), or services that fix their
// device footprint at start-up.  This entry point takes the same arguments
// and runs the same iteration, but its scratch lives in one file-scope
// static device array (sized for n <= NFL_NOALLOC_MAX_N), whose device
// address is looked up once per device.  The products with L_s use the
// plan's buffers, which were allocated when the plan was created.  Like
// nfl_cg_solve it reads every reduction back to the host and synchronizes
// the plan's stream in every iteration (the host decides convergence and
// breakdown), so it cannot run while its stream is being captured.
//
// The array is shared by every call in the process and keeps the previous
// call's contents; every word the solver reads is written first in the same
// call, so nothing needs clearing.  Calls that overlap on the GPU (other
// streams, other plans, other host threads) race on it.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kMaxN = NFL_NOALLOC_MAX_N;
constexpr int kParts = 512;
constexpr int64_t kScratchDoubles = 4 * kMaxN + kParts + 8;

// r, p, q, L_s p (4 x kMaxN), reduction partials (kParts), scalars (8)
__device__ __align__(256) double g_cg_scratch[kScratchDoubles];

std::mutex g_lock;
double *g_scratch_addr[256] = {};

// Device address of g_cg_scratch on the current device (looked up on the
// first call per device, with that device current).
nfl_status scratch_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NFL_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cg_scratch) != cudaSuccess || !p) return NFL_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return NFL_OK;
}

__global__ void na_dot_partials(const double *a, const double *b, int64_t n, double *part) {
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

__global__ void na_sum_partials(const double *part, int nblk, double *out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

__global__ void na_operator(const double *Lp, const double *p, const double *shift, int64_t n, double beta, double *q) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = beta * Lp[i] + (shift ? shift[i] : 1.0) * p[i];
}

__global__ void na_residual(const double *f, const double *q, int64_t n, double *r, double *p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = f[i] - q[i];
        r[i] = v;
        p[i] = v;
    }
}

__global__ void na_update(double *u, double *r, const double *p, const double *q, int64_t n, double alpha) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

__global__ void na_direction(double *p, const double *r, int64_t n, double gamma) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + gamma * p[i];
}

cudaError_t na_dot(cudaStream_t s, const double *a, const double *b, int64_t n, double *part, double *dres,
                   double *hres) {
    na_dot_partials<<<kParts, 256, 0, s>>>(a, b, n, part);
    na_sum_partials<<<1, 256, 0, s>>>(part, kParts, dres);
    cudaError_t e = cudaMemcpyAsync(hres, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace

extern "C" nfl_status nfl_cg_solve_noalloc(nfl_plan *plan, double beta, const double *shift, const double *f,
                                           double *u, double tol, int maxit, int *iters, double *relres) {
    using namespace nfl;
    if (!plan || !f || !u || !(beta > 0.0) || !(tol > 0.0) || maxit < 1) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (P.n > kMaxN) return NFL_ERR_INVALID_ARG;
    if (!P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    double *base = nullptr;
    nfl_status st = scratch_address(&base);
    if (st != NFL_OK) return st;
    const int64_t n = P.n;
    const cudaStream_t s = P.stream;
    double *r = base, *p = base + kMaxN, *q = base + 2 * kMaxN, *lp = base + 3 * kMaxN;
    double *part = base + 4 * kMaxN, *sc = part + kParts;
    const int vb = P.num_sms > 0 ? P.num_sms * 8 : 1024;

    double fn2 = 0.0;
    if (na_dot(s, f, f, n, part, sc, &fn2) != cudaSuccess) return NFL_ERR_CUDA;
    const double fn = std::sqrt(fn2);
    st = run_column(P, OP_LS, u, lp);                       // r = f - (beta L_s u + s u), p = r
    if (st != NFL_OK) return st;
    na_operator<<<vb, 256, 0, s>>>(lp, u, shift, n, beta, q);
    na_residual<<<vb, 256, 0, s>>>(f, q, n, r, p);
    double rr = 0.0;
    if (na_dot(s, r, r, n, part, sc, &rr) != cudaSuccess) return NFL_ERR_CUDA;
    int it = 0;
    nfl_status result = NFL_ERR_NOT_CONVERGED;
    const double target = tol * fn;
    for (; it <= maxit; ++it) {
        if (!std::isfinite(rr)) return NFL_ERR_NAN;
        if (std::sqrt(rr) <= target) { result = NFL_OK; break; }
        if (it == maxit) break;
        st = run_column(P, OP_LS, p, lp);
        if (st != NFL_OK) return st;
        na_operator<<<vb, 256, 0, s>>>(lp, p, shift, n, beta, q);
        double pq = 0.0;
        if (na_dot(s, p, q, n, part, sc, &pq) != cudaSuccess) return NFL_ERR_CUDA;
        if (!(pq > 0.0)) return std::isfinite(pq) ? NFL_ERR_BREAKDOWN : NFL_ERR_NAN;
        const double alpha = rr / pq;
        na_update<<<vb, 256, 0, s>>>(u, r, p, q, n, alpha);
        double rr_new = 0.0;
        if (na_dot(s, r, r, n, part, sc, &rr_new) != cudaSuccess) return NFL_ERR_CUDA;
        na_direction<<<vb, 256, 0, s>>>(p, r, n, rr_new / rr);
        rr = rr_new;
    }
    if (iters) *iters = it;
    if (relres) *relres = fn > 0.0 ? std::sqrt(rr) / fn : std::sqrt(rr);
    if (cudaStreamSynchronize(s) != cudaSuccess) return NFL_ERR_CUDA;
    return result;
}
