// Products with W, A and L_s: Alg. 1 (spread, FFT/multiply/inverse FFT,
// interpolate) with the Alg. 2 step 5 scalings fused into spread and gather.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

namespace nfl {

int kernels_per_column(const Plan &P) {
    const int passes = P.d == 1 ? 1 : (P.d == 2 ? 3 : 5);
    const bool staged = P.d == 3 && column_tile_edge(P.m) == P.tile_edge;
    // the one-column spread and interpolation with dense cells launch the warp-slice and
    // tensor-core kernels for the sparse tiles and the moment kernels for the dense ones
    // (the spreads each only when they have items; the tensor-core launch always counts)
    const bool split = moments_available(P) && P.nslab > 0;
    const int spreads = moments_available(P) ? (P.nsparse > 0 ? 1 : 0) + (P.nslab > 0 ? 1 : 0) : 1;
    const int gathers = split && gather_tc_available(P) ? 2 : 1;
    return (staged || P.prec == NFL_PREC_FP32C ? 1 : 0) + spreads + passes + gathers;
}

// stage events: 5 per timed product (before prep, spread, fft, gather, after); a
// product of nc columns (a block) counts nc columns
static cudaError_t mark(Plan &P, int stage, int nc = 1) {
    if (!P.profile) return cudaSuccess;
    const size_t idx = P.events_used + stage;
    while (P.events.size() <= idx) {
        cudaEvent_t e;
        NFL_CUDA_TRY(cudaEventCreate(&e));
        P.events.push_back(e);
    }
    NFL_CUDA_TRY(cudaEventRecord(P.events[idx], P.stream));
    if (stage == 4) {
        P.events_used += 5;
        P.event_cols.push_back(nc);
    }
    return cudaSuccess;
}

nfl_status run_column(Plan &P, int op, const double *x, double *y) {
    const bool ones = (op == OP_DEGREE);
    const bool scale = (op == OP_A || op == OP_LS);
    NFL_STATUS_TRY(mark(P, 0));
    NFL_STATUS_TRY(prepare_spread(P, op, x, P.n, 1, ones, scale));
    NFL_STATUS_TRY(mark(P, 1));
    NFL_STATUS_TRY(launch_spread(P, x, 0, ones, scale));
    NFL_STATUS_TRY(mark(P, 2));
    NFL_STATUS_TRY(launch_fft(P));
    NFL_STATUS_TRY(mark(P, 3));
    NFL_STATUS_TRY(launch_gather(P, op, x, y));
    NFL_STATUS_TRY(mark(P, 4));
    return NFL_OK;
}

bool block_path_available(const Plan &P) { return spread_warp_available(P) && gather_tc_available(P); }

// nc <= kBlockCols columns (x + c ldx -> y + c ldy) through each stage in one launch
static nfl_status run_block_stages(Plan &P, int op, const double *x, int64_t ldx, double *y, int64_t ldy, int nc) {
    const bool scale = (op == OP_A || op == OP_LS);
    NFL_STATUS_TRY(mark(P, 0));
    NFL_STATUS_TRY(prepare_spread(P, op, x, ldx, nc, false, scale));
    NFL_STATUS_TRY(mark(P, 1));
    NFL_STATUS_TRY(launch_spread3_warp(P, nc));
    NFL_STATUS_TRY(mark(P, 2));
    NFL_STATUS_TRY(launch_fft(P, nc));
    NFL_STATUS_TRY(mark(P, 3));
    NFL_STATUS_TRY(launch_gather_tc(P, op, x, y, ldy, nc));
    NFL_STATUS_TRY(mark(P, 4, nc));
    return NFL_OK;
}

static nfl_status run_block(Plan &P, int op, const double *x, int64_t ldx, double *y, int64_t ldy, int nc) {
    const nfl_status st = ensure_columns(P, nc);
    if (st != NFL_OK) return st;
    // the launches of this block take the block buffers (kernel arguments are copied at
    // launch, so the one-column pointers are restored right after)
    const BlockBuffers one{P.grid, P.bufA, P.bufB, P.g, P.xsort, P.xsorted};
    P.grid = P.blk.grid; P.bufA = P.blk.bufA; P.bufB = P.blk.bufB; P.g = P.blk.g;
    P.xsort = P.blk.xsort; P.xsorted = P.blk.xsorted;
    const nfl_status rs = run_block_stages(P, op, x, ldx, y, ldy, nc);
    P.grid = one.grid; P.bufA = one.bufA; P.bufB = one.bufB; P.g = one.g;
    P.xsort = one.xsort; P.xsorted = one.xsorted;
    return rs;
}

// The second staging buffers, their stream and events, made once (refused under stream
// capture, which allocation would invalidate: the caller then takes the plain loop).
static bool ensure_pipeline(Plan &P) {
    if (P.pipe_stream) return true;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(P.stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return false;
    if (cudaMalloc(&P.pipe_xsort, P.n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&P.pipe_xsorted, P.n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P.pipe_scratch, 64 * sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.pipe_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.pipe_spread_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.pipe_staged[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.pipe_staged[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&P.pipe_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Several one-column products (3-D, FP32 / FP32C, staged): the staging of column c + 1
// (a DRAM-bound gather of x) runs on the pipeline stream into the other staging buffer
// while column c's FFT passes and interpolation run, the kernels that leave it room on
// the SMs.  Column c waits for its staging; the staging of c + 1 waits for the spread of
// c, after which nothing reads its buffer (columns c - 1 and c + 1 share it).  Cols gives
// each column's device x and y and the hooks of host-buffer products (copies in before
// the staging, the y slot free before the interpolation, the copy out after it).
struct DeviceColumns {
    const double *x;
    int64_t ldx;
    double *y;
    int64_t ldy;
    const double *xc(int c) const { return x + c * ldx; }
    double *yc(int c) const { return y + c * ldy; }
    cudaError_t before_stage(int, cudaStream_t) { return cudaSuccess; }
    cudaError_t before_gather(int, cudaStream_t) { return cudaSuccess; }
    cudaError_t after_column(int, cudaStream_t) { return cudaSuccess; }
};

template <class Cols>
static nfl_status run_columns_pipelined(Plan &P, int op, int nrhs, Cols &cols) {
    const bool scale = (op == OP_A || op == OP_LS);
    const cudaStream_t M = P.stream, S = P.pipe_stream;
    void *const xs[2] = {P.xsort, P.pipe_xsort};
    double *const zs[2] = {P.xsorted, P.pipe_xsorted};
    double *const sc[2] = {P.scratch, P.pipe_scratch};
    // the plan's stream and staging buffers as they were, however the products end
    struct Restore {
        Plan &P;
        cudaStream_t s;
        void *x;
        double *z, *c;
        ~Restore() {
            P.stream = s;
            P.xsort = x;
            P.xsorted = z;
            P.scratch = c;
        }
    } restore{P, M, xs[0], zs[0], sc[0]};
    auto use = [&](int b, cudaStream_t s) {
        P.stream = s;
        P.xsort = xs[b];
        P.xsorted = zs[b];
        P.scratch = sc[b];
    };
    auto stage = [&](int c) -> cudaError_t {
        NFL_CUDA_TRY(cols.before_stage(c, S));
        use(c & 1, S);
        NFL_CUDA_TRY(stage_spread3_values(P, op, cols.xc(c), P.n, 1, false, scale));
        return cudaEventRecord(P.pipe_staged[c & 1], S);
    };
    NFL_STATUS_TRY(cudaEventRecord(P.pipe_fork, M));
    NFL_STATUS_TRY(cudaStreamWaitEvent(S, P.pipe_fork, 0));
    NFL_STATUS_TRY(stage(0));
    for (int c = 0; c < nrhs; ++c) {
        const int b = c & 1;
        use(b, M);
        NFL_STATUS_TRY(cudaStreamWaitEvent(M, P.pipe_staged[b], 0));
        NFL_STATUS_TRY(mark(P, 0));
        NFL_STATUS_TRY(clear_spread(P, 1));
        NFL_STATUS_TRY(mark(P, 1));
        NFL_STATUS_TRY(launch_spread(P, cols.xc(c), 0, false, scale));
        NFL_STATUS_TRY(mark(P, 2));
        if (c + 1 < nrhs) {
            NFL_STATUS_TRY(cudaEventRecord(P.pipe_spread_done, M));
            NFL_STATUS_TRY(cudaStreamWaitEvent(S, P.pipe_spread_done, 0));
            NFL_STATUS_TRY(stage(c + 1));
            use(b, M);
        }
        NFL_STATUS_TRY(launch_fft(P));
        NFL_STATUS_TRY(mark(P, 3));
        NFL_STATUS_TRY(cols.before_gather(c, M));
        NFL_STATUS_TRY(launch_gather(P, op, cols.xc(c), cols.yc(c)));
        NFL_STATUS_TRY(mark(P, 4));
        NFL_STATUS_TRY(cols.after_column(c, M));
    }
    return NFL_OK;
}

static bool pipeline_available(const Plan &P) {
    return P.d == 3 && column_tile_edge(P.m) == P.tile_edge && P.prec != NFL_PREC_FP64;
}

static nfl_status apply(nfl_plan *plan, int op, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs) {
    if (!plan || !x || !y || nrhs < 1) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (ldx < P.n || ldy < P.n) return NFL_ERR_INVALID_ARG;
    if (op != OP_W && !P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    if (nrhs > 1 && P.block_cols > 1 && block_path_available(P)) {
        for (int c = 0; c < nrhs; c += P.block_cols) {
            const int nc = nrhs - c < P.block_cols ? nrhs - c : P.block_cols;
            const nfl_status st = run_block(P, op, x + c * ldx, ldx, y + c * ldy, ldy, nc);
            if (st != NFL_OK) return st;
        }
        return NFL_OK;
    }
    if (nrhs > 1 && pipeline_available(P) && ensure_pipeline(P)) {
        DeviceColumns cols{x, ldx, y, ldy};
        return run_columns_pipelined(P, op, nrhs, cols);
    }
    for (int c = 0; c < nrhs; ++c) {
        nfl_status st = run_column(P, op, x + c * ldx, y + c * ldy);
        if (st != NFL_OK) return st;
    }
    return NFL_OK;
}

// Library streams for batched products, one set per device, made on first use and
// kept for the life of the process (a captured CUDA graph may refer to them).
BatchStreams *batch_streams() {
    static std::mutex mu;
    static BatchStreams pools[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    BatchStreams &b = pools[dev];
    if (b.ready) return &b;
    for (int k = 0; k < kBatchStreams; ++k) {
        if (!b.s[k] && cudaStreamCreateWithFlags(&b.s[k], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (!b.join[k] && cudaEventCreateWithFlags(&b.join[k], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    if (!b.fork && cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    b.ready = true;
    return &b;
}

// Products with host-resident blocks.  Column c goes through device slot
// c mod kHostSlots: copied in on the h2d stream, multiplied on the plan's
// stream, copied out on the d2h stream.  Events order the three streams, so
// column c + 1 travels in and column c - 1 travels out while column c is
// multiplied, and a slot is refilled only after its previous column is done
// with it.
static cudaError_t host_pipeline_init(Plan &P) {
    if (!P.host_stage) NFL_CUDA_TRY(cudaMalloc(&P.host_stage, sizeof(double) * 2 * kHostSlots * (size_t)P.n));
    if (!P.h2d) NFL_CUDA_TRY(cudaStreamCreateWithFlags(&P.h2d, cudaStreamNonBlocking));
    if (!P.d2h) NFL_CUDA_TRY(cudaStreamCreateWithFlags(&P.d2h, cudaStreamNonBlocking));
    if (!P.ev_start) NFL_CUDA_TRY(cudaEventCreateWithFlags(&P.ev_start, cudaEventDisableTiming));
    for (int s = 0; s < kHostSlots; ++s) {
        if (!P.ev_in[s]) NFL_CUDA_TRY(cudaEventCreateWithFlags(&P.ev_in[s], cudaEventDisableTiming));
        if (!P.ev_done[s]) NFL_CUDA_TRY(cudaEventCreateWithFlags(&P.ev_done[s], cudaEventDisableTiming));
        if (!P.ev_out[s]) NFL_CUDA_TRY(cudaEventCreateWithFlags(&P.ev_out[s], cudaEventDisableTiming));
    }
    return cudaSuccess;
}

static cudaError_t issue_host_column(Plan &P, int op, const double *x, double *y, int c, nfl_status &st) {
    const int s = c % kHostSlots;
    const size_t bytes = sizeof(double) * (size_t)P.n;
    double *xs = P.host_stage + (size_t)s * P.n;
    double *ys = P.host_stage + (size_t)(kHostSlots + s) * P.n;
    if (c >= kHostSlots) NFL_CUDA_TRY(cudaStreamWaitEvent(P.h2d, P.ev_done[s], 0));   // slot's x read
    NFL_CUDA_TRY(cudaMemcpyAsync(xs, x, bytes, cudaMemcpyDefault, P.h2d));
    NFL_CUDA_TRY(cudaEventRecord(P.ev_in[s], P.h2d));
    NFL_CUDA_TRY(cudaStreamWaitEvent(P.stream, P.ev_in[s], 0));
    if (c >= kHostSlots) NFL_CUDA_TRY(cudaStreamWaitEvent(P.stream, P.ev_out[s], 0));  // slot's y sent
    st = run_column(P, op, xs, ys);
    if (st != NFL_OK) return cudaSuccess;
    NFL_CUDA_TRY(cudaEventRecord(P.ev_done[s], P.stream));
    NFL_CUDA_TRY(cudaStreamWaitEvent(P.d2h, P.ev_done[s], 0));
    NFL_CUDA_TRY(cudaMemcpyAsync(y, ys, bytes, cudaMemcpyDefault, P.d2h));
    return cudaEventRecord(P.ev_out[s], P.d2h);
}

// The columns of a host-buffer product in the pipelined order: column c's x copied into
// slot c mod kHostSlots before its staging, its y slot free (the copy out of column
// c - kHostSlots done) before its interpolation, its y copied out after it.
struct HostColumns {
    Plan &P;
    const double *x;
    int64_t ldx;
    double *y;
    int64_t ldy;
    const double *xc(int c) const { return P.host_stage + (size_t)(c % kHostSlots) * P.n; }
    double *yc(int c) const { return P.host_stage + (size_t)(kHostSlots + c % kHostSlots) * P.n; }
    cudaError_t before_stage(int c, cudaStream_t S) {
        const int s = c % kHostSlots;
        if (c >= kHostSlots) NFL_CUDA_TRY(cudaStreamWaitEvent(P.h2d, P.ev_done[s], 0));   // slot's x read
        NFL_CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(xc(c)), x + c * ldx, sizeof(double) * (size_t)P.n,
                                     cudaMemcpyDefault, P.h2d));
        NFL_CUDA_TRY(cudaEventRecord(P.ev_in[s], P.h2d));
        return cudaStreamWaitEvent(S, P.ev_in[s], 0);
    }
    cudaError_t before_gather(int c, cudaStream_t M) {
        return c >= kHostSlots ? cudaStreamWaitEvent(M, P.ev_out[c % kHostSlots], 0) : cudaSuccess;
    }
    cudaError_t after_column(int c, cudaStream_t M) {
        const int s = c % kHostSlots;
        NFL_CUDA_TRY(cudaEventRecord(P.ev_done[s], M));
        NFL_CUDA_TRY(cudaStreamWaitEvent(P.d2h, P.ev_done[s], 0));
        NFL_CUDA_TRY(cudaMemcpyAsync(y + c * ldy, yc(c), sizeof(double) * (size_t)P.n, cudaMemcpyDefault, P.d2h));
        return cudaEventRecord(P.ev_out[s], P.d2h);
    }
};

static nfl_status apply_host(nfl_plan *plan, int op, const double *x, int64_t ldx, double *y, int64_t ldy,
                             int nrhs) {
    if (!plan || !x || !y || nrhs < 1 || op < 0 || op > 2) return NFL_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (ldx < P.n || ldy < P.n) return NFL_ERR_INVALID_ARG;
    const int ops[3] = {OP_W, OP_A, OP_LS};
    if (ops[op] != OP_W && !P.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    NFL_STATUS_TRY(host_pipeline_init(P));
    nfl_status st = NFL_OK;
    cudaError_t e = cudaEventRecord(P.ev_start, P.stream);   // copies follow the work queued before
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.h2d, P.ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.d2h, P.ev_start, 0);
    if (e == cudaSuccess && nrhs > 1 && pipeline_available(P) && ensure_pipeline(P)) {
        HostColumns cols{P, x, ldx, y, ldy};
        st = run_columns_pipelined(P, ops[op], nrhs, cols);
    } else {
        for (int c = 0; c < nrhs && e == cudaSuccess && st == NFL_OK; ++c)
            e = issue_host_column(P, ops[op], x + c * ldx, y + c * ldy, c, st);
    }
    // wait for everything issued, also after an error: y is final and x free on return
    const cudaError_t e1 = cudaStreamSynchronize(P.h2d);
    const cudaError_t e2 = cudaStreamSynchronize(P.stream);
    const cudaError_t e3 = cudaStreamSynchronize(P.d2h);
    if (st != NFL_OK) return st;
    for (cudaError_t ei : {e, e1, e2, e3})
        if (ei != cudaSuccess) return ei == cudaErrorMemoryAllocation ? NFL_ERR_OUT_OF_MEMORY : NFL_ERR_CUDA;
    return NFL_OK;
}

}  // namespace nfl

extern "C" {

nfl_status nfl_apply_host(nfl_plan *plan, int op, const double *x, int64_t ldx, double *y, int64_t ldy,
                          int nrhs) {
    return nfl::apply_host(plan, op, x, ldx, y, ldy, nrhs);
}

nfl_status nfl_apply_W(nfl_plan *plan, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs) {
    return nfl::apply(plan, nfl::OP_W, x, ldx, y, ldy, nrhs);
}

nfl_status nfl_apply_A(nfl_plan *plan, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs) {
    return nfl::apply(plan, nfl::OP_A, x, ldx, y, ldy, nrhs);
}

nfl_status nfl_apply_Ls(nfl_plan *plan, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs) {
    return nfl::apply(plan, nfl::OP_LS, x, ldx, y, ldy, nrhs);
}

nfl_status nfl_apply_batched(nfl_plan *const *plans, int G, int op, const double *const *x, double *const *y,
                             const int64_t *ld, int nrhs) {
    if (!plans || !x || !y || !ld || G < 0 || op < 0 || op > 2) return NFL_ERR_INVALID_ARG;
    if (G == 0) return NFL_OK;
    for (int g = 0; g < G; ++g)
        if (!plans[g]) return NFL_ERR_INVALID_ARG;
    nfl::BatchStreams *pool = nfl::batch_streams();
    if (!pool) return NFL_ERR_CUDA;
    const cudaStream_t origin = reinterpret_cast<nfl::Plan *>(plans[0])->stream;
    const int K = G < nfl::kBatchStreams ? G : nfl::kBatchStreams;
    // plans to streams, largest first to the least loaded (longest-processing-time order)
    std::vector<int> order(G), lane(G);
    std::vector<int64_t> load(K, 0);
    for (int g = 0; g < G; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return reinterpret_cast<nfl::Plan *>(plans[a])->n > reinterpret_cast<nfl::Plan *>(plans[b])->n;
    });
    for (int g : order) {
        const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
        lane[g] = k;
        load[k] += reinterpret_cast<nfl::Plan *>(plans[g])->n;
    }
    // fork from the origin stream, issue, join back (also after an error, so that the
    // origin stream is ordered after everything issued)
    if (cudaEventRecord(pool->fork, origin) != cudaSuccess) return NFL_ERR_CUDA;
    for (int k = 0; k < K; ++k)
        if (cudaStreamWaitEvent(pool->s[k], pool->fork, 0) != cudaSuccess) return NFL_ERR_CUDA;
    const int ops[3] = {nfl::OP_W, nfl::OP_A, nfl::OP_LS};
    nfl_status st = NFL_OK;
    for (int g = 0; g < G && st == NFL_OK; ++g) {
        nfl::Plan &P = *reinterpret_cast<nfl::Plan *>(plans[g]);
        P.stream = pool->s[lane[g]];
        st = nfl::apply(plans[g], ops[op], x[g], ld[g], y[g], ld[g], nrhs);
    }
    for (int k = 0; k < K; ++k) {
        if (cudaEventRecord(pool->join[k], pool->s[k]) != cudaSuccess ||
            cudaStreamWaitEvent(origin, pool->join[k], 0) != cudaSuccess)
            return NFL_ERR_CUDA;
    }
    for (int g = 0; g < G; ++g) reinterpret_cast<nfl::Plan *>(plans[g])->stream = origin;
    return st;
}

nfl_status nfl_plan_autotune(nfl_plan *plan, double *best_ms) {
    if (!plan) return NFL_ERR_INVALID_ARG;
    nfl::Plan &P = *reinterpret_cast<nfl::Plan *>(plan);
    const int64_t n = P.n;
    double *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release = [&]() {
        cudaFree(x);
        cudaFree(y);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&x, n * 8) != cudaSuccess || cudaMalloc(&y, n * 8) != cudaSuccess) {
        release();
        return NFL_ERR_OUT_OF_MEMORY;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        release();
        return NFL_ERR_CUDA;
    }
    nfl_status st = NFL_OK;
    // x = 1 (the degree product's input), on the plan's stream
    {
        const double one = 1.0;
        std::vector<double> h(std::min<int64_t>(n, 1 << 20), one);
        for (int64_t o = 0; o < n && st == NFL_OK; o += (int64_t)h.size()) {
            const int64_t c = std::min<int64_t>((int64_t)h.size(), n - o);
            if (cudaMemcpyAsync(x + o, h.data(), c * 8, cudaMemcpyHostToDevice, P.stream) != cudaSuccess ||
                cudaStreamSynchronize(P.stream) != cudaSuccess)
                st = NFL_ERR_CUDA;
        }
    }
    const bool prof = P.profile;
    P.profile = false;
    // fastest of five timed products after one untimed one
    auto time_config = [&](double &ms) -> nfl_status {
        float best = 1e30f;
        for (int r = 0; r < 6; ++r) {
            if (cudaEventRecord(e0, P.stream) != cudaSuccess) return NFL_ERR_CUDA;
            const nfl_status rs = nfl::run_column(P, nfl::OP_W, x, y);
            if (rs != NFL_OK) return rs;
            if (cudaEventRecord(e1, P.stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return NFL_ERR_CUDA;
            float t = 0.f;
            if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return NFL_ERR_CUDA;
            if (r > 0 && t < best) best = t;
        }
        ms = best;
        return NFL_OK;
    };
    // One parameter: the current value is timed first and a candidate replaces it only
    // when at least 2 % faster (run-to-run differences are about 1 %).  set(v) applies
    // value v (rebuilding whatever depends on it).
    double best = 1e30;
    auto tune = [&](int &param, const int *cand, int ncand, auto set) -> nfl_status {
        const int start = param;
        int keep = start;
        nfl_status rs = set(start);
        double ms = 0.0;
        if (rs == NFL_OK) rs = time_config(ms);
        if (rs != NFL_OK) return rs;
        best = ms;
        for (int c = 0; c < ncand; ++c) {
            if (cand[c] == start) continue;
            rs = set(cand[c]);
            if (rs == NFL_OK) rs = time_config(ms);
            if (rs != NFL_OK) break;
            if (ms < 0.98 * best) {
                best = ms;
                keep = cand[c];
            }
        }
        const nfl_status fin = set(keep);
        return rs != NFL_OK ? rs : fin;
    };
    if (st == NFL_OK) {
        const int caps[4] = {256, 512, 1024, 2048};
        st = tune(P.fft_cap, caps, 4, [&](int v) { P.fft_cap = v; return NFL_OK; });
    }
    if (st == NFL_OK && P.d == 3) {
        // work-item size: chunks of at most 2048, 4096 or 8192 nodes
        const int chunks[3] = {2048, 4096, 8192};
        int cur = P.chunk;
        st = tune(cur, chunks, 3, [&](int v) { return nfl::rechunk_items(P, v); });
    }
    if (st == NFL_OK && nfl::moments_available(P)) {
        // nodes per occupied cell from which a tile goes to the moment kernels
        const int dens[3] = {16, 32, 64};
        st = tune(P.dense_cell, dens, 3, [&](int v) {
            P.dense_cell = v;
            return nfl::rebuild_spread_items(P);
        });
        // most nodes per slab piece of the moment spread
        const int dch[3] = {2048, 4096, 8192};
        if (st == NFL_OK)
            st = tune(P.dense_chunk, dch, 3, [&](int v) {
                P.dense_chunk = v;
                return nfl::rebuild_spread_items(P);
            });
    }
    if (st == NFL_OK && nfl::spread_warp_available(P)) {
        const int runs[4] = {1, 4, 8, 16};
        st = tune(P.slide_tiles, runs, 4, [&](int v) {
            P.slide_tiles = v;
            return nfl::rebuild_spread_items(P);
        });
    }
    P.profile = prof;
    if (st == NFL_OK && best_ms) *best_ms = best;
    if (cudaStreamSynchronize(P.stream) != cudaSuccess && st == NFL_OK) st = NFL_ERR_CUDA;
    release();
    return st;
}

nfl_status nfl_plan_set_profiling(nfl_plan *plan, int enable) {
    if (!plan) return NFL_ERR_INVALID_ARG;
    nfl::Plan &P = *reinterpret_cast<nfl::Plan *>(plan);
    P.profile = enable != 0;
    P.events_used = 0;
    P.event_cols.clear();
    return NFL_OK;
}

nfl_status nfl_plan_stage_times(nfl_plan *plan, double *ms, int64_t *columns) {
    if (!plan || !ms) return NFL_ERR_INVALID_ARG;
    nfl::Plan &P = *reinterpret_cast<nfl::Plan *>(plan);
    if (cudaStreamSynchronize(P.stream) != cudaSuccess) return NFL_ERR_CUDA;
    for (int s = 0; s < 4; ++s) ms[s] = 0.0;
    const size_t sets = P.events_used / 5;
    int64_t cols = 0;
    for (size_t c = 0; c < sets; ++c) {
        for (int s = 0; s < 4; ++s) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, P.events[5 * c + s], P.events[5 * c + s + 1]) != cudaSuccess)
                return NFL_ERR_CUDA;
            ms[s] += t;
        }
        cols += c < P.event_cols.size() ? P.event_cols[c] : 1;
    }
    if (columns) *columns = cols;
    P.events_used = 0;
    P.event_cols.clear();
    return NFL_OK;
}

nfl_status nfl_plan_kernels(const nfl_plan *plan, int nrhs, int *kernels) {
    if (!plan || !kernels || nrhs < 1) return NFL_ERR_INVALID_ARG;
    const nfl::Plan &P = *reinterpret_cast<const nfl::Plan *>(plan);
    if (nrhs > 1 && P.block_cols > 1 && nfl::block_path_available(P)) {
        const int blocks = (nrhs + P.block_cols - 1) / P.block_cols;
        // one launch per stage and block (a block spreads and interpolates every tile with
        // the warp-slice and tensor-core kernels)
        const bool split = nfl::moments_available(P) && P.nslab > 0;
        const int spreads = nfl::moments_available(P) ? (P.nsparse > 0 ? 1 : 0) + (P.nslab > 0 ? 1 : 0) : 1;
        const int gathers = split && nfl::gather_tc_available(P) ? 2 : 1;
        *kernels = blocks * (nfl::kernels_per_column(P) - spreads + 1 - gathers + 1);
    } else {
        *kernels = nrhs * nfl::kernels_per_column(P);
    }
    return NFL_OK;
}

nfl_status nfl_plan_kernels_per_column(const nfl_plan *plan, int *kernels) {
    if (!plan || !kernels) return NFL_ERR_INVALID_ARG;
    *kernels = nfl::kernels_per_column(*reinterpret_cast<const nfl::Plan *>(plan));
    return NFL_OK;
}

}  // extern "C"
