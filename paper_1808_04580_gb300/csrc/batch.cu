// Products of many graphs with one launch per stage (Alg. 1 with the Alg. 2 step 5
// scalings, for a batch of plans): staging, spread, the five FFT passes and the
// interpolation each run once over every member's (work item, column) pairs.
//
// A batch binds its members' plans, the caller's input and output blocks and its
// own contiguous buffers (staged values, spreading and interpolation grids, FFT
// intermediates for every member and column), so a run is a fixed sequence of
// two memsets and eight kernel launches on one stream: nothing is allocated and
// the host is not synchronized, and a run can be captured into a CUDA graph.
// The spread and the interpolation take their work from one list of all members'
// items, largest first, through one counter each; the FFT passes and the staging
// map each CTA to its member by a binary search over per-member CTA offsets.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.h"

namespace nfl {

// The warp spread's and the interpolation's item lists of a member, as the plan
// holds them on the device (both built on the host from the per-tile chunks).
static std::vector<WorkItem> gather_item_list(const Plan &P) {
    std::vector<WorkItem> h = P.tile_items;
    std::stable_sort(h.begin(), h.end(), [](const WorkItem &x, const WorkItem &y) { return x.count > y.count; });
    return h;
}

static void free_batch(Batch *B) {
    if (!B) return;
    for (cudaEvent_t e : B->events) cudaEventDestroy(e);
    cudaFree(B->desc);
    cudaFree(B->sitems);
    cudaFree(B->gitems);
    cudaFree(B->stage_start);
    cudaFree(B->counter);
    cudaFree(B->grid_all);
    cudaFree(B->abs_all);
    cudaFree(B->xs_all);
    cudaFree(B->zd_all);
    cudaFree(B->g_all);
    cudaFree(B->bufA_all);
    cudaFree(B->bufB_all);
    for (int i = 0; i < 5; ++i) {
        cudaFree(B->pass_args[i]);
        cudaFree(B->pass_start[i]);
    }
    delete B;
}

// Checks that every member can take part: 3-D, the same mixed precision, m and N,
// the warp-spread / tensor-core path, positive degrees unless op is W.
static nfl_status check_members(const Plan *const *P, int G, int op) {
    const Plan &F = *P[0];
    for (int g = 0; g < G; ++g) {
        const Plan &Q = *P[g];
        for (int h = 0; h < g; ++h)
            if (P[h] == P[g]) return NFL_ERR_INVALID_ARG;
        if (Q.d != 3 || Q.prec == NFL_PREC_FP64 || Q.prec != F.prec || Q.bf16_taps != F.bf16_taps || Q.m != F.m ||
            Q.N != F.N || !block_path_available(Q))
            return NFL_ERR_INVALID_ARG;
        if (op != OP_W && !Q.degree_ok) return NFL_ERR_NONPOSITIVE_DEGREE;
    }
    return NFL_OK;
}

// stage events of a timed run: 0 before the memsets and staging, 1 before the spread,
// 2 before the FFT, 3 before the interpolation, 4 after it
static cudaError_t mark(Batch &B, int stage, cudaStream_t s) {
    if (!B.profile) return cudaSuccess;
    const size_t idx = B.events_used + stage;
    while (B.events.size() <= idx) {
        cudaEvent_t e;
        NFL_CUDA_TRY(cudaEventCreate(&e));
        B.events.push_back(e);
    }
    NFL_CUDA_TRY(cudaEventRecord(B.events[idx], s));
    if (stage == 4) B.events_used += 5;
    return cudaSuccess;
}

template <typename T>
static cudaError_t upload(T *&dst, const std::vector<T> &src) {
    NFL_CUDA_TRY(cudaMalloc(&dst, std::max<size_t>(src.size(), 1) * sizeof(T)));
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// One part of a batch: the members mem[j] of the caller's arrays, with their own
// descriptors, item lists and buffers; its runs are eight launches on one stream.
static nfl_status create_part(const std::vector<const Plan *> &PA, const std::vector<int> &mem, int opi,
                              const double *const *xa, const int64_t *ldxa, double *const *ya, const int64_t *ldya,
                              int nrhs, Batch **out) {
    const int G = (int)mem.size();
    std::vector<const Plan *> P(G);
    std::vector<const double *> x(G);
    std::vector<double *> y(G);
    std::vector<int64_t> ldx(G), ldy(G);
    for (int j = 0; j < G; ++j) {
        P[j] = PA[mem[j]];
        x[j] = xa[mem[j]];
        y[j] = ya[mem[j]];
        ldx[j] = ldxa[mem[j]];
        ldy[j] = ldya[mem[j]];
    }
    Batch *B = new (std::nothrow) Batch();
    if (!B) return NFL_ERR_OUT_OF_MEMORY;
    const Plan &F = *P[0];
    B->G = G;
    B->op = opi;
    B->ncol = nrhs;
    B->m = F.m;
    B->N = F.N;
    B->prec = F.prec;
    B->bf16 = F.bf16_taps;
    B->num_sms = F.num_sms;
    B->fft_cap = F.fft_cap;
    for (int j = 0; j < 2 * kMaxM; ++j)
        for (int k = 0; k < kPolyCoef; ++k) B->poly[j][k] = F.kb_poly[j][k];
    for (int g = 0; g < G; ++g) B->plans.push_back(const_cast<Plan *>(P[g]));
    const int64_t nc = nrhs;
    const size_t grid_sz = F.prec == NFL_PREC_FP32 ? 4 : 8;
    // contiguous buffers: element offsets of each member
    std::vector<int64_t> on(G + 1, 0), ob(G + 1, 0), oa(G + 1, 0), obb(G + 1, 0);
    for (int g = 0; g < G; ++g) {
        on[g + 1] = on[g] + P[g]->n * nc;
        ob[g + 1] = ob[g] + P[g]->box_elems * nc;
        oa[g + 1] = oa[g] + P[g]->bufA_elems * nc;
        obb[g + 1] = obb[g] + P[g]->bufB_elems * nc;
    }
    B->grid_bytes = (size_t)ob[G] * grid_sz;
    auto fail = [&](nfl_status s) {
        free_batch(B);
        return s;
    };
    if (cudaMalloc(&B->grid_all, B->grid_bytes) != cudaSuccess ||
        cudaMalloc(&B->abs_all, (size_t)G * nc * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&B->xs_all, (size_t)on[G] * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&B->zd_all, (size_t)on[G] * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&B->g_all, (size_t)ob[G] * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&B->bufA_all, (size_t)oa[G] * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&B->bufB_all, (size_t)obb[G] * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&B->counter, 2 * sizeof(unsigned)) != cudaSuccess)
        return fail(NFL_ERR_OUT_OF_MEMORY);
    // member descriptors, item lists, staging and FFT CTA offsets
    std::vector<BatchPlanDev> desc(G);
    std::vector<BatchItem> sitems, gitems;
    std::vector<int> sc_s, sc_g;   // item sizes for the ordering
    std::vector<int64_t> stage_start(G + 1, 0);
    std::vector<PassArgs> pass(5 * (size_t)G);
    std::vector<int64_t> pass_start(5 * (size_t)(G + 1), 0);
    for (int g = 0; g < G; ++g) {
        const Plan &Q = *P[g];
        BatchPlanDev &D = desc[g];
        D.pts = reinterpret_cast<const PointF *>(Q.pts);
        D.perm = Q.perm;
        D.dinv = Q.dinv_sorted;
        D.tile_start = Q.tile_start;
        D.items = Q.items;
        D.sitems = Q.sitems;
        D.x = x[g];
        D.y = y[g];
        D.ldx = ldx[g];
        D.ldy = ldy[g];
        D.xs = static_cast<float *>(B->xs_all) + on[g];
        D.zd = static_cast<double *>(B->zd_all) + on[g];
        D.grid = static_cast<unsigned char *>(B->grid_all) + ob[g] * grid_sz;
        D.g = static_cast<float *>(B->g_all) + ob[g];
        D.abs_sum = B->abs_all + (size_t)g * nc;
        D.n = Q.n;
        D.box = Q.box_elems;
        for (int i = 0; i < 3; ++i) {
            D.ntile[i] = Q.ntile[i];
            D.L[i] = Q.L[i];
            D.wrap[i] = Q.wrap[i];
        }
        D.k0 = Q.k0;
        D.out_scale = Q.out_scale;
        D.error_flag = Q.error_flag;
        const std::vector<WorkItem> si = spread_item_list(Q), gi = gather_item_list(Q);
        if ((int64_t)si.size() != Q.nsitems || (int64_t)gi.size() != Q.nitems) return fail(NFL_ERR_INVALID_ARG);
        for (size_t i = 0; i < si.size(); ++i) {
            sitems.push_back(BatchItem{g, (int32_t)i});
            sc_s.push_back(si[i].count);
        }
        for (size_t i = 0; i < gi.size(); ++i) {
            gitems.push_back(BatchItem{g, (int32_t)i});
            sc_g.push_back(gi[i].count);
        }
        // staging: about 2048 nodes per CTA
        stage_start[g + 1] = stage_start[g] + std::max<int64_t>(1, (Q.n + 2047) / 2048);
        PassArgs f[5];
        int ctas[5];
        fft_passes_3d(Q, D.grid, static_cast<float2 *>(B->bufA_all) + oa[g], static_cast<float2 *>(B->bufB_all) + obb[g],
                      D.g, Q.bufA_elems, Q.bufB_elems, B->fft_cap, f, nrhs, ctas);
        f[0].abs_sum = D.abs_sum;
        for (int i = 0; i < 5; ++i) {
            pass[(size_t)i * G + g] = f[i];
            pass_start[(size_t)i * (G + 1) + g + 1] = pass_start[(size_t)i * (G + 1) + g] + ctas[i];
        }
    }
    // all members' items, largest first (stable: member order, then the member's order)
    auto by_size = [](const std::vector<BatchItem> &v, const std::vector<int> &cnt) {
        std::vector<size_t> idx(v.size());
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return cnt[a] > cnt[b]; });
        std::vector<BatchItem> out(v.size());
        for (size_t i = 0; i < idx.size(); ++i) out[i] = v[idx[i]];
        return out;
    };
    sitems = by_size(sitems, sc_s);
    gitems = by_size(gitems, sc_g);
    B->nsitems = (int64_t)sitems.size();
    B->ngitems = (int64_t)gitems.size();
    int64_t most_ctas = stage_start[G];
    for (int i = 0; i < 5; ++i) most_ctas = std::max<int64_t>(most_ctas, pass_start[(size_t)i * (G + 1) + G]);
    if (most_ctas > 0x7fffffff || B->nsitems * nc > 0xffffffffll || B->ngitems * nc > 0xffffffffll)
        return fail(NFL_ERR_INVALID_ARG);
    B->stage_ctas = (int)stage_start[G];
    const std::vector<int> ss(stage_start.begin(), stage_start.end());
    bool ok = upload(B->desc, desc) == cudaSuccess && upload(B->sitems, sitems) == cudaSuccess &&
              upload(B->gitems, gitems) == cudaSuccess && upload(B->stage_start, ss) == cudaSuccess;
    for (int i = 0; i < 5 && ok; ++i) {
        std::vector<PassArgs> pi(pass.begin() + (size_t)i * G, pass.begin() + (size_t)(i + 1) * G);
        std::vector<int> si(pass_start.begin() + (size_t)i * (G + 1), pass_start.begin() + (size_t)(i + 1) * (G + 1));
        B->pass_ctas[i] = si[G];
        ok = upload(B->pass_args[i], pi) == cudaSuccess && upload(B->pass_start[i], si) == cudaSuccess;
    }
    if (!ok) return fail(NFL_ERR_CUDA);
    *out = B;
    return NFL_OK;
}

static nfl_status run_part(Batch &B, cudaStream_t s) {
    B.last_stream = s;
    NFL_STATUS_TRY(mark(B, 0, s));
    NFL_STATUS_TRY(cudaMemsetAsync(B.grid_all, 0, B.grid_bytes, s));
    NFL_STATUS_TRY(cudaMemsetAsync(B.counter, 0, 2 * sizeof(unsigned), s));
    if (B.prec == NFL_PREC_FP32C) NFL_STATUS_TRY(cudaMemsetAsync(B.abs_all, 0, (size_t)B.G * B.ncol * sizeof(double), s));
    NFL_STATUS_TRY(launch_stage_batch(B, s));
    NFL_STATUS_TRY(mark(B, 1, s));
    NFL_STATUS_TRY(launch_spread3_warp_batch(B, s));
    NFL_STATUS_TRY(mark(B, 2, s));
    NFL_STATUS_TRY(launch_fft_batch(B, s));
    NFL_STATUS_TRY(mark(B, 3, s));
    NFL_STATUS_TRY(launch_gather_tc_batch(B, s));
    NFL_STATUS_TRY(mark(B, 4, s));
    return NFL_OK;
}

// The public batch: parts that run concurrently on library streams forked from the
// caller's stream and joined back.
struct BatchGroup {
    std::vector<Batch *> parts;
};

static void free_group(BatchGroup *H) {
    if (!H) return;
    for (Batch *B : H->parts) free_batch(B);
    delete H;
}

// Estimated time of a member's product per column (ns): the spread and the
// interpolation scale with the window taps per node, the FFT passes with the box
// (relative weights measured on GB300 at N = 64, m = 4).
static double member_cost(const Plan &P) {
    const double taps = std::pow(2.0 * P.m, 3);
    return double(P.n) * taps / 512.0 * 0.17 + double(P.box_elems) * 0.066;
}

}  // namespace nfl

using nfl::BatchGroup;

extern "C" {

nfl_status nfl_batch_create(nfl_plan *const *plans, int G, int op, const double *const *x, const int64_t *ldx,
                            double *const *y, const int64_t *ldy, int nrhs, int parts, nfl_batch **out) {
    using namespace nfl;
    if (!out) return NFL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || !x || !y || !ldx || !ldy || G < 1 || op < 0 || op > 2 || nrhs < 1 || nrhs > 65535 || parts < 1 ||
        parts > 8)
        return NFL_ERR_INVALID_ARG;
    std::vector<const Plan *> P(G);
    for (int g = 0; g < G; ++g) {
        if (!plans[g] || !x[g] || !y[g]) return NFL_ERR_INVALID_ARG;
        P[g] = reinterpret_cast<const Plan *>(plans[g]);
        if (ldx[g] < P[g]->n || ldy[g] < P[g]->n) return NFL_ERR_INVALID_ARG;
    }
    const int ops[3] = {OP_W, OP_A, OP_LS};
    nfl_status st = check_members(P.data(), G, ops[op]);
    if (st != NFL_OK) return st;
    if (parts > G) parts = G;
    if (parts > 1 && !batch_streams()) return NFL_ERR_CUDA;
    // members to parts, most expensive first to the least loaded
    std::vector<int> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return member_cost(*P[a]) > member_cost(*P[b]); });
    std::vector<std::vector<int>> mem(parts);
    std::vector<double> load(parts, 0.0);
    for (int g : order) {
        const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
        mem[k].push_back(g);
        load[k] += member_cost(*P[g]);
    }
    BatchGroup *H = new (std::nothrow) BatchGroup();
    if (!H) return NFL_ERR_OUT_OF_MEMORY;
    for (int k = 0; k < parts; ++k) {
        std::sort(mem[k].begin(), mem[k].end());
        Batch *B = nullptr;
        st = create_part(P, mem[k], ops[op], x, ldx, y, ldy, nrhs, &B);
        if (st != NFL_OK) {
            free_group(H);
            return st;
        }
        H->parts.push_back(B);
    }
    *out = reinterpret_cast<nfl_batch *>(H);
    return NFL_OK;
}

nfl_status nfl_batch_run(nfl_batch *batch, void *stream) {
    using namespace nfl;
    if (!batch) return NFL_ERR_INVALID_ARG;
    BatchGroup &H = *reinterpret_cast<BatchGroup *>(batch);
    const cudaStream_t origin = (cudaStream_t)stream;
    const int K = (int)H.parts.size();
    if (K == 1) return run_part(*H.parts[0], origin);
    BatchStreams *pool = batch_streams();
    if (!pool) return NFL_ERR_CUDA;
    NFL_STATUS_TRY(cudaEventRecord(pool->fork, origin));
    nfl_status st = NFL_OK;
    for (int k = 0; k < K; ++k) {
        NFL_STATUS_TRY(cudaStreamWaitEvent(pool->s[k], pool->fork, 0));
        if (st == NFL_OK) st = run_part(*H.parts[k], pool->s[k]);
    }
    // join back, also after an error, so that the caller's stream follows everything issued
    for (int k = 0; k < K; ++k) {
        NFL_STATUS_TRY(cudaEventRecord(pool->join[k], pool->s[k]));
        NFL_STATUS_TRY(cudaStreamWaitEvent(origin, pool->join[k], 0));
    }
    return st;
}

nfl_status nfl_batch_set_profiling(nfl_batch *batch, int enable) {
    using namespace nfl;
    if (!batch) return NFL_ERR_INVALID_ARG;
    for (Batch *B : reinterpret_cast<BatchGroup *>(batch)->parts) {
        B->profile = enable != 0;
        B->events_used = 0;
    }
    return NFL_OK;
}

nfl_status nfl_batch_stage_times(nfl_batch *batch, double *ms, int64_t *runs) {
    using namespace nfl;
    if (!batch || !ms) return NFL_ERR_INVALID_ARG;
    for (int s = 0; s < 4; ++s) ms[s] = 0.0;
    int64_t nr = 0;
    for (Batch *Bp : reinterpret_cast<BatchGroup *>(batch)->parts) {
        Batch &B = *Bp;
        if (B.events_used > 0 && cudaStreamSynchronize(B.last_stream) != cudaSuccess) return NFL_ERR_CUDA;
        const size_t sets = B.events_used / 5;
        for (size_t c = 0; c < sets; ++c)
            for (int s = 0; s < 4; ++s) {
                float t = 0.f;
                if (cudaEventElapsedTime(&t, B.events[5 * c + s], B.events[5 * c + s + 1]) != cudaSuccess)
                    return NFL_ERR_CUDA;
                ms[s] += t;
            }
        nr = std::max<int64_t>(nr, (int64_t)sets);
        B.events_used = 0;
    }
    if (runs) *runs = nr;
    return NFL_OK;
}

nfl_status nfl_batch_parts(const nfl_batch *batch, int *parts) {
    if (!batch || !parts) return NFL_ERR_INVALID_ARG;
    *parts = (int)reinterpret_cast<const BatchGroup *>(batch)->parts.size();
    return NFL_OK;
}

void nfl_batch_destroy(nfl_batch *batch) {
    if (!batch) return;
    cudaDeviceSynchronize();
    nfl::free_group(reinterpret_cast<BatchGroup *>(batch));
}

}  // extern "C"
