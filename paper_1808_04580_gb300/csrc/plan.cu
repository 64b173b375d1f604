// Plan creation: Alg. 2 steps 1-4 (Sec. 3.1) on the device.
//   step 1  shift by the bounding-box midpoint c, scale by
//           rho = (1/4 - eps_B/2) / max_j ||v_j - c||                    (Sec. 3)
//   step 2  sigma~ = rho sigma
//   step 3  b_l = N^{-d} sum_{j in I_N} K_R(j/N) e^{-2 pi i j.l/N}       (Sec. 3, eq. (b_l::K_RF))
//   step 4  d_E = W~_E 1 - K(0) 1, D_E^{-1/2}
// plus the layout work of the fast path: each node's base cell and
// fractional offsets on the oversampled grid, a counting sort of the nodes
// into tiles, and the list of tile chunks the spread/gather grids walk.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace nfl {

static constexpr int kChunk = 8192;  // nodes per work item

// ---------------------------------------------------------------- reductions
__global__ void bbox_partials(const double *v, int64_t n, int d, double *part) {
    __shared__ double lo[3][256], hi[3][256];
    double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;   // fmin/fmax drop NaNs, so non-finite input is tracked separately
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < d; ++a) {
            const double x = v[i * d + a];
            l[a] = fmin(l[a], x);
            h[a] = fmax(h[a], x);
            bad = bad || !isfinite(x);
        }
    for (int a = 0; a < 3; ++a) {
        lo[a][threadIdx.x] = bad ? NAN : l[a];
        hi[a][threadIdx.x] = bad ? NAN : h[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                const double l1 = lo[a][threadIdx.x], l2 = lo[a][threadIdx.x + s];
                const double h1 = hi[a][threadIdx.x], h2 = hi[a][threadIdx.x + s];
                lo[a][threadIdx.x] = (l1 != l1 || l2 != l2) ? NAN : fmin(l1, l2);
                hi[a][threadIdx.x] = (h1 != h1 || h2 != h2) ? NAN : fmax(h1, h2);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) { part[blockIdx.x * 6 + a] = lo[a][0]; part[blockIdx.x * 6 + 3 + a] = hi[a][0]; }
}

__global__ void radius_partials(const double *v, int64_t n, int d, double c0, double c1, double c2, double *part) {
    __shared__ double red[256];
    const double c[3] = {c0, c1, c2};
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
            const double t = v[i * d + a] - c[a];
            r2 += t * t;
        }
        mx = fmax(mx, r2);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void minmax_partials(const double *x, int64_t n, double *part) {
    __shared__ double lo[256], hi[256];
    double l = INFINITY, h = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = x[i];
        if (t != t) { l = -INFINITY; h = INFINITY; }  // NaN degree: report as failure
        l = fmin(l, t);
        h = fmax(h, t);
    }
    lo[threadIdx.x] = l;
    hi[threadIdx.x] = h;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            lo[threadIdx.x] = fmin(lo[threadIdx.x], lo[threadIdx.x + s]);
            hi[threadIdx.x] = fmax(hi[threadIdx.x], hi[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = lo[0]; part[2 * blockIdx.x + 1] = hi[0]; }
}

// ------------------------------------------------------- node layout / sort
struct Geometry {
    int d;
    double c[3];
    double rho;
    double ngrid;
    int64_t t0[3];
    int tile_edge;
    int ntile[3];
};

__device__ __forceinline__ void node_cell(const double *v, int64_t i, const Geometry &G, int *cell, double *frac) {
    for (int a = 0; a < G.d; ++a) {
        const double u = G.ngrid * (G.rho * (v[i * G.d + a] - G.c[a]));
        const double base = floor(u);
        frac[a] = u - base;
        cell[a] = (int)((int64_t)base - G.t0[a]);
    }
}

__device__ __forceinline__ int tile_of(const int *cell, const Geometry &G) {
    int t = 0;
    for (int a = 0; a < G.d; ++a) t = t * G.ntile[a] + cell[a] / G.tile_edge;
    return t;
}

// Sort key of a node: its tile, then (when cells_per_tile > 1) its cell inside
// the tile, so that the nodes of one cell are contiguous.
__global__ void count_keys(const double *v, int64_t n, Geometry G, int cells_per_tile, int32_t *key_of,
                           int32_t *rank, int32_t *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int cell[3];
        double frac[3];
        node_cell(v, i, G, cell, frac);
        // cell inside the tile; in 3-D ordered (axis 0, axis 2, axis 1) so that the
        // cells of one (axis 0, axis 2) column of the tile are contiguous
        int local = 0;
        if (cells_per_tile > 1) {
            if (G.d == 3) {
                const int te = G.tile_edge;
                local = ((cell[0] % te) * te + cell[2] % te) * te + cell[1] % te;
            } else {
                for (int a = 0; a < G.d; ++a) local = local * G.tile_edge + cell[a] % G.tile_edge;
            }
        }
        const int key = tile_of(cell, G) * cells_per_tile + local;
        key_of[i] = key;
        rank[i] = atomicAdd(&count[key], 1);
    }
}

// Per-tile node counts and starts from the per-key offsets.
__global__ void tiles_from_keys(const int64_t *kstart, int64_t ntiles, int cells_per_tile, int32_t *count,
                                int64_t *start) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        start[t] = kstart[t * cells_per_tile];
        count[t] = (int32_t)(kstart[(t + 1) * cells_per_tile] - kstart[t * cells_per_tile]);
    }
}

template <typename PT, typename T>
__global__ void scatter_nodes(const double *v, int64_t n, Geometry G, const int32_t *key_of, const int32_t *rank,
                              const int64_t *start, PT *pts, int32_t *perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int cell[3] = {0, 0, 0};
        double frac[3] = {0, 0, 0};
        node_cell(v, i, G, cell, frac);
        const int64_t pos = start[key_of[i]] + rank[i];
        PT p;
        for (int a = 0; a < 3; ++a) p.f[a] = T(a < G.d ? frac[a] : 0.0);
        p.cell = cell[0] | (cell[1] << 10) | (cell[2] << 20);
        pts[pos] = p;
        perm[pos] = (int32_t)i;
    }
}

// Single-block exclusive scan of 32-bit counts into 64-bit offsets; out[n] = total.
__global__ void exclusive_scan(const int32_t *in, int64_t n, int64_t *out) {
    __shared__ int64_t part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per, hi = min(n, lo + per);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int64_t v = part[t];
            part[t] = acc;
            acc += v;
        }
        out[n] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        out[i] = acc;
        acc += in[i];
    }
}

// First sorted node of every tile (and n at index ntiles), from the per-key offsets.
__global__ void tile_starts(const int64_t *kstart, int64_t ntiles, int cells_per_tile, int32_t *out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= ntiles; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (int32_t)kstart[t * cells_per_tile];
}

// Occupied cells of every tile and the nodes of each of its te slabs (the cells that
// share one axis-0 position: te^2 consecutive keys), from the per-key (tile, cell)
// offsets; out holds te + 1 entries per tile.
__global__ void occupied_cells(const int64_t *kstart, int64_t ntiles, int cells_per_tile, int te, int32_t *out) {
    const int per_slab = cells_per_tile / te;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        for (int k = 0; k < cells_per_tile; ++k)
            c += kstart[t * cells_per_tile + k + 1] > kstart[t * cells_per_tile + k] ? 1 : 0;
        out[t * (te + 1)] = c;
        for (int s = 0; s < te; ++s)
            out[t * (te + 1) + 1 + s] = (int32_t)(kstart[t * cells_per_tile + (s + 1) * per_slab] -
                                                  kstart[t * cells_per_tile + s * per_slab]);
    }
}

// Work items of the warp-slice spread from the per-tile chunks (in tile order): a tile
// with several chunks keeps them as items of one tile; runs of single-chunk tiles that
// follow each other along axis 2 in one row are joined while they hold at most `chunk`
// nodes together (pad = tiles in the run), so the spread slides one tile window along
// the run and merges only the planes that leave it.
static std::vector<WorkItem> slide_items(const std::vector<WorkItem> &h, int nt2, int max_tiles, int chunk) {
    std::vector<WorkItem> s;
    size_t i = 0;
    while (i < h.size()) {
        size_t j = i;
        while (j < h.size() && h[j].tile == h[i].tile) ++j;
        if (j - i > 1) {
            for (size_t k = i; k < j; ++k) {
                WorkItem w = h[k];
                w.pad = 1;
                s.push_back(w);
            }
            i = j;
            continue;
        }
        WorkItem g = h[i];
        g.pad = 1;
        ++i;
        while (i < h.size() && g.pad < max_tiles) {
            const WorkItem &x = h[i];
            if (x.tile != g.tile + g.pad || x.tile % nt2 == 0) break;        // not the next tile of the row
            if (i + 1 < h.size() && h[i + 1].tile == x.tile) break;          // a tile of several chunks
            if (g.count + x.count > chunk) break;
            g.count += x.count;
            ++g.pad;
            ++i;
        }
        s.push_back(g);
    }
    return s;
}

// The block buffers (block_cols columns of staged values, grids and FFT buffers),
// allocated on the first block product and kept until the plan is destroyed: the
// one-column buffers are never touched, and neither set is ever reallocated, so
// products captured into a CUDA graph stay valid.
nfl_status ensure_columns(Plan &P, int nc) {
    if (nc > P.block_cols) return NFL_ERR_INVALID_ARG;
    if (P.blk.grid) return NFL_OK;
    // a stream under capture refuses cudaMalloc (and the capture would be invalidated):
    // the first block product has to come before any capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(P.stream, &cap) != cudaSuccess) return NFL_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return NFL_ERR_INVALID_ARG;
    const int64_t bc = P.block_cols;
    const bool fd = fft_is_double(P.prec);
    const size_t real_sz = fd ? 8 : 4, cplx_sz = 2 * real_sz;
    const size_t grid_sz = P.prec == NFL_PREC_FP32 ? 4 : 8;
    if (cudaMalloc(&P.blk.xsort, P.n * 8 * bc) != cudaSuccess ||
        cudaMalloc(&P.blk.xsorted, P.n * 8 * bc) != cudaSuccess ||
        cudaMalloc(&P.blk.bufA, P.bufA_elems * cplx_sz * bc) != cudaSuccess ||
        cudaMalloc(&P.blk.bufB, P.bufB_elems * cplx_sz * bc) != cudaSuccess ||
        cudaMalloc(&P.blk.g, P.box_elems * real_sz * bc) != cudaSuccess ||
        cudaMalloc(&P.blk.grid, P.box_elems * grid_sz * bc) != cudaSuccess) {
        cudaFree(P.blk.xsort); cudaFree(P.blk.xsorted); cudaFree(P.blk.bufA);
        cudaFree(P.blk.bufB); cudaFree(P.blk.g); cudaFree(P.blk.grid);
        P.blk = BlockBuffers{};
        return NFL_ERR_OUT_OF_MEMORY;
    }
    return NFL_OK;
}

// The warp spread's work list: runs of at most slide_tiles tiles, largest first.
std::vector<WorkItem> spread_item_list(const Plan &P) {
    std::vector<WorkItem> s = slide_items(P.tile_items, P.ntile[P.d - 1], P.slide_tiles, P.chunk);
    std::stable_sort(s.begin(), s.end(), [](const WorkItem &x, const WorkItem &y) { return x.count > y.count; });
    return s;
}

cudaError_t side_fork(Plan &P) {
    if (!P.side) return cudaSuccess;
    NFL_CUDA_TRY(cudaEventRecord(P.fork_ev, P.stream));
    return cudaStreamWaitEvent(P.side, P.fork_ev, 0);
}

cudaError_t side_join(Plan &P) {
    if (!P.side) return cudaSuccess;
    NFL_CUDA_TRY(cudaEventRecord(P.join_ev, P.side));
    return cudaStreamWaitEvent(P.stream, P.join_ev, 0);
}

bool moments_available(const Plan &P) {
    return spread_warp_available(P) && P.m == 6 && !P.bf16_taps && !P.tile_cells.empty();
}

// Dense tiles (at least dense_cell nodes per occupied cell) go to the moment kernels
// as their slabs (the cells of one axis-0 position, item pad = the slab) in pieces of
// at most dense_chunk nodes; the other tiles keep the sliding runs of the warp-slice
// spread and the chunks of the tensor-core interpolation.
ItemLists split_item_lists(const Plan &P) {
    ItemLists L;
    std::vector<WorkItem> rest;
    const int te = P.tile_edge;
    const size_t nti = P.tile_items.size();
    for (size_t i = 0; i < nti;) {
        size_t e = i;                                     // the chunks of one tile: [i, e)
        int64_t nodes = 0;
        while (e < nti && P.tile_items[e].tile == P.tile_items[i].tile) nodes += P.tile_items[e++].count;
        const int32_t tile = P.tile_items[i].tile;
        const int32_t *tc = P.tile_cells.data() + (size_t)tile * (te + 1);
        if (tc[0] > 0 && nodes >= (int64_t)P.dense_cell * tc[0]) {
            int32_t start = P.tile_items[i].start;
            for (int sl = 0; sl < te; ++sl) {
                for (int32_t s0 = 0; s0 < tc[1 + sl]; s0 += P.dense_chunk)
                    L.slab.push_back(WorkItem{tile, start + s0, std::min(P.dense_chunk, tc[1 + sl] - s0), sl});
                for (int32_t s0 = 0; s0 < tc[1 + sl]; s0 += kGatherPiece)
                    L.gslab.push_back(WorkItem{tile, start + s0, std::min(kGatherPiece, tc[1 + sl] - s0), sl});
                start += tc[1 + sl];
            }
        } else {
            rest.insert(rest.end(), P.tile_items.begin() + i, P.tile_items.begin() + e);
        }
        i = e;
    }
    L.sparse = slide_items(rest, P.ntile[P.d - 1], P.slide_tiles, P.chunk);
    L.gsparse = rest;
    const auto by_size = [](const WorkItem &x, const WorkItem &y) { return x.count > y.count; };
    for (std::vector<WorkItem> *v : {&L.sparse, &L.gsparse, &L.slab, &L.gslab})
        std::stable_sort(v->begin(), v->end(), by_size);
    return L;
}

// (Re)allocates dst for cnt items when it holds fewer (old lists are never read again)
static nfl_status ensure_list(WorkItem *&dst, int64_t &have, int64_t cnt) {
    if (dst && cnt <= have) return NFL_OK;
    cudaFree(dst);
    dst = nullptr;
    have = 0;
    if (cudaMalloc(&dst, std::max<int64_t>(cnt, 1) * sizeof(WorkItem)) != cudaSuccess) return NFL_ERR_OUT_OF_MEMORY;
    return NFL_OK;
}

// Stores the four lists on the device: through the page-locked staging (room for all
// four lists, copied on `stream`) at plan creation, by synchronous copies otherwise.
static nfl_status store_item_lists(Plan &P, const ItemLists &L, WorkItem *staging, cudaStream_t stream) {
    const std::vector<WorkItem> *src[4] = {&L.sparse, &L.gsparse, &L.slab, &L.gslab};
    WorkItem **dst[4] = {&P.sparse_items, &P.gsparse_items, &P.slab_items, &P.gslab_items};
    int64_t *cnt[4] = {&P.nsparse, &P.ngsparse, &P.nslab, &P.ngslab};
    if (!staging && cudaStreamSynchronize(P.stream) != cudaSuccess) return NFL_ERR_CUDA;
    for (int k = 0; k < 4; ++k) {
        int64_t have = *cnt[k];
        if (ensure_list(*dst[k], have, (int64_t)src[k]->size()) != NFL_OK) return NFL_ERR_OUT_OF_MEMORY;
        *cnt[k] = (int64_t)src[k]->size();
        if (src[k]->empty()) continue;
        const size_t bytes = src[k]->size() * sizeof(WorkItem);
        if (staging) {
            std::copy(src[k]->begin(), src[k]->end(), staging);
            if (cudaMemcpyAsync(*dst[k], staging, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
                return NFL_ERR_CUDA;
            staging += src[k]->size();
        } else if (cudaMemcpy(*dst[k], src[k]->data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            return NFL_ERR_CUDA;
        }
    }
    return NFL_OK;
}

static size_t list_items(const ItemLists &L) {
    return L.sparse.size() + L.gsparse.size() + L.slab.size() + L.gslab.size();
}

nfl_status rebuild_spread_items(Plan &P) {
    if (moments_available(P)) {
        const nfl_status st = store_item_lists(P, split_item_lists(P), nullptr, P.stream);
        if (st != NFL_OK) return st;
    }
    const std::vector<WorkItem> s = spread_item_list(P);
    if ((int64_t)s.size() > P.nsitems || !P.sitems) {
        cudaFree(P.sitems);
        P.sitems = nullptr;
        P.nsitems = 0;
        if (cudaMalloc(&P.sitems, std::max<size_t>(s.size(), 1) * sizeof(WorkItem)) != cudaSuccess)
            return NFL_ERR_OUT_OF_MEMORY;
    }
    // ordered after any product already queued that reads the old list
    if (cudaStreamSynchronize(P.stream) != cudaSuccess) return NFL_ERR_CUDA;
    if (!s.empty() && cudaMemcpy(P.sitems, s.data(), s.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
        return NFL_ERR_CUDA;
    P.nsitems = (int64_t)s.size();
    return NFL_OK;
}

nfl_status rechunk_items(Plan &P, int chunk) {
    if (chunk < 256 || chunk > kChunk) return NFL_ERR_INVALID_ARG;
    std::vector<WorkItem> h;
    size_t i = 0;
    while (i < P.tile_items.size()) {
        // the tile's node range from its consecutive chunks
        const int32_t tile = P.tile_items[i].tile, start = P.tile_items[i].start;
        int32_t end = start;
        for (; i < P.tile_items.size() && P.tile_items[i].tile == tile; ++i)
            end = P.tile_items[i].start + P.tile_items[i].count;
        for (int32_t s = start; s < end; s += chunk) h.push_back(WorkItem{tile, s, std::min(chunk, end - s), 0});
    }
    P.chunk = chunk;
    P.tile_items = h;
    std::vector<WorkItem> sorted = h;
    std::stable_sort(sorted.begin(), sorted.end(), [](const WorkItem &x, const WorkItem &y) { return x.count > y.count; });
    int64_t have = P.nitems;
    if (ensure_list(P.items, have, (int64_t)sorted.size()) != NFL_OK) return NFL_ERR_OUT_OF_MEMORY;
    if (cudaStreamSynchronize(P.stream) != cudaSuccess ||
        cudaMemcpy(P.items, sorted.data(), sorted.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
        return NFL_ERR_CUDA;
    P.nitems = (int64_t)sorted.size();
    return rebuild_spread_items(P);
}

__global__ void chunks_per_tile(const int32_t *count, int64_t ntiles, int32_t *chunks, unsigned long long *nonempty) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = count[t];
        chunks[t] = (c + kChunk - 1) / kChunk;
        if (c > 0) atomicAdd(nonempty, 1ull);
    }
}

__global__ void fill_items(const int32_t *count, const int64_t *start, const int64_t *item_off, int64_t ntiles, WorkItem *items) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = count[t];
        int64_t o = item_off[t];
        for (int s = 0; s < c; s += kChunk) {
            WorkItem w;
            w.tile = (int32_t)t;
            w.start = (int32_t)(start[t] + s);
            w.count = min(kChunk, c - s);
            w.pad = 0;
            items[o++] = w;
        }
    }
}

// ----------------------------------------------------------- coefficients
struct KRParams {
    int N, d, kind;
    double sigma_t, eps_B;
    int ncoef;
    double coef[32];
};

// K_R(j / N) for j in I_N^d, axis 0 slowest (Sec. 3, the K_R ansatz).
__global__ void kr_samples(double *S, KRParams p) {
    int64_t total = 1;
    for (int a = 0; a < p.d; ++a) total *= p.N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e;
        double r2 = 0.0;
        for (int a = p.d - 1; a >= 0; --a) {
            const int j = (int)(r % p.N) - p.N / 2;
            r /= p.N;
            const double y = double(j) / p.N;
            r2 += y * y;
        }
        const double rr = sqrt(r2);
        double val;
        const double a0 = 0.5 - p.eps_B;
        if (p.eps_B <= 0.0 || rr <= a0) {
            const double r = fmin(rr, 0.5), st = p.sigma_t;
            switch (p.kind) {
                case NFL_KERNEL_LAPLACIAN_RBF: val = exp(-r / st); break;
                case NFL_KERNEL_MULTIQUADRIC: val = sqrt(r * r + st * st); break;
                case NFL_KERNEL_INV_MULTIQUADRIC: val = 1.0 / sqrt(r * r + st * st); break;
                case NFL_KERNEL_GAUSSIAN_DSIGMA: val = 2.0 * r * r / (st * st * st) * exp(-(r / st) * (r / st)); break;
                default: val = exp(-(r / st) * (r / st)); break;
            }
        } else {
            const double s = (fmin(rr, 0.5) - a0) / p.eps_B;
            val = 0.0;
            for (int k = p.ncoef - 1; k >= 0; --k) val = val * s + p.coef[k];
        }
        S[e] = val;
    }
}

// out = sum_{j in I_N} in[.., j, ..] cos(2 pi j l / N), l in [0, N/2], along axis ax.
__global__ void cosine_axis(const double *in, double *out, int64_t outer, int N, int64_t inner, const double *ctab) {
    const int K = N / 2 + 1;
    const int64_t total = outer * K * inner;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ii = e % inner;
        const int64_t rest = e / inner;
        const int l = (int)(rest % K);
        const int64_t o = rest / K;
        const double *src = in + o * N * inner + ii;
        double acc = 0.0;
        for (int jj = 0; jj < N; ++jj) {
            const int j = jj - N / 2;
            int q = (j * l) % N;
            if (q < 0) q += N;
            acc += src[(int64_t)jj * inner] * ctab[q];
        }
        out[e] = acc;
    }
}

struct MultParams {
    int N, d;
    int64_t nA, nB;
    double inv_Nd;
};

// M_eff(l) = b_|l| * prod_a dec(|l_a|) * w(l) in the fused pass's layout.
// w(l) keeps the real part of the sum over I_N exactly: 1 when no |l_a| = N/2,
// 1/2 when all components with |l_a| = N/2 have the same sign, else 0.
template <typename T>
__global__ void build_multiplier(const double *bsum, const double *dec, MultParams p, T *M) {
    const int N = p.N, K0 = N + 1, Kh = N / 2 + 1;
    const int64_t total = p.nA * p.nB * K0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j0 = (int)(e % K0);
        const int64_t line = e / K0;
        const int64_t a = line % p.nA;
        const int64_t b = line / p.nA;
        int k[3] = {0, 0, 0};
        k[0] = j0 - N / 2;
        if (p.d == 2) k[1] = (int)b;                 // R2C axis, >= 0
        if (p.d == 3) { k[1] = (int)b - N / 2; k[2] = (int)a; }
        int64_t bi = 0;
        double prod = 1.0;
        int npos = 0, nneg = 0;
        for (int ax = 0; ax < p.d; ++ax) {
            const int ak = abs(k[ax]);
            bi = bi * Kh + ak;
            prod *= dec[ak];
            if (ak == N / 2) { if (k[ax] > 0) ++npos; else ++nneg; }
        }
        double w = 1.0;
        if (npos + nneg > 0) w = (npos == 0 || nneg == 0) ? 0.5 : 0.0;
        M[e] = T(bsum[bi] * p.inv_Nd * prod * w);
    }
}

// ---------------------------------------------------------------- host math
static double hermite_phys(int k, double x) {
    double h0 = 1.0, h1 = 2.0 * x;
    if (k == 0) return h0;
    for (int j = 1; j < k; ++j) {
        const double h2 = 2.0 * x * h1 - 2.0 * j * h0;
        h0 = h1;
        h1 = h2;
    }
    return h1;
}

// k-th r-derivative of exp(-(r/sigma)^2): (-1/sigma)^k H_k(r/sigma) exp(-(r/sigma)^2).
static double gauss_deriv(double r, double sigma, int k) {
    const double x = r / sigma;
    return std::pow(-1.0 / sigma, k) * hermite_phys(k, x) * std::exp(-x * x);
}

// The radial kernel K(r) of each NFL_KERNEL_* with shape parameter s.
static double kernel_value(int kind, double r, double s) {
    switch (kind) {
        case NFL_KERNEL_LAPLACIAN_RBF: return std::exp(-r / s);
        case NFL_KERNEL_MULTIQUADRIC: return std::sqrt(r * r + s * s);
        case NFL_KERNEL_INV_MULTIQUADRIC: return 1.0 / std::sqrt(r * r + s * s);
        case NFL_KERNEL_GAUSSIAN_DSIGMA: return 2.0 * r * r / (s * s * s) * std::exp(-(r / s) * (r / s));
        default: return std::exp(-(r / s) * (r / s));
    }
}

// Taylor coefficients t_k = K^(k)(a) / k!, k < p, of the radial kernel at r = a.
// Multiquadrics: K(a + h) = P(h)^alpha with P(h) = a^2 + s^2 + 2 a h + h^2 and
// alpha = +-1/2; the coefficients of a power of a power series follow from
// P u' = alpha P' u:  k P_0 u_k = sum_{j=1,2} ((alpha + 1) j - k) P_j u_{k-j}.
static void kernel_taylor(int kind, double a, double s, int p, double *t) {
    if (kind == NFL_KERNEL_MULTIQUADRIC || kind == NFL_KERNEL_INV_MULTIQUADRIC) {
        const double alpha = kind == NFL_KERNEL_MULTIQUADRIC ? 0.5 : -0.5;
        const double P0 = a * a + s * s, P[3] = {P0, 2.0 * a, 1.0};
        t[0] = std::pow(P0, alpha);
        for (int k = 1; k < p; ++k) {
            double acc = 0.0;
            for (int j = 1; j <= 2 && j <= k; ++j) acc += ((alpha + 1.0) * j - k) * P[j] * t[k - j];
            t[k] = acc / (k * P0);
        }
        return;
    }
    double fact = 1.0;
    for (int k = 0; k < p; ++k) {
        if (k > 0) fact *= k;
        double dk;
        if (kind == NFL_KERNEL_LAPLACIAN_RBF) {
            dk = std::pow(-1.0 / s, k) * std::exp(-a / s);
        } else if (kind == NFL_KERNEL_GAUSSIAN_DSIGMA) {
            // (2/s^3) d^k [r^2 g(r)] = (2/s^3) (r^2 g^(k) + 2 k r g^(k-1) + k (k-1) g^(k-2))
            dk = a * a * gauss_deriv(a, s, k);
            if (k >= 1) dk += 2.0 * k * a * gauss_deriv(a, s, k - 1);
            if (k >= 2) dk += k * (k - 1.0) * gauss_deriv(a, s, k - 2);
            dk *= 2.0 / (s * s * s);
        } else {
            dk = gauss_deriv(a, s, k);
        }
        t[k] = dk / fact;
    }
}

// Two-point Taylor polynomial T_B(r) = sum_k c_k s^k, s = (r - a)/eps_B, a = 1/2 - eps_B:
// T_B^(k)(a) = K^(k)(a) for k < p;  T_B(1/2) = K(1/2), T_B^(k)(1/2) = 0 for 1 <= k < p.
static bool boundary_coefficients(int kind, double sigma, double eps_B, int p, double *c) {
    const double a = 0.5 - eps_B;
    kernel_taylor(kind, a, sigma, p, c);
    for (int k = 0; k < p; ++k) c[k] *= std::pow(eps_B, k);
    auto dpow = [](int k, int j) {
        if (k < j) return 0.0;
        double r = 1.0;
        for (int t = k - j + 1; t <= k; ++t) r *= t;
        return r;
    };
    std::vector<double> A(p * p), rhs(p);
    for (int j = 0; j < p; ++j) {
        double s = (j == 0) ? kernel_value(kind, 0.5, sigma) : 0.0;
        for (int k = 0; k < p; ++k) s -= c[k] * dpow(k, j);
        rhs[j] = s;
        for (int col = 0; col < p; ++col) A[j * p + col] = dpow(p + col, j);
    }
    for (int col = 0; col < p; ++col) {  // Gaussian elimination, partial pivoting
        int piv = col;
        for (int r = col + 1; r < p; ++r)
            if (std::fabs(A[r * p + col]) > std::fabs(A[piv * p + col])) piv = r;
        if (A[piv * p + col] == 0.0) return false;
        if (piv != col) {
            for (int t = 0; t < p; ++t) std::swap(A[col * p + t], A[piv * p + t]);
            std::swap(rhs[col], rhs[piv]);
        }
        for (int r = col + 1; r < p; ++r) {
            const double f = A[r * p + col] / A[col * p + col];
            for (int t = col; t < p; ++t) A[r * p + t] -= f * A[col * p + t];
            rhs[r] -= f * rhs[col];
        }
    }
    for (int r = p - 1; r >= 0; --r) {
        double s = rhs[r];
        for (int t = r + 1; t < p; ++t) s -= A[r * p + t] * c[p + t];
        c[p + r] = s / A[r * p + r];
    }
    return true;
}

// Modified Bessel function I_0 by its power series sum ((z/2)^2)^k / (k!)^2.
static double bessel_i0(double z) {
    const double q = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / (double(k) * k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

// Step 3 (b_l by the trapezoidal rule) and the fused multiplier, launched on the
// plan's stream without a host synchronization: the kernel samples, the three
// separable cosine sums and the multiplier.  tab (page-locked host memory that
// stays valid until the stream has passed these launches) receives the cosine
// table (N values) and the deconvolution factors (N/2 + 1); S, T1, ctab, dec
// are device temporaries the caller frees after the stream has passed them.
static nfl_status coefficients_launch(Plan &P, double *tab, double *&S, double *&T1, double *&ctab, double *&dec) {
    const int N = P.N, d = P.d, Kh = N / 2 + 1;
    KRParams kp{};
    kp.N = N;
    kp.d = d;
    kp.kind = P.kernel;
    kp.sigma_t = P.sigma_t;
    kp.eps_B = P.eps_B;
    kp.ncoef = 0;
    if (P.eps_B > 0.0) {
        if (2 * P.p > 32) return NFL_ERR_INVALID_ARG;
        if (!boundary_coefficients(P.kernel, P.sigma_t, P.eps_B, P.p, kp.coef)) return NFL_ERR_INVALID_ARG;
        kp.ncoef = 2 * P.p;
    }
    int64_t full = 1;
    for (int a = 0; a < d; ++a) full *= N;
    if (cudaMalloc(&S, full * sizeof(double)) != cudaSuccess || cudaMalloc(&T1, full * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctab, N * sizeof(double)) != cudaSuccess || cudaMalloc(&dec, Kh * sizeof(double)) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    double *h_ct = tab, *h_dec = tab + N;
    for (int q = 0; q < N; ++q) h_ct[q] = std::cos(2.0 * M_PI * q / N);
    // dec(k) = (phi(0) / (n phi_hat(k)))^2 = (phi(0) / I_0(m sqrt(b^2 - (2 pi k / n)^2)))^2
    const double b = P.kb_b, m = P.m, n = P.ngrid;
    const double phi0 = std::sinh(b * m) / (M_PI * m);
    for (int k = 0; k < Kh; ++k) {
        const double arg = b * b - std::pow(2.0 * M_PI * k / n, 2);
        const double r = phi0 / bessel_i0(m * std::sqrt(arg));
        h_dec[k] = r * r;
    }
    cudaStream_t s = P.stream;
    if (cudaMemcpyAsync(ctab, h_ct, N * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dec, h_dec, Kh * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return NFL_ERR_CUDA;
    const int blocks = P.num_sms * 8;
    kr_samples<<<blocks, 256, 0, s>>>(S, kp);
    // cosine transform along each axis, last axis first
    int64_t ext[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) ext[a] = N;
    double *src = S, *dst = T1;
    for (int ax = d - 1; ax >= 0; --ax) {
        int64_t outer = 1, inner = 1;
        for (int a = 0; a < ax; ++a) outer *= ext[a];
        for (int a = ax + 1; a < d; ++a) inner *= ext[a];
        cosine_axis<<<blocks, 256, 0, s>>>(src, dst, outer, N, inner, ctab);
        ext[ax] = Kh;
        std::swap(src, dst);
    }
    MultParams mp;
    mp.N = N;
    mp.d = d;
    mp.inv_Nd = 1.0 / double(full);
    if (d == 1) { mp.nA = 1; mp.nB = 1; }
    else if (d == 2) { mp.nA = 1; mp.nB = Kh; }
    else { mp.nA = Kh; mp.nB = N + 1; }
    if (fft_is_double(P.prec)) build_multiplier<double><<<blocks, 256, 0, s>>>(src, dec, mp, (double *)P.mult);
    else build_multiplier<float><<<blocks, 256, 0, s>>>(src, dec, mp, (float *)P.mult);
    return cudaGetLastError() == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

static void free_plan(Plan *P) {
    if (!P) return;
    if (P->side) {
        cudaStreamSynchronize(P->side);
        cudaStreamDestroy(P->side);
    }
    if (P->fork_ev) cudaEventDestroy(P->fork_ev);
    if (P->join_ev) cudaEventDestroy(P->join_ev);
    if (P->pipe_stream) {
        cudaStreamSynchronize(P->pipe_stream);
        cudaStreamDestroy(P->pipe_stream);
    }
    for (cudaEvent_t e : {P->pipe_fork, P->pipe_spread_done, P->pipe_staged[0], P->pipe_staged[1]})
        if (e) cudaEventDestroy(e);
    cudaFree(P->pipe_xsort);
    cudaFree(P->pipe_xsorted);
    cudaFree(P->pipe_scratch);
    for (cudaEvent_t e : P->events) cudaEventDestroy(e);
    if (P->h2d) cudaStreamSynchronize(P->h2d);
    if (P->d2h) cudaStreamSynchronize(P->d2h);
    for (int s = 0; s < kHostSlots; ++s) {
        if (P->ev_in[s]) cudaEventDestroy(P->ev_in[s]);
        if (P->ev_done[s]) cudaEventDestroy(P->ev_done[s]);
        if (P->ev_out[s]) cudaEventDestroy(P->ev_out[s]);
    }
    if (P->ev_start) cudaEventDestroy(P->ev_start);
    if (P->h2d) cudaStreamDestroy(P->h2d);
    if (P->d2h) cudaStreamDestroy(P->d2h);
    cudaFree(P->host_stage);
    cudaFree(P->items);
    cudaFree(P->blk.xsort); cudaFree(P->blk.xsorted); cudaFree(P->blk.bufA);
    cudaFree(P->blk.bufB); cudaFree(P->blk.g); cudaFree(P->blk.grid);
    cudaFree(P->sitems);
    cudaFree(P->sparse_items);
    cudaFree(P->gsparse_items);
    cudaFree(P->slab_items);
    cudaFree(P->gslab_items);
    cudaFree(P->tile_start);
    cudaFree(P->pts);
    cudaFree(P->perm);
    cudaFree(P->dinv_sorted);
    cudaFree(P->xsort);
    cudaFree(P->xsorted);
    cudaFree(P->degree);
    cudaFree(P->grid);
    cudaFree(P->bufA);
    cudaFree(P->bufB);
    cudaFree(P->g);
    cudaFree(P->mult);
    cudaFree(P->twiddle);
    cudaFree(P->scratch);
    cudaFree(P->error_flag);
    cudaFree(P->work_counter);
    delete P;
}

// phi(delta) / phi(0) for the normalized Kaiser-Bessel window, in FP64 on the host.
static double host_window(double delta, double m, double b, double inv_den) {
    const double s2 = std::max(m * m - delta * delta, 0.0);
    const double s = std::sqrt(s2);
    const double head = std::exp(-b * delta * delta / (s + m));
    const double tail = s > 0.0 ? -std::expm1(-2.0 * b * s) / s : 2.0 * b;
    return head * m * tail * inv_den;
}

// Per-tap polynomials of the window for the FP32 kernels: tap j of a node at
// fractional offset f sees phi(f + m - 1 - j); on f in [0, 1) this is
// interpolated at the kPolyCoef Chebyshev points of t = 2 f - 1 and the
// Chebyshev series is re-expanded in powers of t.  The window is an entire
// function of delta, so degree 9 reaches FP32 rounding of the peak for
// every m here (about 7e-8 of phi(0), measured on a dense grid of f).
static void window_poly(Plan &P) {
    constexpr int NC = kPolyCoef;
    const double m = P.m;
    for (int j = 0; j < 2 * P.m && j < 2 * kMaxM; ++j) {
        double fv[NC], c[NC], mono[NC] = {0}, tkm1[NC] = {0}, tk[NC] = {0}, tn[NC];
        for (int i = 0; i < NC; ++i) {
            const double t = std::cos(M_PI * (i + 0.5) / NC);
            fv[i] = host_window(0.5 * (t + 1.0) + m - 1.0 - j, m, P.kb_b, P.kb_inv_sinh_bm);
        }
        for (int k = 0; k < NC; ++k) {
            double acc = 0.0;
            for (int i = 0; i < NC; ++i) acc += fv[i] * std::cos(M_PI * k * (i + 0.5) / NC);
            c[k] = (k == 0 ? 1.0 : 2.0) * acc / NC;
        }
        // sum_k c_k T_k(t) with T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1}
        tkm1[0] = 1.0;
        tk[1] = 1.0;
        mono[0] = c[0];
        for (int q = 0; q < NC; ++q) mono[q] += c[1] * tk[q];
        for (int k = 2; k < NC; ++k) {
            for (int q = 0; q < NC; ++q) tn[q] = (q > 0 ? 2.0 * tk[q - 1] : 0.0) - tkm1[q];
            for (int q = 0; q < NC; ++q) {
                tkm1[q] = tk[q];
                tk[q] = tn[q];
                mono[q] += c[k] * tn[q];
            }
        }
        for (int q = 0; q < NC; ++q) P.kb_poly[j][q] = static_cast<float>(mono[q]);
        // degree kCheb - 1 interpolant at kCheb Chebyshev points, kept in the Chebyshev basis
        for (int k = 0; k < kCheb; ++k) {
            double acc = 0.0;
            for (int i = 0; i < kCheb; ++i) {
                const double t = std::cos(M_PI * (i + 0.5) / kCheb);
                acc += host_window(0.5 * (t + 1.0) + m - 1.0 - j, m, P.kb_b, P.kb_inv_sinh_bm) *
                       std::cos(M_PI * k * (i + 0.5) / kCheb);
            }
            P.kb_cheb[j][k] = static_cast<float>((k == 0 ? 1.0 : 2.0) * acc / kCheb);
        }
    }
}

// ------------------------------------------------------------ plan creation
// Alg. 2 steps 1-4 run as phases, each of which only issues work on the plan's
// stream and ends with device-to-host reads into page-locked memory; the host
// synchronizes once between phases.  nfl_plan_create runs the phases for one
// plan; nfl_plan_create_batched runs each phase for every plan of a batch
// (spread over the library's streams) before the one synchronization, so a
// batch costs as many host synchronizations as one plan.
constexpr int kRBlocks = 1024;   // reduction partials per pass

struct Builder {
    Plan *P = nullptr;
    const double *v = nullptr;
    int64_t n = 0;
    int d = 0, kernel = 0, N = 0, m = 0, p = 0, prec = 0;
    double sigma = 0, eps_B = 0;
    cudaStream_t stream = 0;
    nfl_status st = NFL_OK;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    Geometry G{};
    int cpt = 1;
    double *part = nullptr;              // device reduction partials (kRBlocks x 6)
    double *hp = nullptr;                // page-locked: the partials and counts read back
    int32_t *key_of = nullptr, *rank = nullptr, *kcount = nullptr, *count = nullptr, *chunks = nullptr;
    int64_t *kstart = nullptr, *start = nullptr, *item_off = nullptr;
    unsigned long long *nonempty = nullptr;
    WorkItem *hitems = nullptr;          // page-locked: chunks read back, then the lists uploaded
    WorkItem *hlists = nullptr;          // page-locked: the dense-cell work lists uploaded
    int32_t *occ = nullptr, *hocc = nullptr;   // occupied cells per tile (device, page-locked)
    double *htab = nullptr;              // page-locked: twiddles, cosine table, deconvolution factors
    double *S = nullptr, *T1 = nullptr, *ctab = nullptr, *dec = nullptr;   // coefficient temporaries
};

static void release_temporaries(Builder &B) {
    cudaFree(B.part); cudaFree(B.key_of); cudaFree(B.rank); cudaFree(B.kcount); cudaFree(B.count);
    cudaFree(B.chunks); cudaFree(B.kstart); cudaFree(B.start); cudaFree(B.item_off); cudaFree(B.nonempty);
    cudaFree(B.S); cudaFree(B.T1); cudaFree(B.ctab); cudaFree(B.dec);
    cudaFreeHost(B.hp); cudaFreeHost(B.hitems); cudaFreeHost(B.hlists); cudaFreeHost(B.htab);
    cudaFree(B.occ); cudaFreeHost(B.hocc);
    B.occ = B.hocc = nullptr;
    B.part = B.S = B.T1 = B.ctab = B.dec = B.hp = B.htab = nullptr;
    B.key_of = B.rank = B.kcount = B.count = B.chunks = nullptr;
    B.kstart = B.start = B.item_off = nullptr;
    B.nonempty = nullptr;
    B.hitems = B.hlists = nullptr;
}

// Fields, window polynomials, per-plan scalars; step 1: bounding-box partials.
static nfl_status phase_setup(Builder &B) {
    Plan *P = B.P;
    int prec = B.prec;
    // BF16W is the FP32 form with BF16-rounded window taps
    P->bf16_taps = prec == NFL_PREC_BF16W;
    if (P->bf16_taps) prec = NFL_PREC_FP32;
    P->n = B.n; P->d = B.d; P->N = B.N; P->m = B.m; P->p = B.p; P->prec = prec;
    P->sigma = B.sigma; P->eps_B = B.eps_B; P->stream = B.stream;
    P->kernel = B.kernel;
    P->ngrid = 2 * B.N;
    P->kb_b = M_PI * (2.0 - 1.0 / 2.0);
    P->kb_inv_sinh_bm = 1.0 / -std::expm1(-2.0 * P->kb_b * B.m);   // 1 / (1 - e^{-2 b m})
    window_poly(*P);
    int dev = 0;
    NFL_STATUS_TRY(cudaGetDevice(&dev));
    NFL_STATUS_TRY(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev));
    NFL_STATUS_TRY(cudaDeviceGetAttribute(&P->l2_bytes, cudaDevAttrL2CacheSize, dev));
    NFL_STATUS_TRY(cudaMalloc(&P->scratch, 64 * sizeof(double)));
    NFL_STATUS_TRY(cudaMalloc(&P->error_flag, sizeof(int)));
    NFL_STATUS_TRY(cudaMalloc(&P->work_counter, 4 * sizeof(unsigned)));
    NFL_STATUS_TRY(cudaMemsetAsync(P->error_flag, 0, sizeof(int), B.stream));
    NFL_STATUS_TRY(cudaMalloc(&B.part, kRBlocks * 6 * sizeof(double)));
    NFL_STATUS_TRY(cudaHostAlloc(&B.hp, kRBlocks * 6 * sizeof(double), cudaHostAllocDefault));
    bbox_partials<<<kRBlocks, 256, 0, B.stream>>>(B.v, B.n, B.d, B.part);
    NFL_STATUS_TRY(cudaMemcpyAsync(B.hp, B.part, kRBlocks * 6 * sizeof(double), cudaMemcpyDeviceToHost, B.stream));
    return NFL_OK;
}

// Step 1: bounding box and centre; radius partials.
static nfl_status phase_radius(Builder &B) {
    Plan *P = B.P;
    const double *hp = B.hp;
    for (int a = 0; a < B.d; ++a) {
        B.lo[a] = INFINITY;
        B.hi[a] = -INFINITY;
        bool bad = false;   // a block saw a non-finite coordinate (fmin/fmax would drop NaN)
        for (int b = 0; b < kRBlocks; ++b) {
            bad = bad || std::isnan(hp[b * 6 + a]) || std::isnan(hp[b * 6 + 3 + a]);
            B.lo[a] = std::fmin(B.lo[a], hp[b * 6 + a]);
            B.hi[a] = std::fmax(B.hi[a], hp[b * 6 + 3 + a]);
        }
        if (bad || !std::isfinite(B.lo[a]) || !std::isfinite(B.hi[a])) return NFL_ERR_INVALID_ARG;
        P->center[a] = 0.5 * (B.lo[a] + B.hi[a]);
    }
    radius_partials<<<kRBlocks, 256, 0, B.stream>>>(B.v, B.n, B.d, P->center[0], P->center[1], P->center[2], B.part);
    NFL_STATUS_TRY(cudaMemcpyAsync(B.hp, B.part, kRBlocks * sizeof(double), cudaMemcpyDeviceToHost, B.stream));
    return NFL_OK;
}

// Steps 1-2: rho and sigma~; the active box, tiles, and the counting sort of the nodes.
static nfl_status phase_sort(Builder &B) {
    Plan *P = B.P;
    const int d = B.d, m = B.m;
    const int64_t n = B.n;
    const cudaStream_t stream = B.stream;
    double r2 = 0.0;
    for (int b = 0; b < kRBlocks; ++b) r2 = std::fmax(r2, B.hp[b]);
    const double radius = std::sqrt(r2);
    P->rho = radius > 0.0 ? (0.25 - 0.5 * B.eps_B) / radius : 1.0;   // all nodes coincide: any rho fits
    P->sigma_t = P->rho * B.sigma;                                   // step 2
    // the scaled kernel is rho^(+-1) times the caller's for the multiquadrics
    const int kernel = B.kernel;
    P->out_scale = kernel == NFL_KERNEL_MULTIQUADRIC ? 1.0 / P->rho
                   : ((kernel == NFL_KERNEL_INV_MULTIQUADRIC || kernel == NFL_KERNEL_GAUSSIAN_DSIGMA) ? P->rho : 1.0);
    P->k0 = kernel_value(kernel, 0.0, B.sigma);

    // active box: cells floor(n v~) - t0 with t0 leaving m taps (and one cell) of room
    Geometry &G = B.G;
    G.d = d;
    G.rho = P->rho;
    G.ngrid = P->ngrid;
    for (int a = 0; a < 3; ++a) G.c[a] = P->center[a];
    // 3-D: the column spreading kernel's tile edge where it exists; otherwise
    // tile + halo must fit shared memory at 8 bytes per cell: (T + 2m - 1)^3 <= 29^3
    if (d == 3) P->tile_edge = column_tile_edge(m) > 0 ? column_tile_edge(m) : std::min(8, 30 - 2 * m);
    else P->tile_edge = d == 2 ? 32 : 256;
    G.tile_edge = P->tile_edge;
    P->box_elems = 1;
    for (int a = 0; a < d; ++a) {
        const double umin = P->ngrid * (P->rho * (B.lo[a] - P->center[a]));
        const double umax = P->ngrid * (P->rho * (B.hi[a] - P->center[a]));
        const int64_t bmin = (int64_t)std::floor(umin), bmax = (int64_t)std::floor(umax);
        P->t0[a] = bmin - (m - 1) - 1;
        G.t0[a] = P->t0[a];
        const int64_t span = bmax - P->t0[a] + m + 2;   // box positions touched, unwrapped
        if (span > 1023) return NFL_ERR_INVALID_ARG;
        P->wrap[a] = span > P->ngrid ? 1 : 0;
        P->L[a] = (int)(span > P->ngrid ? P->ngrid : span);
        P->ntile[a] = (int)((span + P->tile_edge - 1) / P->tile_edge);
        G.ntile[a] = P->ntile[a];
        P->box_elems *= P->L[a];
    }
    P->tiles_total = 1;
    for (int a = 0; a < d; ++a) P->tiles_total *= P->ntile[a];

    // counting sort of the nodes by tile and, inside a tile, by cell
    const int64_t nt = P->tiles_total;
    int cpt = 1;
    for (int a = 0; a < d; ++a) cpt *= P->tile_edge;
    if (nt * cpt > (int64_t)1 << 26) cpt = 1;   // very large grids: sort by tile only
    B.cpt = cpt;
    const int64_t nkeys = nt * cpt;
    if (cudaMalloc(&B.key_of, n * 4) != cudaSuccess || cudaMalloc(&B.rank, n * 4) != cudaSuccess ||
        cudaMalloc(&B.kcount, nkeys * 4) != cudaSuccess || cudaMalloc(&B.kstart, (nkeys + 1) * 8) != cudaSuccess ||
        cudaMalloc(&B.count, nt * 4) != cudaSuccess || cudaMalloc(&B.chunks, nt * 4) != cudaSuccess ||
        cudaMalloc(&B.start, (nt + 1) * 8) != cudaSuccess || cudaMalloc(&B.item_off, (nt + 1) * 8) != cudaSuccess ||
        cudaMalloc(&B.nonempty, 8) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    const bool dbl = points_are_double(P->prec);
    if (cudaMalloc(&P->pts, n * (dbl ? sizeof(PointD) : sizeof(PointF))) != cudaSuccess ||
        cudaMalloc(&P->perm, n * 4) != cudaSuccess || cudaMalloc(&P->dinv_sorted, n * 8) != cudaSuccess ||
        cudaMalloc(&P->degree, n * 8) != cudaSuccess || cudaMalloc(&P->xsort, n * 8) != cudaSuccess ||
        cudaMalloc(&P->xsorted, n * 8) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    const int blocks = P->num_sms * 8;
    NFL_STATUS_TRY(cudaMemsetAsync(B.kcount, 0, nkeys * 4, stream));
    NFL_STATUS_TRY(cudaMemsetAsync(B.nonempty, 0, 8, stream));
    count_keys<<<blocks, 256, 0, stream>>>(B.v, n, G, cpt, B.key_of, B.rank, B.kcount);
    exclusive_scan<<<1, 1024, 0, stream>>>(B.kcount, nkeys, B.kstart);
    tiles_from_keys<<<blocks, 256, 0, stream>>>(B.kstart, nt, cpt, B.count, B.start);
    if (dbl) scatter_nodes<PointD, double><<<blocks, 256, 0, stream>>>(B.v, n, G, B.key_of, B.rank, B.kstart,
                                                                       (PointD *)P->pts, P->perm);
    else scatter_nodes<PointF, float><<<blocks, 256, 0, stream>>>(B.v, n, G, B.key_of, B.rank, B.kstart,
                                                                  (PointF *)P->pts, P->perm);
    chunks_per_tile<<<blocks, 256, 0, stream>>>(B.count, nt, B.chunks, B.nonempty);
    exclusive_scan<<<1, 1024, 0, stream>>>(B.chunks, nt, B.item_off);
    NFL_STATUS_TRY(cudaMemcpyAsync(B.hp, B.item_off + nt, 8, cudaMemcpyDeviceToHost, stream));
    NFL_STATUS_TRY(cudaMemcpyAsync(B.hp + 1, B.nonempty, 8, cudaMemcpyDeviceToHost, stream));
    return cudaGetLastError() == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

// The work items (tile chunks) and tile starts; the chunks are read back.
static nfl_status phase_items(Builder &B) {
    Plan *P = B.P;
    const cudaStream_t stream = B.stream;
    std::memcpy(&P->nitems, B.hp, 8);
    unsigned long long ne = 0;
    std::memcpy(&ne, B.hp + 1, 8);
    P->tiles_nonempty = (int64_t)ne;
    const int64_t nt = P->tiles_total;
    if (cudaMalloc(&P->items, std::max<int64_t>(P->nitems, 1) * sizeof(WorkItem)) != cudaSuccess ||
        cudaMalloc(&P->tile_start, (nt + 1) * sizeof(int32_t)) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    const int blocks = P->num_sms * 8;
    fill_items<<<blocks, 256, 0, stream>>>(B.count, B.start, B.item_off, nt, P->items);
    tile_starts<<<blocks, 256, 0, stream>>>(B.kstart, nt, B.cpt, P->tile_start);
    // occupied cells and slab nodes per tile (for the dense-cell spread and interpolation;
    // only when the nodes of a tile are sorted by cell, in 3-D)
    if (B.cpt > 1 && B.d == 3) {
        const int te = P->tile_edge;
        const int64_t per = (int64_t)nt * (te + 1);
        NFL_STATUS_TRY(cudaMalloc(&B.occ, std::max<int64_t>(per, 1) * sizeof(int32_t)));
        NFL_STATUS_TRY(cudaHostAlloc(&B.hocc, std::max<int64_t>(per, 1) * sizeof(int32_t), cudaHostAllocDefault));
        occupied_cells<<<blocks, 256, 0, stream>>>(B.kstart, nt, B.cpt, te, B.occ);
        NFL_STATUS_TRY(cudaMemcpyAsync(B.hocc, B.occ, per * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    }
    // room for the sorted chunks and the warp spread's list (at most one entry per chunk)
    NFL_STATUS_TRY(cudaHostAlloc(&B.hitems, std::max<int64_t>(2 * P->nitems, 1) * sizeof(WorkItem),
                                 cudaHostAllocDefault));
    if (P->nitems > 0)
        NFL_STATUS_TRY(cudaMemcpyAsync(B.hitems, P->items, P->nitems * sizeof(WorkItem), cudaMemcpyDeviceToHost,
                                       stream));
    return cudaGetLastError() == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

// Work lists, FFT buffers, twiddles; step 3 (coefficients) and step 4 (degrees, one
// fast product with x = 1); the degree partials are read back.
static nfl_status phase_finish(Builder &B) {
    Plan *P = B.P;
    const cudaStream_t stream = B.stream;
    const int64_t n = B.n;
    const int N = B.N, d = B.d;
    const int prec = P->prec;
    if (P->nitems > 0) {
        // largest chunks first: the kernels that take items from a shared counter
        // then end with small ones (longest-processing-time order)
        P->tile_items.assign(B.hitems, B.hitems + P->nitems);
        if (B.hocc) P->tile_cells.assign(B.hocc, B.hocc + P->tiles_total * (P->tile_edge + 1));
        const std::vector<WorkItem> s = spread_item_list(*P);
        if (cudaMalloc(&P->sitems, std::max<size_t>(s.size(), 1) * sizeof(WorkItem)) != cudaSuccess)
            return NFL_ERR_OUT_OF_MEMORY;
        P->nsitems = (int64_t)s.size();
        std::vector<WorkItem> h = P->tile_items;
        std::stable_sort(h.begin(), h.end(), [](const WorkItem &x, const WorkItem &y) { return x.count > y.count; });
        std::copy(h.begin(), h.end(), B.hitems);
        std::copy(s.begin(), s.end(), B.hitems + P->nitems);
        NFL_STATUS_TRY(cudaMemcpyAsync(P->items, B.hitems, P->nitems * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                       stream));
        if (!s.empty())
            NFL_STATUS_TRY(cudaMemcpyAsync(P->sitems, B.hitems + P->nitems, s.size() * sizeof(WorkItem),
                                           cudaMemcpyHostToDevice, stream));
        if (moments_available(*P)) {
            if (cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&P->join_ev, cudaEventDisableTiming) != cudaSuccess)
                return NFL_ERR_CUDA;
            const ItemLists L = split_item_lists(*P);
            NFL_STATUS_TRY(cudaHostAlloc(&B.hlists, std::max<size_t>(list_items(L), 1) * sizeof(WorkItem),
                                         cudaHostAllocDefault));
            const nfl_status st = store_item_lists(*P, L, B.hlists, stream);
            if (st != NFL_OK) return st;
        }
    }

    // FFT buffers, twiddles, multiplier
    const bool fd = fft_is_double(prec);
    const size_t real_sz = fd ? 8 : 4, cplx_sz = 2 * real_sz;
    const int64_t Kh = N / 2 + 1, K0 = N + 1;
    const int64_t L0 = P->L[0], L1 = P->L[1];
    int64_t bufA = 1, bufB = 1, mult = K0;
    if (d == 2) { bufA = Kh * L0; bufB = Kh * L0; mult = Kh * K0; }
    if (d == 3) {
        bufA = std::max(Kh * L0 * L1, Kh * K0 * L0);
        bufB = std::max(K0 * Kh * L0, L1 * L0 * Kh);
        mult = K0 * Kh * K0;
    }
    const size_t grid_sz = prec == NFL_PREC_FP32 ? 4 : 8;
    P->bufA_elems = bufA;
    P->bufB_elems = bufB;
    {
        // block width: as many columns as keep their staged values, grids and FFT
        // buffers within half of L2 (so consecutive stages find their inputs there)
        const double per_col = double(n) * (4 + 8) + double(P->box_elems) * (grid_sz + real_sz) +
                               double(bufA + bufB) * cplx_sz;
        const double budget = 0.5 * double(P->l2_bytes > 0 ? P->l2_bytes : (64 << 20));
        const int w = int(budget / per_col);
        P->block_cols = w < 1 ? 1 : (w > kBlockCols ? kBlockCols : w);
    }
    if (cudaMalloc(&P->grid, P->box_elems * grid_sz) != cudaSuccess ||
        cudaMalloc(&P->bufA, bufA * cplx_sz) != cudaSuccess || cudaMalloc(&P->bufB, bufB * cplx_sz) != cudaSuccess ||
        cudaMalloc(&P->g, P->box_elems * real_sz) != cudaSuccess || cudaMalloc(&P->mult, mult * real_sz) != cudaSuccess ||
        cudaMalloc(&P->twiddle, (P->ngrid / 2) * cplx_sz) != cudaSuccess)
        return NFL_ERR_OUT_OF_MEMORY;
    // page-locked table: twiddles (ngrid / 2 complex), cosine table (N), deconvolution (N / 2 + 1)
    const int half = P->ngrid / 2;
    NFL_STATUS_TRY(cudaHostAlloc(&B.htab, (2 * half + N + Kh) * sizeof(double), cudaHostAllocDefault));
    if (fd) {
        for (int q = 0; q < half; ++q) {
            B.htab[2 * q] = std::cos(2.0 * M_PI * q / P->ngrid);
            B.htab[2 * q + 1] = -std::sin(2.0 * M_PI * q / P->ngrid);
        }
        NFL_STATUS_TRY(cudaMemcpyAsync(P->twiddle, B.htab, 2 * half * 8, cudaMemcpyHostToDevice, stream));
    } else {
        float *tf = reinterpret_cast<float *>(B.htab);
        for (int q = 0; q < half; ++q) {
            tf[2 * q] = static_cast<float>(std::cos(2.0 * M_PI * q / P->ngrid));
            tf[2 * q + 1] = static_cast<float>(-std::sin(2.0 * M_PI * q / P->ngrid));
        }
        NFL_STATUS_TRY(cudaMemcpyAsync(P->twiddle, B.htab, 2 * half * 4, cudaMemcpyHostToDevice, stream));
    }
    nfl_status st = coefficients_launch(*P, B.htab + 2 * half, B.S, B.T1, B.ctab, B.dec);   // step 3
    if (st != NFL_OK) return st;

    // step 4: degrees through the fast path with x = 1
    st = run_column(*P, OP_DEGREE, nullptr, nullptr);
    if (st != NFL_OK) return st;
    minmax_partials<<<kRBlocks, 256, 0, stream>>>(P->degree, n, B.part);
    NFL_STATUS_TRY(cudaMemcpyAsync(B.hp, B.part, kRBlocks * 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    return cudaGetLastError() == cudaSuccess ? NFL_OK : NFL_ERR_CUDA;
}

// Degree summary (Lemma 3.1: A and L_s need min d_E > 0).
static nfl_status phase_summary(Builder &B) {
    Plan *P = B.P;
    P->min_deg = INFINITY;
    P->max_deg = -INFINITY;
    for (int b = 0; b < kRBlocks; ++b) {
        P->min_deg = std::fmin(P->min_deg, B.hp[2 * b]);
        P->max_deg = std::fmax(P->max_deg, B.hp[2 * b + 1]);
    }
    P->degree_ok = P->min_deg > 0.0 && std::isfinite(P->max_deg);
    return NFL_OK;
}

// Runs every phase for all builders, with one synchronization of the streams in
// use between phases; a builder that fails skips the later phases.  Temporaries
// are released at the end (after the streams have passed them).
static void run_phases(std::vector<Builder> &Bs) {
    typedef nfl_status (*Phase)(Builder &);
    const Phase phases[] = {phase_setup, phase_radius, phase_sort, phase_items, phase_finish, phase_summary};
    std::vector<cudaStream_t> streams;
    for (const Builder &B : Bs)
        if (std::find(streams.begin(), streams.end(), B.stream) == streams.end()) streams.push_back(B.stream);
    for (Phase ph : phases) {
        for (Builder &B : Bs)
            if (B.st == NFL_OK) B.st = ph(B);
        for (cudaStream_t s : streams) {
            if (cudaStreamSynchronize(s) == cudaSuccess) continue;
            for (Builder &B : Bs)
                if (B.stream == s && B.st == NFL_OK) B.st = NFL_ERR_CUDA;
        }
    }
    for (Builder &B : Bs) release_temporaries(B);
}

// Argument checks of the create calls; p <= 0 and eps_B < 0 take their defaults.
static nfl_status check_plan_args(int64_t n, int d, int kernel, double sigma, int N, int m, int &p, double &eps_B,
                                  int precision) {
    if (n < 1 || n > 0x7fffffff || d < 1 || d > 3 || kernel < NFL_KERNEL_GAUSSIAN || kernel > NFL_KERNEL_GAUSSIAN_DSIGMA)
        return NFL_ERR_INVALID_ARG;
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return NFL_ERR_INVALID_ARG;
    if (N < 4 || N > 512 || (N & (N - 1)) != 0) return NFL_ERR_INVALID_ARG;
    if (m < 1 || m > kMaxM) return NFL_ERR_INVALID_ARG;
    if (p <= 0) p = m;
    if (p > 16) return NFL_ERR_INVALID_ARG;
    if (eps_B < 0.0) eps_B = double(p) / N;
    if (!(eps_B < 0.5)) return NFL_ERR_INVALID_ARG;
    if (precision != NFL_PREC_FP64 && precision != NFL_PREC_FP32 && precision != NFL_PREC_FP32C &&
        precision != NFL_PREC_BF16W)
        return NFL_ERR_INVALID_ARG;
    return NFL_OK;
}

static void fill_builder(Builder &B, Plan *P, const double *v, int64_t n, int d, int kernel, double sigma, int N,
                         int m, int p, double eps_B, int precision, cudaStream_t stream) {
    B.P = P;
    B.v = v;
    B.n = n;
    B.d = d;
    B.kernel = kernel;
    B.sigma = sigma;
    B.N = N;
    B.m = m;
    B.p = p;
    B.eps_B = eps_B;
    B.prec = precision;
    B.stream = stream;
}

}  // namespace nfl

using nfl::Plan;

extern "C" {

const char *nfl_status_string(int s) {
    switch (s) {
        case NFL_OK: return "ok";
        case NFL_ERR_INVALID_ARG: return "invalid argument";
        case NFL_ERR_NONPOSITIVE_DEGREE: return "non-positive degree: D^{-1/2} undefined";
        case NFL_ERR_BREAKDOWN: return "Lanczos breakdown (invariant subspace)";
        case NFL_ERR_NOT_CONVERGED: return "not converged";
        case NFL_ERR_NAN: return "NaN or Inf in solver scalars";
        case NFL_ERR_TIMEOUT: return "bounded device wait timed out";
        case NFL_ERR_CUDA: return "CUDA runtime error";
        case NFL_ERR_OUT_OF_MEMORY: return "out of device memory";
    }
    return "unknown status";
}

nfl_status nfl_plan_create(const double *v, int64_t n, int d, int kernel, double sigma, int N, int m, int p,
                           double eps_B, int precision, void *stream, nfl_plan **out) {
    if (!out) return NFL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!v) return NFL_ERR_INVALID_ARG;
    const nfl_status ck = nfl::check_plan_args(n, d, kernel, sigma, N, m, p, eps_B, precision);
    if (ck != NFL_OK) return ck;
    Plan *P = new (std::nothrow) Plan();
    if (!P) return NFL_ERR_OUT_OF_MEMORY;
    std::vector<nfl::Builder> Bs(1);
    nfl::fill_builder(Bs[0], P, v, n, d, kernel, sigma, N, m, p, eps_B, precision, (cudaStream_t)stream);
    nfl::run_phases(Bs);
    if (Bs[0].st != NFL_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        nfl::free_plan(P);
        return Bs[0].st;
    }
    *out = reinterpret_cast<nfl_plan *>(P);
    return NFL_OK;
}

nfl_status nfl_plan_create_batched(int G, const double *const *v, const int64_t *n, int d, int kernel,
                                   const double *sigma, int N, int m, int p, double eps_B, int precision,
                                   void *stream, nfl_plan **out) {
    if (!out || !v || !n || !sigma || G < 1) return NFL_ERR_INVALID_ARG;
    for (int g = 0; g < G; ++g) out[g] = nullptr;
    int pg = p;
    double eg = eps_B;
    for (int g = 0; g < G; ++g) {
        if (!v[g]) return NFL_ERR_INVALID_ARG;
        pg = p;
        eg = eps_B;
        const nfl_status ck = nfl::check_plan_args(n[g], d, kernel, sigma[g], N, m, pg, eg, precision);
        if (ck != NFL_OK) return ck;
    }
    nfl::BatchStreams *pool = nfl::batch_streams();
    if (!pool) return NFL_ERR_CUDA;
    const cudaStream_t origin = (cudaStream_t)stream;
    const int K = G < nfl::kBatchStreams ? G : nfl::kBatchStreams;
    // plans to library streams, largest first to the least loaded, forked from the caller's stream
    if (cudaEventRecord(pool->fork, origin) != cudaSuccess) return NFL_ERR_CUDA;
    for (int k = 0; k < K; ++k)
        if (cudaStreamWaitEvent(pool->s[k], pool->fork, 0) != cudaSuccess) return NFL_ERR_CUDA;
    std::vector<int> order(G);
    std::vector<int64_t> load(K, 0);
    for (int g = 0; g < G; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    std::vector<nfl::Builder> Bs(G);
    for (int g : order) {
        const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += n[g];
        Plan *P = new (std::nothrow) Plan();
        if (!P) {
            for (nfl::Builder &B : Bs) delete B.P;
            return NFL_ERR_OUT_OF_MEMORY;
        }
        nfl::fill_builder(Bs[g], P, v[g], n[g], d, kernel, sigma[g], N, m, pg, eg, precision, pool->s[k]);
    }
    nfl::run_phases(Bs);   // every phase ends with the library streams synchronized
    nfl_status st = NFL_OK;
    for (const nfl::Builder &B : Bs)
        if (B.st != NFL_OK) {
            st = B.st;
            break;
        }
    if (st != NFL_OK) {
        for (int k = 0; k < K; ++k) cudaStreamSynchronize(pool->s[k]);
        for (nfl::Builder &B : Bs) nfl::free_plan(B.P);
        return st;
    }
    for (int g = 0; g < G; ++g) {
        Bs[g].P->stream = origin;
        out[g] = reinterpret_cast<nfl_plan *>(Bs[g].P);
    }
    return NFL_OK;
}

void nfl_plan_destroy(nfl_plan *plan) {
    if (!plan) return;
    Plan *P = reinterpret_cast<Plan *>(plan);
    cudaStreamSynchronize(P->stream);
    nfl::free_plan(P);
}

nfl_status nfl_plan_inject_fault(nfl_plan *plan, int kind) {
    if (!plan || kind < 0 || kind > 1) return NFL_ERR_INVALID_ARG;
    reinterpret_cast<nfl::Plan *>(plan)->fault_kind = kind;
    return NFL_OK;
}

nfl_status nfl_plan_info(const nfl_plan *plan, nfl_info *info) {
    if (!plan || !info) return NFL_ERR_INVALID_ARG;
    const Plan *P = reinterpret_cast<const Plan *>(plan);
    std::memset(info, 0, sizeof(*info));
    info->n = P->n;
    info->d = P->d;
    info->N = P->N;
    info->m = P->m;
    info->p = P->p;
    info->precision = P->bf16_taps ? NFL_PREC_BF16W : P->prec;
    info->sigma = P->sigma;
    info->eps_B = P->eps_B;
    info->rho = P->rho;
    info->sigma_tilde = P->sigma_t;
    info->kernel = P->kernel;
    info->k0 = P->k0;
    info->out_scale = P->out_scale;
    info->fft_lines_cap = P->fft_cap;
    info->slide_tiles = P->slide_tiles;
    info->block_cols = P->block_cols;
    info->dense_items = moments_available(*P) ? P->nslab : 0;
    info->chunk = P->chunk;
    info->dense_cell = P->dense_cell;
    info->dense_chunk = P->dense_chunk;
    for (int a = 0; a < 3; ++a) {
        info->center[a] = P->center[a];
        info->box[a] = a < P->d ? P->L[a] : 1;
    }
    info->tiles = P->tiles_nonempty;
    info->work_items = P->nitems;
    info->min_degree = P->min_deg;
    info->max_degree = P->max_deg;
    info->degree_ok = P->degree_ok ? 1 : 0;
    int flag = 0;
    if (P->error_flag) {
        if (cudaMemcpyAsync(&flag, P->error_flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
            cudaStreamSynchronize(P->stream) != cudaSuccess)
            return NFL_ERR_CUDA;
    }
    info->device_error = flag;
    return NFL_OK;
}

nfl_status nfl_set_stream(nfl_plan *plan, void *stream) {
    if (!plan) return NFL_ERR_INVALID_ARG;
    reinterpret_cast<Plan *>(plan)->stream = (cudaStream_t)stream;
    return NFL_OK;
}

nfl_status nfl_degree(const nfl_plan *plan, double *d) {
    if (!plan || !d) return NFL_ERR_INVALID_ARG;
    const Plan *P = reinterpret_cast<const Plan *>(plan);
    return cudaMemcpyAsync(d, P->degree, P->n * sizeof(double), cudaMemcpyDeviceToDevice, P->stream) == cudaSuccess
               ? NFL_OK
               : NFL_ERR_CUDA;
}

}  // extern "C"
