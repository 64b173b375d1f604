// Window spreading in 3-D (Alg. 1 step 1, the window half of the adjoint NFFT):
//   h_t = sum_i x~_i phi(n v~_i0 - t_0) phi(n v~_i1 - t_1) phi(n v~_i2 - t_2).
//
// A first kernel writes x~ = D_E^{-1/2} x (Alg. 2 step 5) in the plan's
// tile-sorted node order, so the spread reads node records and values with
// coalesced loads, one batch ahead of use.
//
// The plan sorts the nodes of every tile by cell, so the nodes of one cell
// are contiguous; they share the whole (2M)^3 support.  A CTA takes one chunk
// of one tile (TE^3 cells) and keeps the tile plus halo (PA = TE + 2M - 1 per
// axis) in shared memory, one copy per thread group.  Nodes are staged in
// batches of 32 per group; group g takes the g-th slice of 32 consecutive
// nodes, whose cell runs the staging warp marks in a bit mask.  In a group,
// thread (jb, jc) owns one support-relative column of the current cell and
// 2M registers along axis 0; each node of a run adds coef * w0[ja],
// coef = x~ w1[jb] w2[jc], for ja = 0..2M-1 (FP32: two lanes per
// fma.rn.f32x2).  Every multiply-add lands in the support, with no range
// tests.  When the cell changes, the group meets at a named barrier and each
// thread adds its 2M values to the group's tile with plain read-modify-write:
// in one flush the threads of a group touch distinct positions, and the
// barrier orders flushes of different cells.  At the end of the chunk the
// non-zero tile cells go to the global grid with one atomic each.
//
// FP32 window weights come from the plan's per-tap polynomials (Horner in
// t = 2f - 1, two taps per fma.rn.f32x2); FP64 evaluates the window itself.
//
// FP32C: each group's FP32 tile only ever holds the sums of 8 slices (256 of
// its nodes); then both tiles are carried into a 64-bit fixed-point tile
// (scale 2^k from sum |x~|, so no partial sum can overflow).  Everything
// after that is exact integer addition.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

struct Spread3Args {
    const void *pts;
    const void *xs;                 // x~ in sorted order (spread type)
    const WorkItem *items;
    int64_t nitems;
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    void *grid;
    const double *abs_sum;
    double b, inv_den;
    int bf16;                       // BF16W: FP32 taps rounded to BF16
    float poly[2 * kMaxM][kPolyCoef];
};

// x~_k = x[perm[k]] * dinv[k] (or dinv[k] / 1 for the all-ones vector) in sorted
// order; with abs_sum, also sum_k |x~_k| (the fixed-point scale of FP32C).
// z_k, the x-only part of the interpolation epilogue y = z + s f (Alg. 2 step 5,
// K(0) = k0, d = dinv):
//   W: z = -k0 x,  A: z = -k0 d^2 x,  L_s: z = x + k0 d^2 x   (none for the degree).
// Column blockIdx.y of a block: x + c ldx in, out + c n and z_out + c n out, abs_sum[c].
template <typename T>
__device__ __forceinline__ void stage_body(const double *x, const int32_t *perm, const double *dinv, int64_t n, int ones,
                                           T *out, double *z_out, int op, double k0, double *abs_sum, int64_t blk,
                                           int64_t nblk) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t k = blk * (int64_t)blockDim.x + threadIdx.x; k < n; k += nblk * blockDim.x) {
        const double xv = ones ? 1.0 : x[perm[k]];
        const double dk = dinv ? dinv[k] : 1.0;
        const double v = dinv ? xv * dk : xv;
        out[k] = T(v);
        if (op == OP_W) z_out[k] = -k0 * xv;
        else if (op == OP_A) z_out[k] = -k0 * dk * v;
        else if (op == OP_LS) z_out[k] = fma(k0 * dk, v, xv);
        acc += fabs(v);
    }
    if (!abs_sum) return;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(abs_sum, red[0]);
}

template <typename T>
__global__ void __launch_bounds__(256) stage_values(const double *x, int64_t ldx, const int32_t *perm,
                                                    const double *dinv, int64_t n, int ones, T *out, double *z_out,
                                                    int op, double k0, double *abs_sum) {
    const int col = blockIdx.y;
    stage_body<T>(x + col * ldx, perm, dinv, n, ones, out + col * n, z_out + col * n, op, k0,
                  abs_sum ? abs_sum + col : nullptr, blockIdx.x, gridDim.x);
}

// The staging of every member of a batch in one launch: CTA x-index b belongs to the
// plan g with start[g] <= b < start[g + 1]; column blockIdx.y.
__global__ void __launch_bounds__(256) stage_values_batch(const BatchPlanDev *D, const int *start, int G, int op,
                                                          int fixed) {
    const int b = blockIdx.x;
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const BatchPlanDev &P = D[lo];
    const int col = blockIdx.y;
    const bool scale = op == OP_A || op == OP_LS;
    stage_body<float>(P.x + col * P.ldx, P.perm, scale ? P.dinv : nullptr, P.n, 0, P.xs + col * P.n,
                      P.zd + col * P.n, op, P.k0, fixed ? P.abs_sum + col : nullptr, b - start[lo],
                      start[lo + 1] - start[lo]);
}

cudaError_t launch_stage_batch(Batch &B, cudaStream_t s) {
    if (B.stage_ctas < 1) return cudaSuccess;
    stage_values_batch<<<dim3(B.stage_ctas, B.ncol), 256, 0, s>>>(B.desc, B.stage_start, B.G, B.op,
                                                                   B.prec == NFL_PREC_FP32C ? 1 : 0);
    return cudaGetLastError();
}

__device__ __forceinline__ void group_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}


constexpr int kCarry = 8;   // FP32C: slices (of 32 nodes per group) per fixed-point carry

template <int M, int TE>
struct CellGeom {
    static constexpr int PA = TE + 2 * M - 1;     // tile + halo per axis
    static constexpr int PA3 = PA * PA * PA;
    static constexpr int TAPS = 2 * M;
    static constexpr int TAPS4 = (TAPS + 3) / 4 * 4;
    static constexpr int PAIRS = TAPS / 2;
    static constexpr int OWN = TAPS * TAPS;       // threads of a group owning a support column (jb, jc)
    static constexpr int NTG = (OWN + 31) / 32 * 32;
    static constexpr int GROUPS = 2;
    static constexpr int NT = GROUPS * NTG;
    static constexpr int S = 32;                  // nodes per group per batch (one staging warp)
    static constexpr int B = S * GROUPS;          // nodes staged per batch
};

// CTAs per SM that shared memory admits (at most 3, and no fewer than 64
// registers per thread): the register budget is set to match, so registers
// do not limit occupancy below shared memory.
template <typename T, int M, int TE, bool FIXED>
constexpr int cells_min_blocks() {
    using G = CellGeom<M, TE>;
    constexpr int dyn = G::GROUPS * ((G::PA3 * (int)sizeof(T) + 15) / 16) * 16 + (FIXED ? G::PA3 * 8 : 0);
    constexpr int stat = G::B * (G::TAPS4 + 2 * G::TAPS + 4) * (int)sizeof(T) + G::B * 4 + G::PAIRS * kPolyCoef * 8 + 64;
    constexpr int by_smem = 232448 / (dyn + stat + 1024);
    constexpr int by_threads = 65536 / (G::NT * 64);    // keep 64 registers per thread
    constexpr int b = by_smem < by_threads ? by_smem : by_threads;
    return b < 1 ? 1 : (b > 3 ? 3 : b);
}

// Register accumulator of one support column: 2M values along axis 0.
template <typename T, int TAPS> struct ColumnAcc {
    T v[TAPS];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int q = 0; q < TAPS; ++q) v[q] = T(0);
    }
    __device__ __forceinline__ void add(T coef, const T *row) {
        const double2 *r2 = reinterpret_cast<const double2 *>(row);
#pragma unroll
        for (int q = 0; q < TAPS / 2; ++q) {
            const double2 w = r2[q];
            v[2 * q] += coef * w.x;
            v[2 * q + 1] += coef * w.y;
        }
    }
    __device__ __forceinline__ T get(int q) const { return v[q]; }
};
template <int TAPS> struct ColumnAcc<float, TAPS> {
    unsigned long long v[TAPS / 2];               // taps (2q, 2q + 1)
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int q = 0; q < TAPS / 2; ++q) v[q] = 0ull;
    }
    __device__ __forceinline__ void add(float coef, const float *row) {
        const ulonglong2 *r = reinterpret_cast<const ulonglong2 *>(row);
        const unsigned long long c2 = pack2(coef, coef);
#pragma unroll
        for (int q = 0; q < (TAPS + 3) / 4; ++q) {
            const ulonglong2 w = r[q];
            v[2 * q] = ffma2(c2, w.x, v[2 * q]);
            if (2 * q + 1 < TAPS / 2) v[2 * q + 1] = ffma2(c2, w.y, v[2 * q + 1]);
        }
    }
    __device__ __forceinline__ float get(int q) const { return lane_of(v[q >> 1], q & 1); }
};

template <typename T, int M, int TE, bool FIXED>
__global__ void __launch_bounds__(CellGeom<M, TE>::NT, (cells_min_blocks<T, M, TE, FIXED>()))
    spread3_cells(Spread3Args a) {
    using G = CellGeom<M, TE>;
    constexpr int PA = G::PA, PA3 = G::PA3, TAPS = G::TAPS, TAPS4 = G::TAPS4, S = G::S, B = G::B, NT = G::NT;
    constexpr int TILE_STRIDE = ((PA3 * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T);
    using Pt = typename PointOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tiles = reinterpret_cast<T *>(smem_raw);                                       // GROUPS x PA^3, [a][b][c]
    unsigned long long *itile =
        reinterpret_cast<unsigned long long *>(smem_raw + G::GROUPS * TILE_STRIDE * sizeof(T));
    __shared__ __align__(16) T w0s[B][TAPS4];
    __shared__ T w1s[B][TAPS], w2s[B][TAPS];
    __shared__ T frs[B][3];
    __shared__ T xs[B];
    __shared__ int org[B];                                // tile-local base cell, 8 bits per axis
    __shared__ unsigned runs[G::GROUPS];                  // bit i: slice node i starts a cell run
    __shared__ __align__(16) float2 polys[G::PAIRS][kPolyCoef];   // (tap 2q, tap 2q+1) coefficients

    const int tid = threadIdx.x;
    const int grp = tid / G::NTG, gtid = tid - grp * G::NTG;
    const bool owner = gtid < G::OWN;
    const int jb = owner ? gtid / TAPS : 0;
    const int jc = owner ? gtid % TAPS : 0;
    T *tile = tiles + grp * TILE_STRIDE;
    const Pt *pts = reinterpret_cast<const Pt *>(a.pts);
    const T *xsrc = reinterpret_cast<const T *>(a.xs);
    T fscale = T(1);
    if (FIXED) fscale = T(fixed_scale_of(*a.abs_sum));
    for (int e = tid; e < G::GROUPS * TILE_STRIDE; e += NT) tiles[e] = T(0);
    if (FIXED)
        for (int e = tid; e < PA3; e += NT) itile[e] = 0ull;
    for (int e = tid; e < G::PAIRS * kPolyCoef; e += NT) {
        const int q = e / kPolyCoef, k = e - q * kPolyCoef;
        polys[q][k] = make_float2(a.poly[2 * q][k], a.poly[2 * q + 1][k]);
    }

    ColumnAcc<T, TAPS> acc;
    // group barrier, then add this thread's 2M values of cell o to the group's tile
    auto flush = [&](int o) {
        group_barrier(1 + grp, G::NTG);
        if (owner) {
            const int s0 = o & 255, s1 = (o >> 8) & 255, s2 = o >> 16;
            T *col = tile + (s0 * PA + s1 + jb) * PA + s2 + jc;
#pragma unroll
            for (int ja = 0; ja < TAPS; ++ja) col[ja * PA * PA] += acc.get(ja);
        }
        acc.clear();
    };

    for (int64_t it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        const int wend = w.start + w.count;
        int tc[3];
        tile_coords<3>(w.tile, a.ntile, tc);
        acc.clear();
        int cur = -1;
        int bcount = 0;
        // node record and value of this thread's slot, one batch ahead
        Pt pn;
        T xn = T(0);
        if (tid < B && w.start + tid < wend) {
            pn = pts[w.start + tid];
            xn = xsrc[w.start + tid];
        }

        for (int base = w.start; base < wend; base += B) {
            const int nb = min(B, wend - base);
            if (tid < B) {                                // warps 0 .. GROUPS-1: one slice each
                const bool valid = tid < nb;
                int o = -1;
                if (valid) {
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        o = (ax == 0 ? 0 : o) | ((cell_axis(pn.cell, ax) - tc[ax] * TE) << (8 * ax));
                        frs[tid][ax] = T(pn.f[ax]);
                    }
                    xs[tid] = xn;
                    org[tid] = o;
                }
                const int lane = tid & 31;
                const int prev = __shfl_up_sync(0xffffffffu, o, 1);
                const unsigned m = __ballot_sync(0xffffffffu, valid && (lane == 0 || o != prev));
                if (lane == 0) runs[tid >> 5] = m;
                const int kn = base + B + tid;
                if (kn < wend) {
                    pn = pts[kn];
                    xn = xsrc[kn];
                }
            }
            __syncthreads();
            if constexpr (std::is_same<T, float>::value) {
                // one (axis, node) per item; the lanes of a warp read the same coefficients
                for (int e = tid; e < 3 * B; e += NT) {
                    const int ax = e / B, pt = e - ax * B;
                    if (pt >= nb) continue;
                    const float t = fmaf(2.f, frs[pt][ax], -1.f);
                    const unsigned long long t2 = pack2(t, t);
                    const float sc = ax == 1 ? xs[pt] : 1.f;    // x~ folded into the axis-1 window
                    float *dst = ax == 0 ? w0s[pt] : (ax == 1 ? w1s[pt] : w2s[pt]);
                    const unsigned long long *pc = reinterpret_cast<const unsigned long long *>(&polys[0][0]);
#pragma unroll 1
                    for (int q = 0; q < G::PAIRS; ++q) {
                        unsigned long long h = pc[q * kPolyCoef + kPolyCoef - 1];
#pragma unroll
                        for (int k = kPolyCoef - 2; k >= 0; --k) h = ffma2(h, t2, pc[q * kPolyCoef + k]);
                        float w0 = lane_of(h, 0), w1 = lane_of(h, 1);
                        if (a.bf16) {
                            w0 = round_bf16(w0);
                            w1 = round_bf16(w1);
                        }
                        dst[2 * q] = w0 * sc;
                        dst[2 * q + 1] = w1 * sc;
                    }
                }
            } else {
                const T tm = T(M), tb = T(a.b), tden = T(a.inv_den);
                for (int e = tid; e < nb * 3 * TAPS; e += NT) {
                    const int pt = e / (3 * TAPS);
                    const int r = e - pt * 3 * TAPS;
                    const int ax = r / TAPS;
                    const int j = r - ax * TAPS;
                    const T wv = kb_weight<T>(frs[pt][ax] + T(M - 1) - T(j), tm, tb, tden);
                    if (ax == 0) w0s[pt][j] = wv;
                    else if (ax == 1) w1s[pt][j] = wv * xs[pt];
                    else w2s[pt][j] = wv;
                }
            }
            __syncthreads();
            {
                // this group's slice, one cell run at a time
                const unsigned rm = runs[grp];
                const int s0 = grp * S;
                const int cnt = max(0, min(S, nb - s0));
                int i = 0;
                while (i < cnt) {
                    const unsigned rest = i + 1 < 32 ? (rm >> (i + 1)) : 0u;
                    const int j = rest ? min(cnt, i + __ffs(rest)) : cnt;
                    const int o = org[s0 + i];
                    if (o != cur) {
                        if (cur >= 0) flush(cur);
                        cur = o;
                    }
                    if (owner) {
#pragma unroll 2
                        for (int q = s0 + i; q < s0 + j; ++q) acc.add(w1s[q][jb] * w2s[q][jc], w0s[q]);
                    }
                    i = j;
                }
            }
            // FP32C carries the FP32 sums into fixed point every kCarry batches and at the chunk end
            const bool carry = FIXED && ((++bcount % kCarry) == 0 || base + B >= wend);
            if (carry && cur >= 0) flush(cur);
            __syncthreads();
            if (carry) {
                for (int e = tid; e < PA3; e += NT) {
                    long long add = 0;
#pragma unroll
                    for (int g = 0; g < G::GROUPS; ++g) {
                        T &tv = tiles[g * TILE_STRIDE + e];
                        if (tv != T(0)) {
                            add += to_fixed(tv * fscale);
                            tv = T(0);
                        }
                    }
                    if (add != 0) itile[e] += (unsigned long long)add;
                }
                __syncthreads();
            }
        }
        if (!FIXED && cur >= 0) flush(cur);
        __syncthreads();

        // tile -> global grid (c fastest, matching the grid's x2 axis), then clear it
        for (int e = tid; e < PA3; e += NT) {
            const int q2 = e % PA, q1 = (e / PA) % PA, q0 = e / (PA * PA);
            int p0 = tc[0] * TE - (M - 1) + q0;
            int p1 = tc[1] * TE - (M - 1) + q1;
            int p2 = tc[2] * TE - (M - 1) + q2;
            if (a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
            if (a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
            if (a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
            const bool ok = p0 >= 0 && p0 < a.L[0] && p1 >= 0 && p1 < a.L[1] && p2 >= 0 && p2 < a.L[2];
            const int64_t gidx = ((int64_t)p0 * a.L[1] + p1) * a.L[2] + p2;
            if (FIXED) {
                const unsigned long long val = itile[e];
                if (val != 0ull) {
                    itile[e] = 0ull;
                    if (ok) atomicAdd(reinterpret_cast<unsigned long long *>(a.grid) + gidx, val);
                }
            } else {
                T val = T(0);
#pragma unroll
                for (int g = 0; g < G::GROUPS; ++g) {
                    val += tiles[g * TILE_STRIDE + e];
                    tiles[g * TILE_STRIDE + e] = T(0);
                }
                if (val != T(0) && ok) atomicAdd(reinterpret_cast<T *>(a.grid) + gidx, val);
            }
        }
        __syncthreads();
    }
}

template <typename T, int M, int TE, bool FIXED>
static cudaError_t launch_cols(Plan &P, const Spread3Args &a) {
    using G = CellGeom<M, TE>;
    auto kern = spread3_cells<T, M, TE, FIXED>;
    const int smem = G::GROUPS * ((G::PA3 * (int)sizeof(T) + 15) / 16) * 16 + (FIXED ? G::PA3 * 8 : 0);
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > P.nitems) grid = P.nitems;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, G::NT, smem, P.stream>>>(a);
    return cudaGetLastError();
}

// Tile edge used with the column kernel for cut-off m (3-D), 0 if none.
int column_tile_edge(int m) {
    switch (m) {
        case 2: case 3: case 4: return 8;
        case 6: return 4;
        case 7: case 8: return 2;
    }
    return 0;
}

template <typename T, bool FIXED>
static cudaError_t dispatch_cols(Plan &P, const Spread3Args &a) {
    switch (P.m) {
        case 2: return launch_cols<T, 2, 8, FIXED>(P, a);
        case 3: return launch_cols<T, 3, 8, FIXED>(P, a);
        case 4: return launch_cols<T, 4, 8, FIXED>(P, a);
        case 6: return launch_cols<T, 6, 4, FIXED>(P, a);
        case 7: return launch_cols<T, 7, 2, FIXED>(P, a);
        case 8: return launch_cols<T, 8, 2, FIXED>(P, a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t stage_spread3_values(Plan &P, int op, const double *x, int64_t ldx, int nc, bool ones,
                                 bool scale_dinv) {
    const double *dinv = scale_dinv ? P.dinv_sorted : nullptr;
    double *abs_sum = nullptr;
    if (P.prec == NFL_PREC_FP32C) {
        NFL_CUDA_TRY(cudaMemsetAsync(P.scratch, 0, nc * sizeof(double), P.stream));
        abs_sum = P.scratch;
    }
    const dim3 blocks((P.num_sms * 4 + nc - 1) / nc, nc);
    if (P.prec == NFL_PREC_FP64)
        stage_values<double><<<blocks, 256, 0, P.stream>>>(x, ldx, P.perm, dinv, P.n, ones ? 1 : 0,
                                                           static_cast<double *>(P.xsort), P.xsorted, op, P.k0,
                                                           abs_sum);
    else
        stage_values<float><<<blocks, 256, 0, P.stream>>>(x, ldx, P.perm, dinv, P.n, ones ? 1 : 0,
                                                          static_cast<float *>(P.xsort), P.xsorted, op, P.k0,
                                                          abs_sum);
    return cudaGetLastError();
}

cudaError_t launch_spread3_columns(Plan &P, const double *, bool, bool) {
    Spread3Args a;
    a.pts = P.pts;
    a.xs = P.xsort;
    a.items = P.items;
    a.nitems = P.nitems;
    for (int i = 0; i < 3; ++i) {
        a.ntile[i] = P.ntile[i];
        a.L[i] = P.L[i];
        a.wrap[i] = P.wrap[i];
    }
    a.ngrid = P.ngrid;
    a.grid = P.grid;
    a.abs_sum = P.scratch;
    a.b = P.kb_b;
    a.inv_den = P.kb_inv_sinh_bm;
    a.bf16 = P.bf16_taps ? 1 : 0;
    for (int j = 0; j < 2 * kMaxM; ++j)
        for (int k = 0; k < kPolyCoef; ++k) a.poly[j][k] = P.kb_poly[j][k];
    if (P.prec == NFL_PREC_FP64) return dispatch_cols<double, false>(P, a);
    if (P.prec == NFL_PREC_FP32C) return dispatch_cols<float, true>(P, a);
    return dispatch_cols<float, false>(P, a);
}

}  // namespace nfl
