// Window spreading in 3-D (Alg. 1 step 1, the window half of the adjoint NFFT):
//   h_t = sum_i x~_i phi(n v~_i0 - t_0) phi(n v~_i1 - t_1) phi(n v~_i2 - t_2).
//
// The plan sorts the nodes of every tile by cell, so the nodes of one cell
// are contiguous; they share the whole (2M)^3 support.  A CTA takes one chunk
// of one tile (TE^3 cells) and keeps the tile plus halo (PA = TE + 2M - 1 per
// axis) in shared memory.  One or two thread groups take alternate nodes; in
// each, thread (jb, jc) owns one support-relative column of its current cell
// and 2M registers along axis 0; each node adds
// coef * w0[ja], coef = x~ w1[jb] w2[jc], for ja = 0..2M-1: every fused
// multiply-add lands in the support, with no range tests.  When the cell
// changes (and before every fixed-point carry for FP32C) each thread adds
// its 2M values to the shared tile with shared-memory atomics (supports of
// neighbouring cells overlap); at the end of the chunk the non-zero tile
// cells go to the global grid with one atomic each.
//
// FP32C: the shared FP32 tile only ever holds the sums of 8 batches (256
// nodes); then it is carried into a 64-bit fixed-point tile (scale 2^k from
// sum |x~|, so no partial sum can overflow).  Everything after that is
// exact integer addition; only the order in which the FP32 partial sums of a
// carry interval meet in the shared tile varies from run to run.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

struct Spread3Args {
    const void *pts;
    const int32_t *perm;
    const double *x;
    const double *dinv;
    const WorkItem *items;
    int64_t nitems;
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    void *grid;
    const double *abs_sum;
    int ones;
    double b, inv_den;
};

__device__ __forceinline__ double fixed_scale_of(double abs_sum) {
    if (!(abs_sum > 0.0)) return 1.0;
    int e;
    frexp(abs_sum, &e);
    int k = 62 - e;
    k = k > 1000 ? 1000 : (k < -1000 ? -1000 : k);
    return ldexp(1.0, k);
}

// acc[q] += coef * row[q], q < PA, with 16-byte shared loads of the row.
template <typename T, int PA>
__device__ __forceinline__ void fma_row(T *acc, T coef, const T *row) {
    if (sizeof(T) == 4) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < (PA + 3) / 4; ++q) {
            const float4 w = r4[q];
            if (4 * q + 0 < PA) acc[4 * q + 0] += coef * T(w.x);
            if (4 * q + 1 < PA) acc[4 * q + 1] += coef * T(w.y);
            if (4 * q + 2 < PA) acc[4 * q + 2] += coef * T(w.z);
            if (4 * q + 3 < PA) acc[4 * q + 3] += coef * T(w.w);
        }
    } else {
        const double2 *r2 = reinterpret_cast<const double2 *>(row);
#pragma unroll
        for (int q = 0; q < (PA + 1) / 2; ++q) {
            const double2 w = r2[q];
            if (2 * q + 0 < PA) acc[2 * q + 0] += coef * T(w.x);
            if (2 * q + 1 < PA) acc[2 * q + 1] += coef * T(w.y);
        }
    }
}

// acc0[q] += k0 * row[q], acc1[q] += k1 * row[q]: one pass over the row for two columns.
template <typename T, int PA>
__device__ __forceinline__ void fma_row2(T *acc0, T *acc1, T k0, T k1, const T *row) {
    if (sizeof(T) == 4) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < (PA + 3) / 4; ++q) {
            const float4 w = r4[q];
            const T v[4] = {T(w.x), T(w.y), T(w.z), T(w.w)};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (4 * q + u < PA) {
                    acc0[4 * q + u] += k0 * v[u];
                    acc1[4 * q + u] += k1 * v[u];
                }
        }
    } else {
        const double2 *r2 = reinterpret_cast<const double2 *>(row);
#pragma unroll
        for (int q = 0; q < (PA + 1) / 2; ++q) {
            const double2 w = r2[q];
            const T v[2] = {T(w.x), T(w.y)};
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (2 * q + u < PA) {
                    acc0[2 * q + u] += k0 * v[u];
                    acc1[2 * q + u] += k1 * v[u];
                }
        }
    }
}

// FP32 value (already scaled by 2^k, |v| < 2^62) -> nearest int64 with 32-bit
// conversions only.  |v| = h 2^32 + l with h = floor(|v| 2^-32) and
// 0 <= l < 2^32: both parts are exact in FP32 (power-of-two scaling; l keeps
// a subset of the bits of |v|), and the sign is applied to the integer.
__device__ __forceinline__ long long to_fixed(float v) {
    const float av = fabsf(v);
    const float hf = floorf(av * 2.3283064365386963e-10f);
    const float lf = fmaf(hf, -4294967296.0f, av);
    const unsigned long long mag = ((unsigned long long)__float2uint_rn(hf) << 32) + __float2uint_rn(lf);
    return v < 0.f ? -(long long)mag : (long long)mag;
}
__device__ __forceinline__ long long to_fixed(double v) { return __double2ll_rn(v); }

constexpr int kCarry = 8;   // FP32C: batches (of 32 nodes) per fixed-point carry

// GROUPS thread groups per CTA take alternate nodes: two for FP32C, whose
// larger shared footprint (FP32 + int64 tiles) leaves fewer CTAs per SM.
template <int M, int TE, int GROUPS_>
struct CellGeom {
    static constexpr int PA = TE + 2 * M - 1;     // tile + halo per axis
    static constexpr int TAPS = 2 * M;
    static constexpr int TAPS4 = (TAPS + 3) / 4 * 4;
    static constexpr int OWN = TAPS * TAPS;       // threads of a group owning a support column (jb, jc)
    static constexpr int NTG = (OWN + 31) / 32 * 32;
    static constexpr int GROUPS = GROUPS_;
    static constexpr int NT = GROUPS * NTG;
    static constexpr int B = 32 * GROUPS;         // nodes staged per batch
};

template <typename T, int M, int TE, bool FIXED>
__global__ void __launch_bounds__(CellGeom<M, TE, FIXED ? 2 : 1>::NT) spread3_cells(Spread3Args a) {
    using G = CellGeom<M, TE, FIXED ? 2 : 1>;
    constexpr int PA = G::PA, PA3 = PA * PA * PA, TAPS = G::TAPS, TAPS4 = G::TAPS4, B = G::B, NT = G::NT;
    using Pt = typename PointOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);                                        // PA^3, [a][b][c]
    unsigned long long *itile = reinterpret_cast<unsigned long long *>(smem_raw + ((PA3 * sizeof(T) + 15) / 16) * 16);
    __shared__ __align__(16) T w0s[B][TAPS4];
    __shared__ T w1s[B][TAPS], w2s[B][TAPS];
    __shared__ T frs[B][3];
    __shared__ T xs[B];
    __shared__ int org[B];                                // tile-local base cell, 8 bits per axis

    const int tid = threadIdx.x;
    const int grp = tid / G::NTG, gtid = tid - grp * G::NTG;
    const bool owner = gtid < G::OWN;
    const int jb = owner ? gtid / TAPS : 0;
    const int jc = owner ? gtid % TAPS : 0;
    const T tm = T(M), tb = T(a.b), tden = T(a.inv_den);
    const Pt *pts = reinterpret_cast<const Pt *>(a.pts);
    T fscale = T(1);
    if (FIXED) fscale = T(fixed_scale_of(*a.abs_sum));
    for (int e = tid; e < PA3; e += NT) {
        tile[e] = T(0);
        if (FIXED) itile[e] = 0ull;
    }

    // add this thread's 2M values along a for the support column (jb, jc) of cell o
    auto flush = [&](int o, T *acc) {
        const int s0 = o & 255, s1 = (o >> 8) & 255, s2 = o >> 16;
        T *col = tile + (s0 * PA + s1 + jb) * PA + s2 + jc;
#pragma unroll
        for (int ja = 0; ja < TAPS; ++ja) {
            if (acc[ja] != T(0)) atomicAdd(col + ja * PA * PA, acc[ja]);
            acc[ja] = T(0);
        }
    };

    for (int64_t it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        int tc[3];
        tile_coords<3>(w.tile, a.ntile, tc);
        T acc[TAPS];
#pragma unroll
        for (int q = 0; q < TAPS; ++q) acc[q] = T(0);
        int cur = -1;
        int bcount = 0;

        for (int base = w.start; base < w.start + w.count; base += B) {
            const int nb = min(B, w.start + w.count - base);
            if (tid < nb) {
                const int k = base + tid;
                const Pt p = pts[k];
                double xv = a.ones ? 1.0 : a.x[a.perm[k]];
                if (a.dinv) xv *= a.dinv[k];
                xs[tid] = T(xv);
                int o = 0;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    o |= (cell_axis(p.cell, ax) - tc[ax] * TE) << (8 * ax);
                    frs[tid][ax] = T(p.f[ax]);
                }
                org[tid] = o;
            }
            __syncthreads();
            for (int e = tid; e < nb * 3 * TAPS; e += NT) {
                const int pt = e / (3 * TAPS);
                const int r = e - pt * 3 * TAPS;
                const int ax = r / TAPS;
                const int j = r - ax * TAPS;
                const T wv = kb_weight<T>(frs[pt][ax] + T(M - 1) - T(j), tm, tb, tden);
                if (ax == 0) w0s[pt][j] = wv;
                else if (ax == 1) w1s[pt][j] = wv * xs[pt];   // x~ folded into the axis-1 window
                else w2s[pt][j] = wv;
            }
            __syncthreads();
            if (owner) {
                for (int pt = grp; pt < nb; pt += G::GROUPS) {
                    const int o = org[pt];
                    if (o != cur) {
                        if (cur >= 0) flush(cur, acc);
                        cur = o;
                    }
                    const T coef = w1s[pt][jb] * w2s[pt][jc];
                    fma_row<T, TAPS>(acc, coef, w0s[pt]);
                }
            }
            // FP32C carries the FP32 sums into fixed point every kCarry batches and at the chunk end
            const bool carry = FIXED && ((++bcount % kCarry) == 0 || base + B >= w.start + w.count);
            if (carry && owner && cur >= 0) flush(cur, acc);
            __syncthreads();
            if (carry) {
                // FP32C: carry the FP32 tile into fixed point and clear it
                for (int e = tid; e < PA3; e += NT) {
                    const T v = tile[e];
                    if (v != T(0)) {
                        itile[e] += (unsigned long long)to_fixed(v * fscale);
                        tile[e] = T(0);
                    }
                }
                __syncthreads();
            }
        }
        if (owner && cur >= 0 && !FIXED) flush(cur, acc);
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
                const T val = tile[e];
                if (val != T(0)) {
                    tile[e] = T(0);
                    if (ok) atomicAdd(reinterpret_cast<T *>(a.grid) + gidx, val);
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int M, int TE, bool FIXED>
static cudaError_t launch_cols(Plan &P, const Spread3Args &a) {
    using G = CellGeom<M, TE, FIXED ? 2 : 1>;
    auto kern = spread3_cells<T, M, TE, FIXED>;
    const int pa3 = G::PA * G::PA * G::PA;
    const int smem = ((pa3 * (int)sizeof(T) + 15) / 16) * 16 + (FIXED ? pa3 * 8 : 0);
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

cudaError_t launch_spread3_columns(Plan &P, const double *x, bool ones, bool scale_dinv) {
    Spread3Args a;
    a.pts = P.pts;
    a.perm = P.perm;
    a.x = x;
    a.dinv = scale_dinv ? P.dinv_sorted : nullptr;
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
    a.ones = ones ? 1 : 0;
    a.b = P.kb_b;
    a.inv_den = P.kb_inv_sinh_bm;
    if (P.prec == NFL_PREC_FP64) return dispatch_cols<double, false>(P, a);
    if (P.prec == NFL_PREC_FP32C) return dispatch_cols<float, true>(P, a);
    return dispatch_cols<float, false>(P, a);
}

}  // namespace nfl
