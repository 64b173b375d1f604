// Window spreading in 3-D without atomics in the inner loop (Alg. 1 step 1,
// spreading half of the adjoint NFFT):
//   h_t = sum_i x~_i phi(n v~_i0 - t_0) phi(n v~_i1 - t_1) phi(n v~_i2 - t_2).
//
// A CTA takes one chunk of one tile of TE^3 cells.  The tile with its halo
// spans PA = TE + 2M - 1 grid positions per axis.  Thread (b, c) owns the
// two grid columns t_1 = b, t_2 = c, c + 1 (c even) and keeps their 2 PA
// values along t_0 in registers (the checks, coefficients and row loads of a
// node are shared by both columns).  Nodes are handled in batches of 32: the CTA stages each
// node's 3 x 2M window weights in shared memory (axis-0 weights placed at
// their offset in a zero-padded row of length PA), then every thread whose
// column lies under a node's support adds
//   coef * w0row[a],  coef = x~ * w1[b - s1] * w2[c - s2],   a = 0..PA-1,
// to its registers: PA fused multiply-adds per node and column, in node
// order, with no shared-memory atomics.  At the end of the chunk each column
// adds its PA values to the global grid (one atomic per non-zero cell).
//
// FP32C: after every batch the FP32 partial sums are converted to 64-bit
// fixed point (scale 2^k from sum |x~|, as in the generic kernel) and added to
// thread-private int64 slots in shared memory, so everything beyond a 32-node
// partial sum is exact and the result does not depend on the order of the
// global atomics.
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

template <int M, int TE>
struct ColGeom {
    static constexpr int PA = TE + 2 * M - 1;
    static constexpr int PA4 = (PA + 3) / 4 * 4;
    static constexpr int CP = (PA + 1) / 2;              // column pairs per row b
    static constexpr int OWN = PA * CP;                  // threads owning a pair (b, c0..c0+1)
    static constexpr int NT = (OWN + 31) / 32 * 32;
    static constexpr int B = 32;
};

template <typename T, int M, int TE, bool FIXED>
__global__ void __launch_bounds__(ColGeom<M, TE>::NT) spread3_columns(Spread3Args a) {
    using G = ColGeom<M, TE>;
    constexpr int PA = G::PA, PA4 = G::PA4, CP = G::CP, B = G::B, TAPS = 2 * M, NT = G::NT;
    using Pt = typename PointOf<T>::type;
    __shared__ __align__(16) T w0row[B][PA4];
    __shared__ T w1s[B][TAPS], w2s[B][TAPS];
    __shared__ T frs[B][3];
    __shared__ T xs[B];
    __shared__ int ss[B][3];
    // FP32C: exact int64 partial sums per owned cell, [q][half][thread] (thread-private slots)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long *iacc = reinterpret_cast<long long *>(smem_raw);

    const int tid = threadIdx.x;
    const bool owner = tid < G::OWN;
    const int cb = owner ? tid / CP : 0;
    const int c0 = owner ? 2 * (tid % CP) : 0;
    const bool has1 = owner && c0 + 1 < PA;
    const T tm = T(M), tb = T(a.b), tden = T(a.inv_den);
    const Pt *pts = reinterpret_cast<const Pt *>(a.pts);
    T fscale = T(1);
    if (FIXED) fscale = T(fixed_scale_of(*a.abs_sum));
    if (FIXED)
        for (int e = tid; e < PA * 2 * NT; e += NT) iacc[e] = 0;

    for (int64_t it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        int tc[3];
        tile_coords<3>(w.tile, a.ntile, tc);
        T acc0[PA], acc1[PA];
#pragma unroll
        for (int q = 0; q < PA; ++q) { acc0[q] = T(0); acc1[q] = T(0); }

        for (int base = w.start; base < w.start + w.count; base += B) {
            const int nb = min(B, w.start + w.count - base);
            for (int e = tid; e < B * PA4; e += NT) (&w0row[0][0])[e] = T(0);
            if (tid < nb) {
                const int k = base + tid;
                const Pt p = pts[k];
                double xv = a.ones ? 1.0 : a.x[a.perm[k]];
                if (a.dinv) xv *= a.dinv[k];
                xs[tid] = T(xv);
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    ss[tid][ax] = cell_axis(p.cell, ax) - tc[ax] * TE;
                    frs[tid][ax] = T(p.f[ax]);
                }
            }
            __syncthreads();
            for (int e = tid; e < nb * 3 * TAPS; e += NT) {
                const int pt = e / (3 * TAPS);
                const int r = e - pt * 3 * TAPS;
                const int ax = r / TAPS;
                const int j = r - ax * TAPS;
                const T wv = kb_weight<T>(frs[pt][ax] + T(M - 1) - T(j), tm, tb, tden);
                if (ax == 0) w0row[pt][ss[pt][0] + j] = wv;
                else if (ax == 1) w1s[pt][j] = wv * xs[pt];   // x~ folded into the axis-1 window
                else w2s[pt][j] = wv;
            }
            __syncthreads();
            if (owner) {
                for (int pt = 0; pt < nb; ++pt) {
                    const int jb = cb - ss[pt][1];
                    if ((unsigned)jb >= (unsigned)TAPS) continue;
                    const int jc = c0 - ss[pt][2];
                    const bool in0 = (unsigned)jc < (unsigned)TAPS;
                    const bool in1 = has1 && (unsigned)(jc + 1) < (unsigned)TAPS;
                    if (!in0 && !in1) continue;
                    const T w1v = w1s[pt][jb];
                    const T k0 = in0 ? w1v * w2s[pt][jc] : T(0);
                    const T k1 = in1 ? w1v * w2s[pt][jc + 1] : T(0);
                    fma_row2<T, PA>(acc0, acc1, k0, k1, w0row[pt]);
                }
                if (FIXED) {
#pragma unroll
                    for (int q = 0; q < PA; ++q) {
                        iacc[(q * 2 + 0) * NT + tid] += to_fixed(acc0[q] * fscale);
                        iacc[(q * 2 + 1) * NT + tid] += to_fixed(acc1[q] * fscale);
                        acc0[q] = T(0);
                        acc1[q] = T(0);
                    }
                }
            }
            __syncthreads();
        }

        if (owner) {
            const int b0 = tc[0] * TE - (M - 1);
            int p1 = tc[1] * TE - (M - 1) + cb;
            if (a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && !has1) break;
                int p2 = tc[2] * TE - (M - 1) + c0 + half;
                if (a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
                const bool ok12 = p1 >= 0 && p1 < a.L[1] && p2 >= 0 && p2 < a.L[2];
#pragma unroll
                for (int q = 0; q < PA; ++q) {
                    int p0 = b0 + q;
                    if (a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                    const bool ok = ok12 && p0 >= 0 && p0 < a.L[0];
                    const int64_t idx = ((int64_t)p0 * a.L[1] + p1) * a.L[2] + p2;
                    if (FIXED) {
                        long long &slot = iacc[(q * 2 + half) * NT + tid];
                        if (ok && slot != 0)
                            atomicAdd(reinterpret_cast<unsigned long long *>(a.grid) + idx, (unsigned long long)slot);
                        slot = 0;
                    } else {
                        const T v = half == 0 ? acc0[q] : acc1[q];
                        if (ok && v != T(0)) atomicAdd(reinterpret_cast<T *>(a.grid) + idx, v);
                    }
                }
            }
        }
    }
}

template <typename T, int M, int TE, bool FIXED>
static cudaError_t launch_cols(Plan &P, const Spread3Args &a) {
    using G = ColGeom<M, TE>;
    auto kern = spread3_columns<T, M, TE, FIXED>;
    const int smem = FIXED ? G::PA * 2 * G::NT * (int)sizeof(long long) : 0;
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
