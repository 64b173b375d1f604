// Window spreading: the first half of the adjoint NFFT in Alg. 1 step 1,
//   h_t = sum_i x~_i prod_a phi(n v~_ia - t_a),   x~ = D_E^{-1/2} x (Alg. 2 step 5),
// onto the active box of the oversampled grid (n = 2N points per axis).
//
// Nodes are sorted into tiles of tile_edge^d cells.  A CTA takes one chunk of
// one tile, accumulates its nodes' (2m)^d taps in a shared-memory copy of the
// tile plus its halo ((tile_edge + 2m - 1)^d cells), then adds the non-zero
// cells to the global grid.  FP32C accumulates in 64-bit fixed point
// (value * 2^k rounded to an integer, k chosen per call from sum |x~| so that
// no partial sum can overflow): integer addition is exact and associative, so
// the long random-sign sums of dense clusters lose nothing.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

struct SpreadArgs {
    const void *pts;
    const int32_t *perm;
    const double *x;
    const double *dinv;          // sorted order, or nullptr
    const WorkItem *items;
    int64_t nitems;
    int ntile[3];
    int tile_edge, m, P;
    int L[3];
    int wrap[3];
    int ngrid;
    void *grid;
    const double *abs_sum;       // fixed point: device sum_i |x~_i|
    int ones;
    double b, inv_sinh_bm;
    int bf16;                    // BF16W: FP32 taps rounded to BF16
};

// 2^k with k the largest integer such that sum|x~| * 2^k < 2^62.
__device__ __forceinline__ double fixed_point_scale(double abs_sum) {
    if (!(abs_sum > 0.0)) return 1.0;
    int e;
    frexp(abs_sum, &e);          // abs_sum < 2^e
    int k = 62 - e;
    k = k > 120 ? 120 : (k < -120 ? -120 : k);     // 2^k stays a normal FP32 number
    return ldexp(1.0, k);
}

template <typename Acc>
__device__ __forceinline__ void shared_add(Acc *p, Acc v) { atomicAdd(p, v); }

// MT > 0: the cut-off m fixed at compile time (weights stay in registers);
// MT = 0: m read from the arguments.
template <typename T, int D, bool FIXED, int MT>
__global__ void __launch_bounds__(256) spread_kernel(SpreadArgs a) {
    using Acc = typename std::conditional<FIXED, unsigned long long, T>::type;
    using Pt = typename PointOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc *tile = reinterpret_cast<Acc *>(smem_raw);

    const int P = a.P;
    int Pd = P;
    if (D >= 2) Pd *= P;
    if (D >= 3) Pd *= P;
    const int m = MT > 0 ? MT : a.m;
    const int taps = 2 * m;
    const T tm = T(m), tb = T(a.b), tinv = T(a.inv_sinh_bm);
    T fscale = T(1);
    if (FIXED) fscale = T(fixed_point_scale(*a.abs_sum));
    const Pt *pts = reinterpret_cast<const Pt *>(a.pts);

    for (int64_t it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        int tc[3] = {0, 0, 0};
        tile_coords<D>(w.tile, a.ntile, tc);
        for (int e = threadIdx.x; e < Pd; e += blockDim.x) tile[e] = Acc(0);
        __syncthreads();

        for (int k = w.start + threadIdx.x; k < w.start + w.count; k += blockDim.x) {
            const Pt pt = pts[k];
            double xv = a.ones ? 1.0 : a.x[a.perm[k]];
            if (a.dinv) xv *= a.dinv[k];
            T wt[D][2 * (MT > 0 ? MT : kMaxM)];
            int s[3] = {0, 0, 0};
#pragma unroll
            for (int ax = 0; ax < D; ++ax) {
                s[ax] = cell_axis(pt.cell, ax) - tc[ax] * a.tile_edge;
                const T fr = T(pt.f[ax]);
#pragma unroll
                for (int j = 0; j < taps; ++j) {
                    wt[ax][j] = kb_weight<T>(fr + T(m - 1) - T(j), tm, tb, tinv);
                    if constexpr (std::is_same<T, float>::value)
                        if (a.bf16) wt[ax][j] = round_bf16(wt[ax][j]);
                }
            }
            const T xt = T(xv);
            if (D == 1) {
                for (int j0 = 0; j0 < taps; ++j0) {
                    const T val = xt * wt[0][j0];
                    if (FIXED) shared_add(&tile[s[0] + j0], (Acc)(unsigned long long)__double2ll_rn(double(val * fscale)));
                    else shared_add(&tile[s[0] + j0], (Acc)val);
                }
            } else if (D == 2) {
                for (int j0 = 0; j0 < taps; ++j0) {
                    const T w0 = xt * wt[0][j0];
                    Acc *row = tile + (s[0] + j0) * P + s[1];
                    for (int j1 = 0; j1 < taps; ++j1) {
                        const T val = w0 * wt[1][j1];
                        if (FIXED) shared_add(&row[j1], (Acc)(unsigned long long)__double2ll_rn(double(val * fscale)));
                        else shared_add(&row[j1], (Acc)val);
                    }
                }
            } else {
#pragma unroll 1
                for (int j0 = 0; j0 < taps; ++j0) {
                    const T w0 = xt * wt[0][j0];
#pragma unroll
                    for (int j1 = 0; j1 < taps; ++j1) {
                        const T w01 = w0 * wt[1][j1];
                        Acc *row = tile + ((s[0] + j0) * P + (s[1] + j1)) * P + s[2];
#pragma unroll
                        for (int j2 = 0; j2 < taps; ++j2) {
                            const T val = w01 * wt[2][j2];
                            if (FIXED) shared_add(&row[j2], (Acc)(unsigned long long)__double2ll_rn(double(val * fscale)));
                            else shared_add(&row[j2], (Acc)val);
                        }
                    }
                }
            }
        }
        __syncthreads();

        Acc *grid = reinterpret_cast<Acc *>(a.grid);
        for (int e = threadIdx.x; e < Pd; e += blockDim.x) {
            const Acc val = tile[e];
            if (val == Acc(0)) continue;
            int loc[3] = {0, 0, 0};
            int r = e;
            for (int ax = D - 1; ax >= 0; --ax) {
                loc[ax] = r % P;
                r /= P;
            }
            int64_t idx = 0;
            bool ok = true;
            for (int ax = 0; ax < D; ++ax) {
                int bpos = tc[ax] * a.tile_edge - (m - 1) + loc[ax];
                if (a.wrap[ax]) bpos = ((bpos % a.ngrid) + a.ngrid) % a.ngrid;
                ok = ok && bpos >= 0 && bpos < a.L[ax];
                idx = idx * a.L[ax] + bpos;
            }
            if (ok) atomicAdd(&grid[idx], val);
        }
        __syncthreads();
    }
}

__global__ void abs_sum_kernel(const double *x, const double *dinv, const int32_t *perm,
                               int64_t n, int ones, double *out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double v = ones ? 1.0 : fabs(x[perm[k]]);
        if (dinv) v *= dinv[k];
        acc += v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

static int spread_smem_bytes(const Plan &P, int elem) {
    int Pt = P.tile_edge + 2 * P.m - 1;
    int cells = Pt;
    for (int a = 1; a < P.d; ++a) cells *= Pt;
    return cells * elem;
}

template <typename T, int D, bool FIXED, int MT>
static cudaError_t launch_spread_m(Plan &P, SpreadArgs &a) {
    using Acc = typename std::conditional<FIXED, unsigned long long, T>::type;
    const int smem = spread_smem_bytes(P, sizeof(Acc));
    NFL_CUDA_TRY(cudaFuncSetAttribute(spread_kernel<T, D, FIXED, MT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spread_kernel<T, D, FIXED, MT>, 256, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > P.nitems) grid = P.nitems;
    if (grid < 1) return cudaSuccess;
    spread_kernel<T, D, FIXED, MT><<<(unsigned)grid, 256, smem, P.stream>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, bool FIXED>
static cudaError_t launch_spread_t(Plan &P, SpreadArgs &a) {
    if (D == 3) {
        switch (P.m) {
            case 2: return launch_spread_m<T, D, FIXED, 2>(P, a);
            case 3: return launch_spread_m<T, D, FIXED, 3>(P, a);
            case 4: return launch_spread_m<T, D, FIXED, 4>(P, a);
            case 6: return launch_spread_m<T, D, FIXED, 6>(P, a);
            case 7: return launch_spread_m<T, D, FIXED, 7>(P, a);
            case 8: return launch_spread_m<T, D, FIXED, 8>(P, a);
        }
    }
    return launch_spread_m<T, D, FIXED, 0>(P, a);
}

cudaError_t launch_fixed_scale(Plan &P, const double *x, bool ones, bool scale_dinv) {
    NFL_CUDA_TRY(cudaMemsetAsync(P.scratch, 0, sizeof(double), P.stream));
    int blocks = P.num_sms * 4;
    abs_sum_kernel<<<blocks, 256, 0, P.stream>>>(x, scale_dinv ? P.dinv_sorted : nullptr, P.perm,
                                                 P.n, ones ? 1 : 0, P.scratch);
    return cudaGetLastError();
}

cudaError_t clear_spread(Plan &P, int nc) {
    size_t elem = P.prec == NFL_PREC_FP32 ? sizeof(float) : 8;
    NFL_CUDA_TRY(cudaMemsetAsync(P.grid, 0, P.box_elems * elem * nc, P.stream));
    return cudaMemsetAsync(P.work_counter, 0, 4 * sizeof(unsigned), P.stream);
}

cudaError_t prepare_spread(Plan &P, int op, const double *x, int64_t ldx, int nc, bool ones, bool scale_dinv) {
    NFL_CUDA_TRY(clear_spread(P, nc));
    if (P.d == 3 && column_tile_edge(P.m) == P.tile_edge)
        return stage_spread3_values(P, op, x, ldx, nc, ones, scale_dinv);
    if (nc != 1) return cudaErrorInvalidValue;
    if (P.prec == NFL_PREC_FP32C) NFL_CUDA_TRY(launch_fixed_scale(P, x, ones, scale_dinv));
    return cudaSuccess;
}

cudaError_t launch_spread(Plan &P, const double *x, int64_t, bool ones, bool scale_dinv) {
    if (P.d == 3 && column_tile_edge(P.m) == P.tile_edge) {
        if (spread_warp_available(P)) return launch_spread3_warp(P);
        return launch_spread3_columns(P, x, ones, scale_dinv);
    }
    SpreadArgs a;
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
    a.tile_edge = P.tile_edge;
    a.m = P.m;
    a.P = P.tile_edge + 2 * P.m - 1;
    a.ngrid = P.ngrid;
    a.grid = P.grid;
    a.abs_sum = P.scratch;
    a.ones = ones ? 1 : 0;
    a.b = P.kb_b;
    a.inv_sinh_bm = P.kb_inv_sinh_bm;
    a.bf16 = P.bf16_taps ? 1 : 0;

    switch (P.prec * 4 + P.d) {
        case NFL_PREC_FP64 * 4 + 1: return launch_spread_t<double, 1, false>(P, a);
        case NFL_PREC_FP64 * 4 + 2: return launch_spread_t<double, 2, false>(P, a);
        case NFL_PREC_FP64 * 4 + 3: return launch_spread_t<double, 3, false>(P, a);
        case NFL_PREC_FP32 * 4 + 1: return launch_spread_t<float, 1, false>(P, a);
        case NFL_PREC_FP32 * 4 + 2: return launch_spread_t<float, 2, false>(P, a);
        case NFL_PREC_FP32 * 4 + 3: return launch_spread_t<float, 3, false>(P, a);
        case NFL_PREC_FP32C * 4 + 1: return launch_spread_t<float, 1, true>(P, a);
        case NFL_PREC_FP32C * 4 + 2: return launch_spread_t<float, 2, true>(P, a);
        case NFL_PREC_FP32C * 4 + 3: return launch_spread_t<float, 3, true>(P, a);
    }
    return cudaErrorInvalidValue;
}

}  // namespace nfl
