// Interpolation back to the nodes, the second half of the NFFT in Alg. 1
// step 3,  f_j = sum_t g_t prod_a phi(n v~_ja - t_a),  with the epilogue of
// the requested product fused in (K(0) = 1 for the Gaussian):
//   W  : y_j = f_j - x_j                                 (W = W~ - K(0) I, Sec. 3)
//   A  : y_j = dinv_j (f_j - x~_j),  x~ = dinv x         (Alg. 2 step 5)
//   L_s: y_j = x_j - dinv_j (f_j - x~_j)                  (Sec. 2, eq. (nomlap))
//   deg: d_j = f_j - 1 with x = 1; dinv_j = d_j^{-1/2}    (Alg. 2 step 4)
// A CTA loads one tile of g plus halo into shared memory and interpolates
// the nodes of one chunk of that tile.  The tap sum is nested per axis
// (sum_a w_a sum_b w_b sum_c w_c g), which keeps FP32 rounding to a few
// ulps of each partial sum.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

struct GatherArgs {
    const void *pts;
    const int32_t *perm;
    const double *x;
    double *y;
    const double *dinv;   // sorted order
    double *degree_out;   // input order (OP_DEGREE)
    double *dinv_out;     // sorted order (OP_DEGREE)
    const WorkItem *items;
    int64_t nitems;
    int ntile[3];
    int tile_edge, m, P;
    int L[3];
    int wrap[3];
    int ngrid;
    const void *g;        // reversed-axis layout: index (..(x_{d-1} L_{d-2} + ..) L_0 + x_0)
    int op;
    double out_scale, k0;   // W x = out_scale f - K(0) x (caller's coordinates)
    double b, inv_sinh_bm;
    int bf16;                    // BF16W: FP32 taps rounded to BF16
};

// MT > 0: the cut-off m fixed at compile time; MT = 0: m from the arguments.
template <typename T, typename TG, int D, int MT>
__global__ void __launch_bounds__(256) gather_kernel(GatherArgs a) {
    using Pt = typename PointOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    const int P = a.P;
    int Pd = P;
    if (D >= 2) Pd *= P;
    if (D >= 3) Pd *= P;
    const int m = MT > 0 ? MT : a.m;
    const int taps = 2 * m;
    const T tm = T(m), tb = T(a.b), tinv = T(a.inv_sinh_bm);
    const Pt *pts = reinterpret_cast<const Pt *>(a.pts);
    const TG *g = reinterpret_cast<const TG *>(a.g);

    for (int64_t it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        int tc[3] = {0, 0, 0};
        tile_coords<D>(w.tile, a.ntile, tc);
        // load with the global grid's fastest axis (axis 0) fastest
        for (int e = threadIdx.x; e < Pd; e += blockDim.x) {
            int loc[3] = {0, 0, 0};
            int r = e;
            for (int ax = 0; ax < D; ++ax) {
                loc[ax] = r % P;
                r /= P;
            }
            int64_t gidx = 0;
            bool ok = true;
            for (int ax = D - 1; ax >= 0; --ax) {
                int bpos = tc[ax] * a.tile_edge - (m - 1) + loc[ax];
                if (a.wrap[ax]) bpos = ((bpos % a.ngrid) + a.ngrid) % a.ngrid;
                ok = ok && bpos >= 0 && bpos < a.L[ax];
                gidx = gidx * a.L[ax] + bpos;
            }
            int sidx = 0;
            for (int ax = 0; ax < D; ++ax) sidx = sidx * P + loc[ax];
            tile[sidx] = ok ? T(g[gidx]) : T(0);
        }
        __syncthreads();

        for (int k = w.start + threadIdx.x; k < w.start + w.count; k += blockDim.x) {
            const Pt pt = pts[k];
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
            T f = T(0);
            if (D == 1) {
                for (int j0 = 0; j0 < taps; ++j0) f += wt[0][j0] * tile[s[0] + j0];
            } else if (D == 2) {
                for (int j0 = 0; j0 < taps; ++j0) {
                    const T *row = tile + (s[0] + j0) * P + s[1];
                    T acc = T(0);
                    for (int j1 = 0; j1 < taps; ++j1) acc += wt[1][j1] * row[j1];
                    f += wt[0][j0] * acc;
                }
            } else {
#pragma unroll 1
                for (int j0 = 0; j0 < taps; ++j0) {
                    T acc0 = T(0);
#pragma unroll
                    for (int j1 = 0; j1 < taps; ++j1) {
                        const T *row = tile + ((s[0] + j0) * P + (s[1] + j1)) * P + s[2];
                        T acc1 = T(0);
#pragma unroll
                        for (int j2 = 0; j2 < taps; ++j2) acc1 += wt[2][j2] * row[j2];
                        acc0 += wt[1][j1] * acc1;
                    }
                    f += wt[0][j0] * acc0;
                }
            }
            const int i = a.perm[k];
            const double fd = double(f);
            if (a.op == OP_DEGREE) {
                const double dd = a.out_scale * fd - a.k0;
                a.degree_out[i] = dd;
                a.dinv_out[k] = dd > 0.0 ? 1.0 / sqrt(dd) : 0.0;
            } else if (a.op == OP_W) {
                a.y[i] = a.out_scale * fd - a.k0 * a.x[i];
            } else {
                const double di = a.dinv[k];
                const double xi = a.x[i];
                const double ax = di * (a.out_scale * fd - a.k0 * di * xi);
                a.y[i] = a.op == OP_A ? ax : xi - ax;
            }
        }
        __syncthreads();
    }
}

template <typename T, typename TG, int D, int MT>
static cudaError_t launch_gather_m(Plan &P, GatherArgs &a) {
    int Pt = P.tile_edge + 2 * P.m - 1;
    int cells = Pt;
    for (int i = 1; i < D; ++i) cells *= Pt;
    const int smem = cells * (int)sizeof(T);
    NFL_CUDA_TRY(cudaFuncSetAttribute(gather_kernel<T, TG, D, MT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_kernel<T, TG, D, MT>, 256, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > P.nitems) grid = P.nitems;
    if (grid < 1) return cudaSuccess;
    gather_kernel<T, TG, D, MT><<<(unsigned)grid, 256, smem, P.stream>>>(a);
    return cudaGetLastError();
}

template <typename T, typename TG, int D>
static cudaError_t launch_gather_t(Plan &P, GatherArgs &a) {
    if (D == 3) {
        switch (P.m) {
            case 2: return launch_gather_m<T, TG, D, 2>(P, a);
            case 3: return launch_gather_m<T, TG, D, 3>(P, a);
            case 4: return launch_gather_m<T, TG, D, 4>(P, a);
            case 6: return launch_gather_m<T, TG, D, 6>(P, a);
            case 7: return launch_gather_m<T, TG, D, 7>(P, a);
            case 8: return launch_gather_m<T, TG, D, 8>(P, a);
        }
    }
    return launch_gather_m<T, TG, D, 0>(P, a);
}

cudaError_t launch_gather(Plan &P, int op, const double *x, double *y) {
    if (gather_tc_available(P)) return launch_gather_tc(P, op, x, y);
    GatherArgs a;
    a.pts = P.pts;
    a.perm = P.perm;
    a.x = x;
    a.y = y;
    a.dinv = P.dinv_sorted;
    a.degree_out = P.degree;
    a.dinv_out = P.dinv_sorted;
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
    a.g = P.g;
    a.op = op;
    a.out_scale = P.out_scale;
    a.k0 = P.k0;
    a.b = P.kb_b;
    a.inv_sinh_bm = P.kb_inv_sinh_bm;
    a.bf16 = P.bf16_taps ? 1 : 0;
    switch (P.prec * 4 + P.d) {
        case NFL_PREC_FP64 * 4 + 1: return launch_gather_t<double, double, 1>(P, a);
        case NFL_PREC_FP64 * 4 + 2: return launch_gather_t<double, double, 2>(P, a);
        case NFL_PREC_FP64 * 4 + 3: return launch_gather_t<double, double, 3>(P, a);
        case NFL_PREC_FP32 * 4 + 1: return launch_gather_t<float, float, 1>(P, a);
        case NFL_PREC_FP32 * 4 + 2: return launch_gather_t<float, float, 2>(P, a);
        case NFL_PREC_FP32 * 4 + 3: return launch_gather_t<float, float, 3>(P, a);
        case NFL_PREC_FP32C * 4 + 1: return launch_gather_t<float, float, 1>(P, a);
        case NFL_PREC_FP32C * 4 + 2: return launch_gather_t<float, float, 2>(P, a);
        case NFL_PREC_FP32C * 4 + 3: return launch_gather_t<float, float, 3>(P, a);
    }
    return cudaErrorInvalidValue;
}

}  // namespace nfl
