// Window spreading in 3-D for dense cells, FP32 / FP32C, m = 6 (Alg. 1 step 1,
// the window half of the adjoint NFFT):
//   h_t = sum_i x~_i phi(n v~_i0 - t_0) phi(n v~_i1 - t_1) phi(n v~_i2 - t_2).
//
// Every node of one cell sees the same 12 x 12 x 12 support, and each of its 12
// taps per axis is a smooth function of the node's fractional offset f: in the
// Chebyshev basis T_k(t), t = 2 f - 1, tap j is sum_k C[j][k] T_k(t) with 8
// terms to within FP32 rounding of the window's peak (3.6e-8 of phi(0) at
// m = 6, from interpolation at 8 Chebyshev points; the plan holds C).  So the
// support block of a cell is
//   H[a][b][c] = sum_{k0,k1,k2} C[a][k0] C[b][k1] C[c][k2] M[k0][k1][k2],
//   M[k0][k1][k2] = sum_{i in cell} x~_i T_k0(t_i0) T_k1(t_i1) T_k2(t_i2),
// 512 moments per node instead of 1728 taps, and the three small products with
// C once per cell.  Tiles whose nodes number at least kDenseCell per occupied
// cell take this kernel; the others keep the warp-slice kernel.
//
// Layout (one CTA per work item = chunk of one tile, 4 warps, each warp the
// g-th quarter of the chunk in slices of 32 nodes, as the warp-slice kernel):
// lane l accumulates the moments (k0, k1 = l / 4, k2 = 2 (l mod 4) + {0, 1})
// for k0 < 8 as 8 packed pairs over its two k2, one fma.rn.f32x2 per k0 and
// node.  Lane i stages node i of a slice: (T_k(t0), T_k(t0)) pairs, the pairs
// (x~ T_k(t1), x~ T_k(t1)) and T_k(t2).  When the cell changes the warp turns
// its moments into the 12^3 block (axis 0 in registers, axes 1 and 2 through
// shared memory) and adds it to its tile copy; the tile copies are merged into
// the global grid at the end of the chunk exactly as in the warp-slice kernel
// (FP32C: 64-bit fixed point, scale 2^k from sum |x~|).
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

namespace {

constexpr int MM = 6, TE_M = 4, TAPS_M = 12, R = kCheb;
constexpr int PA_M = TE_M + 2 * MM - 1;                 // 15
constexpr int PA3_M = PA_M * PA_M * PA_M;
constexpr int TILE_M = (PA3_M + 3) / 4 * 4;
constexpr int NGM = 4, SM_ = 32;
constexpr int kMomentRun = 256;                         // most nodes summed into one set of moments
constexpr int ROW = 44;                                 // staged floats per node (odd multiple of 16 B)
constexpr int A_STRIDE = 72, B_STRIDE = 104;            // transform buffer strides (conflict-free)
constexpr int BUF = TAPS_M * B_STRIDE;                  // 1248 floats
constexpr int WARP_FLOATS = TILE_M + SM_ * ROW + BUF;
constexpr int SMEM_M = NGM * WARP_FLOATS * 4;
static_assert(R == 8, "lane layout: 8 k1 x 4 lanes x 2 k2");
static_assert(12 * A_STRIDE <= BUF, "buffer holds both stages");
static_assert((WARP_FLOATS * 4) % 16 == 0, "16-byte aligned per-warp areas");

struct MomentArgs {
    const PointF *pts;
    const float *xs;
    const WorkItem *items;
    int64_t nitems;
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    void *grid;
    const double *abs_sum;
    unsigned *counter;
    float cheb[TAPS_M][R];
};

}  // namespace

template <bool FIXED>
__global__ void __launch_bounds__(NGM * 32, 2) spread3_moments(MomentArgs a) {
    extern __shared__ __align__(16) float msm[];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    float *tile = msm + g * WARP_FLOATS;
    float *stage = tile + TILE_M;             // [S][ROW]
    float *buf = stage + SM_ * ROW;           // transform stages
    __shared__ __align__(16) float2 Cd[TAPS_M][R];      // (C[a][k], C[a][k])
    __shared__ __align__(16) float2 Cc[TAPS_M / 2][R];  // (C[2p][k], C[2p + 1][k])
    __shared__ __align__(16) float Cs[TAPS_M][R];
    __shared__ unsigned next_item;
    for (int e = threadIdx.x; e < TAPS_M * R; e += NGM * 32) {
        const int j = e / R, k = e - j * R;
        const float c = a.cheb[j][k];
        Cd[j][k] = make_float2(c, c);
        Cs[j][k] = c;
        if ((j & 1) == 0) Cc[j / 2][k] = make_float2(c, a.cheb[j + 1][k]);
    }
    for (int e = lane; e < TILE_M; e += 32) tile[e] = 0.f;
    const float fscale = FIXED ? float(fixed_scale_of(*a.abs_sum)) : 1.f;
    __syncthreads();

    const int k1 = lane >> 2, c0 = 2 * (lane & 3);
    unsigned long long acc[R];                // (M[k][k1][c0], M[k][k1][c0 + 1])
    bool fresh = true;

    // the moments of cell o -> its 12^3 support block, added to this warp's tile copy
    auto flush = [&](int o) {
        if (fresh) return;                    // nothing summed since the last flush (warp-uniform)
        const int s0 = o & 255, s1 = (o >> 8) & 255, s2 = o >> 16;
        __syncwarp();
        {
            // axis 0 in registers: H0[a][k1][k2] = sum_k C[a][k] M[k][k1][k2] (this lane's two k2)
            const unsigned long long *cd = reinterpret_cast<const unsigned long long *>(&Cd[0][0]);
#pragma unroll
            for (int aa = 0; aa < TAPS_M; ++aa) {
                unsigned long long v = fmul2(cd[aa * R], acc[0]);
#pragma unroll
                for (int k = 1; k < R; ++k) v = ffma2(cd[aa * R + k], acc[k], v);
                *reinterpret_cast<unsigned long long *>(buf + aa * A_STRIDE + k1 * 8 + c0) = v;
            }
        }
        __syncwarp();
        // axis 1: lane (k2, three rows a): H1[a][b][k2] = sum_k1 C[b][k1] H0[a][k1][k2]
        const int k2 = lane & 7, ab = 3 * (lane >> 3);
        float h1[3][TAPS_M];
        {
            float h[3][R];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < R; ++k) h[i][k] = buf[(ab + i) * A_STRIDE + k * 8 + k2];
#pragma unroll
            for (int b = 0; b < TAPS_M; ++b) {
                const float4 cl = *reinterpret_cast<const float4 *>(&Cs[b][0]);
                const float4 ch = *reinterpret_cast<const float4 *>(&Cs[b][4]);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float v = cl.x * h[i][0];
                    v = fmaf(cl.y, h[i][1], v);
                    v = fmaf(cl.z, h[i][2], v);
                    v = fmaf(cl.w, h[i][3], v);
                    v = fmaf(ch.x, h[i][4], v);
                    v = fmaf(ch.y, h[i][5], v);
                    v = fmaf(ch.z, h[i][6], v);
                    v = fmaf(ch.w, h[i][7], v);
                    h1[i][b] = v;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int b = 0; b < TAPS_M; ++b) buf[(ab + i) * B_STRIDE + b * 8 + k2] = h1[i][b];
        __syncwarp();
        // axis 2 and the tile: rows (a, b) of the block, columns c in pairs
        const unsigned long long *cc = reinterpret_cast<const unsigned long long *>(&Cc[0][0]);
        for (int p = lane; p < TAPS_M * TAPS_M; p += 32) {
            const int aa = p / TAPS_M, b = p - aa * TAPS_M;
            const float4 q0 = *reinterpret_cast<const float4 *>(buf + aa * B_STRIDE + b * 8);
            const float4 q1 = *reinterpret_cast<const float4 *>(buf + aa * B_STRIDE + b * 8 + 4);
            const unsigned long long hd[R] = {pack2(q0.x, q0.x), pack2(q0.y, q0.y), pack2(q0.z, q0.z),
                                              pack2(q0.w, q0.w), pack2(q1.x, q1.x), pack2(q1.y, q1.y),
                                              pack2(q1.z, q1.z), pack2(q1.w, q1.w)};
            float *row = tile + ((s0 + aa) * PA_M + s1 + b) * PA_M + s2;
#pragma unroll
            for (int cp = 0; cp < TAPS_M / 2; ++cp) {
                unsigned long long v = fmul2(cc[cp * R], hd[0]);
#pragma unroll
                for (int k = 1; k < R; ++k) v = ffma2(cc[cp * R + k], hd[k], v);
                row[2 * cp] += lane_of(v, 0);
                row[2 * cp + 1] += lane_of(v, 1);
            }
        }
        fresh = true;
    };

    // node q of the staged slice into the moments: acc[k] (+)= (T_k(t0), T_k(t0)) * coef,
    // coef = x~ T_k1(t1) (T_c0(t2), T_c0+1(t2))
    auto node = [&](int q, auto init) {
        constexpr bool INIT = decltype(init)::value;
        const float *r = stage + q * ROW;
        const unsigned long long xt = *reinterpret_cast<const unsigned long long *>(r + 16 + 2 * k1);
        const unsigned long long t2 = *reinterpret_cast<const unsigned long long *>(r + 32 + c0);
        const unsigned long long coef = fmul2(xt, t2);
        const ulonglong2 *t0 = reinterpret_cast<const ulonglong2 *>(r);
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            const ulonglong2 v = t0[j];
            acc[2 * j] = INIT ? fmul2(v.x, coef) : ffma2(v.x, coef, acc[2 * j]);
            acc[2 * j + 1] = INIT ? fmul2(v.y, coef) : ffma2(v.y, coef, acc[2 * j + 1]);
        }
    };

    for (;;) {
        // the CTA's next work item (largest first)
        if (threadIdx.x == 0) next_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const int64_t it = next_item;
        if (it >= a.nitems) break;
        const WorkItem w = a.items[it];
        int tc[3];
        tile_coords<3>(w.tile, a.ntile, tc);
        int cur = -1, since = 0;
        // this warp's quarter of the chunk; this lane's node of the next slice, loaded one slice ahead
        const int share = (w.count + NGM - 1) / NGM;
        int base = w.start + g * share;
        const int gend = min(w.start + w.count, base + share);
        PointF pn = {{0.f, 0.f, 0.f}, 0};
        float xn = 0.f;
        if (base + lane < gend) {
            pn = a.pts[base + lane];
            xn = a.xs[base + lane];
        }
        for (; base < gend; base += SM_) {
            const int cnt = min(SM_, gend - base);
            const bool valid = lane < cnt;
            int o = 0;
            {
                // stage node `lane` of the slice: its cell and its Chebyshev rows
                float T[3][R];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const int sa = valid ? cell_axis(pn.cell, ax) - tc[ax] * TE_M : 0;
                    o |= sa << (8 * ax);
                    const float t = valid ? fmaf(2.f, pn.f[ax], -1.f) : 0.f;
                    const float t2x = t + t;
                    T[ax][0] = 1.f;
                    T[ax][1] = t;
#pragma unroll
                    for (int k = 2; k < R; ++k) T[ax][k] = fmaf(t2x, T[ax][k - 1], -T[ax][k - 2]);
                }
                const float xv = valid ? xn : 0.f;
                const int kn = base + SM_ + lane;
                if (kn < gend) {
                    pn = a.pts[kn];
                    xn = a.xs[kn];
                }
                float4 *r = reinterpret_cast<float4 *>(stage + lane * ROW);
#pragma unroll
                for (int j = 0; j < R / 2; ++j) {
                    r[j] = make_float4(T[0][2 * j], T[0][2 * j], T[0][2 * j + 1], T[0][2 * j + 1]);
                    const float u0 = xv * T[1][2 * j], u1 = xv * T[1][2 * j + 1];
                    r[4 + j] = make_float4(u0, u0, u1, u1);
                }
                r[8] = make_float4(T[2][0], T[2][1], T[2][2], T[2][3]);
                r[9] = make_float4(T[2][4], T[2][5], T[2][6], T[2][7]);
            }
            const int prev = __shfl_up_sync(0xffffffffu, o, 1);
            const unsigned runs = __ballot_sync(0xffffffffu, valid && (lane == 0 || o != prev));
            __syncwarp();
            int i = 0;
            while (i < cnt) {
                const unsigned rest = i + 1 < 32 ? (runs >> (i + 1)) : 0u;
                const int j = rest ? min(cnt, i + __ffs(rest)) : cnt;
                const int oi = __shfl_sync(0xffffffffu, o, i);
                if (oi != cur) {
                    if (cur >= 0) flush(cur);
                    cur = oi;
                    since = 0;
                }
                int q = i;
                if (fresh) node(q++, std::true_type{});
#pragma unroll 2
                for (; q < j; ++q) node(q, std::false_type{});
                fresh = false;
                i = j;
            }
            __syncwarp();                             // the next slice overwrites the staged rows
            // no FP32 moment sum runs over more than kMomentRun nodes: a long run of one
            // cell is expanded and carried into the tile copy in pieces
            since += cnt;
            if (since >= kMomentRun && cur >= 0) {
                flush(cur);
                since = 0;
            }
        }
        if (cur >= 0) flush(cur);
        __syncthreads();
        // sum the tile copies -> global grid (fixed point for FP32C), clear them
        {
            const int b0 = tc[0] * TE_M - (MM - 1), b1 = tc[1] * TE_M - (MM - 1), b2 = tc[2] * TE_M - (MM - 1);
            for (int e = threadIdx.x; e < PA3_M; e += NGM * 32) {
                float v = 0.f;
#pragma unroll
                for (int gg = 0; gg < NGM; ++gg) {
                    float *t = msm + gg * WARP_FLOATS + e;
                    v += *t;
                    *t = 0.f;
                }
                if (v == 0.f) continue;
                const int q2 = e % PA_M, q1 = (e / PA_M) % PA_M, q0 = e / (PA_M * PA_M);
                int p0 = b0 + q0, p1 = b1 + q1, p2 = b2 + q2;
                if (a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                if (a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
                if (a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
                if (p0 < 0 || p0 >= a.L[0] || p1 < 0 || p1 >= a.L[1] || p2 < 0 || p2 >= a.L[2]) continue;
                const int64_t gidx = ((int64_t)p0 * a.L[1] + p1) * a.L[2] + p2;
                if (FIXED)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.grid) + gidx,
                              (unsigned long long)to_fixed(v * fscale));
                else
                    atomicAdd(reinterpret_cast<float *>(a.grid) + gidx, v);
            }
        }
        __syncthreads();
    }
}

template <bool FIXED>
static cudaError_t launch_moments(Plan &P, const MomentArgs &a) {
    auto kern = spread3_moments<FIXED>;
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_M));
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NGM * 32, SMEM_M));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > P.ndense) grid = P.ndense;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, NGM * 32, SMEM_M, P.stream>>>(a);
    return cudaGetLastError();
}

// The dense tiles' chunks of a one-column spread (the warp-slice kernel takes the rest).
cudaError_t launch_spread3_moments(Plan &P) {
    if (P.ndense == 0) return cudaSuccess;
    MomentArgs a{};
    a.pts = reinterpret_cast<const PointF *>(P.pts);
    a.xs = static_cast<const float *>(P.xsort);
    a.items = P.dense_items;
    a.nitems = P.ndense;
    for (int i = 0; i < 3; ++i) {
        a.ntile[i] = P.ntile[i];
        a.L[i] = P.L[i];
        a.wrap[i] = P.wrap[i];
    }
    a.ngrid = P.ngrid;
    a.grid = P.grid;
    a.abs_sum = P.scratch;
    a.counter = P.work_counter + 2;
    for (int j = 0; j < TAPS_M; ++j)
        for (int k = 0; k < R; ++k) a.cheb[j][k] = P.kb_cheb[j][k];
    return P.prec == NFL_PREC_FP32C ? launch_moments<true>(P, a) : launch_moments<false>(P, a);
}

}  // namespace nfl
