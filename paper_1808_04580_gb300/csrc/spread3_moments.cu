// Window spreading in 3-D for dense tiles, FP32 / FP32C, m = 6 (Alg. 1 step 1,
// the window half of the adjoint NFFT):
//   h_t = sum_i x~_i phi(n v~_i0 - t_0) phi(n v~_i1 - t_1) phi(n v~_i2 - t_2).
//
// Every node of one cell sees the same 12 x 12 x 12 support, and each of its 12
// taps per axis is a smooth function of the node's fractional offset f: in the
// Chebyshev basis T_k(t), t = 2 f - 1, tap j is sum_k C[j][k] T_k(t) with 8
// terms to within FP32 rounding of the window's peak (3.6e-8 of phi(0) at
// m = 6, from interpolation at 8 Chebyshev points; the plan holds C).  So the
// support block of cell s is
//   H_s[a][b][c] = sum_{k0,k1,k2} C[a][k0] C[b][k1] C[c][k2] M_s[k0][k1][k2],
//   M_s[k0][k1][k2] = sum_{i in s} x~_i T_k0(t_i0) T_k1(t_i1) T_k2(t_i2),
// 512 moments per node instead of 1728 taps.
//
// A CTA takes one slab of a dense tile (the 16 cells that share an axis-0
// position; the nodes of a tile are sorted by cell with axis 0 slowest, so a
// slab's nodes are contiguous), or a piece of one.  Its 8 warps take one
// eighth of the nodes each, in slices of 32: lane l accumulates the moments
// (k0, k1 = l / 4, k2 = 2 (l mod 4) + {0, 1}) for k0 < 8 as 8 pairs over
// (k0, k0 + 1), one fma.rn.f32x2 per pair and node, from the slice's staged
// Chebyshev rows (the rows of four nodes loaded together); when the cell
// changes the lanes add them to the cell's moments in shared memory.  Then the
// CTA expands the 16 cells' moments into
// the slab's 12 x 15 x 15 block in three contractions shared by the cells that
// overlap along each axis,
//   V2[k0][s1][k1][c] = sum_{s2, c'} C[c'][k2] M_{s1,s2}[k0][k1][k2],  c = s2 + c'
//   V1[k0][b][c]      = sum_{s1, b'} C[b'][k1] V2[k0][s1][k1][c],      b = s1 + b'
//   H[a][b][c]        = sum_k0 C[a][k0] V1[k0][b][c],
// 180,000 multiply-adds per slab instead of 29,000 per occupied cell, and adds
// the block to the global grid: FP32 atomics, or for FP32C 64-bit fixed point
// (scale 2^k from sum |x~|, so nothing can overflow) with integer atomics.
// FP32 moment sums are blocked: a lane sums a run segment of one slice (at most
// 32 nodes), then the segments of the cell in its eighth of the work item, and
// the cell's moments in shared memory add one such sum per warp.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

namespace {

constexpr int MM = 6, TE_M = 4, TAPS_M = 12, R = kCheb;
constexpr int PA_M = TE_M + 2 * MM - 1;                 // 15
constexpr int CELLS_M = TE_M * TE_M;                    // cells of a slab
constexpr int MST = R * R * R;                          // moments per cell
constexpr int NWM = 8, NTM = NWM * 32;                  // warps, threads per CTA
constexpr int ROW = 44;                                 // staged floats per node (odd multiple of 16 B)
constexpr int STAGE_M = NWM * 32 * ROW;                 // staged rows of all warps
constexpr int V2_M = R * TE_M * R * PA_M;               // 3840
constexpr int V1_M = R * PA_M * PA_M;                   // 1800
constexpr int SMEM_M = (CELLS_M * MST + STAGE_M) * 4;
static_assert(R == 8, "lane layout: 8 k1 x 4 lanes x 2 k2");
static_assert(V2_M + V1_M <= STAGE_M, "the expansion reuses the staging area");

struct MomentArgs {
    const PointF *pts;
    const float *xs;
    const WorkItem *items;  // pad = the slab (axis-0 cell position inside the tile)
    int64_t nitems;
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    void *grid;             // layout [x0][x1][x2]
    const double *abs_sum;
    unsigned *counter;
    float cheb[TAPS_M][R];
};

}  // namespace

// One staged node as lane (k1, c0) needs it: the (T_2p(t0), T_2p+1(t0)) pairs and
// the two coefficients (c, c), c = x~ T_k1(t1) T_c0+{0,1}(t2).
struct NodeRow {
    unsigned long long t0[R / 2], ca, cb;

    __device__ __forceinline__ void load(const float *rq, int k1, int c0) {
        const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(rq);
        const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(rq + 4);
        t0[0] = a0.x;
        t0[1] = a0.y;
        t0[2] = a1.x;
        t0[3] = a1.y;
        const unsigned long long xt = *reinterpret_cast<const unsigned long long *>(rq + 8 + 2 * k1);
        const ulonglong2 t2 = *reinterpret_cast<const ulonglong2 *>(rq + 24 + 2 * c0);
        ca = fmul2(xt, t2.x);
        cb = fmul2(xt, t2.y);
    }

    __device__ __forceinline__ void add(unsigned long long (&acc)[2][R / 2]) const {
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
            acc[0][p] = ffma2(t0[p], ca, acc[0][p]);
            acc[1][p] = ffma2(t0[p], cb, acc[1][p]);
        }
    }
};

template <bool FIXED>
__global__ void __launch_bounds__(NTM, 2) spread3_moments(MomentArgs a) {
    extern __shared__ __align__(16) float msm[];
    float *Mom = msm;                          // [cell s2 * 4 + s1][k0][k1][k2]
    float *stage_all = msm + CELLS_M * MST;    // [warp][32][ROW]; the expansion's V2, V1 after
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, tid = threadIdx.x;
    float *stage = stage_all + g * 32 * ROW;
    float *V2 = stage_all, *V1 = stage_all + V2_M;
    __shared__ __align__(16) float Cs[TAPS_M][R];
    __shared__ unsigned next_item;
    for (int e = tid; e < TAPS_M * R; e += NTM) Cs[e / R][e % R] = a.cheb[e / R][e % R];
    for (int e = tid; e < CELLS_M * MST; e += NTM) Mom[e] = 0.f;
    const float fscale = FIXED ? float(fixed_scale_of(*a.abs_sum)) : 1.f;
    const int k1 = lane >> 2, c0 = 2 * (lane & 3);

    for (;;) {
        // the CTA's next work item (largest first); the barrier also ends the previous
        // item's use of the staging area and its clearing of the moments
        if (tid == 0) next_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const int64_t it = next_item;
        if (it >= a.nitems) break;
        const WorkItem w = a.items[it];
        int tc[3];
        tile_coords<3>(w.tile, a.ntile, tc);
        const int end = w.start + w.count;

        // moments: warp g takes the g-th eighth of the item in slices of 32 nodes and
        // carries its sums across slices while the cell stays the same
        // acc sums one run segment of a slice (at most 32 nodes), accr the segments of the
        // current cell (blocked summation: the FP32 error grows with 32 + nodes / 32)
        unsigned long long acc[2][R / 2], accr[2][R / 2];
#pragma unroll
        for (int p = 0; p < R / 2; ++p) accr[0][p] = accr[1][p] = 0ull;
        const unsigned long long one2 = pack2(1.f, 1.f);
        int cur = -1;
        // the sums of cell cur into its moments; the accumulators start again from zero
        auto flush = [&]() {
            float *mrow = Mom + cur * MST + k1 * R + c0;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int p = 0; p < R / 2; ++p) {
                    atomicAdd(mrow + 2 * p * R * R + c, lane_of(accr[c][p], 0));
                    atomicAdd(mrow + (2 * p + 1) * R * R + c, lane_of(accr[c][p], 1));
                    accr[c][p] = 0ull;
                }
        };
        const int share = (w.count + NWM - 1) / NWM;
        const int gbeg = w.start + g * share, gend = min(end, gbeg + share);
        for (int base = gbeg; base < gend; base += 32) {
            const int cnt = min(32, gend - base);
            const bool valid = lane < cnt;
            int cell = 0;
            {
                PointF pn = {{0.5f, 0.5f, 0.5f}, 0};
                float xv = 0.f;
                if (valid) {
                    pn = a.pts[base + lane];
                    xv = a.xs[base + lane];
                    const int s1 = min(max(cell_axis(pn.cell, 1) - tc[1] * TE_M, 0), TE_M - 1);
                    const int s2 = min(max(cell_axis(pn.cell, 2) - tc[2] * TE_M, 0), TE_M - 1);
                    cell = s2 * TE_M + s1;
                }
                float T[3][R];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const float t = fmaf(2.f, pn.f[ax], -1.f), t2x = t + t;
                    T[ax][0] = 1.f;
                    T[ax][1] = t;
#pragma unroll
                    for (int k = 2; k < R; ++k) T[ax][k] = fmaf(t2x, T[ax][k - 1], -T[ax][k - 2]);
                }
                // row: T_k(t0), then (x~ T_k(t1), x~ T_k(t1)) and (T_k(t2), T_k(t2)) pairs
                float4 *r = reinterpret_cast<float4 *>(stage + lane * ROW);
                r[0] = make_float4(T[0][0], T[0][1], T[0][2], T[0][3]);
                r[1] = make_float4(T[0][4], T[0][5], T[0][6], T[0][7]);
#pragma unroll
                for (int j = 0; j < R / 2; ++j) {
                    const float u0 = xv * T[1][2 * j], u1 = xv * T[1][2 * j + 1];
                    r[2 + j] = make_float4(u0, u0, u1, u1);
                    r[6 + j] = make_float4(T[2][2 * j], T[2][2 * j], T[2][2 * j + 1], T[2][2 * j + 1]);
                }
            }
            const int prev = __shfl_up_sync(0xffffffffu, cell, 1);
            const unsigned runs = __ballot_sync(0xffffffffu, valid && (lane == 0 || cell != prev));
            __syncwarp();
            int i = 0;
            while (i < cnt) {
                const unsigned rest = i + 1 < 32 ? (runs >> (i + 1)) : 0u;
                const int j = rest ? min(cnt, i + __ffs(rest)) : cnt;
                const int ci = __shfl_sync(0xffffffffu, cell, i);
                if (ci != cur) {
                    if (cur >= 0) flush();
                    cur = ci;
                }
                // acc[c][p] = sum over the segment of (T_2p(t0), T_2p+1(t0)) x~ T_k1(t1) T_c0+c(t2)
#pragma unroll
                for (int p = 0; p < R / 2; ++p) acc[0][p] = acc[1][p] = 0ull;
                int q = i;
                // four nodes' rows loaded before their multiply-adds
                for (; q + 4 <= j; q += 4) {
                    NodeRow d[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) d[u].load(stage + (q + u) * ROW, k1, c0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) d[u].add(acc);
                }
                for (; q < j; ++q) {
                    NodeRow d;
                    d.load(stage + q * ROW, k1, c0);
                    d.add(acc);
                }
#pragma unroll
                for (int p = 0; p < R / 2; ++p) {
                    accr[0][p] = ffma2(acc[0][p], one2, accr[0][p]);
                    accr[1][p] = ffma2(acc[1][p], one2, accr[1][p]);
                }
                i = j;
            }
            __syncwarp();                             // the next slice overwrites the staged rows
        }
        if (cur >= 0) flush();
        __syncthreads();

        // V2[k0][s1][k1][c] = sum_{s2, c'} C[c'][k2] M_{s1,s2}[k0][k1][k2] (c = s2 + c'):
        // thread (k0, s1, k1)
        {
            const int k0 = tid >> 5, s1 = (tid >> 3) & 3, kk1 = tid & 7;
            float v2[PA_M];
#pragma unroll
            for (int c = 0; c < PA_M; ++c) v2[c] = 0.f;
#pragma unroll
            for (int s2 = 0; s2 < TE_M; ++s2) {
                const float *mp = Mom + (s2 * TE_M + s1) * MST + (k0 * R + kk1) * R;
                const float4 ma = *reinterpret_cast<const float4 *>(mp);
                const float4 mb = *reinterpret_cast<const float4 *>(mp + 4);
                const float m[R] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
#pragma unroll
                for (int cp = 0; cp < TAPS_M; ++cp)
#pragma unroll
                    for (int k = 0; k < R; ++k) v2[s2 + cp] = fmaf(Cs[cp][k], m[k], v2[s2 + cp]);
            }
            float *dst = V2 + ((k0 * TE_M + s1) * R + kk1) * PA_M;
#pragma unroll
            for (int c = 0; c < PA_M; ++c) dst[c] = v2[c];
        }
        __syncthreads();
        // the moments are consumed: clear them for the next item (ordered before its
        // sums by the barrier at the top of the loop)
        for (int e = tid; e < CELLS_M * MST / 4; e += NTM)
            reinterpret_cast<float4 *>(Mom)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        // V1[k0][b][c] = sum_{s1, b'} C[b'][k1] V2[k0][s1][k1][c] (b = s1 + b'): thread (k0, c)
        if (tid < R * PA_M) {
            const int k0 = tid / PA_M, c = tid - k0 * PA_M;
            float v1[PA_M];
#pragma unroll
            for (int b = 0; b < PA_M; ++b) v1[b] = 0.f;
#pragma unroll
            for (int s1 = 0; s1 < TE_M; ++s1) {
                float v[R];
#pragma unroll
                for (int k = 0; k < R; ++k) v[k] = V2[((k0 * TE_M + s1) * R + k) * PA_M + c];
#pragma unroll
                for (int bp = 0; bp < TAPS_M; ++bp)
#pragma unroll
                    for (int k = 0; k < R; ++k) v1[s1 + bp] = fmaf(Cs[bp][k], v[k], v1[s1 + bp]);
            }
#pragma unroll
            for (int b = 0; b < PA_M; ++b) V1[(k0 * PA_M + b) * PA_M + c] = v1[b];
        }
        __syncthreads();
        // H[a][b][c] = sum_k0 C[a][k0] V1[k0][b][c] into the global grid: thread (b, c);
        // a warp's atomics of one a fall on consecutive positions along axis 2
        if (tid < PA_M * PA_M) {
            const int b = tid / PA_M, c = tid - b * PA_M;
            float v[R];
#pragma unroll
            for (int k = 0; k < R; ++k) v[k] = V1[(k * PA_M + b) * PA_M + c];
            int p1 = tc[1] * TE_M - (MM - 1) + b, p2 = tc[2] * TE_M - (MM - 1) + c;
            if (a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
            if (a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
            if (p1 >= 0 && p1 < a.L[1] && p2 >= 0 && p2 < a.L[2]) {
                const int o0 = tc[0] * TE_M - (MM - 1) + w.pad;
#pragma unroll
                for (int aa = 0; aa < TAPS_M; ++aa) {
                    float h = 0.f;
#pragma unroll
                    for (int k = 0; k < R; ++k) h = fmaf(Cs[aa][k], v[k], h);
                    int p0 = o0 + aa;
                    if (a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (h == 0.f || p0 < 0 || p0 >= a.L[0]) continue;
                    const int64_t gidx = ((int64_t)p0 * a.L[1] + p1) * a.L[2] + p2;
                    if (FIXED)
                        atomicAdd(reinterpret_cast<unsigned long long *>(a.grid) + gidx,
                                  (unsigned long long)to_fixed(h * fscale));
                    else
                        atomicAdd(reinterpret_cast<float *>(a.grid) + gidx, h);
                }
            }
        }
    }
}

template <bool FIXED>
static cudaError_t launch_moments(Plan &P, const MomentArgs &a, cudaStream_t s) {
    auto kern = spread3_moments<FIXED>;
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_M));
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTM, SMEM_M));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > a.nitems) grid = a.nitems;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, NTM, SMEM_M, s>>>(a);
    return cudaGetLastError();
}

// The dense tiles' slab pieces of a one-column spread (the warp-slice kernel takes the rest).
cudaError_t launch_spread3_moments(Plan &P, cudaStream_t s) {
    if (P.nslab == 0) return cudaSuccess;
    MomentArgs a{};
    a.pts = reinterpret_cast<const PointF *>(P.pts);
    a.xs = static_cast<const float *>(P.xsort);
    a.items = P.slab_items;
    a.nitems = P.nslab;
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
    return P.prec == NFL_PREC_FP32C ? launch_moments<true>(P, a, s) : launch_moments<false>(P, a, s);
}

}  // namespace nfl
