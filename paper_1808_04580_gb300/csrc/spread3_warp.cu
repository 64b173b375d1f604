// Window spreading in 3-D, FP32 / FP32C, one warp per node slice
// (Alg. 1 step 1, the window half of the adjoint NFFT):
//   h_t = sum_i x~_i phi(n v~_i0 - t_0) phi(n v~_i1 - t_1) phi(n v~_i2 - t_2).
//
// The plan sorts the nodes of every tile by cell, so the nodes of one cell
// are contiguous; they share the whole (2M)^3 support.  A CTA of NG warps
// takes one chunk of one tile (TE^3 cells); every warp owns a copy of the
// tile plus halo (PA = TE + 2M - 1 per axis) in shared memory.  Warp g takes
// the g-th quarter of the chunk's nodes, in slices of 32, so the warps of a
// CTA finish a chunk together.
//
// Per slice, lane i stages node i: its tile-local cell, the 3 x 2M window
// taps (the plan's per-tap polynomials, Horner in t = 2f - 1 with two taps
// per fma.rn.f32x2; x~ folded into the axis-1 taps), written once per node.
// A warp ballot marks the cell runs.  For the accumulation, LPB lanes share
// a support row jb of axis 1 and each owns CPL interleaved columns jc of axis 2;
// a lane keeps 2M x CPL accumulators as pairs of adjacent rows ja and adds,
// per node, (c, c) * (w0[ja], w0[ja + 1]) with c = w1[jb] w2[jc], one
// fma.rn.f32x2 per pair and column.  Every multiply-add lands in the
// support, with no range tests and no shared-memory traffic besides the
// staged taps.
// When the cell changes, the lanes add their accumulators to the warp's
// tile copy with plain read-modify-write: in one flush the lanes touch
// distinct positions, and __syncwarp orders consecutive flushes.
//
// At the end of the chunk the CTA sums the NG tile copies; FP32 adds each
// non-zero sum to the global grid with an FP32 atomic, FP32C converts it to
// 64-bit fixed point (scale 2^k from sum |x~|, so nothing can overflow) and
// adds it with an integer atomic.  So FP32C sums at most 8192 / NG nodes of a
// tile position in FP32 (2048 for NG = 4) before the exact integer part.
//
// A work item may also be a run of tiles that follow each other along axis 2
// (at most 8192 nodes together).  The tile copies then slide along the run:
// axis 2 of a copy is addressed circularly (slot = (q2 + woff) mod PA), and
// between two tiles the CTA merges only the TE planes q2 < TE that the next
// tile's window does not cover, clears them (they become its last TE planes)
// and advances woff by TE.  The full merge follows the last tile.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace nfl {

struct SpreadWarpArgs {
    const PointF *pts;
    const float *xs;                // x~ in sorted order, column c at xs + c * xs_stride
    const WorkItem *items;
    int64_t nitems;                 // items of one column; the grid takes nitems * ncol
    int ncol;                       // columns of a block product (item it: item it / ncol, column it % ncol)
    int64_t xs_stride, grid_stride;
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    void *grid;
    const double *abs_sum;          // column c: abs_sum[c]
    const int32_t *tile_start;      // first sorted node of each tile
    unsigned *counter;              // next work item, shared by all CTAs
    int bf16;                       // BF16W: taps rounded to BF16
    const BatchPlanDev *bplans;     // batch: the members (item it is bitems[it] of member bitems[it].plan)
    const BatchItem *bitems;
    float poly[2 * kMaxM][kPolyCoef];
};

// box extent of axis i of the current item's plan
#define SW_L(i) (BATCH ? ip.L[i] : a.L[i])

template <int M, int TE>
struct WarpGeom {
    static constexpr int PA = TE + 2 * M - 1;
    static constexpr int PA3 = PA * PA * PA;
    static constexpr int TAPS = 2 * M;
    static constexpr int LPB = M == 6 ? 2 : (M == 4 ? 4 : (M == 3 ? 3 : 2));   // lanes per support row jb
    static constexpr int CPL = TAPS / LPB;        // support columns per lane
    static constexpr int RP = TAPS / 2;           // row pairs (ja, ja + 1)
    // FULLB: the lanes cover all PA rows of axis 1 of the tile (when they fit in a
    // warp), so a cell run is a whole (axis 0, axis 2) column of the tile and the
    // flushes are TE times rarer; otherwise the 2M support rows of one cell
    static constexpr bool FULLB = PA * LPB <= 32;
    static constexpr int JB = FULLB ? PA : TAPS;  // axis-1 rows covered by the lanes
    static constexpr int LANES = JB * LPB;        // lanes that accumulate
    static constexpr int NG = 4;                  // warps (tile copies) per CTA
    static constexpr int S = 32;                  // nodes per slice
    static constexpr int TILE = (PA3 + 3) / 4 * 4;
    // per node, rows of staged taps (axes 0, 1, 2) whose strides are odd multiples
    // of 16 bytes, so the 16-byte stores of the 32 lanes fall in distinct bank groups
    static constexpr int R1 = ((TAPS + 3) / 4) % 2 ? (TAPS + 3) / 4 * 4 : (TAPS + 3) / 4 * 4 + 4;   // floats per row
    // axis-1 rows: the taps placed over all JB rows for FULLB
    static constexpr int RB = FULLB ? (JB + 3) / 4 * 4 : R1;
    static constexpr int W_BYTES = S * R1 * 4;
    static constexpr int WB_BYTES = S * RB * 4;
    static constexpr int WARP_BYTES = TILE * 4 + 2 * W_BYTES + WB_BYTES;
    static constexpr int SMEM = NG * WARP_BYTES;
    static_assert(LANES <= 32 && CPL % 2 == 0, "lane layout");
    static_assert(WARP_BYTES % 16 == 0, "16-byte aligned per-warp areas");
};

// Per-item plan fields of a batch, in shared memory (written by thread 0 per item).
struct SpreadItemPlan {
    const PointF *pts;
    const int32_t *tile_start;
    int ntile[3], L[3], wrap[3];
};

// BLOCK: a block product of a.ncol columns (item, column pairs); otherwise one column.
// BATCH (with BLOCK): the items of all members of a batch, each item's plan fields
// read from its member's descriptor.
template <int M, int TE, bool FIXED, bool BLOCK, bool BATCH = false>
__global__ void __launch_bounds__(WarpGeom<M, TE>::NG * 32, 3) spread3_warp(SpreadWarpArgs a) {
    using G = WarpGeom<M, TE>;
    constexpr int PA = G::PA, PA3 = G::PA3, TAPS = G::TAPS, RP = G::RP, CPL = G::CPL, S = G::S, NG = G::NG,
                  R1 = G::R1, RB = G::RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    unsigned char *mine = smem_raw + g * G::WARP_BYTES;
    float *tile = reinterpret_cast<float *>(mine);
    float *w0s = reinterpret_cast<float *>(mine + G::TILE * 4);                     // [S][R1]
    float *w2s = reinterpret_cast<float *>(mine + G::TILE * 4 + G::W_BYTES);       // [S][R1]
    float *w1s = reinterpret_cast<float *>(mine + G::TILE * 4 + 2 * G::W_BYTES);   // [S][RB]
    __shared__ __align__(16) float2 polys[M][kPolyCoef];
    __shared__ unsigned next_item;

    const bool acc_lane = lane < G::LANES;
    const int jb = acc_lane ? lane / G::LPB : 0;   // support row of the cell, or tile row for FULLB
    // columns jc = c * LPB + hseg, c < CPL: interleaved, so that in a flush the
    // lanes (30 for m = 6) address different shared-memory banks
    const int hseg = acc_lane ? lane - jb * G::LPB : 0;
    for (int e = threadIdx.x; e < M * kPolyCoef; e += NG * 32) {
        const int q = e / kPolyCoef, k = e - q * kPolyCoef;
        polys[q][k] = make_float2(a.poly[2 * q][k], a.poly[2 * q + 1][k]);
    }
    for (int e = lane; e < G::TILE; e += 32) tile[e] = 0.f;
    __shared__ float fscales[kBlockCols];           // FP32C scale 2^k of each column of a block
    if (FIXED && BLOCK && !BATCH && threadIdx.x < a.ncol)
        fscales[threadIdx.x] = float(fixed_scale_of(a.abs_sum[threadIdx.x]));
    __shared__ SpreadItemPlan ip;
    __shared__ WorkItem bw;
    __shared__ float bscale;
    __shared__ const float *bxs;
    __shared__ void *bgrid;
    float fscale1 = 1.f;                            // the one column's
    if (FIXED && !BLOCK) fscale1 = float(fixed_scale_of(*a.abs_sum));
    __syncthreads();

    unsigned long long acc[RP][CPL];              // (ja, ja + 1) pairs for each column jc
    bool fresh = true;                            // the next node starts the accumulators

    int woff = 0;                                 // circular offset of axis 2 in the tile copies
    // add the accumulators of cell o to this warp's tile copy
    auto flush = [&](int o) {
        __syncwarp();
        if (acc_lane) {
            const int s0 = o & 255, s1 = G::FULLB ? 0 : (o >> 8) & 255, s2 = o >> 16;
            float *row = tile + (s0 * PA + s1 + jb) * PA;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                int q = s2 + hseg + c * G::LPB + woff;   // < 2 PA
                if (q >= PA) q -= PA;
#pragma unroll
                for (int p = 0; p < RP; ++p) {
                    row[(2 * p) * PA * PA + q] += lane_of(acc[p][c], 0);
                    row[(2 * p + 1) * PA * PA + q] += lane_of(acc[p][c], 1);
                }
            }
        }
        fresh = true;
    };

    // one node's taps into the accumulators: (c, c) * (w0[ja], w0[ja + 1]), c = w1[jb] w2[jc];
    // INIT sets them (first node after a flush), otherwise adds
    auto node = [&](int q, auto init) {
        constexpr bool INIT = decltype(init)::value;
        const float w1v = w1s[q * RB + jb];
        const float2 *r2 = reinterpret_cast<const float2 *>(w2s + q * R1 + hseg * CPL);
        unsigned long long coef[CPL];
#pragma unroll
        for (int c2 = 0; c2 < CPL / 2; ++c2) {
            const float2 v = r2[c2];
            const float c0 = w1v * v.x, c1 = w1v * v.y;
            coef[2 * c2] = pack2(c0, c0);
            coef[2 * c2 + 1] = pack2(c1, c1);
        }
        const unsigned long long *r0 = reinterpret_cast<const unsigned long long *>(w0s + q * R1);
#pragma unroll
        for (int p2 = 0; p2 < (RP + 1) / 2; ++p2) {
            unsigned long long wv[2];
            if (2 * p2 + 1 < RP) {
                const ulonglong2 w2v = reinterpret_cast<const ulonglong2 *>(r0)[p2];
                wv[0] = w2v.x;
                wv[1] = w2v.y;
            } else {
                wv[0] = r0[2 * p2];
                wv[1] = 0ull;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (2 * p2 + u >= RP) continue;
#pragma unroll
                for (int c = 0; c < CPL; ++c)
                    acc[2 * p2 + u][c] = INIT ? fmul2(coef[c], wv[u]) : ffma2(coef[c], wv[u], acc[2 * p2 + u][c]);
            }
        }
    };

    for (;;) {
        // the CTA's next work item (largest first: the plan sorts them by size)
        if (threadIdx.x == 0) {
            next_item = atomicAdd(a.counter, 1u);
            if (BATCH && (int64_t)next_item < a.nitems * a.ncol) {
                // the member of this item and its fields
                const unsigned it0 = next_item / (unsigned)a.ncol;
                const int c0 = (int)(next_item - it0 * (unsigned)a.ncol);
                const BatchItem e = a.bitems[it0];
                const BatchPlanDev &D = a.bplans[e.plan];
                bw = D.sitems[e.item];
                ip.pts = D.pts;
                ip.tile_start = D.tile_start;
                for (int i = 0; i < 3; ++i) {
                    ip.ntile[i] = D.ntile[i];
                    ip.L[i] = D.L[i];
                    ip.wrap[i] = D.wrap[i];
                }
                bxs = D.xs + c0 * D.n;
                bscale = FIXED ? float(fixed_scale_of(D.abs_sum[c0])) : 1.f;
                bgrid = FIXED ? (void *)(reinterpret_cast<unsigned long long *>(D.grid) + c0 * D.box)
                              : (void *)(reinterpret_cast<float *>(D.grid) + c0 * D.box);
            }
        }
        __syncthreads();
        const int64_t itc = next_item;
        if (itc >= a.nitems * (BLOCK ? a.ncol : 1)) break;
        const int64_t it = BLOCK ? (int64_t)((unsigned)itc / (unsigned)a.ncol) : itc;
        const int col = BLOCK ? (int)(itc - it * a.ncol) : 0;
        const float *xs = BATCH ? bxs : (BLOCK ? a.xs + col * a.xs_stride : a.xs);
        const float fscale = !FIXED ? 1.f : (BATCH ? bscale : (BLOCK ? fscales[col] : fscale1));
        void *const gridc = BATCH ? bgrid
                          : !BLOCK ? a.grid
                                   : FIXED ? (void *)(reinterpret_cast<unsigned long long *>(a.grid) + col * a.grid_stride)
                                           : (void *)(reinterpret_cast<float *>(a.grid) + col * a.grid_stride);
        const WorkItem w = BATCH ? bw : a.items[it];
        const int wend = w.start + w.count;
        const int ntl = w.pad;                    // tiles in the item (a run along axis 2), or 1
        // lane l holds the first node of tile w.tile + l of a run (l <= ntl <= 31)
        const int lane_start = (ntl > 1 && lane <= ntl) ? (BATCH ? ip.tile_start : a.tile_start)[w.tile + lane] : 0;
        woff = 0;
        for (int jt = 0; jt < ntl; ++jt) {
            const int tile_id = w.tile + jt;
            int tc[3];
            tile_coords<3>(tile_id, BATCH ? ip.ntile : a.ntile, tc);
            int cur = -1;
            // this tile's nodes: the chunk, or the whole tile within a run
            const int run_s = __shfl_sync(0xffffffffu, lane_start, jt);
            const int run_e = __shfl_sync(0xffffffffu, lane_start, jt + 1);
            const int tstart = ntl == 1 ? w.start : run_s;
            const int tend = ntl == 1 ? wend : run_e;
            // this warp's share of them; this lane's node of the next slice, loaded one slice ahead
            const int share = (tend - tstart + NG - 1) / NG;
            int base = tstart + g * share;
            const int gend = min(tend, base + share);
            PointF pn = {{0.f, 0.f, 0.f}, 0};
            float xn = 0.f;
            if (base + lane < gend) {
                pn = (BATCH ? ip.pts : a.pts)[base + lane];
                xn = xs[base + lane];
            }
            for (; base < gend; base += S) {
                const int cnt = min(S, gend - base);
                const bool valid = lane < cnt;
                int o = 0;
                {
                    // stage node `lane` of the slice
                    float f[3];
                    int s1 = 0;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const int sa = valid ? cell_axis(pn.cell, ax) - tc[ax] * TE : 0;
                        if (ax == 1) s1 = sa;
                        if (ax != 1 || !G::FULLB) o |= sa << (8 * ax);     // FULLB runs ignore axis 1
                        f[ax] = valid ? pn.f[ax] : 0.f;
                    }
                    const float xv = xn;
                    const int kn = base + S + lane;
                    if (kn < gend) {
                        pn = (BATCH ? ip.pts : a.pts)[kn];
                        xn = xs[kn];
                    }
                    const unsigned long long T0 = pack2(fmaf(2.f, f[0], -1.f), fmaf(2.f, f[0], -1.f));
                    const unsigned long long T1 = pack2(fmaf(2.f, f[1], -1.f), fmaf(2.f, f[1], -1.f));
                    const unsigned long long T2 = pack2(fmaf(2.f, f[2], -1.f), fmaf(2.f, f[2], -1.f));
                    const unsigned long long *pc = reinterpret_cast<const unsigned long long *>(&polys[0][0]);
                    float t0[TAPS], t1[TAPS], t2[TAPS];
#pragma unroll
                    for (int q = 0; q < M; ++q) {
                        unsigned long long h0 = pc[q * kPolyCoef + kPolyCoef - 1], h1 = h0, h2 = h0;
#pragma unroll
                        for (int k = kPolyCoef - 2; k >= 0; --k) {
                            const unsigned long long c = pc[q * kPolyCoef + k];
                            h0 = ffma2(h0, T0, c);
                            h1 = ffma2(h1, T1, c);
                            h2 = ffma2(h2, T2, c);
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            float w0 = lane_of(h0, u), w1 = lane_of(h1, u), w2 = lane_of(h2, u);
                            if (a.bf16) {
                                w0 = round_bf16(w0);
                                w1 = round_bf16(w1);
                                w2 = round_bf16(w2);
                            }
                            t0[2 * q + u] = w0;
                            t1[2 * q + u] = w1 * xv;
                            t2[2 * q + u] = w2;
                        }
                    }
                    // 16-byte stores of this lane's rows
                    float4 *r0 = reinterpret_cast<float4 *>(w0s + lane * R1);
                    float4 *r1 = reinterpret_cast<float4 *>(w1s + lane * RB);
                    float4 *r2 = reinterpret_cast<float4 *>(w2s + lane * R1);
#pragma unroll
                    for (int j = 0; j < (TAPS + 3) / 4; ++j) {
                        float v0[4], v2[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const bool in = 4 * j + u < TAPS;
                            v0[u] = in ? t0[(4 * j + u) % TAPS] : 0.f;
                            // axis 2 de-interleaved: position h CPL + c holds tap c LPB + h
                            const int r = (4 * j + u) % TAPS;
                            v2[u] = in ? t2[(r % CPL) * G::LPB + r / CPL] : 0.f;
                        }
                        r0[j] = make_float4(v0[0], v0[1], v0[2], v0[3]);
                        r2[j] = make_float4(v2[0], v2[1], v2[2], v2[3]);
                    }
                    // axis 1: FULLB places the taps at the node's tile row s1 (selects, no indexing)
#pragma unroll
                    for (int j = 0; j < RB / 4; ++j) {
                        float v1[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int row = 4 * j + u;
                            float val = 0.f;
                            if (G::FULLB) {
#pragma unroll
                                for (int d = 0; d < TE; ++d)
                                    if (row - d >= 0 && row - d < TAPS) val = (s1 == d) ? t1[row - d] : val;
                            } else if (row < TAPS) {
                                val = t1[row];
                            }
                            v1[u] = val;
                        }
                        r1[j] = make_float4(v1[0], v1[1], v1[2], v1[3]);
                    }
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
                    }
                    if (acc_lane) {
                        int q = i;
                        if (fresh) node(q++, std::true_type{});
#pragma unroll 2
                        for (; q < j; ++q) node(q, std::false_type{});
                    }
                    fresh = false;
                    i = j;
                }
                __syncwarp();                         // the next slice overwrites the staged taps
            }
            if (cur >= 0) flush(cur);
            __syncthreads();
            if (jt + 1 < ntl) {
                // the TE planes q2 < TE leave the window: merge and clear them, slide by TE
                constexpr int NLEAVE = PA * PA * TE;
                const int b0 = tc[0] * TE - (M - 1), b1 = tc[1] * TE - (M - 1), b2 = tc[2] * TE - (M - 1);
                for (int e = threadIdx.x; e < NLEAVE; e += NG * 32) {
                    const int q = e % TE, r = e / TE;
                    const int q1 = r % PA, q0 = r / PA;
                    int slot = woff + q;
                    if (slot >= PA) slot -= PA;
                    const int pos = (q0 * PA + q1) * PA + slot;
                    float v = 0.f;
#pragma unroll
                    for (int gg = 0; gg < NG; ++gg) {
                        float *t = reinterpret_cast<float *>(smem_raw + gg * G::WARP_BYTES) + pos;
                        v += *t;
                        *t = 0.f;
                    }
                    if (v == 0.f) continue;
                    int p0 = b0 + q0, p1 = b1 + q1, p2 = b2 + q;
                    if (BATCH ? ip.wrap[0] : a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (BATCH ? ip.wrap[1] : a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (BATCH ? ip.wrap[2] : a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (p0 < 0 || p0 >= SW_L(0) || p1 < 0 || p1 >= SW_L(1) || p2 < 0 || p2 >= SW_L(2)) continue;
                    const int64_t gidx = ((int64_t)p0 * SW_L(1) + p1) * SW_L(2) + p2;
                    if (FIXED)
                        atomicAdd(reinterpret_cast<unsigned long long *>(gridc) + gidx,
                                  (unsigned long long)to_fixed(v * fscale));
                    else
                        atomicAdd(reinterpret_cast<float *>(gridc) + gidx, v);
                }
                woff += TE;
                if (woff >= PA) woff -= PA;
                __syncthreads();
                continue;
            }
            // sum the tile copies -> global grid, clear them.  Consecutive threads take
            // consecutive positions (c fastest, the grid's x2 axis), so the atomics of a
            // warp fall on a few contiguous rows of the grid rather than one per sector.
            {
                constexpr int STEP = NG * 32;
                int e = threadIdx.x;
                int q2 = e % PA, q1 = (e / PA) % PA, q0 = e / (PA * PA);
                const int b0 = tc[0] * TE - (M - 1), b1 = tc[1] * TE - (M - 1), b2 = tc[2] * TE - (M - 1);
                for (; e < PA3; e += STEP) {
                    float v = 0.f;
#pragma unroll
                    for (int gg = 0; gg < NG; ++gg) {
                        float *t = reinterpret_cast<float *>(smem_raw + gg * G::WARP_BYTES) + e;
                        v += *t;
                        *t = 0.f;
                    }
                    int lq2 = q2 - woff;                      // local axis-2 plane of this slot
                    if (lq2 < 0) lq2 += PA;
                    int p0 = b0 + q0, p1 = b1 + q1, p2 = b2 + lq2;
                    // advance (q0, q1, q2) by STEP positions
                    q2 += STEP % PA;
                    q1 += (STEP / PA) % PA;
                    q0 += STEP / (PA * PA);
                    if (q2 >= PA) { q2 -= PA; ++q1; }
                    if (q1 >= PA) { q1 -= PA; ++q0; }
                    if (v == 0.f) continue;
                    if (BATCH ? ip.wrap[0] : a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (BATCH ? ip.wrap[1] : a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (BATCH ? ip.wrap[2] : a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
                    if (p0 < 0 || p0 >= SW_L(0) || p1 < 0 || p1 >= SW_L(1) || p2 < 0 || p2 >= SW_L(2)) continue;
                    const int64_t gidx = ((int64_t)p0 * SW_L(1) + p1) * SW_L(2) + p2;
                    if (FIXED)
                        atomicAdd(reinterpret_cast<unsigned long long *>(gridc) + gidx,
                                  (unsigned long long)to_fixed(v * fscale));
                    else
                        atomicAdd(reinterpret_cast<float *>(gridc) + gidx, v);
                }
            }
            __syncthreads();
        }
    }
}

template <int M, int TE, bool FIXED>
static cudaError_t launch_warp(Plan &P, const SpreadWarpArgs &a) {
    using G = WarpGeom<M, TE>;
    auto kern = a.ncol > 1 ? spread3_warp<M, TE, FIXED, true> : spread3_warp<M, TE, FIXED, false>;
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NG * 32, G::SMEM));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > a.nitems * a.ncol) grid = a.nitems * a.ncol;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, G::NG * 32, G::SMEM, P.stream>>>(a);
    return cudaGetLastError();
}

template <int M, int TE, bool FIXED>
static cudaError_t launch_warp_batch(Batch &B, const SpreadWarpArgs &a, cudaStream_t s) {
    using G = WarpGeom<M, TE>;
    auto kern = spread3_warp<M, TE, FIXED, true, true>;
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NG * 32, G::SMEM));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * B.num_sms;
    if (grid > B.nsitems * a.ncol) grid = B.nsitems * a.ncol;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, G::NG * 32, G::SMEM, s>>>(a);
    return cudaGetLastError();
}

// The spread of every member of a batch in one launch: (item, column) pairs of all
// members from one counter, items largest first.
cudaError_t launch_spread3_warp_batch(Batch &B, cudaStream_t s) {
    SpreadWarpArgs a{};
    a.ncol = B.ncol;
    a.nitems = B.nsitems;
    a.bitems = B.sitems;
    a.bplans = B.desc;
    a.ngrid = 2 * B.N;
    a.counter = B.counter;
    a.bf16 = B.bf16 ? 1 : 0;
    for (int j = 0; j < 2 * kMaxM; ++j)
        for (int k = 0; k < kPolyCoef; ++k) a.poly[j][k] = B.poly[j][k];
    const bool fixed = B.prec == NFL_PREC_FP32C;
    switch (B.m) {
        case 2: return fixed ? launch_warp_batch<2, 8, true>(B, a, s) : launch_warp_batch<2, 8, false>(B, a, s);
        case 3: return fixed ? launch_warp_batch<3, 8, true>(B, a, s) : launch_warp_batch<3, 8, false>(B, a, s);
        case 4: return fixed ? launch_warp_batch<4, 8, true>(B, a, s) : launch_warp_batch<4, 8, false>(B, a, s);
        case 6: return fixed ? launch_warp_batch<6, 4, true>(B, a, s) : launch_warp_batch<6, 4, false>(B, a, s);
    }
    return cudaErrorInvalidValue;
}

bool spread_warp_available(const Plan &P) {
    if (P.d != 3 || P.prec == NFL_PREC_FP64 || P.tile_edge != column_tile_edge(P.m)) return false;
    return P.m == 2 || P.m == 3 || P.m == 4 || P.m == 6;
}

cudaError_t launch_spread3_warp(Plan &P, int nc) {
    SpreadWarpArgs a;
    a.ncol = nc;
    a.xs_stride = P.n;
    a.grid_stride = P.box_elems;
    a.pts = reinterpret_cast<const PointF *>(P.pts);
    a.xs = static_cast<const float *>(P.xsort);
    // one column with the dense-cell spread: the warp-slice kernel takes the sparse tiles
    const bool split = nc == 1 && moments_available(P);
    a.items = split ? P.sparse_items : P.sitems;
    a.nitems = split ? P.nsparse : P.nsitems;
    a.tile_start = P.tile_start;
    for (int i = 0; i < 3; ++i) {
        a.ntile[i] = P.ntile[i];
        a.L[i] = P.L[i];
        a.wrap[i] = P.wrap[i];
    }
    a.ngrid = P.ngrid;
    a.grid = P.grid;
    a.abs_sum = P.scratch;
    a.counter = P.work_counter;
    a.bf16 = P.bf16_taps ? 1 : 0;
    for (int j = 0; j < 2 * kMaxM; ++j)
        for (int k = 0; k < kPolyCoef; ++k) a.poly[j][k] = P.kb_poly[j][k];
    const bool fixed = P.prec == NFL_PREC_FP32C;
    switch (P.m) {
        case 2: return fixed ? launch_warp<2, 8, true>(P, a) : launch_warp<2, 8, false>(P, a);
        case 3: return fixed ? launch_warp<3, 8, true>(P, a) : launch_warp<3, 8, false>(P, a);
        case 4: return fixed ? launch_warp<4, 8, true>(P, a) : launch_warp<4, 8, false>(P, a);
        case 6:
            if (!split) return fixed ? launch_warp<6, 4, true>(P, a) : launch_warp<6, 4, false>(P, a);
            // the sparse tiles on the plan's stream, the dense tiles' slabs beside them
            NFL_CUDA_TRY(side_fork(P));
            NFL_CUDA_TRY((fixed ? launch_warp<6, 4, true>(P, a) : launch_warp<6, 4, false>(P, a)));
            NFL_CUDA_TRY(launch_spread3_moments(P, P.side ? P.side : P.stream));
            return side_join(P);
    }
    return cudaErrorInvalidValue;
}

}  // namespace nfl
