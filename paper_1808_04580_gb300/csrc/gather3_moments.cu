// Interpolation in 3-D for dense tiles, FP32 / FP32C, m = 6 (Alg. 1 step 3,
// the window half of the NFFT), with the epilogues of Alg. 2 step 5:
//   f_i = sum_{a,b,c} w0_i(a) w1_i(b) w2_i(c) g[s_i + (a, b, c)].
//
// With the taps in the Chebyshev basis, w(j; f) = sum_k C[j][k] T_k(2 f - 1)
// (8 terms, the plan's C as in the dense-cell spread), the sum over the 12^3
// support block G_s of cell s becomes
//   f_i = sum_{k0,k1,k2} T_k0(t_i0) T_k1(t_i1) T_k2(t_i2) Gt_s[k0][k1][k2],
//   Gt_s = (C^T x C^T x C^T) G_s,
// so a node costs 512 multiply-adds against its cell's 8^3 moments.
//
// A CTA forms the moments of a whole slab at once: the 16 cells of one tile
// that share an axis-0 position (the nodes of a tile are sorted by cell with
// axis 0 slowest, so a slab's nodes are contiguous).  The three contractions
// run over the slab's 12 x 15 x 15 grid block, each shared by the cells that
// overlap along the contracted axes:
//   U1[k0][b][c]           = sum_a  C[a][k0]  G[a][b][c]           (15 x 15 rows)
//   U2[k0][s1][k1][c]      = sum_b' C[b'][k1] U1[k0][s1 + b'][c]   (4 cell rows)
//   Gt[s1, s2][k0][k1][k2] = sum_c' C[c'][k2] U2[k0][s1][k1][s2 + c']
// 166,000 multiply-adds for 16 cells instead of 29,000 per cell.  Then every
// thread evaluates its own nodes against their cells' Gt (one fma.rn.f32x2 per
// (k0, k1 pair, k2): Gt is stored as (k1, k1 + 1) pairs, 520 floats per cell so
// that lanes in neighbouring cells read different banks).
//
// Work items are the slabs of the dense tiles, in pieces of at most 8192 nodes
// (pad = the slab), largest first, from a shared counter.
#include "device.cuh"
#include "internal.h"

namespace nfl {

namespace {

constexpr int SM_M = 6, SM_TE = 4, SM_TAPS = 2 * SM_M, SM_R = kCheb;
constexpr int SM_PA = SM_TE + 2 * SM_M - 1;                      // 15
constexpr int SM_CELLS = SM_TE * SM_TE;                          // cells of a slab
constexpr int SM_GST = SM_R * SM_R * SM_R + 8;                   // floats per cell's Gt
constexpr int SM_U1 = SM_R * SM_PA * SM_PA;                      // 1800
constexpr int SM_U2 = SM_R * SM_TE * SM_R * SM_PA;               // 3840
constexpr int SM_GT = SM_CELLS * SM_GST;                         // 8320
constexpr int SM_NT = 256;                                       // threads per CTA
constexpr int SM_SMEM = (SM_U2 + (SM_GT > SM_U1 ? SM_GT : SM_U1)) * 4;
static_assert(SM_R == 8, "k1 pairs and 8-wide rows");
static_assert(SM_GST % 4 == 0 && SM_U2 % 4 == 0, "16-byte aligned cell moments");

struct GatherMomentArgs {
    const PointF *pts;
    const int32_t *perm;
    const double *zd;       // z in sorted order: y = z + s f
    double *y;
    const double *dinv;
    double *degree_out;
    double *dinv_out;
    const WorkItem *items;  // pad = the slab (axis-0 cell position inside the tile)
    int64_t nitems;
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    const float *g;         // layout [x2][x1][x0]
    int op;
    double out_scale, k0;
    unsigned *counter;
    float cheb[SM_TAPS][SM_R];
};

}  // namespace

// One node of the evaluation: its slab cell, Chebyshev values and epilogue operands.
struct NodeTerms {
    float T0[SM_R], T1[SM_R];
    unsigned long long T2d[SM_R];   // (T2[k], T2[k]) pairs
    int cell, iq;
    double zq, dq;

    __device__ __forceinline__ void load(const GatherMomentArgs &a, int kq, const int *tc) {
        const PointF p = a.pts[kq];
        iq = a.perm[kq];
        zq = a.op != OP_DEGREE ? a.zd[kq] : 0.0;
        dq = (a.op == OP_A || a.op == OP_LS) ? a.dinv[kq] : 0.0;
        const int s1 = min(max(cell_axis(p.cell, 1) - tc[1] * SM_TE, 0), SM_TE - 1);
        const int s2 = min(max(cell_axis(p.cell, 2) - tc[2] * SM_TE, 0), SM_TE - 1);
        cell = s2 * SM_TE + s1;
        float *T[2] = {T0, T1};
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
            const float t = fmaf(2.f, p.f[ax], -1.f), t2x = t + t;
            T[ax][0] = 1.f;
            T[ax][1] = t;
#pragma unroll
            for (int k = 2; k < SM_R; ++k) T[ax][k] = fmaf(t2x, T[ax][k - 1], -T[ax][k - 2]);
        }
        const float t = fmaf(2.f, p.f[2], -1.f), t2x = t + t;
        float u0 = 1.f, u1 = t;
        T2d[0] = pack2(u0, u0);
        T2d[1] = pack2(u1, u1);
#pragma unroll
        for (int k = 2; k < SM_R; ++k) {
            const float u2 = fmaf(t2x, u1, -u0);
            T2d[k] = pack2(u2, u2);
            u0 = u1;
            u1 = u2;
        }
    }

    __device__ __forceinline__ void store(const GatherMomentArgs &a, int kq, float f) const {
        const double fd = double(f);
        if (a.op == OP_DEGREE) {
            const double dd = a.out_scale * fd - a.k0;
            a.degree_out[iq] = dd;
            a.dinv_out[kq] = dd > 0.0 ? 1.0 / sqrt(dd) : 0.0;
        } else {
            const double s = a.op == OP_LS ? -a.out_scale * dq : (a.op == OP_A ? a.out_scale * dq : a.out_scale);
            a.y[iq] = fma(s, fd, zq);
        }
    }
};

// f = sum_k0 T0 sum_k1 T1 sum_k2 T2 Gt for two nodes, (k1, k1 + 1) in one packed lane
// pair; with `same` both read the moments at ga once
__device__ __forceinline__ void eval_pair(const float *ga, const float *gb, const NodeTerms &A, const NodeTerms &B,
                                          float &fa, float &fb, bool same) {
    const ulonglong2 *pa = reinterpret_cast<const ulonglong2 *>(ga);
    const ulonglong2 *pb = reinterpret_cast<const ulonglong2 *>(gb);
    fa = 0.f;
    fb = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < SM_R; ++k0) {
        float ra = 0.f, rb = 0.f;
#pragma unroll
        for (int jp = 0; jp < SM_R / 2; ++jp) {
            unsigned long long acca = 0ull, accb = 0ull;
#pragma unroll
            for (int k2 = 0; k2 < SM_R; k2 += 2) {
                const int q = ((k0 * 4 + jp) * SM_R + k2) / 2;
                const ulonglong2 va = pa[q];
                const ulonglong2 vb = same ? va : pb[q];
                acca = k2 == 0 ? fmul2(va.x, A.T2d[0]) : ffma2(va.x, A.T2d[k2], acca);
                accb = k2 == 0 ? fmul2(vb.x, B.T2d[0]) : ffma2(vb.x, B.T2d[k2], accb);
                acca = ffma2(va.y, A.T2d[k2 + 1], acca);
                accb = ffma2(vb.y, B.T2d[k2 + 1], accb);
            }
            ra = fmaf(A.T1[2 * jp], lane_of(acca, 0), ra);
            ra = fmaf(A.T1[2 * jp + 1], lane_of(acca, 1), ra);
            rb = fmaf(B.T1[2 * jp], lane_of(accb, 0), rb);
            rb = fmaf(B.T1[2 * jp + 1], lane_of(accb, 1), rb);
        }
        fa = fmaf(A.T0[k0], ra, fa);
        fb = fmaf(B.T0[k0], rb, fb);
    }
}

__global__ void __launch_bounds__(SM_NT, 2) gather3_moments(GatherMomentArgs a) {
    extern __shared__ __align__(16) float gsm[];
    __shared__ float Cs[SM_TAPS][SM_R];
    __shared__ unsigned next_item;
    float *U2 = gsm;
    float *U1 = gsm + SM_U2;            // the slab's Gt reuses U1's space once U2 is formed
    float *Gt = U1;
    const int tid = threadIdx.x;
    for (int e = tid; e < SM_TAPS * SM_R; e += SM_NT) Cs[e / SM_R][e % SM_R] = a.cheb[e / SM_R][e % SM_R];

    for (;;) {
        // the CTA's next work item (largest first); the barrier also ends the previous
        // item's use of U1 / U2 / Gt
        if (tid == 0) next_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const int64_t it = next_item;
        if (it >= a.nitems) break;
        const WorkItem w = a.items[it];
        int tc[3];
        tile_coords<3>(w.tile, a.ntile, tc);
        const int o0 = tc[0] * SM_TE - (SM_M - 1) + w.pad;    // first support row of the slab's cells
        const int o1 = tc[1] * SM_TE - (SM_M - 1), o2 = tc[2] * SM_TE - (SM_M - 1);

        // U1: axis 0 contracted along the 12 contiguous grid values of each (b, c) row;
        // positions outside the box count 0
        for (int r = tid; r < SM_PA * SM_PA; r += SM_NT) {
            const int b = r / SM_PA, c = r - b * SM_PA;
            int p1 = o1 + b, p2 = o2 + c;
            if (a.wrap[1]) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
            if (a.wrap[2]) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
            const bool ok = p1 >= 0 && p1 < a.L[1] && p2 >= 0 && p2 < a.L[2];
            const float *row = a.g + ((int64_t)(ok ? p2 : 0) * a.L[1] + (ok ? p1 : 0)) * a.L[0];
            float gv[SM_TAPS];
#pragma unroll
            for (int j = 0; j < SM_TAPS; ++j) {
                int p0 = o0 + j;
                if (a.wrap[0]) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                gv[j] = (ok && p0 >= 0 && p0 < a.L[0]) ? __ldg(row + p0) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < SM_R; ++k) {
                float v = 0.f;
#pragma unroll
                for (int j = 0; j < SM_TAPS; ++j) v = fmaf(Cs[j][k], gv[j], v);
                U1[(k * SM_PA + b) * SM_PA + c] = v;
            }
        }
        __syncthreads();
        // U2[k0][s1][k1][c]: axis 1 contracted for each of the 4 cell rows s1
        for (int r = tid; r < SM_R * SM_TE * SM_PA; r += SM_NT) {
            const int k0 = r / (SM_TE * SM_PA), rem = r - k0 * (SM_TE * SM_PA);
            const int s1 = rem / SM_PA, c = rem - s1 * SM_PA;
            float u[SM_TAPS];
#pragma unroll
            for (int b = 0; b < SM_TAPS; ++b) u[b] = U1[(k0 * SM_PA + s1 + b) * SM_PA + c];
#pragma unroll
            for (int k = 0; k < SM_R; ++k) {
                float v = 0.f;
#pragma unroll
                for (int b = 0; b < SM_TAPS; ++b) v = fmaf(Cs[b][k], u[b], v);
                U2[((k0 * SM_TE + s1) * SM_R + k) * SM_PA + c] = v;
            }
        }
        __syncthreads();
        // Gt of cell (s1, s2): axis 2 contracted; stored per cell (s2 * 4 + s1) as
        // [k0][k1 / 2][k2][k1 & 1]
        for (int r = tid; r < SM_R * SM_TE * SM_R * SM_TE; r += SM_NT) {
            const int s2 = r & 3, k1 = (r >> 2) & 7, s1 = (r >> 5) & 3, k0 = r >> 7;
            float u[SM_TAPS];
#pragma unroll
            for (int c = 0; c < SM_TAPS; ++c) u[c] = U2[((k0 * SM_TE + s1) * SM_R + k1) * SM_PA + s2 + c];
            float *dst = Gt + (s2 * SM_TE + s1) * SM_GST + (k0 * 4 + (k1 >> 1)) * 2 * SM_R + (k1 & 1);
#pragma unroll
            for (int k = 0; k < SM_R; ++k) {
                float v = 0.f;
#pragma unroll
                for (int c = 0; c < SM_TAPS; ++c) v = fmaf(Cs[c][k], u[c], v);
                dst[2 * k] = v;
            }
        }
        __syncthreads();

        // the item's nodes, two adjacent ones per thread: nodes are sorted by cell, so the
        // pair nearly always shares its cell and then each moment load serves both
        for (int kq = w.start + 2 * tid; kq < w.start + w.count; kq += 2 * SM_NT) {
            const bool has_b = kq + 1 < w.start + w.count;
            const int kb = has_b ? kq + 1 : kq;
            NodeTerms A, B;
            A.load(a, kq, tc);
            B.load(a, kb, tc);
            float fa, fb;
            if (A.cell == B.cell) {
                eval_pair(Gt + A.cell * SM_GST, Gt + A.cell * SM_GST, A, B, fa, fb, true);
            } else {
                eval_pair(Gt + A.cell * SM_GST, Gt + B.cell * SM_GST, A, B, fa, fb, false);
            }
            A.store(a, kq, fa);
            if (has_b) B.store(a, kb, fb);
        }
    }
}

// The dense tiles' slab pieces of a one-column interpolation (the tensor-core kernel
// takes the rest).
cudaError_t launch_gather3_moments(Plan &P, int op, double *y, cudaStream_t s) {
    if (P.ngslab == 0) return cudaSuccess;
    GatherMomentArgs a{};
    a.pts = reinterpret_cast<const PointF *>(P.pts);
    a.perm = P.perm;
    a.zd = P.xsorted;
    a.y = y;
    a.dinv = P.dinv_sorted;
    a.degree_out = P.degree;
    a.dinv_out = P.dinv_sorted;
    a.items = P.gslab_items;
    a.nitems = P.ngslab;
    for (int i = 0; i < 3; ++i) {
        a.ntile[i] = P.ntile[i];
        a.L[i] = P.L[i];
        a.wrap[i] = P.wrap[i];
    }
    a.ngrid = P.ngrid;
    a.g = reinterpret_cast<const float *>(P.g);
    a.op = op;
    a.out_scale = P.out_scale;
    a.k0 = P.k0;
    a.counter = P.work_counter + 3;
    for (int j = 0; j < SM_TAPS; ++j)
        for (int k = 0; k < SM_R; ++k) a.cheb[j][k] = P.kb_cheb[j][k];
    NFL_CUDA_TRY(cudaFuncSetAttribute(gather3_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_SMEM));
    int per_sm = 0;
    NFL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather3_moments, SM_NT, SM_SMEM));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * P.num_sms;
    if (grid > P.ngslab) grid = P.ngslab;
    gather3_moments<<<(unsigned)grid, SM_NT, SM_SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nfl
