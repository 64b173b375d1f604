// Interpolation in 3-D on the 5th-generation tensor cores (Alg. 1 step 3,
// the window half of the NFFT):
//   f_i = sum_{b,c} w1_i(b) w2_i(c) T[i, (b,c)],   T[i, (b,c)] = sum_a w0_i(a) G[a, (b,c)].
//
// For one tile of TE^3 cells the grid values G (tile plus halo, PA <= 16
// positions per axis) are the B operand, K = a (padded to 16), N = (b, c)
// (PA^2 padded to a multiple of 16).  Each batch of up to 128 nodes gives the
// A operand W0 (M = 128 nodes, K = 16: node i's axis-0 window placed at its
// offset, zero elsewhere).  T = W0 G is a dense 128 x N x 16 product, computed
// by tcgen05.mma (kind::tf32) into TMEM.  FP32 accuracy comes from splitting
// both operands into TF32 hi + lo parts: T = A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the dropped A_lo B_lo term is ~2^-22 relative).
//
// Then thread i (TMEM lane i) reads its row of T in 16-column pieces and
// contracts it with its own axis-1/axis-2 windows held in registers (column
// n = b PA + c is a compile-time index in the unrolled loop), and applies the
// W / A / L_s / degree epilogue in FP64.
//
// Operands use the canonical K-major layout without swizzle: core matrices
// of 8 rows x 16 bytes (8 x 4 TF32 values), k-blocks of one 8-row group
// 128 B apart (leading-dimension offset), 8-row groups 512 B apart (stride
// offset).  The (b, c) columns are processed in halves of N = 128 so that a
// CTA needs 128 TMEM columns and four CTAs fit an SM.  One thread issues the
// MMAs; tcgen05.commit arrives on an mbarrier
// that the CTA waits on with a bounded spin (a wait that runs out sets an
// error flag and the kernel skips ahead rather than hang).
#include <stdint.h>

#include "device.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace nfl {

struct GatherTCArgs {
    const PointF *pts;
    const int32_t *perm;
    const double *zd;     // z in sorted order: y = z + s f (W: s = out_scale; A, L_s: s = +-out_scale dinv)
    double *y;
    const double *dinv;
    double *degree_out;
    double *dinv_out;
    const WorkItem *items;
    int64_t nitems;   // items of one column; the grid takes nitems * ncol
    int ncol;         // columns of a block product (item it: item it / ncol, column it % ncol)
    int64_t g_stride, z_stride, ldy;   // column strides of g, zd and y
    int ntile[3];
    int L[3];
    int wrap[3];
    int ngrid;
    const float *g;   // layout [x2][x1][x0]
    int op;
    double out_scale, k0;   // W x = out_scale f - K(0) x (caller's coordinates)
    int *error_flag;
    unsigned *counter;    // next work item, shared by all CTAs
    int skip_mma;                 // fault test: the MMAs are never issued, so every wait runs out
    unsigned long long wait_ns;   // limit of each bounded wait
    const BatchPlanDev *bplans;   // batch: the members (item it is bitems[it] of member bitems[it].plan)
    const BatchItem *bitems;
    float poly[2 * kMaxM][kPolyCoef];   // window by taps, as in the plan
};

// out[q] = tap[q - s] for 0 <= q - s < TAPS, else 0, with s in [0, TE) and TE a
// power of two: the node's taps placed at its tile-local cell offset by a
// logarithmic shifter (one select per entry and bit of s, no indexing).
template <int TAPS, int PAD, int TE>
__device__ __forceinline__ void place_taps(const float (&tap)[TAPS], int s, float (&out)[PAD]) {
    static_assert((TE & (TE - 1)) == 0 && TAPS + TE - 1 <= PAD, "shifter layout");
#pragma unroll
    for (int q = 0; q < PAD; ++q) out[q] = q < TAPS ? tap[q] : 0.f;
#pragma unroll
    for (int bit = 1; bit < TE; bit <<= 1) {
        const bool on = (s & bit) != 0;
#pragma unroll
        for (int q = PAD - 1; q >= 0; --q) out[q] = on ? (q >= bit ? out[q - bit] : 0.f) : out[q];
    }
}

template <int M, int TE>
struct TCGeom {
    static constexpr int PA = TE + 2 * M - 1;             // <= 16
    static constexpr int NCOL = PA * PA;                  // (b, c) columns used
    static constexpr int N = 128;                         // MMA N per half
    static constexpr int NH = (NCOL + N - 1) / N;         // halves of the column range
    static constexpr int TMEM_COLS = 128;
    static constexpr int A_BYTES = 128 * 64;              // 128 rows x 16 TF32
    static constexpr int B_BYTES = NH * N * 64;           // all halves
};

// Per-item plan fields of a batch, in shared memory (written by thread 0 per item).
struct GatherItemPlan {
    const PointF *pts;
    const int32_t *perm;
    const double *dinv, *zc;
    const float *gc;
    double *yc;
    double out_scale;
    int *error_flag;
    WorkItem w;
    int ntile[3], L[3], wrap[3];
};

#define GT_L(i) (BATCH ? ip.L[i] : a.L[i])
#define GT_WRAP(i) (BATCH ? ip.wrap[i] : a.wrap[i])

// BF16: the window taps are rounded to BF16 (the BF16W form).  BATCH: the items of
// all members of a batch, each item's plan fields read from its member's descriptor.
template <int M, int TE, bool BF16, bool BATCH = false>
__global__ void __launch_bounds__(128, 4) gather3_tc(GatherTCArgs a) {
    using G = TCGeom<M, TE>;
    constexpr int PA = G::PA, N = G::N, NH = G::NH, NCOL = G::NCOL, TAPS = 2 * M;
    static_assert(PA <= 16, "K is padded to 16");
    static_assert(kPolyCoef % 2 == 0, "coefficients loaded in pairs");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sA_hi = smem_raw;
    unsigned char *sA_lo = sA_hi + G::A_BYTES;
    unsigned char *sB_hi = sA_lo + G::A_BYTES;
    unsigned char *sB_lo = sB_hi + G::B_BYTES;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float2 polys[M][kPolyCoef];   // (tap 2q, tap 2q+1) coefficients
    __shared__ unsigned next_item;
    __shared__ GatherItemPlan ip;

    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < M * kPolyCoef; e += 128) {
        const int q = e / kPolyCoef, k = e - q * kPolyCoef;
        polys[q][k] = make_float2(a.poly[2 * q][k], a.poly[2 * q + 1][k]);
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(G::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0;
    bool failed = false;

    // instruction descriptor: D f32, A/B tf32, both K-major, N, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);

    while (!failed) {
        // the CTA's next work item (largest first: the plan sorts them by size)
        if (tid == 0) {
            next_item = atomicAdd(a.counter, 1u);
            if (BATCH && next_item < (unsigned)(a.nitems * a.ncol)) {
                // the member of this item and its fields
                const unsigned it0 = next_item / (unsigned)a.ncol;
                const int c0 = (int)(next_item - it0 * (unsigned)a.ncol);
                const BatchItem e = a.bitems[it0];
                const BatchPlanDev &D = a.bplans[e.plan];
                ip.w = D.items[e.item];
                ip.pts = D.pts;
                ip.perm = D.perm;
                ip.dinv = D.dinv;
                ip.zc = D.zd + c0 * D.n;
                ip.gc = D.g + c0 * D.box;
                ip.yc = D.y + c0 * D.ldy;
                ip.out_scale = D.out_scale;
                ip.error_flag = D.error_flag;
                for (int i = 0; i < 3; ++i) {
                    ip.ntile[i] = D.ntile[i];
                    ip.L[i] = D.L[i];
                    ip.wrap[i] = D.wrap[i];
                }
            }
        }
        __syncthreads();
        const unsigned itc = next_item;
        if (itc >= (unsigned)(a.nitems * a.ncol)) break;
        const unsigned it = a.ncol == 1 ? itc : itc / (unsigned)a.ncol;
        const int col = (int)(itc - it * (unsigned)a.ncol);
        const float *gc = BATCH ? ip.gc : a.g + col * a.g_stride;
        const double *zc = BATCH ? ip.zc : a.zd + col * a.z_stride;
        double *yc = BATCH ? ip.yc : a.y + col * a.ldy;
        const WorkItem w = BATCH ? ip.w : a.items[it];
        int tc[3];
        tile_coords<3>(w.tile, BATCH ? ip.ntile : a.ntile, tc);
        // B operand: row n = b PA + c holds G[a][(b, c)] for k = a = 0..15, split into TF32
        // hi/lo parts; zero beyond PA^2 rows, beyond PA along a and outside the box
        for (int n = tid; n < NH * N; n += 128) {
            const bool used = n < NCOL;
            const int bq = used ? n / PA : 0, cq = used ? n - bq * PA : 0;
            int p1 = tc[1] * TE - (M - 1) + bq;
            int p2 = tc[2] * TE - (M - 1) + cq;
            if (GT_WRAP(1)) p1 = ((p1 % a.ngrid) + a.ngrid) % a.ngrid;
            if (GT_WRAP(2)) p2 = ((p2 % a.ngrid) + a.ngrid) % a.ngrid;
            const bool ok12 = used && p1 >= 0 && p1 < GT_L(1) && p2 >= 0 && p2 < GT_L(2);
            const float *src = gc + ((int64_t)(ok12 ? p2 : 0) * GT_L(1) + (ok12 ? p1 : 0)) * GT_L(0);
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                int p0 = tc[0] * TE - (M - 1) + k;
                if (GT_WRAP(0)) p0 = ((p0 % a.ngrid) + a.ngrid) % a.ngrid;
                v[k] = (ok12 && k < PA && p0 >= 0 && p0 < GT_L(0)) ? src[p0] : 0.f;
            }
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                float4 h, l;
                h.x = to_tf32(v[4 * kb + 0]); l.x = to_tf32(v[4 * kb + 0] - h.x);
                h.y = to_tf32(v[4 * kb + 1]); l.y = to_tf32(v[4 * kb + 1] - h.y);
                h.z = to_tf32(v[4 * kb + 2]); l.z = to_tf32(v[4 * kb + 2] - h.z);
                h.w = to_tf32(v[4 * kb + 3]); l.w = to_tf32(v[4 * kb + 3] - h.w);
                const uint32_t off = kmajor_off(n, 4 * kb);
                *reinterpret_cast<float4 *>(sB_hi + off) = h;
                *reinterpret_cast<float4 *>(sB_lo + off) = l;
            }
        }

        // this thread's node record (and epilogue operands) of the item's first batch, then of
        // each next batch one batch ahead, so the loads are in flight during a batch's MMAs
        const int wend = w.start + w.count;
        PointF pn = {{0.f, 0.f, 0.f}, 0};
        int in_ = 0;
        double zn = 0.0, dn = 0.0;
        auto fetch = [&](int b) {
            const int k = b + tid;
            if (k < wend) {
                pn = (BATCH ? ip.pts : a.pts)[k];
                in_ = (BATCH ? ip.perm : a.perm)[k];
                if (a.op != OP_DEGREE) zn = zc[k];
                if (a.op == OP_A || a.op == OP_LS) dn = (BATCH ? ip.dinv : a.dinv)[k];
            }
        };
        fetch(w.start);
        for (int base = w.start; base < wend && !failed; base += 128) {
            const int nb = min(128, wend - base);
            const bool live = tid < nb;
            float w1p[PA], w2p[PA];
            int kq = 0, iq = 0;
            double zq = 0.0, dq = 0.0;
            {
                float f0 = 0.f, f1 = 0.f, f2 = 0.f;
                int s0 = 0, s1 = 0, s2 = 0;
                if (live) {
                    kq = base + tid;
                    const PointF p = pn;
                    // epilogue operands, loaded a batch ahead and used after the contraction
                    iq = in_;
                    zq = zn;
                    dq = dn;
                    s0 = cell_axis(p.cell, 0) - tc[0] * TE;
                    s1 = cell_axis(p.cell, 1) - tc[1] * TE;
                    s2 = cell_axis(p.cell, 2) - tc[2] * TE;
                    f0 = p.f[0]; f1 = p.f[1]; f2 = p.f[2];
                }
                fetch(base + 128);
                // window taps: Horner in t = 2f - 1, two taps per fma.rn.f32x2; axes 1 and 2
                // first (kept for the contraction), then axis 0 (the A operand)
                // a warp with no node in this batch leaves its rows of A as they are: they
                // only reach rows of T that nothing reads
                if (warp * 32 < nb) {
                    const unsigned long long *pc = reinterpret_cast<const unsigned long long *>(&polys[0][0]);
                    {
                        float tap1[TAPS], tap2[TAPS];
                        const unsigned long long T1 = pack2(fmaf(2.f, f1, -1.f), fmaf(2.f, f1, -1.f));
                        const unsigned long long T2 = pack2(fmaf(2.f, f2, -1.f), fmaf(2.f, f2, -1.f));
#pragma unroll
                        for (int q = 0; q < M; ++q) {
                            // coefficient pairs (k, k + 1) with 16-byte loads; Horner from k = 9 down
                            const ulonglong2 *pq = reinterpret_cast<const ulonglong2 *>(pc + q * kPolyCoef);
                            ulonglong2 cc = pq[kPolyCoef / 2 - 1];
                            unsigned long long h1 = cc.y, h2 = cc.y;
                            h1 = ffma2(h1, T1, cc.x);
                            h2 = ffma2(h2, T2, cc.x);
#pragma unroll
                            for (int i = kPolyCoef / 2 - 2; i >= 0; --i) {
                                cc = pq[i];
                                h1 = ffma2(h1, T1, cc.y);
                                h2 = ffma2(h2, T2, cc.y);
                                h1 = ffma2(h1, T1, cc.x);
                                h2 = ffma2(h2, T2, cc.x);
                            }
                            tap1[2 * q] = lane_of(h1, 0);
                            tap1[2 * q + 1] = lane_of(h1, 1);
                            tap2[2 * q] = lane_of(h2, 0);
                            tap2[2 * q + 1] = lane_of(h2, 1);
                        }
                        if constexpr (BF16) {
#pragma unroll
                            for (int j = 0; j < TAPS; ++j) {
                                tap1[j] = round_bf16(tap1[j]);
                                tap2[j] = round_bf16(tap2[j]);
                            }
                        }
                        place_taps<TAPS, PA, TE>(tap1, s1, w1p);
                        place_taps<TAPS, PA, TE>(tap2, s2, w2p);
                    }
                    {
                        // A operand row tid: axis-0 window, hi/lo TF32 parts, written four values at a time
                        float tap0[TAPS];
                        const unsigned long long T0 = pack2(fmaf(2.f, f0, -1.f), fmaf(2.f, f0, -1.f));
#pragma unroll
                        for (int q = 0; q < M; ++q) {
                            const ulonglong2 *pq = reinterpret_cast<const ulonglong2 *>(pc + q * kPolyCoef);
                            ulonglong2 cc = pq[kPolyCoef / 2 - 1];
                            unsigned long long h0 = ffma2(cc.y, T0, cc.x);
#pragma unroll
                            for (int i = kPolyCoef / 2 - 2; i >= 0; --i) {
                                cc = pq[i];
                                h0 = ffma2(h0, T0, cc.y);
                                h0 = ffma2(h0, T0, cc.x);
                            }
                            tap0[2 * q] = live ? lane_of(h0, 0) : 0.f;
                            tap0[2 * q + 1] = live ? lane_of(h0, 1) : 0.f;
                        }
                        if constexpr (BF16) {
#pragma unroll
                            for (int j = 0; j < TAPS; ++j) tap0[j] = round_bf16(tap0[j]);
                        }
                        float v0[16];
                        place_taps<TAPS, 16, TE>(tap0, s0, v0);
#pragma unroll
                        for (int kb = 0; kb < 4; ++kb) {
                            float4 h, l;
                            h.x = to_tf32(v0[4 * kb + 0]); l.x = to_tf32(v0[4 * kb + 0] - h.x);
                            h.y = to_tf32(v0[4 * kb + 1]); l.y = to_tf32(v0[4 * kb + 1] - h.y);
                            h.z = to_tf32(v0[4 * kb + 2]); l.z = to_tf32(v0[4 * kb + 2] - h.z);
                            h.w = to_tf32(v0[4 * kb + 3]); l.w = to_tf32(v0[4 * kb + 3] - h.w);
                            const uint32_t off = kmajor_off(tid, 4 * kb);
                            *reinterpret_cast<float4 *>(sA_hi + off) = h;
                            *reinterpret_cast<float4 *>(sA_lo + off) = l;
                        }
                    }
                }
            }
            // make the generic-proxy stores visible to the tensor core
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            // f = sum_b w1[b] sum_c w2[c] T[b, c], one row b at a time
            float f = 0.f, rowsum = 0.f;
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                if (failed) break;   // uniform: decided by __syncthreads_or below
                if (tid == 0 && !a.skip_mma) {
                    const uint32_t aH = smem_u32(sA_hi), aL = smem_u32(sA_lo);
                    const uint32_t bH = smem_u32(sB_hi) + h * (N * 64), bL = smem_u32(sB_lo) + h * (N * 64);
                    int issued = 0;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {          // K = 16 in two steps of 8
                        const uint32_t koff = ks * 256;        // two 128-byte k-blocks per step
                        const uint64_t dAh = smem_desc(aH + koff, 128, 512), dAl = smem_desc(aL + koff, 128, 512);
                        const uint64_t dBh = smem_desc(bH + koff, 128, 512), dBl = smem_desc(bL + koff, 128, 512);
                        const uint64_t As[3] = {dAh, dAh, dAl};
                        const uint64_t Bs[3] = {dBh, dBl, dBh};
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            const uint32_t acc = issued > 0 ? 1u : 0u;
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                                "l"(As[t]), "l"(Bs[t]), "r"(idesc), "r"(acc));
                            ++issued;
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&mbar)));
                }
                // bounded wait for the MMAs
                {
                    const bool done = mbar_wait_bounded(smem_u32(&mbar), phase, kSpinLimit, a.wait_ns);
                    // every thread takes the same decision (barriers below stay matched)
                    if (__syncthreads_or(!done)) {
                        failed = true;
                        if (tid == 0) atomicExch(BATCH ? ip.error_flag : a.error_flag, 1);
                    }
                }
                phase ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;");
                // a warp with no node in this batch (the last, partial batch of an item)
                // skips its rows of T
                if (!failed && warp * 32 < nb) {
                    // thread tid owns TMEM lane tid: contract this half of its row of T with w1 w2
                    const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
                    for (int ch = 0; ch < N / 8; ++ch) {
                        if (h * N + ch * 8 >= NCOL) break;
                        uint32_t r[8];
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                            : "r"(row_addr + ch * 8));
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int n = h * N + ch * 8 + e;
                            if (n < NCOL) {
                                rowsum = fmaf(w2p[n % PA], __uint_as_float(r[e]), rowsum);
                                if (n % PA == PA - 1) {
                                    f = fmaf(w1p[n / PA], rowsum, f);
                                    rowsum = 0.f;
                                }
                            }
                        }
                    }
                }
                // the next half's MMA overwrites the accumulator: order it after these loads
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;");
            }
            if (!failed) {
                if (live) {
                    const double fd = double(f);
                    if (a.op == OP_DEGREE) {
                        const double dd = a.out_scale * fd - a.k0;
                        a.degree_out[iq] = dd;
                        a.dinv_out[kq] = dd > 0.0 ? 1.0 / sqrt(dd) : 0.0;
                    } else {
                        const double osc = BATCH ? ip.out_scale : a.out_scale;
                        const double s = a.op == OP_W ? osc : (a.op == OP_A ? osc : -osc) * dq;
                        yc[iq] = fma(s, fd, zq);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
        __syncthreads();
    }
    if (failed) {
        // give MMAs still in flight a second bounded chance to finish before freeing TMEM
        mbar_wait_bounded(smem_u32(&mbar), phase ^ 1u, kSpinLimit, a.wait_ns);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS));
}

template <int M, int TE>
static cudaError_t launch_tc(Plan &P, const GatherTCArgs &a) {
    using G = TCGeom<M, TE>;
    auto kern = P.bf16_taps ? gather3_tc<M, TE, true> : gather3_tc<M, TE, false>;
    // 52 KB of dynamic shared memory (and <= 128 registers from the launch bounds)
    // keep at most four CTAs, 4 x TMEM_COLS = 512 columns, per SM
    const int smem = 52 * 1024;
    static_assert(2 * G::A_BYTES + 2 * G::B_BYTES + 1024 <= 52 * 1024, "operands fit");
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int64_t grid = 4LL * P.num_sms;
    if (grid > P.nitems * a.ncol) grid = P.nitems * a.ncol;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, 128, smem, P.stream>>>(a);
    return cudaGetLastError();
}

template <int M, int TE>
static cudaError_t launch_tc_batch(Batch &B, const GatherTCArgs &a, cudaStream_t s) {
    using G = TCGeom<M, TE>;
    auto kern = B.bf16 ? gather3_tc<M, TE, true, true> : gather3_tc<M, TE, false, true>;
    const int smem = 52 * 1024;
    static_assert(2 * G::A_BYTES + 2 * G::B_BYTES + 1024 <= 52 * 1024, "operands fit");
    NFL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int64_t grid = 4LL * B.num_sms;
    if (grid > B.ngitems * a.ncol) grid = B.ngitems * a.ncol;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

// The interpolation of every member of a batch in one launch: (item, column) pairs of
// all members from one counter, items largest first.
cudaError_t launch_gather_tc_batch(Batch &B, cudaStream_t s) {
    GatherTCArgs a{};
    a.ncol = B.ncol;
    a.nitems = B.ngitems;
    a.bitems = B.gitems;
    a.bplans = B.desc;
    a.ngrid = 2 * B.N;
    a.op = B.op;
    a.counter = B.counter + 1;
    a.skip_mma = 0;
    a.wait_ns = 2000000000ull;
    for (int j = 0; j < 2 * kMaxM; ++j)
        for (int k = 0; k < kPolyCoef; ++k) a.poly[j][k] = B.poly[j][k];
    switch (B.m) {
        case 2: return launch_tc_batch<2, 8>(B, a, s);
        case 3: return launch_tc_batch<3, 8>(B, a, s);
        case 4: return launch_tc_batch<4, 8>(B, a, s);
        case 6: return launch_tc_batch<6, 4>(B, a, s);
    }
    return cudaErrorInvalidValue;
}

bool gather_tc_available(const Plan &P) {
    if (P.d != 3 || P.prec == NFL_PREC_FP64 || P.tile_edge != column_tile_edge(P.m)) return false;
    return P.m == 2 || P.m == 3 || P.m == 4 || P.m == 6 || P.m == 7;
}

cudaError_t launch_gather_tc(Plan &P, int op, const double *x, double *y, int64_t ldy, int nc) {
    GatherTCArgs a;
    a.ncol = nc;
    a.g_stride = P.box_elems;
    a.z_stride = P.n;
    a.ldy = ldy;
    a.pts = reinterpret_cast<const PointF *>(P.pts);
    a.perm = P.perm;
    a.zd = P.xsorted;
    a.y = y;
    a.dinv = P.dinv_sorted;
    a.degree_out = P.degree;
    a.dinv_out = P.dinv_sorted;
    // a one-column interpolation with dense cells leaves the dense tiles to the moment kernel
    const bool split = nc == 1 && moments_available(P) && P.nslab > 0;
    a.items = split ? P.gsparse_items : P.items;
    a.nitems = split ? P.ngsparse : P.nitems;
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
    a.error_flag = P.error_flag;
    a.counter = P.work_counter + 1;
    a.skip_mma = P.fault_kind == 1 ? 1 : 0;
    a.wait_ns = P.fault_kind == 1 ? 10000000ull : 2000000000ull;
    for (int j = 0; j < 2 * kMaxM; ++j)
        for (int k = 0; k < kPolyCoef; ++k) a.poly[j][k] = P.kb_poly[j][k];
    switch (P.m) {
        case 2: return launch_tc<2, 8>(P, a);
        case 3: return launch_tc<3, 8>(P, a);
        case 4: return launch_tc<4, 8>(P, a);
        case 6:
            // the dense tiles' slabs after the sparse tiles, on the same stream (beside them
            // on a second stream the moment kernel's CTAs held SMs the tensor-core kernel
            // still needed: 3 % slower)
            NFL_CUDA_TRY((launch_tc<6, 4>(P, a)));
            return split ? launch_gather3_moments(P, op, y, P.stream) : cudaSuccess;
        case 7: return launch_tc<7, 2>(P, a);
    }
    return cudaErrorInvalidValue;
}

}  // namespace nfl
