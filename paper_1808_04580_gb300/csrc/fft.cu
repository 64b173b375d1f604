// The FFT part of Alg. 1: forward DFT of the spread grid restricted to the
// kept frequencies, multiplication by the Fourier multiplier (step 2 with
// both window deconvolutions folded in), inverse DFT back to the active box.
//
// The grid holds only the active box (L_a <= n = 2N positions per axis); the
// rest of the n-periodic line is zero, and only frequencies |k| <= N/2 are
// kept (k in [0, N/2] on the last axis, whose transform is real-to-complex).
// Shifting the box origin multiplies the spectrum by a phase that the
// inverse transform removes again, so box position s is used as FFT index s.
//
// Every pass transforms contiguous lines: a CTA loads BB consecutive lines
// (a, b0..b0+BB-1) of length Lin, runs a radix-2 Stockham FFT of length n on
// each line in shared memory, and writes the result "rotated" so that b is
// the fastest output index (out[c' oC + a oA + b]); the next pass then again
// reads contiguous lines.  3-D sequence (x2 fastest in the spread grid):
//   F1 axis 2 R2C   h[x0][x1][x2]  -> A[k2][x0][x1]
//   F2 axis 1 C2C   A[k2][x0][x1]  -> B[k1][k2][x0]
//   F3 axis 0 fwd, multiply, inv   -> C[x0][k2][k1]
//   I2 axis 1 inv   C[x0][k2][k1]  -> D[x1][x0][k2]
//   I1 axis 2 C2R   D[x1][x0][k2]  -> g[x2][x1][x0]
#include <type_traits>

#include "internal.h"

namespace nfl {

enum PassMode { P_FWD_R2C = 0, P_FWD_C2C = 1, P_FUSED = 2, P_INV_C2C = 3, P_INV_C2R = 4 };

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}


// Grid value as a real of the FFT type.  int64 fixed point to FP32 through its
// 32-bit halves (hi 2^32 + lo, both converted exactly or to nearest), which
// stays on the FP32 pipe; the result is within one FP32 rounding of the value.
template <typename T> __device__ __forceinline__ T to_real(float v) { return T(v); }
template <typename T> __device__ __forceinline__ T to_real(double v) { return T(v); }
template <typename T> __device__ __forceinline__ T to_real(long long v);
template <> __device__ __forceinline__ float to_real<float>(long long v) {
    const float hi = __int2float_rn((int)(v >> 32));
    const float lo = __uint2float_rn((unsigned)(v & 0xFFFFFFFFll));
    return fmaf(hi, 4294967296.0f, lo);
}
template <> __device__ __forceinline__ double to_real<double>(long long v) { return double(v); }

// 2^-k for the fixed-point scale 2^k used by the spread kernel.
__device__ __forceinline__ double fixed_point_unscale(double abs_sum) {
    if (!(abs_sum > 0.0)) return 1.0;
    int e;
    frexp(abs_sum, &e);
    int k = 62 - e;
    k = k > 120 ? 120 : (k < -120 ? -120 : k);     // 2^k stays a normal FP32 number
    return ldexp(1.0, -k);
}

// Stockham autosort FFT on nl lines of length n (a power of two) held in x
// (scratch y): radix-4 stages while they fit, then one radix-2 stage if log2 n
// is odd.  Stage with stride s (the product of the earlier radices), radix R,
// for j < n / (R s), k < s, q < R:
//   Y[k + R j s + q s] = w^{q j s} sum_{r < R} X[k + j s + r n / R] e^{-+2 pi i r q / R},
// w = e^{-+2 pi i / n}; the table holds w^m for m < n/2 and w^{m + n/2} = -w^m.
template <typename C>
__device__ __forceinline__ C twiddle(const C *tw, int m, int half, bool inverse) {
    C w = m < half ? tw[m] : C{-tw[m - half].x, -tw[m - half].y};
    if (inverse) w.y = -w.y;
    return w;
}

template <typename C>
__device__ C *stockham(C *x, C *y, int nl, int n, int logn, const C *tw, bool inverse) {
    const int half = n >> 1, quarter = n >> 2;
    int s = 1, logs = 0;
    for (; logs + 2 <= logn; logs += 2, s <<= 2) {
        for (int e = threadIdx.x; e < nl * quarter; e += blockDim.x) {
            const int line = e >> (logn - 2);
            const int b = e & (quarter - 1);
            const int j = b >> logs;
            const int k = b & (s - 1);
            const C *X = x + line * n + k + j * s;
            C *Y = y + line * n + k + 4 * j * s;
            const C a0 = X[0], a1 = X[quarter], a2 = X[half], a3 = X[half + quarter];
            const C b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3), d = csub(a1, a3);
            // (a1 - a3) e^{-+i pi / 2}: -i d forward, +i d inverse
            const C b3 = inverse ? C{-d.y, d.x} : C{d.y, -d.x};
            const int t = j * s;
            Y[0] = cadd(b0, b2);
            Y[s] = cmul(cadd(b1, b3), twiddle(tw, t, half, inverse));
            Y[2 * s] = cmul(csub(b0, b2), twiddle(tw, 2 * t, half, inverse));
            Y[3 * s] = cmul(csub(b1, b3), twiddle(tw, 3 * t, half, inverse));
        }
        __syncthreads();
        C *tmp = x;
        x = y;
        y = tmp;
    }
    if (logs < logn) {
        for (int e = threadIdx.x; e < nl * half; e += blockDim.x) {
            const int line = e >> (logn - 1);
            const int b = e & (half - 1);
            const int j = b >> logs;
            const int k = b & (s - 1);
            const C *X = x + line * n + k + j * s;
            C *Y = y + line * n + k + 2 * j * s;
            const C c0 = X[0], c1 = X[half];
            Y[0] = cadd(c0, c1);
            Y[s] = cmul(csub(c0, c1), twiddle(tw, j * s, half, inverse));
        }
        __syncthreads();
        C *tmp = x;
        x = y;
        y = tmp;
    }
    return x;
}

// R2C and C2R transform two real lines as one complex line (PAIR): forward,
// z = a + i b gives A_k = (Z_k + conj Z_{n-k}) / 2 and B_k = (Z_k - conj Z_{n-k}) / 2i;
// inverse, Z = A + i B over the Hermitian extension of both half spectra gives
// a = Re z, b = Im z.
// One CTA's work of a pass: lines b0 = bxi BB .. of line group ai, column col.
template <typename T, typename TIN, int MODE>
__device__ __forceinline__ void fft_pass_body(const PassArgs &a, int bxi, int ai, int col) {
    using C = typename Cplx<T>::type;
    constexpr bool PAIR = (MODE == P_FWD_R2C || MODE == P_INV_C2R);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NL = PAIR ? (a.BB + 1) / 2 : a.BB;     // complex lines in shared memory
    C *bx = reinterpret_cast<C *>(smem_raw);
    C *by = bx + NL * a.n;
    const int b0 = bxi * a.BB;
    const int nb = min(a.BB, a.nB - b0);
    const int n = a.n, N = a.N;
    const C *tw = reinterpret_cast<const C *>(a.tw);

    for (int e = threadIdx.x; e < NL * n; e += blockDim.x) bx[e] = C{T(0), T(0)};
    __syncthreads();

    T in_scale = T(1);
    if (std::is_same<TIN, long long>::value) in_scale = T(fixed_point_unscale(a.abs_sum[col]));

    // load
    if (MODE == P_INV_C2R) {
        // line pairs (2p, 2p + 1): Z_c = A_c + i B_c and Z_{n-c} = conj A_c + i conj B_c
        // (c = 1 .. Lin - 1 < n / 2); the DC terms are real
        const int np = (nb + 1) / 2;
        const C *in = reinterpret_cast<const C *>(a.in);
        for (int e = threadIdx.x; e < np * a.Lin; e += blockDim.x) {
            const int pp = (int)__umulhi((unsigned)e, a.lin_magic);
            const int c = e - pp * a.Lin;
            const int64_t src = col * a.in_cstride + ai * a.sA + (int64_t)(b0 + 2 * pp) * a.sB + c;
            const C A = in[src];
            const C B = 2 * pp + 1 < nb ? in[src + a.sB] : C{T(0), T(0)};
            if (c == 0) {
                bx[pp * n] = C{A.x, B.x};
            } else {
                bx[pp * n + c] = C{A.x - B.y, A.y + B.x};
                bx[pp * n + (n - c)] = C{A.x + B.y, B.x - A.y};
            }
        }
    }
    for (int e = threadIdx.x; e < (MODE == P_INV_C2R ? 0 : nb * a.Lin); e += blockDim.x) {
        const int bb = (int)__umulhi((unsigned)e, a.lin_magic);
        const int c = e - bb * a.Lin;
        const int64_t src = col * a.in_cstride + ai * a.sA + (int64_t)(b0 + bb) * a.sB + c;
        C v;
        if (MODE == P_FWD_R2C || (MODE == P_FUSED && a.real_in)) {
            const TIN *in = reinterpret_cast<const TIN *>(a.in);
            v = C{to_real<T>(in[src]) * in_scale, T(0)};
        } else {
            v = reinterpret_cast<const C *>(a.in)[src];
        }
        if (MODE == P_INV_C2C) {
            const int k = c - N / 2;
            bx[bb * n + ((k + n) & (n - 1))] = v;
        } else if (MODE == P_FWD_R2C) {
            // line bb is the real (even bb) or imaginary (odd bb) part of pair line bb / 2
            reinterpret_cast<T *>(&bx[(bb >> 1) * n + c])[bb & 1] = v.x;
        } else {
            bx[bb * n + c] = v;
        }
    }
    __syncthreads();

    const bool inverse = (MODE == P_INV_C2C || MODE == P_INV_C2R);
    C *res = stockham<C>(bx, by, NL, n, a.logn, tw, inverse);

    if (MODE == P_FUSED) {
        const T *M = reinterpret_cast<const T *>(a.M);
        for (int e = threadIdx.x; e < a.BB * n; e += blockDim.x) {
            const int bb = e >> a.logn;
            const int q = e & (n - 1);
            const int k = q < n / 2 ? q : q - n;
            C v = res[e];
            if (bb < nb && k >= -N / 2 && k <= N / 2) {
                const T mv = M[((int64_t)(b0 + bb) * a.nA + ai) * (N + 1) + (k + N / 2)];
                v = C{v.x * mv, v.y * mv};
            } else {
                v = C{T(0), T(0)};
            }
            res[e] = v;
        }
        __syncthreads();
        C *other = (res == bx) ? by : bx;
        res = stockham<C>(res, other, a.BB, n, a.logn, tw, true);
    }

    // store, b fastest
    const unsigned nb_magic = 0xFFFFFFFFu / (unsigned)nb + 1u;   // e / nb = umulhi(e, nb_magic), nb <= 32
    for (int e = threadIdx.x; e < nb * a.Lout; e += blockDim.x) {
        const int cc = nb == 1 ? e : (int)__umulhi((unsigned)e, nb_magic);
        const int bb = e - cc * nb;
        int idx;
        if (MODE == P_FWD_R2C) idx = cc;
        else if (MODE == P_FWD_C2C) idx = (cc - N / 2 + n) & (n - 1);
        else idx = cc;
        const int64_t dst = col * a.out_cstride + cc * a.oC + (int64_t)ai * a.oA + b0 + bb;
        if (MODE == P_FWD_R2C) {
            const C zk = res[(bb >> 1) * n + idx], zm = res[(bb >> 1) * n + ((n - idx) & (n - 1))];
            const C v = (bb & 1) == 0 ? C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)}
                                      : C{T(0.5) * (zk.y + zm.y), T(0.5) * (zm.x - zk.x)};
            reinterpret_cast<C *>(a.out)[dst] = v;
        } else if (MODE == P_INV_C2R) {
            const C v = res[(bb >> 1) * n + idx];
            reinterpret_cast<T *>(a.out)[dst] = (bb & 1) == 0 ? v.x : v.y;
        } else {
            const C v = res[bb * n + idx];
            if (MODE == P_FUSED && a.real_out) reinterpret_cast<T *>(a.out)[dst] = v.x;
            else reinterpret_cast<C *>(a.out)[dst] = v;
        }
    }
}

template <typename T, typename TIN, int MODE>
__global__ void __launch_bounds__(256) fft_pass(PassArgs a) {
    fft_pass_body<T, TIN, MODE>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// A pass over the plans of a batch in one launch: CTA b belongs to the plan g with
// start[g] <= b < start[g + 1] and is its (line block, line group, column) in that
// plan's grid of the per-plan launch.
template <typename T, typename TIN, int MODE>
__global__ void __launch_bounds__(256) fft_pass_batch(const PassArgs *args, const int *start, int G) {
    const int b = blockIdx.x;
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const PassArgs a = args[lo];
    const int local = b - start[lo];
    const int gx = (a.nB + a.BB - 1) / a.BB;
    const int bxi = local % gx, rest = local / gx;
    fft_pass_body<T, TIN, MODE>(a, bxi, rest % a.nA, rest / a.nA);
}

template <typename T, typename TIN, int MODE>
static cudaError_t run_pass(Plan &P, PassArgs a, int nc) {
    using C = typename Cplx<T>::type;
    // few lines per CTA and one radix-4 butterfly per thread and stage: small CTAs,
    // many of them resident per SM to hide the global-memory latency of load and store
    const int cap = P.fft_cap;
    constexpr bool PAIR = (MODE == P_FWD_R2C || MODE == P_INV_C2R);
    int NL = cap / a.n;                        // complex lines per CTA
    NL = NL > 16 ? 16 : (NL < 1 ? 1 : NL);
    const int BB = PAIR ? 2 * NL : NL;          // real (PAIR) or complex lines per CTA
    a.BB = BB;
    a.lin_magic = (unsigned)((0x100000000ull + (unsigned)a.Lin - 1) / (unsigned)a.Lin);
    const int smem = 2 * NL * a.n * (int)sizeof(C);
    int threads = NL * a.n / 4;
    threads = threads < 64 ? 64 : (threads > 256 ? 256 : threads);
    NFL_CUDA_TRY(cudaFuncSetAttribute(fft_pass<T, TIN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((a.nB + BB - 1) / BB, a.nA, nc);
    fft_pass<T, TIN, MODE><<<grid, threads, smem, P.stream>>>(a);
    return cudaGetLastError();
}

template <typename T, typename TIN>
static cudaError_t launch_fft_t(Plan &P, int nc) {
    const int N = P.N, n = P.ngrid;
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    PassArgs base{};
    base.n = n;
    base.logn = logn;
    base.N = N;
    base.tw = P.twiddle;
    base.M = P.mult;
    base.abs_sum = P.scratch;
    // column strides (elements) of the block buffers
    const int64_t sg = P.box_elems, sa = P.bufA_elems, sb = P.bufB_elems;
    auto stride_of = [&](const void *buf) -> int64_t {
        return buf == P.grid || buf == P.g ? sg : (buf == P.bufA ? sa : sb);
    };
    auto with_strides = [&](PassArgs a) {
        a.in_cstride = stride_of(a.in);
        a.out_cstride = stride_of(a.out);
        return a;
    };
    const int64_t L0 = P.L[0], L1 = P.L[1], L2 = P.L[2];
    if (P.d == 1) {
        PassArgs a = base;
        a.in = P.grid; a.out = P.g;
        a.nA = 1; a.nB = 1; a.sA = 0; a.sB = 0; a.Lin = (int)L0;
        a.oC = 1; a.oA = 0; a.Lout = (int)L0;
        a.real_in = 1; a.real_out = 1;
        return run_pass<T, TIN, P_FUSED>(P, with_strides(a), nc);
    }
    if (P.d == 2) {
        const int64_t K1 = N / 2 + 1;
        PassArgs f1 = base;
        f1.in = P.grid; f1.out = P.bufA;
        f1.nA = 1; f1.nB = (int)L0; f1.sA = 0; f1.sB = L1; f1.Lin = (int)L1;
        f1.oC = L0; f1.oA = 0; f1.Lout = (int)K1;
        NFL_CUDA_TRY((run_pass<T, TIN, P_FWD_R2C>(P, with_strides(f1), nc)));
        PassArgs f3 = base;
        f3.in = P.bufA; f3.out = P.bufB;
        f3.nA = 1; f3.nB = (int)K1; f3.sA = 0; f3.sB = L0; f3.Lin = (int)L0;
        f3.oC = K1; f3.oA = 0; f3.Lout = (int)L0;
        NFL_CUDA_TRY((run_pass<T, T, P_FUSED>(P, with_strides(f3), nc)));
        PassArgs i1 = base;
        i1.in = P.bufB; i1.out = P.g;
        i1.nA = 1; i1.nB = (int)L0; i1.sA = 0; i1.sB = K1; i1.Lin = (int)K1;
        i1.oC = L0; i1.oA = 0; i1.Lout = (int)L1;
        return run_pass<T, T, P_INV_C2R>(P, with_strides(i1), nc);
    }
    const int64_t K2 = N / 2 + 1, K1 = N + 1;
    PassArgs f1 = base;
    f1.in = P.grid; f1.out = P.bufA;
    f1.nA = (int)L0; f1.nB = (int)L1; f1.sA = L1 * L2; f1.sB = L2; f1.Lin = (int)L2;
    f1.oC = L0 * L1; f1.oA = L1; f1.Lout = (int)K2;
    NFL_CUDA_TRY((run_pass<T, TIN, P_FWD_R2C>(P, with_strides(f1), nc)));
    PassArgs f2 = base;
    f2.in = P.bufA; f2.out = P.bufB;
    f2.nA = (int)K2; f2.nB = (int)L0; f2.sA = L0 * L1; f2.sB = L1; f2.Lin = (int)L1;
    f2.oC = K2 * L0; f2.oA = L0; f2.Lout = (int)K1;
    NFL_CUDA_TRY((run_pass<T, T, P_FWD_C2C>(P, with_strides(f2), nc)));
    PassArgs f3 = base;
    f3.in = P.bufB; f3.out = P.bufA;
    f3.nA = (int)K2; f3.nB = (int)K1; f3.sA = L0; f3.sB = K2 * L0; f3.Lin = (int)L0;
    f3.oC = K2 * K1; f3.oA = K1; f3.Lout = (int)L0;
    NFL_CUDA_TRY((run_pass<T, T, P_FUSED>(P, with_strides(f3), nc)));
    PassArgs i2 = base;
    i2.in = P.bufA; i2.out = P.bufB;
    i2.nA = (int)L0; i2.nB = (int)K2; i2.sA = K2 * K1; i2.sB = K1; i2.Lin = (int)K1;
    i2.oC = L0 * K2; i2.oA = K2; i2.Lout = (int)L1;
    NFL_CUDA_TRY((run_pass<T, T, P_INV_C2C>(P, with_strides(i2), nc)));
    PassArgs i1 = base;
    i1.in = P.bufB; i1.out = P.g;
    i1.nA = (int)L1; i1.nB = (int)L0; i1.sA = L0 * K2; i1.sB = K2; i1.Lin = (int)K2;
    i1.oC = L1 * L0; i1.oA = L0; i1.Lout = (int)L2;
    return run_pass<T, T, P_INV_C2R>(P, with_strides(i1), nc);
}

// Launch shape of a pass of line length n at cap grid points per CTA: complex lines
// per CTA NL, lines BB (real line pairs for R2C / C2R), threads and shared memory.
static void pass_shape(int cap, int n, bool pair, size_t csize, int &BB, int &threads, int &smem) {
    int NL = cap / n;
    NL = NL > 16 ? 16 : (NL < 1 ? 1 : NL);
    BB = pair ? 2 * NL : NL;
    smem = 2 * NL * n * (int)csize;
    threads = NL * n / 4;
    threads = threads < 64 ? 64 : (threads > 256 ? 256 : threads);
}

int fft_passes_3d(const Plan &P, const void *grid, void *bufA, void *bufB, void *g, int64_t sa, int64_t sb, int cap,
                  PassArgs *out, int nc, int *ctas) {
    const int N = P.N, n = P.ngrid;
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    PassArgs base{};
    base.n = n;
    base.logn = logn;
    base.N = N;
    base.tw = P.twiddle;
    base.M = P.mult;
    const int64_t L0 = P.L[0], L1 = P.L[1], L2 = P.L[2], sg = P.box_elems;
    const int64_t K2 = N / 2 + 1, K1 = N + 1;
    PassArgs *f = out;
    f[0] = base;
    f[0].in = grid; f[0].out = bufA; f[0].in_cstride = sg; f[0].out_cstride = sa;
    f[0].nA = (int)L0; f[0].nB = (int)L1; f[0].sA = L1 * L2; f[0].sB = L2; f[0].Lin = (int)L2;
    f[0].oC = L0 * L1; f[0].oA = L1; f[0].Lout = (int)K2;
    f[1] = base;
    f[1].in = bufA; f[1].out = bufB; f[1].in_cstride = sa; f[1].out_cstride = sb;
    f[1].nA = (int)K2; f[1].nB = (int)L0; f[1].sA = L0 * L1; f[1].sB = L1; f[1].Lin = (int)L1;
    f[1].oC = K2 * L0; f[1].oA = L0; f[1].Lout = (int)K1;
    f[2] = base;
    f[2].in = bufB; f[2].out = bufA; f[2].in_cstride = sb; f[2].out_cstride = sa;
    f[2].nA = (int)K2; f[2].nB = (int)K1; f[2].sA = L0; f[2].sB = K2 * L0; f[2].Lin = (int)L0;
    f[2].oC = K2 * K1; f[2].oA = K1; f[2].Lout = (int)L0;
    f[3] = base;
    f[3].in = bufA; f[3].out = bufB; f[3].in_cstride = sa; f[3].out_cstride = sb;
    f[3].nA = (int)L0; f[3].nB = (int)K2; f[3].sA = K2 * K1; f[3].sB = K1; f[3].Lin = (int)K1;
    f[3].oC = L0 * K2; f[3].oA = K2; f[3].Lout = (int)L1;
    f[4] = base;
    f[4].in = bufB; f[4].out = g; f[4].in_cstride = sb; f[4].out_cstride = sg;
    f[4].nA = (int)L1; f[4].nB = (int)L0; f[4].sA = L0 * K2; f[4].sB = K2; f[4].Lin = (int)K2;
    f[4].oC = L1 * L0; f[4].oA = L0; f[4].Lout = (int)L2;
    for (int i = 0; i < 5; ++i) {
        int threads = 0, smem = 0;
        pass_shape(cap, n, i == 0 || i == 4, sizeof(float2), f[i].BB, threads, smem);
        f[i].lin_magic = (unsigned)((0x100000000ull + (unsigned)f[i].Lin - 1) / (unsigned)f[i].Lin);
        ctas[i] = ((f[i].nB + f[i].BB - 1) / f[i].BB) * f[i].nA * nc;
    }
    return 5;
}

template <typename TIN, int MODE>
static cudaError_t batch_pass(Batch &B, int i, cudaStream_t s) {
    int BB = 0, threads = 0, smem = 0;
    pass_shape(B.fft_cap, 2 * B.N, MODE == P_FWD_R2C || MODE == P_INV_C2R, sizeof(float2), BB, threads, smem);
    NFL_CUDA_TRY(cudaFuncSetAttribute(fft_pass_batch<float, TIN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem));
    if (B.pass_ctas[i] < 1) return cudaSuccess;
    fft_pass_batch<float, TIN, MODE><<<B.pass_ctas[i], threads, smem, s>>>(B.pass_args[i], B.pass_start[i], B.G);
    return cudaGetLastError();
}

// The five passes over every member of a batch, one launch each.
cudaError_t launch_fft_batch(Batch &B, cudaStream_t s) {
    if (B.prec == NFL_PREC_FP32C) NFL_CUDA_TRY((batch_pass<long long, P_FWD_R2C>(B, 0, s)));
    else NFL_CUDA_TRY((batch_pass<float, P_FWD_R2C>(B, 0, s)));
    NFL_CUDA_TRY((batch_pass<float, P_FWD_C2C>(B, 1, s)));
    NFL_CUDA_TRY((batch_pass<float, P_FUSED>(B, 2, s)));
    NFL_CUDA_TRY((batch_pass<float, P_INV_C2C>(B, 3, s)));
    return batch_pass<float, P_INV_C2R>(B, 4, s);
}

cudaError_t launch_fft(Plan &P, int nc) {
    if (P.prec == NFL_PREC_FP32) return launch_fft_t<float, float>(P, nc);
    if (P.prec == NFL_PREC_FP32C) return launch_fft_t<float, long long>(P, nc);
    return launch_fft_t<double, double>(P, nc);
}

}  // namespace nfl
