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

struct PassArgs {
    const void *in;
    void *out;
    int nA, nB;
    int64_t sA, sB;
    int Lin;
    unsigned lin_magic;   // ceil(2^32 / Lin): e / Lin = umulhi(e, lin_magic) for e < 2^22
    int64_t oC, oA;
    int Lout;
    int n, logn, N;
    int BB;
    const void *tw;       // e^{-2 pi i q / n}, q < n/2
    const void *M;        // fused multiplier, index ((b * nA) + a) * (N + 1) + (k + N/2)
    int real_in, real_out;
    const double *abs_sum;  // int64 fixed-point input: sum |x~| of the spread call, per column
    int64_t in_cstride, out_cstride;   // elements between the columns of a block (grid.z)
};

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
template <typename T, typename TIN, int MODE>
__global__ void __launch_bounds__(256) fft_pass(PassArgs a) {
    using C = typename Cplx<T>::type;
    constexpr bool PAIR = (MODE == P_FWD_R2C || MODE == P_INV_C2R);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NL = PAIR ? (a.BB + 1) / 2 : a.BB;     // complex lines in shared memory
    C *bx = reinterpret_cast<C *>(smem_raw);
    C *by = bx + NL * a.n;
    const int col = blockIdx.z;
    const int ai = blockIdx.y;
    const int b0 = blockIdx.x * a.BB;
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

cudaError_t launch_fft(Plan &P, int nc) {
    if (P.prec == NFL_PREC_FP32) return launch_fft_t<float, float>(P, nc);
    if (P.prec == NFL_PREC_FP32C) return launch_fft_t<float, long long>(P, nc);
    return launch_fft_t<double, double>(P, nc);
}

}  // namespace nfl
