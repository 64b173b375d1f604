"""Kaiser-Bessel window, adjoint NFFT, NFFT and the direct NDFT sums.

Test infrastructure (the oracle); see the package docstring for who may use it.

Sec. 3 applies the d-dimensional adjoint NFFT (Alg. 1 step 1) and NFFT
(Alg. 1 step 3) with NFFT3's default Kaiser-Bessel window, which the paper
names but does not print.  We take its published form (Keiner, Kunis, Potts
2009) with oversampling alpha = 2, grid size n = alpha N per axis and
cut-off m; in grid units delta = n x:

    phi(delta) = sinh(b sqrt(m^2 - delta^2)) / (pi sqrt(m^2 - delta^2)),  |delta| <= m,
    phi_hat(k) = (1/n) I_0(m sqrt(b^2 - (2 pi k / n)^2)),                  b = pi (2 - 1/alpha),

phi_hat being the Fourier transform of the untruncated phi.  The window is
truncated to the 2m grid points t = floor(n x) - m + 1, ..., floor(n x) + m.

Adjoint NFFT:  h_t = sum_i x_i prod_a phi(n v_ia - t_a)  (periodic in t),
               xhat_l = (sum_t h_t exp(-2 pi i l.t / n)) / prod_a (n phi_hat(l_a)).
NFFT:          g_t = sum_{l in I_N} fhat_l / prod_a (n phi_hat(l_a)) exp(2 pi i l.t / n),
               f(v_j) = sum_t g_t prod_a phi(n v_ja - t_a).

BF16 taps (``taps="bf16"``, not a paper construct: the accuracy of storing
the window weights in BF16): every normalized tap phi(delta) / phi(0) is
rounded to FP32 and then to the nearest BF16 value (ties to even) before it
is used, and multiplied back by phi(0).

Pins (tests/test_oracle_nfft.py): phi_hat equals the numerically integrated
Fourier transform of the truncated window to the truncation level; I_0's
power series equals the textbook routine; both transforms equal the direct
NDFT sums to ~1e-14 relative at m = 8 and within the Kaiser-Bessel error at
smaller m.
"""
import itertools
import math

import numpy as np


def kb_shape(alpha=2):
    """b = pi (2 - 1/alpha)."""
    return math.pi * (2.0 - 1.0 / alpha)


def kb_window(delta, m, b):
    """phi at grid-unit offsets delta; zero for |delta| > m; the limit b/pi at |delta| = m."""
    delta = np.asarray(delta, dtype=np.float64)
    arg = m * m - delta * delta
    s = np.sqrt(np.maximum(arg, 0.0))
    safe = np.where(s > 0.0, s, 1.0)
    val = np.where(s > 0.0, np.sinh(b * s) / safe, b) / math.pi
    return np.where(arg >= 0.0, val, 0.0)


def bessel_i0(z):
    """Modified Bessel I_0 by its power series sum_k ((z/2)^2)^k / (k!)^2 (FP64)."""
    z = np.asarray(z, dtype=np.float64)
    q = (z / 2.0) ** 2
    term = np.ones_like(z)
    total = np.ones_like(z)
    for k in range(1, 400):
        term = term * q / (k * k)
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
    return total


def kb_window_hat(k, n, m, b):
    """phi_hat(k) = (1/n) I_0(m sqrt(b^2 - (2 pi k/n)^2)) for |2 pi k / n| <= b."""
    k = np.asarray(k, dtype=np.float64)
    arg = b * b - (2.0 * math.pi * k / n) ** 2
    if np.any(arg < 0.0):
        raise ValueError("frequency outside the window's band")
    return bessel_i0(m * np.sqrt(arg)) / n


def round_bf16(w):
    """Nearest BF16 value (8-bit significand, ties to even) of FP32(w), as FP64."""
    f = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _taps(v, n, m, b, taps="fp64"):
    """Per-axis tap indices (unwrapped) and window values: two (npts, d, 2m) arrays."""
    u = n * v
    base = np.floor(u).astype(np.int64)
    offs = np.arange(-m + 1, m + 1, dtype=np.int64)
    t = base[:, :, None] + offs[None, None, :]
    w = kb_window(u[:, :, None] - t, m, b)
    if taps == "bf16":
        phi0 = float(kb_window(0.0, m, b))
        w = phi0 * round_bf16(w / phi0)
    elif taps != "fp64":
        raise ValueError("taps must be 'fp64' or 'bf16'")
    return t, w


def adjoint_nfft(v, x, N, m, alpha=2, taps="fp64"):
    """xhat_l ~ sum_i x_i exp(-2 pi i l.v_i), l in I_N (index l + N/2 per axis).

    v: (npts, d) nodes in [-1/2, 1/2)^d;  x: (npts,) real or complex.
    """
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    npts, d = v.shape
    n = alpha * N
    b = kb_shape(alpha)
    t, w = _taps(v, n, m, b, taps)
    h = np.zeros((n,) * d, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    for tap in itertools.product(range(2 * m), repeat=d):
        idx = tuple(t[:, a, tap[a]] % n for a in range(d))
        wt = x.copy()
        for a in range(d):
            wt = wt * w[:, a, tap[a]]
        np.add.at(h, idx, wt)
    hhat = np.fft.fftn(h)                       # sum_t h_t exp(-2 pi i k.t/n)
    l = np.arange(-N // 2, N // 2)
    sub = hhat[np.ix_(*([l % n] * d))]
    deconv = n * kb_window_hat(l, n, m, b)      # n phi_hat(l_a) = I_0(...)
    for a in range(d):
        shape = [1] * d
        shape[a] = N
        sub = sub / deconv.reshape(shape)
    return sub


def nfft(v, fhat, N, m, alpha=2, taps="fp64"):
    """f(v_j) ~ sum_{l in I_N} fhat_l exp(2 pi i l.v_j); complex output."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    npts, d = v.shape
    n = alpha * N
    b = kb_shape(alpha)
    l = np.arange(-N // 2, N // 2)
    deconv = n * kb_window_hat(l, n, m, b)
    G = np.asarray(fhat, dtype=np.complex128).copy()
    for a in range(d):
        shape = [1] * d
        shape[a] = N
        G = G / deconv.reshape(shape)
    full = np.zeros((n,) * d, dtype=np.complex128)
    full[np.ix_(*([l % n] * d))] = G
    g = np.fft.ifftn(full) * float(n) ** d      # sum_k G_k exp(+2 pi i k.t/n)
    t, w = _taps(v, n, m, b, taps)
    f = np.zeros(npts, dtype=np.complex128)
    for tap in itertools.product(range(2 * m), repeat=d):
        idx = tuple(t[:, a, tap[a]] % n for a in range(d))
        wt = g[idx]
        for a in range(d):
            wt = wt * w[:, a, tap[a]]
        f += wt
    return f


def _phase_factors(v, N, sign):
    l = np.arange(-N // 2, N // 2)
    return [np.exp(sign * 2j * np.pi * np.outer(v[:, a], l)) for a in range(v.shape[1])]


def ndft_adjoint(v, x, N):
    """Direct sum xhat_l = sum_i x_i exp(-2 pi i l.v_i), O(npts N^d)."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    d = v.shape[1]
    E = _phase_factors(v, N, -1.0)
    letters = "abc"[:d]
    spec = "i," + ",".join("i" + c for c in letters) + "->" + letters
    return np.einsum(spec, np.asarray(x, dtype=np.complex128), *E)


def ndft(v, fhat, N):
    """Direct sum f_j = sum_{l in I_N} fhat_l exp(2 pi i l.v_j), O(npts N^d)."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    d = v.shape[1]
    E = _phase_factors(v, N, +1.0)
    letters = "abc"[:d]
    spec = letters + "," + ",".join("j" + c for c in letters) + "->j"
    return np.einsum(spec, np.asarray(fhat, dtype=np.complex128), *E)
