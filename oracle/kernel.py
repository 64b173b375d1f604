"""Gaussian kernel, boundary regularization K_R and Fourier coefficients b_l.

Test infrastructure (the oracle); see the package docstring for who may use it.

Paper: Sec. 2 eq. (W_gaussian) defines K(y) = exp(-||y||^2 / sigma^2).
Sec. 3 defines the regularized kernel

    K_R(y) = K(y)                 if ||y|| <= 1/2 - eps_B
             T_B(||y||)           if 1/2 - eps_B < ||y|| <= 1/2
             T_B(1/2)             otherwise,

with T_B a polynomial from "two-point Taylor interpolation", and the
trapezoidal-rule coefficients, eq. (b_l::K_RF), which we read with the
d-dimensional normalisation N^{-d} (the printed 1/N is the d = 1 case):

    b_l = N^{-d} sum_{j in I_N} K_R(j / N) exp(-2 pi i j.l / N),  l in I_N,
    I_N = {-N/2, ..., N/2 - 1}^d.

Readings (the paper gives no formula for T_B):
  * T_B is the Hermite (two-point Taylor) polynomial of degree <= 2p-1 in
    r = ||y|| on [a, 1/2], a = 1/2 - eps_B, with T_B^(k)(a) = K^(k)(a) for
    k = 0..p-1 and T_B(1/2) = K(1/2), T_B^(k)(1/2) = 0 for k = 1..p-1.
  * eps_B = 0 leaves no shell: K_R(y) = K(min(||y||, 1/2)).

Pins (tests/test_oracle_kernel.py): the Hermite end conditions checked by
finite differences of exp (not by the Hermite recurrence used here); b_l real
and even; sum_l b_l = K_R(0); K_RF interpolates K_R at the grid nodes j/N;
b_l against the closed-form Fourier transform of the Gaussian for small sigma.
The exact choice of T_B is a reading: "parity unpinned" for T_B's values in
the shell beyond its defining end conditions.

Other kernels (Sec. 2, after eq. (W_gaussian); used by Alg. 2 steps 2, 4, 5):
the Laplacian RBF exp(-||y||/sigma), the multiquadric (||y||^2 + c^2)^{1/2}
and the inverse multiquadric (||y||^2 + c^2)^{-1/2}; and, for gradients with
respect to sigma, the sigma-derivative of the Gaussian,
d/dsigma exp(-||y||^2/sigma^2) = (2 ||y||^2 / sigma^3) exp(-||y||^2/sigma^2).  Every function below
takes the kernel by name (default "gaussian") and its shape parameter
(sigma, or c for the two multiquadrics) in the ``sigma`` argument.
"""
import math

import numpy as np


def gaussian(r, sigma):
    """K as a function of r = ||y||: exp(-r^2 / sigma^2) (Sec. 2, eq. (W_gaussian))."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-(r / sigma) ** 2)


def gaussian_derivative(r, sigma, k):
    """k-th derivative in r of exp(-(r/sigma)^2).

    d^k/dr^k exp(-(r/sigma)^2) = (-1/sigma)^k H_k(r/sigma) exp(-(r/sigma)^2),
    H_k the physicists' Hermite polynomials, H_{k+1}(x) = 2x H_k - 2k H_{k-1}.
    """
    x = np.asarray(r, dtype=np.float64) / sigma
    h_prev = np.ones_like(x)
    h = 2.0 * x
    if k == 0:
        hk = h_prev
    else:
        for j in range(1, k):
            h_prev, h = h, 2.0 * x * h - 2.0 * j * h_prev
        hk = h
    return (-1.0 / sigma) ** k * hk * np.exp(-x * x)


KERNELS = ("gaussian", "laplacian_rbf", "multiquadric", "inverse_multiquadric", "gaussian_dsigma")


def radial(r, sigma, kind="gaussian"):
    """K as a function of r = ||y|| for the kernels of Sec. 2."""
    r = np.asarray(r, dtype=np.float64)
    if kind == "gaussian":
        return gaussian(r, sigma)
    if kind == "laplacian_rbf":
        return np.exp(-r / sigma)
    if kind == "multiquadric":
        return np.sqrt(r * r + sigma * sigma)
    if kind == "inverse_multiquadric":
        return 1.0 / np.sqrt(r * r + sigma * sigma)
    if kind == "gaussian_dsigma":
        return 2.0 * r * r / sigma ** 3 * gaussian(r, sigma)
    raise ValueError("unknown kernel %r" % (kind,))


def _falling(alpha, j):
    """alpha (alpha - 1) ... (alpha - j + 1)."""
    out = 1.0
    for t in range(j):
        out *= alpha - t
    return out


def radial_derivative(r, sigma, k, kind="gaussian"):
    """k-th derivative in r of the radial kernel.

    Laplacian RBF: (-1/sigma)^k exp(-r/sigma).  Multiquadrics: with
    r^2 + c^2 = (r - ic)(r + ic) and alpha = +-1/2, the product rule gives
    sum_j binom(k, j) (alpha)_j (r - ic)^(alpha - j) (alpha)_(k-j) (r + ic)^(alpha - k + j)
    with falling factorials (alpha)_j; the sum is real.
    """
    if kind == "gaussian":
        return gaussian_derivative(r, sigma, k)
    r = np.asarray(r, dtype=np.float64)
    if kind == "laplacian_rbf":
        return (-1.0 / sigma) ** k * np.exp(-r / sigma)
    if kind in ("multiquadric", "inverse_multiquadric"):
        alpha = 0.5 if kind == "multiquadric" else -0.5
        zm = r - 1j * sigma
        zp = r + 1j * sigma
        out = np.zeros_like(zm)
        for j in range(k + 1):
            out = out + (math.comb(k, j) * _falling(alpha, j) * _falling(alpha, k - j)
                         * zm ** (alpha - j) * zp ** (alpha - k + j))
        return out.real
    if kind == "gaussian_dsigma":
        # Leibniz on r^2 g(r): r^2 g^(k) + 2 k r g^(k-1) + k (k - 1) g^(k-2)
        g = lambda j: gaussian_derivative(r, sigma, j) if j >= 0 else 0.0
        return 2.0 / sigma ** 3 * (r * r * g(k) + 2.0 * k * r * g(k - 1) + k * (k - 1) * g(k - 2))
    raise ValueError("unknown kernel %r" % (kind,))


def boundary_polynomial(sigma, eps_B, p, kind="gaussian"):
    """Coefficients c_0..c_{2p-1} of T_B(r) = sum_k c_k s^k, s = (r - a)/eps_B.

    a = 1/2 - eps_B.  Left end: T_B^(k)(a) = K^(k)(a), k < p, which fixes
    c_k = K^(k)(a) eps_B^k / k!.  Right end (s = 1): T_B(1/2) = K(1/2) and
    T_B^(j)(1/2) = 0 for 1 <= j < p, a p x p linear system for c_p..c_{2p-1}.
    """
    if eps_B <= 0.0:
        raise ValueError("boundary polynomial needs eps_B > 0")
    a = 0.5 - eps_B
    c = np.zeros(2 * p)
    for k in range(p):
        c[k] = radial_derivative(a, sigma, k, kind) * eps_B ** k / math.factorial(k)
    # j-th derivative of s^k at s = 1 is k!/(k-j)! for k >= j, else 0.
    def dpow(k, j):
        return math.factorial(k) / math.factorial(k - j) if k >= j else 0.0
    M = np.zeros((p, p))
    rhs = np.zeros(p)
    for j in range(p):
        rhs[j] = (float(radial(0.5, sigma, kind)) if j == 0 else 0.0) - sum(
            c[k] * dpow(k, j) for k in range(p))
        for col, k in enumerate(range(p, 2 * p)):
            M[j, col] = dpow(k, j)
    c[p:] = np.linalg.solve(M, rhs)
    return c


def boundary_polynomial_eval(r, sigma, eps_B, p, coeffs=None, kind="gaussian"):
    """T_B(r) from the coefficients above (Horner in s = (r - a)/eps_B)."""
    if coeffs is None:
        coeffs = boundary_polynomial(sigma, eps_B, p, kind)
    s = (np.asarray(r, dtype=np.float64) - (0.5 - eps_B)) / eps_B
    out = np.zeros_like(s)
    for ck in coeffs[::-1]:
        out = out * s + ck
    return out


def regularized_kernel(r, sigma, eps_B, p, kind="gaussian"):
    """K_R as a function of r = ||y|| (Sec. 3, the K_R ansatz)."""
    r = np.asarray(r, dtype=np.float64)
    if eps_B <= 0.0:
        return radial(np.minimum(r, 0.5), sigma, kind)
    a = 0.5 - eps_B
    coeffs = boundary_polynomial(sigma, eps_B, p, kind)
    inner = radial(r, sigma, kind)
    shell = boundary_polynomial_eval(np.minimum(r, 0.5), sigma, eps_B, p, coeffs, kind)
    return np.where(r <= a, inner, shell)


def frequency_set(N):
    """I_N along one axis: -N/2, ..., N/2 - 1 (Sec. 3, eq. (K_RF))."""
    return np.arange(-N // 2, N // 2)


def fourier_coefficients(N, d, sigma, eps_B, p, kind="gaussian"):
    """b_l for l in I_N (Sec. 3, eq. (b_l::K_RF)), returned as a complex array.

    Array axis a holds l_a + N/2, i.e. index 0 is l_a = -N/2.  The sum over
    j in I_N is the d-dimensional DFT of the N^d samples K_R(j/N), taken with
    numpy's FFT after placing sample j at index j mod N.
    """
    j = frequency_set(N)
    grids = np.meshgrid(*([j / N] * d), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    samples = regularized_kernel(r, sigma, eps_B, p, kind)  # index j + N/2
    samples_mod = np.fft.ifftshift(samples)                # index j mod N
    dft = np.fft.fftn(samples_mod)                         # index l mod N
    return np.fft.fftshift(dft) / float(N) ** d            # index l + N/2


def trig_polynomial(y, bhat, N):
    """K_RF(y) = sum_{l in I_N} b_l exp(2 pi i l.y) at points y (n x d); complex."""
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    d = y.shape[1]
    l = frequency_set(N)
    out = np.zeros(y.shape[0], dtype=np.complex128)
    for idx in np.ndindex(*([N] * d)):
        lv = l[list(idx)]
        out += bhat[idx] * np.exp(2j * np.pi * (y @ lv))
    return out
