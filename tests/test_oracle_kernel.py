"""Pins for the regularized kernel K_R and the coefficients b_l (Sec. 3)."""
import math

import numpy as np
import pytest
import sympy

from oracle import kernel


def _sympy_derivative(sigma, k, r0):
    r = sympy.symbols("r")
    expr = sympy.exp(-(r / sympy.Float(sigma, 30)) ** 2)
    return float(sympy.diff(expr, r, k).subs(r, sympy.Float(r0, 30)).evalf(30))


@pytest.mark.parametrize("k", range(7))
def test_gaussian_derivatives_symbolic(k):
    for r0 in (0.1, 0.37, 0.5):
        assert kernel.gaussian_derivative(r0, 0.2, k) == pytest.approx(
            _sympy_derivative(0.2, k, r0), rel=1e-11, abs=1e-300)


@pytest.mark.parametrize("sigma,eps_B,p", [(0.2, 0.125, 4), (0.15, 0.0625, 6), (0.3, 0.1, 2)])
def test_boundary_polynomial_end_conditions(sigma, eps_B, p):
    a = 0.5 - eps_B
    c = kernel.boundary_polynomial(sigma, eps_B, p)
    # T_B(r) = P(s), s = (r - a)/eps_B; the r-derivative is P^(k)(s) / eps_B^k.
    P = np.polynomial.Polynomial(c)
    for k in range(p):
        lhs = P.deriv(k)(0.0) / eps_B ** k if k else P(0.0)
        assert lhs == pytest.approx(_sympy_derivative(sigma, k, a), rel=1e-8, abs=1e-14)
    assert P(1.0) == pytest.approx(math.exp(-0.25 / sigma ** 2), rel=1e-10, abs=1e-16)
    for k in range(1, p):
        assert abs(P.deriv(k)(1.0)) / eps_B ** k < 1e-8 * max(1.0, abs(_sympy_derivative(sigma, k, a)))


def test_regularized_kernel_pieces():
    sigma, eps_B, p = 0.2, 0.125, 4
    r = np.linspace(0.0, 0.9, 1001)
    KR = kernel.regularized_kernel(r, sigma, eps_B, p)
    inner = r <= 0.375
    np.testing.assert_array_equal(KR[inner], np.exp(-(r[inner] / sigma) ** 2))
    outer = r > 0.5
    assert np.all(KR[outer] == pytest.approx(math.exp(-0.25 / sigma ** 2), rel=1e-10))
    # continuity across both joins
    for r0 in (0.375, 0.5):
        lo, hi = kernel.regularized_kernel([r0 - 1e-12, r0 + 1e-12], sigma, eps_B, p)
        assert abs(lo - hi) < 1e-10
    # eps_B = 0: K(min(r, 1/2))
    np.testing.assert_array_equal(kernel.regularized_kernel(r, sigma, 0.0, p),
                                  np.exp(-(np.minimum(r, 0.5) / sigma) ** 2))


@pytest.mark.parametrize("d,N", [(1, 16), (2, 16), (3, 16), (3, 8)])
def test_coefficients_real_even_and_sum(d, N):
    sigma, eps_B, p = 0.17, 2.0 / N, 2
    b = kernel.fourier_coefficients(N, d, sigma, eps_B, p)
    assert np.abs(b.imag).max() < 1e-15
    # b_l = b_{-l} for l and -l in I_N (indices 1..N-1 mirror about N/2)
    core = b[(slice(1, None),) * d]
    assert np.abs(core - core[(slice(None, None, -1),) * d]).max() < 1e-15
    # sum_l b_l = K_RF(0) = K_R(0) = 1
    assert b.real.sum() == pytest.approx(1.0, abs=1e-14)


def test_trig_polynomial_interpolates_at_nodes():
    N, d, sigma, eps_B, p = 8, 2, 0.2, 0.25, 2
    b = kernel.fourier_coefficients(N, d, sigma, eps_B, p)
    rng = np.random.default_rng(0)
    j = rng.integers(-N // 2, N // 2, (12, d))
    y = j / N
    KRF = kernel.trig_polynomial(y, b, N)
    KR = kernel.regularized_kernel(np.sqrt((y ** 2).sum(axis=1)), sigma, eps_B, p)
    np.testing.assert_allclose(KRF.real, KR, atol=1e-14)
    assert np.abs(KRF.imag).max() < 1e-14


@pytest.mark.parametrize("d", [1, 2, 3])
def test_coefficients_match_gaussian_fourier_transform(d):
    """Small sigma: b_l ~ (sqrt(pi) sigma)^d exp(-pi^2 sigma^2 ||l||^2), the FT of K.

    N = 64, sigma = 0.06: aliasing ~exp(-(pi sigma N/2)^2) ~ 1e-16 and
    K(1/2 - eps_B) ~ exp(-39), so the two agree to rounding."""
    N, sigma = 64, 0.06
    b = kernel.fourier_coefficients(N, d, sigma, 0.125, 4).real
    l = np.arange(-N // 2, N // 2)
    grids = np.meshgrid(*([l] * d), indexing="ij")
    l2 = sum(g.astype(float) ** 2 for g in grids)
    closed = (math.sqrt(math.pi) * sigma) ** d * np.exp(-(math.pi * sigma) ** 2 * l2)
    assert np.abs(b - closed).max() < 1e-15
