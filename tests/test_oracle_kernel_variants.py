"""Pins for the other kernels of Sec. 2 (Laplacian RBF, multiquadric, inverse
multiquadric) through the whole oracle: values, derivatives (for the boundary
polynomial T_B), the coefficients b_l, the direct sums, and Alg. 2 with its
scaling rule for the multiquadrics.
"""
import math

import numpy as np
import pytest
import sympy

from oracle import direct, fastsum, kernel

KINDS = ["gaussian", "laplacian_rbf", "multiquadric", "inverse_multiquadric", "gaussian_dsigma"]


def _expr(kind, r, s):
    if kind == "gaussian":
        return sympy.exp(-(r / s) ** 2)
    if kind == "laplacian_rbf":
        return sympy.exp(-r / s)
    if kind == "multiquadric":
        return sympy.sqrt(r ** 2 + s ** 2)
    if kind == "gaussian_dsigma":
        return sympy.diff(sympy.exp(-(r / s) ** 2), s)
    return 1 / sympy.sqrt(r ** 2 + s ** 2)


def _sym_derivative(kind, s, k, r0):
    r, sg = sympy.symbols("r sg", positive=True)
    e = _expr(kind, r, sg).subs(sg, sympy.Float(s, 30))
    return float(sympy.diff(e, r, k).subs(r, sympy.Float(r0, 30)).evalf(30))


@pytest.mark.parametrize("kind", KINDS)
def test_values_and_k0(kind):
    c = 0.3
    k0 = {"gaussian": 1.0, "laplacian_rbf": 1.0, "multiquadric": c, "inverse_multiquadric": 1.0 / c,
          "gaussian_dsigma": 0.0}[kind]
    assert float(kernel.radial(0.0, c, kind)) == pytest.approx(k0, rel=1e-15, abs=0.0)
    for r0 in (0.05, 0.4, 1.7):
        assert float(kernel.radial(r0, c, kind)) == pytest.approx(_sym_derivative(kind, c, 0, r0), rel=1e-14)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("k", range(8))
def test_derivatives_symbolic(kind, k):
    for r0, s in ((0.1, 0.2), (0.37, 0.05), (0.5, 0.7)):
        scale = s ** -k * max(1.0, abs(_sym_derivative(kind, s, 0, r0)))   # where the derivative vanishes
        assert float(kernel.radial_derivative(r0, s, k, kind)) == pytest.approx(
            _sym_derivative(kind, s, k, r0), rel=1e-10, abs=1e-12 * scale)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("s,eps_B,p", [(0.2, 0.125, 4), (0.05, 0.0625, 6), (0.7, 0.1, 3)])
def test_boundary_polynomial_end_conditions(kind, s, eps_B, p):
    a = 0.5 - eps_B
    P = np.polynomial.Polynomial(kernel.boundary_polynomial(s, eps_B, p, kind))
    for k in range(p):
        lhs = P.deriv(k)(0.0) / eps_B ** k if k else P(0.0)
        ref = _sym_derivative(kind, s, k, a)
        assert lhs == pytest.approx(ref, rel=1e-8, abs=1e-12 * max(1.0, abs(ref)))
    assert P(1.0) == pytest.approx(_sym_derivative(kind, s, 0, 0.5), rel=1e-10)
    for k in range(1, p):
        # zero to rounding: relative to the sum of the magnitudes that make up P^(k)(1)
        terms = np.abs(P.deriv(k).coef).sum()
        assert abs(P.deriv(k)(1.0)) < 1e-12 * terms


@pytest.mark.parametrize("kind", KINDS)
def test_coefficients_sum_to_regularized_kernel_at_zero(kind):
    # sum_l b_l = K_RF(0) = K_R(0) (the trapezoidal rule interpolates at the nodes)
    b = kernel.fourier_coefficients(16, 3, 0.3, 0.125, 4, kind)
    assert abs(b.imag).max() < 1e-12 * abs(b.real).max()
    assert b.real.sum() == pytest.approx(float(kernel.radial(0.0, 0.3, kind)), rel=1e-12,
                                         abs=1e-12 * abs(b.real).max())


@pytest.mark.parametrize("kind", KINDS)
def test_direct_two_nodes_closed_form(kind):
    v = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])   # distance 0.5
    c = 0.8
    w = {"gaussian": math.exp(-0.25 / 0.64), "laplacian_rbf": math.exp(-0.5 / 0.8),
         "multiquadric": math.sqrt(0.25 + 0.64), "inverse_multiquadric": 1.0 / math.sqrt(0.25 + 0.64),
         "gaussian_dsigma": 2.0 * 0.25 / 0.8 ** 3 * math.exp(-0.25 / 0.64)}[kind]
    x = np.array([2.0, -3.0])
    np.testing.assert_allclose(direct.apply_W(v, c, x, kind), [-3.0 * w, 2.0 * w], rtol=1e-15)
    np.testing.assert_allclose(direct.apply_A(v, c, x, kind), [-3.0, 2.0], rtol=1e-14)


@pytest.mark.parametrize("kind", KINDS)
def test_c_rows_match_dense(kind):
    rng = np.random.default_rng(6)
    v = rng.standard_normal((200, 3))
    x = rng.standard_normal(200)
    rows = np.array([0, 11, 199])
    ref = direct.weight_matrix(v, 0.6, kind) @ x
    np.testing.assert_allclose(direct.rows_W(v, 0.6, x, rows, kernel=kind), ref[rows], rtol=1e-13)


@pytest.fixture(scope="module")
def cloud():
    rng = np.random.default_rng(0)
    return rng.standard_normal((300, 3)), rng.standard_normal(300)


@pytest.mark.parametrize("kind,tol", [("gaussian", 1e-12), ("multiquadric", 1e-5),
                                      ("inverse_multiquadric", 1e-6), ("gaussian_dsigma", 1e-12)])
def test_alg2_matches_direct_sum(cloud, kind, tol):
    v, x = cloud
    ref = direct.apply_W(v, 0.7, x, kind)
    fs = fastsum.NormalizedFastsum(v, 0.7, 128, 8, 8, kernel=kind)
    assert np.linalg.norm(fs.apply_W(x) - ref) / np.linalg.norm(ref) < tol
    np.testing.assert_allclose(fs.degree, direct.degree(v, 0.7, kind), rtol=10 * tol)


def test_laplacian_rbf_converges_in_N(cloud):
    """The cusp of exp(-r/sigma) at r = 0 makes b_l decay slowly: the error
    falls with N, but stays far above the smooth kernels' (Sec. 6.2.2 uses it)."""
    v, x = cloud
    ref = direct.apply_W(v, 0.7, x, "laplacian_rbf")
    errs = []
    for N in (32, 64, 128):
        fs = fastsum.NormalizedFastsum(v, 0.7, N, 8, 8, kernel="laplacian_rbf")
        errs.append(np.linalg.norm(fs.apply_W(x) - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-2 and errs[0] / errs[2] > 10


def test_printed_multiquadric_rule_misses_the_kernel(cloud):
    """Alg. 2 prints c := c/rho with the output scaled by rho; with v := rho v
    that is not the caller's kernel, while c~ = rho c with output / rho is."""
    v, x = cloud
    c = 0.7
    ref = direct.apply_W(v, c, x, "multiquadric")
    ours = fastsum.NormalizedFastsum(v, c, 64, 8, 8, kernel="multiquadric")
    b_printed = kernel.fourier_coefficients(64, 3, c / ours.rho, ours.eps_B, 8, "multiquadric")
    printed = ours.rho * fastsum.fastsum(ours.vt, x, b_printed, 64, 8).real - c * x
    assert np.linalg.norm(ours.apply_W(x) - ref) / np.linalg.norm(ref) < 1e-4
    assert np.linalg.norm(printed - ref) / np.linalg.norm(ref) > 0.1


def test_gaussian_dsigma_is_the_sigma_derivative(cloud):
    """W_sigma x equals the central difference in sigma of the Gaussian W x."""
    v, x = cloud
    h = 1e-5
    fd = (direct.apply_W(v, 0.7 + h, x) - direct.apply_W(v, 0.7 - h, x)) / (2 * h)
    ex = direct.apply_W(v, 0.7, x, "gaussian_dsigma")
    assert np.abs(fd - ex).max() < 1e-8 * np.abs(ex).max()
