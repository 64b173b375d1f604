"""Pins for the Kaiser-Bessel window and the (adjoint) NFFT against direct sums."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import nfft


def test_i0_series_matches_library():
    z = np.linspace(0.0, 45.0, 91)
    np.testing.assert_allclose(nfft.bessel_i0(z), special.i0(z), rtol=1e-14)


@pytest.mark.parametrize("m,tol", [(2, 2e-4), (4, 2e-8), (6, 2e-12), (8, 1e-13)])
def test_window_transform_pair(m, tol):
    """phi_hat is the Fourier transform of phi; truncating phi to |n x| <= m
    costs the Kaiser-Bessel truncation error, which falls with m."""
    n = 64
    b = nfft.kb_shape(2)
    for k in (0, 3, 10, 16):
        val = integrate.quad(lambda x: nfft.kb_window(n * x, m, b) * math.cos(2 * math.pi * k * x),
                             -m / n, m / n, limit=400, epsabs=0, epsrel=1e-13)[0]
        ref = nfft.kb_window_hat(k, n, m, b)
        assert abs(val - ref) / ref < tol


def test_window_support_and_limit():
    b = nfft.kb_shape(2)
    assert nfft.kb_window(4.0, 4, b) == pytest.approx(b / math.pi)
    assert nfft.kb_window(4.0000001, 4, b) == 0.0
    assert nfft.kb_window(0.0, 4, b) == pytest.approx(math.sinh(4 * b) / (4 * math.pi))


def test_ndft_single_node_closed_form():
    v = np.array([[0.1, -0.2, 0.05]])
    N = 8
    xhat = nfft.ndft_adjoint(v, np.array([2.0]), N)
    l = np.arange(-N // 2, N // 2)
    la, lb, lc = np.meshgrid(l, l, l, indexing="ij")
    ref = 2.0 * np.exp(-2j * math.pi * (0.1 * la - 0.2 * lb + 0.05 * lc))
    np.testing.assert_allclose(xhat, ref, rtol=1e-14, atol=1e-14)
    f = nfft.ndft(v, ref / 2.0, N)          # sum_l e^{-2 pi i l.v} e^{+2 pi i l.v} = N^3
    assert f[0] == pytest.approx(N ** 3, rel=1e-13)


@pytest.mark.parametrize("d,N,m,tol", [(1, 16, 8, 1e-13), (2, 16, 8, 1e-13), (3, 16, 8, 1e-13),
                                       (3, 16, 4, 1e-6), (2, 32, 3, 1e-4), (3, 8, 2, 5e-3)])
def test_transforms_match_direct_sums(d, N, m, tol):
    rng = np.random.default_rng(d * 100 + N + m)
    v = rng.uniform(-0.5, 0.5, (200, d))          # nodes anywhere on the torus
    x = rng.standard_normal(200)
    a = nfft.adjoint_nfft(v, x, N, m)
    e = nfft.ndft_adjoint(v, x, N)
    assert np.abs(a - e).max() / np.abs(e).max() < tol
    fh = rng.standard_normal((N,) * d) + 1j * rng.standard_normal((N,) * d)
    f = nfft.nfft(v, fh, N, m)
    g = nfft.ndft(v, fh, N)
    assert np.abs(f - g).max() / np.abs(g).max() < tol


# ---------------------------------------------------------------- BF16 taps
def test_round_bf16_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    w = np.concatenate([rng.uniform(0, 1, 20000), rng.uniform(0, 1e-5, 2000), 10.0 ** rng.uniform(-30, 3, 2000)])
    ref = torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nfft.round_bf16(w), ref)


def test_round_bf16_ties_to_even():
    assert nfft.round_bf16(1.0 + 2.0 ** -8) == 1.0                       # tie, even neighbour 1
    assert nfft.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie, even neighbour above
    assert nfft.round_bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7           # representable
    assert nfft.round_bf16(0.5 + 3 * 2.0 ** -10) == 0.5 + 2.0 ** -8           # above the tie: up


def test_bf16_taps_perturb_adjoint_within_rounding():
    """Each tap moves by at most 2^-9 relative, a product of d = 3 taps by < 3.01 * 2^-9."""
    rng = np.random.default_rng(9)
    v = rng.uniform(-0.25, 0.25, (200, 3))
    x = rng.uniform(0.5, 1.5, 200)                  # positive: |sum| = sum |terms|
    a = nfft.adjoint_nfft(v, x, 16, 4)
    b = nfft.adjoint_nfft(v, x, 16, 4, taps="bf16")
    # compare the spread grids through l = 0 (the plain sum of all window products)
    i0 = (8, 8, 8)
    assert 0.0 < abs(b[i0] - a[i0]) <= 3.01 * 2.0 ** -9 * abs(a[i0])
