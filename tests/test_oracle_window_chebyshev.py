"""The Chebyshev form of the window taps that the slab-moment kernels use (m = 6).

For the dense tiles the product writes each of the 2m = 12 taps of the
Kaiser-Bessel window (Sec. 3, the window of Alg. 1), as a function of the
node's fractional cell offset f in [0, 1), in the Chebyshev basis T_k(2f - 1)
with 8 terms (the interpolant at 8 Chebyshev points), so that a cell's nodes
reduce to 8^3 moments.  That is a reading of ours, not a construct of the
paper: it holds only if 8 terms reproduce every tap to the FP32 rounding of the
window's peak.  Checked here with the oracle's own window (oracle/nfft.py),
independent of the product's: 8 terms stay within 4e-8 of phi(0), with the
coefficients rounded to FP32 as the product holds them, while 7 terms miss by
more than 1e-7 (so the bound discriminates and 8 is the smallest count).
"""
import numpy as np

from oracle import nfft

M = 6


def _max_tap_error(terms, fp32_coefficients):
    b = nfft.kb_shape(2)
    phi0 = float(nfft.kb_window(0.0, M, b))
    f = np.linspace(0.0, 1.0, 4001)
    t = 2.0 * f - 1.0
    nodes = np.cos(np.pi * (np.arange(terms) + 0.5) / terms)
    worst = 0.0
    for j in range(2 * M):
        # tap j of a node at offset f sits at window argument f + m - 1 - j
        values = nfft.kb_window(0.5 * (nodes + 1.0) + M - 1 - j, M, b)
        coef = np.array([(1.0 if k == 0 else 2.0) / terms *
                         np.sum(values * np.cos(np.pi * k * (np.arange(terms) + 0.5) / terms))
                         for k in range(terms)])
        if fp32_coefficients:
            coef = coef.astype(np.float32).astype(np.float64)
        exact = nfft.kb_window(f + M - 1 - j, M, b)
        approx = np.polynomial.chebyshev.chebval(t, coef)
        worst = max(worst, float(np.abs(approx - exact).max()) / phi0)
    return worst


def test_eight_chebyshev_terms_reach_fp32_rounding_of_the_peak():
    assert _max_tap_error(8, fp32_coefficients=False) < 2e-8
    assert _max_tap_error(8, fp32_coefficients=True) < 4e-8


def test_seven_terms_are_not_enough():
    assert _max_tap_error(7, fp32_coefficients=False) > 1e-7
