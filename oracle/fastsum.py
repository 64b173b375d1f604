"""O2 (exact trigonometric-polynomial sum) and O3 (Alg. 1 and Alg. 2 in plain numpy).

Test infrastructure (the oracle); see the package docstring for who may use it.

Alg. 1 (Sec. 3): with Fourier coefficients b_l of K_RF, nodes v_j with
||v_j|| <= 1/4 - eps_B/2 and a vector x,
  step 1  xhat_l = adjoint NFFT of x            (~ sum_i x_i e^{-2 pi i l.v_i})
  step 2  fhat_l = b_l xhat_l
  step 3  f_RF(v_j) = NFFT of fhat              (~ sum_l fhat_l e^{2 pi i l.v_j})
and f_RF(v_j) ~ (W~ x)_j with W~ = W + K(0) I (Sec. 3, eq. (nfftWtilde_x)).

Alg. 2 (Sec. 3.1), steps 1-4 once per setup:
  step 1  rho with ||rho v_j|| <= 1/4 - eps_B/2, v_j := rho v_j
  step 2  sigma := rho sigma (Gaussian, Laplacian RBF); for the multiquadrics
          see the reading below
  step 3  control parameters (N, m, p, eps_B; defaults p = m, eps_B = p/N,
          Fig. tab:fastsum_param) and b_l by eq. (b_l::K_RF)
  step 4  D_E = diag(W~_E 1 - K(0) 1)
  step 5  y = D_E^{-1/2} (W~_E (D_E^{-1/2} x) - K(0) D_E^{-1/2} x) ~ A x.

Readings:
  * Shift and scale (Sec. 3 asks to "shift and scale"; Alg. 2 step 1 only
    scales): nodes are shifted by the bounding-box midpoint c, then scaled
    with the largest admissible rho = (1/4 - eps_B/2) / max_j ||v_j - c||,
    also when the nodes already fit.  K is translation invariant, so the
    shift changes nothing exact.
  * When all nodes coincide the scale is free; rho = 1.
  * Alg. 1's output is complex because I_N is not symmetric; the matrix
    product for real x is its real part.  The real part of a Hermitian form
    is symmetric, so the resulting operator is exactly symmetric.
  * L_s x = x - A x (Sec. 2, eq. (nomlap)).
  * Multiquadric kernels (Alg. 2 steps 2, 4, 5): the printed rule "c := c/rho,
    scale the output by rho (multiquadric) or 1/rho (inverse multiquadric)"
    does not reproduce the kernel in the scaled coordinates.  With
    v~ = rho v, (||v~_j - v~_i||^2 + (rho c)^2)^(+-1/2) = rho^(+-1) K(v_j - v_i),
    so this oracle uses c~ = rho c and scales Alg. 1's output by 1/rho
    (multiquadric) or rho (inverse multiquadric); the test against the
    direct sum pins this reading, and shows that the printed rule misses it.
    The sigma-derivative of the Gaussian scales as rho^-1 in the same way
    (output times rho).

Pins: O3 against O2 at m = 8 (~1e-13 relative), O2 against the direct sum
O1 for parameters where the kernel error is tiny, the a-priori bound of
eq. (KERR_estimate), Lemma 3.1, and exact symmetry (tests/test_oracle_fastsum.py).
"""
import numpy as np

from . import kernel as _kernel
from . import nfft as _nfft


def scale_nodes(v, eps_B):
    """Alg. 2 steps 1-2 geometry: (v - c) rho with c the bounding-box midpoint."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    c = 0.5 * (v.min(axis=0) + v.max(axis=0))
    radius = np.sqrt(((v - c) ** 2).sum(axis=1)).max()
    # all nodes coincide (n = 1 included): after the shift every node is 0,
    # so any rho satisfies ||rho v_j|| <= 1/4 - eps_B/2; take rho = 1.
    rho = (0.25 - 0.5 * eps_B) / radius if radius > 0.0 else 1.0
    return (v - c) * rho, rho, c


def fastsum(vt, x, bhat, N, m, alpha=2, taps="fp64"):
    """Alg. 1: complex f_RF at the (already scaled) nodes vt."""
    xhat = _nfft.adjoint_nfft(vt, x, N, m, alpha, taps)   # step 1
    fhat = bhat * xhat                                    # step 2
    return _nfft.nfft(vt, fhat, N, m, alpha, taps)        # step 3


def trig_polynomial_sum(vt, x, bhat, N):
    """O2: sum_i x_i K_RF(vt_j - vt_i) exactly, via direct NDFT sums (complex)."""
    xhat = _nfft.ndft_adjoint(vt, x, N)
    return _nfft.ndft(vt, bhat * xhat, N)


class NormalizedFastsum:
    """Alg. 2: setup (steps 1-4) and products (step 5) for the kernels of Sec. 2."""

    def __init__(self, v, sigma, N, m, p=None, eps_B=None, alpha=2, kernel="gaussian", taps="fp64"):
        if N % 2:
            raise ValueError("N must be even")
        if kernel not in _kernel.KERNELS:
            raise ValueError("unknown kernel %r" % (kernel,))
        self.kernel = kernel
        self.taps = taps                 # "bf16": window taps rounded to BF16 (not a paper construct)
        self.N, self.m, self.alpha = int(N), int(m), int(alpha)
        self.p = int(m if p is None else p)
        self.eps_B = float(self.p / self.N if eps_B is None else eps_B)
        self.vt, self.rho, self.center = scale_nodes(v, self.eps_B)       # step 1
        self.sigma = float(sigma)
        self.sigma_t = self.rho * self.sigma                               # step 2
        # output scale of Alg. 1 back to the original coordinates, and K(0) there
        self.out_scale = {"multiquadric": 1.0 / self.rho, "inverse_multiquadric": self.rho,
                          "gaussian_dsigma": self.rho}.get(kernel, 1.0)
        self.K0 = float(_kernel.radial(0.0, self.sigma, kernel))
        self.d = self.vt.shape[1]
        self.bhat = _kernel.fourier_coefficients(                          # step 3
            self.N, self.d, self.sigma_t, self.eps_B, self.p, kernel)
        ones = np.ones(self.vt.shape[0])
        self.degree = self.apply_Wtilde(ones) - self.K0 * ones             # step 4
        with np.errstate(divide="ignore", invalid="ignore"):
            self.dinv = 1.0 / np.sqrt(self.degree)

    def apply_Wtilde(self, x):
        """W~_E x, the real part of Alg. 1's output in the original coordinates."""
        return self.out_scale * fastsum(self.vt, x, self.bhat, self.N, self.m, self.alpha, self.taps).real

    def apply_W(self, x):
        """W_E x = W~_E x - K(0) x (Sec. 3, the diagonal identity)."""
        x = np.asarray(x, dtype=np.float64)
        return self.apply_Wtilde(x) - self.K0 * x

    def apply_A(self, x):
        """Alg. 2 step 5."""
        xs = self.dinv * np.asarray(x, dtype=np.float64)
        return self.dinv * (self.apply_Wtilde(xs) - self.K0 * xs)

    def apply_Ls(self, x):
        """L_s x = x - A x."""
        x = np.asarray(x, dtype=np.float64)
        return x - self.apply_A(x)

    def apply_W_exact_trig(self, x):
        """O2: W with K replaced by Re K_RF exactly (no window error)."""
        x = np.asarray(x, dtype=np.float64)
        return self.out_scale * trig_polynomial_sum(self.vt, x, self.bhat, self.N).real - self.K0 * x
