"""O1, the ground truth: direct FP64 sums with the kernel weight matrix.

Test infrastructure (the oracle); see the package docstring for who may use it.

Sec. 2, eq. (W_gaussian): W_ji = exp(-||v_j - v_i||^2 / sigma^2) for j != i,
W_jj = 0; the other kernels of Sec. 2 (Laplacian RBF exp(-r/sigma), the
multiquadric (r^2 + c^2)^{1/2} and its inverse, r = ||v_j - v_i||, shape
parameter in ``sigma``) and the sigma-derivative of the Gaussian by name.  Degree d_j = sum_i W_ji; D = diag(d); L = D - W;
A = D^{-1/2} W D^{-1/2}; L_s = I - A (Sec. 2, eq. (nomlap)).
Everything is in the original coordinates (no scaling, no shift).

Dense numpy versions for small n; ``rows_W`` sums selected rows over all n
sources in plain C (direct.c, built by oracle/build.py) for large n.

Pins (tests/test_oracle_direct.py): n = 1 and n = 2 closed forms; L 1 = 0;
L_s D^{1/2} 1 = 0; the quadratic form u^T L u = 1/2 sum W_ji (u_j - u_i)^2
(Sec. 2) by an explicit pair loop; spectrum of L_s in [0, 2] with a zero
eigenvalue; c well-separated clusters give c (numerically) zero eigenvalues;
the C row sums against the dense matrix; the node-coordinate gradient of
a^T A b against central differences of the dense form, its translation
invariance (the node gradients sum to zero) and n = 2 (A is constant).
"""
import ctypes
import os

import numpy as np


def _radial(r2, sigma, kernel):
    """K from the squared distance, written out for each kernel of Sec. 2."""
    if kernel == "gaussian":
        return np.exp(-r2 / sigma ** 2)
    if kernel == "laplacian_rbf":
        return np.exp(-np.sqrt(r2) / sigma)
    if kernel == "multiquadric":
        return np.sqrt(r2 + sigma ** 2)
    if kernel == "inverse_multiquadric":
        return 1.0 / np.sqrt(r2 + sigma ** 2)
    if kernel == "gaussian_dsigma":
        return 2.0 * r2 / sigma ** 3 * np.exp(-r2 / sigma ** 2)
    raise ValueError("unknown kernel %r" % (kernel,))


def weight_matrix(v, sigma, kernel="gaussian"):
    """Dense W (n x n), zero diagonal."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    diff = v[:, None, :] - v[None, :, :]
    W = _radial((diff ** 2).sum(axis=2), sigma, kernel)
    np.fill_diagonal(W, 0.0)
    return W


def degree(v, sigma, kernel="gaussian"):
    return weight_matrix(v, sigma, kernel).sum(axis=1)


def apply_W(v, sigma, x, kernel="gaussian"):
    return weight_matrix(v, sigma, kernel) @ np.asarray(x, dtype=np.float64)


def normalized_adjacency(v, sigma, kernel="gaussian"):
    """A = D^{-1/2} W D^{-1/2}."""
    W = weight_matrix(v, sigma, kernel)
    dinv = 1.0 / np.sqrt(W.sum(axis=1))
    return dinv[:, None] * W * dinv[None, :]


def apply_A(v, sigma, x, kernel="gaussian"):
    return normalized_adjacency(v, sigma, kernel) @ np.asarray(x, dtype=np.float64)


def apply_Ls(v, sigma, x, kernel="gaussian"):
    x = np.asarray(x, dtype=np.float64)
    return x - apply_A(v, sigma, x, kernel)


def laplacian(v, sigma, kernel="gaussian"):
    """L = D - W."""
    W = weight_matrix(v, sigma, kernel)
    return np.diag(W.sum(axis=1)) - W


# --------------------------------------------------------------------------
# Plain-C row sums for large n.

_LIB = None


def form_grad_nodes(v, sigma, a, b):
    """Gradient of G(v) = a^T A(v) b in the node coordinates (Gaussian kernel), by
    the chain rule on the dense matrices: A_ij = W_ij / sqrt(d_i d_j) with
    d_i = sum_l W_il, so dG/dW_ij = a~_i b~_j + dG/dd_i with a~ = a / sqrt(d),
    b~ = b / sqrt(d), dG/dd_i = -(a~_i (W b~)_i + b~_i (W a~)_i) / (2 d_i); and
    dW_ij/dv_k = -(2 / sigma^2) W_ij (v_i - v_j) (delta_ik - delta_jk)
    (Sec. 2, eqs. (W_gaussian) and (nomlap)).  Returns n x d.
    """
    v = np.asarray(v, dtype=np.float64)
    W = weight_matrix(v, sigma)
    d = W.sum(axis=1)
    at, bt = a / np.sqrt(d), b / np.sqrt(d)
    gd = -0.5 * (at * (W @ bt) + bt * (W @ at)) / d
    M = np.outer(at, bt) + gd[:, None]                  # dG/dW_ij
    T = (M * W)[:, :, None] * (v[:, None, :] - v[None, :, :])
    return -(2.0 / sigma ** 2) * (T.sum(axis=1) - T.sum(axis=0))


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(__file__), "_build", "liboracle_direct.so")
        if not os.path.exists(path):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_kernel_rows.restype = ctypes.c_int
        lib.oracle_kernel_rows.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        _LIB = lib
    return _LIB


def max_threads():
    return int(_lib().oracle_max_threads())


_KIND = {"gaussian": 0, "laplacian_rbf": 1, "multiquadric": 2, "inverse_multiquadric": 3, "gaussian_dsigma": 4}


def rows_W(v, sigma, x, rows, nthreads=0, kernel="gaussian"):
    """(W x)_j for j in rows, each summed over all n sources, x (n,) or (n, r)."""
    v = np.ascontiguousarray(np.atleast_2d(v), dtype=np.float64)
    n, d = v.shape
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    X = np.asfortranarray(x.reshape(n, -1))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((rows.size, X.shape[1]), dtype=np.float64, order="F")
    rc = _lib().oracle_kernel_rows(
        v.ctypes.data, n, d, _KIND[kernel], float(sigma), X.ctypes.data, X.shape[1], n,
        rows.ctypes.data, rows.size, out.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle_kernel_rows: bad arguments")
    return out[:, 0] if squeeze else out
