"""O4/O5: dense eigendecomposition and dense solves for small n.

Test infrastructure (the oracle); see the package docstring for who may use it.

Sec. 2: the k smallest eigenvalues of L_s are 1 minus the k largest of
A = D^{-1/2} W D^{-1/2}.  Sec. 6.1 measures eigenvalue error as
max_j |lambda_j - lambda_j^direct| (eq. (max_ev_error)) and residuals as
max_j ||A v_j - lambda_j v_j||_2 (eq. (max_res_norm)).  Sec. 6.2.2 solves
(I + beta L_s) u = f (eq. (ssl::system)) by CG; O5 solves the general
(beta L_s + diag(s)) u = f densely.

numpy.linalg.eigh / solve are the library primitives; nothing else.
"""
import numpy as np

from . import direct as _direct


def smallest_Ls(v, sigma, k):
    """(eigenvalues ascending, eigenvectors as columns) of the k smallest of L_s."""
    A = _direct.normalized_adjacency(v, sigma)
    n = A.shape[0]
    lam, V = np.linalg.eigh(np.eye(n) - A)
    return lam[:k], V[:, :k]


def smallest_of_matrix(M, k):
    lam, V = np.linalg.eigh(0.5 * (M + M.T))
    return lam[:k], V[:, :k]


def solve_shifted(v, sigma, beta, shift, f):
    """Solve (beta L_s + diag(shift)) u = f densely."""
    A = _direct.normalized_adjacency(v, sigma)
    n = A.shape[0]
    M = beta * (np.eye(n) - A) + np.diag(np.asarray(shift, dtype=np.float64))
    return np.linalg.solve(M, np.asarray(f, dtype=np.float64))


def residual_norms(Aop, lam, V):
    """max_j ||A v_j - lambda_j v_j||_2 with A given as a callable."""
    res = []
    for j in range(V.shape[1]):
        res.append(np.linalg.norm(Aop(V[:, j]) - lam[j] * V[:, j]))
    return np.array(res)
