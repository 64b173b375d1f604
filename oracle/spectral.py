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


def nystrom_gaussian(apply_A, G, k, M):
    """Alg. 3 (Sec. 5.2, "Nystrom-Gaussian-NFFT"), step by step in numpy.

    apply_A  callable: n x c block -> A times the block (column by column).
    G        n x L random Gaussian block (passed in, so both sides use the same).
    Returns the k largest approximate eigenvalues of A (descending) and the
    matching orthonormal vectors (n x k).  numpy.linalg.qr / eigh are the
    library primitives of the QR and eigen-decomposition steps.
    """
    G = np.asarray(G, dtype=np.float64)
    Y = apply_A(G)                                   # step 3: Y = A G
    Q, _ = np.linalg.qr(Y)                           #         Q = orth(Y)
    B1 = apply_A(Q)                                  # step 4: B1 = A Q
    B2 = Q.T @ B1                                    #         B2 = Q^T B1
    B2 = 0.5 * (B2 + B2.T)
    sig, U = np.linalg.eigh(B2)                      # step 5: M largest positive
    order = np.argsort(sig)[::-1][:M]
    sig, U = sig[order], U[:, order]
    if not np.all(sig > 0.0):
        raise ValueError("B2 has fewer than M positive eigenvalues")
    Qh, Rh = np.linalg.qr(B1 @ U)                    # step 6: Qh Rh = B1 U_M
    T = Rh @ np.diag(1.0 / sig) @ Rh.T               # step 7: eig of Rh Sigma^-1 Rh^T
    lam, Uh = np.linalg.eigh(0.5 * (T + T.T))
    V = Qh @ Uh
    order = np.argsort(lam)[::-1][:k]                # step 8: k largest
    return lam[order], V[:, order]
