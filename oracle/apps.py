"""Downstream consumers of the eigenpairs of L_s (Sec. 6.2), plain numpy.

Test infrastructure (the oracle); see the package docstring for who may use it.

* ``spectral_clustering`` -- Sec. 6.2.1: the k eigenvectors of the smallest
  eigenvalues of L_s (the largest of A) as columns of V, every row of V
  scaled to unit length, then k-means on the rows (Lloyd's iteration from
  given initial centres; the paper names k-means without fixing its
  initialisation).
* ``allen_cahn`` -- Sec. 6.2.1 (phase field): the convexity-splitting step
      (u - u_bar) / tau + eps L_s u + c u = -(1/eps) psi'(u_bar) + c u_bar + Omega (f - u_bar),
  psi(u) = (u^2 - 1)^2, written in the coefficients of u = V u_coef over the
  k eigenpairs (lambda_j, v_j) of L_s:
      u_j = (u_bar_j / tau + c u_bar_j - v_j^T psi'(u_bar) / eps + v_j^T Omega (f - u_bar))
            / (1 / tau + eps lambda_j + c),
  from u(0) = f, until the squared relative change of u falls below tol.
  The paper states the two-class form (f in {-1, 0, 1}); for C > 2 classes
  the reading used here is one-vs-rest: one run per class c with
  f = +1 on class-c training nodes, -1 on the other training nodes, and
  the class of the largest u.

Pins (tests/test_oracle_apps.py): clustering recovers well-separated blobs
exactly; with all n eigenpairs one coefficient step equals the node-space
linear solve of the same step; a fully labelled two-class f with a large
omega_0 stays at its signs; the step leaves u = f unchanged where psi'(f) = 0
and L_s f = 0.
"""
import numpy as np


def kmeans(X, centres, iters=100):
    """Lloyd's iteration: labels of the nearest centre, centres the label means."""
    C = np.array(centres, dtype=np.float64, copy=True)
    labels = None
    for _ in range(iters):
        d2 = ((X[:, None, :] - C[None, :, :]) ** 2).sum(axis=2)
        new = d2.argmin(axis=1)
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for j in range(C.shape[0]):
            if np.any(labels == j):
                C[j] = X[labels == j].mean(axis=0)
    return labels, C


def spectral_clustering(V, k, init_rows):
    """Ng-Jordan-Weiss: rows of the n x k eigenvector block to unit length, k-means
    from the rows init_rows as initial centres."""
    Y = V / np.linalg.norm(V, axis=1, keepdims=True)
    labels, _ = kmeans(Y, Y[np.asarray(init_rows)])
    return labels


def allen_cahn_step(u_bar, lam, V, f, omega, tau, eps, c):
    """One convexity-splitting step in the eigen-coefficients; returns the new u."""
    ub = V.T @ u_bar
    psi_p = 4.0 * u_bar ** 3 - 4.0 * u_bar
    rhs = ub / tau + c * ub - (V.T @ psi_p) / eps + V.T @ (omega * (f - u_bar))
    return V @ (rhs / (1.0 / tau + eps * lam + c))


def allen_cahn(lam, V, f, omega, tau=0.1, eps=10.0, c=None, tol=1e-10, maxit=500):
    """Two-class phase-field SSL from u(0) = f; returns u and the number of steps."""
    if c is None:
        c = 2.0 / eps + float(np.max(omega))
    u = np.asarray(f, dtype=np.float64).copy()
    for it in range(1, maxit + 1):
        new = allen_cahn_step(u, lam, V, f, omega, tau, eps, c)
        change = float(((new - u) ** 2).sum() / max((new ** 2).sum(), 1e-300))
        u = new
        if change < tol:
            return u, it
    return u, maxit


def allen_cahn_classes(lam, V, train_idx, train_lab, C, omega0=1e4, **kw):
    """One-vs-rest over C classes: argmax over the per-class u."""
    n = V.shape[0]
    omega = np.zeros(n)
    omega[train_idx] = omega0
    U = np.zeros((n, C))
    for cl in range(C):
        f = np.zeros(n)
        f[train_idx] = np.where(np.asarray(train_lab) == cl, 1.0, -1.0)
        U[:, cl], _ = allen_cahn(lam, V, f, omega, **kw)
    return U.argmax(axis=1), U
