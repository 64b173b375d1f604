"""Downstream consumers of the eigenpairs of L_s (Sec. 6.2): spectral clustering
and semi-supervised learning by the phase-field (Allen-Cahn) method.

The eigenpairs come from the library's Lanczos process (nfl_lanczos_k_smallest,
Sec. 4).  What follows them is small and dense -- n x k blocks with k of order
ten -- and runs as torch operations on the device: row normalisation and
k-means (Lloyd's iteration) for Sec. 6.2.1, and the convexity-splitting step
of Sec. 6.2.1 (phase field) in the k eigen-coefficients,

    u_j = (ub_j / tau + c ub_j - v_j^T psi'(ub) / eps + v_j^T Omega (f - ub))
          / (1 / tau + eps lambda_j + c),          psi(u) = (u^2 - 1)^2,

from u(0) = f until the squared relative change of u = V u_coef is below tol.
The paper gives the two-class form; more classes are handled one-vs-rest
(one run per class, the class of the largest u).
"""
import numpy as np
import torch

from .nfl import Plan


def kmeans(X, centres, iters=100):
    """Lloyd's iteration on the rows of X (n x k, device) from the given centres:
    (labels, centres)."""
    C = centres.clone()
    labels = None
    for _ in range(iters):
        new = torch.cdist(X, C).argmin(dim=1)
        if labels is not None and torch.equal(new, labels):
            break
        labels = new
        for j in range(C.shape[0]):
            sel = labels == j
            if bool(sel.any()):
                C[j] = X[sel].mean(dim=0)
    return labels, C


def spectral_clustering(plan, k, init_rows=None, tol=1e-10, seed=0):
    """Ng-Jordan-Weiss clustering into k classes (Sec. 6.2.1): the k eigenvectors of
    the smallest eigenvalues of L_s, rows to unit length, k-means.  init_rows picks
    the rows that start k-means (default: farthest-point choice from row 0).
    Returns (labels on the device, eigenvalues ascending)."""
    if not isinstance(plan, Plan):
        raise TypeError("plan must be a Plan")
    lam, V, _, _ = plan.lanczos_k_smallest(k, tol=tol, seed=seed)
    Y = V / torch.linalg.norm(V, dim=1, keepdim=True)
    if init_rows is None:
        init_rows = [0]
        d = torch.linalg.norm(Y - Y[0], dim=1)
        for _ in range(1, k):
            nxt = int(d.argmax())
            init_rows.append(nxt)
            d = torch.minimum(d, torch.linalg.norm(Y - Y[nxt], dim=1))
    labels, _ = kmeans(Y, Y[torch.as_tensor(init_rows, device=Y.device)])
    return labels, lam


def allen_cahn(lam, V, f, omega, tau=0.1, eps=10.0, c=None, tol=1e-10, maxit=500):
    """Two-class phase-field SSL from u(0) = f (Sec. 6.2.1); lam (k,) eigenvalues of
    L_s, V (n, k) its eigenvectors, f and omega (n,) on the device.  Returns (u, steps)."""
    lam = torch.as_tensor(np.asarray(lam), dtype=torch.float64, device=V.device)
    if c is None:
        c = 2.0 / eps + float(omega.max())
    den = 1.0 / tau + eps * lam + c
    u = f.clone()
    for it in range(1, maxit + 1):
        ub = V.t() @ u
        psi_p = 4.0 * u ** 3 - 4.0 * u
        rhs = ub / tau + c * ub - (V.t() @ psi_p) / eps + V.t() @ (omega * (f - u))
        new = V @ (rhs / den)
        change = float(((new - u) ** 2).sum() / torch.clamp((new ** 2).sum(), min=1e-300))
        u = new
        if change < tol:
            return u, it
    return u, maxit


def allen_cahn_classes(lam, V, train_idx, train_lab, C, omega0=1e4, **kw):
    """One-vs-rest phase-field SSL over C classes: (labels, U (n, C)) on the device."""
    n = V.shape[0]
    idx = torch.as_tensor(train_idx, device=V.device)
    lab = torch.as_tensor(train_lab, device=V.device)
    omega = torch.zeros(n, dtype=torch.float64, device=V.device)
    omega[idx] = omega0
    U = torch.zeros((n, C), dtype=torch.float64, device=V.device)
    for cl in range(C):
        f = torch.zeros(n, dtype=torch.float64, device=V.device)
        f[idx] = torch.where(lab == cl, 1.0, -1.0).to(torch.float64)
        U[:, cl], _ = allen_cahn(lam, V, f, omega, **kw)
    return U.argmax(dim=1), U
