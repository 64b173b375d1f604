"""Pins for the oracle's Alg. 3 (Nystrom-Gaussian-NFFT, Sec. 5.2).

Alg. 3 builds the rank-M approximation (A Q)(Q^T A Q)^+_M (A Q)^T with
Q = orth(A G).  When A has rank <= M <= L the approximation is exact, and
with L = n (Q spans everything) it returns the exact top eigenpairs; both
reduce to a dense eigh of A, which is what these tests compare with.
"""
import numpy as np

from oracle import direct, fastsum, spectral


def _apply(A):
    return lambda X: A @ X


def test_exact_for_low_rank_matrices():
    rng = np.random.default_rng(0)
    n, r = 300, 8
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    lam_true = np.sort(rng.uniform(0.5, 2.0, r))[::-1]
    A = U @ np.diag(lam_true) @ U.T
    G = rng.standard_normal((n, 20))
    lam, V = spectral.nystrom_gaussian(_apply(A), G, 5, r)
    np.testing.assert_allclose(lam, lam_true[:5], rtol=1e-12)
    res = np.linalg.norm(A @ V - V * lam, axis=0)
    assert res.max() < 1e-12
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-12)


def test_full_sample_gives_the_exact_top_eigenpairs():
    rng = np.random.default_rng(1)
    v = rng.standard_normal((120, 3))
    A = direct.normalized_adjacency(v, 1.5)
    lam_ref = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert lam_ref[9] > 0.0                  # the M = 10 largest are positive
    G = rng.standard_normal((120, 120))
    lam, V = spectral.nystrom_gaussian(_apply(A), G, 10, 10)
    np.testing.assert_allclose(lam, lam_ref[:10], rtol=1e-10)
    assert np.linalg.norm(A @ V - V * lam, axis=0).max() < 1e-9


def test_with_the_fast_operator_approximates_the_top_eigenvalues():
    """L = 50, M = 10 on a 2000-node cloud (the paper's setup #2 kind)."""
    rng = np.random.default_rng(2)
    c = rng.uniform(-1, 1, (5, 3))
    v = c[rng.integers(0, 5, 2000)] + 0.3 * rng.standard_normal((2000, 3))
    fs = fastsum.NormalizedFastsum(v, 1.0, 32, 4, 4)
    A = direct.normalized_adjacency(v, 1.0)
    lam_ref = np.sort(np.linalg.eigvalsh(A))[::-1][:5]
    G = rng.standard_normal((2000, 50))
    apply_fast = lambda X: np.stack([fs.apply_A(X[:, j]) for j in range(X.shape[1])], axis=1)
    lam, _ = spectral.nystrom_gaussian(apply_fast, G, 5, 10)
    assert np.abs(lam - lam_ref).max() < 1e-3
