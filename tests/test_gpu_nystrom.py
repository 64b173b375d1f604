"""Alg. 3 (Nystrom-Gaussian-NFFT, Sec. 5.2) through the C ABI against the
oracle's step-by-step version, with the same random block G and the same
fast operator parameters, and against the dense top eigenpairs."""
import numpy as np
import pytest
import torch

from oracle import direct, fastsum, spectral
from paper_1808_04580_gb300 import NflError, Plan

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.fixture(scope="module")
def cloud():
    rng = np.random.default_rng(7)
    c = rng.uniform(-1, 1, (5, 3))
    v = c[rng.integers(0, 5, 2000)] + 0.3 * rng.standard_normal((2000, 3))
    G = rng.standard_normal((2000, 50))
    return v, G


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32c", 2e-6)])
def test_matches_oracle_alg3(cloud, prec, tol):
    v, G = cloud
    fs = fastsum.NormalizedFastsum(v, 1.0, 32, 4, 4)
    apply_fast = lambda X: np.stack([fs.apply_A(X[:, j]) for j in range(X.shape[1])], axis=1)
    lam_ref, V_ref = spectral.nystrom_gaussian(apply_fast, G, 5, 10)
    plan = Plan(gpu(v), 1.0, 32, 4, 4, -1.0, prec)
    lam, V = plan.nystrom_k_largest(5, 50, 10, G=gpu(G))
    np.testing.assert_allclose(lam, lam_ref, rtol=tol, atol=tol)
    V = V.cpu().numpy()
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-10)
    # vectors up to sign, where the eigenvalues are separated
    for j in range(3):
        cosang = abs(V[:, j] @ V_ref[:, j])
        assert cosang > 1 - 100 * tol


def test_close_to_dense_top_eigenpairs(cloud):
    v, _ = cloud
    A = direct.normalized_adjacency(v, 1.0)
    lam_dense = np.sort(np.linalg.eigvalsh(A))[::-1][:5]
    plan = Plan(gpu(v), 1.0, 32, 4, 4, -1.0, "fp64")
    lam, V = plan.nystrom_k_largest(5, 50, 10, seed=11)   # G drawn on the device
    assert np.abs(lam - lam_dense).max() < 1e-3
    res = np.linalg.norm(A @ V.cpu().numpy() - V.cpu().numpy() * lam, axis=0)
    assert res.max() < 5e-2


def test_invalid_sizes_rejected(cloud):
    v, _ = cloud
    plan = Plan(gpu(v), 1.0, 32, 4, 4, -1.0, "fp64")
    for k, L, M in [(0, 10, 5), (6, 10, 5), (5, 4, 5), (5, 600, 10)]:
        with pytest.raises(NflError):
            plan.nystrom_k_largest(k, L, M)


@pytest.mark.parametrize("k,L,M", [(3, 37, 9), (5, 64, 21)])
def test_odd_and_larger_sizes_match_oracle_alg3(cloud, k, L, M):
    """The device eigensolves of Alg. 3 (steps 5 and 7) at odd orders and L = 64,
    against the oracle's Alg. 3 with the same random block."""
    v, _ = cloud
    G = np.random.default_rng(L).standard_normal((v.shape[0], L))
    fs = fastsum.NormalizedFastsum(v, 1.0, 32, 4, 4)
    apply_fast = lambda X: np.stack([fs.apply_A(X[:, j]) for j in range(X.shape[1])], axis=1)
    lam_ref, _ = spectral.nystrom_gaussian(apply_fast, G, k, M)
    plan = Plan(gpu(v), 1.0, 32, 4, 4, -1.0, "fp64")
    lam, V = plan.nystrom_k_largest(k, L, M, G=gpu(G))
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-9, atol=1e-9)
    V = V.cpu().numpy()
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-10)
