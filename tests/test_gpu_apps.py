"""Downstream consumers of the eigenpairs (Sec. 6.2) on the GPU path against the
oracle's versions on dense eigenpairs: spectral clustering (Ng-Jordan-Weiss +
k-means) and phase-field (Allen-Cahn) semi-supervised learning."""
import numpy as np
import pytest
import torch

from oracle import apps as oapps
from oracle import spectral
from paper_1808_04580_gb300 import Plan, apps, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def same_partition(a, b):
    """Fraction of nodes on which two labellings agree under the best one-to-one
    relabelling (greedy on the contingency table; exact for near-equal partitions)."""
    a, b = np.asarray(a), np.asarray(b)
    ka, kb = a.max() + 1, b.max() + 1
    T = np.zeros((ka, kb), dtype=np.int64)
    np.add.at(T, (a, b), 1)
    hit = 0
    while T.size and T.max() > 0:
        i, j = np.unravel_index(T.argmax(), T.shape)
        hit += T[i, j]
        T[i, :] = -1
        T[:, j] = -1
    return hit / a.size


def test_spectral_clustering_blobs_exact():
    rng = np.random.default_rng(4)
    cent = rng.uniform(-3, 3, (4, 3))
    truth = np.repeat(np.arange(4), 500)
    v = cent[truth] + 0.05 * rng.standard_normal((2000, 3))
    p = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp64")
    init = [0, 500, 1000, 1500]
    lab, lam = apps.spectral_clustering(p, 4, init_rows=init)
    assert same_partition(lab.cpu().numpy(), truth) == 1.0
    lam_o, V_o = spectral.smallest_Ls(v, 0.5, 4)
    assert same_partition(lab.cpu().numpy(), oapps.spectral_clustering(V_o, 4, init)) == 1.0
    # eigenvalues of the fast operator: within its approximation error at N = 64 (the
    # blobs span [-3, 3]^3, so the scaled sigma is small) of the dense ones
    assert np.abs(lam - lam_o).max() < 5e-6


def test_spectral_clustering_voronoi_image_matches_dense():
    """A 60 x 60 image of 12 Voronoi colours, segmented into k = 4 classes (Sec. 6.2.1)."""
    v, _ = workloads.voronoi_image(60, 60, seed=3)
    p = Plan(gpu(v), 0.1, 128, 8, 8, -1.0, "fp64")
    init = [0, 1000, 2000, 3000]
    lab, lam = apps.spectral_clustering(p, 4, init_rows=init)
    lam_o, V_o = spectral.smallest_Ls(v, 0.1, 4)
    ref = oapps.spectral_clustering(V_o, 4, init)
    assert same_partition(lab.cpu().numpy(), ref) >= 0.999
    assert np.abs(lam - lam_o).max() < 1e-8


def test_allen_cahn_two_moons_matches_dense():
    v, y = workloads.two_moons(2000, noise=0.05, seed=1)
    p = Plan(gpu(v), 0.2, 128, 8, 8, -1.0, "fp64")
    lam, V, _, _ = p.lanczos_k_smallest(10, tol=1e-11)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.where(y < 0)[0], 5, replace=False),
                          rng.choice(np.where(y > 0)[0], 5, replace=False)])
    f = np.zeros(2000)
    f[idx] = y[idx]
    om = np.zeros(2000)
    om[idx] = 1e4
    u, steps = apps.allen_cahn(lam, V, gpu(f), gpu(om), tol=0.0, maxit=300)
    assert steps == 300
    lam_o, V_o = spectral.smallest_Ls(v, 0.2, 10)
    u_o, _ = oapps.allen_cahn(lam_o, V_o, f, om, tol=0.0, maxit=300)
    u = u.cpu().numpy()
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) < 1e-6
    assert (np.sign(u) == y).mean() > 0.85


def test_allen_cahn_five_classes_one_vs_rest():
    v, cls = workloads.five_centres(2000, seed=5)
    p = Plan(gpu(v), 1.0, 64, 8, 8, -1.0, "fp64")
    lam, V, _, _ = p.lanczos_k_smallest(5, tol=1e-11)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(np.where(cls == c)[0], 5, replace=False) for c in range(5)])
    pred, _ = apps.allen_cahn_classes(lam, V, idx, cls[idx], 5, maxit=300, tol=0.0)
    pred = pred.cpu().numpy()
    lam_o, V_o = spectral.smallest_Ls(v, 1.0, 5)
    ref, _ = oapps.allen_cahn_classes(lam_o, V_o, idx, cls[idx], 5, maxit=300, tol=0.0)
    assert (pred == ref).mean() >= 0.999
    assert (pred == cls).mean() > 0.95
