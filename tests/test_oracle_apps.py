"""Pins of the oracle's downstream consumers (spectral clustering, phase-field SSL)."""
import numpy as np

from oracle import apps, direct, spectral


def _blobs(k, per, seed):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-3, 3, (k, 3))
    lab = np.repeat(np.arange(k), per)
    return centres[lab] + 0.05 * rng.standard_normal((k * per, 3)), lab


def test_spectral_clustering_recovers_separated_blobs():
    v, lab = _blobs(4, 60, 1)
    lam, V = spectral.smallest_Ls(v, 0.5, 4)
    got = apps.spectral_clustering(V, 4, init_rows=[0, 60, 120, 180])
    # the same partition up to a relabelling
    pairs = {(a, b) for a, b in zip(lab, got)}
    assert len(pairs) == 4 and len({a for a, _ in pairs}) == 4 and len({b for _, b in pairs}) == 4


def test_kmeans_fixed_point_of_exact_centres():
    X = np.array([[0.0, 0.0], [0.0, 1.0], [10.0, 0.0], [10.0, 1.0]])
    lab, C = apps.kmeans(X, np.array([[0.0, 0.5], [10.0, 0.5]]))
    assert list(lab) == [0, 0, 1, 1]
    np.testing.assert_allclose(C, [[0.0, 0.5], [10.0, 0.5]])


def test_coefficient_step_with_all_eigenpairs_is_the_node_space_solve():
    rng = np.random.default_rng(2)
    v = rng.standard_normal((40, 3))
    Ls = np.eye(40) - direct.normalized_adjacency(v, 1.0)
    lam, V = np.linalg.eigh(Ls)
    f = np.zeros(40)
    f[:5] = [1, -1, 1, 1, -1]
    omega = np.zeros(40)
    omega[:5] = 7.0
    u_bar = rng.uniform(-1, 1, 40)
    tau, eps, c = 0.1, 2.0, 3.0
    got = apps.allen_cahn_step(u_bar, lam, V, f, omega, tau, eps, c)
    rhs = u_bar / tau + c * u_bar - (4 * u_bar ** 3 - 4 * u_bar) / eps + omega * (f - u_bar)
    ref = np.linalg.solve(np.eye(40) / tau + eps * Ls + c * np.eye(40), rhs)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_step_keeps_a_stationary_labelling():
    # f = +-1 on whole connected components of a graph with no edges between
    # them: L_s f = 0 needs f proportional to D^{1/2} 1 per component, so take
    # components of two nodes at equal degree; psi'(+-1) = 0, Omega (f - f) = 0
    v = np.array([[0.0, 0, 0], [0.1, 0, 0], [50.0, 0, 0], [50.1, 0, 0]])
    Ls = np.eye(4) - direct.normalized_adjacency(v, 0.5)
    lam, V = np.linalg.eigh(Ls)
    f = np.array([1.0, 1.0, -1.0, -1.0])
    u = apps.allen_cahn_step(f, lam, V, f, np.full(4, 10.0), 0.1, 10.0, 11.0)
    np.testing.assert_allclose(u, f, atol=1e-12)


def test_fully_labelled_two_classes_keep_their_signs():
    v, lab = _blobs(2, 50, 3)
    lam, V = spectral.smallest_Ls(v, 0.5, 6)
    f = np.where(lab == 0, 1.0, -1.0)
    u, it = apps.allen_cahn(lam, V, f, np.full(100, 1e4))
    assert np.array_equal(np.sign(u), f) and it < 500
