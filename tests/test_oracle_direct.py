"""Pins for O1 (direct sums) against closed forms and the identities of Sec. 2."""
import math

import numpy as np
import pytest

from oracle import direct


def test_single_node_has_no_edges():
    v = np.array([[0.3, -0.1, 2.0]])
    assert direct.weight_matrix(v, 0.7).shape == (1, 1)
    assert direct.apply_W(v, 0.7, np.array([5.0]))[0] == 0.0


def test_two_nodes_closed_form():
    v = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])   # distance 0.5
    sigma = 0.8
    w = math.exp(-0.25 / 0.64)
    x = np.array([2.0, -3.0])
    np.testing.assert_allclose(direct.apply_W(v, sigma, x), [w * -3.0, w * 2.0], rtol=1e-15)
    np.testing.assert_allclose(direct.degree(v, sigma), [w, w], rtol=1e-15)
    # A = D^{-1/2} W D^{-1/2} = [[0, 1], [1, 0]] for two nodes
    np.testing.assert_allclose(direct.apply_A(v, sigma, x), [-3.0, 2.0], rtol=1e-14)


def test_weight_matrix_structure():
    rng = np.random.default_rng(0)
    v = rng.standard_normal((40, 3))
    W = direct.weight_matrix(v, 1.3)
    assert np.all(np.diag(W) == 0.0)
    assert np.array_equal(W, W.T)
    off = W[~np.eye(40, dtype=bool)]
    assert np.all(off > 0.0) and np.all(off <= 1.0)
    i, j = 3, 17
    assert W[i, j] == pytest.approx(math.exp(-np.sum((v[i] - v[j]) ** 2) / 1.3 ** 2), rel=1e-15)


def test_laplacian_identities():
    rng = np.random.default_rng(1)
    v = rng.uniform(-1.0, 1.0, (50, 2))
    sigma = 0.6
    L = direct.laplacian(v, sigma)
    np.testing.assert_allclose(L @ np.ones(50), 0.0, atol=1e-13)
    d = direct.degree(v, sigma)
    np.testing.assert_allclose(direct.apply_Ls(v, sigma, np.sqrt(d)), 0.0, atol=1e-13)


def test_quadratic_form_pair_loop():
    """u^T L u = 1/2 sum_{j,i} W_ji (u_j - u_i)^2 (Sec. 2), by an explicit pair loop."""
    rng = np.random.default_rng(2)
    v = rng.standard_normal((25, 3))
    u = rng.standard_normal(25)
    sigma = 0.9
    total = 0.0
    for j in range(25):
        for i in range(25):
            if i != j:
                w = math.exp(-sum((v[j, a] - v[i, a]) ** 2 for a in range(3)) / sigma ** 2)
                total += 0.5 * w * (u[j] - u[i]) ** 2
    assert u @ direct.laplacian(v, sigma) @ u == pytest.approx(total, rel=1e-13)


def test_normalized_spectrum():
    rng = np.random.default_rng(3)
    v = rng.standard_normal((80, 3))
    A = direct.normalized_adjacency(v, 1.0)
    lam = np.linalg.eigvalsh(np.eye(80) - A)
    assert lam.min() > -1e-12 and lam.max() < 2.0 + 1e-12
    assert abs(lam[0]) < 1e-12


def test_separated_clusters_give_zero_eigenvalues():
    """c clusters 100 sigma apart: exp underflows, c exact zero eigenvalues."""
    rng = np.random.default_rng(4)
    centres = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0], [0.0, 100.0, 0.0]])
    v = np.concatenate([c + 0.3 * rng.standard_normal((20, 3)) for c in centres])
    A = direct.normalized_adjacency(v, 1.0)
    lam = np.linalg.eigvalsh(np.eye(60) - A)
    assert np.all(np.abs(lam[:3]) < 1e-12)
    assert lam[3] > 1e-3


def test_c_rows_match_dense():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((300, 3))
    x = rng.standard_normal((300, 3))
    rows = np.array([0, 7, 150, 299])
    out = direct.rows_W(v, 0.8, x, rows)
    ref = direct.weight_matrix(v, 0.8) @ x
    np.testing.assert_allclose(out, ref[rows], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(direct.rows_W(v, 0.8, x[:, 1], rows), ref[rows, 1], rtol=1e-13)


# ---------------------------------------------------------------- node gradient
def _form(v, sigma, a, b):
    return float(a @ direct.normalized_adjacency(v, sigma) @ b)


def test_form_grad_nodes_central_differences():
    rng = np.random.default_rng(21)
    n, sigma = 25, 0.7
    v = rng.standard_normal((n, 3))
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    g = direct.form_grad_nodes(v, sigma, a, b)
    h = 1e-6
    fd = np.zeros_like(v)
    for k in range(n):
        for al in range(3):
            vp, vm = v.copy(), v.copy()
            vp[k, al] += h
            vm[k, al] -= h
            fd[k, al] = (_form(vp, sigma, a, b) - _form(vm, sigma, a, b)) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * np.abs(fd).max()


def test_form_grad_nodes_translation_invariant():
    rng = np.random.default_rng(22)
    v = rng.standard_normal((40, 2)) + 100.0
    a, b = rng.standard_normal(40), rng.standard_normal(40)
    g = direct.form_grad_nodes(v, 0.9, a, b)
    assert np.abs(g.sum(axis=0)).max() < 1e-12 * np.abs(g).sum()
    g0 = direct.form_grad_nodes(v - 100.0, 0.9, a, b)
    np.testing.assert_allclose(g, g0, rtol=1e-9, atol=1e-12 * np.abs(g).max())


def test_form_grad_nodes_two_nodes_is_zero():
    # n = 2: d_1 = d_2 = W_12, so A = [[0, 1], [1, 0]] whatever the nodes
    v = np.array([[0.1, 0.2, 0.3], [0.5, -0.1, 0.0]])
    a, b = np.array([1.3, -0.7]), np.array([0.2, 2.0])
    g = direct.form_grad_nodes(v, 0.4, a, b)
    # zero to rounding of its terms, each of size ~ (2 / sigma^2) |a| |b| ||v_1 - v_2||
    scale = 2.0 / 0.4 ** 2 * np.abs(a).max() * np.abs(b).max() * np.linalg.norm(v[0] - v[1])
    assert np.abs(g).max() < 1e-14 * scale
