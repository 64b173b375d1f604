"""Gradients through the solve (beta L_s + diag(s)) u = f (Sec. 6.2.2).

The backward of the library (adjoint solve + assembly in its kernels) is
checked against central differences of the library's own forward solves in
f, s, beta and sigma, and the sigma gradient also against the dense oracle
(direct sums, numpy solves, central differences in sigma), which shares no
code with the GPU path.  torch autograd through paper_1808_04580_gb300.cg_solve
must give the same numbers.
"""
import numpy as np
import pytest
import torch

from oracle import direct
from paper_1808_04580_gb300 import Plan, cg_solve, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ARGS = dict(N=64, m=8, p=8)


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.fixture(scope="module")
def problem():
    rng = np.random.default_rng(3)
    n = 1200
    c = rng.uniform(-1, 1, (4, 3))
    v = c[rng.integers(0, 4, n)] + 0.2 * rng.standard_normal((n, 3))
    f = workloads.rhs(n, seed=4)
    s = rng.uniform(0.5, 2.0, n)
    w = rng.standard_normal(n)
    return v, f, s, w


def plans(v, sigma):
    p = Plan(gpu(v), sigma, ARGS["N"], ARGS["m"], ARGS["p"], -1.0, "fp64")
    dp = Plan(gpu(v), sigma, ARGS["N"], ARGS["m"], ARGS["p"], -1.0, "fp64", kernel="gaussian_dsigma")
    return p, dp


def loss(plan, f, s, beta, w):
    u, _, _, st = plan.cg_solve(gpu(f), beta=beta, shift=gpu(s), tol=1e-13, maxit=2000)
    assert st == 0
    return float(torch.dot(u, gpu(w)))


def test_backward_against_central_differences(problem):
    v, f, s, w = problem
    sigma, beta = 0.5, 0.7
    p, dp = plans(v, sigma)
    u, _, _, _ = p.cg_solve(gpu(f), beta=beta, shift=gpu(s), tol=1e-13, maxit=2000)
    gf, gs, gb, gsig, _, rel = p.cg_solve_backward(u, gpu(w), beta=beta, shift=gpu(s), dplan=dp, tol=1e-13, maxit=2000)
    assert rel <= 1e-13
    rng = np.random.default_rng(9)
    df, ds = rng.standard_normal(f.size), rng.standard_normal(s.size) * 0.1
    h = 1e-3
    fd_f = (loss(p, f + h * df, s, beta, w) - loss(p, f - h * df, s, beta, w)) / (2 * h)
    assert float(torch.dot(gf, gpu(df))) == pytest.approx(fd_f, rel=1e-8)
    fd_s = (loss(p, f, s + h * ds, beta, w) - loss(p, f, s - h * ds, beta, w)) / (2 * h)
    assert float(torch.dot(gs, gpu(ds))) == pytest.approx(fd_s, rel=1e-6)
    hb = 1e-4
    fd_b = (loss(p, f, s, beta + hb, w) - loss(p, f, s, beta - hb, w)) / (2 * hb)
    assert gb == pytest.approx(fd_b, rel=1e-6)
    hs = 1e-4
    pp, _ = plans(v, sigma + hs)
    pm, _ = plans(v, sigma - hs)
    fd_sig = (loss(pp, f, s, beta, w) - loss(pm, f, s, beta, w)) / (2 * hs)
    assert gsig == pytest.approx(fd_sig, rel=1e-6)


def test_sigma_gradient_against_dense_oracle(problem):
    """Dense O1 matrices, numpy solves, central differences in sigma."""
    v, f, s, w = problem
    sigma, beta = 0.5, 0.7
    n = v.shape[0]

    def dense_loss(sg):
        Ls = np.eye(n) - direct.normalized_adjacency(v, sg)
        u = np.linalg.solve(beta * Ls + np.diag(s), f)
        return float(w @ u)

    h = 1e-5
    ref = (dense_loss(sigma + h) - dense_loss(sigma - h)) / (2 * h)
    p, dp = plans(v, sigma)
    u, _, _, _ = p.cg_solve(gpu(f), beta=beta, shift=gpu(s), tol=1e-13, maxit=2000)
    _, _, _, gsig, _, _ = p.cg_solve_backward(u, gpu(w), beta=beta, shift=gpu(s), dplan=dp, tol=1e-13, maxit=2000)
    assert gsig == pytest.approx(ref, rel=1e-6)


def test_torch_autograd_matches_backward(problem):
    v, f, s, w = problem
    sigma, beta = 0.5, 0.7
    p, dp = plans(v, sigma)
    ft = gpu(f).requires_grad_(True)
    st = gpu(s).requires_grad_(True)
    bt = torch.tensor(beta, dtype=torch.float64, device=DEV, requires_grad=True)
    sgt = torch.tensor(sigma, dtype=torch.float64, device=DEV, requires_grad=True)
    u = cg_solve(p, ft, st, bt, sigma=sgt, dplan=dp, tol=1e-13, maxit=2000)
    (u * gpu(w)).sum().backward()
    gf, gs, gb, gsig, _, _ = p.cg_solve_backward(u.detach(), gpu(w), beta=beta, shift=gpu(s), dplan=dp,
                                                tol=1e-13, maxit=2000)
    assert torch.allclose(ft.grad, gf, rtol=1e-9, atol=1e-12)
    assert torch.allclose(st.grad, gs, rtol=1e-9, atol=1e-12)
    assert float(bt.grad) == pytest.approx(gb, rel=1e-9)
    assert float(sgt.grad) == pytest.approx(gsig, rel=1e-9)


def test_dsigma_plan_against_oracle(problem):
    """W_sigma x of the GAUSSIAN_DSIGMA plan against the dense oracle."""
    v, f, _, _ = problem
    p = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp64", kernel="gaussian_dsigma")
    y = p.apply_W(gpu(f)).cpu().numpy()
    ref = direct.apply_W(v, 0.5, f, "gaussian_dsigma")
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-9


def test_backward_rejects_mismatched_plans(problem):
    v, f, s, w = problem
    p, _ = plans(v, 0.5)
    other = Plan(gpu(v), 0.6, 64, 8, 8, -1.0, "fp64", kernel="gaussian_dsigma")
    u, _, _, _ = p.cg_solve(gpu(f), beta=0.7, shift=gpu(s), tol=1e-10, maxit=2000)
    from paper_1808_04580_gb300 import NflError
    with pytest.raises(NflError):
        p.cg_solve_backward(u, gpu(w), beta=0.7, shift=gpu(s), dplan=other)


# ---------------------------------------------------------------- node coordinates
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32c", 2e-5), ("fp32", 2e-5)])
@pytest.mark.parametrize("d", [3, 2])
def test_form_grad_nodes_against_dense_oracle(problem, prec, tol, d):
    """d(a^T A b)/dv of the library, element by element against the oracle's dense chain rule."""
    v, _, _, _ = problem
    v = np.ascontiguousarray(v[:, :d])
    rng = np.random.default_rng(31)
    a, b = rng.standard_normal(v.shape[0]), rng.standard_normal(v.shape[0])
    p = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, prec)
    g = p.form_grad_nodes(gpu(v), gpu(a), gpu(b)).cpu().numpy()
    ref = direct.form_grad_nodes(v, 0.5, a, b)
    assert g.shape == ref.shape
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < tol


def test_node_gradient_of_solve_against_dense_oracle(problem):
    """torch autograd dl/dv through cg_solve: element by element against
    beta * dense form gradient at the dense lambda, u; and the directional
    derivative against central differences of the dense loss."""
    v, f, s, w = problem
    sigma, beta = 0.5, 0.7
    n = v.shape[0]

    def dense_solution(vv):
        Ls = np.eye(n) - direct.normalized_adjacency(vv, sigma)
        return np.linalg.solve(beta * Ls + np.diag(s), f), beta * Ls + np.diag(s)

    vt = gpu(v).requires_grad_(True)
    p = Plan(vt.detach(), sigma, ARGS["N"], ARGS["m"], ARGS["p"], -1.0, "fp64")
    u = cg_solve(p, gpu(f), gpu(s), beta, v=vt, tol=1e-13, maxit=2000)
    (u * gpu(w)).sum().backward()
    g = vt.grad.cpu().numpy()

    ud, Md = dense_solution(v)
    lam = np.linalg.solve(Md, w)
    ref = beta * direct.form_grad_nodes(v, sigma, lam, ud)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-8

    dv = np.random.default_rng(5).standard_normal(v.shape)
    h = 1e-5
    fd = (w @ dense_solution(v + h * dv)[0] - w @ dense_solution(v - h * dv)[0]) / (2 * h)
    assert float((g * dv).sum()) == pytest.approx(fd, rel=1e-6)


def test_form_grad_nodes_rejects_other_kernels(problem):
    v, f, _, _ = problem
    from paper_1808_04580_gb300 import NflError
    p = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp64", kernel="inverse_multiquadric")
    with pytest.raises(NflError):
        p.form_grad_nodes(gpu(v), gpu(f), gpu(f))
