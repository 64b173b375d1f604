"""GPU path (through the C ABI) against the CPU oracle, element by element.

FP64 plans must match the oracle's plain Alg. 1/2 (O3, same N, m, p, eps_B,
Kaiser-Bessel window, oversampling 2) to 1e-10 relative; the mixed forms are
held to their own tolerances against the same O3 output.  Sizes span several
tiles and ragged tails; edge cases: n = 1, 2, 3, coincident nodes, supports
that wrap around the periodic grid, d = 1, 2, 3.
"""
import math

import numpy as np
import pytest
import torch
from _norms import assert_close

from oracle import direct, fastsum, spectral
from paper_1808_04580_gb300 import KERNELS, NflError, Plan, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cloud(kind, n, d, seed):
    rng = np.random.default_rng(seed)
    if kind == "spiral":
        return workloads.two_arm_spiral(n, seed=seed)[:, :d]
    if kind == "normal":
        return rng.standard_normal((n, d))
    if kind == "clusters":
        c = rng.uniform(-1, 1, (4, d))
        return c[rng.integers(0, 4, n)] + 0.05 * rng.standard_normal((n, d))
    raise ValueError(kind)


# (kind, n, d, sigma, N, m, p, eps_B)
FP64_CASES = [
    ("spiral", 1000, 3, 0.5, 16, 4, 4, -1.0),
    ("normal", 17, 3, 1.0, 8, 2, 2, -1.0),
    ("normal", 3, 3, 1.0, 16, 3, 3, -1.0),
    ("clusters", 2500, 3, 0.3, 32, 3, 3, -1.0),
    ("normal", 700, 2, 0.5, 32, 3, 3, -1.0),
    ("clusters", 900, 2, 0.2, 64, 6, 6, -1.0),
    ("normal", 500, 1, 0.3, 64, 5, 5, -1.0),
    ("normal", 200, 3, 1.0, 8, 4, 4, 0.125),     # taps wrap around the periodic grid
    ("normal", 300, 2, 1.0, 8, 6, 2, 0.125),     # wrap, d = 2
    ("spiral", 800, 3, 3.5, 16, 2, 2, 0.0),      # eps_B = 0 (paper's setup #1 form)
]


@pytest.mark.parametrize("case", FP64_CASES, ids=lambda c: "%s-n%d-d%d-N%d-m%d" % (c[0], c[1], c[2], c[4], c[5]))
def test_fp64_matches_alg2_oracle(case):
    kind, n, d, sigma, N, m, p, eps_B = case
    v = _cloud(kind, n, d, seed=n + d)
    x = workloads.rhs(n, seed=n)
    ref = fastsum.NormalizedFastsum(v, sigma, N, m, p, None if eps_B < 0 else eps_B)
    plan = Plan(gpu(v), sigma, N, m, p, eps_B, "fp64")
    info = plan.info()
    assert info["rho"] == pytest.approx(ref.rho, rel=1e-14)
    xt = gpu(x)
    assert_close(plan.apply_W(xt).cpu().numpy(), ref.apply_W(x), 1e-10)
    deg = plan.degree().cpu().numpy()
    np.testing.assert_allclose(deg, ref.degree, rtol=1e-10, atol=1e-12 * np.abs(ref.degree).max())
    # Lemma 3.1: a coarse plan can push a small degree below zero (eps >= eta);
    # the oracle sees the same degrees, and the GPU must then refuse A and L_s.
    assert info["degree_ok"] == int(ref.degree.min() > 0)
    if not info["degree_ok"]:
        with pytest.raises(NflError):
            plan.apply_A(xt)
        return
    assert_close(plan.apply_A(xt).cpu().numpy(), ref.apply_A(x), 1e-10)
    assert_close(plan.apply_Ls(xt).cpu().numpy(), ref.apply_Ls(x), 1e-10)


def _dense_clusters(n, n_dense, seed):
    """Four normal clusters (std 0.05 in [-1, 1]^3) plus n_dense nodes in one very tight
    cluster (std 0.002), which puts more than one 8192-node chunk into a tile."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (4, 3))
    v = c[rng.integers(0, 4, n)] + 0.05 * rng.standard_normal((n, 3))
    v[:n_dense] = c[0] + 0.002 * rng.standard_normal((n_dense, 3))
    return v


# the plain FP64 form at the large windows in 3-D: the cell-run spread (m = 6 on 4^3-cell
# tiles, m = 7, 8 on 2^3-cell tiles) and the FP64 interpolation, N = 128 (the grid of the
# 10^7-node workload) included; (m, N, n, sigma)
FP64_LARGE_M = [(6, 128, 12000, 0.3), (6, 32, 12000, 0.6), (7, 32, 10000, 0.6), (8, 32, 10000, 0.6)]


@pytest.mark.parametrize("case", FP64_LARGE_M, ids=lambda c: "m%d-N%d-n%d" % c[:3])
def test_fp64_large_windows_match_alg2_oracle(case):
    m, N, n, sigma = case
    v = _dense_clusters(n, 9000, seed=70 + m + N)
    x = workloads.rhs(n, seed=71 + m)
    ref = fastsum.NormalizedFastsum(v, sigma, N, m, m)
    plan = Plan(gpu(v), sigma, N, m, m, -1.0, "fp64")
    info = plan.info()
    assert info["work_items"] > info["tiles"]          # a tile of several chunks
    xt = gpu(x)
    err = assert_close(plan.apply_W(xt).cpu().numpy(), ref.apply_W(x), 1e-10, x=x)
    print("FP64 m=%d N=%d W x against Alg. 2:" % (m, N), err)
    deg = plan.degree().cpu().numpy()
    np.testing.assert_allclose(deg, ref.degree, rtol=1e-10, atol=1e-12 * np.abs(ref.degree).max())
    assert info["degree_ok"] == 1
    yl = plan.apply_Ls(xt).cpu().numpy()
    # L_s x = x - A x: the A x parts
    assert_close(x - yl, x - ref.apply_Ls(x), 1e-10)


def test_spiral5k_fp64_against_alg2_and_direct():
    """Small FP64 workload: n = 5000 two-arm spiral, sigma 0.5, N 32, m 4, p 4."""
    v = workloads.two_arm_spiral(5000, seed=0)
    x = workloads.rhs(5000, seed=1)
    plan = Plan(gpu(v), 0.5, 32, 4, 4, -1.0, "fp64")
    y = plan.apply_W(gpu(x)).cpu().numpy()
    ref = fastsum.NormalizedFastsum(v, 0.5, 32, 4, 4)
    assert_close(y, ref.apply_W(x), 1e-10)
    # against the exact sum: within the method's own error (window m = 4 ~ 1e-7)
    assert_close(y, direct.apply_W(v, 0.5, x), 5e-7)
    yl = plan.apply_Ls(gpu(x)).cpu().numpy()
    assert_close(yl, ref.apply_Ls(x), 1e-10)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("fp32c", 1e-6)])
def test_mixed_precision_forms(prec, tol):
    v = _cloud("clusters", 3000, 3, seed=11)
    x = workloads.rhs(3000, seed=12)
    ref = fastsum.NormalizedFastsum(v, 0.3, 32, 4, 4)
    plan = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, prec)
    assert_close(plan.apply_W(gpu(x)).cpu().numpy(), ref.apply_W(x), tol)
    assert_close(plan.apply_A(gpu(x)).cpu().numpy(), ref.apply_A(x), tol)
    assert plan.info()["device_error"] == 0


# every 3-D tile shape of the spread kernels (warp-slice: m = 2, 3, 4, 6; cell-run:
# m = 7, 8; shared-tile: m = 5) and of the tensor-core interpolation, both mixed forms


@pytest.mark.parametrize("prec,tol", [("fp32c", 2e-6), ("fp32", 1e-5)])
@pytest.mark.parametrize("dense", [False, True])
def test_dense_cell_spread_matches_alg2_oracle(prec, tol, dense):
    """m = 6 in 3-D: tiles with many nodes per occupied cell are spread by Chebyshev
    moments (one-column products), the others by the warp-slice kernel; both kinds of
    cloud against the oracle's Alg. 2, and the one-column product against a block
    product (every tile by the warp-slice kernel)."""
    n = 6000
    rng = np.random.default_rng(33)
    if dense:
        c = rng.uniform(-1, 1, (3, 3))
        v = c[rng.integers(0, 3, n)] + 0.02 * rng.standard_normal((n, 3))
    else:
        v = rng.uniform(-1, 1, (n, 3))
    x = workloads.rhs(n, seed=34)
    ref = fastsum.NormalizedFastsum(v, 0.5, 32, 6, 6)
    plan = Plan(gpu(v), 0.5, 32, 6, 6, -1.0, prec)
    info = plan.info()
    assert (info["dense_items"] > 0) == dense
    y = plan.apply_W(gpu(x)).cpu().numpy()
    err = assert_close(y, ref.apply_W(x), tol, x=x)
    print("m=6 %s dense=%s (%d dense items):" % (prec, dense, info["dense_items"]), err)
    np.testing.assert_allclose(plan.degree().cpu().numpy(), ref.degree, rtol=tol)
    X = np.stack([x, -x], axis=1)
    Yb = plan.apply_W(gpu(X)).cpu().numpy()                 # block of 2 columns
    assert_close(Yb[:, 0], y, tol)


def _slab_cloud(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "hot_cell":
        # 85 % of the nodes inside one cell: one slab cut into several work items
        v = rng.uniform(-1, 1, (n, 3))
        hot = rng.random(n) < 0.85
        v[hot] = 0.3 + 1e-4 * rng.standard_normal((int(hot.sum()), 3))
        return v
    # a few tight clusters
    c = rng.uniform(-1, 1, (3, 3))
    return c[rng.integers(0, 3, n)] + 0.03 * rng.standard_normal((n, 3))


@pytest.mark.parametrize("prec,tol", [("fp32c", 2e-6), ("fp32", 1e-5)])
@pytest.mark.parametrize("kind,n,N,p,eps_B", [("hot_cell", 12000, 32, 6, -1.0), ("clusters", 4000, 8, 2, 0.125)])
def test_slab_moments_edge_cases(kind, n, N, p, eps_B, prec, tol):
    """The slab-moment spread and interpolation (m = 6, dense tiles) on a cell holding
    most of the nodes (one slab cut into several work items, each adding its block into
    the same grid positions) and on clusters whose supports wrap around the periodic
    grid (N = 8, eps_B = 1/8: the box spans 7 + 2m + 2 > 2N positions per axis): W, L_s
    and the degrees against the oracle's Alg. 2, before and after the autotuner re-cuts
    the slabs."""
    v = _slab_cloud(kind, n, 41)
    x = workloads.rhs(n, seed=42)
    ref = fastsum.NormalizedFastsum(v, 0.5, N, 6, p, None if eps_B < 0 else eps_B)
    plan = Plan(gpu(v), 0.5, N, 6, p, eps_B, prec)
    info = plan.info()
    assert info["dense_items"] > 0
    if kind == "hot_cell":
        # the hot slab alone (10,200 nodes) is at least two pieces of the spread's
        # and of the interpolation's list (at most 8192 nodes each)
        assert info["dense_items"] >= 2 and info["dense_chunk"] <= 8192
    yw_ref, yl_ref = ref.apply_W(x), ref.apply_Ls(x)
    for tuned in (False, True):
        if tuned:
            plan.autotune()
        err = assert_close(plan.apply_W(gpu(x)).cpu().numpy(), yw_ref, tol, x=x)
        print("slab %s %s tuned=%s:" % (kind, prec, tuned), err)
        yl = plan.apply_Ls(gpu(x)).cpu().numpy()
        assert_close(x - yl, x - yl_ref, tol)
    # degrees here span two orders of magnitude (87 beside the hot cell's 10^4): the FP32
    # error is relative to the largest sums, as in the paper's error measure of W x
    # (max error over ||x||_1 K(0); x = 1), so the bound is absolute at tol * max d
    deg = plan.degree().cpu().numpy()
    np.testing.assert_allclose(deg, ref.degree, rtol=tol, atol=tol * ref.degree.max())
    assert plan.info()["device_error"] == 0


@pytest.mark.parametrize("prec,tol", [("fp32c", 2e-6), ("fp32", 1e-5)])
@pytest.mark.parametrize("m,N", [(2, 16), (3, 16), (4, 32), (6, 32), (7, 32), (5, 32), (8, 32)])
def test_mixed_forms_each_window_size(m, N, prec, tol):
    n = 2600
    v = _cloud("clusters", n, 3, seed=30 + m)
    x = workloads.rhs(n, seed=31 + m)
    ref = fastsum.NormalizedFastsum(v, 0.4, N, m, m)
    plan = Plan(gpu(v), 0.4, N, m, m, -1.0, prec)
    y = plan.apply_W(gpu(x)).cpu().numpy()
    assert_close(y, ref.apply_W(x), tol)
    np.testing.assert_allclose(plan.degree().cpu().numpy(), ref.degree, rtol=tol)
    yl = plan.apply_Ls(gpu(x)).cpu().numpy()
    assert_close(x - yl, x - ref.apply_Ls(x), tol)
    assert plan.info()["device_error"] == 0


# supports that wrap around the periodic grid (span > 2N), and d = 1, 2, in the mixed forms
MIXED_EDGE_CASES = [
    ("normal", 200, 3, 1.0, 8, 4, 4, 0.125),
    ("normal", 300, 3, 1.0, 8, 2, 2, 0.125),
    ("normal", 300, 2, 1.0, 8, 6, 2, 0.125),
    ("normal", 700, 2, 0.5, 32, 3, 3, -1.0),
    ("normal", 500, 1, 0.3, 64, 5, 5, -1.0),
]


@pytest.mark.parametrize("prec,tol", [("fp32c", 2e-6), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", MIXED_EDGE_CASES, ids=lambda c: "n%d-d%d-N%d-m%d" % (c[1], c[2], c[4], c[5]))
def test_mixed_forms_wrap_and_low_dimensions(case, prec, tol):
    kind, n, d, sigma, N, m, p, eps_B = case
    v = _cloud(kind, n, d, seed=40 + n)
    x = workloads.rhs(n, seed=41 + n)
    ref = fastsum.NormalizedFastsum(v, sigma, N, m, p, None if eps_B < 0 else eps_B)
    plan = Plan(gpu(v), sigma, N, m, p, eps_B, prec)
    assert_close(plan.apply_W(gpu(x)).cpu().numpy(), ref.apply_W(x), tol)
    assert plan.info()["device_error"] == 0


# the other kernels of Sec. 2 through Alg. 2 (scaling rule, K(0), output scale)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 2e-6)])
@pytest.mark.parametrize("kind,d", [("laplacian_rbf", 3), ("multiquadric", 3), ("inverse_multiquadric", 3),
                                    ("multiquadric", 2), ("inverse_multiquadric", 1)])


def test_kernel_variants_match_alg2_oracle(kind, d, prec, tol):
    n = 1500
    v = _cloud("clusters", n, d, seed=50 + d)
    x = workloads.rhs(n, seed=51)
    ref = fastsum.NormalizedFastsum(v, 0.5, 32, 4, 4, kernel=kind)
    plan = Plan(gpu(v), 0.5, 32, 4, 4, -1.0, prec, kernel=kind)
    info = plan.info()
    assert info["kernel"] == KERNELS[kind]
    assert info["k0"] == pytest.approx(ref.K0, rel=1e-15)
    assert info["out_scale"] == pytest.approx(ref.out_scale, rel=1e-12)
    xt = gpu(x)
    assert_close(plan.apply_W(xt).cpu().numpy(), ref.apply_W(x), tol)
    np.testing.assert_allclose(plan.degree().cpu().numpy(), ref.degree, rtol=tol)
    assert_close(plan.apply_A(xt).cpu().numpy(), ref.apply_A(x), tol)
    assert info["device_error"] == 0


def test_block_of_right_hand_sides_equals_columns():
    v = workloads.two_arm_spiral(1200, seed=3)
    X = workloads.rhs(1200, nrhs=3, seed=4)
    plan = Plan(gpu(v), 0.5, 32, 4, 4, -1.0, "fp64")
    Y = plan.apply_Ls(gpu(X)).cpu().numpy()
    for c in range(3):
        yc = plan.apply_Ls(gpu(X[:, c])).cpu().numpy()
        np.testing.assert_allclose(Y[:, c], yc, rtol=1e-12, atol=1e-14)


def test_single_node():
    v = np.array([[0.2, -0.3, 1.0]])
    plan = Plan(gpu(v), 0.7, 16, 3, 3, -1.0, "fp64")
    y = plan.apply_W(gpu(np.array([3.0]))).cpu().numpy()
    # W = [0]; the fast sum returns its own error, K_RF(0) - K(0), times x
    ref = fastsum.NormalizedFastsum(v, 0.7, 16, 3, 3).apply_W(np.array([3.0]))
    assert abs(y[0] - ref[0]) < 1e-12
    assert abs(y[0]) < 1e-3
    assert plan.info()["degree_ok"] == int(ref[0] / 3.0 > 0)
    plan = Plan(gpu(v), 0.7, 16, 3, 3, -1.0, "fp64")
    if not plan.info()["degree_ok"]:
        with pytest.raises(NflError) as e:
            plan.apply_A(gpu(np.array([1.0])))
        assert e.value.name == "NFL_ERR_NONPOSITIVE_DEGREE"


def test_two_nodes_closed_form():
    v = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    w = math.exp(-0.25 / 0.64)
    x = np.array([2.0, -3.0])
    plan = Plan(gpu(v), 0.8, 64, 8, 4, -1.0, "fp64")
    y = plan.apply_W(gpu(x)).cpu().numpy()
    ref = fastsum.NormalizedFastsum(v, 0.8, 64, 8, 4)
    assert_close(y, ref.apply_W(x), 1e-10)
    # sigma~ = 0.7 after scaling: a wide kernel on the torus, method error ~3e-4
    np.testing.assert_allclose(y, [-3.0 * w, 2.0 * w], rtol=2e-3)
    np.testing.assert_allclose(plan.degree().cpu().numpy(), ref.degree, rtol=1e-10)


def test_coincident_nodes():
    v = np.tile([[1.0, 2.0, 3.0]], (5, 1))
    x = np.arange(1.0, 6.0)
    plan = Plan(gpu(v), 0.5, 16, 4, 4, -1.0, "fp64")
    y = plan.apply_W(gpu(x)).cpu().numpy()
    ref = fastsum.NormalizedFastsum(v, 0.5, 16, 4, 4)
    assert_close(y, ref.apply_W(x), 1e-10)
    np.testing.assert_allclose(y, x.sum() - x, rtol=1e-4)          # W = 1 1^T - I exactly


def test_invalid_arguments_raise():
    v = gpu(np.random.default_rng(0).standard_normal((10, 3)))
    for kw in [dict(N=30), dict(m=0), dict(eps_B=0.6), dict(sigma=0.0)]:
        args = dict(sigma=1.0, N=16, m=3)
        args.update(kw)
        with pytest.raises(NflError) as e:
            Plan(v, args["sigma"], args["N"], args["m"], 0, kw.get("eps_B", -1.0), "fp64")
        assert e.value.name == "NFL_ERR_INVALID_ARG"
    bad = np.random.default_rng(0).standard_normal((10, 3))
    bad[4, 1] = np.nan
    with pytest.raises(NflError):
        Plan(gpu(bad), 1.0, 16, 3)


def test_operator_symmetry_and_degree_identity():
    v = _cloud("clusters", 4000, 3, seed=21)
    for prec, tol in (("fp64", 1e-13), ("fp32c", 1e-6)):
        plan = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, prec)
        rng = np.random.default_rng(5)
        u, w = rng.standard_normal(4000), rng.standard_normal(4000)
        Wu = plan.apply_W(gpu(u)).cpu().numpy()
        Ww = plan.apply_W(gpu(w)).cpu().numpy()
        scale = np.abs(u) @ plan.apply_W(gpu(np.abs(w))).cpu().numpy()
        assert abs(u @ Ww - Wu @ w) < tol * scale
        d = plan.degree().cpu().numpy()
        Ls_sqrtd = plan.apply_Ls(gpu(np.sqrt(d))).cpu().numpy()
        assert np.abs(Ls_sqrtd).max() < 10 * tol * np.sqrt(d).max()


def test_lanczos_smallest_eigenpairs():
    """10 smallest of L_s to 1e-8 against the dense eigendecomposition (Sec. 6.1 setup)."""
    n = 2000
    v = workloads.two_arm_spiral(n, seed=2)
    lam_ref, V_ref = spectral.smallest_Ls(v, 0.5, 10)
    plan = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp64")    # kernel error ~1e-14 (high-accuracy plan)
    evals, evecs, iters, st = plan.lanczos_k_smallest(10, tol=1e-10, maxit=200, seed=1)
    assert np.abs(evals - lam_ref).max() < 1e-8
    E = evecs.cpu().numpy()
    # residual of each pair against the exact operator (eq. (max_res_norm))
    A = direct.normalized_adjacency(v, 0.5)
    res = np.linalg.norm(A @ E - E * (1.0 - evals)[None, :], axis=0)
    assert res.max() < 1e-6
    assert np.abs(E.T @ E - np.eye(10)).max() < 1e-8


def test_cg_solve_matches_dense_solve():
    n = 1500
    v = workloads.two_arm_spiral(n, seed=4)
    rng = np.random.default_rng(6)
    f = rng.standard_normal(n)
    shift = np.where(rng.uniform(size=n) < 0.1, 10.0, 0.0) + 0.5
    beta = 2.0
    u_ref = spectral.solve_shifted(v, 0.5, beta, shift, f)
    plan = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp64")
    u, iters, relres, st = plan.cg_solve(gpu(f), beta=beta, shift=gpu(shift), tol=1e-12, maxit=2000)
    assert relres <= 1e-12
    assert_close(u.cpu().numpy(), u_ref, 1e-9)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32c", 1e-6), ("fp32", 1e-6)])
def test_repeat_products_agree(prec, tol):
    """Run-to-run spread of the same product (atomic order varies, nothing else)."""
    v = _cloud("clusters", 20000, 3, seed=60)
    x = workloads.rhs(20000, seed=61)
    plan = Plan(gpu(v), 0.3, 32, 6, 6, -1.0, prec)
    xt = gpu(x)
    ys = [plan.apply_W(xt) for _ in range(3)]
    for y in ys[1:]:
        assert float(torch.linalg.norm(y - ys[0]) / torch.linalg.norm(ys[0])) < tol


@pytest.mark.parametrize("m,N,d", [(6, 32, 3), (4, 32, 3), (8, 32, 3), (4, 32, 2), (2, 16, 3)])
def test_bf16w_matches_bf16_tap_oracle(m, N, d):
    """BF16W (taps rounded to BF16) against the oracle's Alg. 2 with BF16 taps: the
    same approximation, up to FP32 arithmetic and rare rounding-boundary flips;
    the rounding itself moves the product by ~1e-3 (checked to be in effect)."""
    v = _cloud("clusters", 2500, d, seed=40 + m)
    x = np.random.default_rng(41).standard_normal(2500)
    p = Plan(gpu(v), 0.3, N, m, m, -1.0, "bf16w")
    assert p.info()["precision"] == 3
    y = p.apply_W(gpu(x)).cpu().numpy()
    ref = fastsum.NormalizedFastsum(v, 0.3, N, m, m, taps="bf16").apply_W(x)
    ref64 = fastsum.NormalizedFastsum(v, 0.3, N, m, m).apply_W(x)
    assert_close(y, ref, 2e-5)
    assert rel(y, ref64) > 1e-4
    ya = p.apply_A(gpu(x)).cpu().numpy()
    refa = fastsum.NormalizedFastsum(v, 0.3, N, m, m, taps="bf16").apply_A(x)
    assert_close(ya, refa, 2e-5)


@pytest.mark.parametrize("prec,m,tol", [("fp32c", 6, 2e-6), ("fp32", 4, 1e-5), ("fp64", 4, 1e-10)])
def test_autotune_keeps_the_products(prec, m, tol):
    """nfl_plan_autotune picks FFT CTA size, work-item size, dense-cell threshold and
    sliding-run length among its candidates; the products stay those of the oracle's
    Alg. 2."""
    v = _cloud("clusters", 6000, 3, seed=77)
    x = np.random.default_rng(78).standard_normal(6000)
    p = Plan(gpu(v), 0.3, 32, m, m, -1.0, prec)
    before = p.info()
    assert before["fft_lines_cap"] == 512 and before["slide_tiles"] == 8
    t = p.autotune()
    assert t["fft_lines_cap"] in (256, 512, 1024, 2048)
    assert t["slide_tiles"] in (1, 4, 8, 16)
    assert t["chunk"] in (2048, 4096, 8192) and t["dense_cell"] in (16, 32, 64)
    assert p.info()["work_items"] >= before["work_items"]
    assert t["best_ms"] > 0.0
    ref = fastsum.NormalizedFastsum(v, 0.3, 32, m, m).apply_W(x)
    assert_close(p.apply_W(gpu(x)).cpu().numpy(), ref, tol)


@pytest.mark.parametrize("prec,tol", [("fp32c", 2e-6), ("fp32", 1e-5)])
@pytest.mark.parametrize("m,N,n", [(7, 32, 3000), (6, 128, 20000)])
def test_column_pipeline_equals_single_columns(m, N, n, prec, tol):
    """Several columns in one call without a block path (m = 7; or N = 128, whose grids
    leave no room for blocks): the staging of each next column runs on a second stream
    into a second buffer.  Every column equals the same column in a call of its own
    (bit for bit with FP32C's fixed-point sums), and for m = 7 L_s matches the oracle."""
    # N = 128: the ball workload's shape, whose full box leaves no room for blocks
    v = _cloud("clusters", n, 3, seed=95) if m == 7 else workloads.ball_plus_clusters(n, seed=95)
    p = Plan(gpu(v), 0.3, N, m, m, -1.0, prec)
    assert p.info()["block_cols"] == 1 or m == 7
    X = np.random.default_rng(96).standard_normal((n, 5))
    for op in ("W", "Ls"):
        fn = getattr(p, "apply_" + op)
        Y = fn(gpu(X)).cpu().numpy()
        for c in range(5):
            yc = fn(gpu(X[:, c])).cpu().numpy()
            if prec == "fp32c":
                np.testing.assert_array_equal(Y[:, c], yc)
            else:
                assert rel(Y[:, c], yc) < 1e-6
    if m == 7:
        ref = fastsum.NormalizedFastsum(v, 0.3, N, m, m).apply_Ls(X[:, 3])
        assert_close(X[:, 3] - Y[:, 3], X[:, 3] - ref, tol)


@pytest.mark.parametrize("prec,m,tol", [("fp32c", 6, 1e-6), ("fp32", 4, 5e-6), ("bf16w", 3, 5e-6)])
@pytest.mark.parametrize("op", ["W", "A", "Ls"])
def test_block_products_equal_column_products(prec, m, tol, op):
    """Block products (several columns per launch, each stage) against the same
    columns one at a time and the oracle: 11 columns = a block of 8 and one of 3."""
    v = _cloud("clusters", 5000, 3, seed=90 + m)
    p = Plan(gpu(v), 0.3, 32, m, m, -1.0, prec)
    inf = p.info()
    assert inf["block_cols"] == 8
    assert p.kernels(11) == 2 * p.kernels(8)             # two blocks, one launch per stage each
    assert p.kernels(8) <= p.kernels_per_column()
    X = np.random.default_rng(91).standard_normal((5000, 11))
    Xg = gpu(X)
    fn = getattr(p, "apply_" + op)
    Y = fn(Xg).cpu().numpy()
    for c in (0, 5, 7, 8, 10):
        yc = fn(gpu(X[:, c])).cpu().numpy()
        # L_s x = x - A x: compare the A x parts
        ref = (X[:, c] - yc) if op == "Ls" else yc
        got = (X[:, c] - Y[:, c]) if op == "Ls" else Y[:, c]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    o = fastsum.NormalizedFastsum(v, 0.3, 32, m, m, taps="bf16" if prec == "bf16w" else "fp64")
    r = getattr(o, "apply_" + op)(X[:, 9])
    got = Y[:, 9]
    if op == "Ls":
        r, got = X[:, 9] - r, X[:, 9] - got
    assert np.linalg.norm(got - r) / np.linalg.norm(r) < max(tol, 2e-6)
