"""Refined CG (nfl_cg_solve_refined): FP64 residuals, FP32C correction solves.

The refinement loop's answer is the FP64 plan's solution of the system of
Sec. 6.2.2, (beta L_s + diag(s)) u = f: checked against a dense solve of the
exact matrix (oracle O5) with a high-accuracy plan, against nfl_cg_solve on
the FP64 plan, and at the full two-moons size against the FP64 CG solution.
"""
import time

import numpy as np
import pytest
import torch
from _norms import assert_close, errors

from oracle import spectral
from paper_1808_04580_gb300 import NflError, Plan, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def test_refined_cg_matches_dense_solve_and_fp64_cg():
    n = 3000
    v = workloads.two_arm_spiral(n, seed=14)
    rng = np.random.default_rng(15)
    f = rng.standard_normal(n)
    shift = np.where(rng.uniform(size=n) < 0.1, 10.0, 0.0) + 0.5
    beta = 2.0
    u_ref = spectral.solve_shifted(v, 0.5, beta, shift, f)
    p64 = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp64")      # kernel error ~1e-14
    p32 = Plan(gpu(v), 0.5, 64, 8, 8, -1.0, "fp32c")
    u, iters, outer, relres, st = p64.cg_solve_refined(p32, gpu(f), beta=beta, shift=gpu(shift), tol=1e-12,
                                                       inner_tol=1e-4, maxit=2000, max_outer=10)
    assert st == 0 and relres <= 1e-12
    assert 1 <= outer <= 6, outer
    assert_close(u.cpu().numpy(), u_ref, 1e-9)
    u64, it64, rel64, st64 = p64.cg_solve(gpu(f), beta=beta, shift=gpu(shift), tol=1e-12, maxit=2000)
    assert st64 == 0
    assert_close(u.cpu().numpy(), u64.cpu().numpy(), 1e-10)
    # the mixed form alone stops at its own accuracy
    u32, _, _, st32 = p32.cg_solve(gpu(f), beta=beta, shift=gpu(shift), tol=1e-12, maxit=2000, check=False)
    print("refined: %d outer, %d inner steps; FP64 CG %d steps; FP32C CG alone vs dense %s" % (
        outer, iters, it64, errors(u32.cpu().numpy(), u_ref)))


def test_refined_cg_rejects_plans_of_other_nodes():
    v = workloads.two_arm_spiral(500, seed=1)
    w = workloads.two_arm_spiral(500, seed=2)
    p = Plan(gpu(v), 0.5, 32, 4, 4, -1.0, "fp64")
    q = Plan(gpu(w), 0.5, 32, 4, 4, -1.0, "fp32c")
    with pytest.raises(NflError) as e:
        p.cg_solve_refined(q, gpu(np.ones(500)))
    assert e.value.name == "NFL_ERR_INVALID_ARG"
    with pytest.raises(NflError):
        p.cg_solve_refined(p, gpu(np.ones(500)))


def test_refined_cg_moons500k_matches_fp64_cg():
    """(L_s + 10 diag(mask)) u = f on the 5e5-node two-moon cloud (sigma 0.2, N 128,
    m 4): the refined solve (FP32C corrections) against FP64 CG, both to 1e-11."""
    v, lab = workloads.two_moons(500_000, seed=1)
    n = v.shape[0]
    rng = np.random.default_rng(4)
    mask = (rng.uniform(size=n) < 0.01).astype(np.float64)
    f, s = gpu(mask * lab), gpu(10.0 * mask)
    vg = gpu(v)
    p64 = Plan(vg, 0.2, 128, 4, 4, -1.0, "fp64")
    p32 = Plan(vg, 0.2, 128, 4, 4, -1.0, "fp32c")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u64, it64, rel64, st64 = p64.cg_solve(f, beta=1.0, shift=s, tol=1e-11, maxit=5000)
    t1 = time.perf_counter()
    u, iters, outer, relres, st = p64.cg_solve_refined(p32, f, beta=1.0, shift=s, tol=1e-11, inner_tol=1e-4,
                                                       maxit=5000, max_outer=12)
    t2 = time.perf_counter()
    assert st64 == 0 and st == 0
    err = errors(u.cpu().numpy(), u64.cpu().numpy())
    print("moons500k: FP64 CG %d steps %.2f s; refined %d outer + %d FP32C steps %.2f s; difference %s" % (
        it64, t1 - t0, outer, iters, t2 - t1, err))
    assert_close(u.cpu().numpy(), u64.cpu().numpy(), 1e-8)
