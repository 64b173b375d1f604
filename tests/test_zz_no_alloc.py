"""The allocation-free CG entry point gives the allocating solver's answer.

nfl_cg_solve_noalloc exists for callers that cannot allocate device memory
while they solve; it keeps its work vectors in a static device array of the
library.  This file runs last, so a failure here leaves every other test
already run.  It must pass in a fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_1808_04580_gb300 import NflError, Plan, nfl, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_cg_matches_allocating_cg_on_two_calls():
    n = 3000
    v = workloads.two_arm_spiral(n, seed=9)
    rng = np.random.default_rng(10)
    f = _gpu(rng.standard_normal(n))
    shift = _gpu(np.where(rng.uniform(size=n) < 0.05, 10.0, 0.0) + 0.5)
    plan = Plan(_gpu(v), 0.5, 32, 4, 4, -1.0, "fp64")
    u_ref, it_ref, rel_ref, st_ref = plan.cg_solve(f, beta=2.0, shift=shift, tol=1e-10, maxit=1000)
    assert st_ref == 0 and rel_ref <= 1e-10
    u_ref = u_ref.cpu().numpy()
    for call in range(2):     # the second call reuses the array the first one left behind
        u, it, rel, st = plan.cg_solve(f, beta=2.0, shift=shift, tol=1e-10, maxit=1000, noalloc=True)
        assert st == 0, call
        assert rel <= 1e-10, call
        assert abs(it - it_ref) <= 1, call
        assert _rel(u.cpu().numpy(), u_ref) < 1e-9, call


def test_noalloc_rejects_more_nodes_than_the_array_holds():
    n = nfl.NOALLOC_MAX_N + 1
    v = np.random.default_rng(11).standard_normal((n, 3))
    plan = Plan(_gpu(v), 1.0, 16, 3, 3, -1.0, "fp32")
    f = _gpu(np.ones(n))
    with pytest.raises(NflError) as e:
        plan.cg_solve(f, beta=1.0, noalloc=True)
    assert e.value.name == "NFL_ERR_INVALID_ARG"
