"""Failure detection without a GPU fault: a bounded wait that runs out.

The tensor-core interpolation waits on an mbarrier for its MMAs with a limit
of polls and device time.  The plan's fault hook makes the issuing thread skip
the MMAs, so every wait runs out (after 10 ms in this mode): the kernel must
set the plan's device_error, skip its remaining work, free its tensor memory
and return; the context must stay usable for new plans.
"""
import time

import numpy as np
import pytest
import torch

from oracle import fastsum
from paper_1808_04580_gb300 import NflError, Plan, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def test_interpolation_wait_runs_out_and_is_reported():
    n = 20000
    v = workloads.gaussian_mixture(n, seed=3)
    x = workloads.rhs(n, seed=4)
    plan = Plan(gpu(v), 0.4, 32, 6, 6, -1.0, "fp32c")        # m = 6: tensor-core interpolation
    assert plan.info()["device_error"] == 0
    plan.inject_fault(1)
    t0 = time.time()
    plan.apply_W(gpu(x))
    torch.cuda.synchronize()
    assert time.time() - t0 < 20.0                            # bounded: no hang
    assert plan.info()["device_error"] == 1
    plan.inject_fault(0)
    with pytest.raises(NflError):
        plan.inject_fault(7)
    # the context is intact: a fresh plan is exact again
    fresh = Plan(gpu(v[:3000]), 0.4, 32, 6, 6, -1.0, "fp32c")
    y = fresh.apply_W(gpu(x[:3000])).cpu().numpy()
    ref = fastsum.NormalizedFastsum(v[:3000], 0.4, 32, 6, 6).apply_W(x[:3000])
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 2e-6
    assert fresh.info()["device_error"] == 0
