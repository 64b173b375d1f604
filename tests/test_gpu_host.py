"""Products with host-resident blocks (nfl_apply_host): the copy/compute
pipeline must give the device products of the same plan, for every op, more
columns than staging slots, page-locked and pageable memory, leading
dimensions above n, and the oracle's Alg. 2 on an FP64 plan.
"""
import ctypes

import numpy as np
import pytest
import torch
from _norms import assert_close

from oracle import fastsum
from paper_1808_04580_gb300 import NflError, Plan, workloads
from paper_1808_04580_gb300.nfl import library

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.fixture(scope="module")
def cloud():
    v = workloads.ball_plus_clusters(6000, seed=11)
    x = np.random.default_rng(12).standard_normal((6000, 7))
    return v, x


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32c", 2e-6), ("fp32", 2e-6)])
@pytest.mark.parametrize("op", ["W", "A", "Ls"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_block_equals_device_product(cloud, precision, tol, op, pinned):
    v, x = cloud
    p = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, precision)
    xh = torch.from_numpy(np.ascontiguousarray(x.T)).t()      # (n, 7), column-major storage
    if pinned:
        xh = xh.t().contiguous().pin_memory().t()
    yh = p.apply_host(xh, op)
    assert not yh.is_cuda and yh.shape == (6000, 7)
    ref = getattr(p, "apply_" + op)(gpu(x))
    assert_close(yh.to(DEV), ref, tol)
    y1 = p.apply_host(xh[:, 2].contiguous(), op)              # one column
    assert_close(y1.to(DEV), ref[:, 2], tol)


def test_host_fp64_matches_oracle(cloud):
    v, x = cloud
    p = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, "fp64")
    ref = fastsum.NormalizedFastsum(v, 0.3, 32, 4, 4)
    y = p.apply_host(torch.from_numpy(x[:, :4].copy()), "A").numpy()
    for c in range(4):
        r = ref.apply_A(x[:, c])
        assert np.linalg.norm(y[:, c] - r) / np.linalg.norm(r) < 1e-10


def test_host_leading_dimensions_above_n(cloud):
    v, x = cloud
    n, r, ldx, ldy = 6000, 5, 6013, 6100
    p = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, "fp64")
    xb = torch.full((r, ldx), float("nan"), dtype=torch.float64).pin_memory()
    xb[:, :n] = torch.from_numpy(np.ascontiguousarray(x[:, :r].T))
    yb = torch.full((r, ldy), -7.0, dtype=torch.float64).pin_memory()
    st = library().nfl_apply_host(p._h, 2, xb.data_ptr(), ldx, yb.data_ptr(), ldy, r)
    assert st == 0
    ref = p.apply_Ls(gpu(x[:, :r])).cpu().numpy().T
    assert np.abs(yb[:, :n].numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    assert torch.all(yb[:, n:] == -7.0)                       # padding untouched


def test_host_repeated_calls_reuse_the_staging(cloud):
    v, x = cloud
    p = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, "fp32c")
    xh = torch.from_numpy(np.ascontiguousarray(x.T)).pin_memory()
    out = torch.empty_like(xh).pin_memory()
    ref = p.apply_Ls(gpu(x))
    for _ in range(3):
        y = p.apply_host(xh.t(), "Ls", out=out)
        assert y.data_ptr() == out.data_ptr()
        assert_close(y.to(DEV), ref, 2e-6)


def test_host_rejects_bad_arguments(cloud):
    v, x = cloud
    p = Plan(gpu(v), 0.3, 32, 4, 4, -1.0, "fp64")
    xb = torch.zeros(6000, dtype=torch.float64)
    with pytest.raises(TypeError):
        p.apply_host(xb.to(DEV))
    with pytest.raises(ValueError):
        p.apply_host(torch.zeros(5999, dtype=torch.float64))
    assert library().nfl_apply_host(p._h, 2, xb.data_ptr(), 5999, xb.data_ptr(), 6000, 1) == 1


def test_host_nonpositive_degree_reported(cloud):
    """sigma = 0.1 with N = 32 gives negative degree estimates on this cloud
    (the oracle's Alg. 2 does too): A and L_s refuse, W still works."""
    v, x = cloud
    p = Plan(gpu(v), 0.1, 32, 4, 4, -1.0, "fp64")
    xh = torch.from_numpy(x[:, 0].copy())
    for op in ("A", "Ls"):
        with pytest.raises(NflError):
            p.apply_host(xh, op)
    y = p.apply_host(xh, "W")
    assert_close(y.to(DEV), p.apply_W(gpu(x[:, 0])), 1e-13)
