"""Batches with one launch per stage (nfl_batch_create / nfl_batch_run).

A batch runs the products of all its members with one staging launch, one
spread, five FFT passes and one interpolation: its results must equal each
member's own products (to the mixed form's budget: the FP32 partial sums meet
in another order), replay from a captured CUDA graph, and match the oracle's
Alg. 2 on a member.  Members that cannot share the launches are refused.
"""
import numpy as np
import pytest
import torch

from oracle import fastsum
from paper_1808_04580_gb300 import Batch, NflError, Plan, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def cols(a):
    """Column-major device block (the layout the library takes without a copy)."""
    return torch.from_numpy(np.asfortranarray(a, dtype=np.float64)).to(DEV)


def _rel_Ax(x, y, ref, op):
    if op == "Ls":   # L_s x = x - A x: compare the A x parts
        y, ref = x - y, x - ref
    return float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))


@pytest.mark.parametrize("prec,m,op,nrhs,parts", [("fp32c", 4, "Ls", 8, 1), ("fp32c", 4, "Ls", 8, 3),
                                                  ("fp32", 6, "W", 3, 2), ("fp32c", 6, "A", 1, 1),
                                                  ("bf16w", 3, "Ls", 2, 8)])
def test_batch_equals_member_products_and_replays(prec, m, op, nrhs, parts):
    sizes = [1000, 3700, 15000, 800, 42000, 2500, 9000]
    clouds = [workloads.gaussian_mixture(n, seed=90 + g) for g, n in enumerate(sizes)]
    plans = [Plan(gpu(v), 0.5, 32, m, m, -1.0, prec) for v in clouds]
    xs = [cols(workloads.rhs(n, nrhs=nrhs, seed=100 + g)) if nrhs > 1 else gpu(workloads.rhs(n, seed=100 + g))
          for g, n in enumerate(sizes)]
    b = Batch(plans, xs, op, parts=parts)
    assert b.parts == min(parts, len(plans))
    ys = [y.clone() for y in b.run()]
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        ref = getattr(p, "apply_" + op)(x)
        assert _rel_Ax(x, y, ref, op) < 1e-6
        assert p.info()["device_error"] == 0
    # captured into a CUDA graph and replayed
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        b.run()
    for o in b.outputs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for x, o, y in zip(xs, b.outputs, ys):
        assert _rel_Ax(x, o, y, op) < 1e-6
    # a member against the oracle's Alg. 2
    o = fastsum.NormalizedFastsum(clouds[1], 0.5, 32, m, m, taps="bf16" if prec == "bf16w" else "fp64")
    x1 = (xs[1][:, 0] if nrhs > 1 else xs[1]).cpu().numpy()
    r = getattr(o, "apply_" + op)(x1)
    got = (ys[1][:, 0] if nrhs > 1 else ys[1]).cpu().numpy()
    if op == "Ls":
        r, got = x1 - r, x1 - got
    assert np.linalg.norm(got - r) / np.linalg.norm(r) < (2e-5 if prec == "bf16w" else 2e-6)
    b.close()


def test_batch_refuses_members_that_cannot_share_launches():
    v1, v2 = workloads.gaussian_mixture(2000, seed=1), workloads.gaussian_mixture(3000, seed=2)
    x1, x2 = gpu(workloads.rhs(2000, seed=3)), gpu(workloads.rhs(3000, seed=4))
    cases = [
        (Plan(gpu(v1), 0.5, 32, 4, 4, -1.0, "fp32c"), Plan(gpu(v2), 0.5, 32, 6, 6, -1.0, "fp32c")),   # m
        (Plan(gpu(v1), 0.5, 32, 4, 4, -1.0, "fp32c"), Plan(gpu(v2), 0.5, 64, 4, 4, -1.0, "fp32c")),   # N
        (Plan(gpu(v1), 0.5, 32, 4, 4, -1.0, "fp32c"), Plan(gpu(v2), 0.5, 32, 4, 4, -1.0, "fp32")),    # precision
        (Plan(gpu(v1), 0.5, 32, 4, 4, -1.0, "fp64"), Plan(gpu(v2), 0.5, 32, 4, 4, -1.0, "fp64")),     # FP64
    ]
    for p1, p2 in cases:
        with pytest.raises(NflError) as e:
            Batch([p1, p2], [x1, x2], "Ls")
        assert e.value.name == "NFL_ERR_INVALID_ARG"
    p = Plan(gpu(v1), 0.5, 32, 4, 4, -1.0, "fp32c")
    with pytest.raises(NflError):
        Batch([p, p], [x1, x1], "W")                       # the same plan twice


def test_batch_256_uneven_graphs_against_member_products():
    """The 256-graph workload (n log-uniform in [1e3, 2e5], 8 columns, FP32C, sigma 0.5,
    N 64, m 4) through one batch: every member's columns against its own products."""
    clouds = workloads.many_graphs(256, seed=0)
    sizes = [c.shape[0] for c in clouds]
    plans = [Plan(gpu(v), 0.5, 64, 4, 4, -1.0, "fp32c") for v in clouds]
    xs = [cols(workloads.rhs(n, nrhs=8, seed=g + 7)) for g, n in enumerate(sizes)]
    b = Batch(plans, xs, "Ls", parts=4)
    ys = b.run()
    torch.cuda.synchronize()
    worst = 0.0
    for g in range(0, 256, 5):
        ref = plans[g].apply_Ls(xs[g])
        worst = max(worst, _rel_Ax(xs[g], ys[g], ref, "Ls"))
    print("graphs256 batch vs member products, worst A x difference: %.2e" % worst)
    assert worst < 1e-6
