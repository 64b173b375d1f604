"""Many independent graphs of uneven size in one call, and in one CUDA graph.

nfl_apply_batched issues every plan's products on one stream without host
synchronization; captured into a CUDA graph, the whole batch replays as a
single launch.  Batched, per-plan and replayed FP32C results agree to the
FP32C budget (the order in which FP32 partial sums meet in shared memory is
not fixed); one graph is also checked against the oracle's Alg. 2.
"""
import numpy as np
import pytest
import torch

from oracle import fastsum
from paper_1808_04580_gb300 import Plan, apply_batched, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def test_batched_equals_per_plan_and_graph_replay():
    sizes = [1000, 3700, 15000, 800, 42000, 2500]
    clouds = [workloads.gaussian_mixture(n, seed=20 + g) for g, n in enumerate(sizes)]
    plans = [Plan(gpu(v), 0.5, 32, 4, 4, -1.0, "fp32c") for v in clouds]
    xs = [gpu(workloads.rhs(n, nrhs=8, seed=40 + g)) for g, n in enumerate(sizes)]
    ys = apply_batched(plans, xs, "Ls")
    torch.cuda.synchronize()
    def close(a, b):
        # L_s x = x - A x: compare the A x parts, which x would otherwise hide
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) < 1e-6

    for plan, x, y in zip(plans, xs, ys):
        ref = plan.apply_Ls(x)
        assert close(x - y, x - ref)
        assert plan.info()["device_error"] == 0

    outs = [torch.empty((8, n), dtype=torch.float64, device=DEV) for n in sizes]
    apply_batched(plans, xs, "Ls", outs=outs)          # warm-up before capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        apply_batched(plans, xs, "Ls", outs=outs)
    for o in outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for o, x, y in zip(outs, xs, ys):
        assert close(x - o.t(), x - y)

    # one member against the oracle's Alg. 2 (FP32C tolerance)
    v, x = clouds[0], xs[0][:, 3].cpu().numpy()
    ref = fastsum.NormalizedFastsum(v, 0.5, 32, 4, 4).apply_Ls(x)
    got = ys[0][:, 3].cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(x - ref) < 2e-6
