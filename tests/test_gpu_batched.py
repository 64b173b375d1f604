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


def test_batched_256_uneven_graphs_full_size():
    """256 Gaussian-mixture graphs, n log-uniform in [1e3, 2e5] (sum ~1.2e7), 8 columns
    each, FP32C, sigma 0.5, N 64, m 4, one captured CUDA graph: every degree positive,
    the replay equal to the eager batch, small members against the oracle's Alg. 2 on
    all rows, large members against the direct sum on sampled rows."""
    from oracle import direct
    clouds = workloads.many_graphs(256, seed=0)
    sizes = [c.shape[0] for c in clouds]
    plans = [Plan(gpu(v), 0.5, 64, 4, 4, -1.0, "fp32c") for v in clouds]
    assert all(p.info()["degree_ok"] for p in plans)
    for p in plans:                                       # launch parameters per graph
        p.autotune()
    xs = [gpu(workloads.rhs(n, nrhs=8, seed=g + 7)) for g, n in enumerate(sizes)]
    eager = [y.clone() for y in apply_batched(plans, xs, "Ls")]
    outs = [torch.empty((8, n), dtype=torch.float64, device=DEV) for n in sizes]
    apply_batched(plans, xs, "Ls", outs=outs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        apply_batched(plans, xs, "Ls", outs=outs)
    for o in outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for o, x, e in zip(outs, xs, eager):
        a, b = x - o.t(), x - e
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) < 1e-6
    order = np.argsort(sizes)
    for g in order[:3]:                                   # smallest: oracle Alg. 2, all rows
        ref = fastsum.NormalizedFastsum(clouds[g], 0.5, 64, 4, 4)
        for c in (0, 5):
            x = xs[g][:, c].cpu().numpy()
            r = ref.apply_Ls(x)
            got = outs[g][c].cpu().numpy()
            assert np.linalg.norm(got - r) / np.linalg.norm(x - r) < 2e-6
    rows = np.random.default_rng(3).choice(int(sizes[order[-1]]), 128, replace=False)
    for g in order[-2:]:                                  # largest: direct sum on sampled rows
        rows_g = rows[rows < sizes[g]]
        x = xs[g][:, 2].contiguous()
        w = plans[g].apply_W(x).cpu().numpy()
        ref = direct.rows_W(clouds[g], 0.5, x.cpu().numpy(), rows_g)
        assert np.linalg.norm(w[rows_g] - ref) / np.linalg.norm(ref) < 1e-5


def test_captured_graph_survives_block_products():
    """A one-column product captured into a CUDA graph still replays correctly after
    block products on the same plan (the plan never reallocates its buffers)."""
    v = workloads.gaussian_mixture(20000, seed=61)
    p = Plan(gpu(v), 0.5, 32, 4, 4, -1.0, "fp32c")
    assert p.info()["block_cols"] > 1
    x = gpu(workloads.rhs(20000, seed=62))
    y = torch.empty_like(x)
    p.apply_Ls(x, out=y)                                  # warm-up before capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        p.apply_Ls(x, out=y)
    ref = p.apply_Ls(x).clone()
    X8 = gpu(workloads.rhs(20000, nrhs=8, seed=63))
    Y8 = p.apply_Ls(X8)                                   # block product
    y.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert float(torch.linalg.norm((x - y) - (x - ref)) / torch.linalg.norm(x - ref)) < 1e-6
    assert float(torch.linalg.norm((X8[:, 3] - Y8[:, 3]) - (X8[:, 3] - p.apply_Ls(X8[:, 3].contiguous())))) \
        < 1e-6 * float(torch.linalg.norm(X8[:, 3] - Y8[:, 3]))


def test_first_block_product_under_capture_is_refused():
    """The first block product allocates the plan's block buffers; under stream capture
    it returns NFL_ERR_INVALID_ARG instead (cudaMalloc would invalidate the capture),
    and after one uncaptured block product the same call captures and replays."""
    from paper_1808_04580_gb300 import NflError
    n = 3000
    plan = Plan(gpu(workloads.gaussian_mixture(n, seed=5)), 0.5, 32, 4, 4, -1.0, "fp32c")
    assert plan.info()["block_cols"] == 8
    x = gpu(workloads.rhs(n, nrhs=8, seed=6))
    out = torch.empty((8, n), dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(NflError) as e:
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            plan.apply_Ls(x, out=out)
    assert e.value.name == "NFL_ERR_INVALID_ARG"
    ref = plan.apply_Ls(x).clone()                 # uncaptured: allocates the block buffers
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        plan.apply_Ls(x, out=out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert float(torch.linalg.norm((x - out.t()) - (x - ref)) / torch.linalg.norm(x - ref)) < 1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 1e-6)])
def test_create_batched_equals_single_plans(prec, tol):
    """nfl_plan_create_batched builds the same plans as one nfl_plan_create per node
    set (same scaling, box, work items and degrees), and the products agree."""
    from paper_1808_04580_gb300 import NflError, create_batched
    sizes = [1000, 3700, 15000, 800, 42000, 2500, 1, 2]
    sig = [0.5, 0.4, 0.5, 0.6, 0.5, 0.45, 0.5, 0.5]
    clouds = [workloads.gaussian_mixture(n, seed=60 + g) for g, n in enumerate(sizes)]
    plans = create_batched([gpu(v) for v in clouds], sig, 32, 4, 4, -1.0, prec)
    for g, (v, s, p) in enumerate(zip(clouds, sig, plans)):
        q = Plan(gpu(v), s, 32, 4, 4, -1.0, prec)
        ip, iq = p.info(), q.info()
        for key in ("n", "rho", "sigma_tilde", "center", "box", "tiles", "work_items", "block_cols", "degree_ok"):
            assert ip[key] == iq[key], (g, key)
        np.testing.assert_allclose(p.degree().cpu().numpy(), q.degree().cpu().numpy(), rtol=tol, atol=0)
        if ip["degree_ok"]:
            x = gpu(workloads.rhs(sizes[g], seed=80 + g))
            a, b = p.apply_Ls(x), q.apply_Ls(x)
            assert float(torch.linalg.norm((x - a) - (x - b)) / torch.linalg.norm(x - b)) < tol, g
    # one member against the oracle's Alg. 2
    x = workloads.rhs(sizes[1], seed=81)
    ref = fastsum.NormalizedFastsum(clouds[1], sig[1], 32, 4, 4).apply_W(x)
    y = plans[1].apply_W(gpu(x)).cpu().numpy()
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < (1e-10 if prec == "fp64" else 1e-6)
    # an invalid member: no plan is returned
    with pytest.raises(NflError) as e:
        create_batched([gpu(v) for v in clouds[:3]], [0.5, -1.0, 0.5], 32, 4, 4, -1.0, prec)
    assert e.value.name == "NFL_ERR_INVALID_ARG"
