#!/usr/bin/env python
"""Throughput of the normalized-Laplacian product L_s x on one GB300.

Workload (one "step" = one pass of the whole hot path over one batch):
  n = 10,000,000 nodes in d = 3: half uniform in the unit ball, half in five
  Gaussian clusters (centres at radius 0.6, std 0.04); Gaussian kernel
  sigma = 0.08; fast summation N = 128, m = 6, p = 6, eps_B = 6/128.
  A step applies L_s to a block of ``--nrhs`` right-hand sides x ~ N(0, 1)
  (spread, FFT with the fused multiplier, gather with the fused D^{-1/2}
  epilogue, per column), in the FP32C form (FP32 window arithmetic, spreading
  sums carried into 64-bit fixed point).

Reported: L_s matvecs/s (columns per second, all ranks), the same through
host buffers (e2e), the plain FP64 single-vector form on the same data, the
error of the product against the FP64 direct sum on sampled rows, a
precision sweep (W x in FP64, FP32, FP32C and BF16W, each against the direct
sum on the sampled rows and the GPU FP64 form on all rows), the
roofline of the dominant kernel from CUDA events recorded around each stage
inside the timed region, and the direct-sum oracle timed on the host cores.

``--impl reference`` times the CPU oracle (direct FP64 sums, plain C with
OpenMP) on a bounded sample of the same workload instead.
Multi-GPU (torchrun): every rank runs an independent replica on its own GPU
(weak scaling); the only collectives are the timing barrier and max.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_NODES = 10_000_000
CFG = dict(sigma=0.08, N=128, m=6, p=6)
WORKLOAD = ("ball10M: n=10,000,000 d=3, 50% uniform in the unit ball + 50% in 5 Gaussian clusters "
            "(centres at radius 0.6, std 0.04); Gaussian sigma=0.08; N=128, m=6, p=6, eps_B=6/128")
METRIC = "L_s matvecs/s (n=10M, d=3) mixed+batched vs FP64 plain, rel err <=1e-6"
FP32_LANES_PER_SM = 128
SMS = 152
SM_MAX_MHZ = 2070.0


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


PEAKS = _peaks()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=4)
    ap.add_argument("--points", type=int, default=N_NODES)
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp32", "fp64"])
    ap.add_argument("--baseline-rows", type=int, default=1024)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-sweep", action="store_true", help="skip the W x precision sweep (FP32, FP32C, BF16W)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch parameters")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip the spiral5k, image1M and graphs256 fields")
    return ap.parse_args()


def dist_setup():
    """Process group from the torchrun environment: NCCL with one GPU per rank, or gloo on a host without GPUs."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def max_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=timestamp," + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 - 0.25 <= t <= t1 + 0.25] or [l for (_, l) in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_sha(path):
    return hashlib.sha1(open(path, "rb").read()).hexdigest()[:12]


def profiled_traffic(summary, kernel_file):
    """dram bytes per launch from the committed ncu summary, if it matches the current source."""
    summ = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(summ):
        return None
    vals = {}
    for line in open(summ):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != source_sha(kernel_file):
        return None
    try:
        return float(vals["traffic_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def oracle_rows(v, x, rows):
    from oracle import direct
    t = time.perf_counter()
    out = direct.rows_W(v, CFG["sigma"], x, rows)
    return out, time.perf_counter() - t, direct.max_threads()


def run_reference(args, world, rank):
    """The oracle (direct FP64 sums on the host cores) as the reference arm."""
    if rank != 0:
        return
    import numpy as np
    from paper_1808_04580_gb300 import workloads
    v = workloads.ball_plus_clusters(args.points, seed=0)
    x = workloads.rhs(args.points, seed=1)
    rng = np.random.default_rng(2)
    rows_per_step = 64
    for _ in range(args.warmup):
        oracle_rows(v, x, rng.choice(args.points, 8, replace=False))
    total = 0.0
    cores = 1
    for _ in range(args.steps):
        _, dt, cores = oracle_rows(v, x, rng.choice(args.points, rows_per_step, replace=False))
        total += dt
    value = rows_per_step * args.steps / total / args.points
    sample = "%d steps x %d of %d target rows, each summed over all %d sources; matvecs/s extrapolated as rows/s / n" % (
        args.steps, rows_per_step, args.points, args.points)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "rows_per_step": rows_per_step},
        "cpu_baseline": {"value": value, "unit": "matvecs/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _events_ms(fn, reps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def other_workloads(dev):
    """The paper-shaped workloads beside the headline one (not part of the timed step):
    spiral5k (FP64 W x and the 10 smallest eigenpairs), image1M (L_s in FP32C and FP64),
    graphs256 (batched plan creation and one captured CUDA graph of 8 columns per graph)."""
    import numpy as np
    import torch
    from paper_1808_04580_gb300 import Batch, Plan, apply_batched, create_batched, workloads
    stream = torch.cuda.current_stream()
    gpu = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)   # noqa: E731
    # column blocks in column-major storage (the layout the library takes without a copy)
    cols = lambda a: torch.from_numpy(np.asfortranarray(a, dtype=np.float64)).to(dev)   # noqa: E731
    out = {}

    # spiral5k: n = 5000 two-arm spiral, sigma 0.5, N 32, m 4, p 4, FP64
    v = workloads.two_arm_spiral(5000, seed=0)
    x = gpu(workloads.rhs(5000, seed=1))
    p = Plan(gpu(v), 0.5, 32, 4, 4, -1.0, "fp64")
    ms = _events_ms(lambda: p.apply_W(x), 20, stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ev, V, iters, st = p.lanczos_k_smallest(10, tol=1e-10, maxit=300, seed=1)
    lz = time.perf_counter() - t
    R = p.apply_A(V) - V * torch.from_numpy(1.0 - ev).to(dev)[None, :]
    out["spiral5k"] = {"workload": "n=5000 two-arm spiral d=3, sigma=0.5, N=32, m=4, p=4, FP64",
                       "W_matvecs_per_s": 1000.0 / ms, "ms_per_W_matvec": ms,
                       "lanczos_10_smallest_s": lz, "lanczos_steps": iters, "status": st,
                       "max_residual": float(torch.linalg.norm(R, dim=0).max())}
    p.close()

    # image1M: 1000 x 1000 Voronoi image (12 regions), sigma 0.1, N 64, m 4
    v, _ = workloads.voronoi_image(seed=0)
    n = v.shape[0]
    X = cols(workloads.rhs(n, nrhs=4, seed=2))
    vg = gpu(v)
    res = {"workload": "n=1,000,000 pixels of a 1000x1000 image, 12 Voronoi regions, RGB features d=3, "
                       "sigma=0.1, N=64, m=4"}
    ys = {}
    for prec in ("fp32c", "fp64"):
        pp = Plan(vg, 0.1, 64, 4, 4, -1.0, prec)
        if prec == "fp32c":
            pp.autotune()
        Y = torch.empty((4, n), dtype=torch.float64, device=dev)
        ms = _events_ms(lambda: pp.apply_Ls(X, out=Y), 5 if prec == "fp32c" else 2, stream)
        res[prec] = {"Ls_matvecs_per_s": 4 * 1000.0 / ms, "ms_per_step_of_4": ms}
        ys[prec] = Y.clone()
        pp.close()
    a, b = X.t() - ys["fp32c"], X.t() - ys["fp64"]
    res["fp32c_rel_err_vs_fp64_Ax"] = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    res["speedup_fp32c_vs_fp64"] = res["fp32c"]["Ls_matvecs_per_s"] / res["fp64"]["Ls_matvecs_per_s"]
    out["image1M"] = res
    del X, vg, ys

    # graphs256: 256 Gaussian-mixture graphs, n log-uniform in [1e3, 2e5], 8 columns each, FP32C
    clouds = workloads.many_graphs(256, seed=0)
    sizes = [c.shape[0] for c in clouds]
    vgs = [gpu(c) for c in clouds]
    torch.cuda.synchronize()
    t = time.perf_counter()
    plans = create_batched(vgs, 0.5, 64, 4, 4, -1.0, "fp32c")
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t
    t = time.perf_counter()
    single = [Plan(vv, 0.5, 64, 4, 4, -1.0, "fp32c") for vv in vgs]
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t
    for q in single:
        q.close()
    for q in plans:
        q.autotune()
    xs = [cols(workloads.rhs(nn, nrhs=8, seed=g + 7)) for g, nn in enumerate(sizes)]
    outs = [torch.empty((8, nn), dtype=torch.float64, device=dev) for nn in sizes]
    apply_batched(plans, xs, "Ls", outs=outs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        apply_batched(plans, xs, "Ls", outs=outs)
    ms = _events_ms(graph.replay, 5, stream)
    # the same products with one launch per stage and part (nfl_batch_run), the members
    # split into parts that run on parallel library streams
    ncols = 8 * len(plans)
    sweep = {}
    for parts in (1, 2, 4, 8):
        b = Batch(plans, xs, "Ls", parts=parts)
        b.run()
        torch.cuda.synchronize()
        graph_b = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_b, capture_error_mode="thread_local"):
            b.run()
        ms_b = _events_ms(graph_b.replay, 5, stream)
        b.set_profiling(True)
        b.run()
        st = b.stage_times()
        worst = 0.0
        for o, x, y in zip(b.outputs, xs, outs):
            a1, a2 = x - o, x - y.t()
            worst = max(worst, float(torch.linalg.norm(a1 - a2) / torch.linalg.norm(a2)))
        b.close()
        del graph_b
        sweep[parts] = {"ms_per_replay": ms_b, "Ls_matvecs_per_s": ncols * 1000.0 / ms_b,
                        "kernel_launches_per_replay": 8 * parts,
                        "stage_ms_summed_over_parts": {k: st[k] for k in ("prep", "spread", "fft", "gather")},
                        "rel_diff_vs_per_plan_products": worst}
    best = min(sweep, key=lambda k: sweep[k]["ms_per_replay"])
    out["graphs256_one_launch_per_stage"] = dict(sweep[best], parts=best,
                                                 point_rhs_per_s=8 * sum(sizes) * 1000.0 / sweep[best]["ms_per_replay"],
                                                 parts_sweep={k: v["ms_per_replay"] for k, v in sweep.items()},
                                                 stage_ms_one_part=sweep[1]["stage_ms_summed_over_parts"])
    out["graphs256"] = {"workload": "256 Gaussian-mixture graphs d=3, n log-uniform in [1e3, 2e5] (sum %d), "
                                    "8 right-hand sides each, FP32C, sigma=0.5, N=64, m=4" % sum(sizes),
                        "ms_per_replay": ms, "Ls_matvecs_per_s": ncols * 1000.0 / ms,
                        "point_rhs_per_s": 8 * sum(sizes) * 1000.0 / ms,
                        "launches_per_replay": int(sum(q.kernels(8) for q in plans)),
                        "api": "nfl_apply_batched: per-plan block products over 16 library streams",
                        "plan_create_batched_s": t_batched, "plan_create_one_by_one_s": t_single}
    for q in plans:
        q.close()
    return out


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch
    from paper_1808_04580_gb300 import Plan, fma_rate, workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n, nrhs = args.points, args.nrhs
    v = workloads.ball_plus_clusters(n, seed=rank)
    X = workloads.rhs(n, nrhs=nrhs, seed=rank + 1)
    X = X.reshape(n, nrhs)
    vg = torch.from_numpy(v).to(dev)
    xg = torch.from_numpy(np.asfortranarray(X)).to(dev)
    # measured multiply-add rates of this GPU (the ALU roofline's denominator)
    rates = {}
    for kind in ("fp32", "fp32x2", "fp64"):
        try:
            rates[kind] = fma_rate(kind)[0]
        except Exception:  # a refused measurement leaves the derived peak
            rates[kind] = None
    plan = Plan(vg, CFG["sigma"], CFG["N"], CFG["m"], CFG["p"], -1.0, args.precision)
    tuned = plan.autotune() if not args.no_autotune else None   # launch parameters, outside the timed region
    info = plan.info()
    ycols = torch.empty((nrhs, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.apply_Ls(xg, out=ycols)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    plan.set_profiling(True)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall1 = time.time()
    sampler.stop()
    stages = plan.stage_times()
    plan.set_profiling(False)
    ms_local = e0.elapsed_time(e1)
    ms = max_over_ranks(ms_local, world)
    columns = nrhs * args.steps
    value = world * columns / (ms / 1000.0)
    clocks = sampler.summary(t_wall0, t_wall1)

    # dominant kernel and its roofline (ALU: one multiply-add per window tap)
    taps = (2 * CFG["m"]) ** 3
    box_elems = int(np.prod(info["box"]))
    spread_ms = stages["spread"] / max(1, stages["columns"])
    gather_ms = stages["gather"] / max(1, stages["columns"])
    fft_ms = stages["fft"] / max(1, stages["columns"])
    dom = "spread" if spread_ms >= gather_ms else "gather"
    # columns one spread / gather launch takes (blocks of up to 8 on the tensor-core path)
    cpl = min(nrhs, info["block_cols"]) if plan.kernels(nrhs) < nrhs * plan.kernels_per_column() else 1
    dom_ms = max(spread_ms, gather_ms) * cpl
    flops = 2.0 * taps * n * cpl
    achieved = flops / (dom_ms / 1000.0) / 1e12
    # the measured FP32 multiply-add rate (the faster of scalar and packed fma), else the
    # unit-count figure 152 SMs x 128 lanes x 2 flop x 2070 MHz
    if rates.get("fp32") or rates.get("fp32x2"):
        peak = max(rates.get("fp32") or 0.0, rates.get("fp32x2") or 0.0) / 1e12
        peak_note = ("measured: nfl_fma_rate, max of fma.rn.f32 (%.1f TFLOP/s) and fma.rn.f32x2 (%.1f TFLOP/s) "
                     "register-resident chains on all SMs, CUDA events" % ((rates.get("fp32") or 0.0) / 1e12,
                                                                       (rates.get("fp32x2") or 0.0) / 1e12))
    else:
        peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        peak_note = "derived: 152 SMs x 128 lanes x 2 flop x 2070 MHz (no measured FP32 rate)"
    # each stage is two kernels (sparse tiles: warp-slice spread / tensor-core interpolation;
    # dense tiles: slab Chebyshev moments)
    parts = ([("spread3_warp.cu", "spread3_warp_ball10M.md"), ("spread3_moments.cu", "spread3_moments_ball10M.md")]
             if dom == "spread" else
             [("gather_tc.cu", "gather3_tc_ball10M.md"), ("gather3_moments.cu", "gather3_moments_ball10M.md")])
    kname = "spread3_warp + spread3_moments" if dom == "spread" else "gather3_tc + gather3_moments"
    traffic = 0.0 if n == 10_000_000 else None
    for src, summary in parts:
        t = profiled_traffic(summary, os.path.join(ROOT, "paper_1808_04580_gb300", "csrc", src)) if traffic is not None else None
        traffic = None if t is None else traffic + t
    if traffic is not None:
        traffic *= cpl                # the profile is of a one-column launch
    # algorithmic HBM bytes per column: the spread reads the 16-byte node record and the
    # FP32 x~ and adds into the 8-byte fixed-point grid of the active box; the gather reads
    # the record, perm, the staged z, D^{-1/2} and the FP32 interpolation grid, writes y
    spread_bytes = n * (16 + 4) + box_elems * 8
    gather_bytes = n * (16 + 4 + 8 + 8 + 8) + box_elems * 4
    dom_bytes = (spread_bytes if dom == "spread" else gather_bytes) * cpl
    hbm_peak = float(PEAKS.get("hbm_gbs") or 6768.0)
    peak_units = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_from_unit_counts": peak_units,
                "traffic": traffic, "kernel": kname,
                "flops_per_launch": flops, "ms_per_launch": dom_ms, "columns_per_launch": cpl,
                "algorithmic_bytes_per_launch": dom_bytes,
                "hbm_achieved_gbs": dom_bytes / (dom_ms / 1000.0) / 1e9,
                "peak_note": peak_note}
    # spread + gather together against both ceilings: the HBM fraction of their algorithmic
    # bytes is far below 50 % because the taps, not the bytes, bound them
    sg_ms = spread_ms + gather_ms
    spread_gather = {"ms_per_column": sg_ms, "algorithmic_bytes_per_column": spread_bytes + gather_bytes,
                     "hbm_gbs": (spread_bytes + gather_bytes) / (sg_ms / 1000.0) / 1e9,
                     "hbm_frac": (spread_bytes + gather_bytes) / (sg_ms / 1000.0) / 1e9 / hbm_peak,
                     "hbm_peak_gbs": hbm_peak,
                     "alu_tflops": 2 * 2.0 * taps * n / (sg_ms / 1000.0) / 1e12,
                     "alu_frac": 2 * 2.0 * taps * n / (sg_ms / 1000.0) / 1e12 / peak,
                     "hbm_target_0.5_met": bool((spread_bytes + gather_bytes) / (sg_ms / 1000.0) / 1e9 / hbm_peak >= 0.5),
                     "note": "arithmetic-bound: the taps need %.2f ms per column at the FP32 peak, the bytes %.3f ms "
                             "at the HBM peak" % (2 * 2.0 * taps * n / (peak * 1e12) * 1e3,
                                                  (spread_bytes + gather_bytes) / (hbm_peak * 1e9) * 1e3)}

    # end to end through the C ABI with page-locked host buffers (nfl_apply_host:
    # each step's columns go to the device and back inside the timed region)
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    Yh = torch.empty((nrhs, n), dtype=torch.float64).pin_memory()
    plan.apply_host(Xh.t(), "Ls", out=Yh)          # staging allocated outside the timed region
    torch.cuda.synchronize()
    barrier(world)
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.apply_host(Xh.t(), "Ls", out=Yh)
    e2e_s = max_over_ranks(time.perf_counter() - t, world)
    yd = ycols.cpu()
    e2e = {"value": world * nrhs * args.e2e_steps / e2e_s, "unit": "matvecs/s",
           "h2d_bytes_per_step": n * nrhs * 8, "d2h_bytes_per_step": n * nrhs * 8,
           "api": "nfl_apply_host (page-locked host blocks, copies overlapped with the products)",
           "rel_diff_vs_device_product": float(torch.linalg.norm(Yh - yd) / torch.linalg.norm(yd))}

    # plain FP64 single-vector form on the same data
    fp64 = None
    x0 = xg[:, 0].contiguous()
    if args.fp64_steps > 0:
        p64 = Plan(vg, CFG["sigma"], CFG["N"], CFG["m"], CFG["p"], -1.0, "fp64")
        y64 = p64.apply_Ls(x0)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.fp64_steps):
            p64.apply_Ls(x0, out=y64)
        s1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(s0.elapsed_time(s1) / args.fp64_steps, world)
        w64 = p64.apply_W(x0).cpu().numpy()
        p64.close()
        fp64 = {"value": world * 1000.0 / ms64, "unit": "matvecs/s", "ms_per_matvec": ms64}

    # accuracy of the timed form: W x on sampled rows against the direct FP64 sum
    wmix = plan.apply_W(x0).cpu().numpy()
    err = {}
    if fp64 is not None:
        err["vs_gpu_fp64_all_rows"] = float(np.linalg.norm(wmix - w64) / np.linalg.norm(w64))
    cpu_baseline = None
    rows, ref = None, None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        rows = np.random.default_rng(3).choice(n, args.baseline_rows, replace=False)
        ref, secs, cores = oracle_rows(v, X[:, 0].copy(), rows)
        err["vs_direct_sample"] = float(np.linalg.norm(wmix[rows] - ref) / np.linalg.norm(ref))
        err["sample_rows"] = int(args.baseline_rows)
        cpu_baseline = {"value": args.baseline_rows / secs / n, "unit": "matvecs/s", "cores": cores,
                        "kind": "oracle",
                        "sample": "direct FP64 sum of W x for %d of %d target rows over all %d sources "
                                  "(plain C, OpenMP), %.1f s; extrapolated as rows/s / n" % (
                                      args.baseline_rows, n, n, secs)}

    # precision sweep: W x (one column) in every form on the same nodes, each against the
    # direct FP64 sum on the sampled rows and the GPU FP64 form on all rows
    sweep = None
    if not args.no_sweep:
        sweep = {args.precision: {"rel_err_vs_gpu_fp64": err.get("vs_gpu_fp64_all_rows"),
                                  "rel_err_vs_direct_sample": err.get("vs_direct_sample")}}
        if fp64 is not None and ref is not None:
            sweep["fp64"] = {"rel_err_vs_direct_sample": float(np.linalg.norm(w64[rows] - ref) / np.linalg.norm(ref))}
        for form in ("fp32", "fp32c", "bf16w"):
            if form == args.precision:
                continue
            pf = Plan(vg, CFG["sigma"], CFG["N"], CFG["m"], CFG["p"], -1.0, form)
            yf = pf.apply_W(x0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                pf.apply_W(x0, out=yf)
            e1.record(stream)
            torch.cuda.synchronize()
            wf = yf.cpu().numpy()
            entry = {"ms_per_matvec_W": e0.elapsed_time(e1) / 3}
            if fp64 is not None:
                entry["rel_err_vs_gpu_fp64"] = float(np.linalg.norm(wf - w64) / np.linalg.norm(w64))
            if ref is not None:
                entry["rel_err_vs_direct_sample"] = float(np.linalg.norm(wf[rows] - ref) / np.linalg.norm(ref))
            sweep[form] = entry
            pf.close()

    others = None
    if rank == 0 and not args.no_other:
        others = other_workloads(dev)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32+i64" if args.precision == "fp32c" else args.precision,
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nrhs_per_step": nrhs, "precision": args.precision,
                       "l2": "inputs larger than L2 (x block %d MB, node records %d MB)" % (
                           n * nrhs * 8 // 2**20, n * 16 // 2**20),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "box": info["box"], "work_items": info["work_items"],
                       "launch_params": {"fft_lines_cap": info["fft_lines_cap"], "slide_tiles": info["slide_tiles"],
                                         "block_cols": info["block_cols"], "chunk": info["chunk"],
                                         "dense_cell": info["dense_cell"], "dense_chunk": info["dense_chunk"],
                                         "dense_items": info["dense_items"],
                                         "autotuned": tuned is not None}},
            "point_rhs_per_s": value * n,
            "stage_ms_per_column": {"prep": stages["prep"] / max(1, stages["columns"]), "spread": spread_ms,
                                    "fft": fft_ms, "gather": gather_ms},
            "fp64_plain": fp64,
            "speedup_vs_fp64_plain": (value / world) / fp64["value"] * world if fp64 else None,
            "rel_err_W": err,
            "precision_sweep": sweep,
            "roofline": roofline,
            "spread_gather": spread_gather,
            "fma_rates_tflops": {k: (v / 1e12 if v else None) for k, v in rates.items()},
            "cpu_baseline": cpu_baseline,
            "other_workloads": others,
            "e2e": e2e,
            "gpu_launches": plan.kernels(nrhs) * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(out))
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
