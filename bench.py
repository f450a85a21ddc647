"""Benchmark: Mpoints/s per FMM evaluation of the headline workload on one B300.

Workload (synthetic, seeded): N = 1,000,000 points, 90 % from 8 Gaussian
clusters (sigma log-uniform in [0.01, 0.1]) + 10 % uniform background in the
unit square, complex strengths with N(0,1) real and imaginary parts, p = 17,
theta = 0.5, N_levels seeded by the cost model of eqs (2.4)-(2.5) with unit
costs measured on this GPU and refined by the library's AT3b autotuner during
warm-up.

One step = the whole hot path for one evaluation: rebuild the pyramid tree and
coupling lists for the step's coordinates (the paper re-partitions at every
time step) + one FMM evaluation (P2M, M2M, M2L, L2L, L2P, P2P) on the FP32
(mixed) path.  `value` is device time with inputs resident in HBM; `e2e` is the
same through the C ABI with host (pinned) buffers: H2D copy of points and
strengths, build, evaluate, D2H copy of the potentials, every step.  The FP64
path, the adjoint, the logarithmic kernel, theta tuning and the other four
workloads (plain FP64 at 1e4, the 20-snapshot dynamic sequence at 2e6, the
512-instance batch, the differentiated 1e6 set) are timed beside it, each with
its sampled error against the oracle's exact sums.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "Mpoints/s per FMM eval at N=1e6, rel err<=1e-5: FP32 vs FP64 path; bwd/fwd"
UNIT = "Mpoints/s"
N_POINTS = 1_000_000
P_TERMS = 17
THETA = 0.5
WORKLOAD = "cluster_mix_1e6_p17_theta0.5"
# N_levels the autotuner settles on for the headline workload (leaves of ~15
# points); the reference arm evaluates the oracle at this N_levels
HEADLINE_NLEVELS = 9
# dram__bytes_read.sum + dram__bytes_write.sum of one P2P launch (k_p2p_pairs) at
# N_levels = 9 on this workload, from one ncu capture of the kernel as it is built
P2P_TRAFFIC_BYTES = 82_951_424 + 4_469_504
# algorithmic FP32 flops of one point-pair interaction Gamma_j / (z_i - z_j) with
# complex Gamma (FMA = 2): difference 2, |d|^2 3, the two scalings by 1/|d|^2 2,
# complex product and accumulation 8 (the reciprocal runs on the MUFU unit)
P2P_FLOPS = 15.0
# what the kernel issues per pair: the hi/lo compensated difference adds 4
# additions, the guard of |d|^2 one (context, not the method's work)
P2P_FLOPS_ISSUED = 20.0
# the same for the logarithmic kernel: difference 2, |d|^2 3, the complex
# accumulation of Gamma_j log2|d|^2 4 (plus one log2 on the MUFU unit)
P2P_LOG_FLOPS = 9.0
FP32_FLOP_PER_CLK_SM = 256  # 128 FP32 lanes x FMA


def _config(nlevels):
    """The workload both arms time (the same dict on the reference arm's line)."""
    return {"workload": WORKLOAD, "n_points": N_POINTS, "p": P_TERMS, "theta": THETA, "nlevels": int(nlevels)}


def _peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _inputs():
    from paper_1311_1006_b300 import workloads as W

    g = W.rng(W.W_CLUSTER_1M)
    xy = W.cluster_mix(N_POINTS, g)
    gam = W.complex_strengths(N_POINTS, g)
    return xy, gam


class _Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value, on every rank (the value itself on one process)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Replicas: every rank processes units_per_rank per step; the whole job's
    rate is the units all ranks processed over the slowest rank's step time
    (millions per second)."""
    return units_per_rank * world / (ms * 1e-3) / 1e6


def _timed_ms(fn, reps, stream, flush):
    """CUDA-event times (ms) of `reps` calls of fn on `stream`, L2 flushed before each."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for _ in range(reps):
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _mps(n, ms):
    return round(n / (ms * 1e-3) / 1e6, 3)


def _seed_and_tune(F, tree, X, G, out, stream, steps):
    """N_levels of the headline tree: one evaluation with every phase timed alone
    calibrates the unit costs of eqs (2.4)-(2.5); the cost-model seed starts an
    AT3b walk (Algorithm 4) over `steps` rebuild + evaluate steps."""
    import torch

    tree.rebuild(X, flags=F.FMM_FLAG_TIMING | F.FMM_FLAG_SERIAL)
    for _ in range(2):
        tree.eval(G, out=out)
    alpha, beta = tree.calibrate_cost_model()
    seed = F.default_nlevels(tree.n, tree.params.p, "fp32")
    tree.rebuild(X, nlevels=seed, flags=0)
    tree.autotune_config(cap=0.2, window=3, period=3)
    L = seed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        e0.record(stream)
        tree.rebuild(X, nlevels=L)
        tree.eval(G, out=out)
        e1.record(stream)
        e1.synchronize()
        L = tree.autotune_step(e0.elapsed_time(e1) * 1e-3)
    return {"alpha_s": alpha, "beta_s": beta, "seed": seed, "tuned": int(tree.info()["autotune_nlevels"]),
            "tuning_steps": steps}


# ---------------------------------------------------------------- other workloads
def leg_c1(F, orc, dev, stream, flush):
    """Plain FMM, FP64: N = 1e4 uniform, real N(0,1) strengths, p = 20, theta = 0.5,
    N_levels = 5 (39 points per leaf); error against the full direct sum."""
    import torch
    from paper_1311_1006_b300 import workloads as W

    n, p, L = 10_000, 20, 5
    g = W.rng(W.W_PLAIN_FP64)
    xy, gam = W.uniform(n, g), W.real_strengths(n, g)
    X, G = torch.tensor(xy, device=dev), torch.tensor(gam, device=dev)
    t = F.Tree.build(X, p=p, theta=THETA, nlevels=L, path="fp64")
    out = torch.empty(n, dtype=torch.complex128, device=dev)
    step = lambda: t.step(X, G, out=out)  # noqa: E731
    _timed_ms(step, 5, stream, flush)
    ms = float(np.median(_timed_ms(step, 20, stream, flush)))
    phi = out.cpu().numpy()
    exact = orc.direct(xy, gam)
    ofmm = orc.fmm(xy, gam, L, THETA, p)["phi"]
    t.close()
    # the oracle on the same workload, all host cores and one thread, median of 5 evaluations each
    cpu = {}
    for label, th in (("all_cores", os.cpu_count() or 1), ("one_thread", 1)):
        orc.set_threads(th)
        ts = []
        for _ in range(5):
            t0 = time.time()
            orc.fmm(xy, gam, L, THETA, p)
            ts.append(time.time() - t0)
        cpu[label] = {"seconds": round(float(np.median(ts)), 4), "value": _mps(n, float(np.median(ts)) * 1e3),
                      "threads": orc.max_threads()}
    orc.set_threads(os.cpu_count() or 1)
    return {"workload": "uniform_1e4_p20_theta0.5_fp64", "n_points": n, "p": p, "nlevels": L, "path": "fp64",
            "ms_per_step": round(ms, 4), "value": _mps(n, ms), "unit": UNIT,
            "rel_err_vs_direct": _rel(phi, exact), "rel_err_vs_oracle_fmm": _rel(phi, ofmm),
            "oracle_fmm_rel_err_vs_direct": _rel(ofmm, exact),
            "cpu_oracle": cpu, "step": "fmm_step (rebuild + evaluate), median of 20, L2 flushed"}


def leg_c3(F, orc, dev, stream, flush):
    """Dynamic sequence: 20 snapshots at N = 2e6 (uniform, then 4 Gaussians with
    sigma = 0.2 * 0.8^k), real U(-1,1) strengths, theta = 0.5, p in {12, 30},
    FP32 and FP64 paths.  Each snapshot is a time step: the tree is rebuilt for
    its points and the AT3b tuner, carried across snapshots, retunes N_levels
    from every step's time."""
    import torch
    from paper_1311_1006_b300 import workloads as W

    n, K = 2_000_000, 20
    snaps = []
    for k in range(K):
        g = W.rng(W.W_DYNAMIC, k)
        xy, gam = W.snapshot(n, k, g), W.uniform_real_strengths(n, g)
        tg = np.random.default_rng(200 + k).choice(n, 64, replace=False)
        snaps.append((torch.tensor(xy, device=dev), torch.tensor(gam, device=dev), tg,
                      orc.direct(xy, gam, targets=tg)))
        del xy, gam
    res = {"workload": "dynamic_20x2e6_theta0.5", "n_points": n, "snapshots": K,
           "step": "per snapshot: steps of tree rebuild + evaluation, the tuner fed every step's time; "
                   "value = points of all steps / their summed time; L2 flushed before every step",
           "error": "rel. max-norm vs the exact sum on 64 sampled points per snapshot (last step)"}
    for path in ("fp32", "fp64"):
        for p in (12, 30):
            S = 8 if path == "fp32" else 3
            L = F.default_nlevels(n, p, path)
            seed = L
            tree = F.Tree.build(snaps[0][0], p=p, theta=THETA, nlevels=L, path=path)
            tree.autotune_config(cap=0.2, window=2, period=2)
            out = torch.empty(n, dtype=tree.out_dtype, device=dev)
            tree.eval(snaps[0][1], out=out)
            per_ms, levels, errs, tot = [], [], [], 0.0
            for X, G, tg, exact in snaps:
                ts = []
                for _ in range(S):
                    Lc = L

                    def _one():
                        tree.rebuild(X, nlevels=Lc)
                        tree.eval(G, out=out)

                    ms = _timed_ms(_one, 1, stream, flush)[0]
                    ts.append(ms)
                    L = tree.autotune_step(ms * 1e-3)
                tot += sum(ts)
                per_ms.append(round(float(np.median(ts)), 3))
                levels.append(int(tree.info()["autotune_nlevels"]))
                errs.append(_rel(out.cpu().numpy().astype(np.complex128)[tg], exact))
            tree.close()
            res[f"{path}_p{p}"] = {"value": _mps(n * S * K, tot), "unit": UNIT, "steps_per_snapshot": S,
                                   "nlevels_seed": seed, "nlevels": levels, "ms_median": per_ms,
                                   "rel_err_max": max(errs), "rel_err": [float(f"{e:.3g}") for e in errs]}
    return res


def leg_c4(F, orc, dev, stream, flush):
    """Batched: 512 independent instances, N_b = floor(10^U(3,5)), each uniform or
    one Gaussian (sigma 0.05), real N(0,1) strengths, p = 16, theta = 0.5, FP32
    path; per-instance N_levels from the cost-model seed.  One step = forest
    rebuild + one evaluation of all instances (each phase one launch)."""
    import torch
    from paper_1311_1006_b300 import workloads as W

    g = W.rng(W.W_BATCHED)
    sizes = W.batch_sizes(512, g)
    pts = [W.batch_instance(int(m), g) for m in sizes]
    gam = [W.real_strengths(int(m), g) for m in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xy, G = np.vstack(pts), np.concatenate(gam)
    n = int(offs[-1])
    X, Gd = torch.tensor(xy, device=dev), torch.tensor(G, device=dev)
    t = F.Tree.build_batched(X, offs, p=16, theta=THETA, path="fp32")
    out = torch.empty(n, dtype=torch.complex64, device=dev)
    step = lambda: t.step(X, Gd, out=out)  # noqa: E731
    _timed_ms(step, 3, stream, flush)
    ms = float(np.median(_timed_ms(step, 7, stream, flush)))
    ev = float(np.median(_timed_ms(lambda: t.eval(Gd, out=out), 7, stream, flush)))
    phi = out.cpu().numpy().astype(np.complex128)
    pick = np.random.default_rng(41)
    picks = []
    for b in pick.choice(512, 8, replace=False):
        s, e = offs[b], offs[b + 1]
        tg = pick.choice(e - s, min(32, e - s), replace=False)
        picks.append((s, e, tg, orc.direct(xy[s:e], G[s:e], targets=tg)))

    def _err(ph):
        return max(_rel(ph[s:e][tg], ex) for s, e, tg, ex in picks)

    err = _err(phi)
    lev = t.export("inst")[:, 2]
    info = t.info()
    # the same forest evaluated by the persistent kernel: one launch over a device work queue
    t.rebuild(X, flags=F.FMM_FLAG_PERSISTENT)
    t.eval(Gd, out=out)
    t.eval_status()
    ms_p = float(np.median(_timed_ms(step, 7, stream, flush)))
    ev_p = float(np.median(_timed_ms(lambda: t.eval(Gd, out=out), 7, stream, flush)))
    err_p = _err(out.cpu().numpy().astype(np.complex128))
    t.close()
    return {"workload": "batched_512_p16_theta0.5_fp32", "instances": 512, "n_points": n, "p": 16,
            "ms_per_step": round(ms, 4), "value": _mps(n, ms), "unit": UNIT,
            "eval_ms": round(ev, 4), "eval_mpoints_s": _mps(n, ev),
            "nlevels_range": [int(lev.min()), int(lev.max())], "launches_per_step":
                int(info["launches_build"] + info["launches_eval"]),
            "rel_err_sampled": err, "mode": "per-phase forest: one launch per phase over all instances",
            "persistent": {"ms_per_step": round(ms_p, 4), "value": _mps(n, ms_p), "eval_ms": round(ev_p, 4),
                           "eval_mpoints_s": _mps(n, ev_p), "rel_err_sampled": err_p,
                           "mode": "one persistent launch per evaluation over a device work queue "
                                   "(M2L on the CUDA cores)"},
            "error": "rel. max-norm per instance vs the exact sum, 8 instances x 32 points, max"}


def leg_c5(F, orc, dev, stream, flush):
    """Differentiated: N = 1e6 uniform, real N(0,1) strengths, p = 17, theta = 0.5,
    FP32 path; upstream gradient w + i v with w, v ~ N(0,1).  Forward = one
    evaluation, backward = fmm_eval_backward (strength and position gradients)."""
    import torch
    from paper_1311_1006_b300 import workloads as W

    n = 1_000_000
    g = W.rng(W.W_DIFFERENTIATED)
    xy, gam = W.uniform(n, g), W.real_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    X, G, GP = (torch.tensor(a, device=dev) for a in (xy, gam, gphi))
    t = F.Tree.build(X, p=17, theta=THETA, path="fp32")
    out = torch.empty(n, dtype=torch.complex64, device=dev)
    t.eval(G, out=out)
    fwd = float(np.median(_timed_ms(lambda: t.eval(G, out=out), 7, stream, flush)))
    grads = [t.backward(G, GP)]

    def _bwd():
        grads[0] = t.backward(G, GP)

    bwd = float(np.median(_timed_ms(_bwd, 7, stream, flush)))
    gg, gxy = grads[0]
    tg = np.random.default_rng(51).choice(n, 128, replace=False)
    rg, rxy = orc.direct_grad(xy, gam, gphi, targets=tg)
    info = t.info()
    t.close()
    # the oracle on the same workload (all host cores, one run each): forward FMM, and the frozen-tree gradient
    orc.set_threads(os.cpu_count() or 1)
    t0 = time.time()
    orc.fmm(xy, gam, info["nlevels_max"], THETA, 17)
    t_fwd = time.time() - t0
    t0 = time.time()
    orc.fmm_grad(xy, gam, gphi, info["nlevels_max"], THETA, 17)
    t_bwd = time.time() - t0
    return {"workload": "differentiated_uniform_1e6_p17_theta0.5_fp32", "n_points": n, "p": 17,
            "nlevels": info["nlevels_max"], "fwd_ms": round(fwd, 4), "bwd_ms": round(bwd, 4),
            "bwd_over_fwd": round(bwd / fwd, 3), "value": _mps(n, fwd + bwd), "unit": UNIT,
            "value_note": "points per second of forward + backward",
            "rel_err_grad_gamma": _rel(gg.cpu().numpy()[tg], rg),
            "rel_err_grad_xy": _rel(gxy.cpu().numpy()[tg], rxy),
            "cpu_oracle": {"threads": orc.max_threads(), "fwd_s": round(t_fwd, 3), "grad_s": round(t_bwd, 3),
                           "note": "oracle FMM and its frozen-tree gradient (plain FP64 C, all host cores)"},
            "error": "rel. max-norm vs the direct-sum gradient on 128 sampled points"}


def leg_targets(F, orc, dev, stream, flush):
    """Separate evaluation points (eq 2.2), M = N: the headline's 1e6 sources
    (cluster mixture, complex strengths) and 1e6 evaluation points uniform in
    the unit square; p = 17, theta = 0.5, FP32 path, N_levels from the seed for
    the 2e6 points.  One step = rebuild over both sets + evaluation at the
    evaluation points."""
    import torch
    from paper_1311_1006_b300 import workloads as W

    src, gam = _inputs()
    tgt = W.uniform(N_POINTS, np.random.default_rng(W.BASE_SEED + 77))
    S, T, G = (torch.tensor(a, device=dev) for a in (src, tgt, gam))
    t = F.Tree.build_targets(S, T, p=P_TERMS, theta=THETA, path="fp32")
    out = torch.empty(N_POINTS, dtype=torch.complex64, device=dev)
    t.eval_targets(G, out=out)

    def _step():
        t.rebuild_targets(S, T)
        t.eval_targets(G, out=out)

    _timed_ms(_step, 3, stream, flush)
    ms = float(np.median(_timed_ms(_step, 7, stream, flush)))
    ev = float(np.median(_timed_ms(lambda: t.eval_targets(G, out=out), 7, stream, flush)))
    pick = np.random.default_rng(61).choice(N_POINTS, 256, replace=False)
    err = _rel(out.cpu().numpy().astype(np.complex128)[pick], orc.direct_points(src, gam, tgt[pick]))
    info = t.info()
    t.close()
    return {"workload": "targets_1e6_sources_1e6_uniform_points_p17", "n_sources": N_POINTS,
            "n_targets": N_POINTS, "nlevels": info["nlevels_max"], "ms_per_step": round(ms, 4),
            "value": _mps(N_POINTS, ms), "unit": "M evaluation points/s", "eval_ms": round(ev, 4),
            "rel_err_sampled": err,
            "error": "rel. max-norm vs the exact sum over the sources at 256 sampled evaluation points"}


def run_gpu(args):
    import torch

    import paper_1311_1006_b300 as F
    from paper_1311_1006_b300 import _lib

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the single-thread oracle run goes in its own process, started before any
    # GPU work, on one host core while the GPU legs run
    st_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not (args.only_step or args.log_kernel):
        st_proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-leg", "1"],
                                   stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream(device=dev)
    xy, gam = _inputs()
    X = torch.tensor(xy, device=dev)
    G = torch.tensor(gam, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 126 MB L2

    with torch.cuda.stream(stream):
        # --- N_levels: cost-model seed from measured unit costs, then AT3b -----
        L0 = args.nlevels or F.default_nlevels(N_POINTS, P_TERMS, "fp32")
        tree = F.Tree.build(X, p=P_TERMS, theta=THETA, nlevels=L0, path="fp32")
        phi = torch.empty(N_POINTS, dtype=torch.complex64, device=dev)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        tuning = None
        if args.nlevels:
            tuned = args.nlevels
        else:
            tuning = _seed_and_tune(F, tree, X, G, phi, stream, max(30, args.warmup))
            tuned = tuning["tuned"]
        tree.rebuild(X, nlevels=tuned, flags=0)
        info = tree.info()

        # --- timed: build + eval, inputs resident ------------------------------
        # one step = fmm_step (rebuild + evaluation in one call); the logarithmic
        # kernel's profiling mode keeps the two calls
        if args.log_kernel:
            def one_step():
                tree.rebuild(X)
                tree.eval_log(G, out=phi)
        else:
            def one_step():
                tree.step(X, G, out=phi)
        for _ in range(args.warmup):
            one_step()
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with _Clocks(local) as clk:
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                one_step()
                ends[k].record(stream)
            torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        ms = _max_over_ranks(float(np.mean(step_ms)), dist, dev)
        if args.only_step or args.log_kernel:
            if rank == 0:
                print(json.dumps({"metric": METRIC, "value": round(_whole_job_rate(N_POINTS, world, ms), 2),
                                  "unit": UNIT, "ms_per_step": round(ms, 4), "nlevels": tuned,
                                  "kernel": "log" if args.log_kernel else "harmonic", "only_step": True}))
            return

        # --- end to end through the public API with host buffers -----------------
        # Every step copies its inputs from pinned host memory and reads its result
        # back; the copies run on a copy stream, double-buffered, so that step k+1's
        # inputs travel while step k computes and step k's result travels while
        # step k+1 computes.  The timed region spans all K steps, first copy to
        # last read-back.
        h_xy = torch.tensor(xy).pin_memory()
        h_g = torch.tensor(gam).pin_memory()
        h_phi = [torch.empty(N_POINTS, dtype=torch.complex64).pin_memory() for _ in range(2)]
        d_xy = [torch.empty_like(X) for _ in range(2)]
        d_g = [torch.empty_like(G) for _ in range(2)]
        d_phi = [torch.empty(N_POINTS, dtype=torch.complex64, device=dev) for _ in range(2)]
        cstream = torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_last = torch.cuda.Event()

        def _copy_in(bi):
            cstream.wait_event(ev_done[bi])  # the step that last read buffer bi has finished
            with torch.cuda.stream(cstream):
                d_xy[bi].copy_(h_xy, non_blocking=True)
                d_g[bi].copy_(h_g, non_blocking=True)
            ev_in[bi].record(cstream)

        def _step(k):
            bi = k % 2
            stream.wait_event(ev_in[bi])
            flush.zero_()
            tree.step(d_xy[bi], d_g[bi], out=d_phi[bi])
            ev_done[bi].record(stream)
            cstream.wait_event(ev_done[bi])
            with torch.cuda.stream(cstream):
                h_phi[bi].copy_(d_phi[bi], non_blocking=True)

        def _pipeline(K):
            for bi in range(2):
                ev_done[bi].record(stream)
            e0.record(stream)
            cstream.wait_event(e0)
            _copy_in(0)
            for k in range(K):
                if k + 1 < K:
                    _copy_in((k + 1) % 2)
                _step(k)
            ev_last.record(cstream)
            stream.wait_event(ev_last)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        _pipeline(2)
        e2e_ms = _pipeline(args.steps) / args.steps
        if not np.allclose(h_phi[(args.steps - 1) % 2].numpy(), phi.cpu().numpy()):
            raise RuntimeError("end-to-end result differs from the device-resident step")

        # --- phase times (events recorded by the library on the streams the kernels
        # run on): once as in the step (P2P overlapped with the far field), once
        # with every phase alone (FMM_FLAG_SERIAL) for the per-kernel roofline
        def _phases(flags):
            tree.rebuild(X, flags=flags)
            ph = []
            for _ in range(5):
                flush.zero_()
                tree.eval(G, out=phi)
                ph.append(tree.phase_times())
            return {k: float(np.median([p[k] for p in ph])) for k in ph[0]}

        phases = _phases(F.FMM_FLAG_TIMING)
        phases_alone = _phases(F.FMM_FLAG_TIMING | F.FMM_FLAG_SERIAL)
        tree.rebuild(X, flags=0)
        build_ms = float(np.median(_timed_ms(lambda: tree.rebuild(X), 15, stream, flush)))
        eval_ms = float(np.median(_timed_ms(lambda: tree.eval(G, out=phi), 15, stream, flush)))

        # --- accuracy on sampled points vs the exact sum (oracle) -----------------
        orc = None
        err32 = None
        if rank == 0:
            import oracle as orc

            tg = np.random.default_rng(7).choice(N_POINTS, 1024, replace=False)
            exact = orc.direct(xy, gam, targets=tg)
            err32 = _rel(phi.cpu().numpy().astype(np.complex128)[tg], exact)

        # --- FP64 path on the same workload -------------------------------------
        t64 = F.Tree.build(X, p=P_TERMS, theta=THETA, nlevels=tuned, path="fp64")
        phi64 = torch.empty(N_POINTS, dtype=torch.complex128, device=dev)

        def _step64():
            t64.rebuild(X)
            t64.eval(G, out=phi64)

        _step64()
        ms64 = float(np.median(_timed_ms(_step64, 3, stream, flush)))
        err64 = _rel(phi64.cpu().numpy()[tg], exact) if rank == 0 else None
        # the FP64 path at its own smallest p that meets the same 1e-5 on the sampled points
        fp64_pmin = None
        if rank == 0:
            for pp in range(8, P_TERMS + 1):
                t64.rebuild(X, p=pp)
                t64.eval(G, out=phi64)
                e_pp = _rel(phi64.cpu().numpy()[tg], exact)
                if e_pp <= 1e-5:
                    # N_levels re-chosen for this p: the FP64 balance of P2P and M2L differs from FP32's
                    best = None
                    for Lp in (tuned - 1, tuned, tuned + 1):
                        if Lp < 1 or 4 ** (Lp - 1) > N_POINTS:
                            continue
                        t64.rebuild(X, nlevels=Lp)
                        t64.eval(G, out=phi64)
                        e_l = _rel(phi64.cpu().numpy()[tg], exact)
                        mp = float(np.median(_timed_ms(_step64, 3, stream, flush)))
                        if e_l <= 1e-5 and (best is None or mp < best[0]):
                            best = (mp, Lp, e_l)
                    if best is not None:
                        mp, Lp, e_l = best
                        fp64_pmin = {"p": pp, "nlevels": Lp, "ms_per_step": round(mp, 4),
                                     "value": round(N_POINTS / (mp * 1e-3) / 1e6, 2), "rel_err_sampled": e_l}
                    break
        t64.close()

        # --- logarithmic kernel (Sec. 3.3) on the same tree and workload -----------
        log_kernel = None
        try:
            phil = torch.empty(N_POINTS, dtype=torch.complex64, device=dev)
            tree.eval_log(G, out=phil)
            tree.rebuild(X, flags=F.FMM_FLAG_TIMING | F.FMM_FLAG_SERIAL)
            lp = []
            for _ in range(5):
                flush.zero_()
                tree.eval_log(G, out=phil)
                lp.append(tree.phase_times()["p2p"])
            tree.rebuild(X, flags=0)
            ls, le = [], []
            for _ in range(5):
                flush.zero_()
                e0.record(stream)
                tree.rebuild(X)
                e1.record(stream)
                tree.eval_log(G, out=phil)
                e2.record(stream)
                e2.synchronize()
                ls.append(e0.elapsed_time(e2))
                le.append(e1.elapsed_time(e2))
            log_p2p_ms = float(np.median(lp))
            log_ms = float(np.median(ls))
            log_eval_ms = float(np.median(le))
            lerr = None
            if rank == 0:
                tgl = np.random.default_rng(9).choice(N_POINTS, 512, replace=False)
                lerr = _rel(phil.cpu().numpy().astype(np.complex128)[tgl], orc.direct_log(xy, gam, targets=tgl))
            log_kernel = {"ms_per_step": round(log_ms, 4), "eval_ms": round(log_eval_ms, 4),
                          "value": round(N_POINTS / (log_ms * 1e-3) / 1e6, 2), "unit": UNIT,
                          "eval_over_harmonic_eval": round(log_eval_ms / eval_ms, 3),
                          "p2p_ms_alone": round(log_p2p_ms, 4),
                          "p2p_tflops": round(info["p2p_pairs"] * P2P_LOG_FLOPS / (log_p2p_ms * 1e-3) / 1e12, 3),
                          "rel_err_sampled": lerr,
                          "step": "tree rebuild + lists + one log-kernel evaluation (FP32 path, same tree)"}
        except _lib.FMMError:
            log_kernel = None

        # --- adjoint / forward ratio (same tree) ------------------------------
        bwd_ratio = None
        try:
            gphi = torch.complex(torch.randn(N_POINTS, device=dev, dtype=torch.float64),
                                 torch.randn(N_POINTS, device=dev, dtype=torch.float64))
            tree.backward(G, gphi)
            bb = _timed_ms(lambda: tree.backward(G, gphi), 3, stream, flush)
            bwd_ratio = float(np.median(bb)) / eval_ms
        except _lib.FMMError:
            bwd_ratio = None

        # --- theta autotuning (the second control of Sec. 4.2): N_levels and theta
        # tuned together at TOL = 1e-6, p following theta, on the same workload;
        # two independent walks, to show whether they agree -------------------------
        theta_tune = None
        if rank == 0 and not args.no_theta_tune:
            tol = 1e-6
            tg2 = np.random.default_rng(8).choice(N_POINTS, 1024, replace=False)
            ex2 = orc.direct(xy, gam, targets=tg2)
            walks = []
            start_ms = None
            for walk in range(2):
                th, L2 = THETA, tuned
                pp = F.p_for_tolerance(tol, th)
                tt = F.Tree.build(X, p=pp, theta=th, nlevels=L2, path="fp32")
                ph = torch.empty(N_POINTS, dtype=torch.complex64, device=dev)

                def _tt_step():
                    tt.rebuild(X)
                    tt.eval(G, out=ph)

                tt.eval(G, out=ph)
                if start_ms is None:  # the starting point (theta of the workload, p from the tolerance rule)
                    start_ms = float(np.median(_timed_ms(_tt_step, 10, stream, flush)))
                tt.autotune_config(cap=0.2, window=4, period=4)
                tt.autotune_theta(tol, 0.35, 0.65)
                for _ in range(120):
                    e0.record(stream)
                    tt.rebuild(X, nlevels=L2, theta=th, p=pp)
                    tt.eval(G, out=ph)
                    e1.record(stream)
                    e1.synchronize()
                    L2, th, pp = tt.autotune_params(e0.elapsed_time(e1) * 1e-3)
                inf2 = tt.info()
                L2, th = int(inf2["autotune_nlevels"]), float(inf2["autotune_theta"])
                pp = F.p_for_tolerance(tol, th)
                tt.rebuild(X, nlevels=L2, theta=th, p=pp)
                tt.eval(G, out=ph)
                tuned_ms = float(np.median(_timed_ms(_tt_step, 10, stream, flush)))
                walks.append({"theta": round(th, 4), "p": pp, "nlevels": L2, "ms_per_step": round(tuned_ms, 4),
                              "value": round(N_POINTS / (tuned_ms * 1e-3) / 1e6, 2),
                              "rel_err_sampled": _rel(ph.cpu().numpy().astype(np.complex128)[tg2], ex2)})
                tt.close()
            theta_tune = dict(walks[0])
            theta_tune.update({"tol": tol, "tuning_steps": 120, "window": 4, "period": 4,
                               "start": {"theta": THETA, "p": F.p_for_tolerance(tol, THETA), "nlevels": tuned,
                                         "ms_per_step": round(start_ms, 4)},
                               "second_walk": walks[1]})

        # --- the other four workloads ----------------------------------------------
        legs = {}
        if rank == 0:
            tree.close()
            for name, fn in (("c1", leg_c1), ("c3", leg_c3), ("c4", leg_c4), ("c5", leg_c5),
                             ("targets", leg_targets)):
                if name in args.skip_legs:
                    continue
                torch.cuda.empty_cache()
                t_leg = time.time()
                legs[name] = fn(F, orc, dev, stream, flush)
                legs[name]["wall_s"] = round(time.time() - t_leg, 1)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    value = _whole_job_rate(N_POINTS, world, ms)
    clocks = clk.summary()
    # dominant kernel: P2P, bound by the FP32 pipe.  Peak = SMs x 256 flop/clk x
    # SM clock (the median sampled under load; also given at the 2032 MHz max).
    sm_mhz = clocks.get("sm_mhz") or 2032.0
    peak = sm_count * FP32_FLOP_PER_CLK_SM * sm_mhz * 1e6 / 1e12
    peak_max = sm_count * FP32_FLOP_PER_CLK_SM * 2032e6 / 1e12
    p2p_ms = phases_alone["p2p"]
    achieved = info["p2p_pairs"] * P2P_FLOPS / (p2p_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (P2P/M2L/P2M/L2P) + f64 (M2M/L2L)",
        "data": "synthetic (seeded Gaussian-cluster mixture)",
        "config": _config(info["nlevels_max"]),
        "path": "fp32",
        "l2": "flushed (256 MB write) between steps",
        "step": "fmm_step: tree rebuild + lists + one evaluation (upward pass overlapped with the list build)",
        "parallelism": "replicas" if world > 1 else "1 gpu",
        "nlevels_tuning": tuning,
        "breakdown_ms": {"build": round(build_ms, 4), "eval": round(eval_ms, 4),
                         "in_step": {k: round(v, 4) for k, v in phases.items()},
                         "alone": {k: round(v, 4) for k, v in phases_alone.items()}},
        "eval_only_mpoints_s": round(N_POINTS / (eval_ms * 1e-3) / 1e6, 2),
        "fp64_path": {"p": P_TERMS, "ms_per_step": round(ms64, 4), "value": round(N_POINTS / (ms64 * 1e-3) / 1e6, 2),
                      "rel_err_sampled": err64, "smallest_p_within_1e-5": fp64_pmin},
        "rel_err_sampled": err32,
        "bwd_over_fwd": bwd_ratio,
        "log_kernel": log_kernel,
        "theta_autotune": theta_tune,
        "roofline": {"kernel": "k_p2p_pairs (P2P, FP32 f32x2)", "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": P2P_TRAFFIC_BYTES, "kernel_ms": round(p2p_ms, 4),
                     "frac_at_max_clock": round(achieved / peak_max, 4),
                     "flops_per_pair": P2P_FLOPS,
                     "frac_issued": round(achieved / peak * P2P_FLOPS_ISSUED / P2P_FLOPS, 4),
                     "peak_note": f"FP32 peak from unit counts: {sm_count} SMs (device property) x 256 flop/clk x "
                                  f"{sm_mhz:.0f} MHz (median SM clock sampled during the timed steps); "
                                  f"{P2P_FLOPS:.0f} algorithmic flops per point pair (FMA = 2; frac_issued counts "
                                  f"the kernel's {P2P_FLOPS_ISSUED:.0f} with the hi/lo compensation); launch time "
                                  "from CUDA events with the pass alone; traffic from one ncu capture of this "
                                  "kernel at this workload"},
        "e2e": {"value": round(N_POINTS / (e2e_ms * 1e-3) / 1e6, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(xy.nbytes + gam.nbytes), "d2h_bytes_per_step": int(N_POINTS * 8),
                "ms_per_step": round(e2e_ms, 4),
                "note": "fmm_step per step, inputs copied from pinned host memory and the result "
                        "read back every step on a copy stream, double-buffered (step k+1's copies overlap step k); "
                        "L2 flushed before every step's rebuild"},
        "gpu_launches": int(args.steps * (info["launches_build"] + info["launches_eval"])),
        "interactions": {"p2p_pairs": info["p2p_pairs"], "m2l_pairs": info["n_weak"]},
    }
    line.update(legs)
    line["clocks"] = clocks
    if peaks:
        line["peaks_used"] = {"hbm_gbs": peaks.get("hbm_gbs")}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(info["nlevels_max"], st_proc)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def _oracle_eval_s(threads, nlevels=HEADLINE_NLEVELS):
    """Seconds of one oracle evaluation (plain FP64 C, OpenMP over boxes) of the
    headline workload itself: tree, lists and every pass, at `threads` threads."""
    import oracle

    xy, gam = _inputs()
    oracle.set_threads(threads)
    t = time.time()
    oracle.fmm(xy, gam, nlevels, THETA, P_TERMS)
    return time.time() - t, oracle.max_threads()


def cpu_baseline(nlevels=HEADLINE_NLEVELS, st_proc=None):
    """The oracle on the headline workload (1e6 points, p = 17, theta = 0.5, the
    GPU's N_levels) on the host's cores: one evaluation with all cores, and the
    single-thread run from the process started at the beginning of the benchmark."""
    single = None
    if st_proc is not None:
        try:
            out, _ = st_proc.communicate(timeout=900)
            single = json.loads(out.strip().splitlines()[-1])
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            st_proc.kill()
            single = None
    cores = os.cpu_count() or 1
    dt, used = _oracle_eval_s(cores, nlevels)
    res = {"value": round(N_POINTS / dt / 1e6, 4), "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"the headline workload itself: {N_POINTS} cluster-mixture points, p={P_TERMS}, "
                     f"theta={THETA}, N_levels={nlevels}; one evaluation incl. tree and lists ({dt:.2f} s)",
           "seconds": round(dt, 3)}
    if single is not None:
        res["single_thread"] = {"value": round(N_POINTS / single["seconds"] / 1e6, 4), "unit": UNIT, "cores": 1,
                                "seconds": round(single["seconds"], 3),
                                "note": "same evaluation on one thread, run while the GPU legs ran"}
        res["speedup_all_cores_vs_one"] = round(single["seconds"] / dt, 2)
    return res


def run_reference(args):
    """The oracle as the reference arm: every step is one full oracle evaluation
    of the headline workload (all host cores, N_levels of the headline)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    xy, gam = _inputs()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    for _ in range(args.warmup):
        oracle.fmm(xy, gam, HEADLINE_NLEVELS, THETA, P_TERMS)
    t0 = time.time()
    for _ in range(args.steps):
        oracle.fmm(xy, gam, HEADLINE_NLEVELS, THETA, P_TERMS)
    ms = (time.time() - t0) / args.steps * 1e3
    v = N_POINTS / (ms * 1e-3) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": _config(HEADLINE_NLEVELS),
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "kind": "oracle", "cores": oracle.max_threads(),
                             "sample": "every step is one full oracle evaluation of the headline workload "
                                       f"({N_POINTS} points, p={P_TERMS}, theta={THETA}, "
                                       f"N_levels={HEADLINE_NLEVELS}) incl. tree and lists"},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nlevels", type=int, default=0, help="fix N_levels (skip the calibration and autotuner)")
    ap.add_argument("--no-theta-tune", action="store_true", help="skip the theta autotuning run")
    ap.add_argument("--skip-legs", default="", help="comma-separated legs to skip (c1,c3,c4,c5,targets)")
    ap.add_argument("--only-step", action="store_true",
                    help="time the step only (no phase split, FP64 path, adjoint, e2e, accuracy); for profiling")
    ap.add_argument("--log-kernel", action="store_true",
                    help="time the logarithmic-kernel step only (as --only-step, with fmm_eval_log); for profiling")
    ap.add_argument("--oracle-leg", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    args.skip_legs = [x for x in args.skip_legs.split(",") if x]
    if args.oracle_leg:
        dt, used = _oracle_eval_s(args.oracle_leg)
        print(json.dumps({"seconds": dt, "threads": used}))
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
