"""Benchmark: Mpoints/s per FMM evaluation of the headline workload on one B300.

Workload (synthetic, seeded): N = 1,000,000 points, 90 % from 8 Gaussian
clusters (sigma log-uniform in [0.01, 0.1]) + 10 % uniform background in the
unit square, complex strengths with N(0,1) real and imaginary parts, p = 17,
theta = 0.5, N_levels picked by the library's AT3b autotuner during warm-up.

One step = the whole hot path for one evaluation: rebuild the pyramid tree and
coupling lists for the step's coordinates (the paper re-partitions at every
time step) + one FMM evaluation (P2M, M2M, M2L, L2L, L2P, P2P) on the FP32
(mixed) path.  `value` is device time with inputs resident in HBM; `e2e` is the
same through the C ABI with host (pinned) buffers: H2D copy of points and
strengths, build, evaluate, D2H copy of the potentials, every step.  The FP64
path and the adjoint are timed on the same workload and reported beside it.

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
# dram__bytes_read.sum + dram__bytes_write.sum of one P2P launch (k_p2p_pairs) at
# N_levels = 9 on this workload, from one ncu capture (profiles/p2p_pairs_cluster1e6_L9.md)
P2P_TRAFFIC_BYTES = 82_333_440 + 5_691_136
# algorithmic FP32 flops of one point-pair interaction (FMA = 2): compensated
# difference 6, |d|^2 4, the two scalings 2, the complex accumulation 8
P2P_FLOPS = 20.0
# the same for the logarithmic kernel: compensated difference 6, |d|^2 3, the
# complex accumulation of Gamma_j log2|d|^2 4 (plus one log2 on the MUFU unit)
P2P_LOG_FLOPS = 13.0
SM_COUNT = 148
FP32_FLOP_PER_CLK_SM = 256  # 128 FP32 lanes x FMA


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


def run_gpu(args):
    import torch

    import paper_1311_1006_b300 as F
    from paper_1311_1006_b300 import _lib

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    xy, gam = _inputs()
    X = torch.tensor(xy, device=dev)
    G = torch.tensor(gam, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 126 MB L2

    with torch.cuda.stream(stream):
        # --- N_levels: AT3b autotuner over a warm-up sequence -----------------
        L0 = F.default_nlevels(N_POINTS, P_TERMS, "fp32")
        tree = F.Tree.build(X, p=P_TERMS, theta=THETA, nlevels=L0, path="fp32")
        tree.autotune_config(cap=0.2, window=2, period=2)
        phi = torch.empty(N_POINTS, dtype=torch.complex64, device=dev)
        L = L0
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        for _ in range(0 if args.nlevels else max(24, args.warmup)):
            e0.record(stream)
            tree.rebuild(X, nlevels=L)
            tree.eval(G, out=phi)
            e1.record(stream)
            e1.synchronize()
            L = tree.autotune_step(e0.elapsed_time(e1) * 1e-3)
        tuned = args.nlevels or int(tree.info()["autotune_nlevels"])
        tree.rebuild(X, nlevels=tuned)
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
        bld = []
        for _ in range(5):
            flush.zero_()
            e0.record(stream)
            tree.rebuild(X)
            e1.record(stream)
            e1.synchronize()
            bld.append(e0.elapsed_time(e1))
        build_ms = float(np.median(bld))
        ev = []
        for _ in range(5):
            flush.zero_()
            e0.record(stream)
            tree.eval(G, out=phi)
            e1.record(stream)
            e1.synchronize()
            ev.append(e0.elapsed_time(e1))
        eval_ms = float(np.median(ev))

        # --- accuracy on sampled points vs the exact sum (oracle) -----------------
        err32 = None
        if rank == 0:
            import oracle

            tg = np.random.default_rng(7).choice(N_POINTS, 1024, replace=False)
            exact = oracle.direct(xy, gam, targets=tg)
            err32 = _rel(phi.cpu().numpy().astype(np.complex128)[tg], exact)

        # --- FP64 path on the same workload -------------------------------------
        t64 = F.Tree.build(X, p=P_TERMS, theta=THETA, nlevels=tuned, path="fp64")
        phi64 = torch.empty(N_POINTS, dtype=torch.complex128, device=dev)
        t64.rebuild(X)
        t64.eval(G, out=phi64)
        s64 = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            t64.rebuild(X)
            t64.eval(G, out=phi64)
            e1.record(stream)
            e1.synchronize()
            s64.append(e0.elapsed_time(e1))
        ms64 = float(np.median(s64))
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
                        sp = []
                        for _ in range(3):
                            flush.zero_()
                            e0.record(stream)
                            t64.rebuild(X)
                            t64.eval(G, out=phi64)
                            e1.record(stream)
                            e1.synchronize()
                            sp.append(e0.elapsed_time(e1))
                        mp = float(np.median(sp))
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
                import oracle as _orcl

                tgl = np.random.default_rng(9).choice(N_POINTS, 512, replace=False)
                lerr = _rel(phil.cpu().numpy().astype(np.complex128)[tgl], _orcl.direct_log(xy, gam, targets=tgl))
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
            bb = []
            for _ in range(3):
                flush.zero_()
                e0.record(stream)
                tree.backward(G, gphi)
                e1.record(stream)
                e1.synchronize()
                bb.append(e0.elapsed_time(e1))
            bwd_ratio = float(np.median(bb)) / eval_ms
        except _lib.FMMError:
            bwd_ratio = None

        # --- theta autotuning (the second control of Sec. 4.2): N_levels and theta
        # tuned together at TOL = 1e-6, p following theta, on the same workload ----
        theta_tune = None
        if rank == 0 and not args.no_theta_tune:
            tol = 1e-6
            th, L2 = THETA, tuned
            pp = F.p_for_tolerance(tol, th)
            tt = F.Tree.build(X, p=pp, theta=th, nlevels=L2, path="fp32")
            ph = torch.empty(N_POINTS, dtype=torch.complex64, device=dev)

            def _tt_ms():
                ms_ = []
                for _ in range(10):
                    flush.zero_()
                    e0.record(stream)
                    tt.rebuild(X)
                    tt.eval(G, out=ph)
                    e1.record(stream)
                    e1.synchronize()
                    ms_.append(e0.elapsed_time(e1))
                return float(np.median(ms_))

            tt.eval(G, out=ph)
            start_ms = _tt_ms()  # the starting point (theta of the workload, p from the tolerance rule)
            tt.autotune_config(cap=0.2, window=2, period=2)
            tt.autotune_theta(tol, 0.35, 0.65)
            for _ in range(60):
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
            tuned_ms = _tt_ms()
            import oracle as _orc

            tg2 = np.random.default_rng(8).choice(N_POINTS, 1024, replace=False)
            ex2 = _orc.direct(xy, gam, targets=tg2)
            theta_tune = {"tol": tol, "theta": round(th, 4), "p": pp, "nlevels": L2,
                          "ms_per_step": round(tuned_ms, 4),
                          "value": round(N_POINTS / (tuned_ms * 1e-3) / 1e6, 2),
                          "start": {"theta": THETA, "p": F.p_for_tolerance(tol, THETA), "nlevels": tuned,
                                    "ms_per_step": round(start_ms, 4)},
                          "rel_err_sampled": _rel(ph.cpu().numpy().astype(np.complex128)[tg2], ex2),
                          "tuning_steps": 60}
            tt.close()

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
    peak = SM_COUNT * FP32_FLOP_PER_CLK_SM * sm_mhz * 1e6 / 1e12
    peak_max = SM_COUNT * FP32_FLOP_PER_CLK_SM * 2032e6 / 1e12
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
        "config": {"workload": WORKLOAD, "n_points": N_POINTS, "p": P_TERMS, "theta": THETA,
                   "nlevels": info["nlevels_max"], "path": "fp32", "l2": "flushed (256 MB write) between steps",
                   "step": "fmm_step: tree rebuild + lists + one evaluation (upward pass overlapped with the list build)", "parallelism": "replicas" if world > 1 else "1 gpu"},
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
                     "peak_note": f"FP32 peak from unit counts: {SM_COUNT} SMs x 256 flop/clk x {sm_mhz:.0f} MHz "
                                  f"(median SM clock sampled during the timed steps); {P2P_FLOPS:.0f} algorithmic "
                                  "flops per point pair (FMA = 2), launch time from CUDA events with the pass alone"},
        "e2e": {"value": round(N_POINTS / (e2e_ms * 1e-3) / 1e6, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(xy.nbytes + gam.nbytes), "d2h_bytes_per_step": int(N_POINTS * 8),
                "ms_per_step": round(e2e_ms, 4),
                "note": "fmm_step per step, inputs copied from pinned host memory and the result "
                        "read back every step on a copy stream, double-buffered (step k+1's copies overlap step k); "
                        "L2 flushed before every step's rebuild"},
        "gpu_launches": int(args.steps * (info["launches_build"] + info["launches_eval"])),
        "interactions": {"p2p_pairs": info["p2p_pairs"], "m2l_pairs": info["n_weak"]},
    }
    line["clocks"] = clocks
    if peaks:
        line["peaks_used"] = {"hbm_gbs": peaks.get("hbm_gbs")}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(n=250_000, levels=8):
    """The oracle (plain FP64 C, OpenMP over boxes) on a bounded sample of the
    same workload: a 250k-point draw of the same generator, N_levels 8."""
    import oracle
    from paper_1311_1006_b300 import workloads as W

    g = W.rng(W.W_CLUSTER_1M)
    xy = W.cluster_mix(n, g)
    gam = W.complex_strengths(n, g)
    oracle.set_threads(os.cpu_count() or 1)
    t = time.time()
    oracle.fmm(xy, gam, levels, THETA, P_TERMS)
    dt = time.time() - t
    return {"value": round(n / dt / 1e6, 4), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} points of the same cluster-mixture generator, N_levels={levels}, p=17, one evaluation "
                      f"incl. tree ({dt:.2f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline()
    for _ in range(args.steps):
        vals.append(cpu_baseline())
    v = float(np.mean([x["value"] for x in vals]))
    ms = N_POINTS / (v * 1e6) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "n_points": N_POINTS, "p": P_TERMS, "theta": THETA},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "kind": "oracle", "cores": vals[0]["cores"],
                             "sample": vals[0]["sample"]},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nlevels", type=int, default=0, help="fix N_levels (skip the autotuner warm-up)")
    ap.add_argument("--no-theta-tune", action="store_true", help="skip the theta autotuning run")
    ap.add_argument("--only-step", action="store_true",
                    help="time the step only (no phase split, FP64 path, adjoint, e2e, accuracy); for profiling")
    ap.add_argument("--log-kernel", action="store_true",
                    help="time the logarithmic-kernel step only (as --only-step, with fmm_eval_log); for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
