#!/usr/bin/env python
"""Benchmark of the MCL expansion hot path on GB300.

A step is one whole MCL iteration through the C ABI (mcl_expand):
expansion A*A fused with prune / top-k select / recovery, inflation,
FP64 renormalisation and chaos, on the 1M-vertex power-law workload
(Zipf(2) degrees, mean ~50, capped at 5,000; ~49M nnz; lognormal(0,1)
weights; self-loops; column-stochastic).  value = expansion GFLOP/s
(2 x multiply-adds / step time), whole job.  The path does not shard:
with --gpus N each rank runs an independent replica (weak scaling).

--impl reference times the FP64 CPU oracle on the host cores on bounded
column samples of the same workload (the only CPU code bench.py runs
besides the cpu_baseline leg of the default arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "expansion GFLOP/s & MCL iters/s, learned+batched vs plain, 1 GB300 at 1e-5"
WORKLOAD = ("zipf1m: one MCL iteration (expand + prune theta=1e-4 / select k=1100 / recover 90% "
            "+ inflate r=2 + renormalise + chaos) on a 1M-vertex Zipf(2) power-law graph, "
            "mean degree ~50 capped at 5,000, lognormal(0,1) weights, int32 CSC, seed 0")
PARAMS = dict(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0)


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(flops):
    """DRAM bytes of one numeric-pass launch: the ncu capture recorded under
    profiles/ (read + write bytes of a smaller graph of the same family),
    scaled by multiply-adds; None when the kernel sources changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_expand_traffic.json")) as f:
            d = json.load(f)
        for path, sha in d["sources_sha256"].items():
            with open(os.path.join(ROOT, path), "rb") as g:
                if hashlib.sha256(g.read()).hexdigest() != sha:
                    return None
        per_mac = (d["dram_bytes_read"] + d["dram_bytes_write"]) / d["multiply_adds"]
        return int(per_mac * flops)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.idx], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, dist, device: str = "cpu") -> float:
    """The slowest rank's time (every rank gets it)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_rank: int, ms: float, world: int) -> float:
    """Whole-job expansion GFLOP/s: every rank runs a replica of the step,
    so the job does world x flops multiply-adds in the slowest rank's time."""
    return 2.0 * flops_per_rank * world / (ms / 1000.0) / 1e9


def make_workload(name: str, seed: int = 0, n: int | None = None):
    from paper_2002_10083_gb300 import synth
    cache = os.environ.get("MCL_BENCH_CACHE", "/tmp/mcl_bench_cache")
    path = os.path.join(cache, f"{name}_n{n}_s{seed}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return synth.CSC(n=int(z["n"]), colptr=z["colptr"], rowidx=z["rowidx"], val=z["val"])
    A = synth.config(name, seed=seed, **({"n": n} if n else {}))
    A = synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=A.val.astype(np.float32))
    try:
        os.makedirs(cache, exist_ok=True)
        np.savez(path + ".tmp.npz", n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=A.val)
        os.replace(path + ".tmp.npz", path)
    except Exception:
        pass
    return A


def oracle_gflops(A, seconds: float, seed: int = 1):
    """The FP64 oracle as it stands on random column samples: GFLOP/s."""
    import oracle
    prm = oracle.Params(theta=float(np.float32(PARAMS["threshold"])), K=PARAMS["select_k"],
                        p=float(np.float32(PARAMS["recover_pct"])), r=PARAMS["inflation"])
    Ad = synth_as_f64(A)
    rng = np.random.default_rng(seed)
    flops, ncols, t0 = 0, 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        cols = rng.choice(A.n, 2048, replace=False).astype(np.int32)
        res = oracle.expand_cols(Ad, prm, cols=cols, kcap=PARAMS["select_k"])
        flops += int(res.flops.sum())
        ncols += len(cols)
    dt = time.perf_counter() - t0
    return 2.0 * flops / dt / 1e9, dt, ncols, oracle.num_threads()


def synth_as_f64(A):
    from paper_2002_10083_gb300 import synth
    return synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=A.val.astype(np.float64))


def run_reference(args):
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    A = make_workload(args.workload, n=args.n)
    per_step = float(os.environ.get("MCL_REF_STEP_SECONDS", "6"))
    vals = []
    for i in range(args.warmup + args.steps):
        g, dt, ncols, cores = oracle_gflops(A, per_step, seed=100 + i)
        if i >= args.warmup:
            vals.append((g, dt, ncols))
    v = statistics.median([x[0] for x in vals])
    ms = statistics.median([x[1] / x[2] * A.n * 1000.0 for x in vals])  # extrapolated full step
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz,
                       "sample": f"{vals[0][2]} random columns per step (~{per_step:.0f} s of CPU work)"},
            "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"random column samples, ~{per_step:.0f} s per step"},
            "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_form(ctx, D, prm, steps, stream, torch, mcl):
    """Time `steps` mcl_expand calls; returns (ms per step, median numeric ms, stats)."""
    ms_num = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = None
    for _ in range(steps):
        out, ch = ctx.expand(D, prm)
        st = ctx.stats()
        ms_num.append(st["ms_numeric"])
        del out
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, statistics.median(ms_num), st


def time_e2e(ctx, A, prm, nnz_out, dev, steps, torch, mcl):
    """End-to-end steps through the C ABI with pinned host buffers (see run_gpu)."""
    n = A.n
    cuda = f"cuda:{dev}"
    hcp = torch.from_numpy(np.ascontiguousarray(A.colptr, np.int64)).pin_memory()
    hri = torch.from_numpy(np.ascontiguousarray(A.rowidx, np.int32)).pin_memory()
    hva = torch.from_numpy(np.ascontiguousarray(A.val, np.float32)).pin_memory()
    dcp = torch.empty_like(hcp, device=cuda)
    dri = torch.empty_like(hri, device=cuda)
    dva = torch.empty_like(hva, device=cuda)
    Dh = mcl.DeviceCSC(n, dcp, dri, dva)
    # two pinned result buffers, used alternately (the result size is fixed for a fixed input)
    cap = nnz_out + 1
    bufs = [(torch.empty(n + 1, dtype=torch.int64, pin_memory=True),
             torch.empty(cap, dtype=torch.int32, pin_memory=True),
             torch.empty(cap, dtype=torch.float32, pin_memory=True)) for _ in range(2)]
    stream = torch.cuda.current_stream(dev)
    copy_stream = torch.cuda.Stream(dev)
    in_bytes = hcp.numel() * 8 + hri.numel() * 4 + hva.numel() * 4
    out_bytes = 0
    # achieved link bandwidth, one upload and one download timed alone
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record(stream)
    dcp.copy_(hcp, non_blocking=True)
    dri.copy_(hri, non_blocking=True)
    dva.copy_(hva, non_blocking=True)
    e1.record(stream)
    out, _ = ctx.expand(Dh, prm)
    m = int(out.rowidx.numel())
    e2.record(stream)
    cp, ri, va = bufs[0]
    cp.copy_(out.colptr, non_blocking=True)
    ri[:m].copy_(out.rowidx, non_blocking=True)
    va[:m].copy_(out.val, non_blocking=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e3.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = in_bytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    d2h_gbs = ((n + 1) * 8 + 8 * m) / (e2.elapsed_time(e3) * 1e-3) / 1e9
    del out
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        dcp.copy_(hcp, non_blocking=True)
        dri.copy_(hri, non_blocking=True)
        dva.copy_(hva, non_blocking=True)
        out, _ = ctx.expand(Dh, prm)
        m = int(out.rowidx.numel())
        if m > cap:  # never for a fixed input; kept correct regardless
            copy_stream.synchronize()
            cap = m
            bufs = [(b[0], torch.empty(cap, dtype=torch.int32, pin_memory=True),
                     torch.empty(cap, dtype=torch.float32, pin_memory=True)) for b in bufs]
        ev = torch.cuda.Event()
        ev.record(stream)
        cp, ri, va = bufs[i % 2]
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev)
            cp.copy_(out.colptr, non_blocking=True)
            ri[:m].copy_(out.rowidx, non_blocking=True)
            va[:m].copy_(out.val, non_blocking=True)
        for t in (out.colptr, out.rowidx, out.val):
            t.record_stream(copy_stream)
        out_bytes = (n + 1) * 8 + m * 4 + m * 4
        del out
    copy_stream.synchronize()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000.0 / steps
    return {"ms": ms, "steps": steps, "h2d_bytes": in_bytes, "d2h_bytes": out_bytes,
            "h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs}


def run_gpu(args):
    import torch
    rank, local, world = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2002_10083_gb300 import estimator, mcl
    dev = local
    torch.cuda.set_device(dev)
    A = make_workload(args.workload, n=args.n)
    n, nnz = A.n, A.nnz
    D = mcl.DeviceCSC.from_host(A, device=f"cuda:{dev}")
    ctx = mcl.Context(dev)
    meta = estimator.install(ctx)
    # numeric-pass settings the autotuner stored for this device and workload class
    from paper_2002_10083_gb300 import autotune
    tuned = autotune.apply(ctx, autotune.load(), torch.cuda.get_device_name(dev),
                           autotune.class_of_host(A))
    if args.bucket_budget_gb:
        ctx.set_option(mcl.OPT_BUCKET_BUDGET, int(args.bucket_budget_gb * (1 << 30)))
    prm_plain = mcl.Params(**PARAMS)
    prm_learn = mcl.Params(**PARAMS, use_estimator=1)
    prm_main = prm_plain if args.form == "plain" else prm_learn
    stream = torch.cuda.current_stream()

    # warm-up (both forms)
    for _ in range(args.warmup):
        for prm in (prm_plain, prm_learn):
            out, ch = ctx.expand(D, prm)
            del out
    torch.cuda.synchronize()

    # timed region: device-resident inputs (A is ~400 MB, larger than L2)
    gpu_idx = os.environ.get("CUDA_VISIBLE_DEVICES", str(dev)).split(",")[dev if world == 1 else local]
    clk = ClockSampler(gpu_idx) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clk:
        clk.start()
        time.sleep(0.3)
    l0 = mcl.launch_count()
    ms, t_num, st = _time_form(ctx, D, prm_main, args.steps, stream, torch, mcl)
    launches = mcl.launch_count() - l0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop() if clk else None
    if dist:
        ms = max_over_ranks(ms, dist, device=f"cuda:{dev}")
    flops = int(st["flops"])
    nnz_out, nnz_b = int(st["nnz_out"]), int(st["nnz_b"])
    # the other form, same workload, for the comparison the metric asks for
    other = prm_plain if prm_main is prm_learn else prm_learn
    ms_o, t_num_o, st_o = _time_form(ctx, D, other, args.steps, stream, torch, mcl)
    # Cohen's probabilistic estimate (Section V) as the size estimate
    ctx.set_option(mcl.OPT_SIZING, mcl.SIZING_COHEN)
    out, ch = ctx.expand(D, prm_plain)
    del out
    ms_c, t_num_c, st_c = _time_form(ctx, D, prm_plain, args.steps, stream, torch, mcl)
    ctx.set_option(mcl.OPT_SIZING, mcl.SIZING_PARAMS)

    # end to end through the C ABI with host buffers (pinned): every step
    # copies A host -> device, runs the iteration and copies the resulting
    # matrix device -> host.  The device input buffers and the pinned result
    # buffers are allocated before the timed region; the result's copy runs on
    # a second stream, overlapping the next step's upload and iteration.
    e2e = None if args.no_e2e else time_e2e(ctx, A, prm_main, int(nnz_out), dev,
                                              max(1, min(args.steps, 5)), torch, mcl)

    if rank != 0:
        return 0
    gflops = job_gflops(flops, ms, world)
    in_bytes = A.colptr.nbytes + A.rowidx.nbytes + A.val.astype(np.float32).nbytes
    peak, peak_kind = _peaks()
    b_alg = 8 * nnz + 8 * flops + 8 * nnz_out + 16 * n
    achieved = b_alg / (t_num / 1000.0) / 1e9
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        g, dt, ncols, cores = oracle_gflops(A, args.cpu_seconds)
        cpu = {"value": round(g, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"{ncols} random columns of the same workload ({dt:.1f} s)"}
    main_name = "learned" if prm_main is prm_learn else "plain"
    other_name = "plain" if main_name == "learned" else "learned"

    def form_line(msv, tnum, s):
        return {"value": round(job_gflops(flops, msv, world), 2), "unit": "GFLOP/s",
                "ms_per_step": round(msv, 3), "iters_per_s": round(1000.0 / msv, 4),
                "numeric_ms": round(tnum, 3), "estimate_ms": round(s["ms_estimate"], 3),
                "estimator_misses": int(s["estimator_misses"]), "window_cuts": int(s["range_splits"])}

    line = {
        "metric": METRIC, "value": round(gflops, 2), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": nnz, "flops_per_step": flops,
                   "nnz_b": nnz_b, "nnz_out": nnz_out,
                   "form": main_name + (" (MLP sizing; one estimator trained on power-law graphs of "
                                        "100k-1M vertices and planted-partition batches, the bench "
                                        "graph held out; held-out median |log ratio| %.4f)" % (
                                            meta.get("eval_stats", {}).get("median_abs_log_ratio", -1))
                                        if main_name == "learned" else " (exact symbolic sizing)"),
                   "l2": "inputs larger than L2 (A is %.0f MB)" % (in_bytes / 1e6),
                   "tuning": tuned if tuned is not None else "library defaults",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iters_per_s": round(world * 1000.0 / ms, 3),
        main_name: form_line(ms, t_num, st),
        other_name: form_line(ms_o, t_num_o, st_o),
        "cohen": form_line(ms_c, t_num_c, st_c),
        "speedup_learned_vs_plain": round((ms_o / ms) if main_name == "learned" else (ms / ms_o), 4),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": _traffic(flops),
                     "kernel": "k_expand (numeric pass, both configurations, one step)",
                     "algorithmic_bytes": b_alg, "kernel_ms": round(t_num, 3),
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": ({"value": round(job_gflops(flops, e2e["ms"], world), 2), "unit": "GFLOP/s",
                 "h2d_bytes_per_step": e2e["h2d_bytes"], "d2h_bytes_per_step": e2e["d2h_bytes"],
                 "ms_per_step": round(e2e["ms"], 3), "steps": e2e["steps"],
                 "h2d_gbs": round(e2e["h2d_gbs"], 1), "d2h_gbs": round(e2e["d2h_gbs"], 1),
                 "vs_device_step": round(e2e["ms"] / ms, 3),
                 "how": "pinned host buffers; H2D of A and the iteration on the launch stream, "
                        "D2H of the result on a second stream overlapping the next step"}
                if e2e else None),
        "gpu_launches": int(launches),
        "clocks": clocks,
        "stage_ms": {k: round(v, 3) for k, v in st.items() if k.startswith("ms_")},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _clocked(fn):
    """Run fn() with nvidia-smi clock sampling; returns (fn's result, clocks)."""
    clk = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clk.start()
    time.sleep(0.3)
    try:
        res = fn()
    finally:
        clocks = clk.stop()
    return res, clocks


def run_batched(args):
    """Batched MCL to convergence over independent components (each stops on
    its own chaos), or column-batched iterations of the 4M-vertex graph."""
    if args.workload == "zipf4m":
        return run_zipf4m(args)
    import torch
    from paper_2002_10083_gb300 import autotune, estimator, mcl, synth
    t0 = time.time()
    A = synth.config("batch4096", seed=0, ncomp=args.ncomp)
    offs = A.comp_offsets
    gen_s = time.time() - t0
    A32 = synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=A.val.astype(np.float32))
    D = mcl.DeviceCSC.from_host(A32)
    ctx = mcl.Context(0)
    # the estimator trained on this workload's graph family (other seeds), if there is one
    est_path = args.estimator or estimator.DEFAULT_WEIGHTS
    est_meta = estimator.install(ctx, est_path)
    tuned = autotune.apply(ctx, autotune.load(), torch.cuda.get_device_name(0),
                           args.tuning_class or autotune.class_of_host(A))
    if args.group_budget_gb:
        ctx.set_option(mcl.OPT_GROUP_BUDGET, int(args.group_budget_gb * (1 << 30)))
    torch.cuda.synchronize()
    peak, peak_kind = _peaks()

    # pinned host copies of A and of the labels for the end-to-end measurement
    host = None
    if not args.no_e2e:
        host = (torch.from_numpy(np.ascontiguousarray(A32.colptr, np.int64)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(A32.rowidx, np.int32)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(A32.val, np.float32)).pin_memory(),
                torch.empty(A.n, dtype=torch.int32).pin_memory())
    e2e = {}

    def timed_run(graph: int, batched: int, use_est: int, with_e2e: bool = False):
        ctx.set_option(mcl.OPT_GRAPH, graph)
        p = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0,
                       chaos_eps=1e-3, max_iters=args.max_iters, batched=batched,
                       use_estimator=use_est)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        if with_e2e:  # the input from pinned host memory, inside the timed region
            D.colptr.copy_(host[0], non_blocking=True)
            D.rowidx.copy_(host[1], non_blocking=True)
            D.val.copy_(host[2], non_blocking=True)
        ev[1].record()
        out = ctx.run(D, p, comp_offsets=offs, keep_final=False)
        ev[2].record()
        if with_e2e:  # the labels back to the host
            host[3].copy_(out[0], non_blocking=True)
        ev[3].record()
        torch.cuda.synchronize()
        if with_e2e:
            e2e["ms"] = ev[0].elapsed_time(ev[3])
            e2e["h2d_ms"] = ev[0].elapsed_time(ev[1])
            e2e["d2h_ms"] = ev[2].elapsed_time(ev[3])
        return out, ev[1].elapsed_time(ev[2]), ctx.stats()

    def summary(res, ms, st):
        lab_, iters_, hist_, _, nc_ = res
        sec = ms / 1000.0
        return {"seconds": round(sec, 2), "iterations": iters_,
                "iters_per_s": round(iters_ / sec, 4), "converged": not nc_,
                "gflops": round(2.0 * st["flops_run"] / sec / 1e9, 2),
                "multiply_adds": int(st["flops_run"]),
                "hbm_frac_alg": round(st["alg_bytes_run"] / sec / 1e9 / peak, 4),
                "graph_replays": int(st["graph_replays"]), "groups": int(st["groups"])}

    # learned + batched (per-component retirement, iterations after the first as
    # CUDA graph replays), the same with exact sizing, and plain: exact sizing,
    # eager, no per-component retirement (each group of components iterates until
    # the group's chaos < eps)
    wanted = args.forms.split(",")
    runs = [r for r in [("learned_batched", 1, 1, 1), ("batched_exact", 1, 1, 0), ("plain", 0, 0, 0)]
            if r[0] in wanted or r[0] == "learned_batched"]
    results, forms = {}, {}
    clocks = None
    for name, graph, batched, ue in runs:
        if name == "learned_batched":
            (res, ms, st), clocks = _clocked(
                lambda: timed_run(graph, batched, ue, with_e2e=host is not None))
        else:
            res, ms, st = timed_run(graph, batched, ue)
        results[name] = res
        forms[name] = summary(res, ms, st)
    lab = results["learned_batched"][0].cpu().numpy()
    labels_equal = {k: bool(np.array_equal(lab, results[k][0].cpu().numpy()))
                    for k in results if k != "learned_batched"}
    parity = None if args.no_check else check_batch(ctx, A32, offs, lab, results, args)
    cpu = None if args.no_cpu_baseline else batch_cpu_baseline(A32, offs, args.cpu_seconds)
    main = forms["learned_batched"]
    line = {"metric": METRIC, "workload": f"batch{len(offs) - 1}: {len(offs) - 1} planted-partition "
            "components, sizes log-uniform in [50, 50000], p_in 0.05, p_out 0.0005, weights U(0.1, 1], "
            "K 1100, theta 1e-4, p 0.9, r 2, to per-component chaos < 1e-3",
            "n": A.n, "nnz": A.nnz, "components": len(offs) - 1,
            "value": main["iters_per_s"], "unit": "MCL iters/s", "higher_is_better": True,
            "form": "learned_batched", "forms": forms,
            "speedup_learned_batched_vs_plain": (round(forms["plain"]["seconds"] / main["seconds"], 4)
                                                 if "plain" in forms else None),
            "speedup_learned_vs_exact_batched": (round(forms["batched_exact"]["seconds"] / main["seconds"], 4)
                                                 if "batched_exact" in forms else None),
            "labels_learned_equal": labels_equal,
            "e2e": None if not e2e else {
                "value": round(main["iterations"] / (e2e["ms"] / 1000.0), 4), "unit": "MCL iters/s",
                "h2d_bytes_per_step": int((A.n + 1) * 8 + A.nnz * 8),
                "d2h_bytes_per_step": int(A.n * 4), "seconds": round(e2e["ms"] / 1000.0, 2),
                "h2d_ms": round(e2e["h2d_ms"], 1), "d2h_ms": round(e2e["d2h_ms"], 1),
                "vs_device_run": round(e2e["ms"] / 1000.0 / main["seconds"], 4),
                "how": "pinned host buffers: H2D of A, the whole run, D2H of the labels"},
            "roofline": {"bound": "hbm", "achieved": round(main["hbm_frac_alg"] * peak, 1),
                         "peak": peak, "unit": "GB/s", "frac": main["hbm_frac_alg"],
                         "kernel": "whole run (algorithmic bytes of every iteration / run time)",
                         "peak_kind": peak_kind},
            "parity": parity, "cpu_baseline": cpu, "clocks": clocks,
            "generation_s": round(gen_s, 1), "group_budget_gb": args.group_budget_gb,
            "tuning": tuned if tuned is not None else "library defaults",
            "tuning_class": args.tuning_class or autotune.class_of_host(A),
            "workload_class": autotune.class_of_host(A),
            "estimator": {"weights": os.path.basename(est_path),
                          "trained_on": est_meta.get("workload"),
                          "train_seeds": est_meta.get("train_seeds")}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def check_batch(ctx, A, offs, lab, results, args):
    """Oracle parity of the batched run: clusters and iteration counts of
    sampled small components against per-component oracle runs, and the
    largest component's first iterations on sampled columns against the
    oracle fed the GPU's own input (its clusters: the batched labels equal a
    run of that component alone)."""
    import torch
    import oracle
    from paper_2002_10083_gb300 import mcl
    from tests.parity import compare_iteration
    t0 = time.time()
    oprm = oracle.Params(theta=float(np.float32(1e-4)), K=1100, p=float(np.float32(0.9)), r=2.0,
                         eps=1e-3, max_iters=args.max_iters)
    sizes = np.diff(offs)
    rng = np.random.default_rng(7)
    small = np.nonzero(sizes <= 300)[0]
    medium = np.nonzero((sizes > 300) & (sizes <= 5000))[0]
    pick = np.concatenate([rng.choice(small, min(64, len(small)), replace=False),
                           rng.choice(medium, min(8, len(medium)), replace=False)]).astype(np.int64)
    big = int(np.argmax(sizes))
    mism = []
    for c in pick:
        lo, hi = int(offs[c]), int(offs[c + 1])
        sub = oracle.submatrix(A, lo, hi)
        _, it_o, _, lab_o = oracle.run_mcl(sub, oprm)
        if not np.array_equal(lab[lo:hi] - lo, lab_o):
            mism.append(int(c))
    # the largest component alone, iteration by iteration
    lo, hi = int(offs[big]), int(offs[big + 1])
    sub = oracle.submatrix(A, lo, hi)
    Dc = mcl.DeviceCSC.from_host(sub)
    prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0)
    big_ok, big_cols = True, 0
    for it in range(3):
        Hin = Dc.to_host()
        out, _ = ctx.expand(Dc, prm)
        cols = rng.choice(hi - lo, min(200, hi - lo), replace=False).astype(np.int32)
        rep, _ = compare_iteration(Hin, out.to_host(), oprm, cols=cols, rtol=1e-5)
        big_ok = big_ok and rep.ok()
        big_cols += len(cols)
        Dc = out
    p1 = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0, chaos_eps=1e-3,
                    max_iters=args.max_iters)
    lab1, *_ = ctx.run(mcl.DeviceCSC.from_host(sub), p1, keep_final=False)
    big_same = bool(np.array_equal(lab1.cpu().numpy(), lab[lo:hi] - lo))
    torch.cuda.synchronize()
    # the largest component's clusters from the oracle's whole loop
    tb = time.time()
    _, it_big, _, lab_big = oracle.run_mcl(sub, oprm)
    big_oracle = bool(np.array_equal(lab[lo:hi] - lo, lab_big))
    big_oracle_s = time.time() - tb
    return {"sampled_components": len(pick), "sampled_max_size": int(sizes[pick].max()),
            "clusters_equal_oracle": len(pick) - len(mism), "mismatched_components": mism,
            "largest_component": {"size": int(hi - lo), "iterations_checked": 3,
                                  "columns_checked": big_cols, "values_within_1e-5": big_ok,
                                  "batched_labels_equal_alone": big_same,
                                  "clusters_equal_oracle": big_oracle,
                                  "oracle_iterations": int(it_big),
                                  "oracle_seconds": round(big_oracle_s, 1)},
            "seconds": round(time.time() - t0, 1)}


def batch_cpu_baseline(A, offs, seconds):
    """The oracle's whole loop on randomly drawn components (bounded time):
    multiply-adds per second over the components it finished."""
    import oracle
    oprm = oracle.Params(theta=float(np.float32(1e-4)), K=1100, p=float(np.float32(0.9)), r=2.0,
                         eps=1e-3, max_iters=30)
    rng = np.random.default_rng(11)
    sizes = np.diff(offs)
    order = rng.permutation(np.nonzero(sizes <= 2000)[0])
    flops, comps, vert = 0, 0, 0
    t0 = time.perf_counter()
    for c in order:
        if time.perf_counter() - t0 > seconds:
            break
        sub = oracle.submatrix(A, int(offs[c]), int(offs[c + 1]))
        M = sub
        for _ in range(oprm.max_iters):
            M, ch, res = oracle.expand(M, oprm)
            flops += int(res.flops.sum())
            if ch < oprm.eps:
                break
        comps += 1
        vert += sub.n
    dt = time.perf_counter() - t0
    return {"value": round(2.0 * flops / dt / 1e9, 4), "unit": "GFLOP/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{comps} whole components of <= 2000 vertices "
            f"({vert} vertices) run to convergence, {dt:.1f} s"}


def run_zipf4m(args):
    """The 4M-vertex power-law graph: MCL iterations through mcl_expand with
    learned sizing and column batches under the staging budget (180 GB), each
    timed with CUDA events."""
    import torch
    from paper_2002_10083_gb300 import autotune, estimator, mcl
    t0 = time.time()
    A = make_workload("zipf4m", n=args.n)
    gen_s = time.time() - t0
    D = mcl.DeviceCSC.from_host(A)
    ctx = mcl.Context(0)
    est_meta = estimator.install(ctx, args.estimator or estimator.DEFAULT_WEIGHTS)
    tuned = autotune.apply(ctx, autotune.load(), torch.cuda.get_device_name(0),
                           args.tuning_class or autotune.class_of_host(A))
    budget = args.phase_budget_gb or 180.0
    ctx.set_option(mcl.OPT_PHASE_BUDGET, int(budget * (1 << 30)))
    peak, peak_kind = _peaks()
    prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0, use_estimator=1)
    iters = []

    def loop():
        Dc = D
        for it in range(1, args.max_iters + 1):
            ctx.set_option(mcl.OPT_ITERATION, it)
            nin = Dc.nnz
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out, ch = ctx.expand(Dc, prm)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st = ctx.stats()
            b_alg = 8 * nin + 8 * st["flops"] + 8 * st["nnz_out"] + 16 * A.n
            iters.append({"iteration": it, "ms": round(ms, 1), "multiply_adds": int(st["flops"]),
                          "nnz_in": int(nin), "nnz_out": int(st["nnz_out"]),
                          "gflops": round(2.0 * st["flops"] / (ms / 1000.0) / 1e9, 2),
                          "numeric_ms": round(st["ms_numeric"], 1), "phases": int(st["phases"]),
                          "hbm_frac_alg_numeric": round(b_alg / (st["ms_numeric"] / 1000.0) / 1e9 / peak, 4),
                          "estimator_misses": int(st["estimator_misses"]), "chaos": round(ch, 6)})
            if Dc is not D:
                del Dc
            Dc = out
        return Dc

    _, clocks = _clocked(loop)
    tot_ms = sum(x["ms"] for x in iters)
    tot_f = sum(x["multiply_adds"] for x in iters)
    line = {"metric": METRIC, "workload": "zipf4m: 4M-vertex Zipf(2) power-law graph, mean degree ~120 "
            "capped at 5,000, lognormal(0,1) weights; learned sizing, column batches under a "
            f"{budget:.0f} GB staging budget, K 1100, theta 1e-4, p 0.9, r 2",
            "n": A.n, "nnz": A.nnz, "iterations": len(iters),
            "value": round(len(iters) / (tot_ms / 1000.0), 4), "unit": "MCL iters/s",
            "gflops": round(2.0 * tot_f / (tot_ms / 1000.0) / 1e9, 2),
            "seconds": round(tot_ms / 1000.0, 2), "per_iteration": iters, "clocks": clocks,
            "generation_s": round(gen_s, 1), "phase_budget_gb": budget,
            "tuning": tuned if tuned is not None else "library defaults",
            "tuning_class": args.tuning_class or autotune.class_of_host(A),
            "estimator": {"trained_on": est_meta.get("workload"), "train_seeds": est_meta.get("train_seeds")}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_planted(args):
    """The 2,000-vertex planted partition to convergence (K 100): GPU time of
    mcl_run, and as cpu_baseline the FP64 oracle's whole loop on the host cores."""
    import torch
    from paper_2002_10083_gb300 import mcl, synth
    A = synth.config("planted2k", seed=0)
    A32 = synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=A.val.astype(np.float32))
    D = mcl.DeviceCSC.from_host(A32)
    ctx = mcl.Context(0)
    prm = mcl.Params(threshold=1e-4, select_k=100, recover_pct=0.9, inflation=2.0,
                     chaos_eps=1e-3, max_iters=30)
    for _ in range(max(args.warmup, 1)):
        ctx.run(D, prm, keep_final=False)
    torch.cuda.synchronize()
    reps = max(args.steps, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        lab, iters, hist, _, nc = ctx.run(D, prm, keep_final=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oprm = oracle.Params(theta=float(np.float32(1e-4)), K=100, p=float(np.float32(0.9)),
                             r=2.0, eps=1e-3, max_iters=30)
        Ad = synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx,
                       val=A.val.astype(np.float32).astype(np.float64))
        t0 = time.perf_counter()
        _, o_iters, _, o_lab = oracle.run_mcl(Ad, oprm)
        dt = time.perf_counter() - t0
        cpu = {"value": round(o_iters / dt, 4), "unit": "MCL iters/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"the whole run ({o_iters} iterations, {dt:.2f} s)"}
    line = {"metric": METRIC, "workload": "planted2k: 20 clusters x 100 vertices, p_in 0.1, "
            "p_out 0.001, K 100, theta 1e-4, p 0.9, r 2, to chaos < 1e-3",
            "n": A.n, "nnz": A.nnz, "iterations": iters, "converged": not nc,
            "ms_per_run": round(ms, 3), "iters_per_s": round(iters / (ms / 1000.0), 2),
            "clusters": int(len(np.unique(lab.cpu().numpy()))), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_split(args):
    """One MCL iteration of the power-law graph through mcl_expand and through
    the split expansion with the binary merge (Section IV, Algorithm 2): time,
    equality, and the merge's memory against a multiway merge's."""
    import torch
    from paper_2002_10083_gb300 import mcl
    n = args.n or 100_000
    A = make_workload("zipf1m", n=n)
    D = mcl.DeviceCSC.from_host(A)
    ctx = mcl.Context(0)
    prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0)

    def timed(fn):
        fn()  # warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    (ref, _), ms_ref = timed(lambda: ctx.expand(D, prm))
    flops = int(ctx.stats()["flops"])
    rows = []
    for ns in (4, 8, 16):
        (out, _, st), ms = timed(lambda: ctx.expand_split(D, prm, ns))
        same = (torch.equal(out.colptr, ref.colptr) and torch.equal(out.rowidx, ref.rowidx)
                and torch.equal(out.val.view(torch.int32), ref.val.view(torch.int32)))
        rows.append({"stages": ns, "ms": round(ms, 1), "equal_to_one_pass": bool(same),
                     "merges": st["merges"], "multiway_entries": st["partial_entries"],
                     "binary_peak_entries": st["binary_peak_entries"],
                     "binary_saving": round(1.0 - st["binary_peak_entries"] / max(1, st["partial_entries"]), 4),
                     "live_peak_entries": st["live_peak_entries"],
                     "merged_entries": st["merged_entries"]})
        del out
    line = {"metric": "split expansion with binary merge vs one pass", "workload":
            f"zipf1m graph family at n={n}: one MCL iteration (K 1100, theta 1e-4, p 0.9, r 2)",
            "n": A.n, "nnz": A.nnz, "multiply_adds": flops, "one_pass_ms": round(ms_ref, 1),
            "bytes_per_entry": 12, "stages": rows}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="zipf1m")
    ap.add_argument("--form", default="learned", choices=["learned", "plain"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="override the vertex count (profiling cases)")
    ap.add_argument("--ncomp", type=int, default=4096, help="components of batch4096")
    ap.add_argument("--max-iters", type=int, default=30)
    ap.add_argument("--estimator", default=None, help="estimator weights (.npz) for the batched runs")
    ap.add_argument("--phase-budget-gb", type=float, default=0.0,
                    help="column-batch staging budget for zipf4m (0: 180 GB)")
    ap.add_argument("--group-budget-gb", type=float, default=150.0,
                    help="device bytes per group of components for batch4096 (0: one group)")
    ap.add_argument("--no-check", action="store_true", help="skip the batch4096 oracle checks")
    ap.add_argument("--tuning-class", default=None,
                    help="batch4096: apply the autotuner's setting stored for this workload class "
                         "(e.g. one tuned on a smaller batch of the same family)")
    ap.add_argument("--forms", default="learned_batched,batched_exact,plain",
                    help="batch4096 forms to time (learned_batched always runs)")
    ap.add_argument("--bucket-budget-gb", type=float, default=0.0,
                    help="device memory of the numeric pass's product buckets (0: library default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch4096", "zipf4m"):
        return run_batched(args)
    if args.workload == "planted2k":
        return run_planted(args)
    if args.workload == "zipf_split":
        return run_split(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
