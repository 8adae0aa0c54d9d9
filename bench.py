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

    # end to end through the C ABI with host buffers (pinned): H2D of A,
    # the iteration, D2H of the resulting matrix
    hcp = torch.from_numpy(A.colptr).pin_memory()
    hri = torch.from_numpy(A.rowidx).pin_memory()
    hva = torch.from_numpy(A.val.astype(np.float32)).pin_memory()
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 3))
    out_bytes = 0
    # pinned host buffers for the result, allocated once outside the timed
    # region (the result's size is the same every step: the timed steps above)
    cap_out = int(nnz_out) + 1
    ocp = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
    ori = torch.empty(cap_out, dtype=torch.int32, pin_memory=True) if e2e_steps else None
    ova = torch.empty(cap_out, dtype=torch.float32, pin_memory=True) if e2e_steps else None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Dh = mcl.DeviceCSC(n, hcp.to(f"cuda:{dev}", non_blocking=True),
                           hri.to(f"cuda:{dev}", non_blocking=True),
                           hva.to(f"cuda:{dev}", non_blocking=True))
        out, ch = ctx.expand(Dh, prm_main)
        m = int(out.rowidx.numel())
        if m > cap_out:  # never for a fixed input; kept correct regardless
            ori = torch.empty(m, dtype=torch.int32, pin_memory=True)
            ova = torch.empty(m, dtype=torch.float32, pin_memory=True)
            cap_out = m
        ocp.copy_(out.colptr, non_blocking=True)
        ori[:m].copy_(out.rowidx, non_blocking=True)
        ova[:m].copy_(out.val, non_blocking=True)
        torch.cuda.synchronize()
        out_bytes = (n + 1) * 8 + m * 4 + m * 4
        del out, Dh
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / max(e2e_steps, 1)
    in_bytes = hcp.numel() * 8 + hri.numel() * 4 + hva.numel() * 4

    if rank != 0:
        return 0
    gflops = job_gflops(flops, ms, world)
    e2e_gflops = job_gflops(flops, e2e_ms, world) if e2e_steps else None
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
                   "form": main_name + (" (MLP sizing; estimator trained on seeds %s, held-out "
                                        "median |log ratio| %.4f)" % (
                                            "1-20", meta.get("eval", {}).get("median_abs_log_ratio", -1))
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
        "e2e": ({"value": round(e2e_gflops, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": in_bytes,
                 "d2h_bytes_per_step": out_bytes, "ms_per_step": round(e2e_ms, 3)}
                if e2e_steps else None),
        "gpu_launches": int(launches),
        "clocks": clocks,
        "stage_ms": {k: round(v, 3) for k, v in st.items() if k.startswith("ms_")},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched MCL to convergence over independent components (each stops on
    its own chaos), or column-batched iterations of the 4M-vertex graph."""
    import torch
    from paper_2002_10083_gb300 import estimator, mcl, synth
    t0 = time.time()
    if args.workload == "batch4096":
        A = synth.config("batch4096", seed=0, ncomp=args.ncomp)
        offs = A.comp_offsets
        prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0,
                         chaos_eps=1e-3, max_iters=args.max_iters, batched=1,
                         use_estimator=0)
    else:
        A = synth.config("zipf4m", seed=0, **({"n": args.n} if args.n else {}))
        offs = None
        prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, inflation=2.0,
                         chaos_eps=1e-3, max_iters=args.max_iters, use_estimator=1)
    gen_s = time.time() - t0
    D = mcl.DeviceCSC.from_host(synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx,
                                          val=A.val.astype(np.float32)))
    ctx = mcl.Context(0)
    # the estimator trained on this workload's graph family (other seeds), if there is one
    est_path = args.estimator or (estimator.BATCH_WEIGHTS if args.workload == "batch4096" and
                                  os.path.exists(estimator.BATCH_WEIGHTS)
                                  else estimator.DEFAULT_WEIGHTS)
    est_meta = estimator.install(ctx, est_path)
    from paper_2002_10083_gb300 import autotune
    tuned = autotune.apply(ctx, autotune.load(), torch.cuda.get_device_name(0),
                           autotune.class_of_host(A))
    if args.phase_budget_gb:
        ctx.set_option(mcl.OPT_PHASE_BUDGET, int(args.phase_budget_gb * (1 << 30)))
    torch.cuda.synchronize()

    def timed_run(graph: int, offsets, use_est: int):
        ctx.set_option(mcl.OPT_GRAPH, graph)
        p = mcl.Params(threshold=prm.threshold, select_k=prm.select_k,
                       recover_pct=prm.recover_pct, inflation=prm.inflation,
                       chaos_eps=prm.chaos_eps, max_iters=prm.max_iters,
                       batched=1 if offsets is not None else 0, use_estimator=use_est)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = ctx.run(D, p, comp_offsets=offsets, keep_final=False)
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1), ctx.stats()

    def summary(res, ms, st):
        lab_, iters_, hist_, _, nc_ = res
        return {"ms_total": round(ms, 1), "iterations": iters_,
                "iters_per_s": round(iters_ / (ms / 1000.0), 4), "converged": not nc_,
                "graph_replays": int(st["graph_replays"])}

    forms = {}
    if offs is not None:
        # plain: the whole block-diagonal matrix until its global chaos < eps,
        # exact sizing, eager loop; batched: per-component retirement with
        # iterations after the first replayed as CUDA graphs (exact sizing),
        # then eager, then with the learned sizing
        runs = [("plain", 0, None, 0), ("batched", 1, offs, 0), ("batched_eager", 0, offs, 0),
                ("learned_batched", 1, offs, 1)]
    else:
        runs = [("learned", 1, None, prm.use_estimator)]
    results = {}
    for name, graph, o, ue in runs:
        res, ms, st = timed_run(graph, o, ue)
        results[name] = (res, ms, st)
        forms[name] = summary(res, ms, st)
    main_name = "learned_batched" if offs is not None else "learned"
    (lab, iters, hist, final, notconv), ms, st = results[main_name]
    labels_equal = {k: bool(torch.equal(v[0][0], lab)) for k, v in results.items()}
    line = {"metric": METRIC, "workload": args.workload, "n": A.n, "nnz": A.nnz,
            "components": None if offs is None else len(offs) - 1,
            "form": main_name, "iterations": iters, "converged": not notconv,
            "ms_total": round(ms, 1), "iters_per_s": round(iters / (ms / 1000.0), 4),
            "chaos_history": [round(h, 6) for h in hist],
            "clusters": int(len(np.unique(lab.cpu().numpy()))),
            "last_iteration": {k: st[k] for k in ("flops", "nnz_b", "nnz_out", "phases",
                                                  "estimator_misses")},
            "forms": forms, "labels_equal_to_main": labels_equal,
            "generation_s": round(gen_s, 1), "phase_budget_gb": args.phase_budget_gb,
            "tuning": tuned if tuned is not None else "library defaults",
            "estimator": {"weights": os.path.basename(est_path),
                          "trained_on": est_meta.get("workload"),
                          "train_seeds": est_meta.get("train_seeds")}}
    print(json.dumps(line), flush=True)
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
                    help="column-batch staging budget for zipf4m (0: one batch)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch4096", "zipf4m"):
        return run_batched(args)
    if args.workload == "planted2k":
        return run_planted(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
