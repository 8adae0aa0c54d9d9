"""Autotuner of the fused numeric pass.

The numeric pass has three run-time knobs (context options of the C ABI):

* ``table`` (MCL_OPT_TABLE): the shape of the large configuration, threads x
  table slots x CTAs per SM: 0 = 256 x 2048 x 4, 1 = 512 x 4096 x 2,
  2 = 256 x 4096 x 2;
* ``plan`` (MCL_OPT_PLAN): entries a hashed window of that table is planned
  for (0 = half the table);
* ``small_max`` (MCL_OPT_SMALL_MAX): columns whose size estimate is at most
  this use the small configuration (128 threads, 1024 slots).

``tune`` times ``mcl_expand`` on the GPU for candidate settings (coordinate
descent: table shape, then plan, then the small bound), keeps only settings
whose result is bit-identical to the default one (the numeric pass sums in
exact fixed point, so no setting may change a single bit), and returns the
fastest.  Winners are stored in a JSON table keyed by device name and
workload class; ``apply`` looks a workload up and sets the options.  Every
timing runs through the library; this module only chooses among its
settings.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import numpy as np

OPT_SMALL_MAX, OPT_TABLE, OPT_PLAN = 11, 12, 13
DEFAULTS = {"table": 0, "plan": 0, "small_max": 512}
TABLE_SLOTS = {0: 2048, 1: 4096, 2: 4096}
HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_PATH = os.path.join(HERE, "autotune_gb300.json")


def workload_class(n: int, nnz: int, max_deg: int) -> str:
    """Coarse workload key: log2 of n, of the mean degree and of the maximum degree."""
    mean = nnz / max(n, 1)
    lg = lambda x: int(math.floor(math.log2(max(x, 1.0))))  # noqa: E731
    return f"n{lg(n)}-mean{lg(mean)}-max{lg(max_deg)}"


def class_of_host(A) -> str:
    deg = np.diff(np.asarray(A.colptr))
    return workload_class(int(A.n), int(A.colptr[-1]), int(deg.max()) if len(deg) else 0)


def set_tuning(ctx, setting: dict) -> None:
    ctx.set_option(OPT_TABLE, int(setting["table"]))
    ctx.set_option(OPT_PLAN, int(setting["plan"]))
    ctx.set_option(OPT_SMALL_MAX, int(setting["small_max"]))


def candidates(stage: str, best: dict) -> list[dict]:
    """Settings one coordinate-descent stage tries around the current best."""
    out = []
    if stage == "table":
        for t in (0, 1, 2):
            out.append(dict(best, table=t, plan=0))
    elif stage == "plan":
        hs = TABLE_SLOTS[best["table"]]
        for frac in (0.25, 0.375, 0.5, 0.625):
            out.append(dict(best, plan=int(hs * frac)))
    elif stage == "small_max":
        for sm in (0, 256, 512):
            out.append(dict(best, small_max=sm))
    return out


def _same(out, ref) -> bool:
    """The result of a setting against the default one: bit-identical."""
    import torch
    return (out.n == ref.n and torch.equal(out.colptr, ref.colptr)
            and torch.equal(out.rowidx, ref.rowidx)
            and torch.equal(out.val.view(torch.int32), ref.val.view(torch.int32)))


def time_setting(ctx, D, prm, setting: dict, reps: int = 3):
    """Median numeric-pass milliseconds of `reps` expansions (after one warm-up)."""
    set_tuning(ctx, setting)
    out, _ = ctx.expand(D, prm)
    ms = []
    for _ in range(reps):
        del out
        out, _ = ctx.expand(D, prm)
        ms.append(float(ctx.stats()["ms_numeric"]))
    return statistics.median(ms), out


def tune(ctx, D, prm, reps: int = 3, stages=("table", "plan", "small_max")) -> dict:
    """Coordinate descent over the knobs; returns {"best", "best_ms", "default_ms", "trials"}."""
    best = dict(DEFAULTS)
    base_ms, ref = time_setting(ctx, D, prm, best, reps)
    best_ms = base_ms
    trials = [{"setting": dict(best), "ms": round(base_ms, 3), "same": True}]
    seen = {tuple(sorted(best.items()))}
    for stage in stages:
        for cand in candidates(stage, best):
            key = tuple(sorted(cand.items()))
            if key in seen:
                continue
            seen.add(key)
            ms, out = time_setting(ctx, D, prm, cand, reps)
            ok = _same(out, ref)
            del out
            trials.append({"setting": dict(cand), "ms": round(ms, 3), "same": ok})
            if ok and ms < best_ms:
                best, best_ms = dict(cand), ms
    set_tuning(ctx, best)
    return {"best": best, "best_ms": round(best_ms, 3), "default_ms": round(base_ms, 3),
            "trials": trials}


def load(path: str = TABLE_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(table: dict, path: str = TABLE_PATH) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def record(table: dict, device: str, wclass: str, result: dict) -> dict:
    table.setdefault(device, {})[wclass] = {"setting": result["best"], "ms": result["best_ms"],
                                            "default_ms": result["default_ms"]}
    return table


def lookup(table: dict, device: str, wclass: str):
    """The stored setting for (device, workload class), else None."""
    entry = table.get(device, {}).get(wclass)
    return None if entry is None else dict(entry["setting"])


def apply(ctx, table: dict, device: str, wclass: str):
    """Set the tuned options for this device and workload class (if any); returns them."""
    setting = lookup(table, device, wclass)
    if setting is not None:
        set_tuning(ctx, setting)
    return setting


def main(argv=None) -> int:
    """Tune a synthetic workload on cuda:0 and record the winner in the table."""
    import argparse
    import sys

    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2002_10083_gb300 import mcl, synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="zipf1m")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--ncomp", type=int, default=None)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--select-k", type=int, default=1100)
    ap.add_argument("--out", default=TABLE_PATH)
    ap.add_argument("--record-class", default=None,
                    help="record the winner under this workload class instead of the input's "
                         "(a larger member of the same graph family)")
    ap.add_argument("--from-iteration", type=int, default=1,
                    help="time the expansion of A_{k-1} (k > 1: after k - 1 default iterations)")
    args = ap.parse_args(argv)
    kw = {}
    if args.n:
        kw["n"] = args.n
    if args.ncomp:
        kw["ncomp"] = args.ncomp
    A = synth.config(args.workload, seed=0, **kw).with_val32()
    D = mcl.DeviceCSC.from_host(A)
    ctx = mcl.Context(0)
    prm = mcl.Params(threshold=1e-4, select_k=args.select_k, recover_pct=0.9, inflation=2.0)
    wc = args.record_class or class_of_host(A)  # the class of the input the run starts from
    for _ in range(args.from_iteration - 1):
        D, _ = ctx.expand(D, prm)
    res = tune(ctx, D, prm, reps=args.reps)
    res["from_iteration"] = args.from_iteration
    dev = torch.cuda.get_device_name(0)
    table = record(load(args.out), dev, wc, res)
    save(table, args.out)
    print(json.dumps({"device": dev, "class": wc, "workload": args.workload, **res}))
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
