"""Training and loading of the learned output-size estimator.

Training data: per-column features (mcl_features) and exact labels from
the symbolic pass (mcl_symbolic: nnz((AA)_*j), flops_j) on MCL iterations
1-3 of seeded power-law graphs; the network is trained on the GPU by the
library's own forward / backward / Adam kernels (mcl_mlp_backward,
mcl_adam_step).  Only data plumbing (batching, shuffling, the feature
standardisation statistics) happens in PyTorch / numpy.

The learned estimate sizes the numeric pass in place of the exact
symbolic SpGEMM (Sections II and V: the memory estimate made before every
iteration); the symbolic pass stays the fallback and judges the estimate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import mcl, synth

HERE = os.path.dirname(os.path.abspath(__file__))
# one network for every workload: trained on power-law graphs of 100k to 1M
# vertices (two degree laws) and on batches of planted-partition components
DEFAULT_WEIGHTS = os.path.join(HERE, "estimator_mix.npz")
# the default mixed training and held-out sets: workload, keyword arguments, seeds
TRAIN_MIX = "zipf1m:n=100000:1-3,zipf1m:n=200000:1-3,zipf1m:n=400000:1-3,zipf1m:1-6," \
            "zipf4m:n=1000000:1-2,batch4096:ncomp=64:1-3,batch4096:ncomp=256:1-4," \
            "batch4096:ncomp=1024:1-2"
EVAL_MIX = "zipf1m:n=400000:100-101,zipf1m:100-101,batch4096:ncomp=128:100-101," \
           "batch4096:ncomp=256:100-101"
NH = 64
SHAPES = [("W1", (NH, mcl.NFEATURES)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (2, NH)), ("b3", (2,))]


def init_master(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-initialised FP32 master weights in the library's flat layout."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[1]
            std = math.sqrt(2.0 / fan_in) if name != "W3" else 0.1 / math.sqrt(fan_in)
            parts.append(torch.randn(shp, generator=g) * std)
        else:
            parts.append(torch.zeros(shp))
    w = torch.cat([p.reshape(-1) for p in parts]).float()
    assert w.numel() == mcl.MLP_NPARAM
    return w.to(device)


def labels(flops: torch.Tensor, nnz: torch.Tensor) -> torch.Tensor:
    """(log(1 + nnz_j), log cf_j) with cf_j = flops_j / max(nnz_j, 1)."""
    f = flops.double()
    z = nnz.double()
    y0 = torch.log1p(z)
    y1 = torch.where(f > 0, torch.log(f / torch.clamp(z, min=1.0)), torch.zeros_like(f))
    return torch.stack([y0, y1], 1).float()


def collect(ctx: mcl.Context, A, iterations=3, sample=200_000, prm=None, seed=0):
    """Features and exact labels of MCL iterations 1..iterations of A."""
    prm = prm or mcl.Params()
    D = mcl.DeviceCSC.from_host(A)
    rng = np.random.default_rng(seed)
    X, T = [], []
    prev = None
    for it in range(1, iterations + 1):
        F = ctx.features(D, it, prev)
        fl, nz = ctx.symbolic(D)
        Y = labels(fl, nz)
        if sample and sample < D.n:
            idx = torch.from_numpy(rng.choice(D.n, sample, replace=False)).to(F.device)
            X.append(F[idx].clone())
            T.append(Y[idx].clone())
        else:
            X.append(F.clone())
            T.append(Y.clone())
        prev = Y[:, 1].contiguous()
        if it < iterations:
            D, _ = ctx.expand(D, prm)
    return torch.cat(X), torch.cat(T)


def standardisation(X: torch.Tensor) -> np.ndarray:
    x = X.double().cpu().numpy()
    mu = x.mean(0)
    sg = x.std(0)
    sg[sg < 1e-6] = 1.0
    mu[15] = 0.0  # the constant feature passes through
    sg[15] = 1.0
    return np.concatenate([mu, sg]).astype(np.float32)


def train(ctx: mcl.Context, X: torch.Tensor, T: torch.Tensor, epochs=8, batch=8192, lr=3e-3,
          seed=0, log=None):
    """Adam on the FP32 master weights with the library's kernels.
    Returns (w_bf16 device tensor, norm device tensor, loss history)."""
    dev = X.device
    norm = torch.from_numpy(standardisation(X)).to(dev)
    master = init_master(seed, dev)
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    grad = torch.zeros_like(master)
    wb = torch.zeros(mcl.MLP_NPARAM, dtype=torch.int16, device=dev)
    # an Adam step with lr = 0 and zero moments only rounds master -> BF16
    ctx.adam_step(master, m, v, grad, 1, 0.0, wb)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        loss.zero_()
        lr_ep = lr * (0.5 ** max(0, ep - epochs // 2))
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            xb = X[idx].contiguous()
            tb = T[idx].contiguous()
            grad.zero_()
            ctx.mlp_backward(xb, tb, wb, norm, 1.0 / len(idx), grad, loss)
            step += 1
            ctx.adam_step(master, m, v, grad, step, lr_ep, wb)
        torch.cuda.synchronize()
        hist.append(float(loss.item()) / n)
        if log:
            log(f"epoch {ep}: train mse {hist[-1]:.5f}")
    return wb, norm, hist


def evaluate(ctx, X, T, wb, norm):
    """Prediction quality on (X, T): mse, median |log ratio| of nnz."""
    Y = ctx.mlp_forward(X, wb, norm)
    mse = float(((Y - T) ** 2).sum(1).mean().item())
    true_nnz = torch.expm1(T[:, 0].double())
    pred_nnz = torch.expm1(Y[:, 0].double()).clamp(min=1.0)
    ratio = (true_nnz.clamp(min=1.0) / pred_nnz)
    return {"mse": mse, "median_abs_log_ratio": float(torch.log(ratio).abs().median().item()),
            "q95_ratio": float(torch.quantile(ratio.float(), 0.95).item()),
            "q99_ratio": float(torch.quantile(ratio.float(), 0.99).item())}, ratio


def save(path, wb, norm, safety, meta):
    np.savez(path, w_bf16=wb.view(torch.int16).cpu().numpy().view(np.uint16),
             norm=norm.cpu().numpy().astype(np.float32), safety=np.float32(safety),
             meta=json.dumps(meta))


def load(path=DEFAULT_WEIGHTS):
    z = np.load(path)
    meta = json.loads(str(z["meta"])) if "meta" in z else {}
    return z["w_bf16"].astype(np.uint16), z["norm"].astype(np.float32), float(z["safety"]), meta


def install(ctx: mcl.Context, path=DEFAULT_WEIGHTS, safety=None):
    w, norm, s, meta = load(path)
    ctx.estimator_load(w, norm, s if safety is None else safety)
    return meta


def _gen(args):
    name, seed, kw = args
    A = synth.config(name, seed=seed, **kw)
    return synth.CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=A.val.astype(np.float32))


def parse_mix(spec: str):
    """'workload[:key=value...]:a-b,...' -> [(workload, kwargs, seed), ...]."""
    out = []
    for item in spec.split(","):
        parts = item.strip().split(":")
        name, rest = parts[0], parts[1:]
        a, b = rest[-1].split("-")
        kw = {}
        for kv in rest[:-1]:
            k, v = kv.split("=")
            kw[k] = int(v)
        out.extend((name, kw, s) for s in range(int(a), int(b) + 1))
    return out


def main():
    ap = argparse.ArgumentParser(description="train the learned nnz estimator")
    ap.add_argument("--train", default=TRAIN_MIX, help="training graphs (see parse_mix)")
    ap.add_argument("--eval", default=EVAL_MIX, help="held-out graphs")
    ap.add_argument("--iterations", type=int, default=3)
    ap.add_argument("--sample", type=int, default=200_000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--quantile", type=float, default=0.98)
    ap.add_argument("--procs", type=int, default=8)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args()
    tr, ev = parse_mix(args.train), parse_mix(args.eval)
    t0 = time.time()
    # graphs are generated in worker processes started before any CUDA call
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(args.procs) as pool:
        graphs = pool.map(_gen, [(name, seed, kw) for name, kw, seed in tr + ev])
    print(f"generated {len(graphs)} graphs in {time.time() - t0:.0f}s", flush=True)
    ctx = mcl.Context(0)

    def gather(items, gs, seed0):
        Xs, Ts, per = [], [], []
        for i, ((name, kw, seed), A) in enumerate(zip(items, gs)):
            X, T = collect(ctx, A, args.iterations, args.sample, seed=seed0 + i)
            Xs.append(X)
            Ts.append(T)
            per.append((name, kw, seed, X.shape[0]))
        return torch.cat(Xs), torch.cat(Ts), per

    X, T, _ = gather(tr, graphs[:len(tr)], 0)
    Xe, Te, per_e = gather(ev, graphs[len(tr):], 1000)
    print(f"collected {X.shape[0]} train / {Xe.shape[0]} eval samples in {time.time() - t0:.0f}s",
          flush=True)
    wb, norm, hist = train(ctx, X, T, epochs=args.epochs, log=lambda s: print(s, flush=True))
    tr_stats, _ = evaluate(ctx, X, T, wb, norm)
    ev_stats, ratio = evaluate(ctx, Xe, Te, wb, norm)
    # held-out quality per graph family and size
    groups = {}
    at = 0
    for name, kw, seed, m in per_e:
        key = name + "".join(f":{k}={v}" for k, v in sorted(kw.items()))
        groups.setdefault(key, []).append((at, at + m))
        at += m
    per_group = {}
    for key, spans in groups.items():
        idx = torch.cat([torch.arange(a, b, device=Xe.device) for a, b in spans])
        st, _ = evaluate(ctx, Xe[idx].contiguous(), Te[idx].contiguous(), wb, norm)
        per_group[key] = st
    safety = max(1.0, float(torch.quantile(ratio.float(), args.quantile).item()))
    meta = {"workload": "mix", "train": [f"{n}:{kw}:{s}" for n, kw, s in tr],
            "eval": [f"{n}:{kw}:{s}" for n, kw, s in ev], "iterations": args.iterations,
            "samples_per_iteration": args.sample, "epochs": args.epochs, "train_stats": tr_stats,
            "eval_stats": ev_stats, "eval_by_family": per_group, "loss_history": hist,
            "safety_quantile": args.quantile, "safety": safety,
            "train_seeds": sorted({s for _, _, s in tr})}
    save(args.out, wb, norm, safety, meta)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
