"""Train the learned warm start on solves of the method itself (needs a CUDA GPU).

1. Data: `--train` instances at N=16, J=300 (seeded, `instances.warmstart_instance`),
   solved in batches of 256 by the batched solver (FP32 then DF64 sweeps, step
   tolerance 1e-9); each (layer n = 1..N-1, unit i) pair is one training row: its 9
   inputs (hq_mlp_features) and target logit(q_i(n)), q_i(n) = P(unit i busy | n busy)
   summed from the solved conditional vector.  `--val` further instances are held out.
2. Training: the library's own forward / backward kernels and Adam step
   (hq_mlp_train_step), mini-batches of 8192 rows, cosine-decayed learning rate.
3. Output: the flat FP32 weights (`--out`, raw little-endian float32, the parameter
   order of include/hq.h) and a JSON summary beside it (losses, data sizes, seeds).

    python -m paper_2603_03019_gb300.train_warmstart --out path/warmstart_mlp_h256.f32
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import hq
from . import instances as I

N_TRAIN, J_TRAIN = 16, 300
SEED_TRAIN, SEED_VAL = 50_000, 90_000


def solve_rows(seeds, batch=256, N=N_TRAIN, J=J_TRAIN, stream=None):
    """(inputs, logit q) rows of the instances `seeds`, solved in batches."""
    import torch

    dev = torch.device("cuda", 0)
    S = 1 << N
    states = torch.arange(S, device=dev)
    bits = ((states[:, None] >> torch.arange(N, device=dev)[None, :]) & 1).double()  # S x N
    layer = torch.nn.functional.one_hot(bits.sum(1).long(), N + 1).double()  # S x (N+1)
    cond = torch.empty(S, dtype=torch.float64, device=dev)
    X, T = [], []
    solvers = [hq.Solver(N, J, I.LOSS, 0, stream=stream) for _ in range(min(batch, len(seeds)))]
    o = hq.hq_default_opts()
    o.tol = 1e-9
    o.tol_kind = hq.HQ_TOL_STEP
    o.precision = hq.HQ_PREC_FP32_DF64
    o.check_every = 8
    for c0 in range(0, len(seeds), batch):
        chunk = seeds[c0:c0 + batch]
        insts = [I.warmstart_instance(s, N=N, J=J) for s in chunk]
        for s, inst in zip(solvers, insts):
            s.load(inst.lam_j, inst.nu, inst.pref)
        b = hq.hq_batch_create([s.h for s in solvers[:len(insts)]], stream=stream)
        rc, stats, _ = hq.hq_batch_solve(b, len(insts), o)
        hq.hq_batch_destroy(b)
        for s, st in zip(solvers, stats):
            if not st["converged"]:
                continue
            hq.hq_get_conditional(s.h, cond)
            q = (layer.T @ (cond[:, None] * bits))[1:N].clamp(1e-6, 1 - 1e-6)  # layers 1..N-1
            X.append(hq.hq_mlp_features(s.h, N=N))
            T.append(torch.log(q / (1 - q)).reshape(-1).float().cpu().numpy())
    for s in solvers:
        s.close()
    torch.cuda.synchronize()
    return np.concatenate(X), np.concatenate(T)


def train(X, T, Xv, Tv, hidden=256, epochs=8, batch=8192, lr=2e-3, seed=7):
    import torch

    dev = torch.device("cuda", 0)
    m = hq.hq_mlp_create(hidden, seed)
    Xd = torch.tensor(X, device=dev)
    Td = torch.tensor(T, device=dev)
    Xvd = torch.tensor(Xv, device=dev)
    Tvd = torch.tensor(Tv, device=dev)
    yv = torch.empty(len(Tv), device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * math.ceil(len(T) / batch)
    k = 0
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(len(T), generator=g).to(dev)
        ep_loss = []
        for b0 in range(0, len(T) - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = Xd[idx].contiguous()
            tb = Td[idx].contiguous()
            a = lr * 0.5 * (1 + math.cos(math.pi * k / steps))
            ep_loss.append(hq.hq_mlp_train_step(m, xb, tb, max(a, lr * 1e-3), want_loss=True))
            k += 1
        hq.hq_mlp_forward(m, Xvd, yv)
        val = float(torch.mean((yv - Tvd) ** 2))
        hist.append({"epoch": ep, "train_mse": float(np.mean(ep_loss)), "val_mse": val})
    w = hq.hq_mlp_get_weights(m)
    hq.hq_mlp_destroy(m)
    return w, hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train", type=int, default=20_000)
    ap.add_argument("--val", type=int, default=1_000)
    ap.add_argument("--hidden", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=8)
    args = ap.parse_args()
    import torch

    hq.load()
    stream = torch.cuda.Stream()
    t0 = time.time()
    X, T = solve_rows(list(range(SEED_TRAIN, SEED_TRAIN + args.train)), stream=stream)
    Xv, Tv = solve_rows(list(range(SEED_VAL, SEED_VAL + args.val)), stream=stream)
    t1 = time.time()
    w, hist = train(X, T, Xv, Tv, hidden=args.hidden, epochs=args.epochs)
    t2 = time.time()
    w.astype("<f4").tofile(args.out)
    meta = {"hidden": args.hidden, "features": 9, "params": int(w.size), "N": N_TRAIN, "J": J_TRAIN,
            "train_instances": args.train, "train_rows": int(len(T)), "val_instances": args.val,
            "val_rows": int(len(Tv)), "seeds": {"train": SEED_TRAIN, "val": SEED_VAL},
            "solve_seconds": round(t1 - t0, 2), "train_seconds": round(t2 - t1, 2),
            "target": "logit(q_i(n)), one row per (layer n, unit i)", "history": hist,
            "baseline_val_mse_predict_mean": float(np.mean((Tv - T.mean()) ** 2))}
    with open(args.out + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps({k: v for k, v in meta.items() if k != "history"} | {"final": hist[-1]}))


if __name__ == "__main__":
    main()
