"""Write the oracle's solution of a large instance to a compressed golden file.

Calls only the CPU oracle (``oracle``) and the seeded input generator; nothing here
runs or reads the GPU library.  The oracle runs Algorithm 1 (literal inner loop, FP64)
on all host threads to a step max|p^k - p^{k-1}| <= --eps, then the birth-death step
of the Remark (infinite buffer) or Eq. (10) / Proposition 2 and the performance
measures, and stores:

  * p(n) (layer marginals), the queued mass, rho_i, R (J x N), W (N x J), the
    throughput and the oracle's own relative balance residual;
  * P{B} at every state of layers 1, 2, N-2 and N-1 and at `--samples` further states
    drawn from the counter-based stream of ``instances.Stream(seed, 77)`` (the test
    draws the same indices).

Usage (one-off, minutes on a many-core host):
    python tests/golden/make_large_golden.py --workload n24 --out tests/golden/inf_n24_j1000_s3001.npz
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_03019_gb300 import instances as I  # noqa: E402

WORKLOADS = {
    "n24": lambda: I.large_infinite_n24(3001),
    "n22": lambda: I.large_infinite_n24(3001, N=22),
}


def sample_states(N: int, count: int, seed: int) -> np.ndarray:
    """Every state of layers 1, 2, N-2, N-1, then `count` states from the splitmix64
    stream (seed, 77), as sorted unique y-order indices."""
    y = np.arange(1 << N, dtype=np.int64)
    pc = np.zeros(1 << N, dtype=np.int8)
    for u in range(N):
        pc += ((y >> u) & 1).astype(np.int8)
    edge = y[np.isin(pc, [1, 2, N - 2, N - 1])]
    rnd = I.Stream(seed, 77).integers(count, 0, (1 << N) - 1)
    return np.unique(np.concatenate([edge, rnd])).astype(np.int64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="n24", choices=sorted(WORKLOADS))
    ap.add_argument("--eps", type=float, default=1e-15)
    ap.add_argument("--samples", type=int, default=100_000)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    inst = WORKLOADS[args.workload]()
    t0 = time.time()
    o = oracle.Oracle(inst, threads=args.threads)
    o.build_table()
    t_table = time.time() - t0
    print(f"table {t_table:.1f} s", flush=True)
    o.init()
    steps = []
    t1 = time.time()
    k = 0
    while True:
        step, _ = o.sweep()
        steps.append(step)
        k += 1
        if k % 25 == 0:
            print(f"sweep {k} step {step:.3e} ({time.time() - t1:.0f} s)", flush=True)
        if step <= args.eps or k >= 20000:
            break
    t_iter = time.time() - t1
    res = o.results(with_R=True, with_residual=True)
    o.close()
    ys = sample_states(inst.N, args.samples, 3001)
    np.savez_compressed(
        args.out, name=inst.name, N=inst.N, J=inst.J, mode=inst.mode, eps=args.eps,
        sweeps=k, steps=np.array(steps), seconds_table=t_table, seconds_iter=t_iter,
        threads=oracle.max_threads() if args.threads == 0 else args.threads,
        y=ys.astype(np.uint32), P=res["P"][ys], pn=res["pn"], queue_tail=res["queue_tail"],
        rho=res["rho"], R=res["R"], W=res["W"], throughput=res["throughput"],
        residual=res["residual"])
    print(f"{inst.name}: {k} sweeps to step {steps[-1]:.2e} in {t_iter:.0f} s, residual "
          f"{res['residual']:.2e}, {len(ys)} sampled states -> {args.out}", flush=True)


if __name__ == "__main__":
    main()
