"""Training and evaluation of the learned bound proposer (GPU).

    python -m paper_1808_05458_gb300.proposer train --out weights/proposer_rhg16_d64.bin
    python -m paper_1808_05458_gb300.proposer eval --weights ... --log2n 23 --deg 64

Training data: random hyperbolic graphs (n = 2^log2n, average degree `deg`,
exponent 5) labelled with the sides of the minimum cuts the GPU solver finds
on them.  Every step is one forward + backward + Adam update on one graph,
all in the library's CUDA kernels.  Evaluation compares, on fresh graphs, the
degree bound, the label-propagation bound and the proposer's sweep-cut bound,
and the solve time with each.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

import graphgen

from . import mincut as mc

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "proposer_rhg16_d64.bin")


def labelled(seeds, log2n, deg):
    """(graph arrays, Graph, solver side bitmap, lambda) per seed."""
    out = []
    for s in seeds:
        g = graphgen.rhg(s, 1 << log2n, float(deg))
        G = mc.Graph(*g)
        res = G.min_cut()
        out.append((g, G, np.asarray(res.bitmap, dtype=np.uint32), res.lam))
    return out


def train(args):
    data = labelled(range(args.seed0, args.seed0 + args.graphs), args.log2n, args.deg)
    held = labelled(range(10_000, 10_000 + args.held), args.log2n, args.deg)
    P = mc.Proposer(seed=args.seed0)
    log = []
    t0 = time.time()
    for ep in range(args.epochs):
        losses = [P.train_step(G, bits, args.lr) for _, G, bits, _ in data]
        hl = [P.grad(G, bits)[0] for _, G, bits, _ in held]
        log.append({"epoch": ep, "train": float(np.mean(losses)), "held": float(np.mean(hl))})
        print(json.dumps(log[-1]), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    P.save(args.out)
    print(json.dumps({"saved": args.out, "seconds": time.time() - t0,
                      "graphs": args.graphs, "epochs": args.epochs}), flush=True)


def evaluate(args):
    P = mc.Proposer.load(args.weights) if args.weights else mc.Proposer(seed=1)
    for s in range(args.seed0, args.seed0 + args.graphs):
        g = graphgen.rhg(s, 1 << args.log2n, float(args.deg))
        n, m = len(g[0]) - 1, len(g[1]) // 2
        with mc.Graph(*g) as G:
            row = {"seed": s, "n": n, "m": m}
            t = time.perf_counter()
            cut, _ = P.bound(G)
            row["proposer_bound"] = cut
            row["proposer_ms"] = (time.perf_counter() - t) * 1e3
            for name, b in (("degree", mc.MC_BOUND_DEGREE), ("lp", mc.MC_BOUND_LP),
                            ("learned", mc.MC_BOUND_LEARNED), ("best", mc.MC_BOUND_BEST)):
                G.min_cut(mc.options(bound=b, proposer=P.handle))  # warm
                t = time.perf_counter()
                r = G.min_cut(mc.options(bound=b, proposer=P.handle))
                row[f"{name}_ms"] = (time.perf_counter() - t) * 1e3
                row[f"{name}_bound"] = r.stats["bound_initial"]
                row["lambda"] = r.lam
        print(json.dumps(row), flush=True)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--graphs", type=int, default=16)
    t.add_argument("--held", type=int, default=2)
    t.add_argument("--log2n", type=int, default=16)
    t.add_argument("--deg", type=float, default=64)
    t.add_argument("--epochs", type=int, default=30)
    t.add_argument("--lr", type=float, default=3e-3)
    t.add_argument("--seed0", type=int, default=1)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--log2n", type=int, default=23)
    e.add_argument("--deg", type=float, default=64)
    e.add_argument("--graphs", type=int, default=1)
    e.add_argument("--seed0", type=int, default=1)
    args = ap.parse_args()
    if args.cmd == "train":
        train(args)
    else:
        evaluate(args)


if __name__ == "__main__":
    main()
