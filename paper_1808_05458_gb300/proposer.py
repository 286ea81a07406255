"""Training and evaluation of the learned bound proposer (GPU).

    python -m paper_1808_05458_gb300.proposer train --out weights/proposer_prhg16_d64.bin
    python -m paper_1808_05458_gb300.proposer eval --weights ... --log2n 16

The network runs inside mc_min_cut on one level of label-propagation
clusters, so it is trained on those cluster graphs.  Training data: planted-
cut random hyperbolic graphs (two RHG blocks of 2^log2n points, average
degree `deg`, exponent 5, joined by a few random unit edges, so that the
minimum cut lies below the minimum degree and splits the graph in two large
sides), each coarsened by mc_graph_coarsen and labelled with the side of the
minimum cut the solver finds (a cluster takes the side of most of its
vertices).  Every step is one forward + backward + Adam update on one graph,
all in the library's CUDA kernels.  Evaluation compares, on held-out graphs,
the degree bound, the label-propagation bound and the proposer's bound with
trained and untrained weights: the bound each reaches, the rounds and the
solve time.
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
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "proposer_prhg16_d64.bin")
CROSS = (4, 6, 8, 10, 12)


def planted_graph(seed, log2n, deg):
    """The training family: two RHG blocks joined by CROSS[seed % 5] edges."""
    return graphgen.planted_rhg(seed, 1 << log2n, float(deg), cross=CROSS[seed % len(CROSS)])


def to_bits(side):
    b = np.packbits(np.asarray(side, dtype=np.uint8), bitorder="little")
    b = np.concatenate([b, np.zeros((-len(b)) % 4, np.uint8)])
    return b.view(np.uint32)


def cluster_example(g, lp_iters=2):
    """(cluster Graph, cluster labels as a bitmap, lambda, delta) of graph g:
    the solver's minimum-cut side, taken per cluster by majority."""
    G = mc.Graph(*g)
    res = G.min_cut()
    side = res.side(G.n)
    C, cl = G.coarsen(lp_iters)
    votes = np.bincount(cl, weights=side, minlength=C.n)
    size = np.bincount(cl, minlength=C.n)
    lab = (2 * votes > size).astype(np.uint8)
    delta = int(G.degrees().min())
    G.close()
    return C, to_bits(lab), res.lam, delta


def train(args):
    data = [cluster_example(planted_graph(s, args.log2n, args.deg))
            for s in range(args.seed0, args.seed0 + args.graphs)]
    held = [cluster_example(planted_graph(s, args.log2n, args.deg))
            for s in range(10_000, 10_000 + args.held)]
    P = mc.Proposer(seed=args.seed0)
    t0 = time.time()
    rng = np.random.default_rng(args.seed0)
    for ep in range(args.epochs):
        losses = [P.train_step(data[i][0], data[i][1], args.lr) for i in rng.permutation(len(data))]
        hl = [P.grad(C, bits)[0] for C, bits, _, _ in held]
        hb = [P.bound(C)[0] for C, _, _, _ in held]
        print(json.dumps({"epoch": ep, "train": float(np.mean(losses)), "held": float(np.mean(hl)),
                          "held_bounds": [int(x) for x in hb],
                          "held_lambda": [int(l) for _, _, l, _ in held]}), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    P.save(args.out)
    print(json.dumps({"saved": args.out, "seconds": time.time() - t0, "graphs": args.graphs,
                      "epochs": args.epochs, "family": f"planted RHG 2x2^{args.log2n} d{args.deg}"}),
          flush=True)
    for C, _, _, _ in data + held:
        C.close()


def evaluate(args):
    import torch
    T = mc.Proposer.load(args.weights)
    U = mc.Proposer(seed=123)
    for s in range(args.seed0, args.seed0 + args.graphs):
        g = planted_graph(s, args.log2n, args.deg)
        with mc.Graph(*g) as G:
            row = {"seed": s, "n": G.n, "m": G.m, "delta": int(G.degrees().min())}
            for name, b, P in (("degree", mc.MC_BOUND_DEGREE, None), ("lp", mc.MC_BOUND_LP, None),
                               ("learned", mc.MC_BOUND_LEARNED, T), ("untrained", mc.MC_BOUND_LEARNED, U),
                               ("best", mc.MC_BOUND_BEST, T)):
                o = mc.options(bound=b, proposer=P.handle if P else None)
                G.min_cut(o)
                torch.cuda.synchronize()
                r = G.min_cut(o)
                row[name] = {"bound": r.stats["bound_initial"], "rounds": r.stats["rounds"],
                             "ms": r.stats["ms_total"], "ms_bound": r.stats["ms_bound"]}
                row["lambda"] = r.lam
        print(json.dumps(row), flush=True)
    T.close()
    U.close()


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--graphs", type=int, default=24)
    t.add_argument("--held", type=int, default=4)
    t.add_argument("--log2n", type=int, default=16)
    t.add_argument("--deg", type=float, default=64)
    t.add_argument("--epochs", type=int, default=40)
    t.add_argument("--lr", type=float, default=3e-3)
    t.add_argument("--seed0", type=int, default=1)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--log2n", type=int, default=16)
    e.add_argument("--deg", type=float, default=64)
    e.add_argument("--graphs", type=int, default=4)
    e.add_argument("--seed0", type=int, default=20_000)
    args = ap.parse_args()
    if args.cmd == "train":
        train(args)
    else:
        evaluate(args)


if __name__ == "__main__":
    main()
