"""Write batch_lambdas_seed1.json: the exact minimum cut of every graph of the
batched workload (graphgen.batch(1): 4096 graphs, n in 50..2000, average
degree 4..16, weights 1..100), computed by the CPU oracle's sequential NOI
and checked against Stoer-Wagner on the graphs with at most 300 vertices.

    python tests/golden/make_batch_lambdas.py

The benchmark checks every lambda of its batched form against this file."""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle  # noqa: E402


def batch_digest(b):
    """First 16 hex digits of the SHA-256 of the batch's five arrays."""
    h = hashlib.sha256()
    for a in b:
        h.update(a.tobytes())
    return h.hexdigest()[:16]


def main():
    b = graphgen.batch(1)
    G = len(b[3]) - 1
    lam = []
    for k in range(G):
        g = graphgen.batch_graph(b, k)
        x = oracle.noi(*g)[0]
        if len(g[0]) - 1 <= 300:
            assert oracle.stoer_wagner(*g)[0] == x
        lam.append(int(x))
    out = {"workload": "graphgen.batch(1)", "solver": "oracle.noi (Stoer-Wagner on n <= 300)",
           "arrays_sha256_16": batch_digest(b), "lambdas": lam}
    with open(os.path.join(HERE, "batch_lambdas_seed1.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
