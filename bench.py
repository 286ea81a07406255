#!/usr/bin/env python3
"""Benchmark of the exact minimum-cut hot path on one GB300 (or N replicas).

Workload (the plain GPU path): a threshold random hyperbolic graph with
n = 2^20 points, average degree 32, power-law exponent 5, largest connected
component, unit int32 weights (the paper's Fig. 1a instance family).  One
step = one complete mc_min_cut (Alg. 2: bound, PR tests, concurrent capped
CAPFOREST rounds, contraction, until one vertex is left) on the resident
graph; metric = input edges per second.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(sequential NOI, one core) on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s"
UNIT = "edges/s"
# Fig. 1a of the paper: NOI_lambda-BStack, 32.91 ns per edge on RHG n=2^20,
# average degree 32, exponent 5 (1 core, Xeon E5-2643 v4) -- the fastest
# variant the paper reports at this point.
PAPER_EDGES_PER_S = 1e9 / 32.91
WORKLOAD = "rhg_n2^20_deg32_gamma5_lcc_unit"
LEARNED_WEIGHTS = os.path.join(ROOT, "paper_1808_05458_gb300", "weights", "proposer_prhg16_d64.bin")


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist, device):
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(m_per_rank, world, ms_per_step):
    """Whole-job throughput: every rank solves its own replica of the
    workload (no data-path collective), so all ranks' edges count, over the
    slowest rank's step time."""
    return world * m_per_rank / (ms_per_step / 1000.0)


def make_graph(seed, log2n=20):
    import graphgen
    return graphgen.rhg(seed, 1 << log2n, 32.0, 5.0)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(kernel_name):
    """DRAM bytes per launch from the committed ncu summary, only while the
    kernel's source is unchanged since the capture (hash check)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[kernel_name]
        h = hashlib.sha256()
        for src in ent["sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        if h.hexdigest()[:16] != ent["sources_sha256_16"]:
            return None
        return ent
    except (OSError, KeyError, ValueError):
        return None


def cpu_oracle_time(g, reps=1):
    import oracle
    t = []
    lam = None
    for _ in range(reps):
        t0 = time.perf_counter()
        lam, _, _ = oracle.noi(*g)
        t.append(time.perf_counter() - t0)
    return min(t), lam


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle (sequential NOI) on the host cores."""
    if rank != 0:
        return 0
    g = make_graph(args.seed, args.rhg_log2)
    m = len(g[1]) // 2
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.noi(*g)
    times = []
    lam = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        lam, _, _ = oracle.noi(*g)
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = m / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_EDGES_PER_S,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": len(g[0]) - 1, "m": m, "lambda": lam,
                   "solver": "oracle sequential NOI, capped heap, 1 core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"full workload graph, {args.steps} solves"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def form_batched(mc, peak, seed=1):
    """The batched form (4096 graphs, n in 50..2000, degree 4..16, weights
    1..100): one mc_batch_min_cut per step through the C ABI from pinned host
    arrays (H2D of the batch, one persistent launch, D2H of the lambdas and
    side bitmaps), every lambda checked against the oracle's lambdas stored
    in tests/golden/batch_lambdas_seed1.json (written by the script beside
    it), and the plain path (mc_graph_create + mc_min_cut per graph) timed on
    every 16th graph of the same batch."""
    import graphgen
    b = graphgen.batch(seed)
    G = len(b[3]) - 1
    with open(os.path.join(ROOT, "tests", "golden", f"batch_lambdas_seed{seed}.json")) as f:
        stored = json.load(f)
    h = hashlib.sha256()
    for a in b:
        h.update(a.tobytes())
    assert h.hexdigest()[:16] == stored["arrays_sha256_16"], "batch generator output changed"
    ref = np.array(stored["lambdas"], dtype=np.int64)
    # the batch's host arrays in pinned memory, as a serving process keeps
    # its staging buffers (the timed region copies them to the device)
    import torch
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in b]
    b = tuple(t.numpy() for t in pinned)
    mc.batch_autotune(*b)
    for _ in range(2):
        lam, _, _, st = mc.batch_min_cut(*b, bitmaps=True)
    assert (lam == ref).all()
    wall, dev = [], []
    for _ in range(5):
        t0 = time.perf_counter()
        lam, _, _, st = mc.batch_min_cut(*b, bitmaps=True)
        wall.append(time.perf_counter() - t0)
        dev.append(st["ms_total"] / 1e3)
        assert (lam == ref).all()
    sample = range(0, G, 16)
    p_wall = p_dev = 0.0
    for k in sample:
        g = graphgen.batch_graph(b, k)
        t0 = time.perf_counter()
        with mc.Graph(*g) as gr:
            r = gr.min_cut()
        p_wall += time.perf_counter() - t0
        p_dev += r.stats["ms_total"] / 1e3
        assert r.lam == ref[k]
    scale = G / len(sample)
    vo, ao = b[3], b[4]
    n_tot, a_tot = int(vo[-1]), int(ao[-1])
    # algorithmic bytes of one batched solve, counted as the least the method
    # moves: the input CSR read once (4 B per row offset, 8 B per arc), one
    # full capped scan (8 B per arc, 24 B per vertex) and one contraction
    # (12 B read, 16 B written per arc)
    alg = 4 * (n_tot + G) + 8 * a_tot + (8 * a_tot + 24 * n_tot) + 28 * a_tot
    kern = min(dev)
    return {
        "workload": "batch_4096_n50-2000_deg4-16_w1-100",
        "graphs": G, "vertices": n_tot, "edges": a_tot // 2,
        "solves_per_s": G / kern, "ms_kernel": kern * 1e3,
        "e2e_solves_per_s": G / min(wall), "ms_e2e": min(wall) * 1e3,
        "h2d_bytes_per_step": int(4 * (len(b[0]) + len(b[1]) + len(b[2])) + 16 * (G + 1)),
        "plain_solves_per_s": G / (p_dev * scale), "plain_e2e_solves_per_s": G / (p_wall * scale),
        "plain_sample": f"every 16th graph ({len(sample)} graphs), scaled to {G}",
        "vs_plain": p_dev * scale / kern, "vs_plain_e2e": p_wall * scale / min(wall),
        "lambda_checked": f"all {G} equal to the oracle's stored NOI results",
        "roofline": {"bound": "hbm", "achieved": alg / kern / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / kern / 1e9 / peak, "traffic": None,
                     "note": "one warp per graph; latency-bound (dependent per-pop loads)"},
    }


def form_bounds(mc, peak, name, g, proposer):
    """Solve times of one resident graph with each initial bound: minimum
    degree (the plain path), label propagation (VieCut), the learned
    proposer, and the best of both; lambda must not change."""
    import torch
    n, m = len(g[0]) - 1, len(g[1]) // 2
    out = {"workload": name, "n": n, "m": m}
    stream = torch.cuda.current_stream()
    with mc.Graph(*g) as G:
        lam = None
        for label, b in (("degree", mc.MC_BOUND_DEGREE), ("lp", mc.MC_BOUND_LP),
                         ("learned", mc.MC_BOUND_LEARNED), ("best", mc.MC_BOUND_BEST)):
            o = mc.options(bound=b, proposer=proposer.handle, cuda_stream=stream.cuda_stream)
            G.min_cut(o)
            ms, r = [], None
            for _ in range(3):
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = G.min_cut(o)
                e.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(e))
            lam = r.lam if lam is None else lam
            assert r.lam == lam, (label, r.lam, lam)
            t = min(ms)
            out[label] = {"ms": t, "edges_per_s": m / (t / 1e3), "bound": r.stats["bound_initial"],
                          "rounds": r.stats["rounds"], "ms_bound": r.stats["ms_bound"],
                          "hbm_frac_whole_solve": r.stats["bytes_alg"] / (t / 1e3) / 1e9 / peak}
        out["lambda"] = lam
        out["delta"] = int(G.degrees().min())
    return out


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_1808_05458_gb300 as mc

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    g = make_graph(args.seed, args.rhg_log2)
    rp, col, w = g
    n = len(rp) - 1
    m = len(col) // 2
    stream = torch.cuda.current_stream()
    opts = mc.options(cuda_stream=stream.cuda_stream, seed=args.seed)
    G = mc.Graph(rp, col, w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # 256 MB > 129 MB L2

    res = None
    for _ in range(args.warmup):
        res = G.min_cut(opts)
    lam = res.lam if res is not None else None

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        res = G.min_cut(opts)
        ev[k][1].record(stream)
        stats.append(res.stats)
        lam = res.lam
    barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_value(m, world, ms_per_step)

    # end to end through the public API with host buffers: H2D of the CSR
    # from pinned host memory, canonicalise + solve on the device, D2H of
    # lambda and the side bitmap.  An unweighted graph is passed as it is
    # stored by a user, without a weight array (mc_graph_create with w NULL).
    unweighted = bool((w == 1).all())
    host = (rp, col) if unweighted else (rp, col, w)
    pinned = [torch.from_numpy(a).pin_memory().numpy() for a in host]
    e2e_steps = max(1, min(args.steps, 5))
    with mc.Graph(*pinned) as Ge:  # untimed: the allocator's first growth
        Ge.min_cut(mc.options(seed=args.seed))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with mc.Graph(*pinned) as Ge:
            r2 = Ge.min_cut(mc.options(seed=args.seed))
        assert r2.lam == lam
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, "cuda")
    h2d = sum(a.nbytes for a in host)
    d2h = 8 + 4 * ((n + 31) // 32)

    # dominant kernel: the concurrent CAPFOREST scan kernel
    scan_ms = sum(s["ms_scan_kernel"] for s in stats)
    scan_launches = sum(s["scan_launches"] for s in stats)
    scanned_arcs = sum(s["scanned_arcs"] for s in stats)
    scanned_verts = sum(s["scanned_verts"] for s in stats)
    # per scanned arc: 8 B {neighbour, weight}; per scanned vertex: 8 B row
    # offsets + 8 B degree + 4 B owner claim + 4 B visit order
    alg_bytes = scanned_arcs * 8 + scanned_verts * 24
    per_launch_bytes = alg_bytes / max(1, scan_launches)
    per_launch_s = scan_ms / max(1, scan_launches) / 1000.0
    peak, peak_kind = measured_peaks()
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    tr = kernel_traffic("k_capforest")
    roofline = {"kernel": "k_capforest (concurrent capped CAPFOREST scans)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs",
                # one capture on RHG n=2^19 round 0, scaled by algorithmic bytes
                "traffic": tr["traffic_over_alg"] * per_launch_bytes if tr else None,
                "traffic_source": "profiles/k_capforest_rhg2e19.md" if tr else None,
                "alg_bytes_per_launch": per_launch_bytes,
                "ms_per_launch": per_launch_s * 1000.0,
                "share_of_step": scan_ms / max(1e-9, total_ms)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        secs, lam_cpu = cpu_oracle_time(g)
        assert lam_cpu == lam, (lam_cpu, lam)
        cpu = {"value": m / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "oracle sequential NOI on the full workload graph, one solve"}

    s0 = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_EDGES_PER_S, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.rhg_log2 == 20 else
                   f"rhg_n2^{args.rhg_log2}_deg32_gamma5_lcc_unit", "n": n, "m": m, "lambda": lam,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "256 MB buffer written between timed steps; CSR 402 MB > L2",
                   "e2e_input": "row_ptr + col, unweighted (w NULL)" if unweighted
                                 else "row_ptr + col + w",
                   "rounds": s0["rounds"], "fallback_rounds": s0["fallback_rounds"],
                   "ms_phase": {k: s0[k] for k in ("ms_bound", "ms_pr", "ms_capforest",
                                                    "ms_contract")},
                   "vs_baseline_ref": "paper Fig.1a NOI_lambda-BStack 32.91 ns/edge, 1 core"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": world * m / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "clocks": clocks,
    }
    G.close()
    del flush
    if rank == 0 and world == 1 and not args.no_forms:
        # the metric's chosen forms beside the plain path
        import graphgen
        forms = {"batched": form_batched(mc, peak, args.seed)}
        P = mc.Proposer.load(LEARNED_WEIGHTS)
        forms["bounds"] = [
            form_bounds(mc, peak, "rhg_n2^23_deg64_gamma5_lcc_unit",
                        graphgen.rhg(args.seed, 1 << 23, 64.0), P),
            form_bounds(mc, peak, "planted_rhg_2x2^20_deg64_gamma5_cross8_unit",
                        graphgen.planted_rhg(args.seed, 1 << 20, 64.0, cross=8), P)]
        P.close()
        line["forms"] = forms
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and bound-form measurements")
    ap.add_argument("--rhg-log2", type=int, default=20,
                    help="log2 of the RHG point count (20 = the benchmark workload; smaller "
                         "sizes are for profiling captures)")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    from paper_1808_05458_gb300 import build
    build.build_library()
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
