"""Writes the CPU oracle's results on the paper-shaped synthetic workloads at
full size, for the GPU parity tests.

Calls only the seeded generators (inputs) and the oracle; nothing here comes
from the GPU path.

  single  -> expected_full.json: per single-graph workload (Erdos-Renyi
             n = 10,000; road 4096^2; RMAT scale 22) the input graph's FNV-1a
             hash (so a test can tell a changed input from a changed result),
             the SHA-256 of the oracle's colour array (little-endian int32),
             the round count, the colour count and |WL| and the worklist's
             degree sum at the start of every round (about two minutes);
  batch   -> expected_batch.json: the batched workload (4,096 graphs, n
             log-uniform in [100, 200,000], half Erdos-Renyi with average
             degree U(4, 32), half RMAT with edge factor 8, seed 4): the
             FNV-1a hash of the concatenated input and, per graph, the first
             16 hex digits of the SHA-256 of its oracle colours, its rounds
             and its colour count (one oracle run per graph, in worker
             processes forked before anything else runs; a few minutes);
  serving -> expected_serving.json: the serving workload's graphs: the pool
             of 512 batch-shaped graphs (seed 5) in the same per-graph form,
             and the four RMAT scale-20, edge-factor-16 graphs (seeds 500-503)
             with their full colour SHA-256, rounds and colour count.

Run: python tests/golden/make_expected.py [single|batch|serving|all]
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1912_01478_gb300 import graphgen  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS = ["er_n10000_deg8_seed1", "road_4096_seed3", "rmat_s22_ef16_seed2"]

# the serving workload's graphs (the same recipe as bench.py's serving leg)
SERVING_POOL = dict(num_graphs=512, seed=5, nmin=100, nmax=200_000)
SERVING_BIG = [(20, 16, 500 + k) for k in range(4)]


def colours_sha256(colors) -> str:
    return hashlib.sha256(np.ascontiguousarray(colors, dtype="<i4").tobytes()).hexdigest()


def batch_hash(bt) -> int:
    """FNV-1a 64 over the concatenated rowptr, then the concatenated col."""
    return graphgen.graph_hash(bt["rowptr_cat"], bt["col_cat"])


def single():
    path = os.path.join(HERE, "expected_full.json")
    out = {}
    for name in WORKLOADS:
        rp, cl = graphgen.workload(name)
        t = time.time()
        res = oracle.color(rp, cl)
        dt = time.time() - t
        out[name] = dict(
            n=int(rp.size - 1),
            nnz=int(cl.size),
            graph_hash=graphgen.graph_hash(rp, cl),
            colors_sha256=colours_sha256(res.colors),
            rounds=int(res.rounds),
            num_colors=int(res.num_colors),
            wl_sizes=[int(x) for x in res.wl_sizes],
            deg_sums=[int(x) for x in res.deg_sums],
            oracle_seconds=round(dt, 2),
        )
        print(name, out[name]["rounds"], out[name]["num_colors"], f"{dt:.1f}s", flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


# The batch being coloured, set before the worker processes are forked (they
# inherit it; nothing is copied back but the per-graph results).
_BATCH = None


def _one_graph(g):
    rp, cl = graphgen.batch_graph(_BATCH, g)
    res = oracle.color(np.ascontiguousarray(rp), np.ascontiguousarray(cl), trace=False)
    return g, colours_sha256(res.colors)[:16], int(res.rounds), int(res.num_colors)


def per_graph_results(bt, workers):
    """Oracle results of every graph of a batch, in graph order."""
    global _BATCH
    _BATCH = bt
    G = bt["node_off"].size - 1
    oracle.build()
    # largest graphs first, so the pool ends evenly
    sizes = np.diff(bt["edge_off"])
    order = [int(g) for g in np.argsort(-sizes, kind="stable")]
    res = [None] * G
    with mp.get_context("fork").Pool(workers) as pool:
        for g, h, r, k in pool.imap_unordered(_one_graph, order, chunksize=4):
            res[g] = (h, r, k)
    _BATCH = None
    return dict(
        n=[int(x) for x in np.diff(bt["node_off"])],
        nnz=[int(x) for x in sizes],
        colors_sha256_16=[x[0] for x in res],
        rounds=[x[1] for x in res],
        num_colors=[x[2] for x in res],
    )


def batch(workers):
    path = os.path.join(HERE, "expected_batch.json")
    t = time.time()
    bt = graphgen.batch_workload(4096, seed=4)
    gen_s = time.time() - t
    t = time.time()
    per = per_graph_results(bt, workers)
    out = dict(
        workload="4096 graphs, n log-uniform in [100, 200000]; even index Erdos-Renyi with average "
                 "degree U(4, 32), odd index RMAT edge factor 8 (a, b, c = 0.57, 0.19, 0.19, IDs "
                 "permuted); seed 4",
        num_graphs=4096,
        seed=4,
        nodes=int(bt["node_off"][-1]),
        entries=int(bt["edge_off"][-1]),
        input_hash=batch_hash(bt),
        **per,
    )
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"wrote {path}: generation {gen_s:.0f}s, oracle {time.time() - t:.0f}s", flush=True)


def serving(workers):
    path = os.path.join(HERE, "expected_serving.json")
    bt = graphgen.batch(**SERVING_POOL)
    pool = per_graph_results(bt, workers)
    pool.update(input_hash=batch_hash(bt), **SERVING_POOL)
    big = []
    for scale, ef, seed in SERVING_BIG:
        rp, cl = graphgen.rmat(scale, ef, seed=seed)
        t = time.time()
        res = oracle.color(rp, cl, trace=False)
        big.append(dict(scale=scale, edge_factor=ef, seed=seed, n=int(rp.size - 1),
                        nnz=int(cl.size), graph_hash=graphgen.graph_hash(rp, cl),
                        colors_sha256=colours_sha256(res.colors), rounds=int(res.rounds),
                        num_colors=int(res.num_colors), oracle_seconds=round(time.time() - t, 1)))
        print("rmat", scale, seed, big[-1]["rounds"], f"{big[-1]['oracle_seconds']}s", flush=True)
    out = dict(workload="the serving workload's graphs: 512 batch-shaped graphs (seed 5) and four "
                        "RMAT scale-20 edge-factor-16 graphs (seeds 500-503)",
               pool=pool, rmat_s20=big)
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote", path, flush=True)


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    workers = max(1, os.cpu_count() or 1)
    if what in ("single", "all"):
        single()
    if what in ("batch", "all"):
        batch(workers)
    if what in ("serving", "all"):
        serving(workers)


if __name__ == "__main__":
    main()
