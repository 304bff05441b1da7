"""The byte count bench.py reports for the paper's loop (the roofline's
algorithmic bytes), against a direct round-by-round count over the oracle's
active sets: the cumulative sums the bench uses must give the same total."""
import os
import sys

import numpy as np

import oracle
from paper_1912_01478_gb300 import graphgen

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def direct_count(rp, cl, fin, modes):
    n = rp.size - 1
    deg = np.diff(rp).astype(np.int64)
    low = np.array([int((cl[rp[v]:rp[v + 1]] < v).sum()) for v in range(n)], dtype=np.int64)
    total = 4 * (n + 1) + 4 * int((deg > 0).sum()) + 8 * n + 4 * int((fin >= 2).sum())
    for r in range(2, int(fin.max()) + 1):
        active = fin >= r
        a = int(active.sum())
        d = int(deg[active].sum())
        lo = int(low[active].sum())
        w = int((fin == r).sum())
        sweep = 4 * n if modes[r - 1] == 1 else 4 * a
        total += (12 * a + 8 * d) + (12 * a + 8 * lo + 4 * w + 4 * (a - w)) + 2 * sweep
    return total


def test_algorithmic_bytes_match_a_direct_count():
    for rp, cl in (graphgen.rmat(10, 8, seed=51), graphgen.er(2_000, 9_000, seed=52),
                   graphgen.road(40, seed=53)):
        ref = oracle.color(rp, cl, trace=True)
        n = rp.size - 1
        modes = [1] + [1 if w > int(0.6 * n) else 2 for w in ref.wl_sizes[1:]]
        fin = np.asarray(ref.fin_round, dtype=np.int32)
        got = bench.algorithmic_bytes(rp, cl, fin, modes)
        assert got == direct_count(rp, cl, fin, modes)
        # topology-driven sweeps read every node's state: never fewer bytes
        assert bench.algorithmic_bytes(rp, cl, fin, [1] * (ref.rounds + 1)) >= got
