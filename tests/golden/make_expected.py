"""Writes tests/golden/expected_full.json: the CPU oracle's results on the
paper-shaped synthetic workloads at full size.

Calls only the seeded generators (inputs) and the oracle; nothing here comes
from the GPU path. Stored per workload: the input graph's FNV-1a hash (so a
test can tell a changed input from a changed result), the SHA-256 of the
oracle's colour array (little-endian int32), the round count, the colour
count and |WL| at the start of every round.

Run: python tests/golden/make_expected.py   (about two minutes)
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1912_01478_gb300 import graphgen  # noqa: E402

WORKLOADS = ["er_n10000_deg8_seed1", "road_4096_seed3", "rmat_s22_ef16_seed2"]


def main():
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
            colors_sha256=hashlib.sha256(res.colors.astype("<i4").tobytes()).hexdigest(),
            rounds=int(res.rounds),
            num_colors=int(res.num_colors),
            wl_sizes=[int(x) for x in res.wl_sizes],
            deg_sums=[int(x) for x in res.deg_sums],
            oracle_seconds=round(dt, 2),
        )
        print(name, out[name]["rounds"], out[name]["num_colors"], f"{dt:.1f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expected_full.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
