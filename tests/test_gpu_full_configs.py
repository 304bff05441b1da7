"""The batched and the served forms at their workloads' own sizes, against the
CPU oracle's stored results (tests/golden/expected_batch.json and
expected_serving.json, written by tests/golden/make_expected.py from the
generators and the oracle alone).

  - The batched workload: 4,096 graphs (n log-uniform in [100, 200,000],
    half Erdos-Renyi with average degree U(4, 32), half RMAT with edge
    factor 8; seed 4; 108.7 M nodes, 1.77 G entries) in one launch, with the
    default schedule and with the schedule the native autotuner picks; every
    graph's colours (SHA-256), rounds and colour count must equal the
    oracle's for that graph alone (Section II-C's loop; the schedule and the
    mode never change a colour).
  - The serving workload's graphs: the four RMAT scale-20, edge-factor-16
    graphs and the pool of 512 batch-shaped graphs (seed 5), all submitted to
    the continuous-batching server at once, so they share launches and
    device memory; every result must equal the oracle's for the graph alone.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1912_01478_gb300 import graphgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def sha(colors) -> str:
    return hashlib.sha256(np.ascontiguousarray(colors, dtype="<i4").tobytes()).hexdigest()


def batch_hash(bt) -> int:
    return graphgen.graph_hash(bt["rowptr_cat"], bt["col_cat"])


def check_batch(colors, st, node_off, exp):
    G = node_off.size - 1
    wrong = []
    for g in range(G):
        got = colors[node_off[g]:node_off[g + 1]]
        if (sha(got)[:16] != exp["colors_sha256_16"][g] or int(st["rounds"][g]) != exp["rounds"][g]
                or int(st["num_colors"][g]) != exp["num_colors"][g] or int(st["error"][g]) != 0):
            wrong.append(g)
    assert not wrong, f"{len(wrong)} graphs differ from the oracle, first {wrong[:10]}"


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    c = ipgc.Context(0)
    yield c
    c.close()


def test_full_batched_workload_matches_the_oracle(ctx):
    import torch

    from paper_1912_01478_gb300 import batched

    exp = load("expected_batch.json")
    bt = graphgen.batch_workload(exp["num_graphs"], seed=exp["seed"])
    assert batch_hash(bt) == exp["input_hash"], "the generator's output changed"
    no, eo = bt["node_off"], bt["edge_off"]
    assert int(no[-1]) == exp["nodes"] and int(eo[-1]) == exp["entries"]
    drp = torch.from_numpy(bt["rowptr_cat"]).cuda()
    dcl = torch.from_numpy(bt["col_cat"]).cuda()
    del bt
    out = torch.empty(int(no[-1]), dtype=torch.int32, device="cuda")
    # the default schedule
    colors, st = batched.color_batched(ctx, no, eo, drp, dcl, out, batched.options())
    check_batch(colors.cpu().numpy(), st, no, exp)
    # the autotuned schedule (tuned on the first 256 graphs, then checked
    # against the starting options on the whole batch)
    out.fill_(-1)
    opts, ms = batched.autotune(ctx, no, eo, drp, dcl, out, sample_graphs=256, reps=1)
    assert ms > 0
    out.fill_(-1)
    colors, st = batched.color_batched(ctx, no, eo, drp, dcl, out, opts)
    check_batch(colors.cpu().numpy(), st, no, exp)


def test_serving_workload_graphs_match_the_oracle():
    import time

    import torch

    from paper_1912_01478_gb300 import _build, server

    _build.build()
    exp = load("expected_serving.json")
    pe = exp["pool"]
    bt = graphgen.batch(pe["num_graphs"], seed=pe["seed"], nmin=pe["nmin"], nmax=pe["nmax"])
    assert batch_hash(bt) == pe["input_hash"], "the generator's output changed"
    reqs = []  # (rowptr, col, expected sha (full or first 16), rounds, colours)
    for b in exp["rmat_s20"]:
        rp, cl = graphgen.rmat(b["scale"], b["edge_factor"], seed=b["seed"])
        assert graphgen.graph_hash(rp, cl) == b["graph_hash"]
        reqs.append((rp, cl, b["colors_sha256"], b["rounds"], b["num_colors"]))
    for g in range(pe["num_graphs"]):
        rp, cl = (np.ascontiguousarray(a) for a in graphgen.batch_graph(bt, g))
        reqs.append((rp, cl, pe["colors_sha256_16"][g], pe["rounds"][g], pe["num_colors"][g]))
    del bt
    # pinned copies, submitted by reference (as a serving front end would)
    pinned = [(torch.from_numpy(rp).pin_memory(), torch.from_numpy(cl).pin_memory())
              for rp, cl, *_ in reqs]
    srv = server.Server(0, server.options(hbm_budget=8 << 30, inflight=2, max_batch_graphs=256))
    try:
        tickets = {}
        # the RMAT scale-20 graphs first and again in the middle of the pool,
        # so they run beside small requests
        order = list(range(4)) + list(range(4, 4 + 256)) + list(range(4 + 256, len(reqs)))
        for i in order:
            prp, pcl = pinned[i]
            while True:
                try:
                    tickets[srv.submit_ref(prp.numpy(), pcl.numpy())] = i
                    break
                except Exception as e:
                    if getattr(e, "code", None) != -6:  # busy: retry
                        raise
                    time.sleep(0.001)
        done = 0
        t0 = time.time()
        wrong = []
        while done < len(tickets) and time.time() - t0 < 300:
            t = srv.next_done(timeout_s=5.0)
            if t is None:
                continue
            colors, st, _ = srv.poll(t)
            i = tickets[t]
            _, _, h, rounds, k = reqs[i]
            if sha(colors)[:len(h)] != h or st.rounds != rounds or st.num_colors != k or st.error:
                wrong.append(i)
            done += 1
        assert done == len(tickets), f"{len(tickets) - done} requests did not complete"
        assert not wrong, f"requests {wrong[:10]} differ from the oracle"
        c = srv.counters()
        assert c.completed == len(tickets) and c.status == 0
    finally:
        srv.close()
