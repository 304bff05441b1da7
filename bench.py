"""Benchmark: hybrid IPGC colouring of the RMAT scale-22 graph on GB300.

One step = one whole colouring (every round of the loop, hybrid schedule,
persistent driver) of the RMAT scale-22, edge-factor-16 graph (a, b, c, d =
0.57, 0.19, 0.19, 0.05; symmetrised, deduplicated, IDs permuted; seed 2;
4,194,304 nodes, 128,304,280 CSR entries). value = CSR entries coloured per
second of device time (edges/s), inputs resident in HBM.

Also reported:
  roofline      algorithmic bytes of one colouring (the paper's loop, which
                rescans the active nodes' rows every round) / its average
                duration (CUDA events on the launch stream around the call:
                the pushing kernel, then the rescanning kernel, which returns
                at once when the first one coloured the graph), against the
                measured HBM copy peak; per-kernel bytes and device times from
                the round trace; DRAM traffic from the committed ncu summary
                when it was taken on the current kernel sources;
  roofline_dram the DRAM bytes the kernels really move per colouring (ncu
                summary in profiles/, when taken on the current sources) over
                the same duration;
  roofline_own  the bytes the pushing kernel's own steps must move (rows read
                once at commit, bitmap words, list entries, push atomics, the
                low-degree nodes' rescans; pushing_bytes) over the duration;
  e2e           the same metric through ipgc_color_host (host buffers, the
                copies inside the timed region);
  cpu_baseline  the CPU oracle, single-threaded, on the headline graph itself
                (host core count and CPU model recorded);
  clocks        nvidia-smi samples taken during the timed region;
  validate_ms   the device CSR check of the headline graph, and default_ms a
                default ipgc_color_ex call (check included);
  road, er      the road-network workload (4096^2 grid, seed 3): edges/s and
                its roofline; the Erdos-Renyi workload (n = 10,000): edges/s;
  batched, serving, mode_rules: compact summaries of those legs (the full
                records go to --detail FILE).

--impl reference times the CPU oracle on the same metric (host cores).
With torchrun (N > 1 processes) every rank colours its own replica on its
GPU (the single-graph loop does not shard); value sums over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "rmat_s22_ef16_seed2"
WORKLOAD_DESC = (
    "RMAT scale 22, edge factor 16 (a,b,c,d=0.57,0.19,0.19,0.05), symmetrised, "
    "deduplicated, no self-loops, IDs permuted, seed 2"
)
METRIC = "IPGC edges/s"
UNIT = "edges/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="threshold")
    ap.add_argument("--driver", default="persistent")
    ap.add_argument("--forbidden", default="auto", choices=["auto", "rescan", "push"],
                    help="how assignment steps find forbidden colours (default: the library's)")
    ap.add_argument("--batch-graphs", type=int, default=4096,
                    help="graphs of the batched workload (0 = skip the batched leg)")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-rates", default="1000,2000,5000,10000,20000",
                    help="request rates of the serving leg (empty = skip)")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--plain-seconds", type=float, default=3.0,
                    help="wall-time cap of the plain comparator on each rate's stream")
    ap.add_argument("--suite", type=int, default=0,
                    help="Table III analogue on the ten stand-in graphs (slow; 1 = run)")
    ap.add_argument("--mode-rules", type=int, default=1,
                    help="compare per-round mode rules on held-out graphs (0 = skip)")
    ap.add_argument("--worklist-leg", type=int, default=1,
                    help="compare the kept and the rebuilt worklist (0 = skip)")
    ap.add_argument("--micro-n", type=int, default=50_912_018,
                    help="nodes of the Section III micro-benchmark leg (0 = skip)")
    ap.add_argument("--road", type=int, default=1, help="the road-network workload leg (0 = skip)")
    ap.add_argument("--detail", default="",
                    help="write the full records of every leg to this JSON file")
    return ap.parse_args()


def serving_leg(args, ctx, dev, stream):
    """Serving: Poisson request streams at each rate, graphs drawn from a pool
    shaped like the batched workload (512 graphs) plus RMAT scale-20 graphs
    (edge factor 16) for 1 % of the requests; seed 5. Requests go to the
    continuous-batching server by reference from pinned memory; latency =
    submission to completion. The plain path serves the same stream one
    request at a time through ipgc_color_host (copies inside each call)."""
    import torch

    from paper_1912_01478_gb300 import graphgen, ipgc, server

    rates = [int(r) for r in args.serve_rates.split(",") if r]
    if not rates:
        return None
    bt = graphgen.batch(512, seed=5, nmin=100, nmax=200_000)
    pool = [graphgen.batch_graph(bt, g) for g in range(512)]
    big = [graphgen.rmat(20, 16, seed=500 + k) for k in range(4)]
    pinned = []
    for rp, cl in pool + big:
        prp = torch.from_numpy(np.ascontiguousarray(rp)).pin_memory()
        pcl = torch.from_numpy(np.ascontiguousarray(cl)).pin_memory()
        pinned.append((prp, pcl, prp.numpy(), pcl.numpy()))
    del bt
    rng = np.random.default_rng(5)
    out_rates = []
    for rate in rates:
        N = max(1, int(rate * args.serve_seconds))
        gaps = rng.exponential(1.0 / rate, N)
        arrivals = np.cumsum(gaps) - gaps[0]
        pick = np.where(rng.uniform(size=N) < 0.01, 512 + rng.integers(0, 4, N), rng.integers(0, 512, N))
        so = server.options(hbm_budget=24 << 30, host_budget=2 << 30, inflight=2,
                            max_batch_graphs=1024)
        so.batch.base.forbidden = ipgc.FORBIDDEN[args.forbidden]
        # teams of at most 64 CTAs: a large request leaves the rest of its
        # slot to the small ones (same-GPU sweep of slots and team caps)
        so.batch.max_team = 64
        srv = server.Server(dev.index or 0, so)
        lat = []
        done_n = [0]

        def drain():
            while done_n[0] < N:
                t = srv.next_done(timeout_s=5.0)
                if t is None:
                    break
                r = srv.poll(t)
                lat.append(r[2])
                done_n[0] += 1

        import threading

        th = threading.Thread(target=drain, daemon=True)
        th.start()
        t0 = time.perf_counter()
        busy_retries = 0
        for i in range(N):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            _, _, rp, cl = pinned[pick[i]]
            while True:
                try:
                    srv.submit_ref(rp, cl)
                    break
                except Exception as e:  # queue or staging momentarily full
                    if getattr(e, "code", None) != -6:
                        raise
                    busy_retries += 1
                    time.sleep(0.0001)
        th.join(timeout=120)
        wall = time.perf_counter() - t0
        c = srv.counters()
        srv.close()
        lat_ms = np.array(lat, dtype=np.float64) / 1e6
        # the plain path (one ipgc_color_host call per request) on the same
        # stream, for at most --plain-seconds of wall time (it saturates
        # near 1 K req/s, so at high rates it serves a prefix of the stream)
        plain_lat = []
        tp0 = time.perf_counter()
        for i in range(N):
            if time.perf_counter() - tp0 > args.plain_seconds:
                break
            while time.perf_counter() - tp0 < arrivals[i]:
                pass
            _, _, rp, cl = pinned[pick[i]]
            ctx.color_host(rp, cl, options=None, stream=stream)
            plain_lat.append(time.perf_counter() - tp0 - arrivals[i])
        M = len(plain_lat)
        plain_wall = time.perf_counter() - tp0
        pl = np.array(plain_lat) * 1e3
        out_rates.append({
            "rate_rps": rate,
            "requests": N,
            "completed": int(len(lat)),
            "throughput_rps": len(lat) / wall,
            "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None,
            "batches": int(c.batches),
            "mean_batch": c.graphs_in_batches / max(int(c.batches), 1),
            "hbm_peak_gb": c.hbm_peak / 2**30,
            "busy_retries": busy_retries,
            "plain_requests": M,
            "plain_throughput_rps": M / plain_wall,
            "plain_p50_ms": float(np.percentile(pl, 50)),
            "plain_p99_ms": float(np.percentile(pl, 99)),
        })
    return {
        "workload": "Poisson arrivals per rate; graphs drawn from 512 graphs shaped like the batched "
                    "workload (seed 5) and, for 1 % of requests, 4 RMAT scale-20 edge-factor-16 graphs",
        "server": "2 slots, teams of at most 64 CTAs, 24 GiB device arena, forbidden "
                  "colours: " + ("rows rescanned" if args.forbidden == "rescan" else "bitmaps"),
        "seconds_per_rate": args.serve_seconds,
        "rates": out_rates,
    }


def worklist_leg(args, ctx, drp, dcl, stream):
    """The paper's hybrid (the worklist kept in every round) against the
    discard-and-rebuild hybrid (topology-driven rounds keep no worklist; it
    is rebuilt on the way back), both without neighbour filtering, on the
    headline graph at three thresholds H = frac * n; best of 3 colourings
    each (CUDA events)."""
    import torch

    from paper_1912_01478_gb300 import ipgc

    if not args.worklist_leg:
        return None
    nnz = dcl.numel()
    out = []
    for frac in (0.6, 0.2, 0.05):
        row = {"threshold_frac": frac}
        for wl in ("keep", "rebuild"):
            o = ipgc.ColorOptions(validate=False, filter_degree=-1, worklist=wl, threshold_frac=frac,
                                  forbidden="rescan")
            ctx.color(drp, dcl, options=o, stream=stream)
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.color(drp, dcl, options=o, stream=stream, wait=False)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            st = ctx.last_stats()
            row[wl] = {"ms": min(ts), "edges_per_s": nnz / (min(ts) / 1e3),
                       "rounds_topo": int(st.rounds_topo), "rounds_data": int(st.rounds_data)}
        row["rebuild_over_keep"] = row["rebuild"]["ms"] / row["keep"]["ms"]
        out.append(row)
    return {"workload": "the headline RMAT scale-22 graph",
            "engine": "rows rescanned every round (the paper's loop), no filtering, for both",
            "rows": out}


def suite_leg(args, ctx, stream):
    """Table III analogue: the stand-ins for the paper's ten graphs (Table I
    shapes, see graphgen.SUITE), each coloured by Plain (every round
    data-driven) and Hybrid (the paper's threshold rule), both rescanning
    rows without neighbour filtering (the paper's loop), by Hybrid with
    filtering, and by Hybrid with forbidden-colour bitmaps (this build's
    default); best of 3 colourings each (CUDA events). All colourings must be
    identical (the mode never changes a colour) and proper."""
    import torch

    from paper_1912_01478_gb300 import graphgen, ipgc

    if not args.suite:
        return None
    rows = []
    for name in graphgen.SUITE:
        t0 = time.perf_counter()
        rp, cl = graphgen.suite_graph(name)
        gen_s = time.perf_counter() - t0
        deg = np.diff(rp)
        drp = torch.from_numpy(rp).cuda()
        dcl = torch.from_numpy(cl).cuda()
        if ctx.validate(drp, dcl, stream=stream) != ipgc.IPGC_OK:
            raise SystemExit(f"{name}: generated graph failed validation")
        row = {"graph": name, "n": int(rp.size - 1), "nnz": int(cl.size),
               "deg_min_med_max": [int(deg.min()), int(np.median(deg)), int(deg.max())],
               "generation_s": gen_s}
        ref = None
        R = "rescan"
        for label, kw in (("plain", dict(mode="data", filter_degree=-1, forbidden=R)),
                          ("hybrid", dict(filter_degree=-1, forbidden=R)),
                          ("hybrid_filtered", dict(forbidden=R)),
                          ("hybrid_push", dict())):
            o = ipgc.ColorOptions(validate=False, **kw)
            colors, st = ctx.color(drp, dcl, options=o, stream=stream)
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.color(drp, dcl, colors, options=o, stream=stream, wait=False)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            h = colors.cpu().numpy()
            if ref is None:
                ref = h
                src = np.repeat(np.arange(rp.size - 1), deg)
                if np.any(h[src] == h[cl]) or h.min(initial=1) < 1:
                    raise SystemExit(f"{name}: improper colouring")
            elif not np.array_equal(ref, h):
                raise SystemExit(f"{name}: {label} coloured differently")
            row[label] = {"ms": min(ts), "rounds": int(st.rounds), "colors": int(st.num_colors),
                          "rounds_topo": int(st.rounds_topo)}
        row["hybrid_over_plain"] = row["plain"]["ms"] / row["hybrid"]["ms"]
        row["filtered_over_plain"] = row["plain"]["ms"] / row["hybrid_filtered"]["ms"]
        row["push_over_plain"] = row["plain"]["ms"] / row["hybrid_push"]["ms"]
        rows.append(row)
        del drp, dcl
        torch.cuda.empty_cache()
    geo = lambda k: float(np.exp(np.mean([np.log(r[k]) for r in rows])))
    return {"graphs": rows, "geomean_hybrid_over_plain": geo("hybrid_over_plain"),
            "geomean_filtered_over_plain": geo("filtered_over_plain"),
            "geomean_push_over_plain": geo("push_over_plain")}


def training_graphs():
    """The learned switch's training graphs: RMAT, road grids, Erdos-Renyi,
    and 2-D and 3-D random geometric graphs and a lattice (mesh-like), none of
    them a held-out graph."""
    from paper_1912_01478_gb300 import graphgen

    gs = [graphgen.rmat(a, b, seed=sd) for a, b, sd in [(15, 16, 1), (16, 8, 2), (17, 16, 3),
                                                         (18, 8, 8)]]
    gs += [graphgen.road(512, seed=4), graphgen.road(1024, seed=5),
           graphgen.er(200_000, 800_000, seed=6), graphgen.er(60_000, 960_000, seed=7)]
    gs += [graphgen.rgg(60_000, 3, 60.0, seed=9), graphgen.rgg(150_000, 3, 40.0, seed=10),
           graphgen.rgg(300_000, 2, 16.0, seed=11), graphgen.lattice3(40, 6),
           graphgen.rgg(1_000_000, 2, 16.0, seed=13), graphgen.rgg(50_000, 3, 90.0, seed=14),
           graphgen.rgg(600_000, 2, 10.0, seed=15)]
    return gs


def mode_rules_leg(args, ctx):
    """Per-round mode rules on held-out graphs (the ten suite stand-ins at 5 %
    scale), from forced-mode round times of the default colouring: the
    paper's H = 0.6 n, the byte model's H (policy.BYTES_KAPPA), a threshold
    fitted to training graphs, the learned switch trained on the same
    training graphs, and the per-round best. Totals are summed round times
    (ns -> ms). Then whole colourings of the held-out graphs under the
    threshold rule and under the learned switch (best of 3 each, CUDA events,
    same colours checked). Returns (record, trained weights)."""
    import torch

    from paper_1912_01478_gb300 import graphgen, ipgc, policy

    if not args.mode_rules:
        return None, None
    train = policy.collect(ctx, training_graphs())
    held_graphs = [graphgen.suite_graph(nm, 0.05) for nm in graphgen.SUITE]
    held = policy.collect(ctx, held_graphs)
    fit = policy.fit_threshold(train)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    w, _ = policy.train(ctx, dev(train.x), dev(train.y), dev(train.w / max(train.w.mean(), 1e-9)),
                        epochs=1500, lr=0.01)
    learned, _ = policy.decisions(w, held.x, 0.05, held.thr_topo)
    rules = {"paper_0.6": policy.threshold_choices(held, 0.6),
             "byte_model": policy.threshold_choices(held, policy.BYTES_KAPPA),
             "fitted": policy.threshold_choices(held, fit=fit),
             "learned": learned,
             "all_data": np.zeros(held.wl.size, bool)}
    out = {k: held.totals(v) / 1e6 for k, v in rules.items()}
    out["per_round_best"] = float(np.minimum(held.t_topo, held.t_data).sum() / 1e6)
    a, b, c = fit
    # whole colourings: the threshold rule against the learned switch
    policy.load(ctx, w)
    real = {"threshold": 0.0, "learned": 0.0}
    for rp, cl in held_graphs:
        drp, dcl = torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda()
        col = torch.empty(rp.size - 1, dtype=torch.int32, device="cuda")
        ref = None
        for mode in real:
            o = ipgc.ColorOptions(mode=mode, validate=False)
            ctx.color(drp, dcl, col, o)
            ts = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.color(drp, dcl, col, o, wait=False)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            real[mode] += min(ts)
            h = col.cpu().numpy()
            if ref is None:
                ref = h
            elif not np.array_equal(ref, h):
                raise SystemExit("the learned switch changed a colour")
    policy.load(ctx, None)
    return ({"held_out": "the ten suite stand-ins at 5 % scale", "rounds": int(held.wl.size),
             "total_round_ms": out, "colouring_ms": real, "byte_model_kappa": policy.BYTES_KAPPA,
             "fitted": {"a_ns_per_node": a, "b_ns_per_wl": b, "c_ns": c,
                        "H_over_n_at_1M": (a * 1e6 + c) / b / 1e6}}, w)


def micro_leg(args, ctx):
    """Section III micro-benchmark at the europe_osm size (n = 50,912,018,
    COUNT = 1000, 50,913 iterations in one launch): per-iteration time (TTI)
    of Push_NoWL (topology-driven) and Push_WL (data-driven), their crossover
    (first window of 500 iterations where Push_WL is faster on average), and
    the hybrid switching at the worklist size of the crossover. Bytes moved:
    Push_NoWL writes 4 |WL_next|; Push_WL reads 4 |WL| and writes 4 |WL_next|."""
    n, count = args.micro_n, 1000
    if n <= 0:
        return None
    out = {"workload": f"n = {n} (europe_osm's node count), COUNT = {count}", "n": n}
    tti = {}
    for mode in ("nowl", "wl"):
        ctx.push_bench(n, count, mode)  # warm-up
        it, rec = ctx.push_bench(n, count, mode)
        t = rec[:, 3].astype(np.float64)
        sizes = rec[:, 0].astype(np.float64)
        before = np.concatenate([[n], sizes[:-1]])
        moved = 4 * sizes.sum() + (4 * before.sum() if mode == "wl" else 0.0)
        tti[mode] = t
        out[mode] = {"iterations": int(it), "total_ms": t.sum() / 1e6,
                     "tti_us_first100": t[:100].mean() / 1e3, "tti_us_last100": t[-100:].mean() / 1e3,
                     "bytes_moved": moved, "gbs": moved / t.sum()}
    d = tti["wl"] - tti["nowl"]
    w = 500
    cs = np.convolve(d, np.ones(w) / w, mode="valid")
    x = int(np.argmax(cs < 0)) if (cs < 0).any() else len(d)
    switch = max(n - count * (x + 1), 0)
    it, rec = ctx.push_bench(n, count, "hybrid", switch)
    out["crossover_iteration"] = x
    out["crossover_wl"] = switch
    out["hybrid"] = {"switch_wl": switch, "total_ms": rec[:, 3].sum() / 1e6}
    out["per_iteration_best_ms"] = float(np.minimum(tti["wl"], tti["nowl"]).sum() / 1e6)
    return out


def batched_leg(args, ctx, dev, stream, policy_w=None):
    """Batched workload: G graphs (n log-uniform in [100, 200000], half
    Erdos-Renyi with average degree U(4, 32), half RMAT with edge factor 8,
    seed 4) coloured in one persistent launch with the autotuned schedule,
    against the plain path of one ipgc_color_ex launch per graph. Inputs
    resident in HBM; graphs/s = G / device time."""
    import torch

    from paper_1912_01478_gb300 import batched, graphgen, ipgc

    t0 = time.perf_counter()
    bt = graphgen.batch_workload(args.batch_graphs, seed=4)
    gen_s = time.perf_counter() - t0
    no, eo = bt["node_off"], bt["edge_off"]
    G = no.size - 1
    drp = torch.from_numpy(bt["rowptr_cat"]).to(dev)
    dcl = torch.from_numpy(bt["col_cat"]).to(dev)
    del bt
    out = torch.empty(int(no[-1]), dtype=torch.int32, device=dev)
    # schedule chosen by the native autotuner on the first 256 graphs
    sample = min(G, 256)
    opts, tune_ms = batched.autotune(ctx, no, eo, drp, dcl, out, sample_graphs=sample, reps=2,
                                     stream=stream)
    opts_default = batched.options()

    def run(o, reps):
        for _ in range(2):
            batched.color_batched(ctx, no, eo, drp, dcl, out, o, stream=stream, want_stats=False)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            batched.color_batched(ctx, no, eo, drp, dcl, out, o, stream=stream, want_stats=False)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_tuned = run(opts, args.batch_steps)
    ms_default = run(opts_default, args.batch_steps)
    _, st = batched.color_batched(ctx, no, eo, drp, dcl, out, opts, stream=stream)
    assert int(st["error"].max()) == 0
    batch_colors = out.clone()
    ms_learned = None
    if policy_w is not None:  # the same schedule, each round's mode from the learned switch
        from paper_1912_01478_gb300 import policy

        policy.load(ctx, policy_w)
        ol = batched.BatchOptions.from_buffer_copy(opts)
        ol.base.mode = ipgc.MODE_LEARNED
        ms_learned = run(ol, args.batch_steps)
        policy.load(ctx, None)
        assert torch.equal(out, batch_colors), "the learned switch changed a colour"

    # plain path: one ipgc_color_ex launch per graph, same schedule, one stream
    plain = ipgc.ColorOptions(validate=False, t1=opts.base.t1, chunk=opts.base.chunk,
                              block_size=opts.base.block_size)
    po = plain.to_c()
    L = ipgc.lib()
    base_rp, base_cl, base_out = drp.data_ptr(), dcl.data_ptr(), out.data_ptr()

    def plain_pass():
        for g in range(G):
            n = int(no[g + 1] - no[g])
            if n == 0:
                continue
            rc = L.ipgc_color_ex(ctx.handle, base_rp + 4 * (int(no[g]) + g), base_cl + 4 * int(eo[g]),
                                 n, int(eo[g + 1] - eo[g]), base_out + 4 * int(no[g]), None,
                                 ctypes.byref(po), int(stream.cuda_stream))
            assert rc == 0

    import ctypes

    plain_pass()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plain_pass()
    e1.record(stream)
    stream.synchronize()
    ms_plain = e0.elapsed_time(e1)
    assert torch.equal(out, batch_colors), "batched and plain colourings differ"
    entries = int(eo[-1])
    return {
        "workload": f"{G} graphs, n log-uniform in [100, 200000]; even index Erdos-Renyi avg degree "
                    f"U(4,32), odd index RMAT edge factor 8 (a,b,c=0.57,0.19,0.19, permuted); seed 4",
        "graphs": G,
        "nodes": int(no[-1]),
        "entries": entries,
        "graphs_per_s": G / (ms_tuned / 1e3),
        "edges_per_s": entries / (ms_tuned / 1e3),
        "ms_per_batch": ms_tuned,
        "ms_per_batch_default_schedule": ms_default,
        "plain_graphs_per_s": G / (ms_plain / 1e3),
        "plain_ms": ms_plain,
        "speedup_vs_plain": ms_plain / ms_tuned,
        "ms_learned": ms_learned,
        "learned_speedup_vs_plain": ms_plain / ms_learned if ms_learned else None,
        "autotuned": batched.describe(opts),
        "autotune_sample_graphs": sample,
        "identical_colours_batched_vs_plain": True,
        "generation_s": round(gen_s, 1),
    }


def road_leg(args, ctx, dev, stream, hbm):
    """The road-network workload: a 4096 x 4096 4-neighbour grid, 30 % of the
    edges deleted, 1 % long-range edges added (seed 3; 16.8 M nodes, 47.4 M
    entries, the long tail of small rounds). Default options (no node is
    above t1, so the rescanning kernel colours it), inputs resident; K timed
    colourings (CUDA events) after W warm-ups; roofline as for the headline
    (the paper's loop's bytes from one traced run)."""
    import torch

    from paper_1912_01478_gb300 import graphgen, ipgc

    if not args.road:
        return None
    rp, cl = graphgen.workload("road_4096_seed3")
    n, nnz = rp.size - 1, cl.size
    drp = torch.from_numpy(rp).to(dev)
    dcl = torch.from_numpy(cl).to(dev)
    colors = torch.empty(n, dtype=torch.int32, device=dev)
    opts = ipgc.ColorOptions(validate=False)
    trace = ipgc.trace_buffer(n + 2, dev.index or 0)
    fin = torch.zeros(n, dtype=torch.int32, device=dev)
    _, st = ctx.color(drp, dcl, colors, opts, stream=stream, trace=trace, fin_round=fin)
    tr = ipgc.read_trace(trace, st.rounds)
    alg = algorithmic_bytes(rp, cl, fin.cpu().numpy(), tr["mode"].tolist())
    del trace, fin
    for _ in range(args.warmup):
        ctx.color(drp, dcl, colors, opts, stream=stream, wait=False)
    stream.synchronize()
    ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.color(drp, dcl, colors, opts, stream=stream, wait=False)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    st2 = ctx.last_stats()
    assert st2.error == 0 and st2.rounds == st.rounds
    avg = float(np.mean(ms))
    gbs = alg / (avg / 1e3) / 1e9
    return {"workload": "road 4096^2, 30 % deleted, 1 % long-range, seed 3", "n": int(n),
            "nnz": int(nnz), "rounds": int(st.rounds), "colors": int(st.num_colors),
            "ms": avg, "edges_per_s": nnz / (avg / 1e3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "algorithmic_bytes_per_step": int(alg)}}


def er_leg(args, ctx, dev, stream):
    """The small Erdos-Renyi workload (n = 10,000, m = 40,000, seed 1):
    K timed colourings after W warm-ups (CUDA events), default options
    without the check."""
    import torch

    from paper_1912_01478_gb300 import graphgen, ipgc

    rp, cl = graphgen.workload("er_n10000_deg8_seed1")
    drp = torch.from_numpy(rp).to(dev)
    dcl = torch.from_numpy(cl).to(dev)
    colors = torch.empty(rp.size - 1, dtype=torch.int32, device=dev)
    o = ipgc.ColorOptions(validate=False)
    for _ in range(max(args.warmup, 3)):
        _, st = ctx.color(drp, dcl, colors, o, stream=stream)
    ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.color(drp, dcl, colors, o, stream=stream, wait=False)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    avg = float(np.mean(ms))
    return {"ms": _r(avg), "edges_per_s": _r(cl.size / (avg / 1e3)), "rounds": int(st.rounds)}


def validate_leg(ctx, drp, dcl, stream, opts_default):
    """Device CSR check of the headline graph alone, and a default
    ipgc_color_ex call (check included), CUDA events, best of 5."""
    import torch

    from paper_1912_01478_gb300 import ipgc

    def best(f):
        f()
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    colors = torch.empty(drp.numel() - 1, dtype=torch.int32, device=drp.device)
    v = best(lambda: ctx.validate(drp, dcl, stream=stream))
    d = best(lambda: ctx.color(drp, dcl, colors, opts_default, stream=stream))
    assert ctx.validate(drp, dcl, stream=stream) == ipgc.IPGC_OK
    return v, d


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) while running."""

    Q = (
        "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
            )
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (timing: the slowest rank sets the job's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed / the slowest rank's time."""
    return units_per_rank * steps * world / (max_ms / 1e3)


COLOURING_SOURCES = ("ipgc_api.cu", "ipgc_color.cu", "ipgc_device.cuh", "ipgc_internal.h",
                     "ipgc_phases.cuh")


def kernel_sources_hash():
    """sha256 over the sources the single-graph colouring kernels are built
    from and the public header (what the ncu counters in profiles/ were
    taken on)."""
    import hashlib

    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1912_01478_gb300", "csrc")
    for f in COLOURING_SOURCES:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "include", "ipgc.h"), "rb") as fh:
        h.update(b"ipgc.h\0" + fh.read())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per colouring of this workload from the ncu summary in
    profiles/ (line 'traffic_bytes_per_step: B sources: H'), or None when the
    summary was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "rmat_s22_dram_traffic.md")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_step:"):
                    parts = line.split()
                    b, h = int(parts[1]), parts[3]
                    return b if h == kernel_sources_hash() else None
    except (OSError, ValueError, IndexError):
        return None
    return None


def round_bytes(rp, cl, fin, modes):
    """Per-round algorithmic bytes (index r - 1 for round r); see algorithmic_bytes."""
    n = rp.size - 1
    deg = np.diff(rp).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    nlow = np.bincount(src[cl < src], minlength=n).astype(np.int64)
    R = int(fin.max())
    cnt_fin = np.bincount(fin, minlength=R + 2).astype(np.int64)
    deg_fin = np.bincount(fin, weights=deg, minlength=R + 2).astype(np.int64)
    low_fin = np.bincount(fin, weights=nlow, minlength=R + 2).astype(np.int64)
    A = np.cumsum(cnt_fin[::-1])[::-1]
    D = np.cumsum(deg_fin[::-1])[::-1]
    L = np.cumsum(low_fin[::-1])[::-1]
    out = [4 * (n + 1) + 4 * int((deg > 0).sum()) + 8 * n + 4 * int(A[2] if R >= 2 else 0)]
    for r in range(2, R + 1):
        a, d, l, w = int(A[r]), int(D[r]), int(L[r]), int(cnt_fin[r])
        x = a - w
        sweep = 4 * n if modes[r - 1] == 1 else 4 * a
        out.append(8 * a + 8 * d + 4 * a + 12 * a + 8 * l + 4 * w + 4 * x + 2 * sweep)
    return out


def algorithmic_bytes(rp, cl, fin, modes):
    """Bytes the method must move, summed over rounds:
    round 1 (implicit assignment): rowptr, the first neighbour of every
    non-isolated node, colour and tentative-colour writes, loser pushes;
    round r >= 2 over the active set A (D = sum deg, L = sum of lower-ID
    neighbours, W winners, X losers):
      assign  8|A| + 4D (col) + 4D (colour gathers) + 4|A| (tent write)
      detect  8|A| + 4|A| (own tent) + 4L (col) + 4L (tent gathers) + 4W + 4X
      + per phase 4|A| worklist reads (data-driven) or 4n state reads (topology)."""
    n = rp.size - 1
    deg = np.diff(rp).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    nlow = np.bincount(src[cl < src], minlength=n).astype(np.int64)
    R = int(fin.max())
    cnt_fin = np.bincount(fin, minlength=R + 2).astype(np.int64)
    deg_fin = np.bincount(fin, weights=deg, minlength=R + 2).astype(np.int64)
    low_fin = np.bincount(fin, weights=nlow, minlength=R + 2).astype(np.int64)
    # active at round r: fin >= r  -> reverse cumulative sums
    A = np.cumsum(cnt_fin[::-1])[::-1]
    D = np.cumsum(deg_fin[::-1])[::-1]
    L = np.cumsum(low_fin[::-1])[::-1]
    total = 4 * (n + 1) + 4 * int((deg > 0).sum()) + 8 * n + 4 * int(A[2] if R >= 2 else 0)
    for r in range(2, R + 1):
        a, d, l, w = int(A[r]), int(D[r]), int(L[r]), int(cnt_fin[r])
        x = a - w
        assign = 8 * a + 8 * d + 4 * a
        detect = 12 * a + 8 * l + 4 * w + 4 * x
        sweep = 4 * n if modes[r - 1] == 1 else 4 * a
        total += assign + detect + 2 * sweep
    return total


def host_facts():
    """The host's logical core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform

    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "arch": platform.machine()}


def _active_sums(fin, R, weights=None):
    """x[r] = sum of weights over the nodes still active at round r (fin >= r)."""
    c = np.bincount(fin, weights=weights, minlength=R + 2).astype(np.float64)
    return np.cumsum(c[::-1])[::-1]


def pushing_bytes(rp, cl, fin, modes, t1=64, chunk=1024, maxc_push=2048):
    """Bytes the pushing kernel's own steps move in one colouring (a model of
    its algorithm, not of its caches), from the per-node finalisation rounds:
      degree pass   rowptr 4(n + 1) and the bitmaps cleared, 4 per word
                    (ceil(min(d, 2048) / 32) words for d > t1);
      round 1       rowptr, the first neighbour of each non-isolated node,
                    colour and tentative-colour writes, loser pushes;
      every commit  the node's row read once (4 d) with a check of each
                    neighbour (rowptr pair and colour, 12 B), and a 4-byte
                    atomic OR for each neighbour that keeps a bitmap and is
                    still active;
      round r >= 2  low-degree nodes (d <= t1) rescan their rows: 8 + 8 d +
                    4 (assign) and 12 + 8 (lower neighbours) (detect);
                    nodes above t1 read their bitmap (4 per word) and write
                    tent (assign: 8 + 4 words + 4); nodes of one work item
                    (d <= chunk) scan the lower part of their row, nodes of
                    several scan their list of active lower-ID neighbours
                    (8 per entry with its tentative colour; + 4 to write
                    each list entry in round 2); commits, loser pushes and
                    worklist reads (4n per phase when topology-driven)."""
    n = rp.size - 1
    deg = np.diff(rp).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    lowmask = cl < src
    nlow = np.bincount(src[lowmask], minlength=n).astype(np.int64)
    R = int(fin.max())
    big = deg > t1
    words = np.where(big, (np.minimum(deg, maxc_push) + 31) // 32, 0)
    total = 4.0 * (n + 1) + 4.0 * words.sum()                          # degree pass
    A = _active_sums(fin, R)
    total += 4 * (n + 1) + 4 * int((deg > 0).sum()) + 8 * n + 4 * A[2]  # round 1
    # commits: row read once, neighbour checks, atomics to active bitmapped neighbours
    total += 16.0 * deg.sum()
    fs, fd = fin[src], fin[cl]
    total += 4.0 * np.count_nonzero(big[cl] & (fd > fs))
    # per-round sums over the active set
    low = ~big
    A_low = _active_sums(fin, R, low.astype(np.float64))
    D_low = _active_sums(fin, R, np.where(low, deg, 0).astype(np.float64))
    L_low = _active_sums(fin, R, np.where(low, nlow, 0).astype(np.float64))
    A_big = _active_sums(fin, R, big.astype(np.float64))
    W_big = _active_sums(fin, R, words.astype(np.float64))
    row1 = big & (deg <= chunk)
    L_row = _active_sums(fin, R, np.where(row1, nlow, 0).astype(np.float64))
    listed = deg > chunk
    e = lowmask & listed[src]
    m = np.minimum(fs[e], fd[e])  # a list entry is active while both ends are
    Ecnt = np.bincount(m, minlength=R + 2).astype(np.float64)
    E = np.cumsum(Ecnt[::-1])[::-1]
    for r in range(2, R + 1):
        a, w = A[r], A[r] - A[r + 1]
        x = a - w
        assign = A_low[r] * 12 + 8 * D_low[r] + A_big[r] * 12 + 4 * W_big[r]
        detect = A_low[r] * 12 + 8 * L_low[r] + A_big[r] * 4 + 8 * L_row[r] + 8 * E[r]
        if r == 2:
            detect += 4 * E[r]
        sweep = 4 * n if modes[r - 1] == 1 else 4 * a
        total += assign + detect + 4 * w + 4 * x + 2 * sweep
    return int(total)


def cpu_baseline_leg(rp, cl):
    """The oracle, single-threaded, on the headline graph itself (one colouring)."""
    import oracle

    t = time.perf_counter()
    oracle.color(rp, cl, trace=False)
    dt = time.perf_counter() - t
    h = host_facts()
    return {
        "value": cl.size / dt,
        "unit": UNIT,
        "cores": 1,
        "kind": "oracle",
        "sample": f"one oracle colouring of the headline RMAT scale-22 graph, {dt:.1f} s on 1 core",
        "host_nproc": h["nproc"],
        "host_cpu": f"{h['arch']} {h['cpu_model']}",
        "seconds": dt,
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1912_01478_gb300 import graphgen

    # bounded sample of the workload per step: RMAT scale 18 from the same generator
    rp, cl = graphgen.rmat(18, 16, seed=2)
    for _ in range(args.warmup):
        oracle.color(rp, cl, trace=False)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.color(rp, cl, trace=False)
    dt = time.perf_counter() - t
    value = cl.size * args.steps / dt
    sample = (f"per step one oracle colouring of RMAT scale 18 (same generator, edge factor 16, "
              f"seed 2; {rp.size - 1} nodes, {cl.size} entries)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC + "; oracle sample: RMAT scale 18", "driver": "cpu oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host_nproc": os.cpu_count(), "host_cpu": host_facts()["cpu_model"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()

    import torch

    from paper_1912_01478_gb300 import _build, graphgen, ipgc

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()

    rp, cl = graphgen.workload(WORKLOAD)
    n, nnz = rp.size - 1, cl.size
    # the CPU baseline (the oracle on this graph, one core) runs before any GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(rp, cl)
    drp = torch.from_numpy(rp).to(dev)
    dcl = torch.from_numpy(cl).to(dev)
    colors = torch.empty(n, dtype=torch.int32, device=dev)
    ctx = ipgc.Context(local)
    stream = torch.cuda.Stream(device=dev)
    if ctx.validate(drp, dcl, stream=stream) != ipgc.IPGC_OK:
        raise SystemExit("input graph failed validation")
    opts = ipgc.ColorOptions(mode=args.mode, driver=args.driver, validate=False,
                             forbidden=args.forbidden)
    pushing = args.driver == "persistent" and args.forbidden in ("auto", "push")

    # one traced run (untimed): per-round modes and finalisation rounds for the byte count
    trace = ipgc.trace_buffer(n + 2, local)
    fin = torch.zeros(n, dtype=torch.int32, device=dev)
    _, st = ctx.color(drp, dcl, colors, opts, stream=stream, trace=trace, fin_round=fin)
    tr = ipgc.read_trace(trace, st.rounds)
    rounds, ncolors, r0 = st.rounds, st.num_colors, st.filter_round
    fin_h = fin.cpu().numpy()
    alg_bytes = algorithmic_bytes(rp, cl, fin_h, tr["mode"].tolist())
    maxdeg = int(np.diff(rp).max()) if n else 0
    t1_used = maxdeg if maxdeg <= 255 else 64  # the library's rule when t1 = 0
    own_bytes = (pushing_bytes(rp, cl, fin_h, tr["mode"].tolist(), t1=t1_used)
                 if pushing and maxdeg > t1_used else alg_bytes)
    # per kernel: rounds before the hand-over round r0 and from it on, their
    # bytes and device times (%globaltimer of the trace)
    rb = round_bytes(rp, cl, fin_h, tr["mode"].tolist())
    t_round_end = tr["t_detect"].astype(np.int64)
    split = r0 - 1 if r0 > 0 else rounds
    per_kernel = [{
        "kernel": "persistent_push_kernel<256>" if pushing else "persistent_kernel<256>",
        "rounds": [1, split],
        "algorithmic_bytes": int(sum(rb[:split])),
        "device_ms": float(t_round_end[split - 1] - tr["t_begin"][0]) / 1e6,
    }]
    if r0 > 0:
        per_kernel.append({
            "kernel": "persistent_filt_kernel<256>",
            "rounds": [r0, rounds],
            "algorithmic_bytes": int(sum(rb[split:])),
            "device_ms": float(t_round_end[rounds - 1] - tr["t_begin"][split]) / 1e6,
        })
    for k in per_kernel:
        k["algorithmic_gbs"] = k["algorithmic_bytes"] / max(k["device_ms"], 1e-9) / 1e6
    if args.driver == "hostloop":  # round 1, two per later round, the finishing kernel
        launches_per_step = 2 + 2 * (rounds - 1)
    elif pushing:  # the pushing kernel, then the rescanning ones (they return at once; the
        # filtering kernel is enqueued too when the choice is automatic)
        launches_per_step = 3 if args.forbidden == "auto" else 2
    else:  # the persistent kernel, then the filtering kernel (returns at once without a hand-over)
        launches_per_step = 2 if opts.filter_degree >= 0 else 1
    del trace, fin

    # warm-up, then K timed steps bracketed by barrier + synchronize
    for _ in range(args.warmup):
        ctx.color(drp, dcl, colors, opts, stream=stream, wait=False)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            ctx.color(drp, dcl, colors, opts, stream=stream, wait=False)
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    total_ms = t_start.elapsed_time(t_end)
    per_launch_ms = [a.elapsed_time(b) for a, b in ev]
    st = ctx.last_stats()
    assert st.error == 0 and st.rounds == rounds and st.num_colors == ncolors
    total_ms = max_over_ranks(total_ms, world)
    if world > 1:
        dist.barrier()

    # end to end through the host-buffer entry point: copies inside the region
    hrp = torch.from_numpy(rp).pin_memory().numpy()
    hcl = torch.from_numpy(cl).pin_memory().numpy()
    hout = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    ctx.color_host(hrp, hcl, hout, opts, stream=stream)
    t0 = time.perf_counter()
    e2e_calls = []  # per call, for the detail file (the host link and the host vary by box)
    for _ in range(args.e2e_steps):
        tc = time.perf_counter()
        ctx.color_host(hrp, hcl, hout, opts, stream=stream)
        e2e_calls.append(round((time.perf_counter() - tc) * 1e3, 3))
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world)
    e2e_val = job_value(nnz, 1, world, e2e_s * 1e3)

    if rank != 0:
        dist.destroy_process_group()
        return
    hbm, src = peaks()
    validate_ms = default_ms = None
    if world == 1:
        validate_ms, default_ms = validate_leg(ctx, drp, dcl, stream, ipgc.ColorOptions(
            mode=args.mode, driver=args.driver, forbidden=args.forbidden))
    worklist_out = worklist_leg(args, ctx, drp, dcl, stream) if world == 1 else None
    rules_out, policy_w = mode_rules_leg(args, ctx) if world == 1 else (None, None)
    batched_out = None
    if world == 1 and args.batch_graphs > 0:
        del drp, dcl, colors
        torch.cuda.empty_cache()
        batched_out = batched_leg(args, ctx, dev, stream, policy_w)
    road_out = er_out = None
    if world == 1:
        torch.cuda.empty_cache()
        road_out = road_leg(args, ctx, dev, stream, hbm)
        er_out = er_leg(args, ctx, dev, stream)
    suite_out = suite_leg(args, ctx, stream) if world == 1 else None
    micro_out = None
    if world == 1 and args.micro_n > 0:
        torch.cuda.empty_cache()
        micro_out = micro_leg(args, ctx)
    serving_out = None
    if world == 1 and args.serve_rates:
        torch.cuda.empty_cache()
        serving_out = serving_leg(args, ctx, dev, stream)
    traffic = measured_traffic()
    avg_launch_s = float(np.mean(per_launch_ms)) / 1e3
    achieved_gbs = alg_bytes / avg_launch_s / 1e9
    value = job_value(nnz, args.steps, world, total_ms)
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD_DESC,
            "n": int(n),
            "nnz": int(nnz),
            "rounds": int(rounds),
            "colors": int(ncolors),
            "rounds_topo": int(st.rounds_topo),
            "rounds_data": int(st.rounds_data),
            "schedule": f"{args.mode} (H = 0.6 n), driver {args.driver}",
            "forbidden_colours": ("bitmaps filled by pushes, lower-neighbour lists for conflicts"
                                  if pushing else "rows rescanned every round"),
            "neighbour_filtering": (f"filter_degree 1024, start |WL| <= n/32, round {int(r0)}"
                                    if not pushing else "off (pushing)"),
            "l2": "inputs larger than L2 (col 513 MB vs 129 MB L2); no flush",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "roofline": {
            "bound": "hbm",
            "achieved": achieved_gbs,
            "peak": hbm,
            "unit": "GB/s",
            "frac": achieved_gbs / hbm,
            "traffic": traffic,
            "peak_source": src,
            "algorithmic_bytes_per_step": int(alg_bytes),
            "bytes_model": "the paper's loop (rows rescanned every round), exact from the trace",
            "avg_step_ms": avg_launch_s * 1e3,
            "kernels": " + ".join(k["kernel"] for k in per_kernel),
            "launches_per_step": launches_per_step,
            "traffic_source": "profiles/rmat_s22_dram_traffic.md (ncu dram__bytes_read.sum + "
                              "dram__bytes_write.sum, both launches, one colouring)"
                              if traffic is not None else "no ncu summary for these kernel sources",
        },
        "e2e": {
            "value": e2e_val,
            "unit": UNIT,
            "h2d_bytes_per_step": int(4 * (n + 1) + 4 * nnz),
            "d2h_bytes_per_step": int(4 * n),
        },
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clk.summary(),
        "cpu_baseline": ({k: v for k, v in cpu.items() if k != "seconds"} if cpu else None),
        "micro_benchmark": compact_micro(micro_out),
        "worklist_policy": compact_worklist(worklist_out),
        "suite": ({"geomean_hybrid_over_plain": suite_out["geomean_hybrid_over_plain"],
                   "geomean_push_over_plain": suite_out["geomean_push_over_plain"]}
                  if suite_out else None),
        # (the driver keeps the line's end: what matters most comes last)
        "roofline_dram": ({"achieved": _r(traffic / avg_launch_s / 1e9), "peak": hbm, "unit": "GB/s",
                           "frac": _r(traffic / avg_launch_s / 1e9 / hbm, 3),
                           "bytes_per_step": traffic, "what": "ncu DRAM bytes"}
                          if traffic is not None else None),
        "roofline_own": {"achieved": _r(own_bytes / avg_launch_s / 1e9), "peak": hbm, "unit": "GB/s",
                         "frac": _r(own_bytes / avg_launch_s / 1e9 / hbm, 3),
                         "bytes_per_step": int(own_bytes), "what": "pushing_bytes"},
        "validate_ms": _r(validate_ms),
        "default_call_ms": _r(default_ms),
        "er": er_out,
        "road": compact_road(road_out),
        "batched": compact_batched(batched_out),
        "serving": compact_serving(serving_out),
        "mode_rules": compact_rules(rules_out),
    }
    if args.detail:
        with open(args.detail, "w") as f:
            json.dump({"headline_per_kernel": per_kernel, "e2e_calls_ms": e2e_calls, "batched": batched_out,
                       "serving": serving_out, "micro_benchmark": micro_out,
                       "worklist_policy": worklist_out, "suite": suite_out,
                       "mode_rules": rules_out, "road": road_out}, f, indent=1)
    print(json.dumps(out, separators=(",", ":")), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _r(x, k=4):
    """x rounded to k significant digits (None stays None)."""
    if x is None:
        return None
    return float(f"{x:.{k}g}")


def compact_road(r):
    if not r:
        return None
    return {"edges_per_s": _r(r["edges_per_s"]), "ms": _r(r["ms"]), "rounds": r["rounds"],
            "frac": _r(r["roofline"]["frac"], 3)}


def compact_batched(b):
    if not b:
        return None
    out = {"graphs": b["graphs"], "graphs_per_s": _r(b["graphs_per_s"]),
           "edges_per_s": _r(b["edges_per_s"]), "ms": _r(b["ms_per_batch"]),
           "ms_default": _r(b["ms_per_batch_default_schedule"]),
           "plain_graphs_per_s": _r(b["plain_graphs_per_s"]),
           "speedup_vs_plain": _r(b["speedup_vs_plain"], 3),
           "same_colours_as_plain": b["identical_colours_batched_vs_plain"],
           "tuned": "{forbidden} t1={t1} chunk={chunk} team<={max_team}".format(**b["autotuned"])}
    if b.get("ms_learned"):
        out["ms_learned"] = _r(b["ms_learned"])
        out["learned_speedup_vs_plain"] = _r(b["learned_speedup_vs_plain"], 3)
    return out


def compact_serving(s):
    if not s:
        return None
    rates = s["rates"]
    col = lambda k, d=3: [_r(r[k], d) for r in rates]  # noqa: E731
    return {"rate_rps": [r["rate_rps"] for r in rates], "rps": col("throughput_rps"),
            "p50_ms": col("p50_ms"), "p99_ms": col("p99_ms"), "plain_rps": col("plain_throughput_rps"),
            "plain_p50_ms": col("plain_p50_ms"), "plain_p99_ms": col("plain_p99_ms"),
            "plain_requests": [r["plain_requests"] for r in rates]}


def compact_rules(m):
    if not m:
        return None
    out = {k: _r(v) for k, v in m["total_round_ms"].items()}
    out.update({f"colouring_{k}": _r(v) for k, v in m["colouring_ms"].items()})
    return out


def compact_micro(m):
    if not m:
        return None
    return {"crossover_iteration": m["crossover_iteration"], "nowl_ms": _r(m["nowl"]["total_ms"]),
            "wl_ms": _r(m["wl"]["total_ms"]), "hybrid_ms": _r(m["hybrid"]["total_ms"]),
            "best_ms": _r(m["per_iteration_best_ms"])}


def compact_worklist(w):
    if not w:
        return None
    return {str(r["threshold_frac"]): [_r(r["keep"]["ms"]), _r(r["rebuild"]["ms"])] for r in w["rows"]}


if __name__ == "__main__":
    main()
