"""GPU parity of the forbidden-colour bitmaps (IPGC_FORBIDDEN_PUSH).

With pushing, a node of degree > t1 finds its tentative colour in a bitmap
that its neighbours fill when they are committed, instead of rescanning its
row each round (Section II-C defines the colour, not how the finalised
neighbours' colours are found). The colours, the rounds and every round's
worklist must stay those of the oracle: for every mode policy, bucket split
and worklist policy; for hubs whose rows are pushed by the whole team; for
complete graphs whose colours leave the bitmaps (K_2049 and up fall back to
rescanning); and for the full-size workloads against the stored oracle
results.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen
from test_gpu_parity import assert_parity, band_network, complete, csr, gpu_color, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PUSH = dict(forbidden="push")


@pytest.fixture(scope="module")
def ctx():
    import torch

    assert torch.cuda.is_available()
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    return ipgc.Context(0)


@pytest.mark.parametrize("mode", ["threshold", "topo", "data"])
def test_er_all_modes(ctx, er_graph, mode):
    rp, cl = er_graph
    for t1 in (0, 1, 4):  # 0: every node on the low-degree path (no bitmaps at all)
        assert_parity(ctx, rp, cl, mode=mode, t1=t1, **PUSH)


@pytest.mark.parametrize("t1,chunk", [(0, 0), (1, 32), (3, 64), (8, 100), (63, 4096), (24, 33),
                                      (1, 4096), (255, 32), (16, 1024)])
def test_bucket_thresholds(ctx, t1, chunk):
    # RMAT: hubs with many items (pushed by the whole team), single-item
    # nodes (pushed by their own warp) and low-degree nodes (edge-balanced)
    rp, cl = graphgen.rmat(14, 16, seed=21)
    ref = oracle.color(rp, cl)
    for mode in ("threshold", "data", "topo"):
        assert_parity(ctx, rp, cl, ref, t1=t1, chunk=chunk, mode=mode, **PUSH)


@pytest.mark.parametrize("leaves", [10, 64, 1023, 1024, 70000])
def test_stars(ctx, leaves):
    # the centre (ID 0) wins round 1 and pushes colour 1 to every leaf; with
    # the centre last (highest ID) the leaves win round 1 and push into the
    # centre's bitmap
    for centre in (0, leaves):
        others = [v for v in range(leaves + 1) if v != centre]
        rp, cl = csr(leaves + 1, [(centre, v) for v in others])
        for t1 in (1, 8):
            assert_parity(ctx, rp, cl, t1=t1, chunk=32, **PUSH)


@pytest.mark.parametrize("n", [65, 300, 1100, 2046, 2047, 2048, 2049, 2100])
def test_complete_graphs_leave_the_bitmap(ctx, n):
    # K_n: colour v + 1 for node v in round v + 1; from the round that starts
    # with colour 2048 committed the colours no longer fit the bitmaps and
    # the assignment step rescans rows again
    rp, cl = complete(n)
    ref = oracle.color(rp, cl)
    assert ref.num_colors == n
    for mode in ("data", "topo"):
        assert_parity(ctx, rp, cl, ref, mode=mode, t1=16, chunk=512, **PUSH)


def test_trace_and_finalisation_rounds(ctx):
    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.rmat(15, 16, seed=31)
    ref = oracle.color(rp, cl)
    drp, dcl = to_dev(rp, cl)
    fin = torch.zeros(len(rp) - 1, dtype=torch.int32, device="cuda")
    tr = ipgc.trace_buffer(ref.rounds + 2)
    colors, st = ctx.color(drp, dcl, options=ipgc.ColorOptions(**PUSH), trace=tr, fin_round=fin)
    assert np.array_equal(colors.cpu().numpy(), ref.colors)
    assert np.array_equal(fin.cpu().numpy(), ref.fin_round)
    t = ipgc.read_trace(tr, st.rounds)
    assert t["wl_size"].tolist() == list(ref.wl_sizes)
    assert t["deg_sum"].tolist() == list(ref.deg_sums)


@pytest.mark.parametrize("graph", ["rmat", "road"])
def test_worklist_rebuild_and_thresholds(ctx, graph):
    rp, cl = {"rmat": lambda: graphgen.rmat(14, 16, seed=22),
              "road": lambda: graphgen.road(300, seed=23)}[graph]()
    ref = oracle.color(rp, cl)
    for frac in (0.6, 0.2, 0.0, 1.0, 5.0):
        for wl in ("keep", "rebuild"):
            assert_parity(ctx, rp, cl, ref, threshold_frac=frac, worklist=wl, t1=8, **PUSH)


def test_learned_switch_band(ctx):
    import torch

    from paper_1912_01478_gb300 import ipgc, policy

    rp, cl = graphgen.rmat(14, 16, seed=24)
    ref = oracle.color(rp, cl)
    policy.load(ctx, band_network(20 / 84, 40 / 104))
    try:
        drp, dcl = to_dev(rp, cl)
        for wl in ("rebuild", "keep"):
            colors, st = ctx.color(drp, dcl, options=ipgc.ColorOptions(mode="learned", worklist=wl,
                                                                       **PUSH))
            assert np.array_equal(colors.cpu().numpy(), ref.colors) and st.rounds == ref.rounds
    finally:
        policy.load(ctx, None)


def test_grid_shapes_and_block_sizes(ctx):
    rp, cl = graphgen.rmat(13, 16, seed=9)
    ref = oracle.color(rp, cl)
    for bs in (256, 512):
        for bps in (1, 2):
            assert_parity(ctx, rp, cl, ref, block_size=bs, blocks_per_sm=bps, **PUSH)


def test_repeat_reuses_the_workspace(ctx):
    # bitmaps are cleared by every colouring: a second graph and a repeat of
    # the first must not see stale bits
    a = graphgen.rmat(13, 16, seed=41)
    b = graphgen.rmat(12, 32, seed=42)
    ra, rb = oracle.color(*a), oracle.color(*b)
    for g, r in ((a, ra), (b, rb), (a, ra), (a, ra)):
        assert_parity(ctx, *g, r, **PUSH)


def test_needs_the_persistent_driver(ctx):
    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.er(500, 1500, seed=5)
    with pytest.raises(ipgc.IpgcError) as ei:
        gpu_color(ctx, rp, cl, driver="hostloop", **PUSH)
    assert ei.value.code == ipgc.IPGC_ERR_UNSUPPORTED


@pytest.mark.slow
@pytest.mark.parametrize("name", ["road_4096_seed3", "rmat_s22_ef16_seed2"])
def test_full_size_workloads(ctx, name):
    with open(os.path.join(GOLDEN, "expected_full.json")) as f:
        exp = json.load(f)[name]
    rp, cl = graphgen.workload(name)
    assert graphgen.graph_hash(rp, cl) == exp["graph_hash"], "input changed"
    for kw in (dict(), dict(mode="data"), dict(mode="topo")):
        got, st, tr = gpu_color(ctx, rp, cl, trace_rounds=exp["rounds"] + 4, validate=False,
                                **kw, **PUSH)
        assert hashlib.sha256(got.astype("<i4").tobytes()).hexdigest() == exp["colors_sha256"], kw
        assert st.rounds == exp["rounds"] and st.num_colors == exp["num_colors"]
        assert tr["wl_size"].tolist() == exp["wl_sizes"]


def test_repeated_colourings_match(ctx):
    # races between CTAs show up as rare, run-to-run differences: colour the
    # same graphs many times (RMAT's last rounds run late: every active node
    # keeps a one-item list, winners push along their lists and the next
    # round collects lower-ID winners from them, with no push phase)
    rp, cl = graphgen.rmat(17, 16, seed=2)
    ref = oracle.color(rp, cl)
    drp, dcl = to_dev(rp, cl)
    from paper_1912_01478_gb300 import ipgc

    for mode in ("threshold", "data"):
        o = ipgc.ColorOptions(validate=False, mode=mode, **PUSH)
        for _ in range(60):
            colors, st = ctx.color(drp, dcl, options=o)
            assert np.array_equal(colors.cpu().numpy(), ref.colors), mode
            assert st.rounds == ref.rounds and st.num_colors == ref.num_colors


@pytest.mark.slow
def test_repeated_full_size_colourings_match(ctx):
    with open(os.path.join(GOLDEN, "expected_full.json")) as f:
        exp = json.load(f)["rmat_s22_ef16_seed2"]
    rp, cl = graphgen.workload("rmat_s22_ef16_seed2")
    drp, dcl = to_dev(rp, cl)
    from paper_1912_01478_gb300 import ipgc

    o = ipgc.ColorOptions(validate=False, **PUSH)
    for _ in range(40):
        colors, st = ctx.color(drp, dcl, options=o)
        got = colors.cpu().numpy()
        assert hashlib.sha256(got.astype("<i4").tobytes()).hexdigest() == exp["colors_sha256"]


def test_automatic_choice_between_pushing_and_rescanning(ctx):
    # by default (IPGC_FORBIDDEN_AUTO) the bitmaps are used only when the rows
    # of the nodes above t1 hold at least half of the entries: on a graph of a
    # few giant hubs over a sparse base (the circuit5M stand-in, 29 % of its
    # entries in rows of degree > 64) no round pushes; on RMAT (most entries
    # in long rows) the rounds push; the colours are the oracle's either way
    import torch

    from paper_1912_01478_gb300 import ipgc

    for rp, cl, pushes in ((*graphgen.suite_graph("circuit5M", 0.05), False),
                           (*graphgen.rmat(15, 16, seed=23), True)):
        deg = np.diff(rp)
        share = deg[deg > 64].sum() / cl.size
        assert (share >= 0.5) == pushes
        ref = oracle.color(rp, cl, trace=False)
        drp, dcl = to_dev(rp, cl)
        tr = ipgc.trace_buffer(rp.size + 1)
        colors, st = ctx.color(drp, dcl, options=ipgc.ColorOptions(validate=False), trace=tr)
        assert np.array_equal(colors.cpu().numpy(), ref.colors) and st.rounds == ref.rounds
        rec = ipgc.read_trace(tr, st.rounds)
        assert (int(rec["push_ns"].sum()) > 0) == pushes
        # forced pushing still pushes
        tr2 = ipgc.trace_buffer(rp.size + 1)
        colors2, st2 = ctx.color(drp, dcl, options=ipgc.ColorOptions(validate=False, **PUSH),
                                 trace=tr2)
        assert np.array_equal(colors2.cpu().numpy(), ref.colors)
        assert int(ipgc.read_trace(tr2, st2.rounds)["push_ns"].sum()) > 0
