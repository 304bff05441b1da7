"""Batched colouring: every graph of a batch gets, bit for bit, the colouring
the CPU oracle gives it alone, whatever the team split, team size, mode or
block size (the schedule must never change a colour)."""
import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen

pytestmark = pytest.mark.gpu


def make_batch(graphs):
    """Concatenate (rowptr, col) pairs into the batched layout."""
    node_off = np.zeros(len(graphs) + 1, np.int64)
    edge_off = np.zeros(len(graphs) + 1, np.int64)
    rps, cls = [], []
    for g, (rp, cl) in enumerate(graphs):
        node_off[g + 1] = node_off[g] + rp.size - 1
        edge_off[g + 1] = edge_off[g] + cl.size
        rps.append(rp)
        cls.append(cl)
    return dict(
        node_off=node_off,
        edge_off=edge_off,
        rowptr_cat=np.concatenate(rps).astype(np.int32),
        col_cat=np.concatenate(cls).astype(np.int32) if edge_off[-1] else np.zeros(0, np.int32),
    )


def run_batch(ctx, bt, **kw):
    import torch

    from paper_1912_01478_gb300 import batched

    drp = torch.from_numpy(bt["rowptr_cat"]).cuda()
    dcl = torch.from_numpy(bt["col_cat"]).cuda()
    colors, st = batched.color_batched(ctx, bt["node_off"], bt["edge_off"], drp, dcl,
                                       opts=batched.options(**kw))
    return colors.cpu().numpy(), st


def check_against_oracle(bt, colors, st, refs=None):
    no = bt["node_off"]
    G = no.size - 1
    for g in range(G):
        rp, cl = graphgen.batch_graph(bt, g)
        ref = refs[g] if refs is not None else oracle.color(rp, cl, trace=False)
        got = colors[no[g]:no[g + 1]]
        assert np.array_equal(got, ref.colors), g
        assert st["rounds"][g] == ref.rounds and st["num_colors"][g] == ref.num_colors, g
        assert st["error"][g] == 0


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    return ipgc.Context(0)


@pytest.fixture(scope="module")
def mixed_batch():
    bt = graphgen.batch(48, seed=4, nmin=100, nmax=40_000)
    refs = []
    for g in range(48):
        rp, cl = graphgen.batch_graph(bt, g)
        refs.append(oracle.color(rp, cl, trace=False))
    return bt, refs


@pytest.mark.parametrize(
    "kw",
    [
        dict(),
        dict(nnz_per_cta=1),                     # every graph on a grid-sized team
        dict(nnz_per_cta=1, max_team=2),
        dict(nnz_per_cta=5_000, max_team=16),    # teams of 1..16 CTAs
        dict(nnz_per_cta=1 << 40),               # every graph on one CTA
        dict(mode="data"),
        dict(mode="topo", nnz_per_cta=20_000),
        dict(block_size=512, chunk=256, t1=8),
        # rows rescanned every round (the default pushes into bitmaps)
        dict(forbidden="rescan"),
        dict(forbidden="rescan", nnz_per_cta=5_000, max_team=16),
        dict(forbidden="rescan", mode="topo", nnz_per_cta=20_000),
        # small t1: most graphs keep bitmaps; big chunk: few list items
        dict(t1=4, chunk=4096, nnz_per_cta=5_000),
    ],
)
def test_batch_matches_oracle(ctx, mixed_batch, kw):
    bt, refs = mixed_batch
    colors, st = run_batch(ctx, bt, **kw)
    check_against_oracle(bt, colors, st, refs)


def test_degenerate_graphs_in_a_batch(ctx):
    import itertools

    edgeless = graphgen.from_edges(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    one = graphgen.from_edges(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    empty = (np.zeros(1, np.int32), np.zeros(0, np.int32))
    k = 70
    e = np.array(list(itertools.combinations(range(k), 2)), np.int32)
    clique = graphgen.from_edges(k, e[:, 0], e[:, 1])
    star = graphgen.from_edges(3000, np.zeros(2999, np.int32), np.arange(1, 3000, dtype=np.int32))
    graphs = [edgeless, empty, one, clique, graphgen.rmat(12, 8, seed=5), empty, star]
    bt = make_batch(graphs)
    colors, st = run_batch(ctx, bt, nnz_per_cta=2000, max_team=8)
    check_against_oracle(bt, colors, st)
    assert st["rounds"][1] == 0 and st["rounds"][5] == 0


def test_batch_equals_single_graph_calls(ctx):
    import torch

    bt = graphgen.batch(16, seed=7, nmin=2_000, nmax=60_000)
    colors, st = run_batch(ctx, bt, nnz_per_cta=30_000)
    no = bt["node_off"]
    for g in range(16):
        rp, cl = graphgen.batch_graph(bt, g)
        one, st1 = ctx.color(torch.from_numpy(np.ascontiguousarray(rp)).cuda(),
                             torch.from_numpy(np.ascontiguousarray(cl)).cuda())
        assert np.array_equal(one.cpu().numpy(), colors[no[g]:no[g + 1]])
        assert st1.rounds == st["rounds"][g]


def test_batch_validation(ctx):
    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.er(300, 900, seed=3)
    bad = cl.copy()
    bad[0] = 10_000
    bt = make_batch([graphgen.er(200, 500, seed=2), (rp, bad)])
    with pytest.raises(ipgc.IpgcError) as ei:
        run_batch(ctx, bt, validate=True)
    assert ei.value.code == ipgc.IPGC_ERR_INVALID


def test_autotuners_keep_colours(ctx):
    import ctypes

    import torch

    from paper_1912_01478_gb300 import batched, ipgc

    bt = graphgen.batch(24, seed=9, nmin=500, nmax=30_000)
    drp = torch.from_numpy(bt["rowptr_cat"]).cuda()
    dcl = torch.from_numpy(bt["col_cat"]).cuda()
    out = torch.empty(int(bt["node_off"][-1]), dtype=torch.int32, device="cuda")
    o, ms = batched.autotune(ctx, bt["node_off"], bt["edge_off"], drp, dcl, out, sample_graphs=12)
    assert ms > 0 and o.base.chunk in (0, 512, 1024, 2048) and o.max_team in (0, 4, 16, 64)
    colors, st = batched.color_batched(ctx, bt["node_off"], bt["edge_off"], drp, dcl, opts=o)
    check_against_oracle(bt, colors.cpu().numpy(), st)
    # single-graph tuner
    rp, cl = graphgen.rmat(14, 16, seed=3)
    ref = oracle.color(rp, cl, trace=False)
    g_rp, g_cl = torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda()
    scratch = torch.empty(rp.size - 1, dtype=torch.int32, device="cuda")
    opt = ipgc.ColorOptions().to_c()
    best = ctypes.c_float(0)
    rc = ipgc.lib().ipgc_autotune(ctx.handle, g_rp.data_ptr(), g_cl.data_ptr(), rp.size - 1, cl.size,
                                  scratch.data_ptr(), 2, ctypes.byref(opt), ctypes.byref(best), None)
    assert rc == 0 and best.value > 0 and opt.chunk in (256, 512, 1024, 2048, 4096)
    st1 = ipgc.Stats()
    rc = ipgc.lib().ipgc_color_ex(ctx.handle, g_rp.data_ptr(), g_cl.data_ptr(), rp.size - 1, cl.size,
                                  scratch.data_ptr(), ctypes.byref(st1), ctypes.byref(opt), None)
    assert rc == 0 and np.array_equal(scratch.cpu().numpy(), ref.colors)


def test_batch_with_the_learned_switch(ctx, mixed_batch):
    # the learned switch in a batched launch: a hand-built network that says
    # "topology-driven" while the largest colour is in a band (so rounds of
    # both modes alternate within a graph, and late rounds follow), loaded
    # into the context; every graph keeps the oracle's colours, with the
    # pushing and the rescanning batched kernels
    from paper_1912_01478_gb300 import policy
    from test_gpu_parity import band_network

    bt, refs = mixed_batch
    policy.load(ctx, band_network(3 / 67, 8 / 72))  # maxc in (3, 8)
    try:
        for forbidden in ("auto", "rescan"):
            colors, st = run_batch(ctx, bt, mode="learned", forbidden=forbidden)
            check_against_oracle(bt, colors, st, refs)
            # some graph ran topology-driven rounds after the first
            assert int(st["rounds_topo"].max()) > 1
    finally:
        policy.load(ctx, None)
