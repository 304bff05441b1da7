"""GPU parity: the CUDA path against the CPU oracle, bit for bit.

Colouring is integer work, so per-node colours, the round count and the
colour count must be identical for every mode policy (topology, data,
threshold hybrid), driver (persistent, host loop) and degree-bucket setting:
the mode never changes a colour (the paper's Plain and Hybrid use the same
colours, Section V). Sizes span many warps, CTAs and all three degree buckets
with ragged tails; the full-size workloads are compared against stored oracle
results written by tests/golden/make_expected.py.
"""
import hashlib
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MODES = [
    ("threshold", "persistent"),
    ("topo", "persistent"),
    ("data", "persistent"),
    ("threshold", "hostloop"),
    ("data", "hostloop"),
    ("topo", "hostloop"),
]


@pytest.fixture(scope="module")
def ctx():
    import torch

    assert torch.cuda.is_available()
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    return ipgc.Context(0)


def to_dev(rp, cl):
    import torch

    return (
        torch.from_numpy(np.ascontiguousarray(rp, np.int32)).cuda(),
        torch.from_numpy(np.ascontiguousarray(cl, np.int32)).cuda(),
    )


def gpu_color(ctx, rp, cl, trace_rounds=0, **kw):
    from paper_1912_01478_gb300 import ipgc

    drp, dcl = to_dev(rp, cl)
    tr = ipgc.trace_buffer(trace_rounds) if trace_rounds else None
    colors, st = ctx.color(drp, dcl, options=ipgc.ColorOptions(**kw), trace=tr)
    out = colors.cpu().numpy()
    if trace_rounds:
        return out, st, ipgc.read_trace(tr, min(st.rounds, trace_rounds))
    return out, st


def assert_parity(ctx, rp, cl, ref=None, **kw):
    ref = ref if ref is not None else oracle.color(rp, cl)
    colors, st = gpu_color(ctx, rp, cl, **kw)
    assert st.error == 0
    assert np.array_equal(colors, ref.colors), (kw, np.flatnonzero(colors != ref.colors)[:10])
    assert st.rounds == ref.rounds, kw
    assert st.num_colors == ref.num_colors, kw
    assert st.rounds_topo + st.rounds_data == st.rounds
    return st


def csr(n, edges):
    if not edges:
        return graphgen.from_edges(n, np.zeros(0, np.int32), np.zeros(0, np.int32))
    e = np.array(edges, np.int32)
    return graphgen.from_edges(n, e[:, 0], e[:, 1])


@pytest.mark.parametrize("mode,driver", MODES)
def test_er_workload_all_modes(ctx, er_graph, mode, driver):
    rp, cl = er_graph
    st = assert_parity(ctx, rp, cl, mode=mode, driver=driver)
    if mode == "topo":
        assert st.rounds_data == 0
    if mode == "data":
        assert st.rounds_topo == 1  # round 1 always sweeps every node


@pytest.mark.parametrize("name", ["handworked_g7.txt", "handworked_g8.txt"])
def test_handworked(ctx, name):
    from test_oracle_pins import load_golden

    n, edges, colors, rounds, k, wl = load_golden(name)
    rp, cl = csr(n, edges)
    for mode, driver in MODES:
        got, st = gpu_color(ctx, rp, cl, mode=mode, driver=driver)
        assert got.tolist() == colors.tolist() and st.rounds == rounds and st.num_colors == k


def test_trivial_graphs(ctx):
    import torch

    from paper_1912_01478_gb300 import ipgc

    # n = 0
    colors, st = ctx.color(torch.zeros(1, dtype=torch.int32, device="cuda"),
                           torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert colors.numel() == 0 and st.rounds == 0 and st.num_colors == 0
    # n = 1 and edgeless graphs of ragged sizes
    for n in (1, 2, 31, 33, 1000, 70001):
        got, st = gpu_color(ctx, *csr(n, []))
        assert np.all(got == 1) and st.rounds == 1 and st.num_colors == 1


@pytest.mark.parametrize("n", [2, 3, 33, 64, 65, 300, 1100, 1500])
def test_complete_graphs(ctx, n):
    # K_n: colour(v) = v + 1 and n rounds; crosses every degree bucket and
    # (n > 1024) the CTA bitmap beyond the per-warp window
    rp, cl = csr(n, list(itertools.combinations(range(n), 2)))
    got, st = gpu_color(ctx, rp, cl)
    assert np.array_equal(got, np.arange(1, n + 1)) and st.rounds == n and st.num_colors == n


@pytest.mark.parametrize("leaves", [10, 64, 1023, 1024, 70000])
def test_stars(ctx, leaves):
    n = leaves + 1
    rp, cl = csr(n, [(0, i) for i in range(1, n)])
    got, st = gpu_color(ctx, rp, cl)
    assert got[0] == 1 and np.all(got[1:] == 2) and st.rounds == 2
    rp, cl = csr(n, [(i, n - 1) for i in range(n - 1)])
    got, st = gpu_color(ctx, rp, cl)
    assert np.all(got[:-1] == 1) and got[-1] == 2 and st.rounds == 2


@pytest.mark.parametrize("n", [2, 7, 1000, 4097])
def test_paths(ctx, n):
    rp, cl = csr(n, [(i, i + 1) for i in range(n - 1)])
    got, st = gpu_color(ctx, rp, cl)
    assert np.array_equal(got, np.array([1 + i % 2 for i in range(n)])) and st.rounds == n // 2 + 1


@pytest.mark.parametrize("t1,chunk", [(0, 0), (1, 32), (3, 64), (8, 100), (63, 4096), (24, 33), (1, 4096),
                                      (128, 1024), (255, 64), (200, 2048)])
def test_bucket_thresholds(ctx, t1, chunk):
    # the same graph through every split of nodes between the low-degree path
    # and chunked work items, with ragged chunk sizes
    rp, cl = graphgen.rmat(13, 16, seed=11)
    ref = oracle.color(rp, cl)
    for mode in ("threshold", "topo", "data"):
        for forbidden in ("auto", "rescan"):  # (auto: bitmaps with the persistent driver)
            assert_parity(ctx, rp, cl, ref, mode=mode, t1=t1, chunk=chunk, forbidden=forbidden)


@pytest.mark.parametrize("fdeg,t1,chunk,start", [(-1, 0, 0, 0.0), (1, 1, 32, 1.0), (24, 24, 64, 0.05),
                                                  (100, 8, 33, 0.2), (256, 24, 1024, 1.0),
                                                  (2000, 24, 256, 1.0), (0, 63, 4096, 0.01),
                                                  (0, 0, 0, 0.0)])
def test_neighbour_filtering(ctx, fdeg, t1, chunk, start):
    # filtered lists for none, some or all high-degree nodes, handed over in
    # an early or a late round, with one or many work items per node, in
    # every mode and driver: the colours never change
    rp, cl = graphgen.rmat(14, 16, seed=21)
    ref = oracle.color(rp, cl)
    for mode, driver in MODES:
        assert_parity(ctx, rp, cl, ref, mode=mode, driver=driver, filter_degree=fdeg, t1=t1,
                      chunk=chunk, filter_start=start, forbidden="rescan")


def complete(n):
    a, b = np.triu_indices(n, 1)
    return graphgen.from_edges(n, a.astype(np.int32), b.astype(np.int32))


@pytest.mark.parametrize("n", [2046, 2047, 2048, 2049, 2100])
def test_filtering_hands_over_beyond_the_bitmap(ctx, n):
    # K_n: colour(v) = v + 1 and n rounds. Past 2046 colours the filtered
    # nodes' bitmap could not hold every colour, so they go back to reading
    # their rows: the hand-over round must not change a colour
    rp, cl = complete(n)
    for mode, driver, chunk in (("data", "persistent", 0), ("topo", "persistent", 512),
                                ("threshold", "hostloop", 256)):
        got, st = gpu_color(ctx, rp, cl, mode=mode, driver=driver, chunk=chunk, filter_degree=64,
                            filter_start=1.0, forbidden="rescan")
        assert st.error == 0
        assert np.array_equal(got, np.arange(1, n + 1)), (mode, driver)
        assert st.rounds == n and st.num_colors == n


@pytest.mark.parametrize("frac", [0.0, 0.3, 0.6, 0.9, 1.0, 5.0])
def test_threshold_fraction_invariance(ctx, frac):
    rp, cl = graphgen.rmat(14, 8, seed=12)
    assert_parity(ctx, rp, cl, threshold_frac=frac)


@pytest.mark.parametrize("bps", [1, 2])
def test_grid_shapes(ctx, bps):
    rp, cl = graphgen.road(300, seed=13)
    assert_parity(ctx, rp, cl, blocks_per_sm=bps)


@pytest.mark.parametrize("mode,driver", MODES)
def test_rmat_medium(ctx, mode, driver):
    # RMAT scale 16 (65,536 nodes), edge factor 16, permuted IDs
    rp, cl = graphgen.rmat(16, 16, seed=2)
    ref = oracle.color(rp, cl)
    assert_parity(ctx, rp, cl, ref, mode=mode, driver=driver)
    if driver == "persistent":  # the default there pushes colours; rescanning rows as well
        assert_parity(ctx, rp, cl, ref, mode=mode, driver=driver, forbidden="rescan")


@pytest.mark.parametrize("mode", ["threshold", "data", "topo"])
def test_road_medium(ctx, mode):
    rp, cl = graphgen.road(700, seed=3)
    assert_parity(ctx, rp, cl, mode=mode)


def test_batch_shapes_single(ctx):
    bt = graphgen.batch(24, seed=4, nmin=100, nmax=30000)
    for g in range(24):
        rp, cl = graphgen.batch_graph(bt, g)
        assert_parity(ctx, rp, cl)


def test_finalisation_rounds_when_no_node_keeps_a_bitmap(ctx):
    # graphs without a node above t1 (a road grid, a mesh): the pushing
    # kernel hands them to the rescanning kernel after its degree pass; the
    # per-node finalisation rounds and the trace must still be the oracle's
    import torch

    from paper_1912_01478_gb300 import ipgc

    for rp, cl in (graphgen.road(300, seed=41), graphgen.lattice3(24, 6)):
        ref = oracle.color(rp, cl, trace=True)
        assert int(np.diff(rp).max()) <= 255
        drp, dcl = to_dev(rp, cl)
        fin = torch.zeros(rp.size - 1, dtype=torch.int32, device="cuda")
        tr = ipgc.trace_buffer(ref.rounds + 2)
        colors, st = ctx.color(drp, dcl, trace=tr, fin_round=fin)
        assert np.array_equal(colors.cpu().numpy(), ref.colors)
        assert np.array_equal(fin.cpu().numpy(), ref.fin_round)
        t = ipgc.read_trace(tr, st.rounds)
        assert t["wl_size"].tolist() == list(ref.wl_sizes)


def test_buffers_zeroed_on_the_current_stream_before_a_side_stream_colouring(ctx):
    # the binding orders a colouring on another torch stream after the work
    # queued on the current one: a large trace buffer and the finalisation
    # array are zeroed there just before the call, and the zero fill must not
    # land on what the colouring writes
    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.road(1000, seed=43)
    ref = oracle.color(rp, cl, trace=True)
    drp, dcl = to_dev(rp, cl)
    side = torch.cuda.Stream()
    for _ in range(3):
        tr = ipgc.trace_buffer(rp.size + 1)  # about 56 MB of zero fill first
        fin = torch.zeros(rp.size - 1, dtype=torch.int32, device="cuda")
        colors, st = ctx.color(drp, dcl, stream=side, trace=tr, fin_round=fin)
        assert np.array_equal(colors.cpu().numpy(), ref.colors)
        assert np.array_equal(fin.cpu().numpy(), ref.fin_round)
        t = ipgc.read_trace(tr, st.rounds)
        assert t["wl_size"].tolist() == list(ref.wl_sizes)


def test_trace_matches_oracle(ctx):
    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.rmat(15, 16, seed=21)
    ref = oracle.color(rp, cl)
    got, st, tr = gpu_color(ctx, rp, cl, trace_rounds=ref.rounds + 4)
    assert np.array_equal(got, ref.colors)
    # per-node finalisation rounds
    drp, dcl = to_dev(rp, cl)
    fin = torch.zeros(rp.size - 1, dtype=torch.int32, device="cuda")
    for mode in ("threshold", "data", "topo"):
        fin.zero_()
        ctx.color(drp, dcl, options=ipgc.ColorOptions(mode=mode), fin_round=fin)
        assert np.array_equal(fin.cpu().numpy(), ref.fin_round), mode
    assert tr["round"].tolist() == list(range(1, ref.rounds + 1))
    assert tr["wl_size"].tolist() == ref.wl_sizes.tolist()
    assert tr["deg_sum"].tolist() == ref.deg_sums.tolist()
    assert st.edges_processed == int(ref.deg_sums.sum())
    n = rp.size - 1
    H = int(0.6 * n)
    expect_mode = [1 if w > H else 2 for w in ref.wl_sizes]
    assert tr["mode"].tolist() == expect_mode
    assert np.all(tr["t_assign"] >= tr["t_begin"]) and np.all(tr["t_detect"] >= tr["t_assign"])


def test_repeat_and_resize(ctx):
    # the context's workspace is reused across sizes; results stay exact
    for scale in (12, 10, 14, 11):
        rp, cl = graphgen.rmat(scale, 8, seed=scale)
        ref = oracle.color(rp, cl)
        for _ in range(2):
            assert_parity(ctx, rp, cl, ref)


def test_stream_and_async(ctx):
    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.rmat(13, 8, seed=5)
    ref = oracle.color(rp, cl)
    drp, dcl = to_dev(rp, cl)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        colors, st = ctx.color(drp, dcl, stream=s, wait=False)
    assert st is None
    st = ctx.last_stats()
    s.synchronize()
    assert np.array_equal(colors.cpu().numpy(), ref.colors) and st.rounds == ref.rounds


def test_color_host(ctx):
    rp, cl = graphgen.rmat(14, 16, seed=6)
    ref = oracle.color(rp, cl)
    got, st = ctx.color_host(rp, cl)
    assert np.array_equal(got, ref.colors) and st.rounds == ref.rounds


def test_simple_entry_point():
    import ctypes

    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.er(3000, 9000, seed=8)
    ref = oracle.color(rp, cl)
    drp, dcl = to_dev(rp, cl)
    out = torch.empty(rp.size - 1, dtype=torch.int32, device="cuda")
    st = ipgc.Stats()
    rc = ipgc.lib().ipgc_color(drp.data_ptr(), dcl.data_ptr(), rp.size - 1, cl.size, out.data_ptr(),
                               ctypes.byref(st))
    assert rc == 0 and np.array_equal(out.cpu().numpy(), ref.colors) and st.rounds == ref.rounds


def test_device_validation(ctx):
    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.er(500, 2000, seed=9)
    drp, dcl = to_dev(rp, cl)
    assert ctx.validate(drp, dcl) == ipgc.IPGC_OK
    bad = cl.copy()
    bad[5] = 10**6
    assert ctx.validate(*to_dev(rp, bad)) == ipgc.IPGC_ERR_INVALID
    bad = cl.copy()
    bad[rp[7]] = 7
    assert ctx.validate(*to_dev(rp, bad)) == ipgc.IPGC_ERR_INVALID
    # validation on by default: the colouring refuses the bad graph
    with pytest.raises(ipgc.IpgcError) as ei:
        ctx.color(*to_dev(rp, bad))
    assert ei.value.code == ipgc.IPGC_ERR_INVALID


def test_max_rounds_guard(ctx):
    from paper_1912_01478_gb300 import ipgc

    rp, cl = csr(12, list(itertools.combinations(range(12), 2)))
    for driver in ("persistent", "hostloop"):
        with pytest.raises(ipgc.IpgcError) as ei:
            gpu_color(ctx, rp, cl, max_rounds=5, driver=driver)
        assert ei.value.code == ipgc.IPGC_ERR_NO_CONVERGE
    # the context stays usable
    assert_parity(ctx, rp, cl)


def test_bounded_barrier_timeout(ctx):
    # every grid barrier waits for a CTA that never arrives; each wait gives
    # up after timeout_ns, the launch ends and reports IPGC_ERR_TIMEOUT
    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.er(5000, 20000, seed=10)
    with pytest.raises(ipgc.IpgcError) as ei:
        gpu_color(ctx, rp, cl, fault_inject=1, timeout_ns=2_000_000)
    assert ei.value.code == ipgc.IPGC_ERR_TIMEOUT
    assert_parity(ctx, rp, cl)


def _expected():
    with open(os.path.join(GOLDEN, "expected_full.json")) as f:
        return json.load(f)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["road_4096_seed3", "rmat_s22_ef16_seed2"])
def test_full_size_workloads(ctx, name):
    # full-size paper-shaped inputs against the stored oracle results, in the
    # launch configuration the benchmark times (persistent, threshold 0.6)
    exp = _expected()[name]
    rp, cl = graphgen.workload(name)
    assert graphgen.graph_hash(rp, cl) == exp["graph_hash"], "input changed"
    got, st, tr = gpu_color(ctx, rp, cl, trace_rounds=exp["rounds"] + 4, validate=False)
    assert hashlib.sha256(got.astype("<i4").tobytes()).hexdigest() == exp["colors_sha256"]
    assert st.rounds == exp["rounds"] and st.num_colors == exp["num_colors"]
    assert tr["wl_size"].tolist() == exp["wl_sizes"]
    assert tr["deg_sum"].tolist() == exp["deg_sums"]
    # the same through the host loop driver and forced modes
    for kw in (dict(mode="data"), dict(mode="topo"), dict(driver="hostloop"),
               dict(forbidden="rescan")):
        got2, st2 = gpu_color(ctx, rp, cl, validate=False, **kw)
        assert np.array_equal(got2, got) and st2.rounds == st.rounds


@pytest.mark.parametrize("graph", ["rmat", "road", "er"])
def test_worklist_rebuild(ctx, graph, er_graph):
    # the discard-and-rebuild hybrid (Section I) gives the same colours: for
    # every threshold, mode and bucket split
    rp, cl = {"rmat": lambda: graphgen.rmat(14, 16, seed=22), "road": lambda: graphgen.road(300, seed=23),
              "er": lambda: er_graph}[graph]()
    ref = oracle.color(rp, cl)
    for frac in (0.6, 0.2, 0.0, 1.0):
        for mode in ("threshold", "topo", "data"):
            assert_parity(ctx, rp, cl, ref, mode=mode, threshold_frac=frac, worklist="rebuild")
    for t1, chunk in ((1, 32), (63, 4096), (8, 100)):
        assert_parity(ctx, rp, cl, ref, t1=t1, chunk=chunk, threshold_frac=0.3, worklist="rebuild")


def band_network(lo, hi, k=200.0):
    """A learned-switch network (8 -> 16 -> 16 -> 1) that says 'topology' iff
    the largest colour lies in a band: feature 7 = maxc / (maxc + 64) in
    (lo, hi). Layer 1: tanh(k (f7 - lo)), tanh(k (f7 - hi)); layer 2:
    tanh((h0 - h1) / 2); output 10 (h2 - 0.38)."""
    w = np.zeros(433, np.float32)
    W1, B1, W2, B2, W3, B3 = 0, 128, 144, 400, 416, 432
    w[W1 + 0 * 8 + 7], w[B1 + 0] = k, -k * lo
    w[W1 + 1 * 8 + 7], w[B1 + 1] = k, -k * hi
    w[W2 + 0 * 16 + 0], w[W2 + 0 * 16 + 1] = 0.5, -0.5
    w[W3 + 0], w[B3] = 10.0, -3.8
    return w


def test_worklist_rebuild_many_switches(ctx):
    # topology-driven rounds in a band of colours in the middle of the run:
    # topology (round 1), data (rebuild), topology (discard), data (rebuild)
    import torch

    from paper_1912_01478_gb300 import ipgc, policy

    rp, cl = graphgen.rmat(14, 16, seed=24)
    ref = oracle.color(rp, cl)
    lo, hi = 20 / 84, 40 / 104  # maxc in (20, 40)
    policy.load(ctx, band_network(lo, hi))
    try:
        drp, dcl = to_dev(rp, cl)
        tr = ipgc.trace_buffer(ref.rounds + 2)
        for wl in ("rebuild", "keep"):
            colors, st = ctx.color(drp, dcl, trace=tr,
                                   options=ipgc.ColorOptions(mode="learned", worklist=wl))
            assert np.array_equal(colors.cpu().numpy(), ref.colors) and st.rounds == ref.rounds
            modes = ipgc.read_trace(tr, st.rounds)["mode"]
            switches = int(np.sum(modes[1:] != modes[:-1]))
            assert switches >= 3, modes  # topo -> data -> topo -> data at least
    finally:
        policy.load(ctx, None)


def test_worklist_rebuild_needs_the_persistent_driver(ctx):
    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.er(500, 1500, seed=5)
    with pytest.raises(ipgc.IpgcError) as ei:
        gpu_color(ctx, rp, cl, worklist="rebuild", driver="hostloop")
    assert ei.value.code == ipgc.IPGC_ERR_UNSUPPORTED
