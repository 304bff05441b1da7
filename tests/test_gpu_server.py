"""Colouring server: continuous batching gives every request the colouring
it gets alone (the CPU oracle's), whatever else is in flight, with
forbidden-colour bitmaps (the default) and with rescanning; admission by
device memory, slot reuse, errors."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen

pytestmark = pytest.mark.gpu


def pool(k, seed, nmax=60_000):
    bt = graphgen.batch(k, seed=seed, nmin=100, nmax=nmax)
    return [tuple(np.ascontiguousarray(a) for a in graphgen.batch_graph(bt, g)) for g in range(k)]


@pytest.fixture(scope="module")
def graphs():
    gs = pool(40, seed=5)
    gs.append(graphgen.rmat(16, 16, seed=6))  # one large request (teams)
    refs = [oracle.color(rp, cl, trace=False) for rp, cl in gs]
    return gs, refs


def check(res, ref):
    colors, st, lat = res
    assert np.array_equal(colors, ref.colors)
    assert st.rounds == ref.rounds and st.num_colors == ref.num_colors and st.error == 0
    assert lat > 0


@pytest.mark.parametrize("forbidden", ["auto", "rescan"])
def test_results_same_alone_and_in_the_mix(graphs, forbidden):
    # the default server colours with forbidden-colour bitmaps (graphs
    # without a node above t1 rescan in the same launch); "rescan" rereads
    # rows in every launch
    from paper_1912_01478_gb300 import _build, ipgc, server

    _build.build()
    gs, refs = graphs
    o = server.options(inflight=2, max_batch_graphs=8)
    o.batch.base.forbidden = ipgc.FORBIDDEN[forbidden]
    srv = server.Server(0, o)
    # alone: one request at a time
    alone = []
    for rp, cl in gs[:6]:
        t = srv.submit(rp, cl)
        while (r := srv.poll(t)) is None:
            time.sleep(0.0005)
        alone.append(r)
    for r, ref in zip(alone, refs[:6]):
        check(r, ref)
    # in the mix: everything at once from two submitting threads, results
    # polled in completion order; small batches force several overlapping ones
    tickets = [None] * len(gs)

    def submit_range(lo, hi):
        for i in range(lo, hi):
            tickets[i] = srv.submit(*gs[i])

    th = [threading.Thread(target=submit_range, args=(0, 20)),
          threading.Thread(target=submit_range, args=(20, len(gs)))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = {}
    deadline = time.time() + 60
    while len(got) < len(gs) and time.time() < deadline:
        t = srv.next_done(timeout_s=1.0)
        if t is not None:
            got[t] = srv.poll(t)
    assert len(got) == len(gs)
    for i, t in enumerate(tickets):
        check(got[t], refs[i])
    c = srv.counters()
    assert c.batches >= 2 and c.completed == c.submitted and c.hbm_used == 0 and c.status == 0
    srv.close()


def test_admission_by_device_memory(graphs):
    # a budget that holds only a couple of requests at a time: the rest wait
    # in the queue and are admitted as memory frees up
    from paper_1912_01478_gb300 import server

    gs, refs = graphs
    small = gs[:30]
    srv = server.Server(0, server.options(hbm_budget=24 << 20, inflight=2, max_batch_graphs=4))
    tickets = [srv.submit(rp, cl) for rp, cl in small]
    for t, ref in zip(tickets, refs[:30]):
        while (r := srv.poll(t)) is None:
            time.sleep(0.0005)
        check(r, ref)
    c = srv.counters()
    assert c.hbm_peak <= 24 << 20 and c.hbm_used == 0 and c.batches >= 8
    srv.close()


def test_errors_and_ticket_reuse(graphs):
    from paper_1912_01478_gb300 import ipgc, server

    gs, refs = graphs
    srv = server.Server(0, server.options(hbm_budget=8 << 20, host_budget=64 << 20))
    rp, cl = graphgen.rmat(17, 16, seed=1)  # needs more than 8 MB on the device
    with pytest.raises(ipgc.IpgcError) as ei:
        srv.submit(rp, cl)
    assert ei.value.code == ipgc.IPGC_ERR_TOO_LARGE
    t = srv.submit(*gs[0])
    while (r := srv.poll(t)) is None:
        time.sleep(0.0005)
    check(r, refs[0])
    with pytest.raises(ipgc.IpgcError) as ei:
        srv.poll(t)  # released
    assert ei.value.code == ipgc.IPGC_ERR_NOT_FOUND
    # an empty graph completes at once
    t0 = srv.submit(np.zeros(1, np.int32), np.zeros(0, np.int32))
    r0 = srv.poll(t0)
    assert r0 is not None and r0[1].rounds == 0
    # destroy with work queued: no hang, no leak of the context
    for rp2, cl2 in gs[:10]:
        srv.submit(rp2, cl2)
    srv.close()


def test_submission_by_reference(graphs):
    import torch

    from paper_1912_01478_gb300 import server

    gs, refs = graphs
    srv = server.Server(0, server.options(inflight=2, max_batch_graphs=16))
    keep = []
    tickets = []
    for rp, cl in gs:
        prp = torch.from_numpy(rp).pin_memory()
        pcl = torch.from_numpy(cl).pin_memory()
        keep.append((prp, pcl))
        tickets.append(srv.submit_ref(prp.numpy(), pcl.numpy()))
    for t, ref in zip(tickets, refs):
        while (r := srv.poll(t)) is None:
            time.sleep(0.0005)
        check(r, ref)
    srv.close()


def test_small_requests_finish_before_a_large_one_in_the_same_launch():
    # with one batch slot, a first request keeps the slot busy while a large
    # graph (on a small team) and many tiny graphs queue up; they then share
    # one launch, and each tiny request completes as soon as its own CTA is
    # done, before the large one, not when the launch ends
    from paper_1912_01478_gb300 import server

    blocker = graphgen.rmat(18, 16, seed=10)
    big = graphgen.rmat(18, 16, seed=11)
    tiny = pool(64, seed=12, nmax=1_500)
    ref_blocker = oracle.color(*blocker, trace=False)
    ref_big = oracle.color(*big, trace=False)
    refs = [oracle.color(rp, cl, trace=False) for rp, cl in tiny]
    o = server.options(inflight=1, max_batch_graphs=256)
    o.batch.max_team = 4
    srv = server.Server(0, o)
    t0 = srv.submit(*blocker)
    time.sleep(0.01)  # let the blocker launch
    tb = srv.submit(*big)
    ts = [srv.submit(rp, cl) for rp, cl in tiny]
    order = []
    done = {}
    deadline = time.time() + 120
    while len(done) < len(ts) + 2 and time.time() < deadline:
        t = srv.next_done(timeout_s=1.0)
        if t is not None:
            order.append(t)
            done[t] = srv.poll(t)
    assert len(done) == len(ts) + 2
    check(done[t0], ref_blocker)
    check(done[tb], ref_big)
    for t, ref in zip(ts, refs):
        check(done[t], ref)
    c = srv.counters()
    srv.close()
    assert c.batches == 2 and c.max_batch == len(ts) + 1
    assert order[0] == t0 and order[-1] == tb


def test_learned_switch_in_the_server(graphs):
    # with the learned mode switch the server's launches ask the loaded
    # network every round: one that always answers "topology-driven" makes
    # every round of every request topology-driven, one that always answers
    # "data-driven" every round after the first; without a network the
    # threshold rule decides; the colours are the oracle's throughout
    from paper_1912_01478_gb300 import ipgc, server

    gs, refs = graphs
    o = server.options(inflight=2, max_batch_graphs=8)
    o.batch.base.mode = ipgc.MODE_LEARNED
    srv = server.Server(0, o)
    with pytest.raises(ipgc.IpgcError) as ei:
        srv.load_policy(np.zeros(10, np.float32))
    assert ei.value.code == ipgc.IPGC_ERR_INVALID
    topo = np.zeros(433, np.float32)
    topo[432] = 10.0  # output bias: p(topology faster) ~ 1
    data = np.zeros(433, np.float32)
    data[432] = -10.0
    wl = [oracle.color(rp, cl).wl_sizes for rp, cl in gs[:12]]
    for w, want in ((None, "threshold"), (topo, "topo"), (data, "data")):
        srv.load_policy(w)
        tickets = [srv.submit(rp, cl) for rp, cl in gs[:12]]
        for t, ref, (rp, cl), sizes in zip(tickets, refs[:12], gs[:12], wl):
            while (r := srv.poll(t)) is None:
                time.sleep(0.0005)
            check(r, ref)
            st = r[1]
            if want == "topo":
                assert st.rounds_topo == st.rounds
            elif want == "data":
                assert st.rounds_topo == min(st.rounds, 1)
            else:
                H = int(np.float64(np.float32(0.6)) * (rp.size - 1))  # the library's floor(0.6f n)
                assert st.rounds_topo == sum(int(x > H) for x in sizes)
    srv.close()
