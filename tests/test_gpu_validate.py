"""The device CSR check (ipgc_validate_csr with on_device = 1) accepts exactly
the inputs the method is defined on: the undirected graph of Section II-A
(symmetric CSR) with Section V's self-loops and multi-edges removed, in the
layout the kernels read (rowptr from 0 to nnz, non-decreasing; entries in
range; rows strictly ascending).

Every verdict is compared with a plain numpy statement of those rules on the
same arrays. The mutations cover each rule, and for symmetry both ways a
missing reverse can show: the entry that would find it is the one that
searches (a failed lookup), or the other one (only the count of searched
entries can show it). Sizes span many warp tiles of the edge-balanced layout
and ragged ends (a hub row across tiles, runs of empty rows)."""
import numpy as np
import pytest

from paper_1912_01478_gb300 import graphgen

pytestmark = pytest.mark.gpu


def reference_ok(rp, cl) -> bool:
    """The rules, written out with numpy (no shortcuts)."""
    rp = np.asarray(rp, np.int64)
    cl = np.asarray(cl, np.int64)
    n, nnz = rp.size - 1, cl.size
    if rp[0] != 0 or rp[-1] != nnz or np.any(np.diff(rp) < 0) or rp.min() < 0 or rp.max() > nnz:
        return False
    if nnz == 0:
        return True
    if cl.min() < 0 or cl.max() >= n:
        return False
    src = np.repeat(np.arange(n), np.diff(rp))
    if np.any(src == cl):
        return False
    same_row = src[1:] == src[:-1]
    if np.any(same_row & (cl[1:] <= cl[:-1])):
        return False
    fwd = set(zip(src.tolist(), cl.tolist()))
    return all((u, v) in fwd for v, u in fwd)


def entries(rp):
    n = rp.size - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))


def from_entries(n, src, dst):
    """CSR of directed entries given as (src, dst), rows sorted (no dedup)."""
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp).astype(np.int32), dst.astype(np.int32)


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    return ipgc.Context(0)


def dev_check(ctx, rp, cl):
    import torch

    from paper_1912_01478_gb300 import ipgc

    d_rp = torch.from_numpy(np.ascontiguousarray(rp, np.int32)).cuda()
    d_cl = torch.from_numpy(np.ascontiguousarray(cl, np.int32)).cuda()
    rc = ctx.validate(d_rp, d_cl)
    assert rc in (ipgc.IPGC_OK, ipgc.IPGC_ERR_INVALID)
    return rc == ipgc.IPGC_OK


GRAPHS = {
    "er": lambda: graphgen.er(3000, 9000, seed=41),
    "rmat": lambda: graphgen.rmat(13, 16, seed=42),  # hubs over many tiles, isolated runs
    "star": lambda: graphgen.from_edges(5000, np.zeros(4999, np.int32),
                                        np.arange(1, 5000, dtype=np.int32)),
    "road": lambda: graphgen.road(60, seed=43),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_valid_graphs_pass(ctx, name):
    rp, cl = GRAPHS[name]()
    assert reference_ok(rp, cl)
    assert dev_check(ctx, rp, cl)


def test_degenerate_inputs(ctx):
    # edgeless, one node, and a single edge
    for rp, cl in [(np.zeros(6, np.int32), np.zeros(0, np.int32)),
                   (np.zeros(2, np.int32), np.zeros(0, np.int32)),
                   (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))]:
        assert reference_ok(rp, cl) and dev_check(ctx, rp, cl)
    # a one-way single entry
    rp, cl = np.array([0, 1, 1], np.int32), np.array([1], np.int32)
    assert not reference_ok(rp, cl) and not dev_check(ctx, rp, cl)


@pytest.mark.parametrize("name", ["er", "rmat", "star"])
def test_missing_reverse_either_side(ctx, name):
    # drop one directed entry: its reverse then has no partner; whether the
    # remaining entry is the one that searches depends on the degrees, so
    # entries at both ends of hub-leaf and leaf-hub pairs are dropped
    rp, cl = GRAPHS[name]()
    src = entries(rp)
    deg = np.diff(rp).astype(np.int64)
    rng = np.random.default_rng(7)
    hub_side = np.flatnonzero(deg[src] > deg[cl])
    leaf_side = np.flatnonzero(deg[src] < deg[cl])
    picks = list(rng.choice(hub_side, 3, replace=False)) if hub_side.size >= 3 else []
    picks += list(rng.choice(leaf_side, 3, replace=False)) if leaf_side.size >= 3 else []
    picks += list(rng.choice(src.size, 3, replace=False))
    for e in picks:
        keep = np.ones(src.size, bool)
        keep[e] = False
        r2, c2 = from_entries(rp.size - 1, src[keep], cl[keep].astype(np.int64))
        assert not reference_ok(r2, c2)
        assert not dev_check(ctx, r2, c2), int(e)


@pytest.mark.parametrize("name", ["er", "rmat"])
def test_redirected_entry(ctx, name):
    # one entry (u, v) replaced by (u, w) with w not a neighbour of u: the
    # entry count stays even and every row stays sorted and simple
    rp, cl = GRAPHS[name]()
    n = rp.size - 1
    src = entries(rp)
    rng = np.random.default_rng(11)
    for e in rng.choice(src.size, 6, replace=False):
        u = int(src[e])
        row = set(cl[rp[u]:rp[u + 1]].tolist())
        w = int(rng.integers(0, n))
        while w == u or w in row:
            w = int(rng.integers(0, n))
        dst = cl.astype(np.int64).copy()
        dst[e] = w
        r2, c2 = from_entries(n, src, dst)
        assert not reference_ok(r2, c2)
        assert not dev_check(ctx, r2, c2), int(e)


def test_layout_rule_violations(ctx):
    rp, cl = graphgen.rmat(12, 16, seed=44)
    n = rp.size - 1
    rng = np.random.default_rng(13)
    deg = np.diff(rp)
    big = int(np.argmax(deg))
    cases = []
    c = cl.copy()
    c[rp[big] + 5] = n  # out of range
    cases.append((rp, c))
    c = cl.copy()
    c[rp[big] + 3] = -1  # negative
    cases.append((rp, c))
    c = cl.copy()
    c[rp[big] + 2] = big  # self-loop
    cases.append((rp, c))
    c = cl.copy()
    k = rp[big] + 7
    c[k], c[k + 1] = c[k + 1], c[k]  # unsorted row
    cases.append((rp, c))
    c = cl.copy()
    k = rp[big] + 9
    c[k + 1] = c[k]  # duplicate entry
    cases.append((rp, c))
    r = rp.copy()
    r[n // 2] = r[n // 2 + 1] + 1  # rowptr decreasing
    cases.append((r, cl))
    r = rp.copy()
    r[0] = 1  # does not start at 0
    cases.append((r, cl))
    cases.append((rp, cl[:-1]))  # rowptr[n] != nnz
    for r, c in cases:
        assert not reference_ok(r, c)
        assert not dev_check(ctx, r, c)
    # random single-entry corruptions, each judged like the reference
    for _ in range(10):
        c = cl.copy()
        k = int(rng.integers(0, c.size))
        c[k] = int(rng.integers(-2, n + 2))
        assert dev_check(ctx, rp, c) == reference_ok(rp, c)


def test_repeated_checks_reset_their_state(ctx):
    # the count of searched entries is reset by the check itself, so valid,
    # invalid and valid graphs in a row each get their own verdict
    good = GRAPHS["rmat"]()
    rp, cl = good
    src = entries(rp)
    r2, c2 = from_entries(rp.size - 1, src[1:], cl[1:].astype(np.int64))
    for g, want in [(good, True), ((r2, c2), False), (good, True), (good, True)]:
        assert dev_check(ctx, *g) == want
