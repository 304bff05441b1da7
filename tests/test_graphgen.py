"""Seeded generators: structure, determinism and recorded hashes (CPU)."""
import numpy as np
import pytest

from paper_1912_01478_gb300 import graphgen


def check_simple_symmetric(rp, cl):
    n = rp.size - 1
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == cl.size
    if cl.size == 0:
        return
    assert cl.min() >= 0 and cl.max() < n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    assert not np.any(src == cl), "self-loop"
    # rows strictly ascending (sorted, no duplicates)
    same_row = src[1:] == src[:-1]
    assert np.all(cl[1:][same_row] > cl[:-1][same_row])
    # symmetric: the multiset of (u, v) equals that of (v, u)
    a = np.sort(src * n + cl)
    b = np.sort(cl.astype(np.int64) * n + src)
    assert np.array_equal(a, b)


def test_er_shape_and_determinism():
    rp, cl = graphgen.er(10_000, 40_000, seed=1)
    check_simple_symmetric(rp, cl)
    assert cl.size == 80_000
    rp2, cl2 = graphgen.er(10_000, 40_000, seed=1)
    assert np.array_equal(rp, rp2) and np.array_equal(cl, cl2)
    rp3, _ = graphgen.er(10_000, 40_000, seed=2)
    assert not np.array_equal(rp, rp3)


def test_er_hash_recorded():
    # FNV-1a of the ER n=10^4, m=4*10^4, seed-1 workload (rowptr then col)
    rp, cl = graphgen.er(10_000, 40_000, seed=1)
    assert graphgen.graph_hash(rp, cl) == 10912466498579925223


def test_rmat_small():
    rp, cl = graphgen.rmat(12, 16, seed=2)
    check_simple_symmetric(rp, cl)
    assert rp.size == 4097
    deg = np.diff(rp)
    assert deg.max() > 20 * max(np.median(deg), 1)  # skewed degrees


def test_rmat_n_limit_and_thread_independence():
    rp, cl = graphgen.rmat(10, 8, seed=9, n_limit=700)
    check_simple_symmetric(rp, cl)
    assert rp.size == 701


def test_road_small():
    rp, cl = graphgen.road(64, seed=3)
    check_simple_symmetric(rp, cl)
    n = 64 * 64
    assert rp.size == n + 1
    avg = cl.size / n
    assert 2.5 < avg < 3.1  # 4 * 0.7 * (1 - 1/side) * 1.01


def test_from_edges_dedups():
    rp, cl = graphgen.from_edges(4, [0, 1, 1, 2, 3], [1, 0, 1, 3, 2])
    assert rp.tolist() == [0, 1, 2, 3, 4]
    assert cl.tolist() == [1, 0, 3, 2]


def test_batch_small():
    bt = graphgen.batch(12, seed=4, nmin=100, nmax=2000)
    no, eo = bt["node_off"], bt["edge_off"]
    assert no.size == 13 and eo.size == 13
    for g in range(12):
        rp, cl = graphgen.batch_graph(bt, g)
        assert 100 <= rp.size - 1 <= 2000
        check_simple_symmetric(rp, cl)
    bt2 = graphgen.batch(12, seed=4, nmin=100, nmax=2000)
    assert np.array_equal(bt["col_cat"], bt2["col_cat"])
