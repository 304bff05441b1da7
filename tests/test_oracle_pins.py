"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself:
  * hand-worked examples (tests/golden/handworked_*.txt, derived on paper
    from Section II-C);
  * closed forms derived by hand from Section II-C for edgeless, complete,
    star, path and complete bipartite graphs;
  * brute force: the exact chromatic number of every labelled graph on up
    to 5 nodes (and random graphs on 6..8 nodes) is a lower bound on the
    colour count;
  * invariants that any correct IPGC run has (Section II-C): a proper
    colouring, colours in 1..max degree + 1, the first-fit property (every
    smaller colour appears on a neighbour), a worklist that shrinks every
    round, round-1 winners are exactly the nodes below all their neighbours,
    and the colour count equals the number of distinct colours;
  * the micro-benchmark iteration count ceil(n / COUNT) (Section III text).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_from_edges(n, edges):
    if edges:
        src = np.array([e[0] for e in edges], np.int32)
        dst = np.array([e[1] for e in edges], np.int32)
    else:
        src = dst = np.zeros(0, np.int32)
    return graphgen.from_edges(n, src, dst)


def neighbours(rowptr, col, v):
    return col[rowptr[v] : rowptr[v + 1]]


def check_invariants(rowptr, col, res):
    n = rowptr.size - 1
    colors = res.colors
    if n == 0:
        assert res.rounds == 0 and res.num_colors == 0
        return
    deg = np.diff(rowptr)
    # colours are 1..max degree + 1
    assert colors.min() >= 1
    assert res.num_colors == colors.max() <= deg.max() + 1
    # proper colouring
    src = np.repeat(np.arange(n), deg)
    assert not np.any(colors[src] == colors[col])
    # colour count = number of distinct colours
    assert len(np.unique(colors)) == res.num_colors
    # first-fit: every colour below color(v) appears on a neighbour of v
    for v in range(n):
        nb = set(colors[neighbours(rowptr, col, v)].tolist())
        for c in range(1, colors[v]):
            assert c in nb, (v, c)
    # per-node colour bound: color(v) <= deg(v) + 1
    assert np.all(colors <= deg + 1)
    # worklist shrinks strictly; starts at n; rounds <= n
    wl = res.wl_sizes
    assert wl[0] == n
    assert np.all(np.diff(wl) < 0)
    assert res.rounds == wl.size <= n
    # round-1 winners: nodes with no lower-ID neighbour
    first = np.array(
        [deg[v] == 0 or neighbours(rowptr, col, v).min() > v for v in range(n)]
    )
    assert np.array_equal(res.fin_round == 1, first)


def chromatic_number(n, edges):
    """Exact chromatic number by dynamic programming over vertex subsets."""
    if n == 0:
        return 0
    adj = [0] * n
    for a, b in edges:
        adj[a] |= 1 << b
        adj[b] |= 1 << a
    full = (1 << n) - 1
    indep = [True] * (1 << n)
    for s in range(1, 1 << n):
        low = (s & -s).bit_length() - 1
        rest = s & ~(1 << low)
        indep[s] = indep[rest] and not (adj[low] & rest)
    chi = [0] * (1 << n)
    for s in range(1, 1 << n):
        low = s & -s
        best = n
        sub = s
        while sub:
            if (sub & low) and indep[sub]:
                c = chi[s & ~sub] + 1
                if c < best:
                    best = c
            sub = (sub - 1) & s
        chi[s] = best
    return chi[full]


def load_golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            d[key] = vals
    n = int(d["n"][0])
    edges = [tuple(int(x) for x in e.split("-")) for e in d["edges"]]
    return (
        n,
        edges,
        np.array([int(x) for x in d["colors"]], np.int32),
        int(d["rounds"][0]),
        int(d["num_colors"][0]),
        [int(x) for x in d["wl"]],
    )


@pytest.mark.parametrize("name", ["handworked_g7.txt", "handworked_g8.txt"])
def test_handworked(name):
    n, edges, colors, rounds, k, wl = load_golden(name)
    rp, cl = csr_from_edges(n, edges)
    res = oracle.color(rp, cl)
    assert np.array_equal(res.colors, colors)
    assert res.rounds == rounds
    assert res.num_colors == k
    assert res.wl_sizes.tolist() == wl
    check_invariants(rp, cl, res)


def test_empty_graph():
    res = oracle.color(np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert res.rounds == 0 and res.num_colors == 0 and res.colors.size == 0


@pytest.mark.parametrize("n", [1, 2, 7, 100])
def test_edgeless(n):
    rp, cl = csr_from_edges(n, [])
    res = oracle.color(rp, cl)
    assert np.all(res.colors == 1) and res.rounds == 1 and res.num_colors == 1


@pytest.mark.parametrize("n", [2, 3, 5, 8, 20])
def test_complete_graph(n):
    # one node (the lowest active ID) wins per round; colour(v) = v + 1
    edges = list(itertools.combinations(range(n), 2))
    rp, cl = csr_from_edges(n, edges)
    res = oracle.color(rp, cl)
    assert np.array_equal(res.colors, np.arange(1, n + 1))
    assert res.rounds == n and res.num_colors == n
    check_invariants(rp, cl, res)


@pytest.mark.parametrize("leaves", [1, 4, 50])
def test_star_low_centre(leaves):
    # centre 0 wins round 1 with colour 1; the leaves get colour 2 in round 2
    n = leaves + 1
    rp, cl = csr_from_edges(n, [(0, i) for i in range(1, n)])
    res = oracle.color(rp, cl)
    assert res.colors[0] == 1 and np.all(res.colors[1:] == 2)
    assert res.rounds == 2 and res.num_colors == 2


@pytest.mark.parametrize("leaves", [1, 4, 50])
def test_star_high_centre(leaves):
    # leaves win round 1 with colour 1; the centre gets colour 2 in round 2
    n = leaves + 1
    c = n - 1
    rp, cl = csr_from_edges(n, [(i, c) for i in range(c)])
    res = oracle.color(rp, cl)
    assert np.all(res.colors[:c] == 1) and res.colors[c] == 2
    assert res.rounds == 2 and res.num_colors == 2


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 11, 40])
def test_path_in_id_order(n):
    # 0-1-2-..: round 1 finalises only node 0 (every other node has a lower
    # neighbour with the same tentative colour, even one that itself loses);
    # afterwards two nodes per round. Colours alternate 1, 2, 1, 2, ...
    rp, cl = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    res = oracle.color(rp, cl)
    assert np.array_equal(res.colors, np.array([1 + (i % 2) for i in range(n)], np.int32))
    assert res.rounds == n // 2 + 1
    check_invariants(rp, cl, res)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (5, 4)])
def test_complete_bipartite_blocks(a, b):
    # side {0..a-1} lies below side {a..a+b-1}: side A wins round 1 (colour 1),
    # side B gets colour 2 in round 2
    edges = [(i, a + j) for i in range(a) for j in range(b)]
    rp, cl = csr_from_edges(a + b, edges)
    res = oracle.color(rp, cl)
    assert np.all(res.colors[:a] == 1) and np.all(res.colors[a:] == 2)
    assert res.rounds == 2


@pytest.mark.parametrize("m", [2, 3, 6])
def test_complete_bipartite_interleaved(m):
    # evens vs odds: round 1 finalises only node 0; in round 2 every odd node
    # sees colour 1 (node 0) and takes 2, every even node takes 1; no conflicts
    edges = [(i, j) for i in range(0, 2 * m, 2) for j in range(1, 2 * m, 2)]
    rp, cl = csr_from_edges(2 * m, edges)
    res = oracle.color(rp, cl)
    assert np.array_equal(res.colors, np.array([1 + (i % 2) for i in range(2 * m)], np.int32))
    assert res.rounds == 2
    assert res.wl_sizes.tolist() == [2 * m, 2 * m - 1]


def all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [p for i, p in enumerate(pairs) if mask >> i & 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_small_graphs(n):
    # every labelled simple graph on n nodes: invariants + chi <= K
    for edges in all_graphs(n):
        rp, cl = csr_from_edges(n, edges)
        res = oracle.color(rp, cl)
        check_invariants(rp, cl, res)
        assert chromatic_number(n, edges) <= res.num_colors


def test_random_small_graphs_brute_force():
    rng = np.random.default_rng(12345)
    for _ in range(150):
        n = int(rng.integers(6, 9))
        p = float(rng.uniform(0.1, 0.9))
        edges = [e for e in itertools.combinations(range(n), 2) if rng.random() < p]
        rp, cl = csr_from_edges(n, edges)
        res = oracle.color(rp, cl)
        check_invariants(rp, cl, res)
        assert chromatic_number(n, edges) <= res.num_colors


def test_disjoint_union_is_componentwise():
    # components interact only through edges: colouring a disjoint union
    # (second component's IDs shifted above the first's) equals colouring
    # each component alone, and rounds = the max over components
    rng = np.random.default_rng(7)
    n1, n2 = 30, 25
    e1 = [e for e in itertools.combinations(range(n1), 2) if rng.random() < 0.2]
    e2 = [e for e in itertools.combinations(range(n2), 2) if rng.random() < 0.3]
    r1 = oracle.color(*csr_from_edges(n1, e1))
    r2 = oracle.color(*csr_from_edges(n2, e2))
    ru = oracle.color(*csr_from_edges(n1 + n2, e1 + [(a + n1, b + n1) for a, b in e2]))
    assert np.array_equal(ru.colors, np.concatenate([r1.colors, r2.colors]))
    assert ru.rounds == max(r1.rounds, r2.rounds)


def test_er_workload_invariants(er_graph):
    rp, cl = er_graph
    res = oracle.color(rp, cl)
    check_invariants(rp, cl, res)


def test_micro_benchmark_iterations():
    # Section III: each iteration deactivates the next COUNT IDs, so the
    # worklist empties after ceil(n / COUNT) iterations, |WL| = n - COUNT*(i+1)
    for n, count in [(1, 1000), (999, 1000), (1000, 1000), (1001, 1000), (25_000, 1000)]:
        it, sizes = oracle.push_iterations(n, count, cap=64)
        assert it == -(-n // count)
        k = min(it, 64)
        assert sizes[:k].tolist() == [max(n - count * (i + 1), 0) for i in range(k)]


@pytest.mark.parametrize("mode", ["wl", "nowl"])
def test_push_kernels_closed_form(mode):
    # Section III: both kernels deactivate the same COUNT IDs per iteration, so
    # after iteration i the worklist is {COUNT*(i+1), ..., n-1}: its size and
    # the sum of its IDs are closed forms (a slip such as the listing's strict
    # comparison keeps one extra node per iteration and fails here)
    for n, count in [(0, 1000), (1, 1000), (999, 1000), (1000, 1000), (1001, 1000),
                     (25_000, 1000), (10_007, 7), (5, 1)]:
        it, sizes, sums = oracle.push_run(n, count, mode)
        assert it == -(-n // count)
        for i in range(it):
            a = count * (i + 1)
            m = max(n - a, 0)
            assert sizes[i] == m
            assert sums[i] == (m * (a + n - 1) // 2 if m else 0)


def test_push_kernels_agree():
    # the data-driven and topology-driven kernels do the same work (Section III)
    a = oracle.push_run(12_345, 100, "wl")
    b = oracle.push_run(12_345, 100, "nowl")
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
