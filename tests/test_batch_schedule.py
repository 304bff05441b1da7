"""Gang schedule of batched colouring (host logic, no GPU): team sizes,
aligned CTA blocks, a job order under which every team meets at its barriers,
and a makespan within the list-scheduling bound."""
import numpy as np
import pytest

from paper_1912_01478_gb300 import _build


@pytest.fixture(scope="module")
def batched():
    _build.build()
    from paper_1912_01478_gb300 import batched

    return batched


def shapes(G, seed, heavy=0.05):
    rng = np.random.default_rng(seed)
    n = rng.integers(1, 60_000, G).astype(np.int32)
    nnz = (n.astype(np.int64) * rng.integers(1, 16, G)).astype(np.int64)
    big = rng.random(G) < heavy
    n[big] = rng.integers(200_000, 2_000_000, big.sum())
    nnz[big] = n[big].astype(np.int64) * 16
    n[rng.random(G) < 0.03] = 0
    nnz[n == 0] = 0
    return n, nnz


def expected_team(nnz, n, grid, max_team, npc):
    """Smallest power of two covering nnz / npc, else the cap."""
    cap = max_team if 0 < max_team < grid else grid
    if n == 0:
        return 0
    need = -(-int(nnz) // npc)
    k = 1
    while k < need:
        k *= 2
    return min(k, cap)


@pytest.mark.parametrize("grid,max_team,npc", [(456, 0, 131072), (228, 16, 65536), (304, 0, 1),
                                               (456, 4, 1 << 40), (7, 0, 1000)])
def test_plan_properties(batched, grid, max_team, npc):
    n, nnz = shapes(600, seed=grid + max_team)
    team, first, seq = batched.plan(n, nnz, grid, max_team, npc)
    G = n.size
    for g in range(G):
        k = expected_team(nnz[g], n[g], grid, max_team, npc)
        assert team[g] == k, g
        if k >= 2:
            assert first[g] % k == 0 and 0 <= first[g] and first[g] + k <= grid
        else:
            assert first[g] == -1
        assert (seq[g] < 0) == (k == 0)
    # the single-CTA queue: a permutation, largest work first
    solo = np.flatnonzero(team == 1)
    q = solo[np.argsort(seq[solo])]
    assert sorted(seq[solo]) == list(range(solo.size))
    w = (n.astype(np.int64) + nnz)[q]
    assert np.all(w[:-1] >= w[1:])
    # the teams: one gang order, larger teams first
    tg = np.flatnonzero(team >= 2)
    order = tg[np.argsort(seq[tg])]
    assert sorted(seq[tg]) == list(range(tg.size))
    assert np.all(team[order][:-1] >= team[order][1:])
    # every CTA runs its team jobs in the gang order; executing any job whose
    # CTAs all have it at the head of their lists must finish every job (no
    # two teams wait on each other)
    lists = [[] for _ in range(grid)]
    for g in order:
        for c in range(first[g], first[g] + team[g]):
            lists[c].append(g)
    head = [0] * grid
    left = tg.size
    progress = True
    while left and progress:
        progress = False
        for g in order:
            cs = range(first[g], first[g] + team[g])
            if all(head[c] < len(lists[c]) and lists[c][head[c]] == g for c in cs):
                for c in cs:
                    head[c] += 1
                left -= 1
                progress = True
    assert left == 0
    # list scheduling on aligned blocks: the blocks of size k are evenly
    # loaded when a team of k is placed (larger teams came first), so it
    # starts no later than the mean load of the CTAs its blocks cover, and
    # finishes within total / (that many CTAs) + its own duration
    load = np.zeros(grid)
    total = sum((int(n[g]) + int(nnz[g])) for g in tg)
    for g in order:
        k = int(team[g])
        cs = slice(first[g], first[g] + k)
        assert np.all(load[cs] == load[cs][0])
        dur = (int(n[g]) + int(nnz[g])) / k
        load[cs] = load[cs][0] + dur
        usable = (grid // k) * k
        assert load[cs][0] <= total / usable + dur + 1e-6


def test_plan_rejects_bad_arguments(batched):
    from paper_1912_01478_gb300 import ipgc

    n = np.array([10, 20], np.int32)
    nnz = np.array([30, 40], np.int64)
    for kw in (dict(grid=0), dict(grid=8, max_team=-1), dict(grid=8, nnz_per_cta=0)):
        with pytest.raises(ipgc.IpgcError) as ei:
            batched.plan(n, nnz, **kw)
        assert ei.value.code == ipgc.IPGC_ERR_INVALID
    with pytest.raises(ipgc.IpgcError):
        batched.plan(np.array([-1], np.int32), np.array([0], np.int64), 8)
    team, first, seq = batched.plan(np.zeros(0, np.int32), np.zeros(0, np.int64), 8)
    assert team.size == 0
