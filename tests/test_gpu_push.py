"""Section III micro-benchmark on the GPU: every iteration's worklist (its
size and the sum of its IDs) equals the oracle's for Push_WL, Push_NoWL and
the hybrid, which switches from the topology-driven to the data-driven
kernel by worklist size; at the europe_osm size (n = 50.9 M, COUNT = 1000)
the records are checked against the closed forms the oracle tests pin."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    return ipgc.Context(0)


CASES = [(1, 1000), (999, 1000), (1000, 1000), (1001, 1000), (123_457, 1000), (5_000, 1),
         (300_000, 4096), (4_096 * 37 + 5, 7)]


@pytest.mark.parametrize("n,count", CASES)
def test_push_kernels_match_oracle(ctx, n, count):
    it_ref, sizes, sums = oracle.push_run(n, count, "wl")
    for mode, switch in (("wl", 0), ("nowl", 0), ("hybrid", n // 2), ("hybrid", 0), ("hybrid", n)):
        it, rec = ctx.push_bench(n, count, mode, switch)
        assert it == it_ref, (mode, switch)
        assert np.array_equal(rec[:, 0], sizes), (mode, switch)
        assert np.array_equal(rec[:, 1], sums), (mode, switch)
        assert np.all(rec[:, 3] > 0)
        # the kernel each iteration used: the topology-driven one while the
        # worklist it starts from is above the switch size
        before = np.concatenate([[n], sizes[:-1]])
        want = {"wl": np.zeros(it, bool), "nowl": np.ones(it, bool),
                "hybrid": before > switch}[mode]
        assert np.array_equal(rec[:, 2] == 1, want), (mode, switch)


def test_empty_and_invalid(ctx):
    from paper_1912_01478_gb300 import ipgc

    assert ctx.push_bench(0, 1000, "wl") == (0, None)
    for kw in (dict(n=10, count=0), dict(n=-1, count=10)):
        with pytest.raises(ipgc.IpgcError) as ei:
            ctx.push_bench(kw["n"], kw["count"], "wl")
        assert ei.value.code == ipgc.IPGC_ERR_INVALID


def test_europe_osm_size(ctx):
    # n = 50,912,018 (europe_osm's node count), COUNT = 1000: 50,913 iterations
    n, count = 50_912_018, 1000
    for mode, switch in (("nowl", 0), ("wl", 0), ("hybrid", n // 4)):
        it, rec = ctx.push_bench(n, count, mode, switch)
        assert it == -(-n // count)
        a = count * (np.arange(it, dtype=np.int64) + 1)
        m = np.maximum(n - a, 0)
        assert np.array_equal(rec[:, 0], m)
        assert np.array_equal(rec[:, 1], np.where(m > 0, m * (a + n - 1) // 2, 0))
