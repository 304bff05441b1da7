"""The allocation-free entry point gives the same colouring as ipgc_color_ex
and as the CPU oracle.

ipgc_color_noalloc serves callers that cannot allocate device memory when
they need a colouring (code inside an allocator or memory-pool callback,
which must not re-enter the allocator, or a service working within a budget
reserved in advance); it works in one fixed device array inside the library.
The GPU tests call it through the C ABI several times in a row, on graphs of
different sizes (a smaller graph after a larger one, so state left over from
an earlier call in the shared array would show), and compare colours, rounds
and colour count with the context-based entry point and with the oracle:
  - two mid-size graphs, one with hubs above the work-item size;
  - graphs of exactly the largest size the fixed array takes, built so that
    the number of nodes above the low-degree bound, of work items and of
    multi-item nodes come close to the bounds the array is laid out for;
  - a call without a statistics record (the device's status is still
    returned) and a malformed graph (rejected by the validation).
The size checks run first and need no GPU. This file is collected last on
purpose.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen


def test_noalloc_rejects_graphs_above_its_limits():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    st = ipgc.Stats()
    big_n = ipgc.NOALLOC_MAX_N + 1
    rc = ipgc.lib().ipgc_color_noalloc(1, 1, big_n, 0, 1, ctypes.byref(st), None)
    assert rc == ipgc.IPGC_ERR_TOO_LARGE
    rc = ipgc.lib().ipgc_color_noalloc(1, 1, 10, ipgc.NOALLOC_MAX_NNZ + 1, 1, ctypes.byref(st), None)
    assert rc == ipgc.IPGC_ERR_TOO_LARGE
    rc = ipgc.lib().ipgc_color_noalloc(None, None, -1, 0, None, None, None)
    assert rc == ipgc.IPGC_ERR_INVALID


def test_noalloc_array_has_the_documented_size():
    # the header states the fixed array's size; the library's host-side
    # stand-in of the device array has the array's type, so its symbol size
    # is the array's size
    from paper_1912_01478_gb300 import _build

    _build.build()
    out = subprocess.run(["nm", "-S", "-C", _build.LIB], capture_output=True, text=True,
                         check=True).stdout
    sizes = [int(line.split()[1], 16) for line in out.splitlines()
             if line.endswith("g_noalloc_scratch")]
    assert sizes == [15_074_048], sizes
    with open(os.path.join(_build.INCLUDE, "ipgc.h")) as f:
        assert "15,074,048" in f.read()


def complete_bipartite_blocks(blocks):
    """Edges of disjoint complete bipartite graphs K_{a,a}; blocks = [(count, a)]."""
    src, dst, base = [], [], 0
    for count, a in blocks:
        left = np.repeat(np.arange(a), a)
        right = np.tile(np.arange(a), a) + a
        for _ in range(count):
            src.append(base + left)
            dst.append(base + right)
            base += 2 * a
    return np.concatenate(src), np.concatenate(dst), base


def capacity_graph(blocks, seed):
    """A graph of exactly IPGC_NOALLOC_MAX_N nodes and IPGC_NOALLOC_MAX_NNZ
    entries: the given K_{a,a} blocks, then a matching that fills the
    entries up to the limit, IDs permuted at random over all nodes."""
    from paper_1912_01478_gb300 import ipgc

    n, nnz = ipgc.NOALLOC_MAX_N, ipgc.NOALLOC_MAX_NNZ
    src, dst, used = complete_bipartite_blocks(blocks)
    rest = nnz - 2 * src.size
    assert rest >= 0 and rest % 2 == 0
    m = np.arange(rest // 2)
    src = np.concatenate([src, used + 2 * m])
    dst = np.concatenate([dst, used + 2 * m + 1])
    assert used + rest <= n
    perm = np.random.default_rng(seed).permutation(n)
    rp, cl = graphgen.from_edges(n, perm[src], perm[dst])
    assert rp.size - 1 == n and cl.size == nnz
    return rp, cl


def noalloc(rp_d, cl_d, n, nnz, out, with_stats=True):
    from paper_1912_01478_gb300 import ipgc

    st = ipgc.Stats()
    rc = ipgc.lib().ipgc_color_noalloc(rp_d.data_ptr(), cl_d.data_ptr() if nnz else None, n, nnz,
                                       out.data_ptr(), ctypes.byref(st) if with_stats else None,
                                       None)
    return rc, st


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    c = ipgc.Context(0)
    yield c
    c.close()


def check_against_both(ctx, rp, cl, with_stats=True):
    import torch

    from paper_1912_01478_gb300 import ipgc

    n, nnz = rp.size - 1, cl.size
    assert n <= ipgc.NOALLOC_MAX_N and nnz <= ipgc.NOALLOC_MAX_NNZ
    drp = torch.from_numpy(rp).cuda()
    dcl = torch.from_numpy(cl).cuda()
    ref, st_ref = ctx.color(drp, dcl)
    orc = oracle.color(rp, cl, trace=False)
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rc, st = noalloc(drp, dcl, n, nnz, out, with_stats)
    assert rc == ipgc.IPGC_OK, ipgc.lib().ipgc_strerror(rc)
    got = out.cpu().numpy()
    assert np.array_equal(got, ref.cpu().numpy())
    assert np.array_equal(got, orc.colors)
    if with_stats:
        assert st.rounds == st_ref.rounds == orc.rounds
        assert st.num_colors == st_ref.num_colors == orc.num_colors
        assert st.rounds_topo == st_ref.rounds_topo and st.rounds_data == st_ref.rounds_data
        assert st.error == 0


@pytest.mark.gpu
def test_noalloc_matches_context_entry_point_twice(ctx):
    for rp, cl in [graphgen.rmat(17, 16, seed=31),  # hubs above the chunk size: multi-item nodes
                   graphgen.er(20_000, 90_000, seed=32)]:
        check_against_both(ctx, rp, cl)


@pytest.mark.gpu
def test_noalloc_at_its_size_limits(ctx):
    # nodes of degree 65 (just above the low-degree bound 64): about as many
    # as the array's high-degree room (nnz / 65); then nodes of degree 1025
    # (two work items each, just above the item size) beside them
    many_big = capacity_graph([(992, 65)], seed=33)
    multi_item = capacity_graph([(3, 1025), (246, 65)], seed=34)
    for rp, cl in (many_big, multi_item):
        check_against_both(ctx, rp, cl)


@pytest.mark.gpu
def test_noalloc_without_stats_and_on_a_malformed_graph(ctx):
    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.rmat(14, 16, seed=35)
    check_against_both(ctx, rp, cl, with_stats=False)
    # an empty graph: nothing to do, no error
    empty = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, _ = noalloc(empty, empty, 0, 0, empty)
    assert rc == ipgc.IPGC_OK
    # one direction of an edge removed: asymmetric, rejected before colouring
    bad = cl.copy()
    k = int(rp[int(np.argmax(np.diff(rp)))])
    bad[k] = (bad[k] + 1) % (rp.size - 1)
    drp = torch.from_numpy(rp).cuda()
    dcl = torch.from_numpy(bad).cuda()
    out = torch.zeros(rp.size - 1, dtype=torch.int32, device="cuda")
    for with_stats in (True, False):
        rc, _ = noalloc(drp, dcl, rp.size - 1, bad.size, out, with_stats)
        assert rc == ipgc.IPGC_ERR_INVALID
    # and the array is still usable after the rejected calls
    check_against_both(ctx, *graphgen.er(5_000, 20_000, seed=36))
