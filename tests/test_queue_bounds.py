"""The per-round queues of the pushing colouring are sized from n and nnz
alone (the workspace is laid out before the graph is seen): one-window push
items for the rows of winners above t1, one-window units for list rewrites
of nodes with several work items. A window is 128 entries aligned to 16
bytes, so a row of d entries starting at s takes ceil(((s mod 4) + d) / 128)
of them. These checks take every qualifying node at once (the most a round
can queue) on real row layouts and compare with the sizes the library uses:
nnz / 128 + 2 x (nodes above t1) + 1 and nnz / 128 + 2 x (merge-state
slots) + 1."""
import numpy as np

from paper_1912_01478_gb300 import graphgen

WINDOW = 128


def windows(rp, sel):
    s = rp[:-1][sel].astype(np.int64)
    d = np.diff(rp)[sel].astype(np.int64)
    return int((((s & 3) + d + WINDOW - 1) // WINDOW).sum())


def graphs():
    yield graphgen.rmat(14, 16, seed=61)
    yield graphgen.rmat(13, 32, seed=62)
    yield graphgen.er(20_000, 200_000, seed=63)
    yield graphgen.hubs(20_000, 60_000, 40, 15_000, 1.0, seed=64)  # a few very long rows


def test_push_and_rewrite_queues_hold_a_worst_round():
    for rp, cl in graphs():
        n, nnz = rp.size - 1, cl.size
        deg = np.diff(rp)
        for t1 in (16, 64):
            nbig = min(n, nnz // (t1 + 1))
            assert int((deg > t1).sum()) <= nbig
            assert windows(rp, deg > t1) <= nnz // WINDOW + 2 * nbig + 1
        for chunk in (512, 1024):
            slots = nnz // (chunk + 1) + 1
            assert int((deg > chunk).sum()) <= slots
            assert windows(rp, deg > chunk) <= nnz // WINDOW + 2 * slots + 1
