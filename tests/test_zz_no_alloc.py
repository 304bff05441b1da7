"""The allocation-free entry point gives the same colouring as ipgc_color_ex.

ipgc_color_noalloc serves callers that cannot allocate device memory when
they need a colouring (inside an allocator callback, under a budget reserved
in advance); it works in one fixed device array inside the library. This test
calls it through the C ABI twice in a row, on two different graphs (the
second smaller than the first, so state left over from the first call in the
shared array would show), and compares colours, rounds and colour count with
the context-based entry point. The size check runs first and needs no GPU.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.gpu
def test_noalloc_matches_context_entry_point_twice():
    import torch

    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    ctx = ipgc.Context(0)
    graphs = [
        graphgen.rmat(17, 16, seed=31),  # hubs above the chunk size: multi-item nodes
        graphgen.er(20_000, 90_000, seed=32),
    ]
    for rp, cl in graphs:
        n, nnz = rp.size - 1, cl.size
        assert n <= ipgc.NOALLOC_MAX_N and nnz <= ipgc.NOALLOC_MAX_NNZ
        drp = torch.from_numpy(rp).cuda()
        dcl = torch.from_numpy(cl).cuda()
        ref, st_ref = ctx.color(drp, dcl)
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st = ipgc.Stats()
        rc = ipgc.lib().ipgc_color_noalloc(
            drp.data_ptr(), dcl.data_ptr(), n, nnz, out.data_ptr(), ctypes.byref(st), None
        )
        assert rc == ipgc.IPGC_OK, ipgc.lib().ipgc_strerror(rc)
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
        assert st.rounds == st_ref.rounds and st.num_colors == st_ref.num_colors
        assert st.error == 0
    ctx.close()
