"""The stand-ins for the paper's ten graphs (Table I shapes), small
versions: Plain (data-driven), Hybrid and Hybrid with neighbour filtering
(rescanning rows), Hybrid with forbidden-colour bitmaps (the default) and
the worklist rebuild colour each exactly as the CPU oracle does."""
import numpy as np
import pytest

import oracle
from paper_1912_01478_gb300 import graphgen

pytestmark = pytest.mark.gpu

SCALE = {"europe_osm": 0.005, "rgg_n_2_24_s0": 0.005, "indochina-2004": 0.005,
         "Queen_4147": 0.01, "kron_g500-logn21": 0.01, "hollywood-2009": 0.01}


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_01478_gb300 import _build, ipgc

    _build.build()
    return ipgc.Context(0)


@pytest.mark.parametrize("name", list(graphgen.SUITE))
def test_suite_graph_matches_oracle(ctx, name):
    import torch

    from paper_1912_01478_gb300 import ipgc

    rp, cl = graphgen.suite_graph(name, SCALE.get(name, 0.02))
    ref = oracle.color(rp, cl, trace=False)
    drp, dcl = torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda()
    R = "rescan"
    for kw in (dict(mode="data", filter_degree=-1, forbidden=R), dict(filter_degree=-1, forbidden=R),
               dict(filter_start=1.0, filter_degree=32, chunk=32, forbidden=R), dict(),
               dict(mode="data", t1=16, chunk=32), dict(worklist="rebuild")):
        colors, st = ctx.color(drp, dcl, options=ipgc.ColorOptions(**kw))
        assert np.array_equal(colors.cpu().numpy(), ref.colors), (name, kw)
        assert st.rounds == ref.rounds and st.num_colors == ref.num_colors
