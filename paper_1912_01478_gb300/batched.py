"""Binding of the batched entry point (ctypes; argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import ipgc


class BatchOptions(ctypes.Structure):
    _fields_ = [
        ("base", ipgc.Options),
        ("max_team", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("nnz_per_cta", ctypes.c_int64),
    ]


_P = ctypes.c_void_p
SIGNATURES = {
    "ipgc_batch_options_default": (None, [ctypes.POINTER(BatchOptions)]),
    "ipgc_color_batched": (
        ctypes.c_int,
        [_P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.POINTER(ipgc.Stats),
         ctypes.POINTER(BatchOptions), _P],
    ),
    "ipgc_batch_plan": (
        ctypes.c_int,
        [ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P, _P],
    ),
    "ipgc_batched_autotune": (
        ctypes.c_int,
        [_P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
         ctypes.POINTER(BatchOptions), ctypes.POINTER(ctypes.c_float), _P],
    ),
}


def autotune(ctx: "ipgc.Context", node_off, edge_off, rowptr_cat, col_cat, colors_cat,
             opts: BatchOptions | None = None, sample_graphs: int = 0, reps: int = 2, stream=None):
    """Run the native schedule autotuner; returns (BatchOptions, best ms)."""
    node_off = np.ascontiguousarray(node_off, dtype=np.int64)
    edge_off = np.ascontiguousarray(edge_off, dtype=np.int64)
    o = opts if opts is not None else options()
    best = ctypes.c_float(0)
    ipgc._after_current(stream)
    rc = lib().ipgc_batched_autotune(
        ctx.handle, node_off.size - 1, node_off.ctypes.data, edge_off.ctypes.data,
        rowptr_cat.data_ptr(), col_cat.data_ptr(), colors_cat.data_ptr(), sample_graphs, reps,
        ctypes.byref(o), ctypes.byref(best), ipgc._stream_handle(stream) or None,
    )
    if rc != ipgc.IPGC_OK:
        raise ipgc.IpgcError(rc, "ipgc_batched_autotune")
    return o, best.value


def plan(n, nnz, grid: int, max_team: int = 0, nnz_per_cta: int = 131072):
    """The gang schedule of a batch on `grid` CTAs (host only): per graph its
    team size, the first CTA of its block (-1: single CTA or empty) and its
    position in the gang order or the single-CTA queue (-1: empty)."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    nnz = np.ascontiguousarray(nnz, dtype=np.int64)
    G = n.size
    team = np.zeros(G, np.int32)
    first = np.zeros(G, np.int32)
    seq = np.zeros(G, np.int32)
    rc = lib().ipgc_batch_plan(G, n.ctypes.data, nnz.ctypes.data, grid, max_team, nnz_per_cta,
                               team.ctypes.data, first.ctypes.data, seq.ctypes.data)
    if rc != ipgc.IPGC_OK:
        raise ipgc.IpgcError(rc, "ipgc_batch_plan")
    return team, first, seq


def describe(o: BatchOptions) -> dict:
    forbidden = {v: k for k, v in ipgc.FORBIDDEN.items()}.get(o.base.forbidden, o.base.forbidden)
    return dict(t1=o.base.t1, chunk=o.base.chunk, block_size=o.base.block_size,
                max_team=o.max_team, nnz_per_cta=int(o.nnz_per_cta), mode=o.base.mode,
                forbidden=forbidden)

_bound = False


def lib():
    global _bound
    L = ipgc.lib()
    if not _bound:
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


def options(max_team: int = -1, nnz_per_cta: int = 0, **base) -> BatchOptions:
    """Batch options: defaults, then team settings (max_team: largest team in
    CTAs, 0 = the grid; nnz_per_cta: entries per team CTA) and
    ipgc.ColorOptions fields."""
    o = BatchOptions()
    lib().ipgc_batch_options_default(ctypes.byref(o))
    if base:
        b = ipgc.ColorOptions(**{"validate": False, **base}).to_c()
        o.base = b
    if max_team >= 0:
        o.max_team = max_team
    if nnz_per_cta:
        o.nnz_per_cta = nnz_per_cta
    return o


def color_batched(ctx: "ipgc.Context", node_off: np.ndarray, edge_off: np.ndarray, rowptr_cat,
                  col_cat, colors_cat=None, opts: BatchOptions | None = None, stream=None,
                  want_stats: bool = True):
    """Colour every graph of a concatenated batch held in CUDA int32 tensors.

    node_off / edge_off: host int64 arrays of G + 1 offsets. Returns
    (colors_cat, stats) where stats is a numpy structured array (or None).
    """
    import torch

    node_off = np.ascontiguousarray(node_off, dtype=np.int64)
    edge_off = np.ascontiguousarray(edge_off, dtype=np.int64)
    G = node_off.size - 1
    total_n = int(node_off[-1])
    if colors_cat is None:
        colors_cat = torch.empty(max(total_n, 0), dtype=torch.int32, device=rowptr_cat.device)
    st = (ipgc.Stats * max(G, 1))() if want_stats else None
    ipgc._after_current(stream)
    rc = lib().ipgc_color_batched(
        ctx.handle, G, node_off.ctypes.data, edge_off.ctypes.data, rowptr_cat.data_ptr(),
        col_cat.data_ptr() if col_cat.numel() else None,
        colors_cat.data_ptr() if total_n else None,
        st if want_stats else None, ctypes.byref(opts) if opts is not None else None,
        ipgc._stream_handle(stream) or None,
    )
    if rc != ipgc.IPGC_OK:
        raise ipgc.IpgcError(rc, "ipgc_color_batched")
    if not want_stats:
        return colors_cat, None
    arr = np.array([(s.rounds, s.num_colors, s.rounds_topo, s.rounds_data, s.edges_processed, s.ns,
                     s.error) for s in st[:G]],
                   dtype=[("rounds", np.int32), ("num_colors", np.int32), ("rounds_topo", np.int32),
                          ("rounds_data", np.int32), ("edges_processed", np.int64),
                          ("ns", np.uint64), ("error", np.int32)])
    return colors_cat, arr
