"""Seeded synthetic graph generators (inputs only; no colouring arithmetic).

Thin ctypes binding over ``libgraphgen.so`` (built from ``graphgen.c`` beside
this file by :func:`build`; its C ABI is declared in
``include/ipgc_graphgen.h``). Every graph is undirected, symmetric, has no
self-loops or duplicate edges and sorted CSR rows, matching the preprocessing
the paper applies to its inputs (Section V). Arrays come back as numpy int32
(rowptr, col) or int64 (batch offsets).

Both the CPU oracle's tests and the GPU path consume these bytes; the graphs
stand in for the paper's UFL/SuiteSparse inputs (Table I), which are not
available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_HEADER = os.path.join(os.path.dirname(os.path.dirname(_HERE)), "include", "ipgc_graphgen.h")
_lock = threading.Lock()
_lib = None

# Paper-shaped workload parameters (seeded, synthetic).
RMAT_ABC = (0.57, 0.19, 0.19)


class _Csr(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("nnz", ctypes.c_int64),
        ("rowptr", ctypes.POINTER(ctypes.c_int32)),
        ("col", ctypes.POINTER(ctypes.c_int32)),
    ]


class _Batch(ctypes.Structure):
    _fields_ = [
        ("num_graphs", ctypes.c_int32),
        ("node_off", ctypes.POINTER(ctypes.c_int64)),
        ("edge_off", ctypes.POINTER(ctypes.c_int64)),
        ("rowptr_cat", ctypes.POINTER(ctypes.c_int32)),
        ("col_cat", ctypes.POINTER(ctypes.c_int32)),
    ]


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (OpenMP over graphs of a batch)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_HEADER)
        ):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fvisibility=hidden",
                   "-I", os.path.dirname(_HEADER), "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.POINTER
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    lib.ipgc_gen_er.argtypes = [u64, i32, i64, P(_Csr)]
    lib.ipgc_gen_rmat.argtypes = [u64, i32, i64, dbl, dbl, dbl, i32, i32, P(_Csr)]
    lib.ipgc_gen_road.argtypes = [u64, i32, dbl, dbl, P(_Csr)]
    lib.ipgc_gen_from_edges.argtypes = [i32, i64, P(i32), P(i32), P(_Csr)]
    lib.ipgc_gen_rgg.argtypes = [u64, i32, i32, dbl, P(_Csr)]
    lib.ipgc_gen_lattice3.argtypes = [i32, i32, P(_Csr)]
    lib.ipgc_gen_hubs.argtypes = [u64, i32, i64, i32, i64, dbl, P(_Csr)]
    lib.ipgc_gen_batch.argtypes = [u64, i32, i32, i32, dbl, dbl, i32, dbl, dbl, dbl, P(_Batch)]
    lib.ipgc_gen_free_csr.argtypes = [P(_Csr)]
    lib.ipgc_gen_free_batch.argtypes = [P(_Batch)]
    lib.ipgc_gen_hash_words.argtypes = [P(i32), i64, u64]
    lib.ipgc_gen_hash_words.restype = u64
    lib.ipgc_gen_derive_seed.argtypes = [u64, u64]
    lib.ipgc_gen_derive_seed.restype = u64
    lib.ipgc_gen_num_threads.restype = ctypes.c_int
    for f in (lib.ipgc_gen_er, lib.ipgc_gen_rmat, lib.ipgc_gen_road, lib.ipgc_gen_from_edges,
              lib.ipgc_gen_batch, lib.ipgc_gen_rgg, lib.ipgc_gen_lattice3, lib.ipgc_gen_hubs):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _take(c: _Csr):
    lib = _load()
    n, nnz = int(c.n), int(c.nnz)
    rowptr = np.ctypeslib.as_array(c.rowptr, shape=(n + 1,)).copy()
    col = (
        np.ctypeslib.as_array(c.col, shape=(nnz,)).copy() if nnz > 0 else np.zeros(0, np.int32)
    )
    lib.ipgc_gen_free_csr(ctypes.byref(c))
    return rowptr, col


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"graphgen {what} failed with code {rc}")


def er(n: int, m: int, seed: int):
    """Erdos-Renyi G(n, m) with exactly m undirected edges. Returns (rowptr, col)."""
    c = _Csr()
    _check(_load().ipgc_gen_er(seed, n, m, ctypes.byref(c)), "er")
    return _take(c)


def rmat(scale: int, edge_factor: int, seed: int, abc=RMAT_ABC, n_limit: int = 0, permute=True):
    """RMAT with edge_factor * 2^scale directed draws, symmetrised, IDs permuted."""
    a, b, cc = abc
    c = _Csr()
    nedges = int(edge_factor) * (n_limit if n_limit > 0 else (1 << scale))
    _check(
        _load().ipgc_gen_rmat(seed, scale, nedges, a, b, cc, n_limit, 1 if permute else 0,
                              ctypes.byref(c)),
        "rmat",
    )
    return _take(c)


def road(side: int, seed: int, p_delete: float = 0.30, frac_long: float = 0.01):
    """side x side grid, p_delete of edges removed, frac_long long-range edges added."""
    c = _Csr()
    _check(_load().ipgc_gen_road(seed, side, p_delete, frac_long, ctypes.byref(c)), "road")
    return _take(c)


def rgg(n: int, dim: int, avg_degree: float, seed: int):
    """Random geometric graph in the unit square (dim 2) or cube (dim 3), mean
    degree avg_degree away from the border, IDs in grid-cell order."""
    c = _Csr()
    _check(_load().ipgc_gen_rgg(seed, n, dim, avg_degree, ctypes.byref(c)), "rgg")
    return _take(c)


def lattice3(side: int, r2: int):
    """side^3 lattice, edges between nodes at squared distance <= r2 (r2 = 6:
    80 neighbours inside)."""
    c = _Csr()
    _check(_load().ipgc_gen_lattice3(side, r2, ctypes.byref(c)), "lattice3")
    return _take(c)


def hubs(n: int, m_base: int, nhubs: int, max_deg: int, alpha: float, seed: int):
    """Uniform base of m_base pairs plus nhubs hubs of degree max_deg / (h+1)^alpha."""
    c = _Csr()
    _check(_load().ipgc_gen_hubs(seed, n, m_base, nhubs, max_deg, alpha, ctypes.byref(c)), "hubs")
    return _take(c)


def from_edges(n: int, src, dst):
    """CSR (symmetrised, deduplicated, self-loops dropped, rows sorted) from pairs."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    assert src.shape == dst.shape
    c = _Csr()
    P = ctypes.POINTER(ctypes.c_int32)
    _check(
        _load().ipgc_gen_from_edges(
            n, src.size, src.ctypes.data_as(P), dst.ctypes.data_as(P), ctypes.byref(c)
        ),
        "from_edges",
    )
    return _take(c)


def batch(
    num_graphs: int,
    seed: int,
    nmin: int = 100,
    nmax: int = 200_000,
    deg_lo: float = 4.0,
    deg_hi: float = 32.0,
    rmat_ef: int = 8,
    abc=RMAT_ABC,
):
    """Concatenated batch: dict(node_off, edge_off, rowptr_cat, col_cat)."""
    b = _Batch()
    a, bb, c = abc
    lib = _load()
    _check(
        lib.ipgc_gen_batch(seed, num_graphs, nmin, nmax, deg_lo, deg_hi, rmat_ef, a, bb, c,
                           ctypes.byref(b)),
        "batch",
    )
    G = int(b.num_graphs)
    node_off = np.ctypeslib.as_array(b.node_off, shape=(G + 1,)).copy()
    edge_off = np.ctypeslib.as_array(b.edge_off, shape=(G + 1,)).copy()
    nrp = int(node_off[-1]) + G
    ncol = int(edge_off[-1])
    rowptr_cat = np.ctypeslib.as_array(b.rowptr_cat, shape=(nrp,)).copy()
    col_cat = (
        np.ctypeslib.as_array(b.col_cat, shape=(ncol,)).copy() if ncol > 0 else np.zeros(0, np.int32)
    )
    lib.ipgc_gen_free_batch(ctypes.byref(b))
    return dict(node_off=node_off, edge_off=edge_off, rowptr_cat=rowptr_cat, col_cat=col_cat)


def batch_graph(bt: dict, g: int):
    """(rowptr, col) views of graph g inside a batch dict."""
    no, eo = bt["node_off"], bt["edge_off"]
    n = int(no[g + 1] - no[g])
    rp = bt["rowptr_cat"][int(no[g]) + g : int(no[g]) + g + n + 1]
    cl = bt["col_cat"][int(eo[g]) : int(eo[g + 1])]
    return rp, cl


def graph_hash(rowptr, col) -> int:
    """FNV-1a 64 over rowptr then col (little-endian int32 words)."""
    lib = _load()
    P = ctypes.POINTER(ctypes.c_int32)
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    h = lib.ipgc_gen_hash_words(rp.ctypes.data_as(P), rp.size, 0)
    return int(lib.ipgc_gen_hash_words(cl.ctypes.data_as(P), cl.size, h))


def derive_seed(seed: int, index: int) -> int:
    return int(_load().ipgc_gen_derive_seed(seed, index))


def num_threads() -> int:
    return int(_load().ipgc_gen_num_threads())


def batch_workload(num_graphs: int = 4096, seed: int = 4):
    """The batched workload: num_graphs graphs, n log-uniform in [100, 200000],
    even index Erdos-Renyi with average degree U(4, 32), odd index RMAT with
    edge factor 8 (IDs permuted), per-graph seeds derived from `seed`."""
    return batch(num_graphs, seed=seed, nmin=100, nmax=200_000, deg_lo=4.0, deg_hi=32.0, rmat_ef=8)


# Stand-ins for the paper's ten UFL graphs (Table I: nodes, entries, degree
# minimum / median / maximum), each built to that shape; `scale` shrinks the
# node count (and hub sizes) with the degrees kept, for tests.
SUITE = {
    # hub-heavy circuit: median degree 4, one hub of ~1.29 M neighbours
    "circuit5M": lambda s: hubs(int(5_500_000 * s), int(12_000_000 * s), max(1, int(3000 * s)),
                                int(1_290_500 * s), 0.9, seed=11),
    # finite-element meshes: regular, median degrees 68 / 44 / 80
    "Audikw_1": lambda s: rgg(int(943_695 * s), 3, 90.0, seed=12),
    "Bump_2911": lambda s: rgg(int(2_911_419 * s), 3, 46.0, seed=13),
    "Queen_4147": lambda s: lattice3(max(2, round(160 * s ** (1 / 3))), 6),
    # Kronecker (Graph 500) generator, scale 21
    "kron_g500-logn21": lambda s: rmat(21, 48, seed=14, n_limit=int((1 << 21) * s) if s < 1 else 0),
    # web crawl: very skewed, IDs in crawl order (not permuted)
    "indochina-2004": lambda s: rmat(23, 24, seed=15, abc=(0.6, 0.15, 0.15),
                                     n_limit=int(7_414_866 * s), permute=False),
    # collaboration graph: dense, moderately skewed
    "hollywood-2009": lambda s: rmat(21, 55, seed=16, abc=(0.45, 0.22, 0.22),
                                     n_limit=int(1_139_905 * s)),
    # random geometric graph, n = 2^24
    "rgg_n_2_24_s0": lambda s: rgg(int((1 << 24) * s), 2, 16.0, seed=17),
    # social network
    "soc-LiveJournal1": lambda s: rmat(23, 10, seed=18, abc=(0.5, 0.2, 0.2),
                                       n_limit=int(4_847_571 * s)),
    # road network: average degree ~2.1, degrees 1..13
    "europe_osm": lambda s: road(max(2, round(7135 * s ** 0.5)), seed=19, p_delete=0.47,
                                 frac_long=0.005),
}


def suite_graph(name: str, scale: float = 1.0):
    """(rowptr, col) of the stand-in for one of the paper's ten graphs."""
    return SUITE[name](scale)


# Named workloads: the paper-shaped synthetic inputs (sizes as stated).
def workload(name: str):
    """Return (rowptr, col) for a named single-graph workload."""
    if name == "er_n10000_deg8_seed1":
        return er(10_000, 40_000, seed=1)
    if name == "rmat_s22_ef16_seed2":
        return rmat(22, 16, seed=2)
    if name == "road_4096_seed3":
        return road(4096, seed=3)
    raise KeyError(name)
