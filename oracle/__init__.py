"""IPGC CPU oracle -- TEST INFRASTRUCTURE ONLY.

ctypes binding over ``liboracle.so`` built from ``ipgc_oracle.c`` (plain C,
single-threaded, -O2). Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product library
never imports, links or calls it, and it shares no code with the CUDA path.

The oracle follows the IPGC iteration of Section II-C (speculative first-fit
colouring of every uncoloured node, then conflict removal until the worklist
is empty) with fixed round semantics: colours read from the previous round's
snapshot, and the higher node ID losing a conflict. Its header comment states
every reading taken where the paper is silent.

Pins (tests/test_oracle_pins.py): closed forms for edgeless, complete, star,
path and complete bipartite graphs derived by hand from Section II-C; two
hand-worked examples in tests/golden/; the exhaustive set of labelled graphs on up to 5
nodes against a brute-force chromatic number (chi <= K); invariants on random
and paper-shaped graphs (proper colouring, K <= max degree + 1, first-fit
property, strictly shrinking worklist). The micro-benchmark iteration count
is pinned by the closed form ceil(n / COUNT).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ipgc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2, single-threaded)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(
                ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC], check=True
            )
            os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Load an oracle shared library built from ipgc_oracle.c (or a variant)."""
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_color.argtypes = [P(i32), P(i32), i32, P(i32), P(i32), P(i32), P(i32), P(i64), P(i64), i32]
    lib.oracle_color.restype = ctypes.c_int
    lib.oracle_push_iterations.argtypes = [i32, i32, P(i64), i64]
    lib.oracle_push_iterations.restype = i64
    lib.oracle_push_run.argtypes = [i32, i32, i32, P(i64), P(i64), i64]
    lib.oracle_push_run.restype = i64
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_LIB)
    return _lib


class Result:
    """colors (int32[n]), rounds, num_colors, fin_round (int32[n]),
    wl_sizes (|A| per round), deg_sums (sum of degrees over A per round)."""

    def __init__(self, colors, rounds, num_colors, fin_round, wl_sizes, deg_sums):
        self.colors = colors
        self.rounds = rounds
        self.num_colors = num_colors
        self.fin_round = fin_round
        self.wl_sizes = wl_sizes
        self.deg_sums = deg_sums


def color(rowptr, col, trace: bool = True, cap: int | None = None, lib=None) -> Result:
    """Run the oracle on a CSR graph (numpy int32 arrays)."""
    lib = lib if lib is not None else _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = rowptr.size - 1
    P = ctypes.POINTER
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    colors = np.zeros(max(n, 0), np.int32)
    fin = np.zeros(max(n, 0), np.int32) if trace else None
    if cap is None:
        cap = n + 1 if trace else 0
    wl = np.zeros(cap, np.int64) if trace else None
    ds = np.zeros(cap, np.int64) if trace else None
    rounds, k = i32(0), i32(0)
    null32, null64 = P(i32)(), P(i64)()
    rc = lib.oracle_color(
        rowptr.ctypes.data_as(P(i32)),
        col.ctypes.data_as(P(i32)) if col.size else null32,
        n,
        colors.ctypes.data_as(P(i32)),
        ctypes.byref(rounds),
        ctypes.byref(k),
        fin.ctypes.data_as(P(i32)) if trace else null32,
        wl.ctypes.data_as(P(i64)) if trace else null64,
        ds.ctypes.data_as(P(i64)) if trace else null64,
        cap,
    )
    if rc != 0:
        raise RuntimeError(f"oracle_color failed: {rc}")
    r = rounds.value
    return Result(
        colors,
        r,
        k.value,
        fin,
        wl[: min(r, cap)] if trace else None,
        ds[: min(r, cap)] if trace else None,
    )


def push_run(n: int, count: int = 1000, mode: str = "wl"):
    """Both Section III push kernels as written (mode "wl": Push_WL pops the
    worklist; "nowl": Push_NoWL visits every node), run until the worklist is
    empty. Returns (iterations, |WL| per iteration, sum of WL IDs per iteration)."""
    lib = _load()
    P = ctypes.POINTER(ctypes.c_int64)
    cap = (n + count - 1) // count + 1 if count > 0 else 1
    sizes = np.zeros(cap, np.int64)
    sums = np.zeros(cap, np.int64)
    it = lib.oracle_push_run(n, count, {"wl": 0, "nowl": 1}[mode], sizes.ctypes.data_as(P),
                             sums.ctypes.data_as(P), cap)
    if it < 0:
        raise RuntimeError("oracle_push_run failed")
    return int(it), sizes[:it], sums[:it]


def push_iterations(n: int, count: int = 1000, cap: int = 0):
    """Iterations of the Section III micro-benchmark until |WL| = 0, and the
    |WL| after each iteration (first ``cap`` entries)."""
    lib = _load()
    sizes = np.zeros(max(cap, 1), np.int64)
    it = lib.oracle_push_iterations(n, count, sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
    if it < 0:
        raise RuntimeError("oracle_push_iterations failed")
    return int(it), sizes[:cap]
