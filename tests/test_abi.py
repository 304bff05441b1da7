"""The C-ABI library loads and exports every declared entry point (CPU only;
no compute calls that need a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1912_01478_gb300 import _build, ipgc
from paper_1912_01478_gb300 import graphgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ipgc.lib()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"IPGC_API\s+[\w\s\*]+?\b(ipgc_\w+)\s*\(", txt))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("ipgc_color", "ipgc_color_ex", "ipgc_ctx_create", "ipgc_validate_csr", "ipgc_color_host"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\bT (ipgc_\w+)", out.stdout))
    missing = declared_symbols() - exported
    assert not missing, missing
    for name in declared_symbols():
        assert hasattr(lib, name)
    # nothing but the API is exported
    others = [l for l in out.stdout.splitlines() if " T " in l and " ipgc_" not in l]
    assert not others, others


def test_binding_covers_header():
    assert declared_symbols() <= set(ipgc.SIGNATURES) | extra_bound()


def extra_bound():
    import importlib
    names = set()
    for mod in ("paper_1912_01478_gb300.ipgc", "paper_1912_01478_gb300.batched",
                "paper_1912_01478_gb300.server", "paper_1912_01478_gb300.policy"):
        try:
            m = importlib.import_module(mod)
        except ImportError:
            continue
        names |= set(getattr(m, "SIGNATURES", {}))
    return names


def test_strerror_and_defaults(lib):
    assert lib.ipgc_strerror(0) == b"ok"
    assert b"invalid" in lib.ipgc_strerror(-1)
    o = ipgc.Options()
    lib.ipgc_options_default(ctypes.byref(o))
    assert o.mode == ipgc.MODE_THRESHOLD and abs(o.threshold_frac - 0.6) < 1e-7
    assert o.driver == ipgc.DRIVER_PERSISTENT and o.validate == 1
    assert abs(o.policy_margin - 0.05) < 1e-7


def test_ctypes_layouts_match_the_header(tmp_path):
    # a C program compiled against include/ipgc.h prints the real sizes and
    # field offsets; the ctypes mirrors must agree field by field
    from paper_1912_01478_gb300 import batched, server

    structs = {
        "ipgc_options": ipgc.Options,
        "ipgc_stats": ipgc.Stats,
        "ipgc_trace_rec": ipgc.TraceRec,
        "ipgc_batch_options": batched.BatchOptions,
        "ipgc_server_options": server.ServerOptions,
        "ipgc_server_counters": server.ServerCounters,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ipgc.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_workspace_size(lib):
    assert lib.ipgc_workspace_size(0, 0, None) == 0
    assert lib.ipgc_workspace_size(1000, 8000, None) >= 3 * 4000  # tent + 2 worklists
    # smaller t2: more high-degree nodes possible, more work-item room
    o = ipgc.Options()
    lib.ipgc_options_default(ctypes.byref(o))
    o.t1 = 2
    assert lib.ipgc_workspace_size(1000, 8000, ctypes.byref(o)) > lib.ipgc_workspace_size(1000, 8000, None)


def test_workspace_size_by_forbidden_colour_source(lib):
    # the default (persistent driver) pushes: rescanning's arrays plus the
    # bitmaps (4 bytes per entry), the winners list (4 per node) and the
    # push queue; rescanning with filtering holds the two list buffers (8
    # bytes per entry), without filtering neither; the host-loop driver
    # rescans whatever `forbidden` says by default
    n, nnz = 4_194_304, 128_304_280

    def size(**kw):
        return lib.ipgc_workspace_size(n, nnz, ctypes.byref(ipgc.ColorOptions(**kw).to_c()))

    auto, push = size(), size(forbidden="push")
    rescan, plain = size(forbidden="rescan"), size(forbidden="rescan", filter_degree=-1)
    assert auto == push
    assert size(driver="hostloop") == rescan
    assert rescan - plain >= 8 * nnz
    # + bitmaps (4 nnz) + winners (4 n) + queue, - the filtered items (2 x 16 B per item)
    assert 3.5 * nnz < push - rescan < 4 * nnz + 4 * n + 16 * (nnz // 128 + n + 1)


def test_host_validation(lib):
    rp, cl = graphgen.er(200, 600, seed=5)
    assert ipgc.validate_host(rp, cl) == ipgc.IPGC_OK
    bad = cl.copy()
    bad[0] = rp.size  # out of range
    assert ipgc.validate_host(rp, bad) == ipgc.IPGC_ERR_INVALID
    # self loop
    bad = cl.copy()
    bad[rp[3]] = 3
    assert ipgc.validate_host(rp, bad) == ipgc.IPGC_ERR_INVALID
    # asymmetric: drop one direction of an edge by re-pointing it
    rp2, cl2 = graphgen.from_edges(3, [0, 1], [1, 2])
    cl2 = cl2.copy()
    cl2[0] = 2  # row 0: {2} but row 2 lacks 0
    assert ipgc.validate_host(rp2, cl2) == ipgc.IPGC_ERR_INVALID
    # unsorted row
    rp3, cl3 = graphgen.from_edges(4, [0, 0], [1, 2])
    cl3 = cl3.copy()
    cl3[0], cl3[1] = cl3[1], cl3[0]
    assert ipgc.validate_host(rp3, cl3) == ipgc.IPGC_ERR_INVALID
    # bad rowptr
    assert ipgc.validate_host(np.array([0, 2, 1], np.int32), np.array([1, 0], np.int32)) == ipgc.IPGC_ERR_INVALID


def test_ctx_create_reports_no_device_without_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.ipgc_ctx_create(ctypes.byref(h), 0)
    assert rc in (ipgc.IPGC_ERR_INVALID, ipgc.IPGC_ERR_CUDA)
    assert not h.value
