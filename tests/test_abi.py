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
    # the automatic choice also holds the filtered nodes' work items (two lists
    # of 16-byte items), for the graphs it leaves to the rescanning kernels
    items = 16 * (nnz // 1024 + min(n, nnz // 65) + 1)
    assert push < auto <= push + 2 * items + 512
    assert size(driver="hostloop") == rescan
    assert rescan - plain >= 8 * nnz
    # + bitmaps (4 nnz) + winners (4 n) + push targets (8 n) + the push and list
    # rewrite queues (16 B per 128 entries each, plus per node), - the filtered
    # items (2 x 16 B per item)
    assert 3.5 * nnz < push - rescan < 4 * nnz + 12 * n + 32 * (nnz // 128 + n + 1)


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


def test_server_options_checked_before_any_device_call(lib):
    # bad options are refused before the device is touched (no GPU needed):
    # the forbidden-colour source must be one of the three
    from paper_1912_01478_gb300 import server

    for bad in (-1, 3):
        o = server.options()
        o.batch.base.forbidden = bad
        h = ctypes.c_void_p()
        assert lib.ipgc_server_create(ctypes.byref(h), 0, ctypes.byref(o)) == ipgc.IPGC_ERR_INVALID
        assert not h.value
    o = server.options(inflight=0)
    h = ctypes.c_void_p()
    assert lib.ipgc_server_create(ctypes.byref(h), 0, ctypes.byref(o)) == ipgc.IPGC_ERR_INVALID


# ------------------------------------------------ the generator library --

def declared_generator_symbols():
    txt = open(os.path.join(ROOT, "include", "ipgc_graphgen.h")).read()
    return set(re.findall(r"IPGC_GEN_API\s+[\w\s\*]+?\b(ipgc_gen_\w+)\s*\(", txt))


def test_generator_library_exports_exactly_its_header():
    path = graphgen.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True)
    exported = set(re.findall(r"\bT (\w+)", out.stdout))
    declared = declared_generator_symbols()
    assert {"ipgc_gen_er", "ipgc_gen_rmat", "ipgc_gen_road", "ipgc_gen_batch",
            "ipgc_gen_from_edges", "ipgc_gen_free_csr", "ipgc_gen_free_batch"} <= declared
    assert exported == declared, (exported ^ declared)


def test_generator_c_abi_from_a_c_program(tmp_path):
    # a C program compiled against include/ipgc_graphgen.h and linked with
    # libgraphgen.so: the symmetriser on a hand-made edge list (a triangle
    # 0-1-2 given with a repeat, a reversed copy and a self-loop, plus the
    # pendant edge 3-1) must give rows {1,2} {0,2,3} {0,1} {1}; an argument
    # out of range must be refused without memory; the layouts of both
    # records must match the ctypes mirrors
    path = graphgen.build()
    src = tmp_path / "gen.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "ipgc_graphgen.h"
int main(void) {
  const int32_t s[] = {0, 1, 2, 1, 2, 3, 2};
  const int32_t d[] = {1, 2, 0, 0, 2, 1, 1};
  ipgc_gen_csr g;
  int rc = ipgc_gen_from_edges(4, 7, s, d, &g);
  printf("rc %d n %d nnz %lld\n", rc, g.n, (long long)g.nnz);
  printf("rowptr"); for (int i = 0; i <= g.n; ++i) printf(" %d", g.rowptr[i]); printf("\n");
  printf("col"); for (long long i = 0; i < g.nnz; ++i) printf(" %d", g.col[i]); printf("\n");
  ipgc_gen_free_csr(&g);
  ipgc_gen_free_csr(&g);
  ipgc_gen_csr bad;
  const int32_t s2[] = {0}, d2[] = {4};
  bad.rowptr = (int32_t*)&rc;
  rc = ipgc_gen_from_edges(4, 1, s2, d2, &bad);
  printf("bad %d %d\n", rc, bad.rowptr == NULL && bad.col == NULL);
  printf("er %d\n", ipgc_gen_er(1, 3, 4, &bad));
  printf("csr %zu %zu %zu %zu %zu\n", sizeof(ipgc_gen_csr), offsetof(ipgc_gen_csr, n),
         offsetof(ipgc_gen_csr, nnz), offsetof(ipgc_gen_csr, rowptr), offsetof(ipgc_gen_csr, col));
  printf("batch %zu %zu %zu %zu %zu %zu\n", sizeof(ipgc_gen_batch_t),
         offsetof(ipgc_gen_batch_t, num_graphs), offsetof(ipgc_gen_batch_t, node_off),
         offsetof(ipgc_gen_batch_t, edge_off), offsetof(ipgc_gen_batch_t, rowptr_cat),
         offsetof(ipgc_gen_batch_t, col_cat));
  return 0;
}
''')
    exe = tmp_path / "gen"
    libdir = os.path.dirname(path)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src),
                    "-L", libdir, "-l:libgraphgen.so", f"-Wl,-rpath,{libdir}"], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    assert lines[0] == "rc 0 n 4 nnz 8"
    assert lines[1] == "rowptr 0 2 5 7 8"
    assert lines[2] == "col 1 2 0 2 3 0 1 1"
    assert lines[3] == "bad -1 1"
    assert lines[4] == "er -1"  # 4 edges do not fit on 3 nodes
    csr = [int(x) for x in lines[5].split()[1:]]
    C = graphgen._Csr
    assert csr == [ctypes.sizeof(C), C.n.offset, C.nnz.offset, C.rowptr.offset, C.col.offset]
    bat = [int(x) for x in lines[6].split()[1:]]
    B = graphgen._Batch
    assert bat == [ctypes.sizeof(B), B.num_graphs.offset, B.node_off.offset, B.edge_off.offset,
                   B.rowptr_cat.offset, B.col_cat.offset]
