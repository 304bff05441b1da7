"""Python binding of libipgc.so (ctypes; argument marshalling only).

Every step of the colouring runs in the library's CUDA kernels. PyTorch is
used here only to hold device memory and to name streams: tensors are passed
by ``data_ptr()``. There is no CPU fallback: if the library cannot be loaded
the import of :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libipgc.so")

IPGC_OK = 0
IPGC_PENDING = 1
IPGC_ERR_INVALID = -1
IPGC_ERR_OOM = -2
IPGC_ERR_TIMEOUT = -3
IPGC_ERR_NO_CONVERGE = -4
IPGC_ERR_CUDA = -5
IPGC_ERR_BUSY = -6
IPGC_ERR_UNSUPPORTED = -7
IPGC_ERR_NOT_FOUND = -8
IPGC_ERR_TOO_LARGE = -9

# limits of ipgc_color_noalloc's fixed scratch
NOALLOC_MAX_N = 524288
NOALLOC_MAX_NNZ = 8388608

MODE_THRESHOLD, MODE_TOPO, MODE_DATA, MODE_LEARNED = 0, 1, 2, 3
DRIVER_PERSISTENT, DRIVER_HOSTLOOP = 0, 1
PUSH_WL, PUSH_NOWL, PUSH_HYBRID = 0, 1, 2
WORKLIST_KEEP, WORKLIST_REBUILD = 0, 1
FORBIDDEN_AUTO, FORBIDDEN_RESCAN, FORBIDDEN_PUSH = 0, 1, 2
FORBIDDEN = {"auto": FORBIDDEN_AUTO, "rescan": FORBIDDEN_RESCAN, "push": FORBIDDEN_PUSH}
MODES = {"threshold": MODE_THRESHOLD, "topo": MODE_TOPO, "data": MODE_DATA, "learned": MODE_LEARNED}
DRIVERS = {"persistent": DRIVER_PERSISTENT, "hostloop": DRIVER_HOSTLOOP}


class Stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int32),
        ("num_colors", ctypes.c_int32),
        ("rounds_topo", ctypes.c_int32),
        ("rounds_data", ctypes.c_int32),
        ("edges_processed", ctypes.c_int64),
        ("ns", ctypes.c_uint64),
        ("error", ctypes.c_int32),
        ("filter_round", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TraceRec(ctypes.Structure):
    _fields_ = [
        ("round", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("wl_size", ctypes.c_int64),
        ("deg_sum", ctypes.c_int64),
        ("max_color", ctypes.c_int32),
        ("shortcut", ctypes.c_int32),
        ("wl_small", ctypes.c_int32),
        ("push_ns", ctypes.c_int32),
        ("t_begin", ctypes.c_uint64),
        ("t_assign", ctypes.c_uint64),
        ("t_detect", ctypes.c_uint64),
    ]


TRACE_DTYPE = np.dtype(
    [
        ("round", np.int32),
        ("mode", np.int32),
        ("wl_size", np.int64),
        ("deg_sum", np.int64),
        ("max_color", np.int32),
        ("shortcut", np.int32),
        ("wl_small", np.int32),
        ("push_ns", np.int32),
        ("t_begin", np.uint64),
        ("t_assign", np.uint64),
        ("t_detect", np.uint64),
    ]
)
assert TRACE_DTYPE.itemsize == ctypes.sizeof(TraceRec)


class Options(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("threshold_frac", ctypes.c_float),
        ("driver", ctypes.c_int32),
        ("max_rounds", ctypes.c_int32),
        ("timeout_ns", ctypes.c_uint64),
        ("validate", ctypes.c_int32),
        ("t1", ctypes.c_int32),
        ("chunk", ctypes.c_int32),
        ("block_size", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("trace", ctypes.c_void_p),
        ("fin_round", ctypes.c_void_p),
        ("trace_cap", ctypes.c_int32),
        ("fault_inject", ctypes.c_int32),
        ("policy_margin", ctypes.c_float),
        ("filter_degree", ctypes.c_int32),
        ("filter_start", ctypes.c_float),
        ("worklist", ctypes.c_int32),
        ("forbidden", ctypes.c_int32),
    ]


class IpgcError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {lib().ipgc_strerror(code).decode()} ({code})")


_lib = None

# name -> (restype, argtypes); every entry point the header declares
_P = ctypes.c_void_p
_I32, _I64, _INT = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
SIGNATURES = {
    "ipgc_options_default": (None, [ctypes.POINTER(Options)]),
    "ipgc_strerror": (ctypes.c_char_p, [_INT]),
    "ipgc_ctx_create": (_INT, [ctypes.POINTER(_P), _INT]),
    "ipgc_ctx_destroy": (_INT, [_P]),
    "ipgc_ctx_cuda_error": (_INT, [_P]),
    "ipgc_workspace_size": (ctypes.c_size_t, [_I32, _I64, ctypes.POINTER(Options)]),
    "ipgc_color": (_INT, [_P, _P, _I32, _I64, _P, ctypes.POINTER(Stats)]),
    "ipgc_color_ex": (
        _INT,
        [_P, _P, _P, _I32, _I64, _P, ctypes.POINTER(Stats), ctypes.POINTER(Options), _P],
    ),
    "ipgc_ctx_last_stats": (_INT, [_P, ctypes.POINTER(Stats)]),
    "ipgc_color_host": (
        _INT,
        [_P, _P, _P, _I32, _I64, _P, ctypes.POINTER(Stats), ctypes.POINTER(Options), _P],
    ),
    "ipgc_validate_csr": (_INT, [_P, _P, _P, _I32, _I64, _INT, _P]),
    "ipgc_push_bench": (_INT, [_P, _I64, _I32, _I32, _I64, _P, _I64, ctypes.POINTER(_I64), _P]),
    "ipgc_color_noalloc": (_INT, [_P, _P, _I32, _I64, _P, ctypes.POINTER(Stats), _P]),
    "ipgc_autotune": (
        _INT,
        [_P, _P, _P, _I32, _I64, _P, _I32, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_float), _P],
    ),
}


def lib():
    """Load libipgc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_1912_01478_gb300._build.build()"
            )
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


@dataclass
class ColorOptions:
    mode: str = "threshold"
    threshold_frac: float = 0.6
    driver: str = "persistent"
    max_rounds: int = 0
    timeout_ns: int = 0
    validate: bool = True
    t1: int = 0
    chunk: int = 0
    block_size: int = 0
    blocks_per_sm: int = 0
    fault_inject: int = 0
    policy_margin: float = 0.05
    filter_degree: int = 0  # 0: library default; < 0: neighbour filtering off
    filter_start: float = 0.0  # 0: library default
    worklist: str = "keep"  # "keep" (the paper's hybrid) or "rebuild" (discard and rebuild)
    forbidden: str = "auto"  # "auto", "rescan" (reread rows every round) or "push" (bitmaps)

    def to_c(self, trace_ptr: int = 0, trace_cap: int = 0, fin_ptr: int = 0) -> Options:
        o = Options()
        lib().ipgc_options_default(ctypes.byref(o))
        o.mode = MODES[self.mode]
        o.threshold_frac = self.threshold_frac
        o.driver = DRIVERS[self.driver]
        o.max_rounds = self.max_rounds
        o.timeout_ns = self.timeout_ns
        o.validate = 1 if self.validate else 0
        o.t1, o.chunk = self.t1, self.chunk
        o.block_size, o.blocks_per_sm = self.block_size, self.blocks_per_sm
        o.trace = trace_ptr or None
        o.trace_cap = trace_cap
        o.fin_round = fin_ptr or None
        o.fault_inject = self.fault_inject
        o.policy_margin = self.policy_margin
        o.filter_degree = self.filter_degree
        o.filter_start = self.filter_start
        o.worklist = {"keep": WORKLIST_KEEP, "rebuild": WORKLIST_REBUILD}[self.worklist]
        o.forbidden = FORBIDDEN[self.forbidden]
        return o


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _after_current(stream) -> None:
    """Order a torch stream after the work already queued on the current torch
    stream of its device, where the caller's buffers were allocated, zeroed or
    copied (a trace buffer or finalisation array zeroed there could otherwise
    be zeroed again while the colouring writes it). Raw stream handles are the
    caller's to order."""
    if stream is None or isinstance(stream, int):
        return
    import torch

    cur = torch.cuda.current_stream(stream.device)
    if cur != stream:
        stream.wait_stream(cur)


def _check(rc: int, what: str):
    if rc != IPGC_OK:
        raise IpgcError(rc, what)


class Context:
    """An ipgc_ctx on one CUDA device (owns the library's workspace)."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().ipgc_ctx_create(ctypes.byref(h), device), "ipgc_ctx_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().ipgc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cuda_error(self) -> int:
        return lib().ipgc_ctx_cuda_error(self.handle)

    def color(self, rowptr, col, colors_out=None, options: ColorOptions | None = None, stream=None,
              trace=None, wait: bool = True, fin_round=None):
        """Colour a graph held in CUDA int32 tensors. Returns (colors, Stats or None).

        trace: optional CUDA uint8 tensor of k * sizeof(TraceRec) bytes that
        receives one record per round (see :func:`read_trace`).
        """
        import torch

        n = rowptr.numel() - 1
        nnz = col.numel()
        assert rowptr.dtype == torch.int32 and col.dtype == torch.int32
        assert rowptr.is_cuda and (nnz == 0 or col.is_cuda)
        if colors_out is None:
            colors_out = torch.empty(max(n, 0), dtype=torch.int32, device=rowptr.device)
        opts = options or ColorOptions()
        tptr, tcap = 0, 0
        if trace is not None:
            tptr, tcap = trace.data_ptr(), trace.numel() // ctypes.sizeof(TraceRec)
        o = opts.to_c(tptr, tcap, fin_round.data_ptr() if fin_round is not None else 0)
        st = Stats()
        _after_current(stream)
        rc = lib().ipgc_color_ex(
            self.handle,
            rowptr.data_ptr(),
            col.data_ptr() if nnz else None,
            n,
            nnz,
            colors_out.data_ptr() if n else None,
            ctypes.byref(st) if wait else None,
            ctypes.byref(o),
            _stream_handle(stream) or None,
        )
        _check(rc, "ipgc_color_ex")
        return colors_out, (st if wait else None)

    def last_stats(self) -> Stats:
        st = Stats()
        _check(lib().ipgc_ctx_last_stats(self.handle, ctypes.byref(st)), "ipgc_ctx_last_stats")
        return st

    def color_host(self, rowptr: np.ndarray, col: np.ndarray, colors_out: np.ndarray | None = None,
                   options: ColorOptions | None = None, stream=None):
        """Colour a graph held in host int32 arrays (copies inside the call)."""
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n = rowptr.size - 1
        if colors_out is None:
            colors_out = np.empty(max(n, 0), np.int32)
        o = (options or ColorOptions()).to_c()
        st = Stats()
        rc = lib().ipgc_color_host(
            self.handle,
            rowptr.ctypes.data,
            col.ctypes.data if col.size else None,
            n,
            col.size,
            colors_out.ctypes.data if n else None,
            ctypes.byref(st),
            ctypes.byref(o),
            _stream_handle(stream) or None,
        )
        _check(rc, "ipgc_color_host")
        return colors_out, st

    def push_bench(self, n: int, count: int = 1000, mode: str = "wl", switch_wl: int = 0,
                   record: bool = True, stream=None):
        """The Section III micro-benchmark (mode "wl", "nowl" or "hybrid").
        Returns (iterations, records): records is a numpy int64 [iterations, 4]
        array of (|WL| after, sum of its IDs, kernel used, time ns) or None."""
        import torch

        cap = (n + count - 1) // count if record and count > 0 else 0
        rec = torch.zeros(max(cap, 1) * 4, dtype=torch.int64, device=f"cuda:{self.device}")
        it = _I64(0)
        m = {"wl": PUSH_WL, "nowl": PUSH_NOWL, "hybrid": PUSH_HYBRID}[mode]
        rc = lib().ipgc_push_bench(self.handle, n, count, m, switch_wl,
                                   rec.data_ptr() if cap else None, cap, ctypes.byref(it),
                                   _stream_handle(stream) or None)
        _check(rc, "ipgc_push_bench")
        out = rec[: it.value * 4].view(-1, 4).cpu().numpy() if cap else None
        return it.value, out

    def validate(self, rowptr, col, stream=None) -> int:
        """IPGC_OK or IPGC_ERR_INVALID for a CSR held in CUDA tensors."""
        _after_current(stream)
        return lib().ipgc_validate_csr(
            self.handle, rowptr.data_ptr(), col.data_ptr() if col.numel() else None,
            rowptr.numel() - 1, col.numel(), 1, _stream_handle(stream) or None,
        )


def validate_host(rowptr: np.ndarray, col: np.ndarray) -> int:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return lib().ipgc_validate_csr(
        None, rowptr.ctypes.data, col.ctypes.data if col.size else None, rowptr.size - 1, col.size, 0, None
    )


def read_trace(trace_tensor, rounds: int) -> np.ndarray:
    """Copy the first `rounds` trace records of a CUDA trace buffer to numpy."""
    raw = trace_tensor[: rounds * TRACE_DTYPE.itemsize].cpu().numpy()
    return raw.view(TRACE_DTYPE).copy()


def trace_buffer(rounds: int, device=0):
    import torch

    return torch.zeros(rounds * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=f"cuda:{device}")


_default_ctx: dict[int, Context] = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


def color(rowptr, col, colors_out=None, options: ColorOptions | None = None, stream=None, trace=None):
    """ipgc_color_ex on the default context of the tensors' device."""
    dev = rowptr.device.index or 0
    return default_context(dev).color(rowptr, col, colors_out, options, stream, trace)


def color_noalloc(rowptr, col, colors_out=None, stream=None):
    """ipgc_color_noalloc: colour without any allocation inside the library.

    For callers that cannot allocate device memory at that moment; the library
    works in one fixed device array (see include/ipgc.h for the limits), so
    calls on one GPU must not overlap. colors_out must be given when the
    caller itself cannot allocate (this helper only allocates it when absent).
    """
    import torch

    n = rowptr.numel() - 1
    nnz = col.numel()
    if colors_out is None:
        colors_out = torch.empty(max(n, 0), dtype=torch.int32, device=rowptr.device)
    st = Stats()
    rc = lib().ipgc_color_noalloc(
        rowptr.data_ptr(), col.data_ptr() if nnz else None, n, nnz,
        colors_out.data_ptr() if n else None, ctypes.byref(st), _stream_handle(stream) or None,
    )
    _check(rc, "ipgc_color_noalloc")
    return colors_out, st
