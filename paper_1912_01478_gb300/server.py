"""Binding of the colouring server (ctypes; argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import batched, ipgc


class ServerOptions(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_size_t),
        ("host_budget", ctypes.c_size_t),
        ("inflight", ctypes.c_int32),
        ("max_batch_graphs", ctypes.c_int32),
        ("max_pending", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("batch", batched.BatchOptions),
    ]


class ServerCounters(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("batches", ctypes.c_uint64),
        ("graphs_in_batches", ctypes.c_uint64),
        ("pending", ctypes.c_int64),
        ("ready", ctypes.c_int64),
        ("running_batches", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("hbm_used", ctypes.c_int64),
        ("hbm_peak", ctypes.c_int64),
        ("host_used", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_P = ctypes.c_void_p
SIGNATURES = {
    "ipgc_server_options_default": (None, [ctypes.POINTER(ServerOptions)]),
    "ipgc_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ServerOptions)]),
    "ipgc_server_submit": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "ipgc_server_submit_ref": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_uint64)]),
    "ipgc_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.POINTER(ipgc.Stats),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "ipgc_server_next_done": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64]),
    "ipgc_server_query": (ctypes.c_int, [_P, ctypes.POINTER(ServerCounters)]),
    "ipgc_server_policy_load": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "ipgc_server_destroy": (ctypes.c_int, [_P]),
}
_bound = False


def lib():
    global _bound
    L = batched.lib()
    if not _bound:
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


def options(**kw) -> ServerOptions:
    """Defaults, then ServerOptions fields by name (hbm_budget, inflight, ...)."""
    o = ServerOptions()
    lib().ipgc_server_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Server:
    """A colouring server on one device (owns its arenas and scheduler thread)."""

    def __init__(self, device: int = 0, opts: ServerOptions | None = None):
        h = ctypes.c_void_p()
        o = opts if opts is not None else options()
        rc = lib().ipgc_server_create(ctypes.byref(h), device, ctypes.byref(o))
        if rc != ipgc.IPGC_OK:
            raise ipgc.IpgcError(rc, "ipgc_server_create")
        self.handle = h
        self._n = {}

    def submit(self, rowptr: np.ndarray, col: np.ndarray) -> int:
        """Queue a graph; returns its ticket. Raises IpgcError (code BUSY, TOO_LARGE, ...)."""
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        t = ctypes.c_uint64(0)
        rc = lib().ipgc_server_submit(self.handle, rowptr.ctypes.data, col.ctypes.data if col.size else None,
                                      rowptr.size - 1, col.size, ctypes.byref(t))
        if rc != ipgc.IPGC_OK:
            raise ipgc.IpgcError(rc, "ipgc_server_submit")
        self._n[t.value] = rowptr.size - 1
        return t.value

    def submit_ref(self, rowptr: np.ndarray, col: np.ndarray) -> int:
        """Queue a graph by reference: the arrays (int32, contiguous, ideally in
        pinned memory) must stay alive and unchanged until the ticket completes."""
        assert rowptr.dtype == np.int32 and col.dtype == np.int32
        assert rowptr.flags.c_contiguous and col.flags.c_contiguous
        t = ctypes.c_uint64(0)
        rc = lib().ipgc_server_submit_ref(self.handle, rowptr.ctypes.data,
                                          col.ctypes.data if col.size else None,
                                          rowptr.size - 1, col.size, ctypes.byref(t))
        if rc != ipgc.IPGC_OK:
            raise ipgc.IpgcError(rc, "ipgc_server_submit_ref")
        self._n[t.value] = rowptr.size - 1
        return t.value

    def try_submit(self, rowptr, col):
        """Like submit, but returns None when the server is busy right now."""
        try:
            return self.submit(rowptr, col)
        except ipgc.IpgcError as e:
            if e.code == ipgc.IPGC_ERR_BUSY:
                return None
            raise

    def poll(self, ticket: int):
        """None while pending; else (colors, Stats, latency_ns). Releases the ticket."""
        n = self._n.get(ticket, 0)
        out = np.empty(max(n, 0), np.int32)
        st = ipgc.Stats()
        lat = ctypes.c_int64(0)
        rc = lib().ipgc_server_poll(self.handle, ticket, out.ctypes.data if n else None,
                                    ctypes.byref(st), ctypes.byref(lat))
        if rc == ipgc.IPGC_PENDING:
            return None
        self._n.pop(ticket, None)
        if rc != ipgc.IPGC_OK:
            raise ipgc.IpgcError(rc, "ipgc_server_poll")
        return out, st, lat.value

    def next_done(self, timeout_s: float = 1.0):
        t = ctypes.c_uint64(0)
        rc = lib().ipgc_server_next_done(self.handle, ctypes.byref(t), int(timeout_s * 1e9))
        return t.value if rc == ipgc.IPGC_OK else None

    def load_policy(self, w):
        """Load (or with None unload) the network of the learned mode switch."""
        if w is None:
            rc = lib().ipgc_server_policy_load(self.handle, None, 0)
        else:
            w = np.ascontiguousarray(w, dtype=np.float32)
            rc = lib().ipgc_server_policy_load(
                self.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size)
        if rc != ipgc.IPGC_OK:
            raise ipgc.IpgcError(rc, "ipgc_server_policy_load")

    def counters(self) -> ServerCounters:
        c = ServerCounters()
        lib().ipgc_server_query(self.handle, ctypes.byref(c))
        return c

    def close(self):
        if getattr(self, "handle", None):
            lib().ipgc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
