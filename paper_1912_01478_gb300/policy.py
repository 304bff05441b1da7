"""Learned per-round mode switch: traces -> features -> GPU training -> policy.

The colouring is the same in every mode (Section V: the versions differ only
in speed), so a graph coloured once with every round forced topology-driven
and once forced data-driven passes through the same sequence of worklists;
round r of the two runs is the same state, and the two trace records give
that round's time in each mode. Those pairs are the training data:
  x = the round's 8 features (computed on the device by
      ipgc_policy_features, the same function the colouring kernel uses),
  y = 1 if topology-driven was faster,
  w = |t_topo - t_data| (a wrong choice costs the time difference).
The network is trained with the library's own CUDA kernels (ipgc_mlp_train)
and loaded into a context with ipgc_policy_load; IPGC_MODE_LEARNED then
evaluates it on the device at the start of every round, the threshold rule
(Section IV) deciding whenever the network is unsure or absent.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import ipgc

NPARAMS = 433
NIN = 8

_P = ctypes.c_void_p
SIGNATURES = {
    "ipgc_policy_features": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P]),
    "ipgc_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "ipgc_mlp_grad": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, _P, _P, _P, _P]),
    "ipgc_mlp_train": (
        ctypes.c_int,
        [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P,
         ctypes.POINTER(ctypes.c_float), _P],
    ),
    "ipgc_policy_load": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
}
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


def _check(rc, what):
    if rc != ipgc.IPGC_OK:
        raise ipgc.IpgcError(rc, what)


def init_weights(seed: int = 0, scale: float = 0.3) -> np.ndarray:
    """Seeded initial parameters (normal, std `scale`; biases zero)."""
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, scale, NPARAMS).astype(np.float32)
    # b1 = [128, 144), b2 = [400, 416), b3 = 432
    w[128:144] = 0
    w[400:416] = 0
    w[432] = 0
    return w


def features(trace_tensor, rounds: int, n: int, nnz: int):
    """Device features (torch float32 [rounds, 8]) of the first `rounds` records."""
    import torch

    out = torch.empty((rounds, NIN), dtype=torch.float32, device=trace_tensor.device)
    _check(lib().ipgc_policy_features(trace_tensor.data_ptr(), rounds, n, nnz, out.data_ptr(), None),
           "ipgc_policy_features")
    return out


def forward(w, x):
    """Network probabilities for CUDA tensors w [433], x [n, 8]."""
    import torch

    p = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().ipgc_mlp_forward(w.data_ptr(), x.data_ptr(), x.shape[0], p.data_ptr(), None),
           "ipgc_mlp_forward")
    return p


def grad(w, x, y, wt):
    """(gradient [433], loss) of the weighted logistic loss on the device."""
    import torch

    n = x.shape[0]
    g = torch.empty(NPARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    scratch = torch.empty((NPARAMS + 1) * n, dtype=torch.float32, device=x.device)
    _check(lib().ipgc_mlp_grad(w.data_ptr(), x.data_ptr(), y.data_ptr(), wt.data_ptr(), n,
                               g.data_ptr(), loss.data_ptr(), scratch.data_ptr(), None),
           "ipgc_mlp_grad")
    return g, float(loss.item())


def train(ctx: "ipgc.Context", x, y, wt, epochs: int = 1500, lr: float = 0.01, seed: int = 0,
          w0: np.ndarray | None = None):
    """Train on the GPU; returns (weights as numpy float32, final loss)."""
    import torch

    w = torch.from_numpy(w0 if w0 is not None else init_weights(seed)).to(x.device).contiguous()
    loss = ctypes.c_float(0)
    _check(lib().ipgc_mlp_train(ctx.handle, x.data_ptr(), y.data_ptr(), wt.data_ptr(), x.shape[0],
                                epochs, lr, w.data_ptr(), ctypes.byref(loss), None),
           "ipgc_mlp_train")
    return w.cpu().numpy(), loss.value


def load(ctx: "ipgc.Context", w: np.ndarray | None):
    """Load (or with None unload) the network used by IPGC_MODE_LEARNED."""
    if w is None:
        _check(lib().ipgc_policy_load(ctx.handle, None, 0), "ipgc_policy_load")
        return
    w = np.ascontiguousarray(w, dtype=np.float32)
    _check(lib().ipgc_policy_load(ctx.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                  w.size), "ipgc_policy_load")


@dataclass
class Traces:
    """Per-round samples of one or more graphs (round 1, always topology-driven, excluded)."""

    x: np.ndarray        # [m, 8] features
    t_topo: np.ndarray   # [m] ns, topology-driven
    t_data: np.ndarray   # [m] ns, data-driven
    thr_topo: np.ndarray  # [m] bool, the threshold rule's choice
    graph: np.ndarray    # [m] index of the graph
    nodes: np.ndarray = None  # [m] n of the round's graph
    wl: np.ndarray = None     # [m] |WL| at the start of the round

    @property
    def y(self):
        return (self.t_topo < self.t_data).astype(np.float32)

    @property
    def w(self):
        return np.abs(self.t_topo - self.t_data).astype(np.float32)

    def totals(self, choose_topo: np.ndarray):
        """Summed round time of a per-round schedule (ns)."""
        return float(np.where(choose_topo, self.t_topo, self.t_data).sum())

    def subset(self, mask):
        return Traces(self.x[mask], self.t_topo[mask], self.t_data[mask], self.thr_topo[mask],
                      self.graph[mask], None if self.nodes is None else self.nodes[mask],
                      None if self.wl is None else self.wl[mask])


def _round_times(tr):
    return (tr["t_detect"].astype(np.int64) - tr["t_begin"].astype(np.int64)).astype(np.float64)


def collect(ctx: "ipgc.Context", graphs, reps: int = 3, threshold_frac: float = 0.6,
            forbidden: str = "auto") -> Traces:
    """Forced-mode traces of every (rowptr, col) graph: the median of `reps`
    runs per mode and round, by default of the library's default colouring
    (forbidden = "auto": bitmaps filled by pushes where a node is above t1);
    forbidden = "rescan" gives the paper's loop (rows rescanned every round,
    which the byte model BYTES_KAPPA describes)."""
    import torch

    xs, tt, td, thr, gi, ns, ws = [], [], [], [], [], [], []
    for g, (rp, cl) in enumerate(graphs):
        n, nnz = rp.size - 1, cl.size
        drp = torch.from_numpy(np.ascontiguousarray(rp, np.int32)).cuda()
        dcl = torch.from_numpy(np.ascontiguousarray(cl, np.int32)).cuda()
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        times = {}
        feats = None
        for mode in ("topo", "data"):
            runs = []
            for _ in range(reps + 1):
                trb = ipgc.trace_buffer(n + 2)
                _, st = ctx.color(drp, dcl, out,
                                  ipgc.ColorOptions(mode=mode, validate=False, forbidden=forbidden),
                                  trace=trb)
                runs.append(_round_times(ipgc.read_trace(trb, st.rounds)))
            times[mode] = np.median(np.stack(runs[1:]), axis=0)  # first run warms up
            if feats is None:
                rec = ipgc.read_trace(trb, st.rounds)
                feats = features(trb, st.rounds, n, nnz).cpu().numpy()
                wl = rec["wl_size"]
        R = len(times["topo"])
        assert len(times["data"]) == R
        sl = slice(1, R)
        xs.append(feats[sl])
        tt.append(times["topo"][sl])
        td.append(times["data"][sl])
        thr.append(wl[sl] > int(threshold_frac * n))
        gi.append(np.full(R - 1, g))
        ns.append(np.full(R - 1, n))
        ws.append(wl[sl])
    cat = lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt)  # noqa: E731
    return Traces(np.concatenate(xs).astype(np.float32) if xs else np.zeros((0, NIN), np.float32),
                  cat(tt, np.float64), cat(td, np.float64), cat(thr, bool), cat(gi, np.int32),
                  cat(ns, np.float64), cat(ws, np.float64))


# Analytical thresholds H (Section VII leaves H to be derived analytically).
#
# Byte model of one round of this build's kernels. Topology-driven, every node
# is visited in order: the row offsets and the colour of each node (assign),
# the row offsets, colour and tentative colour (detect): about 8 + 12 = 20
# bytes per node, read coalesced. Data-driven, every worklist entry costs its
# own read (4 bytes per phase) plus random 32-byte sectors for the node's row
# offsets (each phase) and its tentative colour (detect): about 36 + 68 = 104
# bytes per active node. The neighbour work is the same in both modes, so
# topology-driven is cheaper iff 20 n < 104 |WL|.
BYTES_KAPPA = 20.0 / 104.0


def fit_threshold(tr: Traces):
    """Calibrated model: least squares of t_topo - t_data = a n - b |WL| + c
    over the rounds of the traces; topology-driven iff |WL| > (a n + c) / b.
    Returns (a, b, c)."""
    A = np.stack([tr.nodes, -tr.wl, np.ones_like(tr.wl)], axis=1)
    coef, *_ = np.linalg.lstsq(A, tr.t_topo - tr.t_data, rcond=None)
    return tuple(float(v) for v in coef)


def threshold_choices(tr: Traces, kappa: float | None = None, fit=None):
    """Per-round choices (topology = True) of a threshold rule: |WL| > kappa n,
    or the calibrated rule of fit_threshold's coefficients."""
    if fit is not None:
        a, b, c = fit
        return tr.wl * b > a * tr.nodes + c
    return tr.wl > kappa * tr.nodes


def decisions(w: np.ndarray, x: np.ndarray, margin: float, thr_topo: np.ndarray):
    """The learned policy's per-round choices (topology = True), with the
    threshold rule where |p - 1/2| < margin; evaluated by the device kernel."""
    import torch

    p = forward(torch.from_numpy(w).cuda(), torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    learned = p > 0.5
    return np.where(np.abs(p - 0.5) >= margin, learned, thr_topo), p
