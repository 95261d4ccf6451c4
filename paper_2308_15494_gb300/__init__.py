"""Python binding of the upr C ABI (include/upr.h).

Argument marshalling only: every step of the refinement runs in the CUDA
library libupr.so built next to this file (see build.py).  Arrays may be
numpy arrays (host) or torch CUDA tensors (device); torch supplies device
memory and the current stream.  Importing this package does not load the
library; the first call does, and raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libupr.so")

UPR_OK, UPR_PENDING = 0, 1
UPR_ERR_INVALID, UPR_ERR_OOM, UPR_ERR_CUDA, UPR_ERR_INFEASIBLE = -1, -2, -3, -4
UPR_ERR_BUSY, UPR_ERR_TIMEOUT, UPR_ERR_NOT_FOUND = -5, -6, -7
NSLOT = 73

P = ctypes.c_void_p
I32, I64, U64, D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


class Graph(ctypes.Structure):
    _fields_ = [("n", I64), ("m", I64), ("xadj", P), ("adjncy", P), ("vwgt", P), ("adjwgt", P), ("on_device", I32)]


class Params(ctypes.Structure):
    _fields_ = [("t_num", I32), ("t_den", I32), ("tau1_num", I32), ("tau1_den", I32), ("max_subrounds", I32),
                ("validate", I32), ("round_offset", I32), ("total_rounds", I32), ("autotune", I32), ("table", I32),
                ("graphs", I32), ("schedule", I32), ("gain_priority", I32), ("append", I32),
                ("lp_rounds", I32), ("lock_rebalanced", I32), ("stream", P)]


class Stats(ctypes.Structure):
    _fields_ = [("cut_in", I64), ("cut_out", I64), ("rounds_run", I32), ("repaired_input", I32),
                ("n_candidates", I64), ("n_moves", I64), ("n_rebalance_moves", I64), ("n_sequence", I64),
                ("n_applied", I64), ("subrounds", I32), ("kernel_launches", I32), ("ms_device", D),
                ("ms_gain_table", D), ("gain_table_builds", I32), ("gain_table_bytes", I64),
                ("ms_select", D), ("ms_rebalance", D), ("ms_sequence", D), ("ms_host", D),
                ("batch_graphs", I32), ("select_lanes", I32), ("propose_lanes", I32),
                ("sparse_table", I32), ("rebalance_graphs", I32), ("constrained_rounds", I32),
                ("lp_rounds", I32), ("lp_table_builds", I32), ("seq_degree_sum", I64), ("bytes_algorithmic", I64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("max_jobs", I32), ("queue_capacity", I32), ("memory_budget", I64), ("params", Params),
                ("batch_max_jobs", I32), ("batch_max_nodes", I32), ("batch_max_total_nodes", I64)]


class Trace(ctypes.Structure):
    _fields_ = [("avail", P), ("slot", P), ("bucket", P), ("factor", P),
                ("cand_target", P), ("cand_s0", P), ("cand_gain", P), ("n_cand", I64),
                ("n_moves", I64), ("M_node", P), ("M_to", P), ("M_score", P),
                ("n_rebal", I64), ("subrounds", I32),
                ("R_node", P), ("R_from", P), ("R_to", P), ("R_subround", P),
                ("n_inter", I64), ("X_node", P), ("X_from", P), ("X_to", P),
                ("n_seq", I64), ("I_node", P), ("I_from", P), ("I_to", P),
                ("I_gain", P), ("I_eligible", P),
                ("best_len", I64), ("best_gain", I64), ("cut_before", I64), ("cut_after", I64)]


# Every symbol include/upr.h declares, with its ctypes signature.
SIGNATURES = {
    "upr_params_default": (None, [ctypes.POINTER(Params)]),
    "upr_status_str": (ctypes.c_char_p, [I32]),
    "upr_create": (I32, [ctypes.POINTER(Graph), I32, D, ctypes.POINTER(Params), ctypes.POINTER(P)]),
    "upr_refine": (I32, [P, P, I32, U64, ctypes.POINTER(Stats)]),
    "upr_cut": (I32, [P, P, ctypes.POINTER(I64), P]),
    "upr_destroy": (None, [P]),
    "upr_cut_noalloc": (I32, [ctypes.POINTER(Graph), I32, P, P, ctypes.POINTER(I64), P]),
    "upr_server_params_default": (None, [ctypes.POINTER(ServerParams)]),
    "upr_server_create": (I32, [ctypes.POINTER(ServerParams), ctypes.POINTER(P)]),
    "upr_submit": (I32, [P, ctypes.POINTER(Graph), I32, D, P, I32, U64, ctypes.POINTER(U64)]),
    "upr_poll": (I32, [P, U64, P, ctypes.POINTER(I64), ctypes.POINTER(Stats)]),
    "upr_wait": (I32, [P, U64, I64, P, ctypes.POINTER(I64), ctypes.POINTER(Stats)]),
    "upr_server_destroy": (None, [P]),
    "upr_debug_gain_table": (I32, [P, P, P, P]),
    "upr_debug_round": (I32, [P, P, I32, I32, I32, ctypes.POINTER(Trace)]),
    "upr_batch_create": (I32, [ctypes.POINTER(Graph), I32, I32, P, ctypes.POINTER(Params), ctypes.POINTER(P)]),
    "upr_batch_create_mixed": (I32, [ctypes.POINTER(Graph), I32, P, P, ctypes.POINTER(Params), ctypes.POINTER(P)]),
    "upr_batch_rebind": (I32, [P, ctypes.POINTER(Graph), I32, P, P]),
    "upr_batch_refine": (I32, [P, P, I32, U64, P, P, P, ctypes.POINTER(Stats)]),
    "upr_batch_cut": (I32, [P, P, P, P]),
    "upr_batch_info": (I32, [P, ctypes.POINTER(I32), P, P]),
}

_lib = None


class UprError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_name(status)} ({status})")


def load(path: str = LIB_PATH):
    """Loads libupr.so and binds every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run paper_2308_15494_gb300.build.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(s: int) -> str:
    return load().upr_status_str(s).decode()


# --------------------------------------------------------------- marshalling
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(P)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def upr_params_default() -> Params:
    p = Params()
    load().upr_params_default(ctypes.byref(p))
    return p


@dataclass
class Context:
    handle: ctypes.c_void_p
    n: int
    m: int
    k: int
    _keep: tuple = ()

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.upr_destroy(self.handle)
            self.handle = None


def _graph_struct(xadj, adj, vwgt=None, adjw=None):
    n = (xadj.shape[0] if _is_torch(xadj) else len(xadj)) - 1
    m = adj.shape[0] if _is_torch(adj) else len(adj)
    g = Graph(n, m, _ptr(xadj), _ptr(adj), _ptr(vwgt), _ptr(adjw), int(_is_torch(xadj) and xadj.is_cuda))
    return g, n, m


def upr_create(xadj, adj, k: int, eps: float, vwgt=None, adjw=None, params: Optional[Params] = None,
               stream=None) -> Context:
    """upr_create: xadj int64[n+1], adj int32[m], optional vwgt int32[n] / adjw int32[m]."""
    lib = load()
    g, n, m = _graph_struct(xadj, adj, vwgt, adjw)
    p = params if params is not None else upr_params_default()
    if stream is not None:
        p.stream = stream
    elif not p.stream:
        p.stream = _current_stream()
    h = ctypes.c_void_p()
    st = lib.upr_create(ctypes.byref(g), k, eps, ctypes.byref(p), ctypes.byref(h))
    if st != UPR_OK:
        raise UprError(st, "upr_create")
    return Context(h, n, m, k)


def create_from_workload(w, params: Optional[Params] = None, device: bool = False) -> Context:
    arrs = [w.xadj, w.adj, w.vwgt, w.adjw]
    if device:
        import torch
        arrs = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    xa, ad, vw, aw = arrs
    return upr_create(xa, ad, w.k, w.eps, vwgt=vw, adjw=aw, params=params)


def upr_refine(ctx: Context, part, rounds: int, seed: int = 0) -> Stats:
    """Refines part (numpy int32 or torch CUDA int32) in place; returns the stats."""
    st = Stats()
    rc = load().upr_refine(ctx.handle, _ptr(part), rounds, seed, ctypes.byref(st))
    if rc != UPR_OK:
        raise UprError(rc, "upr_refine")
    return st


def upr_cut(ctx: Context, part) -> tuple[int, np.ndarray]:
    cut = ctypes.c_int64()
    bw = np.zeros(ctx.k, np.int64)
    rc = load().upr_cut(ctx.handle, _ptr(part), ctypes.byref(cut), _ptr(bw))
    if rc != UPR_OK:
        raise UprError(rc, "upr_cut")
    return int(cut.value), bw


def upr_cut_noalloc(xadj, adj, part, k: int, vwgt=None, adjw=None, stream=None) -> tuple[int, np.ndarray]:
    """upr_cut_noalloc: graph arrays and part are torch CUDA tensors (the
    caller's memory); returns (cut, block weights) without any allocation in
    the library."""
    g, n, m = _graph_struct(xadj, adj, vwgt, adjw)
    cut = ctypes.c_int64()
    bw = np.zeros(k, np.int64)
    s = stream if stream is not None else _current_stream()
    rc = load().upr_cut_noalloc(ctypes.byref(g), k, _ptr(part), s, ctypes.byref(cut), _ptr(bw))
    if rc != UPR_OK:
        raise UprError(rc, "upr_cut_noalloc")
    return int(cut.value), bw


def upr_destroy(ctx: Context) -> None:
    if ctx.handle:
        load().upr_destroy(ctx.handle)
        ctx.handle = None


def upr_debug_gain_table(ctx: Context, part) -> tuple[np.ndarray, np.ndarray]:
    W = np.zeros((ctx.n, ctx.k), np.int32)
    wI = np.zeros(ctx.n, np.int64)
    rc = load().upr_debug_gain_table(ctx.handle, _ptr(part), _ptr(W), _ptr(wI))
    if rc != UPR_OK:
        raise UprError(rc, "upr_debug_gain_table")
    return W, wI


def upr_debug_round(ctx: Context, part: np.ndarray, r: int, R: int, rebalance_only: bool = False):
    """One round on a copy of part; returns (status, new_part, trace dict)."""
    n, k = ctx.n, ctx.k
    part = np.array(part, dtype=np.int32, copy=True)
    a = dict(
        avail=np.zeros(n, np.int8), slot=np.zeros(n, np.int32), bucket=np.zeros(k * NSLOT, np.int64),
        factor=np.zeros(NSLOT, np.int64), cand_target=np.zeros(n, np.int32),
        cand_s0=np.zeros(n, np.int64), cand_gain=np.zeros(n, np.int64),
        M_node=np.zeros(n, np.int32), M_to=np.zeros(n, np.int32), M_score=np.zeros(n, np.int64),
        R_node=np.zeros(n, np.int32), R_from=np.zeros(n, np.int32), R_to=np.zeros(n, np.int32),
        R_subround=np.zeros(n, np.int32),
        X_node=np.zeros(2 * n, np.int32), X_from=np.zeros(2 * n, np.int32), X_to=np.zeros(2 * n, np.int32),
        I_node=np.zeros(n, np.int32), I_from=np.zeros(n, np.int32), I_to=np.zeros(n, np.int32),
        I_gain=np.zeros(n, np.int64), I_eligible=np.zeros(n + 1, np.int8))
    t = Trace(**{key: _ptr(v) for key, v in a.items()})
    rc = load().upr_debug_round(ctx.handle, _ptr(part), r, R, int(rebalance_only), ctypes.byref(t))
    tr = {f: getattr(t, f) for f in ("n_cand", "n_moves", "n_rebal", "subrounds", "n_inter", "n_seq", "best_len",
                                     "best_gain", "cut_before", "cut_after")}
    tr.update(avail=a["avail"], slot=a["slot"], bucket=a["bucket"].reshape(k, NSLOT), factor=a["factor"],
              cand_target=a["cand_target"], cand_s0=a["cand_s0"], cand_gain=a["cand_gain"])
    nm, nr, nx, ns = t.n_moves, t.n_rebal, t.n_inter, t.n_seq
    tr["M"] = (a["M_node"][:nm], a["M_to"][:nm], a["M_score"][:nm])
    tr["R"] = (a["R_node"][:nr], a["R_from"][:nr], a["R_to"][:nr], a["R_subround"][:nr])
    tr["X"] = (a["X_node"][:nx], a["X_from"][:nx], a["X_to"][:nx])
    tr["I"] = (a["I_node"][:ns], a["I_from"][:ns], a["I_to"][:ns], a["I_gain"][:ns])
    tr["eligible"] = a["I_eligible"][: ns + 1].astype(bool)
    return rc, part, tr


# --------------------------------------------------------------- batches
@dataclass
class BatchContext:
    handle: ctypes.c_void_p
    n_graphs: int
    k: int                       # the graphs' k (0: a mixed context, see ks)
    offsets: np.ndarray          # node offsets, n_graphs + 1
    lmax: np.ndarray             # L_max per graph
    ks: Optional[np.ndarray] = None   # per graph k of a mixed context

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.upr_destroy(self.handle)
            self.handle = None


def upr_batch_create(graphs, k: int, eps, params: Optional[Params] = None, stream=None) -> BatchContext:
    """upr_batch_create: graphs = [(xadj, adj, vwgt or None, adjw or None), ...]
    (numpy or torch CUDA arrays, graph-local node ids), one eps or one per graph."""
    lib = load()
    ng = len(graphs)
    arr = (Graph * max(ng, 1))()
    for i, (xa, ad, vw, aw) in enumerate(graphs):
        arr[i], _, _ = _graph_struct(xa, ad, vw, aw)
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (ng,)))
    p = params if params is not None else upr_params_default()
    if stream is not None:
        p.stream = stream
    elif not p.stream:
        p.stream = _current_stream()
    h = ctypes.c_void_p()
    st = lib.upr_batch_create(arr, ng, k, _ptr(e), ctypes.byref(p), ctypes.byref(h))
    if st != UPR_OK:
        raise UprError(st, "upr_batch_create")
    cnt = I32()
    off = np.zeros(ng + 1, np.int64)
    lm = np.zeros(max(ng, 1), np.int64)
    lib.upr_batch_info(h, ctypes.byref(cnt), _ptr(off), _ptr(lm))
    return BatchContext(h, ng, k, off, lm[:ng])


def upr_batch_create_mixed(graphs, ks, eps, params: Optional[Params] = None, stream=None) -> BatchContext:
    """upr_batch_create_mixed: graphs as upr_batch_create, ks[i] = graph i's k."""
    lib = load()
    ng = len(graphs)
    arr = (Graph * max(ng, 1))()
    for i, (xa, ad, vw, aw) in enumerate(graphs):
        arr[i], _, _ = _graph_struct(xa, ad, vw, aw)
    kk = np.ascontiguousarray(np.asarray(ks, np.int32))
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (ng,)))
    p = params if params is not None else upr_params_default()
    if stream is not None:
        p.stream = stream
    elif not p.stream:
        p.stream = _current_stream()
    h = ctypes.c_void_p()
    st = lib.upr_batch_create_mixed(arr, ng, _ptr(kk), _ptr(e), ctypes.byref(p), ctypes.byref(h))
    if st != UPR_OK:
        raise UprError(st, "upr_batch_create_mixed")
    cnt = I32()
    off = np.zeros(ng + 1, np.int64)
    lm = np.zeros(max(ng, 1), np.int64)
    lib.upr_batch_info(h, ctypes.byref(cnt), _ptr(off), _ptr(lm))
    return BatchContext(h, ng, 0, off, lm[:ng], kk.copy())


def upr_rebind(ctx: Context, xadj, adj, k: int, eps: float, vwgt=None, adjw=None) -> Context:
    """upr_batch_rebind of a one-graph context to another graph (its device
    memory reused where it is large enough)."""
    g, n, m = _graph_struct(xadj, adj, vwgt, adjw)
    kk = np.array([k], np.int32)
    e = np.array([eps], np.float64)
    st = load().upr_batch_rebind(ctx.handle, ctypes.byref(g), 1, _ptr(kk), _ptr(e))
    if st != UPR_OK:
        raise UprError(st, "upr_batch_rebind")
    ctx.n, ctx.m, ctx.k = n, m, k
    ctx._keep = (xadj, adj, vwgt, adjw)
    return ctx


def upr_batch_rebind(ctx: BatchContext, graphs, ks, eps) -> BatchContext:
    """upr_batch_rebind: the context bound to other graphs (reusing its device
    memory where it is large enough); returns ctx with its offsets, L_max and
    k updated."""
    lib = load()
    ng = len(graphs)
    arr = (Graph * max(ng, 1))()
    for i, (xa, ad, vw, aw) in enumerate(graphs):
        arr[i], _, _ = _graph_struct(xa, ad, vw, aw)
    kk = np.ascontiguousarray(np.asarray(ks, np.int32))
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (ng,)))
    st = lib.upr_batch_rebind(ctx.handle, arr, ng, _ptr(kk), _ptr(e))
    if st != UPR_OK:
        raise UprError(st, "upr_batch_rebind")
    cnt = I32()
    off = np.zeros(ng + 1, np.int64)
    lm = np.zeros(max(ng, 1), np.int64)
    lib.upr_batch_info(ctx.handle, ctypes.byref(cnt), _ptr(off), _ptr(lm))
    ctx.n_graphs, ctx.offsets, ctx.lmax = ng, off, lm[:ng]
    if ctx.ks is not None:
        ctx.ks = kk.copy()
    else:
        ctx.k = int(kk[0])
    return ctx


def create_batch_from_workloads(ws, params: Optional[Params] = None, device: bool = False) -> BatchContext:
    """One batch context for the workloads (their own eps each): upr_batch_create
    when they share k, upr_batch_create_mixed otherwise."""
    ks = {w.k for w in ws}
    graphs = []
    for w in ws:
        arrs = [w.xadj, w.adj, w.vwgt, w.adjw]
        if device:
            import torch
            arrs = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
        graphs.append(tuple(arrs))
    if len(ks) > 1:
        return upr_batch_create_mixed(graphs, [w.k for w in ws], [w.eps for w in ws], params=params)
    return upr_batch_create(graphs, ws[0].k, [w.eps for w in ws], params=params)


def upr_batch_refine(ctx: BatchContext, part, rounds: int, seed: int = 0):
    """Refines the packed partition in place; returns (status, cut_in, cut_out, stats) arrays per graph."""
    ng = ctx.n_graphs
    status = np.zeros(max(ng, 1), np.int32)
    cin = np.zeros(max(ng, 1), np.int64)
    cout = np.zeros(max(ng, 1), np.int64)
    st = Stats()
    rc = load().upr_batch_refine(ctx.handle, _ptr(part), rounds, seed, _ptr(status), _ptr(cin), _ptr(cout),
                                 ctypes.byref(st))
    if rc != UPR_OK:
        raise UprError(rc, "upr_batch_refine")
    return status[:ng], cin[:ng], cout[:ng], st


def upr_batch_cut(ctx: BatchContext, part):
    """Per-graph cuts and block weights: an (n_graphs, k) array, or for a mixed
    context a list with graph i's k_i weights."""
    cut = np.zeros(max(ctx.n_graphs, 1), np.int64)
    total = int(ctx.ks.sum()) if ctx.ks is not None else ctx.n_graphs * ctx.k
    bw = np.zeros(max(total, 1), np.int64)
    rc = load().upr_batch_cut(ctx.handle, _ptr(part), _ptr(cut), _ptr(bw))
    if rc != UPR_OK:
        raise UprError(rc, "upr_batch_cut")
    if ctx.ks is not None:
        ends = np.cumsum(ctx.ks)
        return cut[: ctx.n_graphs], [bw[e - k:e] for e, k in zip(ends, ctx.ks)]
    return cut[: ctx.n_graphs], bw[: ctx.n_graphs * ctx.k].reshape(ctx.n_graphs, ctx.k)


# --------------------------------------------------------------- serving
class Server:
    """upr_server_create / upr_submit / upr_poll / upr_wait / upr_server_destroy."""

    def __init__(self, max_jobs: int = 8, queue_capacity: int = 4096, memory_budget: int = 0,
                 params: Optional[Params] = None, batch_max_jobs: Optional[int] = None,
                 batch_max_nodes: Optional[int] = None):
        lib = load()
        sp = ServerParams()
        lib.upr_server_params_default(ctypes.byref(sp))
        sp.max_jobs, sp.queue_capacity, sp.memory_budget = max_jobs, queue_capacity, memory_budget
        if batch_max_jobs is not None:
            sp.batch_max_jobs = batch_max_jobs
        if batch_max_nodes is not None:
            sp.batch_max_nodes = batch_max_nodes
        if params is not None:
            sp.params = params
        h = ctypes.c_void_p()
        rc = lib.upr_server_create(ctypes.byref(sp), ctypes.byref(h))
        if rc != UPR_OK:
            raise UprError(rc, "upr_server_create")
        self.handle = h
        self._n = {}

    def submit(self, w, part=None, rounds: Optional[int] = None, seed: int = 0) -> int:
        g, n, m = _graph_struct(np.ascontiguousarray(w.xadj, np.int64), np.ascontiguousarray(w.adj, np.int32),
                                None if w.vwgt is None else np.ascontiguousarray(w.vwgt, np.int32),
                                None if w.adjw is None else np.ascontiguousarray(w.adjw, np.int32))
        keep = (w.xadj, w.adj, w.vwgt, w.adjw)
        part = np.ascontiguousarray(w.part if part is None else part, np.int32)
        t = ctypes.c_uint64()
        rc = load().upr_submit(self.handle, ctypes.byref(g), w.k, w.eps, _ptr(part),
                               w.rounds if rounds is None else rounds, seed, ctypes.byref(t))
        del keep
        if rc != UPR_OK:
            raise UprError(rc, "upr_submit")
        self._n[t.value] = n
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (part, cut, stats)."""
        n = self._n[ticket]
        part = np.zeros(max(n, 1), np.int32)
        cut = ctypes.c_int64()
        st = Stats()
        rc = load().upr_poll(self.handle, ticket, _ptr(part), ctypes.byref(cut), ctypes.byref(st))
        if rc == UPR_PENDING:
            return None
        del self._n[ticket]
        if rc != UPR_OK:
            raise UprError(rc, "upr_poll")
        return part[:n], int(cut.value), st

    def wait(self, ticket: int, timeout_ms: int = 600000):
        n = self._n[ticket]
        part = np.zeros(max(n, 1), np.int32)
        cut = ctypes.c_int64()
        st = Stats()
        rc = load().upr_wait(self.handle, ticket, timeout_ms, _ptr(part), ctypes.byref(cut), ctypes.byref(st))
        if rc == UPR_ERR_TIMEOUT:
            raise UprError(rc, "upr_wait")
        del self._n[ticket]
        if rc != UPR_OK:
            raise UprError(rc, "upr_wait")
        return part[:n], int(cut.value), st

    def close(self):
        if self.handle:
            load().upr_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
