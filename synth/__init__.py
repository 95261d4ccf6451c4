"""Seeded synthetic inputs: graphs, weights and initial partitions.

This package is shared by the CUDA library's tests and benchmark and by the
CPU oracle.  It holds no refinement arithmetic: it only draws graphs with the
structure of the paper's benchmark classes (skewed-degree Chung-Lu and R-MAT
graphs, and random geometric graphs; Sec. 7.1, Table 1), node and edge
weights, and initial partitions.  The paper's own datasets are not used; these
generators stand in for them.

The heavy lifting is in ``gen.c`` (compiled on first use with gcc into
``libsynth.so`` next to it).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

GRAPH_SEED = 0x5EED0001
PART_SEED = 0x5EED1001


def build() -> str:
    """Compile gen.c into libsynth.so if it is missing or older than the source."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64, I32, U64, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        _lib.synth_permutation.argtypes = [I64, U64, P]
        _lib.synth_relabel.argtypes = [I64, P, P, P]
        _lib.synth_chung_lu_edges.argtypes = [I64, D, D, U64, P, P]
        _lib.synth_chung_lu_edges.restype = I64
        _lib.synth_rmat_edges.argtypes = [ctypes.c_int, I64, D, D, D, U64, P, P]
        _lib.synth_rgg_edges.argtypes = [I64, D, U64, P, P, P]
        _lib.synth_rgg_edges.restype = I64
        _lib.synth_build_csr.argtypes = [I64, I64, P, P, P, P]
        _lib.synth_build_csr.restype = I64
        _lib.synth_edge_weights_uniform.argtypes = [I64, P, P, I32, I32, U64, P]
        _lib.synth_node_weights_zipf.argtypes = [I64, D, I32, I32, U64, P]
        _lib.synth_part_random_balanced.argtypes = [I64, I32, U64, P]
        _lib.synth_part_strip.argtypes = [I64, I32, P, P, P]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Workload:
    """A refinement input: CSR graph, weights, k, epsilon, initial partition, rounds."""
    name: str
    n: int
    xadj: np.ndarray                 # int64[n+1]
    adj: np.ndarray                  # int32[m]
    adjw: Optional[np.ndarray]       # int32[m] or None (unit)
    vwgt: Optional[np.ndarray]       # int32[n] or None (unit)
    k: int
    eps: float
    part: np.ndarray                 # int32[n]
    rounds: int
    info: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.xadj[-1])


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray):
    """Symmetrise, drop self loops, dedup and sort an undirected edge list into CSR."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    xadj = np.zeros(n + 1, dtype=np.int64)
    adj = np.empty(max(2 * len(src), 1), dtype=np.int32)
    m = lib.synth_build_csr(n, len(src), _p(src), _p(dst), _p(xadj), _p(adj))
    if m < 0:
        raise MemoryError("synth_build_csr failed")
    return xadj, adj[:m].copy()


def _permute(n, src, dst, seed):
    lib = _load()
    perm = np.empty(n, dtype=np.int32)
    lib.synth_permutation(n, seed, _p(perm))
    lib.synth_relabel(len(src), _p(perm), _p(src), _p(dst))


def chung_lu(n: int, avg_deg: float, gamma: float, seed: int, permute: bool = True):
    lib = _load()
    ne = int(avg_deg * n / 2.0)
    src = np.empty(max(ne, 1), dtype=np.int32)
    dst = np.empty(max(ne, 1), dtype=np.int32)
    ne = lib.synth_chung_lu_edges(n, avg_deg, gamma, seed, _p(src), _p(dst))
    src, dst = src[:ne], dst[:ne]
    if permute:
        _permute(n, src, dst, seed ^ 0xA5A5A5A5)
    return csr_from_edges(n, src, dst)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    lib = _load()
    n = 1 << scale
    ne = edge_factor * n
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    lib.synth_rmat_edges(scale, ne, a, b, c, seed, _p(src), _p(dst))
    _permute(n, src, dst, seed ^ 0xA5A5A5A5)
    return csr_from_edges(n, src, dst)


def rgg(n: int, avg_deg: float, seed: int):
    """Random geometric graph; returns (xadj, adj, xy)."""
    lib = _load()
    radius = math.sqrt(avg_deg / (math.pi * n))
    cnt = lib.synth_rgg_edges(n, radius, seed, None, None, None)
    src = np.empty(max(cnt, 1), dtype=np.int32)
    dst = np.empty(max(cnt, 1), dtype=np.int32)
    xy = np.empty(2 * n, dtype=np.float64)
    cnt2 = lib.synth_rgg_edges(n, radius, seed, _p(src), _p(dst), _p(xy))
    assert cnt2 == cnt
    xadj, adj = csr_from_edges(n, src[:cnt], dst[:cnt])
    return xadj, adj, xy


def edge_weights_uniform(xadj, adj, lo, hi, seed):
    lib = _load()
    n = len(xadj) - 1
    w = np.empty(len(adj), dtype=np.int32)
    lib.synth_edge_weights_uniform(n, _p(xadj), _p(adj), lo, hi, seed, _p(w))
    return w


def node_weights_zipf(n, s, lo, hi, seed):
    lib = _load()
    w = np.empty(n, dtype=np.int32)
    lib.synth_node_weights_zipf(n, s, lo, hi, seed, _p(w))
    return w


def part_random_balanced(n, k, seed):
    lib = _load()
    part = np.empty(max(n, 1), dtype=np.int32)
    lib.synth_part_random_balanced(n, k, seed, _p(part))
    return part[:n].copy()


def part_strip(n, k, xy, vwgt):
    lib = _load()
    part = np.empty(max(n, 1), dtype=np.int32)
    lib.synth_part_strip(n, k, _p(xy), _p(vwgt), _p(part))
    return part[:n].copy()


def cached(fn, *args):
    """Call a workload builder through an on-disk cache (env UPR_SYNTH_CACHE,
    default /tmp/upr_synth_cache) keyed by builder, arguments and gen.c."""
    import hashlib, pickle
    d = os.environ.get("UPR_SYNTH_CACHE", "/tmp/upr_synth_cache")
    h = hashlib.sha1(open(_SRC, "rb").read() + repr((fn.__name__, args)).encode()).hexdigest()[:16]
    path = os.path.join(d, f"{fn.__name__}_{h}.pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    w = fn(*args)
    try:
        os.makedirs(d, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            pickle.dump(w, f, protocol=4)
        os.replace(tmp, path)
    except OSError:
        pass
    return w


# ---------------------------------------------------------------------------
# The five workloads.  `shrink` divides the node count by 2**shrink (same
# generator, degree structure and k), for tests that must finish on the CPU.

def plain_tiny(shrink: int = 0) -> Workload:
    """Chung-Lu power law, n=16384, avg degree 16, exponent 2.2, unit weights, k=8, 4 rounds."""
    n = 16384 >> shrink
    xadj, adj = chung_lu(n, 16.0, 2.2, GRAPH_SEED + 0)
    part = part_random_balanced(n, 8, PART_SEED + 0)
    return Workload(f"chung_lu_n{n}_k8", n, xadj, adj, None, None, 8, 0.03, part, 4,
                    {"generator": "chung-lu", "avg_deg": 16, "gamma": 2.2})


def plain_large(shrink: int = 0) -> Workload:
    """R-MAT scale 22 (a=.57, b=c=.19), edge factor 16, symmetrised+dedup, unit weights, k=64, 8 rounds."""
    scale = 22 - shrink
    xadj, adj = rmat(scale, 16, 0.57, 0.19, 0.19, GRAPH_SEED + 1)
    n = 1 << scale
    part = part_random_balanced(n, 64, PART_SEED + 1)
    return Workload(f"rmat_s{scale}_ef16_k64", n, xadj, adj, None, None, 64, 0.03, part, 8,
                    {"generator": "r-mat", "scale": scale, "edge_factor": 16})


def plain_weighted(shrink: int = 0) -> Workload:
    """RGG 2^22 nodes, avg degree 12, node weights Zipf(1.5) in [1,1024], edge weights U[1,64], k=256, strip split, 8 rounds."""
    n = (1 << 22) >> shrink
    xadj, adj, xy = rgg(n, 12.0, GRAPH_SEED + 2)
    adjw = edge_weights_uniform(xadj, adj, 1, 64, GRAPH_SEED + 102)
    vwgt = node_weights_zipf(n, 1.5, 1, 1024, GRAPH_SEED + 202)
    k = 256
    part = part_strip(n, k, xy, vwgt)
    return Workload(f"rgg_n{n}_k{k}_weighted", n, xadj, adj, adjw, vwgt, k, 0.03, part, 8,
                    {"generator": "rgg", "avg_deg_target": 12})


def batch_graph(i: int, seed: int = GRAPH_SEED + 3) -> Workload:
    """Graph i of the 4096-graph Chung-Lu batch: n log-uniform in [2^10, 2^16],
    avg degree U[4,32], exponent U[2.0,2.8], k from {2,4,8,16,32}."""
    rng = np.random.Generator(np.random.PCG64([seed, i]))
    n = int(round(2.0 ** rng.uniform(10.0, 16.0)))
    d = float(rng.uniform(4.0, 32.0))
    g = float(rng.uniform(2.0, 2.8))
    k = int(rng.choice([2, 4, 8, 16, 32]))
    xadj, adj = chung_lu(n, d, g, seed * 7919 + i)
    part = part_random_balanced(n, k, PART_SEED + 3 + 7919 * i)
    return Workload(f"batch{i}_n{n}_k{k}", n, xadj, adj, None, None, k, 0.03, part, 4,
                    {"generator": "chung-lu", "avg_deg": d, "gamma": g})


def served_rmat(scale: int, k: int, i: int) -> Workload:
    """R-MAT graph i of the served mix: scale 18 or 21, edge factor 16,
    symmetrised+dedup, unit weights, k from {8, 64}, 8 rounds."""
    xadj, adj = rmat(scale, 16, 0.57, 0.19, 0.19, GRAPH_SEED + 5 + 7919 * i + 104729 * scale)
    n = 1 << scale
    part = part_random_balanced(n, k, PART_SEED + 5 + 7919 * i)
    return Workload(f"served_rmat_s{scale}_k{k}_{i}", n, xadj, adj, None, None, k, 0.03, part, 8,
                    {"generator": "r-mat", "scale": scale, "edge_factor": 16})


def _batch_graph_cached(i: int) -> None:
    cached(batch_graph, i)


def batch_graphs(count: int, start: int = 0, workers: Optional[int] = None) -> list:
    """Graphs start .. start+count-1 of the Chung-Lu batch, generated in a
    pool of spawned processes (safe after CUDA is initialised) through the
    on-disk cache, then loaded in order."""
    idx = list(range(start, start + count))
    workers = workers or min(16, os.cpu_count() or 1)
    if workers > 1 and count > 8:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_batch_graph_cached, idx, chunksize=8)
    return [cached(batch_graph, i) for i in idx]


def random_small(seed: int, n: int, avg_deg: float, k: int, weighted: bool = True,
                 hubs: int = 0, isolated: int = 0, max_vw: int = 8, max_ew: int = 9,
                 balanced: bool = True) -> Workload:
    """A small seeded random graph for parity cases: uniform edges plus optional
    hub nodes adjacent to a large share of the graph and isolated nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = int(avg_deg * n / 2)
    src = rng.integers(0, max(n, 1), size=ne, dtype=np.int64)
    dst = rng.integers(0, max(n, 1), size=ne, dtype=np.int64)
    extra_s, extra_d = [], []
    for h in range(min(hubs, n)):
        nb = rng.choice(n, size=max(1, n // 2), replace=False)
        extra_s.append(np.full(len(nb), h)); extra_d.append(nb)
    if extra_s:
        src = np.concatenate([src] + extra_s); dst = np.concatenate([dst] + extra_d)
    if isolated > 0 and n > isolated:
        iso = n - isolated                     # the last `isolated` ids get no edges
        keep = (src < iso) & (dst < iso)
        src, dst = src[keep], dst[keep]
    xadj, adj = csr_from_edges(n, src.astype(np.int32), dst.astype(np.int32))
    adjw = vwgt = None
    if weighted:
        adjw = edge_weights_uniform(xadj, adj, 1, max_ew, seed + 11)
        vwgt = rng.integers(1, max_vw + 1, size=n, dtype=np.int32)
    eps = 0.03
    if balanced:
        if weighted:
            # heaviest first into the lightest block (ties: seeded order, smallest block)
            order = rng.permutation(n)
            order = order[np.argsort(-vwgt[order], kind="stable")]
            part = np.zeros(n, np.int32)
            load = np.zeros(k, np.int64)
            for v in order:
                b = int(np.argmin(load))
                part[v] = b
                load[b] += int(vwgt[v])
            total = int(vwgt.sum())
            while True:            # smallest eps on a 0.01 grid (>= 0.03) that admits this partition
                avg = -(-total // k)
                if load.max() <= (avg * (1000000 + int(round(eps * 1e6)))) // 1000000:
                    break
                eps = round(eps + 0.01, 2)
        else:
            part = part_random_balanced(n, k, seed + 17)
    else:
        part = rng.integers(0, k, size=n, dtype=np.int32)
        part[: n // 2] = 0                     # skew half the nodes into block 0
    return Workload(f"small{seed}_n{n}_k{k}", n, xadj, adj, adjw, vwgt, k, eps, part, 3, {})
