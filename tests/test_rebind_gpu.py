"""Rebinding a context to a graph of the same shape, and the whole-call graph
after label propagation.

A context with params.graphs = 2 runs a call's rounds as one captured graph
from the binding's second call on.  A rebinding whose host values (sizes,
schedule counts, key widths, arena, parameters, graph offsets and limits)
all equal the previous binding's keeps that graph: the next call replays it
on the new graph's data.  The cases below rebind to graphs with the same
offsets but other neighbours (nodes relabelled within their degree class),
and then to a graph of another shape; every call must give the oracle's
partition and cut, and the calls after a same-shape rebinding must run the
captured graph (no per-phase times: those come from host-driven rounds).
Batches bound from page-locked host arrays (one gather launch per array
kind instead of a copy per graph) must give the oracle's results too."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def upr():
    from paper_2308_15494_gb300 import build
    build.build()
    import paper_2308_15494_gb300 as m
    m.load()
    return m


def _relabelled(w, seed):
    """The graph with its nodes permuted within each degree class: the same
    offsets array, other rows; a fresh balanced random partition."""
    rng = np.random.default_rng(seed)
    n = w.n
    deg = np.diff(w.xadj)
    pi = np.arange(n)
    for d in np.unique(deg):
        idx = np.nonzero(deg == d)[0]
        pi[idx] = rng.permutation(idx)
    inv = np.empty(n, np.int64)
    inv[pi] = np.arange(n)
    adj = np.empty_like(w.adj)
    for u in range(n):
        v = inv[u]
        adj[w.xadj[u]:w.xadj[u + 1]] = np.sort(pi[w.adj[w.xadj[v]:w.xadj[v + 1]]])
    assert w.adjw is None and w.vwgt is None
    part = synth.part_random_balanced(n, w.k, seed)
    return synth.Workload(w.name + f"_relabelled{seed}", n, w.xadj.copy(), adj.astype(np.int32), None, None, w.k,
                          w.eps, part, w.rounds)


def _refine_checked(upr, ctx, w, rounds):
    rc, p0, c0, _ = oracle.refine(w, w.part, rounds=rounds)
    assert rc == oracle.OK
    p = np.asarray(w.part, np.int32).copy()
    st = upr.upr_refine(ctx, p, rounds)
    assert np.array_equal(p, p0), w.name
    assert st.cut_out == c0, w.name
    return st


def test_same_shape_rebind_keeps_the_step_graph(upr):
    a = synth.cached(synth.plain_large, 10)          # R-MAT, 4096 nodes, k = 64
    b, b2 = _relabelled(a, 1), _relabelled(a, 2)
    assert np.array_equal(a.xadj, b.xadj) and not np.array_equal(a.adj, b.adj)
    prm = upr.upr_params_default()
    prm.graphs = 2
    ctx = upr.create_from_workload(a, params=prm)
    rounds = 4
    sts = [_refine_checked(upr, ctx, a, rounds) for _ in range(3)]
    assert sts[0].ms_select > 0 and sts[2].ms_select == 0      # host rounds first, then the graph
    for w in (b, b2, a):
        upr.upr_rebind(ctx, w.xadj, w.adj, w.k, w.eps)
        st = _refine_checked(upr, ctx, w, rounds)
        assert st.ms_select == 0, w.name                        # the kept graph
    other = synth.random_small(77, 3000, 6.0, 64, weighted=False)
    upr.upr_rebind(ctx, other.xadj, other.adj, other.k, other.eps)
    st = _refine_checked(upr, ctx, other, rounds)
    assert st.ms_select > 0                                     # another shape: host rounds again
    for _ in range(2):
        _refine_checked(upr, ctx, other, rounds)
    upr.upr_rebind(ctx, b.xadj, b.adj, b.k, b.eps)
    st = _refine_checked(upr, ctx, b, rounds)
    assert st.ms_select > 0                                     # not the key of the last binding


def test_same_shape_rebind_of_a_batch(upr):
    a = [synth.cached(synth.plain_large, 10), synth.random_small(78, 2500, 5.0, 64, weighted=False)]
    b = [_relabelled(a[0], 3), _relabelled(a[1], 4)]
    prm = upr.upr_params_default()
    prm.graphs = 2
    ctx = upr.create_batch_from_workloads(a, params=prm)
    rounds = 3

    def check(ws):
        part = np.concatenate([np.asarray(w.part, np.int32) for w in ws])
        status, cin, cout, st = upr.upr_batch_refine(ctx, part, rounds)
        off = ctx.offsets
        for i, w in enumerate(ws):
            rc, p0, c0, _ = oracle.refine(w, w.part, rounds)
            assert rc == oracle.OK and status[i] == 0
            assert np.array_equal(part[off[i]:off[i + 1]], p0), w.name
            assert cout[i] == c0
        return st

    sts = [check(a) for _ in range(3)]
    assert sts[2].ms_select == 0
    for ws in (b, a):
        upr.upr_batch_rebind(ctx, [(w.xadj, w.adj, w.vwgt, w.adjw) for w in ws], [w.k for w in ws],
                             [w.eps for w in ws])
        assert check(ws).ms_select == 0


@pytest.mark.parametrize("shrink", [10, 8])
def test_label_propagation_then_the_step_graph(upr, shrink):
    """Label propagation (Sec. 5), then the FM rounds as one captured graph
    from the second call on: every call equals the oracle."""
    w = synth.cached(synth.plain_large, shrink)
    rounds = 3
    rc, p0, c0, _ = oracle.refine(w, w.part, rounds=rounds, p=oracle.params(lp_rounds=5))
    assert rc == oracle.OK
    prm = upr.upr_params_default()
    prm.graphs = 2
    prm.lp_rounds = 5
    ctx = upr.create_from_workload(w, params=prm)
    sts = []
    for _ in range(3):
        p = np.asarray(w.part, np.int32).copy()
        st = upr.upr_refine(ctx, p, rounds)
        assert np.array_equal(p, p0) and st.cut_out == c0
        sts.append(st)
    assert sts[0].ms_select > 0 and sts[2].ms_select == 0


def test_batches_from_page_locked_host_arrays(upr):
    """A batch bound from page-locked host arrays (read by one gather launch
    per array kind) and rebound to other graphs: weighted and unweighted
    graphs, isolated nodes, one graph without edges, several k; every graph
    equals the oracle."""
    import torch

    def pinned(a):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    def graphs_of(seed, k_list):
        ws = []
        for i, k in enumerate(k_list):
            n = [40, 700, 1500, 90, 3000, 12][i % 6]
            ws.append(synth.random_small(seed + i, n, [3, 6, 4, 8, 5, 0.1][i % 6], k, weighted=i % 3 != 2,
                                         hubs=2 if i % 4 == 1 else 0, isolated=4 if i % 5 == 3 else 0))
        return ws

    def check(ctx, ws, rounds=3):
        part = np.concatenate([np.asarray(w.part, np.int32) for w in ws])
        status, cin, cout, st = upr.upr_batch_refine(ctx, part, rounds)
        off = ctx.offsets
        for i, w in enumerate(ws):
            rc, p0, c0, _ = oracle.refine(w, w.part, rounds)
            assert status[i] == rc, (i, w.name)
            if rc == oracle.OK:
                assert np.array_equal(part[off[i]:off[i + 1]], p0), (i, w.name)
                assert cout[i] == c0, (i, w.name)

    for mixed in (False, True):
        a = graphs_of(700, [8] * 7 if not mixed else [4, 8, 16, 8, 4, 16, 8])
        b = graphs_of(800, [8] * 9 if not mixed else [16, 4, 8, 8, 16, 4, 8, 8, 4])
        ga = [tuple(pinned(x) for x in (w.xadj, w.adj, w.vwgt, w.adjw)) for w in a]
        gb = [tuple(pinned(x) for x in (w.xadj, w.adj, w.vwgt, w.adjw)) for w in b]
        if mixed:
            ctx = upr.upr_batch_create_mixed(ga, [w.k for w in a], [w.eps for w in a])
        else:
            ctx = upr.upr_batch_create(ga, 8, [w.eps for w in a])
        check(ctx, a)
        upr.upr_batch_rebind(ctx, gb, [w.k for w in b], [w.eps for w in b])
        check(ctx, b)
        upr.upr_destroy(ctx)
