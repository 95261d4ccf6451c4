"""Batches through the C ABI: many graphs refined by one context must give,
graph by graph, exactly what the oracle gives for that graph alone
(partition, cut, block weights), and what the one-graph entry points give.

The batch form keeps every step per graph (own blocks, own L_max, own move
sequence and best prefix), so there is nothing approximate to allow for:
the comparison is bit-exact."""
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


def _mixed(k: int, count: int, seed: int):
    """Graphs of one k with different sizes, weights, hubs and isolated nodes."""
    ws = []
    for i in range(count):
        s = seed * 1000 + i
        n = [30, 200, 700, 64, 1500, 9][i % 6]
        ws.append(synth.random_small(s, n, [3, 6, 4, 8, 5, 2][i % 6], k, weighted=i % 3 != 2,
                                     hubs=i % 4 == 1 and 2 or 0, isolated=i % 5 == 3 and 4 or 0))
    return ws


def _packed(ws):
    return np.concatenate([np.asarray(w.part, np.int32) for w in ws]) if ws else np.zeros(0, np.int32)


def _check_batch(upr, ws, rounds, device):
    import torch
    ctx = upr.create_batch_from_workloads(ws, device=device)
    part = _packed(ws)
    buf = torch.from_numpy(part.copy()).cuda() if device else part.copy()
    status, cin, cout, st = upr.upr_batch_refine(ctx, buf, rounds)
    got = buf.cpu().numpy() if device else buf
    off = ctx.offsets
    cut_b, bw_b = upr.upr_batch_cut(ctx, got)
    for i, w in enumerate(ws):
        rc, ref, cut, _ = oracle.refine(w, w.part, rounds)
        mine = got[off[i]:off[i + 1]]
        if rc == 0:
            assert status[i] == 0, (i, w.name)
            assert np.array_equal(mine, ref), (i, w.name)
            assert cout[i] == cut, (i, w.name)
        else:
            assert status[i] == rc, (i, w.name, status[i], rc)
            assert np.array_equal(mine, w.part), (i, w.name)
            assert cout[i] == cin[i]
        assert cin[i] == oracle.cut(w, w.part)[0], (i, w.name)
        assert cut_b[i] == cout[i]
        bw = np.bincount(mine, weights=w.vwgt if w.vwgt is not None else None, minlength=w.k).astype(np.int64)
        assert np.array_equal(bw_b[i], bw)
    assert st.cut_out == int(cout.sum())
    return ctx


@pytest.mark.parametrize("k", [2, 4, 6, 8, 12, 32, 64])
def test_batch_matches_oracle_per_graph(upr, k):
    _check_batch(upr, _mixed(k, 12, k), rounds=3, device=False)


@pytest.mark.parametrize("k", [8, 256])
def test_batch_device_buffers(upr, k):
    _check_batch(upr, _mixed(k, 7, 50 + k), rounds=2, device=True)


def test_batch_repairs_and_infeasible(upr):
    """Imbalanced inputs in the batch are repaired per graph; a graph that cannot
    be balanced keeps its input and reports UPR_ERR_INFEASIBLE while the others
    are refined as if alone."""
    k = 4
    ws = _mixed(k, 6, 77)
    bad = synth.random_small(91, 120, 4, k, balanced=False)
    # an infeasible graph: one node heavier than L_max allows
    n = 12
    xadj = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    adj = np.array([sorted(((v + 1) % n, (v - 1) % n)) for v in range(n)], np.int32).ravel()
    vw = np.ones(n, np.int32)
    vw[0] = 40
    inf = synth.Workload("infeasible", n, xadj, adj, None, vw, k, 0.03, np.arange(n, dtype=np.int32) % k, 2)
    ws = [ws[0], bad, ws[1], inf, ws[2]]
    _check_batch(upr, ws, rounds=2, device=False)


def test_batch_equals_single_graph_calls(upr):
    ws = _mixed(16, 5, 5)
    ctx = upr.create_batch_from_workloads(ws)
    part = _packed(ws)
    upr.upr_batch_refine(ctx, part, 3)
    off = ctx.offsets
    for i, w in enumerate(ws):
        c1 = upr.create_from_workload(w)
        p1 = np.asarray(w.part, np.int32).copy()
        upr.upr_refine(c1, p1, 3)
        assert np.array_equal(part[off[i]:off[i + 1]], p1)


def test_batch_chung_lu_sample(upr):
    """A sample of the 4096-graph Chung-Lu batch (n log-uniform in [2^10, 2^16]):
    graphs grouped by k, one context per group, against the oracle."""
    ws = [synth.cached(synth.batch_graph, i) for i in range(12)]
    by_k = {}
    for w in ws:
        by_k.setdefault(w.k, []).append(w)
    for k, group in sorted(by_k.items()):
        _check_batch(upr, group, rounds=group[0].rounds, device=True)


def test_one_graph_through_batch_entry(upr):
    w = synth.random_small(3, 300, 5, 8)
    _check_batch(upr, [w], rounds=2, device=False)


def test_batch_rejects_bad_input(upr):
    ws = _mixed(4, 3, 9)
    ctx = upr.create_batch_from_workloads(ws)
    part = _packed(ws)
    part[5] = 4
    with pytest.raises(upr.UprError) as e:
        upr.upr_batch_refine(ctx, part, 1)
    assert e.value.status == upr.UPR_ERR_INVALID
    # a neighbour id outside its own graph
    w = ws[1]
    adj = np.asarray(w.adj, np.int32).copy()
    adj[0] = w.n
    with pytest.raises(upr.UprError) as e:
        upr.upr_batch_create([(ws[0].xadj, ws[0].adj, ws[0].vwgt, ws[0].adjw), (w.xadj, adj, w.vwgt, w.adjw)], 4,
                             0.03)
    assert e.value.status == upr.UPR_ERR_INVALID


def test_batch_repeated_calls_graph_loop(upr):
    """A batch context refined again and again: from the ninth round of the
    binding on, the rebalancing loop runs as a CUDA graph; every call still
    equals the oracle graph by graph."""
    ws = _mixed(16, 10, 77)
    ctx = upr.create_batch_from_workloads(ws)
    used = 0
    for _ in range(3):
        part = _packed(ws)
        status, cin, cout, st = upr.upr_batch_refine(ctx, part, 4)
        used += st.rebalance_graphs
        off = ctx.offsets
        for i, w in enumerate(ws):
            rc, ref, cut, _ = oracle.refine(w, w.part, 4)
            assert status[i] == rc
            if rc == 0:
                assert np.array_equal(part[off[i]:off[i + 1]], ref), i
                assert cout[i] == cut
    assert used > 0


@pytest.mark.parametrize("k", [4, 16, 64])
def test_step_graph_equals_oracle(upr, k):
    """params.graphs = 2: from a binding's second call on, all rounds of a
    call run as one CUDA graph launch (every round's kernels, each
    rebalancing loop a while node).  Calls 1-4 (host-driven, graph built,
    graph replayed, a different round count) and an imbalanced input (its
    repair round runs first, the graph after) equal the oracle graph by
    graph; the graph calls report every round as a graph round."""
    ws = _mixed(k, 8, 91 + k)
    prm = upr.upr_params_default()
    prm.graphs = 2
    ctx = upr.create_batch_from_workloads(ws, params=prm)
    off = ctx.offsets
    seen_graph = 0
    for call, rounds in enumerate((3, 3, 3, 5)):
        part = _packed(ws)
        status, cin, cout, st = upr.upr_batch_refine(ctx, part, rounds)
        for i, w in enumerate(ws):
            rc, ref, cut, _ = oracle.refine(w, w.part, rounds)
            assert status[i] == rc, (call, i)
            if rc == 0:
                assert np.array_equal(part[off[i]:off[i + 1]], ref), (call, i)
                assert cout[i] == cut, (call, i)
        if call >= 1:
            assert st.rebalance_graphs == rounds and st.rounds_run == rounds
            seen_graph += 1
    assert seen_graph == 3
    # an imbalanced graph in the batch: repaired first, then the graph's rounds
    bad = [synth.random_small(1234 + j, 300, 5.0, k, balanced=False) for j in range(2)]
    ws2 = ws[:3] + bad
    ctx2 = upr.create_batch_from_workloads(ws2, params=prm)
    off2 = ctx2.offsets
    for call in range(3):
        part = _packed(ws2)
        status, cin, cout, st = upr.upr_batch_refine(ctx2, part, 3)
        for i, w in enumerate(ws2):
            rc, ref, cut, _ = oracle.refine(w, w.part, 3)
            assert status[i] == rc, (call, i)
            if rc == 0:
                assert np.array_equal(part[off2[i]:off2[i + 1]], ref), (call, i)


@pytest.mark.parametrize("name", ["plain_tiny", "rmat_s12_k64", "weighted"])
def test_step_graph_one_graph(upr, name):
    """The same for one graph (plain tau schedule): partition and cut equal
    the oracle on the host-driven first call and on the graph calls, also
    with the oscillation guard."""
    w = (synth.plain_tiny(3) if name == "plain_tiny" else
         synth.random_small(5, 4000, 10.0, 64, weighted=False, hubs=2) if name == "rmat_s12_k64" else
         synth.random_small(6, 3000, 6.0, 16, max_vw=40, max_ew=30))
    for lock in (0, 1):
        prm = upr.upr_params_default()
        prm.graphs = 2
        prm.lock_rebalanced = lock
        ctx = upr.create_from_workload(w, params=prm)
        rc, ref, cut, _ = oracle.refine_schedule(w, w.part, 4, 0, p=oracle.params(lock_rebalanced=lock))[:4]
        for call in range(3):
            p = w.part.copy()
            st = upr.upr_refine(ctx, p, 4)
            assert np.array_equal(p, ref) and st.cut_out == cut, (call, lock)
            if call >= 1:
                assert st.rebalance_graphs == 4


@pytest.mark.parametrize("graphs_mode", [1, 2])
def test_mixed_k_context_equals_oracle(upr, graphs_mode):
    """One context over graphs of different k (upr_batch_create_mixed): the
    graphs with the same k form one batch each, refined concurrently; every
    graph's partition, status and cut equal the oracle's for that graph
    alone, in the caller's graph order, over several calls (with
    params.graphs = 2 the later calls run each batch's rounds as one graph
    launch), from host and from device buffers; upr_batch_cut gives the
    oracle's cut and k_i block weights per graph."""
    import torch
    ks = [2, 8, 4, 32, 8, 2, 16, 4, 64, 8, 6, 32]
    ws = [synth.random_small(700 + i, [40, 300, 120, 900, 60, 500, 250, 33, 1200, 80, 400, 150][i],
                             [3, 5, 4, 8, 3, 6, 5, 2, 9, 4, 5, 6][i], k, weighted=i % 3 != 1, hubs=1 if i % 4 == 2 else 0)
          for i, k in enumerate(ks)]
    ws.append(synth.random_small(799, 200, 5.0, 8, balanced=False))        # a repair in one of the batches
    prm = upr.upr_params_default()
    prm.graphs = graphs_mode
    ctx = upr.create_batch_from_workloads(ws, params=prm)
    assert ctx.k == 0 and list(ctx.ks) == [w.k for w in ws]
    off = ctx.offsets
    ref = [oracle.refine(w, w.part, 3) for w in ws]
    for call in range(3):
        part = _packed(ws)
        buf = torch.from_numpy(part.copy()).cuda() if call == 1 else part
        status, cin, cout, st = upr.upr_batch_refine(ctx, buf, 3)
        got = buf.cpu().numpy() if call == 1 else buf
        for i, (w, (rc, p0, c0, _)) in enumerate(zip(ws, ref)):
            assert status[i] == rc, (call, i)
            if rc == 0:
                assert np.array_equal(got[off[i]:off[i + 1]], p0), (call, i)
                assert cout[i] == c0, (call, i)
    cuts, bws = upr.upr_batch_cut(ctx, got)
    for i, w in enumerate(ws):
        c, bw = oracle.cut(w, got[off[i]:off[i + 1]])
        assert cuts[i] == c and np.array_equal(bws[i], bw), i


def test_mixed_k_context_refuses_single_graph_calls(upr):
    """upr_refine and upr_cut refuse a mixed context (it is not one graph)."""
    import ctypes
    ws = [synth.random_small(810, 100, 4.0, 4), synth.random_small(811, 100, 4.0, 8)]
    ctx = upr.create_batch_from_workloads(ws)
    part = _packed(ws)
    lib = upr.load()
    assert lib.upr_refine(ctx.handle, part.ctypes.data_as(ctypes.c_void_p), 1, 0, None) == upr.UPR_ERR_INVALID
    cut = ctypes.c_int64()
    assert lib.upr_cut(ctx.handle, part.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cut), None) == upr.UPR_ERR_INVALID


def _check_ctx(upr, ctx, ws, rounds=3):
    part = _packed(ws)
    status, cin, cout, st = upr.upr_batch_refine(ctx, part, rounds)
    off = ctx.offsets
    for i, w in enumerate(ws):
        rc, ref, cut, _ = oracle.refine(w, w.part, rounds)
        assert status[i] == rc, i
        if rc == 0:
            assert np.array_equal(part[off[i]:off[i + 1]], ref), i
            assert cout[i] == cut, i


@pytest.mark.parametrize("graphs_mode", [1, 2])
def test_rebind_contexts(upr, graphs_mode):
    """upr_batch_rebind: a mixed context bound to graphs of other k (a k it
    had reused, a new one added, one dropped) and back, a same-k batch bound
    to other graphs, a one-graph context bound to another graph (smaller:
    its memory reused); every result equals the oracle's; a same-k context
    refuses graphs of several k and stays usable."""
    prm = upr.upr_params_default()
    prm.graphs = graphs_mode
    a = [synth.random_small(900 + i, 150 + 50 * i, 5.0, [4, 8, 4, 8][i]) for i in range(4)]
    b = [synth.random_small(950 + i, 300 + 40 * i, 4.0, [8, 16, 16, 8, 16][i]) for i in range(5)]
    ctx = upr.create_batch_from_workloads(a, params=prm)
    for ws in (a, b, a, b):
        upr.upr_batch_rebind(ctx, [(w.xadj, w.adj, w.vwgt, w.adjw) for w in ws], [w.k for w in ws],
                             [w.eps for w in ws])
        for _ in range(2):
            _check_ctx(upr, ctx, ws)
    same = [synth.random_small(980 + i, 200 + 30 * i, 5.0, 8) for i in range(3)]
    other = [synth.random_small(990 + i, 120 + 30 * i, 6.0, 8) for i in range(4)]
    bctx = upr.create_batch_from_workloads(same, params=prm)
    _check_ctx(upr, bctx, same)
    upr.upr_batch_rebind(bctx, [(w.xadj, w.adj, w.vwgt, w.adjw) for w in other], [8] * 4, [w.eps for w in other])
    _check_ctx(upr, bctx, other)
    with pytest.raises(upr.UprError) as e:
        upr.upr_batch_rebind(bctx, [(w.xadj, w.adj, w.vwgt, w.adjw) for w in b], [w.k for w in b],
                             [w.eps for w in b])
    assert e.value.status == upr.UPR_ERR_INVALID
    _check_ctx(upr, bctx, other)                # unchanged and usable
    big, small = synth.random_small(1001, 3000, 6.0, 16), synth.random_small(1002, 1000, 5.0, 16)
    one = upr.create_batch_from_workloads([big], params=prm)
    _check_ctx(upr, one, [big])
    upr.upr_batch_rebind(one, [(small.xadj, small.adj, small.vwgt, small.adjw)], [16], [small.eps])
    _check_ctx(upr, one, [small])
