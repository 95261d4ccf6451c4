"""Serving through the C ABI: continuous batching must not change any result.

Jobs of mixed sizes are submitted in waves while earlier ones run; small
jobs with equal k and rounds are refined together as batches, large ones
alone, on concurrent slots.  Every job's partition and cut must equal the
oracle's for that job alone (and the one-graph entry point's)."""
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


def _mix():
    ws = []
    for i in range(48):
        k = [4, 8, 6][i % 3]
        w = synth.random_small(300 + i, [40, 300, 900, 150][i % 4], [3, 5, 7][i % 3], k,
                               weighted=i % 2 == 0, hubs=1 if i % 7 == 0 else 0)
        w.rounds = 2 + (i % 2)
        ws.append(w)
    ws.insert(5, synth.plain_tiny(1))          # 8k nodes, k=8
    ws.insert(20, synth.plain_large(10))       # 4k nodes, k=64
    ws.insert(33, synth.batch_graph(3))
    return ws


def _expect(w):
    rc, p, c, _ = oracle.refine(w, w.part, rounds=w.rounds)
    return rc, p, c


def _serve(upr, ws, **kw):
    srv = upr.Server(**kw)
    out = {}
    try:
        half = len(ws) // 2
        tickets = [srv.submit(w) for w in ws[:half]]
        # the second wave arrives while the first is on the device
        p0, c0, st0 = srv.wait(tickets[0])
        out[0] = (p0, c0, st0)
        tickets += [srv.submit(w) for w in ws[half:]]
        for i, t in enumerate(tickets):
            if i == 0:
                continue
            try:
                out[i] = srv.wait(t)
            except upr.UprError as e:
                out[i] = e.status
    finally:
        srv.close()
    return out


def _check(ws, out):
    batched = 0
    for i, w in enumerate(ws):
        rc, p, c = _expect(w)
        if rc != 0:
            assert out[i] == rc, (i, w.name)
            continue
        p2, c2, st = out[i]
        assert np.array_equal(p2, p), (i, w.name)
        assert c2 == c, (i, w.name)
        batched += st.batch_graphs > 1
    return batched


def test_continuous_batching_equals_alone(upr):
    ws = _mix()
    out = _serve(upr, ws, max_jobs=3)
    assert _check(ws, out) > 0           # some jobs were refined in batches


def test_batching_off_same_results(upr):
    ws = _mix()[:20]
    out = _serve(upr, ws, max_jobs=2, batch_max_jobs=1)
    assert _check(ws, out) == 0


def test_small_budget_serialises(upr):
    """A budget of a few contexts: work waits for memory, slots give arenas back,
    and nothing changes in the results."""
    ws = _mix()[:24]
    fp = max(w.n for w in ws) * 2000 + (64 << 20)
    out = _serve(upr, ws, max_jobs=4, memory_budget=fp)
    _check(ws, out)


def test_infeasible_job_in_a_batch(upr):
    k = 4
    n = 12
    xadj = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    adj = np.array([sorted(((v + 1) % n, (v - 1) % n)) for v in range(n)], np.int32).ravel()
    vw = np.ones(n, np.int32)
    vw[0] = 40
    inf = synth.Workload("infeasible", n, xadj, adj, None, vw, k, 0.03, np.arange(n, dtype=np.int32) % k, 2)
    ws = [synth.random_small(700 + i, 100, 4, k) for i in range(6)]
    for w in ws:
        w.rounds = 2
    ws.insert(3, inf)
    out = _serve(upr, ws, max_jobs=1)
    _check(ws, out)
    assert out[3] == upr.UPR_ERR_INFEASIBLE


def test_one_slot_rebinds_between_single_and_batch(upr):
    """One slot re-binds its context (and reuses its arena) between large
    single jobs and batches of small ones, so every word a kernel reads must
    be set by the binding itself, whatever the arena held before."""
    ws = []
    for i in range(4):
        ws.append(synth.plain_large(9 + (i % 2)))            # 8k / 4k nodes, k=64, alone
        for j in range(6):
            w = synth.random_small(900 + 10 * i + j, 200 + 50 * j, 5, 64)
            w.rounds = 8
            ws.append(w)                                      # batched together (k=64, 8 rounds)
    out = _serve(upr, ws, max_jobs=1)
    assert _check(ws, out) > 0
