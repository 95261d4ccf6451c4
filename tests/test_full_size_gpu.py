"""Full-size parity: the CUDA library on the full workloads, in the launch
configuration bench.py times (graph and partition resident on the device),
against the oracle's results stored in tests/golden/full_size.json (written
by tests/golden/make_golden.py, which calls only the oracle).

Per workload: the generated input must hash to the stored digest (the
generators are deterministic across machines; a mismatch means the input
changed and the comparison would be meaningless), then the final partition,
cut and block weights must match exactly."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size.json")


def _digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        if a is None:
            h.update(b"none")
        else:
            a = np.ascontiguousarray(a)
            h.update(str(a.dtype).encode())
            h.update(a.tobytes())
    return h.hexdigest()


def _golden():
    if not os.path.exists(GOLDEN):
        return {}
    return json.load(open(GOLDEN))


@pytest.fixture(scope="module")
def upr():
    from paper_2308_15494_gb300 import build
    build.build()
    import paper_2308_15494_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("builder", ["plain_tiny", "plain_large", "plain_weighted"])
def test_full_size_matches_oracle(upr, builder):
    import torch
    g = _golden().get(builder)
    if g is None:
        pytest.skip("no stored oracle result for this workload")
    w = synth.cached(getattr(synth, builder), 0)
    assert _digest(w.xadj, w.adj, w.adjw, w.vwgt, w.part) == g["input_sha256"], "generated input differs"
    ctx = upr.create_from_workload(w, device=True)
    part = torch.from_numpy(w.part.copy()).cuda()
    st = upr.upr_refine(ctx, part, w.rounds)
    torch.cuda.synchronize()
    got = part.cpu().numpy()
    assert st.cut_in == g["cut_in"]
    assert st.cut_out == g["cut_out"]
    assert _digest(got) == g["part_sha256"]
    cut, bw = upr.upr_cut(ctx, part)
    assert cut == g["cut_out"] and list(bw) == g["block_weights"]
    L = (-(-int(np.sum(w.vwgt if w.vwgt is not None else np.ones(w.n))) // w.k) * (10**6 + round(w.eps * 1e6))) // 10**6
    assert max(g["block_weights"]) <= L


def _oracle_job(args):
    """One graph through the oracle (runs in a spawned worker)."""
    import oracle as orc
    import synth as syn
    kind, spec = args
    w = syn.cached(syn.batch_graph, spec) if kind == "batch" else syn.cached(syn.served_rmat, *spec)
    orc.build()
    rc, p, c, _ = orc.refine(w, w.part, w.rounds)
    return rc, p, c


def _oracle_pool(jobs):
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_oracle_job, jobs)


def test_batch_4096_graphs_sampled(upr):
    """The 4096-graph Chung-Lu batch in the bench's launch configuration: one
    context over all graphs (k from {2, 4, 8, 16, 32}: upr_batch_create_mixed,
    one batch per k refined concurrently), params.graphs = 2 (from the second
    call on each batch's rounds are one graph launch), refined twice; every
    graph's status and cut against its balance, and 32 graphs sampled across
    the k values against the oracle bit for bit, on both calls."""
    import torch
    graphs = synth.batch_graphs(4096)
    prm = upr.upr_params_default()
    prm.graphs = 2
    ctx = upr.upr_batch_create_mixed([(w.xadj, w.adj, w.vwgt, w.adjw) for w in graphs], [w.k for w in graphs],
                                     [w.eps for w in graphs], params=prm)
    init = np.concatenate([w.part for w in graphs]).astype(np.int32)
    rounds = graphs[0].rounds
    calls = []
    for call in range(2):
        part = torch.from_numpy(init.copy()).cuda()
        status, cin, cout, stats = upr.upr_batch_refine(ctx, part, rounds)
        torch.cuda.synchronize()
        assert (status == 0).all()
        assert (cout <= cin).all()
        host = part.cpu().numpy()
        calls.append((host, cout.copy(), stats))
        for i, w in enumerate(graphs):
            mine = host[ctx.offsets[i]:ctx.offsets[i + 1]]
            assert np.bincount(mine, minlength=w.k).max() <= ctx.lmax[i], i
    assert np.array_equal(calls[0][0], calls[1][0]) and np.array_equal(calls[0][1], calls[1][1])
    assert calls[1][2].rebalance_graphs == 5 * rounds           # five batches, every round in the graph
    parts = {i: (calls[1][0][ctx.offsets[i]:ctx.offsets[i + 1]], int(calls[1][1][i])) for i in range(len(graphs))}
    sample = sorted({int(x) for x in np.linspace(0, 4095, 32).round()})
    for i, (rc, p, c) in zip(sample, _oracle_pool([("batch", i) for i in sample])):
        assert rc == 0
        assert np.array_equal(parts[i][0], p), i
        assert parts[i][1] == c, i


def test_served_mix_sampled(upr):
    """A burst of the served mix (Chung-Lu batch graphs with their own k, R-MAT
    scale-18 graphs with k from {8, 64}) into the continuous-batching server
    with 8 slots, as the bench serves it: every repeat of an input gives the
    same result, and sampled jobs equal the oracle bit for bit."""
    small = [synth.cached(synth.batch_graph, i) for i in range(48)]
    rmat = [synth.cached(synth.served_rmat, 18, 8 if i < 2 else 64, i) for i in range(4)]
    rng = np.random.default_rng(5)
    jobs = []
    for _ in range(160):
        if rng.random() < 0.55:
            jobs.append(("batch", int(rng.integers(len(small)))))
        else:
            jobs.append(("rmat", int(rng.integers(len(rmat)))))
    srv = upr.Server(max_jobs=8)
    try:
        tickets = [srv.submit(small[j] if kind == "batch" else rmat[j]) for kind, j in jobs]
        out = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    seen = {}
    batched = 0
    for (kind, j), (p, c, st) in zip(jobs, out):
        key = (kind, j)
        if key in seen:
            assert np.array_equal(seen[key][0], p) and seen[key][1] == c
        else:
            seen[key] = (p, c)
        batched += st.batch_graphs > 1
    assert batched > 0
    sample = sorted(seen)[:: max(1, len(seen) // 12)]
    specs = [("batch", j) if kind == "batch" else ("rmat", (18, 8 if j < 2 else 64, j)) for kind, j in sample]
    for key, (rc, p, c) in zip(sample, _oracle_pool(specs)):
        assert rc == 0
        assert np.array_equal(seen[key][0], p), key
        assert seen[key][1] == c, key
