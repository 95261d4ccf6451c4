"""Parity of the CUDA library with the CPU oracle, through the C ABI.

Everything the round computes is an integer, so the bar is bit-exact: the
gain table, availability, slots, bucket weights, penalty factors, candidate
targets and scores, the move list M, the rebalancing moves R with their
sub-rounds, the interleaved sequence, the merged sequence I with its exact
gains and balanced prefixes, the applied prefix, the partition, the cut and
the block weights."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def upr():
    from paper_2308_15494_gb300 import build
    build.build()
    import paper_2308_15494_gb300 as m
    m.load()
    return m


def _star_plus(seed, n=6000, k=8):
    """A hub adjacent to every other node (degree above the hub threshold) plus random edges."""
    rng = np.random.default_rng(seed)
    src = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(0, n, 3 * n)])
    dst = np.concatenate([np.arange(1, n), rng.integers(0, n, 3 * n)])
    xadj, adj = synth.csr_from_edges(n, src.astype(np.int32), dst.astype(np.int32))
    part = synth.part_random_balanced(n, k, seed)
    return synth.Workload(f"star{n}", n, xadj, adj, None, None, k, 0.03, part, 3)


def _near_hubs(seed=11, n=9000, k=8, heavy=12, deg=4090):
    """Several nodes of degree just below the hub threshold next to low-degree nodes,
    so tiles of the table build close on their entry budget."""
    rng = np.random.default_rng(seed)
    src = [np.repeat(np.arange(heavy), deg)]
    dst = [np.concatenate([rng.choice(np.arange(heavy, n), size=deg, replace=False) for _ in range(heavy)])]
    src.append(rng.integers(0, n, 2 * n)); dst.append(rng.integers(0, n, 2 * n))
    xadj, adj = synth.csr_from_edges(n, np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32))
    part = synth.part_random_balanced(n, k, seed)
    return synth.Workload("near_hubs", n, xadj, adj, None, None, k, 0.03, part, 3)


def _isolated(n=100, k=4):
    xadj = np.zeros(n + 1, np.int64)
    adj = np.zeros(0, np.int32)
    return synth.Workload("isolated", n, xadj, adj, None, None, k, 0.03, synth.part_random_balanced(n, k, 3), 2)


def _heavy(seed=9, n=300, k=4):
    """Node weights up to 2^20 (wide exact rebalancing keys)."""
    w = synth.random_small(seed, n, 4.0, k, max_vw=(1 << 20) - 1, max_ew=100)
    return w


CASES = {
    "small1": lambda: synth.random_small(1, 40, 4, 3),
    "small2_hubs_isolated": lambda: synth.random_small(2, 64, 6, 4, hubs=2, isolated=3),
    "small3_isolated": lambda: synth.random_small(3, 100, 3, 5, isolated=10),
    "small4_hubs": lambda: synth.random_small(4, 200, 8, 8, hubs=3),
    "small5_unit": lambda: synth.random_small(5, 150, 5, 2, weighted=False),
    "small6_wide": lambda: synth.random_small(6, 300, 10, 16, hubs=1, max_vw=30, max_ew=64),
    "small7_k_gt_n": lambda: synth.random_small(7, 9, 2, 12),
    "k11_odd": lambda: synth.random_small(8, 500, 6, 11, max_vw=5),
    "star_hub": lambda: _star_plus(10),
    "near_hubs": _near_hubs,
    "isolated": _isolated,
    "heavy_weights": _heavy,
    "chung_lu_1k": lambda: synth.plain_tiny(4),
    "rmat_s12_k64": lambda: synth.plain_large(10),
}


def _repaired(w):
    """Imbalanced inputs get the round-0 repair first (as upr_refine does)."""
    rc, p, _, _ = oracle.refine(w, w.part, rounds=0, total_rounds=1)
    if rc == oracle.OK:
        w.part = p
    return w


@pytest.fixture(params=sorted(CASES))
def case(request):
    return _repaired(CASES[request.param]())


def test_cut_and_block_weights(upr, case):
    ctx = upr.create_from_workload(case)
    c, bw = upr.upr_cut(ctx, case.part)
    c0, bw0 = oracle.cut(case, case.part)
    assert c == c0 and np.array_equal(bw, bw0)


def test_gain_table(upr, case):
    ctx = upr.create_from_workload(case)
    W, wI = upr.upr_debug_gain_table(ctx, case.part)
    W0, wI0 = oracle.gain_table(case, case.part)
    assert np.array_equal(W, W0) and np.array_equal(wI, wI0)


def _compare_traces(t, o):
    for key in ("n_cand", "n_moves", "n_rebal", "subrounds", "n_inter", "n_seq", "best_len", "best_gain",
                "cut_before", "cut_after"):
        assert t[key] == o[key], key
    for key in ("avail", "slot", "bucket", "factor", "cand_target", "cand_s0", "cand_gain", "eligible"):
        assert np.array_equal(np.asarray(t[key]), np.asarray(o[key])), key
    for key in ("M", "R", "X", "I"):
        for a, b in zip(t[key], o[key]):
            assert np.array_equal(a, b), key


@pytest.mark.parametrize("r,R", [(1, 4), (4, 4), (1, 1)])
def test_round_trace(upr, case, r, R):
    ctx = upr.create_from_workload(case)
    rc, p, t = upr.upr_debug_round(ctx, case.part, r, R)
    rc0, p0, c0, o = oracle.run_round(case, case.part, r, R)
    assert rc == rc0
    _compare_traces(t, o)
    assert np.array_equal(p, p0)


def test_round_zero_repair_trace(upr):
    w = synth.random_small(41, 400, 5.0, 4, balanced=False)
    assert np.any(brute.block_weights(w, w.part) > brute.lmax(w))
    ctx = upr.create_from_workload(w)
    rc, p, t = upr.upr_debug_round(ctx, w.part, 0, 4, rebalance_only=True)
    rc0, p0, c0, o = oracle.run_round(w, w.part, 0, 4, rebalance_only=True)
    assert rc == rc0 == oracle.OK
    _compare_traces(t, o)
    assert np.array_equal(p, p0)


def test_refine(upr, case):
    ctx = upr.create_from_workload(case)
    part = case.part.copy()
    st = upr.upr_refine(ctx, part, case.rounds)
    rc0, p0, c0, _ = oracle.refine(case, case.part, rounds=case.rounds)
    assert rc0 == oracle.OK
    assert np.array_equal(part, p0) and st.cut_out == c0
    assert st.cut_out <= st.cut_in
    # the input cut (from the first table build when the graph has tiles)
    assert st.cut_in == oracle.cut(case, case.part)[0]


@pytest.mark.parametrize("builder,shrink", [("plain_tiny", 0), ("plain_large", 6), ("plain_weighted", 6)])
def test_refine_configs_scaled(upr, builder, shrink):
    w = _repaired(synth.cached(getattr(synth, builder), shrink))
    ctx = upr.create_from_workload(w)
    part = w.part.copy()
    st = upr.upr_refine(ctx, part, w.rounds)
    rc0, p0, c0, rcuts = oracle.refine(w, w.part, rounds=w.rounds)
    assert np.array_equal(part, p0) and st.cut_out == c0 == rcuts[-1]
    c, bw = upr.upr_cut(ctx, part)
    assert c == c0 and np.array_equal(bw, oracle.cut(w, p0)[1])


def test_device_pointers_match_host(upr):
    import torch
    w = synth.plain_tiny(2)
    host = upr.create_from_workload(w)
    dev = upr.create_from_workload(w, device=True)
    p_host = w.part.copy()
    upr.upr_refine(host, p_host, 3)
    p_dev = torch.from_numpy(w.part.copy()).cuda()
    upr.upr_refine(dev, p_dev, 3)
    torch.cuda.synchronize()
    assert np.array_equal(p_dev.cpu().numpy(), p_host)


def test_imbalanced_input_repaired(upr):
    w = synth.random_small(42, 500, 5.0, 6, balanced=False)
    ctx = upr.create_from_workload(w)
    part = w.part.copy()
    st = upr.upr_refine(ctx, part, 2)
    rc0, p0, c0, _ = oracle.refine(w, w.part, rounds=2)
    assert st.repaired_input == 1 and np.array_equal(part, p0) and st.cut_out == c0


def test_infeasible_input_leaves_part_unchanged(upr):
    xadj, adj = synth.csr_from_edges(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    vw = np.array([10, 1, 1], np.int32)
    w = synth.Workload("heavy", 3, xadj, adj, None, vw, 2, 0.03, np.array([0, 0, 1], np.int32), 1)
    ctx = upr.create_from_workload(w)
    part = w.part.copy()
    with pytest.raises(upr.UprError) as e:
        upr.upr_refine(ctx, part, 1)
    assert e.value.status == upr.UPR_ERR_INFEASIBLE
    assert np.array_equal(part, w.part)
    assert oracle.refine(w, w.part, rounds=1)[0] == oracle.ERR_INFEASIBLE


def test_invalid_inputs_rejected(upr):
    w = synth.random_small(43, 50, 4.0, 3)
    # asymmetric: drop one direction of an edge by editing a neighbour id
    adj = w.adj.copy()
    adj[0] = (adj[0] + 1) % w.n if (adj[0] + 1) % w.n != 0 else 2
    with pytest.raises(upr.UprError) as e:
        upr.upr_create(w.xadj, adj, w.k, w.eps, vwgt=w.vwgt, adjw=w.adjw)
    assert e.value.status == upr.UPR_ERR_INVALID
    # self loop
    xadj, adj2 = synth.csr_from_edges(3, np.array([0], np.int32), np.array([1], np.int32))
    adj_self = np.array([0, 0], np.int32)
    with pytest.raises(upr.UprError):
        upr.upr_create(xadj, adj_self, 2, 0.03)
    # partition out of range: part untouched
    ctx = upr.create_from_workload(w)
    part = w.part.copy()
    part[3] = w.k
    keep = part.copy()
    with pytest.raises(upr.UprError) as e:
        upr.upr_refine(ctx, part, 1)
    assert e.value.status == upr.UPR_ERR_INVALID and np.array_equal(part, keep)
    with pytest.raises(upr.UprError):
        upr.upr_create(w.xadj, w.adj, 1, 0.03)            # k < 2


def _with_duplicate(xadj, adj, v, u):
    """The CSR with the pair {v, u} listed a second time in both rows (still
    symmetric, so only the duplicate check can refuse it)."""
    rows = [list(adj[xadj[i]:xadj[i + 1]]) for i in range(len(xadj) - 1)]
    rows[v].append(u)
    rows[u].append(v)
    x = np.zeros(len(rows) + 1, np.int64)
    x[1:] = np.cumsum([len(r) for r in rows])
    return x, np.array([a for r in rows for a in r], np.int32)


def test_duplicate_entries_rejected(upr):
    """E is a set of pairs (Sec. 2): a row that lists a neighbour twice is
    refused with UPR_ERR_INVALID, in a short row, a row of a few hundred
    entries (the shared-memory hash set) and a hub row of more than 4096
    entries (the bitmap pass), one graph and in a batch; the same graphs
    without the duplicate are accepted."""
    w = synth.random_small(44, 300, 6.0, 4)
    v = 7
    u = int(w.adj[w.xadj[v]])
    x, a = _with_duplicate(w.xadj, w.adj, v, u)
    with pytest.raises(upr.UprError) as e:
        upr.upr_create(x, a, w.k, w.eps)
    assert e.value.status == upr.UPR_ERR_INVALID
    # a row of a few hundred entries: node 0 joined to every third node
    n = 900
    src = np.array([0] * (n // 3 - 1), np.int32)
    dst = np.arange(3, n, 3, dtype=np.int32)[:len(src)]
    ring_s = np.arange(1, n - 1, dtype=np.int32)
    xadj, adj = synth.csr_from_edges(n, np.concatenate([src, ring_s]), np.concatenate([dst, ring_s + 1]))
    upr.upr_destroy(upr.upr_create(xadj, adj, 4, 0.03))
    x, a = _with_duplicate(xadj, adj, 0, 3)
    with pytest.raises(upr.UprError) as e:
        upr.upr_create(x, a, 4, 0.03)
    assert e.value.status == upr.UPR_ERR_INVALID
    # a hub: node 0 joined to all 5999 others, plus a ring
    n = 6000
    src = np.concatenate([np.zeros(n - 1, np.int32), np.arange(1, n - 1, dtype=np.int32)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int32), np.arange(2, n, dtype=np.int32)])
    xadj, adj = synth.csr_from_edges(n, src, dst)
    assert xadj[1] - xadj[0] > 4096
    upr.upr_destroy(upr.upr_create(xadj, adj, 8, 0.03))
    x, a = _with_duplicate(xadj, adj, 0, 4321)
    with pytest.raises(upr.UprError) as e:
        upr.upr_create(x, a, 8, 0.03)
    assert e.value.status == upr.UPR_ERR_INVALID
    # in a batch: one graph with a duplicate makes the call fail
    ws = [synth.random_small(45 + i, 200, 5.0, 4) for i in range(3)]
    xd, ad = _with_duplicate(ws[1].xadj, ws[1].adj, 5, int(ws[1].adj[ws[1].xadj[5]]))
    graphs = [(g.xadj, g.adj, None, None) for g in ws]
    graphs[1] = (xd, ad, None, None)
    with pytest.raises(upr.UprError) as e:
        upr.upr_batch_create(graphs, 4, 0.03)
    assert e.value.status == upr.UPR_ERR_INVALID


@pytest.mark.parametrize("seed", [71, 72, 73])
def test_wide_rebalancing_key_same_results(upr, seed):
    """Node weights near 2^24 with heavy edges: the exact rebalancing key
    (class bit, g*c or floor(|g| 2^(2 cb) / c)) needs 1 + gb + 2 cb > 63 bits
    and is sorted as two words.  Round traces (with the rebalancing sequence
    and its sub-rounds), a repair of an imbalanced input and whole
    refinements equal the oracle's, for the g/c priority and the gain-only
    variant."""
    w = synth.random_small(seed, 1500, 6.0, 8, max_vw=(1 << 24) - 1, max_ew=1 << 20)
    w.eps = 0.01
    wI = np.add.reduceat(w.adjw.astype(np.int64), w.xadj[:-1]) if w.m else np.zeros(1)
    gb, cb = int(wI.max()).bit_length(), int(w.vwgt.max()).bit_length()
    assert 1 + gb + 2 * cb > 63 and wI.max() < 2 ** 31
    ctx = upr.create_from_workload(w)
    for r, R in ((1, 4), (3, 4)):
        rc, p, t = upr.upr_debug_round(ctx, w.part, r, R)
        rc0, p0, c0, o = oracle.run_round(w, w.part, r, R)
        assert rc == rc0
        _compare_traces(t, o)
        assert np.array_equal(p, p0)
    for gp in (0, 1):
        prm = upr.upr_params_default()
        prm.gain_priority = gp
        ctx = upr.create_from_workload(w, params=prm)
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, 4)
        rc0, p0, c0, _ = oracle.refine(w, w.part, rounds=4, p=oracle.params(gain_priority=gp))
        assert np.array_equal(p, p0) and st.cut_out == c0, gp
    # an imbalanced input: everything of block 0 moved to block 1 first
    bad = w.part.copy()
    bad[bad == 0] = 1
    ctx = upr.create_from_workload(w)
    rc0, p0, c0, _ = oracle.refine(w, bad, rounds=2)
    p = bad.copy()
    if rc0 == oracle.OK:
        st = upr.upr_refine(ctx, p, 2)
        assert st.repaired_input == 1 and np.array_equal(p, p0) and st.cut_out == c0
    else:
        with pytest.raises(upr.UprError):
            upr.upr_refine(ctx, p, 2)


def test_unsorted_rows_without_duplicates_accepted(upr):
    """Rows need not be sorted: with every row reversed (so the exact
    duplicate check runs, on short rows, long rows and a hub row) the graph
    is accepted and refines to the oracle's result for the same graph."""
    n = 6000
    src = np.concatenate([np.zeros(n - 1, np.int32), np.arange(1, n - 1, dtype=np.int32),
                          np.arange(0, n - 3, 7, dtype=np.int32)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int32), np.arange(2, n, dtype=np.int32),
                          (np.arange(0, n - 3, 7, dtype=np.int32) * 13 + 5) % n])
    xadj, adj = synth.csr_from_edges(n, src, dst)
    rev = np.concatenate([adj[xadj[v]:xadj[v + 1]][::-1] for v in range(n)]).astype(np.int32)
    w = synth.Workload("rows_reversed", n, xadj, adj, None, None, 8, 0.03, synth.part_random_balanced(n, 8, 5), 3)
    rc0, p0, c0, _ = oracle.refine(w, w.part, 3)
    ctx = upr.upr_create(xadj, rev, 8, 0.03)
    p = w.part.copy()
    st = upr.upr_refine(ctx, p, 3)
    assert np.array_equal(p, p0) and st.cut_out == c0


def test_split_resume_and_seed_independence(upr):
    w = synth.plain_tiny(3)
    full = upr.create_from_workload(w)
    p8 = w.part.copy()
    upr.upr_refine(full, p8, 8, seed=1)
    p8b = w.part.copy()
    upr.upr_refine(full, p8b, 8, seed=12345)
    assert np.array_equal(p8, p8b)
    prm = upr.upr_params_default()
    prm.round_offset, prm.total_rounds = 0, 8
    a = upr.create_from_workload(w, params=prm)
    p = w.part.copy()
    upr.upr_refine(a, p, 3)
    prm2 = upr.upr_params_default()
    prm2.round_offset, prm2.total_rounds = 3, 8
    b = upr.create_from_workload(w, params=prm2)
    upr.upr_refine(b, p, 5)
    assert np.array_equal(p, p8)
    rc0, p0, c0, _ = oracle.refine(w, w.part, rounds=8)
    assert np.array_equal(p8, p0)


def test_server_results_equal_alone_and_in_mix(upr):
    ws = [synth.random_small(50 + i, 200 + 97 * i, 5.0, 2 + (i % 5)) for i in range(6)]
    ws += [synth.plain_tiny(2), synth.plain_large(11)]
    alone = []
    for w in ws:
        ctx = upr.create_from_workload(w)
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, w.rounds)
        alone.append((p, st.cut_out))
    srv = upr.Server(max_jobs=4)
    try:
        tickets = [srv.submit(w) for w in ws]
        for t, (p, c), w in zip(tickets, alone, ws):
            p2, c2, st = srv.wait(t)
            assert np.array_equal(p2, p) and c2 == c
            rc0, p0, c0, _ = oracle.refine(w, w.part, rounds=w.rounds)
            assert np.array_equal(p2, p0)
    finally:
        srv.close()


def _params(upr, table):
    p = upr.upr_params_default()
    p.table = table
    return p


@pytest.mark.parametrize("table", [2, 3])
@pytest.mark.parametrize("name", ["small4_hubs", "small6_wide", "k11_odd", "star_hub", "chung_lu_1k",
                                  "rmat_s12_k64", "heavy_weights"])
def test_sparse_table_same_results(upr, name, table):
    """The sparse gain table (2: rows of min(k, 2 deg) + 1 slots; 3: rows of
    min(k, deg) + 1 slots, which overflow in busy rounds and send the round
    back to the dense table) changes nothing: table, partition and cut equal
    the oracle's."""
    w = CASES[name]()
    ctx = upr.create_from_workload(w, params=_params(upr, table))
    if w.k % 4 == 0:
        W, _ = upr.upr_debug_gain_table(ctx, w.part)
        Wo, _ = oracle.gain_table(w, w.part)
        assert np.array_equal(W, Wo)
    p = w.part.copy()
    st = upr.upr_refine(ctx, p, w.rounds)
    rc, p0, c0, _ = oracle.refine(w, w.part, rounds=w.rounds)
    assert np.array_equal(p, p0)
    assert st.cut_out == c0


@pytest.mark.parametrize("table", [2, 3])
def test_sparse_rows_carried_over_rounds(upr, table):
    """Hashed rows are built once and then follow the moves, the rebalancing
    moves and the end-of-round rollback as delta updates, round after round
    and across calls on one context; a row that runs out of slots sends the
    round back to rows built afresh (then to the dense table).  Nothing of
    this shows in the results."""
    for w in (CASES["rmat_s12_k64"](), synth.random_small(23, 4000, 9, 256, weighted=True, hubs=2)):
        ctx = upr.create_from_workload(w, params=_params(upr, table))
        rounds = 6
        rc, p0, c0, _ = oracle.refine(w, w.part, rounds=rounds)
        for _ in range(2):
            p = w.part.copy()
            st = upr.upr_refine(ctx, p, rounds)
            assert np.array_equal(p, p0), w.name
            assert st.cut_out == c0
        if table == 2:
            assert st.sparse_table == 1
            assert st.gain_table_builds < rounds


def test_sparse_rows_in_a_batch(upr):
    ws = [synth.random_small(40 + i, [300, 900, 50, 2000][i % 4], [5, 9, 3, 7][i % 4], 128,
                             weighted=i % 2 == 0, hubs=1 if i == 1 else 0) for i in range(6)]
    ctx = upr.create_batch_from_workloads(ws, params=_params(upr, 2))
    part = np.concatenate([w.part for w in ws]).astype(np.int32)
    status, cin, cout, st = upr.upr_batch_refine(ctx, part, 4)
    assert st.sparse_table == 1
    off = ctx.offsets
    for i, w in enumerate(ws):
        rc, ref, cut, _ = oracle.refine(w, w.part, rounds=4)
        assert status[i] == rc
        if rc == 0:
            assert np.array_equal(part[off[i]:off[i + 1]], ref), i
            assert cout[i] == cut


def test_rebalancing_graph_same_results(upr):
    """The rebalancing loop run as one CUDA graph launch per round (a while
    node over one sub-round, the stop test on the device) gives what the
    host-driven loop gives; a small binding switches to it after 8 rounds."""
    for w in (CASES["rmat_s12_k64"](), synth.random_small(31, 3000, 6, 8, weighted=True, hubs=1)):
        rc, p0, c0, _ = oracle.refine(w, w.part, rounds=12)
        for graphs in (0, 1):
            prm = upr.upr_params_default()
            prm.graphs = graphs
            ctx = upr.create_from_workload(w, params=prm)
            p = w.part.copy()
            st = upr.upr_refine(ctx, p, 12)
            assert np.array_equal(p, p0), (w.name, graphs)
            assert st.cut_out == c0
            assert (st.rebalance_graphs > 0) == (graphs == 1)


def test_tuned_schedules_shared_between_contexts(upr):
    """A context bound to a graph of the same shape as one tuned before starts
    with the schedules found then (no candidates timed again); results equal."""
    w = synth.cached(synth.plain_large, 2)          # R-MAT, 2^20 nodes, k = 64
    runs = []
    for _ in range(2):
        ctx = upr.create_from_workload(w)
        p = w.part.copy()
        runs.append((p, upr.upr_refine(ctx, p, 2)))
        del ctx
    (p1, s1), (p2, s2) = runs
    assert np.array_equal(p1, p2) and s1.cut_out == s2.cut_out
    assert (s2.select_lanes, s2.propose_lanes) == (s1.select_lanes, s1.propose_lanes)


@pytest.mark.parametrize("schedule", [6, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("name", ["small4_hubs", "small6_wide", "k11_odd", "chung_lu_1k", "rmat_s12_k64",
                                  "heavy_weights", "isolated"])
def test_round_driver_same_results(upr, name, schedule):
    """The round driver of Sec. 4.4 / 6.2 (6: the paper's final
    configuration, unconstrained rounds with tau annealed to 1 and the
    switch below 0.002 of the cut, two closing constrained rounds; 1: dynamic
    activation, the constrained / tau = 1/2 decision of the first two rounds;
    2: constrained rounds only) and the variants of Sec. 7.2 in the final
    configuration's frame (3: constant tau = 1/2, 4: fully unconstrained, 5:
    limited imbalance 2 -> 1.1) equal the oracle's."""
    w = CASES[name]()
    rounds = 7
    op = oracle.params(tau1=(1, 2)) if schedule == 3 else None
    rc, p0, c0, cuts, kinds = oracle.refine_schedule(w, w.part, rounds, schedule, p=op)
    prm = upr.upr_params_default()
    prm.schedule = schedule
    if schedule == 3:
        prm.tau1_num, prm.tau1_den = 1, 2
    ctx = upr.create_from_workload(w, params=prm)
    p = w.part.copy()
    if rc != oracle.OK:
        with pytest.raises(upr.UprError):
            upr.upr_refine(ctx, p, rounds)
        return
    st = upr.upr_refine(ctx, p, rounds)
    assert np.array_equal(p, p0), name
    assert st.cut_out == c0
    assert st.constrained_rounds == int((kinds == oracle.CONSTRAINED).sum())


@pytest.mark.parametrize("name", ["small4_hubs", "small6_wide", "k11_odd", "heavy_weights", "rmat_s12_k64"])
def test_gain_priority_same_results(upr, name):
    """Rebalancing by the gain alone (the variant of Sec. 7.2) equals the oracle."""
    w = CASES[name]()
    w.eps = 0.01
    rc, p0, c0, _ = oracle.refine(w, w.part, rounds=4, p=oracle.params(gain_priority=1))
    prm = upr.upr_params_default()
    prm.gain_priority = 1
    ctx = upr.create_from_workload(w, params=prm)
    p = w.part.copy()
    if rc != oracle.OK:
        with pytest.raises(upr.UprError):
            upr.upr_refine(ctx, p, 4)
        return
    st = upr.upr_refine(ctx, p, 4)
    assert np.array_equal(p, p0) and st.cut_out == c0


@pytest.mark.parametrize("name", ["small4_hubs", "small6_wide", "k11_odd", "heavy_weights", "rmat_s12_k64"])
def test_appended_sequence_same_results(upr, name):
    """The rebalancing moves appended after M (the variant of Sec. 7.2): the
    round's lists and the refinement equal the oracle's."""
    w = CASES[name]()
    w.eps = 0.01
    prm = upr.upr_params_default()
    prm.append = 1
    ctx = upr.create_from_workload(w, params=prm)
    op = oracle.params(append=1)
    rc, p, t = upr.upr_debug_round(ctx, w.part, 1, 3)
    rc0, p0, c0, o = oracle.run_round(w, w.part, 1, 3, p=op)
    assert rc == rc0
    if rc0 == oracle.OK:
        _compare_traces(t, o)
        assert np.array_equal(p, p0)
    rc, p0, c0, _ = oracle.refine(w, w.part, rounds=4, p=op)
    p = w.part.copy()
    if rc != oracle.OK:
        with pytest.raises(upr.UprError):
            upr.upr_refine(ctx, p, 4)
        return
    st = upr.upr_refine(ctx, p, 4)
    assert np.array_equal(p, p0) and st.cut_out == c0


@pytest.mark.parametrize("name", ["small4_hubs", "small6_wide", "k11_odd", "chung_lu_1k", "rmat_s12_k64",
                                  "heavy_weights", "isolated", "star_hub"])
def test_label_propagation_same_results(upr, name):
    """Unconstrained label propagation (Sec. 5) before the FM rounds, alone
    (no FM round) and followed by FM rounds, equals the oracle."""
    w = CASES[name]()
    prm = upr.upr_params_default()
    prm.lp_rounds = 5
    ctx = upr.create_from_workload(w, params=prm)
    if np.all(brute.block_weights(w, w.part) <= brute.lmax(w)):
        kept, q, c = oracle.label_propagation(w, w.part, 5)      # label propagation alone
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, 0)
        assert st.lp_rounds == kept and np.array_equal(p, q) and st.cut_out == c
    rc, p0, c0, _ = oracle.refine(w, w.part, rounds=3, p=oracle.params(lp_rounds=5))
    p = w.part.copy()
    if rc != oracle.OK:
        with pytest.raises(upr.UprError):
            upr.upr_refine(ctx, p, 3)
        return
    st = upr.upr_refine(ctx, p, 3)
    assert np.array_equal(p, p0), name
    assert st.cut_out == c0


@pytest.mark.parametrize("table", [2, 3])
def test_label_propagation_on_hashed_rows(upr, table):
    for w in (CASES["rmat_s12_k64"](), synth.random_small(23, 4000, 9, 256, weighted=True, hubs=2)):
        rc, p0, c0, _ = oracle.refine(w, w.part, rounds=2, p=oracle.params(lp_rounds=5))
        prm = upr.upr_params_default()
        prm.lp_rounds = 5
        prm.table = table
        ctx = upr.create_from_workload(w, params=prm)
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, 2)
        assert np.array_equal(p, p0) and st.cut_out == c0


@pytest.mark.parametrize("schedule", [6, 1])
def test_label_propagation_with_the_round_driver(upr, schedule):
    """Label propagation (Sec. 5) before the FM rounds of the paper's final
    configuration (6) and of dynamic activation (1)."""
    w = CASES["chung_lu_1k"]()
    rc, p0, c0, cuts, kinds = oracle.refine_schedule(w, w.part, 6, schedule, p=oracle.params(lp_rounds=5))
    prm = upr.upr_params_default()
    prm.lp_rounds = 5
    prm.schedule = schedule
    ctx = upr.create_from_workload(w, params=prm)
    p = w.part.copy()
    st = upr.upr_refine(ctx, p, 6)
    assert np.array_equal(p, p0) and st.cut_out == c0


@pytest.mark.parametrize("seed", [41, 44, 45, 47])
def test_oscillation_guard_same_results(upr, seed):
    """The oscillation guard of Sec. 2 (a node whose applied move came from
    rebalancing alone is no candidate in the next round), with the plain
    rounds and with the fully unconstrained variant (where it changes the
    outcome), equals the oracle."""
    w = synth.random_small(seed, 600, 8, 4, weighted=seed % 2 == 0)
    w.eps = 0.01
    for schedule in (0, 4):
        rc, p0, c0, cuts, kinds = oracle.refine_schedule(w, w.part, 5, schedule,
                                                         p=oracle.params(lock_rebalanced=1))
        prm = upr.upr_params_default()
        prm.schedule = schedule
        prm.lock_rebalanced = 1
        ctx = upr.create_from_workload(w, params=prm)
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, 5)
        assert np.array_equal(p, p0), (seed, schedule)
        assert st.cut_out == c0


def test_round_driver_on_a_tight_case(upr):
    w = synth.random_small(11, 4000, 8, 16, weighted=True, max_vw=20)
    w.eps = 0.005
    for schedule in (6, 1, 2, 4, 5):
        rc, p0, c0, cuts, kinds = oracle.refine_schedule(w, w.part, 6, schedule)
        prm = upr.upr_params_default()
        prm.schedule = schedule
        ctx = upr.create_from_workload(w, params=prm)
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, 6)
        assert np.array_equal(p, p0) and st.cut_out == c0


@pytest.mark.parametrize("schedule", [6, 1])
def test_round_driver_needs_one_graph_and_a_whole_schedule(upr, schedule):
    prm = upr.upr_params_default()
    prm.schedule = schedule
    ws = [synth.random_small(60 + i, 100, 4, 4) for i in range(3)]
    ctx = upr.create_batch_from_workloads(ws, params=prm)
    with pytest.raises(upr.UprError):
        upr.upr_batch_refine(ctx, np.concatenate([w.part for w in ws]).astype(np.int32), 3)
    w = ws[0]
    prm.round_offset = 1
    ctx = upr.create_from_workload(w, params=prm)
    with pytest.raises(upr.UprError):
        upr.upr_refine(ctx, w.part.copy(), 3)


def test_sparse_table_chosen_by_size(upr):
    """Auto layout: hashed rows for k >= 128 when they take at most half the
    dense table's bytes (sparse graphs), the dense table otherwise."""
    for k, deg, want in ((256, 6, 1), (64, 6, 0), (128, 200, 0)):
        w = synth.random_small(21, 3000, deg, k, max_vw=20)
        ctx = upr.create_from_workload(w)
        p = w.part.copy()
        st = upr.upr_refine(ctx, p, 3)
        assert st.sparse_table == want, (k, deg)
        rc, p0, c0, _ = oracle.refine(w, w.part, rounds=3)
        assert np.array_equal(p, p0) and st.cut_out == c0
