"""upr_cut_noalloc, the allocation-free variant of upr_cut for callers that
cannot allocate device memory themselves through the library (their memory
belongs to another allocator, or cudaMalloc's implicit synchronisation is
not acceptable in their loop).  Its results must equal upr_cut's and the
CPU oracle's on the same inputs, on two calls in a row (the shared static
scratch keeps the previous call's contents, which the call must clear), and
it must refuse, before any kernel indexes with them, CSR arrays that would
send the cut kernels out of bounds.  Collected last on purpose."""
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


def _dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _both(upr, w, part):
    ctx = upr.create_from_workload(w)
    ref = upr.upr_cut(ctx, part)
    upr.upr_destroy(ctx)
    got = upr.upr_cut_noalloc(_dev(w.xadj), _dev(w.adj), _dev(part), w.k, vwgt=_dev(w.vwgt), adjw=_dev(w.adjw))
    return ref, got


def test_noalloc_cut_equals_upr_cut_on_two_calls_in_a_row(upr):
    import torch
    a = synth.random_small(61, 3000, 6.0, 16, hubs=2, max_vw=50, max_ew=20)
    b = synth.plain_tiny(3)                      # different n, m, k, unit weights
    for w, part in ((a, a.part), (b, b.part)):
        (c_ref, bw_ref), (c, bw) = _both(upr, w, part)
        c_or, bw_or = oracle.cut(w, part)
        assert c == c_ref == c_or and np.array_equal(bw, bw_ref) and np.array_equal(bw, bw_or)
    # the same graph again with another partition: nothing left over from before
    p2 = synth.part_random_balanced(a.n, a.k, 99)
    (c_ref, bw_ref), (c, bw) = _both(upr, a, p2)
    c_or, bw_or = oracle.cut(a, p2)
    assert c == c_ref == c_or and np.array_equal(bw, bw_ref) and np.array_equal(bw, bw_or)
    torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_scratch(upr):
    w = synth.random_small(62, 100, 4.0, 3)
    with pytest.raises(upr.UprError) as e:
        upr.upr_cut_noalloc(_dev(w.xadj), _dev(w.adj), _dev(w.part), 4097, vwgt=_dev(w.vwgt), adjw=_dev(w.adjw))
    assert e.value.status == upr.UPR_ERR_INVALID
    bad = w.part.copy()
    bad[0] = 3                                   # outside [0, k)
    with pytest.raises(upr.UprError) as e:
        upr.upr_cut_noalloc(_dev(w.xadj), _dev(w.adj), _dev(bad), w.k, vwgt=_dev(w.vwgt), adjw=_dev(w.adjw))
    assert e.value.status == upr.UPR_ERR_INVALID
    # host arrays are refused: the call cannot copy them without allocating
    with pytest.raises(upr.UprError):
        upr.upr_cut_noalloc(w.xadj, w.adj, w.part, w.k)


def test_noalloc_rejects_a_malformed_csr(upr):
    """Offsets that do not end at m, offsets that decrease, and a neighbour id
    outside [0, n) are refused with UPR_ERR_INVALID (checked on the device
    before the cut kernels read anything through them); a correct call after
    them still gives the oracle's cut."""
    w = synth.random_small(63, 200, 5.0, 4)
    cases = []
    x = w.xadj.copy()
    x[-1] = w.m - 1                              # xadj[n] != m
    cases.append((x, w.adj))
    x = w.xadj.copy()
    x[5], x[6] = x[6], x[5]                      # not non-decreasing
    cases.append((x, w.adj))
    a = w.adj.copy()
    a[0] = w.n                                   # neighbour id outside [0, n)
    cases.append((w.xadj, a))
    a = w.adj.copy()
    a[-1] = -1
    cases.append((w.xadj, a))
    for x, a in cases:
        with pytest.raises(upr.UprError) as e:
            upr.upr_cut_noalloc(_dev(x), _dev(a), _dev(w.part), w.k, vwgt=_dev(w.vwgt), adjw=_dev(w.adjw))
        assert e.value.status == upr.UPR_ERR_INVALID
    c, bw = upr.upr_cut_noalloc(_dev(w.xadj), _dev(w.adj), _dev(w.part), w.k, vwgt=_dev(w.vwgt), adjw=_dev(w.adjw))
    c_or, bw_or = oracle.cut(w, w.part)
    assert c == c_or and np.array_equal(bw, bw_or)
