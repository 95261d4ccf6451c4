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
