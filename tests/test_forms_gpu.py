"""The equivalent forms of the rebalancing sub-round, each against the oracle.

The library computes a one-graph sub-round (K <= 256) in one cooperative
launch by default; UPR_MEGA=0 selects the separate fused kernels (whose
captured form skips the sort's later passes with a conditional node) and
UPR_FUSED=0 the general form.  The switches are read once per process, so
each form runs in a child process that refines the workloads and hands the
partitions back; every form must give the oracle's partition and cut."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (builder, args, rounds): small weighted graphs with hubs, a hub adjacent to
# every node, and R-MAT / weighted RGG cases large enough for multi-tile lists
WORKLOADS = [
    ("random_small", (4, 200, 8, 8), {"hubs": 3}),
    ("random_small", (6, 300, 10, 16), {"hubs": 1, "max_vw": 30, "max_ew": 64}),
    ("plain_large", (10,), {}),
    ("plain_large", (6,), {}),
    ("plain_weighted", (6,), {}),
]

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth
from paper_2308_15494_gb300 import build
build.build()
import paper_2308_15494_gb300 as upr
upr.load()
inp = np.load({inp!r})
out = {{}}
for i, (name, args, kw) in enumerate({workloads!r}):
    fn = getattr(synth, name)
    w = synth.cached(fn, *args) if not kw else fn(*args, **kw)
    ctx = upr.create_from_workload(w)
    for call in range(2):            # the second call runs the captured form
        part = inp[f"p{{i}}"].copy()
        st = upr.upr_refine(ctx, part, w.rounds)
    out[f"p{{i}}"] = part
    out[f"c{{i}}"] = np.array([st.cut_out])
    upr.upr_destroy(ctx)
np.savez({path!r}, **out)
"""


def _workload(name, args, kw):
    fn = getattr(synth, name)
    return synth.cached(fn, *args) if not kw else fn(*args, **kw)


@pytest.fixture(scope="module")
def expected():
    """Per workload: the input partition (an imbalanced one repaired first, as
    upr_refine does) and the oracle's partition and cut from it."""
    oracle.build()
    res = []
    for name, args, kw in WORKLOADS:
        w = _workload(name, args, kw)
        rc, p_in, _, _ = oracle.refine(w, w.part, rounds=0, total_rounds=1)
        if rc != oracle.OK:
            p_in = w.part
        rc, p, c, _ = oracle.refine(w, p_in, rounds=w.rounds)
        assert rc == oracle.OK
        res.append((np.asarray(p_in, np.int32), p, c))
    return res


@pytest.mark.parametrize("env", [{}, {"UPR_MEGA": "0"}, {"UPR_MEGA": "0", "UPR_SORT_IF": "0"}, {"UPR_FUSED": "0"}])
def test_rebalancing_forms_match_oracle(expected, env):
    with tempfile.TemporaryDirectory() as d:
        inp, path = os.path.join(d, "in.npz"), os.path.join(d, "out.npz")
        np.savez(inp, **{f"p{i}": p_in for i, (p_in, _, _) in enumerate(expected)})
        code = CHILD.format(root=ROOT, workloads=WORKLOADS, inp=inp, path=path)
        e = dict(os.environ)
        e.update(env)
        subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=e, check=True, timeout=900)
        got = np.load(path)
        for i, (_, p, c) in enumerate(expected):
            assert np.array_equal(got[f"p{i}"], p), (env, WORKLOADS[i])
            assert int(got[f"c{i}"][0]) == c, (env, WORKLOADS[i])
