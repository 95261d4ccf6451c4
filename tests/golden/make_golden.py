"""Writes tests/golden/full_size.json: the CPU oracle's results on the
full-size workloads (Chung-Lu n=16384 k=8 4 rounds; R-MAT scale 22 k=64
8 rounds; weighted RGG 2^22 k=256 8 rounds).  Calls only oracle/ and synth/.

Each entry records a digest of the generated input (so a test can tell that
the generator produced the same graph on another machine), the final cut,
the block weights, a digest of the final partition and the cut after every
round.  Run from the repository root: python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size.json")


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        if a is None:
            h.update(b"none")
        else:
            a = np.ascontiguousarray(a)
            h.update(str(a.dtype).encode())
            h.update(a.tobytes())
    return h.hexdigest()


def entry(builder: str):
    w = synth.cached(getattr(synth, builder), 0)
    t = time.time()
    rc, part, cut, rcuts = oracle.refine(w, w.part, rounds=w.rounds)
    assert rc == oracle.OK
    _, bw = oracle.cut(w, part)
    return {
        "builder": builder, "name": w.name, "n": w.n, "m": w.m, "k": w.k, "eps": w.eps, "rounds": w.rounds,
        "input_sha256": digest(w.xadj, w.adj, w.adjw, w.vwgt, w.part),
        "cut_in": int(oracle.cut(w, w.part)[0]), "cut_out": int(cut), "round_cuts": [int(x) for x in rcuts],
        "block_weights": [int(x) for x in bw], "part_sha256": digest(part),
        "source": "oracle.refine (oracle/upr_oracle.cpp), written by tests/golden/make_golden.py",
        "oracle_seconds": round(time.time() - t, 1),
    }


def main(builders):
    data = {}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    for b in builders:
        data[b] = entry(b)
        print(b, data[b]["cut_in"], "->", data[b]["cut_out"], f'{data[b]["oracle_seconds"]} s', flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["plain_tiny", "plain_large", "plain_weighted"])
