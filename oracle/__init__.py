"""CPU oracle for the unconstrained-FM refinement round -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product (the CUDA library and its binding)
never does.  The oracle shares no code with the CUDA path; see
``upr_oracle.cpp`` for the step-by-step statement of the round (Algorithm 1
of the paper in its synchronous reading).

What pins each step (tests/test_oracle_pins.py):
  step 0  block weights / cut ........ closed form from an independent COO edge list
  step 1  gain table ................. brute force over COO; delta update == rebuild
  step 2  slots, buckets, F_r ........ defining inequality 1.5^(s-1) < w/c <= 1.5^s in
                                       exact rationals; bucket sums; F_r vs Fraction
  step 2-4 penalty ................... Lemma 1 (Sec. 4.3): level sequence equals the
                                       slots of the cheapest available nodes and the
                                       constructive rebalancing costs <= (1/t) sum pen
  step 3  selection .................. brute-force argmax with gains from cut
                                       differences (parity of the definition only)
  step 4  inflow / order of M ........ M re-derived per target from the candidates with
                                       brute-force penalties of the cumulative inflow;
                                       order (score desc, id asc)
  step 6  rebalancing ................ the whole sequence (node, from, to, sub-round)
                                       equals the sub-rounds of Sec. 6.1 evaluated from
                                       the definitions (gains as cut differences,
                                       priorities in exact rationals, prefixes by
                                       search); post-conditions: balanced when
                                       feasible, every admitted move fits
  step 7  interleave ................. independent re-derivation of the sequential rule
  step 9  exact gains ................ G(j) == cut(P) - cut(P o I^j) by brute force
  step 10 best prefix ................ brute-force max over balanced prefixes; cut never
                                       worse; result balanced
  round   ............................ cut >= exhaustive optimum (n <= 12); two cliques
                                       with one misplaced node reach cut 0
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "upr_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NSLOT = 73
SLOT_LO = -32
OK, ERR_INVALID, ERR_INFEASIBLE = 0, -1, -4


def build() -> str:
    """Compile upr_oracle.cpp (plain g++ -O2) into liboracle.so if stale."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


P = ctypes.c_void_p


class Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("xadj", P), ("adj", P), ("adjw", P), ("vwgt", P)]


class Params(ctypes.Structure):
    _fields_ = [("t_num", ctypes.c_int32), ("t_den", ctypes.c_int32),
                ("tau1_num", ctypes.c_int32), ("tau1_den", ctypes.c_int32),
                ("max_subrounds", ctypes.c_int32), ("gain_priority", ctypes.c_int32), ("append", ctypes.c_int32),
                ("lp_rounds", ctypes.c_int32), ("lock_rebalanced", ctypes.c_int32)]


class Trace(ctypes.Structure):
    _fields_ = [("avail", P), ("slot", P), ("bucket", P), ("factor", P),
                ("cand_target", P), ("cand_s0", P), ("cand_gain", P), ("n_cand", ctypes.c_int64),
                ("n_moves", ctypes.c_int64), ("M_node", P), ("M_to", P), ("M_score", P),
                ("n_rebal", ctypes.c_int64), ("subrounds", ctypes.c_int32),
                ("R_node", P), ("R_from", P), ("R_to", P), ("R_subround", P),
                ("n_inter", ctypes.c_int64), ("X_node", P), ("X_from", P), ("X_to", P),
                ("n_seq", ctypes.c_int64), ("I_node", P), ("I_from", P), ("I_to", P),
                ("I_gain", P), ("I_eligible", P),
                ("best_len", ctypes.c_int64), ("best_gain", ctypes.c_int64),
                ("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        I32, I64 = ctypes.c_int32, ctypes.c_int64
        GP, PP, TP = ctypes.POINTER(Graph), ctypes.POINTER(Params), ctypes.POINTER(Trace)
        lib.upro_params_default.argtypes = [PP]
        lib.upro_lmax.argtypes = [I64, I32, I64]; lib.upro_lmax.restype = I64
        lib.upro_slot.argtypes = [I64, I64]; lib.upro_slot.restype = I32
        lib.upro_factors.argtypes = [I32, I32, PP, P]; lib.upro_factors.restype = ctypes.c_int
        lib.upro_cut.argtypes = [GP, I32, P, P, P]; lib.upro_cut.restype = ctypes.c_int
        lib.upro_gain_table.argtypes = [GP, I32, P, P, P]; lib.upro_gain_table.restype = ctypes.c_int
        lib.upro_penalty_sequence.argtypes = [GP, I32, I64, PP, I32, I32, P, I32, I64, P, P, P]
        lib.upro_penalty_sequence.restype = ctypes.c_int
        lib.upro_round.argtypes = [GP, I32, I64, PP, I32, I32, I32, P, P, TP]
        lib.upro_round.restype = ctypes.c_int
        lib.upro_refine.argtypes = [GP, I32, I64, PP, P, I32, I32, I32, P, P]
        lib.upro_refine.restype = ctypes.c_int
        lib.upro_refine_schedule.argtypes = [GP, I32, I64, PP, P, I32, I32, P, P, P]
        lib.upro_round_kind.argtypes = [GP, I32, I64, PP, I32, I64, I64, I64, P, P, TP]
        lib.upro_round_kind.restype = ctypes.c_int
        lib.upro_round_guard.argtypes = [GP, I32, I64, PP, I32, I32, I64, P, P, P, P, TP]
        lib.upro_round_guard.restype = ctypes.c_int
        lib.upro_lp_round.argtypes = [GP, I32, I64, PP, P, P, P, P, TP]
        lib.upro_lp_round.restype = ctypes.c_int
        lib.upro_label_propagation.argtypes = [GP, I32, I64, PP, P, I32, P]
        lib.upro_label_propagation.restype = ctypes.c_int
        lib.upro_refine_schedule.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(P)


def eps_ppm(eps: float) -> int:
    """epsilon in parts per million, rounded to nearest (the integer form of Sec. 2's epsilon)."""
    return int(round(eps * 1e6))


class _G:
    """Keeps the numpy arrays alive for as long as the ctypes struct is used."""

    def __init__(self, w):
        self.arrays = [np.ascontiguousarray(w.xadj, np.int64), np.ascontiguousarray(w.adj, np.int32),
                       None if w.adjw is None else np.ascontiguousarray(w.adjw, np.int32),
                       None if w.vwgt is None else np.ascontiguousarray(w.vwgt, np.int32)]
        xa, ad, aw, vw = self.arrays
        self.s = Graph(w.n, _ptr(xa), _ptr(ad), _ptr(aw), _ptr(vw))


def params(t=(7, 10), tau1=(1, 4), max_subrounds=64, gain_priority=0, append=0, lp_rounds=0,
           lock_rebalanced=0) -> Params:
    return Params(t[0], t[1], tau1[0], tau1[1], max_subrounds, gain_priority, append, lp_rounds, lock_rebalanced)


def lmax(total_weight: int, k: int, eps: float) -> int:
    return int(_load().upro_lmax(total_weight, k, eps_ppm(eps)))


def slot(omega: int, c: int) -> int:
    return int(_load().upro_slot(omega, c))


def factors(r: int, R: int, p: Optional[Params] = None) -> np.ndarray:
    F = np.zeros(NSLOT, np.int64)
    rc = _load().upro_factors(r, R, ctypes.byref(p) if p else None, _ptr(F))
    if rc != OK:
        raise ValueError("invalid schedule")
    return F


def cut(w, part) -> tuple[int, np.ndarray]:
    g = _G(w)
    part = np.ascontiguousarray(part, np.int32)
    c = ctypes.c_int64(0)
    bw = np.zeros(w.k, np.int64)
    _load().upro_cut(ctypes.byref(g.s), w.k, _ptr(part), ctypes.byref(c), _ptr(bw))
    return int(c.value), bw


def gain_table(w, part) -> tuple[np.ndarray, np.ndarray]:
    g = _G(w)
    part = np.ascontiguousarray(part, np.int32)
    W = np.zeros((w.n, w.k), np.int32)
    wI = np.zeros(w.n, np.int64)
    _load().upro_gain_table(ctypes.byref(g.s), w.k, _ptr(part), _ptr(W), _ptr(wI))
    return W, wI


def penalty_sequence(w, part, block: int, nodes, r: int = 1, R: int = 1,
                     p: Optional[Params] = None) -> tuple[np.ndarray, np.ndarray]:
    g = _G(w)
    part = np.ascontiguousarray(part, np.int32)
    nodes = np.ascontiguousarray(nodes, np.int32)
    pen = np.zeros(len(nodes), np.int64)
    lvl = np.zeros(len(nodes), np.int32)
    _load().upro_penalty_sequence(ctypes.byref(g.s), w.k, eps_ppm(w.eps), ctypes.byref(p) if p else None,
                                  r, R, _ptr(part), block, len(nodes), _ptr(nodes), _ptr(pen), _ptr(lvl))
    return pen, lvl


def run_round(w, part, r: int, R: int, rebalance_only: bool = False, p: Optional[Params] = None,
              kind: Optional[tuple] = None):
    """One round on a copy of part.  Returns (rc, new_part, cut, trace dict).
    kind (Sec. 6.2, 7.2): ("constrained",), ("tau", num, den) or ("limit",
    L) (no penalty, no block above L) instead of the schedule's tau_r."""
    n, k = w.n, w.k
    g = _G(w)
    part = np.array(part, dtype=np.int32, copy=True)
    c0, _ = cut(w, part)
    c = ctypes.c_int64(c0)
    a = dict(
        avail=np.zeros(n, np.int8), slot=np.zeros(n, np.int32), bucket=np.zeros(k * NSLOT, np.int64),
        factor=np.zeros(NSLOT, np.int64), cand_target=np.zeros(n, np.int32),
        cand_s0=np.zeros(n, np.int64), cand_gain=np.zeros(n, np.int64),
        M_node=np.zeros(n, np.int32), M_to=np.zeros(n, np.int32), M_score=np.zeros(n, np.int64),
        R_node=np.zeros(n, np.int32), R_from=np.zeros(n, np.int32), R_to=np.zeros(n, np.int32),
        R_subround=np.zeros(n, np.int32),
        X_node=np.zeros(2 * n, np.int32), X_from=np.zeros(2 * n, np.int32), X_to=np.zeros(2 * n, np.int32),
        I_node=np.zeros(n, np.int32), I_from=np.zeros(n, np.int32), I_to=np.zeros(n, np.int32),
        I_gain=np.zeros(n, np.int64), I_eligible=np.zeros(n + 1, np.int8))
    t = Trace(**{key: _ptr(v) for key, v in a.items()})
    if kind is None:
        rc = _load().upro_round(ctypes.byref(g.s), k, eps_ppm(w.eps), ctypes.byref(p) if p else None,
                                r, R, int(rebalance_only), _ptr(part), ctypes.byref(c), ctypes.byref(t))
    else:
        con = kind[0] == "constrained"
        num, den = (kind[1], kind[2]) if kind[0] == "tau" else (0, 0)
        limit = kind[1] if kind[0] == "limit" else 0
        rc = _load().upro_round_kind(ctypes.byref(g.s), k, eps_ppm(w.eps), ctypes.byref(p) if p else None,
                                     int(con), num, den, limit, _ptr(part), ctypes.byref(c), ctypes.byref(t))
    tr = {"n_cand": t.n_cand, "n_moves": t.n_moves, "n_rebal": t.n_rebal, "subrounds": t.subrounds,
          "n_inter": t.n_inter, "n_seq": t.n_seq, "best_len": t.best_len, "best_gain": t.best_gain,
          "cut_before": t.cut_before, "cut_after": t.cut_after}
    tr["avail"], tr["slot"] = a["avail"], a["slot"]
    tr["bucket"] = a["bucket"].reshape(k, NSLOT)
    tr["factor"] = a["factor"]
    tr["cand_target"], tr["cand_s0"], tr["cand_gain"] = a["cand_target"], a["cand_s0"], a["cand_gain"]
    nm, nr, nx, ns = t.n_moves, t.n_rebal, t.n_inter, t.n_seq
    tr["M"] = (a["M_node"][:nm], a["M_to"][:nm], a["M_score"][:nm])
    tr["R"] = (a["R_node"][:nr], a["R_from"][:nr], a["R_to"][:nr], a["R_subround"][:nr])
    tr["X"] = (a["X_node"][:nx], a["X_from"][:nx], a["X_to"][:nx])
    tr["I"] = (a["I_node"][:ns], a["I_from"][:ns], a["I_to"][:ns], a["I_gain"][:ns])
    tr["eligible"] = a["I_eligible"][: ns + 1].astype(bool)
    return rc, part, int(c.value), tr


def refine(w, part, rounds: Optional[int] = None, round_offset: int = 0,
           total_rounds: Optional[int] = None, p: Optional[Params] = None):
    """Rounds round_offset+1..round_offset+rounds of a total_rounds schedule.
    Returns (rc, new_part, cut, per-round cuts [rounds+1])."""
    rounds = w.rounds if rounds is None else rounds
    total_rounds = rounds + round_offset if total_rounds is None else total_rounds
    g = _G(w)
    part = np.array(part, dtype=np.int32, copy=True)
    c = ctypes.c_int64(0)
    rcuts = np.zeros(rounds + 1, np.int64)
    rc = _load().upro_refine(ctypes.byref(g.s), w.k, eps_ppm(w.eps), ctypes.byref(p) if p else None,
                             _ptr(part), rounds, round_offset, total_rounds, ctypes.byref(c), _ptr(rcuts))
    return rc, part, int(c.value), rcuts


# Round kinds reported by refine_schedule (the round driver of Sec. 4.4 / 6.2
# and the variants of Sec. 7.2).
UNCONSTRAINED, CONSTRAINED, UNCONSTRAINED_HALF, CONSTANT_TAU, NO_PENALTY, LIMITED = 0, 1, 2, 3, 4, 5


def refine_schedule(w, part, rounds: int, schedule: int, p: Optional[Params] = None):
    """The round driver of Sec. 4.4 / Sec. 6.2.  schedule 0 = every round
    unconstrained (tau schedule over the rounds); 6 = the paper's final
    configuration (unconstrained rounds with tau annealed from tau_1 to 1
    over the first U rounds, U = R - 2 for R >= 3, 1 for R = 2, 0 for R = 1,
    the switch to constrained rounds below an improvement of 0.002 of the
    cut, constrained rounds after them); 3-5 = the variants of Sec. 7.2 in
    the same frame (3 constant tau = tau_1, 4 fully unconstrained, 5 limited
    imbalance 2 -> 1.1); 1 = dynamic activation (Sec. 4.4, not in the
    paper's final configuration: constrained round, unconstrained round with
    tau = 1/2, then unconstrained or constrained rounds by the improvements,
    constrained last round); 2 = every round constrained.  Returns (rc,
    new_part, cut, per-round cuts [rounds+1], kind of each round [rounds])."""
    g = _G(w)
    part = np.array(part, dtype=np.int32, copy=True)
    c = ctypes.c_int64(0)
    rcuts = np.zeros(rounds + 1, np.int64)
    kinds = np.zeros(max(rounds, 1), np.int8)
    rc = _load().upro_refine_schedule(ctypes.byref(g.s), w.k, eps_ppm(w.eps), ctypes.byref(p) if p else None,
                                      _ptr(part), rounds, schedule, ctypes.byref(c), _ptr(rcuts), _ptr(kinds))
    return rc, part, int(c.value), rcuts, kinds[:rounds]


def lp_round(w, part, active, p: Optional[Params] = None):
    """One round of unconstrained label propagation (Sec. 5) on a copy of part
    over the active nodes.  Returns (rc, kept, new_part, cut, trace dict with
    the moves "M" = (node, to, gain) and the rebalancing "R")."""
    n = w.n
    g = _G(w)
    part = np.array(part, dtype=np.int32, copy=True)
    active = np.ascontiguousarray(active, np.int8)
    c = ctypes.c_int64(cut(w, part)[0])
    kept = ctypes.c_int32(0)
    a = dict(M_node=np.zeros(n, np.int32), M_to=np.zeros(n, np.int32), M_score=np.zeros(n, np.int64),
             R_node=np.zeros(n, np.int32), R_from=np.zeros(n, np.int32), R_to=np.zeros(n, np.int32),
             R_subround=np.zeros(n, np.int32))
    t = Trace(**{key: _ptr(v) for key, v in a.items()})
    rc = _load().upro_lp_round(ctypes.byref(g.s), w.k, eps_ppm(w.eps), ctypes.byref(p) if p else None, _ptr(active),
                               _ptr(part), ctypes.byref(c), ctypes.byref(kept), ctypes.byref(t))
    nm, nr = t.n_moves, t.n_rebal
    tr = {"M": (a["M_node"][:nm], a["M_to"][:nm], a["M_score"][:nm]),
          "R": (a["R_node"][:nr], a["R_from"][:nr], a["R_to"][:nr], a["R_subround"][:nr]),
          "cut_before": t.cut_before, "cut_after": t.cut_after}
    return rc, bool(kept.value), part, int(c.value), tr


def label_propagation(w, part, max_rounds: int = 5, p: Optional[Params] = None):
    """Unconstrained label propagation alone (Sec. 5).  Returns (rounds kept
    or an error code, new_part, cut)."""
    g = _G(w)
    part = np.array(part, dtype=np.int32, copy=True)
    c = ctypes.c_int64(0)
    kept = _load().upro_label_propagation(ctypes.byref(g.s), w.k, eps_ppm(w.eps), ctypes.byref(p) if p else None,
                                          _ptr(part), max_rounds, ctypes.byref(c))
    return kept, part, int(c.value)


def round_guard(w, part, r: int, R: int, locked, limit: int = 0, p: Optional[Params] = None):
    """One round under the oscillation guard of Sec. 2 (locked nodes are no
    candidates).  Returns (rc, new_part, cut, locked_out, trace dict with
    cand_target, M, R, I, best_len)."""
    n = w.n
    g = _G(w)
    part = np.array(part, dtype=np.int32, copy=True)
    locked = np.ascontiguousarray(locked, np.int8)
    out = np.zeros(n, np.int8)
    c = ctypes.c_int64(cut(w, part)[0])
    a = dict(cand_target=np.zeros(n, np.int32), cand_s0=np.zeros(n, np.int64), cand_gain=np.zeros(n, np.int64),
             M_node=np.zeros(n, np.int32), M_to=np.zeros(n, np.int32), M_score=np.zeros(n, np.int64),
             R_node=np.zeros(n, np.int32), R_from=np.zeros(n, np.int32), R_to=np.zeros(n, np.int32),
             R_subround=np.zeros(n, np.int32), I_node=np.zeros(n, np.int32), I_from=np.zeros(n, np.int32),
             I_to=np.zeros(n, np.int32), I_gain=np.zeros(n, np.int64))
    t = Trace(**{key: _ptr(v) for key, v in a.items()})
    rc = _load().upro_round_guard(ctypes.byref(g.s), w.k, eps_ppm(w.eps), ctypes.byref(p) if p else None, r, R, limit,
                                  _ptr(locked), _ptr(out), _ptr(part), ctypes.byref(c), ctypes.byref(t))
    nm, nr, ns = t.n_moves, t.n_rebal, t.n_seq
    tr = {"cand_target": a["cand_target"], "M": (a["M_node"][:nm], a["M_to"][:nm]),
          "R": (a["R_node"][:nr], a["R_from"][:nr], a["R_to"][:nr]),
          "I": (a["I_node"][:ns], a["I_from"][:ns], a["I_to"][:ns]), "best_len": t.best_len}
    return rc, part, int(c.value), out, tr
