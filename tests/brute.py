"""Brute-force definitions used to pin the oracle, written from the paper's
definitions (Sec. 2, Sec. 4.3) over a COO edge list, independently of the
oracle's code.  Exact rationals (fractions.Fraction) wherever the paper's
quantity is a real number."""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def coo(w):
    """Undirected edge list (u < v) with weights, from the CSR."""
    src = np.repeat(np.arange(w.n, dtype=np.int64), np.diff(w.xadj))
    dst = w.adj.astype(np.int64)
    ew = np.ones(len(dst), np.int64) if w.adjw is None else w.adjw.astype(np.int64)
    keep = src < dst
    return src[keep], dst[keep], ew[keep]


def node_w(w):
    return np.ones(w.n, np.int64) if w.vwgt is None else w.vwgt.astype(np.int64)


def cut(w, part, edges=None):
    """cut(P) = sum of omega over edges whose endpoints lie in different blocks (Sec. 2)."""
    u, v, ew = coo(w) if edges is None else edges
    part = np.asarray(part)
    return int(ew[part[u] != part[v]].sum())


def block_weights(w, part):
    return np.bincount(np.asarray(part), weights=node_w(w), minlength=w.k).astype(np.int64)


def table(w, part):
    """W[v][b] = omega(v, V_b), from both directions of every COO edge."""
    u, v, ew = coo(w)
    part = np.asarray(part)
    W = np.zeros((w.n, w.k), np.int64)
    np.add.at(W, (u, part[v]), ew)
    np.add.at(W, (v, part[u]), ew)
    return W


def lmax(w):
    """L_max = floor((1 + eps) * ceil(c(V) / k)) (Sec. 2), eps taken as an exact decimal."""
    tot = int(node_w(w).sum())
    eps = Fraction(round(w.eps * 1e6), 10**6)
    avg = -(-tot // w.k)
    return int((1 + eps) * avg)


def slot(omega: int, c: int, lo: int = -32, hi: int = 40) -> int:
    """ceil(log_{3/2}(omega / c)) clamped to [lo, hi], found from the defining
    inequality (3/2)^(s-1) < omega/c <= (3/2)^s by a search over s in exact rationals."""
    if omega == 0:
        return lo
    r = Fraction(omega, c)
    s = 0
    while Fraction(3, 2) ** s < r:
        s += 1
    while Fraction(3, 2) ** (s - 1) >= r:
        s -= 1
    return max(lo, min(hi, s))


def tau(r: int, R: int, tau1=Fraction(1, 4)) -> Fraction:
    """Linear interpolation from tau_1 (round 1) to 1 (round R) (Sec. 4.4)."""
    if R <= 1:
        return Fraction(tau1)
    return Fraction(tau1) + (1 - Fraction(tau1)) * Fraction(r - 1, R - 1)


def factor(l: int, t: Fraction, q: int = 20) -> int:
    """floor(tau * (3/2)^l * 2^q)."""
    v = t * Fraction(3, 2) ** l * 2**q
    return v.numerator // v.denominator


def apply(part, nodes, to):
    p = np.array(part, copy=True)
    p[np.asarray(nodes, dtype=np.int64)] = np.asarray(to)
    return p
