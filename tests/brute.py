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


def rebalance_subrounds(w, part, L: int, max_subrounds: int = 64, gain_only: bool = False):
    """The rebalancing sub-rounds of Sec. 6.1 in the synchronous reading,
    evaluated from the definitions on a tiny graph.  Per sub-round: every node
    of an overloaded block proposes a move into an allowed block (not
    overloaded when rebalancing started, never rejected a move, room for the
    node): the allowed block it is most connected to, ties to the smaller id,
    else the lightest allowed block, ties to the smaller id; the gain of a
    proposal is the cut difference of the move.  Proposals are ordered by
    priority (g * c for g >= 0 before g / c for g < 0, higher first, ties by
    node id; the gain alone when gain_only), compared in exact rationals.  A
    source selects the shortest prefix of its proposals whose weight covers
    its excess; a target admits the longest prefix of the selected proposals
    to it that keeps it within L and is never a target again if that prefix
    is not all of them.  The loop ends when no block is overloaded, when a
    sub-round admits nothing and rejects nowhere new, or after max_subrounds.
    Returns the admitted moves (node, from, to, sub-round) in sub-round order,
    priority order within a sub-round."""
    part = np.array(part, copy=True)
    c = node_w(w)
    edges = coo(w)
    C = block_weights(w, part)
    first_over = set(np.nonzero(C > L)[0].tolist())
    rejected = set()
    out = []
    for h in range(1, max_subrounds + 1):
        over = [b for b in range(w.k) if C[b] > L]
        if not over:
            break
        base = cut(w, part, edges)
        props = []
        for u in range(w.n):
            a = int(part[u])
            if a not in over:
                continue
            allowed = [b for b in range(w.k)
                       if b != a and b not in first_over and b not in rejected and C[b] + c[u] <= L]
            if not allowed:
                continue
            nbr_blocks = set(part[w.adj[w.xadj[u]:w.xadj[u + 1]]].tolist())
            linked = [b for b in allowed if b in nbr_blocks]
            if linked:
                # most connected = largest cut decrease (the own block's share is fixed)
                gains = {}
                for b in linked:
                    q = part.copy()
                    q[u] = b
                    gains[b] = base - cut(w, q, edges)
                t = max(linked, key=lambda b: (gains[b], -b))
            else:
                t = min(allowed, key=lambda b: (C[b], b))
            q = part.copy()
            q[u] = t
            g = base - cut(w, q, edges)
            props.append((u, a, t, g, int(c[u])))

        def key(p):
            u, _, _, g, cu = p
            if gain_only:
                return (0, -Fraction(g), u)
            return (0, -Fraction(g * cu), u) if g >= 0 else (1, -Fraction(g, cu), u)

        props.sort(key=key)
        selected = []
        for a in over:
            mine = [p for p in props if p[1] == a]
            excess = int(C[a]) - L
            j = 0
            while j < len(mine) and sum(p[4] for p in mine[:j]) < excess:
                j += 1
            selected += mine[:j]
        selected.sort(key=key)
        admitted = []
        grew = False
        for t in sorted({p[2] for p in selected}):
            mine = [p for p in selected if p[2] == t]
            j = len(mine)
            while j > 0 and C[t] + sum(p[4] for p in mine[:j]) > L:
                j -= 1
            admitted += mine[:j]
            if j < len(mine) and t not in rejected:
                rejected.add(t)
                grew = True
        admitted.sort(key=key)
        for u, a, t, _, cu in admitted:
            part[u] = t
            C[a] -= cu
            C[t] += cu
            out.append((u, a, t, h))
        if not admitted and not grew:
            break
    return out
