/*
 * CPU oracle for one deterministic synchronous round of unconstrained FM
 * refinement (Maas, Gottesbueren, Seemaier, "Parallel Unconstrained Local
 * Search for Partitioning Irregular Graphs", arXiv 2308.15494).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA library: both are
 * written independently from the paper, and this file is the plain,
 * sequential, slow statement of what the CUDA path must reproduce bit for
 * bit.  Every quantity is an integer; 128-bit integers are used wherever a
 * product could exceed 64 bits.
 *
 * The round follows Algorithm 1 in the paper's order, in the synchronous
 * reading documented in the repository's design notes:
 *   0. block weights c(V_b) and cut (Sec. 2)
 *   1. gain table omega(v, V_b) and omega(I(v)) (Sec. 2, Sec. 6.1)
 *   2. rebalancing-availability, slots, bucket weights, penalty factors
 *      (Alg. 1, Sec. 4.3, Sec. 4.4 for the tau schedule)
 *   3. per boundary node, the best target by gain minus penalty (Alg. 1,
 *      Sec. 4.3)
 *   4. penalties including the inflow of better-ranked candidates into the
 *      same block, keep gain - penalty > 0, global move order M (Alg. 1,
 *      Sec. 4.4 first paragraph, Lemma 1's sequence)
 *   5. apply M (Alg. 1)
 *   6. rebalancing into R_1..R_k (Alg. 1, Sec. 6)
 *   7. interleaving of M and R (Sec. 4.4)
 *   8. merging of a node's two moves into one (Sec. 4.4 footnote)
 *   9. exact gains of the interleaved sequence (Sec. 4.4; gains per Sec. 2)
 *  10. best balanced prefix and its application (Alg. 1, Sec. 4.1)
 * Parity status of each step is listed in the oracle's package docstring.
 */
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <vector>

typedef __int128 i128;
typedef unsigned __int128 u128;

extern "C" {

/* ---------------------------------------------------------------- ABI -- */
typedef struct {
    int64_t n;
    const int64_t *xadj;   /* [n+1] */
    const int32_t *adj;    /* [m]   */
    const int32_t *adjw;   /* [m] or NULL: unit edge weights */
    const int32_t *vwgt;   /* [n] or NULL: unit node weights */
} upro_graph;

typedef struct {
    int32_t t_num, t_den;       /* availability threshold t (Sec. 4.3); 7/10 */
    int32_t tau1_num, tau1_den; /* tau_1 of the penalty schedule (Sec. 4.4); 1/4 */
    int32_t max_subrounds;      /* rebalancing sub-round limit; 64 */
    int32_t gain_priority;      /* 1: rebalancing priority = gain alone (the variant of Sec. 7.2); 0 */
    int32_t append;             /* 1: the rebalancing moves appended after M instead of
                                   interleaved (the variant of Sec. 7.2); 0 */
    int32_t lp_rounds;          /* rounds of unconstrained label propagation before the
                                   FM rounds (Sec. 5; the paper uses 5); 0 */
    int32_t lock_rebalanced;    /* 1: the oscillation guard of Sec. 2: a node whose applied
                                   move in a round came from rebalancing alone is not a
                                   candidate in the next round; 0 */
} upro_params;

/* Optional per-round trace; every pointer may be NULL.  Node-sized arrays
 * hold n entries, the pre-merge sequence 2n. */
typedef struct {
    /* step 2 */
    int8_t  *avail;       /* [n] 1 if available for rebalancing          */
    int32_t *slot;        /* [n] bucket slot                              */
    int64_t *bucket;      /* [k*73] c(B_{slot,b}), row b, column slot+32  */
    int64_t *factor;      /* [73] F_r[l]                                  */
    /* step 3 (node-indexed) */
    int32_t *cand_target; /* [n] target of v, -1 if v is no candidate     */
    int64_t *cand_s0;     /* [n] gain - penalty at the round-start weight */
    int64_t *cand_gain;   /* [n] gain of that move                        */
    int64_t  n_cand;
    /* step 4 */
    int64_t  n_moves;
    int32_t *M_node, *M_to;
    int64_t *M_score;     /* gain - penalty with inflow                   */
    /* step 6 */
    int64_t  n_rebal;
    int32_t  subrounds;
    int32_t *R_node, *R_from, *R_to, *R_subround;
    /* step 7 (before merging; capacity 2n) */
    int64_t  n_inter;
    int32_t *X_node, *X_from, *X_to;
    /* steps 8-9 */
    int64_t  n_seq;
    int32_t *I_node, *I_from, *I_to;
    int64_t *I_gain;
    int8_t  *I_eligible;  /* [n+1] eligible(j) for j = 0..|I|            */
    /* step 10 */
    int64_t  best_len, best_gain, cut_before, cut_after;
} upro_trace;

enum { UPRO_OK = 0, UPRO_ERR_INVALID = -1, UPRO_ERR_INFEASIBLE = -4 };

} /* extern "C" */

namespace {

const int SLOT_LO = -32;                 /* slots are clamped to [-32, 40] */
const int SLOT_HI = 40;
const int NSLOT = SLOT_HI - SLOT_LO + 1; /* 73 */
const int QBITS = 20;                    /* fixed-point scale of F_r */
const int64_t FORBID = -1;               /* "no such slot: forbid the move" */

struct Graph {
    int64_t n;
    const int64_t *xadj;
    const int32_t *adj;
    const int32_t *adjw;
    const int32_t *vwgt;
    int64_t c(int64_t v) const { return vwgt ? (int64_t)vwgt[v] : 1; }
    int64_t w(int64_t e) const { return adjw ? (int64_t)adjw[e] : 1; }
};

Graph wrap(const upro_graph *g) { return Graph{g->n, g->xadj, g->adj, g->adjw, g->vwgt}; }

u128 pow_u128(u128 b, int e) { u128 r = 1; while (e-- > 0) r *= b; return r; }

/* Sec. 2: L_max = (1 + eps) * ceil(c(V) / k), eps given in parts per million. */
int64_t lmax_of(int64_t total, int32_t k, int64_t eps_ppm) {
    int64_t avg = (total + k - 1) / k;
    return (int64_t)(((i128)avg * (1000000 + eps_ppm)) / 1000000);
}

/* Sec. 4.3: slot(v) = ceil(log_{3/2}(omega(v, Pi(v)) / c(v))), i.e. the smallest
 * integer s with (3/2)^s >= omega / c, clamped to [SLOT_LO, SLOT_HI].
 * (3/2)^s >= w / c  <=>  3^s c >= 2^s w   (s >= 0)
 *                   <=>  2^-s c >= 3^-s w (s < 0). */
int slot_of(int64_t omega, int64_t c) {
    for (int s = SLOT_LO; s <= SLOT_HI; s++) {
        bool ok;
        if (s >= 0) ok = pow_u128(3, s) * (u128)c >= pow_u128(2, s) * (u128)omega;
        else ok = pow_u128(2, -s) * (u128)c >= pow_u128(3, -s) * (u128)omega;
        if (ok) return s;
    }
    return SLOT_HI;
}

/* Sec. 4.4: tau_r interpolates linearly from tau_1 (round 1) to 1 (round R).
 * Returned as an exact fraction num/den. */
void tau_of(int32_t r, int32_t R, const upro_params &p, int64_t *num, int64_t *den) {
    int64_t a = p.tau1_num, b = p.tau1_den;
    int64_t D = R > 1 ? (int64_t)R - 1 : 1;
    *num = a * D + (b - a) * (int64_t)(r - 1);
    *den = b * D;
}

/* F_r[l] = floor(tau_r * (3/2)^l * 2^Q): the penalty factor of slot l
 * (Sec. 4.3 penalty (3/2)^l c(u), scaled by tau_r of Sec. 4.4). */
void factors_of(int64_t tnum, int64_t tden, int64_t *F) {
    for (int l = SLOT_LO; l <= SLOT_HI; l++) {
        u128 num, den;
        if (l >= 0) { num = (u128)tnum * pow_u128(3, l) << QBITS; den = (u128)tden * pow_u128(2, l); }
        else { num = (u128)tnum * pow_u128(2, -l) << QBITS; den = (u128)tden * pow_u128(3, -l); }
        F[l - SLOT_LO] = (int64_t)(num / den);
    }
}

/* Sec. 4.3: the penalty of moving a node of weight cu into block b when the
 * block would exceed L_max by x.  l is the minimal slot whose cumulative
 * bucket weight sum_{i <= l} c(B_{i,b}) covers x; none -> the move is
 * forbidden (footnote in Sec. 4.3).  penalty = floor(cu * F_r[l] / 2^Q). */
int64_t penalty(const std::vector<int64_t> &BW, int32_t b, int64_t x, int64_t cu,
                const int64_t *F, int *level) {
    *level = SLOT_LO - 1;
    if (x <= 0) return 0;
    int64_t acc = 0;
    for (int l = 0; l < NSLOT; l++) {
        acc += BW[(size_t)b * NSLOT + l];
        if (acc >= x) {
            *level = l + SLOT_LO;
            return (int64_t)(((u128)cu * (u128)F[l]) >> QBITS);
        }
    }
    return FORBID;
}

struct Move { int32_t v, from, to; int8_t rebal; };  /* rebal: produced by rebalancing */

struct Proposal { int32_t u, from, to; int64_t g, c; };

/* Sec. 6.1 priority: g / c(u) if g < 0, g * c(u) if g >= 0; higher first;
 * equal priorities by smaller node id.  Compared exactly by integer
 * cross-multiplication. */
bool higher_priority(const Proposal &a, const Proposal &b) {
    bool pa = a.g >= 0, pb = b.g >= 0;
    if (pa != pb) return pa;
    if (pa) {
        i128 x = (i128)a.g * a.c, y = (i128)b.g * b.c;
        if (x != y) return x > y;
    } else {
        i128 x = (i128)a.g * b.c, y = (i128)b.g * a.c;   /* a.g/a.c > b.g/b.c */
        if (x != y) return x > y;
    }
    return a.u < b.u;
}

struct Table {
    int64_t n; int32_t k;
    std::vector<int32_t> W;   /* W[v*k + b] = omega(v, V_b) */
    std::vector<int64_t> wI;  /* omega(I(v)) */
    int32_t &at(int64_t v, int32_t b) { return W[(size_t)v * k + b]; }
};

/* Sec. 2 / Sec. 6.1: the gain table, built by one pass over every adjacency list. */
void build_table(const Graph &g, int32_t k, const int32_t *part, Table &T) {
    T.n = g.n; T.k = k;
    T.W.assign((size_t)g.n * k, 0);
    T.wI.assign((size_t)g.n, 0);
    for (int64_t v = 0; v < g.n; v++)
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
            T.at(v, part[g.adj[e]]) += (int32_t)g.w(e);
            T.wI[v] += g.w(e);
        }
}

/* Moving v from a to b changes omega(x, V_a) and omega(x, V_b) of each neighbour x. */
void table_move(const Graph &g, Table &T, int32_t v, int32_t a, int32_t b) {
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
        T.at(g.adj[e], a) -= (int32_t)g.w(e);
        T.at(g.adj[e], b) += (int32_t)g.w(e);
    }
}

int64_t cut_of(const Graph &g, const int32_t *part) {
    int64_t twice = 0;
    for (int64_t v = 0; v < g.n; v++)
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++)
            if (part[v] != part[g.adj[e]]) twice += g.w(e);
    return twice / 2;
}

struct RoundOut {
    int64_t n_cand = 0, n_moves = 0, n_rebal = 0, n_seq = 0, best_len = 0, best_gain = 0;
    int32_t subrounds = 0;
    bool lp_kept = false;     /* label propagation: the round's result was kept */
};

/*
 * One round.  rebalance_only: the round-0 repair of an imbalanced input
 * (steps 2-5 skipped, M empty).  Returns UPRO_ERR_INFEASIBLE (part unchanged)
 * if no prefix of the sequence is balanced.
 */
/* The kind of a round in the round driver of Sec. 6.2 ("integration"):
 * an unconstrained round whose penalty factor is tau_r of the schedule
 * (tau_den == 0) or a given tau, or a constrained round, read as the same
 * round in which no move may leave its target above L_max (an infinite
 * penalty, so such a move is never a candidate and never kept in M). */
struct RoundKind {
    bool constrained = false;
    int64_t tau_num = 0, tau_den = 0;
    /* the variants of Sec. 7.2: limit > 0 replaces the penalty by a block
     * limit: a move that would leave its target above `limit` (with the
     * inflow of better-ranked candidates) is forbidden, every other move
     * pays nothing.  A constrained round is limit = L_max. */
    int64_t limit = 0;
    /* unconstrained label propagation (Sec. 5): active[v] != 0 marks V_a;
     * the round moves every active node to its best positive-gain block,
     * rebalances, and keeps the result only if it is balanced and cuts less */
    const int8_t *lp_active = nullptr;
    /* the oscillation guard (Sec. 2): locked[v] != 0 keeps v out of the
     * selection of this round (rebalancing may still move it); locked_out
     * receives the nodes whose applied move came from rebalancing alone */
    const int8_t *locked = nullptr;
    int8_t *locked_out = nullptr;
};

int round_impl(const Graph &g, int32_t k, int64_t Lmax, const upro_params &p, int32_t r,
               int32_t R, bool rebalance_only, int32_t *part, int64_t *cut, upro_trace *tr,
               RoundOut *out, const RoundKind &kind = RoundKind()) {
    const int64_t n = g.n;

    /* ---- step 0: block weights c(V_b) (Sec. 2) ---- */
    std::vector<int64_t> C(k, 0);
    for (int64_t v = 0; v < n; v++) C[part[v]] += g.c(v);
    const int64_t cut0 = *cut;

    /* ---- step 1: gain table ---- */
    Table T;
    build_table(g, k, part, T);

    std::vector<Move> M;
    std::vector<int32_t> Pp(part, part + n);  /* P' = P o M */
    std::vector<int64_t> Cp(C);

    if (kind.lp_active) {
        /* ---- label propagation (Sec. 5): every active node to the
         * neighbouring block of the highest positive gain (ties to the smaller
         * block), all against the round-start partition, balance ignored ---- */
        for (int64_t v = 0; v < n; v++) {
            if (!kind.lp_active[v]) continue;
            const int64_t own = T.at(v, part[v]);
            int64_t best = 0; int32_t bt = -1;
            for (int32_t b = 0; b < k; b++) {
                if (b == part[v] || T.at(v, b) <= 0) continue;
                const int64_t gv = (int64_t)T.at(v, b) - own;
                if (gv > best) { best = gv; bt = b; }
            }
            if (bt >= 0) {
                M.push_back(Move{(int32_t)v, part[v], bt, 0});
                if (tr && tr->M_node) { tr->M_node[M.size() - 1] = (int32_t)v; tr->M_to[M.size() - 1] = bt; tr->M_score[M.size() - 1] = best; }
            }
        }
        out->n_moves = (int64_t)M.size();
        for (const Move &mv : M) {
            Pp[mv.v] = mv.to;
            Cp[mv.from] -= g.c(mv.v);
            Cp[mv.to] += g.c(mv.v);
            table_move(g, T, mv.v, mv.from, mv.to);
        }
    } else if (!rebalance_only) {
        /* ---- step 2: V_r, slots, buckets B_{i,j} (Alg. 1, Sec. 4.3) ---- */
        std::vector<int64_t> BW((size_t)k * NSLOT, 0);
        for (int64_t v = 0; v < n; v++) {
            int64_t own = T.at(v, part[v]);
            bool avail = (int64_t)p.t_den * own >= (int64_t)p.t_num * T.wI[v];
            int s = slot_of(own, g.c(v));
            if (avail) BW[(size_t)part[v] * NSLOT + (s - SLOT_LO)] += g.c(v);
            if (tr && tr->avail) tr->avail[v] = avail ? 1 : 0;
            if (tr && tr->slot) tr->slot[v] = s;
        }
        int64_t tnum, tden, F[NSLOT];
        if (kind.tau_den > 0) { tnum = kind.tau_num; tden = kind.tau_den; }
        else tau_of(r, R, p, &tnum, &tden);
        factors_of(tnum, tden, F);
        /* the penalty of a move that leaves b exceeding L_max by x */
        auto pen_of = [&](int32_t b, int64_t x, int64_t cu) -> int64_t {
            int lvl;
            if (kind.constrained) return x > 0 ? FORBID : 0;
            if (kind.limit > 0) return x + Lmax > kind.limit ? FORBID : 0;   /* x + L_max: the new weight */
            return penalty(BW, b, x, cu, F, &lvl);
        };
        if (tr && tr->bucket) memcpy(tr->bucket, BW.data(), sizeof(int64_t) * BW.size());
        if (tr && tr->factor) memcpy(tr->factor, F, sizeof(F));

        /* ---- step 3: best target of every boundary node (Alg. 1, Sec. 4.3) ---- */
        std::vector<int32_t> tgt(n, -1);
        std::vector<int64_t> s0(n, 0), gain(n, 0);
        for (int64_t v = 0; v < n; v++) {
            int64_t own = T.at(v, part[v]);
            if (own >= T.wI[v]) continue;              /* not a boundary node (Sec. 2) */
            if (kind.locked && kind.locked[v]) continue; /* locked by the oscillation guard */
            bool have = false;
            int64_t best = 0, bestg = 0; int32_t bt = -1;
            for (int32_t b = 0; b < k; b++) {
                if (b == part[v] || T.at(v, b) <= 0) continue;
                int64_t gv = (int64_t)T.at(v, b) - own;
                int64_t pen = pen_of(b, C[b] + g.c(v) - Lmax, g.c(v));
                if (pen == FORBID) continue;
                int64_t sc = gv - pen;
                if (!have || sc > best) { have = true; best = sc; bt = b; bestg = gv; }
            }
            if (have && best > 0) { tgt[v] = bt; s0[v] = best; gain[v] = bestg; out->n_cand++; }
        }
        if (tr && tr->cand_target) memcpy(tr->cand_target, tgt.data(), sizeof(int32_t) * n);
        if (tr && tr->cand_s0) memcpy(tr->cand_s0, s0.data(), sizeof(int64_t) * n);
        if (tr && tr->cand_gain) memcpy(tr->cand_gain, gain.data(), sizeof(int64_t) * n);

        /* ---- step 4: penalties with inflow, keep gain - penalty > 0 ---- */
        std::vector<std::vector<int32_t>> into(k);
        for (int64_t v = 0; v < n; v++) if (tgt[v] >= 0) into[tgt[v]].push_back((int32_t)v);
        struct Kept { int32_t v, to; int64_t s; };
        std::vector<Kept> kept;
        for (int32_t t = 0; t < k; t++) {
            std::vector<int32_t> &L = into[t];
            std::sort(L.begin(), L.end(), [&](int32_t a, int32_t b) {
                if (s0[a] != s0[b]) return s0[a] > s0[b];
                return a < b;
            });
            int64_t inflow = 0;                          /* c(U^{i-1}) of Lemma 1 */
            for (int32_t v : L) {
                int64_t pen = pen_of(t, C[t] + inflow + g.c(v) - Lmax, g.c(v));
                inflow += g.c(v);
                if (pen == FORBID) continue;
                int64_t sc = gain[v] - pen;
                if (sc > 0) kept.push_back(Kept{v, t, sc});
            }
        }
        std::sort(kept.begin(), kept.end(), [](const Kept &a, const Kept &b) {
            if (a.s != b.s) return a.s > b.s;
            return a.v < b.v;
        });
        for (size_t i = 0; i < kept.size(); i++) {
            M.push_back(Move{kept[i].v, part[kept[i].v], kept[i].to, 0});
            if (tr && tr->M_node) { tr->M_node[i] = kept[i].v; tr->M_to[i] = kept[i].to; tr->M_score[i] = kept[i].s; }
        }
        out->n_moves = (int64_t)M.size();

        /* ---- step 5: apply M (P' = P o M, Alg. 1) ---- */
        for (const Move &mv : M) {
            Pp[mv.v] = mv.to;
            Cp[mv.from] -= g.c(mv.v);
            Cp[mv.to] += g.c(mv.v);
            table_move(g, T, mv.v, mv.from, mv.to);
        }
    }

    /* ---- step 6: rebalancing (Alg. 1, Sec. 6) ---- */
    std::vector<Move> Rseq;
    std::vector<int32_t> Rsub;
    std::vector<char> over1(k, 0), forb(k, 0);
    for (int32_t b = 0; b < k; b++) over1[b] = Cp[b] > Lmax;
    for (int32_t h = 1; h <= p.max_subrounds; h++) {
        std::vector<char> over(k, 0);
        bool any = false;
        for (int32_t b = 0; b < k; b++) { over[b] = Cp[b] > Lmax; any = any || over[b]; }
        if (!any) break;
        out->subrounds = h;
        /* insertion: every node of an overloaded block proposes its move (Sec. 6.1) */
        std::vector<Proposal> props;
        for (int64_t u = 0; u < n; u++) {
            int32_t a = Pp[u];
            if (!over[a]) continue;
            int64_t own = T.at(u, a), cu = g.c(u);
            bool have = false; int32_t bt = -1; int64_t bg = 0;
            for (int32_t b = 0; b < k; b++) {          /* best-gain balanced target */
                if (b == a || over1[b] || forb[b] || Cp[b] + cu > Lmax) continue;
                if (T.at(u, b) <= 0) continue;
                int64_t gv = (int64_t)T.at(u, b) - own;
                if (!have || gv > bg) { have = true; bt = b; bg = gv; }
            }
            if (!have) {                                /* not connected: lightest block */
                for (int32_t b = 0; b < k; b++) {
                    if (b == a || over1[b] || forb[b] || Cp[b] + cu > Lmax) continue;
                    if (!have || Cp[b] < Cp[bt]) { have = true; bt = b; }
                }
                bg = -own;
            }
            if (have) props.push_back(Proposal{(int32_t)u, a, bt, bg, cu});
        }
        if (p.gain_priority)      /* Sec. 7.2 variant: the gain alone, higher first, then smaller id */
            std::sort(props.begin(), props.end(), [](const Proposal &a, const Proposal &b) {
                return a.g != b.g ? a.g > b.g : a.u < b.u;
            });
        else
            std::sort(props.begin(), props.end(), higher_priority);
        /* per source: the minimal prefix that removes the excess */
        std::vector<int64_t> taken(k, 0);
        std::vector<Proposal> sel;
        for (const Proposal &q : props) {
            if (taken[q.from] < Cp[q.from] - Lmax) { sel.push_back(q); taken[q.from] += q.c; }
        }
        /* per target: the longest prefix that keeps it within L_max */
        std::vector<int64_t> inflow(k, 0);
        std::vector<char> stopped(k, 0);
        std::vector<Proposal> adm;
        bool grew = false;
        for (const Proposal &q : sel) {
            if (!stopped[q.to] && Cp[q.to] + inflow[q.to] + q.c <= Lmax) {
                inflow[q.to] += q.c;
                adm.push_back(q);
            } else {
                stopped[q.to] = 1;
                if (!forb[q.to]) { forb[q.to] = 1; grew = true; }
            }
        }
        for (const Proposal &q : adm) {
            Pp[q.u] = q.to;
            Cp[q.from] -= q.c;
            Cp[q.to] += q.c;
            table_move(g, T, q.u, q.from, q.to);
            Rseq.push_back(Move{q.u, q.from, q.to, 1});
            Rsub.push_back(h);
        }
        if (adm.empty() && !grew) break;
    }
    out->n_rebal = (int64_t)Rseq.size();
    if (tr && tr->R_node)
        for (size_t i = 0; i < Rseq.size(); i++) {
            tr->R_node[i] = Rseq[i].v; tr->R_from[i] = Rseq[i].from;
            tr->R_to[i] = Rseq[i].to; tr->R_subround[i] = Rsub[i];
        }
    if (kind.lp_active) {
        /* label propagation: keep the moved and rebalanced partition only if
         * it is balanced and cuts strictly less (Sec. 5: the net improvement
         * check, else the rollback) */
        bool bal = true;
        for (int32_t b = 0; b < k; b++) bal = bal && Cp[b] <= Lmax;
        const int64_t cut1 = cut_of(g, Pp.data());
        out->lp_kept = bal && cut1 < cut0;
        if (tr) {
            tr->n_cand = out->n_moves; tr->n_moves = out->n_moves; tr->n_rebal = out->n_rebal;
            tr->subrounds = out->subrounds; tr->cut_before = cut0;
        }
        if (out->lp_kept) {
            memcpy(part, Pp.data(), sizeof(int32_t) * n);
            *cut = cut1;
        }
        if (tr) tr->cut_after = *cut;
        return UPRO_OK;
    }

    /* ---- step 7: interleaved sequence I (Sec. 4.4) ---- */
    std::vector<std::vector<Move>> Rb(k);
    for (const Move &mv : Rseq) Rb[mv.from].push_back(mv);
    std::vector<Move> X;
    if (p.append) {             /* Sec. 7.2 variant: M, then the rebalancing moves in their order */
        X = M;
        X.insert(X.end(), Rseq.begin(), Rseq.end());
    } else {
        std::vector<int64_t> Xw(C);
        std::vector<size_t> q(k, 0);
        for (const Move &mv : M) {
            X.push_back(mv);
            Xw[mv.from] -= g.c(mv.v);
            Xw[mv.to] += g.c(mv.v);
            int32_t b = mv.to;
            while (Xw[b] > Lmax && q[b] < Rb[b].size()) {
                const Move &rm = Rb[b][q[b]++];
                X.push_back(rm);
                Xw[rm.from] -= g.c(rm.v);
                Xw[rm.to] += g.c(rm.v);
            }
        }
        for (int32_t b = 0; b < k; b++)
            while (q[b] < Rb[b].size()) X.push_back(Rb[b][q[b]++]);
    }
    if (tr && tr->X_node)
        for (size_t i = 0; i < X.size(); i++) { tr->X_node[i] = X[i].v; tr->X_from[i] = X[i].from; tr->X_to[i] = X[i].to; }

    /* ---- step 8: a node moved twice becomes one move (Sec. 4.4 footnote) ----
     * A node has at most one move from M and one from R.  The merged move goes
     * from its round-start block to its block after R, at the position of its
     * M move; it is dropped when both blocks are equal. */
    std::vector<Move> I;
    {
        std::vector<int64_t> mpos(n, -1), rpos(n, -1);
        std::vector<int32_t> rto(n, -1);
        for (size_t i = 0; i < X.size(); i++) {
            if (X[i].rebal) { rpos[X[i].v] = (int64_t)i; rto[X[i].v] = X[i].to; }
            else mpos[X[i].v] = (int64_t)i;
        }
        for (size_t i = 0; i < X.size(); i++) {
            int32_t v = X[i].v;
            if (X[i].rebal && mpos[v] >= 0) continue;        /* folded into v's M move */
            int32_t to = (!X[i].rebal && rpos[v] >= 0) ? rto[v] : X[i].to;
            if (part[v] != to) I.push_back(Move{v, part[v], to, X[i].rebal});
        }
    }

    /* ---- step 9: exact gains of I (Sec. 4.4; gain per Sec. 2) ---- */
    std::vector<int64_t> pos(n, INT64_MAX);
    std::vector<int32_t> dest(n, -1);
    for (size_t i = 0; i < I.size(); i++) { pos[I[i].v] = (int64_t)i; dest[I[i].v] = I[i].to; }
    std::vector<int64_t> gI(I.size(), 0);
    for (size_t i = 0; i < I.size(); i++) {
        int32_t v = I[i].v, a = I[i].from, b = I[i].to;
        int64_t gsum = 0;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
            int32_t u = g.adj[e];
            int32_t bu = pos[u] < (int64_t)i ? dest[u] : part[u];
            if (bu == b) gsum += g.w(e);
            if (bu == a) gsum -= g.w(e);
        }
        gI[i] = gsum;
    }

    /* ---- step 10: best balanced prefix (Alg. 1, Sec. 4.1) ---- */
    std::vector<int64_t> Xw(C);
    int64_t overloaded = 0;
    for (int32_t b = 0; b < k; b++) overloaded += Xw[b] > Lmax;
    bool have_best = overloaded == 0;
    int64_t best_len = 0, best_gain = 0, G = 0;
    if (tr && tr->I_eligible) tr->I_eligible[0] = overloaded == 0;
    for (size_t j = 1; j <= I.size(); j++) {
        const Move &mv = I[j - 1];
        overloaded -= Xw[mv.from] > Lmax;
        Xw[mv.from] -= g.c(mv.v);
        overloaded += Xw[mv.from] > Lmax;
        overloaded -= Xw[mv.to] > Lmax;
        Xw[mv.to] += g.c(mv.v);
        overloaded += Xw[mv.to] > Lmax;
        G += gI[j - 1];
        bool elig = overloaded == 0;
        if (tr && tr->I_eligible) tr->I_eligible[j] = elig;
        if (elig && (!have_best || G > best_gain)) { have_best = true; best_gain = G; best_len = (int64_t)j; }
    }
    if (tr) {
        tr->n_cand = out->n_cand; tr->n_moves = out->n_moves; tr->n_rebal = out->n_rebal;
        tr->subrounds = out->subrounds; tr->n_inter = (int64_t)X.size(); tr->n_seq = (int64_t)I.size();
        if (tr->I_node)
            for (size_t i = 0; i < I.size(); i++) {
                tr->I_node[i] = I[i].v; tr->I_from[i] = I[i].from; tr->I_to[i] = I[i].to; tr->I_gain[i] = gI[i];
            }
        tr->cut_before = cut0;
    }
    out->n_seq = (int64_t)I.size();
    if (!have_best) return UPRO_ERR_INFEASIBLE;
    for (int64_t j = 0; j < best_len; j++) part[I[j].v] = I[j].to;
    if (kind.locked_out) {
        memset(kind.locked_out, 0, (size_t)n);
        for (int64_t j = 0; j < best_len; j++)
            if (I[j].rebal) kind.locked_out[I[j].v] = 1;
    }
    *cut = cut0 - best_gain;
    out->best_len = best_len; out->best_gain = best_gain;
    if (tr) { tr->best_len = best_len; tr->best_gain = best_gain; tr->cut_after = *cut; }
    return UPRO_OK;
}

/* V_a after a kept label-propagation round (Sec. 5): the neighbours of the
 * nodes whose block changed that did not change block themselves. */
void lp_next_active(const Graph &g, const int32_t *before, const int32_t *after, std::vector<int8_t> &active) {
    std::fill(active.begin(), active.end(), 0);
    for (int64_t v = 0; v < g.n; v++) {
        if (before[v] == after[v]) continue;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
            const int32_t u = g.adj[e];
            if (before[u] == after[u]) active[u] = 1;
        }
    }
}

/* Unconstrained label propagation before the FM rounds (Sec. 5): V_a starts
 * as the boundary nodes; a round that is not kept ends it, as do
 * max_rounds rounds, an empty V_a, or a kept round whose improvement is below
 * 0.001 of the cut before it.  Returns the rounds kept. */
int32_t label_propagation(const Graph &g, int32_t k, int64_t Lmax, const upro_params &p, int32_t max_rounds,
                          int32_t *P, int64_t *cut) {
    std::vector<int8_t> active(g.n, 0);
    {
        Table T;
        build_table(g, k, P, T);
        for (int64_t v = 0; v < g.n; v++) active[v] = T.at(v, P[v]) < T.wI[v];   /* boundary nodes */
    }
    int32_t kept = 0;
    for (int32_t r = 1; r <= max_rounds; r++) {
        bool any = false;
        for (int8_t a : active) any = any || a;
        if (!any) break;
        std::vector<int32_t> before(P, P + g.n);
        const int64_t cut_before = *cut;
        RoundKind kind;
        kind.lp_active = active.data();
        RoundOut o;
        round_impl(g, k, Lmax, p, 1, 1, false, P, cut, nullptr, &o, kind);
        if (!o.lp_kept) break;
        kept++;
        if (1000 * (cut_before - *cut) < cut_before) break;
        lp_next_active(g, before.data(), P, active);
    }
    return kept;
}

bool params_ok(const upro_params &p) {
    return p.t_den > 0 && p.t_num >= 0 && p.t_num <= p.t_den && p.tau1_den > 0 && p.tau1_num >= 0 &&
           p.tau1_num <= p.tau1_den && p.tau1_den <= 65536 && p.max_subrounds >= 1 &&
           (p.gain_priority == 0 || p.gain_priority == 1) && (p.append == 0 || p.append == 1) &&
           p.lp_rounds >= 0 && p.lp_rounds <= 64 && (p.lock_rebalanced == 0 || p.lock_rebalanced == 1);
}

upro_params defaults() { return upro_params{7, 10, 1, 4, 64, 0, 0, 0, 0}; }

} /* namespace */

extern "C" {

void upro_params_default(upro_params *p) { *p = defaults(); }

int64_t upro_lmax(int64_t total_weight, int32_t k, int64_t eps_ppm) { return lmax_of(total_weight, k, eps_ppm); }

int32_t upro_slot(int64_t omega, int64_t c) { return slot_of(omega, c); }

/* F_r[l] for l = -32..40 into F[0..72]. */
int upro_factors(int32_t r, int32_t R, const upro_params *pp, int64_t *F) {
    upro_params p = pp ? *pp : defaults();
    if (!params_ok(p) || R < 1 || R > 65536 || r < 1 || r > R) return UPRO_ERR_INVALID;
    int64_t tn, td;
    tau_of(r, R, p, &tn, &td);
    factors_of(tn, td, F);
    return UPRO_OK;
}

/* Block weights and cut of a partition (Sec. 2). */
int upro_cut(const upro_graph *gg, int32_t k, const int32_t *part, int64_t *cut, int64_t *block_weights) {
    Graph g = wrap(gg);
    if (block_weights) {
        for (int32_t b = 0; b < k; b++) block_weights[b] = 0;
        for (int64_t v = 0; v < g.n; v++) block_weights[part[v]] += g.c(v);
    }
    if (cut) *cut = cut_of(g, part);
    return UPRO_OK;
}

/* Dense gain table W[v*k + b] = omega(v, V_b) and omega(I(v)). */
int upro_gain_table(const upro_graph *gg, int32_t k, const int32_t *part, int32_t *W, int64_t *wI) {
    Graph g = wrap(gg);
    Table T;
    build_table(g, k, part, T);
    if (W) memcpy(W, T.W.data(), sizeof(int32_t) * T.W.size());
    if (wI) memcpy(wI, T.wI.data(), sizeof(int64_t) * T.wI.size());
    return UPRO_OK;
}

/* Penalties pen(u_i, V_b u U^{i-1}) of a sequence of nodes all moved into
 * block b, in the given order (the scenario of Lemma 1), at round r of R. */
int upro_penalty_sequence(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp,
                          int32_t r, int32_t R, const int32_t *part, int32_t b, int64_t count,
                          const int32_t *nodes, int64_t *pen, int32_t *level) {
    upro_params p = pp ? *pp : defaults();
    Graph g = wrap(gg);
    Table T;
    build_table(g, k, part, T);
    std::vector<int64_t> C(k, 0);
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) { C[part[v]] += g.c(v); tot += g.c(v); }
    int64_t Lmax = lmax_of(tot, k, eps_ppm);
    std::vector<int64_t> BW((size_t)k * NSLOT, 0);
    for (int64_t v = 0; v < g.n; v++) {
        int64_t own = T.at(v, part[v]);
        if ((int64_t)p.t_den * own >= (int64_t)p.t_num * T.wI[v])
            BW[(size_t)part[v] * NSLOT + (slot_of(own, g.c(v)) - SLOT_LO)] += g.c(v);
    }
    int64_t tn, td, F[NSLOT];
    tau_of(r, R, p, &tn, &td);
    factors_of(tn, td, F);
    int64_t inflow = 0;
    for (int64_t i = 0; i < count; i++) {
        int lvl;
        pen[i] = penalty(BW, b, C[b] + inflow + g.c(nodes[i]) - Lmax, g.c(nodes[i]), F, &lvl);
        level[i] = lvl;
        inflow += g.c(nodes[i]);
    }
    return UPRO_OK;
}

/* One round r of R on part (in/out).  cut is in/out: the caller passes the
 * cut of part.  rebalance_only selects the round-0 repair. */
int upro_round(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, int32_t r,
               int32_t R, int32_t rebalance_only, int32_t *part, int64_t *cut, upro_trace *tr) {
    upro_params p = pp ? *pp : defaults();
    if (!params_ok(p) || k < 2 || R < 1 || R > 65536 || (!rebalance_only && (r < 1 || r > R)))
        return UPRO_ERR_INVALID;
    Graph g = wrap(gg);
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    RoundOut o;
    std::vector<int32_t> backup(part, part + g.n);
    int rc = round_impl(g, k, lmax_of(tot, k, eps_ppm), p, r, R, rebalance_only != 0, part, cut, tr, &o);
    if (rc != UPRO_OK) memcpy(part, backup.data(), sizeof(int32_t) * g.n);
    return rc;
}

/* One round of unconstrained label propagation (Sec. 5) over the active
 * nodes (active[v] != 0); *kept = 1 when its result was kept (part and cut
 * updated), 0 when it was rolled back.  The trace's M holds the label
 * propagation moves (M_score = their gain), R the rebalancing. */
int upro_lp_round(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, const int8_t *active,
                  int32_t *part, int64_t *cut, int32_t *kept, upro_trace *tr) {
    upro_params p = pp ? *pp : defaults();
    if (!params_ok(p) || k < 2 || !active) return UPRO_ERR_INVALID;
    Graph g = wrap(gg);
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    RoundOut o;
    RoundKind kind;
    kind.lp_active = active;
    int rc = round_impl(g, k, lmax_of(tot, k, eps_ppm), p, 1, 1, false, part, cut, tr, &o, kind);
    if (kept) *kept = o.lp_kept ? 1 : 0;
    return rc;
}

/* Unconstrained label propagation alone (Sec. 5) on a balanced partition:
 * returns the number of rounds kept, or an error. */
int upro_label_propagation(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, int32_t *part,
                           int32_t max_rounds, int64_t *cut_out) {
    upro_params p = pp ? *pp : defaults();
    if (!params_ok(p) || k < 2 || max_rounds < 0) return UPRO_ERR_INVALID;
    Graph g = wrap(gg);
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    int64_t cut = cut_of(g, part);
    const int32_t kept = label_propagation(g, k, lmax_of(tot, k, eps_ppm), p, max_rounds, part, &cut);
    if (cut_out) *cut_out = cut;
    return kept;
}

/* One round r of R (as upro_round) under the oscillation guard of Sec. 2:
 * nodes with locked[v] != 0 are not candidates; locked_out[v] = 1 for the
 * nodes whose applied move came from rebalancing alone (the next round's
 * locks).  limit > 0: the fully unconstrained / limited variant instead of
 * the penalty (as in upro_round_kind). */
int upro_round_guard(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, int32_t r, int32_t R,
                     int64_t limit, const int8_t *locked, int8_t *locked_out, int32_t *part, int64_t *cut,
                     upro_trace *tr) {
    upro_params p = pp ? *pp : defaults();
    if (!params_ok(p) || k < 2 || R < 1 || R > 65536 || r < 1 || r > R || limit < 0) return UPRO_ERR_INVALID;
    Graph g = wrap(gg);
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    RoundOut o;
    RoundKind kind;
    kind.limit = limit;
    kind.locked = locked;
    kind.locked_out = locked_out;
    std::vector<int32_t> backup(part, part + g.n);
    int rc = round_impl(g, k, lmax_of(tot, k, eps_ppm), p, r, R, false, part, cut, tr, &o, kind);
    if (rc != UPRO_OK) memcpy(part, backup.data(), sizeof(int32_t) * g.n);
    return rc;
}

/* One round of a given kind (Sec. 6.2): constrained != 0, or unconstrained
 * with tau = tau_num / tau_den.  Otherwise as upro_round with r = R = 1. */
int upro_round_kind(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, int32_t constrained,
                    int64_t tau_num, int64_t tau_den, int64_t limit, int32_t *part, int64_t *cut, upro_trace *tr) {
    upro_params p = pp ? *pp : defaults();
    if (!params_ok(p) || k < 2 || limit < 0 ||
        (!constrained && limit == 0 && (tau_den <= 0 || tau_num < 0 || tau_num > tau_den || tau_den > 65536)))
        return UPRO_ERR_INVALID;
    Graph g = wrap(gg);
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    RoundOut o;
    RoundKind kind;
    kind.constrained = constrained != 0;
    kind.tau_num = constrained ? 0 : tau_num;
    kind.tau_den = constrained ? 0 : tau_den;
    kind.limit = constrained ? 0 : limit;
    std::vector<int32_t> backup(part, part + g.n);
    int rc = round_impl(g, k, lmax_of(tot, k, eps_ppm), p, 1, 1, false, part, cut, tr, &o, kind);
    if (rc != UPRO_OK) memcpy(part, backup.data(), sizeof(int32_t) * g.n);
    return rc;
}

/* Rounds round_offset+1 .. round_offset+rounds of a total_rounds schedule,
 * preceded by the round-0 repair if part is imbalanced.  part is changed
 * only on success.  cut_out and per-round stats are optional. */
int upro_refine(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, int32_t *part,
                int32_t rounds, int32_t round_offset, int32_t total_rounds, int64_t *cut_out,
                int64_t *round_cuts /* [rounds+1] or NULL */) {
    upro_params p = pp ? *pp : defaults();
    Graph g = wrap(gg);
    if (!params_ok(p) || k < 2 || rounds < 0 || round_offset < 0 || total_rounds < 1 ||
        round_offset + rounds > total_rounds || total_rounds > 65536)
        return UPRO_ERR_INVALID;
    for (int64_t v = 0; v < g.n; v++) if (part[v] < 0 || part[v] >= k) return UPRO_ERR_INVALID;
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    int64_t Lmax = lmax_of(tot, k, eps_ppm);
    std::vector<int32_t> P(part, part + g.n);
    int64_t cut = cut_of(g, P.data());
    std::vector<int64_t> C(k, 0);
    for (int64_t v = 0; v < g.n; v++) C[P[v]] += g.c(v);
    bool bal = true;
    for (int32_t b = 0; b < k; b++) bal = bal && C[b] <= Lmax;
    RoundOut o;
    if (!bal) {
        int rc = round_impl(g, k, Lmax, p, 0, total_rounds, true, P.data(), &cut, nullptr, &o);
        if (rc != UPRO_OK) return rc;
    }
    if (p.lp_rounds > 0) label_propagation(g, k, Lmax, p, p.lp_rounds, P.data(), &cut);
    if (round_cuts) round_cuts[0] = cut;
    std::vector<int8_t> locked(p.lock_rebalanced ? g.n : 0, 0), locked_next(locked);
    for (int32_t i = 1; i <= rounds; i++) {
        RoundKind kind;
        if (p.lock_rebalanced) { kind.locked = locked.data(); kind.locked_out = locked_next.data(); }
        int rc = round_impl(g, k, Lmax, p, round_offset + i, total_rounds, false, P.data(), &cut, nullptr, &o, kind);
        if (rc != UPRO_OK) return rc;
        if (round_cuts) round_cuts[i] = cut;
        locked.swap(locked_next);
    }
    memcpy(part, P.data(), sizeof(int32_t) * g.n);
    if (cut_out) *cut_out = cut;
    return UPRO_OK;
}

/* The round driver of Sec. 4.4 / Sec. 6.2 over R = `rounds` rounds.
 *
 * The frame of the paper's final configuration (Sec. 4.4, "Integration into
 * the Overall Algorithm", with the parameters of Sec. 7.2): the first U
 * rounds are unconstrained, the others constrained, where U = R - 2 for
 * R >= 3 (ten rounds: eight unconstrained and two constrained, the split
 * Sec. 7.2 compares the switch against), U = 1 for R = 2 and U = 0 for
 * R = 1, so at least one constrained round follows the unconstrained ones;
 * once an unconstrained round improves the cut by less than 0.002 of the
 * cut before it, every later round is constrained.
 *
 * schedule 0: every round unconstrained with tau_r of the rounds' schedule
 *   (as upro_refine; no switch, no constrained round).
 * schedule 6: the paper's final configuration: the frame above with tau_i
 *   of a schedule over the U unconstrained rounds (tau_1 in round 1, 1 in
 *   round U).
 * schedules 3-5, the variants of Sec. 7.2 in the same frame (every variant
 *   there starts unconstrained and switches at 0.002): 3 constant penalty,
 *   tau = tau_1 in every unconstrained round; 4 fully unconstrained, no
 *   penalty and nothing forbidden; 5 limited imbalance, no penalty but no
 *   block above alpha_i * L_max, alpha going linearly from 2 (round 1) to
 *   1.1 (round U), the limit rounded down.
 * schedule 1: dynamic activation (Sec. 4.4, last paragraph), which Sec. 7.2
 *   tested and left out of the final configuration: round 1 constrained,
 *   round 2 unconstrained with tau = 1/2; if round 2 improved the cut by
 *   more than round 1, rounds 3..R-1 are unconstrained with tau_i of a
 *   schedule over those R-3 rounds (i = 1, 2, ...) until one of them
 *   improves the cut by less than 0.002 of the cut before it, the remaining
 *   ones constrained; otherwise rounds 3..R-1 are constrained; round R
 *   (R >= 3) is constrained.
 * schedule 2: every round constrained.
 * kinds[i-1] (may be NULL) receives round i's kind: 0 unconstrained (tau of
 * the schedule), 1 constrained, 2 unconstrained with tau = 1/2, 3 constant
 * tau, 4 no penalty, 5 limited imbalance. */
static int32_t unconstrained_rounds(int32_t R) { return R >= 3 ? R - 2 : R == 2 ? 1 : 0; }

int upro_refine_schedule(const upro_graph *gg, int32_t k, int64_t eps_ppm, const upro_params *pp, int32_t *part,
                         int32_t rounds, int32_t schedule, int64_t *cut_out, int64_t *round_cuts, int8_t *kinds) {
    upro_params p = pp ? *pp : defaults();
    Graph g = wrap(gg);
    if (!params_ok(p) || k < 2 || rounds < 0 || rounds > 65536 || schedule < 0 || schedule > 6)
        return UPRO_ERR_INVALID;
    for (int64_t v = 0; v < g.n; v++) if (part[v] < 0 || part[v] >= k) return UPRO_ERR_INVALID;
    int64_t tot = 0;
    for (int64_t v = 0; v < g.n; v++) tot += g.c(v);
    int64_t Lmax = lmax_of(tot, k, eps_ppm);
    std::vector<int32_t> P(part, part + g.n);
    int64_t cut = cut_of(g, P.data());
    std::vector<int64_t> C(k, 0);
    for (int64_t v = 0; v < g.n; v++) C[P[v]] += g.c(v);
    bool bal = true;
    for (int32_t b = 0; b < k; b++) bal = bal && C[b] <= Lmax;
    RoundOut o;
    if (!bal) {
        int rc = round_impl(g, k, Lmax, p, 0, rounds > 0 ? rounds : 1, true, P.data(), &cut, nullptr, &o);
        if (rc != UPRO_OK) return rc;
    }
    if (p.lp_rounds > 0) label_propagation(g, k, Lmax, p, p.lp_rounds, P.data(), &cut);
    if (round_cuts) round_cuts[0] = cut;
    bool unconstrained_rest = false, switched = false;
    int64_t imp1 = 0;
    const int32_t U1 = rounds - 3;                      /* unconstrained rounds 3..R-1 of schedule 1 */
    const int32_t U = unconstrained_rounds(rounds);     /* unconstrained rounds of schedules 3-6 */
    std::vector<int8_t> locked(p.lock_rebalanced ? g.n : 0, 0), locked_next(locked);
    for (int32_t i = 1; i <= rounds; i++) {
        RoundKind kind;
        int8_t code = 0;
        int32_t r = i, R = rounds;
        if (schedule == 2 || (schedule >= 3 && (i > U || switched))) {
            kind.constrained = true; code = 1;
        } else if (schedule == 3) {
            kind.tau_num = p.tau1_num; kind.tau_den = p.tau1_den; code = 3;
        } else if (schedule == 4) {
            kind.limit = INT64_MAX; code = 4;
        } else if (schedule == 5) {
            const int64_t D = U > 1 ? U - 1 : 1;                    /* alpha over rounds 1..U */
            kind.limit = (int64_t)(((i128)Lmax * (20 * D - 9 * (int64_t)(i - 1))) / (10 * D));
            code = 5;
        } else if (schedule == 6) {
            r = i; R = U;                                             /* tau_i of the U unconstrained rounds */
        } else if (schedule == 1) {
            if (i == 1 || (rounds >= 3 && i == rounds) || (i >= 3 && (!unconstrained_rest || switched))) {
                kind.constrained = true; code = 1;
            } else if (i == 2) {
                kind.tau_num = 1; kind.tau_den = 2; code = 2;
            } else {
                r = i - 2; R = U1;             /* tau_{i-2} of the U1 unconstrained rounds */
            }
        }
        const int64_t before = cut;
        if (p.lock_rebalanced) { kind.locked = locked.data(); kind.locked_out = locked_next.data(); }
        int rc = round_impl(g, k, Lmax, p, r, R, false, P.data(), &cut, nullptr, &o, kind);
        locked.swap(locked_next);
        if (rc != UPRO_OK) return rc;
        if (round_cuts) round_cuts[i] = cut;
        if (kinds) kinds[i - 1] = code;
        const int64_t imp = before - cut;
        if (schedule == 1) {
            if (i == 1) imp1 = imp;
            if (i == 2) unconstrained_rest = imp > imp1;
            if (i >= 3 && code == 0 && 500 * imp < before) switched = true;
        }
        if (schedule >= 3 && code != 1 && 500 * imp < before) switched = true;
    }
    memcpy(part, P.data(), sizeof(int32_t) * g.n);
    if (cut_out) *cut_out = cut;
    return UPRO_OK;
}

} /* extern "C" */
