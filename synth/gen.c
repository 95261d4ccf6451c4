/*
 * Seeded synthetic graph and partition generators.
 *
 * This module only produces inputs: CSR graphs with the degree structure of
 * the paper's benchmark classes (power-law Chung-Lu, R-MAT and random
 * geometric graphs; Sec. 7.1, Table 1), node and edge weights, and initial
 * partitions.  It contains none of the refinement arithmetic, so both the
 * CUDA library and the CPU oracle may consume what it writes.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), one stream per call, seeded by the
 * caller.  Every routine is deterministic for a given seed and gives the
 * same output on x86_64 and aarch64 (no floating-point reductions whose
 * order could differ, no platform intrinsics).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform double in [0,1) with 53 random bits */
static double sm64_unit(sm64 *r) { return (double)(sm64_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, bound) by rejection (bound > 0) */
static uint64_t sm64_below(sm64 *r, uint64_t bound) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
    uint64_t x;
    do { x = sm64_next(r); } while (x >= lim);
    return x % bound;
}

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* Seeded permutation of 0..n-1 (Fisher-Yates).                         */
void synth_permutation(int64_t n, uint64_t seed, int32_t *perm) {
    sm64 r = {seed};
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)sm64_below(&r, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Relabel both endpoints of an edge list through perm. */
void synth_relabel(int64_t ne, const int32_t *perm, int32_t *src, int32_t *dst) {
    for (int64_t e = 0; e < ne; e++) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
}

/* ------------------------------------------------------------------ */
/* Chung-Lu: expected degree w_i proportional to (i+1)^(-1/(gamma-1)),   */
/* scaled so that sum w = avg_deg * n.  ne = avg_deg*n/2 endpoint pairs */
/* are drawn, each endpoint proportional to w (inverse CDF).            */
int64_t synth_chung_lu_edges(int64_t n, double avg_deg, double gamma, uint64_t seed,
                             int32_t *src, int32_t *dst) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)n);
    if (!cdf) return -1;
    double ex = -1.0 / (gamma - 1.0), acc = 0.0;
    for (int64_t i = 0; i < n; i++) { acc += pow((double)(i + 1), ex); cdf[i] = acc; }
    for (int64_t i = 0; i < n; i++) cdf[i] /= acc;
    cdf[n - 1] = 1.0;
    int64_t ne = (int64_t)(avg_deg * (double)n / 2.0);
    sm64 r = {seed};
    for (int64_t e = 0; e < ne; e++) {
        for (int side = 0; side < 2; side++) {
            double u = sm64_unit(&r);
            int64_t lo = 0, hi = n - 1;           /* first i with cdf[i] > u */
            while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
            if (side == 0) src[e] = (int32_t)lo; else dst[e] = (int32_t)lo;
        }
    }
    free(cdf);
    return ne;
}

/* ------------------------------------------------------------------ */
/* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge descends    */
/* `scale` levels of the adjacency matrix, picking a quadrant with      */
/* probabilities (a, b, c, 1-a-b-c), quantised to 1/65536; one 64-bit   */
/* draw serves four levels.                                             */
void synth_rmat_edges(int scale, int64_t ne, double a, double b, double c, uint64_t seed,
                      int32_t *src, int32_t *dst) {
    sm64 r = {seed};
    uint32_t ta = (uint32_t)(a * 65536.0 + 0.5), tab = (uint32_t)((a + b) * 65536.0 + 0.5);
    uint32_t tabc = (uint32_t)((a + b + c) * 65536.0 + 0.5);
    for (int64_t e = 0; e < ne; e++) {
        uint32_t u = 0, v = 0;
        uint64_t bits = 0;
        for (int l = 0; l < scale; l++) {
            if ((l & 3) == 0) bits = sm64_next(&r);
            uint32_t x = (uint32_t)(bits & 0xFFFFu);
            bits >>= 16;
            uint32_t bu = (uint32_t)(x >= tab);
            uint32_t bv = (uint32_t)((x >= ta) & (x < tab)) | (uint32_t)(x >= tabc);
            u = (u << 1) | bu; v = (v << 1) | bv;
        }
        src[e] = (int32_t)u; dst[e] = (int32_t)v;
    }
}

/* ------------------------------------------------------------------ */
/* Random geometric graph in the unit square: n points, edge iff the    */
/* Euclidean distance is below `radius`.  Points are bucketed into a    */
/* square grid of cells of side >= radius; node ids are assigned in     */
/* (cell_x, cell_y, draw order) order, so ids are spatially local.      */
/* Two passes: with src == NULL only the number of pairs (u < v) is     */
/* returned.  xy (2n doubles, may be NULL) receives the coordinates in  */
/* id order.                                                            */
typedef struct { double x, y; int64_t cell; int64_t draw; } rpt;

static int rpt_cmp(const void *pa, const void *pb) {
    const rpt *p = (const rpt *)pa, *q = (const rpt *)pb;
    if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
    return p->draw < q->draw ? -1 : (p->draw > q->draw);
}

int64_t synth_rgg_edges(int64_t n, double radius, uint64_t seed, int32_t *src, int32_t *dst,
                        double *xy) {
    int64_t g = (int64_t)floor(1.0 / radius);
    if (g < 1) g = 1;
    rpt *p = (rpt *)malloc(sizeof(rpt) * (size_t)n);
    int64_t *start = (int64_t *)calloc((size_t)(g * g + 1), sizeof(int64_t));
    if (!p || !start) { free(p); free(start); return -1; }
    sm64 r = {seed};
    for (int64_t i = 0; i < n; i++) {
        p[i].x = sm64_unit(&r); p[i].y = sm64_unit(&r); p[i].draw = i;
        int64_t cx = (int64_t)(p[i].x * (double)g), cy = (int64_t)(p[i].y * (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        p[i].cell = cx * g + cy;
    }
    qsort(p, (size_t)n, sizeof(rpt), rpt_cmp);
    for (int64_t i = 0; i < n; i++) start[p[i].cell + 1]++;
    for (int64_t cidx = 0; cidx < g * g; cidx++) start[cidx + 1] += start[cidx];
    if (xy) for (int64_t i = 0; i < n; i++) { xy[2 * i] = p[i].x; xy[2 * i + 1] = p[i].y; }
    double r2 = radius * radius;
    int64_t cnt = 0;
    for (int64_t cx = 0; cx < g; cx++)
        for (int64_t cy = 0; cy < g; cy++) {
            int64_t c0 = cx * g + cy;
            for (int64_t i = start[c0]; i < start[c0 + 1]; i++)
                for (int64_t dx = -1; dx <= 1; dx++)
                    for (int64_t dy = -1; dy <= 1; dy++) {
                        int64_t nx = cx + dx, ny = cy + dy;
                        if (nx < 0 || ny < 0 || nx >= g || ny >= g) continue;
                        int64_t c1 = nx * g + ny;
                        for (int64_t j = start[c1]; j < start[c1 + 1]; j++) {
                            if (j <= i) continue;
                            double ddx = p[i].x - p[j].x, ddy = p[i].y - p[j].y;
                            if (ddx * ddx + ddy * ddy < r2) {
                                if (src) { src[cnt] = (int32_t)i; dst[cnt] = (int32_t)j; }
                                cnt++;
                            }
                        }
                    }
        }
    free(p); free(start);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Build a symmetric CSR from an undirected edge list: self loops are   */
/* dropped, both directions are inserted, parallel entries collapse to  */
/* one, and each adjacency list is sorted by neighbour id.  adj must    */
/* hold 2*ne entries.  Returns m (number of directed entries).          */
int64_t synth_build_csr(int64_t n, int64_t ne, const int32_t *src, const int32_t *dst,
                        int64_t *xadj, int32_t *adj) {
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int32_t *tmp_u = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne + 1));
    int32_t *tmp_v = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne + 1));
    if (!cnt || !tmp_u || !tmp_v) { free(cnt); free(tmp_u); free(tmp_v); return -1; }
    /* pass 1: counting sort of directed entries by neighbour (secondary key) */
    for (int64_t e = 0; e < ne; e++) if (src[e] != dst[e]) { cnt[dst[e] + 1]++; cnt[src[e] + 1]++; }
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t tot = cnt[n];
    for (int64_t e = 0; e < ne; e++) {
        int32_t a = src[e], b = dst[e];
        if (a == b) continue;
        int64_t p = cnt[b]++; tmp_u[p] = a; tmp_v[p] = b;   /* entry a -> b, keyed by b */
        p = cnt[a]++; tmp_u[p] = b; tmp_v[p] = a;           /* entry b -> a, keyed by a */
    }
    /* pass 2: stable counting sort by owner (primary key) */
    memset(cnt, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t p = 0; p < tot; p++) cnt[tmp_u[p] + 1]++;
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    for (int64_t p = 0; p < tot; p++) { int32_t u = tmp_u[p]; adj[cnt[u]++] = tmp_v[p]; }
    /* cnt[u] now holds the end of u's segment; segments are sorted; dedup in place */
    int64_t w = 0, beg = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t end = cnt[u];
        xadj[u] = w;
        for (int64_t p = beg; p < end; p++)
            if (p == beg || adj[p] != adj[p - 1]) adj[w++] = adj[p];
        beg = end;
    }
    xadj[n] = w;
    free(cnt); free(tmp_u); free(tmp_v);
    return w;
}

/* ------------------------------------------------------------------ */
/* Symmetric edge weights uniform in [lo, hi]: the weight of {u,v} is a */
/* hash of (min, max, seed), so both directions agree.                  */
void synth_edge_weights_uniform(int64_t n, const int64_t *xadj, const int32_t *adj, int32_t lo,
                                int32_t hi, uint64_t seed, int32_t *adjw) {
    uint64_t span = (uint64_t)(hi - lo + 1);
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = xadj[u]; e < xadj[u + 1]; e++) {
            uint64_t a = (uint64_t)(u < adj[e] ? u : adj[e]), b = (uint64_t)(u < adj[e] ? adj[e] : u);
            uint64_t h = mix64(mix64(seed ^ (a * 0x9E3779B97F4A7C15ull)) + b);
            adjw[e] = lo + (int32_t)(h % span);
        }
}

/* Node weights from a Zipf(s) law truncated to [lo, hi] (inverse CDF). */
void synth_node_weights_zipf(int64_t n, double s, int32_t lo, int32_t hi, uint64_t seed, int32_t *vwgt) {
    int64_t span = (int64_t)hi - lo + 1;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)span);
    double acc = 0.0;
    for (int64_t i = 0; i < span; i++) { acc += pow((double)(lo + i), -s); cdf[i] = acc; }
    for (int64_t i = 0; i < span; i++) cdf[i] /= acc;
    cdf[span - 1] = 1.0;
    sm64 r = {seed};
    for (int64_t v = 0; v < n; v++) {
        double u = sm64_unit(&r);
        int64_t a = 0, b = span - 1;
        while (a < b) { int64_t mid = (a + b) >> 1; if (cdf[mid] > u) b = mid; else a = mid + 1; }
        vwgt[v] = (int32_t)(lo + a);
    }
    free(cdf);
}

/* ------------------------------------------------------------------ */
/* Random balanced partition: a seeded permutation, block = rank mod k. */
void synth_part_random_balanced(int64_t n, int32_t k, uint64_t seed, int32_t *part) {
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    synth_permutation(n, seed, perm);
    for (int64_t i = 0; i < n; i++) part[perm[i]] = (int32_t)(i % k);
    free(perm);
}

/* Spatial strip split: nodes ordered by (x, id); block = min(k-1,       */
/* floor(k * prefix_excl / c(V))) where prefix_excl is the node weight  */
/* of all nodes before it in that order.                                */
typedef struct { double x; int32_t id; } xid;
static int xid_cmp(const void *pa, const void *pb) {
    const xid *p = (const xid *)pa, *q = (const xid *)pb;
    if (p->x != q->x) return p->x < q->x ? -1 : 1;
    return p->id < q->id ? -1 : (p->id > q->id);
}

void synth_part_strip(int64_t n, int32_t k, const double *xy, const int32_t *vwgt, int32_t *part) {
    xid *o = (xid *)malloc(sizeof(xid) * (size_t)(n > 0 ? n : 1));
    int64_t total = 0;
    for (int64_t i = 0; i < n; i++) { o[i].x = xy[2 * i]; o[i].id = (int32_t)i; total += vwgt ? vwgt[i] : 1; }
    qsort(o, (size_t)n, sizeof(xid), xid_cmp);
    int64_t pre = 0;
    for (int64_t i = 0; i < n; i++) {
        int32_t v = o[i].id;
        int64_t b = (int64_t)(((__int128)k * pre) / (total > 0 ? total : 1));
        if (b > k - 1) b = k - 1;
        part[v] = (int32_t)b;
        pre += vwgt ? vwgt[v] : 1;
    }
    free(o);
}
