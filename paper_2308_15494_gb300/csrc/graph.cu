// Step (e): block weights and edge cut (Sec. 2); step (a): the gain table
// omega(v, V_b) (Sec. 2, Sec. 6.1), built from the partition (its delta
// update after moves is in delta.cu); create-time graph checks and incident
// weights omega(I(v)).
#include "kernels.h"

namespace upr {
namespace {

constexpr int kChunk = 1024;   // adjacency entries per warp in entry-parallel passes

// Owner of adjacency entry e: the v with xadj[v] <= e < xadj[v+1] (rows may be empty).
__device__ __forceinline__ int64_t owner_of(const int64_t *__restrict__ xadj, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (xadj[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Block weights: per-CTA accumulators (BlockDelta), lanes with the same
// block combined with __match_any_sync first.
__global__ void k_block_weights(const int32_t *__restrict__ part, const int32_t *__restrict__ vwgt, int64_t n, int32_t K,
                                int64_t *__restrict__ C) {
    extern __shared__ unsigned long long s_c[];
    BlockDelta bd = make_block_delta(s_c, K, (unsigned long long *)C);
    bd.init();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        bd.add(v < n ? part[v] : -1, v < n ? (vwgt ? vwgt[v] : 1) : 0);
    }
    bd.flush((unsigned long long *)C);
}

// Edge cut per graph: warp per chunk of adjacency entries; a warp whose
// entries all belong to one graph adds once, otherwise each lane adds its own.
__global__ void k_edge_cut(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                           const int32_t *__restrict__ adjw, const int32_t *__restrict__ part,
                           const int32_t *__restrict__ gid, int64_t n, int64_t m, unsigned long long *__restrict__ out) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t e0 = warp * kChunk, e1 = min(m, e0 + kChunk);
    long long acc = 0;
    int32_t g0 = 0, g1 = 0;
    if (e0 < m) {                                 // warp-uniform
        int64_t e = e0 + lane;
        int64_t v = e < e1 ? owner_of(xadj, n, e) : 0;
        g0 = gid ? gid[owner_of(xadj, n, e0)] : 0;
        g1 = gid ? gid[owner_of(xadj, n, e1 - 1)] : 0;
        for (; e < e1; e += 32) {
            while (xadj[v + 1] <= e) v++;
            const int32_t u = adj[e];
            if (v < u && part[v] != part[u]) {    // each undirected edge once
                const long long w = adjw ? adjw[e] : 1;
                if (g0 == g1) acc += w;
                else atomicAdd(&out[gid[v]], (unsigned long long)w);
            }
        }
    }
    acc = warp_sum(acc);
    if (gid) {
        if (lane == 0 && acc && g0 == g1) atomicAdd(&out[g0], (unsigned long long)acc);
        return;
    }
    // one graph: one atomic per CTA (one per warp would queue on the word)
    __shared__ long long s_acc[8];
    if (lane == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) acc += s_acc[w];
        if (acc) atomicAdd(&out[0], (unsigned long long)acc);
    }
}

// omega(I(v)) per node (warp per node); records the maximum and overflow.
// omega(I(v)) per node (warp per node, grid-stride) and its maximum: one
// atomic per CTA (one per node would queue on the single word).
__global__ void __launch_bounds__(256) k_incident(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adjw,
                                                  int64_t n, int32_t *__restrict__ wI,
                                                  unsigned long long *__restrict__ wmax) {
    __shared__ unsigned long long s_max[8];
    const int lane = threadIdx.x & 31;
    unsigned long long mx = 0;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n;
         v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        long long acc = 0;
        for (int64_t e = xadj[v] + lane; e < xadj[v + 1]; e += 32) acc += adjw ? adjw[e] : 1;
        acc = warp_sum(acc);
        if (lane == 0) wI[v] = acc > 0x7fffffffLL ? 0x7fffffff : (int32_t)acc;
        mx = (unsigned long long)acc > mx ? (unsigned long long)acc : mx;
    }
    if (lane == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = s_max[w] > mx ? s_max[w] : mx;
        if (mx) atomicMax(wmax, mx);
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t entry_hash(uint64_t a, uint64_t b, uint64_t w) {
    return mix64(mix64(mix64(a + 0x1234567ull) ^ b) + w);
}

// Validation bits: 1 xadj, 2 neighbour range (or, in a batch, a neighbour in
// another graph), 4 self loop, 8 edge weight, 16 node weight, 32 duplicate
// neighbour in a row, 128 a row not strictly increasing (no error: rows with
// strictly increasing ids have no duplicates, others get the exact duplicate
// check); asymmetry shows as differing sums of hash(v,u,w) and
// hash(u,v,w) over the entries (an asymmetric graph whose sums agree passes:
// probability about 2^-64 for a graph not built against the hash).
__global__ void k_validate_entries(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                                   const int32_t *__restrict__ adjw, const int32_t *__restrict__ gid, int64_t n,
                                   int64_t m, unsigned long long *__restrict__ acc, int32_t *__restrict__ flags) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t e0 = warp * kChunk, e1 = min(m, e0 + kChunk);
    unsigned long long h1 = 0, h2 = 0;
    int32_t f = 0;
    if (e0 < m) {
        int64_t e = e0 + lane;
        int64_t v = e < e1 ? owner_of(xadj, n, e) : 0;
        for (; e < e1; e += 32) {
            while (xadj[v + 1] <= e) v++;
            int32_t u = adj[e];
            int32_t w = adjw ? adjw[e] : 1;
            // a row whose next entry is not larger: unsorted, or a duplicate
            // (bit 128, not an error by itself: the exact duplicate check runs)
            if (e + 1 < xadj[v + 1] && adj[e + 1] <= u) f |= 128;
            if (u < 0 || u >= n || (gid && gid[u] != gid[v])) { f |= 2; continue; }
            if (u == v) f |= 4;
            if (w <= 0) f |= 8;
            h1 += entry_hash((uint64_t)v, (uint64_t)u, (uint64_t)(uint32_t)w);
            h2 += entry_hash((uint64_t)u, (uint64_t)v, (uint64_t)(uint32_t)w);
        }
    }
    h1 = warp_sum(h1);
    h2 = warp_sum(h2);
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    // one set of atomics per CTA (the sums wrap modulo 2^64 in any order)
    __shared__ unsigned long long s_h[2][8];
    __shared__ int32_t s_f[8];
    if (lane == 0) {
        s_h[0][threadIdx.x >> 5] = h1;
        s_h[1][threadIdx.x >> 5] = h2;
        s_f[threadIdx.x >> 5] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            h1 += s_h[0][w];
            h2 += s_h[1][w];
            f |= s_f[w];
        }
        if (h1) atomicAdd(&acc[0], h1);
        if (h2) atomicAdd(&acc[1], h2);
        if (f) atomicOr(flags, f);
    }
}

__global__ void k_validate_nodes(const int64_t *__restrict__ xadj, const int32_t *__restrict__ vwgt, int64_t n, int64_t m,
                                 int32_t *__restrict__ flags) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n) return;
    int32_t f = 0;
    if (v == 0 && xadj[0] != 0) f |= 1;
    if (v == n && xadj[n] != m) f |= 1;
    if (v < n && xadj[v + 1] < xadj[v]) f |= 1;
    if (v < n && vwgt && vwgt[v] <= 0) f |= 16;
    if (f) atomicOr(flags, f);
}

// The cut of a partition from its gain table (Sec. 2): every edge leaving v
// is counted once from each end, so cut = (sum of omega(I(v)) - sum of
// omega(v, V_P(v))) / 2; one read of the own-block entry per node instead of
// a pass over the edges.  One graph; *out (zero) receives twice the cut
// first, halved by the last step below.
__global__ void k_cut_from_table(const GraphDev g, const int32_t *__restrict__ part, const int32_t *__restrict__ W,
                                 unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s_w[8];
    unsigned long long acc = 0;
    UPR_FOR(v, g.n) {
        const int32_t own = g.sp.on() ? sp_get(g.sp, v, part[v]) : W[(int64_t)v * g.k + part[v]];
        acc += (unsigned long long)((int64_t)g.wI[v] - own);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
        if (t) atomicAdd(out, t);
    }
}

__global__ void k_halve(int64_t *x) { *x /= 2; }

// Duplicate adjacency entries (E is a set of pairs {v, u}, Sec. 2, so a row
// lists each neighbour once).  Rows of degree <= kHubDegree: a CTA takes the
// rows that start in a chunk of kDupChunk entries (they may run into the
// next chunk, by less than kHubDegree entries) and inserts (row, neighbour)
// into a hash set in shared memory: kDupSlots 64-bit keys, linear probing, a
// key that meets itself is a duplicate.  Keys carry the CTA's iteration
// number, so a slot holding another iteration's key counts as empty and the
// set is never cleared between chunks.  Hub rows: k_dup_hubs.  Both set
// validation bit 32.
constexpr int kDupChunk = 4096;
constexpr int kDupSlots = 4 * kDupChunk;             // >= 2 x the entries of one chunk's rows (< 2 kDupChunk)
constexpr int64_t kDupRange = (int64_t)1 << 20;     // neighbour ids per bitmap of k_dup_hubs
static_assert(kHubDegree <= kDupChunk, "a row of a chunk ends within the next chunk");
static_assert((kDupSlots & (kDupSlots - 1)) == 0, "power of two");

__device__ __forceinline__ uint64_t dup_key(uint64_t iter, int64_t row, int32_t u) {
    // iteration: 20 bits; row: its first entry's offset from the chunk's first
    // row start, 13 bits (< kDupChunk + kHubDegree); neighbour: 31 bits
    return (iter << 44) | ((uint64_t)row << 31) | (uint64_t)(uint32_t)u;
}

// first[c] = the first row starting at or after entry c * kDupChunk (n if
// none), c = 0 .. chunks: one pass over the rows instead of a search per chunk.
__global__ void k_dup_chunk_first(const int64_t *__restrict__ xadj, int64_t n, int64_t chunks,
                                  int32_t *__restrict__ first) {
    UPR_FOR(v, n + 1) {
        // chunks c with xadj[v - 1] < c * kDupChunk <= xadj[v] start at row v
        const int64_t hi = v < n ? xadj[v] : (int64_t)chunks * kDupChunk;
        const int64_t lo = v > 0 ? xadj[v - 1] : -1;
        const int64_t c0 = lo < 0 ? 0 : lo / kDupChunk + 1;
        const int64_t c1 = v < n ? hi / kDupChunk : chunks;
        for (int64_t c = c0; c <= c1 && c <= chunks; c++) first[c] = (int32_t)v;
    }
}

__global__ void __launch_bounds__(512) k_dup_rows(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                                                  int64_t n, int64_t m, const int32_t *__restrict__ chunk_first,
                                                  int32_t *__restrict__ flags) {
    extern __shared__ unsigned long long s_set[];
    __shared__ int64_t s_v[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    for (int i = threadIdx.x; i < kDupSlots; i += blockDim.x) s_set[i] = ~0ull;     // iteration field all ones
    bool dup = false;
    const int64_t chunks = (m + kDupChunk - 1) / kDupChunk;
    uint64_t iter = 0;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x, iter = (iter + 1) & 0xFFFFF) {
        const int64_t e0 = c * kDupChunk, e1 = min(m, e0 + kDupChunk);
        __syncthreads();
        if (threadIdx.x == 0 && chunk_first) {
            s_v[0] = chunk_first[c];
            s_v[1] = chunk_first[c + 1];
        } else if (threadIdx.x == 0) {
            // the rows that start in [e0, e1): first row starting at or after
            // e0, first row starting at or after e1
            int64_t lo = 0, hi = n;
            while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (xadj[mid] < e0) lo = mid + 1; else hi = mid; }
            s_v[0] = lo;
            hi = n;
            while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (xadj[mid] < e1) lo = mid + 1; else hi = mid; }
            s_v[1] = lo;
        }
        __syncthreads();
        const int64_t va = s_v[0], vb = s_v[1];
        if (va >= vb) continue;
        const int64_t f0 = xadj[va];
        for (int64_t v = va + warp; v < vb; v += warps) {
            const int64_t r0 = xadj[v], r1 = xadj[v + 1];
            if (r1 - r0 < 2 || r1 - r0 > kHubDegree) continue;
            for (int64_t e = r0 + lane; e < r1; e += 32) {
                const uint64_t key = dup_key(iter, r0 - f0, adj[e]);
                uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 50) & (kDupSlots - 1);
                for (int probe = 0; probe < kDupSlots;) {
                    const unsigned long long cur = s_set[h];
                    if ((cur >> 44) != iter) {            // another iteration's key: empty
                        if (atomicCAS(&s_set[h], cur, key) == cur) break;
                        continue;                         // lost the slot: look at it again
                    }
                    if (cur == key) { dup = true; break; }
                    h = (h + 1) & (kDupSlots - 1);
                    probe++;
                }
            }
        }
    }
    if (__syncthreads_or(dup) && threadIdx.x == 0) atomicOr(flags, 32);
}

// Hub rows (degree > kHubDegree): CTA (h, r) takes hub h's neighbours in
// [lo + r * kDupRange, lo + (r + 1) * kDupRange) over the node ids [lo, hi)
// of the hub's graph, sets their bits in a shared-memory bitmap (8 loads in
// flight per thread); a bit found set is a duplicate.
__global__ void __launch_bounds__(256) k_dup_hubs(const int32_t *__restrict__ hubs, const int64_t *__restrict__ xadj,
                                                  const int32_t *__restrict__ adj, int64_t n,
                                                  const int32_t *__restrict__ gid, const int64_t *__restrict__ noff,
                                                  int32_t *__restrict__ flags) {
    extern __shared__ uint32_t s_bits[];
    const int32_t v = hubs[blockIdx.x];
    const int64_t e0 = xadj[v], e1 = xadj[v + 1];
    const int64_t hi = noff ? noff[gid[v] + 1] : n;
    const int64_t lo = (noff ? noff[gid[v]] : 0) + (int64_t)blockIdx.y * kDupRange;
    if (lo >= hi) return;                                   // uniform over the CTA
    for (int i = threadIdx.x; i < (int)(kDupRange / 32); i += blockDim.x) s_bits[i] = 0;
    __syncthreads();
    bool dup = false;
    constexpr int kU = 8;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += (int64_t)blockDim.x * kU) {
        int32_t u[kU];
#pragma unroll
        for (int j = 0; j < kU; j++) {
            const int64_t x = e + (int64_t)j * blockDim.x;
            u[j] = x < e1 ? adj[x] : -1;
        }
#pragma unroll
        for (int j = 0; j < kU; j++) {
            const int64_t x = (int64_t)u[j] - lo;
            if (u[j] < 0 || x < 0 || x >= kDupRange) continue;
            const uint32_t bit = 1u << (x & 31);
            dup |= (atomicOr(&s_bits[x >> 5], bit) & bit) != 0;
        }
    }
    if (__syncthreads_or(dup) && threadIdx.x == 0) atomicOr(flags, 32);
}

// Dense gain table, tiled: one CTA per tile of consecutive nodes whose
// adjacency (without hubs) is one contiguous range of entries.  The CTA
// streams that range with 16-byte loads (4 * UNROLL entries in flight per
// thread), gathers the neighbours' blocks, finds each entry's owner (binary
// search in the tile's xadj slice for the first of four consecutive entries,
// then a forward walk), accumulates all rows of the tile in shared memory and
// writes them as one contiguous block with streaming stores.  WEIGHTED: edge
// weights are read (else unit); LOCAL: 0 = one graph (block ids are
// columns), 1 = a batch with k a power of two (mask), 2 = a batch with other
// k (remainder).  Hub rows stay zero.
template <int LOCAL>
__device__ __forceinline__ int tile_col(int32_t p, int32_t k, int32_t kmask) {
    return LOCAL == 0 ? p : LOCAL == 1 ? (p & kmask) : p % k;
}

__device__ __forceinline__ int tile_owner(const int64_t *s_x, int nn, int64_t e) {
    int lo = 0, hi = nn - 1;            // last i with s_x[i] <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_x[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool WEIGHTED, int LOCAL, int UNROLL>
__device__ __forceinline__ void table_tile(const TableTile t, const int64_t *__restrict__ xadj,
                                           const int32_t *__restrict__ adj, const int32_t *__restrict__ adjw,
                                           const int32_t *__restrict__ part, int32_t k, int32_t kmask,
                                           int32_t *__restrict__ W, const SparseRows &sp, bool bulk) {
    extern __shared__ int4 s_raw[];
    const int nn = t.v1 - t.v0;
    int64_t *s_x = reinterpret_cast<int64_t *>(s_raw);           // nn + 1 row starts
    int *rows = reinterpret_cast<int *>(s_x + ((nn + 2) & ~1));    // nn * k
    for (int i = threadIdx.x; i <= nn; i += blockDim.x) s_x[i] = xadj[t.v0 + i];
    // hashed rows: the tile's row offsets, fetched now so that the write-out
    // does not wait for them row by row
    int64_t *s_off = sp.on() ? reinterpret_cast<int64_t *>(reinterpret_cast<int2 *>(rows + nn * k) + 8 * sp.buf_cap)
                             : nullptr;
    if (sp.on())
        for (int i = threadIdx.x; i <= nn; i += blockDim.x) s_off[i] = sp.off[t.v0 + i];
    // (k % 4 != 0: the rows' block is not a whole number of 16-byte words)
    const bool quads = k % 4 == 0;
    const int words4 = nn * k / 4;
    const int4 z = make_int4(0, 0, 0, 0);
    if (quads)
        for (int i = threadIdx.x; i < words4; i += blockDim.x) reinterpret_cast<int4 *>(rows)[i] = z;
    else
        for (int i = threadIdx.x; i < nn * k; i += blockDim.x) rows[i] = 0;
    __syncthreads();
    // ragged head and tail (fewer than 4 entries each) element by element
    const int64_t qa = (t.e0 + 3) >> 2, qb = t.e1 >> 2;     // aligned quads [qa, qb)
    if (threadIdx.x < 8) {
        const int64_t e = threadIdx.x < 4 ? t.e0 + threadIdx.x : (qb << 2) + (threadIdx.x - 4);
        const bool in_head = threadIdx.x < 4 && e < min(qa << 2, t.e1);
        const bool in_tail = threadIdx.x >= 4 && qb >= qa && e < t.e1;
        if (in_head || in_tail) {
            const int o = tile_owner(s_x, nn, e);
            atomicAdd(&rows[o * k + tile_col<LOCAL>(part[adj[e]], k, kmask)], WEIGHTED ? adjw[e] : 1);
        }
    }
    const int4 *adj4 = reinterpret_cast<const int4 *>(adj);
    const int4 *adjw4 = reinterpret_cast<const int4 *>(adjw);
    for (int64_t q0 = qa + threadIdx.x; q0 < qb; q0 += (int64_t)blockDim.x * UNROLL) {
        int4 u[UNROLL], w[UNROLL];
#pragma unroll
        for (int r = 0; r < UNROLL; r++) {
            const int64_t q = q0 + (int64_t)r * blockDim.x;
            u[r] = q < qb ? __ldcs(adj4 + q) : make_int4(0, 0, 0, 0);
            if (WEIGHTED) w[r] = q < qb ? __ldcs(adjw4 + q) : make_int4(0, 0, 0, 0);
        }
        int pb[UNROLL][4];
#pragma unroll
        for (int r = 0; r < UNROLL; r++) {
            const bool ok = q0 + (int64_t)r * blockDim.x < qb;
            pb[r][0] = ok ? tile_col<LOCAL>(part[u[r].x], k, kmask) : 0;
            pb[r][1] = ok ? tile_col<LOCAL>(part[u[r].y], k, kmask) : 0;
            pb[r][2] = ok ? tile_col<LOCAL>(part[u[r].z], k, kmask) : 0;
            pb[r][3] = ok ? tile_col<LOCAL>(part[u[r].w], k, kmask) : 0;
        }
#pragma unroll
        for (int r = 0; r < UNROLL; r++) {
            const int64_t q = q0 + (int64_t)r * blockDim.x;
            if (q >= qb) continue;
            const int64_t e = q << 2;
            int o = tile_owner(s_x, nn, e);
            int ww[4] = {1, 1, 1, 1};
            if (WEIGHTED) { ww[0] = w[r].x; ww[1] = w[r].y; ww[2] = w[r].z; ww[3] = w[r].w; }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                while (s_x[o + 1] <= e + j) o++;
                atomicAdd(&rows[o * k + pb[r][j]], ww[j]);
            }
        }
    }
    __syncthreads();
    if (sp.on()) {
        // sparse table: a warp per row fills the row's slots in its own shared
        // buffer (each non-zero column is claimed once, by the lane that holds
        // it), then stores them with coalesced 8-byte stores
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int2 *buf = reinterpret_cast<int2 *>(rows + nn * k) + warp * sp.buf_cap;
        for (int r = warp; r < nn; r += (int)(blockDim.x >> 5)) {
            const int64_t o = s_off[r];
            const uint32_t cap = (uint32_t)(s_off[r + 1] - o);
            if (cap > (uint32_t)sp.buf_cap) {
                // a hub: its row is empty here, the chunk pass fills it
                for (uint32_t i = lane; i < cap; i += 32) sp.slot[o + i] = make_int2(kEmpty, 0);
                continue;
            }
            for (uint32_t i = lane; i < cap; i += 32) buf[i] = make_int2(kEmpty, 0);
            __syncwarp();
            for (int c = lane; c < k; c += 32) {
                const int w = rows[r * k + c];
                if (!w) continue;
                uint32_t h = sp_home(c, cap);
                for (uint32_t i = 0; i < cap; i++) {
                    if (atomicCAS(&buf[h].x, kEmpty, c) == kEmpty) { buf[h].y = w; break; }
                    h = (h + 1) & (cap - 1);
                }
            }
            __syncwarp();
            for (uint32_t i = lane; i < cap; i += 32) sp.slot[o + i] = buf[i];
            __syncwarp();
        }
        return;
    }
    if (!quads) {
        int32_t *dst1 = W + (int64_t)t.v0 * k;
        for (int i = threadIdx.x; i < nn * k; i += blockDim.x) __stcs(dst1 + i, rows[i]);
        return;
    }
    int4 *dst = reinterpret_cast<int4 *>(W + (int64_t)t.v0 * k);
    if (bulk) {
        // one bulk copy of the row block by the tensor memory accelerator
        // (k % 4 == 0: the block's bytes and both addresses are multiples of
        // 16); the rows' shared-memory writes made visible to the async proxy
        // first, and the copy's reads of them finished before the shared
        // memory is reused or released
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0 && words4 > 0) {
            const uint32_t src = (uint32_t)__cvta_generic_to_shared(rows);
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                         :: "l"(dst), "r"(src), "r"(words4 * 16) : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        return;
    }
    for (int i = threadIdx.x; i < words4; i += blockDim.x) __stcs(dst + i, reinterpret_cast<const int4 *>(rows)[i]);
}

// One tile per CTA for a build (grid = tiles); the rebuild alternatives,
// which usually return at once, run on one wave of CTAs that loop over the
// tiles, so that their early return costs a wave, not tens of thousands of CTAs.
template <bool WEIGHTED, int LOCAL, int UNROLL>
__global__ void __launch_bounds__(256) k_table_tiles(const TableTile *__restrict__ tiles, int64_t n_tiles,
                                                        const int64_t *__restrict__ xadj,
                                                        const int32_t *__restrict__ adj,
                                                        const int32_t *__restrict__ adjw,
                                                        const int32_t *__restrict__ part, int32_t k, int32_t kmask,
                                                        int32_t *__restrict__ W, const int64_t *__restrict__ deg_sum,
                                                        int64_t m, SparseRows sp, bool bulk) {
    if (deg_sum && *deg_sum * 4 < m) return;      // the delta update handles this case
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        table_tile<WEIGHTED, LOCAL, UNROLL>(tiles[ti], xadj, adj, adjw, part, k, kmask, W, sp, bulk);
        __syncthreads();                          // the next tile reuses the shared memory
    }
}

// Hub rows: one CTA per chunk of a hub's adjacency, shared-memory row, then
// atomic adds of the non-zero entries into the (zeroed) global row.
__global__ void __launch_bounds__(512) k_table_hub_chunks(const HubChunk *__restrict__ chunks, const int32_t *__restrict__ adj,
                                                          const int32_t *__restrict__ adjw,
                                                          const int32_t *__restrict__ part, int32_t k,
                                                          int32_t kmask, int32_t *__restrict__ W,
                                                          const int64_t *__restrict__ deg_sum, int64_t m,
                                                          SparseRows sp) {
    if (deg_sum && *deg_sum * 4 < m) return;
    extern __shared__ int s_row[];
    const HubChunk ch = chunks[blockIdx.x];
    for (int b = threadIdx.x; b < k; b += blockDim.x) s_row[b] = 0;
    __syncthreads();
    for (int64_t e = ch.begin + threadIdx.x; e < ch.end; e += blockDim.x)
        atomicAdd(&s_row[blk_local(part[adj[e]], k, kmask)], adjw ? adjw[e] : 1);
    __syncthreads();
    if (sp.on()) {
        for (int b = threadIdx.x; b < k; b += blockDim.x)
            if (s_row[b]) sp_add(sp, ch.v, b, s_row[b]);
        return;
    }
    int32_t *dst = W + (int64_t)ch.v * k;
    for (int b = threadIdx.x; b < k; b += blockDim.x)
        if (s_row[b]) atomicAdd(&dst[b], s_row[b]);
}

__global__ void k_node_graph(const int64_t *__restrict__ noff, int32_t ng, int64_t n, int32_t *__restrict__ gid) {
    UPR_FOR(v, n) {
        int32_t lo = 0, hi = ng - 1;            // last g with noff[g] <= v
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (noff[mid] <= v) lo = mid; else hi = mid - 1;
        }
        gid[v] = lo;
    }
}

__global__ void k_shift_adj(const int64_t *__restrict__ xadj, const int64_t *__restrict__ noff,
                            const int32_t *__restrict__ gid, int64_t n, int32_t *__restrict__ adj) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n;
         v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t off = noff[gid[v]];
        for (int64_t e = xadj[v] + lane; e < xadj[v + 1]; e += 32) {
            const int64_t u = (int64_t)adj[e] + off;
            adj[e] = (u < 0 || u >= n) ? -1 : (int32_t)u;
        }
    }
}

// Dense rows from the sparse table (inspection only): warp per row.
__global__ void k_sparse_to_dense(SparseRows sp, int64_t n, int32_t k, int32_t *__restrict__ W) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n;
         v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int32_t *row = W + v * k;
        for (int c = lane; c < k; c += 32) row[c] = 0;
        __syncwarp();
        for (int64_t i = sp.off[v] + lane; i < sp.off[v + 1]; i += 32) {
            const int2 e = sp.slot[i];
            if (e.x != kEmpty) row[e.x] = e.y;
        }
        __syncwarp();
    }
}

int sm_count() {
    static int cnt = 0;
    if (!cnt) {
        int dev = 0;
        UPR_CUDA(cudaGetDevice(&dev));
        UPR_CUDA(cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev));
    }
    return cnt;
}

}  // namespace

void block_weights(const GraphDev &g, const int32_t *part, int64_t *C, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(C, 0, sizeof(int64_t) * g.K(), s));
    if (g.n == 0) return;
    int64_t blocks = std::min<int64_t>(ceil_div(g.n, 256), (int64_t)sm_count() * 8);
    k_block_weights<<<(unsigned)blocks, 256, block_delta_smem(g.K()), s>>>(part, g.vwgt, g.n, g.K(), C);
    UPR_LAUNCH_CHECK();
}

void edge_cut(const GraphDev &g, const int32_t *part, int64_t *cut, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(cut, 0, sizeof(int64_t) * g.ng, s));
    if (g.m == 0) return;
    int64_t warps = ceil_div(g.m, kChunk);
    k_edge_cut<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, s>>>(g.xadj, g.adj, g.adjw, part, g.gid, g.n, g.m,
                                                                   (unsigned long long *)cut);
    UPR_LAUNCH_CHECK();
}

void cut_from_table(const GraphDev &g, const int32_t *part, const int32_t *W, int64_t *cut, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(cut, 0, sizeof(int64_t), s));
    if (g.n == 0) return;
    k_cut_from_table<<<grid_for(g.n), 256, 0, s>>>(g, part, W, (unsigned long long *)cut);
    UPR_LAUNCH_CHECK();
    k_halve<<<1, 1, 0, s>>>(cut);
    UPR_LAUNCH_CHECK();
}

void incident_weights(const GraphDev &g, int32_t *wI, int64_t *wmax, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(wmax, 0, sizeof(int64_t), s));
    if (g.n == 0) return;
    k_incident<<<wave_grid((const void *)k_incident, 256, 0, ceil_div(g.n * 32, 256)), 256, 0, s>>>(
        g.xadj, g.adjw, g.n, wI, (unsigned long long *)wmax);
    UPR_LAUNCH_CHECK();
}

void pack_batch(const GraphDev &g, const int64_t *noff, int32_t *gid, int32_t *adj, cudaStream_t s) {
    if (g.n == 0) return;
    k_node_graph<<<grid_for(g.n), 256, 0, s>>>(noff, g.ng, g.n, gid);
    UPR_LAUNCH_CHECK();
    const int64_t blocks = std::min<int64_t>(ceil_div(g.n * 32, 256), (int64_t)sm_count() * 16);
    k_shift_adj<<<(unsigned)blocks, 256, 0, s>>>(g.xadj, noff, gid, g.n, adj);
    UPR_LAUNCH_CHECK();
}

void sparse_to_dense(const GraphDev &g, int32_t *W, cudaStream_t s) {
    if (g.n == 0 || !g.sp.on()) return;
    const int64_t blocks = std::min<int64_t>(ceil_div(g.n * 32, 256), (int64_t)sm_count() * 16);
    k_sparse_to_dense<<<(unsigned)blocks, 256, 0, s>>>(g.sp, g.n, g.k, W);
    UPR_LAUNCH_CHECK();
}

void validate_graph(const GraphDev &g, uint64_t *d_acc, int32_t *d_flags, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(d_acc, 0, 2 * sizeof(uint64_t), s));
    UPR_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int32_t), s));
    k_validate_nodes<<<(unsigned)ceil_div(g.n + 1, 256), 256, 0, s>>>(g.xadj, g.vwgt, g.n, g.m, d_flags);
    UPR_LAUNCH_CHECK();
    if (g.m > 0 && g.n > 0) {
        int64_t warps = ceil_div(g.m, kChunk);
        k_validate_entries<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, s>>>(
            g.xadj, g.adj, g.adjw, g.gid, g.n, g.m, (unsigned long long *)d_acc, d_flags);
        UPR_LAUNCH_CHECK();
    }
}

void validate_duplicates(const GraphDev &g, int32_t *d_flags, const int32_t *hubs, int64_t n_hubs,
                         const int64_t *noff, int64_t max_graph_nodes, int32_t *scratch, int64_t scratch_ints,
                         cudaStream_t s) {
    if (g.m == 0 || g.n == 0) return;
    // rows up to kHubDegree by chunks of entries, hub rows by CTAs
    const size_t shm_rows = (size_t)kDupSlots * sizeof(unsigned long long);
    const size_t shm_hubs = (size_t)(kDupRange / 32) * sizeof(uint32_t);
    kernel_setup((const void *)k_dup_rows, -1);
    kernel_setup((const void *)k_dup_hubs, -1);
    const int64_t chunks = ceil_div(g.m, (int64_t)kDupChunk);
    int32_t *first = chunks + 1 <= scratch_ints ? scratch : nullptr;
    if (first) {
        k_dup_chunk_first<<<grid_for(g.n + 1), 256, 0, s>>>(g.xadj, g.n, chunks, first);
        UPR_LAUNCH_CHECK();
    }
    const unsigned grid = wave_grid((const void *)k_dup_rows, 512, shm_rows, chunks);
    k_dup_rows<<<grid, 512, shm_rows, s>>>(g.xadj, g.adj, g.n, g.m, first, d_flags);
    UPR_LAUNCH_CHECK();
    if (n_hubs > 0) {
        // ranges of node ids per hub: those of the largest graph
        const int64_t ranges = ceil_div(std::max<int64_t>(max_graph_nodes, 1), kDupRange);
        k_dup_hubs<<<dim3((unsigned)n_hubs, (unsigned)ranges), 256, shm_hubs, s>>>(
            hubs, g.xadj, g.adj, g.n, g.gid, g.ng > 1 ? noff : nullptr, d_flags);
        UPR_LAUNCH_CHECK();
    }
}

size_t table_tile_smem(int32_t k, int32_t nodes, int32_t sparse_buf_cap) {
    const size_t rows = sizeof(int64_t) * (size_t)((nodes + 2) & ~1) + sizeof(int) * (size_t)nodes * k;
    // hashed rows: 8 warps' staging buffers and the tile's nodes + 1 row offsets
    return sparse_buf_cap > 0 ? ((rows + 15) & ~(size_t)15) + 8 * sizeof(int2) * (size_t)sparse_buf_cap +
                                    sizeof(int64_t) * (size_t)(nodes + 1)
                              : rows;
}

// The tiles' dense row blocks are written by one bulk copy each (about 1.5 %
// faster on the R-MAT build than the threads' streaming stores);
// UPR_TILE_BULK=0 selects the stores (an A/B switch between equivalent forms)
bool bulk_rows() {
    static int env = -1;
    if (env < 0) { const char *v = getenv("UPR_TILE_BULK"); env = (v && *v == '0') ? 0 : 1; }
    return env == 1;
}

void gain_table(const GraphDev &g, const int32_t *part, int32_t *W, const HubChunk *hub_chunks, int64_t n_chunks,
                const TableTile *tiles, int64_t n_tiles, int32_t tile_nodes, const int64_t *deg_sum, cudaStream_t s) {
    if (g.n == 0) return;
    if (tiles && n_tiles > 0) {
        const size_t shm = table_tile_smem(g.k, tile_nodes, g.sp.on() ? g.sp.buf_cap : 0);
        const int local = g.ng == 1 ? 0 : g.kmask ? 1 : 2;
        auto launch = [&](auto kern) {
            // about four tiles per SM and the rest of the unified memory as L1:
            // the gathers of part[] need the L1 more than extra CTAs
            kernel_setup((const void *)kern, 64);
            const unsigned grid = deg_sum ? wave_grid((const void *)kern, 256, shm, n_tiles) : (unsigned)n_tiles;
            kern<<<grid, 256, shm, s>>>(tiles, n_tiles, g.xadj, g.adj, g.adjw, part, g.k, g.kmask, W, deg_sum, g.m,
                                        g.sp, bulk_rows());
        };
        // 16 entries in flight per thread (8 with weights); the default
        // shared/L1 split: a smaller L1 slows the gathers of part[] down
        if (g.adjw) {
            if (local == 0) launch(k_table_tiles<true, 0, 2>);
            else if (local == 1) launch(k_table_tiles<true, 1, 2>);
            else launch(k_table_tiles<true, 2, 2>);
        } else {
            if (local == 0) launch(k_table_tiles<false, 0, 4>);
            else if (local == 1) launch(k_table_tiles<false, 1, 4>);
            else launch(k_table_tiles<false, 2, 4>);
        }
        UPR_LAUNCH_CHECK();
    } else {
        throw CudaError{cudaErrorInvalidValue, "gain_table: a binding without table tiles"};
    }
    if (n_chunks > 0) {
        k_table_hub_chunks<<<(unsigned)n_chunks, 512, sizeof(int) * g.k, s>>>(hub_chunks, g.adj, g.adjw, part, g.k,
                                                                             g.kmask, W, deg_sum, g.m, g.sp);
        UPR_LAUNCH_CHECK();
    }
}

}  // namespace upr
