// Internal interface between the kernel translation units and the engine.
// Every function enqueues work on the given stream and returns at once.
#pragma once
#include "common.cuh"

namespace upr {

// The graph as the kernels see it (device pointers; adjw / vwgt may be null =
// unit weights).  wI[v] = omega(I(v)) < 2^31.
//
// Sparse form of the gain table for large k: row v holds the blocks adjacent
// to v in off[v+1] - off[v] slots (a power of two, at least min(k, 2 deg(v))
// + 1), each (local block or kEmpty, weight), open addressing with linear
// probing from a hashed home slot.  Keys are only ever inserted (a weight may
// drop to 0 and its key stays), so concurrent inserts of one block meet at
// the same first free slot; the table is rebuilt at every round start.  A row
// without a free slot for a new block sets *overflow, and the round is run
// again with the dense table.
constexpr int32_t kEmpty = -1;
constexpr int kSparseRowMax = 512;   // slots of the largest sparse row (k <= 256: 2k rounded up)
struct SparseRows {
    const int64_t *off;   // [n+1] first slot of each row
    int2 *slot;           // (local block or kEmpty, weight); null: the table is dense
    int32_t *overflow;
    int32_t buf_cap;      // largest row of a node of degree <= kHubDegree (the build's staging buffer)
    __host__ __device__ bool on() const { return slot != nullptr; }
};

// A context holds one graph or a batch of ng independent graphs packed as one
// CSR (graph g owns the nodes [noff[g], noff[g+1]) and no edge joins two
// graphs).  Blocks are numbered globally: graph g owns blocks [g*k, g*k + k),
// part[] holds global block ids, and everything indexed by block has K = ng*k
// entries.  Gain-table rows keep k columns: the column of global block p is
// p mod k (blk_local).  With one graph, global and local ids coincide.
struct GraphDev {
    int64_t n, m;
    int32_t k;            // blocks per graph
    int32_t ng;           // graphs in the context
    int32_t kmask;        // blk_local(p) = p & kmask when non-zero (-1 for one graph, k-1 for k a power of two)
    const int64_t *xadj;
    const int32_t *adj;
    const int32_t *adjw;
    const int32_t *vwgt;
    const int32_t *wI;
    const int64_t *Lb;    // [K] L_max of the graph each block belongs to
    const int32_t *gid;   // [n] graph of each node (null for one graph)
    SparseRows sp;        // sparse gain table when sp.on(), else the dense W[n][k]
    __host__ __device__ int32_t K() const { return ng * k; }
};

__device__ __forceinline__ uint32_t sp_home(int32_t b, uint32_t cap) {
    return (((uint32_t)b * 0x9E3779B1u) >> 8) & (cap - 1);
}
// omega(v, block column b)
__device__ __forceinline__ int32_t sp_get(const SparseRows &t, int64_t v, int32_t b) {
    const int64_t o = t.off[v];
    const uint32_t cap = (uint32_t)(t.off[v + 1] - o);
    uint32_t h = sp_home(b, cap);
    for (uint32_t i = 0; i < cap; i++) {
        const int2 e = t.slot[o + h];
        if (e.x == b) return e.y;
        if (e.x == kEmpty) return 0;
        h = (h + 1) & (cap - 1);
    }
    return 0;
}
// omega(v, b) += w, inserting b at the first free slot of its probe sequence
__device__ __forceinline__ void sp_add(const SparseRows &t, int64_t v, int32_t b, int32_t w) {
    const int64_t o = t.off[v];
    const uint32_t cap = (uint32_t)(t.off[v + 1] - o);
    uint32_t h = sp_home(b, cap);
    for (uint32_t i = 0; i < cap; i++) {
        int *key = &t.slot[o + h].x;
        int kk = *(volatile int *)key;
        if (kk == kEmpty) {
            kk = atomicCAS(key, kEmpty, b);
            if (kk == kEmpty) kk = b;
        }
        if (kk == b) {
            atomicAdd(&t.slot[o + h].y, w);
            return;
        }
        h = (h + 1) & (cap - 1);
    }
    atomicOr(t.overflow, 1);
}
// omega(v, b) -= w for a block b that is in the row
__device__ __forceinline__ void sp_sub(const SparseRows &t, int64_t v, int32_t b, int32_t w) {
    const int64_t o = t.off[v];
    const uint32_t cap = (uint32_t)(t.off[v + 1] - o);
    uint32_t h = sp_home(b, cap);
    for (uint32_t i = 0; i < cap; i++) {
        const int kk = *(volatile int *)&t.slot[o + h].x;
        if (kk == b) {
            atomicSub(&t.slot[o + h].y, w);
            return;
        }
        if (kk == kEmpty) break;
        h = (h + 1) & (cap - 1);
    }
    atomicOr(t.overflow, 2);      // cannot happen: the block of a neighbour is always in the row
}

__device__ __forceinline__ int32_t blk_local(int32_t p, int32_t k, int32_t kmask) {
    return kmask ? (p & kmask) : p % k;
}
__device__ __forceinline__ int32_t blk_local(const GraphDev &g, int32_t p) { return blk_local(p, g.k, g.kmask); }
// first global block of p's graph
__device__ __forceinline__ int32_t blk_base(const GraphDev &g, int32_t p) { return p - blk_local(g, p); }
__device__ __forceinline__ int32_t blk_graph(const GraphDev &g, int32_t p) { return g.ng == 1 ? 0 : p / g.k; }

__device__ __forceinline__ int64_t node_c(const GraphDev &g, int64_t v) { return g.vwgt ? (int64_t)g.vwgt[v] : 1; }
__device__ __forceinline__ int32_t edge_w(const GraphDev &g, int64_t e) { return g.adjw ? g.adjw[e] : 1; }

// An element count that may live in device memory: d (nullable) holds the
// actual count, max is a static upper bound used to size grids and buffers.
struct Count {
    const int32_t *d;
    int64_t max;
};
inline Count fixed(int64_t n) { return Count{nullptr, n}; }

// Scratch memory of the primitives: status words and partial results, tile
// and ticket counters (zero between calls: the last CTA of a call resets
// them), the call counter whose value tags status words (host memory,
// advanced at every call; calls on one scratch are serialised by their
// stream) and an error word set when a bounded wait gives up.
struct Scratch {
    char *mem;              // radix status and digit counts (radix_temp_bytes(tiles_cap * 2048))
    char *scan;             // scan / compaction status (scan_temp_bytes(tiles_cap * 2048)); never overlaps mem
    size_t mem_bytes, scan_bytes;
    int64_t tiles_cap;      // tiles of the longest list; fixes the layout of both regions
    unsigned int *ticket;   // [0] next tile, [1] finished CTAs, [2] radix count ticket
    uint32_t *epoch;        // device word: the primitives' last call tag
    int32_t *err;
};

// Grid-stride loop over a device-held count (all threads of the grid).
#define UPR_FOR(i, cnt) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (cnt); i += (int64_t)gridDim.x * blockDim.x)

// A grid of 256-thread blocks for up to `max` items, at most 8 blocks per SM.
inline unsigned grid_for(int64_t max) {
    const int64_t b = ceil_div(max > 0 ? max : 1, 256);
    return (unsigned)std::min<int64_t>(b, (int64_t)device_sm_count() * 8);
}

// ---- prim.cu
size_t scan_temp_bytes(int64_t n);
size_t radix_temp_bytes(int64_t n);
void exclusive_sum_i32(const int32_t *in, int32_t *out, Count n, Scratch tmp, cudaStream_t s);
void exclusive_sum_i64(const int64_t *in, int64_t *out, Count n, Scratch tmp, cudaStream_t s);
void inclusive_sum_i64(const int64_t *in, int64_t *out, Count n, Scratch tmp, cudaStream_t s);
void exclusive_sum_i32_to_i64(const int32_t *in, int64_t *out, Count n, Scratch tmp, cudaStream_t s);
void inclusive_max_u64(const uint64_t *in, uint64_t *out, Count n, Scratch tmp, cudaStream_t s);
void iota_u32(uint32_t *v, int64_t n, cudaStream_t s);
// Stable LSD sort on key bits [0, bits); returns true if the result is in the *_alt buffers
// (a property of `bits` alone, known when the launches are enqueued).
bool radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, Count n, int bits,
                      Scratch tmp, cudaStream_t s);
// out_idx[0..*d_count) = indices i < n with flags[i] != 0, ascending.
void select_flags(const int32_t *flags, int32_t *out_idx, int32_t *d_count, Count n, Scratch tmp, cudaStream_t s);
// out[j] = vals[i] for the j-th i with flags[i] != 0 (index order); out may be vals.
void select_values(const int32_t *flags, const int32_t *vals, int32_t *out, int32_t *d_count, Count n, Scratch tmp,
                   cudaStream_t s);

// ---- graph.cu: step (e), step (a), create-time work
struct HubChunk { int32_t v; int32_t pad; int64_t begin, end; };
// C[0..K) = block weights of part.
void block_weights(const GraphDev &g, const int32_t *part, int64_t *C, cudaStream_t s);
// cut[0..ng) = edge cut of each graph.
void edge_cut(const GraphDev &g, const int32_t *part, int64_t *cut, cudaStream_t s);
void incident_weights(const GraphDev &g, int32_t *wI, int64_t *wmax, cudaStream_t s);
// *cut = the cut of part (one graph) from the gain table W = W(part) (dense or hashed rows) and omega(I(v)).
void cut_from_table(const GraphDev &g, const int32_t *part, const int32_t *W, int64_t *cut, cudaStream_t s);
// A tile of the table build: nodes [v0, v1) and the adjacency entries [e0, e1)
// of its non-hub nodes (a hub, if any, is the tile's last node).
struct TableTile { int64_t e0, e1; int32_t v0, v1; };
// Static schedules from the packed offsets (bind.cu), over segments of
// kSchedSegment nodes.  sched_count: cnt[4 s + 0..3] = exclusive offsets of
// segment s's hub chunks, tiles, hashed-row slots and hubs; tot[0..3] = the
// totals; *cap_max = the largest hashed row of a non-hub node.  sp_mode 0:
// no hashed rows, 1: min(k, 2 deg) + 1 slots rounded up to a power of two,
// 3: min(k, deg) + 1.  sched_write fills the arrays (nullptr: not written).
constexpr int64_t kSchedSegment = 1024;
int64_t sched_segments(int64_t n);
void sched_count(const int64_t *xadj, int64_t n, int64_t m, int tile_nodes, int sp_mode, int32_t k, int64_t *cnt,
                 int64_t *tot, unsigned long long *cap_max, cudaStream_t s);
void sched_write(const int64_t *xadj, int64_t n, int64_t m, int tile_nodes, int sp_mode, int32_t k,
                 const int64_t *off, HubChunk *chunks, TableTile *tiles, int64_t *sp_off, int32_t *hubs,
                 cudaStream_t s);
// *bad = 1 unless xadj[0] = 0, xadj[n] = m and xadj is non-decreasing
void xadj_check(const int64_t *xadj, int64_t n, int64_t m, int32_t *bad, cudaStream_t s);
// A batch's packed offsets from each graph's own (graph i's n_i + 1 offsets at
// raw + noff[i] + i), shifted by the entries before it (eoff), checked as
// xadj_check checks one graph
// One segment of a gather of host arrays: len elements from src (page-locked
// host memory, read by the GPU directly) to the destination + off.
struct HostSeg {
    const void *src;
    int64_t off, len;
};
constexpr int64_t kGatherChunk = 1 << 16;
// d_segs (device memory): the segments; elem: 4 or 8 bytes per element
void gather_host(const HostSeg *d_segs, int64_t nseg, size_t elem, void *dst, cudaStream_t s);
void xadj_pack(const int64_t *raw, const int64_t *noff, const int64_t *eoff, int32_t ng, int64_t n, int64_t *out,
               int32_t *bad, cudaStream_t s);
// Shared memory of one tile of `nodes` rows (plus per-warp row buffers for the sparse table).
size_t table_tile_smem(int32_t k, int32_t nodes, int32_t sparse_buf_cap);
// W must hold n*k ints.  Rows of hubs (degree > kHubDegree) are completed by the chunk pass.
// By the binding's tiles (every binding with nodes has them).
// With deg_sum: runs only when 4 * (*deg_sum) >= m (the rebuild alternative to table_move).
void gain_table(const GraphDev &g, const int32_t *part, int32_t *W, const HubChunk *hub_chunks, int64_t n_chunks,
                const TableTile *tiles, int64_t n_tiles, int32_t tile_nodes, const int64_t *deg_sum, cudaStream_t s);
// How moved hubs are found for the chunked delta update: through m_pos (moves
// of M: from/to are M_from/M_to) or, when m_pos is null, through r_to/r_at
// (moves of the current rebalancing sub-round: R indices in [*r_base,
// *r_base + *r_count), from/to are R_from/R_to).
struct HubMoves {
    const int32_t *m_pos;
    const int32_t *r_to, *r_at, *r_base, *r_count;
    const int32_t *from, *to;
};
// For each listed node v moving from[i] -> to[i] (i < *d_count, entries start at
// *d_offset when given): W[u][from] -= w, W[u][to] += w for every neighbour u.
// With deg_sum: runs only when 4 * (*deg_sum) < m (otherwise a rebuild is cheaper).
// Hubs are handled chunk by chunk through hub_chunks and hm.
void table_move(const GraphDev &g, int32_t *W, const int32_t *nodes, const int32_t *from, const int32_t *to,
                const int32_t *d_count, const int32_t *d_offset, const int64_t *deg_sum, int64_t max_count,
                const HubChunk *hub_chunks, int64_t n_chunks, HubMoves hm, cudaStream_t s);
// Batches: gid[v] = graph of node v (noff: [ng + 1] first nodes), and each
// graph's neighbour ids (local to the graph on input) shifted by its first
// node; an id that leaves [0, n) becomes -1 for the checks to report.
void pack_batch(const GraphDev &g, const int64_t *noff, int32_t *gid, int32_t *adj, cudaStream_t s);
// W[v][b] = omega(v, V_b) from the sparse table (inspection only).
void sparse_to_dense(const GraphDev &g, int32_t *W, cudaStream_t s);
// Graph checks; writes a bitmask of violations into *d_flags (see engine.cu).
// Checks the CSR on the device (bits of *d_flags, hash sums in d_acc[0..1]):
// ranges, self loops, weights, symmetry by a multiset hash, and bit 128 for a
// row whose ids are not strictly increasing.
void validate_graph(const GraphDev &g, uint64_t *d_acc, int32_t *d_flags, cudaStream_t s);
// Exact duplicate check (bit 32 of *d_flags) for graphs with an unsorted row:
// hubs lists the n_hubs nodes of degree > kHubDegree, noff the batch's node
// offsets (ignored for one graph), max_graph_nodes the largest graph's node
// count, scratch: scratch_ints free ints.
void validate_duplicates(const GraphDev &g, int32_t *d_flags, const int32_t *hubs, int64_t n_hubs,
                         const int64_t *noff, int64_t max_graph_nodes, int32_t *scratch, int64_t scratch_ints,
                         cudaStream_t s);

// ---- select.cu: step (b) and applying M
struct Penalty {
    const int64_t *PW;    // [K][73] inclusive prefix over slots of available node weight
    const int64_t *F;     // [73] floor(tau_r * (3/2)^l * 2^Q)
    const int64_t *C;     // [K] round-start block weights
    const int64_t *Lb;    // [K] L_max of each block's graph
    const int8_t *first;  // [K] smallest slot l with PW[b][l] >= 1, -1 if none (the excess-1 case)
    // > 0 (unit node weights, one graph, gb + pack_bits <= 30): the dense
    // selection kernel scores a column as one integer, ((gain - penalty) <<
    // pack_bits) + (2^pack_bits - 1 - b), pack_bits = the bits of a column index
    int pack_bits = 0;
    int gbits = 0;
};
// With cut2 (kCutParts + 1 words; one graph): also sums twice the cut of part
// (Sec. 2: the sum over v of omega(I(v)) - omega(v, V_P(v))) into
// cut2[kCutParts] and writes the cut to *cut.
constexpr int kCutParts = 256;
void buckets(const GraphDev &g, const int32_t *part, const int32_t *W, int32_t t_num, int32_t t_den, int64_t *BW,
             int64_t *PW, int8_t *first, int8_t *avail_out, int32_t *slot_out, cudaStream_t s,
             int64_t *cut2 = nullptr, int64_t *cut = nullptr);
// Lanes per node (G) and 16-byte chunks per lane (CH) of the vectorised
// selection and proposal kernels (k % 4 == 0, k <= 256, 4*G*CH >= k).  A
// schedule only decides how the work is spread over lanes, never the
// result.  G = 0: the default (the fewest chunks per lane).
struct LaneCfg { int32_t G, CH; };
// The schedules worth timing for k (the default first); returns their number (0..3).
int lane_candidates(int32_t k, LaneCfg *out);
void select_moves(const GraphDev &g, const int32_t *part, const int32_t *W, Penalty pen, int32_t *cand_tgt,
                  int64_t *cand_s0, int32_t *cand_gain, int32_t *flags, LaneCfg cfg, cudaStream_t s);
void cand_keys(const int32_t *cand_idx, const int32_t *d_count, const int32_t *cand_tgt, const int64_t *cand_s0,
               int gbits, uint64_t *keys, uint32_t *vals, int64_t max_count, cudaStream_t s);
void cand_gather(const GraphDev &g, const int32_t *cand_idx, const uint32_t *order, const int32_t *d_count,
                 const int32_t *cand_tgt, int64_t *c_sorted, int32_t *seg_first, int64_t max_count, cudaStream_t s);
void inflow_filter(const GraphDev &g, const int32_t *cand_idx, const uint32_t *order, const int32_t *d_count,
                   const int32_t *cand_tgt, const int32_t *cand_gain, const int64_t *c_excl, const int32_t *seg_first,
                   Penalty pen, int32_t *keep_flag, int64_t *score, int64_t max_count, cudaStream_t s);
void move_keys(const int32_t *m_idx, const int32_t *d_count, const int64_t *score, int gbits, uint64_t *keys,
               uint32_t *vals, int64_t max_count, cudaStream_t s);
void apply_moves(const GraphDev &g, const int32_t *cand_idx, const int32_t *m_idx, const uint32_t *order,
                 const int32_t *d_count, const int32_t *cand_tgt, const int64_t *score, const int32_t *part0,
                 int32_t *part, int64_t *C, int32_t *M_node, int32_t *M_from, int32_t *M_to, int64_t *M_score,
                 int32_t *m_pos, int64_t *deg_sum, int64_t max_count, cudaStream_t s);

// ---- rebalance.cu: step (d)
// Device-resident control block of the rebalancing loop.
struct RebalCtl {
    int32_t active;      // the current sub-round runs
    int32_t stopped;     // the loop has finished
    int32_t light;       // one graph: lightest block that may receive moves, or -1
    int32_t subrounds;   // sub-rounds that ran
    int32_t nR;          // rebalancing moves so far (length of R)
    int32_t n1_active;   // length of the node list if this sub-round runs, else 0
    int32_t flag;        // batch controllers: "some block is overloaded" / "the excluded set grew"
    uint32_t ticket;     // batch controllers: CTAs finished (the last one updates the control block)
};
struct RebalState {
    const int64_t *C;     // [K] current block weights
    const int8_t *over;   // [K] overloaded now
    const int8_t *excl;   // [K] not a target: overloaded at the first sub-round, or rejected a move
    const int32_t *light; // [ng] lightest non-excluded block of each graph, or -1
    const int64_t *Lb;    // [K] L_max of each block's graph
    // optional (null: not written): per listed node i with a proposal, its
    // block and gain by list index, so that later passes over the list read
    // them in order instead of gathering them by node
    int32_t *lsrc = nullptr, *lgain = nullptr;
    // > 0 (unit node weights, one graph, 1 + gb + pack_bits <= 32): the dense
    // proposal kernel scores a column as one integer, (omega << pack_bits) +
    // (2^pack_bits - 1 - b), pack_bits = the bits of a column index
    int pack_bits = 0;
};
// flags[v] = 1 for the nodes of the marked blocks
void rebalance_flag_in_blocks(const int32_t *part, int64_t n, const int8_t *mark, int32_t *flags, cudaStream_t s);
// Proposals of the listed nodes in overloaded blocks: prop_tgt/prop_gain by node, flags by list position.
void rebalance_propose_scalar_list(const GraphDev &g, const int32_t *list, const int32_t *d_n1, int64_t n1_max,
                                   const int32_t *part, const int32_t *W, RebalState st, int32_t *prop_tgt,
                                   int32_t *prop_gain, int32_t *flags, cudaStream_t s);
void rebalance_propose_list(const GraphDev &g, const int32_t *list, const int32_t *d_n1, int64_t n1_max,
                            const int32_t *part, const int32_t *W, RebalState st, int32_t *prop_tgt,
                            int32_t *prop_gain, int32_t *flags, LaneCfg cfg, cudaStream_t s);
// Proposal prefilter (exact): a source's proposals in the priority bins after
// the one where its cumulative weight reaches the excess can never be in its
// minimal prefix.  keep[i] = 1 for listed node i (list/d_n1; flags from the
// proposal kernel, or null when every listed node proposes) when it proposes
// and is not in such a bin.  hist (K * kPrioBins, zero on entry) is left zero.
constexpr int kPrioBins = 256;
void rebalance_prefilter(const GraphDev &g, const int32_t *list, const int32_t *d_n1, int64_t n1_max,
                         const int32_t *flags, const int32_t *prop_gain, const int32_t *part, const int8_t *over,
                         const int64_t *C, int gbits, int cbits, int gain_only, unsigned long long *hist,
                         int32_t *cut, int32_t *keep, cudaStream_t s);
// The four buffers of a two-array radix sort (keys and values, and their alternates).
struct SortPairs { uint64_t *k, *ka; uint32_t *v, *va; };
// A priority key wider than 63 bits (1 + gbits + 2 cbits > 63): the proposals
// P[0..*d_np) ordered by their 128-bit keys, two stable sorts (low word, then
// high word); *order receives the buffer holding the order (indices into P).
void rebalance_prio_sort_wide(const GraphDev &g, const int32_t *P, const int32_t *d_np, const int32_t *prop_gain,
                              int gbits, int cbits, int gain_only, SortPairs sp, int64_t np_max, Scratch tmp,
                              cudaStream_t s, uint32_t **order);
// ---- mixed.cu: one context over batches of different k (one batch per k)
struct MixedBatch;
upr_status mixed_create(const upr_graph *graphs, int32_t n_graphs, const int32_t *k, const double *eps,
                        const upr_params *params, MixedBatch **out);
upr_status mixed_rebind(MixedBatch *mb, const upr_graph *graphs, int32_t n_graphs, const int32_t *k,
                        const double *eps);
void mixed_destroy(MixedBatch *mb);
// engine.cu: a context bound to other graphs (its arena reused when large enough)
upr_status ctx_rebind(upr_ctx *c, const upr_graph *g, int32_t k, double eps, const upr_params *params);
upr_status ctx_rebind_batch(upr_ctx *c, const upr_graph *gs, int32_t ng, int32_t k, const double *eps,
                            const upr_params *params);
int64_t mixed_nodes(const MixedBatch *mb);
upr_status mixed_refine(MixedBatch *mb, int32_t *part, int32_t rounds, uint64_t seed, upr_status *status,
                        int64_t *cut_in, int64_t *cut_out, upr_stats *stats);
upr_status mixed_cut(MixedBatch *mb, const int32_t *part, int64_t *cut, int64_t *block_weights);
upr_status mixed_info(const MixedBatch *mb, int32_t *n_graphs, int64_t *node_offsets, int64_t *lmax);

// ---- reb_fused.cu: one rebalancing sub-round in fused passes (one graph,
// K <= 256, a key of at most 63 bits, the prefilter on); same results as the
// general form.  K * ceil(n / 2048) must not exceed the histogram buffers.
bool rebalance_fused_ok(const GraphDev &g, int key_bits, bool prefilter);
// list[0..*d_out) = the listed nodes with flags set (in place, in order), and
// the prefilter's (source, bin) weights added to hist
// (rep: [kPrioBins] one key per bin; *exact set to 1 for k_fr_keep_keys to clear)
// (lgain, lsrc: the proposals' gains and blocks by list index, compacted with the list)
void rebalance_fused_compact_hist(const GraphDev &g, const int32_t *flags, int32_t *list, const int32_t *d_n,
                                  int64_t n_max, int32_t *d_out, int32_t *lgain, int32_t *lsrc, int gbits, int cbits,
                                  int gain_only, unsigned long long *hist, uint64_t *rep, int32_t *exact, Scratch tmp,
                                  cudaStream_t s);
// (keys, vals)[0..*d_out) = (priority key, node) of the proposals whose bin is
// not after their source's cut; *exact cleared when a kept key differs from its bin's rep
void rebalance_fused_keep_keys(const GraphDev &g, const int32_t *list, const int32_t *d_n, int64_t n_max,
                               const int32_t *lgain, const int32_t *lsrc, const int32_t *cut, int gbits, int cbits,
                               int gain_only, uint64_t *keys, uint32_t *vals, int32_t *d_out, const uint64_t *rep,
                               int32_t *exact, Scratch tmp, cudaStream_t s);
// Steps 1 and 3-7 of the fused sub-round (compaction with the prefilter
// histogram, cut bins, kept keys, the sort, selection, admission and the
// moves) in one cooperative launch with grid barriers: the same results as
// the separate fused kernels.  The wrapper sets the fields after `exact`.
struct RebalMega {
    const int32_t *flags;                    // [n1] proposer flags by list index
    int32_t *list, *lsrc, *lgain;            // [n1] the list (becomes the proposers), their blocks and gains
    const int32_t *d_n1;                     // n1
    int32_t *list2, *lsrc2, *lgain2;         // [n] the compacted proposers, their blocks and gains
    int gbits, cbits, gain_only;
    unsigned long long *hist;                // [K * kPrioBins] prefilter weights (rows of overloaded sources cleared)
    uint64_t *rep;                           // [kPrioBins] some proposal's key per bin
    int32_t *cut;                            // [K] cut bin per source
    const int8_t *over;
    const int64_t *C;
    uint64_t *keys, *keys_alt;               // [n] kept keys; the sorted keys
    uint32_t *vals, *vals_alt;               // [n] kept nodes; the sorted nodes
    int32_t *part;
    const int32_t *prop_tgt;
    int8_t *sel;                             // [n] per sorted proposal: 1 selected, 2 admitted
    long long *h0, *h1;                      // [K * tiles] per-(block, tile) weights and their row prefixes
    int8_t *reject;
    const RebalCtl *ctl;
    int32_t *R_node, *R_from, *R_to, *R_sub, *r_to, *r_at;
    long long *Cd;
    int32_t *d_np, *d_nk, *d_na;             // proposers, kept, admitted
    int32_t *exact;
    // set by rebalance_fused_mega
    const int32_t *vwgt = nullptr;
    const int64_t *Lb = nullptr;
    int K = 0, passes = 0, vec = 0;
    int32_t *tab = nullptr;                  // tile counts 3 x [tcap], digit totals [256], digit counts [256 * tcap]
    int64_t tcap = 0;
    unsigned long long *bar = nullptr;       // the grid barrier's arrival counter
    int32_t *err = nullptr;
};
void rebalance_fused_mega(const GraphDev &g, RebalMega m, int key_bits, int64_t n_max, Scratch tmp, cudaStream_t s);
// Stable sort of (keys, vals)[0..*d_n) by key (key_bits, an odd number of
// 8-bit passes), or by the key's prefilter bin alone when *exact; the result
// is in the alternate buffers (returns true).  While s is being captured and
// s_aux and later_runs are given, the passes after the first are captured on
// s_aux as the body of a conditional node that runs only when they sort
// anything; each run adds 1 to *later_runs, and *later_kernels = the body's
// kernels (0 when no such node was made).
bool rebalance_fused_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, const int32_t *d_n,
                          int64_t n_max, int key_bits, int gbits, int cbits, const int32_t *exact, Scratch tmp,
                          cudaStream_t s, cudaStream_t s_aux = nullptr, int32_t *later_runs = nullptr,
                          int *later_kernels = nullptr);
// U[0..*d_np): proposals (nodes) in priority order.  Minimal prefix per
// source, longest fitting prefix per target, the admitted appended to R at
// ctl->nR (count *d_na), part / r_to / r_at updated, block-weight changes
// added to Cd; sel (np int8) and the two histograms (K * ceil(np / 2048)
// int64 each) are scratch.
void rebalance_fused_select_admit(const GraphDev &g, const uint32_t *U, const int32_t *d_np, int64_t np_max,
                                  int32_t *part, const int32_t *prop_tgt, const int64_t *C, int8_t *sel,
                                  long long *h0, long long *h1, int32_t *d_hist_n, int8_t *reject,
                                  const RebalCtl *ctl, int32_t *R_node, int32_t *R_from, int32_t *R_to,
                                  int32_t *R_sub, int32_t *r_to, int32_t *r_at, long long *Cd, int32_t *d_na,
                                  Scratch tmp, cudaStream_t s);
// C += Cd, Cd = 0; then k_reb_end's update of the excluded set and the stop
// flag; with cond (a graph-resident loop) also the loop's condition, as
// rebalance_continue sets it.  With begin_next (over, reject and d_n1
// given) the next sub-round's begin follows in the same kernel (as
// rebalance_begin) and the condition is "that sub-round runs".
void rebalance_fused_end(const GraphDev &g, int64_t *C, long long *Cd, int8_t *excl, const int8_t *reject,
                         const int32_t *d_na, RebalCtl *ctl, cudaStream_t s, cudaGraphConditionalHandle cond = 0,
                         int32_t max_subrounds = 0, int8_t *over = nullptr, int8_t *reject_next = nullptr,
                         const int32_t *d_n1 = nullptr);
// The prefilter's cut bin of every overloaded source (hist rows read are cleared).
void rebalance_prio_cut(const GraphDev &g, const int8_t *over, const int64_t *C, unsigned long long *hist, int32_t *cut,
                        cudaStream_t s);
// gain_only: the priority is the gain alone (a variant of Sec. 7.2), else g/c
// for g < 0 and g*c for g >= 0 (Sec. 6.1)
void rebalance_prio_keys(const GraphDev &g, const int32_t *P, const int32_t *d_np, const int32_t *prop_gain,
                         int gbits, int cbits, int gain_only, uint64_t *keys, uint32_t *vals, int64_t np_max,
                         cudaStream_t s);
void rebalance_block_keys(const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *d_cnt,
                          const int32_t *blk_of_node, uint64_t *keys, uint32_t *vals, int64_t cnt_max, cudaStream_t s);
void rebalance_seg_weights(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S,
                           const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, int64_t *c_sorted,
                           int32_t *seg_first, int64_t cnt_max, cudaStream_t s);
void rebalance_mark_selected(const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_excl,
                             const int32_t *seg_first, RebalState st, int32_t *sel, int64_t cnt_max, cudaStream_t s);
void rebalance_mark_admitted(const uint32_t *T, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_sorted,
                             const int64_t *c_excl, const int32_t *seg_first, RebalState st, int32_t *adm,
                             int8_t *reject, int64_t cnt_max, cudaStream_t s);
void rebalance_apply(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *Adm,
                     const int32_t *d_na, const int32_t *prop_tgt, int32_t *part, int64_t *C, const RebalCtl *ctl,
                     int32_t *R_node, int32_t *R_from, int32_t *R_to, int32_t *R_sub, int32_t *r_to, int32_t *r_at,
                     int64_t na_max, cudaStream_t s);
// Loop control over the K blocks of g (C = current block weights).  light
// receives each graph's lightest non-excluded block (&ctl->light for one graph).
void rebalance_init(const GraphDev &g, const int64_t *C, int8_t *excl, RebalCtl *ctl, cudaStream_t s);
// cond (one graph, a graph-resident loop whose body does not begin with this
// kernel): also sets the loop's condition to "this sub-round runs"
void rebalance_begin(const GraphDev &g, const int64_t *C, const int8_t *excl, int8_t *over, int8_t *reject,
                     const int32_t *d_n1, int32_t max_subrounds, RebalCtl *ctl, int32_t *light, cudaStream_t s,
                     cudaGraphConditionalHandle cond = 0);
// Sets the condition of a graph's while node: another sub-round is due.
void rebalance_continue(const RebalCtl *ctl, int32_t max_subrounds, cudaGraphConditionalHandle handle,
                        cudaStream_t s);
void rebalance_end(const GraphDev &g, const int64_t *C, int8_t *excl, const int8_t *reject, const int32_t *d_na,
                   RebalCtl *ctl, cudaStream_t s);

// ---- sequence.cu: step (c); every count lives in device memory, `max` bounds it
void count_affine(const int32_t *a, int32_t a_mul, const int32_t *b, int32_t add, int32_t *out, cudaStream_t s);
void fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t s);
void clear_count(int32_t *a, const int32_t *d_n, int32_t extra, int64_t max, cudaStream_t s);
void reset_nodes(const int32_t *nodes, const int32_t *d_cnt, int64_t max, int32_t *arr, int32_t val, cudaStream_t s);
// out[g] = number of blocks of graph g above L_max
void count_over(const GraphDev &g, const int64_t *C, int32_t *out, cudaStream_t s);
void seq_rb_keys(const int32_t *R_from, const int32_t *d_nR, int64_t max, uint64_t *keys, uint32_t *vals,
                 cudaStream_t s);
void seq_rb_bounds(const int32_t *R_node, const int32_t *R_from, const uint32_t *RB, const int32_t *d_nR, int64_t max,
                   const int32_t *vwgt, int64_t *rc, int32_t *rbeg, int32_t *rend, cudaStream_t s);
void seq_ev_keys(const int32_t *M_from, const int32_t *M_to, const int32_t *d_nM, int64_t max, uint64_t *keys,
                 uint32_t *vals, cudaStream_t s);
void seq_ev_delta(const int32_t *M_node, const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nM, int64_t max,
                  const int32_t *vwgt, int64_t *delta, int32_t *ebeg, int32_t *eend, cudaStream_t s);
void seq_ev_need(const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nM, int64_t max, const int64_t *delta,
                 const int64_t *d_excl, const int32_t *ebeg, const int64_t *C0, const int64_t *Lb,
                 const int32_t *rbeg, const int32_t *rend, const int64_t *rc_excl, const int64_t *rc, uint64_t *packed,
                 cudaStream_t s);
void seq_ev_emit(const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nM, int64_t max, const uint64_t *qmax,
                 const int32_t *ebeg, int32_t *emit, int32_t *qbefore_m, cudaStream_t s);
void seq_block_final(int32_t K, const int32_t *ebeg, const int32_t *eend, const uint64_t *qmax, const int32_t *rbeg,
                     const int32_t *rend, int32_t *qfin, int32_t *left, cudaStream_t s);
void seq_place_m(const int32_t *M_node, const int32_t *M_from, const int32_t *M_to, const int32_t *d_nM, int64_t max,
                 const int32_t *em_excl, int32_t *pos_m, int32_t *X_node, int32_t *X_from, int32_t *X_to,
                 int8_t *X_isr, cudaStream_t s);
// X = M followed by R (the appended sequence, a variant of Sec. 7.2); max
// bounds |M| + |R|
void seq_append(const int32_t *M_node, const int32_t *M_from, const int32_t *M_to, const int32_t *d_nM,
                const int32_t *R_node, const int32_t *R_from, const int32_t *R_to, const int32_t *d_nR, int64_t max,
                int32_t *X_node, int32_t *X_from, int32_t *X_to, int8_t *X_isr, cudaStream_t s);
void seq_place_r(const int32_t *R_node, const int32_t *R_from, const int32_t *R_to, const uint32_t *RB,
                 const int32_t *d_nR, int64_t max, const int32_t *rbeg, const uint32_t *EV, const int32_t *ebeg,
                 const int32_t *eend, const uint64_t *qmax, const int32_t *pos_m, const int32_t *qfin,
                 const int32_t *left_excl, const int32_t *em_excl, const int32_t *emit, const int32_t *d_nM,
                 int32_t *X_node, int32_t *X_from, int32_t *X_to, int8_t *X_isr, cudaStream_t s);
void seq_merge_flags(const int32_t *X_node, const int32_t *X_to, const int8_t *X_isr, const int32_t *d_nX, int64_t max,
                     const int32_t *m_pos, const int32_t *r_to, const int32_t *part0, int32_t *keep, int32_t *final_to,
                     cudaStream_t s);
void seq_build_I(const int32_t *Ix, const int32_t *d_nI, int64_t max, const int32_t *X_node, const int32_t *final_to,
                 const int32_t *part0, int32_t *I_node, int32_t *I_from, int32_t *I_to, int32_t *pos, int32_t *dest,
                 cudaStream_t s);
// pk: n words of scratch (each node's position in I and blocks before/after)
void seq_gains(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
               const int32_t *d_nI, int64_t max, const int32_t *part0, int2 *pk, int64_t *gain,
               const HubChunk *hub_chunks, int64_t n_chunks, int64_t *deg_sum, cudaStream_t s);
void seq_iev_keys(const int32_t *I_from, const int32_t *I_to, const int32_t *d_nI, int64_t max, uint64_t *keys,
                  uint32_t *vals, cudaStream_t s);
void seq_iev_delta(const int32_t *I_node, const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nI, int64_t max,
                   const int32_t *vwgt, int64_t *delta, int32_t *ebeg, cudaStream_t s);
void seq_iev_transitions(const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nI, int64_t max,
                         const int64_t *delta, const int64_t *d_excl, const int32_t *ebeg, const int64_t *C0,
                         const int64_t *Lb, int32_t *diff, cudaStream_t s);
void seq_best(const int64_t *Gsum, const int32_t *diff, const int32_t *diff_excl, const int32_t *d_nI, int64_t max,
              const int32_t *d_over0, long long *parts, long long *out, int32_t *infeasible, cudaStream_t s);
void seq_apply_prefix(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
                      int64_t max, const long long *best, int32_t *part0, int64_t *C0, int64_t *cut, cudaStream_t s);
// The moves of I undone after the best prefix: positions i >= j* (one graph,
// best[1] = j*, -1 = none kept) or i - seg_beg[g] >= best_j[g] (a batch, gid set).
struct Rollback {
    const int32_t *I_node, *I_from, *I_to;
    const int32_t *d_nI;
    const long long *best;
    const int32_t *gid, *seg_beg;
    const long long *best_j;
};
// The oscillation guard of Sec. 2: locked[v] = 1 exactly for the nodes of the
// applied prefix of I whose move came from rebalancing alone (m_pos < 0,
// r_to >= 0); and no candidate among the locked nodes.
void guard_locks(const struct Rollback &rb, int64_t max, int64_t n, const int32_t *m_pos, const int32_t *r_to,
                 int8_t *locked, cudaStream_t s);
void guard_filter(const int8_t *locked, int64_t n, int32_t *flags, int32_t *cand_tgt, int64_t *cand_s0,
                  int32_t *cand_gain, cudaStream_t s);
// W(P o I) -> W(P o I^{j*}): delta updates of the undone moves (pos = positions
// in I), or nothing when 4 * (their degree sum, left in *deg_sum) >= m, in which
// case the caller rebuilds with gain_table(..., deg_sum).
void table_rollback(const GraphDev &g, const Rollback &rb, int64_t max, const int32_t *pos, int32_t *W,
                    const HubChunk *hub_chunks, int64_t n_chunks, int64_t *deg_sum, cudaStream_t s);
// Batches: I (length *d_nI) stably sorted by graph into O_*; pos/dest of the
// moved nodes set from the sorted order; seg_beg/seg_end[g] bound graph g's
// moves (both 0 for a graph without moves).
void seq_sort_by_graph(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
                       const int32_t *d_nI, int64_t max, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                       uint32_t *vals_alt, Scratch tmp, int32_t *O_node, int32_t *O_from, int32_t *O_to, int32_t *pos,
                       int32_t *dest, int32_t *seg_beg, int32_t *seg_end, cudaStream_t s);
// Per graph: the best eligible prefix j* (ties: shortest; none: infeasible,
// j* = 0), cut[g] -= G_g(j*); tot = (sum j*, sum G(j*), infeasible graphs).
void seq_best_seg(const GraphDev &g, const int32_t *I_node, const int32_t *d_nI, int64_t max, const int32_t *seg_beg,
                  const int64_t *Gsum, const int32_t *diff, const int32_t *diff_excl, const int32_t *over0,
                  long long *best_g, long long *best_j, int64_t *cut, int32_t *infeasible, int64_t *tot,
                  cudaStream_t s);
void seq_apply_prefix_seg(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
                          const int32_t *d_nI, int64_t max, const int32_t *seg_beg, const long long *best_j,
                          int32_t *part0, int64_t *C0, cudaStream_t s);

// ---- lp.cu: unconstrained label propagation (Sec. 5)
// active[v] = 1 for the boundary nodes of part (table W of part)
void lp_boundary(const GraphDev &g, const int32_t *part, const int32_t *W, int8_t *active, cudaStream_t s);
// flags[v] = 0 where active[v] = 0
void lp_filter(int32_t *flags, const int8_t *active, int64_t n, cudaStream_t s);
// the listed movers (d_cnt of them, node order) to cand_tgt: part (a copy of
// part0), C, the move list, m_pos markers and the movers' degree sum
void lp_apply(const GraphDev &g, const int32_t *movers, const int32_t *d_cnt, const int32_t *cand_tgt,
              const int32_t *cand_gain, const int32_t *part0, int32_t *part, int64_t *C, int32_t *M_node,
              int32_t *M_from, int32_t *M_to, int64_t *M_score, int32_t *m_pos, int64_t *deg_sum, int64_t max_count,
              cudaStream_t s);
// next[u] = 1 for the unmoved neighbours u of the nodes whose block changed
// from before to after, every such node being in nodes1[0..*d_cnt1) or
// nodes2[0..*d_cnt2) (the hubs' rows by their chunks); *d_count = their number
void lp_next(const GraphDev &g, const int32_t *before, const int32_t *after, const int32_t *nodes1,
             const int32_t *d_cnt1, const int32_t *nodes2, const int32_t *d_cnt2, const HubChunk *hub_chunks,
             int64_t n_chunks, int8_t *next, int32_t *d_count, cudaStream_t s);
// *d_count = the number of non-zero entries of active
void lp_count(const int8_t *active, int64_t n, int32_t *d_count, cudaStream_t s);

}  // namespace upr
