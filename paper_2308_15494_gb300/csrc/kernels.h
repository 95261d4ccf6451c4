// Internal interface between the kernel translation units and the engine.
// Every function enqueues work on the given stream and returns at once.
#pragma once
#include "common.cuh"

namespace upr {

// The graph as the kernels see it (device pointers; adjw / vwgt may be null =
// unit weights).  wI[v] = omega(I(v)) < 2^31.
struct GraphDev {
    int64_t n, m;
    int32_t k;
    const int64_t *xadj;
    const int32_t *adj;
    const int32_t *adjw;
    const int32_t *vwgt;
    const int32_t *wI;
};

__device__ __forceinline__ int64_t node_c(const GraphDev &g, int64_t v) { return g.vwgt ? (int64_t)g.vwgt[v] : 1; }
__device__ __forceinline__ int32_t edge_w(const GraphDev &g, int64_t e) { return g.adjw ? g.adjw[e] : 1; }

// ---- prim.cu
size_t scan_temp_bytes(int64_t n);
size_t radix_temp_bytes(int64_t n);
void exclusive_sum_i32(const int32_t *in, int32_t *out, int64_t n, void *tmp, cudaStream_t s);
void exclusive_sum_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
void inclusive_sum_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
void exclusive_sum_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
void inclusive_max_u64(const uint64_t *in, uint64_t *out, int64_t n, void *tmp, cudaStream_t s);
void iota_u32(uint32_t *v, int64_t n, cudaStream_t s);
// Stable LSD sort on key bits [0, bits); returns true if the result is in the *_alt buffers.
bool radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int64_t n, int bits,
                      void *tmp, cudaStream_t s);
// out_idx[0..*d_count) = indices i with flags[i] != 0, ascending.  excl: n scratch ints.
void select_flags(const int32_t *flags, int32_t *excl, int32_t *out_idx, int32_t *d_count, int64_t n, void *tmp,
                  cudaStream_t s);

// ---- graph.cu: step (e), step (a), create-time work
struct HubChunk { int32_t v; int32_t pad; int64_t begin, end; };
void block_weights(const GraphDev &g, const int32_t *part, int64_t *C, cudaStream_t s);
void edge_cut(const GraphDev &g, const int32_t *part, int64_t *cut, cudaStream_t s);
void incident_weights(const GraphDev &g, int32_t *wI, int64_t *wmax, cudaStream_t s);
// W must hold n*k ints.  Rows of hubs (degree > kHubDegree) are completed by the chunk pass.
void gain_table(const GraphDev &g, const int32_t *part, int32_t *W, const HubChunk *hub_chunks, int64_t n_chunks,
                cudaStream_t s);
// For each listed node v moving from[i] -> to[i]: W[u][from] -= w, W[u][to] += w for every neighbour u.
void table_move(const GraphDev &g, int32_t *W, const int32_t *nodes, const int32_t *from, const int32_t *to,
                const int32_t *d_count, int64_t max_count, cudaStream_t s);
// Graph checks; writes a bitmask of violations into *d_flags (see engine.cu).
void validate_graph(const GraphDev &g, uint64_t *d_acc, int32_t *d_flags, cudaStream_t s);

// ---- select.cu: step (b) and applying M
struct Penalty {
    const int64_t *PW;    // [k][73] inclusive prefix over slots of available node weight
    const int64_t *F;     // [73] floor(tau_r * (3/2)^l * 2^Q)
    const int64_t *C;     // [k] round-start block weights
    int64_t Lmax;
};
void buckets(const GraphDev &g, const int32_t *part, const int32_t *W, int32_t t_num, int32_t t_den, int64_t *BW,
             int64_t *PW, int8_t *avail_out, int32_t *slot_out, cudaStream_t s);
void select_moves(const GraphDev &g, const int32_t *part, const int32_t *W, Penalty pen, int32_t *cand_tgt,
                  int64_t *cand_s0, int32_t *cand_gain, int32_t *flags, cudaStream_t s);
void cand_keys(const int32_t *cand_idx, const int32_t *d_count, const int32_t *cand_tgt, const int64_t *cand_s0,
               uint64_t *keys, uint32_t *vals, int64_t max_count, cudaStream_t s);
void cand_gather(const GraphDev &g, const int32_t *cand_idx, const uint32_t *order, const int32_t *d_count,
                 const int32_t *cand_tgt, int64_t *c_sorted, int32_t *seg_first, int64_t max_count, cudaStream_t s);
void inflow_filter(const GraphDev &g, const int32_t *cand_idx, const uint32_t *order, const int32_t *d_count,
                   const int32_t *cand_tgt, const int32_t *cand_gain, const int64_t *c_excl, const int32_t *seg_first,
                   Penalty pen, int32_t *keep_flag, int64_t *score, int64_t max_count, cudaStream_t s);
void move_keys(const int32_t *m_idx, const int32_t *d_count, const int64_t *score, uint64_t *keys, uint32_t *vals,
               int64_t max_count, cudaStream_t s);
void apply_moves(const GraphDev &g, const int32_t *cand_idx, const int32_t *m_idx, const uint32_t *order,
                 const int32_t *d_count, const int32_t *cand_tgt, const int64_t *score, const int32_t *part0,
                 int32_t *part, int64_t *C, int32_t *M_node, int32_t *M_from, int32_t *M_to, int64_t *M_score,
                 int32_t *m_pos, int64_t max_count, cudaStream_t s);

// ---- rebalance.cu: step (d)
struct RebalState {
    const int64_t *C;     // current block weights
    const int8_t *over;   // [k] overloaded now
    const int8_t *excl;   // [k] not a target: overloaded at the first sub-round, or rejected a move
    int32_t light;        // lightest non-excluded block, or -1
    int64_t Lmax;
};
void rebalance_propose(const GraphDev &g, const int32_t *part, const int32_t *W, RebalState st, int32_t *prop_tgt,
                       int32_t *prop_gain, int32_t *flags, cudaStream_t s);
void rebalance_prio_keys(const GraphDev &g, const int32_t *P, const int32_t *d_np, const int32_t *prop_gain,
                         int gbits, int cbits, uint64_t *keys, uint32_t *vals, int64_t np, cudaStream_t s);
void rebalance_block_keys(const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *d_cnt,
                          const int32_t *blk_of_node, uint64_t *keys, uint32_t *vals, int64_t cnt, cudaStream_t s);
void rebalance_seg_weights(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S,
                           const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, int64_t *c_sorted,
                           int32_t *seg_first, int64_t cnt, cudaStream_t s);
void rebalance_mark_selected(const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_excl,
                             const int32_t *seg_first, RebalState st, int32_t *sel, int64_t cnt, cudaStream_t s);
void rebalance_mark_admitted(const uint32_t *T, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_sorted,
                             const int64_t *c_excl, const int32_t *seg_first, RebalState st, int32_t *adm,
                             int8_t *reject, int64_t cnt, cudaStream_t s);
void rebalance_apply(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *Adm,
                     const int32_t *d_na, const int32_t *prop_tgt, int32_t *part, int64_t *C, int32_t subround,
                     int32_t *R_node, int32_t *R_from, int32_t *R_to, int32_t *R_sub, int32_t *r_to, int64_t na,
                     cudaStream_t s);

// ---- sequence.cu: step (c)
void fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t s);
void reset_nodes(const int32_t *nodes, int64_t cnt, int32_t *arr, int32_t val, cudaStream_t s);
void seq_rb_keys(const int32_t *R_from, int64_t nR, uint64_t *keys, uint32_t *vals, cudaStream_t s);
void seq_rb_bounds(const int32_t *R_node, const int32_t *R_from, const uint32_t *RB, int64_t nR, const int32_t *vwgt,
                   int64_t *rc, int32_t *rbeg, int32_t *rend, cudaStream_t s);
void seq_ev_keys(const int32_t *M_from, const int32_t *M_to, int64_t nM, uint64_t *keys, uint32_t *vals,
                 cudaStream_t s);
void seq_ev_delta(const int32_t *M_node, const uint32_t *EV, const uint64_t *ekeys, int64_t nev, const int32_t *vwgt,
                  int64_t *delta, int32_t *ebeg, int32_t *eend, cudaStream_t s);
void seq_ev_need(const uint32_t *EV, const uint64_t *ekeys, int64_t nev, const int64_t *delta, const int64_t *d_excl,
                 const int32_t *ebeg, const int64_t *C0, int64_t Lmax, const int32_t *rbeg, const int32_t *rend,
                 const int64_t *rc_excl, const int64_t *rc, uint64_t *packed, cudaStream_t s);
void seq_ev_emit(const uint32_t *EV, const uint64_t *ekeys, int64_t nev, const uint64_t *qmax, const int32_t *ebeg,
                 int32_t *emit, int32_t *qbefore_m, cudaStream_t s);
void seq_block_final(int32_t k, const int32_t *ebeg, const int32_t *eend, const uint64_t *qmax, const int32_t *rbeg,
                     const int32_t *rend, int32_t *qfin, int32_t *left, cudaStream_t s);
void seq_place_m(const int32_t *M_node, const int32_t *M_from, const int32_t *M_to, int64_t nM, const int32_t *em_excl,
                 int32_t *pos_m, int32_t *X_node, int32_t *X_from, int32_t *X_to, int8_t *X_isr, cudaStream_t s);
void seq_place_r(const int32_t *R_node, const int32_t *R_from, const int32_t *R_to, const uint32_t *RB, int64_t nR,
                 const int32_t *rbeg, const uint32_t *EV, const int32_t *ebeg, const int32_t *eend,
                 const uint64_t *qmax, const int32_t *pos_m, const int32_t *qfin, const int32_t *left_excl,
                 const int32_t *em_excl, const int32_t *emit, int64_t nM, int32_t *X_node, int32_t *X_from,
                 int32_t *X_to, int8_t *X_isr, cudaStream_t s);
void seq_merge_flags(const int32_t *X_node, const int32_t *X_to, const int8_t *X_isr, int64_t nX, const int32_t *m_pos,
                     const int32_t *r_to, const int32_t *part0, int32_t *keep, int32_t *final_to, cudaStream_t s);
void seq_build_I(const int32_t *Ix, const int32_t *d_nI, int64_t nI_max, const int32_t *X_node, const int32_t *final_to,
                 const int32_t *part0, int32_t *I_node, int32_t *I_from, int32_t *I_to, int32_t *pos, int32_t *dest,
                 cudaStream_t s);
void seq_gains(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to, int64_t nI,
               const int32_t *pos, const int32_t *dest, const int32_t *part0, int64_t *gain, int32_t *hub_flag,
               int32_t *hub_excl, int32_t *hubs, int32_t *d_nh, void *tmp, cudaStream_t s);
void seq_iev_keys(const int32_t *I_from, const int32_t *I_to, int64_t nI, uint64_t *keys, uint32_t *vals,
                  cudaStream_t s);
void seq_iev_delta(const int32_t *I_node, const uint32_t *EV, const uint64_t *ekeys, int64_t nev, const int32_t *vwgt,
                   int64_t *delta, int32_t *ebeg, cudaStream_t s);
void seq_iev_transitions(const uint32_t *EV, const uint64_t *ekeys, int64_t nev, const int64_t *delta,
                         const int64_t *d_excl, const int32_t *ebeg, const int64_t *C0, int64_t Lmax, int32_t *diff,
                         cudaStream_t s);
void seq_best(const int64_t *Gsum, const int32_t *diff, const int32_t *diff_excl, int64_t nI, int32_t over0,
              long long *parts, long long *out, cudaStream_t s);
void seq_apply_prefix(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to, int64_t nI,
                      const long long *best, int32_t *part0, int64_t *C0, int64_t *cut, cudaStream_t s);

}  // namespace upr
