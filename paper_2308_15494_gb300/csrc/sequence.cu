// Step (c): the interleaved move sequence I of M and R_1..R_k (Sec. 4.4),
// merging of a node's two moves (Sec. 4.4 footnote), exact gains of I, the
// balanced prefixes and the best one (Alg. 1, Sec. 4.1).
//
// Interleaving in parallel.  Walking M, after each move into block b the
// sequential rule emits the shortest further prefix of R_b that brings b to
// L_max.  Blocks with R_b non-empty were overloaded when rebalancing started
// and never receive rebalancing moves, so b's weight at that point is
// D_b(i) - (weight of R_b already emitted), with D_b(i) the weight of b after
// M's first i moves.  Hence the emitted count after M move i is
// min(|R_b|, max over inflow events i' <= i of need_b(i')), need_b = the
// shortest prefix of R_b whose weight covers D_b - L_max.  Every move of M
// becomes two block events (-c at its source, +c at its target); events are
// sorted by block (stable, so M order within a block), D_b is a segmented
// sum and the running maximum of need a segmented max-scan.
//
// All list lengths (|M|, |R|, |I|) are read from device memory.
#include <climits>

#include "kernels.h"

namespace upr {
namespace {

__device__ __forceinline__ int64_t cw(const int32_t *vwgt, int32_t v) { return vwgt ? (int64_t)vwgt[v] : 1; }

// out = a_mul * (*a) + (b ? *b : 0) + add
__global__ void k_count_affine(const int32_t *__restrict__ a, int32_t a_mul, const int32_t *__restrict__ b,
                               int32_t add, int32_t *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = a_mul * (*a) + (b ? *b : 0) + add;
}

// keys/vals for R grouped by source block
__global__ void k_rb_keys(const int32_t *__restrict__ R_from, const int32_t *__restrict__ d_nR,
                          uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t nR = *d_nR;
    UPR_FOR(i, nR) {
        keys[i] = (uint64_t)R_from[i];
        vals[i] = (uint32_t)i;
    }
}

// per R_b position: node weight; block bounds [rbeg[b], rend[b])
__global__ void k_rb_bounds(const int32_t *__restrict__ R_node, const int32_t *__restrict__ R_from,
                            const uint32_t *__restrict__ RB, const int32_t *__restrict__ d_nR,
                            const int32_t *__restrict__ vwgt, int64_t *__restrict__ rc, int32_t *__restrict__ rbeg,
                            int32_t *__restrict__ rend) {
    const int64_t nR = *d_nR;
    UPR_FOR(q, nR) {
        const uint32_t i = RB[q];
        rc[q] = cw(vwgt, R_node[i]);
        const int32_t b = R_from[i];
        if (q == 0 || R_from[RB[q - 1]] != b) rbeg[b] = (int32_t)q;
        if (q == nR - 1 || R_from[RB[q + 1]] != b) rend[b] = (int32_t)(q + 1);
    }
}

// events of M: 2i = leave M_from[i], 2i+1 = enter M_to[i]
__global__ void k_ev_keys(const int32_t *__restrict__ M_from, const int32_t *__restrict__ M_to,
                          const int32_t *__restrict__ d_nM, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t nev = 2 * (int64_t)*d_nM;
    UPR_FOR(e, nev) {
        const int64_t i = e >> 1;
        keys[e] = (uint64_t)((e & 1) ? M_to[i] : M_from[i]);
        vals[e] = (uint32_t)e;
    }
}

__global__ void k_ev_delta(const int32_t *__restrict__ M_node, const uint32_t *__restrict__ EV,
                           const uint64_t *__restrict__ ekeys, const int32_t *__restrict__ d_nM,
                           const int32_t *__restrict__ vwgt, int64_t *__restrict__ delta, int32_t *__restrict__ ebeg,
                           int32_t *__restrict__ eend) {
    const int64_t nev = 2 * (int64_t)*d_nM;
    UPR_FOR(q, nev) {
        const uint32_t e = EV[q];
        const int64_t c = cw(vwgt, M_node[e >> 1]);
        delta[q] = (e & 1) ? c : -c;
        const int32_t b = (int32_t)ekeys[q];
        if (q == 0 || (int32_t)ekeys[q - 1] != b) ebeg[b] = (int32_t)q;
        if (q == nev - 1 || (int32_t)ekeys[q + 1] != b) eend[b] = (int32_t)(q + 1);
    }
}

// need(q) for inflow events into blocks with R_b non-empty; packed with the block for the max-scan
__global__ void k_ev_need(const uint32_t *__restrict__ EV, const uint64_t *__restrict__ ekeys,
                          const int32_t *__restrict__ d_nM, const int64_t *__restrict__ delta,
                          const int64_t *__restrict__ d_excl, const int32_t *__restrict__ ebeg,
                          const int64_t *__restrict__ C0, const int64_t *__restrict__ Lb,
                          const int32_t *__restrict__ rbeg, const int32_t *__restrict__ rend,
                          const int64_t *__restrict__ rc_excl, const int64_t *__restrict__ rc,
                          uint64_t *__restrict__ packed) {
    const int64_t nev = 2 * (int64_t)*d_nM;
    UPR_FOR(q, nev) {
        const uint32_t e = EV[q];
        const int32_t b = (int32_t)ekeys[q];
        uint32_t need = 0;
        const int32_t r0 = rbeg[b], r1 = rend[b];
        if ((e & 1) && r1 > r0) {
            const int64_t D = C0[b] + (d_excl[q] + delta[q]) - d_excl[ebeg[b]];
            const int64_t Lmax = Lb[b];
            if (D > Lmax) {
                // smallest x in [1, |R_b|] with D - (weight of R_b[0..x)) <= L_max, else |R_b|
                const int64_t base = rc_excl[r0];
                int lo = 1, hi = r1 - r0;
                while (lo < hi) {
                    const int mid = lo + ((hi - lo) >> 1);
                    const int64_t w = rc_excl[r0 + mid - 1] + rc[r0 + mid - 1] - base;
                    if (D - w <= Lmax) hi = mid; else lo = mid + 1;
                }
                need = (uint32_t)lo;
            }
        }
        packed[q] = ((uint64_t)(uint32_t)b << 32) | need;
    }
}

// per M move: emissions after it (e_i) and the R_b count before them
__global__ void k_ev_emit(const uint32_t *__restrict__ EV, const uint64_t *__restrict__ ekeys,
                          const int32_t *__restrict__ d_nM, const uint64_t *__restrict__ qmax,
                          const int32_t *__restrict__ ebeg, int32_t *__restrict__ emit,
                          int32_t *__restrict__ qbefore_m) {
    const int64_t nev = 2 * (int64_t)*d_nM;
    UPR_FOR(q, nev) {
        const uint32_t e = EV[q];
        if (!(e & 1)) continue;
        const int32_t b = (int32_t)ekeys[q];
        const uint32_t after = (uint32_t)qmax[q];
        const uint32_t before = q == ebeg[b] ? 0u : (uint32_t)qmax[q - 1];
        emit[e >> 1] = (int32_t)(after - before);
        qbefore_m[e >> 1] = (int32_t)before;
    }
}

// per block: final emitted count and leftover count
__global__ void k_block_final(int32_t K, const int32_t *__restrict__ ebeg, const int32_t *__restrict__ eend,
                              const uint64_t *__restrict__ qmax, const int32_t *__restrict__ rbeg,
                              const int32_t *__restrict__ rend, int32_t *__restrict__ qfin,
                              int32_t *__restrict__ left) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= K) return;
    const int32_t f = eend[b] > ebeg[b] ? (int32_t)(uint32_t)qmax[eend[b] - 1] : 0;
    qfin[b] = f;
    left[b] = (rend[b] - rbeg[b]) - f;
}

// positions of M moves in X
__global__ void k_place_m(const int32_t *__restrict__ M_node, const int32_t *__restrict__ M_from,
                          const int32_t *__restrict__ M_to, const int32_t *__restrict__ d_nM,
                          const int32_t *__restrict__ em_excl, int32_t *__restrict__ pos_m,
                          int32_t *__restrict__ X_node, int32_t *__restrict__ X_from, int32_t *__restrict__ X_to,
                          int8_t *__restrict__ X_isr) {
    const int64_t nM = *d_nM;
    UPR_FOR(i, nM) {
        const int32_t p = (int32_t)i + em_excl[i];
        pos_m[i] = p;
        X_node[p] = M_node[i];
        X_from[p] = M_from[i];
        X_to[p] = M_to[i];
        X_isr[p] = 0;
    }
}

// positions of R moves in X
__global__ void k_place_r(const int32_t *__restrict__ R_node, const int32_t *__restrict__ R_from,
                          const int32_t *__restrict__ R_to, const uint32_t *__restrict__ RB,
                          const int32_t *__restrict__ d_nR, const int32_t *__restrict__ rbeg,
                          const uint32_t *__restrict__ EV, const int32_t *__restrict__ ebeg,
                          const int32_t *__restrict__ eend, const uint64_t *__restrict__ qmax,
                          const int32_t *__restrict__ pos_m, const int32_t *__restrict__ qfin,
                          const int32_t *__restrict__ left_excl, const int32_t *__restrict__ em_excl,
                          const int32_t *__restrict__ emit, const int32_t *__restrict__ d_nM,
                          int32_t *__restrict__ X_node, int32_t *__restrict__ X_from, int32_t *__restrict__ X_to,
                          int8_t *__restrict__ X_isr) {
    const int64_t nR = *d_nR, nM = *d_nM;
    const int64_t tail0 = nM + (nM > 0 ? (int64_t)em_excl[nM - 1] + emit[nM - 1] : 0);
    UPR_FOR(q, nR) {
        const uint32_t i = RB[q];
        const int32_t b = R_from[i];
        const uint32_t r = (uint32_t)(q - rbeg[b]);
        int64_t p;
        if ((int32_t)r < qfin[b]) {
            // first event of b with running max > r (an inflow event)
            int lo = ebeg[b], hi = eend[b] - 1;
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if ((uint32_t)qmax[mid] > r) hi = mid; else lo = mid + 1;
            }
            const uint32_t before = lo == ebeg[b] ? 0u : (uint32_t)qmax[lo - 1];
            p = (int64_t)pos_m[EV[lo] >> 1] + 1 + (r - before);
        } else {
            p = tail0 + left_excl[b] + (r - (uint32_t)qfin[b]);
        }
        X_node[p] = R_node[i];
        X_from[p] = R_from[i];
        X_to[p] = R_to[i];
        X_isr[p] = 1;
    }
}

// merging: an R move of a node that also has an M move folds into the M move
__global__ void k_merge_flags(const int32_t *__restrict__ X_node, const int32_t *__restrict__ X_to,
                              const int8_t *__restrict__ X_isr, const int32_t *__restrict__ d_nX,
                              const int32_t *__restrict__ m_pos, const int32_t *__restrict__ r_to,
                              const int32_t *__restrict__ part0, int32_t *__restrict__ keep,
                              int32_t *__restrict__ final_to) {
    const int64_t nX = *d_nX;
    UPR_FOR(x, nX) {
        const int32_t v = X_node[x];
        int32_t to = X_to[x];
        bool k = true;
        if (X_isr[x]) {
            if (m_pos[v] >= 0) k = false;
        } else if (r_to[v] >= 0) {
            to = r_to[v];
        }
        if (k && to == part0[v]) k = false;
        keep[x] = k ? 1 : 0;
        final_to[x] = to;
    }
}

__global__ void k_build_I(const int32_t *__restrict__ Ix, const int32_t *__restrict__ d_nI,
                          const int32_t *__restrict__ X_node, const int32_t *__restrict__ final_to,
                          const int32_t *__restrict__ part0, int32_t *__restrict__ I_node,
                          int32_t *__restrict__ I_from, int32_t *__restrict__ I_to, int32_t *__restrict__ pos,
                          int32_t *__restrict__ dest) {
    const int64_t nI = *d_nI;
    UPR_FOR(i, nI) {
        const int32_t x = Ix[i];
        const int32_t v = X_node[x];
        I_node[i] = v;
        I_from[i] = part0[v];
        I_to[i] = final_to[x];
        pos[v] = (int32_t)i;
        dest[v] = final_to[x];
    }
}

// Exact gain of the i-th move of I: neighbours moved earlier in I count in
// their new block, all others in their round-start block.  Warp per move;
// hub moves (degree > kHubDegree) are left to k_gains_hub.
// Block of each node at every step of I, packed for one 8-byte gather per
// adjacency entry: x = the node's position in I (INT32_MAX when it does not
// move), y = (local block before its move) | (local block after it) << 16.
// Before step i a neighbour u is in its later block iff x < i.
__global__ void k_pk_fill(const int32_t *__restrict__ part0, int64_t n, int32_t k, int32_t kmask,
                          int2 *__restrict__ pk) {
    UPR_FOR(u, n) {
        const uint32_t l = (uint32_t)blk_local(part0[u], k, kmask);
        pk[u] = make_int2(INT32_MAX, (int32_t)(l | (l << 16)));
    }
}

// Also adds the degrees of the moved nodes to *deg_sum (the adjacency the
// exact gains read: the step's algorithmic bytes).
__global__ void k_pk_moves(const int32_t *__restrict__ I_node, const int32_t *__restrict__ I_from,
                           const int32_t *__restrict__ I_to, const int32_t *__restrict__ d_nI, int32_t k,
                           int32_t kmask, const int64_t *__restrict__ xadj, int2 *__restrict__ pk,
                           unsigned long long *__restrict__ deg_sum) {
    const int64_t nI = *d_nI;
    unsigned long long deg = 0;
    UPR_FOR(i, nI) {
        const int32_t v = I_node[i];
        const uint32_t a = (uint32_t)blk_local(I_from[i], k, kmask), b = (uint32_t)blk_local(I_to[i], k, kmask);
        pk[v] = make_int2((int32_t)i, (int32_t)(a | (b << 16)));
        deg += (unsigned long long)(xadj[v + 1] - xadj[v]);
    }
    deg = warp_sum(deg);
    if ((threadIdx.x & 31) == 0 && deg) atomicAdd(deg_sum, deg);
}

__device__ __forceinline__ uint32_t block_before(int2 p, int64_t i) {
    const uint32_t code = (uint32_t)p.y;
    return p.x < i ? (code >> 16) : (code & 0xffffu);
}

// Exact gain of every move of I against the partition just before it (Sec.
// 4.4): warp per move, hubs (degree > kHubDegree) are left to the chunk kernel.
__global__ void k_gains_warp(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                             const int32_t *__restrict__ adjw, const int32_t *__restrict__ I_node,
                             const int32_t *__restrict__ I_from, const int32_t *__restrict__ I_to,
                             const int32_t *__restrict__ d_nI, const int2 *__restrict__ pk, int32_t k, int32_t kmask,
                             int64_t *__restrict__ gain) {
    const int lane = threadIdx.x & 31;
    const int64_t nI = *d_nI;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nI;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t v = I_node[i];
        const uint32_t a = (uint32_t)blk_local(I_from[i], k, kmask), b = (uint32_t)blk_local(I_to[i], k, kmask);
        const int64_t e0 = xadj[v], e1 = xadj[v + 1];
        if (e1 - e0 > kHubDegree) {
            if (lane == 0) gain[i] = 0;
            continue;
        }
        long long acc = 0;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const uint32_t bu = block_before(pk[adj[e]], i);
            const int32_t w = adjw ? adjw[e] : 1;
            acc += (bu == b ? w : 0) - (bu == a ? w : 0);
        }
        acc = warp_sum(acc);
        if (lane == 0) gain[i] = acc;
    }
}

// Exact gains of hub moves, one CTA per static chunk of a hub's adjacency:
// partial sums added to gain[i] (set to 0 by k_gains_warp) with 64-bit
// integer atomics, whose result does not depend on their order.
__global__ void __launch_bounds__(512) k_gains_hub_chunks(const HubChunk *__restrict__ chunks,
                                                          const int32_t *__restrict__ adj,
                                                          const int32_t *__restrict__ adjw,
                                                          const int2 *__restrict__ pk,
                                                          int64_t *__restrict__ gain) {
    __shared__ long long s_w[16];
    const HubChunk ch = chunks[blockIdx.x];
    const int2 me = pk[ch.v];
    const int32_t i = me.x;
    if (i == INT32_MAX) return;                  // this hub is not in I
    const uint32_t a = (uint32_t)me.y & 0xffffu, b = (uint32_t)me.y >> 16;
    long long acc = 0;
    for (int64_t e = ch.begin + threadIdx.x; e < ch.end; e += blockDim.x) {
        const uint32_t bu = block_before(pk[adj[e]], i);
        const int32_t w = adjw ? adjw[e] : 1;
        acc += (bu == b ? w : 0) - (bu == a ? w : 0);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
        if (t) atomicAdd(reinterpret_cast<unsigned long long *>(&gain[i]), (unsigned long long)t);
    }
}

// block events of I for the weight trajectory: 2i = leave I_from[i], 2i+1 = enter I_to[i]
__global__ void k_iev_keys(const int32_t *__restrict__ I_from, const int32_t *__restrict__ I_to,
                           const int32_t *__restrict__ d_nI, uint64_t *__restrict__ keys,
                           uint32_t *__restrict__ vals) {
    const int64_t nev = 2 * (int64_t)*d_nI;
    UPR_FOR(e, nev) {
        const int64_t i = e >> 1;
        keys[e] = (uint64_t)((e & 1) ? I_to[i] : I_from[i]);
        vals[e] = (uint32_t)e;
    }
}

__global__ void k_iev_delta(const int32_t *__restrict__ I_node, const uint32_t *__restrict__ EV,
                            const uint64_t *__restrict__ ekeys, const int32_t *__restrict__ d_nI,
                            const int32_t *__restrict__ vwgt, int64_t *__restrict__ delta,
                            int32_t *__restrict__ ebeg) {
    const int64_t nev = 2 * (int64_t)*d_nI;
    UPR_FOR(q, nev) {
        const uint32_t e = EV[q];
        const int64_t c = cw(vwgt, I_node[e >> 1]);
        delta[q] = (e & 1) ? c : -c;
        const int32_t b = (int32_t)ekeys[q];
        if (q == 0 || (int32_t)ekeys[q - 1] != b) ebeg[b] = (int32_t)q;
    }
}

// Changes of the number of overloaded blocks, at prefix length j = i + 1.
__global__ void k_iev_transitions(const uint32_t *__restrict__ EV, const uint64_t *__restrict__ ekeys,
                                  const int32_t *__restrict__ d_nI, const int64_t *__restrict__ delta,
                                  const int64_t *__restrict__ d_excl, const int32_t *__restrict__ ebeg,
                                  const int64_t *__restrict__ C0, const int64_t *__restrict__ Lb,
                                  int32_t *__restrict__ diff) {
    const int64_t nev = 2 * (int64_t)*d_nI;
    UPR_FOR(q, nev) {
        const int32_t b = (int32_t)ekeys[q];
        const int64_t Lmax = Lb[b];
        const int64_t before = C0[b] + d_excl[q] - d_excl[ebeg[b]];
        const int64_t after = before + delta[q];
        const int t = (after > Lmax ? 1 : 0) - (before > Lmax ? 1 : 0);
        if (t) atomicAdd(&diff[(EV[q] >> 1) + 1], t);
    }
}

// number of blocks above L_max, per graph (out[0..ng) zeroed by the caller)
__global__ void k_count_over(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t K, int32_t k,
                             int32_t *__restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < K; b += gridDim.x * blockDim.x)
        if (C[b] > Lb[b]) atomicAdd(&out[b / k], 1);
}

// best prefix: max G(j) over eligible j (ties: smallest j); G(0) = 0, eligible(0) = (over0 == 0)
struct Best { long long g; long long j; };

__device__ __forceinline__ Best better(Best x, Best y) {
    if (x.j < 0) return y;
    if (y.j < 0) return x;
    if (y.g > x.g || (y.g == x.g && y.j < x.j)) return y;
    return x;
}

__global__ void k_best_partial(const int64_t *__restrict__ Gsum, const int32_t *__restrict__ diff,
                               const int32_t *__restrict__ diff_excl, const int32_t *__restrict__ d_nI,
                               const int32_t *__restrict__ d_over0, long long *__restrict__ part_g,
                               long long *__restrict__ part_j) {
    __shared__ long long s_g[8], s_j[8];
    const int64_t nI = *d_nI;
    const int32_t over0 = *d_over0;
    Best b{0, -1};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= nI; j += (int64_t)gridDim.x * blockDim.x) {
        const bool elig = over0 + diff_excl[j] + diff[j] == 0;
        if (elig) b = better(b, Best{j == 0 ? 0 : Gsum[j - 1], j});
    }
    for (int o = 16; o > 0; o >>= 1) {
        Best y{__shfl_xor_sync(0xffffffffu, b.g, o), __shfl_xor_sync(0xffffffffu, b.j, o)};
        b = better(b, y);
    }
    if ((threadIdx.x & 31) == 0) { s_g[threadIdx.x >> 5] = b.g; s_j[threadIdx.x >> 5] = b.j; }
    __syncthreads();
    if (threadIdx.x == 0) {
        Best t{0, -1};
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = better(t, Best{s_g[w], s_j[w]});
        part_g[blockIdx.x] = t.g;
        part_j[blockIdx.x] = t.j;
    }
}

__global__ void __launch_bounds__(1024) k_best_final(const long long *__restrict__ part_g,
                                                    const long long *__restrict__ part_j, int parts,
                                                    long long *__restrict__ out, int32_t *__restrict__ infeasible) {
    __shared__ long long s_g[32], s_j[32];
    Best b{0, -1};
    for (int p = threadIdx.x; p < parts; p += blockDim.x) b = better(b, Best{part_g[p], part_j[p]});
    for (int o = 16; o > 0; o >>= 1) {
        Best y{__shfl_xor_sync(0xffffffffu, b.g, o), __shfl_xor_sync(0xffffffffu, b.j, o)};
        b = better(b, y);
    }
    if ((threadIdx.x & 31) == 0) { s_g[threadIdx.x >> 5] = b.g; s_j[threadIdx.x >> 5] = b.j; }
    __syncthreads();
    if (threadIdx.x == 0) {
        Best t{0, -1};
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = better(t, Best{s_g[w], s_j[w]});
        out[0] = t.g;
        out[1] = t.j;
        if (t.j < 0) *infeasible = 1;
    }
}

__global__ void k_apply_prefix(const int32_t *__restrict__ I_node, const int32_t *__restrict__ I_from,
                               const int32_t *__restrict__ I_to, const long long *__restrict__ best,
                               const int32_t *__restrict__ vwgt, int32_t *__restrict__ part0,
                               unsigned long long *__restrict__ C0, int32_t K, long long *__restrict__ cut) {
    extern __shared__ unsigned long long s_delta[];
    BlockDelta bd = make_block_delta(s_delta, K, C0);
    bd.init();
    const long long len = best[1];
    if (blockIdx.x == 0 && threadIdx.x == 0 && len >= 0) atomicAdd((unsigned long long *)cut, (unsigned long long)(-best[0]));
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < len; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = base + threadIdx.x;
        int32_t a = -1, b = -1;
        long long c = 0;
        if (j < len) {
            const int32_t v = I_node[j];
            a = I_from[j];
            b = I_to[j];
            c = vwgt ? vwgt[v] : 1;
            part0[v] = b;
        }
        bd.add(a, -c);
        bd.add(b, c);
    }
    bd.flush(C0);
}

// ---- batches: I sorted by graph (stable), then per-graph segments
// [seg_beg[g], seg_end[g]) of I; G_g(j) and eligibility are differences of
// the global prefix sums taken at the segment start.

// keys: graph of each move of I
__global__ void k_i_graph_keys(const int32_t *__restrict__ I_node, const int32_t *__restrict__ d_nI,
                               const int32_t *__restrict__ gid, uint64_t *__restrict__ keys,
                               uint32_t *__restrict__ vals) {
    const int64_t nI = *d_nI;
    UPR_FOR(i, nI) {
        keys[i] = (uint64_t)gid[I_node[i]];
        vals[i] = (uint32_t)i;
    }
}

// I in graph order (out arrays), pos/dest of the moved nodes, segment bounds
__global__ void k_i_permute(const uint32_t *__restrict__ order, const uint64_t *__restrict__ gkeys,
                            const int32_t *__restrict__ d_nI, const int32_t *__restrict__ I_node,
                            const int32_t *__restrict__ I_from, const int32_t *__restrict__ I_to,
                            int32_t *__restrict__ O_node, int32_t *__restrict__ O_from, int32_t *__restrict__ O_to,
                            int32_t *__restrict__ pos, int32_t *__restrict__ dest, int32_t *__restrict__ seg_beg,
                            int32_t *__restrict__ seg_end) {
    const int64_t nI = *d_nI;
    UPR_FOR(q, nI) {
        const uint32_t i = order[q];
        const int32_t v = I_node[i];
        O_node[q] = v;
        O_from[q] = I_from[i];
        O_to[q] = I_to[i];
        pos[v] = (int32_t)q;
        dest[v] = I_to[i];
        const int32_t g = (int32_t)gkeys[q];
        if (q == 0 || (int32_t)gkeys[q - 1] != g) seg_beg[g] = (int32_t)q;
        if (q == nI - 1 || (int32_t)gkeys[q + 1] != g) seg_end[g] = (int32_t)(q + 1);
    }
}

// per graph: best gain so far = 0 if the empty prefix is eligible, else "none"
__global__ void k_best_seg_init(const int32_t *__restrict__ over0, int32_t ng, long long *__restrict__ best_g,
                                long long *__restrict__ best_j) {
    UPR_FOR(g, ng) {
        best_g[g] = over0[g] == 0 ? 0 : LLONG_MIN;
        best_j[g] = LLONG_MAX;
    }
}

struct SegPoint { int32_t g; long long G; long long j; bool elig; };

// Prefix of length j = i - seg_beg + 1 of move i's graph: its gain and eligibility.
__device__ __forceinline__ SegPoint seg_point(int64_t i, const int32_t *I_node, const int32_t *gid,
                                              const int32_t *seg_beg, const int64_t *Gsum, const int32_t *diff,
                                              const int32_t *diff_excl, const int32_t *over0) {
    const int32_t g = gid[I_node[i]];
    const int32_t s = seg_beg[g];
    const long long G = Gsum[i] - (s > 0 ? Gsum[s - 1] : 0);
    const int32_t over = over0[g] + (diff_excl[i + 1] + diff[i + 1]) - (diff_excl[s] + diff[s]);
    return SegPoint{g, G, (long long)(i - s + 1), over == 0};
}

__global__ void k_best_seg_max(const int32_t *__restrict__ I_node, const int32_t *__restrict__ d_nI,
                               const int32_t *__restrict__ gid, const int32_t *__restrict__ seg_beg,
                               const int64_t *__restrict__ Gsum, const int32_t *__restrict__ diff,
                               const int32_t *__restrict__ diff_excl, const int32_t *__restrict__ over0,
                               long long *__restrict__ best_g) {
    const int64_t nI = *d_nI;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nI; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int32_t key = -1;
        long long val = LLONG_MIN;
        if (i < nI) {
            const SegPoint p = seg_point(i, I_node, gid, seg_beg, Gsum, diff, diff_excl, over0);
            if (p.elig) { key = p.g; val = p.G; }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        long long m = val;
        for (unsigned r = peers; r; r &= r - 1) m = max(m, __shfl_sync(peers, val, __ffs(r) - 1));
        if (key >= 0 && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicMax(&best_g[key], m);
    }
}

__global__ void k_best_seg_min(const int32_t *__restrict__ I_node, const int32_t *__restrict__ d_nI,
                               const int32_t *__restrict__ gid, const int32_t *__restrict__ seg_beg,
                               const int64_t *__restrict__ Gsum, const int32_t *__restrict__ diff,
                               const int32_t *__restrict__ diff_excl, const int32_t *__restrict__ over0,
                               const long long *__restrict__ best_g, long long *__restrict__ best_j) {
    const int64_t nI = *d_nI;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nI; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int32_t key = -1;
        long long val = LLONG_MAX;
        if (i < nI) {
            const SegPoint p = seg_point(i, I_node, gid, seg_beg, Gsum, diff, diff_excl, over0);
            if (p.elig && p.G == best_g[p.g]) { key = p.g; val = p.j; }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        long long m = val;
        for (unsigned r = peers; r; r &= r - 1) m = min(m, __shfl_sync(peers, val, __ffs(r) - 1));
        if (key >= 0 && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicMin(&best_j[key], m);
    }
}

// per graph: j* (the empty prefix wins ties), cut update; totals for the
// round statistics in tot[0..3) = (sum of j*, sum of gains, infeasible graphs)
__global__ void k_best_seg_final(const int32_t *__restrict__ over0, int32_t ng, long long *__restrict__ best_g,
                                 long long *__restrict__ best_j, long long *__restrict__ cut,
                                 int32_t *__restrict__ infeasible, unsigned long long *__restrict__ tot) {
    long long sj = 0, sg = 0, ninf = 0;
    UPR_FOR(g, ng) {
        long long G = best_g[g], j;
        if (G == LLONG_MIN) {
            infeasible[g] = 1;
            G = 0;
            j = 0;
            ninf++;
        } else {
            infeasible[g] = 0;
            j = (over0[g] == 0 && G == 0) ? 0 : best_j[g];
            cut[g] -= G;
        }
        best_g[g] = G;
        best_j[g] = j;
        sj += j;
        sg += G;
    }
    sj = warp_sum(sj);
    sg = warp_sum(sg);
    ninf = warp_sum(ninf);
    if ((threadIdx.x & 31) == 0) {
        if (sj) atomicAdd(&tot[0], (unsigned long long)sj);
        if (sg) atomicAdd(&tot[1], (unsigned long long)sg);
        if (ninf) atomicAdd(&tot[2], (unsigned long long)ninf);
    }
}

__global__ void k_apply_prefix_seg(const int32_t *__restrict__ I_node, const int32_t *__restrict__ I_from,
                                   const int32_t *__restrict__ I_to, const int32_t *__restrict__ d_nI,
                                   const int32_t *__restrict__ gid, const int32_t *__restrict__ seg_beg,
                                   const long long *__restrict__ best_j, const int32_t *__restrict__ vwgt,
                                   int32_t *__restrict__ part0, unsigned long long *__restrict__ C0, int32_t K) {
    extern __shared__ unsigned long long s_delta[];
    BlockDelta bd = make_block_delta(s_delta, K, C0);
    bd.init();
    const int64_t nI = *d_nI;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nI; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int32_t a = -1, b = -1;
        long long c = 0;
        if (i < nI) {
            const int32_t v = I_node[i];
            const int32_t g = gid[v];
            if (i - seg_beg[g] < best_j[g]) {
                a = I_from[i];
                b = I_to[i];
                c = vwgt ? vwgt[v] : 1;
                part0[v] = b;
            }
        }
        bd.add(a, -c);
        bd.add(b, c);
    }
    bd.flush(C0);
}

// ---- carrying the gain table into the next round.  After rebalancing the
// table is W(P o M o R) = W(P o I); the next round starts from P o I^{j*},
// so the moves of I after the best prefix are undone in the table (delta
// updates), or the table is rebuilt when they touch many entries.
__device__ __forceinline__ bool rolled_back(const Rollback &rb, int64_t i) {
    if (!rb.gid) {
        const long long j = rb.best[1];
        return i >= (j < 0 ? 0 : j);
    }
    const int32_t g = rb.gid[rb.I_node[i]];
    return i - rb.seg_beg[g] >= rb.best_j[g];
}

__global__ void k_rollback_degsum(Rollback rb, const int64_t *__restrict__ xadj, unsigned long long *__restrict__ out) {
    const int64_t nI = *rb.d_nI;
    long long acc = 0;
    UPR_FOR(i, nI) {
        if (rolled_back(rb, i)) {
            const int32_t v = rb.I_node[i];
            acc += xadj[v + 1] - xadj[v];
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

// warp per move of I; hubs are left to k_table_rollback_hubs
// (sparse rows: both blocks are keys of the row already, so nothing is inserted)
__global__ void k_table_rollback(Rollback rb, const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                                 const int32_t *__restrict__ adjw, int32_t k, int32_t kmask, int32_t *__restrict__ W,
                                 const int64_t *__restrict__ deg_sum, int64_t m, SparseRows sp) {
    if (*deg_sum * 4 >= m) return;          // the rebuild handles this case
    const int lane = threadIdx.x & 31;
    const int64_t nI = *rb.d_nI;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nI;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        if (!rolled_back(rb, i)) continue;
        const int32_t v = rb.I_node[i];
        const int64_t e0 = xadj[v], e1 = xadj[v + 1];
        if (e1 - e0 > kHubDegree) continue;
        const int32_t a = blk_local(rb.I_to[i], k, kmask), b = blk_local(rb.I_from[i], k, kmask);
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t w = adjw ? adjw[e] : 1;
            if (sp.on()) {
                sp_sub(sp, adj[e], a, w);
                sp_add(sp, adj[e], b, w);
                continue;
            }
            int32_t *row = W + (int64_t)adj[e] * k;
            atomicSub(&row[a], w);
            atomicAdd(&row[b], w);
        }
    }
}

__global__ void __launch_bounds__(512) k_table_rollback_hubs(Rollback rb, const HubChunk *__restrict__ chunks,
                                                             const int32_t *__restrict__ pos,
                                                             const int32_t *__restrict__ adj,
                                                             const int32_t *__restrict__ adjw, int32_t k,
                                                             int32_t kmask, int32_t *__restrict__ W,
                                                             const int64_t *__restrict__ deg_sum, int64_t m,
                                                             SparseRows sp) {
    if (*deg_sum * 4 >= m) return;
    const HubChunk ch = chunks[blockIdx.x];
    const int32_t i = pos[ch.v];
    if (i == INT32_MAX || !rolled_back(rb, i)) return;
    const int32_t a = blk_local(rb.I_to[i], k, kmask), b = blk_local(rb.I_from[i], k, kmask);
    for (int64_t e = ch.begin + threadIdx.x; e < ch.end; e += blockDim.x) {
        const int32_t w = adjw ? adjw[e] : 1;
        if (sp.on()) {
            sp_sub(sp, adj[e], a, w);
            sp_add(sp, adj[e], b, w);
            continue;
        }
        int32_t *row = W + (int64_t)adj[e] * k;
        atomicSub(&row[a], w);
        atomicAdd(&row[b], w);
    }
}

// The variant of Sec. 7.2 without interleaving: X = M, then R in its order.
__global__ void k_seq_append(const int32_t *__restrict__ M_node, const int32_t *__restrict__ M_from,
                             const int32_t *__restrict__ M_to, const int32_t *__restrict__ d_nM,
                             const int32_t *__restrict__ R_node, const int32_t *__restrict__ R_from,
                             const int32_t *__restrict__ R_to, const int32_t *__restrict__ d_nR,
                             int32_t *__restrict__ X_node, int32_t *__restrict__ X_from, int32_t *__restrict__ X_to,
                             int8_t *__restrict__ X_isr) {
    const int64_t nM = *d_nM, nR = *d_nR;
    UPR_FOR(i, nM + nR) {
        const bool r = i >= nM;
        const int64_t j = r ? i - nM : i;
        X_node[i] = r ? R_node[j] : M_node[j];
        X_from[i] = r ? R_from[j] : M_from[j];
        X_to[i] = r ? R_to[j] : M_to[j];
        X_isr[i] = r ? 1 : 0;
    }
}

// The oscillation guard of Sec. 2: lock the nodes of the applied prefix whose
// move comes from rebalancing alone (an R move and no M move).
__global__ void k_guard_locks(Rollback rb, const int32_t *__restrict__ m_pos, const int32_t *__restrict__ r_to,
                              int8_t *__restrict__ locked) {
    const int64_t nI = *rb.d_nI;
    UPR_FOR(i, nI) {
        if (rolled_back(rb, i)) continue;
        const int32_t v = rb.I_node[i];
        if (m_pos[v] < 0 && r_to[v] >= 0) locked[v] = 1;
    }
}

// no candidate among the locked nodes
__global__ void k_guard_filter(const int8_t *__restrict__ locked, int64_t n, int32_t *__restrict__ flags,
                               int32_t *__restrict__ cand_tgt, int64_t *__restrict__ cand_s0,
                               int32_t *__restrict__ cand_gain) {
    UPR_FOR(v, n) {
        if (!locked[v]) continue;
        flags[v] = 0;
        cand_tgt[v] = -1;
        cand_s0[v] = 0;
        cand_gain[v] = 0;
    }
}

__global__ void k_reset_nodes(const int32_t *__restrict__ nodes, const int32_t *__restrict__ d_cnt,
                              int32_t *__restrict__ arr, int32_t val) {
    const int64_t cnt = *d_cnt;
    UPR_FOR(i, cnt) arr[nodes[i]] = val;
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
    UPR_FOR(i, n) a[i] = v;
}

// a[0 .. *d_n + extra) = 0
__global__ void k_clear_count(int32_t *a, const int32_t *__restrict__ d_n, int32_t extra) {
    const int64_t n = (int64_t)*d_n + extra;
    UPR_FOR(i, n) a[i] = 0;
}

}  // namespace

// ---------------------------------------------------------------- wrappers
void count_affine(const int32_t *a, int32_t a_mul, const int32_t *b, int32_t add, int32_t *out, cudaStream_t s) {
    k_count_affine<<<1, 32, 0, s>>>(a, a_mul, b, add, out);
    UPR_LAUNCH_CHECK();
}

void fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t s) {
    if (n <= 0) return;
    k_fill_i32<<<grid_for(n), 256, 0, s>>>(a, n, v);
    UPR_LAUNCH_CHECK();
}

void clear_count(int32_t *a, const int32_t *d_n, int32_t extra, int64_t max, cudaStream_t s) {
    k_clear_count<<<grid_for(max + extra), 256, 0, s>>>(a, d_n, extra);
    UPR_LAUNCH_CHECK();
}

void reset_nodes(const int32_t *nodes, const int32_t *d_cnt, int64_t max, int32_t *arr, int32_t val, cudaStream_t s) {
    if (max <= 0) return;
    k_reset_nodes<<<grid_for(max), 256, 0, s>>>(nodes, d_cnt, arr, val);
    UPR_LAUNCH_CHECK();
}

void count_over(const GraphDev &g, const int64_t *C, int32_t *out, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t) * g.ng, s));
    k_count_over<<<grid_for(g.K()), 256, 0, s>>>(C, g.Lb, g.K(), g.k, out);
    UPR_LAUNCH_CHECK();
}

void seq_rb_keys(const int32_t *R_from, const int32_t *d_nR, int64_t max, uint64_t *keys, uint32_t *vals,
                 cudaStream_t s) {
    k_rb_keys<<<grid_for(max), 256, 0, s>>>(R_from, d_nR, keys, vals);
    UPR_LAUNCH_CHECK();
}

void seq_rb_bounds(const int32_t *R_node, const int32_t *R_from, const uint32_t *RB, const int32_t *d_nR, int64_t max,
                   const int32_t *vwgt, int64_t *rc, int32_t *rbeg, int32_t *rend, cudaStream_t s) {
    k_rb_bounds<<<grid_for(max), 256, 0, s>>>(R_node, R_from, RB, d_nR, vwgt, rc, rbeg, rend);
    UPR_LAUNCH_CHECK();
}

void seq_ev_keys(const int32_t *M_from, const int32_t *M_to, const int32_t *d_nM, int64_t max, uint64_t *keys,
                 uint32_t *vals, cudaStream_t s) {
    k_ev_keys<<<grid_for(2 * max), 256, 0, s>>>(M_from, M_to, d_nM, keys, vals);
    UPR_LAUNCH_CHECK();
}

void seq_ev_delta(const int32_t *M_node, const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nM, int64_t max,
                  const int32_t *vwgt, int64_t *delta, int32_t *ebeg, int32_t *eend, cudaStream_t s) {
    k_ev_delta<<<grid_for(2 * max), 256, 0, s>>>(M_node, EV, ekeys, d_nM, vwgt, delta, ebeg, eend);
    UPR_LAUNCH_CHECK();
}

void seq_ev_need(const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nM, int64_t max, const int64_t *delta,
                 const int64_t *d_excl, const int32_t *ebeg, const int64_t *C0, const int64_t *Lb,
                 const int32_t *rbeg, const int32_t *rend, const int64_t *rc_excl, const int64_t *rc, uint64_t *packed,
                 cudaStream_t s) {
    k_ev_need<<<grid_for(2 * max), 256, 0, s>>>(EV, ekeys, d_nM, delta, d_excl, ebeg, C0, Lb, rbeg, rend, rc_excl, rc,
                                                packed);
    UPR_LAUNCH_CHECK();
}

void seq_ev_emit(const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nM, int64_t max, const uint64_t *qmax,
                 const int32_t *ebeg, int32_t *emit, int32_t *qbefore_m, cudaStream_t s) {
    k_ev_emit<<<grid_for(2 * max), 256, 0, s>>>(EV, ekeys, d_nM, qmax, ebeg, emit, qbefore_m);
    UPR_LAUNCH_CHECK();
}

void seq_block_final(int32_t K, const int32_t *ebeg, const int32_t *eend, const uint64_t *qmax, const int32_t *rbeg,
                     const int32_t *rend, int32_t *qfin, int32_t *left, cudaStream_t s) {
    k_block_final<<<(unsigned)ceil_div(K, 256), 256, 0, s>>>(K, ebeg, eend, qmax, rbeg, rend, qfin, left);
    UPR_LAUNCH_CHECK();
}

void seq_place_m(const int32_t *M_node, const int32_t *M_from, const int32_t *M_to, const int32_t *d_nM, int64_t max,
                 const int32_t *em_excl, int32_t *pos_m, int32_t *X_node, int32_t *X_from, int32_t *X_to,
                 int8_t *X_isr, cudaStream_t s) {
    k_place_m<<<grid_for(max), 256, 0, s>>>(M_node, M_from, M_to, d_nM, em_excl, pos_m, X_node, X_from, X_to, X_isr);
    UPR_LAUNCH_CHECK();
}

void seq_place_r(const int32_t *R_node, const int32_t *R_from, const int32_t *R_to, const uint32_t *RB,
                 const int32_t *d_nR, int64_t max, const int32_t *rbeg, const uint32_t *EV, const int32_t *ebeg,
                 const int32_t *eend, const uint64_t *qmax, const int32_t *pos_m, const int32_t *qfin,
                 const int32_t *left_excl, const int32_t *em_excl, const int32_t *emit, const int32_t *d_nM,
                 int32_t *X_node, int32_t *X_from, int32_t *X_to, int8_t *X_isr, cudaStream_t s) {
    k_place_r<<<grid_for(max), 256, 0, s>>>(R_node, R_from, R_to, RB, d_nR, rbeg, EV, ebeg, eend, qmax, pos_m, qfin,
                                            left_excl, em_excl, emit, d_nM, X_node, X_from, X_to, X_isr);
    UPR_LAUNCH_CHECK();
}

void seq_merge_flags(const int32_t *X_node, const int32_t *X_to, const int8_t *X_isr, const int32_t *d_nX, int64_t max,
                     const int32_t *m_pos, const int32_t *r_to, const int32_t *part0, int32_t *keep, int32_t *final_to,
                     cudaStream_t s) {
    k_merge_flags<<<grid_for(max), 256, 0, s>>>(X_node, X_to, X_isr, d_nX, m_pos, r_to, part0, keep, final_to);
    UPR_LAUNCH_CHECK();
}

void seq_build_I(const int32_t *Ix, const int32_t *d_nI, int64_t max, const int32_t *X_node, const int32_t *final_to,
                 const int32_t *part0, int32_t *I_node, int32_t *I_from, int32_t *I_to, int32_t *pos, int32_t *dest,
                 cudaStream_t s) {
    k_build_I<<<grid_for(max), 256, 0, s>>>(Ix, d_nI, X_node, final_to, part0, I_node, I_from, I_to, pos, dest);
    UPR_LAUNCH_CHECK();
}

void seq_gains(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
               const int32_t *d_nI, int64_t max, const int32_t *part0, int2 *pk, int64_t *gain,
               const HubChunk *hub_chunks, int64_t n_chunks, int64_t *deg_sum, cudaStream_t s) {
    k_pk_fill<<<grid_for(g.n), 256, 0, s>>>(part0, g.n, g.k, g.kmask, pk);
    UPR_LAUNCH_CHECK();
    k_pk_moves<<<grid_for(max), 256, 0, s>>>(I_node, I_from, I_to, d_nI, g.k, g.kmask, g.xadj, pk,
                                             reinterpret_cast<unsigned long long *>(deg_sum));
    UPR_LAUNCH_CHECK();
    // two waves of CTAs (moved nodes differ widely in degree)
    const unsigned blocks = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(max * 32, 256), (int64_t)device_sm_count() * 16));
    k_gains_warp<<<blocks, 256, 0, s>>>(g.xadj, g.adj, g.adjw, I_node, I_from, I_to, d_nI, pk, g.k, g.kmask, gain);
    UPR_LAUNCH_CHECK();
    if (n_chunks > 0) {
        k_gains_hub_chunks<<<(unsigned)n_chunks, 512, 0, s>>>(hub_chunks, g.adj, g.adjw, pk, gain);
        UPR_LAUNCH_CHECK();
    }
}

void seq_iev_keys(const int32_t *I_from, const int32_t *I_to, const int32_t *d_nI, int64_t max, uint64_t *keys,
                  uint32_t *vals, cudaStream_t s) {
    k_iev_keys<<<grid_for(2 * max), 256, 0, s>>>(I_from, I_to, d_nI, keys, vals);
    UPR_LAUNCH_CHECK();
}

void seq_iev_delta(const int32_t *I_node, const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nI, int64_t max,
                   const int32_t *vwgt, int64_t *delta, int32_t *ebeg, cudaStream_t s) {
    k_iev_delta<<<grid_for(2 * max), 256, 0, s>>>(I_node, EV, ekeys, d_nI, vwgt, delta, ebeg);
    UPR_LAUNCH_CHECK();
}

void seq_iev_transitions(const uint32_t *EV, const uint64_t *ekeys, const int32_t *d_nI, int64_t max,
                         const int64_t *delta, const int64_t *d_excl, const int32_t *ebeg, const int64_t *C0,
                         const int64_t *Lb, int32_t *diff, cudaStream_t s) {
    k_iev_transitions<<<grid_for(2 * max), 256, 0, s>>>(EV, ekeys, d_nI, delta, d_excl, ebeg, C0, Lb, diff);
    UPR_LAUNCH_CHECK();
}

void seq_best(const int64_t *Gsum, const int32_t *diff, const int32_t *diff_excl, const int32_t *d_nI, int64_t max,
              const int32_t *d_over0, long long *parts, long long *out, int32_t *infeasible, cudaStream_t s) {
    const int nparts = (int)std::min<int64_t>(ceil_div(max + 1, 256), 1024);
    k_best_partial<<<nparts, 256, 0, s>>>(Gsum, diff, diff_excl, d_nI, d_over0, parts, parts + 1024);
    UPR_LAUNCH_CHECK();
    k_best_final<<<1, 1024, 0, s>>>(parts, parts + 1024, nparts, out, infeasible);
    UPR_LAUNCH_CHECK();
}

void seq_apply_prefix(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
                      int64_t max, const long long *best, int32_t *part0, int64_t *C0, int64_t *cut, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>(ceil_div(max > 0 ? max : 1, 256), (int64_t)device_sm_count() * 4);
    k_apply_prefix<<<(unsigned)blocks, 256, block_delta_smem(g.K()), s>>>(
        I_node, I_from, I_to, best, g.vwgt, part0, (unsigned long long *)C0, g.K(), (long long *)cut);
    UPR_LAUNCH_CHECK();
}

void table_rollback(const GraphDev &g, const Rollback &rb, int64_t max, const int32_t *pos, int32_t *W,
                    const HubChunk *hub_chunks, int64_t n_chunks, int64_t *deg_sum, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(deg_sum, 0, sizeof(int64_t), s));
    if (max <= 0) return;
    k_rollback_degsum<<<grid_for(max), 256, 0, s>>>(rb, g.xadj, (unsigned long long *)deg_sum);
    UPR_LAUNCH_CHECK();
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(max * 32, 256), (int64_t)device_sm_count() * 16);
    k_table_rollback<<<blocks, 256, 0, s>>>(rb, g.xadj, g.adj, g.adjw, g.k, g.kmask, W, deg_sum, g.m,
                                                      g.sp);
    UPR_LAUNCH_CHECK();
    if (n_chunks > 0) {
        k_table_rollback_hubs<<<(unsigned)n_chunks, 512, 0, s>>>(rb, hub_chunks, pos, g.adj, g.adjw, g.k, g.kmask, W,
                                                                 deg_sum, g.m, g.sp);
        UPR_LAUNCH_CHECK();
    }
}

void seq_append(const int32_t *M_node, const int32_t *M_from, const int32_t *M_to, const int32_t *d_nM,
                const int32_t *R_node, const int32_t *R_from, const int32_t *R_to, const int32_t *d_nR, int64_t max,
                int32_t *X_node, int32_t *X_from, int32_t *X_to, int8_t *X_isr, cudaStream_t s) {
    if (max <= 0) return;
    k_seq_append<<<grid_for(max), 256, 0, s>>>(M_node, M_from, M_to, d_nM, R_node, R_from, R_to, d_nR, X_node, X_from,
                                              X_to, X_isr);
    UPR_LAUNCH_CHECK();
}

void guard_locks(const Rollback &rb, int64_t max, int64_t n, const int32_t *m_pos, const int32_t *r_to,
                 int8_t *locked, cudaStream_t s) {
    if (n > 0) UPR_CUDA(cudaMemsetAsync(locked, 0, (size_t)n, s));
    if (max <= 0) return;
    k_guard_locks<<<grid_for(max), 256, 0, s>>>(rb, m_pos, r_to, locked);
    UPR_LAUNCH_CHECK();
}

void guard_filter(const int8_t *locked, int64_t n, int32_t *flags, int32_t *cand_tgt, int64_t *cand_s0,
                  int32_t *cand_gain, cudaStream_t s) {
    if (n <= 0) return;
    k_guard_filter<<<grid_for(n), 256, 0, s>>>(locked, n, flags, cand_tgt, cand_s0, cand_gain);
    UPR_LAUNCH_CHECK();
}

void seq_sort_by_graph(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
                       const int32_t *d_nI, int64_t max, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                       uint32_t *vals_alt, Scratch tmp, int32_t *O_node, int32_t *O_from, int32_t *O_to, int32_t *pos,
                       int32_t *dest, int32_t *seg_beg, int32_t *seg_end, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(seg_beg, 0, sizeof(int32_t) * g.ng, s));
    UPR_CUDA(cudaMemsetAsync(seg_end, 0, sizeof(int32_t) * g.ng, s));
    if (max <= 0) return;
    k_i_graph_keys<<<grid_for(max), 256, 0, s>>>(I_node, d_nI, g.gid, keys, vals);
    UPR_LAUNCH_CHECK();
    int gbits = 1;
    while ((1ll << gbits) < g.ng) gbits++;
    const bool alt = radix_sort_pairs(keys, vals, keys_alt, vals_alt, Count{d_nI, max}, gbits, tmp, s);
    k_i_permute<<<grid_for(max), 256, 0, s>>>(alt ? vals_alt : vals, alt ? keys_alt : keys, d_nI, I_node, I_from, I_to,
                                              O_node, O_from, O_to, pos, dest, seg_beg, seg_end);
    UPR_LAUNCH_CHECK();
}

void seq_best_seg(const GraphDev &g, const int32_t *I_node, const int32_t *d_nI, int64_t max, const int32_t *seg_beg,
                  const int64_t *Gsum, const int32_t *diff, const int32_t *diff_excl, const int32_t *over0,
                  long long *best_g, long long *best_j, int64_t *cut, int32_t *infeasible, int64_t *tot,
                  cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(tot, 0, 3 * sizeof(int64_t), s));
    k_best_seg_init<<<grid_for(g.ng), 256, 0, s>>>(over0, g.ng, best_g, best_j);
    UPR_LAUNCH_CHECK();
    if (max > 0) {
        k_best_seg_max<<<grid_for(max), 256, 0, s>>>(I_node, d_nI, g.gid, seg_beg, Gsum, diff, diff_excl, over0, best_g);
        UPR_LAUNCH_CHECK();
        k_best_seg_min<<<grid_for(max), 256, 0, s>>>(I_node, d_nI, g.gid, seg_beg, Gsum, diff, diff_excl, over0, best_g,
                                                     best_j);
        UPR_LAUNCH_CHECK();
    }
    k_best_seg_final<<<grid_for(g.ng), 256, 0, s>>>(over0, g.ng, best_g, best_j, (long long *)cut, infeasible,
                                                    (unsigned long long *)tot);
    UPR_LAUNCH_CHECK();
}

void seq_apply_prefix_seg(const GraphDev &g, const int32_t *I_node, const int32_t *I_from, const int32_t *I_to,
                          const int32_t *d_nI, int64_t max, const int32_t *seg_beg, const long long *best_j,
                          int32_t *part0, int64_t *C0, cudaStream_t s) {
    if (max <= 0) return;
    const int64_t blocks = std::min<int64_t>(ceil_div(max, 256), (int64_t)device_sm_count() * 4);
    k_apply_prefix_seg<<<(unsigned)blocks, 256, block_delta_smem(g.K()), s>>>(
        I_node, I_from, I_to, d_nI, g.gid, seg_beg, best_j, g.vwgt, part0, (unsigned long long *)C0, g.K());
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
