// Unconstrained label propagation (Sec. 5): the kernels of one round that the
// FM round does not already have.  The round itself (selection without a
// penalty, rebalancing, the net-improvement check) is driven from engine.cu.
#include "kernels.h"

namespace upr {
namespace {

// V_a of the first round: the boundary nodes, omega(v, V_P(v)) < omega(I(v)).
__global__ void k_lp_boundary(const GraphDev g, const int32_t *__restrict__ part, const int32_t *__restrict__ W,
                              int8_t *__restrict__ active) {
    UPR_FOR(v, g.n) {
        const int32_t wI = g.wI[v];
        const int32_t a = blk_local(g, part[v]);
        const int32_t own = wI == 0 ? 0 : g.sp.on() ? sp_get(g.sp, v, a) : W[v * (int64_t)g.k + a];
        active[v] = own < wI ? 1 : 0;
    }
}

// a node outside V_a does not move
__global__ void k_lp_filter(int32_t *__restrict__ flags, const int8_t *__restrict__ active, int64_t n) {
    UPR_FOR(v, n) if (flags[v] && !active[v]) flags[v] = 0;
}

// All moves at once: the listed nodes (node order) to their targets; the move
// list M (for the table update and the markers), block weights, and the
// degree sum of the moved nodes (delta update or rebuild).
__global__ void k_lp_apply(const int32_t *__restrict__ movers, const int32_t *__restrict__ d_cnt,
                           const int32_t *__restrict__ cand_tgt, const int32_t *__restrict__ cand_gain,
                           const int32_t *__restrict__ vwgt, const int64_t *__restrict__ xadj,
                           const int32_t *__restrict__ part0, int32_t *__restrict__ part,
                           unsigned long long *__restrict__ C, int32_t K, int32_t *__restrict__ M_node,
                           int32_t *__restrict__ M_from, int32_t *__restrict__ M_to, int64_t *__restrict__ M_score,
                           int32_t *__restrict__ m_pos, unsigned long long *__restrict__ deg_sum) {
    extern __shared__ unsigned long long s_delta[];
    BlockDelta bd = make_block_delta(s_delta, K, C);
    bd.init();
    const int64_t cnt = *d_cnt;
    long long degs = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < cnt; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        int32_t a = -1, b = -1;
        long long c = 0;
        if (p < cnt) {
            const int32_t v = movers[p];
            a = part0[v];
            b = cand_tgt[v];
            c = vwgt ? vwgt[v] : 1;
            M_node[p] = v;
            M_from[p] = a;
            M_to[p] = b;
            M_score[p] = cand_gain[v];
            m_pos[v] = (int32_t)p;
            part[v] = b;
            degs += xadj[v + 1] - xadj[v];
        }
        bd.add(a, -c);
        bd.add(b, c);
    }
    bd.flush(C);
    degs = warp_sum(degs);
    if ((threadIdx.x & 31) == 0 && degs) atomicAdd(deg_sum, (unsigned long long)degs);
}

// V_a of the next round: the neighbours of the nodes whose block changed that
// did not change block themselves.  One byte per node holds the state: 2
// moved, 1 unmoved with a moved neighbour, 0 otherwise; then the bytes
// become the 0/1 markers.  With few moved nodes the moved nodes push (their
// rows, from the round's two move lists: a node in both, or moved back, is
// looked at twice or skipped); with more than a quarter of the nodes moved
// the unmoved nodes pull (their rows until the first moved neighbour).  Hubs'
// rows go by their chunks, a CTA each.
__global__ void k_lp_state(const int32_t *__restrict__ before, const int32_t *__restrict__ after, int64_t n,
                           int8_t *__restrict__ state, int32_t *__restrict__ d_moved) {
    int32_t c = 0;
    UPR_FOR(v, n) {
        const bool moved = before[v] != after[v];
        state[v] = moved ? 2 : 0;
        c += moved;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(d_moved, c);
}

__global__ void __launch_bounds__(256) k_lp_mark(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                                                 int64_t n, const int32_t *__restrict__ nodes1,
                                                 const int32_t *__restrict__ d_cnt1,
                                                 const int32_t *__restrict__ nodes2,
                                                 const int32_t *__restrict__ d_cnt2,
                                                 const HubChunk *__restrict__ chunks, int64_t n_chunks,
                                                 const int32_t *__restrict__ d_moved, int8_t *state) {
    const bool pull = 4 * (int64_t)*d_moved > n;           // uniform over the grid
    const int lane = threadIdx.x & 31;
    __shared__ int s_hit;
    for (int64_t ci = blockIdx.x; ci < n_chunks; ci += gridDim.x) {
        const HubChunk ch = chunks[ci];
        const int8_t sh = state[ch.v];
        if (pull ? sh == 2 : sh != 2) continue;            // uniform over the CTA
        if (threadIdx.x == 0) s_hit = 0;
        __syncthreads();
        int hit = 0;
        for (int64_t e = ch.begin + threadIdx.x; e < ch.end; e += blockDim.x) {
            const int32_t u = adj[e];
            const int8_t su = state[u];
            if (pull) hit |= su == 2;
            else if (su == 0) state[u] = 1;
        }
        if (pull && hit) s_hit = 1;
        __syncthreads();
        if (pull && threadIdx.x == 0 && s_hit && state[ch.v] == 0) state[ch.v] = 1;
    }
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pull) {
        // 32 consecutive nodes per warp; the unmoved ones scan their rows in turn
        for (int64_t base = w0 * 32; base < n; base += warps * 32) {
            const int64_t v = base + lane;
            uint32_t todo = __ballot_sync(0xffffffffu, v < n && state[v] == 0);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t x = base + src;
                const int64_t e0 = xadj[x], e1 = xadj[x + 1];
                if (e1 - e0 > kHubDegree) continue;         // its chunks above
                bool found = false;
                for (int64_t e = e0; e < e1 && !found; e += 32)
                    found = __any_sync(0xffffffffu, e + lane < e1 && state[adj[e + lane]] == 2);
                if (found && lane == 0) state[x] = 1;
            }
        }
        return;
    }
    // 32 listed nodes per warp, spread over the list (neighbouring ids can
    // share high degrees), their rows (non-hub, moved) in turn
    const int64_t c1 = *d_cnt1, c2 = *d_cnt2;
    for (int64_t base = w0; base < c1 + c2; base += warps * 32) {
        const int64_t j = base + lane * warps;
        int64_t e0 = 0, e1 = 0;
        if (j < c1 + c2) {
            const int32_t v = j < c1 ? nodes1[j] : nodes2[j - c1];
            if (state[v] == 2) {
                e0 = xadj[v];
                e1 = xadj[v + 1];
                if (e1 - e0 > kHubDegree) e1 = e0;          // its chunks above
            }
        }
        uint32_t todo = __ballot_sync(0xffffffffu, e1 > e0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t a = __shfl_sync(0xffffffffu, e0, src), b = __shfl_sync(0xffffffffu, e1, src);
            for (int64_t e = a + lane; e < b; e += 32) {
                const int32_t u = adj[e];
                if (state[u] == 0) state[u] = 1;
            }
        }
    }
}

// The states become the markers (1 for state 1, else 0); *out += their number.
__global__ void k_lp_final(int8_t *__restrict__ state, int64_t n, int32_t *__restrict__ out) {
    __shared__ int32_t s_c[8];
    int32_t c = 0;
    UPR_FOR(i, n) {
        const int8_t m = state[i] == 1 ? 1 : 0;
        state[i] = m;
        c += m;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) c += s_c[w];
        if (c) atomicAdd(out, c);
    }
}

// *out += the number of non-zero entries (one atomic per CTA)
__global__ void k_count_i8(const int8_t *__restrict__ a, int64_t n, int32_t *__restrict__ out) {
    __shared__ int32_t s_c[8];
    int32_t c = 0;
    UPR_FOR(i, n) c += a[i] != 0;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) c += s_c[w];
        if (c) atomicAdd(out, c);
    }
}

}  // namespace

void lp_boundary(const GraphDev &g, const int32_t *part, const int32_t *W, int8_t *active, cudaStream_t s) {
    if (g.n == 0) return;
    k_lp_boundary<<<grid_for(g.n), 256, 0, s>>>(g, part, W, active);
    UPR_LAUNCH_CHECK();
}

void lp_filter(int32_t *flags, const int8_t *active, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    k_lp_filter<<<grid_for(n), 256, 0, s>>>(flags, active, n);
    UPR_LAUNCH_CHECK();
}

void lp_apply(const GraphDev &g, const int32_t *movers, const int32_t *d_cnt, const int32_t *cand_tgt,
              const int32_t *cand_gain, const int32_t *part0, int32_t *part, int64_t *C, int32_t *M_node,
              int32_t *M_from, int32_t *M_to, int64_t *M_score, int32_t *m_pos, int64_t *deg_sum, int64_t max_count,
              cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(deg_sum, 0, sizeof(int64_t), s));
    if (max_count <= 0) return;
    const int32_t K = g.K();
    const size_t shm = block_delta_smem(K);
    const int64_t blocks = std::min<int64_t>(ceil_div(max_count, 256), (int64_t)device_sm_count() * 4);
    k_lp_apply<<<(unsigned)blocks, 256, shm, s>>>(movers, d_cnt, cand_tgt, cand_gain, g.vwgt, g.xadj, part0, part,
                                                  (unsigned long long *)C, K, M_node, M_from, M_to, M_score, m_pos,
                                                  (unsigned long long *)deg_sum);
    UPR_LAUNCH_CHECK();
}

void lp_next(const GraphDev &g, const int32_t *before, const int32_t *after, const int32_t *nodes1,
             const int32_t *d_cnt1, const int32_t *nodes2, const int32_t *d_cnt2, const HubChunk *hub_chunks,
             int64_t n_chunks, int8_t *next, int32_t *d_count, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s));
    if (g.n == 0) return;
    k_lp_state<<<grid_for(g.n), 256, 0, s>>>(before, after, g.n, next, d_count);
    UPR_LAUNCH_CHECK();
    const int64_t blocks = std::max<int64_t>(std::min<int64_t>(ceil_div(g.n, 256), (int64_t)device_sm_count() * 8),
                                             std::min<int64_t>(n_chunks, (int64_t)device_sm_count() * 8));
    k_lp_mark<<<(unsigned)blocks, 256, 0, s>>>(g.xadj, g.adj, g.n, nodes1, d_cnt1, nodes2, d_cnt2, hub_chunks,
                                               n_chunks, d_count, next);
    UPR_LAUNCH_CHECK();
    UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s));
    k_lp_final<<<grid_for(g.n), 256, 0, s>>>(next, g.n, d_count);
    UPR_LAUNCH_CHECK();
}

void lp_count(const int8_t *active, int64_t n, int32_t *d_count, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s));
    if (n == 0) return;
    k_count_i8<<<grid_for(n), 256, 0, s>>>(active, n, d_count);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
