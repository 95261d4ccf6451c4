// Delta update of the gain table after moves (Sec. 6.2: when a node moves,
// its neighbours' entries in the gain table change): for every neighbour u of
// a node v moved from block a to block b, W[u][a] -= w(u, v) and
// W[u][b] += w(u, v), with integer atomics, so the result does not depend on
// their order.
#include "kernels.h"

namespace upr {
namespace {

// Delta update: warp per moved node; hubs (degree > kHubDegree) are left to
// k_table_move_hubs, which splits them into the static chunks.
__global__ void k_table_move(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                             const int32_t *__restrict__ adjw, int32_t k, int32_t kmask, int32_t *__restrict__ W,
                             const int32_t *__restrict__ nodes, const int32_t *__restrict__ from,
                             const int32_t *__restrict__ to, const int32_t *__restrict__ d_count,
                             const int32_t *__restrict__ d_offset, const int64_t *__restrict__ deg_sum, int64_t m,
                             SparseRows sp) {
    if (deg_sum && *deg_sum * 4 >= m) return;     // a rebuild handles this case
    const int lane = threadIdx.x & 31;
    const int64_t cnt = *d_count;
    const int64_t off = d_offset ? *d_offset : 0;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t v = nodes[off + j];
        const int32_t a = blk_local(from[off + j], k, kmask), b = blk_local(to[off + j], k, kmask);
        const int64_t e0 = xadj[v], e1 = xadj[v + 1];
        if (e1 - e0 > kHubDegree) continue;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t w = adjw ? adjw[e] : 1;
            const int32_t u = adj[e];
            if (sp.on()) {
                sp_sub(sp, u, a, w);
                sp_add(sp, u, b, w);
                continue;
            }
            int32_t *row = W + (int64_t)u * k;
            atomicSub(&row[a], w);
            atomicAdd(&row[b], w);
        }
    }
}

// Moved hubs over the static chunks.  A hub moved in M has m_pos >= 0 (from
// its round-start block to its M target); a hub moved in the current
// rebalancing sub-round has an R index in [*r_base, *r_base + *r_count).
// CTA c owns chunks c, c + gridDim.x, ...: its threads test those chunks at
// once, then the whole CTA updates the rows of each moved one, so a call with
// no moved hub costs one wave of tests.
__device__ __forceinline__ bool hub_moved(int32_t v, const HubMoves &hm, int32_t k, int32_t kmask, int32_t *a,
                                          int32_t *b) {
    if (hm.m_pos) {
        const int32_t p = hm.m_pos[v];
        if (p < 0) return false;
        *a = blk_local(hm.from[p], k, kmask);
        *b = blk_local(hm.to[p], k, kmask);
        return true;
    }
    if (hm.r_to[v] < 0) return false;
    const int32_t ri = hm.r_at[v], base = *hm.r_base;
    if (ri < base || ri >= base + *hm.r_count) return false;
    *a = blk_local(hm.from[ri], k, kmask);
    *b = blk_local(hm.to[ri], k, kmask);
    return true;
}

__global__ void __launch_bounds__(512) k_table_move_hubs(const HubChunk *__restrict__ chunks, int64_t n_chunks,
                                                         const int32_t *__restrict__ adj,
                                                         const int32_t *__restrict__ adjw, int32_t k,
                                                         int32_t kmask, int32_t *__restrict__ W, HubMoves hm,
                                                         const int64_t *__restrict__ deg_sum, int64_t m,
                                                         SparseRows sp) {
    if (deg_sum && *deg_sum * 4 >= m) return;
    __shared__ int s_cnt;
    __shared__ int64_t s_ci[512];
    __shared__ int32_t s_a[512], s_b[512];
    const int64_t stride = gridDim.x;
    for (int64_t j0 = 0; (int64_t)blockIdx.x + j0 * stride < n_chunks; j0 += blockDim.x) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const int64_t ci = (int64_t)blockIdx.x + (j0 + threadIdx.x) * stride;
        int32_t a, b;
        if (ci < n_chunks && hub_moved(chunks[ci].v, hm, k, kmask, &a, &b)) {
            const int q = atomicAdd(&s_cnt, 1);
            s_ci[q] = ci;
            s_a[q] = a;
            s_b[q] = b;
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int q = 0; q < cnt; q++) {
            const HubChunk ch = chunks[s_ci[q]];
            const int32_t qa = s_a[q], qb = s_b[q];
            for (int64_t e = ch.begin + threadIdx.x; e < ch.end; e += blockDim.x) {
                const int32_t w = adjw ? adjw[e] : 1;
                const int32_t u = adj[e];
                if (sp.on()) {
                    sp_sub(sp, u, qa, w);
                    sp_add(sp, u, qb, w);
                    continue;
                }
                int32_t *row = W + (int64_t)u * k;
                atomicSub(&row[qa], w);
                atomicAdd(&row[qb], w);
            }
        }
        __syncthreads();
    }
}

// Both in one launch (256 threads): the CTA's share of the hub chunks as in
// k_table_move_hubs, then its share of the other moved nodes as in
// k_table_move (the updates are integer atomics: their order does not matter).
__global__ void __launch_bounds__(256) k_table_move_all(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj,
                                                        const int32_t *__restrict__ adjw, int32_t k, int32_t kmask,
                                                        int32_t *__restrict__ W, const int32_t *__restrict__ nodes,
                                                        const int32_t *__restrict__ from, const int32_t *__restrict__ to,
                                                        const int32_t *__restrict__ d_count,
                                                        const int32_t *__restrict__ d_offset,
                                                        const int64_t *__restrict__ deg_sum, int64_t m, SparseRows sp,
                                                        const HubChunk *__restrict__ chunks, int64_t n_chunks,
                                                        HubMoves hm) {
    if (deg_sum && *deg_sum * 4 >= m) return;     // a rebuild handles this case
    __shared__ int s_cnt;
    __shared__ int64_t s_ci[256];
    __shared__ int32_t s_a[256], s_b[256];
    const int64_t stride = gridDim.x;
    for (int64_t j0 = 0; (int64_t)blockIdx.x + j0 * stride < n_chunks; j0 += blockDim.x) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const int64_t ci = (int64_t)blockIdx.x + (j0 + threadIdx.x) * stride;
        int32_t a, b;
        if (ci < n_chunks && hub_moved(chunks[ci].v, hm, k, kmask, &a, &b)) {
            const int q = atomicAdd(&s_cnt, 1);
            s_ci[q] = ci;
            s_a[q] = a;
            s_b[q] = b;
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int q = 0; q < cnt; q++) {
            const HubChunk ch = chunks[s_ci[q]];
            const int32_t qa = s_a[q], qb = s_b[q];
            for (int64_t e = ch.begin + threadIdx.x; e < ch.end; e += blockDim.x) {
                const int32_t w = adjw ? adjw[e] : 1;
                const int32_t u = adj[e];
                if (sp.on()) {
                    sp_sub(sp, u, qa, w);
                    sp_add(sp, u, qb, w);
                    continue;
                }
                int32_t *row = W + (int64_t)u * k;
                atomicSub(&row[qa], w);
                atomicAdd(&row[qb], w);
            }
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t cnt = *d_count;
    const int64_t off = d_offset ? *d_offset : 0;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t v = nodes[off + j];
        const int32_t a = blk_local(from[off + j], k, kmask), b = blk_local(to[off + j], k, kmask);
        const int64_t e0 = xadj[v], e1 = xadj[v + 1];
        if (e1 - e0 > kHubDegree) continue;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t w = adjw ? adjw[e] : 1;
            const int32_t u = adj[e];
            if (sp.on()) {
                sp_sub(sp, u, a, w);
                sp_add(sp, u, b, w);
                continue;
            }
            int32_t *row = W + (int64_t)u * k;
            atomicSub(&row[a], w);
            atomicAdd(&row[b], w);
        }
    }
}

}  // namespace

void table_move(const GraphDev &g, int32_t *W, const int32_t *nodes, const int32_t *from, const int32_t *to,
                const int32_t *d_count, const int32_t *d_offset, const int64_t *deg_sum, int64_t max_count,
                const HubChunk *hub_chunks, int64_t n_chunks, HubMoves hm, cudaStream_t s) {
    if (max_count <= 0) return;
    int64_t blocks = std::min<int64_t>(ceil_div(max_count * 32, 256), (int64_t)device_sm_count() * 16);
    if (n_chunks > 0) {
        // one launch for the hubs and the other nodes, on at least one wave
        const unsigned wave = wave_grid((const void *)k_table_move_all, 256, 0, (int64_t)1 << 40);
        const unsigned grid = (unsigned)std::max<int64_t>(blocks, std::min<int64_t>(wave, n_chunks));
        k_table_move_all<<<grid, 256, 0, s>>>(g.xadj, g.adj, g.adjw, g.k, g.kmask, W, nodes, from, to, d_count,
                                              d_offset, deg_sum, g.m, g.sp, hub_chunks, n_chunks, hm);
        UPR_LAUNCH_CHECK();
        return;
    }
    k_table_move<<<(unsigned)blocks, 256, 0, s>>>(g.xadj, g.adj, g.adjw, g.k, g.kmask, W, nodes, from, to, d_count,
                                                  d_offset, deg_sum, g.m, g.sp);
    UPR_LAUNCH_CHECK();
    if (n_chunks > 0) {
        const unsigned grid = wave_grid((const void *)k_table_move_hubs, 512, 0, n_chunks);
        k_table_move_hubs<<<grid, 512, 0, s>>>(hub_chunks, n_chunks, g.adj, g.adjw, g.k, g.kmask, W, hm, deg_sum,
                                               g.m, g.sp);
        UPR_LAUNCH_CHECK();
    }
}

}  // namespace upr
