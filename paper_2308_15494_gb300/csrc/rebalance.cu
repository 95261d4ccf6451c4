// Step (d): rebalancing (Sec. 6) in synchronous sub-rounds.  Per sub-round:
// every node of an overloaded block proposes its best-gain move into a block
// that stays within L_max (unconnected nodes: the lightest block, Sec. 6.1);
// proposals are ordered by the priority of Sec. 6.1 (g * c(u) for g >= 0,
// g / c(u) for g < 0, higher first, ties by node id) through an exact integer
// key; each source keeps the minimal prefix that removes its excess; each
// target admits the longest prefix that fits.  engine.cu runs the loop, from
// the host or as one CUDA graph whose condition k_reb_continue sets.
#include <cstddef>

#include "kernels.h"

namespace upr {
namespace {

int sm_count_reb() {
    static int cnt = 0;
    if (!cnt) {
        int dev = 0;
        UPR_CUDA(cudaGetDevice(&dev));
        UPR_CUDA(cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev));
    }
    return cnt;
}

template <int G>
__global__ void __launch_bounds__(256) k_propose(const GraphDev g, const int32_t *__restrict__ list,
                                                 const int32_t *__restrict__ d_n1, const int32_t *__restrict__ part,
                                                 const int32_t *__restrict__ W, RebalState st,
                                                 int32_t *__restrict__ prop_tgt, int32_t *__restrict__ prop_gain,
                                                 int32_t *__restrict__ flags) {
    const int64_t n1 = *d_n1;
    const int32_t k = g.k;
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n1; base += (int64_t)gridDim.x * kGroups) {
        const int64_t i = base + gid;
        const int32_t v = i < n1 ? list[i] : 0;
        const int32_t ag = i < n1 ? part[v] : 0;
        const bool src = i < n1 && st.over[ag];
        const int32_t a = blk_local(g, ag), b0 = ag - a;
        int64_t best = 0;
        int32_t bt = -1;
        int32_t own = 0;
        int64_t c = 1;
        if (src) {
            const int32_t *row = W + (int64_t)v * k;
            own = row[a];
            c = g.vwgt ? g.vwgt[v] : 1;
            for (int b = gl; b < k; b += G) {
                const int32_t w = row[b];
                const int32_t gb = b0 + b;
                if (b == a || w <= 0 || st.excl[gb] || st.C[gb] + c > st.Lb[gb]) continue;
                const int64_t gain = (int64_t)w - own;
                if (bt < 0 || gain > best) { best = gain; bt = b; }
            }
        }
        int64_t s = best;
        int32_t id = bt;
        group_argmax<G>(s, id);
        if (i < n1 && gl == 0) {
            int32_t tgt = src && id >= 0 ? b0 + id : -1;
            int64_t gain = s;
            const int32_t light = src ? st.light[blk_graph(g, ag)] : -1;
            if (src && tgt < 0 && light >= 0 && st.C[light] + c <= st.Lb[light]) { tgt = light; gain = -(int64_t)own; }
            if (tgt >= 0) {
                prop_tgt[v] = tgt;
                prop_gain[v] = (int32_t)gain;
                if (st.lgain) { st.lgain[i] = (int32_t)gain; st.lsrc[i] = ag; }
            }
            flags[i] = tgt >= 0 ? 1 : 0;
        }
    }
}

__device__ __forceinline__ int32_t int4_at(const int4 &x, int c) {
    return c == 0 ? x.x : c == 1 ? x.y : c == 2 ? x.z : x.w;
}

// Proposals of the listed nodes (the nodes of blocks overloaded when
// rebalancing started; those that left them are skipped).  Vectorised rows
// as in selection; room(b) = L_max - C[b] for an allowed target, -1 for an
// excluded one, so one comparison c <= room(b) tests validity.  With one
// graph the rooms are staged in shared memory; in a batch each node reads its
// graph's blocks from global memory.
template <int G, int CH, bool EXACT, bool BATCH, bool PACK = false>
__global__ void __launch_bounds__(256) k_propose_vec(const GraphDev g, const int32_t *__restrict__ list,
                                                     const int32_t *__restrict__ d_n1,
                                                     const int32_t *__restrict__ part, const int32_t *__restrict__ W,
                                                     RebalState st, int32_t *__restrict__ prop_tgt,
                                                     int32_t *__restrict__ prop_gain, int32_t *__restrict__ flags) {
    // EXACT: k == 4 * G * CH, every lane's four blocks exist.  The room of an
    // excluded block (which includes every overloaded block, so the node's own
    // block) is -1, so "c <= room" alone decides whether a block may receive
    // the node; room is clamped to 2^31 - 1 since c < 2^31.
    const int64_t n1 = *d_n1;
    if (n1 == 0) return;
    const int32_t k = g.k;
    extern __shared__ int32_t s_room[];
    int8_t *s_over = reinterpret_cast<int8_t *>(s_room + k);
    if (!BATCH) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const int64_t room = st.Lb[i] - st.C[i];
            s_room[i] = st.excl[i] ? -1 : (int32_t)(room > 0x7fffffffLL ? 0x7fffffffLL : room);
            s_over[i] = st.over[i];
        }
        __syncthreads();
    }
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    // PACK (unit weights, one graph): the lane's columns that have room for a
    // node of weight 1, as a bit mask fixed for the launch, and a column's
    // score as one integer whose maximum is the largest omega, ties to the
    // smaller block
    uint32_t okm = 0;
    const int kb = st.pack_bits;
    const int32_t kmask = (1 << kb) - 1, lbase = kmask - 4 * gl;
    if (PACK) {
#pragma unroll
        for (int j = 0; j < CH; j++)
#pragma unroll
            for (int cc = 0; cc < 4; cc++) {
                const int b = 4 * (gl + G * j) + cc;
                if ((EXACT || b < k) && s_room[b] >= 1) okm |= 1u << (4 * j + cc);
            }
    }
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n1; base += (int64_t)gridDim.x * kGroups) {
        const int64_t i = base + gid;
        const int32_t v = i < n1 ? list[i] : 0;
        const int32_t ag = i < n1 ? part[v] : 0;
        const int32_t a = BATCH ? blk_local(g, ag) : ag, b0 = ag - a;
        const bool src = i < n1 && (BATCH ? st.over[ag] : s_over[a]);
        const int4 zero = make_int4(0, 0, 0, 0);
        int4 r[CH];
        // the row is loaded as soon as v is known, beside its block (a
        // listed node that is no longer a source ignores it)
        if (i < n1) {
            const int4 *row4 = reinterpret_cast<const int4 *>(W + (int64_t)v * k);
#pragma unroll
            for (int j = 0; j < CH; j++) {
                const int q = gl + G * j;
                r[j] = (EXACT || 4 * q < k) ? row4[q] : zero;
            }
        } else {
#pragma unroll
            for (int j = 0; j < CH; j++) r[j] = zero;
        }
        const int q4 = a >> 2;
        int32_t mine = 0;
#pragma unroll
        for (int j = 0; j < CH; j++)
            if (j == q4 / G) mine = int4_at(r[j], a & 3);
        const int32_t own = __shfl_sync(0xffffffffu, mine, gbase + (q4 % G));
        const int32_t c = src ? (g.vwgt ? g.vwgt[v] : 1) : 1;
        // best valid block: the largest omega(v, V_b) (gain = omega - own), ties to the smaller b
        int32_t bw = 0, bt = -1;
        if (PACK) {
            int32_t best = 0;
#pragma unroll
            for (int j = 0; j < CH; j++) {
#pragma unroll
                for (int cc = 0; cc < 4; cc++) {
                    const int32_t w = int4_at(r[j], cc);
                    const int32_t key = (w << kb) + (lbase - 4 * G * j - cc);
                    const bool ok = ((okm >> (4 * j + cc)) & 1u) && w > 0;
                    best = max(best, ok ? key : 0);
                }
            }
            for (int o = G / 2; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
            if (src && best > 0) { bw = best >> kb; bt = kmask - (best & kmask); }
        } else if (src) {
#pragma unroll
            for (int j = 0; j < CH; j++) {
#pragma unroll
                for (int cc = 0; cc < 4; cc++) {
                    const int b = 4 * (gl + G * j) + cc;
                    const int32_t w = int4_at(r[j], cc);
                    if ((!EXACT && b >= k) || w <= 0) continue;
                    int32_t room;
                    if (BATCH) {
                        const int64_t rm = st.Lb[b0 + b] - st.C[b0 + b];
                        room = st.excl[b0 + b] ? -1 : (int32_t)(rm > 0x7fffffffLL ? 0x7fffffffLL : rm);
                    } else {
                        room = s_room[b];
                    }
                    if (c > room) continue;
                    if (bt < 0 || w > bw) { bw = w; bt = b; }
                }
            }
        }
        int32_t id = bt;
        if (!PACK) group_argmax32<G>(bw, id);
        if (i < n1 && gl == 0) {
            int32_t tgt = src && id >= 0 ? b0 + id : -1;
            int32_t gain = bw - own;
            if (src && tgt < 0) {
                const int32_t light = st.light[BATCH ? blk_graph(g, ag) : 0];
                if (light >= 0) {
                    const int64_t lroom = st.Lb[light] - st.C[light];
                    if ((int64_t)c <= lroom) { tgt = light; gain = -own; }
                }
            }
            if (tgt >= 0) {
                prop_tgt[v] = tgt;
                prop_gain[v] = gain;
                if (st.lgain) { st.lgain[i] = gain; st.lsrc[i] = ag; }
            }
            flags[i] = tgt >= 0 ? 1 : 0;
        }
    }
}

// Proposals over the sparse table: G lanes per node walk the node's slots;
// the best valid block has the largest omega(v, V_b), ties to the smaller b.
template <int G>
__global__ void __launch_bounds__(256) k_propose_sparse(const GraphDev g, const int32_t *__restrict__ list,
                                                        const int32_t *__restrict__ d_n1,
                                                        const int32_t *__restrict__ part, RebalState st,
                                                        int32_t *__restrict__ prop_tgt, int32_t *__restrict__ prop_gain,
                                                        int32_t *__restrict__ flags) {
    const int64_t n1 = *d_n1;
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    const SparseRows &sp = g.sp;
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n1; base += (int64_t)gridDim.x * kGroups) {
        const int64_t i = base + gid;
        const int32_t v = i < n1 ? list[i] : 0;
        const int32_t ag = i < n1 ? part[v] : 0;
        const bool src = i < n1 && st.over[ag];
        const int32_t a = blk_local(g, ag), b0 = ag - a;
        int32_t bw = 0, bt = -1, own = 0;
        const int32_t c = src ? (g.vwgt ? g.vwgt[v] : 1) : 1;
        if (src) {
            own = sp_get(sp, v, a);
            for (int64_t q = sp.off[v] + gl; q < sp.off[v + 1]; q += G) {
                const int2 e = sp.slot[q];
                if (e.x == kEmpty || e.y <= 0) continue;
                const int32_t gb = b0 + e.x;
                if (st.excl[gb] || st.C[gb] + c > st.Lb[gb]) continue;
                if (bt < 0 || e.y > bw || (e.y == bw && e.x < bt)) { bw = e.y; bt = e.x; }
            }
        }
        int32_t id = bt;
        group_argmax32<G>(bw, id);
        if (i < n1 && gl == 0) {
            int32_t tgt = src && id >= 0 ? b0 + id : -1;
            int32_t gain = bw - own;
            if (src && tgt < 0) {
                const int32_t light = st.light[blk_graph(g, ag)];
                if (light >= 0 && (int64_t)c <= st.Lb[light] - st.C[light]) { tgt = light; gain = -own; }
            }
            if (tgt >= 0) {
                prop_tgt[v] = tgt;
                prop_gain[v] = gain;
                if (st.lgain) { st.lgain[i] = gain; st.lsrc[i] = ag; }
            }
            flags[i] = tgt >= 0 ? 1 : 0;
        }
    }
}

// list[i] = nodes of the blocks marked in `mark`
__global__ void k_flag_in_blocks(const int32_t *__restrict__ part, int64_t n, const int8_t *__restrict__ mark,
                                 int32_t *__restrict__ flags) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flags[v] = mark[part[v]] ? 1 : 0;
}

// ---- loop control.  One graph: one CTA each (K = k <= 4096).  A batch: a
// grid over the graphs, warp per graph; the last CTA to finish (ticket)
// updates the control block.
// Start of rebalancing: the blocks overloaded now are never targets.
__global__ void k_reb_init(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t K,
                           int8_t *__restrict__ excl, RebalCtl *__restrict__ ctl) {
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
        const bool o = C[b] > Lb[b];
        excl[b] = o ? 1 : 0;
        if (o) s_any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->active = 0;
        ctl->stopped = s_any ? 0 : 1;
        ctl->light = -1;
        ctl->subrounds = 0;
        ctl->nR = 0;
        ctl->n1_active = 0;
        ctl->flag = 0;
        ctl->ticket = 0;
    }
}

// The last CTA of a batch controller grid: true in thread 0 of that CTA.
__device__ __forceinline__ bool last_cta(RebalCtl *ctl) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_last) {
        __threadfence();
        return true;
    }
    return false;
}

__global__ void k_reb_init_batch(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t K,
                                 int8_t *__restrict__ excl, RebalCtl *__restrict__ ctl) {
    int any = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < K; b += gridDim.x * blockDim.x) {
        const bool o = C[b] > Lb[b];
        excl[b] = o ? 1 : 0;
        any |= o;
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&ctl->flag, 1);
    if (last_cta(ctl)) {
        const int f = atomicAdd(&ctl->flag, 0);
        ctl->active = 0;
        ctl->stopped = f ? 0 : 1;
        ctl->light = -1;
        ctl->subrounds = 0;
        ctl->nR = 0;
        ctl->n1_active = 0;
        ctl->flag = 0;
        ctl->ticket = 0;
    }
}

// Start of the next sub-round (h = the number run so far + 1): overloaded
// set, lightest allowed block, activity.
__global__ void k_reb_begin(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t k,
                            const int8_t *__restrict__ excl, int8_t *__restrict__ over, int8_t *__restrict__ reject,
                            const int32_t *__restrict__ d_n1, int32_t max_subrounds, RebalCtl *__restrict__ ctl,
                            cudaGraphConditionalHandle cond) {
    __shared__ int s_any;
    __shared__ long long s_w[256];
    __shared__ int s_b[256];
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    long long bw = 0;
    int bb = -1;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
        const bool o = C[b] > Lb[b];
        over[b] = o ? 1 : 0;
        reject[b] = 0;
        if (o) s_any = 1;
        if (!excl[b] && (bb < 0 || C[b] < bw)) { bw = C[b]; bb = b; }
    }
    s_w[threadIdx.x] = bw;
    s_b[threadIdx.x] = bb;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const int b2 = s_b[threadIdx.x + o];
            const long long w2 = s_w[threadIdx.x + o];
            const int b1 = s_b[threadIdx.x];
            if (b2 >= 0 && (b1 < 0 || w2 < s_w[threadIdx.x] || (w2 == s_w[threadIdx.x] && b2 < b1))) {
                s_b[threadIdx.x] = b2;
                s_w[threadIdx.x] = w2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int32_t h = ctl->subrounds + 1;
        const bool run = !ctl->stopped && s_any && h <= max_subrounds;
        ctl->active = run ? 1 : 0;
        if (!run) ctl->stopped = 1;
        if (run) ctl->subrounds = h;
        ctl->light = s_b[0];
        ctl->n1_active = run ? *d_n1 : 0;
        // a graph-resident loop whose body starts without this kernel: its condition
        if (cond) cudaGraphSetConditional(cond, run ? 1u : 0u);
    }
}

// Batch form: warp per graph.
__global__ void k_reb_begin_batch(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t k,
                                  int32_t ng, const int8_t *__restrict__ excl, int8_t *__restrict__ over,
                                  int8_t *__restrict__ reject, const int32_t *__restrict__ d_n1,
                                  int32_t max_subrounds, RebalCtl *__restrict__ ctl, int32_t *__restrict__ light) {
    const int lane = threadIdx.x & 31;
    int any = 0;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t bw = 0;
        int32_t bb = -1;
        for (int32_t j = lane; j < k; j += 32) {
            const int32_t b = (int32_t)g * k + j;
            const bool o = C[b] > Lb[b];
            over[b] = o ? 1 : 0;
            reject[b] = 0;
            any |= o;
            // lightest: smallest weight, ties to the smaller block (b grows with j)
            if (!excl[b] && (bb < 0 || C[b] < bw)) { bw = C[b]; bb = b; }
        }
        // argmin over the warp: negate weights for group_argmax (larger score wins, ties to smaller id)
        int64_t sc = -bw;
        group_argmax<32>(sc, bb);
        if (lane == 0) light[g] = bb;
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&ctl->flag, 1);
    if (last_cta(ctl)) {
        const int f = atomicAdd(&ctl->flag, 0);
        const int32_t h = ctl->subrounds + 1;
        const bool run = !ctl->stopped && f && h <= max_subrounds;
        ctl->active = run ? 1 : 0;
        if (!run) ctl->stopped = 1;
        if (run) ctl->subrounds = h;
        ctl->n1_active = run ? *d_n1 : 0;
        ctl->flag = 0;
        ctl->ticket = 0;
    }
}

// End of a sub-round: targets that rejected a move are excluded from now on;
// stop when nothing was admitted and no target was newly excluded, or when no
// block is overloaded any more (the next sub-round would find nothing to do).
__global__ void k_reb_end(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t K,
                          int8_t *__restrict__ excl, const int8_t *__restrict__ reject,
                          const int32_t *__restrict__ d_na, RebalCtl *__restrict__ ctl) {
    __shared__ int s_grew, s_over;
    if (threadIdx.x == 0) s_grew = 0, s_over = 0;
    __syncthreads();
    if (!ctl->active) return;
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
        if (reject[b] && !excl[b]) { excl[b] = 1; s_grew = 1; }
        if (C[b] > Lb[b]) s_over = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t na = *d_na;
        ctl->nR += na;
        if ((na == 0 && !s_grew) || !s_over) ctl->stopped = 1;
    }
}

__global__ void k_reb_end_batch(const int64_t *__restrict__ C, const int64_t *__restrict__ Lb, int32_t K,
                                int8_t *__restrict__ excl, const int8_t *__restrict__ reject,
                                const int32_t *__restrict__ d_na, RebalCtl *__restrict__ ctl) {
    if (!ctl->active) return;                 // uniform over the grid: no CTA takes a ticket
    int grew = 0, over = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < K; b += gridDim.x * blockDim.x) {
        if (reject[b] && !excl[b]) { excl[b] = 1; grew = 1; }
        if (C[b] > Lb[b]) over = 1;
    }
    if (__syncthreads_or(grew) && threadIdx.x == 0) atomicOr(&ctl->flag, 1);
    if (__syncthreads_or(over) && threadIdx.x == 0) atomicOr(&ctl->flag, 2);
    if (last_cta(ctl)) {
        const int f = atomicAdd(&ctl->flag, 0);
        const int32_t na = *d_na;
        ctl->nR += na;
        if ((na == 0 && !(f & 1)) || !(f & 2)) ctl->stopped = 1;
        ctl->flag = 0;
        ctl->ticket = 0;
    }
}

// Ascending key = descending priority.  Class 0 (g >= 0): (2^(gb+cb) - 1) - g*c.
// Class 1 (g < 0): 2^(gb+2cb) + floor(|g| * 2^(2cb) / c), exact for c < 2^cb.
// Equal priorities give equal keys; the stable sort then keeps node order.
// The key has 1 + gb + 2cb bits; up to 63 it is one word (prio_key), above
// it the 128-bit form (prio_key_wide) is sorted as two words, low word first.
__device__ __forceinline__ uint64_t prio_key(int64_t g, uint64_t c, int gbits, int cbits) {
    const int S = 2 * cbits;
    if (g >= 0) return ((1ull << (gbits + cbits)) - 1ull) - (uint64_t)g * c;
    const uint64_t num = ((uint64_t)(-g)) << S;
    return (1ull << (gbits + S)) | (c == 1 ? num : num / c);     // unit weights need no division
}

__device__ __forceinline__ unsigned __int128 prio_key_wide(int64_t g, uint64_t c, int gbits, int cbits) {
    typedef unsigned __int128 u128;
    const int S = 2 * cbits;
    if (g >= 0) return (u128)(((1ull << (gbits + cbits)) - 1ull) - (uint64_t)g * c);     // gb + cb <= 62
    const u128 num = ((u128)(uint64_t)(-g)) << S;
    return ((u128)1 << (gbits + S)) | (c == 1 ? num : num / (u128)c);
}

// gain_only (the variant of Sec. 7.2): the priority is the gain alone, the
// key of weight 1 (g >= 0 first by g, then g < 0 by |g|: g descending).
__global__ void k_prio_keys(const int32_t *__restrict__ P, const int32_t *__restrict__ d_np,
                            const int32_t *__restrict__ prop_gain, const int32_t *__restrict__ vwgt, int gbits,
                            int cbits, int gain_only, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t cnt = *d_np;
    UPR_FOR(i, cnt) {
        const int32_t u = P[i];
        keys[i] = prio_key(prop_gain[u], (vwgt && !gain_only) ? (uint64_t)vwgt[u] : 1ull, gbits, cbits);
        vals[i] = (uint32_t)i;
    }
}

// The two words of a wide key: the low words of the proposals in list order
// (sorted first), then the high words in the order of that sort (A0), whose
// stable sort completes the order.
__global__ void k_prio_keys_lo(const int32_t *__restrict__ P, const int32_t *__restrict__ d_np,
                               const int32_t *__restrict__ prop_gain, const int32_t *__restrict__ vwgt, int gbits,
                               int cbits, int gain_only, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t cnt = *d_np;
    UPR_FOR(i, cnt) {
        const int32_t u = P[i];
        keys[i] = (uint64_t)prio_key_wide(prop_gain[u], (vwgt && !gain_only) ? (uint64_t)vwgt[u] : 1ull, gbits, cbits);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_prio_keys_hi(const int32_t *__restrict__ P, const uint32_t *__restrict__ A0,
                               const int32_t *__restrict__ d_np, const int32_t *__restrict__ prop_gain,
                               const int32_t *__restrict__ vwgt, int gbits, int cbits, int gain_only,
                               uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t cnt = *d_np;
    UPR_FOR(j, cnt) {
        const uint32_t i = A0[j];
        const int32_t u = P[i];
        keys[j] = (uint64_t)(prio_key_wide(prop_gain[u], (vwgt && !gain_only) ? (uint64_t)vwgt[u] : 1ull, gbits,
                                           cbits) >> 64);
        vals[j] = i;
    }
}

// ---- prefilter of the proposals.  A source keeps the minimal prefix of its
// proposals (priority order) that covers its excess; that prefix is usually a
// few percent of them.  A coarse bin, non-decreasing in the key, splits each
// source's proposals into ranges: every proposal in a bin below the bin where
// the source's cumulative weight reaches the excess is in the prefix, none
// above it is, so only the proposals up to that bin need the exact ordering.
// Keeping them (in their order) and dropping the rest leaves every kept
// proposal with the same weight before it in its source's order.
// The bin of a proposal of gain g and weight c (c = 1 for the gain-only
// priority), from g and c directly so that it needs no key of any width.  It
// equals the bin of the key: class 0 keys bin by g*c (127 - g*c, larger values
// all in bin 0), class 1 keys by floor(|g| * 2^cb / c), the key's class-1
// part shifted right by cb (128 + that value, larger values all in bin 255).
__device__ __forceinline__ int prio_bin(int64_t g, uint64_t c, int cbits) {
    if (g >= 0) {
        const uint64_t v = (uint64_t)g * c;
        return 127 - (int)(v < 127ull ? v : 127ull);
    }
    const uint64_t r = (((uint64_t)(-g)) << cbits) / c;     // |g| < 2^31, cb <= 31
    return 128 + (int)(r < 127ull ? r : 127ull);
}

// Per source block, the weight of its proposals by bin.  The proposals are
// the listed nodes with a set flag.  Each CTA sums into a small shared hash
// table keyed by (block, bin) first (the weight piles up on a few bins of each
// block), then adds its entries to the global histogram.
constexpr int kHistSlots = 2048;
constexpr uint32_t kHistEmpty = 0xffffffffu;

__global__ void __launch_bounds__(256) k_prio_hist(const int32_t *__restrict__ list, const int32_t *__restrict__ d_n1,
                                                   const int32_t *__restrict__ flags,
                                                   const int32_t *__restrict__ prop_gain,
                                                   const int32_t *__restrict__ vwgt, const int32_t *__restrict__ part,
                                                   int gbits, int cbits, int gain_only,
                                                   unsigned long long *__restrict__ hist) {
    __shared__ uint32_t s_key[kHistSlots];
    __shared__ unsigned long long s_val[kHistSlots];
    for (int i = threadIdx.x; i < kHistSlots; i += blockDim.x) { s_key[i] = kHistEmpty; s_val[i] = 0; }
    __syncthreads();
    const int64_t n1 = *d_n1;
    UPR_FOR(i, n1) {
        if (flags && !flags[i]) continue;
        const int32_t u = list[i];
        const uint64_t c = vwgt ? (uint64_t)vwgt[u] : 1ull;
        const uint32_t key = (uint32_t)part[u] * kPrioBins + prio_bin(prop_gain[u], gain_only ? 1ull : c, cbits);
        uint32_t h = (key * 0x9E3779B1u) >> 21;          // 11 bits: kHistSlots
        bool done = false;
        for (int probe = 0; probe < 32 && !done; probe++) {
            uint32_t cur = s_key[h];
            if (cur == kHistEmpty) {
                cur = atomicCAS(&s_key[h], kHistEmpty, key);
                if (cur == kHistEmpty) cur = key;
            }
            if (cur == key) {
                atomicAdd(&s_val[h], (unsigned long long)c);
                done = true;
            }
            h = (h + 1) & (kHistSlots - 1);
        }
        if (!done) atomicAdd(&hist[key], (unsigned long long)c);   // crowded table: straight to the histogram
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistSlots; i += blockDim.x)
        if (s_key[i] != kHistEmpty) atomicAdd(&hist[s_key[i]], s_val[i]);
}

// Per overloaded source: the first bin where the cumulative weight reaches the
// excess C - L_max (the last bin when it never does); the histogram row is
// cleared for the next sub-round.  One CTA of kPrioBins threads per block.
__global__ void __launch_bounds__(kPrioBins) k_prio_cut(int32_t K, const int8_t *__restrict__ over,
                                                       const int64_t *__restrict__ C, const int64_t *__restrict__ Lb,
                                                       unsigned long long *__restrict__ hist,
                                                       int32_t *__restrict__ cut) {
    __shared__ unsigned long long s_warp[kPrioBins / 32];
    __shared__ int s_cut;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int32_t a = blockIdx.x; a < K; a += gridDim.x) {
        if (!over[a]) continue;                       // uniform over the CTA
        unsigned long long *row = hist + (int64_t)a * kPrioBins;
        const unsigned long long v = row[t];
        unsigned long long inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        if (t == 0) s_cut = kPrioBins - 1;
        __syncthreads();
        for (int w = 0; w < warp; w++) inc += s_warp[w];
        const unsigned long long excess = (unsigned long long)(C[a] - Lb[a]);
        if (inc >= excess) atomicMin(&s_cut, t);
        row[t] = 0;
        __syncthreads();
        if (t == 0) cut[a] = s_cut;
        __syncthreads();
    }
}

// keep[i]: listed node i proposes and its bin is not after its source's cut
__global__ void k_prio_keep(const int32_t *__restrict__ list, const int32_t *__restrict__ d_n1,
                            const int32_t *__restrict__ flags, const int32_t *__restrict__ prop_gain,
                            const int32_t *__restrict__ vwgt, const int32_t *__restrict__ part,
                            const int32_t *__restrict__ cut, int gbits, int cbits, int gain_only,
                            int32_t *__restrict__ keep) {
    const int64_t n1 = *d_n1;
    UPR_FOR(i, n1) {
        int32_t k = 0;
        if (!flags || flags[i]) {
            const int32_t u = list[i];
            const uint64_t c = vwgt ? (uint64_t)vwgt[u] : 1ull;
            k = prio_bin(prop_gain[u], gain_only ? 1ull : c, cbits) <= cut[part[u]] ? 1 : 0;
        }
        keep[i] = k;
    }
}

// Block-id key (source or target) of the entries listed through idx/order.
__global__ void k_block_keys(const int32_t *__restrict__ P, const uint32_t *__restrict__ A,
                             const int32_t *__restrict__ S, const int32_t *__restrict__ d_cnt,
                             const int32_t *__restrict__ blk_of_node, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
    const int64_t cnt = *d_cnt;
    UPR_FOR(i, cnt) {
        const int64_t j = S ? S[i] : i;
        const int32_t u = P[A[j]];
        keys[i] = (uint64_t)blk_of_node[u];
        vals[i] = (uint32_t)i;
    }
}

// For entries in block-sorted order: weights, and the first position of each block.
__global__ void k_seg_weights(const int32_t *__restrict__ P, const uint32_t *__restrict__ A,
                              const int32_t *__restrict__ S, const uint32_t *__restrict__ B,
                              const uint64_t *__restrict__ bkeys, const int32_t *__restrict__ d_cnt,
                              const int32_t *__restrict__ vwgt, int64_t *__restrict__ c_sorted,
                              int32_t *__restrict__ seg_first) {
    const int64_t cnt = *d_cnt;
    UPR_FOR(q, cnt) {
        const int64_t i = B[q];
        const int64_t j = S ? S[i] : i;
        const int32_t u = P[A[j]];
        c_sorted[q] = vwgt ? vwgt[u] : 1;
        const int32_t b = (int32_t)bkeys[q];
        if (q == 0 || (int32_t)bkeys[q - 1] != b) seg_first[b] = (int32_t)q;
    }
}

// Minimal prefix per source: entry selected iff the weight before it in its
// source's priority order is below the source's excess.
__global__ void k_mark_selected(const uint32_t *__restrict__ B, const uint64_t *__restrict__ bkeys,
                                const int32_t *__restrict__ d_cnt, const int64_t *__restrict__ c_excl,
                                const int32_t *__restrict__ seg_first, RebalState st, int32_t *__restrict__ sel) {
    const int64_t cnt = *d_cnt;
    UPR_FOR(q, cnt) {
        const int32_t b = (int32_t)bkeys[q];
        const int64_t before = c_excl[q] - c_excl[seg_first[b]];
        sel[B[q]] = before < st.C[b] - st.Lb[b] ? 1 : 0;
    }
}

// Longest fitting prefix per target; a rejected entry marks its target.
__global__ void k_mark_admitted(const uint32_t *__restrict__ T, const uint64_t *__restrict__ bkeys,
                                const int32_t *__restrict__ d_cnt, const int64_t *__restrict__ c_sorted,
                                const int64_t *__restrict__ c_excl, const int32_t *__restrict__ seg_first,
                                RebalState st, int32_t *__restrict__ adm, int8_t *__restrict__ reject) {
    const int64_t cnt = *d_cnt;
    UPR_FOR(q, cnt) {
        const int32_t t = (int32_t)bkeys[q];
        const int64_t incl = c_excl[q] - c_excl[seg_first[t]] + c_sorted[q];
        const bool ok = st.C[t] + incl <= st.Lb[t];
        adm[T[q]] = ok ? 1 : 0;
        if (!ok) reject[t] = 1;
    }
}

__global__ void k_apply_rebal(const int32_t *__restrict__ P, const uint32_t *__restrict__ A,
                              const int32_t *__restrict__ S, const int32_t *__restrict__ Adm,
                              const int32_t *__restrict__ d_na, const int32_t *__restrict__ prop_tgt,
                              const int32_t *__restrict__ vwgt, int32_t *__restrict__ part,
                              unsigned long long *__restrict__ C, int32_t K, const RebalCtl *__restrict__ ctl,
                              int32_t *__restrict__ R_node, int32_t *__restrict__ R_from,
                              int32_t *__restrict__ R_to, int32_t *__restrict__ R_sub, int32_t *__restrict__ r_to,
                              int32_t *__restrict__ r_at) {
    extern __shared__ unsigned long long s_delta[];
    BlockDelta bd = make_block_delta(s_delta, K, C);
    bd.init();
    const int64_t cnt = *d_na;
    const int64_t off = ctl->nR;
    const int32_t subround = ctl->subrounds;
    R_node += off; R_from += off; R_to += off; R_sub += off;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < cnt; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        int32_t a = -1, b = -1;
        long long c = 0;
        if (p < cnt) {
            const int32_t u = P[A[S[Adm[p]]]];
            a = part[u];
            b = prop_tgt[u];
            c = vwgt ? vwgt[u] : 1;
            R_node[p] = u;
            R_from[p] = a;
            R_to[p] = b;
            R_sub[p] = subround;
            r_to[u] = b;
            r_at[u] = (int32_t)(off + p);
            part[u] = b;
        }
        bd.add(a, -c);
        bd.add(b, c);
    }
    bd.flush(C);
}

inline unsigned grid1(int64_t n) { return (unsigned)ceil_div(n > 0 ? n : 1, 256); }

}  // namespace

int rebalance_group(int k) {
    int G = k / 4;
    return G >= 32 ? 32 : G >= 16 ? 16 : G >= 8 ? 8 : k >= 4 ? 4 : 2;
}

void rebalance_propose_scalar_list(const GraphDev &g, const int32_t *list, const int32_t *d_n1, int64_t n1_max,
                                   const int32_t *part, const int32_t *W, RebalState st, int32_t *prop_tgt,
                                   int32_t *prop_gain, int32_t *flags, cudaStream_t s) {
    if (n1_max <= 0) return;
    const int G = rebalance_group(g.k);
    const int64_t groups = 256 / G;
    const int64_t blocks = std::min<int64_t>(ceil_div(n1_max, groups), (int64_t)sm_count_reb() * 16);
#define UPR_PROP(GG) k_propose<GG><<<(unsigned)blocks, 256, 0, s>>>(g, list, d_n1, part, W, st, prop_tgt, prop_gain, \
                                                                    flags)
    switch (G) {
        case 2: UPR_PROP(2); break;
        case 4: UPR_PROP(4); break;
        case 8: UPR_PROP(8); break;
        case 16: UPR_PROP(16); break;
        default: UPR_PROP(32); break;
    }
#undef UPR_PROP
    UPR_LAUNCH_CHECK();
}

void rebalance_flag_in_blocks(const int32_t *part, int64_t n, const int8_t *mark, int32_t *flags, cudaStream_t s) {
    if (n <= 0) return;
    k_flag_in_blocks<<<grid1(n), 256, 0, s>>>(part, n, mark, flags);
    UPR_LAUNCH_CHECK();
}

namespace {

template <int G, int CH>
void launch_propose_vec(bool exact, bool batch, unsigned blocks, size_t shm, cudaStream_t s, const GraphDev &g,
                        const int32_t *list, const int32_t *d_n1, const int32_t *part, const int32_t *W,
                        const RebalState &st, int32_t *prop_tgt, int32_t *prop_gain, int32_t *flags) {
    // one full wave of CTAs at most (the kernel loops over the list)
    auto go = [&](auto kern) {
        kern<<<wave_grid((const void *)kern, 256, shm, blocks), 256, shm, s>>>(g, list, d_n1, part, W, st, prop_tgt,
                                                                             prop_gain, flags);
    };
    const bool pack = !batch && st.pack_bits > 0 && g.vwgt == nullptr;
    if constexpr (CH == 1 || (G == 32 && CH == 2)) {
        if (!exact) {
            if (batch) go(k_propose_vec<G, CH, false, true>);
            else if (pack) go(k_propose_vec<G, CH, false, false, true>);
            else go(k_propose_vec<G, CH, false, false>);
            return;
        }
    }
    if (batch) go(k_propose_vec<G, CH, true, true>);
    else if (pack) go(k_propose_vec<G, CH, true, false, true>);
    else go(k_propose_vec<G, CH, true, false>);
}

}  // namespace

void rebalance_propose_list(const GraphDev &g, const int32_t *list, const int32_t *d_n1, int64_t n1_max,
                            const int32_t *part, const int32_t *W, RebalState st, int32_t *prop_tgt,
                            int32_t *prop_gain, int32_t *flags, LaneCfg cfg, cudaStream_t s) {
    if (n1_max <= 0) return;
    const int k = g.k;
    const bool batch = g.ng > 1;
    if (g.sp.on()) {
        const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n1_max, 256 / 8), (int64_t)sm_count_reb() * 8);
        k_propose_sparse<8><<<blocks, 256, 0, s>>>(g, list, d_n1, part, st, prop_tgt, prop_gain, flags);
        UPR_LAUNCH_CHECK();
        return;
    }
    const size_t shm = batch ? 0 : sizeof(int32_t) * (size_t)k + (size_t)k + 16;
    LaneCfg cands[3];
    if (lane_candidates(k, cands) > 0) {
        if (cfg.G <= 0) cfg = cands[0];
        const int G = cfg.G, CH = cfg.CH;
        const bool exact = k == 4 * G * CH;
        const int64_t groups = 256 / G;
        const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n1_max, groups), (int64_t)sm_count_reb() * 8);
#define UPR_PVC(GG, CC)                                                                                        \
    if (G == GG && CH == CC) {                                                                                 \
        launch_propose_vec<GG, CC>(exact, batch, blocks, shm, s, g, list, d_n1, part, W, st, prop_tgt,         \
                                   prop_gain, flags);                                                          \
        UPR_LAUNCH_CHECK();                                                                                    \
        return;                                                                                                \
    }
        UPR_PVC(1, 1) UPR_PVC(2, 1) UPR_PVC(4, 1) UPR_PVC(8, 1) UPR_PVC(16, 1) UPR_PVC(32, 1)
        UPR_PVC(1, 2) UPR_PVC(2, 2) UPR_PVC(4, 2) UPR_PVC(8, 2) UPR_PVC(16, 2) UPR_PVC(32, 2)
        UPR_PVC(1, 4) UPR_PVC(2, 4) UPR_PVC(4, 4) UPR_PVC(8, 4) UPR_PVC(16, 4)
#undef UPR_PVC
        throw CudaError{cudaErrorInvalidValue, "rebalance_propose_list: unsupported lane schedule"};
    }
    rebalance_propose_scalar_list(g, list, d_n1, n1_max, part, W, st, prop_tgt, prop_gain, flags, s);
}

void rebalance_prefilter(const GraphDev &g, const int32_t *list, const int32_t *d_n1, int64_t n1_max,
                         const int32_t *flags, const int32_t *prop_gain, const int32_t *part, const int8_t *over,
                         const int64_t *C, int gbits, int cbits, int gain_only, unsigned long long *hist,
                         int32_t *cut, int32_t *keep, cudaStream_t s) {
    if (n1_max <= 0) return;
    const unsigned hist_grid = (unsigned)std::min<int64_t>(ceil_div(n1_max, 256), (int64_t)device_sm_count() * 4);
    k_prio_hist<<<hist_grid, 256, 0, s>>>(list, d_n1, flags, prop_gain, g.vwgt, part, gbits, cbits, gain_only,
                                          hist);
    UPR_LAUNCH_CHECK();
    k_prio_cut<<<(unsigned)std::min<int64_t>(g.K(), 4096), kPrioBins, 0, s>>>(g.K(), over, C, g.Lb, hist, cut);
    UPR_LAUNCH_CHECK();
    k_prio_keep<<<grid_for(n1_max), 256, 0, s>>>(list, d_n1, flags, prop_gain, g.vwgt, part, cut, gbits, cbits,
                                                 gain_only, keep);
    UPR_LAUNCH_CHECK();
}

void rebalance_prio_cut(const GraphDev &g, const int8_t *over, const int64_t *C, unsigned long long *hist, int32_t *cut,
                        cudaStream_t s) {
    k_prio_cut<<<(unsigned)std::min<int64_t>(g.K(), 4096), kPrioBins, 0, s>>>(g.K(), over, C, g.Lb, hist, cut);
    UPR_LAUNCH_CHECK();
}

void rebalance_prio_keys(const GraphDev &g, const int32_t *P, const int32_t *d_np, const int32_t *prop_gain,
                         int gbits, int cbits, int gain_only, uint64_t *keys, uint32_t *vals, int64_t np_max,
                         cudaStream_t s) {
    if (np_max <= 0) return;
    k_prio_keys<<<grid_for(np_max), 256, 0, s>>>(P, d_np, prop_gain, g.vwgt, gbits, cbits, gain_only, keys, vals);
    UPR_LAUNCH_CHECK();
}

void rebalance_prio_sort_wide(const GraphDev &g, const int32_t *P, const int32_t *d_np, const int32_t *prop_gain,
                              int gbits, int cbits, int gain_only, SortPairs sp, int64_t np_max, Scratch tmp,
                              cudaStream_t s, uint32_t **order) {
    if (np_max <= 0) { *order = sp.v; return; }
    const Count cnt{d_np, np_max};
    k_prio_keys_lo<<<grid_for(np_max), 256, 0, s>>>(P, d_np, prop_gain, g.vwgt, gbits, cbits, gain_only, sp.k, sp.v);
    UPR_LAUNCH_CHECK();
    // 64 bits = 8 passes, an even number: the result is back in (k, v)
    radix_sort_pairs(sp.k, sp.v, sp.ka, sp.va, cnt, 64, tmp, s);
    k_prio_keys_hi<<<grid_for(np_max), 256, 0, s>>>(P, sp.v, d_np, prop_gain, g.vwgt, gbits, cbits, gain_only, sp.ka,
                                                    sp.va);
    UPR_LAUNCH_CHECK();
    const bool alt = radix_sort_pairs(sp.ka, sp.va, sp.k, sp.v, cnt, 1 + gbits + 2 * cbits - 64, tmp, s);
    *order = alt ? sp.v : sp.va;
}

void rebalance_block_keys(const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *d_cnt,
                          const int32_t *blk_of_node, uint64_t *keys, uint32_t *vals, int64_t cnt_max, cudaStream_t s) {
    if (cnt_max <= 0) return;
    k_block_keys<<<grid_for(cnt_max), 256, 0, s>>>(P, A, S, d_cnt, blk_of_node, keys, vals);
    UPR_LAUNCH_CHECK();
}

void rebalance_seg_weights(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S,
                           const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, int64_t *c_sorted,
                           int32_t *seg_first, int64_t cnt_max, cudaStream_t s) {
    if (cnt_max <= 0) return;
    k_seg_weights<<<grid_for(cnt_max), 256, 0, s>>>(P, A, S, B, bkeys, d_cnt, g.vwgt, c_sorted, seg_first);
    UPR_LAUNCH_CHECK();
}

void rebalance_mark_selected(const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_excl,
                             const int32_t *seg_first, RebalState st, int32_t *sel, int64_t cnt_max, cudaStream_t s) {
    if (cnt_max <= 0) return;
    k_mark_selected<<<grid_for(cnt_max), 256, 0, s>>>(B, bkeys, d_cnt, c_excl, seg_first, st, sel);
    UPR_LAUNCH_CHECK();
}

void rebalance_mark_admitted(const uint32_t *T, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_sorted,
                             const int64_t *c_excl, const int32_t *seg_first, RebalState st, int32_t *adm,
                             int8_t *reject, int64_t cnt_max, cudaStream_t s) {
    if (cnt_max <= 0) return;
    k_mark_admitted<<<grid_for(cnt_max), 256, 0, s>>>(T, bkeys, d_cnt, c_sorted, c_excl, seg_first, st, adm, reject);
    UPR_LAUNCH_CHECK();
}

void rebalance_apply(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *Adm,
                     const int32_t *d_na, const int32_t *prop_tgt, int32_t *part, int64_t *C, const RebalCtl *ctl,
                     int32_t *R_node, int32_t *R_from, int32_t *R_to, int32_t *R_sub, int32_t *r_to, int32_t *r_at,
                     int64_t na_max, cudaStream_t s) {
    if (na_max <= 0) return;
    const int64_t blocks = std::min<int64_t>(ceil_div(na_max, 256), (int64_t)device_sm_count() * 4);
    k_apply_rebal<<<(unsigned)blocks, 256, block_delta_smem(g.K()), s>>>(
        P, A, S, Adm, d_na, prop_tgt, g.vwgt, part, (unsigned long long *)C, g.K(), ctl, R_node, R_from, R_to, R_sub,
        r_to, r_at);
    UPR_LAUNCH_CHECK();
}

// Grid of a batch controller: warp per graph (begin) or thread per block.
inline unsigned ctl_grid(int64_t items) {
    return (unsigned)std::min<int64_t>(ceil_div(items > 0 ? items : 1, 256), (int64_t)sm_count_reb() * 2);
}

// The batch controllers count finished CTAs in ctl->ticket and collect a flag
// in ctl->flag; both are cleared before every such launch, so nothing
// depends on what the control block held before.
inline void clear_ticket(RebalCtl *ctl, cudaStream_t s) {
    static_assert(offsetof(RebalCtl, ticket) == offsetof(RebalCtl, flag) + sizeof(int32_t), "flag, ticket adjacent");
    UPR_CUDA(cudaMemsetAsync(&ctl->flag, 0, sizeof(int32_t) + sizeof(uint32_t), s));
}

void rebalance_init(const GraphDev &g, const int64_t *C, int8_t *excl, RebalCtl *ctl, cudaStream_t s) {
    if (g.ng == 1) {
        k_reb_init<<<1, 256, 0, s>>>(C, g.Lb, g.K(), excl, ctl);
    } else {
        clear_ticket(ctl, s);
        k_reb_init_batch<<<ctl_grid(g.K()), 256, 0, s>>>(C, g.Lb, g.K(), excl, ctl);
    }
    UPR_LAUNCH_CHECK();
}

void rebalance_begin(const GraphDev &g, const int64_t *C, const int8_t *excl, int8_t *over, int8_t *reject,
                     const int32_t *d_n1, int32_t max_subrounds, RebalCtl *ctl, int32_t *light, cudaStream_t s,
                     cudaGraphConditionalHandle cond) {
    if (g.ng == 1) {
        k_reb_begin<<<1, 256, 0, s>>>(C, g.Lb, g.k, excl, over, reject, d_n1, max_subrounds, ctl, cond);
    } else {
        clear_ticket(ctl, s);
        k_reb_begin_batch<<<ctl_grid((int64_t)g.ng * 32), 256, 0, s>>>(C, g.Lb, g.k, g.ng, excl, over, reject, d_n1,
                                                                       max_subrounds, ctl, light);
    }
    UPR_LAUNCH_CHECK();
}

// The loop condition of the graph-resident rebalancing loop: run another
// sub-round while the loop has not stopped and sub-rounds are left.
__global__ void k_reb_continue(const RebalCtl *__restrict__ ctl, int32_t max_subrounds,
                               cudaGraphConditionalHandle handle) {
    if (threadIdx.x == 0)
        cudaGraphSetConditional(handle, (!ctl->stopped && ctl->subrounds < max_subrounds) ? 1u : 0u);
}

void rebalance_continue(const RebalCtl *ctl, int32_t max_subrounds, cudaGraphConditionalHandle handle,
                        cudaStream_t s) {
    k_reb_continue<<<1, 32, 0, s>>>(ctl, max_subrounds, handle);
    UPR_LAUNCH_CHECK();
}

void rebalance_end(const GraphDev &g, const int64_t *C, int8_t *excl, const int8_t *reject, const int32_t *d_na,
                   RebalCtl *ctl, cudaStream_t s) {
    if (g.ng == 1) {
        k_reb_end<<<1, 256, 0, s>>>(C, g.Lb, g.K(), excl, reject, d_na, ctl);
    } else {
        clear_ticket(ctl, s);
        k_reb_end_batch<<<ctl_grid(g.K()), 256, 0, s>>>(C, g.Lb, g.K(), excl, reject, d_na, ctl);
    }
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
