// Step (d): rebalancing (Sec. 6) in synchronous sub-rounds.  Per sub-round:
// every node of an overloaded block proposes its best-gain move into a block
// that stays within L_max (unconnected nodes: the lightest block, Sec. 6.1);
// proposals are ordered by the priority of Sec. 6.1 (g * c(u) for g >= 0,
// g / c(u) for g < 0, higher first, ties by node id) through an exact integer
// key; each source keeps the minimal prefix that removes its excess; each
// target admits the longest prefix that fits.  The host drives the loop.
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
__global__ void __launch_bounds__(256) k_propose(const int32_t *__restrict__ part, const int32_t *__restrict__ W,
                                                 const int32_t *__restrict__ vwgt, int64_t n, int32_t k,
                                                 RebalState st, int32_t *__restrict__ prop_tgt,
                                                 int32_t *__restrict__ prop_gain, int32_t *__restrict__ flags) {
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n; base += (int64_t)gridDim.x * kGroups) {
        const int64_t v = base + gid;
        const bool active = v < n;
        const int32_t a = active ? part[v] : 0;
        const bool src = active && st.over[a];
        int64_t best = 0;
        int32_t bt = -1;
        int32_t own = 0;
        int64_t c = 1;
        if (src) {
            const int32_t *row = W + v * (int64_t)k;
            own = row[a];
            c = vwgt ? vwgt[v] : 1;
            for (int b = gl; b < k; b += G) {
                const int32_t w = row[b];
                if (b == a || w <= 0 || st.excl[b] || st.C[b] + c > st.Lmax) continue;
                const int64_t gain = (int64_t)w - own;
                if (bt < 0 || gain > best) { best = gain; bt = b; }
            }
        }
        int64_t s = best;
        int32_t id = bt;
        group_argmax<G>(s, id);
        if (src && gl == 0) {
            int32_t tgt = id;
            int64_t gain = s;
            if (tgt < 0 && st.light >= 0 && st.C[st.light] + c <= st.Lmax) { tgt = st.light; gain = -(int64_t)own; }
            prop_tgt[v] = tgt;
            prop_gain[v] = (int32_t)gain;
            flags[v] = tgt >= 0 ? 1 : 0;
        } else if (active && gl == 0) {
            flags[v] = 0;
        }
    }
}

// Ascending key = descending priority.  Class 0 (g >= 0): (2^(gb+cb) - 1) - g*c.
// Class 1 (g < 0): floor(|g| * 2^(2cb) / c), exact for c < 2^cb.  Equal
// priorities give equal keys; the stable sort then keeps node order.
__global__ void k_prio_keys(const int32_t *__restrict__ P, const int32_t *__restrict__ d_np,
                            const int32_t *__restrict__ prop_gain, const int32_t *__restrict__ vwgt, int gbits,
                            int cbits, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *d_np) return;
    const int32_t u = P[i];
    const int64_t g = prop_gain[u];
    const uint64_t c = vwgt ? (uint64_t)vwgt[u] : 1ull;
    const int S = 2 * cbits;
    uint64_t key;
    if (g >= 0) {
        key = ((1ull << (gbits + cbits)) - 1ull) - (uint64_t)g * c;
    } else {
        key = (1ull << (gbits + S)) | ((((uint64_t)(-g)) << S) / c);
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

// Block-id key (source or target) of the entries listed through idx/order.
__global__ void k_block_keys(const int32_t *__restrict__ P, const uint32_t *__restrict__ A,
                             const int32_t *__restrict__ S, const int32_t *__restrict__ d_cnt,
                             const int32_t *__restrict__ blk_of_node, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *d_cnt) return;
    const int64_t j = S ? S[i] : i;
    const int32_t u = P[A[j]];
    keys[i] = (uint64_t)blk_of_node[u];
    vals[i] = (uint32_t)i;
}

// For entries in block-sorted order: weights, and the first position of each block.
__global__ void k_seg_weights(const int32_t *__restrict__ P, const uint32_t *__restrict__ A,
                              const int32_t *__restrict__ S, const uint32_t *__restrict__ B,
                              const uint64_t *__restrict__ bkeys, const int32_t *__restrict__ d_cnt,
                              const int32_t *__restrict__ vwgt, int64_t *__restrict__ c_sorted,
                              int32_t *__restrict__ seg_first) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= *d_cnt) return;
    const int64_t i = B[q];
    const int64_t j = S ? S[i] : i;
    const int32_t u = P[A[j]];
    c_sorted[q] = vwgt ? vwgt[u] : 1;
    const int32_t b = (int32_t)bkeys[q];
    if (q == 0 || (int32_t)bkeys[q - 1] != b) seg_first[b] = (int32_t)q;
}

// Minimal prefix per source: entry selected iff the weight before it in its
// source's priority order is below the source's excess.
__global__ void k_mark_selected(const uint32_t *__restrict__ B, const uint64_t *__restrict__ bkeys,
                                const int32_t *__restrict__ d_cnt, const int64_t *__restrict__ c_excl,
                                const int32_t *__restrict__ seg_first, RebalState st, int32_t *__restrict__ sel) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= *d_cnt) return;
    const int32_t b = (int32_t)bkeys[q];
    const int64_t before = c_excl[q] - c_excl[seg_first[b]];
    sel[B[q]] = before < st.C[b] - st.Lmax ? 1 : 0;
}

// Longest fitting prefix per target; a rejected entry marks its target.
__global__ void k_mark_admitted(const uint32_t *__restrict__ T, const uint64_t *__restrict__ bkeys,
                                const int32_t *__restrict__ d_cnt, const int64_t *__restrict__ c_sorted,
                                const int64_t *__restrict__ c_excl, const int32_t *__restrict__ seg_first,
                                RebalState st, int32_t *__restrict__ adm, int8_t *__restrict__ reject) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= *d_cnt) return;
    const int32_t t = (int32_t)bkeys[q];
    const int64_t incl = c_excl[q] - c_excl[seg_first[t]] + c_sorted[q];
    const bool ok = st.C[t] + incl <= st.Lmax;
    adm[T[q]] = ok ? 1 : 0;
    if (!ok) reject[t] = 1;
}

__global__ void k_apply_rebal(const int32_t *__restrict__ P, const uint32_t *__restrict__ A,
                              const int32_t *__restrict__ S, const int32_t *__restrict__ Adm,
                              const int32_t *__restrict__ d_na, const int32_t *__restrict__ prop_tgt,
                              const int32_t *__restrict__ vwgt, int32_t *__restrict__ part,
                              unsigned long long *__restrict__ C, int32_t subround, int32_t *__restrict__ R_node,
                              int32_t *__restrict__ R_from, int32_t *__restrict__ R_to,
                              int32_t *__restrict__ R_sub, int32_t *__restrict__ r_to) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *d_na) return;
    const int32_t u = P[A[S[Adm[p]]]];
    const int32_t a = part[u], b = prop_tgt[u];
    const unsigned long long c = vwgt ? (unsigned long long)vwgt[u] : 1ull;
    R_node[p] = u;
    R_from[p] = a;
    R_to[p] = b;
    R_sub[p] = subround;
    r_to[u] = b;
    part[u] = b;
    atomicAdd(&C[a], (unsigned long long)(-(long long)c));
    atomicAdd(&C[b], c);
}

inline unsigned grid1(int64_t n) { return (unsigned)ceil_div(n > 0 ? n : 1, 256); }

}  // namespace

int rebalance_group(int k) {
    int G = k / 4;
    return G >= 32 ? 32 : G >= 16 ? 16 : G >= 8 ? 8 : 4;
}

void rebalance_propose(const GraphDev &g, const int32_t *part, const int32_t *W, RebalState st, int32_t *prop_tgt,
                       int32_t *prop_gain, int32_t *flags, cudaStream_t s) {
    if (g.n == 0) return;
    const int G = rebalance_group(g.k);
    const int64_t groups = 256 / G;
    const int64_t blocks = std::min<int64_t>(ceil_div(g.n, groups), (int64_t)sm_count_reb() * 16);
#define UPR_PROP(GG) k_propose<GG><<<(unsigned)blocks, 256, 0, s>>>(part, W, g.vwgt, g.n, g.k, st, prop_tgt, prop_gain, flags)
    switch (G) {
        case 4: UPR_PROP(4); break;
        case 8: UPR_PROP(8); break;
        case 16: UPR_PROP(16); break;
        default: UPR_PROP(32); break;
    }
#undef UPR_PROP
    UPR_LAUNCH_CHECK();
}

void rebalance_prio_keys(const GraphDev &g, const int32_t *P, const int32_t *d_np, const int32_t *prop_gain,
                         int gbits, int cbits, uint64_t *keys, uint32_t *vals, int64_t np, cudaStream_t s) {
    if (np <= 0) return;
    k_prio_keys<<<grid1(np), 256, 0, s>>>(P, d_np, prop_gain, g.vwgt, gbits, cbits, keys, vals);
    UPR_LAUNCH_CHECK();
}

void rebalance_block_keys(const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *d_cnt,
                          const int32_t *blk_of_node, uint64_t *keys, uint32_t *vals, int64_t cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    k_block_keys<<<grid1(cnt), 256, 0, s>>>(P, A, S, d_cnt, blk_of_node, keys, vals);
    UPR_LAUNCH_CHECK();
}

void rebalance_seg_weights(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S,
                           const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, int64_t *c_sorted,
                           int32_t *seg_first, int64_t cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    k_seg_weights<<<grid1(cnt), 256, 0, s>>>(P, A, S, B, bkeys, d_cnt, g.vwgt, c_sorted, seg_first);
    UPR_LAUNCH_CHECK();
}

void rebalance_mark_selected(const uint32_t *B, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_excl,
                             const int32_t *seg_first, RebalState st, int32_t *sel, int64_t cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    k_mark_selected<<<grid1(cnt), 256, 0, s>>>(B, bkeys, d_cnt, c_excl, seg_first, st, sel);
    UPR_LAUNCH_CHECK();
}

void rebalance_mark_admitted(const uint32_t *T, const uint64_t *bkeys, const int32_t *d_cnt, const int64_t *c_sorted,
                             const int64_t *c_excl, const int32_t *seg_first, RebalState st, int32_t *adm,
                             int8_t *reject, int64_t cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    k_mark_admitted<<<grid1(cnt), 256, 0, s>>>(T, bkeys, d_cnt, c_sorted, c_excl, seg_first, st, adm, reject);
    UPR_LAUNCH_CHECK();
}

void rebalance_apply(const GraphDev &g, const int32_t *P, const uint32_t *A, const int32_t *S, const int32_t *Adm,
                     const int32_t *d_na, const int32_t *prop_tgt, int32_t *part, int64_t *C, int32_t subround,
                     int32_t *R_node, int32_t *R_from, int32_t *R_to, int32_t *R_sub, int32_t *r_to, int64_t na,
                     cudaStream_t s) {
    if (na <= 0) return;
    k_apply_rebal<<<grid1(na), 256, 0, s>>>(P, A, S, Adm, d_na, prop_tgt, g.vwgt, part, (unsigned long long *)C,
                                            subround, R_node, R_from, R_to, R_sub, r_to);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
