// One batch context for graphs with different k.  A table row keeps exactly
// k columns, so graphs are grouped by k: each group is a batch context of its
// own (upr_batch_create) with its own stream, and a call refines the groups
// concurrently (one host thread per group; with params.graphs = 2 each
// group's rounds are one graph launch).  The caller sees one context: its
// partitions, statuses and cuts in its own graph order.  Every graph's result
// is the one it gets alone (each group is a batch whose graphs are refined
// exactly as alone).
#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "kernels.h"

namespace upr {

struct MixedBatch {
    int device = 0;
    cudaStream_t s = nullptr;                     // the caller's stream
    int64_t n = 0;
    int32_t ng = 0;
    std::vector<int32_t> k_of;                    // k of each group
    std::vector<std::vector<int32_t>> idx;        // caller graph indices of each group
    std::vector<upr_ctx *> sub;
    std::vector<cudaStream_t> streams;
    std::vector<int64_t> noff;                    // caller node offsets [ng + 1]
    std::vector<int64_t> boff;                    // caller offsets of the graphs' block weights [ng + 1]
    std::vector<int64_t> lmax;                    // L_max of each caller graph
    std::vector<int64_t> gnodes;                  // nodes of each group
    upr_params prm{};                             // the parameters every batch is bound with
    int32_t *d_part = nullptr;                    // [n] the partition in caller order
    std::vector<int32_t *> d_sub;                 // [nodes of group g] the group's packed partition
    std::vector<size_t> d_cap;                    // capacity of d_sub[g]
    int32_t **d_ptrs = nullptr;                   // device copy of d_sub
    int64_t *d_map = nullptr;                     // [n] caller node -> (group << 40) | position in the group
    size_t part_cap = 0, map_cap = 0, ptrs_cap = 0;
    int64_t *d_noff = nullptr, *d_gpos = nullptr;  // per caller graph: node offset, first position in its batch
    int32_t *d_grp = nullptr;                     // per caller graph: its batch
    size_t noff_cap = 0, gpos_cap = 0, grp_cap = 0;
    cudaEvent_t ev_fork = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
};

namespace {

constexpr int kPosBits = 40;

__global__ void k_mix_gather(const int32_t *__restrict__ part, const int64_t *__restrict__ map, int64_t n,
                             int32_t *const *__restrict__ sub) {
    UPR_FOR(j, n) {
        const int64_t m = map[j];
        sub[m >> kPosBits][m & ((1ll << kPosBits) - 1)] = part[j];
    }
}

__global__ void k_mix_scatter(int32_t *__restrict__ part, const int64_t *__restrict__ map, int64_t n,
                              int32_t *const *__restrict__ sub) {
    UPR_FOR(j, n) {
        const int64_t m = map[j];
        part[j] = sub[m >> kPosBits][m & ((1ll << kPosBits) - 1)];
    }
}

// map[j] for every caller node j: its batch (group) and its position in the
// batch's packed order, from per-graph node offsets (caller order), groups
// and first positions in their batches.
__global__ void k_mix_map(const int64_t *__restrict__ noff, const int32_t *__restrict__ grp,
                          const int64_t *__restrict__ gpos, int32_t ng, int64_t n, int64_t *__restrict__ map) {
    UPR_FOR(j, n) {
        int32_t lo = 0, hi = ng - 1;            // last graph i with noff[i] <= j
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (noff[mid] <= j) lo = mid; else hi = mid - 1;
        }
        map[j] = ((int64_t)grp[lo] << kPosBits) | (gpos[lo] + (j - noff[lo]));
    }
}

void free_mixed(MixedBatch *mb) {
    if (!mb) return;
    for (upr_ctx *c : mb->sub) upr_destroy(c);
    for (cudaStream_t st : mb->streams)
        if (st) cudaStreamDestroy(st);
    for (int32_t *p : mb->d_sub)
        if (p) cudaFree(p);
    if (mb->d_part) cudaFree(mb->d_part);
    if (mb->d_ptrs) cudaFree(mb->d_ptrs);
    if (mb->d_map) cudaFree(mb->d_map);
    if (mb->d_noff) cudaFree(mb->d_noff);
    if (mb->d_gpos) cudaFree(mb->d_gpos);
    if (mb->d_grp) cudaFree(mb->d_grp);
    if (mb->ev_fork) cudaEventDestroy(mb->ev_fork);
    if (mb->ev_t0) cudaEventDestroy(mb->ev_t0);
    if (mb->ev_t1) cudaEventDestroy(mb->ev_t1);
    delete mb;
}

// The caller's partition (host or device) into the groups' packed buffers.
void gather_part(MixedBatch *mb, const int32_t *part) {
    if (mb->n == 0) return;
    UPR_CUDA(cudaMemcpyAsync(mb->d_part, part, sizeof(int32_t) * mb->n, cudaMemcpyDefault, mb->s));
    k_mix_gather<<<grid_for(mb->n), 256, 0, mb->s>>>(mb->d_part, mb->d_map, mb->n, mb->d_ptrs);
    UPR_LAUNCH_CHECK();
}

}  // namespace

namespace {

// Device buffer of at least `count` elements (grown, never shrunk).
template <typename T>
void reserve(T **p, size_t *cap, size_t count) {
    if (*cap >= count) return;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    UPR_CUDA(cudaMalloc(p, sizeof(T) * std::max<size_t>(count, 1)));
    *cap = count;
}

// Binds the graphs: one batch per k.  A batch of a k the previous binding
// had reuses that batch's context (and its device memory when large
// enough); new k get new contexts; contexts of k no longer present are freed.
upr_status mixed_bind(MixedBatch *mb, const upr_graph *graphs, int32_t n_graphs, const int32_t *k, const double *eps,
                      const upr_params &prm) {
    mb->noff.assign(n_graphs + 1, 0);
    mb->boff.assign(n_graphs + 1, 0);
    for (int32_t i = 0; i < n_graphs; i++) {
        if (k[i] < 2 || k[i] > kMaxK || graphs[i].n < 0) return UPR_ERR_INVALID;
        mb->noff[i + 1] = mb->noff[i] + graphs[i].n;
        mb->boff[i + 1] = mb->boff[i] + k[i];
    }
    if (mb->noff[n_graphs] >= (1ll << 31)) return UPR_ERR_INVALID;
    mb->ng = n_graphs;
    mb->n = mb->noff[n_graphs];
    // groups by k, in increasing k, graphs in caller order within a group
    std::vector<int32_t> ks(k, k + n_graphs);
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    const size_t G = ks.size();
    // the previous binding's contexts, streams and buffers by k
    std::vector<upr_ctx *> sub(G, nullptr);
    std::vector<cudaStream_t> streams(G, nullptr);
    std::vector<int32_t *> d_sub(G, nullptr);
    std::vector<size_t> d_cap(G, 0);
    for (size_t j = 0; j < mb->k_of.size(); j++) {
        const auto it = std::lower_bound(ks.begin(), ks.end(), mb->k_of[j]);
        if (it != ks.end() && *it == mb->k_of[j]) {
            const size_t g = it - ks.begin();
            sub[g] = mb->sub[j];
            streams[g] = mb->streams[j];
            d_sub[g] = mb->d_sub[j];
            d_cap[g] = mb->d_cap[j];
        } else {
            upr_destroy(mb->sub[j]);
            if (mb->streams[j]) cudaStreamDestroy(mb->streams[j]);
            if (mb->d_sub[j]) cudaFree(mb->d_sub[j]);
        }
    }
    mb->k_of = ks;
    mb->sub = sub;
    mb->streams = streams;
    mb->d_sub = d_sub;
    mb->d_cap = d_cap;
    mb->idx.assign(G, {});
    for (int32_t i = 0; i < n_graphs; i++)
        mb->idx[std::lower_bound(ks.begin(), ks.end(), k[i]) - ks.begin()].push_back(i);
    mb->gnodes.assign(G, 0);
    mb->lmax.assign(n_graphs, 0);
    std::vector<int32_t> grp(n_graphs);
    std::vector<int64_t> gpos(n_graphs);
    std::vector<std::vector<upr_graph>> gs(G);
    std::vector<std::vector<double>> es(G);
    for (size_t g = 0; g < G; g++) {
        if (!mb->streams[g]) UPR_CUDA(cudaStreamCreateWithFlags(&mb->streams[g], cudaStreamNonBlocking));
        int64_t pos = 0;
        for (int32_t i : mb->idx[g]) {
            gs[g].push_back(graphs[i]);
            es[g].push_back(eps[i]);
            grp[i] = (int32_t)g;
            gpos[i] = pos;
            pos += graphs[i].n;
        }
        mb->gnodes[g] = pos;
    }
    // the batches are bound concurrently, one host thread each
    std::vector<upr_status> grc(G, UPR_OK);
    std::vector<std::thread> th;
    for (size_t g = 0; g < G; g++)
        th.emplace_back([&, g] {
            cudaSetDevice(mb->device);
            upr_params p = prm;
            p.stream = mb->streams[g];
            grc[g] = mb->sub[g] ? ctx_rebind_batch(mb->sub[g], gs[g].data(), (int32_t)gs[g].size(), ks[g],
                                                   es[g].data(), &p)
                                : upr_batch_create(gs[g].data(), (int32_t)gs[g].size(), ks[g], es[g].data(), &p,
                                                   &mb->sub[g]);
        });
    for (auto &t : th) t.join();
    for (size_t g = 0; g < G; g++)
        if (grc[g] != UPR_OK) return grc[g];
    for (size_t g = 0; g < G; g++) {
        std::vector<int64_t> lm(gs[g].size());
        upr_batch_info(mb->sub[g], nullptr, nullptr, lm.data());
        for (size_t j = 0; j < gs[g].size(); j++) mb->lmax[mb->idx[g][j]] = lm[j];
        reserve(&mb->d_sub[g], &mb->d_cap[g], (size_t)mb->gnodes[g]);
    }
    reserve(&mb->d_part, &mb->part_cap, (size_t)mb->n);
    reserve(&mb->d_map, &mb->map_cap, (size_t)mb->n);
    reserve(&mb->d_ptrs, &mb->ptrs_cap, G);
    UPR_CUDA(cudaMemcpy(mb->d_ptrs, mb->d_sub.data(), sizeof(int32_t *) * G, cudaMemcpyHostToDevice));
    if (mb->n > 0) {
        // the node map on the device, from per-graph offsets, batches and
        // first positions (in buffers kept across bindings)
        reserve(&mb->d_noff, &mb->noff_cap, (size_t)n_graphs + 1);
        reserve(&mb->d_gpos, &mb->gpos_cap, (size_t)n_graphs);
        reserve(&mb->d_grp, &mb->grp_cap, (size_t)n_graphs);
        UPR_CUDA(cudaMemcpy(mb->d_noff, mb->noff.data(), sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice));
        UPR_CUDA(cudaMemcpy(mb->d_gpos, gpos.data(), sizeof(int64_t) * n_graphs, cudaMemcpyHostToDevice));
        UPR_CUDA(cudaMemcpy(mb->d_grp, grp.data(), sizeof(int32_t) * n_graphs, cudaMemcpyHostToDevice));
        k_mix_map<<<grid_for(mb->n), 256, 0, mb->s>>>(mb->d_noff, mb->d_grp, mb->d_gpos, n_graphs, mb->n, mb->d_map);
        UPR_LAUNCH_CHECK();
        UPR_CUDA(cudaStreamSynchronize(mb->s));
    }
    return UPR_OK;
}

}  // namespace

upr_status mixed_create(const upr_graph *graphs, int32_t n_graphs, const int32_t *k, const double *eps,
                        const upr_params *params, MixedBatch **out) {
    if (!graphs || !k || !eps || n_graphs < 1 || !out) return UPR_ERR_INVALID;
    MixedBatch *mb = new (std::nothrow) MixedBatch();
    if (!mb) return UPR_ERR_OOM;
    upr_params_default(&mb->prm);
    if (params) mb->prm = *params;
    mb->s = (cudaStream_t)mb->prm.stream;
    upr_status rc = UPR_OK;
    try {
        UPR_CUDA(cudaGetDevice(&mb->device));
        UPR_CUDA(cudaEventCreateWithFlags(&mb->ev_fork, cudaEventDisableTiming));
        UPR_CUDA(cudaEventCreate(&mb->ev_t0));
        UPR_CUDA(cudaEventCreate(&mb->ev_t1));
        rc = mixed_bind(mb, graphs, n_graphs, k, eps, mb->prm);
    } catch (const CudaError &e) {
        rc = e.e == cudaErrorMemoryAllocation ? UPR_ERR_OOM : UPR_ERR_CUDA;
    } catch (const std::bad_alloc &) {
        rc = UPR_ERR_OOM;
    }
    if (rc != UPR_OK) { free_mixed(mb); return rc; }
    *out = mb;
    return UPR_OK;
}

upr_status mixed_rebind(MixedBatch *mb, const upr_graph *graphs, int32_t n_graphs, const int32_t *k,
                        const double *eps) {
    if (!graphs || !k || !eps || n_graphs < 1) return UPR_ERR_INVALID;
    try {
        UPR_CUDA(cudaSetDevice(mb->device));
        return mixed_bind(mb, graphs, n_graphs, k, eps, mb->prm);
    } catch (const CudaError &e) {
        return e.e == cudaErrorMemoryAllocation ? UPR_ERR_OOM : UPR_ERR_CUDA;
    } catch (const std::bad_alloc &) {
        return UPR_ERR_OOM;
    }
}

void mixed_destroy(MixedBatch *mb) { free_mixed(mb); }

int64_t mixed_nodes(const MixedBatch *mb) { return mb->n; }

upr_status mixed_refine(MixedBatch *mb, int32_t *part, int32_t rounds, uint64_t seed, upr_status *status,
                        int64_t *cut_in, int64_t *cut_out, upr_stats *stats) {
    if ((!part && mb->n > 0) || rounds < 0) return UPR_ERR_INVALID;
    const size_t G = mb->sub.size();
    std::vector<std::vector<upr_status>> gst(G);
    std::vector<std::vector<int64_t>> gin(G), gout(G);
    std::vector<upr_stats> gstats(G);
    std::vector<upr_status> grc(G, UPR_OK);
    try {
        UPR_CUDA(cudaEventRecord(mb->ev_t0, mb->s));
        gather_part(mb, part);
        UPR_CUDA(cudaEventRecord(mb->ev_fork, mb->s));
        for (size_t g = 0; g < G; g++) {
            UPR_CUDA(cudaStreamWaitEvent(mb->streams[g], mb->ev_fork, 0));
            gst[g].assign(mb->idx[g].size(), UPR_OK);
            gin[g].assign(mb->idx[g].size(), 0);
            gout[g].assign(mb->idx[g].size(), 0);
        }
        // the groups concurrently: each call runs on its group's stream and
        // returns after it has synchronised that stream
        std::vector<std::thread> th;
        for (size_t g = 1; g < G; g++)
            th.emplace_back([&, g] {
                cudaSetDevice(mb->device);
                grc[g] = upr_batch_refine(mb->sub[g], mb->d_sub[g], rounds, seed, gst[g].data(), gin[g].data(),
                                          gout[g].data(), &gstats[g]);
            });
        if (G > 0)
            grc[0] = upr_batch_refine(mb->sub[0], mb->d_sub[0], rounds, seed, gst[0].data(), gin[0].data(),
                                      gout[0].data(), &gstats[0]);
        for (auto &t : th) t.join();
        for (upr_status r : grc)
            if (r != UPR_OK) return r;
        if (mb->n > 0) {
            k_mix_scatter<<<grid_for(mb->n), 256, 0, mb->s>>>(mb->d_part, mb->d_map, mb->n, mb->d_ptrs);
            UPR_LAUNCH_CHECK();
            UPR_CUDA(cudaMemcpyAsync(part, mb->d_part, sizeof(int32_t) * mb->n, cudaMemcpyDefault, mb->s));
        }
        UPR_CUDA(cudaEventRecord(mb->ev_t1, mb->s));
        UPR_CUDA(cudaEventSynchronize(mb->ev_t1));
        float ms = 0;
        UPR_CUDA(cudaEventElapsedTime(&ms, mb->ev_t0, mb->ev_t1));
        upr_stats st{};
        for (size_t g = 0; g < G; g++) {
            const upr_stats &x = gstats[g];
            st.cut_in += x.cut_in; st.cut_out += x.cut_out;
            st.rounds_run = std::max(st.rounds_run, x.rounds_run);
            st.repaired_input |= x.repaired_input;
            st.n_candidates += x.n_candidates; st.n_moves += x.n_moves; st.n_rebalance_moves += x.n_rebalance_moves;
            st.n_sequence += x.n_sequence; st.n_applied += x.n_applied; st.subrounds += x.subrounds;
            st.kernel_launches += x.kernel_launches; st.ms_gain_table += x.ms_gain_table;
            st.gain_table_builds += x.gain_table_builds; st.gain_table_bytes += x.gain_table_bytes;
            st.ms_select += x.ms_select; st.ms_rebalance += x.ms_rebalance; st.ms_sequence += x.ms_sequence;
            st.batch_graphs += x.batch_graphs; st.rebalance_graphs += x.rebalance_graphs;
            st.constrained_rounds += x.constrained_rounds; st.seq_degree_sum += x.seq_degree_sum;
            st.bytes_algorithmic += x.bytes_algorithmic;
            for (size_t j = 0; j < mb->idx[g].size(); j++) {
                const int32_t i = mb->idx[g][j];
                if (status) status[i] = gst[g][j];
                if (cut_in) cut_in[i] = gin[g][j];
                if (cut_out) cut_out[i] = gout[g][j];
            }
        }
        st.kernel_launches += mb->n > 0 ? 2 : 0;     // gather, scatter
        st.ms_device = ms;
        if (stats) *stats = st;
    } catch (const CudaError &e) {
        return e.e == cudaErrorMemoryAllocation ? UPR_ERR_OOM : UPR_ERR_CUDA;
    }
    return UPR_OK;
}

upr_status mixed_cut(MixedBatch *mb, const int32_t *part, int64_t *cut, int64_t *block_weights) {
    if (!part || !cut) return UPR_ERR_INVALID;
    try {
        gather_part(mb, part);
        UPR_CUDA(cudaStreamSynchronize(mb->s));
        for (size_t g = 0; g < mb->sub.size(); g++) {
            const size_t m = mb->idx[g].size();
            std::vector<int64_t> c(m), bw(m * (size_t)mb->k_of[g]);
            const upr_status rc = upr_batch_cut(mb->sub[g], mb->d_sub[g], c.data(), bw.data());
            if (rc != UPR_OK) return rc;
            for (size_t j = 0; j < m; j++) {
                const int32_t i = mb->idx[g][j];
                cut[i] = c[j];
                if (block_weights)
                    for (int32_t b = 0; b < mb->k_of[g]; b++)
                        block_weights[mb->boff[i] + b] = bw[j * mb->k_of[g] + b];
            }
        }
    } catch (const CudaError &e) {
        return UPR_ERR_CUDA;
    }
    return UPR_OK;
}

upr_status mixed_info(const MixedBatch *mb, int32_t *n_graphs, int64_t *node_offsets, int64_t *lmax) {
    if (n_graphs) *n_graphs = mb->ng;
    if (node_offsets) std::copy(mb->noff.begin(), mb->noff.end(), node_offsets);
    if (lmax) std::copy(mb->lmax.begin(), mb->lmax.end(), lmax);
    return UPR_OK;
}

}  // namespace upr
