// Serving: upr_server_* / upr_submit / upr_poll / upr_wait of include/upr.h.
//
// Continuous batching.  Submitted jobs wait in a FIFO queue; max_jobs slot
// threads each own a CUDA stream and one context that they re-bind to every
// piece of work they take.  A free slot takes the oldest queued job that fits
// in what is left of the device-memory budget (smaller jobs may overtake a
// large one that does not fit yet).  If that job is small, the slot also
// takes every other queued small job with the same k and rounds that still
// fits, and refines the group as one batch context (one launch per step for
// all of them); jobs that arrive meanwhile are taken by the next free slot.
// Slots run concurrently on their own streams, so batches and large jobs
// overlap on the device.  A job's result is the same as upr_create +
// upr_refine on the same inputs (a batch keeps every step per graph).
//
// Memory accounting is exact: in_use is the sum over slots of the arena
// bytes a slot holds or has reserved for the work it took.  A slot keeps its
// arena between pieces of work when it is at most a fair share of the budget,
// and gives it back when it is larger or when queued work does not fit.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.h"

namespace {

struct Job {
    uint64_t ticket = 0;
    int64_t n = 0, m = 0;
    int32_t k = 0, rounds = 0;
    double eps = 0;
    uint64_t seed = 0;
    std::vector<int64_t> xadj;
    std::vector<int32_t> adj, adjw, vwgt, part;
    bool has_adjw = false, has_vwgt = false;
    size_t footprint = 0;
    // results
    bool done = false;
    upr_status status = UPR_PENDING;
    int64_t cut = 0;
    upr_stats stats{};
};

using JobPtr = std::shared_ptr<Job>;

}  // namespace

// Device bytes of a context for ng graphs with n nodes / m entries in total (engine.cu).
size_t upr_ctx_footprint(int64_t n, int64_t m, int32_t k, int32_t ng);

namespace upr {
upr_status ctx_rebind(upr_ctx *c, const upr_graph *g, int32_t k, double eps, const upr_params *params);
upr_status ctx_rebind_batch(upr_ctx *c, const upr_graph *gs, int32_t ng, int32_t k, const double *eps,
                            const upr_params *params);
size_t ctx_arena_bytes(const upr_ctx *c);
}

struct upr_server {
    upr_server_params p{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<JobPtr> queue;
    std::map<uint64_t, JobPtr> jobs;
    std::vector<std::thread> slots;
    std::vector<size_t> held;      // per slot: arena bytes held or reserved
    size_t budget = 0, in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    int device = 0;

    // batches need the plain round schedule (the round driver decides per graph)
    bool small(const Job &j) const {
        return p.batch_max_jobs > 1 && p.params.schedule == 0 && j.n <= p.batch_max_nodes;
    }

    // Extra bytes slot i must reserve to run work of footprint f.
    size_t extra(int i, size_t f) const { return f > held[i] ? f - held[i] : 0; }

    // Under mu: takes the next piece of work for slot i (empty if none fits).
    std::vector<JobPtr> take(int i, size_t *fp_out) {
        std::vector<JobPtr> group;
        auto it = queue.begin();
        for (; it != queue.end(); ++it) {
            const size_t e = extra(i, (*it)->footprint);
            if (in_use + e <= budget || in_use == held[i]) break;
        }
        if (it == queue.end()) return group;
        JobPtr j0 = *it;
        queue.erase(it);
        group.push_back(j0);
        int64_t nodes = j0->n, edges = j0->m;
        size_t fp = j0->footprint;
        if (small(*j0)) {
            for (auto q = queue.begin(); q != queue.end() && (int32_t)group.size() < p.batch_max_jobs;) {
                const Job &j = **q;
                if (small(j) && j.k == j0->k && j.rounds == j0->rounds && nodes + j.n <= p.batch_max_total_nodes) {
                    const size_t f2 = upr_ctx_footprint(nodes + j.n, edges + j.m, j0->k, (int32_t)group.size() + 1);
                    if (in_use + extra(i, f2) <= budget) {
                        group.push_back(*q);
                        nodes += j.n;
                        edges += j.m;
                        fp = f2;
                        q = queue.erase(q);
                        continue;
                    }
                }
                ++q;
            }
        }
        const size_t e = extra(i, fp);
        in_use += e;
        held[i] += e;
        *fp_out = fp;
        return group;
    }

    void slot_main(int i) {
        cudaSetDevice(device);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
        upr_ctx *ctx = nullptr;     // this slot's context, re-bound to every piece of work
        const size_t share = budget / (size_t)p.max_jobs;
        for (;;) {
            std::vector<JobPtr> group;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop && queue.empty()) break;
                    size_t fp = 0;
                    group = take(i, &fp);
                    if (!group.empty()) break;
                    if (!queue.empty() && ctx) {
                        // queued work does not fit: give this slot's arena back
                        lk.unlock();
                        upr_destroy(ctx);
                        ctx = nullptr;
                        lk.lock();
                        in_use -= held[i];
                        held[i] = 0;
                        cv_work.notify_all();
                        continue;
                    }
                    cv_work.wait(lk);
                }
            }
            if (group.empty()) break;
            run(group, s, &ctx);
            const size_t arena = upr::ctx_arena_bytes(ctx);
            if (ctx && arena > share) {
                upr_destroy(ctx);
                ctx = nullptr;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                const size_t now = ctx ? upr::ctx_arena_bytes(ctx) : 0;
                in_use -= held[i];
                held[i] = now;
                in_use += now;
                for (auto &j : group) j->done = true;
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
        upr_destroy(ctx);
        {
            std::lock_guard<std::mutex> lk(mu);
            in_use -= held[i];
            held[i] = 0;
        }
        if (s) cudaStreamDestroy(s);
    }

    static upr_graph graph_of(const Job &j) {
        upr_graph g{};
        g.n = j.n; g.m = j.m;
        g.xadj = j.xadj.data();
        g.adjncy = j.adj.data();
        g.vwgt = j.has_vwgt ? j.vwgt.data() : nullptr;
        g.adjwgt = j.has_adjw ? j.adjw.data() : nullptr;
        return g;
    }

    void run(std::vector<JobPtr> &group, cudaStream_t s, upr_ctx **ctx) {
        upr_params prm = p.params;
        prm.stream = s;
        if (group.size() == 1) {
            Job *j = group[0].get();
            const upr_graph g = graph_of(*j);
            upr_status st = *ctx ? upr::ctx_rebind(*ctx, &g, j->k, j->eps, &prm)
                                 : upr_create(&g, j->k, j->eps, &prm, ctx);
            if (st == UPR_OK) {
                st = upr_refine(*ctx, j->part.data(), j->rounds, j->seed, &j->stats);
                if (st == UPR_OK) j->cut = j->stats.cut_out;
            }
            j->status = st;
        } else {
            const size_t ng = group.size();
            std::vector<upr_graph> gs(ng);
            std::vector<double> eps(ng);
            std::vector<int64_t> off(ng + 1, 0);
            for (size_t i = 0; i < ng; i++) {
                gs[i] = graph_of(*group[i]);
                eps[i] = group[i]->eps;
                off[i + 1] = off[i] + group[i]->n;
            }
            const int32_t k = group[0]->k;
            upr_status st = UPR_OK;
            if (!*ctx) {
                *ctx = nullptr;
                st = upr_batch_create(gs.data(), (int32_t)ng, k, eps.data(), &prm, ctx);
            } else {
                st = upr::ctx_rebind_batch(*ctx, gs.data(), (int32_t)ng, k, eps.data(), &prm);
            }
            std::vector<int32_t> part((size_t)off[ng]);
            std::vector<upr_status> gst(ng, UPR_OK);
            std::vector<int64_t> cin(ng, 0), cout(ng, 0);
            upr_stats bst{};
            if (st == UPR_OK) {
                for (size_t i = 0; i < ng; i++)
                    if (group[i]->n) memcpy(part.data() + off[i], group[i]->part.data(), sizeof(int32_t) * group[i]->n);
                st = upr_batch_refine(*ctx, part.data(), group[0]->rounds, group[0]->seed, gst.data(), cin.data(),
                                      cout.data(), &bst);
            }
            for (size_t i = 0; i < ng; i++) {
                Job *j = group[i].get();
                j->status = st == UPR_OK ? gst[i] : st;
                if (j->status == UPR_OK) {
                    if (j->n) memcpy(j->part.data(), part.data() + off[i], sizeof(int32_t) * j->n);
                    j->stats = bst;
                    j->stats.cut_in = cin[i];
                    j->stats.cut_out = cout[i];
                    j->cut = cout[i];
                }
            }
        }
        for (auto &jp : group) {
            // the graph copy is no longer needed
            std::vector<int64_t>().swap(jp->xadj);
            std::vector<int32_t>().swap(jp->adj);
            std::vector<int32_t>().swap(jp->adjw);
            std::vector<int32_t>().swap(jp->vwgt);
        }
    }
};

extern "C" {

void upr_server_params_default(upr_server_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->max_jobs = 8;
    p->queue_capacity = 4096;
    p->memory_budget = 0;
    upr_params_default(&p->params);
    p->batch_max_jobs = 4096;
    p->batch_max_nodes = 131072;
    p->batch_max_total_nodes = (int64_t)1 << 25;
}

upr_status upr_server_create(const upr_server_params *p, upr_server **out) {
    if (!out) return UPR_ERR_INVALID;
    upr_server_params prm;
    upr_server_params_default(&prm);
    if (p) prm = *p;
    if (prm.max_jobs < 1 || prm.max_jobs > 256 || prm.queue_capacity < 1 || prm.memory_budget < 0 ||
        prm.batch_max_jobs < 1 || prm.batch_max_nodes < 0 || prm.batch_max_total_nodes < 1)
        return UPR_ERR_INVALID;
    upr_server *s = new (std::nothrow) upr_server();
    if (!s) return UPR_ERR_OOM;
    s->p = prm;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return UPR_ERR_CUDA; }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; return UPR_ERR_CUDA; }
    s->budget = prm.memory_budget > 0 ? (size_t)prm.memory_budget : free_b / 10 * 8;
    s->held.assign(prm.max_jobs, 0);
    try {
        for (int i = 0; i < prm.max_jobs; i++) s->slots.emplace_back([s, i] { s->slot_main(i); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->slots) t.join();
        delete s;
        return UPR_ERR_OOM;
    }
    *out = s;
    return UPR_OK;
}

upr_status upr_submit(upr_server *s, const upr_graph *g, int32_t k, double eps, const int32_t *part, int32_t rounds,
                      uint64_t seed, uint64_t *ticket) {
    if (!s || !g || !part || !ticket || g->n < 0 || g->m < 0 || k < 2 || rounds < 0 || !(eps > 0))
        return UPR_ERR_INVALID;
    auto j = std::make_shared<Job>();
    try {
        j->n = g->n; j->m = g->m; j->k = k; j->eps = eps; j->rounds = rounds; j->seed = seed;
        j->xadj.assign(g->xadj, g->xadj + g->n + 1);
        j->adj.assign(g->adjncy, g->adjncy + g->m);
        if (g->adjwgt) { j->adjw.assign(g->adjwgt, g->adjwgt + g->m); j->has_adjw = true; }
        if (g->vwgt) { j->vwgt.assign(g->vwgt, g->vwgt + g->n); j->has_vwgt = true; }
        j->part.assign(part, part + g->n);
    } catch (const std::bad_alloc &) {
        return UPR_ERR_OOM;
    }
    j->footprint = upr_ctx_footprint(g->n, g->m, k, 1);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((int64_t)s->queue.size() >= s->p.queue_capacity) return UPR_ERR_BUSY;
        if (j->footprint > s->budget) return UPR_ERR_OOM;
        j->ticket = s->next_ticket++;
        s->jobs[j->ticket] = j;
        s->queue.push_back(j);
        *ticket = j->ticket;
    }
    s->cv_work.notify_one();
    return UPR_OK;
}

static upr_status take_result(upr_server *s, std::map<uint64_t, JobPtr>::iterator it, int32_t *part_out,
                              int64_t *cut_out, upr_stats *stats) {
    JobPtr j = it->second;
    s->jobs.erase(it);
    if (j->status == UPR_OK) {
        if (part_out) memcpy(part_out, j->part.data(), sizeof(int32_t) * j->n);
        if (cut_out) *cut_out = j->cut;
        if (stats) *stats = j->stats;
    }
    return j->status;
}

upr_status upr_poll(upr_server *s, uint64_t ticket, int32_t *part_out, int64_t *cut_out, upr_stats *stats) {
    if (!s) return UPR_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return UPR_ERR_NOT_FOUND;
    if (!it->second->done) return UPR_PENDING;
    return take_result(s, it, part_out, cut_out, stats);
}

upr_status upr_wait(upr_server *s, uint64_t ticket, int64_t timeout_ms, int32_t *part_out, int64_t *cut_out,
                    upr_stats *stats) {
    if (!s) return UPR_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return UPR_ERR_NOT_FOUND;
    JobPtr j = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] { return j->done; }))
        return UPR_ERR_TIMEOUT;
    it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return UPR_ERR_NOT_FOUND;
    return take_result(s, it, part_out, cut_out, stats);
}

void upr_server_destroy(upr_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->slots) t.join();
    delete s;
}

}  // extern "C"
