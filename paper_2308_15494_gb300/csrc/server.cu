// Serving: upr_server_* / upr_submit / upr_poll / upr_wait of include/upr.h.
//
// Continuous batching.  Submitted jobs wait in a queue; max_jobs slot threads
// each own a CUDA stream.  A free slot admits the oldest queued job whose
// device footprint fits in what is left of the memory budget (smaller jobs may
// overtake a large one that does not fit yet), creates its context on the
// slot's stream and runs upr_refine, so jobs of different sizes run
// concurrently on the device.  Each job keeps its gain table and partition
// resident for all its rounds; its result stays in host memory until polled.
// A job's result is the same as upr_create + upr_refine on the same inputs.
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

}  // namespace

// Device bytes one context needs (the arena of engine.cu plus slack).
size_t upr_ctx_footprint(int64_t n, int64_t m, int32_t k);

namespace upr {
upr_status ctx_rebind(upr_ctx *c, const upr_graph *g, int32_t k, double eps, const upr_params *params);
}

struct upr_server {
    upr_server_params p{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::vector<std::thread> slots;
    size_t budget = 0, in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    int device = 0;

    void slot_main() {
        cudaSetDevice(device);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
        upr_ctx *ctx = nullptr;     // this slot's context, re-bound to every job it runs
        for (;;) {
            std::shared_ptr<Job> job;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop && queue.empty()) break;
                    auto it = queue.begin();
                    for (; it != queue.end(); ++it)
                        if (in_use + (*it)->footprint <= budget || in_use == 0) break;
                    if (it != queue.end()) {
                        job = *it;
                        queue.erase(it);
                        in_use += job->footprint;
                        break;
                    }
                    cv_work.wait(lk);
                }
            }
            if (!job) break;
            run(job.get(), s, &ctx);
            {
                std::lock_guard<std::mutex> lk(mu);
                in_use -= job->footprint;
                job->done = true;
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
        upr_destroy(ctx);
        if (s) cudaStreamDestroy(s);
    }

    void run(Job *j, cudaStream_t s, upr_ctx **ctx) {
        upr_graph g{};
        g.n = j->n; g.m = j->m;
        g.xadj = j->xadj.data();
        g.adjncy = j->adj.data();
        g.vwgt = j->has_vwgt ? j->vwgt.data() : nullptr;
        g.adjwgt = j->has_adjw ? j->adjw.data() : nullptr;
        upr_params prm = p.params;
        prm.stream = s;
        // the slot's context keeps its device arena, pinned buffers and events
        // between jobs, so admitting a job allocates only when it is larger
        // than every job this slot ran before
        upr_status st = *ctx ? upr::ctx_rebind(*ctx, &g, j->k, j->eps, &prm)
                             : upr_create(&g, j->k, j->eps, &prm, ctx);
        if (st == UPR_OK) {
            st = upr_refine(*ctx, j->part.data(), j->rounds, j->seed, &j->stats);
            if (st == UPR_OK) j->cut = j->stats.cut_out;
        }
        // the graph copy is no longer needed
        std::vector<int64_t>().swap(j->xadj);
        std::vector<int32_t>().swap(j->adj);
        std::vector<int32_t>().swap(j->adjw);
        std::vector<int32_t>().swap(j->vwgt);
        j->status = st;
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
}

upr_status upr_server_create(const upr_server_params *p, upr_server **out) {
    if (!out) return UPR_ERR_INVALID;
    upr_server_params prm;
    upr_server_params_default(&prm);
    if (p) prm = *p;
    if (prm.max_jobs < 1 || prm.max_jobs > 256 || prm.queue_capacity < 1 || prm.memory_budget < 0)
        return UPR_ERR_INVALID;
    upr_server *s = new (std::nothrow) upr_server();
    if (!s) return UPR_ERR_OOM;
    s->p = prm;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return UPR_ERR_CUDA; }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; return UPR_ERR_CUDA; }
    s->budget = prm.memory_budget > 0 ? (size_t)prm.memory_budget : free_b / 10 * 8;
    try {
        for (int i = 0; i < prm.max_jobs; i++) s->slots.emplace_back([s] { s->slot_main(); });
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
    j->footprint = upr_ctx_footprint(g->n, g->m, k);
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

static upr_status take_result(upr_server *s, std::map<uint64_t, std::shared_ptr<Job>>::iterator it, int32_t *part_out,
                              int64_t *cut_out, upr_stats *stats) {
    std::shared_ptr<Job> j = it->second;
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
    std::shared_ptr<Job> j = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] { return j->done; }))
        return UPR_ERR_TIMEOUT;
    it = s->jobs.find(ticket);
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
