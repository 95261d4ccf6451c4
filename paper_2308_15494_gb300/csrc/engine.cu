// The C ABI of include/upr.h: context creation, the round driver and the
// inspection entry points.  The driver enqueues the kernels of one round on
// the context's stream.  List lengths stay in device memory (kernels read
// them; grids are sized by static bounds), so the host reads back counters
// once per round, and after every rebalancing sub-round only when it drives
// that loop itself instead of launching it as one CUDA graph.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <tuple>
#include <vector>

#include "kernels.h"

using namespace upr;

namespace {

int bit_length(uint64_t x) { int b = 0; while (x) { b++; x >>= 1; } return b; }

// UPR_LOG=1 in the environment prints list sizes per round and sub-round to stderr.
bool log_enabled() {
    static int on = -1;
    if (on < 0) { const char *v = getenv("UPR_LOG"); on = (v && *v && *v != '0') ? 1 : 0; }
    return on == 1;
}

// UPR_LOG: name the failing CUDA call and its error.
upr_status cuda_failure(const CudaError &e) {
    if (log_enabled()) fprintf(stderr, "upr: %s failed: %s\n", e.what, cudaGetErrorString(e.e));
    return e.e == cudaErrorMemoryAllocation ? UPR_ERR_OOM : UPR_ERR_CUDA;
}

// Bump allocator over one cudaMalloc; a first pass with base == nullptr sizes it.
struct Arena {
    char *base = nullptr;
    size_t off = 0;
    template <typename T> T *take(size_t count) {
        size_t a = (off + 255) & ~size_t(255);
        off = a + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + a) : nullptr;
    }
};

struct SortBuf {
    uint64_t *k, *ka;
    uint32_t *v, *va;
    // sorts (k, v) on `bits` bits; returns the buffers holding the result
    void run(Count n, int bits, Scratch tmp, cudaStream_t s, uint64_t **ko, uint32_t **vo) {
        bool alt = radix_sort_pairs(k, v, ka, va, n, bits, tmp, s);
        *ko = alt ? ka : k;
        *vo = alt ? va : v;
    }
};

// Host-side F_r[l] = floor(tau_r * (3/2)^l * 2^Q), tau_r = tau_1 + (1 - tau_1)(r-1)/max(R-1,1)
// F[l] = floor(tau * (3/2)^l * 2^Q) for tau = num / den
void factors_tau(u128 num, u128 den, int64_t *F) {
    for (int l = kSlotLo; l <= kSlotHi; l++) {
        u128 p3 = 1, p2 = 1;
        for (int i = 0; i < (l >= 0 ? l : -l); i++) { p3 *= 3; p2 *= 2; }
        u128 a = l >= 0 ? num * p3 : num * p2;
        u128 b = l >= 0 ? den * p2 : den * p3;
        F[l - kSlotLo] = (int64_t)((a << kQ) / b);
    }
}

void penalty_factors(int32_t r, int32_t R, int64_t t1n, int64_t t1d, int64_t *F) {
    const int64_t D = R > 1 ? (int64_t)R - 1 : 1;
    factors_tau((u128)(t1n * D + (t1d - t1n) * (int64_t)(r - 1)), (u128)(t1d * D), F);
}

// The kind of a round (Sec. 4.4, Sec. 6.2): unconstrained with tau_r of the schedule
// (tau_den = 0) or a given tau, or constrained: no move may leave its target
// above L_max.  A constrained round uses the factor 2^51 in every slot: the
// penalty of any move that overfills its target is then at least 2^31, more
// than any gain (omega(I(v)) < 2^31), so such a move is never a candidate
// and never kept, exactly as if it were forbidden; moves that do not
// overfill pay nothing, as in every round.
struct RoundKind {
    bool constrained = false;
    int64_t tau_num = 0, tau_den = 0;
    // the variants of Sec. 7.2: limit > 0 replaces the penalty by a block
    // limit (no move may leave its target above it, every other move pays
    // nothing): the selection sees L = limit and the factor 2^51 as above.
    int64_t limit = 0;
};
constexpr int64_t kConstrainedF = (int64_t)1 << 51;

__global__ void k_fill_i64(int64_t *a, int64_t n, int64_t v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

}  // namespace

namespace {
// Slots of the device counters (upr_ctx::counts).
enum {
    CNT_CAND = 0, CNT_M, CNT_P, CNT_S, CNT_A, CNT_I, CNT_HUB, CNT_BADPART, CNT_L1, CNT_X, CNT_EVM, CNT_EVI,
    CNT_I1, CNT_OVER0, CNT_INFEAS, CNT_HIST, CNT_EXACT, CNT_SORTP, CNT_SLOTS = 32
};

// Per-call sums of the step graph's rounds (upr_ctx::dstats): candidates,
// moves, rebalancing moves, sub-rounds, sequence length, applied moves, the
// primitives' error word, infeasible rounds, interleaved length, runs of the
// sub-rounds' conditional sort passes.
__global__ void k_round_stats(const int32_t *__restrict__ cnt, const RebalCtl *__restrict__ ctl,
                              const long long *__restrict__ best, const int64_t *__restrict__ tot, int batch,
                              const int32_t *__restrict__ err, long long *__restrict__ d) {
    if (threadIdx.x != 0) return;
    const bool infeasible = !batch && cnt[CNT_INFEAS] != 0;
    d[0] += cnt[CNT_CAND];
    d[1] += cnt[CNT_M];
    d[2] += ctl->nR;
    d[3] += ctl->subrounds;
    d[4] += cnt[CNT_I];
    d[5] += infeasible ? 0 : batch ? tot[0] : best[1];
    d[6] |= *err;
    d[7] += infeasible ? 1 : 0;
    d[8] += cnt[CNT_X];
    d[9] += cnt[CNT_SORTP];
}
}  // namespace

// kernels launched by this host thread (a call runs on one thread, so the
// difference over a call counts that call's launches even when other
// threads refine other contexts meanwhile)
thread_local long long upr::g_upr_launches = 0;

int upr::resident_ctas(const void *func, int threads, size_t shm) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    UPR_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, func, threads, shm);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    UPR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, shm));
    n = std::max(n, 1);
    cache[key] = n;
    return n;
}

void upr::kernel_setup(const void *func, int carveout_percent) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    UPR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, func})) return;
    int optin = 0;
    UPR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    UPR_CUDA(cudaFuncGetAttributes(&fa, func));     // static shared memory counts against the same limit
    UPR_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes));
    if (carveout_percent >= 0)
        UPR_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_percent));
    done.insert({dev, func});
}

struct upr_ctx {
    int device = 0;
    MixedBatch *mix = nullptr;        // a context over graphs of different k (mixed.cu); nothing else is used
    int64_t n = 0, m = 0;
    int32_t k = 0;
    int32_t ng = 1;                   // graphs bound (a batch when > 1)
    bool table_valid = false;         // W holds the table of part0 (carried from the previous round)
    // lane schedules of the selection / proposal kernels: chosen by timing the
    // candidates on this binding's inputs (see tune_*), default until then
    LaneCfg sel_cfg{0, 0}, prop_cfg{0, 0};
    bool sel_tuned = false, prop_tuned = false;
    int sel_pending = 0, prop_pending = 0;      // candidates timed in the current round / sub-round
    LaneCfg sel_cands[3], prop_cands[3];
    cudaEvent_t ev_tune[12] = {};
    // sparse gain table (GraphDev::sp): row offsets, slots, overflow word
    int64_t sp_slots = 0;             // slots of all rows (0: dense only)
    bool sparse_on = false;           // the rounds use the sparse table
    int64_t *sp_off = nullptr; int2 *sp_slot = nullptr; int32_t *sp_over = nullptr;
    // with sparse rows there is no dense table in the arena: one is allocated
    // here only if a round falls back to it (or for the debug entry point)
    int32_t *W_own = nullptr; size_t W_own_bytes = 0;
    int32_t sp_buf_cap = 1;
    // the rebalancing loop as one CUDA graph (a while node over one sub-round),
    // built for the binding and the proposal schedule it was captured with
    cudaStream_t s_cap = nullptr;     // capture stream (non-blocking)
    cudaGraphExec_t reb_exec = nullptr;
    uint64_t gen = 0, reb_gen = ~0ull;  // binding generation; the one reb_exec belongs to
    LaneCfg reb_cfg{};
    int reb_body_kernels = 0;
    cudaStream_t s_up = nullptr;      // binding: the early upload of the adjacency
    cudaEvent_t ev_up = nullptr, ev_prev = nullptr;
    int64_t *xs = nullptr;            // binding: the packed offsets and the schedule counts (bind.cu), kept
    int64_t xs_cap = 0;
    HostSeg *segs_d = nullptr;        // binding a batch: the segments of a gather of host arrays, kept
    int64_t segs_cap = 0;
    int reb_if_kernels = 0;           // kernels of the conditional sort passes in the sub-round body
    cudaStream_t s_if = nullptr;      // capture stream of that conditional body
    int64_t rounds_bound = 0;         // rounds run since the binding
    bool cut_pending = false;         // the next build also computes the cut of part0 (load_part skipped it)
    int32_t lp_attempts = 0;          // label propagation rounds run by the current call (kept or not)
    bool reb_failed = false;          // capture or instantiation failed: host-driven loop
    // the whole refinement after round 1's table build as one CUDA graph
    // (params.graphs == 2): every round's launches, each rebalancing loop a
    // while node; built on a binding's second call of the same shape
    cudaGraphExec_t step_exec = nullptr;
    cudaStream_t s_body = nullptr;    // captures the while nodes' bodies
    uint64_t step_gen = ~0ull;
    int32_t step_rounds = -1, step_off = -1, step_total = -1, step_lock = -1;
    bool step_cut = false;            // captured with round 1 summing the input cut (cut_pending)
    LaneCfg step_sel{}, step_prop{};
    bool step_failed = false, capturing = false;
    int32_t cap_round = 0;            // while capturing: index of the round in the call (0-based)
    long long step_kernels = 0;       // kernels of the step graph outside the while bodies
    int64_t *F_all = nullptr; int64_t *hF_all = nullptr; int32_t F_all_cap = 0;   // [rounds][kSlots]
    int64_t calls_bound = 0;          // refinement calls since the binding
    // every host value of a binding that a captured launch can depend on (the
    // sizes, the schedules' counts, the key widths, the arena, the parameters,
    // the graphs' offsets and limits): a rebinding to a graph with the same
    // key, with nothing invalidated since, keeps the captured graphs
    std::vector<int64_t> bkey;
    uint64_t bkey_gen = ~0ull;        // gen when bkey was taken
    int64_t eps_ppm = 0, total_w = 0, Lmax = 0, wmax = 0;   // one graph: its eps, c(V), L_max
    std::vector<int64_t> noff, Lmax_g;                        // per graph: first node, L_max
    int gbits = 1, cbits = 1;
    upr_params prm{};
    cudaStream_t s = nullptr;
    GraphDev G{};

    void *mem = nullptr;
    size_t mem_bytes = 0;
    // graph
    int64_t *xadj; int32_t *adj, *adjw, *vwgt, *wI;
    HubChunk *hub_chunks; int64_t n_chunks = 0;
    TableTile *tiles = nullptr; int64_t n_tiles = 0; int32_t tile_nodes = 0;
    int64_t *Lb; int32_t *gid;          // [K] L_max per block; [n] graph of each node (batches)
    int64_t *Lsel;                      // [K] the selection's block limit in a limited round (Sec. 7.2)
    int8_t *lp_active, *lp_next;        // [n] label propagation: V_a and the next V_a (Sec. 5)
    int8_t *locked;                     // [n] the oscillation guard's locks for the next round (Sec. 2)
    int32_t *seg_beg, *seg_end, *over0_g, *light_g, *infeas_g, *inf0_g; long long *best_g, *best_j; int64_t *tot;
    int32_t *part_in;                   // batches: the input partition (global ids)
    int64_t *noff_d;                    // batches: [ng + 1] first node of each graph
    // state
    int32_t *part0, *part; int64_t *C0, *C, *cut; int32_t *W;
    int64_t *BW, *PW, *F; int8_t *first_slot;
    // node-indexed
    int32_t *cand_tgt, *cand_gain, *flags, *flags2, *excl_i, *m_pos, *r_to, *r_at, *pos, *dest, *prop_tgt, *prop_gain;
    int64_t *cand_s0;
    // lists
    int32_t *idxA, *idxB, *idxC, *idxD, *L1, *Pq;
    int64_t *score;
    int32_t *M_node, *M_from, *M_to; int64_t *M_score;
    int32_t *R_node, *R_from, *R_to, *R_sub;
    int32_t *X_node, *X_from, *X_to, *final_to; int8_t *X_isr;
    int32_t *I_node, *I_from, *I_to; int64_t *I_gain, *Gsum;
    SortBuf sb[3];
    int64_t *c_sorted, *c_excl, *delta, *d_excl;
    uint64_t *packed, *qmax;
    uint64_t *prio_rep;                 // [2 * kPrioBins] rebalancing: a key per prefilter bin
    int32_t *emit, *qbefore, *em_excl, *pos_m;
    int32_t *diff, *diff_excl;
    int32_t *hub_flag, *hub_excl, *hubs;
    int32_t *seg_first, *rbeg, *rend, *ebeg, *eend, *qfin, *left, *left_excl;
    long long *best_parts, *best;
    int8_t *over_d, *excl_d, *reject_d;
    long long *Cd;                   // [K] block-weight changes of a fused rebalancing sub-round
    unsigned long long *prio_hist;   // [K][kPrioBins] proposal prefilter (null: K too large, no prefilter)
    int32_t *prio_cut;               // [K]
    int32_t *counts;          // device counters (CNT_* slots)
    RebalCtl *ctl;            // rebalancing loop control block
    long long *dstats;        // [16] per-call sums of the step graph's rounds
    uint64_t *vacc; int32_t *vflags; int64_t *scal, *cut_parts;
    int2 *pk;                 // exact gains: position in I and blocks before/after, per node
    Scratch tmp;              // scan / sort temporaries
    // pinned host mirrors
    int64_t *h = nullptr;     // pinned scratch
    int8_t *h8 = nullptr;
    int64_t *hF = nullptr, *hcut = nullptr;
    int32_t *hcnt = nullptr;
    long long *hbest = nullptr;
    RebalCtl *hctl = nullptr;
    cudaEvent_t ev[8] = {};
    int64_t *hx = nullptr; int64_t hx_cap = 0;   // pinned staging of a batch's packed xadj (kept across bindings)
};

namespace {

void layout(upr_ctx *c, Arena &A) {
    const size_t n = (size_t)std::max<int64_t>(c->n, 1), m = (size_t)std::max<int64_t>(c->m, 1);
    const size_t kr = (size_t)c->k;                   // table row width
    const size_t k = (size_t)c->k * (size_t)c->ng;    // blocks (K)
    const size_t ng = (size_t)c->ng;
    const size_t n2 = 2 * n;
    c->Lb = A.take<int64_t>(k);
    c->Lsel = A.take<int64_t>(k);
    c->lp_active = A.take<int8_t>(n);
    c->locked = A.take<int8_t>(n);
    c->lp_next = A.take<int8_t>(n);
    c->gid = c->ng > 1 ? A.take<int32_t>(n) : nullptr;
    c->part_in = c->ng > 1 ? A.take<int32_t>(n) : nullptr;
    c->noff_d = A.take<int64_t>(ng + 1);
    for (int32_t **p : {&c->seg_beg, &c->seg_end, &c->over0_g, &c->light_g, &c->infeas_g, &c->inf0_g})
        *p = A.take<int32_t>(ng);
    c->best_g = A.take<long long>(ng);
    c->best_j = A.take<long long>(ng);
    c->tot = A.take<int64_t>(4);
    c->xadj = A.take<int64_t>(n + 1);
    c->adj = A.take<int32_t>(m);
    c->adjw = A.take<int32_t>(m);
    c->vwgt = A.take<int32_t>(n);
    c->wI = A.take<int32_t>(n);
    c->hub_chunks = A.take<HubChunk>((size_t)std::max<int64_t>(c->n_chunks, 1));
    c->tiles = A.take<TableTile>((size_t)std::max<int64_t>(c->n_tiles, 1));
    c->sp_off = c->sp_slots ? A.take<int64_t>(n + 1) : nullptr;
    c->sp_slot = c->sp_slots ? A.take<int2>((size_t)c->sp_slots) : nullptr;
    c->sp_over = A.take<int32_t>(1);
    c->part0 = A.take<int32_t>(n);
    c->part = A.take<int32_t>(n);
    c->C0 = A.take<int64_t>(k);
    c->C = A.take<int64_t>(k);
    c->cut = A.take<int64_t>(std::max<size_t>(ng, 4));
    c->W = c->sp_slots ? nullptr : A.take<int32_t>(n * kr);
    c->BW = A.take<int64_t>(k * kSlots);
    c->PW = A.take<int64_t>(k * kSlots);
    c->F = A.take<int64_t>(kSlots);
    c->first_slot = A.take<int8_t>(k);
    for (int32_t **p : {&c->cand_tgt, &c->cand_gain, &c->flags, &c->m_pos, &c->r_to, &c->pos, &c->dest, &c->prop_tgt,
                        &c->prop_gain, &c->idxA, &c->idxB, &c->idxC, &c->M_node, &c->M_from, &c->M_to, &c->R_node,
                        &c->R_from, &c->R_to, &c->R_sub, &c->I_node, &c->I_from, &c->I_to, &c->emit, &c->qbefore,
                        &c->em_excl, &c->pos_m, &c->hub_flag, &c->hub_excl, &c->hubs, &c->L1, &c->r_at, &c->Pq})
        *p = A.take<int32_t>(n);
    for (int32_t **p : {&c->flags2, &c->excl_i, &c->idxD, &c->X_node, &c->X_from, &c->X_to, &c->final_to})
        *p = A.take<int32_t>(n2 + 1);
    c->diff = A.take<int32_t>(n + 2);
    c->diff_excl = A.take<int32_t>(n + 2);
    c->X_isr = A.take<int8_t>(n2);
    c->cand_s0 = A.take<int64_t>(n);
    c->score = A.take<int64_t>(n);
    c->M_score = A.take<int64_t>(n);
    c->I_gain = A.take<int64_t>(n);
    c->Gsum = A.take<int64_t>(n);
    for (int i = 0; i < 3; i++) {
        c->sb[i].k = A.take<uint64_t>(n2);
        c->sb[i].ka = A.take<uint64_t>(n2);
        c->sb[i].v = A.take<uint32_t>(n2);
        c->sb[i].va = A.take<uint32_t>(n2);
    }
    c->c_sorted = A.take<int64_t>(n2);
    c->c_excl = A.take<int64_t>(n2);
    c->delta = A.take<int64_t>(n2);
    c->d_excl = A.take<int64_t>(n2);
    c->packed = A.take<uint64_t>(n2);
    c->qmax = A.take<uint64_t>(n2);
    c->prio_rep = A.take<uint64_t>(2 * (size_t)kPrioBins);
    for (int32_t **p : {&c->seg_first, &c->rbeg, &c->rend, &c->ebeg, &c->eend, &c->qfin, &c->left, &c->left_excl})
        *p = A.take<int32_t>(k);
    c->best_parts = A.take<long long>(2048);
    c->best = A.take<long long>(2);
    c->over_d = A.take<int8_t>(k);
    c->excl_d = A.take<int8_t>(k);
    c->reject_d = A.take<int8_t>(k);
    c->Cd = A.take<long long>(k);
    const bool prefilter = k * (size_t)kPrioBins <= ((size_t)1 << 22);
    c->prio_hist = prefilter ? A.take<unsigned long long>(k * kPrioBins) : nullptr;
    c->prio_cut = prefilter ? A.take<int32_t>(k) : nullptr;
    c->counts = A.take<int32_t>(64);
    c->ctl = A.take<RebalCtl>(1);
    c->dstats = A.take<long long>(16);
    c->vacc = A.take<uint64_t>(2);
    c->vflags = A.take<int32_t>(2);
    c->scal = A.take<int64_t>(4);    // [0] wmax, [1] degree sum of M, [2] degree sum of undone moves
    c->cut_parts = A.take<int64_t>(kCutParts + 1);   // twice the input cut: partial sums, total
    c->pk = A.take<int2>(n);
    c->tmp.tiles_cap = ceil_div(std::max<int64_t>((int64_t)n2 + 2, (int64_t)k + 2), 2048);   // lists of nodes, events, blocks
    c->tmp.mem_bytes = radix_temp_bytes(c->tmp.tiles_cap * 2048);
    c->tmp.scan_bytes = scan_temp_bytes(c->tmp.tiles_cap * 2048);
    c->tmp.mem = A.take<char>(c->tmp.mem_bytes);
    c->tmp.scan = A.take<char>(c->tmp.scan_bytes);
    c->tmp.ticket = A.take<unsigned int>(64);
    c->tmp.err = A.take<int32_t>(1);
    c->tmp.epoch = A.take<uint32_t>(1);
}

enum MemKind { kHost = 0, kDevice = 1 };

MemKind mem_kind(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { cudaGetLastError(); return kHost; }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? kDevice : kHost;
}

void copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    UPR_CUDA(cudaMemcpyAsync(dst, src, bytes, mem_kind(src) == kDevice ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

void copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    UPR_CUDA(cudaMemcpyAsync(dst, src, bytes, mem_kind(dst) == kDevice ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

// Page-locked host memory that kernels read at the same address.
bool host_locked(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

// The copies dst[off_i .. off_i + len_i) <- src_i (elements of `elem` bytes):
// one gather launch that reads the sources where they are when every one is
// page-locked host memory (a batch's thousands of small arrays would
// otherwise be as many DMA transfers), one copy each otherwise.
void copy_many(upr_ctx *c, const std::vector<const void *> &src, const std::vector<int64_t> &off,
               const std::vector<int64_t> &len, size_t elem, void *dst, cudaStream_t s) {
    bool locked = src.size() > 1;                    // (one array: one DMA transfer)
    for (size_t i = 0; i < src.size() && locked; i++) locked = len[i] <= 0 || host_locked(src[i]);
    if (!locked) {
        for (size_t i = 0; i < src.size(); i++)
            if (len[i] > 0) copy_in(static_cast<char *>(dst) + off[i] * elem, src[i], len[i] * elem, s);
        return;
    }
    std::vector<HostSeg> segs;
    for (size_t i = 0; i < src.size(); i++)
        for (int64_t b = 0; b < len[i]; b += kGatherChunk)
            segs.push_back(HostSeg{static_cast<const char *>(src[i]) + b * elem, off[i] + b,
                                   std::min<int64_t>(kGatherChunk, len[i] - b)});
    if (segs.empty()) return;
    if (c->segs_cap < (int64_t)segs.size()) {
        UPR_CUDA(cudaStreamSynchronize(s));          // (a gather queued earlier may still read them)
        if (c->segs_d) cudaFree(c->segs_d);
        c->segs_d = nullptr;
        c->segs_cap = 0;
        UPR_CUDA(cudaMalloc(&c->segs_d, sizeof(HostSeg) * segs.size()));
        c->segs_cap = (int64_t)segs.size();
    }
    // (from pageable memory: the copy waits for the work queued on s, so an
    // earlier gather has read its segments by then)
    UPR_CUDA(cudaMemcpyAsync(c->segs_d, segs.data(), sizeof(HostSeg) * segs.size(), cudaMemcpyHostToDevice, s));
    gather_host(c->segs_d, (int64_t)segs.size(), elem, dst, s);
}

int32_t read_count(upr_ctx *c, int slot) {
    UPR_CUDA(cudaMemcpyAsync(c->h, c->counts + slot, sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
    UPR_CUDA(cudaStreamSynchronize(c->s));
    return *reinterpret_cast<int32_t *>(c->h);
}

void read_i64(upr_ctx *c, const int64_t *src, int64_t cnt, int64_t *dst) {
    if (cnt <= 4 * (int64_t)kMaxK) {           // through the pinned buffer
        UPR_CUDA(cudaMemcpyAsync(c->h, src, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost, c->s));
        UPR_CUDA(cudaStreamSynchronize(c->s));
        memcpy(dst, c->h, sizeof(int64_t) * cnt);
    } else {
        UPR_CUDA(cudaMemcpyAsync(dst, src, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost, c->s));
        UPR_CUDA(cudaStreamSynchronize(c->s));
    }
}

void read_i32(upr_ctx *c, const int32_t *src, int64_t cnt, int32_t *dst) {
    UPR_CUDA(cudaMemcpyAsync(dst, src, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, c->s));
    UPR_CUDA(cudaStreamSynchronize(c->s));
}

struct RoundInfo {
    int64_t n_cand = 0, n_moves = 0, n_rebal = 0, n_inter = 0, n_seq = 0, best_len = 0, best_gain = 0;
    int32_t subrounds = 0;
    float ms_table = 0, ms_select = 0, ms_rebalance = 0, ms_sequence = 0;
    int tables = 0;
    bool graph = false;         // the rebalancing loop ran as one graph launch
    bool constrained = false;   // a constrained round (Sec. 6.2)
};

// Trace destinations on the host (debug entry only).
struct TraceSink { upr_trace *t; int8_t *avail_d; int32_t *slot_d; };

void d2h(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (dst && bytes) UPR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
}

// ---- lane-schedule tuning.  A kernel whose schedule is not chosen yet runs
// every candidate back to back on the same inputs (each run rewrites the
// same outputs, all equal), timed with events; the times are read after the
// next synchronisation the round makes anyway.  Small inputs keep the
// default (nothing to gain, and their timings would be launch noise).
bool worth_tuning(const upr_ctx *c) { return c->prm.autotune && (int64_t)c->n * c->k >= ((int64_t)1 << 22); }

template <typename F>
void run_tuned(upr_ctx *c, bool tuned, LaneCfg cfg, LaneCfg *cands, int *pending, cudaEvent_t *ev, F launch) {
    *pending = 0;
    if (!tuned && worth_tuning(c)) {
        const int nc = lane_candidates(c->k, cands);
        if (nc > 1) {
            for (int i = 0; i < nc; i++) {
                UPR_CUDA(cudaEventRecord(ev[2 * i], c->s));
                launch(cands[i]);
                UPR_CUDA(cudaEventRecord(ev[2 * i + 1], c->s));
            }
            *pending = nc;
            return;
        }
    }
    launch(cfg);
}

// Schedules found by tuning, shared by the contexts of the process: keyed by
// device, k, the table layout, one graph or a batch, and the size class
// (log2 of n), so a context bound to a graph like one tuned before starts
// with its schedules instead of timing the candidates again.
struct TuneKey {
    int dev, k, sparse, batch, size_class, which;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, k, sparse, batch, size_class, which) <
               std::tie(o.dev, o.k, o.sparse, o.batch, o.size_class, o.which);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, LaneCfg> g_tuned;

TuneKey tune_key(const upr_ctx *c, int which) {
    return TuneKey{c->device, c->k, c->G.sp.on() ? 1 : 0, c->ng > 1 ? 1 : 0, bit_length((uint64_t)c->n), which};
}

void remember_tuning(const upr_ctx *c, int which, LaneCfg cfg) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(c, which)] = cfg;
}

void recall_tuning(upr_ctx *c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto a = g_tuned.find(tune_key(c, 0)), b = g_tuned.find(tune_key(c, 1));
    if (a != g_tuned.end()) { c->sel_cfg = a->second; c->sel_tuned = true; }
    if (b != g_tuned.end()) { c->prop_cfg = b->second; c->prop_tuned = true; }
}

// After a synchronisation: keep the fastest candidate if the work was large
// enough to tell them apart (otherwise try again next time).
void settle_tuning(LaneCfg *cfg, bool *tuned, int *pending, const LaneCfg *cands, cudaEvent_t *ev, float min_ms) {
    if (*pending <= 1) return;
    int best = 0;
    float tbest = 0;
    for (int i = 0; i < *pending; i++) {
        float t = 0;
        UPR_CUDA(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
        if (i == 0 || t < tbest) { tbest = t; best = i; }
    }
    if (tbest >= min_ms) {
        *cfg = cands[best];
        *tuned = true;
    }
    *pending = 0;
}

// The selection's one-integer column scores (unit node weights, one graph,
// gains and column bits within 30 bits).
void set_pack(const upr_ctx *c, Penalty &pen) {
    const int kb = std::max(1, bit_length((uint64_t)(c->G.k - 1)));
    if (c->ng == 1 && !c->G.vwgt && c->gbits + kb <= 30) {
        pen.pack_bits = kb;
        pen.gbits = c->gbits;
    }
}

// The fused form of a rebalancing sub-round applies: one graph, K <= 256, a
// one-word key, the prefilter, and per-(block, tile) sums that fit the
// 2n-entry buffers they use (UPR_FUSED=0 in the environment turns it off:
// the general form computes the same sub-round).
bool fused_rebalance(const upr_ctx *c, int key_bits) {
    static int env = -1;
    if (env < 0) { const char *v = getenv("UPR_FUSED"); env = (v && *v == '0') ? 0 : 1; }
    const int64_t n = std::max<int64_t>(c->n, 1);
    return env == 1 && rebalance_fused_ok(c->G, key_bits, c->prio_hist != nullptr) &&
           (int64_t)c->G.K() * ceil_div(n, (int64_t)2048) <= 2 * n;
}

// The fused sub-round's steps after the proposals in one cooperative launch
// (UPR_MEGA=0 in the environment: one launch per step, the same results).
bool mega_rebalance() {
    static int env = -1;
    if (env < 0) {
        const char *v = getenv("UPR_MEGA");
        int coop = 0, dev = 0;
        UPR_CUDA(cudaGetDevice(&dev));
        UPR_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        env = (v && *v == '0') || !coop ? 0 : 1;
    }
    return env == 1;
}

// One rebalancing sub-round (Sec. 6), enqueued on s.  Every argument is fixed
// for the binding (the sub-round number and every list length live in device
// memory), so the same launches can be captured once and replayed.  first:
// the round's first sub-round, which may time the proposal kernel's lane
// schedules (host-driven loop only).  cond: the condition of a graph-resident
// loop; returns true when the sub-round's last kernel has set it (else the
// caller adds rebalance_continue).
bool enqueue_subround(upr_ctx *c, const RebalState &st, int32_t *light, bool first, cudaStream_t s,
                      cudaGraphConditionalHandle cond = 0) {
    const GraphDev &G = c->G;
    const int64_t n = c->n;
    const int kbits = std::max(1, bit_length((uint64_t)(G.K() - 1)));
    int32_t *cnt = c->counts;
    RebalCtl *ctl = c->ctl;
    const Count cS{cnt + CNT_S, n};
    // a graph-resident loop in the fused form begins each sub-round at the
    // end of the one before (and the first before the loop, merged_loop_head)
    const bool merged = cond && fused_rebalance(c, 1 + c->gbits + 2 * c->cbits);
    if (!merged)
        rebalance_begin(G, c->C, c->excl_d, c->over_d, c->reject_d, cnt + CNT_L1, c->prm.max_subrounds, ctl, light,
                        s);
    if (first)
        run_tuned(c, c->prop_tuned, c->prop_cfg, c->prop_cands, &c->prop_pending, c->ev_tune + 6,
                  [&](LaneCfg cfg) {
                      rebalance_propose_list(G, c->L1, &ctl->n1_active, n, c->part, c->W, st, c->prop_tgt,
                                             c->prop_gain, c->flags, cfg, s);
                  });
    else
        rebalance_propose_list(G, c->L1, &ctl->n1_active, n, c->part, c->W, st, c->prop_tgt, c->prop_gain,
                               c->flags, c->prop_cfg, s);
    // the proposers, in node order, are the next sub-round's list: a listed
    // node without a proposal has no block with room for it (the lightest
    // allowed block has the most room, and rooms only shrink), so it never
    // proposes again
    const int key_bits = 1 + c->gbits + 2 * c->cbits;
    if (fused_rebalance(c, key_bits)) {
        // the same sub-round in fused passes (reb_fused.cu): the proposers
        // with the prefilter histogram, the cut bins, the kept proposals as
        // (key, node), one sort by key, selection and admission from
        // per-tile block sums, R appended and the moves applied
        uint64_t *rep = c->prio_rep;
        int32_t *exact = cnt + CNT_EXACT;
        if (mega_rebalance()) {
            // steps 1 and 3-7 in one cooperative launch (the sort buffers of
            // sb[1] and sb[2] hold the compacted proposers: free here)
            RebalMega m{};
            m.flags = c->flags;
            m.list = c->L1;
            m.lsrc = st.lsrc;
            m.lgain = st.lgain;
            m.d_n1 = &ctl->n1_active;
            m.list2 = reinterpret_cast<int32_t *>(c->sb[1].v);
            m.lsrc2 = reinterpret_cast<int32_t *>(c->sb[1].va);
            m.lgain2 = reinterpret_cast<int32_t *>(c->sb[2].v);
            m.gbits = c->gbits;
            m.cbits = c->cbits;
            m.gain_only = c->prm.gain_priority;
            m.hist = c->prio_hist;
            m.rep = rep;
            m.cut = c->prio_cut;
            m.over = c->over_d;
            m.C = c->C;
            m.keys = c->sb[0].k;
            m.keys_alt = c->sb[0].ka;
            m.vals = c->sb[0].v;
            m.vals_alt = c->sb[0].va;
            m.part = c->part;
            m.prop_tgt = c->prop_tgt;
            m.sel = reinterpret_cast<int8_t *>(c->flags2);
            m.h0 = reinterpret_cast<long long *>(c->c_sorted);
            m.h1 = reinterpret_cast<long long *>(c->c_excl);
            m.reject = c->reject_d;
            m.ctl = ctl;
            m.R_node = c->R_node; m.R_from = c->R_from; m.R_to = c->R_to; m.R_sub = c->R_sub;
            m.r_to = c->r_to; m.r_at = c->r_at;
            m.Cd = c->Cd;
            m.d_np = cnt + CNT_L1;
            m.d_nk = cnt + CNT_P;
            m.d_na = cnt + CNT_A;
            m.exact = exact;
            rebalance_fused_mega(G, m, key_bits, n, c->tmp, s);
            table_move(G, c->W, c->R_node, c->R_from, c->R_to, cnt + CNT_A, &ctl->nR, nullptr, n, c->hub_chunks,
                       c->n_chunks, HubMoves{nullptr, c->r_to, c->r_at, &ctl->nR, cnt + CNT_A, c->R_from, c->R_to}, s);
            rebalance_fused_end(G, c->C, c->Cd, c->excl_d, c->reject_d, cnt + CNT_A, ctl, s, cond,
                                c->prm.max_subrounds, merged ? c->over_d : nullptr, c->reject_d, cnt + CNT_L1);
            return cond != 0;
        }
        rebalance_fused_compact_hist(G, c->flags, c->L1, &ctl->n1_active, n, cnt + CNT_L1, st.lgain, st.lsrc,
                                     c->gbits, c->cbits, c->prm.gain_priority, c->prio_hist, rep, exact, c->tmp, s);
        rebalance_prio_cut(G, c->over_d, c->C, c->prio_hist, c->prio_cut, s);
        rebalance_fused_keep_keys(G, c->L1, cnt + CNT_L1, n, st.lgain, st.lsrc, c->prio_cut, c->gbits, c->cbits,
                                  c->prm.gain_priority, c->sb[0].k, c->sb[0].v, cnt + CNT_P, rep, exact, c->tmp, s);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        static int if_env = -1;
        if (if_env < 0) { const char *v = getenv("UPR_SORT_IF"); if_env = (v && *v == '0') ? 0 : 1; }
        if (if_env) UPR_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusActive && !c->s_if)
            UPR_CUDA(cudaStreamCreateWithFlags(&c->s_if, cudaStreamNonBlocking));
        int if_kernels = 0;
        rebalance_fused_sort(c->sb[0].k, c->sb[0].v, c->sb[0].ka, c->sb[0].va, cnt + CNT_P, n, key_bits, c->gbits,
                             c->cbits, exact, c->tmp, s, c->s_if, cnt + CNT_SORTP, &if_kernels);
        if (cs == cudaStreamCaptureStatusActive) c->reb_if_kernels = if_kernels;
        const uint32_t *U = c->sb[0].va;
        rebalance_fused_select_admit(G, U, cnt + CNT_P, n, c->part, c->prop_tgt, c->C,
                                     reinterpret_cast<int8_t *>(c->flags2), reinterpret_cast<long long *>(c->c_sorted),
                                     reinterpret_cast<long long *>(c->c_excl), cnt + CNT_HIST, c->reject_d, ctl,
                                     c->R_node, c->R_from, c->R_to, c->R_sub, c->r_to, c->r_at, c->Cd, cnt + CNT_A,
                                     c->tmp, s);
        table_move(G, c->W, c->R_node, c->R_from, c->R_to, cnt + CNT_A, &ctl->nR, nullptr, n, c->hub_chunks,
                   c->n_chunks, HubMoves{nullptr, c->r_to, c->r_at, &ctl->nR, cnt + CNT_A, c->R_from, c->R_to}, s);
        rebalance_fused_end(G, c->C, c->Cd, c->excl_d, c->reject_d, cnt + CNT_A, ctl, s, cond, c->prm.max_subrounds,
                            merged ? c->over_d : nullptr, c->reject_d, cnt + CNT_L1);
        return cond != 0;
    }
    select_values(c->flags, c->L1, c->L1, cnt + CNT_L1, Count{&ctl->n1_active, n}, c->tmp, s);
    // proposals that cannot be in their source's minimal prefix are dropped
    // before the ordering; P lists the others in node order
    const int32_t *Pn = c->L1;
    int32_t *dP = cnt + CNT_L1;
    if (c->prio_hist) {
        rebalance_prefilter(G, c->L1, cnt + CNT_L1, n, nullptr, c->prop_gain, c->part, c->over_d, c->C, c->gbits,
                            c->cbits, c->prm.gain_priority, c->prio_hist, c->prio_cut, c->flags2, s);
        select_values(c->flags2, c->L1, c->Pq, cnt + CNT_P, Count{cnt + CNT_L1, n}, c->tmp, s);
        Pn = c->Pq;
        dP = cnt + CNT_P;
    }
    const Count cP{dP, n};
    uint64_t *kA; uint32_t *A;
    if (key_bits <= 63) {
        rebalance_prio_keys(G, Pn, dP, c->prop_gain, c->gbits, c->cbits, c->prm.gain_priority, c->sb[0].k,
                            c->sb[0].v, n, s);
        c->sb[0].run(cP, key_bits, c->tmp, s, &kA, &A);
    } else {                // a 128-bit key: two stable sorts in sb[0]'s buffers
        rebalance_prio_sort_wide(G, Pn, dP, c->prop_gain, c->gbits, c->cbits, c->prm.gain_priority,
                                 SortPairs{c->sb[0].k, c->sb[0].ka, c->sb[0].v, c->sb[0].va}, n, c->tmp, s, &A);
    }
    // per source: the minimal prefix covering the excess
    uint64_t *kB; uint32_t *B;
    rebalance_block_keys(Pn, A, nullptr, dP, c->part, c->sb[1].k, c->sb[1].v, n, s);
    c->sb[1].run(cP, kbits, c->tmp, s, &kB, &B);
    rebalance_seg_weights(G, Pn, A, nullptr, B, kB, dP, c->c_sorted, c->seg_first, n, s);
    exclusive_sum_i64(c->c_sorted, c->c_excl, cP, c->tmp, s);
    rebalance_mark_selected(B, kB, dP, c->c_excl, c->seg_first, st, c->flags2, n, s);
    select_flags(c->flags2, c->idxB, cnt + CNT_S, cP, c->tmp, s);
    // per target: the longest prefix that fits
    uint64_t *kT; uint32_t *Tq;
    rebalance_block_keys(Pn, A, c->idxB, cnt + CNT_S, c->prop_tgt, c->sb[2].k, c->sb[2].v, n, s);
    c->sb[2].run(cS, kbits, c->tmp, s, &kT, &Tq);
    rebalance_seg_weights(G, Pn, A, c->idxB, Tq, kT, cnt + CNT_S, c->c_sorted, c->seg_first, n, s);
    exclusive_sum_i64(c->c_sorted, c->c_excl, cS, c->tmp, s);
    rebalance_mark_admitted(Tq, kT, cnt + CNT_S, c->c_sorted, c->c_excl, c->seg_first, st, c->flags2, c->reject_d,
                            n, s);
    select_flags(c->flags2, c->idxC, cnt + CNT_A, cS, c->tmp, s);
    rebalance_apply(G, Pn, A, c->idxB, c->idxC, cnt + CNT_A, c->prop_tgt, c->part, c->C, ctl, c->R_node,
                    c->R_from, c->R_to, c->R_sub, c->r_to, c->r_at, n, s);
    table_move(G, c->W, c->R_node, c->R_from, c->R_to, cnt + CNT_A, &ctl->nR, nullptr, n, c->hub_chunks,
               c->n_chunks, HubMoves{nullptr, c->r_to, c->r_at, &ctl->nR, cnt + CNT_A, c->R_from, c->R_to}, s);
    rebalance_end(G, c->C, c->excl_d, c->reject_d, cnt + CNT_A, ctl, s);
    return false;
}

// The kernel before a graph-resident loop: the fused form begins the first
// sub-round there (setting the condition), the general form only sets the
// condition (its body begins each sub-round itself).
void loop_head(upr_ctx *c, int32_t *light, cudaGraphConditionalHandle cond, cudaStream_t s) {
    if (fused_rebalance(c, 1 + c->gbits + 2 * c->cbits))
        rebalance_begin(c->G, c->C, c->excl_d, c->over_d, c->reject_d, c->counts + CNT_L1, c->prm.max_subrounds,
                        c->ctl, light, s, cond);
    else
        rebalance_continue(c->ctl, c->prm.max_subrounds, cond, s);
}

// The rebalancing loop as a graph: a kernel sets the condition of a while
// node whose body is one sub-round followed by the same kernel.  Built on
// first use for the binding and the proposal schedule, then replayed; false
// if the graph cannot be built (the host-driven loop is used instead).
bool rebalance_graph(upr_ctx *c, const RebalState &st, int32_t *light) {
    if (c->reb_failed) return false;
    if (c->reb_exec && c->reb_gen == c->gen && c->reb_cfg.G == c->prop_cfg.G && c->reb_cfg.CH == c->prop_cfg.CH)
        return true;
    if (c->reb_exec) { cudaGraphExecDestroy(c->reb_exec); c->reb_exec = nullptr; }
    cudaGraph_t g = nullptr;
    bool capturing = false;
    long long captured = 0;
    try {
        if (!c->s_cap) UPR_CUDA(cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking));
        UPR_CUDA(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle cond;
        UPR_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
        UPR_CUDA(cudaStreamBeginCaptureToGraph(c->s_cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        capturing = true;
        loop_head(c, light, cond, c->s_cap);
        captured++;
        cudaGraph_t out = nullptr;
        capturing = false;
        UPR_CUDA(cudaStreamEndCapture(c->s_cap, &out));
        cudaGraphNode_t head[1];
        size_t n_head = 1;
        UPR_CUDA(cudaGraphGetNodes(g, head, &n_head));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop;
        UPR_CUDA(cudaGraphAddNode(&loop, g, head, nullptr, n_head, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        UPR_CUDA(cudaStreamBeginCaptureToGraph(c->s_cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        capturing = true;
        const long long b0 = g_upr_launches;
        if (!enqueue_subround(c, st, light, false, c->s_cap, cond))
            rebalance_continue(c->ctl, c->prm.max_subrounds, cond, c->s_cap);
        c->reb_body_kernels = (int)(g_upr_launches - b0);
        captured += c->reb_body_kernels;
        capturing = false;
        UPR_CUDA(cudaStreamEndCapture(c->s_cap, &out));
        UPR_CUDA(cudaGraphInstantiate(&c->reb_exec, g, 0));
        cudaGraphDestroy(g);
    } catch (const CudaError &e) {
        if (capturing) {
            cudaGraph_t out = nullptr;
            cudaStreamEndCapture(c->s_cap, &out);
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (log_enabled()) fprintf(stderr, "upr: rebalancing graph not built (%s: %s)\n", e.what,
                                   cudaGetErrorString(e.e));
        c->reb_exec = nullptr;
        c->reb_failed = true;
    }
    g_upr_launches -= (captured);     // captured, not launched: counted when the graph runs
    c->reb_gen = c->gen;
    c->reb_cfg = c->prop_cfg;
    return c->reb_exec != nullptr;
}

// Step (d): the rebalancing sub-rounds (Sec. 6) on c->part / c->C / the table,
// host-driven or as one graph launch.  r: the round (for the log).
void rebalance_phase(upr_ctx *c, int32_t r, RoundInfo &ri, TraceSink *tr) {
    cudaStream_t s = c->s;
    const GraphDev &G = c->G;
    const int64_t n = c->n;
    const int32_t K = G.K();
    const bool batch = c->ng > 1;
    int32_t *cnt = c->counts;
    RebalCtl *ctl = c->ctl;
    const Count cN{nullptr, n};
    if (c->prio_hist)
        UPR_CUDA(cudaMemsetAsync(c->prio_hist, 0, sizeof(unsigned long long) * K * kPrioBins, s));
    rebalance_init(G, c->C, c->excl_d, ctl, s);
    rebalance_flag_in_blocks(c->part, n, c->excl_d, c->flags, s);
    select_flags(c->flags, c->L1, cnt + CNT_L1, cN, c->tmp, s);
    int32_t *light = batch ? c->light_g : &ctl->light;
    RebalState st{c->C, c->over_d, c->excl_d, light, c->Lb};
    {
        const int kb = std::max(1, bit_length((uint64_t)(G.k - 1)));
        if (!batch && !G.vwgt && c->gbits + kb <= 31) st.pack_bits = kb;
    }
    if (fused_rebalance(c, 1 + c->gbits + 2 * c->cbits)) {
        st.lsrc = c->emit;          // list-indexed proposal blocks and gains (sequence-phase arrays, free here)
        st.lgain = c->qbefore;
    }
    if (c->capturing) {
        // inside the step graph: the loop as a while node whose body is one
        // sub-round followed by the condition kernel (captured on a side
        // stream into the node's body graph)
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        UPR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle cond;
        UPR_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
        loop_head(c, light, cond, s);
        UPR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop;
        UPR_CUDA(cudaGraphAddNode(&loop, g, deps, nullptr, nd, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (!c->s_body) UPR_CUDA(cudaStreamCreateWithFlags(&c->s_body, cudaStreamNonBlocking));
        UPR_CUDA(cudaStreamBeginCaptureToGraph(c->s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const long long b0 = g_upr_launches;
        if (!enqueue_subround(c, st, light, false, c->s_body, cond))
            rebalance_continue(ctl, c->prm.max_subrounds, cond, c->s_body);
        c->reb_body_kernels = (int)(g_upr_launches - b0);
        cudaGraph_t out = nullptr;
        UPR_CUDA(cudaStreamEndCapture(c->s_body, &out));
        UPR_CUDA(cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1, cudaStreamSetCaptureDependencies));
        ri.graph = true;
        return;
    }
    auto t_sub = std::chrono::steady_clock::now();
    // the loop runs on the device as one graph once the proposal schedule is
    // settled (the host-driven form times the schedules, logs and traces);
    // a small binding first has to run a few rounds to pay for the capture
    const bool tuning = !c->prop_tuned && worth_tuning(c);
    const bool pays = (int64_t)n * c->k >= ((int64_t)1 << 22) || c->rounds_bound >= 8;
    c->rounds_bound++;
    if (c->prm.graphs && pays && !tuning && !tr && !log_enabled() && rebalance_graph(c, st, light)) {
        UPR_CUDA(cudaGraphLaunch(c->reb_exec, s));
        ri.graph = true;
    } else for (int32_t h = 1; h <= c->prm.max_subrounds; h++) {
        enqueue_subround(c, st, light, h == 1, s);
        UPR_CUDA(cudaMemcpyAsync(c->hctl, ctl, sizeof(RebalCtl), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaStreamSynchronize(s));
        if (c->prop_pending) {
            settle_tuning(&c->prop_cfg, &c->prop_tuned, &c->prop_pending, c->prop_cands, c->ev_tune + 6, 0.02f);
            if (c->prop_tuned) remember_tuning(c, 1, c->prop_cfg);
        }
        if (log_enabled()) {
            int32_t hc[CNT_SLOTS];
            UPR_CUDA(cudaMemcpy(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost));
            const auto t1 = std::chrono::steady_clock::now();
            fprintf(stderr, "upr round %d sub-round %d: listed %d proposals %d kept %d selected %d "
                            "admitted %d (%.3f ms)\n",
                    r, h, c->hctl->n1_active, hc[CNT_L1], c->prio_hist ? hc[CNT_P] : hc[CNT_L1], hc[CNT_S],
                    hc[CNT_A],
                    std::chrono::duration<double, std::milli>(t1 - t_sub).count());
            t_sub = std::chrono::steady_clock::now();
        }
        if (c->hctl->stopped) break;
    }
}

/*
 * One round on c->part0 / c->C0 / c->cut (device state).  Every step is
 * enqueued on c->s with its list lengths in device memory; the host waits
 * only for the rebalancing loop's stop flag after each sub-round and for the
 * end of the round.  Returns UPR_OK or UPR_ERR_INFEASIBLE (state unchanged).
 * rebalance_only: the round-0 repair.
 */
constexpr upr_status kRedoDense = 100;     // internal: run the round again on the dense table
constexpr upr_status kRedoFresh = 101;     // internal: run the round again on freshly built sparse rows

upr_status run_round_once(upr_ctx *c, int32_t r, int32_t R, bool rebalance_only, RoundInfo &ri, TraceSink *tr,
                          const RoundKind &kind) {
    cudaStream_t s = c->s;
    const GraphDev &G = c->G;
    const int64_t n = c->n;
    const int32_t K = G.K();
    const bool batch = c->ng > 1;
    const int kbits = std::max(1, bit_length((uint64_t)(K - 1)));
    upr_trace *T = tr ? tr->t : nullptr;
    int32_t *cnt = c->counts;
    RebalCtl *ctl = c->ctl;
    const Count cN{nullptr, n};
    uint64_t *ko; uint32_t *vo;

    UPR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * CNT_SLOTS, s));
    UPR_CUDA(cudaMemcpyAsync(c->part, c->part0, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    UPR_CUDA(cudaMemcpyAsync(c->C, c->C0, sizeof(int64_t) * K, cudaMemcpyDeviceToDevice, s));
    // ---- (a) gain table of the round-start partition (kept from the previous
    // round of this call when it is valid)
    // (in the step graph the table is always carried: round 1's build runs before it)
    const bool cap = c->capturing;
    const bool build = !cap && (!c->table_valid || tr);
    c->table_valid = false;
    if (!cap) UPR_CUDA(cudaEventRecord(c->ev[0], s));
    if (build)
        gain_table(G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, nullptr, s);
    if (!cap) {
        UPR_CUDA(cudaEventRecord(c->ev[1], s));
        UPR_CUDA(cudaEventRecord(c->ev[4], s));
    }
    if (!rebalance_only) {
        // ---- (b1) availability, slots, bucket weights; F_r
        // (the first round of a call also sums the input cut here)
        buckets(G, c->part0, c->W, c->prm.t_num, c->prm.t_den, c->BW, c->PW, c->first_slot,
                tr ? tr->avail_d : nullptr, tr ? tr->slot_d : nullptr, s, c->cut_pending ? c->cut_parts : nullptr,
                c->cut);
        c->cut_pending = false;
        // the step graph reads round i's factors from the per-call table F_all
        const int64_t *F = cap ? c->F_all + (int64_t)c->cap_round * kSlots : c->F;
        if (!cap) {
            if (kind.constrained || kind.limit > 0)
                for (int l = 0; l < kSlots; l++) c->hF[l] = kConstrainedF;
            else if (kind.tau_den > 0)
                factors_tau((u128)kind.tau_num, (u128)kind.tau_den, c->hF);
            else
                penalty_factors(r, R, c->prm.tau1_num, c->prm.tau1_den, c->hF);
            UPR_CUDA(cudaMemcpyAsync(c->F, c->hF, sizeof(int64_t) * kSlots, cudaMemcpyHostToDevice, s));
        }
        if (kind.limit > 0) {
            k_fill_i64<<<(unsigned)ceil_div(K, 256), 256, 0, s>>>(c->Lsel, K, kind.limit);
            UPR_LAUNCH_CHECK();
        }
        Penalty pen{c->PW, F, c->C0, kind.limit > 0 ? c->Lsel : c->Lb, c->first_slot};
        set_pack(c, pen);
        // ---- (b2) best move per boundary node
        run_tuned(c, c->sel_tuned, c->sel_cfg, c->sel_cands, &c->sel_pending, c->ev_tune, [&](LaneCfg cfg) {
            select_moves(G, c->part0, c->W, pen, c->cand_tgt, c->cand_s0, c->cand_gain, c->flags, cfg, s);
        });
        if (c->prm.lock_rebalanced)        // the oscillation guard (Sec. 2)
            guard_filter(c->locked, n, c->flags, c->cand_tgt, c->cand_s0, c->cand_gain, s);
        select_flags(c->flags, c->idxA, cnt + CNT_CAND, cN, c->tmp, s);
        const Count cC{cnt + CNT_CAND, n};
        // ---- (b3) inflow penalties: order by (target, s0 desc, id)
        cand_keys(c->idxA, cnt + CNT_CAND, c->cand_tgt, c->cand_s0, c->gbits, c->sb[0].k, c->sb[0].v, n, s);
        c->sb[0].run(cC, c->gbits + kbits, c->tmp, s, &ko, &vo);
        cand_gather(G, c->idxA, vo, cnt + CNT_CAND, c->cand_tgt, c->c_sorted, c->seg_first, n, s);
        exclusive_sum_i64(c->c_sorted, c->c_excl, cC, c->tmp, s);
        inflow_filter(G, c->idxA, vo, cnt + CNT_CAND, c->cand_tgt, c->cand_gain, c->c_excl, c->seg_first, pen,
                      c->flags2, c->score, n, s);
        select_flags(c->flags2, c->idxB, cnt + CNT_M, cC, c->tmp, s);
        // ---- M ordered by (score desc, id), applied
        uint64_t *k2; uint32_t *v2;
        move_keys(c->idxB, cnt + CNT_M, c->score, c->gbits, c->sb[1].k, c->sb[1].v, n, s);
        c->sb[1].run(Count{cnt + CNT_M, n}, c->gbits, c->tmp, s, &k2, &v2);
        apply_moves(G, c->idxA, c->idxB, v2, cnt + CNT_M, c->cand_tgt, c->score, c->part0, c->part, c->C, c->M_node,
                    c->M_from, c->M_to, c->M_score, c->m_pos, c->scal + 1, n, s);
        // W' for P o M: the delta update costs two atomics per adjacency entry of a
        // moved node, a rebuild streams the graph and the table once; each kernel
        // checks on the device which of the two applies
        table_move(G, c->W, c->M_node, c->M_from, c->M_to, cnt + CNT_M, nullptr, c->scal + 1, n, c->hub_chunks,
                   c->n_chunks, HubMoves{c->m_pos, nullptr, nullptr, nullptr, nullptr, c->M_from, c->M_to}, s);
        gain_table(G, c->part, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, c->scal + 1, s);
    }
    if (!cap) UPR_CUDA(cudaEventRecord(c->ev[5], s));

    // ---- (d) rebalancing sub-rounds
    rebalance_phase(c, r, ri, tr);
    if (!cap) UPR_CUDA(cudaEventRecord(c->ev[6], s));

    // ---- (c1) interleave M and R_1..R_k (or append R after M: a variant of Sec. 7.2)
    const int32_t *dM = cnt + CNT_M, *dR = &ctl->nR;
    count_affine(dM, 2, nullptr, 0, cnt + CNT_EVM, s);
    count_affine(dM, 1, dR, 0, cnt + CNT_X, s);
    if (c->prm.append) {
        seq_append(c->M_node, c->M_from, c->M_to, dM, c->R_node, c->R_from, c->R_to, dR, 2 * n, c->X_node, c->X_from,
                   c->X_to, c->X_isr, s);
    } else {
    UPR_CUDA(cudaMemsetAsync(c->rbeg, 0, sizeof(int32_t) * K, s));
    UPR_CUDA(cudaMemsetAsync(c->rend, 0, sizeof(int32_t) * K, s));
    UPR_CUDA(cudaMemsetAsync(c->ebeg, 0, sizeof(int32_t) * K, s));
    UPR_CUDA(cudaMemsetAsync(c->eend, 0, sizeof(int32_t) * K, s));
    uint64_t *kRB; uint32_t *RB;
    seq_rb_keys(c->R_from, dR, n, c->sb[0].k, c->sb[0].v, s);
    c->sb[0].run(Count{dR, n}, kbits, c->tmp, s, &kRB, &RB);
    seq_rb_bounds(c->R_node, c->R_from, RB, dR, n, G.vwgt, c->c_sorted, c->rbeg, c->rend, s);
    exclusive_sum_i64(c->c_sorted, c->c_excl, Count{dR, n}, c->tmp, s);
    uint64_t *kEV; uint32_t *EV;
    const Count cEVM{cnt + CNT_EVM, 2 * n};
    seq_ev_keys(c->M_from, c->M_to, dM, n, c->sb[1].k, c->sb[1].v, s);
    c->sb[1].run(cEVM, kbits, c->tmp, s, &kEV, &EV);
    seq_ev_delta(c->M_node, EV, kEV, dM, n, G.vwgt, c->delta, c->ebeg, c->eend, s);
    exclusive_sum_i64(c->delta, c->d_excl, cEVM, c->tmp, s);
    seq_ev_need(EV, kEV, dM, n, c->delta, c->d_excl, c->ebeg, c->C0, c->Lb, c->rbeg, c->rend, c->c_excl,
                c->c_sorted, c->packed, s);
    inclusive_max_u64(c->packed, c->qmax, cEVM, c->tmp, s);
    seq_ev_emit(EV, kEV, dM, n, c->qmax, c->ebeg, c->emit, c->qbefore, s);
    exclusive_sum_i32(c->emit, c->em_excl, Count{dM, n}, c->tmp, s);
    seq_block_final(K, c->ebeg, c->eend, c->qmax, c->rbeg, c->rend, c->qfin, c->left, s);
    exclusive_sum_i32(c->left, c->left_excl, fixed(K), c->tmp, s);
    seq_place_m(c->M_node, c->M_from, c->M_to, dM, n, c->em_excl, c->pos_m, c->X_node, c->X_from, c->X_to, c->X_isr,
                s);
    seq_place_r(c->R_node, c->R_from, c->R_to, RB, dR, n, c->rbeg, EV, c->ebeg, c->eend, c->qmax, c->pos_m, c->qfin,
                c->left_excl, c->em_excl, c->emit, dM, c->X_node, c->X_from, c->X_to, c->X_isr, s);
    }

    // ---- (c1) merge double moves
    const Count cX{cnt + CNT_X, 2 * n};
    seq_merge_flags(c->X_node, c->X_to, c->X_isr, cnt + CNT_X, 2 * n, c->m_pos, c->r_to, c->part0, c->flags2,
                    c->final_to, s);
    select_flags(c->flags2, c->idxD, cnt + CNT_I, cX, c->tmp, s);
    const int32_t *dI = cnt + CNT_I;
    seq_build_I(c->idxD, dI, n, c->X_node, c->final_to, c->part0, c->I_node, c->I_from, c->I_to, c->pos, c->dest, s);
    // a batch: each graph's moves are a subsequence of I in its own order;
    // a stable sort by graph makes them contiguous (X_* are free by now)
    const int32_t *Iv = c->I_node, *If = c->I_from, *It = c->I_to;
    if (batch) {
        seq_sort_by_graph(G, c->I_node, c->I_from, c->I_to, dI, n, c->sb[0].k, c->sb[0].v, c->sb[0].ka, c->sb[0].va,
                          c->tmp, c->X_node, c->X_from, c->X_to, c->pos, c->dest, c->seg_beg, c->seg_end, s);
        Iv = c->X_node; If = c->X_from; It = c->X_to;
    }

    // ---- (c2) exact gains, balanced prefixes, best prefix
    seq_gains(G, Iv, If, It, dI, n, c->part0, c->pk, c->I_gain, c->hub_chunks, c->n_chunks, c->scal + 3, s);
    inclusive_sum_i64(c->I_gain, c->Gsum, Count{dI, n}, c->tmp, s);
    count_affine(dI, 2, nullptr, 0, cnt + CNT_EVI, s);
    count_affine(dI, 1, nullptr, 1, cnt + CNT_I1, s);
    uint64_t *kE; uint32_t *E;
    const Count cEVI{cnt + CNT_EVI, 2 * n};
    seq_iev_keys(If, It, dI, n, c->sb[2].k, c->sb[2].v, s);
    c->sb[2].run(cEVI, kbits, c->tmp, s, &kE, &E);
    UPR_CUDA(cudaMemsetAsync(c->ebeg, 0, sizeof(int32_t) * K, s));
    seq_iev_delta(Iv, E, kE, dI, n, G.vwgt, c->delta, c->ebeg, s);
    exclusive_sum_i64(c->delta, c->d_excl, cEVI, c->tmp, s);
    clear_count(c->diff, dI, 1, n, s);
    seq_iev_transitions(E, kE, dI, n, c->delta, c->d_excl, c->ebeg, c->C0, c->Lb, c->diff, s);
    exclusive_sum_i32(c->diff, c->diff_excl, Count{cnt + CNT_I1, n + 1}, c->tmp, s);
    if (!cap) UPR_CUDA(cudaMemcpyAsync(c->hcut, c->cut, sizeof(int64_t), cudaMemcpyDeviceToHost, s));   // cut before the round
    if (!batch) {
        count_over(G, c->C0, cnt + CNT_OVER0, s);
        seq_best(c->Gsum, c->diff, c->diff_excl, dI, n, cnt + CNT_OVER0, c->best_parts, c->best, cnt + CNT_INFEAS, s);
    } else {
        count_over(G, c->C0, c->over0_g, s);
        seq_best_seg(G, Iv, dI, n, c->seg_beg, c->Gsum, c->diff, c->diff_excl, c->over0_g, c->best_g, c->best_j, c->cut,
                     c->infeas_g, c->tot, s);
    }
    if (G.sp.on() && !cap) {
        // a sparse row without room for a new block: nothing of the round is
        // applied yet; the caller runs it again on rows built afresh (which
        // drop the blocks whose weight went back to zero) or, if these were
        // fresh already, on the dense table
        UPR_CUDA(cudaMemcpyAsync(c->hcnt + 41, c->sp_over, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaStreamSynchronize(s));
        if (c->hcnt[41] != 0) {
            reset_nodes(c->I_node, dI, n, c->pos, INT32_MAX, s);
            reset_nodes(c->M_node, dM, n, c->m_pos, -1, s);
            reset_nodes(c->R_node, dR, n, c->r_to, -1, s);
            UPR_CUDA(cudaMemsetAsync(c->sp_over, 0, sizeof(int32_t), s));
            UPR_CUDA(cudaStreamSynchronize(s));
            return build ? kRedoDense : kRedoFresh;
        }
    }
    if (!batch) seq_apply_prefix(G, c->I_node, c->I_from, c->I_to, n, c->best, c->part0, c->C0, c->cut, s);
    else seq_apply_prefix_seg(G, Iv, If, It, dI, n, c->seg_beg, c->best_j, c->part0, c->C0, s);
    // the table goes from W(P o I) to W(P o I^{j*}) for the next round
    {
        const Rollback rb{Iv, If, It, dI, c->best, batch ? G.gid : nullptr, c->seg_beg, c->best_j};
        if (c->prm.lock_rebalanced && !rebalance_only) guard_locks(rb, n, n, c->m_pos, c->r_to, c->locked, s);
        table_rollback(G, rb, n, c->pos, c->W, c->hub_chunks, c->n_chunks, c->scal + 2, s);
        gain_table(G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, c->scal + 2, s);
    }
    // reset node-indexed markers for the next round
    reset_nodes(c->I_node, dI, n, c->pos, INT32_MAX, s);
    reset_nodes(c->M_node, dM, n, c->m_pos, -1, s);
    reset_nodes(c->R_node, dR, n, c->r_to, -1, s);
    if (cap) {                  // the step graph: the round's counts go to the device sums
        k_round_stats<<<1, 32, 0, s>>>(cnt, ctl, c->best, c->tot, batch ? 1 : 0, c->tmp.err, c->dstats);
        UPR_LAUNCH_CHECK();
        c->table_valid = true;
        return UPR_OK;
    }
    UPR_CUDA(cudaEventRecord(c->ev[7], s));
    UPR_CUDA(cudaMemcpyAsync(c->hcnt, cnt, sizeof(int32_t) * CNT_SLOTS, cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaMemcpyAsync(c->hctl, ctl, sizeof(RebalCtl), cudaMemcpyDeviceToHost, s));
    if (!batch) UPR_CUDA(cudaMemcpyAsync(c->hbest, c->best, sizeof(long long) * 2, cudaMemcpyDeviceToHost, s));
    else UPR_CUDA(cudaMemcpyAsync(c->hbest, c->tot, sizeof(long long) * 3, cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaMemcpyAsync(c->hcnt + 40, c->tmp.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaStreamSynchronize(s));
    if (c->sel_pending) {
        settle_tuning(&c->sel_cfg, &c->sel_tuned, &c->sel_pending, c->sel_cands, c->ev_tune, 0.05f);
        if (c->sel_tuned) remember_tuning(c, 0, c->sel_cfg);
    }
    // a bounded wait of a primitive gave up: the round's lists are not trustworthy
    if (c->hcnt[40] != 0) { c->table_valid = false; throw CudaError{cudaErrorLaunchTimeout, "primitive wait"}; }
    {
        float a = 0, b = 0, d = 0, t = 0;
        UPR_CUDA(cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
        UPR_CUDA(cudaEventElapsedTime(&a, c->ev[4], c->ev[5]));
        UPR_CUDA(cudaEventElapsedTime(&b, c->ev[5], c->ev[6]));
        UPR_CUDA(cudaEventElapsedTime(&d, c->ev[6], c->ev[7]));
        if (build) { ri.ms_table += t; ri.tables++; }
        ri.ms_select = a; ri.ms_rebalance = b; ri.ms_sequence = d;
    }
    const int32_t *hc = c->hcnt;
    ri.n_cand = rebalance_only ? 0 : hc[CNT_CAND];
    ri.n_moves = hc[CNT_M];
    ri.n_rebal = c->hctl->nR;
    ri.subrounds = c->hctl->subrounds;
    if (ri.graph)
        g_upr_launches += (1 + (long long)c->reb_body_kernels * ri.subrounds +
                           (long long)c->reb_if_kernels * hc[CNT_SORTP]);
    ri.n_inter = hc[CNT_X];
    ri.n_seq = hc[CNT_I];
    // one graph: an infeasible round applies nothing and is an error; a
    // batch records it per graph (infeas_g) and the round goes on
    const bool infeasible = !batch && hc[CNT_INFEAS] != 0;
    c->table_valid = !infeasible;
    ri.best_len = infeasible ? 0 : batch ? c->hbest[0] : c->hbest[1];
    ri.best_gain = infeasible ? 0 : batch ? c->hbest[1] : c->hbest[0];
    if (log_enabled())
        fprintf(stderr, "upr round %d: candidates %lld moves %lld rebalance moves %lld in %d sub-rounds, "
                        "sequence %lld, applied %lld (gain %lld)\n",
                r, (long long)ri.n_cand, (long long)ri.n_moves, (long long)ri.n_rebal, ri.subrounds,
                (long long)ri.n_seq, (long long)ri.best_len, (long long)ri.best_gain);
    if (T) {
        const int64_t nM = ri.n_moves, nR = ri.n_rebal, nX = ri.n_inter, nI = ri.n_seq;
        T->n_cand = ri.n_cand; T->n_moves = nM; T->n_rebal = nR; T->subrounds = ri.subrounds; T->n_inter = nX;
        T->n_seq = nI;
        if (!rebalance_only) {
            d2h(T->avail, tr->avail_d, n, s);
            d2h(T->slot, tr->slot_d, sizeof(int32_t) * n, s);
            d2h(T->bucket, c->BW, sizeof(int64_t) * K * kSlots, s);
            if (T->factor) memcpy(T->factor, c->hF, sizeof(int64_t) * kSlots);
            d2h(T->cand_target, c->cand_tgt, sizeof(int32_t) * n, s);
            d2h(T->cand_s0, c->cand_s0, sizeof(int64_t) * n, s);
        }
        std::vector<int32_t> tmp(rebalance_only ? 0 : n);
        if (T->cand_gain && !rebalance_only)
            UPR_CUDA(cudaMemcpyAsync(tmp.data(), c->cand_gain, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        d2h(T->M_node, c->M_node, sizeof(int32_t) * nM, s);
        d2h(T->M_to, c->M_to, sizeof(int32_t) * nM, s);
        d2h(T->M_score, c->M_score, sizeof(int64_t) * nM, s);
        d2h(T->R_node, c->R_node, sizeof(int32_t) * nR, s);
        d2h(T->R_from, c->R_from, sizeof(int32_t) * nR, s);
        d2h(T->R_to, c->R_to, sizeof(int32_t) * nR, s);
        d2h(T->R_subround, c->R_sub, sizeof(int32_t) * nR, s);
        d2h(T->X_node, c->X_node, sizeof(int32_t) * nX, s);
        d2h(T->X_from, c->X_from, sizeof(int32_t) * nX, s);
        d2h(T->X_to, c->X_to, sizeof(int32_t) * nX, s);
        d2h(T->I_node, c->I_node, sizeof(int32_t) * nI, s);
        d2h(T->I_from, c->I_from, sizeof(int32_t) * nI, s);
        d2h(T->I_to, c->I_to, sizeof(int32_t) * nI, s);
        d2h(T->I_gain, c->I_gain, sizeof(int64_t) * nI, s);
        std::vector<int32_t> df(nI + 1), de(nI + 1);
        UPR_CUDA(cudaMemcpyAsync(df.data(), c->diff, sizeof(int32_t) * (nI + 1), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaMemcpyAsync(de.data(), c->diff_excl, sizeof(int32_t) * (nI + 1), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaStreamSynchronize(s));
        if (T->cand_gain && !rebalance_only)
            for (int64_t v = 0; v < n; v++) T->cand_gain[v] = tmp[v];
        if (T->I_eligible)
            for (int64_t j = 0; j <= nI; j++) T->I_eligible[j] = (hc[CNT_OVER0] + de[j] + df[j]) == 0;
        T->cut_before = *c->hcut;
        T->best_len = infeasible ? 0 : c->hbest[1];
        T->best_gain = infeasible ? 0 : c->hbest[0];
        T->cut_after = *c->hcut - T->best_gain;
    }
    return infeasible ? UPR_ERR_INFEASIBLE : UPR_OK;
}

// The dense table of a context bound with sparse rows (allocated on first use).
void ensure_dense(upr_ctx *c) {
    if (c->W) return;
    const size_t bytes = sizeof(int32_t) * (size_t)std::max<int64_t>(c->n, 1) * (size_t)c->k;
    if (c->W_own_bytes < bytes) {
        if (c->W_own) cudaFree(c->W_own);
        c->W_own = nullptr;
        c->W_own_bytes = 0;
        if (cudaMalloc(&c->W_own, bytes) != cudaSuccess) {
            cudaGetLastError();
            throw CudaError{cudaErrorMemoryAllocation, "dense gain table"};
        }
        c->W_own_bytes = bytes;
    }
    c->W = c->W_own;
}

// A round; when a sparse row overflows, the round runs again from the same
// state on rows built afresh, and when fresh rows overflow, on the dense table.
upr_status run_round(upr_ctx *c, int32_t r, int32_t R, bool rebalance_only, RoundInfo &ri, TraceSink *tr,
                     const RoundKind &kind = RoundKind()) {
    for (;;) {
        ri = RoundInfo{};
        const upr_status rc = run_round_once(c, r, R, rebalance_only, ri, tr, kind);
        if (rc == kRedoFresh) {
            c->table_valid = false;
            continue;
        }
        if (rc != kRedoDense) return rc;
        ensure_dense(c);
        c->sparse_on = false;
        c->G.sp.slot = nullptr;
        c->table_valid = false;
        c->gen++;
    }
}

void free_ctx(upr_ctx *c) {
    if (!c) return;
    if (c->mix) mixed_destroy(c->mix);
    if (c->mem) cudaFree(c->mem);
    if (c->W_own) cudaFree(c->W_own);
    if (c->reb_exec) cudaGraphExecDestroy(c->reb_exec);
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    if (c->s_cap) cudaStreamDestroy(c->s_cap);
    if (c->s_body) cudaStreamDestroy(c->s_body);
    if (c->s_if) cudaStreamDestroy(c->s_if);
    if (c->xs) cudaFree(c->xs);
    if (c->segs_d) cudaFree(c->segs_d);
    if (c->s_up) cudaStreamDestroy(c->s_up);
    if (c->ev_up) cudaEventDestroy(c->ev_up);
    if (c->ev_prev) cudaEventDestroy(c->ev_prev);
    if (c->F_all) cudaFree(c->F_all);
    if (c->hF_all) cudaFreeHost(c->hF_all);
    if (c->h) cudaFreeHost(c->h);
    if (c->h8) cudaFreeHost(c->h8);
    if (c->hx) cudaFreeHost(c->hx);
    for (auto &e : c->ev) if (e) cudaEventDestroy(e);
    for (auto &e : c->ev_tune) if (e) cudaEventDestroy(e);
    delete c;
}

// part in [0, k)?
__global__ void k_check_part(const int32_t *part, int64_t n, int32_t k, int32_t *bad) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && (part[v] < 0 || part[v] >= k)) atomicOr(bad, 1);
}

// batches: graph-local block ids -> global ids (and a copy of the input)
__global__ void k_part_to_global(int32_t *part, const int32_t *gid, int64_t n, int32_t k, int32_t *copy) {
    UPR_FOR(v, n) {
        const int32_t p = part[v] + gid[v] * k;
        part[v] = p;
        copy[v] = p;
    }
}

// batches: global -> graph-local ids; graphs flagged in keep_input get their input back
__global__ void k_part_to_local(const int32_t *part, const int32_t *part_in, const int32_t *gid,
                                const int32_t *keep_input, int64_t n, int32_t k, int32_t *out) {
    UPR_FOR(v, n) {
        const int32_t g = gid[v];
        out[v] = (keep_input[g] ? part_in[v] : part[v]) - g * k;
    }
}

// need_cut = false: the cut is left to the first round's bucket pass (one
// graph, a refinement round follows).
upr_status load_part(upr_ctx *c, const int32_t *part, bool need_cut = true) {
    c->table_valid = false;
    copy_in(c->part0, part, sizeof(int32_t) * c->n, c->s);
    UPR_CUDA(cudaMemsetAsync(c->counts + 7, 0, sizeof(int32_t), c->s));
    if (c->n > 0) {
        k_check_part<<<(unsigned)ceil_div(c->n, 256), 256, 0, c->s>>>(c->part0, c->n, c->k, c->counts + 7);
        UPR_LAUNCH_CHECK();
    }
    if (read_count(c, 7)) return UPR_ERR_INVALID;
    if (c->ng > 1 && c->n > 0) {
        k_part_to_global<<<grid_for(c->n), 256, 0, c->s>>>(c->part0, c->gid, c->n, c->k, c->part_in);
        UPR_LAUNCH_CHECK();
    }
    block_weights(c->G, c->part0, c->C0, c->s);
    c->cut_pending = !need_cut;
    if (need_cut) edge_cut(c->G, c->part0, c->cut, c->s);
    return UPR_OK;
}

// Writes the partition (graph-local ids) to `part`; in a batch, graphs with
// keep_input[g] != 0 (host array) get their input partition back.
void store_part(upr_ctx *c, int32_t *part, const std::vector<int32_t> &keep_input) {
    if (c->ng == 1) {
        copy_out(part, c->part0, sizeof(int32_t) * c->n, c->s);
        return;
    }
    UPR_CUDA(cudaMemcpyAsync(c->inf0_g, keep_input.data(), sizeof(int32_t) * c->ng, cudaMemcpyHostToDevice, c->s));
    if (c->n > 0) {
        k_part_to_local<<<grid_for(c->n), 256, 0, c->s>>>(c->part0, c->part_in, c->gid, c->inf0_g, c->n, c->k, c->part);
        UPR_LAUNCH_CHECK();
    }
    copy_out(part, c->part, sizeof(int32_t) * c->n, c->s);
    UPR_CUDA(cudaStreamSynchronize(c->s));      // keep_input is host memory
}

void add_round(upr_stats &st, const RoundInfo &ri, bool repair) {
    st.ms_gain_table += ri.ms_table; st.gain_table_builds += ri.tables;
    st.n_rebalance_moves += ri.n_rebal; st.subrounds += ri.subrounds; st.n_sequence += ri.n_seq;
    st.rebalance_graphs += ri.graph ? 1 : 0;
    st.constrained_rounds += ri.constrained ? 1 : 0;
    st.n_applied += ri.best_len;
    if (repair) return;
    st.rounds_run++;
    st.n_candidates += ri.n_cand; st.n_moves += ri.n_moves;
    st.ms_select += ri.ms_select; st.ms_rebalance += ri.ms_rebalance; st.ms_sequence += ri.ms_sequence;
}

/*
 * upr_refine and upr_batch_refine.  One graph: an infeasible input is an
 * error (part unchanged).  A batch: per-graph status; an infeasible graph
 * keeps its input partition and cut, the others go on.  cut_in / cut_out /
 * status (nullable) have ng entries.
 */
// One round of unconstrained label propagation (Sec. 5) on one graph, from
// part0 (round start) with V_a = c->lp_active: every active node to its best
// positive-gain block (the selection with no penalty and no limit), all moves
// at once, then the rebalancing; the result is kept only if it is balanced and
// cuts less than *cut (then part0, C0, the cut and the table follow it and
// c->lp_active becomes the next V_a), else everything stays as it was.
// Returns whether the round was kept; *active_next = |next V_a|.
constexpr int kLpRedo = 2;     // internal: a hashed row ran out of slots, nothing was kept

int lp_round_once(upr_ctx *c, int64_t *cut, int64_t *active_next, RoundInfo &ri) {
    cudaStream_t s = c->s;
    const GraphDev &G = c->G;
    const int64_t n = c->n;
    const int32_t K = G.K();
    int32_t *cnt = c->counts;
    RebalCtl *ctl = c->ctl;
    const Count cN{nullptr, n};
    UPR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * CNT_SLOTS, s));
    UPR_CUDA(cudaMemcpyAsync(c->part, c->part0, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    UPR_CUDA(cudaMemcpyAsync(c->C, c->C0, sizeof(int64_t) * K, cudaMemcpyDeviceToDevice, s));
    const bool build = !c->table_valid;
    UPR_CUDA(cudaEventRecord(c->ev[0], s));
    if (build)
        gain_table(G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, nullptr, s);
    UPR_CUDA(cudaEventRecord(c->ev[1], s));
    c->table_valid = false;
    // selection without a penalty: no block limit, so no move pays anything
    for (int l = 0; l < kSlots; l++) c->hF[l] = kConstrainedF;
    UPR_CUDA(cudaMemcpyAsync(c->F, c->hF, sizeof(int64_t) * kSlots, cudaMemcpyHostToDevice, s));
    k_fill_i64<<<(unsigned)ceil_div(K, 256), 256, 0, s>>>(c->Lsel, K, INT64_MAX);
    UPR_LAUNCH_CHECK();
    Penalty pen{c->PW, c->F, c->C0, c->Lsel, c->first_slot};
    set_pack(c, pen);
    select_moves(G, c->part0, c->W, pen, c->cand_tgt, c->cand_s0, c->cand_gain, c->flags, c->sel_cfg, s);
    lp_filter(c->flags, c->lp_active, n, s);
    select_flags(c->flags, c->idxA, cnt + CNT_M, cN, c->tmp, s);
    lp_apply(G, c->idxA, cnt + CNT_M, c->cand_tgt, c->cand_gain, c->part0, c->part, c->C, c->M_node, c->M_from,
             c->M_to, c->M_score, c->m_pos, c->scal + 1, n, s);
    table_move(G, c->W, c->M_node, c->M_from, c->M_to, cnt + CNT_M, nullptr, c->scal + 1, n, c->hub_chunks,
               c->n_chunks, HubMoves{c->m_pos, nullptr, nullptr, nullptr, nullptr, c->M_from, c->M_to}, s);
    gain_table(G, c->part, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
               c->tile_nodes, c->scal + 1, s);
    UPR_CUDA(cudaEventRecord(c->ev[5], s));
    rebalance_phase(c, 0, ri, nullptr);
    // balanced, and the cut after: the table follows every move and
    // rebalancing move, so the cut comes from it in a pass over the nodes
    count_over(G, c->C, cnt + CNT_OVER0, s);
    cut_from_table(G, c->part, c->W, c->tot, s);
    int64_t cut1 = 0;
    UPR_CUDA(cudaMemcpyAsync(c->hcnt, cnt, sizeof(int32_t) * CNT_SLOTS, cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaMemcpyAsync(c->hcut, c->tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaMemcpyAsync(c->hctl, ctl, sizeof(RebalCtl), cudaMemcpyDeviceToHost, s));
    if (G.sp.on()) UPR_CUDA(cudaMemcpyAsync(c->hcnt + 41, c->sp_over, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaStreamSynchronize(s));
    cut1 = *c->hcut;
    if (build) {
        float t = 0;
        UPR_CUDA(cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
        ri.ms_table += t;
        ri.tables++;
    }
    ri.n_moves = c->hcnt[CNT_M];
    ri.n_rebal = c->hctl->nR;
    ri.subrounds = c->hctl->subrounds;
    const int32_t *dM = cnt + CNT_M, *dR = &ctl->nR;
    if (G.sp.on() && c->hcnt[41] != 0) {
        // a hashed row ran out of slots: the proposals may have read a wrong
        // row, so nothing of the round is kept; the caller runs it again
        reset_nodes(c->M_node, dM, n, c->m_pos, -1, s);
        reset_nodes(c->R_node, dR, n, c->r_to, -1, s);
        UPR_CUDA(cudaMemsetAsync(c->sp_over, 0, sizeof(int32_t), s));
        UPR_CUDA(cudaStreamSynchronize(s));
        return kLpRedo;
    }
    const bool kept = c->hcnt[CNT_OVER0] == 0 && cut1 < *cut;
    if (kept) {
        lp_next(G, c->part0, c->part, c->M_node, dM, c->R_node, dR, c->hub_chunks, c->n_chunks, c->lp_next,
                cnt + CNT_L1, s);
        std::swap(c->lp_active, c->lp_next);
        UPR_CUDA(cudaMemcpyAsync(c->part0, c->part, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        UPR_CUDA(cudaMemcpyAsync(c->C0, c->C, sizeof(int64_t) * K, cudaMemcpyDeviceToDevice, s));
        UPR_CUDA(cudaMemcpyAsync(c->cut, c->tot, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        c->table_valid = true;              // W follows every move and rebalancing move
        ri.best_gain = *cut - cut1;
        *cut = cut1;
    }
    reset_nodes(c->M_node, dM, n, c->m_pos, -1, s);
    reset_nodes(c->R_node, dR, n, c->r_to, -1, s);
    UPR_CUDA(cudaMemcpyAsync(c->hcnt + 40, c->tmp.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaMemcpyAsync(c->hcnt + CNT_L1, cnt + CNT_L1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaStreamSynchronize(s));
    if (c->hcnt[40] != 0) { c->table_valid = false; throw CudaError{cudaErrorLaunchTimeout, "primitive wait"}; }
    *active_next = kept ? c->hcnt[CNT_L1] : 0;
    return kept ? 1 : 0;
}

// A label propagation round; when hashed rows run out of slots, the round
// runs again on rows built afresh, and then on the dense table.
bool lp_round(upr_ctx *c, int64_t *cut, int64_t *active_next, RoundInfo &ri) {
    for (int attempt = 0;; attempt++) {
        ri = RoundInfo{};
        const int rc = lp_round_once(c, cut, active_next, ri);
        if (rc != kLpRedo) return rc == 1;
        c->table_valid = false;
        if (attempt >= 1) {
            ensure_dense(c);
            c->sparse_on = false;
            c->G.sp.slot = nullptr;
            c->gen++;
        }
    }
}

// Label propagation before the FM rounds (Sec. 5): V_a starts as the boundary
// nodes; stops after max_rounds rounds, at a round that is not kept, at an
// empty V_a, or after a kept round improving the cut by less than 0.001 of
// it.  Returns the rounds kept.
int32_t label_propagation(upr_ctx *c, int32_t max_rounds, int64_t *cut, upr_stats &st) {
    cudaStream_t s = c->s;
    if (!c->table_valid) {
        UPR_CUDA(cudaEventRecord(c->ev[0], s));
        gain_table(c->G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, nullptr, s);
        UPR_CUDA(cudaEventRecord(c->ev[1], s));
        UPR_CUDA(cudaEventSynchronize(c->ev[1]));
        float t = 0;
        UPR_CUDA(cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
        st.ms_gain_table += t;
        st.gain_table_builds++;
        st.lp_table_builds++;
    }
    c->table_valid = true;
    lp_boundary(c->G, c->part0, c->W, c->lp_active, s);
    lp_count(c->lp_active, c->n, c->counts + CNT_L1, s);
    UPR_CUDA(cudaMemcpyAsync(c->hcnt + CNT_L1, c->counts + CNT_L1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaStreamSynchronize(s));
    int64_t active = c->hcnt[CNT_L1];
    int32_t kept = 0;
    for (int32_t r = 1; r <= max_rounds && active > 0; r++) {
        const int64_t before = *cut;
        RoundInfo ri;
        const bool keep = lp_round(c, cut, &active, ri);
        st.ms_gain_table += ri.ms_table;
        st.gain_table_builds += ri.tables;
        st.lp_table_builds += ri.tables;
        c->lp_attempts++;
        if (!keep) break;
        kept++;
        st.n_moves += ri.n_moves;
        st.n_rebalance_moves += ri.n_rebal;
        st.subrounds += ri.subrounds;
        if (1000 * (before - *cut) < before) break;
    }
    return kept;
}

// The step graph of `rounds` rounds (round_offset+1 .. of total): every
// round of run_round_once captured on s_cap with the rebalancing loops as
// while nodes.  False if it cannot be built (the host-driven rounds run).
bool build_step_graph(upr_ctx *c, int32_t rounds, int32_t total) {
    if (c->step_exec) { cudaGraphExecDestroy(c->step_exec); c->step_exec = nullptr; }
    cudaStream_t saved = c->s;
    cudaGraph_t g = nullptr;
    bool capturing = false;
    const long long l0 = g_upr_launches;
    try {
        if (!c->s_cap) UPR_CUDA(cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking));
        UPR_CUDA(cudaStreamBeginCapture(c->s_cap, cudaStreamCaptureModeRelaxed));
        capturing = true;
        c->s = c->s_cap;
        c->capturing = true;
        c->step_cut = c->cut_pending;
        for (int32_t i = 1; i <= rounds; i++) {
            c->cap_round = i - 1;
            RoundInfo ri;
            run_round_once(c, c->prm.round_offset + i, total, false, ri, nullptr, RoundKind());
        }
        c->capturing = false;
        c->s = saved;
        capturing = false;
        UPR_CUDA(cudaStreamEndCapture(c->s_cap, &g));
        UPR_CUDA(cudaGraphInstantiate(&c->step_exec, g, 0));
        cudaGraphDestroy(g);
    } catch (const CudaError &e) {
        c->capturing = false;
        c->s = saved;
        if (capturing) {
            cudaGraph_t out = nullptr;
            cudaStreamEndCapture(c->s_cap, &out);
            if (out) cudaGraphDestroy(out);
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (log_enabled()) fprintf(stderr, "upr: step graph not built (%s: %s)\n", e.what, cudaGetErrorString(e.e));
        c->step_exec = nullptr;
        c->step_failed = true;
    }
    const long long captured = g_upr_launches - l0;
    g_upr_launches -= (captured);     // captured, not launched: counted when the graph runs
    c->step_kernels = captured - (long long)rounds * c->reb_body_kernels;
    c->step_gen = c->gen;
    c->step_rounds = rounds;
    c->step_off = c->prm.round_offset;
    c->step_total = total;
    c->step_lock = c->prm.lock_rebalanced;
    c->step_sel = c->sel_cfg;
    c->step_prop = c->prop_cfg;
    return c->step_exec != nullptr;
}

// Rounds 1..rounds of a call as one graph launch (params.graphs == 2, the
// plain tau schedule, dense table, lane schedules settled): round 1's table
// build runs (timed) before the graph, the rounds' penalty factors are copied
// in one piece, and the rounds' counts are read once at the end.  False: not
// applicable (nothing enqueued but the build); the caller runs the rounds.
bool run_step_graph(upr_ctx *c, int32_t rounds, int32_t total, upr_stats &st) {
    cudaStream_t s = c->s;
    if (c->step_failed) return false;
    const bool same = c->step_exec && c->step_gen == c->gen && c->step_rounds == rounds &&
                      c->step_off == c->prm.round_offset && c->step_total == total &&
                      c->step_lock == c->prm.lock_rebalanced && c->step_cut == c->cut_pending &&
                      c->step_sel.G == c->sel_cfg.G &&
                      c->step_sel.CH == c->sel_cfg.CH && c->step_prop.G == c->prop_cfg.G &&
                      c->step_prop.CH == c->prop_cfg.CH;
    if (!c->table_valid) {
        UPR_CUDA(cudaEventRecord(c->ev[0], s));
        gain_table(c->G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, nullptr, s);
        UPR_CUDA(cudaEventRecord(c->ev[1], s));
        UPR_CUDA(cudaEventSynchronize(c->ev[1]));
        float t = 0;
        UPR_CUDA(cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
        st.ms_gain_table += t;
        st.gain_table_builds++;
        c->table_valid = true;
    }
    if (c->F_all_cap < rounds) {
        if (c->F_all) cudaFree(c->F_all);
        if (c->hF_all) cudaFreeHost(c->hF_all);
        c->F_all = nullptr;
        c->hF_all = nullptr;
        c->F_all_cap = 0;
        UPR_CUDA(cudaMalloc(&c->F_all, sizeof(int64_t) * kSlots * (size_t)rounds));
        UPR_CUDA(cudaMallocHost(&c->hF_all, sizeof(int64_t) * kSlots * (size_t)rounds));
        c->F_all_cap = rounds;
    }
    UPR_CUDA(cudaStreamSynchronize(s));          // hF_all may still be read by the previous call's copy
    for (int32_t i = 1; i <= rounds; i++)
        penalty_factors(c->prm.round_offset + i, total, c->prm.tau1_num, c->prm.tau1_den,
                        c->hF_all + (size_t)(i - 1) * kSlots);
    if (!same && !build_step_graph(c, rounds, total)) return false;
    UPR_CUDA(cudaMemcpyAsync(c->F_all, c->hF_all, sizeof(int64_t) * kSlots * rounds, cudaMemcpyHostToDevice, s));
    UPR_CUDA(cudaMemsetAsync(c->dstats, 0, sizeof(long long) * 16, s));
    UPR_CUDA(cudaGraphLaunch(c->step_exec, s));
    long long d[16];
    UPR_CUDA(cudaMemcpyAsync(d, c->dstats, sizeof(d), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaStreamSynchronize(s));
    if (d[6] != 0) { c->table_valid = false; throw CudaError{cudaErrorLaunchTimeout, "primitive wait"}; }
    if (d[7] != 0) { c->table_valid = false; throw CudaError{cudaErrorInvalidValue, "step graph: infeasible round"}; }
    st.rounds_run += rounds;
    st.n_candidates += d[0];
    st.n_moves += d[1];
    st.n_rebalance_moves += d[2];
    st.subrounds += (int32_t)d[3];
    st.n_sequence += d[4];
    st.n_applied += d[5];
    st.rebalance_graphs += rounds;
    g_upr_launches += (c->step_kernels + (long long)c->reb_body_kernels * d[3] + (long long)c->reb_if_kernels * d[9]);
    return true;
}

upr_status refine_impl(upr_ctx *c, int32_t *part, int32_t rounds, upr_stats *stats, upr_status *status,
                       int64_t *cut_in, int64_t *cut_out) {
    const int32_t total = c->prm.total_rounds > 0 ? c->prm.total_rounds : c->prm.round_offset + rounds;
    if (c->prm.round_offset + rounds > total) return UPR_ERR_INVALID;
    const int32_t ng = c->ng, K = c->G.K();
    // the round driver of Sec. 6.2 decides round by round from one graph's
    // cut, over a whole schedule in one call
    const int sch = c->prm.schedule;
    if (sch != 0 && (ng != 1 || c->prm.round_offset != 0 || c->prm.total_rounds != 0)) return UPR_ERR_INVALID;
    if (c->prm.lp_rounds > 0 && ng != 1) return UPR_ERR_INVALID;     // label propagation: one graph
    upr_stats st{};
    const auto t_host0 = std::chrono::steady_clock::now();
    const long long launches0 = g_upr_launches;
    c->lp_attempts = 0;
    UPR_CUDA(cudaEventRecord(c->ev[2], c->s));
    UPR_CUDA(cudaMemsetAsync(c->scal + 3, 0, sizeof(int64_t), c->s));     // degrees of the sequences' nodes
    // one graph with a balanced input: the first round's bucket pass, which
    // reads omega(v, V_P(v)) and omega(I(v)) of every node anyway, gives the
    // cut, instead of a pass over the edges
    bool defer_cut = ng == 1 && rounds >= 1 && sch == 0 && c->prm.lp_rounds == 0;
    // label propagation on the dense table: its first build gives the cut
    const bool lp_cut = ng == 1 && c->prm.lp_rounds > 0 && !c->G.sp.on();
    upr_status rc = load_part(c, part, !defer_cut && !lp_cut);
    if (rc != UPR_OK) return rc;
    std::vector<int64_t> cin(ng), cout(ng), C0h(K);
    read_i64(c, c->C0, K, C0h.data());
    bool bal_in = true;
    for (int32_t b = 0; b < K; b++) bal_in = bal_in && C0h[b] <= c->Lmax_g[b / c->k];
    if (defer_cut && !bal_in) {     // the repair round comes first and has no bucket pass
        edge_cut(c->G, c->part0, c->cut, c->s);
        c->cut_pending = false;
        defer_cut = false;
    }
    if (lp_cut) {
        if (bal_in) {
            UPR_CUDA(cudaEventRecord(c->ev[0], c->s));
            gain_table(c->G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                       c->tile_nodes, nullptr, c->s);
            UPR_CUDA(cudaEventRecord(c->ev[1], c->s));
            cut_from_table(c->G, c->part0, c->W, c->cut, c->s);
            UPR_CUDA(cudaEventSynchronize(c->ev[1]));
            float t = 0;
            UPR_CUDA(cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
            st.ms_gain_table += t;
            st.gain_table_builds++;
            st.lp_table_builds++;
            c->table_valid = true;
        } else {                    // the repair round comes first
            edge_cut(c->G, c->part0, c->cut, c->s);
        }
        c->cut_pending = false;
    }
    if (!defer_cut) read_i64(c, c->cut, ng, cin.data());
    st.cut_in = 0;
    for (int64_t x : cin) st.cut_in += x;
    const bool balanced = bal_in;
    std::vector<int32_t> keep(ng, 0);
    int64_t repair_gain = 0;
    if (!balanced) {
        RoundInfo ri;
        rc = run_round(c, 0, total, true, ri, nullptr);
        add_round(st, ri, true);
        if (rc != UPR_OK) return rc;
        if (ng > 1) read_i32(c, c->infeas_g, ng, keep.data());
        st.repaired_input = 1;
        repair_gain = ri.best_gain;
    }
    if (c->prm.lock_rebalanced && c->n > 0) UPR_CUDA(cudaMemsetAsync(c->locked, 0, (size_t)c->n, c->s));
    // unconstrained label propagation before the FM rounds (Sec. 5)
    if (c->prm.lp_rounds > 0) {
        int64_t cut_lp = st.cut_in - repair_gain;
        st.lp_rounds = label_propagation(c, c->prm.lp_rounds, &cut_lp, st);
        repair_gain = st.cut_in - cut_lp;       // the rounds below start from this cut
    }
    // The frame of the paper's final configuration (Sec. 4.4, with Sec. 7.2's
    // split of ten rounds into eight unconstrained and two constrained): the
    // first U rounds unconstrained (U = R - 2 for R >= 3, 1 for R = 2, 0 for
    // R = 1), the others constrained, and once an unconstrained round improves
    // the cut by less than 0.002 of the cut before it, every later round is
    // constrained.  Schedule 6 runs its unconstrained rounds with tau_i of a
    // schedule over the U rounds; the variants of Sec. 7.2 (3-5) run theirs
    // in the same frame.  Schedule 1 is dynamic activation (Sec. 4.4, left out
    // of the final configuration in Sec. 7.2): round 1 constrained, round 2
    // unconstrained with tau = 1/2; rounds 3..R-1 unconstrained (tau_i of a
    // schedule over those R-3 rounds) if round 2 improved the cut more than
    // round 1, until one of them improves it by less than 0.002 of the cut
    // before it, constrained otherwise; round R constrained.  Schedule 2:
    // every round constrained.
    const int32_t U = rounds >= 3 ? rounds - 2 : rounds == 2 ? 1 : 0;
    bool unconstrained_rest = false, switched = false;
    int64_t imp1 = 0, cut_now = st.cut_in - repair_gain;
    // params.graphs == 2: from a binding's second call on, the plain schedule's
    // rounds run as one graph launch
    c->calls_bound++;
    // with graphs = 2, a lane schedule still open after two calls had too
    // little work to time (e.g. no rebalancing sub-round ran): it keeps the
    // default, so that the call can run as one graph (other contexts, the
    // server's slots among them, go on timing: settling early there
    // lengthened the served mix's tail latency, p99 87 -> 240-350 ms)
    if (c->prm.graphs == 2 && c->calls_bound >= 3) {
        c->sel_tuned = true;
        c->prop_tuned = true;
    }
    LaneCfg lc[3];
    const bool no_choice = lane_candidates(c->k, lc) <= 1;      // nothing to time: the schedule is fixed
    const bool settled = no_choice || !worth_tuning(c) || (c->sel_tuned && c->prop_tuned);
    const bool step = c->prm.graphs == 2 && sch == 0 && !c->G.sp.on() && rounds >= 1 && !log_enabled() && settled &&
                      c->calls_bound >= 2;
    const int32_t first_round = step && run_step_graph(c, rounds, total, st) ? rounds + 1 : 1;
    for (int32_t i = first_round; i <= rounds; i++) {
        RoundInfo ri;
        RoundKind kind;
        int32_t r = c->prm.round_offset + i, R = total;
        if (sch == 2 || (sch >= 3 && (i > U || switched))) {
            kind.constrained = true;
        } else if (sch == 3) {                       // constant penalty, tau = tau_1
            kind.tau_num = c->prm.tau1_num;
            kind.tau_den = c->prm.tau1_den;
        } else if (sch == 4) {                       // fully unconstrained
            kind.limit = INT64_MAX;
        } else if (sch == 5) {                       // limited imbalance, alpha 2 -> 1.1 over rounds 1..U
            const int64_t D = U > 1 ? U - 1 : 1;
            kind.limit = (int64_t)(((i128)c->Lmax * (20 * D - 9 * (int64_t)(i - 1))) / (10 * D));
        } else if (sch == 6) {                       // tau_i of the U unconstrained rounds
            r = i;
            R = U;
        } else if (sch == 1) {
            if (i == 1 || (rounds >= 3 && i == rounds) || (i >= 3 && (!unconstrained_rest || switched))) {
                kind.constrained = true;
            } else if (i == 2) {
                kind.tau_num = 1;
                kind.tau_den = 2;
            } else {
                r = i - 2;
                R = rounds - 3;
            }
        }
        rc = run_round(c, r, R, false, ri, nullptr, kind);
        if (rc != UPR_OK) return rc;
        ri.constrained = kind.constrained;
        add_round(st, ri, false);
        const int64_t imp = ri.best_gain, before = cut_now;
        cut_now -= imp;
        if (sch == 1) {
            if (i == 1) imp1 = imp;
            if (i == 2) unconstrained_rest = imp > imp1;
            if (i >= 3 && !kind.constrained && 500 * imp < before) switched = true;
        }
        if (sch >= 3 && !kind.constrained && 500 * imp < before) switched = true;
    }
    store_part(c, part, keep);
    read_i64(c, c->cut, ng, cout.data());
    if (defer_cut) {
        read_i64(c, c->cut_parts + kCutParts, 1, cin.data());
        cin[0] /= 2;
        st.cut_in = cin[0];
    }
    st.cut_out = 0;
    for (int32_t g = 0; g < ng; g++) {
        if (keep[g]) cout[g] = cin[g];
        st.cut_out += cout[g];
        if (status) status[g] = keep[g] ? UPR_ERR_INFEASIBLE : UPR_OK;
        if (cut_in) cut_in[g] = cin[g];
        if (cut_out) cut_out[g] = cout[g];
    }
    UPR_CUDA(cudaEventRecord(c->ev[3], c->s));
    UPR_CUDA(cudaEventSynchronize(c->ev[3]));
    float ms = 0;
    UPR_CUDA(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
    st.ms_device = ms;
    st.kernel_launches = (int32_t)(g_upr_launches - launches0);
    st.ms_host = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
    // the rows written by a build: the dense table, or every slot of the hashed rows
    const int64_t table_bytes = c->G.sp.on() ? 8 * c->sp_slots : 4 * c->n * (int64_t)c->k;
    st.gain_table_bytes = 8 * (c->n + 1) + 4 * c->m + (c->G.adjw ? 4 * c->m : 0) + 4 * c->n + table_bytes;
    read_i64(c, c->scal + 3, 1, &st.seq_degree_sum);
    // the rounds' algorithmic bytes (FM rounds and label propagation rounds):
    // each build, per round a read of the table and 16 bytes per node (part,
    // c, omega(I)), the exact gains and delta updates over the adjacency of
    // the sequence's nodes, and one read and one write of 24-byte records per
    // candidate, move and rebalancing move
    st.bytes_algorithmic = (int64_t)st.gain_table_builds * st.gain_table_bytes +
                           (int64_t)(st.rounds_run + c->lp_attempts) * (table_bytes + 16 * c->n) +
                           16 * st.seq_degree_sum + 48 * (st.n_candidates + st.n_moves + st.n_rebalance_moves);
    st.batch_graphs = ng;
    {
        LaneCfg d[3];
        const int nd = lane_candidates(c->k, d);
        st.select_lanes = nd ? (c->sel_cfg.G > 0 ? c->sel_cfg.G : d[0].G) : 0;
        st.propose_lanes = nd ? (c->prop_cfg.G > 0 ? c->prop_cfg.G : d[0].G) : 0;
        st.sparse_table = c->G.sp.on() ? 1 : 0;
        if (c->G.sp.on()) st.select_lanes = st.propose_lanes = 8;
    }
    if (stats) *stats = st;
    return UPR_OK;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

void upr_params_default(upr_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->t_num = 7; p->t_den = 10;
    p->tau1_num = 1; p->tau1_den = 4;
    p->max_subrounds = 64;
    p->validate = 1;
    p->round_offset = 0;
    p->total_rounds = 0;
    p->autotune = 1;
    p->table = 0;
    p->graphs = 1;
    p->schedule = 0;
    p->gain_priority = 0;
    p->append = 0;
    p->lp_rounds = 0;
    p->lock_rebalanced = 0;
    p->stream = nullptr;
}

const char *upr_status_str(upr_status s) {
    switch (s) {
        case UPR_OK: return "UPR_OK";
        case UPR_PENDING: return "UPR_PENDING";
        case UPR_ERR_INVALID: return "UPR_ERR_INVALID";
        case UPR_ERR_OOM: return "UPR_ERR_OOM";
        case UPR_ERR_CUDA: return "UPR_ERR_CUDA";
        case UPR_ERR_INFEASIBLE: return "UPR_ERR_INFEASIBLE";
        case UPR_ERR_BUSY: return "UPR_ERR_BUSY";
        case UPR_ERR_TIMEOUT: return "UPR_ERR_TIMEOUT";
        case UPR_ERR_NOT_FOUND: return "UPR_ERR_NOT_FOUND";
        default: return "UPR_UNKNOWN";
    }
}

static bool params_ok(const upr_params &p) {
    return p.t_den > 0 && p.t_num >= 0 && p.t_num <= p.t_den && p.tau1_den > 0 && p.tau1_den <= 65536 &&
           p.tau1_num >= 0 && p.tau1_num <= p.tau1_den && p.max_subrounds >= 1 && p.round_offset >= 0 &&
           p.total_rounds >= 0 && p.total_rounds <= 65536 && (p.autotune == 0 || p.autotune == 1) &&
           p.table >= 0 && p.table <= 3 && (p.graphs >= 0 && p.graphs <= 2) && p.schedule >= 0 && p.schedule <= 6 && p.lp_rounds >= 0 && p.lp_rounds <= 64 &&
           (p.lock_rebalanced == 0 || p.lock_rebalanced == 1) &&
           (p.gain_priority == 0 || p.gain_priority == 1) && (p.append == 0 || p.append == 1);
}

}  // extern "C"

namespace upr {

// (Re)binds a context to one graph (ng = 1) or to a batch of ng graphs packed
// into one CSR: checks them, lays out the workspace (reusing the context's
// device arena when it is large enough), copies the graphs and computes
// omega(I(v)).  Pinned host buffers and events are created once per context.
// On error the context is left unbound (n = -1) but reusable.
// Host threads for a pass over n nodes: one per 2^18 nodes, at most 16.
int host_threads(int64_t n) {
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    return (int)std::max<int64_t>(1, std::min<int64_t>({hw, (int64_t)16, n >> 18}));
}

// fn(t, v0, v1) on [0, n) split into `parts` contiguous segments, segment t on
// its own thread (the calling thread takes segment 0).
template <typename F>
void parallel_segments(int64_t n, int parts, F fn) {
    if (parts <= 1 || n <= 0) {
        fn(0, 0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 1; t < parts; t++) th.emplace_back(fn, t, n * t / parts, n * (t + 1) / parts);
    fn(0, 0, n / parts);
    for (auto &x : th) x.join();
}

// The binding's key (upr_ctx::bkey): the host values the captured graphs'
// launches were built from.  Everything else they read is device data that
// a binding rewrites in full.
std::vector<int64_t> bind_key(const upr_ctx *c) {
    static_assert(sizeof(upr_params) % sizeof(int64_t) == 0, "parameters as whole words");
    std::vector<int64_t> key = {c->n, c->m, c->k, c->ng, c->G.kmask, c->G.adjw != nullptr, c->G.vwgt != nullptr,
                                c->sp_slots, c->sp_buf_cap, c->sparse_on, c->n_chunks, c->n_tiles, c->tile_nodes,
                                c->gbits, c->cbits, c->wmax, c->Lmax, c->total_w, c->eps_ppm,
                                (int64_t)(uintptr_t)c->mem, (int64_t)c->mem_bytes, (int64_t)(uintptr_t)c->W};
    const size_t words = sizeof(upr_params) / sizeof(int64_t);
    key.resize(key.size() + words);
    memcpy(key.data() + key.size() - words, &c->prm, sizeof(upr_params));
    key.insert(key.end(), c->noff.begin(), c->noff.end());
    key.insert(key.end(), c->Lmax_g.begin(), c->Lmax_g.end());
    return key;
}

upr_status bind_graphs(upr_ctx *c, const upr_graph *gs, int32_t ng, int32_t k, const double *eps,
                       const upr_params &prm) {
    if (!gs || !eps || ng < 1 || k < 2 || k > kMaxK || (int64_t)ng * k >= (1LL << 30) || !params_ok(prm))
        return UPR_ERR_INVALID;
    int64_t n = 0, m = 0;
    bool any_adjw = false, any_vwgt = false;
    for (int32_t i = 0; i < ng; i++) {
        const upr_graph *g = &gs[i];
        if (g->n < 0 || g->m < 0 || !(eps[i] > 0) || eps[i] > 1000.0 || (g->n > 0 && !g->xadj) ||
            (g->m > 0 && !g->adjncy))
            return UPR_ERR_INVALID;
        n += g->n;
        m += g->m;
        any_adjw = any_adjw || g->adjwgt;
        any_vwgt = any_vwgt || g->vwgt;
    }
    if (n >= (1LL << 31) || m >= (1LL << 31)) return UPR_ERR_INVALID;
    const auto t_bind0 = std::chrono::steady_clock::now();
    // the previous binding's key, if nothing invalidated its graphs since
    const bool kept_ok = c->n >= 0 && c->bkey_gen == c->gen;
    const uint64_t gen0 = c->gen;
    const int64_t calls0 = c->calls_bound, rounds0 = c->rounds_bound;
    std::vector<int64_t> key0;
    key0.swap(c->bkey);
    c->bkey_gen = ~0ull;
    c->n = -1;
    c->table_valid = false;
    UPR_CUDA(cudaGetDevice(&c->device));
    c->prm = prm;
    c->s = (cudaStream_t)prm.stream;
    c->ng = ng;
    c->eps_ppm = (int64_t)(eps[0] * 1e6 + 0.5);
    // the packed xadj on the host (the caller's array itself for one graph in
    // host memory) and the per-graph sums for create-time decisions; the
    // passes over the nodes run on several host threads
    c->noff.assign(ng + 1, 0);
    c->Lmax_g.assign(ng, 0);
    std::vector<int64_t> eoff(ng + 1, 0);
    for (int32_t i = 0; i < ng; i++) {
        c->noff[i + 1] = c->noff[i] + gs[i].n;
        eoff[i + 1] = eoff[i] + gs[i].m;
    }
    // the packed xadj of a batch (or of a graph whose xadj is device
    // memory) goes to the context's pinned staging buffer, kept across
    // bindings, so that its upload is a DMA from pinned memory
    const int nthreads = host_threads(n);
    int64_t cmax = 1;
    for (int32_t i = 0; i < ng; i++) {
        const upr_graph *g = &gs[i];
        const int64_t gn = g->n;
        int64_t total = gn;
        if (g->vwgt && gn > 0) {
            std::vector<int32_t> vw(gn);
            if (mem_kind(g->vwgt) == kDevice)
                UPR_CUDA(cudaMemcpy(vw.data(), g->vwgt, sizeof(int32_t) * gn, cudaMemcpyDeviceToHost));
            else
                memcpy(vw.data(), g->vwgt, sizeof(int32_t) * gn);
            total = 0;
            for (int32_t w : vw) {
                if (w <= 0) return UPR_ERR_INVALID;
                total += w;
                cmax = std::max<int64_t>(cmax, w);
            }
        }
        const int64_t eps_ppm = (int64_t)(eps[i] * 1e6 + 0.5);
        const int64_t avg = (total + k - 1) / k;
        c->Lmax_g[i] = (int64_t)(((i128)avg * (1000000 + eps_ppm)) / 1000000);
        if (i == 0) c->total_w = total;
    }
    c->Lmax = c->Lmax_g[0];
    c->cbits = bit_length((uint64_t)cmax);
    // the packed offsets on the device (a staging buffer kept across
    // bindings), checked there for one graph, and the static schedules
    // counted (bind.cu): hub chunks of 8192 entries of one node of degree >
    // kHubDegree, the table build's tiles (at most tile_nodes rows, <= 32 KB
    // of shared memory), the hashed rows' slots, the hubs
    cudaStream_t s = c->s;
    if (!c->h) {
        UPR_CUDA(cudaMallocHost((void **)&c->h, sizeof(int64_t) * (4 * (int64_t)kMaxK + 256)));
        int64_t *hb = c->h + 4 * (int64_t)kMaxK;
        c->hF = hb;                                             // 73
        c->hcut = hb + 80;                                      // 1
        c->hbest = reinterpret_cast<long long *>(hb + 88);      // 3
        c->hctl = reinterpret_cast<RebalCtl *>(hb + 96);        // 4
        c->hcnt = reinterpret_cast<int32_t *>(hb + 112);        // 64 ints
    }
    // one graph rebound to an arena that already has room for its adjacency
    // at the adjacency's offset (which depends only on n, m, k and ng): the
    // adjacency upload starts now on a side stream, beside the offsets'
    // checks and the schedules, after the work already queued on s
    bool early = false;
    size_t adj_off = 0;
    // whatever way the binding ends, the early copy has landed before the
    // arena can be freed or written again
    struct UpGuard {
        upr_ctx *c;
        bool on = false;
        ~UpGuard() { if (on) cudaEventSynchronize(c->ev_up); }
    } up_guard{c};
    if (ng == 1 && m > 0 && c->mem) {
        upr_ctx dry;
        dry.n = n; dry.m = m; dry.k = k; dry.ng = ng;
        Arena D;
        D.base = reinterpret_cast<char *>((uintptr_t)1 << 20);
        layout(&dry, D);
        adj_off = (size_t)(reinterpret_cast<char *>(dry.adj) - D.base);
        if (c->mem_bytes >= adj_off + sizeof(int32_t) * (size_t)m) {
            if (!c->s_up) UPR_CUDA(cudaStreamCreateWithFlags(&c->s_up, cudaStreamNonBlocking));
            if (!c->ev_up) UPR_CUDA(cudaEventCreateWithFlags(&c->ev_up, cudaEventDisableTiming));
            if (!c->ev_prev) UPR_CUDA(cudaEventCreateWithFlags(&c->ev_prev, cudaEventDisableTiming));
            early = true;           // (issued below, after the offsets' copy, which the schedules wait for)
        }
    }
    // staging layout: packed offsets [n + 1], schedule counts [4 nseg], 8
    // words (totals, largest row, check flag); a batch adds each graph's own
    // offsets [n + ng] and the graphs' node and entry offsets [ng + 1] x 2
    const int64_t nseg = sched_segments(n);
    const int64_t xs_need = n + 1 + 4 * nseg + 8 + (ng > 1 ? n + ng + 2 * (ng + 1) : 0);
    if (c->xs_cap < xs_need) {
        if (c->xs) cudaFree(c->xs);
        c->xs = nullptr;
        c->xs_cap = 0;
        if (cudaMalloc(&c->xs, sizeof(int64_t) * (size_t)xs_need) != cudaSuccess) {
            cudaGetLastError();
            return UPR_ERR_OOM;
        }
        c->xs_cap = xs_need;
    }
    int64_t *sx = c->xs, *scnt = c->xs + n + 1, *stot = scnt + 4 * nseg;   // stot: 4 totals, cap, check flag
    UPR_CUDA(cudaMemsetAsync(stot, 0, 8 * sizeof(int64_t), s));
    if (ng == 1) {
        if (n > 0) copy_in(sx, gs[0].xadj, sizeof(int64_t) * (n + 1), s);
        else UPR_CUDA(cudaMemsetAsync(sx, 0, sizeof(int64_t), s));
        if (early) {
            UPR_CUDA(cudaEventRecord(c->ev_prev, s));
            UPR_CUDA(cudaStreamWaitEvent(c->s_up, c->ev_prev, 0));
            copy_in(static_cast<char *>(c->mem) + adj_off, gs[0].adjncy, sizeof(int32_t) * m, c->s_up);
            UPR_CUDA(cudaEventRecord(c->ev_up, c->s_up));
            up_guard.on = true;
        }
        xadj_check(sx, n, m, reinterpret_cast<int32_t *>(stot + 5), s);
    } else {
        // each graph's offsets as given, then packed (shifted by the entries of
        // the graphs before it) and checked on the device
        int64_t *raw = stot + 8, *d_noff = raw + n + ng, *d_eoff = d_noff + ng + 1;
        std::vector<const void *> src(ng);
        std::vector<int64_t> off(ng), len(ng);
        for (int32_t i = 0; i < ng; i++) {
            src[i] = gs[i].xadj;
            off[i] = c->noff[i] + i;
            len[i] = gs[i].n > 0 ? gs[i].n + 1 : 0;
        }
        copy_many(c, src, off, len, sizeof(int64_t), raw, s);
        UPR_CUDA(cudaMemcpyAsync(d_noff, c->noff.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
        UPR_CUDA(cudaMemcpyAsync(d_eoff, eoff.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
        xadj_pack(raw, d_noff, d_eoff, ng, n, sx, reinterpret_cast<int32_t *>(stot + 5), s);
    }
    const int32_t tile_nodes = (int32_t)std::max<int64_t>(4, std::min<int64_t>(512, 8192 / k));
    // sparse rows: a power of two >= min(k, 2 deg(v)) + 1 slots per row (mode 3:
    // min(k, deg(v)) + 1); chosen by size (mode 0) when k >= 128 and the rows
    // take at most half the bytes of the dense table
    const int mode = prm.table;
    const int sp_mode = (k % 4 == 0 && k <= kSparseRowMax / 2 && (mode >= 2 || (mode == 0 && k >= 128)))
                            ? (mode == 3 ? 3 : 1) : 0;
    sched_count(sx, n, m, tile_nodes, sp_mode, k, scnt, stot, reinterpret_cast<unsigned long long *>(stot + 4), s);
    int64_t *ht = c->h;                      // (the pinned block's first words: free outside a call)
    UPR_CUDA(cudaMemcpyAsync(ht, stot, 6 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    UPR_CUDA(cudaStreamSynchronize(s));
    if ((int32_t)ht[5] != 0) return UPR_ERR_INVALID;
    const int64_t n_hubs = ht[3];
    {
        int64_t total = sp_mode ? ht[2] : 0, buf_cap = sp_mode ? std::max<int64_t>(1, ht[4]) : 1;
        if (sp_mode && mode == 0 && total * (int64_t)sizeof(int2) * 2 > n * (int64_t)k * (int64_t)sizeof(int32_t))
            total = 0, buf_cap = 1;
        c->sp_slots = total;
        c->sp_buf_cap = (int32_t)buf_cap;
    }
    const int sp_write = c->sp_slots > 0 ? sp_mode : 0;
    const auto t_sched = std::chrono::steady_clock::now();
    c->m = m; c->k = k;
    c->n = n;                       // layout needs the sizes
    c->n_chunks = ht[0];
    c->n_tiles = tile_nodes ? ht[1] : 0;
    c->tile_nodes = tile_nodes;
    Arena A;
    if (c->W_own) { cudaFree(c->W_own); c->W_own = nullptr; c->W_own_bytes = 0; }
    c->gen++;                       // kernels captured for the previous binding are stale
    c->rounds_bound = 0;
    c->calls_bound = 0;
    c->step_failed = false;
    layout(c, A);
    if (!c->mem || c->mem_bytes < A.off) {
        if (early) { UPR_CUDA(cudaEventSynchronize(c->ev_up)); early = false; }     // (its target is freed)
        if (c->mem) { cudaFree(c->mem); c->mem = nullptr; c->mem_bytes = 0; }
        if (cudaMalloc(&c->mem, A.off) != cudaSuccess) { cudaGetLastError(); c->n = -1; return UPR_ERR_OOM; }
        c->mem_bytes = A.off;
    }
    A.base = (char *)c->mem; A.off = 0;
    layout(c, A);
    const auto t_alloc = std::chrono::steady_clock::now();
    // pinned buffers and events are sized for kMaxK blocks, so a context
    // re-bound to another graph keeps them
    if (!c->h8) UPR_CUDA(cudaMallocHost((void **)&c->h8, 2 * (size_t)kMaxK + 64));
    for (auto &ev : c->ev)
        if (!ev) UPR_CUDA(cudaEventCreate(&ev));
    for (auto &ev : c->ev_tune)
        if (!ev) UPR_CUDA(cudaEventCreate(&ev));
    c->sel_cfg = c->prop_cfg = LaneCfg{0, 0};
    c->sel_tuned = c->prop_tuned = false;
    c->sel_pending = c->prop_pending = 0;
    UPR_CUDA(cudaMemcpyAsync(c->xadj, sx, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
    // the schedules written (the hub list into a sort buffer, free until the
    // first round, for the duplicate check)
    int32_t *hubs_d = reinterpret_cast<int32_t *>(c->sb[0].v);
    sched_write(c->xadj, n, m, tile_nodes, sp_write, k, scnt, c->hub_chunks, c->tiles, c->sp_off, hubs_d, s);
    if (early && reinterpret_cast<char *>(c->adj) != static_cast<char *>(c->mem) + adj_off) {
        UPR_CUDA(cudaEventSynchronize(c->ev_up));       // (not where the layout put it: copied again)
        early = false;
    }
    if (early) UPR_CUDA(cudaStreamWaitEvent(s, c->ev_up, 0));
    {
        // the graphs' arrays (a batch's as one gather each where they are
        // page-locked host memory); unit weights where a graph has none
        std::vector<const void *> sa, sw, sv;
        std::vector<int64_t> oa, la, ow, lw, ov, lv;
        for (int32_t i = 0; i < ng; i++) {
            const upr_graph *g = &gs[i];
            const int64_t v0 = c->noff[i], e0 = eoff[i];
            if (!early) { sa.push_back(g->adjncy); oa.push_back(e0); la.push_back(g->m); }
            if (g->adjwgt) { sw.push_back(g->adjwgt); ow.push_back(e0); lw.push_back(g->m); }
            else if (any_adjw) fill_i32(c->adjw + e0, g->m, 1, s);
            if (g->vwgt) { sv.push_back(g->vwgt); ov.push_back(v0); lv.push_back(g->n); }
            else if (any_vwgt) fill_i32(c->vwgt + v0, g->n, 1, s);
        }
        copy_many(c, sa, oa, la, sizeof(int32_t), c->adj, s);
        copy_many(c, sw, ow, lw, sizeof(int32_t), c->adjw, s);
        copy_many(c, sv, ov, lv, sizeof(int32_t), c->vwgt, s);
    }
    {
        std::vector<int64_t> Lb((size_t)ng * k);
        for (int32_t i = 0; i < ng; i++)
            for (int32_t b = 0; b < k; b++) Lb[(size_t)i * k + b] = c->Lmax_g[i];
        UPR_CUDA(cudaMemcpyAsync(c->Lb, Lb.data(), sizeof(int64_t) * Lb.size(), cudaMemcpyHostToDevice, s));
        UPR_CUDA(cudaStreamSynchronize(s));     // Lb is a local vector
    }

    const int32_t kmask = ng == 1 ? -1 : ((k & (k - 1)) == 0 ? k - 1 : 0);
    c->sparse_on = c->sp_slots > 0;
    UPR_CUDA(cudaMemsetAsync(c->sp_over, 0, sizeof(int32_t), s));
    c->G = GraphDev{n,      m,        k,       ng,   kmask, c->xadj, c->adj, any_adjw ? c->adjw : nullptr,
                    any_vwgt ? c->vwgt : nullptr, c->wI, c->Lb, c->gid,
                    SparseRows{c->sp_off, c->sparse_on ? c->sp_slot : nullptr, c->sp_over, c->sp_buf_cap}};
    if (prm.autotune) recall_tuning(c);
    if (ng > 1) {
        // node -> graph, and graph-local neighbour ids made global
        UPR_CUDA(cudaMemcpyAsync(c->noff_d, c->noff.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
        pack_batch(c->G, c->noff_d, c->gid, c->adj, s);
        UPR_CUDA(cudaStreamSynchronize(s));     // noff is host memory that may be re-assigned
    }
    if (prm.validate) {
        validate_graph(c->G, c->vacc, c->vflags, s);
        uint64_t acc[2]; int32_t flags;
        UPR_CUDA(cudaMemcpyAsync(acc, c->vacc, sizeof(acc), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaMemcpyAsync(&flags, c->vflags, sizeof(flags), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaStreamSynchronize(s));
        if ((flags & ~128) != 0 || acc[0] != acc[1]) { c->n = -1; return UPR_ERR_INVALID; }
        if (flags & 128) {
            // a row that is not strictly increasing: the exact duplicate check
            // (the hub list goes to a sort buffer, free until the first round)
            UPR_CUDA(cudaMemsetAsync(c->vflags, 0, sizeof(int32_t), s));
            int64_t max_nodes = 0;
            for (int32_t i = 0; i < ng; i++) max_nodes = std::max<int64_t>(max_nodes, c->noff[i + 1] - c->noff[i]);
            validate_duplicates(c->G, c->vflags, hubs_d, n_hubs, c->noff_d, max_nodes,
                                reinterpret_cast<int32_t *>(c->sb[1].k), 4 * std::max<int64_t>(n, 1), s);
            UPR_CUDA(cudaMemcpyAsync(&flags, c->vflags, sizeof(flags), cudaMemcpyDeviceToHost, s));
            UPR_CUDA(cudaStreamSynchronize(s));
            if (flags != 0) { c->n = -1; return UPR_ERR_INVALID; }
        }
    }
    const auto t_valid = std::chrono::steady_clock::now();
    incident_weights(c->G, c->wI, c->scal, s);
    read_i64(c, c->scal, 1, &c->wmax);
    if (c->wmax > 0x7fffffffLL) { c->n = -1; return UPR_ERR_INVALID; }
    c->gbits = std::max(1, bit_length((uint64_t)c->wmax));
    // the arena may hold another binding's data: clear every word a kernel
    // reads before writing it
    UPR_CUDA(cudaMemsetAsync(c->tmp.ticket, 0, 64 * sizeof(unsigned int), s));
    UPR_CUDA(cudaMemsetAsync(c->tmp.mem, 0, c->tmp.mem_bytes, s));
    UPR_CUDA(cudaMemsetAsync(c->tmp.scan, 0, c->tmp.scan_bytes, s));
    UPR_CUDA(cudaMemsetAsync(c->tmp.err, 0, sizeof(int32_t), s));
    UPR_CUDA(cudaMemsetAsync(c->tmp.epoch, 0, sizeof(uint32_t), s));
    UPR_CUDA(cudaMemsetAsync(c->ctl, 0, sizeof(RebalCtl), s));
    UPR_CUDA(cudaMemsetAsync(c->counts, 0, 64 * sizeof(int32_t), s));
    UPR_CUDA(cudaMemsetAsync(c->Cd, 0, sizeof(long long) * (size_t)c->G.K(), s));
    fill_i32(c->pos, n, INT32_MAX, s);
    fill_i32(c->m_pos, n, -1, s);
    fill_i32(c->r_to, n, -1, s);
    UPR_CUDA(cudaStreamSynchronize(s));
    c->bkey = bind_key(c);
    if (kept_ok && c->bkey == key0) {
        // the same key: the graphs captured for the previous binding launch
        // the same kernels with the same arguments on this one
        c->gen = gen0;
        c->calls_bound = calls0;
        c->rounds_bound = rounds0;
    }
    c->bkey_gen = c->gen;
    if (log_enabled()) {
        const auto t_end = std::chrono::steady_clock::now();
        auto ms = [](auto a, auto b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
        fprintf(stderr, "upr bind: %lld nodes, %d host threads: schedules %.2f ms, arena %.2f ms (%.2f GB), "
                        "upload and checks %.2f ms, incident weights and clears %.2f ms\n",
                (long long)n, nthreads, ms(t_bind0, t_sched), ms(t_sched, t_alloc), A.off / 1e9,
                ms(t_alloc, t_valid), ms(t_valid, t_end));
    }
    return UPR_OK;
}

template <typename F>
upr_status guarded(upr_ctx *c, F f) {
    try {
        return f();
    } catch (const CudaError &e) {
        c->n = -1;
        return cuda_failure(e);
    } catch (const std::bad_alloc &) {
        c->n = -1;
        return UPR_ERR_OOM;
    }
}

upr_status ctx_rebind(upr_ctx *c, const upr_graph *g, int32_t k, double eps, const upr_params *params) {
    upr_params prm;
    upr_params_default(&prm);
    if (params) prm = *params;
    if (!g) return UPR_ERR_INVALID;
    if (g->n >= (1LL << 31) || g->m >= (1LL << 31)) return UPR_ERR_INVALID;
    return guarded(c, [&] { return bind_graphs(c, g, 1, k, &eps, prm); });
}

// Device bytes of the context's arena.
size_t ctx_arena_bytes(const upr_ctx *c) { return c ? c->mem_bytes + sizeof(int64_t) * (size_t)c->xs_cap : 0; }

upr_status ctx_rebind_batch(upr_ctx *c, const upr_graph *gs, int32_t ng, int32_t k, const double *eps,
                            const upr_params *params) {
    upr_params prm;
    upr_params_default(&prm);
    if (params) prm = *params;
    return guarded(c, [&] { return bind_graphs(c, gs, ng, k, eps, prm); });
}

}  // namespace upr

extern "C" {

upr_status upr_create(const upr_graph *g, int32_t k, double eps, const upr_params *params, upr_ctx **out) {
    if (!out) return UPR_ERR_INVALID;
    upr_ctx *c = new (std::nothrow) upr_ctx();
    if (!c) return UPR_ERR_OOM;
    const upr_status st = upr::ctx_rebind(c, g, k, eps, params);
    if (st != UPR_OK) { free_ctx(c); return st; }
    *out = c;
    return UPR_OK;
}

void upr_destroy(upr_ctx *c) { free_ctx(c); }

upr_status upr_cut(upr_ctx *c, const int32_t *part, int64_t *cut, int64_t *block_weights_out) {
    if (!c || c->mix || c->n < 0 || c->ng != 1 || !part || !cut) return UPR_ERR_INVALID;
    try {
        upr_status st = load_part(c, part);
        if (st != UPR_OK) return st;
        int64_t tmp[1];
        read_i64(c, c->cut, 1, tmp);
        *cut = tmp[0];
        if (block_weights_out) read_i64(c, c->C0, c->k, block_weights_out);
    } catch (const CudaError &e) {
        return cuda_failure(e);
    }
    return UPR_OK;
}

upr_status upr_refine(upr_ctx *c, int32_t *part, int32_t rounds, uint64_t seed, upr_stats *stats) {
    (void)seed;
    if (!c || c->mix || c->n < 0 || c->ng != 1 || (!part && c->n > 0) || rounds < 0) return UPR_ERR_INVALID;
    try {
        return refine_impl(c, part, rounds, stats, nullptr, nullptr, nullptr);
    } catch (const CudaError &e) {
        return cuda_failure(e);
    }
}

upr_status upr_batch_create(const upr_graph *graphs, int32_t n_graphs, int32_t k, const double *eps,
                            const upr_params *params, upr_ctx **out) {
    if (!out || !graphs || !eps || n_graphs < 1) return UPR_ERR_INVALID;
    upr_ctx *c = new (std::nothrow) upr_ctx();
    if (!c) return UPR_ERR_OOM;
    const upr_status st = upr::ctx_rebind_batch(c, graphs, n_graphs, k, eps, params);
    if (st != UPR_OK) { free_ctx(c); return st; }
    *out = c;
    return UPR_OK;
}

upr_status upr_batch_create_mixed(const upr_graph *graphs, int32_t n_graphs, const int32_t *k, const double *eps,
                                  const upr_params *params, upr_ctx **out) {
    if (!out || !graphs || !eps || !k || n_graphs < 1) return UPR_ERR_INVALID;
    upr_ctx *c = new (std::nothrow) upr_ctx();
    if (!c) return UPR_ERR_OOM;
    const upr_status st = upr::mixed_create(graphs, n_graphs, k, eps, params, &c->mix);
    if (st != UPR_OK) { delete c; return st; }
    c->n = upr::mixed_nodes(c->mix);
    c->ng = n_graphs;
    *out = c;
    return UPR_OK;
}

upr_status upr_batch_rebind(upr_ctx *c, const upr_graph *graphs, int32_t n_graphs, const int32_t *k,
                            const double *eps) {
    if (!c || !graphs || !k || !eps || n_graphs < 1) return UPR_ERR_INVALID;
    if (c->mix) {
        const upr_status st = upr::mixed_rebind(c->mix, graphs, n_graphs, k, eps);
        c->n = st == UPR_OK ? upr::mixed_nodes(c->mix) : -1;
        c->ng = n_graphs;
        return st;
    }
    for (int32_t i = 1; i < n_graphs; i++)
        if (k[i] != k[0]) return UPR_ERR_INVALID;        // one k: a mixed context takes several
    if (n_graphs == 1) return upr::ctx_rebind(c, graphs, k[0], eps[0], &c->prm);
    return upr::ctx_rebind_batch(c, graphs, n_graphs, k[0], eps, &c->prm);
}

upr_status upr_batch_refine(upr_ctx *c, int32_t *part, int32_t rounds, uint64_t seed, upr_status *status,
                            int64_t *cut_in, int64_t *cut_out, upr_stats *stats) {
    (void)seed;
    if (c && c->mix) {
        if (c->n < 0) return UPR_ERR_INVALID;
        return upr::mixed_refine(c->mix, part, rounds, seed, status, cut_in, cut_out, stats);
    }
    if (!c || c->n < 0 || (!part && c->n > 0) || rounds < 0) return UPR_ERR_INVALID;
    try {
        upr_status rc = refine_impl(c, part, rounds, stats, status, cut_in, cut_out);
        if (rc == UPR_ERR_INFEASIBLE && c->ng == 1) {
            // one graph through the batch entry: a per-graph status, input kept
            int64_t cut = 0;
            read_i64(c, c->cut, 1, &cut);
            if (status) status[0] = UPR_ERR_INFEASIBLE;
            if (cut_in) cut_in[0] = cut;
            if (cut_out) cut_out[0] = cut;
            if (stats) { *stats = upr_stats{}; stats->cut_in = stats->cut_out = cut; }
            rc = UPR_OK;
        }
        return rc;
    } catch (const CudaError &e) {
        return cuda_failure(e);
    }
}

upr_status upr_batch_cut(upr_ctx *c, const int32_t *part, int64_t *cut, int64_t *block_weights_out) {
    if (c && c->mix) return c->n < 0 ? UPR_ERR_INVALID : upr::mixed_cut(c->mix, part, cut, block_weights_out);
    if (!c || c->n < 0 || !part || !cut) return UPR_ERR_INVALID;
    try {
        upr_status st = load_part(c, part);
        if (st != UPR_OK) return st;
        read_i64(c, c->cut, c->ng, cut);
        if (block_weights_out) read_i64(c, c->C0, c->G.K(), block_weights_out);
    } catch (const CudaError &e) {
        return cuda_failure(e);
    }
    return UPR_OK;
}

upr_status upr_batch_info(const upr_ctx *c, int32_t *n_graphs, int64_t *node_offsets, int64_t *lmax) {
    if (c && c->mix) return c->n < 0 ? UPR_ERR_INVALID : upr::mixed_info(c->mix, n_graphs, node_offsets, lmax);
    if (!c || c->n < 0) return UPR_ERR_INVALID;
    if (n_graphs) *n_graphs = c->ng;
    if (node_offsets) memcpy(node_offsets, c->noff.data(), sizeof(int64_t) * (c->ng + 1));
    if (lmax) memcpy(lmax, c->Lmax_g.data(), sizeof(int64_t) * c->ng);
    return UPR_OK;
}

upr_status upr_debug_gain_table(upr_ctx *c, const int32_t *part, int32_t *W, int64_t *wI) {
    if (!c || c->mix || c->n < 0 || c->ng != 1 || !part) return UPR_ERR_INVALID;
    try {
        upr_status rc = load_part(c, part);
        if (rc != UPR_OK) return rc;
        ensure_dense(c);
        gain_table(c->G, c->part0, c->W, c->hub_chunks, c->n_chunks, c->n_tiles ? c->tiles : nullptr, c->n_tiles,
                   c->tile_nodes, nullptr, c->s);
        sparse_to_dense(c->G, c->W, c->s);
        if (W) UPR_CUDA(cudaMemcpyAsync(W, c->W, sizeof(int32_t) * c->n * c->k, cudaMemcpyDeviceToHost, c->s));
        if (wI && c->n > 0) {
            std::vector<int32_t> w(c->n);
            UPR_CUDA(cudaMemcpyAsync(w.data(), c->wI, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->s));
            UPR_CUDA(cudaStreamSynchronize(c->s));
            for (int64_t v = 0; v < c->n; v++) wI[v] = w[v];
        }
        UPR_CUDA(cudaStreamSynchronize(c->s));
    } catch (const CudaError &e) {
        return cuda_failure(e);
    }
    return UPR_OK;
}

upr_status upr_debug_round(upr_ctx *c, int32_t *part, int32_t r, int32_t R, int32_t rebalance_only, upr_trace *trace) {
    if (!c || c->mix || c->n < 0 || c->ng != 1 || !part || !trace || R < 1 || R > 65536 ||
        (!rebalance_only && (r < 1 || r > R)))
        return UPR_ERR_INVALID;
    int8_t *avail_d = nullptr;
    int32_t *slot_d = nullptr;
    upr_status rc = UPR_OK;
    try {
        rc = load_part(c, part);
        if (rc != UPR_OK) return rc;
        UPR_CUDA(cudaMalloc(&avail_d, std::max<int64_t>(c->n, 1)));
        UPR_CUDA(cudaMalloc(&slot_d, sizeof(int32_t) * std::max<int64_t>(c->n, 1)));
        TraceSink ts{trace, avail_d, slot_d};
        RoundInfo ri;
        rc = run_round(c, r, R, rebalance_only != 0, ri, &ts);
        if (rc == UPR_OK) copy_out(part, c->part0, sizeof(int32_t) * c->n, c->s);
        UPR_CUDA(cudaStreamSynchronize(c->s));
    } catch (const CudaError &e) {
        rc = cuda_failure(e);
    }
    if (avail_d) cudaFree(avail_d);
    if (slot_d) cudaFree(slot_d);
    return rc;
}

}  // extern "C"

// Device bytes a context for ng graphs with n nodes and m adjacency entries
// in total and k blocks each allocates (used by the server's admission).
size_t upr_ctx_footprint(int64_t n, int64_t m, int32_t k, int32_t ng) {
    upr_ctx c;
    c.n = n; c.m = m; c.k = k; c.ng = ng;
    c.n_chunks = m / 4096 + 1;
    c.n_tiles = n + 1;
    c.sp_slots = 0;     // the dense layout bounds the sparse one (rows chosen by size take half as many bytes)
    Arena A;
    layout(&c, A);
    // plus the staging buffer of the offsets and schedule counts
    return A.off + sizeof(int64_t) * (size_t)(n + 1 + 4 * sched_segments(n) + 8) + ((size_t)1 << 20);
}
