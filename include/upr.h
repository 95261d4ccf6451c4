/*
 * upr.h -- unconstrained FM refinement for balanced k-way graph partitioning
 * on one NVIDIA GB300 GPU (sm_103a).
 *
 * The library refines a k-way partition of an undirected graph G = (V, E,
 * c, omega) with integer node weights c > 0 and edge weights omega > 0 (Sec. 2
 * of Maas, Gottesbueren, Seemaier, "Parallel Unconstrained Local Search for
 * Partitioning Irregular Graphs", arXiv 2308.15494).  One round is the
 * deterministic synchronous form of Algorithm 1:
 *   (a) gain table omega(v, V_b) (Sec. 6.1),
 *   (b) selection of moves that ignore the balance constraint, scored by
 *       gain minus the rebalancing-cost penalty of Sec. 4.3, scaled by the
 *       tau schedule of Sec. 4.4,
 *   (d) rebalancing by gain-per-weight priority (Sec. 6),
 *   (c) interleaving of the moves with the rebalancing moves, exact gain
 *       recalculation and application of the best balanced prefix (Sec. 4.4,
 *       Alg. 1), so the cut never increases,
 *   (e) exact cut and block weights (Sec. 2).
 * Every quantity is an integer and every tie is broken by node or block id,
 * so results are bit-for-bit reproducible and equal those of the sequential
 * reference definition of the round.
 *
 * Conventions for every entry point:
 *  - Return value: UPR_OK (0) on success, UPR_PENDING (1) for a job that is not
 *    finished, a negative upr_status on error.  On error no output argument
 *    is modified and the context stays usable unless the status is
 *    UPR_ERR_CUDA (a CUDA error that may have left the device unusable).
 *  - Pointers to graph or partition data may be host or device memory; the
 *    library detects which (cudaPointerGetAttributes).  Device pointers must
 *    be on the device that was current when the context was created.
 *  - All device work of a context runs on the stream given in upr_params
 *    (NULL = the legacy default stream); every call returns after its results
 *    are in the caller's buffers (it synchronises that stream).
 *  - Contexts are not thread-safe: one thread at a time per context.
 */
#ifndef UPR_H
#define UPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t upr_status;
#define UPR_OK               0
#define UPR_PENDING          1
#define UPR_ERR_INVALID     (-1)  /* malformed graph, partition or parameter            */
#define UPR_ERR_OOM         (-2)  /* device or host allocation failed                   */
#define UPR_ERR_CUDA        (-3)  /* a CUDA runtime call failed                          */
#define UPR_ERR_INFEASIBLE  (-4)  /* an imbalanced input could not be rebalanced         */
#define UPR_ERR_BUSY        (-5)  /* server queue full                                  */
#define UPR_ERR_TIMEOUT     (-6)  /* a bounded wait expired                              */
#define UPR_ERR_NOT_FOUND   (-7)  /* unknown ticket                                      */

typedef struct upr_ctx upr_ctx;
typedef struct upr_server upr_server;

/* An undirected graph in CSR form (Sec. 2).  Every edge {u,v} appears twice,
 * as v in u's list and u in v's list, with equal weight, and a list holds each
 * neighbour once (E is a set of pairs).  n < 2^31, m < 2^31.
 * on_device: ignored (the library inspects the pointers); kept for callers
 * that want to state it. */
typedef struct {
    int64_t        n;        /* number of nodes                                      */
    int64_t        m;        /* number of adjacency entries (= 2|E|)                 */
    const int64_t *xadj;     /* [n+1], xadj[0] = 0, non-decreasing, xadj[n] = m      */
    const int32_t *adjncy;   /* [m], neighbour ids in [0, n), no self loops, no
                                duplicates within a row                              */
    const int32_t *vwgt;     /* [n] node weights c(v) > 0, or NULL for unit weights  */
    const int32_t *adjwgt;   /* [m] edge weights omega > 0, or NULL for unit weights */
    int32_t        on_device;
} upr_graph;

typedef struct {
    int32_t t_num, t_den;        /* rebalancing-availability threshold t (Sec. 4.3): a node v
                                    is available if omega(v, P(v)) >= t * omega(I(v)). 7/10  */
    int32_t tau1_num, tau1_den;  /* tau_1, the penalty factor of round 1 (Sec. 4.4); rounds
                                    interpolate linearly to 1. 1/4; tau1_den <= 65536       */
    int32_t max_subrounds;       /* rebalancing sub-rounds per round. 64                      */
    int32_t validate;            /* 1: check the graph in upr_create: offsets, neighbour
                                    ranges, self loops, weights and duplicate neighbours
                                    exactly; symmetry with equal weights by a 64-bit
                                    multiset hash (an asymmetric graph is rejected with
                                    probability 1 - 2^-64 unless built against the hash).
                                    0: the caller guarantees all of it (a duplicate then
                                    counts as a second edge of the same pair). 1            */
    int32_t round_offset;        /* rounds already run of a longer schedule (resume). 0       */
    int32_t total_rounds;        /* length of the tau schedule; 0 = the rounds of each call   */
    int32_t autotune;            /* 1: on a context's first large calls, time the lane
                                    schedules of the selection and proposal kernels on the
                                    actual inputs and keep the fastest (results never depend
                                    on the schedule). 1                                      */
    int32_t table;               /* gain-table layout (results never depend on it): 0 auto
                                    (hashed rows of min(k, 2 deg) + 1 slots when k >= 128
                                    and they take at most half the bytes of the dense
                                    table, else dense), 1 dense, 2 hashed rows of
                                    min(k, 2 deg) + 1 slots, 3 hashed rows of
                                    min(k, deg) + 1 slots.  Hashed rows need k % 4 == 0 and
                                    k <= 256 (else the dense table is used); they carry no
                                    dense table: a round whose rows run out of slots runs
                                    again on rows built afresh, and if those run out too,
                                    on a dense table allocated then. 0                       */
    int32_t graphs;              /* 1: once the proposal schedule is settled, each round's
                                    rebalancing loop runs as one CUDA graph launch (a while
                                    node over one sub-round, the stop test on the device);
                                    2: also, from a binding's second call on, all FM
                                    rounds of a call run as one graph launch (schedule 0,
                                    dense table; after label propagation too; round 1's
                                    table build precedes the graph; the per-phase times of
                                    the stats are then 0); 0: the host launches every
                                    sub-round and reads its stop flag.  Results never
                                    depend on it. 1                                          */
    int32_t schedule;            /* round driver (Sec. 4.4, Sec. 6.2): 0 every round
                                    unconstrained with the tau schedule.  6 the paper's
                                    final configuration: the first U rounds unconstrained
                                    with tau from tau_1 to 1 over them, the rest
                                    constrained (U = R - 2 for R >= 3, the paper's eight
                                    and two of ten; U = 1 for R = 2; U = 0 for R = 1), and
                                    every round after one that improves the cut by less
                                    than 0.002 of it constrained.  The variants of
                                    Sec. 7.2 in the same frame: 3 constant penalty (tau =
                                    tau_1 every round), 4 fully unconstrained (no penalty,
                                    nothing forbidden), 5 limited imbalance (no penalty,
                                    no block above alpha * L_max, alpha from 2 to 1.1).
                                    1 dynamic activation (Sec. 4.4, which Sec. 7.2 leaves
                                    out of the final configuration): round 1 constrained,
                                    round 2 unconstrained with tau = 1/2, rounds 3..R-1
                                    unconstrained (tau schedule over them, with the same
                                    switch) if round 2 improved the cut more than round
                                    1, else constrained; round R constrained.  2 every
                                    round constrained.  A constrained round is the same
                                    round with every move that would leave its target
                                    above L_max forbidden.  1..6 need one graph,
                                    round_offset = 0 and total_rounds = 0. 0             */
    int32_t gain_priority;       /* rebalancing priority: 0 g/c(u) for g < 0 and g*c(u)
                                    for g >= 0 (Sec. 6.1); 1 the gain alone (the variant
                                    of Sec. 7.2), ties by node id either way. 0             */
    int32_t append;              /* move sequence: 0 the rebalancing moves interleaved with
                                    M (Sec. 4.4); 1 appended after M in their order (the
                                    variant of Sec. 7.2). 0                                  */
    int32_t lp_rounds;           /* rounds of unconstrained label propagation before the
                                    FM rounds (Sec. 5; the paper uses 5): every active node
                                    to its best positive-gain block, rebalancing, the round
                                    kept only if balanced and cutting less; next active set
                                    = the unmoved neighbours of moved nodes; stops at a
                                    round not kept, an empty active set or an improvement
                                    below 0.001 of the cut.  One graph only. 0 = off        */
    int32_t lock_rebalanced;     /* 1: the oscillation guard of Sec. 2: a node whose applied
                                    move in a round came from rebalancing alone is not a
                                    candidate in the next round of the call. 0              */
    void   *stream;              /* cudaStream_t for all device work; NULL = default stream   */
} upr_params;

/* Per-call statistics (all optional). */
typedef struct {
    int64_t cut_in, cut_out;     /* cut before and after the call                       */
    int32_t rounds_run;          /* refinement rounds executed                          */
    int32_t repaired_input;      /* 1 if an imbalanced input was rebalanced first       */
    int64_t n_candidates;        /* sum over rounds: nodes with a positive scored move  */
    int64_t n_moves;             /* sum over rounds: |M|                                */
    int64_t n_rebalance_moves;   /* sum over rounds: |R|                                */
    int64_t n_sequence;          /* sum over rounds: |I| after merging                  */
    int64_t n_applied;           /* sum over rounds: length of the applied prefix       */
    int32_t subrounds;           /* sum over rounds: rebalancing sub-rounds             */
    int32_t kernel_launches;     /* kernels launched by the call                        */
    double  ms_device;           /* device time of the call (CUDA events)               */
    double  ms_gain_table;       /* device time of gain-table builds                    */
    int32_t gain_table_builds;   /* number of full gain-table builds                    */
    int64_t gain_table_bytes;    /* algorithmic DRAM bytes of one build                 */
    double  ms_select;           /* device time of step (b) and applying M (with the
                                    table update after M)                               */
    double  ms_rebalance;        /* device time of step (d)                             */
    double  ms_sequence;         /* device time of step (c): interleave to apply        */
    double  ms_host;             /* wall-clock time of the call on the host             */
    int32_t batch_graphs;        /* graphs refined together in this call (batches and
                                    batched server jobs; 1 = one graph)                 */
    int32_t select_lanes;        /* lanes per node of the selection kernel (0: scalar)  */
    int32_t propose_lanes;       /* lanes per node of the proposal kernel (0: scalar)   */
    int32_t sparse_table;        /* 1: the rounds ran on the sparse gain table            */
    int32_t rebalance_graphs;    /* rounds whose rebalancing loop ran as one graph launch */
    int32_t constrained_rounds;  /* constrained rounds (schedules 1-6)                   */
    int32_t lp_rounds;           /* label propagation rounds kept (Sec. 5)               */
    int32_t lp_table_builds;     /* full gain-table builds of label propagation (also in
                                    gain_table_builds)                                  */
    int64_t seq_degree_sum;      /* sum over rounds of the degrees of the nodes of the
                                    move sequence I (the adjacency its exact gains read)  */
    int64_t bytes_algorithmic;   /* the rounds' algorithmic DRAM bytes: every full table
                                    build, per round one read of the table (dense n*k*4
                                    or the hashed rows' slots * 8) and 16 bytes per node,
                                    16 bytes per adjacency entry of a node of I, 48
                                    bytes per candidate, move and rebalancing move       */
} upr_stats;

/* Fills *p with the defaults documented in upr_params. */
void upr_params_default(upr_params *p);

/* Human-readable name of a status code (static string). */
const char *upr_status_str(upr_status s);

/* Creates a refinement context for graph g, k blocks (2 <= k <= 4096) and
 * imbalance eps > 0 (L_max = floor((1 + eps) * ceil(c(V)/k)) with eps rounded
 * to parts per million; Sec. 2).  Copies the graph to the device (the caller
 * may free it on return), computes omega(I(v)) and allocates all workspace
 * for later calls, so upr_refine allocates nothing.  params may be NULL.
 * Errors: UPR_ERR_INVALID (bad sizes, k, eps, params, or with validate=1 a
 * graph that is not a symmetric positive-weight CSR without self loops, or
 * weights so large that omega(I(v)) >= 2^31 or the exact rebalancing key
 * would exceed 63 bits); UPR_ERR_OOM; UPR_ERR_CUDA. */
upr_status upr_create(const upr_graph *g, int32_t k, double eps, const upr_params *params,
                      upr_ctx **out);

/* Refines part (n entries, host or device, values in [0, k)) in place with
 * `rounds` rounds (the tau schedule of Sec. 4.4 runs over rounds
 * round_offset+1 .. round_offset+rounds of total_rounds).  An imbalanced
 * input is first rebalanced (round 0: Sec. 6 rebalancing and best balanced
 * prefix).  The cut never increases.  seed is recorded only: results depend
 * on (graph, k, eps, part, rounds, params) alone.  part is written only on
 * UPR_OK.  Errors: UPR_ERR_INVALID (part out of range, rounds < 0, schedule
 * out of range), UPR_ERR_INFEASIBLE (imbalanced input that cannot be
 * rebalanced), UPR_ERR_CUDA. */
upr_status upr_refine(upr_ctx *ctx, int32_t *part, int32_t rounds, uint64_t seed, upr_stats *stats);

/* Exact cut and block weights (Sec. 2) of part (host or device, n entries).
 * *cut receives sum of omega over cut edges; block_weights (k entries, host,
 * may be NULL) receives c(V_b). Errors: UPR_ERR_INVALID (also for a batch
 * context: see upr_batch_cut), UPR_ERR_CUDA. */
upr_status upr_cut(upr_ctx *ctx, const int32_t *part, int64_t *cut, int64_t *block_weights);

/* Releases the context and all its device memory. NULL is ignored. */
void upr_destroy(upr_ctx *ctx);

/* Cut and block weights of part, like upr_cut, for callers that cannot
 * allocate: code whose device memory is owned by another allocator or
 * budget (a host framework's pool, a fixed-footprint embedded deployment),
 * or latency-critical loops that must not pay the implicit device
 * synchronisation and locking of cudaMalloc / cudaFree.  The paper has no
 * counterpart; it is an operational variant of step (e).
 * It allocates nothing: no context, no cudaMalloc / cudaFree, no allocating
 * library call.  The graph arrays of g and part must be device memory (the
 * caller's); cut (one int64) and block_weights (k int64, may be NULL) may be
 * host or device memory.  The kernels' scratch is one static device array of
 * 4096 + 8 int64 that every GPU loading the library holds until exit, so
 * k must be in [2, 4096] (UPR_ERR_INVALID otherwise).  Every call looks up
 * that array's device address (cudaGetSymbolAddress, which allocates
 * nothing); the first call on a device may load the library's device code,
 * so make it before any stream capture.  Every call on a device shares the
 * one array and clears what it accumulates into, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The call runs on `stream` (cudaStream_t, NULL =
 * default) and returns after synchronising it.  Before any kernel indexes
 * with them it checks, on the device, that part is in [0, k), that xadj[0] =
 * 0, xadj[n] = m and xadj is non-decreasing, and that every neighbour id is
 * in [0, n).  Errors: UPR_ERR_INVALID (sizes, k, pointers that are not
 * device memory of the current device, a failed check above), UPR_ERR_CUDA.
 * Symmetry, self loops and weights are not checked (see upr_create's
 * validate). */
upr_status upr_cut_noalloc(const upr_graph *g, int32_t k, const int32_t *part, void *stream, int64_t *cut,
                           int64_t *block_weights);

/* ------------------------------------------------------------------------
 * Batches: many independent graphs refined together.  The paper refines one
 * graph; a batch runs the same synchronous rounds (Alg. 1, Sec. 4-6) on the
 * disjoint union of its graphs with every step kept per graph: graph g owns
 * its own k blocks and L_max, its candidates, penalties, rebalancing and move
 * sequence involve its blocks only, and its best prefix (Sec. 4.1) is taken
 * over its own moves.  So every graph's result equals upr_refine on that
 * graph alone, while one launch of each step covers all graphs.
 * ------------------------------------------------------------------------ */

/* Creates one context for n_graphs graphs, all with k blocks (2 <= k <=
 * 4096); eps[i] is graph i's imbalance.  The graphs are packed into one
 * device CSR in order (graph i's nodes follow graph i-1's); each graph's
 * arrays are read as in upr_create (host or device, local node ids) and may
 * be freed on return.  Sums of n and of m must stay below 2^31 and
 * n_graphs * k below 2^30.  Errors as upr_create (a graph with an invalid
 * CSR makes the whole call fail). */
upr_status upr_batch_create(const upr_graph *graphs, int32_t n_graphs, int32_t k, const double *eps,
                            const upr_params *params, upr_ctx **out);

/* Creates one context for n_graphs graphs whose block counts may differ:
 * k[i] (2 <= k[i] <= 4096) is graph i's k, eps[i] its imbalance.  A row of
 * the gain table keeps exactly k columns, so the graphs with the same k form
 * one batch (as upr_batch_create) with its own stream, created with params
 * (params.stream is the caller's stream); upr_batch_refine refines the
 * batches concurrently and returns every graph's result in the caller's
 * graph order, each equal to upr_refine on that graph alone.  part holds
 * the graphs' partitions back to back in the caller's order (graph-local
 * block ids), host or device.  upr_batch_cut's block_weights then holds
 * sum(k[i]) entries, graph i's k[i] weights after those of graphs < i;
 * upr_batch_info is as for a batch.  upr_refine, upr_cut and the inspection
 * entry points refuse the context (UPR_ERR_INVALID).  Errors as
 * upr_batch_create. */
upr_status upr_batch_create_mixed(const upr_graph *graphs, int32_t n_graphs, const int32_t *k, const double *eps,
                                  const upr_params *params, upr_ctx **out);

/* Binds other graphs to an existing context, with the parameters it was
 * created with, as upr_create / upr_batch_create / upr_batch_create_mixed
 * would create it, reusing its device memory where it is large enough (a
 * context rebound to graphs no larger than before allocates nothing new on
 * the device).  k and eps have n_graphs entries.  A context of
 * upr_create or upr_batch_create takes graphs of one k (k[i] all equal,
 * else UPR_ERR_INVALID with the context unchanged); a mixed context takes
 * any k (batches of a k it already had are reused, new k get new batches,
 * batches of k no longer present are freed).  The graphs are read as in
 * upr_create and may be freed on return; a batch's arrays in page-locked
 * host memory are read in place by one gather launch per array kind.  A
 * rebinding whose sizes, schedules, key widths, limits and device memory
 * all equal the previous binding's (the same graph, or another of the same
 * shape) keeps the graphs captured for it, so the next call does not
 * capture again.  Any other error leaves the context unusable (every call
 * returns UPR_ERR_INVALID) until a rebind succeeds. */
upr_status upr_batch_rebind(upr_ctx *ctx, const upr_graph *graphs, int32_t n_graphs, const int32_t *k,
                            const double *eps);

/* Refines all graphs of a batch context.  part holds every graph's
 * partition back to back (graph i at node offset sum of n of graphs < i,
 * graph-local block ids in [0, k)), host or device, refined in place.
 * status, cut_in and cut_out (n_graphs entries each, host, may be NULL)
 * receive per graph: UPR_OK or UPR_ERR_INFEASIBLE (an imbalanced input that
 * cannot be rebalanced: that graph's partition and cut stay as given), the
 * cut before and after.  stats sums over graphs.  Returns UPR_OK unless the
 * call itself fails (UPR_ERR_INVALID: a block id out of range, rounds < 0;
 * UPR_ERR_CUDA).  Also accepts a one-graph context. */
upr_status upr_batch_refine(upr_ctx *ctx, int32_t *part, int32_t rounds, uint64_t seed, upr_status *status,
                            int64_t *cut_in, int64_t *cut_out, upr_stats *stats);

/* Per-graph cut (n_graphs entries) and block weights (n_graphs * k entries,
 * graph-major, may be NULL) of a packed partition as in upr_batch_refine. */
upr_status upr_batch_cut(upr_ctx *ctx, const int32_t *part, int64_t *cut, int64_t *block_weights);

/* Number of graphs, node offsets (n_graphs + 1 entries) and L_max of each
 * graph (n_graphs entries); the pointers may be NULL. */
upr_status upr_batch_info(const upr_ctx *ctx, int32_t *n_graphs, int64_t *node_offsets, int64_t *lmax);

/* ------------------------------------------------------------------------
 * Serving with continuous batching.  max_jobs slots, each with its own
 * stream and context, take work from a FIFO queue while device memory
 * allows (a job that does not fit yet may be overtaken by smaller ones).  A
 * slot that takes a small job (n <= batch_max_nodes) also takes every other
 * queued small job with the same k and rounds that fits the budget, up to
 * batch_max_jobs graphs and batch_max_total_nodes nodes, and refines them as
 * one batch (upr_batch_refine); jobs submitted while others run join the
 * next batch a slot takes.  Slots run concurrently, so jobs of different
 * sizes overlap on the device.  Each job's state stays on the device for all
 * its rounds; its result stays in host memory until polled.  Every result is
 * identical to upr_create + upr_refine on the same inputs. */
typedef struct {
    int32_t max_jobs;           /* slots: batches or jobs on the device at once. 8           */
    int32_t queue_capacity;     /* submitted-but-not-admitted jobs before UPR_ERR_BUSY. 4096 */
    int64_t memory_budget;      /* device bytes the server may hold; 0 = 80% of free memory */
    upr_params params;          /* per-job parameters (stream ignored: each slot owns one) */
    int32_t batch_max_jobs;     /* graphs per batch; 1 = no batching. 4096                   */
    int32_t batch_max_nodes;    /* largest graph (nodes) that joins batches. 131072          */
    int64_t batch_max_total_nodes; /* nodes per batch. 2^25                                  */
} upr_server_params;

void upr_server_params_default(upr_server_params *p);

upr_status upr_server_create(const upr_server_params *p, upr_server **out);

/* Queues a job.  The graph and part (host memory) are copied before the call
 * returns.  *ticket identifies the job.  Errors: UPR_ERR_INVALID, UPR_ERR_BUSY,
 * UPR_ERR_OOM. */
upr_status upr_submit(upr_server *s, const upr_graph *g, int32_t k, double eps, const int32_t *part,
                      int32_t rounds, uint64_t seed, uint64_t *ticket);

/* UPR_PENDING while the job runs; on completion writes part_out (n entries,
 * host), *cut_out and stats (each may be NULL), forgets the ticket and returns
 * the job's status.  Errors: UPR_ERR_NOT_FOUND. */
upr_status upr_poll(upr_server *s, uint64_t ticket, int32_t *part_out, int64_t *cut_out,
                    upr_stats *stats);

/* Waits up to timeout_ms for a job (same outputs as upr_poll); UPR_ERR_TIMEOUT
 * if it is still running afterwards. */
upr_status upr_wait(upr_server *s, uint64_t ticket, int64_t timeout_ms, int32_t *part_out,
                    int64_t *cut_out, upr_stats *stats);

/* Stops the worker after finishing admitted jobs and frees everything. */
void upr_server_destroy(upr_server *s);

/* ------------------------------------------------------------------------
 * Inspection entry points used by the parity tests; each runs one step or
 * one round and copies intermediate results to host buffers. */

/* Dense gain table W[v*k + b] = omega(v, V_b) (Sec. 2, Sec. 6.1) of part, and
 * omega(I(v)).  W (n*k int32) and wI (n int64) are host buffers (NULL to skip). */
upr_status upr_debug_gain_table(upr_ctx *ctx, const int32_t *part, int32_t *W, int64_t *wI);

/* Trace of one round (host buffers; any pointer may be NULL).  Capacities:
 * node-indexed arrays n, the pre-merge sequence 2n, I_eligible n+1, bucket
 * k*73 (slot s in column s+32), factor 73. */
typedef struct {
    int8_t  *avail;        int32_t *slot;        int64_t *bucket;      int64_t *factor;
    int32_t *cand_target;  int64_t *cand_s0;     int64_t *cand_gain;   int64_t  n_cand;
    int64_t  n_moves;      int32_t *M_node;      int32_t *M_to;        int64_t *M_score;
    int64_t  n_rebal;      int32_t  subrounds;
    int32_t *R_node;       int32_t *R_from;      int32_t *R_to;        int32_t *R_subround;
    int64_t  n_inter;      int32_t *X_node;      int32_t *X_from;      int32_t *X_to;
    int64_t  n_seq;        int32_t *I_node;      int32_t *I_from;      int32_t *I_to;
    int64_t *I_gain;       int8_t  *I_eligible;
    int64_t  best_len;     int64_t  best_gain;   int64_t  cut_before;  int64_t  cut_after;
} upr_trace;

/* Runs round r of R (rebalance_only = 1: the round-0 repair) on part (host,
 * in/out, written only on UPR_OK) and fills *trace. */
upr_status upr_debug_round(upr_ctx *ctx, int32_t *part, int32_t r, int32_t R, int32_t rebalance_only,
                           upr_trace *trace);

#ifdef __cplusplus
}
#endif
#endif /* UPR_H */
