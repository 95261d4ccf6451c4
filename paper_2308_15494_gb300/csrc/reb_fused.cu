// Step (d), one rebalancing sub-round (Sec. 6.1) in fewer, fused passes, for
// one graph with K <= kFuseMaxK blocks, a one-word priority key and the
// proposal prefilter.  It computes exactly what the general form in
// rebalance.cu computes (the same proposals, the same minimal prefix per
// source, the same longest fitting prefix per target, R in priority order),
// but instead of sorting the kept proposals three times (by key, then by
// source, then by target) it sorts them once by key and finds each
// proposal's weight before it among the proposals of its source (then of its
// target) from per-tile, per-block weight sums:
//   1. compaction of the proposers (in place, node order) fused with the
//      prefilter's (source, bin) weight histogram;
//   2. the prefilter's cut bin per source (rebalance.cu, k_prio_cut);
//   3. the kept proposals as (key, node) pairs, in node order;
//   4. one stable radix sort by key;
//   5. weights per (source, tile) of the sorted list, scanned;
//   6. selection: weight before the proposal in its source = the scanned sum
//      of earlier tiles + the weight of earlier items of the tile with the
//      same source; selected iff that is below the source's excess; weights
//      of the selected per (target, tile), scanned;
//   7. admission in the same way per target (the inclusive weight fits the
//      target's room), compaction of the admitted into R (look-back) and the
//      moves applied; block-weight changes go to a delta array that the
//      sub-round's end folds in, because C is read for admission meanwhile.
#include <type_traits>

#include "prim.cuh"

namespace upr {
namespace {

using namespace prim;

constexpr int kFuseMaxK = 256;
constexpr int kDigits = kFuseMaxK + 1;          // blocks, and one digit for "no item"
constexpr int kHistSlots = 2048;
constexpr uint32_t kHistEmpty = 0xffffffffu;

// The bin of a proposal: the same function as rebalance.cu's prefilter bins.
__device__ __forceinline__ int prio_bin_f(int64_t g, uint64_t c, int cbits) {
    if (g >= 0) {
        const uint64_t v = (uint64_t)g * c;
        return 127 - (int)(v < 127ull ? v : 127ull);
    }
    const uint64_t r = (((uint64_t)(-g)) << cbits) / c;
    return 128 + (int)(r < 127ull ? r : 127ull);
}

// The one-word priority key (ascending = higher priority first): class 0
// (g >= 0) (2^(gb+cb) - 1) - g*c, class 1 (g < 0) 2^(gb+2cb) + floor(|g|
// 2^(2cb) / c); the same function as rebalance.cu's prio_key.
__device__ __forceinline__ uint64_t prio_key_f(int64_t g, uint64_t c, int gbits, int cbits) {
    const int S = 2 * cbits;
    if (g >= 0) return ((1ull << (gbits + cbits)) - 1ull) - (uint64_t)g * c;
    const uint64_t num = ((uint64_t)(-g)) << S;
    return (1ull << (gbits + S)) | (c == 1 ? num : num / c);
}

// Weighted ranks inside a tile: before[r] = the weight of the earlier items
// of the tile (item (r, t) precedes (r', t') iff r < r' or r == r' and
// t < t') with the same digit; digit K = no item.  s_cnt: [2][kWarps][K+1]
// and s_run: [K+1], zero on entry, zero again on return.
template <bool UNIT, int N = kItems>
__device__ __forceinline__ void tile_wprefix(const int (&dig)[N], const int64_t (&w)[N], int64_t (&before)[N],
                                             int64_t *s_cnt, int64_t *s_run, int K) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int stride = kWarps * (K + 1);
#pragma unroll
    for (int r = 0; r < N; r++) {
        int64_t *cnt = s_cnt + (r & 1) * stride;
        const int d = dig[r];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int64_t within;
        if (UNIT) {
            within = __popc(peers & lt);
            if ((peers & lt) == 0) cnt[warp * (K + 1) + d] = __popc(peers);
        } else {
            within = 0;
            for (int j = 0; j < 32; j++) {
                const int dj = __shfl_sync(0xffffffffu, d, j);
                const int64_t wj = __shfl_sync(0xffffffffu, w[r], j);
                if (j < lane && dj == d) within += wj;
            }
            if (lane == 31 - __clz(peers)) cnt[warp * (K + 1) + d] = within + w[r];     // last of the group
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd <= K; dd += kThreads) {
            int64_t run = s_run[dd];
            for (int q = 0; q < kWarps; q++) {
                const int64_t c = cnt[q * (K + 1) + dd];
                cnt[q * (K + 1) + dd] = run;
                run += c;
            }
            s_run[dd] = run;
            int64_t *old = s_cnt + ((r + 1) & 1) * stride;     // read by everyone before the barrier above
            for (int q = 0; q < kWarps; q++) old[q * (K + 1) + dd] = 0;
        }
        __syncthreads();
        before[r] = cnt[warp * (K + 1) + d] + within;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < stride; i += kThreads) s_cnt[((N - 1) & 1) * stride + i] = 0;
    for (int dd = threadIdx.x; dd <= K; dd += kThreads) s_run[dd] = 0;
    __syncthreads();
}

// Per-warp accumulation without atomics: the lanes holding the same digit
// form a group (__match_any_sync); the group's first lane adds the group's
// weight to the warp's own slot of that digit.  Items of a tile sorted by
// priority often share their block, so shared-memory atomics would queue on
// one address.  acc: this warp's K slots; valid = false: no item.
template <bool UNIT>
__device__ __forceinline__ void warp_acc(int d, int64_t w, bool valid, int64_t *acc) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : -1);
    int64_t tot;
    if (UNIT) {
        tot = (int64_t)__popc(peers) * w;        // the group's items share w (+1 or -1)
    } else {
        tot = 0;
        for (unsigned m = peers; m; m &= m - 1) tot += __shfl_sync(peers, w, __ffs(m) - 1);
    }
    if (valid && lane == __ffs(peers) - 1) acc[d] += tot;
}

// Sum of the warps' slots of digit i (threads i < K), then the slots cleared.
__device__ __forceinline__ int64_t warps_total(int64_t *s_acc, int K, int i) {
    int64_t t = 0;
    for (int q = 0; q < kWarps; q++) {
        t += s_acc[q * K + i];
        s_acc[q * K + i] = 0;
    }
    return t;
}

// ---- 1. proposers compacted in place (node order) + prefilter histogram
__global__ void __launch_bounds__(kThreads) k_fr_compact_hist(const int32_t *__restrict__ flags, int32_t *list,
                                                              const int32_t *__restrict__ d_n, int32_t *__restrict__ d_out,
                                                              int32_t *lgain, const int32_t *__restrict__ vwgt,
                                                              int32_t *lsrc, int gbits, int cbits,
                                                              int gain_only, unsigned long long *__restrict__ hist,
                                                              uint64_t *__restrict__ rep, int32_t *__restrict__ exact,
                                                              int vec, ScanState<int32_t> st) {
    __shared__ int32_t s_warp[kWarps];
    __shared__ int32_t s_excl;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_key[kHistSlots];
    __shared__ unsigned long long s_val[kHistSlots];
    __shared__ uint64_t s_rep[kPrioBins];
    __shared__ int s_has[kPrioBins];
    const int64_t n = *d_n;
    const int64_t tiles = tiles_of(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *exact = 1;                              // until k_fr_keep_keys finds a bin holding two keys
        if (tiles == 0) *d_out = 0;
    }
    const unsigned parts = participants(tiles);
    if (blockIdx.x >= parts) return;
    for (int i = threadIdx.x; i < kHistSlots; i += kThreads) { s_key[i] = kHistEmpty; s_val[i] = 0; }
    for (int i = threadIdx.x; i < kPrioBins; i += kThreads) s_has[i] = 0;
    __syncthreads();
    const bool alone = tiles == 1;
    const uint32_t epoch = alone ? 0u : call_epoch(st);
    for (;;) {
        const int64_t tile = alone ? (int64_t)blockIdx.x : next_tile(st.ctr, &s_tile);
        if (tile >= tiles) break;
        int32_t x[kItems], y[kItems], ya[kItems], yg[kItems];
        load_items(flags, tile * kTile, n, (vec & 1) != 0, x);
        load_items((const int32_t *)list, tile * kTile, n, (vec & 2) != 0, y);
        load_items((const int32_t *)lsrc, tile * kTile, n, (vec & 2) != 0, ya);
        load_items((const int32_t *)lgain, tile * kTile, n, (vec & 2) != 0, yg);
        int32_t c = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) c += x[j] != 0;
        int32_t total;
        const int32_t pre = block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x < 32) {
            const int32_t e = alone ? 0 : lookback<OpSum>(st, tile, total, epoch);
            if (threadIdx.x == 0) {
                s_excl = e;
                if (tile == tiles - 1) *d_out = e + total;
            }
        }
        __syncthreads();
        int32_t pos = s_excl + pre;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            uint32_t key = kHistEmpty;
            uint64_t cu = 0;
            if (x[j]) {
                const int32_t u = y[j];
                list[pos] = u;
                lsrc[pos] = ya[j];
                lgain[pos] = yg[j];
                pos++;
                cu = vwgt ? (uint64_t)vwgt[u] : 1ull;
                const int64_t gu = yg[j];
                const int bin = prio_bin_f(gu, gain_only ? 1ull : cu, cbits);
                // some proposal's key per bin (any one: plain stores race, one
                // wins), in shared memory first: one global store per bin and CTA
                s_rep[bin] = prio_key_f(gu, gain_only ? 1ull : cu, gbits, cbits);
                s_has[bin] = 1;
                key = (uint32_t)ya[j] * kPrioBins + bin;
            }
            // the lanes holding the same (source, bin) add their weights
            // first, so that one lane per group updates the table (many
            // proposals share their source and bin)
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            unsigned long long tot;
            if (vwgt) {
                tot = 0;
                for (unsigned mm = peers; mm; mm &= mm - 1) tot += __shfl_sync(peers, cu, __ffs(mm) - 1);
            } else {
                tot = (unsigned long long)__popc(peers);
            }
            if (key == kHistEmpty || lane != __ffs(peers) - 1) continue;
            uint32_t h = (key * 0x9E3779B1u) >> 21;          // 11 bits: kHistSlots
            bool done = false;
            for (int probe = 0; probe < 32 && !done; probe++) {
                uint32_t cur = s_key[h];
                if (cur == kHistEmpty) {
                    cur = atomicCAS(&s_key[h], kHistEmpty, key);
                    if (cur == kHistEmpty) cur = key;
                }
                if (cur == key) {
                    atomicAdd(&s_val[h], tot);
                    done = true;
                }
                h = (h + 1) & (kHistSlots - 1);
            }
            if (!done) atomicAdd(&hist[key], tot);   // crowded table: straight to the histogram
        }
        __syncthreads();
        if (alone) break;
    }
    if (!alone) finish_tiles(st, parts, epoch);
    __syncthreads();
    for (int i = threadIdx.x; i < kHistSlots; i += kThreads)
        if (s_key[i] != kHistEmpty) atomicAdd(&hist[s_key[i]], s_val[i]);
    for (int i = threadIdx.x; i < kPrioBins; i += kThreads)
        if (s_has[i]) rep[i] = s_rep[i];
}

// ---- 3. kept proposals (bin not after their source's cut) as (key, node)
__global__ void __launch_bounds__(kThreads) k_fr_keep_keys(const int32_t *__restrict__ list, const int32_t *__restrict__ d_n,
                                                           const int32_t *__restrict__ lgain,
                                                           const int32_t *__restrict__ vwgt,
                                                           const int32_t *__restrict__ lsrc,
                                                           const int32_t *__restrict__ cut, int gbits, int cbits,
                                                           int gain_only, uint64_t *__restrict__ keys,
                                                           uint32_t *__restrict__ vals, int32_t *__restrict__ d_out,
                                                           const uint64_t *__restrict__ rep,
                                                           int32_t *__restrict__ exact, ScanState<int32_t> st) {
    __shared__ int32_t s_warp[kWarps];
    __shared__ int32_t s_excl;
    __shared__ uint32_t s_tile;
    const int64_t n = *d_n;
    const int64_t tiles = tiles_of(n);
    if (tiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) *d_out = 0;
    const unsigned parts = participants(tiles);
    if (blockIdx.x >= parts) return;
    const bool alone = tiles == 1;
    const uint32_t epoch = alone ? 0u : call_epoch(st);
    for (;;) {
        const int64_t tile = alone ? (int64_t)blockIdx.x : next_tile(st.ctr, &s_tile);
        if (tile >= tiles) break;
        const int64_t first = tile * kTile + (int64_t)threadIdx.x * kItems;
        uint64_t key[kItems];
        int32_t u[kItems];
        int32_t c = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            u[j] = -1;
            if (first + j < n) {
                const int32_t v = list[first + j];
                const uint64_t cv = (vwgt && !gain_only) ? (uint64_t)vwgt[v] : 1ull;
                const int64_t g = lgain[first + j];
                const int bin = prio_bin_f(g, cv, cbits);
                if (bin <= cut[lsrc[first + j]]) {
                    u[j] = v;
                    key[j] = prio_key_f(g, cv, gbits, cbits);
                    if (key[j] != rep[bin]) *exact = 0;
                    c++;
                }
            }
        }
        int32_t total;
        const int32_t pre = block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x < 32) {
            const int32_t e = alone ? 0 : lookback<OpSum>(st, tile, total, epoch);
            if (threadIdx.x == 0) {
                s_excl = e;
                if (tile == tiles - 1) *d_out = e + total;
            }
        }
        __syncthreads();
        int32_t pos = s_excl + pre;
#pragma unroll
        for (int j = 0; j < kItems; j++)
            if (u[j] >= 0) { keys[pos] = key[j]; vals[pos] = (uint32_t)u[j]; pos++; }
        __syncthreads();
        if (alone) break;
    }
    if (!alone) finish_tiles(st, parts, epoch);
}

// ---- 4. the stable sort of the kept proposals by key.  The bin of a key is
// non-decreasing in the key; when every bin holds one key value (the flag
// `exact`, e.g. unit weights with small gains), sorting by the bin alone gives
// the key order, so pass 0 sorts by the bin and the later passes do nothing.
// With an odd number of passes the result lands in the same buffer either way.
__device__ __forceinline__ int bin_of_key(uint64_t key, int gbits, int cbits) {
    const uint64_t top = 1ull << (gbits + 2 * cbits);
    if (key < top) {
        const uint64_t v = ((1ull << (gbits + cbits)) - 1ull) - key;     // g * c
        return 127 - (int)(v < 127ull ? v : 127ull);
    }
    const uint64_t r = (key - top) >> cbits;                            // floor(|g| 2^cb / c)
    return 128 + (int)(r < 127ull ? r : 127ull);
}

__device__ __forceinline__ int sort_digit(uint64_t key, int pass, bool exact, int gbits, int cbits) {
    return exact ? bin_of_key(key, gbits, cbits) : (int)((key >> (8 * pass)) & 0xFF);
}

__global__ void __launch_bounds__(kThreads) k_fr_radix_hist(const uint64_t *__restrict__ keys,
                                                            const int32_t *__restrict__ d_n, int pass, int gbits,
                                                            int cbits, const int32_t *__restrict__ d_exact,
                                                            int32_t *__restrict__ hist, int32_t *__restrict__ d_hist_n) {
    __shared__ int s_h[kBins];
    const int64_t n = *d_n;
    const bool exact = *d_exact != 0;
    const bool skip = n <= kTile || (exact && pass > 0);
    const int64_t T = tiles_of(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_hist_n = skip ? 0 : (int32_t)(kBins * T);
    if (skip) return;
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        for (int i = threadIdx.x; i < kBins; i += kThreads) s_h[i] = 0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = tile * kTile + r * kThreads + threadIdx.x;
            if (g < n) atomicAdd(&s_h[sort_digit(keys[g], pass, exact, gbits, cbits)], 1);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kBins; i += kThreads) hist[(int64_t)i * T + tile] = s_h[i];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_fr_radix_scatter(const uint64_t *__restrict__ keys,
                                                               const uint32_t *__restrict__ vals,
                                                               uint64_t *__restrict__ okeys, uint32_t *__restrict__ ovals,
                                                               const int32_t *__restrict__ d_n, int pass, int gbits,
                                                               int cbits, const int32_t *__restrict__ d_exact,
                                                               const int32_t *__restrict__ offs,
                                                               cudaGraphConditionalHandle later,
                                                               int32_t *__restrict__ later_runs) {
    __shared__ int s_cnt[2 * kWarps * (kBins + 1)];
    __shared__ int s_run[kBins + 1];
    __shared__ int s_off[kBins];
    const int64_t n = *d_n;
    const bool exact = *d_exact != 0;
    if (later_runs && blockIdx.x == 0 && threadIdx.x == 0) {
        // captured form: the later passes are the body of a conditional node,
        // run only when they sort anything
        const bool run = n > kTile && !exact;
        cudaGraphSetConditional(later, run ? 1u : 0u);
        if (run) *later_runs += 1;
    }
    if (n <= kTile || (exact && pass > 0)) return;
    const int64_t T = tiles_of(n);
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
        for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
        for (int i = threadIdx.x; i < kBins; i += kThreads) s_off[i] = offs[(int64_t)i * T + tile];
        __syncthreads();
        uint64_t k[kItems];
        uint32_t v[kItems];
        int dig[kItems], rank[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = tile * kTile + r * kThreads + threadIdx.x;
            if (g < n) { k[r] = keys[g]; v[r] = vals[g]; dig[r] = sort_digit(k[r], pass, exact, gbits, cbits); }
            else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
        }
        tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
        for (int r = 0; r < kItems; r++)
            if (dig[r] < kBins) {
                const int64_t p = (int64_t)s_off[dig[r]] + rank[r];
                okeys[p] = k[r];
                ovals[p] = v[r];
            }
        __syncthreads();
    }
}

// A list of at most one tile: every pass in one CTA (one pass by the bin when exact).
__global__ void __launch_bounds__(kThreads) k_fr_radix_small(const uint64_t *__restrict__ keys,
                                                             const uint32_t *__restrict__ vals, uint64_t *okeys,
                                                             uint32_t *ovals, const int32_t *__restrict__ d_n,
                                                             int passes, int gbits, int cbits,
                                                             const int32_t *__restrict__ d_exact) {
    __shared__ int s_cnt[2 * kWarps * (kBins + 1)];
    __shared__ int s_run[kBins + 1];
    __shared__ int s_off[kBins];
    __shared__ int s_warp[kWarps];
    __shared__ uint64_t s_k[kTile];
    __shared__ uint32_t s_v[kTile];
    const int64_t n64 = *d_n;
    if (n64 > kTile || n64 <= 0) return;
    const int n = (int)n64;
    const bool exact = *d_exact != 0;
    for (int i = threadIdx.x; i < n; i += kThreads) { s_k[i] = keys[i]; s_v[i] = vals[i]; }
    for (int p = 0; p < (exact ? 1 : passes); p++) {
        for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
        for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
        for (int i = threadIdx.x; i < kBins; i += kThreads) s_off[i] = 0;
        __syncthreads();
        uint64_t k[kItems];
        uint32_t v[kItems];
        int dig[kItems], rank[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int g = r * kThreads + threadIdx.x;
            if (g < n) {
                k[r] = s_k[g]; v[r] = s_v[g];
                dig[r] = sort_digit(k[r], p, exact, gbits, cbits);
                atomicAdd(&s_off[dig[r]], 1);
            } else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
        }
        __syncthreads();
        const int c = threadIdx.x < kBins ? s_off[threadIdx.x] : 0;
        int total;
        const int ex = block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x < kBins) s_off[threadIdx.x] = ex;
        __syncthreads();
        tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
        for (int r = 0; r < kItems; r++)
            if (dig[r] < kBins) { const int q = s_off[dig[r]] + rank[r]; s_k[q] = k[r]; s_v[q] = v[r]; }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += kThreads) { okeys[i] = s_k[i]; ovals[i] = s_v[i]; }
}

// Item (r, t) of a tile: index base + r * kThreads + t (the radix order).
__device__ __forceinline__ int64_t item_at(int64_t tile, int r) { return tile * kTile + r * kThreads + threadIdx.x; }

// ---- 5. weight of the sorted proposals per (source, tile), block-major
template <bool UNIT>
__global__ void __launch_bounds__(kThreads) k_fr_src_hist(const uint32_t *__restrict__ U, const int32_t *__restrict__ d_n,
                                                          const int32_t *__restrict__ part,
                                                          const int32_t *__restrict__ vwgt, int K,
                                                          long long *__restrict__ hw, int32_t *__restrict__ d_hist_n) {
    __shared__ int64_t s_acc[kWarps * kFuseMaxK];
    const int64_t n = *d_n;
    const int64_t T = tiles_of(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_hist_n = (int32_t)(K * T);
    int64_t *acc = s_acc + (threadIdx.x >> 5) * K;
    for (int i = threadIdx.x; i < kWarps * K; i += kThreads) s_acc[i] = 0;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = item_at(tile, r);
            const bool ok = g < n;
            const uint32_t u = ok ? U[g] : 0;
            warp_acc<UNIT>(ok ? part[u] : 0, (ok && vwgt) ? vwgt[u] : 1, ok, acc);
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += kThreads) hw[(int64_t)i * T + tile] = warps_total(s_acc, K, i);
        __syncthreads();
    }
}

// ---- 6. selection per source; weights of the selected per (target, tile)
template <bool UNIT>
__global__ void __launch_bounds__(kThreads) k_fr_select(const uint32_t *__restrict__ U, const int32_t *__restrict__ d_n,
                                                        const int32_t *__restrict__ part,
                                                        const int32_t *__restrict__ vwgt,
                                                        const int32_t *__restrict__ prop_tgt, int K,
                                                        const int64_t *__restrict__ C, const int64_t *__restrict__ Lb,
                                                        const long long *__restrict__ hw_ex, int8_t *__restrict__ sel,
                                                        long long *__restrict__ ht, int32_t *__restrict__ d_hist_n) {
    // the warps' accumulators share the ranks' counters: tile_wprefix leaves
    // them zero, warps_total leaves them zero again
    __shared__ int64_t s_cnt[2 * kWarps * kDigits];
    __shared__ int64_t s_run[kDigits];
    int64_t *s_acc = s_cnt;
    const int64_t n = *d_n;
    const int64_t T = tiles_of(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_hist_n = (int32_t)(K * T);
    for (int i = threadIdx.x; i < 2 * kWarps * (K + 1); i += kThreads) s_cnt[i] = 0;
    for (int i = threadIdx.x; i <= K; i += kThreads) s_run[i] = 0;
    int64_t *acc = s_acc + (threadIdx.x >> 5) * K;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        int dig[kItems];
        int64_t w[kItems], before[kItems];
        uint32_t u[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = item_at(tile, r);
            if (g < n) {
                u[r] = U[g];
                dig[r] = part[u[r]];
                w[r] = vwgt ? vwgt[u[r]] : 1;
            } else {
                u[r] = 0;
                dig[r] = K;
                w[r] = 0;
            }
        }
        tile_wprefix<UNIT>(dig, w, before, s_cnt, s_run, K);
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = item_at(tile, r);
            bool s = false;
            if (g < n) {
                const int a = dig[r];
                const int64_t prior = hw_ex[(int64_t)a * T + tile] - hw_ex[(int64_t)a * T] + before[r];
                s = prior < C[a] - Lb[a];
                sel[g] = s ? 1 : 0;
            }
            warp_acc<UNIT>(s ? prop_tgt[u[r]] : 0, w[r], s, acc);
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += kThreads) ht[(int64_t)i * T + tile] = warps_total(s_acc, K, i);
        __syncthreads();
    }
}

// ---- 7. admission per target, compaction of the admitted into R, moves applied
template <bool UNIT>
__global__ void __launch_bounds__(kThreads) k_fr_admit(const uint32_t *__restrict__ U, const int32_t *__restrict__ d_n,
                                                       const int8_t *__restrict__ sel, int32_t *__restrict__ part,
                                                       const int32_t *__restrict__ vwgt,
                                                       const int32_t *__restrict__ prop_tgt, int K,
                                                       const int64_t *__restrict__ C, const int64_t *__restrict__ Lb,
                                                       const long long *__restrict__ ht_ex,
                                                       int8_t *__restrict__ reject, const RebalCtl *__restrict__ ctl,
                                                       int32_t *__restrict__ R_node, int32_t *__restrict__ R_from,
                                                       int32_t *__restrict__ R_to, int32_t *__restrict__ R_sub,
                                                       int32_t *__restrict__ r_to, int32_t *__restrict__ r_at,
                                                       long long *__restrict__ Cd, int32_t *__restrict__ d_out,
                                                       ScanState<int32_t> st) {
    // the warps' accumulators share the ranks' counters (see k_fr_select)
    __shared__ int64_t s_cnt[2 * kWarps * kDigits];
    __shared__ int64_t s_run[kDigits];
    int64_t *s_acc = s_cnt;
    __shared__ uint64_t s_w64[kWarps];
    __shared__ int32_t s_excl;
    __shared__ uint32_t s_tile;
    const int64_t n = *d_n;
    const int64_t T = tiles_of(n);
    if (T == 0 && blockIdx.x == 0 && threadIdx.x == 0) *d_out = 0;
    const unsigned parts = participants(T);
    if (blockIdx.x >= parts) return;
    for (int i = threadIdx.x; i < 2 * kWarps * (K + 1); i += kThreads) s_cnt[i] = 0;
    for (int i = threadIdx.x; i <= K; i += kThreads) s_run[i] = 0;
    int64_t *acc = s_acc + (threadIdx.x >> 5) * K;
    __syncthreads();
    const int64_t off = ctl->nR;
    const int32_t subround = ctl->subrounds;
    const bool alone = T == 1;
    const uint32_t epoch = alone ? 0u : call_epoch(st);
    for (;;) {
        const int64_t tile = alone ? (int64_t)blockIdx.x : next_tile(st.ctr, &s_tile);
        if (tile >= T) break;
        int dig[kItems];
        int64_t w[kItems], before[kItems];
        uint32_t u[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = item_at(tile, r);
            dig[r] = K;
            w[r] = 0;
            u[r] = 0;
            if (g < n) {
                u[r] = U[g];
                if (sel[g]) {
                    dig[r] = prop_tgt[u[r]];
                    w[r] = vwgt ? vwgt[u[r]] : 1;
                }
            }
        }
        tile_wprefix<UNIT>(dig, w, before, s_cnt, s_run, K);
        // admitted: the weight of the target's selected proposals up to this one fits
        bool adm[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            adm[r] = false;
            const int b = dig[r];
            if (b == K) continue;
            const int64_t incl = ht_ex[(int64_t)b * T + tile] - ht_ex[(int64_t)b * T] + before[r] + w[r];
            adm[r] = C[b] + incl <= Lb[b];
            if (!adm[r]) reject[b] = 1;
        }
        // R keeps the sorted (priority) order, which inside a tile is item
        // order (round-major): per-round counts packed 16 bits each into two
        // words, one block scan per word
        uint64_t lo = 0, hi = 0;
#pragma unroll
        for (int r = 0; r < kItems; r++)
            if (adm[r]) {
                if (r < 4) lo += 1ull << (16 * r);
                else hi += 1ull << (16 * (r - 4));
            }
        uint64_t tlo, thi;
        const uint64_t plo = block_exclusive<OpSum>(lo, s_w64, &tlo);
        const uint64_t phi = block_exclusive<OpSum>(hi, s_w64, &thi);
        int32_t total = 0;
#pragma unroll
        for (int r = 0; r < kItems; r++) total += (int32_t)(((r < 4 ? tlo : thi) >> (16 * (r & 3))) & 0xFFFF);
        if (threadIdx.x < 32) {
            const int32_t e = alone ? 0 : lookback<OpSum>(st, tile, total, epoch);
            if (threadIdx.x == 0) {
                s_excl = e;
                if (tile == T - 1) *d_out = e + total;
            }
        }
        __syncthreads();
        int32_t mine[kItems];
        {
            int32_t base = s_excl;
#pragma unroll
            for (int r = 0; r < kItems; r++) {
                const int sh = 16 * (r & 3);
                mine[r] = base + (int32_t)(((r < 4 ? plo : phi) >> sh) & 0xFFFF);
                base += (int32_t)(((r < 4 ? tlo : thi) >> sh) & 0xFFFF);
            }
        }
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            int32_t a = 0;
            const int32_t b = dig[r];
            if (adm[r]) {
                const int32_t v = (int32_t)u[r];
                a = part[v];
                const int64_t p = off + mine[r];
                R_node[p] = v;
                R_from[p] = a;
                R_to[p] = b;
                R_sub[p] = subround;
                r_to[v] = b;
                r_at[v] = (int32_t)p;
                part[v] = b;
            }
            warp_acc<UNIT>(a, -w[r], adm[r], acc);
            __syncwarp();
            warp_acc<UNIT>(b, w[r], adm[r], acc);
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += kThreads) {
            const int64_t d = warps_total(s_acc, K, i);
            if (d) atomicAdd(reinterpret_cast<unsigned long long *>(&Cd[i]), (unsigned long long)d);
        }
        __syncthreads();
        if (alone) break;
    }
    if (!alone) finish_tiles(st, parts, epoch);
}

// ---- end of the sub-round: the block-weight changes folded in, then the
// targets that rejected a move excluded; stop when nothing was admitted and
// no target was newly excluded, or when no block is overloaded any more.
// In a graph-resident loop (cond != 0) it also sets the loop's condition:
// another sub-round while the loop has not stopped and sub-rounds are left.
__global__ void k_fr_end(int64_t *__restrict__ C, long long *__restrict__ Cd, const int64_t *__restrict__ Lb, int32_t K,
                         int8_t *__restrict__ excl, int8_t *reject, const int32_t *__restrict__ d_na,
                         RebalCtl *__restrict__ ctl, cudaGraphConditionalHandle cond, int32_t max_subrounds,
                         int8_t *__restrict__ over, const int32_t *__restrict__ d_n1) {
    __shared__ int s_grew, s_over;
    if (threadIdx.x == 0) s_grew = 0, s_over = 0;
    __syncthreads();
    const bool active = ctl->active != 0;
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
        const int64_t c = C[b] + Cd[b];
        C[b] = c;
        Cd[b] = 0;
        if (!active) continue;
        if (reject[b] && !excl[b]) { excl[b] = 1; s_grew = 1; }
        if (c > Lb[b]) s_over = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && active) {
        const int32_t na = *d_na;
        ctl->nR += na;
        if ((na == 0 && !s_grew) || !s_over) ctl->stopped = 1;
    }
    if (!over) {
        if (threadIdx.x == 0 && cond)
            cudaGraphSetConditional(cond, (!ctl->stopped && ctl->subrounds < max_subrounds) ? 1u : 0u);
        return;
    }
    // the next sub-round's begin (k_reb_begin's steps) on the updated weights
    // and exclusions: overloaded set, lightest allowed block, activity
    __shared__ int s_any;
    __shared__ long long s_w[256];
    __shared__ int s_b[256];
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    long long bw = 0;
    int bb = -1;
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
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
        if (cond) cudaGraphSetConditional(cond, run ? 1u : 0u);
    }
}


// ---- steps 1 and 3-7 of the sub-round in one cooperative launch.  The
// same tiles and the same per-tile code as the kernels above; the prefix of
// a tile over the tiles before it comes from per-tile totals read after a
// grid barrier instead of the look-back, and the per-(block, tile) weight
// sums are scanned row by row (one row per CTA).  Every CTA passes every
// barrier (no early return), and every wait is bounded: a wait that gives up
// sets the error word and the launch runs to its end.

// Grid barrier on a 64-bit arrival counter that only grows: the barrier that
// a CTA reaches with arrival number `old` ends when the count reaches the
// next multiple of the grid size.
__device__ __forceinline__ void grid_sync(unsigned long long *count, int32_t *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long old = atomicAdd(count, 1ull);
        const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
        for (int it = 0;; it++) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (it >= kMaxSpin || ((it & 1023) == 1023 && gave_up(err))) { atomicOr(err, 2); break; }
            if (it >= 16) __nanosleep(32);
        }
    }
    __syncthreads();
}

// Sum of tc[0..t) (all threads get it).
__device__ __forceinline__ int32_t tiles_before(const int32_t *tc, int64_t t, int32_t *s_warp) {
    int32_t v = 0;
    for (int64_t i = threadIdx.x; i < t; i += kThreads) v += tc[i];
    int32_t total;
    block_exclusive<OpSum>(v, s_warp, &total);
    return total;
}

// Row-wise exclusive scan in place: row[0..T) becomes the sum of the entries
// before each one; returns the row's total (all threads).
template <typename T>
__device__ __forceinline__ T scan_row(T *row, int64_t len, T *s_warp) {
    T carry = 0;
    for (int64_t base = 0; base < len; base += kTile) {
        T x[kItems];
        load_items(row, base, len, false, x);
        T c = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) c += x[j];
        T total;
        const T pre = block_exclusive<OpSum>(c, s_warp, &total);
        T run = carry + pre;
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const T v = x[j];
            x[j] = run;
            run += v;
        }
        store_items(row, base, len, false, x);
        carry += total;
    }
    return carry;
}

using MegaArgs = RebalMega;

constexpr int kMegaSmem = 43136;
constexpr int kMI = 4;                       // items per thread in steps 5-7
constexpr int kMT = kThreads * kMI;          // their tiles: 1024 sorted proposals
constexpr uint64_t kNoKey = ~0ull;           // (keys have at most 63 bits)

__device__ __forceinline__ int64_t item_m(int64_t tile, int r) { return tile * kMT + r * kThreads + threadIdx.x; }
__device__ __forceinline__ int64_t tiles_m(int64_t n) { return (n + kMT - 1) / kMT; }

// The proposal at index i of the compacted proposers: kept (its bin not after
// its source's cut), with its key and node; the list takes the node.
__device__ __forceinline__ bool kept_key(const MegaArgs &a, int64_t i, bool copy, uint64_t *key, int32_t *node) {
    const int32_t v = a.list2[i];
    if (copy) a.list[i] = v;
    const uint64_t cv = (a.vwgt && !a.gain_only) ? (uint64_t)a.vwgt[v] : 1ull;
    const int64_t g = a.lgain2[i];
    const int bin = prio_bin_f(g, cv, a.cbits);
    *node = v;
    if (bin > a.cut[a.lsrc2[i]]) return false;
    *key = prio_key_f(g, cv, a.gbits, a.cbits);
    return true;
}

// Sort passes [p0, p1) of n <= kTile (key, node) pairs held in shared memory
// (one CTA; the radix order of the kernels above).
__device__ __forceinline__ void smem_sort(uint64_t *s_k, uint32_t *s_v, int *s_cnt, int *s_run, int *s_off,
                                          int32_t *s_warp, int n, int p0, int p1, bool exact, int gbits, int cbits) {
    for (int p = p0; p < p1; p++) {
        for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
        for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
        for (int i = threadIdx.x; i < kBins; i += kThreads) s_off[i] = 0;
        __syncthreads();
        uint64_t k[kItems];
        uint32_t v[kItems];
        int dig[kItems], rank[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int g = r * kThreads + threadIdx.x;
            if (g < n) {
                k[r] = s_k[g]; v[r] = s_v[g];
                dig[r] = sort_digit(k[r], p, exact, gbits, cbits);
                atomicAdd(&s_off[dig[r]], 1);
            } else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
        }
        __syncthreads();
        const int c = threadIdx.x < kBins ? s_off[threadIdx.x] : 0;
        int total;
        const int ex = block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x < kBins) s_off[threadIdx.x] = ex;
        __syncthreads();
        tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
        for (int r = 0; r < kItems; r++)
            if (dig[r] < kBins) { const int q = s_off[dig[r]] + rank[r]; s_k[q] = k[r]; s_v[q] = v[r]; }
        __syncthreads();
    }
}

template <bool UNIT>
__global__ void __launch_bounds__(kThreads, 2) k_fr_mega(const MegaArgs a) {
    __shared__ __align__(16) unsigned char s_raw[kMegaSmem];
    __shared__ int32_t s_warp[kWarps];
    __shared__ int64_t s_w64s[kWarps];
    __shared__ uint64_t s_w64[kWarps];
    __shared__ int s_inexact;
    const int64_t P = gridDim.x;
    const int K = a.K;
    int32_t *tc1 = a.tab, *tc2 = tc1 + a.tcap, *tc3 = tc2 + a.tcap;       // tc3: 2 * tcap tiles of kMT
    int32_t *dtot = tc3 + 2 * a.tcap, *tbl = dtot + kBins;                 // (digits: more than one tile only)
    uint64_t *grep = a.rep;

    // ---- 1. proposers compacted (node order) with the prefilter histogram;
    // a key per bin, to learn whether every bin holds one key value
    const int64_t n1 = *a.d_n1;
    const int64_t T1 = tiles_of(n1);
    for (int64_t t = blockIdx.x; t < T1; t += P) {
        int32_t x[kItems];
        load_items(a.flags, t * kTile, n1, (a.vec & 1) != 0, x);
        int32_t c = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) c += x[j] != 0;
        int32_t total;
        block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x == 0) tc1[t] = total;
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < kPrioBins; i += kThreads) grep[i] = kNoKey;
        if (threadIdx.x == 0) *a.exact = 1;
    }
    grid_sync(a.bar, a.err);
    {
        // the (source, bin) weights in a shared-memory hash table: 32-bit
        // values with unit weights (a CTA's proposals fit), 64-bit otherwise
        using HV = typename std::conditional<UNIT, unsigned int, unsigned long long>::type;
        uint32_t *s_key = reinterpret_cast<uint32_t *>(s_raw);
        HV *s_val = reinterpret_cast<HV *>(s_raw + 8192);
        for (int i = threadIdx.x; i < kHistSlots; i += kThreads) { s_key[i] = kHistEmpty; s_val[i] = 0; }
        __syncthreads();
        for (int64_t t = blockIdx.x; t < T1; t += P) {
            const int32_t before = tiles_before(tc1, t, s_warp);
            int32_t x[kItems], y[kItems], ya[kItems], yg[kItems];
            load_items(a.flags, t * kTile, n1, (a.vec & 1) != 0, x);
            load_items((const int32_t *)a.list, t * kTile, n1, (a.vec & 2) != 0, y);
            load_items((const int32_t *)a.lsrc, t * kTile, n1, (a.vec & 2) != 0, ya);
            load_items((const int32_t *)a.lgain, t * kTile, n1, (a.vec & 2) != 0, yg);
            int32_t c = 0;
#pragma unroll
            for (int j = 0; j < kItems; j++) c += x[j] != 0;
            int32_t total;
            int32_t pos = before + block_exclusive<OpSum>(c, s_warp, &total);
#pragma unroll
            for (int j = 0; j < kItems; j++) {
                if (!x[j]) continue;
                const int32_t u = y[j];
                a.list2[pos] = u;
                a.lsrc2[pos] = ya[j];
                a.lgain2[pos] = yg[j];
                pos++;
                const uint64_t cu = a.vwgt ? (uint64_t)a.vwgt[u] : 1ull;
                const int64_t gu = yg[j];
                const int bin = prio_bin_f(gu, a.gain_only ? 1ull : cu, a.cbits);
                const uint32_t key = (uint32_t)ya[j] * kPrioBins + bin;
                const HV tot = (HV)cu;
                uint32_t h = (key * 0x9E3779B1u) >> 21;
                bool done = false;
                for (int probe = 0; probe < 32 && !done; probe++) {
                    uint32_t cur = s_key[h];
                    if (cur == kHistEmpty) {
                        cur = atomicCAS(&s_key[h], kHistEmpty, key);
                        if (cur == kHistEmpty) cur = key;
                    }
                    if (cur == key) {
                        atomicAdd(&s_val[h], tot);
                        done = true;
                    }
                    h = (h + 1) & (kHistSlots - 1);
                }
                if (!done) atomicAdd(&a.hist[key], (unsigned long long)tot);
            }
            __syncthreads();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kHistSlots; i += kThreads)
            if (s_key[i] != kHistEmpty) atomicAdd(&a.hist[s_key[i]], (unsigned long long)s_val[i]);
    }
    grid_sync(a.bar, a.err);
    const int64_t np = tiles_before(tc1, T1, s_warp);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.d_np = (int32_t)np;

    // ---- 2. the prefilter's cut bin per overloaded source (one CTA per source)
    {
        unsigned long long *s_pw = reinterpret_cast<unsigned long long *>(s_raw);
        int *s_cut = reinterpret_cast<int *>(s_raw + 64);
        const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
        for (int64_t src = blockIdx.x; src < K; src += P) {
            if (!a.over[src]) continue;                       // uniform over the CTA
            unsigned long long *row = a.hist + src * kPrioBins;
            const unsigned long long v = row[t];
            unsigned long long inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_pw[warp] = inc;
            if (t == 0) *s_cut = kPrioBins - 1;
            __syncthreads();
            for (int w = 0; w < warp; w++) inc += s_pw[w];
            const unsigned long long excess = (unsigned long long)(a.C[src] - a.Lb[src]);
            if (inc >= excess) atomicMin(s_cut, t);
            row[t] = 0;
            __syncthreads();
            if (t == 0) a.cut[src] = *s_cut;
            __syncthreads();
        }
    }
    grid_sync(a.bar, a.err);

    // ---- 3-4. the kept proposals (node order) sorted stably by key, or by
    // the bin alone when every bin holds one key value; the list becomes the
    // proposers
    const int64_t Tp = tiles_of(np);
    int64_t nk = 0;
    if (Tp <= 1) {
        // one tile of proposals: kept keys and the whole sort in one CTA
        if (blockIdx.x == 0) {
            int *s_cnt = reinterpret_cast<int *>(s_raw);
            int *s_run = reinterpret_cast<int *>(s_raw + 16448);
            int *s_off = reinterpret_cast<int *>(s_raw + 17488);
            uint64_t *s_k = reinterpret_cast<uint64_t *>(s_raw + 18512);
            uint32_t *s_v = reinterpret_cast<uint32_t *>(s_raw + 34896);
            const int64_t first = (int64_t)threadIdx.x * kItems;
            uint64_t key[kItems];
            int32_t u[kItems];
            bool kp[kItems];
            int32_t c = 0;
#pragma unroll
            for (int j = 0; j < kItems; j++) {
                kp[j] = first + j < np && kept_key(a, first + j, true, &key[j], &u[j]);
                c += kp[j];
            }
            int32_t total;
            int32_t pos = block_exclusive<OpSum>(c, s_warp, &total);
#pragma unroll
            for (int j = 0; j < kItems; j++)
                if (kp[j]) { s_k[pos] = key[j]; s_v[pos] = (uint32_t)u[j]; pos++; }
            // whether every bin of the kept keys holds one key value
            uint64_t *s_rep = reinterpret_cast<uint64_t *>(s_raw);      // (free until the sort)
            for (int i = threadIdx.x; i < kPrioBins; i += kThreads) s_rep[i] = kNoKey;
            if (threadIdx.x == 0) s_inexact = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < total; i += kThreads) {
                const uint64_t k = s_k[i];
                const int bin = bin_of_key(k, a.gbits, a.cbits);
                unsigned long long r = atomicCAS(reinterpret_cast<unsigned long long *>(&s_rep[bin]), kNoKey, k);
                if (r != kNoKey && r != k) s_inexact = 1;
            }
            __syncthreads();
            const bool exact = s_inexact == 0;
            if (threadIdx.x == 0) *a.exact = exact ? 1 : 0;
            smem_sort(s_k, s_v, s_cnt, s_run, s_off, s_warp, total, 0, exact ? 1 : a.passes, exact, a.gbits, a.cbits);
            for (int i = threadIdx.x; i < total; i += kThreads) { a.keys_alt[i] = s_k[i]; a.vals_alt[i] = s_v[i]; }
            if (threadIdx.x == 0) tc2[0] = total;
        }
        grid_sync(a.bar, a.err);
        nk = Tp == 1 ? tc2[0] : 0;
    } else {
        // (a) per tile of proposals: the kept ones staged in node order at the
        // tile's start, the counts of both candidates for their first sort
        // digit (the bin, or the key's low byte), and whether every bin of
        // the kept keys holds one key value
        int32_t *tbl_b = reinterpret_cast<int32_t *>(a.h1);       // (free until step 5)
        {
            int *s_h = reinterpret_cast<int *>(s_raw);
            int *s_h2 = s_h + kBins;
            uint64_t *s_rep = reinterpret_cast<uint64_t *>(s_raw + 2048);
            for (int i = threadIdx.x; i < kPrioBins; i += kThreads) s_rep[i] = kNoKey;
            if (threadIdx.x == 0) s_inexact = 0;
            for (int64_t t = blockIdx.x; t < Tp; t += P) {
                for (int i = threadIdx.x; i < kBins; i += kThreads) { s_h[i] = 0; s_h2[i] = 0; }
                __syncthreads();
                const int64_t first = t * kTile + (int64_t)threadIdx.x * kItems;
                uint64_t key[kItems];
                int32_t yv[kItems];
                bool kp[kItems];
                int32_t c = 0;
#pragma unroll
                for (int j = 0; j < kItems; j++) {
                    kp[j] = first + j < np && kept_key(a, first + j, true, &key[j], &yv[j]);
                    c += kp[j];
                }
                int32_t total;
                int32_t pos = block_exclusive<OpSum>(c, s_warp, &total);
#pragma unroll
                for (int j = 0; j < kItems; j++)
                    if (kp[j]) {
                        a.keys[t * kTile + pos] = key[j];
                        a.vals[t * kTile + pos] = (uint32_t)yv[j];
                        pos++;
                        const int bin = bin_of_key(key[j], a.gbits, a.cbits);
                        atomicAdd(&s_h[bin], 1);
                        atomicAdd(&s_h2[(int)(key[j] & 0xFF)], 1);
                        uint64_t r = s_rep[bin];
                        if (r == kNoKey) {
                            r = atomicCAS(reinterpret_cast<unsigned long long *>(&s_rep[bin]), kNoKey, key[j]);
                            if (r == kNoKey) r = key[j];
                        }
                        if (r != key[j]) s_inexact = 1;
                    }
                __syncthreads();
                for (int i = threadIdx.x; i < kBins; i += kThreads) {
                    tbl[(int64_t)i * Tp + t] = s_h[i];
                    tbl_b[(int64_t)i * Tp + t] = s_h2[i];
                }
                if (threadIdx.x == 0) tc2[t] = total;
                __syncthreads();
            }
            bool differs = false;
            for (int i = threadIdx.x; i < kPrioBins; i += kThreads)
                if (s_rep[i] != kNoKey) {
                    const unsigned long long g =
                        atomicCAS(reinterpret_cast<unsigned long long *>(&grep[i]), kNoKey, s_rep[i]);
                    if (g != kNoKey && g != s_rep[i]) differs = true;
                }
            if (differs) s_inexact = 1;
            __syncthreads();
            if (threadIdx.x == 0 && s_inexact) *a.exact = 0;
        }
        grid_sync(a.bar, a.err);
        const bool exact = *(volatile const int32_t *)a.exact != 0;
        const int passes = exact ? 1 : a.passes;
        int32_t *tsel = exact ? tbl : tbl_b;
        for (int64_t d = blockIdx.x; d < kBins; d += P) {
            const int32_t tot = scan_row(tsel + d * Tp, Tp, s_warp);
            if (threadIdx.x == 0) dtot[d] = tot;
        }
        grid_sync(a.bar, a.err);
        // (b) the first pass from the staged tiles into the alternate buffers
        {
            int *s_cnt = reinterpret_cast<int *>(s_raw);
            int *s_run = reinterpret_cast<int *>(s_raw + 16448);
            int *s_off = reinterpret_cast<int *>(s_raw + 17488);
            int *s_base = reinterpret_cast<int *>(s_raw + 18512);
            {
                const int c = dtot[threadIdx.x];       // kThreads == kBins
                int total;
                s_base[threadIdx.x] = block_exclusive<OpSum>(c, s_warp, &total);
            }
            for (int64_t t = blockIdx.x; t < Tp; t += P) {
                const int cnt = tc2[t];
                for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
                for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
                for (int i = threadIdx.x; i < kBins; i += kThreads) s_off[i] = s_base[i] + tsel[(int64_t)i * Tp + t];
                __syncthreads();
                uint64_t k[kItems];
                uint32_t v[kItems];
                int dig[kItems], rank[kItems];
#pragma unroll
                for (int r = 0; r < kItems; r++) {
                    const int j = r * kThreads + threadIdx.x;
                    if (j < cnt) {
                        k[r] = a.keys[t * kTile + j];
                        v[r] = a.vals[t * kTile + j];
                        dig[r] = sort_digit(k[r], 0, exact, a.gbits, a.cbits);
                    } else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
                }
                tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
                for (int r = 0; r < kItems; r++)
                    if (dig[r] < kBins) {
                        const int64_t q = (int64_t)s_off[dig[r]] + rank[r];
                        a.keys_alt[q] = k[r];
                        a.vals_alt[q] = v[r];
                    }
                __syncthreads();
            }
        }
        grid_sync(a.bar, a.err);
        nk = tiles_before(tc2, Tp, s_warp);
        // (c) the other passes (none when exact), alternate -> main -> ... ->
        // alternate (an odd number of passes in all)
        if (passes > 1) {
            if (nk <= kTile) {
                if (blockIdx.x == 0 && nk > 0) {
                    int *s_cnt = reinterpret_cast<int *>(s_raw);
                    int *s_run = reinterpret_cast<int *>(s_raw + 16448);
                    int *s_off = reinterpret_cast<int *>(s_raw + 17488);
                    uint64_t *s_k = reinterpret_cast<uint64_t *>(s_raw + 18512);
                    uint32_t *s_v = reinterpret_cast<uint32_t *>(s_raw + 34896);
                    const int n = (int)nk;
                    for (int i = threadIdx.x; i < n; i += kThreads) { s_k[i] = a.keys_alt[i]; s_v[i] = a.vals_alt[i]; }
                    __syncthreads();
                    smem_sort(s_k, s_v, s_cnt, s_run, s_off, s_warp, n, 1, passes, false, a.gbits, a.cbits);
                    for (int i = threadIdx.x; i < n; i += kThreads) { a.keys_alt[i] = s_k[i]; a.vals_alt[i] = s_v[i]; }
                }
            } else {
                const int64_t Tk = tiles_of(nk);
                uint64_t *ka = a.keys_alt, *kb = a.keys;
                uint32_t *va = a.vals_alt, *vb = a.vals;
                for (int p = 1; p < passes; p++) {
                    {
                        int *s_h = reinterpret_cast<int *>(s_raw);
                        for (int64_t t = blockIdx.x; t < Tk; t += P) {
                            for (int i = threadIdx.x; i < kBins; i += kThreads) s_h[i] = 0;
                            __syncthreads();
#pragma unroll
                            for (int r = 0; r < kItems; r++) {
                                const int64_t g = t * kTile + r * kThreads + threadIdx.x;
                                if (g < nk) atomicAdd(&s_h[sort_digit(ka[g], p, false, a.gbits, a.cbits)], 1);
                            }
                            __syncthreads();
                            for (int i = threadIdx.x; i < kBins; i += kThreads) tbl[(int64_t)i * Tk + t] = s_h[i];
                            __syncthreads();
                        }
                    }
                    grid_sync(a.bar, a.err);
                    for (int64_t d = blockIdx.x; d < kBins; d += P) {
                        const int32_t tot = scan_row(tbl + d * Tk, Tk, s_warp);
                        if (threadIdx.x == 0) dtot[d] = tot;
                    }
                    grid_sync(a.bar, a.err);
                    {
                        int *s_cnt = reinterpret_cast<int *>(s_raw);
                        int *s_run = reinterpret_cast<int *>(s_raw + 16448);
                        int *s_off = reinterpret_cast<int *>(s_raw + 17488);
                        int *s_base = reinterpret_cast<int *>(s_raw + 18512);
                        {
                            const int c = dtot[threadIdx.x];
                            int total;
                            s_base[threadIdx.x] = block_exclusive<OpSum>(c, s_warp, &total);
                        }
                        for (int64_t t = blockIdx.x; t < Tk; t += P) {
                            for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
                            for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
                            for (int i = threadIdx.x; i < kBins; i += kThreads)
                                s_off[i] = s_base[i] + tbl[(int64_t)i * Tk + t];
                            __syncthreads();
                            uint64_t k[kItems];
                            uint32_t v[kItems];
                            int dig[kItems], rank[kItems];
#pragma unroll
                            for (int r = 0; r < kItems; r++) {
                                const int64_t g = t * kTile + r * kThreads + threadIdx.x;
                                if (g < nk) { k[r] = ka[g]; v[r] = va[g]; dig[r] = sort_digit(k[r], p, false, a.gbits, a.cbits); }
                                else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
                            }
                            tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
                            for (int r = 0; r < kItems; r++)
                                if (dig[r] < kBins) {
                                    const int64_t q = (int64_t)s_off[dig[r]] + rank[r];
                                    kb[q] = k[r];
                                    vb[q] = v[r];
                                }
                            __syncthreads();
                        }
                    }
                    grid_sync(a.bar, a.err);
                    uint64_t *tk = ka; ka = kb; kb = tk;
                    uint32_t *tv = va; va = vb; vb = tv;
                }
            }
        }
        grid_sync(a.bar, a.err);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.d_nk = (int32_t)nk;
    const uint32_t *U = a.vals_alt;
    const int64_t T2 = tiles_m(nk);

    // ---- 5. weight of the sorted proposals per (source, tile), row prefixes
    {
        int64_t *s_acc = reinterpret_cast<int64_t *>(s_raw);
        int64_t *acc = s_acc + (threadIdx.x >> 5) * K;
        for (int i = threadIdx.x; i < kWarps * K; i += kThreads) s_acc[i] = 0;
        __syncthreads();
        for (int64_t t = blockIdx.x; t < T2; t += P) {
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                const int64_t g = item_m(t, r);
                const bool ok = g < nk;
                const uint32_t u = ok ? U[g] : 0;
                warp_acc<UNIT>(ok ? a.part[u] : 0, (ok && a.vwgt) ? a.vwgt[u] : 1, ok, acc);
                __syncwarp();
            }
            __syncthreads();
            for (int i = threadIdx.x; i < K; i += kThreads) a.h0[(int64_t)i * T2 + t] = warps_total(s_acc, K, i);
            __syncthreads();
        }
    }
    grid_sync(a.bar, a.err);
    for (int64_t b = blockIdx.x; b < K; b += P) {
        long long *row = a.h0 + b * T2;
        long long *out = a.h1 + b * T2;
        for (int64_t i = threadIdx.x; i < T2; i += kThreads) out[i] = row[i];
        __syncthreads();
        scan_row(out, T2, reinterpret_cast<long long *>(s_w64s));
    }
    grid_sync(a.bar, a.err);

    // ---- 6. selection per source; weights of the selected per (target, tile)
    int64_t *s_cnt = reinterpret_cast<int64_t *>(s_raw);
    int64_t *s_run = reinterpret_cast<int64_t *>(s_raw + 32896);
    {
        for (int i = threadIdx.x; i < 2 * kWarps * (K + 1); i += kThreads) s_cnt[i] = 0;
        for (int i = threadIdx.x; i <= K; i += kThreads) s_run[i] = 0;
        int64_t *acc = s_cnt + (threadIdx.x >> 5) * K;
        __syncthreads();
        for (int64_t t = blockIdx.x; t < T2; t += P) {
            int dig[kMI];
            int64_t w[kMI], before[kMI];
            uint32_t u[kMI];
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                const int64_t g = item_m(t, r);
                if (g < nk) {
                    u[r] = U[g];
                    dig[r] = a.part[u[r]];
                    w[r] = a.vwgt ? a.vwgt[u[r]] : 1;
                } else {
                    u[r] = 0;
                    dig[r] = K;
                    w[r] = 0;
                }
            }
            tile_wprefix<UNIT, kMI>(dig, w, before, s_cnt, s_run, K);
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                const int64_t g = item_m(t, r);
                bool sl = false;
                if (g < nk) {
                    const int src = dig[r];
                    const int64_t prior = a.h1[(int64_t)src * T2 + t] + before[r];
                    sl = prior < a.C[src] - a.Lb[src];
                    a.sel[g] = sl ? 1 : 0;
                }
                warp_acc<UNIT>(sl ? a.prop_tgt[u[r]] : 0, w[r], sl, acc);
                __syncwarp();
            }
            __syncthreads();
            for (int i = threadIdx.x; i < K; i += kThreads) a.h0[(int64_t)i * T2 + t] = warps_total(s_cnt, K, i);
            __syncthreads();
        }
    }
    grid_sync(a.bar, a.err);
    for (int64_t b = blockIdx.x; b < K; b += P) {
        long long *row = a.h0 + b * T2;
        long long *out = a.h1 + b * T2;
        for (int64_t i = threadIdx.x; i < T2; i += kThreads) out[i] = row[i];
        __syncthreads();
        scan_row(out, T2, reinterpret_cast<long long *>(s_w64s));
    }
    grid_sync(a.bar, a.err);

    // ---- 7. admission per target (sel = 2), then R in priority order and the moves applied
    {
        for (int i = threadIdx.x; i < 2 * kWarps * (K + 1); i += kThreads) s_cnt[i] = 0;
        for (int i = threadIdx.x; i <= K; i += kThreads) s_run[i] = 0;
        __syncthreads();
        for (int64_t t = blockIdx.x; t < T2; t += P) {
            int dig[kMI];
            int64_t w[kMI], before[kMI];
            uint32_t u[kMI];
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                const int64_t g = item_m(t, r);
                dig[r] = K;
                w[r] = 0;
                u[r] = 0;
                if (g < nk) {
                    u[r] = U[g];
                    if (a.sel[g]) {
                        dig[r] = a.prop_tgt[u[r]];
                        w[r] = a.vwgt ? a.vwgt[u[r]] : 1;
                    }
                }
            }
            tile_wprefix<UNIT, kMI>(dig, w, before, s_cnt, s_run, K);
            int32_t c = 0;
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                const int b = dig[r];
                if (b == K) continue;
                const int64_t incl = a.h1[(int64_t)b * T2 + t] + before[r] + w[r];
                const bool adm = a.C[b] + incl <= a.Lb[b];
                if (!adm) a.reject[b] = 1;
                else { a.sel[item_m(t, r)] = 2; c++; }
            }
            int32_t total;
            block_exclusive<OpSum>(c, s_warp, &total);
            if (threadIdx.x == 0) tc3[t] = total;
        }
    }
    grid_sync(a.bar, a.err);
    {
        int64_t *acc = s_cnt + (threadIdx.x >> 5) * K;
        for (int i = threadIdx.x; i < kWarps * K; i += kThreads) s_cnt[i] = 0;
        __syncthreads();
        const int64_t off = a.ctl->nR;
        const int32_t subround = a.ctl->subrounds;
        for (int64_t t = blockIdx.x; t < T2; t += P) {
            const int32_t tbefore = tiles_before(tc3, t, s_warp);
            bool adm[kMI];
            int32_t b8[kMI];
            int64_t w[kMI];
            uint32_t u[kMI];
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                const int64_t g = item_m(t, r);
                adm[r] = g < nk && a.sel[g] == 2;
                u[r] = adm[r] ? U[g] : 0;
                b8[r] = adm[r] ? a.prop_tgt[u[r]] : 0;
                w[r] = adm[r] ? (a.vwgt ? a.vwgt[u[r]] : 1) : 0;
            }
            // R keeps the sorted (priority) order, which inside a tile is item
            // order (round-major): per-round counts packed 16 bits each
            uint64_t lo = 0;
#pragma unroll
            for (int r = 0; r < kMI; r++)
                if (adm[r]) lo += 1ull << (16 * r);
            uint64_t tlo;
            const uint64_t plo = block_exclusive<OpSum>(lo, s_w64, &tlo);
            int32_t mine[kMI];
            {
                int32_t base = tbefore;
#pragma unroll
                for (int r = 0; r < kMI; r++) {
                    const int sh = 16 * r;
                    mine[r] = base + (int32_t)((plo >> sh) & 0xFFFF);
                    base += (int32_t)((tlo >> sh) & 0xFFFF);
                }
            }
#pragma unroll
            for (int r = 0; r < kMI; r++) {
                int32_t from = 0;
                const int32_t b = b8[r];
                if (adm[r]) {
                    const int32_t v = (int32_t)u[r];
                    from = a.part[v];
                    const int64_t p = off + mine[r];
                    a.R_node[p] = v;
                    a.R_from[p] = from;
                    a.R_to[p] = b;
                    a.R_sub[p] = subround;
                    a.r_to[v] = b;
                    a.r_at[v] = (int32_t)p;
                    a.part[v] = b;
                }
                warp_acc<UNIT>(from, -w[r], adm[r], acc);
                __syncwarp();
                warp_acc<UNIT>(b, w[r], adm[r], acc);
                __syncwarp();
            }
            __syncthreads();
            for (int i = threadIdx.x; i < K; i += kThreads) {
                const int64_t d = warps_total(s_cnt, K, i);
                if (d) atomicAdd(reinterpret_cast<unsigned long long *>(&a.Cd[i]), (unsigned long long)d);
            }
            __syncthreads();
        }
        const int32_t na = tiles_before(tc3, T2, s_warp);
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.d_na = na;
    }
}

}  // namespace

bool rebalance_fused_ok(const GraphDev &g, int key_bits, bool prefilter) {
    return g.ng == 1 && g.K() <= kFuseMaxK && key_bits <= 63 && prefilter && (((key_bits + 7) / 8) & 1);
}

void rebalance_fused_compact_hist(const GraphDev &g, const int32_t *flags, int32_t *list, const int32_t *d_n,
                                  int64_t n_max, int32_t *d_out, int32_t *lgain, int32_t *lsrc, int gbits, int cbits,
                                  int gain_only, unsigned long long *hist, uint64_t *rep, int32_t *exact, Scratch tmp,
                                  cudaStream_t s) {
    if (n_max <= 0) { UPR_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int32_t), s)); return; }
    const int vec = (aligned16(flags) ? 1 : 0) |
                    (aligned16(list) && aligned16(lgain) && aligned16(lsrc) ? 2 : 0);
    const int64_t tiles_max = ceil_div(n_max, kTile);
    k_fr_compact_hist<<<tile_grid((const void *)k_fr_compact_hist, tiles_max), kThreads, 0, s>>>(
        flags, list, d_n, d_out, lgain, g.vwgt, lsrc, gbits, cbits, gain_only, hist, rep, exact, vec,
        scan_state<int32_t>(tmp, tiles_max));
    UPR_LAUNCH_CHECK();
}

void rebalance_fused_keep_keys(const GraphDev &g, const int32_t *list, const int32_t *d_n, int64_t n_max,
                               const int32_t *lgain, const int32_t *lsrc, const int32_t *cut, int gbits, int cbits,
                               int gain_only, uint64_t *keys, uint32_t *vals, int32_t *d_out, const uint64_t *rep,
                               int32_t *exact, Scratch tmp, cudaStream_t s) {
    if (n_max <= 0) { UPR_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int32_t), s)); return; }
    const int64_t tiles_max = ceil_div(n_max, kTile);
    k_fr_keep_keys<<<tile_grid((const void *)k_fr_keep_keys, tiles_max), kThreads, 0, s>>>(
        list, d_n, lgain, g.vwgt, lsrc, cut, gbits, cbits, gain_only, keys, vals, d_out, rep, exact,
        scan_state<int32_t>(tmp, tiles_max));
    UPR_LAUNCH_CHECK();
}

bool rebalance_fused_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, const int32_t *d_n,
                          int64_t n_max, int key_bits, int gbits, int cbits, const int32_t *exact, Scratch tmp,
                          cudaStream_t s, cudaStream_t s_aux, int32_t *later_runs, int *later_kernels) {
    const int passes = (key_bits + 7) / 8;
    if (!(passes & 1)) throw CudaError{cudaErrorInvalidValue, "rebalance_fused_sort: even pass count"};
    if (later_kernels) *later_kernels = 0;
    if (n_max <= 0) return true;
    k_fr_radix_small<<<1, kThreads, 0, s>>>(keys, vals, keys_alt, vals_alt, d_n, passes, gbits, cbits, exact);
    UPR_LAUNCH_CHECK();
    if (n_max <= kTile) return true;
    const int64_t tiles_max = ceil_div(n_max, kTile);
    if (tiles_max > tmp.tiles_cap) throw CudaError{cudaErrorInvalidValue, "sort longer than the scratch"};
    int32_t *hist = reinterpret_cast<int32_t *>(tmp.mem);
    int32_t *d_hist_n = hist + (size_t)kBins * tmp.tiles_cap;
    const unsigned grid_h = wave_grid((const void *)k_fr_radix_hist, kThreads, 0, tiles_max);
    const unsigned grid_s = wave_grid((const void *)k_fr_radix_scatter, kThreads, 0, tiles_max);
    // while s is being captured (and s_aux is given), passes 1.. become the
    // body of a conditional node that pass 0 sets: an exact-bin sort, or a
    // list of one tile, skips them without launching their kernels
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    if (s_aux && later_runs && passes > 1) UPR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    const bool cond = cs == cudaStreamCaptureStatusActive;
    cudaGraphConditionalHandle later = 0;
    if (cond) UPR_CUDA(cudaGraphConditionalHandleCreate(&later, g, 0, 0));
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    auto pass = [&](int p, cudaStream_t st) {
        k_fr_radix_hist<<<grid_h, kThreads, 0, st>>>(ka, d_n, p, gbits, cbits, exact, hist, d_hist_n);
        UPR_LAUNCH_CHECK();
        exclusive_sum_i32(hist, hist, Count{d_hist_n, (int64_t)kBins * tiles_max}, tmp, st);
        k_fr_radix_scatter<<<grid_s, kThreads, 0, st>>>(ka, va, kb, vb, d_n, p, gbits, cbits, exact, hist, later,
                                                         p == 0 && cond ? later_runs : nullptr);
        UPR_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    };
    pass(0, s);
    if (!cond) {
        for (int p = 1; p < passes; p++) pass(p, s);
        return true;
    }
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    UPR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = later;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    UPR_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
    UPR_CUDA(cudaStreamBeginCaptureToGraph(s_aux, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
    const long long l0 = g_upr_launches;
    try {
        for (int p = 1; p < passes; p++) pass(p, s_aux);
    } catch (...) {
        cudaGraph_t out = nullptr;
        cudaStreamEndCapture(s_aux, &out);
        throw;
    }
    // counted when the node runs (later_runs), not with the enclosing graph
    const long long body = g_upr_launches - l0;
    g_upr_launches -= body;
    if (later_kernels) *later_kernels = (int)body;
    cudaGraph_t out = nullptr;
    UPR_CUDA(cudaStreamEndCapture(s_aux, &out));
    UPR_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return true;
}

void rebalance_fused_select_admit(const GraphDev &g, const uint32_t *U, const int32_t *d_np, int64_t np_max,
                                  int32_t *part, const int32_t *prop_tgt, const int64_t *C, int8_t *sel,
                                  long long *h0, long long *h1, int32_t *d_hist_n, int8_t *reject,
                                  const RebalCtl *ctl, int32_t *R_node, int32_t *R_from, int32_t *R_to,
                                  int32_t *R_sub, int32_t *r_to, int32_t *r_at, long long *Cd, int32_t *d_na,
                                  Scratch tmp, cudaStream_t s) {
    if (np_max <= 0) { UPR_CUDA(cudaMemsetAsync(d_na, 0, sizeof(int32_t), s)); return; }
    const int K = g.K();
    const int64_t tiles_max = ceil_div(np_max, kTile);
    const Count ch{d_hist_n, (int64_t)K * tiles_max};
    const bool unit = g.vwgt == nullptr;
    if (unit) {
        const unsigned gh = wave_grid((const void *)k_fr_src_hist<true>, kThreads, 0, tiles_max);
        k_fr_src_hist<true><<<gh, kThreads, 0, s>>>(U, d_np, part, g.vwgt, K, h0, d_hist_n);
    } else {
        const unsigned gh = wave_grid((const void *)k_fr_src_hist<false>, kThreads, 0, tiles_max);
        k_fr_src_hist<false><<<gh, kThreads, 0, s>>>(U, d_np, part, g.vwgt, K, h0, d_hist_n);
    }
    UPR_LAUNCH_CHECK();
    exclusive_sum_i64((const int64_t *)h0, (int64_t *)h1, ch, tmp, s);
    if (unit) {
        const unsigned gs = wave_grid((const void *)k_fr_select<true>, kThreads, 0, tiles_max);
        k_fr_select<true><<<gs, kThreads, 0, s>>>(U, d_np, part, g.vwgt, prop_tgt, K, C, g.Lb, h1, sel, h0, d_hist_n);
    } else {
        const unsigned gs = wave_grid((const void *)k_fr_select<false>, kThreads, 0, tiles_max);
        k_fr_select<false><<<gs, kThreads, 0, s>>>(U, d_np, part, g.vwgt, prop_tgt, K, C, g.Lb, h1, sel, h0, d_hist_n);
    }
    UPR_LAUNCH_CHECK();
    exclusive_sum_i64((const int64_t *)h0, (int64_t *)h1, ch, tmp, s);
    auto launch = [&](auto kern) {
        kern<<<tile_grid((const void *)kern, tiles_max), kThreads, 0, s>>>(
            U, d_np, sel, part, g.vwgt, prop_tgt, K, C, g.Lb, h1, reject, ctl, R_node, R_from, R_to, R_sub, r_to, r_at,
            Cd, d_na, scan_state<int32_t>(tmp, tiles_max));
    };
    if (unit) launch(k_fr_admit<true>);
    else launch(k_fr_admit<false>);
    UPR_LAUNCH_CHECK();
}

void rebalance_fused_mega(const GraphDev &g, RebalMega m, int key_bits, int64_t n_max, Scratch tmp,
                          cudaStream_t s) {
    m.K = g.K();
    m.vwgt = g.vwgt;
    m.Lb = g.Lb;
    m.passes = (key_bits + 7) / 8;
    if (!(m.passes & 1)) throw CudaError{cudaErrorInvalidValue, "rebalance_fused_mega: even pass count"};
    m.tcap = std::max<int64_t>(1, ceil_div(std::max<int64_t>(n_max, 1), kTile));
    // tile counts [tcap] x 2 and [2 tcap], then (more than one tile of
    // proposals) digit totals and counts
    const int64_t need = m.tcap == 1 ? 4 : 4 * m.tcap + kBins + (int64_t)kBins * m.tcap;
    if ((size_t)need * sizeof(int32_t) > tmp.mem_bytes)
        throw CudaError{cudaErrorInvalidValue, "rebalance_fused_mega: scratch too small"};
    m.tab = reinterpret_cast<int32_t *>(tmp.mem);
    m.bar = reinterpret_cast<unsigned long long *>(tmp.ticket + 8);
    m.err = tmp.err;
    m.vec = (aligned16(m.flags) ? 1 : 0) | (aligned16(m.list) && aligned16(m.lsrc) && aligned16(m.lgain) ? 2 : 0);
    const bool unit = g.vwgt == nullptr;
    const void *fn = unit ? (const void *)k_fr_mega<true> : (const void *)k_fr_mega<false>;
    const int per_sm = std::min(2, resident_ctas(fn, kThreads, 0));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(device_sm_count() * per_sm));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (unit) UPR_CUDA(cudaLaunchKernelEx(&cfg, k_fr_mega<true>, m));
    else UPR_CUDA(cudaLaunchKernelEx(&cfg, k_fr_mega<false>, m));
    UPR_LAUNCH_CHECK();
}

void rebalance_fused_end(const GraphDev &g, int64_t *C, long long *Cd, int8_t *excl, const int8_t *reject,
                         const int32_t *d_na, RebalCtl *ctl, cudaStream_t s, cudaGraphConditionalHandle cond,
                         int32_t max_subrounds, int8_t *over, int8_t *reject_next, const int32_t *d_n1) {
    if (over && (!reject_next || reject_next != reject || !d_n1 || g.K() > 256))
        throw CudaError{cudaErrorInvalidValue, "rebalance_fused_end: begin_next needs reject and d_n1, K <= 256"};
    k_fr_end<<<1, 256, 0, s>>>(C, Cd, g.Lb, g.K(), excl, const_cast<int8_t *>(reject), d_na, ctl, cond, max_subrounds,
                               over, d_n1);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
