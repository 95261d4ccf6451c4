// Device-wide primitives written for this library: tile scans (sum / max),
// stable LSD radix sort of (64-bit key, 32-bit value) pairs and stable flag
// compaction.  Every ordered list the refinement produces comes out of these,
// never out of the order of atomic operations, so results are deterministic.
//
// Element counts may live in device memory (Count::d) next to a static upper
// bound (Count::max): grids are sized by the bound and every kernel reads the
// actual count, so a step can be enqueued without the host knowing how long
// the previous step's output was.
//
// Tiles are 2048 items: 256 threads x 8 items, grid-stride over tiles.  A scan
// is reduce-then-scan (per-tile totals, a one-CTA scan of the totals, a
// per-tile scan with its offset).  A radix pass is histogram -> scan of the
// digit-major histogram -> stable scatter; inside a tile, equal digits are
// ranked in item order with __match_any_sync per warp and a per-digit prefix
// over the 8 warps.  Lists of at most one tile are sorted in one CTA.
#include "kernels.h"

namespace upr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 2048
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ int64_t count_of(const int32_t *d, int64_t max) { return d ? (int64_t)*d : max; }
__device__ __forceinline__ int64_t tiles_of(int64_t n) { return (n + kTile - 1) / kTile; }

struct OpSum {
    template <typename T> __device__ __forceinline__ static T apply(T a, T b) { return a + b; }
    template <typename T> __device__ __forceinline__ static T identity() { return T(0); }
};
struct OpMax {
    template <typename T> __device__ __forceinline__ static T apply(T a, T b) { return a > b ? a : b; }
    template <typename T> __device__ __forceinline__ static T identity() { return T(0); }   // unsigned only
};

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix, *total receives the block aggregate.
template <typename Op, typename T>
__device__ __forceinline__ T block_exclusive(T v, T *s_warp, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = Op::template apply<T>(u, inc);
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kWarps ? s_warp[lane] : Op::template identity<T>();
        for (int o = 1; o < kWarps; o <<= 1) {
            T u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = Op::template apply<T>(u, w);
        }
        if (lane < kWarps) s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    T warp_prefix = warp == 0 ? Op::template identity<T>() : s_warp[warp - 1];
    *total = s_warp[kWarps - 1];
    T excl = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) excl = Op::template identity<T>();
    __syncthreads();
    return Op::template apply<T>(warp_prefix, excl);
}

// Thread t of a tile owns items [8t, 8t + 8): loaded with 16-byte vector loads
// when the tile is complete and the input aligned, element by element otherwise.
template <typename T>
__device__ __forceinline__ void load_items(const T *__restrict__ in, int64_t base, int64_t n, bool vec,
                                           T (&x)[kItems]) {
    const int64_t first = base + (int64_t)threadIdx.x * kItems;
    if (vec && first + kItems <= n) {
        const int4 *p = reinterpret_cast<const int4 *>(in + first);
        int4 tmp[kItems * sizeof(T) / 16];
#pragma unroll
        for (int i = 0; i < (int)(kItems * sizeof(T) / 16); i++) tmp[i] = p[i];
        const T *t = reinterpret_cast<const T *>(tmp);
#pragma unroll
        for (int j = 0; j < kItems; j++) x[j] = t[j];
    } else {
#pragma unroll
        for (int j = 0; j < kItems; j++) x[j] = first + j < n ? in[first + j] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store_items(T *__restrict__ out, int64_t base, int64_t n, bool vec,
                                            const T (&x)[kItems]) {
    const int64_t first = base + (int64_t)threadIdx.x * kItems;
    if (vec && first + kItems <= n) {
        int4 *p = reinterpret_cast<int4 *>(out + first);
        const int4 *t = reinterpret_cast<const int4 *>(x);
#pragma unroll
        for (int i = 0; i < (int)(kItems * sizeof(T) / 16); i++) p[i] = t[i];
    } else {
#pragma unroll
        for (int j = 0; j < kItems; j++)
            if (first + j < n) out[first + j] = x[j];
    }
}

// Exclusive scan of the tile totals part[0 .. tiles) by one CTA, in chunks of
// 2048 with a carry; optionally writes the grand total (as int32) to *d_total.
template <typename Op, typename T>
__device__ void scan_partials(T *part, int64_t tiles, int32_t *d_total, T *s_warp) {
    T carry = Op::template identity<T>();
    for (int64_t c0 = 0; c0 < tiles; c0 += kTile) {
        T x[kItems];
        const int64_t first = c0 + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int j = 0; j < kItems; j++) x[j] = first + j < tiles ? __ldcg(part + first + j) : Op::template identity<T>();
        T acc = Op::template identity<T>();
#pragma unroll
        for (int j = 0; j < kItems; j++) acc = Op::template apply<T>(acc, x[j]);
        T total;
        T run = Op::template apply<T>(carry, block_exclusive<Op>(acc, s_warp, &total));
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const T nxt = Op::template apply<T>(run, x[j]);
            if (first + j < tiles) part[first + j] = run;
            run = nxt;
        }
        carry = Op::template apply<T>(carry, total);
    }
    if (d_total && threadIdx.x == 0) *d_total = (int32_t)carry;
}

// Per-tile totals; the CTA that finishes last (ticket counter, no waiting)
// scans them and resets the ticket.
template <typename Op, typename T, typename TIn>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const TIn *__restrict__ in, const int32_t *__restrict__ d_n,
                                                          int64_t n_max, T *__restrict__ part, int vec,
                                                          unsigned int *__restrict__ ticket) {
    __shared__ T s_warp[kWarps];
    __shared__ bool s_last;
    const int64_t n = count_of(d_n, n_max);
    for (int64_t tile = blockIdx.x; tile < tiles_of(n); tile += gridDim.x) {
        TIn x[kItems];
        load_items(in, tile * kTile, n, vec != 0, x);
        T acc = Op::template identity<T>();
#pragma unroll
        for (int j = 0; j < kItems; j++) acc = Op::template apply<T>(acc, (T)x[j]);
        T total;
        block_exclusive<Op>(acc, s_warp, &total);
        if (threadIdx.x == 0) part[tile] = total;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    scan_partials<Op, T>(part, tiles_of(n), nullptr, s_warp);
    if (threadIdx.x == 0) *ticket = 0;
}

// Scans every tile with the offset from part[] (exclusive-scanned totals; null = one tile).
template <typename Op, typename T, typename TIn>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const TIn *__restrict__ in, T *__restrict__ out,
                                                        const int32_t *__restrict__ d_n, int64_t n_max,
                                                        const T *__restrict__ part, int inclusive, int vec) {
    __shared__ T s_warp[kWarps];
    const int64_t n = count_of(d_n, n_max);
    for (int64_t tile = blockIdx.x; tile < tiles_of(n); tile += gridDim.x) {
        TIn x[kItems];
        load_items(in, tile * kTile, n, (vec & 1) != 0, x);
        T acc = Op::template identity<T>();
#pragma unroll
        for (int j = 0; j < kItems; j++) acc = Op::template apply<T>(acc, (T)x[j]);
        T total;
        const T pre = block_exclusive<Op>(acc, s_warp, &total);
        T run = Op::template apply<T>(part ? part[tile] : Op::template identity<T>(), pre);
        T y[kItems];
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const T nxt = Op::template apply<T>(run, (T)x[j]);
            y[j] = inclusive ? nxt : run;
            run = nxt;
        }
        store_items(out, tile * kTile, n, (vec & 2) != 0, y);
    }
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

inline unsigned tile_grid(int64_t tiles_max) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles_max, (int64_t)device_sm_count() * 8));
}

template <typename Op, typename T, typename TIn>
void scan_impl(const TIn *in, T *out, Count n, bool inclusive, Scratch tmp, cudaStream_t s) {
    if (n.max <= 0) return;
    const int vin = aligned16(in) ? 1 : 0;
    const int vio = vin | (aligned16(out) ? 2 : 0);
    const int64_t tiles_max = ceil_div(n.max, kTile);
    if (tiles_max == 1) {
        k_tile_scan<Op, T, TIn><<<1, kThreads, 0, s>>>(in, out, n.d, n.max, (const T *)nullptr, inclusive ? 1 : 0, vio);
        UPR_LAUNCH_CHECK();
        return;
    }
    T *part = (T *)tmp.mem;
    k_tile_reduce<Op, T, TIn><<<tile_grid(tiles_max), kThreads, 0, s>>>(in, n.d, n.max, part, vin, tmp.ticket);
    UPR_LAUNCH_CHECK();
    k_tile_scan<Op, T, TIn><<<tile_grid(tiles_max), kThreads, 0, s>>>(in, out, n.d, n.max, part, inclusive ? 1 : 0,
                                                                      vio);
    UPR_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ compaction
// Pass 1: number of set flags per tile.  One-CTA scan of those.  Pass 2: every
// thread ranks its 8 flags in registers and writes the indices of the set
// ones; tile order, then thread order, then item order = index order.
__global__ void __launch_bounds__(kThreads) k_flag_count(const int32_t *__restrict__ flags, const int32_t *__restrict__ d_n,
                                                         int64_t n_max, int32_t *__restrict__ counts, int vec,
                                                         int32_t *__restrict__ d_count, unsigned int *__restrict__ ticket) {
    __shared__ int32_t s_warp[kWarps];
    __shared__ bool s_last;
    const int64_t n = count_of(d_n, n_max);
    for (int64_t tile = blockIdx.x; tile < tiles_of(n); tile += gridDim.x) {
        int32_t x[kItems];
        load_items(flags, tile * kTile, n, vec != 0, x);
        int32_t c = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) c += x[j] != 0;
        int32_t total;
        block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x == 0) counts[tile] = total;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    scan_partials<OpSum, int32_t>(counts, tiles_of(n), d_count, s_warp);
    if (threadIdx.x == 0) *ticket = 0;
}

__global__ void __launch_bounds__(kThreads) k_flag_scatter(const int32_t *__restrict__ flags, const int32_t *__restrict__ d_n,
                                                           int64_t n_max, const int32_t *__restrict__ offs,
                                                           int32_t *__restrict__ out, int32_t *__restrict__ d_count,
                                                           int vec) {
    __shared__ int32_t s_warp[kWarps];
    const int64_t n = count_of(d_n, n_max);
    if (!offs && blockIdx.x == 0 && threadIdx.x == 0 && n == 0) *d_count = 0;
    for (int64_t tile = blockIdx.x; tile < tiles_of(n); tile += gridDim.x) {
        int32_t x[kItems];
        load_items(flags, tile * kTile, n, vec != 0, x);
        int32_t c = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) c += x[j] != 0;
        int32_t total;
        int32_t pos = block_exclusive<OpSum>(c, s_warp, &total) + (offs ? offs[tile] : 0);
        const int64_t first = tile * kTile + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int j = 0; j < kItems; j++)
            if (x[j]) out[pos++] = (int32_t)(first + j);
        if (!offs && threadIdx.x == 0) *d_count = total;   // single tile
    }
}

// ------------------------------------------------------------------ radix sort
constexpr int kBins = 256;

// Stable ranking of the 8 x 256 items of a tile by digit (0..255, 256 = no item).
// Item (round r, thread t) precedes (r', t') iff r < r' or (r == r' and t < t').
// s_cnt: [2][kWarps][kBins+1] zero-initialised; s_run: [kBins+1] tile-local
// running counts (zero-initialised).  Returns the rank within the tile among
// items of the same digit.
__device__ __forceinline__ void tile_rank(const int (&dig)[kItems], int (&rank)[kItems], int *s_cnt, int *s_run) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    constexpr int kStride = kWarps * (kBins + 1);
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        int *cnt = s_cnt + (r & 1) * kStride;
        const int d = dig[r];
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int within = __popc(peers & lt);
        if (within == 0) cnt[warp * (kBins + 1) + d] = __popc(peers);
        __syncthreads();
        // thread t owns digit t (t < 256); digit 256 (padding) is owned by thread 0 as well
        for (int dd = threadIdx.x; dd <= kBins; dd += kThreads) {
            int run = s_run[dd];
            for (int w = 0; w < kWarps; w++) {
                int c = cnt[w * (kBins + 1) + dd];
                cnt[w * (kBins + 1) + dd] = run;
                run += c;
            }
            s_run[dd] = run;
            // clear the other buffer (used two rounds ago, read by everyone before the barrier above)
            int *old = s_cnt + ((r + 1) & 1) * kStride;
            for (int w = 0; w < kWarps; w++) old[w * (kBins + 1) + dd] = 0;
        }
        __syncthreads();
        rank[r] = cnt[warp * (kBins + 1) + d] + within;
    }
}

// Digit histograms per tile, digit-major with the actual tile count as
// stride; block 0 publishes the histogram length (0 when the list fits one
// tile: the one-CTA sort handles it).
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint64_t *__restrict__ keys, const int32_t *__restrict__ d_n,
                                                         int64_t n_max, int shift, int32_t *__restrict__ hist,
                                                         int32_t *__restrict__ d_hist_n) {
    __shared__ int s_h[kBins];
    const int64_t n = count_of(d_n, n_max);
    const int64_t T = tiles_of(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_hist_n = n > kTile ? (int32_t)(kBins * T) : 0;
    if (n <= kTile) return;
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        for (int i = threadIdx.x; i < kBins; i += kThreads) s_h[i] = 0;
        __syncthreads();
        const int64_t base = tile * kTile;
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = base + r * kThreads + threadIdx.x;
            if (g < n) atomicAdd(&s_h[(int)((keys[g] >> shift) & 0xFF)], 1);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kBins; i += kThreads) hist[(int64_t)i * T + tile] = s_h[i];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                                            uint64_t *__restrict__ okeys, uint32_t *__restrict__ ovals,
                                                            const int32_t *__restrict__ d_n, int64_t n_max, int shift,
                                                            const int32_t *__restrict__ offs) {
    __shared__ int s_cnt[2 * kWarps * (kBins + 1)];
    __shared__ int s_run[kBins + 1];
    __shared__ int s_off[kBins];
    const int64_t n = count_of(d_n, n_max);
    if (n <= kTile) return;
    const int64_t T = tiles_of(n);
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
        for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
        for (int i = threadIdx.x; i < kBins; i += kThreads) s_off[i] = offs[(int64_t)i * T + tile];
        __syncthreads();
        const int64_t base = tile * kTile;
        uint64_t k[kItems];
        uint32_t v[kItems];
        int dig[kItems], rank[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int64_t g = base + r * kThreads + threadIdx.x;
            if (g < n) { k[r] = keys[g]; v[r] = vals[g]; dig[r] = (int)((k[r] >> shift) & 0xFF); }
            else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
        }
        tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            if (dig[r] < kBins) {
                const int64_t p = (int64_t)s_off[dig[r]] + rank[r];
                okeys[p] = k[r];
                ovals[p] = v[r];
            }
        }
        __syncthreads();
    }
}

// All passes of a sort of at most one tile inside one CTA (shared memory);
// reads (keys, vals), writes the result to (okeys, ovals) (may alias the input).
__global__ void __launch_bounds__(kThreads) k_radix_small(const uint64_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ vals, uint64_t *okeys,
                                                          uint32_t *ovals, const int32_t *__restrict__ d_n,
                                                          int64_t n_max, int passes) {
    __shared__ int s_cnt[2 * kWarps * (kBins + 1)];
    __shared__ int s_run[kBins + 1];
    __shared__ int s_off[kBins];
    __shared__ int s_warp[kWarps];
    __shared__ uint64_t s_k[kTile];
    __shared__ uint32_t s_v[kTile];
    const int64_t n64 = count_of(d_n, n_max);
    if (n64 > kTile || n64 <= 0) return;
    const int n = (int)n64;
    for (int i = threadIdx.x; i < n; i += kThreads) { s_k[i] = keys[i]; s_v[i] = vals[i]; }
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
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
            if (g < n) { k[r] = s_k[g]; v[r] = s_v[g]; dig[r] = (int)((k[r] >> shift) & 0xFF); atomicAdd(&s_off[dig[r]], 1); }
            else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
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

__global__ void k_iota_u32(uint32_t *v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    return (size_t)(ceil_div(n > 0 ? n : 1, kTile) + 64) * sizeof(int64_t);
}

size_t radix_temp_bytes(int64_t n) {
    const int64_t tiles = ceil_div(n > 0 ? n : 1, kTile);
    const size_t hist = (size_t)kBins * tiles;
    return hist * sizeof(int32_t) + 256 + scan_temp_bytes((int64_t)hist);
}

void exclusive_sum_i32(const int32_t *in, int32_t *out, Count n, Scratch tmp, cudaStream_t s) {
    scan_impl<OpSum, int32_t, int32_t>(in, out, n, false, tmp, s);
}
void exclusive_sum_i64(const int64_t *in, int64_t *out, Count n, Scratch tmp, cudaStream_t s) {
    scan_impl<OpSum, int64_t, int64_t>(in, out, n, false, tmp, s);
}
void inclusive_sum_i64(const int64_t *in, int64_t *out, Count n, Scratch tmp, cudaStream_t s) {
    scan_impl<OpSum, int64_t, int64_t>(in, out, n, true, tmp, s);
}
void exclusive_sum_i32_to_i64(const int32_t *in, int64_t *out, Count n, Scratch tmp, cudaStream_t s) {
    scan_impl<OpSum, int64_t, int32_t>(in, out, n, false, tmp, s);
}
void inclusive_max_u64(const uint64_t *in, uint64_t *out, Count n, Scratch tmp, cudaStream_t s) {
    scan_impl<OpMax, uint64_t, uint64_t>(in, out, n, true, tmp, s);
}

void iota_u32(uint32_t *v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_iota_u32<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(v, n);
    UPR_LAUNCH_CHECK();
}

bool radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, Count n, int bits,
                      Scratch tmp, cudaStream_t s) {
    if (n.max <= 0 || bits <= 0) return false;
    const int passes = (bits + 7) / 8;
    const bool alt = passes & 1;
    // a list that fits one tile: all passes in one CTA, result where the multi-pass sort would leave it
    k_radix_small<<<1, kThreads, 0, s>>>(keys, vals, alt ? keys_alt : keys, alt ? vals_alt : vals, n.d, n.max, passes);
    UPR_LAUNCH_CHECK();
    if (n.max <= kTile) return alt;
    const int64_t tiles_max = ceil_div(n.max, kTile);
    int32_t *hist = (int32_t *)tmp.mem;
    int32_t *d_hist_n = (int32_t *)(tmp.mem + (size_t)kBins * tiles_max * sizeof(int32_t));
    const Scratch stmp{tmp.mem + (size_t)kBins * tiles_max * sizeof(int32_t) + 256, tmp.ticket};
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; p++) {
        k_radix_hist<<<tile_grid(tiles_max), kThreads, 0, s>>>(ka, n.d, n.max, 8 * p, hist, d_hist_n);
        UPR_LAUNCH_CHECK();
        exclusive_sum_i32(hist, hist, Count{d_hist_n, (int64_t)kBins * tiles_max}, stmp, s);
        k_radix_scatter<<<tile_grid(tiles_max), kThreads, 0, s>>>(ka, va, kb, vb, n.d, n.max, 8 * p, hist);
        UPR_LAUNCH_CHECK();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return alt;
}

void select_flags(const int32_t *flags, int32_t *out_idx, int32_t *d_count, Count n, Scratch tmp, cudaStream_t s) {
    if (n.max <= 0) { UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s)); return; }
    const int vec = aligned16(flags) ? 1 : 0;
    const int64_t tiles_max = ceil_div(n.max, kTile);
    if (tiles_max == 1) {
        k_flag_scatter<<<1, kThreads, 0, s>>>(flags, n.d, n.max, nullptr, out_idx, d_count, vec);
        UPR_LAUNCH_CHECK();
        return;
    }
    int32_t *counts = (int32_t *)tmp.mem;
    k_flag_count<<<tile_grid(tiles_max), kThreads, 0, s>>>(flags, n.d, n.max, counts, vec, d_count, tmp.ticket);
    UPR_LAUNCH_CHECK();
    k_flag_scatter<<<tile_grid(tiles_max), kThreads, 0, s>>>(flags, n.d, n.max, counts, out_idx, d_count, vec);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
