// Device-wide primitives written for this library: tile scans (sum / max),
// stable LSD radix sort of (64-bit key, 32-bit value) pairs and stable flag
// compaction.  Every ordered list the refinement produces comes out of these,
// never out of the order of atomic operations, so results are deterministic.
//
// Tiles are 2048 items: 256 threads x 8 items.  A scan is reduce-then-scan
// (per-tile totals, a recursive scan of the totals, a per-tile scan with its
// offset).  A radix pass is histogram -> scan of the digit-major histogram ->
// stable scatter; inside a tile, equal digits are ranked in item order with
// __match_any_sync per warp and a per-digit prefix over the 8 warps.
#include "kernels.h"

namespace upr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 2048
constexpr int kWarps = kThreads / 32;

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

// Loads the tile striped into shared memory, reduces 8 consecutive items per thread.
template <typename Op, typename T, typename TIn>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const TIn *__restrict__ in, int64_t n, T *__restrict__ part) {
    __shared__ T s_items[kTile];
    __shared__ T s_warp[kWarps];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        s_items[i] = g < n ? (T)in[g] : Op::template identity<T>();
    }
    __syncthreads();
    T acc = Op::template identity<T>();
#pragma unroll
    for (int j = 0; j < kItems; j++) acc = Op::template apply<T>(acc, s_items[threadIdx.x * kItems + j]);
    T total;
    block_exclusive<Op>(acc, s_warp, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Scans one tile with an offset taken from part[] (already exclusive-scanned).
template <typename Op, typename T, typename TIn>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const TIn *__restrict__ in, T *__restrict__ out, int64_t n,
                                                        const T *__restrict__ part, int inclusive) {
    __shared__ T s_items[kTile];
    __shared__ T s_warp[kWarps];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        s_items[i] = g < n ? (T)in[g] : Op::template identity<T>();
    }
    __syncthreads();
    T loc[kItems];
    T acc = Op::template identity<T>();
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        loc[j] = s_items[threadIdx.x * kItems + j];
        acc = Op::template apply<T>(acc, loc[j]);
    }
    T total;
    T pre = block_exclusive<Op>(acc, s_warp, &total);
    T off = part ? part[blockIdx.x] : Op::template identity<T>();
    T run = Op::template apply<T>(off, pre);
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        T nxt = Op::template apply<T>(run, loc[j]);
        s_items[threadIdx.x * kItems + j] = inclusive ? nxt : run;
        run = nxt;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) out[g] = s_items[i];
    }
}

template <typename Op, typename T, typename TIn>
void scan_impl(const TIn *in, T *out, int64_t n, bool inclusive, T *tmp, cudaStream_t s) {
    if (n <= 0) return;
    int64_t tiles = ceil_div(n, kTile);
    if (tiles == 1) {
        k_tile_scan<Op, T, TIn><<<1, kThreads, 0, s>>>(in, out, n, (const T *)nullptr, inclusive ? 1 : 0);
        UPR_LAUNCH_CHECK();
        return;
    }
    T *part = tmp;
    k_tile_reduce<Op, T, TIn><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, part);
    UPR_LAUNCH_CHECK();
    scan_impl<Op, T, T>(part, part, tiles, false, tmp + ceil_div(tiles, 32) * 32, s);
    k_tile_scan<Op, T, TIn><<<(unsigned)tiles, kThreads, 0, s>>>(in, out, n, part, inclusive ? 1 : 0);
    UPR_LAUNCH_CHECK();
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

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                         int32_t *__restrict__ hist, int64_t tiles) {
    __shared__ int s_h[kBins];
    for (int i = threadIdx.x; i < kBins; i += kThreads) s_h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        int64_t g = base + r * kThreads + threadIdx.x;
        if (g < n) atomicAdd(&s_h[(int)((keys[g] >> shift) & 0xFF)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += kThreads) hist[(int64_t)i * tiles + blockIdx.x] = s_h[i];
}

__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                                            uint64_t *__restrict__ okeys, uint32_t *__restrict__ ovals,
                                                            int64_t n, int shift, const int32_t *__restrict__ offs,
                                                            int64_t tiles) {
    __shared__ int s_cnt[2 * kWarps * (kBins + 1)];
    __shared__ int s_run[kBins + 1];
    __shared__ int s_off[kBins];
    for (int i = threadIdx.x; i < 2 * kWarps * (kBins + 1); i += kThreads) s_cnt[i] = 0;
    for (int i = threadIdx.x; i <= kBins; i += kThreads) s_run[i] = 0;
    for (int i = threadIdx.x; i < kBins; i += kThreads) s_off[i] = offs[(int64_t)i * tiles + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint64_t k[kItems];
    uint32_t v[kItems];
    int dig[kItems], rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        int64_t g = base + r * kThreads + threadIdx.x;
        if (g < n) { k[r] = keys[g]; v[r] = vals[g]; dig[r] = (int)((k[r] >> shift) & 0xFF); }
        else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
    }
    tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        if (dig[r] < kBins) {
            int64_t p = (int64_t)s_off[dig[r]] + rank[r];
            okeys[p] = k[r];
            ovals[p] = v[r];
        }
    }
}

// All passes of a sort of at most one tile inside one CTA (shared memory).
__global__ void __launch_bounds__(kThreads) k_radix_small(uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                          int n, int passes) {
    __shared__ int s_cnt[2 * kWarps * (kBins + 1)];
    __shared__ int s_run[kBins + 1];
    __shared__ int s_off[kBins];
    __shared__ int s_warp[kWarps];
    __shared__ uint64_t s_k[kTile];
    __shared__ uint32_t s_v[kTile];
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
            int g = r * kThreads + threadIdx.x;
            if (g < n) { k[r] = s_k[g]; v[r] = s_v[g]; dig[r] = (int)((k[r] >> shift) & 0xFF); atomicAdd(&s_off[dig[r]], 1); }
            else { k[r] = 0; v[r] = 0; dig[r] = kBins; }
        }
        __syncthreads();
        int c = threadIdx.x < kBins ? s_off[threadIdx.x] : 0;
        int total;
        int ex = block_exclusive<OpSum>(c, s_warp, &total);
        if (threadIdx.x < kBins) s_off[threadIdx.x] = ex;
        __syncthreads();
        tile_rank(dig, rank, s_cnt, s_run);
#pragma unroll
        for (int r = 0; r < kItems; r++)
            if (dig[r] < kBins) { int q = s_off[dig[r]] + rank[r]; s_k[q] = k[r]; s_v[q] = v[r]; }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += kThreads) { keys[i] = s_k[i]; vals[i] = s_v[i]; }
}

__global__ void k_select_scatter(const int32_t *__restrict__ flags, const int32_t *__restrict__ excl, int64_t n,
                                 int32_t *__restrict__ out, int32_t *__restrict__ count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[i]) out[excl[i]] = (int32_t)i;
    if (i == n - 1) *count = excl[i] + (flags[i] ? 1 : 0);
}

__global__ void k_iota_u32(uint32_t *v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    // partial sums of every level, each padded to 32 entries, 8 bytes each
    size_t total = 0;
    int64_t m = n;
    while (m > kTile) { m = ceil_div(m, kTile); total += (size_t)ceil_div(m, 32) * 32; }
    return (total + 64) * sizeof(int64_t);
}

size_t radix_temp_bytes(int64_t n) {
    int64_t tiles = ceil_div(n > 0 ? n : 1, kTile);
    size_t hist = (size_t)kBins * tiles;
    return hist * sizeof(int32_t) + 256 + scan_temp_bytes((int64_t)hist);
}

void exclusive_sum_i32(const int32_t *in, int32_t *out, int64_t n, void *tmp, cudaStream_t s) {
    scan_impl<OpSum, int32_t, int32_t>(in, out, n, false, (int32_t *)tmp, s);
}
void exclusive_sum_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    scan_impl<OpSum, int64_t, int64_t>(in, out, n, false, (int64_t *)tmp, s);
}
void inclusive_sum_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    scan_impl<OpSum, int64_t, int64_t>(in, out, n, true, (int64_t *)tmp, s);
}
void exclusive_sum_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    scan_impl<OpSum, int64_t, int32_t>(in, out, n, false, (int64_t *)tmp, s);
}
void inclusive_max_u64(const uint64_t *in, uint64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    scan_impl<OpMax, uint64_t, uint64_t>(in, out, n, true, (uint64_t *)tmp, s);
}

void iota_u32(uint32_t *v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_iota_u32<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(v, n);
    UPR_LAUNCH_CHECK();
}

bool radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int64_t n, int bits,
                      void *tmp, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return false;
    const int passes = (bits + 7) / 8;
    if (n <= kTile) {
        k_radix_small<<<1, kThreads, 0, s>>>(keys, vals, (int)n, passes);
        UPR_LAUNCH_CHECK();
        return false;
    }
    const int64_t tiles = ceil_div(n, kTile);
    int32_t *hist = (int32_t *)tmp;
    void *stmp = (char *)tmp + (size_t)kBins * tiles * sizeof(int32_t) + 256;
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; p++) {
        k_radix_hist<<<(unsigned)tiles, kThreads, 0, s>>>(ka, n, 8 * p, hist, tiles);
        UPR_LAUNCH_CHECK();
        exclusive_sum_i32(hist, hist, (int64_t)kBins * tiles, stmp, s);
        k_radix_scatter<<<(unsigned)tiles, kThreads, 0, s>>>(ka, va, kb, vb, n, 8 * p, hist, tiles);
        UPR_LAUNCH_CHECK();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return passes & 1;
}

void select_flags(const int32_t *flags, int32_t *excl, int32_t *out_idx, int32_t *d_count, int64_t n, void *tmp,
                  cudaStream_t s) {
    if (n <= 0) { UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s)); return; }
    exclusive_sum_i32(flags, excl, n, tmp, s);
    k_select_scatter<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(flags, excl, n, out_idx, d_count);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
