// Building blocks of the single-pass primitives (prim.cu) for kernels that
// fuse a compaction or a scan into other work: tiles of 2048 items (256
// threads x 8 items), block-wide scans, the decoupled look-back over tile
// status words tagged with the call's epoch (every wait bounded; a wait that
// gives up sets the scratch's error word) and the per-call tile counters.
#pragma once

#include "kernels.h"

namespace upr {
namespace prim {


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
// (N items per thread: kItems for the fused kernels' tiles, more for the
// scans and compactions of prim.cu)
template <typename T, int N>
__device__ __forceinline__ void load_items(const T *__restrict__ in, int64_t base, int64_t n, bool vec,
                                           T (&x)[N]) {
    const int64_t first = base + (int64_t)threadIdx.x * N;
    if (vec && first + N <= n) {
        const int4 *p = reinterpret_cast<const int4 *>(in + first);
        int4 tmp[N * sizeof(T) / 16];
#pragma unroll
        for (int i = 0; i < (int)(N * sizeof(T) / 16); i++) tmp[i] = p[i];
        const T *t = reinterpret_cast<const T *>(tmp);
#pragma unroll
        for (int j = 0; j < N; j++) x[j] = t[j];
    } else {
#pragma unroll
        for (int j = 0; j < N; j++) x[j] = first + j < n ? in[first + j] : T(0);
    }
}

template <typename T, int N>
__device__ __forceinline__ void store_items(T *__restrict__ out, int64_t base, int64_t n, bool vec,
                                            const T (&x)[N]) {
    const int64_t first = base + (int64_t)threadIdx.x * N;
    if (vec && first + N <= n) {
        int4 *p = reinterpret_cast<int4 *>(out + first);
        const int4 *t = reinterpret_cast<const int4 *>(x);
#pragma unroll
        for (int i = 0; i < (int)(N * sizeof(T) / 16); i++) p[i] = t[i];
    } else {
#pragma unroll
        for (int j = 0; j < N; j++)
            if (first + j < n) out[first + j] = x[j];
    }
}

// ---- decoupled look-back
constexpr uint32_t kAgg = 1, kIncl = 2;
constexpr int kMaxSpin = 1 << 22;            // polls before a wait gives up (error word set)

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Tile status of the scans: a flag word ((epoch << 2) | state) and separate
// aggregate / inclusive values (a value is never overwritten after its flag).
template <typename T>
struct ScanState {
    uint32_t *flag;
    T *agg, *incl;
    unsigned int *ctr;      // [0] next tile, [1] finished CTAs
    int32_t *err;
    uint32_t *epoch;        // the last epoch used (0 after a clear)
    int64_t flags_cap;      // status words in `flag`
};

// Epochs live in 30 bits; the call that reaches the limit clears every status
// word and starts again from 1, so no stale word can carry a current epoch.
constexpr uint32_t kEpochLimit = (1u << 30) - 1;

template <typename T>
__device__ __forceinline__ uint32_t call_epoch(const ScanState<T> &st) {
    return *(volatile const uint32_t *)st.epoch + 1u;
}

// Waits (bounded) until tile j's flag carries this epoch; returns its state
// (kAgg / kIncl), or 0 after a timeout (recorded in *err).
__device__ __forceinline__ bool gave_up(const int32_t *err) { return *(volatile const int32_t *)err != 0; }

__device__ __forceinline__ uint32_t wait_flag(const uint32_t *flag, uint32_t epoch, int32_t *err) {
    for (int it = 0; it < kMaxSpin; it++) {
        const uint32_t f = ld_acquire(flag);
        if ((f >> 2) == epoch) return f & 3u;
        if (it >= 32) {
            if ((it & 1023) == 0 && gave_up(err)) return 0;   // another wait already timed out
            __nanosleep(64);
        }
    }
    atomicOr(err, 1);
    return 0;
}

// The next tile for this CTA (all threads get it).
__device__ __forceinline__ int64_t next_tile(unsigned int *ctr, uint32_t *s_tile) {
    if (threadIdx.x == 0) *s_tile = atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const int64_t t = *s_tile;
    __syncthreads();
    return t;
}

// CTAs that take part in a pass over `tiles` tiles: no more than there are
// tiles; the others return at once without touching the counters.
__device__ __forceinline__ unsigned participants(int64_t tiles) {
    return (unsigned)min((int64_t)gridDim.x, tiles);
}

// Called by every taking-part CTA once it takes no more tiles: the last one
// resets the counters and advances the epoch (all taking-part CTAs read it
// before they got here).
template <typename T>
__device__ __forceinline__ void finish_tiles(const ScanState<T> &st, unsigned parts, uint32_t epoch) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st.ctr[1], 1u) == parts - 1;
    }
    __syncthreads();
    if (!s_last) return;
    if (epoch >= kEpochLimit) {
        for (int64_t i = threadIdx.x; i < st.flags_cap; i += blockDim.x) st.flag[i] = 0;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st.ctr[0] = 0;
        st.ctr[1] = 0;
        *st.epoch = epoch >= kEpochLimit ? 0u : epoch;
        __threadfence();
    }
}

// Exclusive prefix (over the preceding tiles) of `total` for tile t, computed
// by warp 0 and published by its lane 0: the warp reads the status of 32
// preceding tiles at a time (lane l: tile j - l), adds the published values
// up to the nearest inclusive prefix, and goes on to the next 32 if there is
// none among them.  Returns the prefix in every lane of warp 0.
template <typename Op, typename T>
__device__ __forceinline__ T lookback(const ScanState<T> &st, int64_t t, T total, uint32_t epoch) {
    const int lane = threadIdx.x & 31;
    T excl = Op::template identity<T>();
    if (t == 0) {
        if (lane == 0) {
            st.incl[0] = total;
            st_release(&st.flag[0], (epoch << 2) | kIncl);
        }
        return excl;
    }
    if (lane == 0) {
        st.agg[t] = total;
        st_release(&st.flag[t], (epoch << 2) | kAgg);
    }
    for (int64_t j = t - 1; j >= 0; j -= 32) {
        const int64_t jj = j - lane;
        uint32_t s = 0;
        T v = Op::template identity<T>();
        if (jj >= 0) {
            s = wait_flag(&st.flag[jj], epoch, st.err);
            if (s == kIncl) v = st.incl[jj];
            else if (s == kAgg) v = st.agg[jj];
        }
        const unsigned incl = __ballot_sync(0xffffffffu, s == kIncl);
        const unsigned bad = __ballot_sync(0xffffffffu, jj >= 0 && s == 0);
        // lanes up to the nearest inclusive prefix (all lanes if none) contribute
        const int stop = incl ? __ffs(incl) - 1 : 31;
        if (lane > stop) v = Op::template identity<T>();
        for (int o = 16; o > 0; o >>= 1) v = Op::template apply<T>(v, __shfl_xor_sync(0xffffffffu, v, o));
        excl = Op::template apply<T>(excl, v);
        if (incl || bad) break;                       // done (or a wait timed out: error recorded)
    }
    if (lane == 0) {
        st.incl[t] = Op::template apply<T>(excl, total);
        st_release(&st.flag[t], (epoch << 2) | kIncl);
    }
    return excl;
}


inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Persistent grid of the tile kernels (tiles are taken dynamically): as many
// CTAs as fit on the GPU at once, no more than there are tiles.
inline unsigned tile_grid(const void *func, int64_t tiles_max) {
    return wave_grid(func, kThreads, 0, tiles_max);
}

// The layout depends on the scratch's capacity only, never on the call, so a
// status word is only ever read at a place where status words are written.
template <typename T>
inline ScanState<T> scan_state(const Scratch &tmp, int64_t tiles_max) {
    if (tiles_max > tmp.tiles_cap) throw CudaError{cudaErrorInvalidValue, "scan longer than the scratch"};
    const size_t stride = ((size_t)tmp.tiles_cap * sizeof(int64_t) + 255) & ~(size_t)255;
    ScanState<T> st;
    st.flag = reinterpret_cast<uint32_t *>(tmp.scan);
    st.agg = reinterpret_cast<T *>(tmp.scan + stride);
    st.incl = reinterpret_cast<T *>(tmp.scan + 2 * stride);
    st.ctr = tmp.ticket;
    st.err = tmp.err;
    st.epoch = tmp.epoch;
    st.flags_cap = tmp.tiles_cap;
    return st;
}

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

}  // namespace prim
}  // namespace upr
