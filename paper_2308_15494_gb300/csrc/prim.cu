// Device-wide primitives written for this library: scans (sum / max),
// stable LSD radix sort of (64-bit key, 32-bit value) pairs and stable
// compaction by flags (of the indices, or of values, in place if wanted).  Every ordered list the refinement produces comes out of these,
// never out of the order of atomic operations, so results are deterministic.
//
// Element counts may live in device memory (Count::d) next to a static upper
// bound (Count::max): grids are sized by the bound and every kernel reads the
// actual count, so a step can be enqueued without the host knowing how long
// the previous step's output was.
//
// Scan and compaction tiles are 4096 items (256 threads x 16 items), radix
// tiles 2048 (256 x 8; the tile ranking's shared memory grows with the
// items).  Scans and compaction are single-pass with decoupled look-back: a
// CTA takes the next tile index from an atomic counter, publishes its tile
// total, then walks back over the
// preceding tiles' published totals until it meets an inclusive prefix, and
// publishes its own.  A tile only waits for tiles that running CTAs took
// earlier, so the waits end whatever the scheduling; every wait is bounded
// anyway and records a timeout in an error word instead of spinning on.
// Status words carry the call's epoch, so nothing has to be cleared between
// calls: the epoch is a device word that the taking-part CTAs read when they
// start and the last of them advances when it finishes, so calls replayed
// from a CUDA graph get fresh epochs exactly like calls launched one by one.  A radix
// pass is histogram -> single-pass scan of the digit-major histogram ->
// stable scatter; inside a tile, equal digits are ranked in item order with
// __match_any_sync per warp and a per-digit prefix over the 8 warps.  Lists
// of at most one tile are sorted in one CTA.
#include "prim.cuh"

namespace upr {
namespace {

using namespace prim;
// Single-pass scan (see the top of the file).  A one-tile list needs neither
// the tile counters nor the look-back.
// Items per thread of the scans and compactions (tiles of kThreads * kPI).
constexpr int kPI = 16;
constexpr int kPTile = kThreads * kPI;
__device__ __forceinline__ int64_t ptiles_of(int64_t n) { return (n + kPTile - 1) / kPTile; }

template <typename Op, typename T, typename TIn>
__device__ __forceinline__ void scan_tile(const TIn *in, T *out, int64_t n, int inclusive, int vec,
                                          const ScanState<T> &st, uint32_t epoch, int64_t tile, bool alone,
                                          T *s_warp, T *s_excl) {
    TIn x[kPI];
    load_items(in, tile * kPTile, n, (vec & 1) != 0, x);
    T acc = Op::template identity<T>();
#pragma unroll
    for (int j = 0; j < kPI; j++) acc = Op::template apply<T>(acc, (T)x[j]);
    T total;
    const T pre = block_exclusive<Op>(acc, s_warp, &total);
    if (alone) {
        if (threadIdx.x == 0) *s_excl = Op::template identity<T>();
    } else if (threadIdx.x < 32) {
        const T e = lookback<Op>(st, tile, total, epoch);
        if (threadIdx.x == 0) *s_excl = e;
    }
    __syncthreads();
    T run = Op::template apply<T>(*s_excl, pre);
    T y[kPI];
#pragma unroll
    for (int j = 0; j < kPI; j++) {
        const T nxt = Op::template apply<T>(run, (T)x[j]);
        y[j] = inclusive ? nxt : run;
        run = nxt;
    }
    store_items(out, tile * kPTile, n, (vec & 2) != 0, y);
    __syncthreads();
}

template <typename Op, typename T, typename TIn>
__global__ void __launch_bounds__(kThreads) k_scan(const TIn *in, T *out, const int32_t *__restrict__ d_n,
                                                   int64_t n_max, int inclusive, int vec, ScanState<T> st) {
    __shared__ T s_warp[kWarps];
    __shared__ T s_excl;
    __shared__ uint32_t s_tile;
    const int64_t n = count_of(d_n, n_max);
    const int64_t tiles = ptiles_of(n);
    const unsigned parts = participants(tiles);
    if (blockIdx.x >= parts) return;
    if (tiles == 1) {
        scan_tile<Op>(in, out, n, inclusive, vec, st, 0u, 0, true, s_warp, &s_excl);
        return;
    }
    const uint32_t epoch = call_epoch(st);
    for (;;) {
        const int64_t tile = next_tile(st.ctr, &s_tile);
        if (tile >= tiles) break;
        scan_tile<Op>(in, out, n, inclusive, vec, st, epoch, tile, false, s_warp, &s_excl);
    }
    finish_tiles(st, parts, epoch);
}




template <typename Op, typename T, typename TIn>
void scan_impl(const TIn *in, T *out, Count n, bool inclusive, Scratch tmp, cudaStream_t s) {
    if (n.max <= 0) return;
    const int vin = aligned16(in) ? 1 : 0;
    const int vio = vin | (aligned16(out) ? 2 : 0);
    const int64_t tiles_max = ceil_div(n.max, kPTile);
    k_scan<Op, T, TIn><<<tile_grid((const void *)k_scan<Op, T, TIn>, tiles_max), kThreads, 0, s>>>(in, out, n.d, n.max, inclusive ? 1 : 0, vio,
                                                                  scan_state<T>(tmp, tiles_max));
    UPR_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ compaction
// Single pass: a tile counts its set flags, takes its offset by look-back and
// every thread writes the indices of its set flags (tile order, then thread
// order, then item order = index order); the last tile writes the total.
__device__ __forceinline__ void compact_tile(const int32_t *flags, int64_t n, int64_t tiles, int32_t *out,
                                             int32_t *d_count, int vec, const ScanState<int32_t> &st,
                                             uint32_t epoch, int64_t tile, bool alone, int32_t *s_warp,
                                             int32_t *s_excl) {
    int32_t x[kPI];
    load_items(flags, tile * kPTile, n, vec != 0, x);
    int32_t c = 0;
#pragma unroll
    for (int j = 0; j < kPI; j++) c += x[j] != 0;
    int32_t total;
    const int32_t pre = block_exclusive<OpSum>(c, s_warp, &total);
    if (threadIdx.x < 32) {
        const int32_t e = alone ? 0 : lookback<OpSum>(st, tile, total, epoch);
        if (threadIdx.x == 0) {
            *s_excl = e;
            if (tile == tiles - 1) *d_count = e + total;
        }
    }
    __syncthreads();
    int32_t pos = *s_excl + pre;
    const int64_t first = tile * kPTile + (int64_t)threadIdx.x * kPI;
#pragma unroll
    for (int j = 0; j < kPI; j++)
        if (x[j]) out[pos++] = (int32_t)(first + j);
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_compact(const int32_t *__restrict__ flags, const int32_t *__restrict__ d_n,
                                                      int64_t n_max, int32_t *__restrict__ out,
                                                      int32_t *__restrict__ d_count, int vec, ScanState<int32_t> st) {
    __shared__ int32_t s_warp[kWarps];
    __shared__ int32_t s_excl;
    __shared__ uint32_t s_tile;
    const int64_t n = count_of(d_n, n_max);
    const int64_t tiles = ptiles_of(n);
    if (tiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) *d_count = 0;
    const unsigned parts = participants(tiles);
    if (blockIdx.x >= parts) return;
    if (tiles == 1) {
        compact_tile(flags, n, tiles, out, d_count, vec, st, 0u, 0, true, s_warp, &s_excl);
        return;
    }
    const uint32_t epoch = call_epoch(st);
    for (;;) {
        const int64_t tile = next_tile(st.ctr, &s_tile);
        if (tile >= tiles) break;
        compact_tile(flags, n, tiles, out, d_count, vec, st, epoch, tile, false, s_warp, &s_excl);
    }
    finish_tiles(st, parts, epoch);
}

// Compaction of values: out[j] = vals[i] for the j-th set flag i, in index
// order.  out may be vals itself: a tile loads its flags and values before it
// publishes its count, writes only after its offset is known (so after every
// earlier tile has published, hence loaded), and its output range
// [offset, offset + count) ends within its own input range.
__device__ __forceinline__ void compact_values_tile(const int32_t *flags, const int32_t *vals, int64_t n,
                                                    int64_t tiles, int32_t *out, int32_t *d_count, int vec,
                                                    const ScanState<int32_t> &st, uint32_t epoch, int64_t tile,
                                                    bool alone, int32_t *s_warp, int32_t *s_excl) {
    int32_t x[kPI], y[kPI];
    load_items(flags, tile * kPTile, n, (vec & 1) != 0, x);
    load_items(vals, tile * kPTile, n, (vec & 2) != 0, y);
    int32_t c = 0;
#pragma unroll
    for (int j = 0; j < kPI; j++) c += x[j] != 0;
    int32_t total;
    const int32_t pre = block_exclusive<OpSum>(c, s_warp, &total);
    if (threadIdx.x < 32) {
        const int32_t e = alone ? 0 : lookback<OpSum>(st, tile, total, epoch);
        if (threadIdx.x == 0) {
            *s_excl = e;
            if (tile == tiles - 1) *d_count = e + total;
        }
    }
    __syncthreads();
    int32_t pos = *s_excl + pre;
#pragma unroll
    for (int j = 0; j < kPI; j++)
        if (x[j]) out[pos++] = y[j];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_compact_values(const int32_t *__restrict__ flags, const int32_t *vals,
                                                             const int32_t *__restrict__ d_n, int64_t n_max,
                                                             int32_t *out, int32_t *__restrict__ d_count, int vec,
                                                             ScanState<int32_t> st) {
    __shared__ int32_t s_warp[kWarps];
    __shared__ int32_t s_excl;
    __shared__ uint32_t s_tile;
    const int64_t n = count_of(d_n, n_max);
    const int64_t tiles = ptiles_of(n);
    if (tiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) *d_count = 0;
    const unsigned parts = participants(tiles);
    if (blockIdx.x >= parts) return;
    if (tiles == 1) {
        compact_values_tile(flags, vals, n, tiles, out, d_count, vec, st, 0u, 0, true, s_warp, &s_excl);
        return;
    }
    const uint32_t epoch = call_epoch(st);
    for (;;) {
        const int64_t tile = next_tile(st.ctr, &s_tile);
        if (tile >= tiles) break;
        compact_values_tile(flags, vals, n, tiles, out, d_count, vec, st, epoch, tile, false, s_warp, &s_excl);
    }
    finish_tiles(st, parts, epoch);
}

// ------------------------------------------------------------------ radix sort

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
    const size_t tiles = (size_t)ceil_div(n > 0 ? n : 1, kTile);
    return 3 * ((tiles * sizeof(int64_t) + 255) & ~(size_t)255);
}

size_t radix_temp_bytes(int64_t n) {
    const size_t tiles = (size_t)ceil_div(n > 0 ? n : 1, kTile);
    return ((tiles * kBins + 64) * sizeof(int32_t) + 255) & ~(size_t)255;
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
    if (tiles_max > tmp.tiles_cap) throw CudaError{cudaErrorInvalidValue, "sort longer than the scratch"};
    // digit-major per-tile histograms (kBins x tiles), scanned in place
    int32_t *hist = reinterpret_cast<int32_t *>(tmp.mem);
    int32_t *d_hist_n = hist + (size_t)kBins * tmp.tiles_cap;
    // one full wave each (tiles are assigned by CTA index)
    const unsigned grid_h = wave_grid((const void *)k_radix_hist, kThreads, 0, tiles_max);
    const unsigned grid_s = wave_grid((const void *)k_radix_scatter, kThreads, 0, tiles_max);
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; p++) {
        k_radix_hist<<<grid_h, kThreads, 0, s>>>(ka, n.d, n.max, 8 * p, hist, d_hist_n);
        UPR_LAUNCH_CHECK();
        scan_impl<OpSum, int32_t, int32_t>(hist, hist, Count{d_hist_n, (int64_t)kBins * tiles_max}, false, tmp, s);
        k_radix_scatter<<<grid_s, kThreads, 0, s>>>(ka, va, kb, vb, n.d, n.max, 8 * p, hist);
        UPR_LAUNCH_CHECK();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return alt;
}

void select_flags(const int32_t *flags, int32_t *out_idx, int32_t *d_count, Count n, Scratch tmp, cudaStream_t s) {
    if (n.max <= 0) { UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s)); return; }
    const int vec = aligned16(flags) ? 1 : 0;
    const int64_t tiles_max = ceil_div(n.max, kPTile);
    k_compact<<<tile_grid((const void *)k_compact, tiles_max), kThreads, 0, s>>>(flags, n.d, n.max, out_idx, d_count, vec,
                                                        scan_state<int32_t>(tmp, tiles_max));
    UPR_LAUNCH_CHECK();
}

void select_values(const int32_t *flags, const int32_t *vals, int32_t *out, int32_t *d_count, Count n, Scratch tmp,
                   cudaStream_t s) {
    if (n.max <= 0) { UPR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s)); return; }
    const int vec = (aligned16(flags) ? 1 : 0) | (aligned16(vals) ? 2 : 0);
    const int64_t tiles_max = ceil_div(n.max, kPTile);
    k_compact_values<<<tile_grid((const void *)k_compact_values, tiles_max), kThreads, 0, s>>>(
        flags, vals, n.d, n.max, out, d_count, vec, scan_state<int32_t>(tmp, tiles_max));
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
