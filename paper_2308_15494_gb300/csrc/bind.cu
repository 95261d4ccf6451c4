// Static schedules of a binding, built on the device from the packed row
// offsets (the hub chunks, the table build's tiles, the hashed rows' slot
// offsets and the hub list), in two passes over fixed segments of
// kSchedSegment nodes: one thread per segment counts, a one-CTA scan turns
// the counts into offsets and totals (read back to size the arena), and the
// same walk writes.  A segment boundary also ends a tile; rows are
// independent, so any such tiling gives the same table.
#include "prim.cuh"

namespace upr {
namespace {

using namespace prim;

// Walks the nodes [v0, v1) of one segment: hub chunks (8192 entries of one
// node of degree > kHubDegree), tiles (runs of consecutive nodes with at most
// tile_nodes rows and kTileEntries non-hub entries, a hub closing its tile)
// and the hashed rows' slots (a power of two >= min(k, 2 deg) + 1, or
// min(k, deg) + 1 with sp_mode 3).  With out == nullptr it only counts.
struct SchedOut {
    HubChunk *chunks;
    TableTile *tiles;
    int64_t *sp_off;
    int32_t *hubs;
};

// Offsets outside [0, m] or decreasing (an input the check rejects) count as
// empty rows, so that no walk runs long on them.
__device__ __forceinline__ int64_t row_len(const int64_t *__restrict__ x, int64_t v, int64_t m) {
    const int64_t e0 = x[v], e1 = x[v + 1];
    return (e0 < 0 || e1 < e0 || e1 > m) ? 0 : e1 - e0;
}

__device__ __forceinline__ void sched_walk(const int64_t *__restrict__ x, int64_t m, int64_t v0, int64_t v1,
                                           int tile_nodes,
                                           int sp_mode, int32_t k, const SchedOut *out, int64_t base_chunk,
                                           int64_t base_tile, int64_t base_sp, int64_t base_hub, int64_t *n_chunk,
                                           int64_t *n_tile, int64_t *n_sp, int64_t *n_hub, int64_t *sp_cap_max) {
    constexpr int64_t kTileEntries = 4096;
    int64_t chunks = 0, tiles = 0, sp = 0, hubs = 0, cap_max = 1;
    for (int64_t v = v0; v < v1; v++) {
        const int64_t d = row_len(x, v, m), e0 = x[v], e1 = e0 + d;
        if (d > kHubDegree) {
            if (out) out->hubs[base_hub + hubs] = (int32_t)v;
            hubs++;
            for (int64_t b = e0; b < e1; b += 8192) {
                if (out) out->chunks[base_chunk + chunks] = HubChunk{(int32_t)v, 0, b, min(b + 8192, e1)};
                chunks++;
            }
        }
        if (sp_mode) {
            const int64_t want = min((int64_t)k, sp_mode == 3 ? d : 2 * d) + 1;
            int64_t cap = 1;
            while (cap < want) cap <<= 1;
            if (out) out->sp_off[v] = base_sp + sp;
            sp += cap;
            if (d <= kHubDegree) cap_max = max(cap_max, cap);
        }
    }
    if (tile_nodes) {
        int64_t v = v0;
        while (v < v1) {
            TableTile tl{x[v], x[v], (int32_t)v, (int32_t)v};
            while (v < v1 && tl.v1 - tl.v0 < tile_nodes) {
                const int64_t d = row_len(x, v, m);
                if (d > kHubDegree) { tl.v1 = (int32_t)(++v); break; }     // hub: row zero here, last in tile
                if (tl.e1 + d - tl.e0 > kTileEntries && tl.v1 > tl.v0) break;
                tl.e1 += d;
                tl.v1 = (int32_t)(++v);
            }
            if (out) out->tiles[base_tile + tiles] = tl;
            tiles++;
        }
    }
    *n_chunk = chunks;
    *n_tile = tiles;
    *n_sp = sp;
    *n_hub = hubs;
    *sp_cap_max = cap_max;
}

// Per segment s: cnt[4 s + 0..3] = chunks, tiles, sparse slots, hubs; the
// largest non-hub row capacity into *cap_max.
__global__ void k_sched_count(const int64_t *__restrict__ x, int64_t n, int64_t m, int64_t nseg, int tile_nodes,
                              int sp_mode, int32_t k, int64_t *__restrict__ cnt,
                              unsigned long long *__restrict__ cap_max) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const int64_t v0 = s * kSchedSegment, v1 = min(n, v0 + kSchedSegment);
    int64_t c, t, sp, h, cm;
    sched_walk(x, m, v0, v1, tile_nodes, sp_mode, k, nullptr, 0, 0, 0, 0, &c, &t, &sp, &h, &cm);
    cnt[4 * s + 0] = c;
    cnt[4 * s + 1] = t;
    cnt[4 * s + 2] = sp;
    cnt[4 * s + 3] = h;
    atomicMax(cap_max, (unsigned long long)cm);
}

// Exclusive prefix of each of the four count columns in place, one CTA;
// tot[0..3] = the totals.
__global__ void __launch_bounds__(kThreads) k_sched_scan(int64_t *__restrict__ cnt, int64_t nseg,
                                                         int64_t *__restrict__ tot) {
    __shared__ int64_t s_warp[kWarps];
    for (int col = 0; col < 4; col++) {
        int64_t carry = 0;
        for (int64_t base = 0; base < nseg; base += kThreads) {
            const int64_t i = base + threadIdx.x;
            const int64_t v = i < nseg ? cnt[4 * i + col] : 0;
            int64_t total;
            const int64_t pre = block_exclusive<OpSum>(v, s_warp, &total);
            if (i < nseg) cnt[4 * i + col] = carry + pre;
            carry += total;
        }
        if (threadIdx.x == 0) tot[col] = carry;
    }
}

__global__ void k_sched_write(const int64_t *__restrict__ x, int64_t n, int64_t m, int64_t nseg, int tile_nodes,
                              int sp_mode, int32_t k, const int64_t *__restrict__ off, SchedOut out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const int64_t v0 = s * kSchedSegment, v1 = min(n, v0 + kSchedSegment);
    int64_t c, t, sp, h, cm;
    sched_walk(x, m, v0, v1, tile_nodes, sp_mode, k, &out, off[4 * s + 0], off[4 * s + 1], off[4 * s + 2],
               off[4 * s + 3], &c, &t, &sp, &h, &cm);
    if (sp_mode && v1 == n) out.sp_off[n] = off[4 * s + 2] + sp;
}

// One graph's offsets: x[0] = 0, x[n] = m, non-decreasing; *bad = 1 otherwise.
__global__ void k_xadj_check(const int64_t *__restrict__ x, int64_t n, int64_t m, int32_t *__restrict__ bad) {
    UPR_FOR(v, n) if (x[v + 1] < x[v]) *bad = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (x[0] != 0 || x[n] != m)) *bad = 1;
}

// A batch's packed offsets: node j of graph i (noff[i] <= j < noff[i + 1])
// takes graph i's own offset raw[noff[i] + i + (j - noff[i])] plus eoff[i];
// out[n] = eoff[ng].  *bad = 1 unless each graph's offsets start at 0, end at
// its entry count and do not decrease.
__global__ void k_xadj_pack(const int64_t *__restrict__ raw, const int64_t *__restrict__ noff,
                            const int64_t *__restrict__ eoff, int32_t ng, int64_t n, int64_t *__restrict__ out,
                            int32_t *__restrict__ bad) {
    UPR_FOR(j, n) {
        int32_t lo = 0, hi = ng - 1;            // the last graph i with noff[i] <= j
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (noff[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int64_t p = noff[lo] + lo + (j - noff[lo]);
        const int64_t a = raw[p], b = raw[p + 1];
        out[j] = a + eoff[lo];
        if (b < a) *bad = 1;
        if (j == noff[lo] && a != 0) *bad = 1;
        if (j + 1 == noff[lo + 1] && b != eoff[lo + 1] - eoff[lo]) *bad = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = eoff[ng];
}

// Copies of many host arrays in one launch: the arrays are page-locked host
// memory, which the GPU reads directly; segment i moves len elements from
// src to dst + off (segments of at most kGatherChunk elements, one per CTA
// at a time, eight loads in flight per thread).
template <typename T>
__global__ void __launch_bounds__(256) k_gather_host(const HostSeg *__restrict__ segs, int64_t nseg,
                                                     T *__restrict__ dst) {
    for (int64_t i = blockIdx.x; i < nseg; i += gridDim.x) {
        const HostSeg sg = segs[i];
        const T *src = static_cast<const T *>(sg.src);
        T *out = dst + sg.off;
        for (int64_t b = 0; b < sg.len; b += 8 * 256) {
            T x[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int64_t e = b + u * 256 + threadIdx.x;
                if (e < sg.len) x[u] = src[e];
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int64_t e = b + u * 256 + threadIdx.x;
                if (e < sg.len) out[e] = x[u];
            }
        }
    }
}

}  // namespace

void gather_host(const HostSeg *d_segs, int64_t nseg, size_t elem, void *dst, cudaStream_t s) {
    if (nseg <= 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>(nseg, (int64_t)device_sm_count() * 8);
    if (elem == 8) k_gather_host<int64_t><<<grid, 256, 0, s>>>(d_segs, nseg, static_cast<int64_t *>(dst));
    else k_gather_host<int32_t><<<grid, 256, 0, s>>>(d_segs, nseg, static_cast<int32_t *>(dst));
    UPR_LAUNCH_CHECK();
}

void xadj_pack(const int64_t *raw, const int64_t *noff, const int64_t *eoff, int32_t ng, int64_t n, int64_t *out,
               int32_t *bad, cudaStream_t s) {
    k_xadj_pack<<<grid_for(std::max<int64_t>(n, 1)), 256, 0, s>>>(raw, noff, eoff, ng, n, out, bad);
    UPR_LAUNCH_CHECK();
}

int64_t sched_segments(int64_t n) { return n > 0 ? ceil_div(n, kSchedSegment) : 0; }

void sched_count(const int64_t *xadj, int64_t n, int64_t m, int tile_nodes, int sp_mode, int32_t k, int64_t *cnt,
                 int64_t *tot, unsigned long long *cap_max, cudaStream_t s) {
    const int64_t nseg = sched_segments(n);
    UPR_CUDA(cudaMemsetAsync(cap_max, 0, sizeof(unsigned long long), s));
    if (nseg == 0) {
        UPR_CUDA(cudaMemsetAsync(tot, 0, 4 * sizeof(int64_t), s));
        return;
    }
    k_sched_count<<<(unsigned)ceil_div(nseg, 128), 128, 0, s>>>(xadj, n, m, nseg, tile_nodes, sp_mode, k, cnt,
                                                                cap_max);
    UPR_LAUNCH_CHECK();
    k_sched_scan<<<1, kThreads, 0, s>>>(cnt, nseg, tot);
    UPR_LAUNCH_CHECK();
}

void sched_write(const int64_t *xadj, int64_t n, int64_t m, int tile_nodes, int sp_mode, int32_t k,
                 const int64_t *off, HubChunk *chunks, TableTile *tiles, int64_t *sp_off, int32_t *hubs,
                 cudaStream_t s) {
    const int64_t nseg = sched_segments(n);
    if (nseg == 0) return;
    k_sched_write<<<(unsigned)ceil_div(nseg, 128), 128, 0, s>>>(xadj, n, m, nseg, tile_nodes, sp_mode, k, off,
                                                                SchedOut{chunks, tiles, sp_off, hubs});
    UPR_LAUNCH_CHECK();
}

void xadj_check(const int64_t *xadj, int64_t n, int64_t m, int32_t *bad, cudaStream_t s) {
    k_xadj_check<<<grid_for(std::max<int64_t>(n, 1)), 256, 0, s>>>(xadj, n, m, bad);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
