// Step (b): rebalancing availability, slots and bucket weights (Alg. 1,
// Sec. 4.3), each boundary node's best move by gain minus penalty
// (Alg. 1), penalties with the inflow of better-ranked candidates,
// the global move order M (Sec. 4.4), and the application of M.
#include "kernels.h"

namespace upr {
namespace {

// 3^i for i = 0..40 (3^40 < 2^64).
__constant__ uint64_t c_pow3[41];

int sm_count_sel() {
    static int cnt = 0;
    if (!cnt) {
        int dev = 0;
        UPR_CUDA(cudaGetDevice(&dev));
        UPR_CUDA(cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev));
    }
    return cnt;
}

void ensure_pow3() {
    static int done_dev = -1;
    int dev = 0;
    UPR_CUDA(cudaGetDevice(&dev));
    if (done_dev == dev) return;
    uint64_t p[41];
    p[0] = 1;
    for (int i = 1; i <= 40; i++) p[i] = p[i - 1] * 3;
    UPR_CUDA(cudaMemcpyToSymbol(c_pow3, p, sizeof(p)));
    done_dev = dev;
}

// (3/2)^s * c >= omega, exactly (p3 = the powers of 3, in shared memory).
__device__ __forceinline__ bool slot_ok(int s, uint64_t omega, uint64_t c, const uint64_t *p3) {
    if (s >= 0) return (u128)p3[s] * c >= ((u128)omega << s);
    return ((u128)c << (-s)) >= (u128)p3[-s] * omega;
}

// Smallest s in [kSlotLo, kSlotHi] with (3/2)^s >= omega / c (kSlotHi if none).
// A single-precision logarithm gives a first guess; the exact test, monotone
// in s, then moves it to the answer (one or two tests in practice).
__device__ __forceinline__ int slot_of(uint64_t omega, uint64_t c, const uint64_t *p3) {
    if (omega == 0) return kSlotLo;
    const float guess = (log2f((float)omega) - log2f((float)c)) * 1.7095113f;   // 1 / log2(3/2)
    int s = guess > (float)kSlotHi ? kSlotHi : guess < (float)kSlotLo ? kSlotLo : (int)ceilf(guess);
    while (s > kSlotLo && slot_ok(s - 1, omega, c, p3)) s--;
    while (s < kSlotHi && !slot_ok(s, omega, c, p3)) s++;
    return s;
}

// Penalty of moving weight cu into block b that would then exceed L_max by x;
// -1 = forbidden (no slot's cumulative weight covers x).
// An excess of exactly 1 (every overfilling move of a unit-weight node) takes
// the block's first non-empty slot without a search.
__device__ __forceinline__ int64_t penalty(const Penalty &p, int32_t b, int64_t x, int64_t cu) {
    if (x <= 0) return 0;
    int lo;
    if (x == 1) {
        lo = p.first[b];
        if (lo < 0) return -1;
    } else {
        const int64_t *row = p.PW + (int64_t)b * kSlots;
        if (row[kSlots - 1] < x) return -1;
        lo = 0;
        int hi = kSlots - 1;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (row[mid] >= x) hi = mid; else lo = mid + 1;
        }
    }
    return (int64_t)(((u128)(uint64_t)cu * (uint64_t)p.F[lo]) >> kQ);
}

__global__ void k_buckets(const int32_t *__restrict__ part, const int32_t *__restrict__ W,
                          const int32_t *__restrict__ wI, const int32_t *__restrict__ vwgt, int64_t n, int32_t k,
                          int32_t kmask, int32_t K, int32_t t_num, int32_t t_den, unsigned long long *__restrict__ BW,
                          int use_shared, int8_t *__restrict__ avail_out, int32_t *__restrict__ slot_out,
                          SparseRows sp, unsigned long long *__restrict__ cut2) {
    extern __shared__ unsigned long long s_bw[];
    __shared__ uint64_t s_p3[41];
    for (int i = threadIdx.x; i < 41; i += blockDim.x) s_p3[i] = c_pow3[i];
    const int bins = K * kSlots;
    __syncthreads();
    if (use_shared) {
        // (unit weights: 32-bit counts, half the words)
        unsigned int *s_w32 = reinterpret_cast<unsigned int *>(s_bw);
        for (int i = threadIdx.x; i < (vwgt ? 2 : 1) * bins; i += blockDim.x) s_w32[i] = 0;
        __syncthreads();
    }
    long long out_w = 0;      // weight of the edges leaving v's block, summed over this thread's nodes
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = part[v];
        const int32_t wIv = wI[v];
        // an isolated node's row is zero: no gather
        const int64_t own = wIv == 0 ? 0
                            : sp.on() ? sp_get(sp, v, blk_local(a, k, kmask))
                                      : W[v * (int64_t)k + blk_local(a, k, kmask)];
        const int64_t c = vwgt ? vwgt[v] : 1;
        const bool av = (int64_t)t_den * own >= (int64_t)t_num * (int64_t)wIv;
        out_w += (long long)wIv - own;
        const int s = slot_of((uint64_t)own, (uint64_t)c, s_p3);
        if (av) {
            if (use_shared && !vwgt)      // unit weights: a CTA's counts fit 32-bit shared-memory atomics
                atomicAdd(reinterpret_cast<unsigned int *>(s_bw) + a * kSlots + (s - kSlotLo), 1u);
            else
                atomicAdd(&(use_shared ? s_bw : BW)[a * kSlots + (s - kSlotLo)], (unsigned long long)c);
        }
        if (avail_out) avail_out[v] = av ? 1 : 0;
        if (slot_out) slot_out[v] = s;
    }
    if (use_shared) {
        __syncthreads();
        if (!vwgt) {
            const unsigned int *s_bw32 = reinterpret_cast<const unsigned int *>(s_bw);
            for (int i = threadIdx.x; i < bins; i += blockDim.x)
                if (s_bw32[i]) atomicAdd(&BW[i], (unsigned long long)s_bw32[i]);
        } else {
            for (int i = threadIdx.x; i < bins; i += blockDim.x)
                if (s_bw[i]) atomicAdd(&BW[i], s_bw[i]);
        }
    }
    if (cut2) {
        __shared__ long long s_cw[8];
        out_w = warp_sum(out_w);
        if ((threadIdx.x & 31) == 0) s_cw[threadIdx.x >> 5] = out_w;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_cw[w];
            if (t) atomicAdd(&cut2[blockIdx.x % kCutParts], (unsigned long long)t);
        }
    }
}

// cut2[0 .. kCutParts): partial sums of twice the cut (spread over many words
// so that the CTAs' atomics do not queue on one address); cut2[kCutParts] =
// their total; cut = half of it.
__global__ void __launch_bounds__(kCutParts) k_half_cut(unsigned long long *__restrict__ cut2,
                                                        int64_t *__restrict__ cut) {
    __shared__ unsigned long long s_w[kCutParts / 32];
    unsigned long long v = cut2[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kCutParts / 32; w++) t += s_w[w];
        cut2[kCutParts] = t;
        cut[0] = (int64_t)(t / 2);
    }
}

__global__ void k_bucket_prefix(const int64_t *__restrict__ BW, int64_t *__restrict__ PW, int8_t *__restrict__ first,
                                int32_t K) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= K) return;
    int64_t acc = 0;
    int f = -1;
    for (int l = 0; l < kSlots; l++) {
        acc += BW[b * kSlots + l];
        PW[b * kSlots + l] = acc;
        if (f < 0 && acc >= 1) f = l;
    }
    first[b] = (int8_t)f;
}

// G lanes per node: best target by (gain - penalty) among adjacent blocks,
// ties to the smaller block id; candidate iff the score is positive and v is
// a boundary node.
template <int G>
__global__ void __launch_bounds__(256) k_select(const GraphDev g, const int32_t *__restrict__ part,
                                                const int32_t *__restrict__ W, Penalty pen,
                                                int32_t *__restrict__ cand_tgt, int64_t *__restrict__ cand_s0,
                                                int32_t *__restrict__ cand_gain, int32_t *__restrict__ flags) {
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    const int64_t n = g.n;
    const int32_t k = g.k;
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n; base += (int64_t)gridDim.x * kGroups) {
        const int64_t v = base + gid;
        const bool active = v < n;
        int64_t best = 0;
        int32_t bt = -1, bg = 0, b0 = 0;
        if (active) {
            const int32_t ag = part[v];
            const int32_t a = blk_local(g, ag);
            b0 = ag - a;
            const int32_t *row = W + v * (int64_t)k;
            const int32_t own = row[a];
            if (own < g.wI[v]) {
                const int64_t c = g.vwgt ? g.vwgt[v] : 1;
                for (int b = gl; b < k; b += G) {
                    const int32_t w = row[b];
                    if (b == a || w <= 0) continue;
                    const int64_t gain = (int64_t)w - own;
                    const int32_t gb = b0 + b;
                    const int64_t p = penalty(pen, gb, pen.C[gb] + c - pen.Lb[gb], c);
                    if (p < 0) continue;
                    const int64_t sc = gain - p;
                    if (bt < 0 || sc > best) { best = sc; bt = b; bg = (int32_t)gain; }
                }
            }
        }
        int64_t s = best;
        int32_t id = bt;
        group_argmax<G>(s, id);
        // lanes own disjoint blocks, so exactly one lane holds the winner's gain
        const int32_t gsel = group_sum<G>((id >= 0 && bt == id) ? bg : 0);
        if (active && gl == 0) {
            const bool cand = id >= 0 && s > 0;
            cand_tgt[v] = cand ? b0 + id : -1;
            cand_s0[v] = cand ? s : 0;
            cand_gain[v] = cand ? gsel : 0;
            flags[v] = cand ? 1 : 0;
        }
    }
}

__device__ __forceinline__ int32_t int4_get(const int4 &x, int c) {
    return c == 0 ? x.x : c == 1 ? x.y : c == 2 ? x.z : x.w;
}

// Vectorised form of k_select for k % 4 == 0, k <= 4*G*CH: lane gl of a group
// holds blocks [4(gl + G j), 4(gl + G j) + 4) of the row in one int4 per j.
// With one graph (BATCH false) the per-block slack L_max - C[b] and the
// factors F_r (and, when they fit, the bucket prefixes) are staged in shared
// memory; in a batch each node reads its own graph's blocks from global
// memory.  A move into a block with room for it costs no penalty and needs no
// search.
template <int G, int CH, bool EXACT, bool BATCH, bool PACK = false>
__global__ void __launch_bounds__(256) k_select_vec(const GraphDev g, const int32_t *__restrict__ part,
                                                    const int32_t *__restrict__ W, Penalty pen, int smem_pw,
                                                    int32_t *__restrict__ cand_tgt, int64_t *__restrict__ cand_s0,
                                                    int32_t *__restrict__ cand_gain, int32_t *__restrict__ flags) {
    // s_slack[b] = L_max - C[b] clamped to 2^31 - 1 (blocks start balanced, so
    // it is >= 0): a node of weight c < 2^31 overfills b iff c > s_slack[b],
    // and then x = c - s_slack[b] is exact.
    extern __shared__ int64_t s_mem[];
    const int64_t n = g.n;
    const int32_t k = g.k;
    int64_t *s_F = s_mem;
    int64_t *s_PW = s_mem + kSlots;
    int32_t *s_slack = reinterpret_cast<int32_t *>(s_mem + kSlots + (smem_pw ? (size_t)k * kSlots : 0));
    int8_t *s_first = reinterpret_cast<int8_t *>(s_slack + k);
    if (!BATCH)
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const int64_t sl = pen.Lb[i] - pen.C[i];
            s_slack[i] = (int32_t)(sl > 0x7fffffffLL ? 0x7fffffffLL : sl);
            s_first[i] = pen.first[i];
        }
    for (int i = threadIdx.x; i < kSlots; i += blockDim.x) s_F[i] = pen.F[i];
    if (!BATCH && smem_pw)
        for (int i = threadIdx.x; i < k * kSlots; i += blockDim.x) s_PW[i] = pen.PW[i];
    __syncthreads();
    const int64_t *PW = (!BATCH && smem_pw) ? s_PW : pen.PW;
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    // PACK (unit weights, one graph): a node of weight 1 pays the same
    // penalty p(b) into block b wherever it comes from, so p(b) (-1:
    // forbidden) is fixed for the launch; the lane keeps, per column it
    // scores, a bit "allowed" and the constant (2^kb - 1 - b) - (p(b) << kb)
    const int kb = PACK ? pen.pack_bits : 0;
    const int32_t kmask = (1 << kb) - 1;
    int32_t *s_pen = reinterpret_cast<int32_t *>(s_first + ((k + 3) & ~3));
    uint32_t okm = 0;
    int32_t cst[CH][4];
    if (PACK) {
        for (int b = threadIdx.x; b < k; b += blockDim.x) {
            const int32_t sl = s_slack[b];
            int32_t p = 0;
            if (sl < 1) {
                const int64_t x = 1 - (int64_t)sl;
                int lo;
                if (x == 1) {
                    lo = s_first[b];
                } else {
                    const int64_t *row = PW + (int64_t)b * kSlots;
                    if (row[kSlots - 1] < x) {
                        lo = -1;
                    } else {
                        lo = 0;
                        int hi = kSlots - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (row[mid] >= x) hi = mid; else lo = mid + 1;
                        }
                    }
                }
                if (lo < 0) {
                    p = -1;
                } else {
                    // floor(1 * F / 2^Q); a penalty of at least 2^gb exceeds every gain
                    const uint64_t pp = (uint64_t)s_F[lo] >> kQ;
                    p = pp >= (1ull << pen.gbits) ? -1 : (int32_t)pp;
                }
            }
            s_pen[b] = p;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < CH; j++)
#pragma unroll
            for (int cc = 0; cc < 4; cc++) {
                const int b = 4 * (gl + G * j) + cc;
                const int32_t p = (EXACT || b < k) ? s_pen[b] : -1;
                if (p >= 0) okm |= 1u << (4 * j + cc);
                cst[j][cc] = (kmask - b) - (p >= 0 ? (p << kb) : 0);
            }
    }
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n; base += (int64_t)gridDim.x * kGroups) {
        const int64_t v = base + gid;
        const bool active = v < n;
        int4 r[CH];
        int32_t a = 0, b0 = 0;
        const int4 zero = make_int4(0, 0, 0, 0);
        // (rows are loaded without waiting for omega(I(v)): skipping the zero
        // rows of isolated nodes behind that load measured slower)
        const int32_t wIv = active ? g.wI[v] : 0;
        if (active) {
            const int32_t ag = part[v];
            a = BATCH ? blk_local(g, ag) : ag;
            b0 = ag - a;
            const int4 *row4 = reinterpret_cast<const int4 *>(W + v * (int64_t)k);
#pragma unroll
            for (int j = 0; j < CH; j++) {
                const int q = gl + G * j;
                r[j] = (EXACT || 4 * q < k) ? __ldcs(row4 + q) : zero;
            }
        } else {
#pragma unroll
            for (int j = 0; j < CH; j++) r[j] = zero;
        }
        const int q4 = a >> 2;
        int32_t mine = 0;
#pragma unroll
        for (int j = 0; j < CH; j++)
            if (j == q4 / G) mine = int4_get(r[j], a & 3);
        const int32_t own = __shfl_sync(0xffffffffu, mine, gbase + (q4 % G));
        if (PACK) {
            int32_t pbest = 0;
            if (active && own < wIv) {
                const int32_t ownk = own << kb;
#pragma unroll
                for (int j = 0; j < CH; j++)
#pragma unroll
                    for (int cc = 0; cc < 4; cc++) {
                        const int32_t key = (int4_get(r[j], cc) << kb) - ownk + cst[j][cc];
                        pbest = max(pbest, ((okm >> (4 * j + cc)) & 1u) ? key : 0);
                    }
            }
            for (int o = G / 2; o > 0; o >>= 1) pbest = max(pbest, __shfl_xor_sync(0xffffffffu, pbest, o));
            if (active && gl == 0) {
                // a score >= 1 (key >= 2^kb) makes a candidate
                const bool cand = pbest >= (1 << kb);
                const int32_t b = kmask - (pbest & kmask);
                const int32_t sc = pbest >> kb;
                cand_tgt[v] = cand ? b0 + b : -1;
                cand_s0[v] = cand ? sc : 0;
                cand_gain[v] = cand ? sc + s_pen[b] : 0;
                flags[v] = cand ? 1 : 0;
            }
            continue;
        }
        // Only a positive score makes a candidate and the penalty is never
        // negative, so blocks with gain <= 0 (the own block among them) are
        // skipped and every score kept lies in [1, 2^31).
        int32_t best = 0;
        int32_t bt = -1, bg = 0;
        if (active && own < wIv) {
            const int32_t c = g.vwgt ? g.vwgt[v] : 1;
#pragma unroll
            for (int j = 0; j < CH; j++) {
#pragma unroll
                for (int cc = 0; cc < 4; cc++) {
                    const int b = 4 * (gl + G * j) + cc;
                    const int32_t w = int4_get(r[j], cc);
                    if ((!EXACT && b >= k) || w <= own) continue;
                    const int32_t gain = w - own;
                    int32_t sc = gain;
                    int32_t slack;
                    if (BATCH) {
                        const int64_t sl = pen.Lb[b0 + b] - pen.C[b0 + b];
                        slack = (int32_t)(sl > 0x7fffffffLL ? 0x7fffffffLL : sl);
                    } else {
                        slack = s_slack[b];
                    }
                    if (c > slack) {
                        const int64_t x = (int64_t)c - slack;
                        int lo;
                        if (x == 1) {                               // first non-empty slot
                            lo = BATCH ? pen.first[b0 + b] : s_first[b];
                            if (lo < 0) continue;                   // forbidden
                        } else {
                            const int64_t *row = PW + (int64_t)(b0 + b) * kSlots;
                            if (row[kSlots - 1] < x) continue;      // no slot covers the excess: forbidden
                            lo = 0;
                            int hi = kSlots - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (row[mid] >= x) hi = mid; else lo = mid + 1;
                            }
                        }
                        const int64_t p = (int64_t)(((u128)(uint64_t)c * (uint64_t)s_F[lo]) >> kQ);
                        if (p >= gain) continue;
                        sc = gain - (int32_t)p;
                    }
                    if (bt < 0 || sc > best) { best = sc; bt = b; bg = gain; }
                }
            }
        }
        int32_t sbest = best;
        int32_t id = bt;
        group_argmax32<G>(sbest, id);
        const int32_t gsel = group_sum<G>((id >= 0 && bt == id) ? bg : 0);
        if (active && gl == 0) {
            const bool cand = id >= 0 && sbest > 0;
            cand_tgt[v] = cand ? b0 + id : -1;
            cand_s0[v] = cand ? sbest : 0;
            cand_gain[v] = cand ? gsel : 0;
            flags[v] = cand ? 1 : 0;
        }
    }
}

// Selection over the sparse table: G lanes per node walk the node's slots
// (hash order, so ties compare block ids explicitly); penalties as in
// k_select_vec with the per-block values read from global memory.
template <int G>
__global__ void __launch_bounds__(256) k_select_sparse(const GraphDev g, const int32_t *__restrict__ part,
                                                       Penalty pen, int32_t *__restrict__ cand_tgt,
                                                       int64_t *__restrict__ cand_s0, int32_t *__restrict__ cand_gain,
                                                       int32_t *__restrict__ flags) {
    constexpr int kGroups = 256 / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x % G;
    const int64_t n = g.n;
    const SparseRows &sp = g.sp;
    for (int64_t base = (int64_t)blockIdx.x * kGroups; base < n; base += (int64_t)gridDim.x * kGroups) {
        const int64_t v = base + gid;
        const bool active = v < n;
        int32_t best = 0, bt = -1, bg = 0, b0 = 0;
        if (active) {
            const int32_t ag = part[v];
            const int32_t a = blk_local(g, ag);
            b0 = ag - a;
            const int32_t own = sp_get(sp, v, a);
            if (own < g.wI[v]) {
                const int32_t c = g.vwgt ? g.vwgt[v] : 1;
                for (int64_t i = sp.off[v] + gl; i < sp.off[v + 1]; i += G) {
                    const int2 e = sp.slot[i];
                    if (e.x == kEmpty || e.y <= own) continue;      // gain <= 0 (the own block among them)
                    const int32_t b = e.x, gain = e.y - own;
                    const int64_t sl = pen.Lb[b0 + b] - pen.C[b0 + b];
                    const int32_t slack = (int32_t)(sl > 0x7fffffffLL ? 0x7fffffffLL : sl);
                    int32_t sc = gain;
                    if (c > slack) {
                        const int64_t x = (int64_t)c - slack;
                        int lo;
                        if (x == 1) {
                            lo = pen.first[b0 + b];
                            if (lo < 0) continue;
                        } else {
                            const int64_t *row = pen.PW + (int64_t)(b0 + b) * kSlots;
                            if (row[kSlots - 1] < x) continue;
                            lo = 0;
                            int hi = kSlots - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (row[mid] >= x) hi = mid; else lo = mid + 1;
                            }
                        }
                        const int64_t p = (int64_t)(((u128)(uint64_t)c * (uint64_t)pen.F[lo]) >> kQ);
                        if (p >= gain) continue;
                        sc = gain - (int32_t)p;
                    }
                    if (bt < 0 || sc > best || (sc == best && b < bt)) { best = sc; bt = b; bg = gain; }
                }
            }
        }
        int32_t sbest = best, id = bt;
        group_argmax32<G>(sbest, id);
        const int32_t gsel = group_sum<G>((id >= 0 && bt == id) ? bg : 0);
        if (active && gl == 0) {
            const bool cand = id >= 0 && sbest > 0;
            cand_tgt[v] = cand ? b0 + id : -1;
            cand_s0[v] = cand ? sbest : 0;
            cand_gain[v] = cand ? gsel : 0;
            flags[v] = cand ? 1 : 0;
        }
    }
}

__global__ void k_cand_keys(const int32_t *__restrict__ cand_idx, const int32_t *__restrict__ d_count,
                            const int32_t *__restrict__ cand_tgt, const int64_t *__restrict__ cand_s0, int gbits,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t cnt = *d_count;
    const uint64_t top = (1ull << gbits) - 1ull;
    UPR_FOR(i, cnt) {
        const int32_t v = cand_idx[i];
        keys[i] = ((uint64_t)cand_tgt[v] << gbits) | (top - (uint64_t)cand_s0[v]);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_cand_gather(const int32_t *__restrict__ cand_idx, const uint32_t *__restrict__ order,
                              const int32_t *__restrict__ d_count, const int32_t *__restrict__ cand_tgt,
                              const int32_t *__restrict__ vwgt, int64_t *__restrict__ c_sorted,
                              int32_t *__restrict__ seg_first) {
    const int64_t cnt = *d_count;
    UPR_FOR(j, cnt) {
        const int32_t v = cand_idx[order[j]];
        c_sorted[j] = vwgt ? vwgt[v] : 1;
        const int32_t t = cand_tgt[v];
        if (j == 0 || cand_tgt[cand_idx[order[j - 1]]] != t) seg_first[t] = (int32_t)j;
    }
}

__global__ void k_inflow(const int32_t *__restrict__ cand_idx, const uint32_t *__restrict__ order,
                         const int32_t *__restrict__ d_count, const int32_t *__restrict__ cand_tgt,
                         const int32_t *__restrict__ cand_gain, const int32_t *__restrict__ vwgt,
                         const int64_t *__restrict__ c_excl, const int32_t *__restrict__ seg_first, Penalty pen,
                         int32_t *__restrict__ keep, int64_t *__restrict__ score) {
    const int64_t cnt = *d_count;
    UPR_FOR(j, cnt) {
        const uint32_t i = order[j];
        const int32_t v = cand_idx[i];
        const int32_t t = cand_tgt[v];
        const int64_t c = vwgt ? vwgt[v] : 1;
        const int64_t inflow = c_excl[j] - c_excl[seg_first[t]];
        const int64_t p = penalty(pen, t, pen.C[t] + inflow + c - pen.Lb[t], c);
        const int64_t s = (int64_t)cand_gain[v] - p;
        const bool kp = p >= 0 && s > 0;
        keep[i] = kp ? 1 : 0;
        score[i] = kp ? s : 0;
    }
}

__global__ void k_move_keys(const int32_t *__restrict__ m_idx, const int32_t *__restrict__ d_count,
                            const int64_t *__restrict__ score, int gbits, uint64_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    const int64_t cnt = *d_count;
    UPR_FOR(j, cnt) {
        keys[j] = ((1ull << gbits) - 1ull) - (uint64_t)score[m_idx[j]];
        vals[j] = (uint32_t)j;
    }
}

__global__ void k_apply_moves(const int32_t *__restrict__ cand_idx, const int32_t *__restrict__ m_idx,
                              const uint32_t *__restrict__ order, const int32_t *__restrict__ d_count,
                              const int32_t *__restrict__ cand_tgt, const int64_t *__restrict__ score,
                              const int32_t *__restrict__ vwgt, const int64_t *__restrict__ xadj,
                              const int32_t *__restrict__ part0, int32_t *__restrict__ part,
                              unsigned long long *__restrict__ C, int32_t K, int32_t *__restrict__ M_node,
                              int32_t *__restrict__ M_from, int32_t *__restrict__ M_to,
                              int64_t *__restrict__ M_score, int32_t *__restrict__ m_pos,
                              unsigned long long *__restrict__ deg_sum) {
    extern __shared__ unsigned long long s_delta[];
    BlockDelta bd = make_block_delta(s_delta, K, C);
    bd.init();
    const int64_t cnt = *d_count;
    long long degs = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < cnt; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        int32_t a = -1, b = -1;
        long long c = 0;
        if (p < cnt) {
            const int32_t i = m_idx[order[p]];
            const int32_t v = cand_idx[i];
            a = part0[v];
            b = cand_tgt[v];
            c = vwgt ? vwgt[v] : 1;
            M_node[p] = v;
            M_from[p] = a;
            M_to[p] = b;
            M_score[p] = score[i];
            m_pos[v] = (int32_t)p;
            part[v] = b;
            degs += xadj[v + 1] - xadj[v];
        }
        bd.add(a, -c);
        bd.add(b, c);
    }
    bd.flush(C);
    degs = warp_sum(degs);
    if ((threadIdx.x & 31) == 0 && degs) atomicAdd(deg_sum, (unsigned long long)degs);
}

}  // namespace

void buckets(const GraphDev &g, const int32_t *part, const int32_t *W, int32_t t_num, int32_t t_den, int64_t *BW,
             int64_t *PW, int8_t *first, int8_t *avail_out, int32_t *slot_out, cudaStream_t s, int64_t *cut2,
             int64_t *cut) {
    ensure_pow3();
    const int32_t K = g.K();
    UPR_CUDA(cudaMemsetAsync(BW, 0, sizeof(int64_t) * K * kSlots, s));
    unsigned long long *c2 = nullptr;
    if (cut2) {
        if (g.ng != 1) throw CudaError{cudaErrorInvalidValue, "buckets: the cut is summed for one graph"};
        UPR_CUDA(cudaMemsetAsync(cut2, 0, sizeof(int64_t) * (kCutParts + 1), s));
        c2 = reinterpret_cast<unsigned long long *>(cut2);
    }
    if (g.n > 0) {
        const size_t shm = (g.vwgt ? sizeof(unsigned long long) : sizeof(unsigned int)) * (size_t)K * kSlots;
        const int use_shared = shm <= 200 * 1024;
        if (use_shared && shm > 48 * 1024)
            kernel_setup((const void *)k_buckets, -1);
        const unsigned blocks = wave_grid((const void *)k_buckets, 256, use_shared ? shm : 0, ceil_div(g.n, 256));
        k_buckets<<<blocks, 256, use_shared ? shm : 0, s>>>(part, W, g.wI, g.vwgt, g.n, g.k, g.kmask, K,
                                                                      t_num, t_den, (unsigned long long *)BW,
                                                                      use_shared, avail_out, slot_out, g.sp, c2);
        UPR_LAUNCH_CHECK();
    }
    if (c2) {
        k_half_cut<<<1, kCutParts, 0, s>>>(c2, cut);
        UPR_LAUNCH_CHECK();
    }
    k_bucket_prefix<<<(unsigned)ceil_div(K, 128), 128, 0, s>>>(BW, PW, first, K);
    UPR_LAUNCH_CHECK();
}

int select_group(int k) {
    int G = k / 4;
    return G >= 32 ? 32 : G >= 16 ? 16 : G >= 8 ? 8 : k >= 4 ? 4 : 2;
}

int lane_candidates(int32_t k, LaneCfg *out) {
    if (k % 4 != 0 || k > 256) return 0;
    int G = 1;
    while (G < 32 && 4 * G < k) G <<= 1;
    int CH = (k + 4 * G - 1) / (4 * G);
    int cnt = 0;
    out[cnt++] = LaneCfg{G, CH};
    // fewer lanes per node, more chunks per lane (exact fits only, at most 4 chunks)
    while (cnt < 3 && G > 1 && CH * 2 <= 4 && 4 * (G / 2) * (CH * 2) == k) {
        G /= 2;
        CH *= 2;
        out[cnt++] = LaneCfg{G, CH};
    }
    return cnt;
}

namespace {

template <int G, int CH>
void launch_select_vec(bool exact, bool batch, unsigned blocks, size_t shm, cudaStream_t s, const GraphDev &g,
                       const int32_t *part, const int32_t *W, const Penalty &pen, int smem_pw, int32_t *cand_tgt,
                       int64_t *cand_s0, int32_t *cand_gain, int32_t *flags) {
    // one full wave of CTAs at most (the kernel loops over the nodes)
    auto go = [&](auto kern) {
        kern<<<wave_grid((const void *)kern, 256, shm, blocks), 256, shm, s>>>(g, part, W, pen, smem_pw, cand_tgt,
                                                                             cand_s0, cand_gain, flags);
    };
    const bool pack = !batch && pen.pack_bits > 0 && g.vwgt == nullptr;
    if constexpr (CH == 1 || (G == 32 && CH == 2)) {
        if (!exact) {
            if (batch) go(k_select_vec<G, CH, false, true>);
            else if (pack) go(k_select_vec<G, CH, false, false, true>);
            else go(k_select_vec<G, CH, false, false>);
            return;
        }
    }
    if (batch) go(k_select_vec<G, CH, true, true>);
    else if (pack) go(k_select_vec<G, CH, true, false, true>);
    else go(k_select_vec<G, CH, true, false>);
}

}  // namespace

void select_moves(const GraphDev &g, const int32_t *part, const int32_t *W, Penalty pen, int32_t *cand_tgt,
                  int64_t *cand_s0, int32_t *cand_gain, int32_t *flags, LaneCfg cfg, cudaStream_t s) {
    if (g.n == 0) return;
    const int k = g.k;
    const bool batch = g.ng > 1;
    if (g.sp.on()) {
        const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(g.n, 256 / 8), (int64_t)sm_count_sel() * 8);
        k_select_sparse<8><<<blocks, 256, 0, s>>>(g, part, pen, cand_tgt, cand_s0, cand_gain, flags);
        UPR_LAUNCH_CHECK();
        return;
    }
    LaneCfg cands[3];
    if (lane_candidates(k, cands) > 0) {
        if (cfg.G <= 0) cfg = cands[0];
        const int G = cfg.G, CH = cfg.CH;
        const bool exact = k == 4 * G * CH;
        // the slot prefixes are read only for an excess x > 1, i.e. a node
        // weight c >= 2: with unit node weights they stay in global memory
        // and the smaller shared footprint lets more CTAs run
        const int smem_pw = !batch && g.vwgt && (size_t)k * kSlots * 8 <= 40 * 1024;
        const size_t shm = sizeof(int64_t) * ((size_t)kSlots + (smem_pw ? (size_t)k * kSlots : 0)) +
                           (batch ? 0 : (sizeof(int32_t) + 1) * k + sizeof(int32_t) * (k + 4));
        const int64_t groups = 256 / G;
        const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(g.n, groups), (int64_t)sm_count_sel() * 8);
#define UPR_SELC(GG, CC)                                                                                       \
    if (G == GG && CH == CC) {                                                                                 \
        launch_select_vec<GG, CC>(exact, batch, blocks, shm, s, g, part, W, pen, smem_pw, cand_tgt, cand_s0,   \
                                  cand_gain, flags);                                                           \
        UPR_LAUNCH_CHECK();                                                                                    \
        return;                                                                                                \
    }
        UPR_SELC(1, 1) UPR_SELC(2, 1) UPR_SELC(4, 1) UPR_SELC(8, 1) UPR_SELC(16, 1) UPR_SELC(32, 1)
        UPR_SELC(1, 2) UPR_SELC(2, 2) UPR_SELC(4, 2) UPR_SELC(8, 2) UPR_SELC(16, 2) UPR_SELC(32, 2)
        UPR_SELC(1, 4) UPR_SELC(2, 4) UPR_SELC(4, 4) UPR_SELC(8, 4) UPR_SELC(16, 4)
#undef UPR_SELC
        throw CudaError{cudaErrorInvalidValue, "select_moves: unsupported lane schedule"};
    }
    const int G = select_group(k);
    const int64_t groups = 256 / G;
    const int64_t blocks = std::min<int64_t>(ceil_div(g.n, groups), (int64_t)sm_count_sel() * 16);
#define UPR_SEL(GG) k_select<GG><<<(unsigned)blocks, 256, 0, s>>>(g, part, W, pen, cand_tgt, cand_s0, cand_gain, flags)
    switch (G) {
        case 2: UPR_SEL(2); break;
        case 4: UPR_SEL(4); break;
        case 8: UPR_SEL(8); break;
        case 16: UPR_SEL(16); break;
        default: UPR_SEL(32); break;
    }
#undef UPR_SEL
    UPR_LAUNCH_CHECK();
}

void cand_keys(const int32_t *cand_idx, const int32_t *d_count, const int32_t *cand_tgt, const int64_t *cand_s0,
               int gbits, uint64_t *keys, uint32_t *vals, int64_t max_count, cudaStream_t s) {
    if (max_count <= 0) return;
    k_cand_keys<<<grid_for(max_count), 256, 0, s>>>(cand_idx, d_count, cand_tgt, cand_s0, gbits, keys,
                                                                   vals);
    UPR_LAUNCH_CHECK();
}

void cand_gather(const GraphDev &g, const int32_t *cand_idx, const uint32_t *order, const int32_t *d_count,
                 const int32_t *cand_tgt, int64_t *c_sorted, int32_t *seg_first, int64_t max_count, cudaStream_t s) {
    if (max_count <= 0) return;
    k_cand_gather<<<grid_for(max_count), 256, 0, s>>>(cand_idx, order, d_count, cand_tgt, g.vwgt,
                                                                     c_sorted, seg_first);
    UPR_LAUNCH_CHECK();
}

void inflow_filter(const GraphDev &g, const int32_t *cand_idx, const uint32_t *order, const int32_t *d_count,
                   const int32_t *cand_tgt, const int32_t *cand_gain, const int64_t *c_excl, const int32_t *seg_first,
                   Penalty pen, int32_t *keep_flag, int64_t *score, int64_t max_count, cudaStream_t s) {
    if (max_count <= 0) return;
    k_inflow<<<grid_for(max_count), 256, 0, s>>>(cand_idx, order, d_count, cand_tgt, cand_gain, g.vwgt,
                                                                c_excl, seg_first, pen, keep_flag, score);
    UPR_LAUNCH_CHECK();
}

void move_keys(const int32_t *m_idx, const int32_t *d_count, const int64_t *score, int gbits, uint64_t *keys,
               uint32_t *vals, int64_t max_count, cudaStream_t s) {
    if (max_count <= 0) return;
    k_move_keys<<<grid_for(max_count), 256, 0, s>>>(m_idx, d_count, score, gbits, keys, vals);
    UPR_LAUNCH_CHECK();
}

void apply_moves(const GraphDev &g, const int32_t *cand_idx, const int32_t *m_idx, const uint32_t *order,
                 const int32_t *d_count, const int32_t *cand_tgt, const int64_t *score, const int32_t *part0,
                 int32_t *part, int64_t *C, int32_t *M_node, int32_t *M_from, int32_t *M_to, int64_t *M_score,
                 int32_t *m_pos, int64_t *deg_sum, int64_t max_count, cudaStream_t s) {
    UPR_CUDA(cudaMemsetAsync(deg_sum, 0, sizeof(int64_t), s));
    if (max_count <= 0) return;
    const int64_t blocks = std::min<int64_t>(ceil_div(max_count, 256), (int64_t)device_sm_count() * 4);
    k_apply_moves<<<(unsigned)blocks, 256, block_delta_smem(g.K()), s>>>(
        cand_idx, m_idx, order, d_count, cand_tgt, score, g.vwgt, g.xadj, part0, part, (unsigned long long *)C, g.K(),
        M_node, M_from, M_to, M_score, m_pos, (unsigned long long *)deg_sum);
    UPR_LAUNCH_CHECK();
}

}  // namespace upr
