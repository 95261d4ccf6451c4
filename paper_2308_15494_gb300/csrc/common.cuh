// Shared definitions of the CUDA library: integer types, launch helpers,
// error propagation and warp-level primitives.  Everything here is
// integer-only; no floating point reaches a result.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "../../include/upr.h"

typedef unsigned __int128 u128;
typedef __int128 i128;

namespace upr {

constexpr int kSlotLo = -32;                 // bucket slots are clamped to [-32, 40]
constexpr int kSlotHi = 40;
constexpr int kSlots = kSlotHi - kSlotLo + 1; // 73
constexpr int kQ = 20;                       // fixed-point bits of the penalty factors
constexpr int kMaxK = 4096;
constexpr int kHubDegree = 4096;             // nodes above this degree get CTA-wide treatment

// A failing CUDA call is turned into UPR_ERR_CUDA by the entry points.
struct CudaError { cudaError_t e; const char *what; };

#define UPR_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) throw ::upr::CudaError{_e, #call};          \
    } while (0)

// Counts kernel launches of this library (reported in upr_stats).
extern thread_local long long g_upr_launches;
#define UPR_LAUNCH_CHECK()                                                 \
    do {                                                                   \
        ::upr::g_upr_launches++;     \
        UPR_CUDA(cudaGetLastError());                                      \
    } while (0)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over an aligned group of G lanes (G a power of two <= 32).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lexicographic max of (score, -id) over an aligned group of G lanes: the
// larger score wins, equal scores go to the smaller id; id < 0 marks "none".
template <int G>
__device__ __forceinline__ void group_argmax(int64_t &score, int32_t &id) {
    for (int o = G / 2; o > 0; o >>= 1) {
        int64_t s2 = __shfl_xor_sync(0xffffffffu, score, o);
        int32_t i2 = __shfl_xor_sync(0xffffffffu, id, o);
        bool take = (i2 >= 0) && (id < 0 || s2 > score || (s2 == score && i2 < id));
        if (take) { score = s2; id = i2; }
    }
}

// Per-CTA accumulation of block-weight changes.  Every lane of every warp
// calls add() (key < 0 = nothing to add); lanes with equal keys are combined
// with __match_any_sync and their leader adds the group's total to shared
// memory; flush() adds the CTA's non-zero totals to the global counters.
// With more than kMaxK blocks (a batch of graphs) the shared array would not
// fit: `direct` then points at the global counters and the leaders add there.
// Integer additions commute, so the result is independent of scheduling.
struct BlockDelta {
    unsigned long long *s;
    int k;
    unsigned long long *direct;
    __device__ __forceinline__ void init() {
        if (!direct)
            for (int i = threadIdx.x; i < k; i += blockDim.x) s[i] = 0;
        __syncthreads();
    }
    __device__ __forceinline__ void add(int key, long long d) {
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        long long tot = 0;
        for (unsigned m = peers; m; m &= m - 1) tot += __shfl_sync(peers, d, __ffs(m) - 1);
        if (key >= 0 && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0 && tot != 0)
            atomicAdd(direct ? &direct[key] : &s[key], (unsigned long long)tot);
    }
    __device__ __forceinline__ void flush(unsigned long long *C) {
        if (direct) return;
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += blockDim.x)
            if (s[i]) atomicAdd(&C[i], s[i]);
    }
};
// Shared memory of a BlockDelta over K blocks, and the CTA's accumulator.
inline size_t block_delta_smem(int64_t K) { return K <= kMaxK ? sizeof(unsigned long long) * (size_t)K : 0; }
__device__ __forceinline__ BlockDelta make_block_delta(unsigned long long *smem, int K, unsigned long long *C) {
    return K <= kMaxK ? BlockDelta{smem, K, nullptr} : BlockDelta{nullptr, K, C};
}

// Kernel attributes are per process and device, shared by every host thread:
// a kernel's dynamic shared-memory limit is raised once to the device's
// opt-in maximum less its static shared memory (a ceiling only: occupancy
// follows the launch's actual size)
// and its shared/L1 split set, never changed afterwards, so no thread can
// lower a limit another thread's launch relies on.
void kernel_setup(const void *func, int carveout_percent);   // engine.cu; -1 = no carveout preference
// CTAs of `threads` threads with `shm` bytes of dynamic shared memory that fit
// on one SM at once (at least 1), cached per kernel and size (engine.cu).
int resident_ctas(const void *func, int threads, size_t shm);
// A grid for `want` CTAs of a grid-stride kernel: at most one full wave.
inline unsigned wave_grid(const void *func, int threads, size_t shm, int64_t want);

inline int device_sm_count() {
    static thread_local int cnt = 0, dev_cached = -1;
    int dev = 0;
    UPR_CUDA(cudaGetDevice(&dev));
    if (dev != dev_cached) {
        UPR_CUDA(cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev));
        dev_cached = dev;
    }
    return cnt;
}

inline unsigned wave_grid(const void *func, int threads, size_t shm, int64_t want) {
    const int64_t wave = (int64_t)device_sm_count() * resident_ctas(func, threads, shm);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, wave));
}

// 32-bit form of group_argmax.
template <int G>
__device__ __forceinline__ void group_argmax32(int32_t &score, int32_t &id) {
    for (int o = G / 2; o > 0; o >>= 1) {
        int32_t s2 = __shfl_xor_sync(0xffffffffu, score, o);
        int32_t i2 = __shfl_xor_sync(0xffffffffu, id, o);
        bool take = (i2 >= 0) && (id < 0 || s2 > score || (s2 == score && i2 < id));
        if (take) { score = s2; id = i2; }
    }
}

}  // namespace upr
