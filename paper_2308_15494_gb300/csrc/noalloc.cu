// upr_cut_noalloc: cut and block weights of a partition without allocating
// any memory.  It runs the same kernels as upr_cut, but their scratch (the
// block-weight accumulators, the cut accumulator and a range flag) lives in
// one file-scope __device__ array instead of a context's arena, so the call
// needs no upr_create and no cudaMalloc.  Every GPU that loads the library
// holds this array (kNoAllocMaxK + 8 int64, about 33 KB) until the process
// exits.
#include <algorithm>

#include "kernels.h"

namespace {

constexpr int kNoAllocMaxK = 4096;

// [0, k): block weights, [k]: cut, [k+1]: input-check flag (partition range,
// CSR offsets, neighbour ids).
static __device__ __align__(256) int64_t g_noalloc_scratch[kNoAllocMaxK + 8];

// The device address of g_noalloc_scratch on the current device (host code
// cannot use the symbol itself as an address).  Looked up on every call: the
// lookup allocates nothing, and an address cached across a cudaDeviceReset
// could point into a module that no longer exists.
int64_t *scratch_address() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<int64_t *>(p);
}

__device__ __forceinline__ void set_flag(int32_t flag_slot) {
    atomicOr(reinterpret_cast<unsigned long long *>(&g_noalloc_scratch[flag_slot]), 1ull);
}

__global__ void k_part_in_range(const int32_t *__restrict__ part, int64_t n, int32_t k, int32_t flag_slot) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && (part[v] < 0 || part[v] >= k)) set_flag(flag_slot);
}

// The CSR offsets: xadj[0] = 0, xadj[n] = m, non-decreasing.  The cut kernels
// find an entry's node by walking xadj, so they run only after this holds.
__global__ void k_xadj_valid(const int64_t *__restrict__ xadj, int64_t n, int64_t m, int32_t flag_slot) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n) return;
    const bool bad = (v == 0 && xadj[0] != 0) || (v == n && xadj[n] != m) || (v < n && xadj[v + 1] < xadj[v]);
    if (bad) set_flag(flag_slot);
}

// Neighbour ids in [0, n): the cut kernels read part[] at every neighbour.
__global__ void k_adj_in_range(const int32_t *__restrict__ adj, int64_t m, int64_t n, int32_t flag_slot) {
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        bad |= adj[e] < 0 || adj[e] >= n;
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_flag(flag_slot);
}

// Device memory of the current device (another GPU's memory would be read
// through peer access, which may be off).
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" upr_status upr_cut_noalloc(const upr_graph *g, int32_t k, const int32_t *part, void *stream,
                                      int64_t *cut, int64_t *block_weights) {
    if (!g || !cut || g->n < 0 || g->m < 0 || g->n >= (1LL << 31) || g->m >= (1LL << 31)) return UPR_ERR_INVALID;
    if (k < 2 || k > kNoAllocMaxK) return UPR_ERR_INVALID;      // the scratch holds at most 4096 blocks
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return UPR_ERR_CUDA; }
    if (g->n > 0 && (!part || !g->xadj || !on_device(part, dev) || !on_device(g->xadj, dev))) return UPR_ERR_INVALID;
    if (g->m > 0 && (!g->adjncy || !on_device(g->adjncy, dev))) return UPR_ERR_INVALID;
    if ((g->vwgt && !on_device(g->vwgt, dev)) || (g->adjwgt && !on_device(g->adjwgt, dev))) return UPR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t *scratch = scratch_address();
    if (!scratch) return UPR_ERR_CUDA;
    try {
        upr::GraphDev G{g->n, g->m, k, 1, -1, g->xadj, g->adjncy, g->adjwgt, g->vwgt, nullptr, nullptr, nullptr};
        // the flag keeps the previous call's value: clear it first; then the
        // partition's range and the CSR's offsets and neighbour ids, all
        // before any kernel that indexes with them
        UPR_CUDA(cudaMemsetAsync(scratch + k + 1, 0, sizeof(int64_t), s));
        if (g->n > 0) {
            k_part_in_range<<<(unsigned)upr::ceil_div(g->n, 256), 256, 0, s>>>(part, g->n, k, k + 1);
            UPR_LAUNCH_CHECK();
            k_xadj_valid<<<(unsigned)upr::ceil_div(g->n + 1, 256), 256, 0, s>>>(g->xadj, g->n, g->m, k + 1);
            UPR_LAUNCH_CHECK();
        }
        if (g->m > 0) {
            const int64_t blocks = std::min<int64_t>(upr::ceil_div(g->m, 256), 4096);
            k_adj_in_range<<<(unsigned)blocks, 256, 0, s>>>(g->adjncy, g->m, g->n, k + 1);
            UPR_LAUNCH_CHECK();
        }
        int64_t bad = 0;
        UPR_CUDA(cudaMemcpyAsync(&bad, scratch + k + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        UPR_CUDA(cudaStreamSynchronize(s));
        if (bad) return UPR_ERR_INVALID;
        // both wrappers zero their accumulators before accumulating
        upr::block_weights(G, part, scratch, s);
        upr::edge_cut(G, part, scratch + k, s);
        UPR_CUDA(cudaMemcpyAsync(cut, scratch + k, sizeof(int64_t), cudaMemcpyDefault, s));
        if (block_weights)
            UPR_CUDA(cudaMemcpyAsync(block_weights, scratch, sizeof(int64_t) * k, cudaMemcpyDefault, s));
        UPR_CUDA(cudaStreamSynchronize(s));
    } catch (const upr::CudaError &) {
        return UPR_ERR_CUDA;
    }
    return UPR_OK;
}
