// upr_cut_noalloc: cut and block weights of a partition without allocating
// any memory.  It runs the same kernels as upr_cut, but their scratch (the
// block-weight accumulators, the cut accumulator and a range flag) lives in
// one file-scope __device__ array instead of a context's arena, so the call
// needs no upr_create and no cudaMalloc.  Every GPU that loads the library
// holds this array (kNoAllocMaxK + 8 int64, about 33 KB) until the process
// exits.
#include <mutex>

#include "kernels.h"

namespace {

constexpr int kNoAllocMaxK = 4096;
constexpr int kMaxDevices = 64;

// [0, k): block weights, [k]: cut, [k+1]: partition-range flag.
static __device__ __align__(256) int64_t g_noalloc_scratch[kNoAllocMaxK + 8];

std::mutex g_setup_mu;
int64_t *g_scratch_addr[kMaxDevices] = {};

// The device address of g_noalloc_scratch on the current device, looked up
// once per device (host code cannot use the symbol itself as an address).
int64_t *scratch_address(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_addr[dev] = static_cast<int64_t *>(p);
    }
    return g_scratch_addr[dev];
}

__global__ void k_part_in_range(const int32_t *__restrict__ part, int64_t n, int32_t k, int32_t flag_slot) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && (part[v] < 0 || part[v] >= k))
        atomicOr(reinterpret_cast<unsigned long long *>(&g_noalloc_scratch[flag_slot]), 1ull);
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" upr_status upr_cut_noalloc(const upr_graph *g, int32_t k, const int32_t *part, void *stream,
                                      int64_t *cut, int64_t *block_weights) {
    if (!g || !cut || g->n < 0 || g->m < 0 || g->n >= (1LL << 31) || g->m >= (1LL << 31)) return UPR_ERR_INVALID;
    if (k < 2 || k > kNoAllocMaxK) return UPR_ERR_INVALID;      // the scratch holds at most 4096 blocks
    if (g->n > 0 && (!part || !g->xadj || !on_device(part) || !on_device(g->xadj))) return UPR_ERR_INVALID;
    if (g->m > 0 && (!g->adjncy || !on_device(g->adjncy))) return UPR_ERR_INVALID;
    if ((g->vwgt && !on_device(g->vwgt)) || (g->adjwgt && !on_device(g->adjwgt))) return UPR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return UPR_ERR_CUDA;
    int64_t *scratch = scratch_address(dev);
    if (!scratch) return UPR_ERR_CUDA;
    try {
        upr::GraphDev G{g->n, g->m, k, 1, -1, g->xadj, g->adjncy, g->adjwgt, g->vwgt, nullptr, nullptr, nullptr};
        // the flag keeps the previous call's value: clear it first
        UPR_CUDA(cudaMemsetAsync(scratch + k + 1, 0, sizeof(int64_t), s));
        if (g->n > 0) {
            k_part_in_range<<<(unsigned)upr::ceil_div(g->n, 256), 256, 0, s>>>(part, g->n, k, k + 1);
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
