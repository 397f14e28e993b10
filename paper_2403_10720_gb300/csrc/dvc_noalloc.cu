// dvc_noalloc.cu -- dvc_determinize_noalloc: the determinizer with its
// scratch in a fixed device array instead of memory the library allocates.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// already fully reserved by another framework's caching allocator, or a
// serving process that is not allowed to allocate once it has started.  This
// entry point lets them determinize without creating a context (which
// allocates) and without the context's lazily allocated workspace.
//
// The scratch is one file-scope __device__ array of kNoAllocRoots slots of
// kNoAllocCells counting-table cells (8 MiB).  Every GPU that loads the
// library holds it until the process exits.  All calls share it and it keeps
// the last call's contents; nothing in it needs to start at zero, because
// every table cell is written before it is read.  Calls that overlap on the
// GPU (on different streams, or from several host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "dvc_det.cuh"

using namespace dvc;

namespace {

constexpr int kNoAllocRoots = 64;
constexpr uint32_t kNoAllocCells = 16384;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned long long g_det_scratch[(size_t)kNoAllocRoots * kNoAllocCells];

// Device address of g_det_scratch per device, looked up once per device.
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Device memory of device `dev` (the one the kernel will run on), or managed
// memory.  A pointer into another GPU's memory is refused: the kernel would
// read and write a peer's memory, which faults without peer access.
bool on_device(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// [a, a + n) and [b, b + n) records share a byte.
bool overlaps(const dvc_state* a, const dvc_state* b, int n) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b, len = sizeof(dvc_state) * (uintptr_t)n;
    return a0 < b0 + len && b0 < a0 + len;
}

__global__ void determinize_noalloc_kernel(const dvc_state* roots, int n, int observer, uint64_t seed,
                                           const uint32_t* tree_ids, const uint32_t* iter_ids, dvc_state* out,
                                           int32_t* status, unsigned long long* scratch) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const G g = load_state(roots[idx]);
    if (observer >= (int)g.np) {  // no such seat in this root's game
        out[idx] = roots[idx];
        if (status) status[idx] = DVC_E_INVALID;
        return;
    }
    const uint32_t obs = observer < 0 ? g.cur : (uint32_t)observer;
    DetPlan pl;
    det_plan(g, obs, pl);
    if (pl.cells > kNoAllocCells) {
        out[idx] = roots[idx];
        if (status) status[idx] = DVC_E_UNSUPPORTED;
        return;
    }
    unsigned long long* F = scratch + (size_t)idx * kNoAllocCells;
    det_fill(pl, F, 0u, 1u, [] {});
    Rng r;
    r.open(seed, tree_ids[idx], 0u, iter_ids[idx], kTagDet);
    G o;
    det_sample(pl, F, g, r, o);
    store_state(o, out[idx]);
    if (status) status[idx] = DVC_OK;
}

}  // namespace

extern "C" int dvc_determinize_noalloc(const dvc_state* d_roots, int n, int observer, uint64_t seed,
                                       const uint32_t* d_tree_ids, const uint32_t* d_iter_ids, dvc_state* d_out,
                                       int32_t* d_status, void* stream) {
    if (n < 0 || observer >= 4) return DVC_E_INVALID;
    if (n > kNoAllocRoots) return DVC_E_UNSUPPORTED;
    if (n == 0) return DVC_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DVC_E_CUDA;
    }
    if (!on_device(d_roots, dev) || !on_device(d_tree_ids, dev) || !on_device(d_iter_ids, dev) ||
        !on_device(d_out, dev) || (d_status && !on_device(d_status, dev)))
        return DVC_E_INVALID;
    if (overlaps(d_roots, d_out, n)) return DVC_E_INVALID;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            // The symbol's name is only a host-side stand-in; the kernel needs
            // the device address, looked up with this device current.
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_det_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DVC_E_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    determinize_noalloc_kernel<<<(n + 63) / 64, 64, 0, (cudaStream_t)stream>>>(
        d_roots, n, observer, seed, d_tree_ids, d_iter_ids, d_out, d_status, (unsigned long long*)scratch);
    if (cudaGetLastError() != cudaSuccess) return DVC_E_CUDA;
    return DVC_OK;
}
