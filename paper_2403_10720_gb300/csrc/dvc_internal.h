// dvc_internal.h -- host-side state shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/dvc.h"

struct dvc_value_net;  // value network state (dvc_value.cu)
struct dvc_ctx;
struct dvc_state;
void dvc_value_free(dvc_ctx* c);
// Win probabilities (n x 4, absolute seats) of n leaves by the context's
// value network, enqueued on st; no argument checks (library-internal).
int dvc_value_forward_probs(dvc_ctx* c, const dvc_state* d_leaves, int n, float* d_probs, cudaStream_t st);

// Value-network activations owned by one caller (a forest's value-mode
// pipeline), so that a captured graph never points into the context's own
// workspace, which other calls may reallocate.  rows: a multiple of 128.
struct dvc_value_rows {
    void *X, *H1, *H2, *H3;  // BF16: rows x 640, rows x 512 (three)
    float* L;                // rows x 16 logits
    int rows;
};
int dvc_value_rows_alloc(dvc_ctx* c, dvc_value_rows* r, int rows);
void dvc_value_rows_free(dvc_value_rows* r);
// Set the network kernels' launch attributes; call before capturing a graph.
int dvc_value_prepare(dvc_ctx* c);
// Win probabilities of n leaves into d_probs, with the activations in rows
// [row0, row0 + n rounded up to 128) of r.  Enqueues kernels only: no
// allocation, no synchronisation, so it may be captured into a graph.
int dvc_value_forward_rows(dvc_ctx* c, const dvc_state* d_leaves, int n, dvc_value_rows* r, int row0, float* d_probs,
                           cudaStream_t st);

struct dvc_ctx {
    dvc_config cfg;
    int device;
    std::string err;
    int32_t* d_flags;  // [0]: latched error code (0 = none)
    unsigned long long* d_ws;  // determinization workspace
    size_t ws_cells;
    dvc_value_net* vnet;       // created on first use of a dvc_value_* call
};


namespace dvc_host {

inline int fail(dvc_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

inline int cuda_fail(dvc_ctx* c, cudaError_t e, const char* where) {
    return fail(c, DVC_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device memory of device `dev` (the context's), or managed memory.  A pointer
// into another GPU's memory is refused: kernels run on the context's device
// and would fault on a peer's memory without peer access.
inline bool is_device_ptr(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// [a, a + bytes) and [b, b + bytes) share a byte.
inline bool ranges_overlap(const void* a, const void* b, size_t bytes) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bytes && b0 < a0 + bytes;
}


inline int check_launch(dvc_ctx* c, const char* where) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return DVC_OK;
}

inline int set_device(dvc_ctx* c) {
    const cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return DVC_OK;
}


}  // namespace dvc_host
