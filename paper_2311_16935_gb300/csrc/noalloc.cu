// osmodi_solve_noalloc: the solve of osmodi_solve with its device scratch in
// a fixed, file-scope device array instead of a caller-allocated workspace.
//
// For callers that cannot allocate device memory when they solve: a host
// framework whose caching allocator owns the device memory, or a
// latency-bound acquisition loop in which cudaMalloc / cudaFree (which can
// synchronise the device) are not acceptable.  Such a caller creates its
// plans during set-up and then solves with no allocation at all.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace osm {
osmodi_status solve_into_scratch(osmodi_plan p, const void* grad, int gdt, void* pu, int pdt, double tol, int max_iter,
                                 void* scratch, cudaStream_t s, osmodi_result* res);
}  // namespace osm

// The scratch.  Every GPU that loads this module holds it until the process
// exits.  Host code must never pass `g_noalloc_scratch` itself to a kernel:
// on the host that name is only a stand-in, not a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[OSMODI_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device.  Plan creation does this set-up (osm::noalloc_prepare): looking the
// symbol up loads this module, and with it the array, on that device, which
// under lazy module loading would otherwise happen inside the first solve.
cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

namespace osm {
// Called by osmodi_create with the plan's device current: resolves (and so
// loads) the scratch on that device once, so that osmodi_solve_noalloc finds
// it ready and allocates nothing.  A failure here is not an error of plan
// creation; the solve reports it if it persists.
void noalloc_prepare(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    void* ptr = nullptr;
    if (scratch_address(dev, &ptr) != cudaSuccess) cudaGetLastError();
}
}  // namespace osm

extern "C" osmodi_status osmodi_solve_noalloc(osmodi_plan p, const void* grad, int gdt, void* pu, int pdt, double tol,
                                              int max_iter, void* stream, osmodi_result* res) {
    if (res) std::memset(res, 0, sizeof(*res));
    if (!p || !grad || !pu) return OSMODI_E_INVALID;
    if ((gdt != OSMODI_F32 && gdt != OSMODI_F64) || (pdt != OSMODI_F32 && pdt != OSMODI_F64)) return OSMODI_E_INVALID;
    if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 0) return OSMODI_E_INVALID;
    const size_t need = osmodi_workspace_bytes(p);
    if (need > (size_t)OSMODI_NOALLOC_SCRATCH_BYTES) {
        osm::set_error_text("osmodi_solve_noalloc: the plan needs more scratch than the fixed "
                            "OSMODI_NOALLOC_SCRATCH_BYTES; use osmodi_solve with a workspace");
        return OSMODI_E_WORKSPACE;
    }
    int dev = -1;
    OSM_CUDA(cudaGetDevice(&dev));
    if (dev != p->device || dev < 0 || dev >= kMaxDevices) {
        osm::set_error_text("osmodi_solve_noalloc: the current device is not the plan's device");
        return OSMODI_E_INVALID;
    }
    if (!osm::user_buffer_ok(grad, dev) || !osm::user_buffer_ok(pu, dev)) {
        osm::set_error_text("osmodi_solve_noalloc: gradient and pressure must be device, managed or page-locked host memory");
        return OSMODI_E_INVALID;
    }
    void* scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        osm::set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        return OSMODI_E_CUDA;
    }
    osmodi_status st = osm::solve_into_scratch(p, grad, gdt, pu, pdt, tol, max_iter, scratch, (cudaStream_t)stream, res);
    if (res) res->status = st;
    return st;
}
