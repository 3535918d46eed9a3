// lpdf_pdf_step_static: the particle step for callers that cannot allocate device memory.
//
// Who needs it: a host code that owns every device buffer through its own pool or arena
// (a coupling framework, a solver that pre-reserves all of HBM at start-up, an embedded
// runtime) and forbids cudaMalloc inside its time loop -- cudaMalloc can synchronise the
// device, fragments a pool it does not own, and may simply fail when the pool has taken the
// memory. Such a caller keeps the particle state, the node fields and the output in its own
// buffers and calls this entry point; no lpdf_ctx (which allocates) is needed.
//
// The scratch that the step kernel needs -- the 64-bit fixed-point gridpoint accumulators and
// four status words -- lives in file-scope __device__ arrays of a fixed maximum size. Every
// GPU that loads this library holds them (16 MiB + 32 B) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lpdf_internal.h"

namespace {

// n_nodes * (11 + 2 ns) accumulators at most: 2^21 (e.g. 100k nodes with 4 scalars fit).
constexpr size_t kStaticAccMax = size_t(1) << 21;

static __device__ __align__(256) unsigned long long g_static_acc[kStaticAccMax];
static __device__ __align__(256) unsigned long long g_static_status[4];

struct DevicePtrs {
    bool ready = false;
    unsigned long long* acc = nullptr;
    unsigned long long* status = nullptr;
};
constexpr int kMaxDevices = 64;
DevicePtrs g_ptrs[kMaxDevices];
std::mutex g_mutex;

// In host code the names g_static_acc / g_static_status are host-side stand-ins, not device
// addresses; the device addresses come from cudaGetSymbolAddress with that device current.
cudaError_t device_ptrs(int dev, DevicePtrs& out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    DevicePtrs& p = g_ptrs[dev];
    if (!p.ready) {
        void* a = nullptr;
        void* s = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_static_acc);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&s, g_static_status);
        if (e != cudaSuccess) return e;
        p.acc = static_cast<unsigned long long*>(a);
        p.status = static_cast<unsigned long long*>(s);
        p.ready = true;
    }
    out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" int lpdf_pdf_step_static(const lpdf_mesh* mesh, const lpdf_params* params, int64_t n, float* x,
                                    float* y, float* u, float* v, float* w, float* omega, float* psi,
                                    int32_t* elem, const uint32_t* pid, const float* node_fields, uint64_t step,
                                    double* moments, int64_t* status_out, void* stream)
{
    using namespace lpdf;
    if (!mesh || !params || !node_fields || !moments) {
        lpdf_set_error(LPDF_ERR_ARG, "pdf_step_static: NULL argument");
        return LPDF_ERR_ARG;
    }
    if (mesh->d.n_comp > 1 || mesh->d.edge_walls) {
        lpdf_set_error(LPDF_ERR_UNSUPPORTED, "pdf_step_static: multi-component meshes and walls off the frame need a context");
        return LPDF_ERR_UNSUPPORTED;
    }
    if (params->ns < 1 || params->ns > LPDF_MAX_SCALARS) {
        lpdf_set_error(LPDF_ERR_UNSUPPORTED, "pdf_step_static: ns outside 1..4");
        return LPDF_ERR_UNSUPPORTED;
    }
    if (params->mixing != 0 || params->react_k > 0.0) {
        lpdf_set_error(LPDF_ERR_UNSUPPORTED, "pdf_step_static: IECM and reactive sources need a context");
        return LPDF_ERR_UNSUPPORTED;
    }
    if (params->moment_sums != 0) {
        lpdf_set_error(LPDF_ERR_UNSUPPORTED, "pdf_step_static: compensated moment sums need a context");
        return LPDF_ERR_UNSUPPORTED;
    }
    if (n < 0 || (n > 0 && (!x || !y || !u || !v || !w || !omega || !psi || !elem || !pid))) {
        lpdf_set_error(LPDF_ERR_ARG, "pdf_step_static: bad particle arrays");
        return LPDF_ERR_ARG;
    }
    const int ns = params->ns;
    const size_t nacc = (size_t)mesh->d.n_nodes * (size_t)nquant(ns);
    if (nacc > kStaticAccMax) {
        lpdf_set_error(LPDF_ERR_ARG, "pdf_step_static: n_nodes * (11 + 2 ns) = %zu exceeds the static maximum %zu",
                       nacc, kStaticAccMax);
        return LPDF_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) e = cudaErrorInvalidDevice;
    DevicePtrs ptrs;
    if (e == cudaSuccess) e = device_ptrs(dev, ptrs);
    const cudaStream_t st = (cudaStream_t)stream;
    // the arrays keep the previous call's contents: clear the accumulators and the status words
    if (e == cudaSuccess) e = cudaMemsetAsync(ptrs.acc, 0, nacc * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ptrs.status, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ptrs.status + 2, 0xff, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ptrs.status + 3, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && n > 0) {
        DevState s{x, y, u, v, w, omega, psi, elem, const_cast<uint32_t*>(pid), n, n};
        const StepParams p = make_step_params(*params, mesh, step);
        e = launch_pdf_step(mesh->d, s, ns, node_fields, p, ptrs.acc, ptrs.status, st);
    }
    if (e == cudaSuccess) e = launch_grid_statistics(mesh->d, ns, ptrs.acc, moments, 1, st);
    if (e != cudaSuccess) {
        lpdf_set_error(LPDF_ERR_CUDA, "pdf_step_static: %s", cudaGetErrorString(e));
        return LPDF_ERR_CUDA;
    }
    if (status_out) {
        unsigned long long h[4];
        e = cudaMemcpyAsync(h, ptrs.status, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            lpdf_set_error(LPDF_ERR_CUDA, "pdf_step_static: %s", cudaGetErrorString(e));
            return LPDF_ERR_CUDA;
        }
        status_out[0] = (int64_t)h[0];
        status_out[1] = (int64_t)h[1];
        status_out[2] = h[2] == ~0ull ? -1 : (int64_t)h[2];
        status_out[3] = (int64_t)h[3];
        if (h[0] & kErrLost) {
            lpdf_set_error(LPDF_ERR_LOST_PARTICLE, "%llu particle(s) lost", h[1]);
            return LPDF_ERR_LOST_PARTICLE;
        }
        if (h[0] & kErrNonFinite) {
            lpdf_set_error(LPDF_ERR_NONFINITE, "non-finite particle state");
            return LPDF_ERR_NONFINITE;
        }
        if (h[0] & kErrTimeout) {
            lpdf_set_error(LPDF_ERR_CUDA, "a bulk-copy wait in the step kernel timed out");
            return LPDF_ERR_CUDA;
        }
        if (h[0] & kErrCheck) {
            lpdf_set_error(LPDF_ERR_CUDA, "an internal consistency check of the step kernel failed");
            return LPDF_ERR_CUDA;
        }
        if (h[0] & kErrOverflow) {
            lpdf_set_error(LPDF_ERR_OVERFLOW, "fixed-point moment range exceeded");
            return LPDF_ERR_OVERFLOW;
        }
    }
    return LPDF_OK;
}
