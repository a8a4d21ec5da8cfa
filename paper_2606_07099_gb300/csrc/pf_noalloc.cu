// pf_noalloc.cu -- pf_solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA graph
// is being captured elsewhere in the process, plug-ins that live inside a host
// application whose allocator owns every device byte, or real-time loops whose
// memory budget is fixed at start-up.  For them this file keeps the solver's
// per-scenario scratch (the workspace pf_solve normally receives from the caller)
// in one file-scope device array that exists for as long as the library is loaded.
//
// The array is shared by every call on a device and keeps what the last call left
// in it.  The solver writes every scratch byte it reads before reading it, so
// nothing needs clearing between calls.  Two calls whose kernels overlap on the GPU
// (different streams, or different threads without ordering) race on the array and
// corrupt each other's results: order them on one stream.
#include <cuda_runtime.h>

#include <mutex>

#include "pf.h"

namespace pf {
int handle_device(const pf_handle* h);  // pf_api.cpp: the device the plan lives on
}

namespace {

// PF_NOALLOC_SCRATCH_BYTES (16 MiB): enough for the 118-bus grid with its full
// 4096-scenario batch in the mixed form (about 2.3 KB per scenario when the factor
// stays in shared memory).
constexpr size_t kScratchBytes = PF_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
pf_err scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return PF_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PF_ECUDA;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return PF_OK;
}

}  // namespace

extern "C" {

pf_err pf_solve_noalloc(pf_handle* h, int batch, const double* Pd, const double* Qd,
                        const double* Pg, const double* Vset, double tol, int max_iter,
                        const pf_solve_opts* opts, double* Vm, double* Va, double* Pg_out,
                        double* Qg_out, int* iters, int* status, double* final_mismatch,
                        void* stream) {
    if (!h || !opts || opts->keep_factors) return PF_EINVAL;
    size_t need = 0;
    pf_err e = pf_workspace_size(h, batch, opts, &need);
    if (e != PF_OK) return e;
    if (need > kScratchBytes) return PF_EINVAL;  // beyond the static maximum
    // pf_solve launches on the device the plan lives on: look the array up there, with
    // that device current (the first call on a device does this one-time lookup)
    const int dev = pf::handle_device(h);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return PF_ECUDA;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return PF_ECUDA;
    void* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (prev != dev) cudaSetDevice(prev);
    if (e != PF_OK) return e;
    return pf_solve(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, opts, Vm, Va, Pg_out, Qg_out,
                    iters, status, final_mismatch, scratch, kScratchBytes, stream);
}

}  // extern "C"
