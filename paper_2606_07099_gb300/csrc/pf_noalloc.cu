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
//
// In host code the array's name is only a host-side stand-in, so its device address
// is looked up with cudaGetSymbolAddress.  pf_create does that once per handle, with
// the handle's device current, and keeps the address on the handle: under lazy module
// loading that lookup is what loads this module and commits the array, so it happens
// in the call that allocates anyway, never inside pf_solve_noalloc.  A device reset
// ends the handle and, with it, the address.
#include <cuda_runtime.h>

#include "pf.h"
#include "pf_launch.h"

namespace pf {
int handle_device(const pf_handle* h);             // pf_api.cpp: the plan's device
void* handle_noalloc_scratch(const pf_handle* h);  // pf_api.cpp: the address kept by pf_create
}

namespace {

// PF_NOALLOC_SCRATCH_BYTES (16 MiB): enough for the 118-bus grid with its full
// 4096-scenario batch in the mixed form (about 2.3 KB per scenario when the factor
// stays in shared memory).
constexpr size_t kScratchBytes = PF_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

}  // namespace

namespace pf {
cudaError_t noalloc_lookup(void** out) {
    *out = nullptr;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();  // not sticky: keep it from surfacing at a later launch check
        return e;
    }
    if (!p) return cudaErrorInvalidSymbol;
    *out = p;
    return cudaSuccess;
}
}  // namespace pf

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
    void* scratch = pf::handle_noalloc_scratch(h);
    if (!scratch) return PF_ECUDA;  // pf_create could not look the array up on this device
    return pf_solve(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, opts, Vm, Va, Pg_out, Qg_out,
                    iters, status, final_mismatch, scratch, kScratchBytes, stream);
}

}  // extern "C"
