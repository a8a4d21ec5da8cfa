// pf_launch.h -- host entry points into the device code (internal to libpf).
#pragma once

#include "pf_device.cuh"

namespace pf {
template <typename FT>
cudaError_t launch_solve(const DevPlan& P, const SolveArgs& A, int threads, cudaStream_t s);
template <typename FT>
cudaError_t launch_solve_multi(const MultiArgs& M, int threads, int grid, size_t smem, cudaStream_t s);
template <typename FT>
cudaError_t multi_blocks_per_sm(int threads, size_t smem, int* out);
template <typename FT>
cudaError_t launch_solve_qlim(const DevPlan& P, const SolveArgs& A, int threads, cudaStream_t s);
template <typename FT>
cudaError_t launch_adjoint_qlim(const DevPlan& P, const AdjArgs& A, int threads, cudaStream_t s);
template <typename FT>
cudaError_t launch_adjoint(const DevPlan& P, const AdjArgs& A, int threads, cudaStream_t s);
cudaError_t launch_export_jacobian(const DevPlan& P, int batch, const double* Vm, const double* Va,
                                   double* values, cudaStream_t s);
cudaError_t launch_bde_pattern(const DevPlan& P, int batch, int* row_ptr, int* col_idx,
                               cudaStream_t s);
size_t bde_workspace_bytes(const DevPlan& P, int batch);
cudaError_t solve_bde(const DevPlan& P, int batch, const double* Pd, const double* Qd,
                      const double* Pg, const double* Vset, double tol, int max_iter, double* Vm,
                      double* Va, double* Pg_out, double* Qg_out, int* iters, int* status,
                      double* fmis, void* ws, cudaStream_t s);
// The scenario-interleaved solve (pf_si.cu): one thread-block cluster per pack.
template <typename FT>
cudaError_t launch_solve_si(const DevPlan& P, const SiArgs& A, cudaStream_t s);
// Whether a pack shape can be scheduled on the current device (at least one cluster).
template <typename FT>
cudaError_t si_shape_fits(int S, int cluster, int threads, size_t smem, bool* fits);
// CTAs of the shape one SM holds (cluster 1), or clusters the GPU holds; 0: cannot run.
template <typename FT>
cudaError_t si_resident(int S, int cluster, int threads, size_t smem, int* n);
// Device address of pf_solve_noalloc's static scratch array on the current device
// (pf_noalloc.cu; called once per handle by pf_create).
cudaError_t noalloc_lookup(void** out);
}  // namespace pf
