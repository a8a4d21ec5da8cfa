// pf_kernels.cu -- kernel instantiations and launchers of libpf (sm_103a): the Newton
// solve, the multi-network solve, the adjoint and the block-diagonal export.  The device
// code itself is in pf_body.cuh; pf_qlim.cu instantiates the reactive-limit solve.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "pf_body.cuh"
#include "pf_launch.h"

namespace pf {

// ---------------------------------------------------------------- launchers
// The dynamic shared-memory limit of a kernel is raised once per (device, kernel) to the
// largest size requested so far, so that launches after the first make no attribute
// call (a launch can then be recorded into a CUDA graph).
cudaError_t ensure_smem_limit(const void* k, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = done[{dev, k}];
    if (bytes <= cur && cur > 0) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// ---------------------------------------------------------------- block-diagonal export
// The J1 values of every scenario at the given voltages, written straight into the fixed
// scalar template (Sec. III-A; Alg. 1's element formulas, here jac_block in FP64).  One
// CTA per scenario: first the unit phasor u = e^{j theta} of every bus (one FP64 sincos
// per bus, the costly part on this GPU's FP64 pipe), kept in shared memory (UMEM) when it
// fits, else recomputed per use; then one thread per non-slack bus forms I_i from its
// Ybus row and the 2x2 block of every entry (i, j) of that row, and stores the applicable
// entries at the positions the plan holds for them.
template <bool UMEM>
__global__ void __launch_bounds__(256) export_j1_kernel(DevPlan P, int batch, const double* Vm,
                                                        const double* Va, double* values) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* su = reinterpret_cast<double2*>(smem_raw);
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        const double* vm = Vm + (size_t)b * P.n_bus;
        const double* va = Va + (size_t)b * P.n_bus;
        auto unit = [&](int j) {
            if (UMEM) return su[j];
            double sj, cj;
            sincos(va[j], &sj, &cj);
            return make_double2(cj, sj);
        };
        if (UMEM) {
            for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
                double si, ci;
                sincos(va[i], &si, &ci);
                su[i] = make_double2(ci, si);
            }
            __syncthreads();
        }
        double* out = values + (size_t)b * P.nnz_j1;
        for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
            if (__ldg(P.bus_type + i) == 2) continue;
            const double2 ui = unit(i);
            const double vmi = vm[i], vri = vmi * ui.x, vii = vmi * ui.y;
            const int k0 = __ldg(P.y_ptr + i), k1 = __ldg(P.y_ptr + (i + 1));
            double ir = 0.0, ii = 0.0;
            for (int k = k0; k < k1; ++k) {
                const int j = __ldg(P.y_idx + k);
                const double2 y = __ldg(P.y_gb + k);
                const double2 uj = unit(j);
                const double vr = vm[j] * uj.x, vi = vm[j] * uj.y;
                ir = fma(y.x, vr, fma(-y.y, vi, ir));
                ii = fma(y.x, vi, fma(y.y, vr, ii));
            }
            const double pu = ui.x * ir + ui.y * ii, qu = ui.y * ir - ui.x * ii;  // u_i conj(I_i)
            for (int k = k0; k < k1; ++k) {
                const int j = __ldg(P.y_idx + k);
                const double2 y = __ldg(P.y_gb + k);
                const double2 uj = unit(j);
                const Blk<double> m = jac_block<double>(i == j, y.x, y.y, vri, vii, uj.x, uj.y,
                                                        vm[j], vmi, pu, qu);
                const int4 pos = __ldg(P.j1_pos + k);
                if (pos.x >= 0) out[pos.x] = m.a;
                if (pos.y >= 0) out[pos.y] = m.b;
                if (pos.z >= 0) out[pos.z] = m.c;
                if (pos.w >= 0) out[pos.w] = m.d;
            }
        }
        if (UMEM) __syncthreads();  // the next scenario overwrites the phasors
    }
}

// Index arrays of the block-diagonal embedding: block k is the template shifted by k n1.
__global__ void __launch_bounds__(256) bde_pattern_kernel(DevPlan P, int batch, int* row_ptr,
                                                          int* col_idx) {
    const long long rows = (long long)batch * P.n1, nz = (long long)batch * P.nnz_j1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= rows; r += stride) {
        const long long b = r / P.n1, rr = r - b * P.n1;
        row_ptr[r] = (r == rows) ? (int)nz : (int)(b * P.nnz_j1 + __ldg(P.j1_ptr + rr));
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nz; e += stride) {
        const long long b = e / P.nnz_j1, ee = e - b * P.nnz_j1;
        col_idx[e] = (int)(b * P.n1 + __ldg(P.j1_col + ee));
    }
}


template <typename FT, bool VSM, bool FSM, bool XSM>
cudaError_t launch_solve_cfg(const DevPlan& P, const SolveArgs& A, int threads, cudaStream_t s) {
    if (A.ipc <= 1) return launch_one(nr_solve_kernel<FT, VSM, FSM, XSM>, P, A, A.L.fwd, threads, s);
    auto k = nr_solve_warps_kernel<FT, VSM, FSM, XSM>;
    const size_t smem = A.L.fwd.smem_bytes * (size_t)A.ipc;
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(k), smem);
    if (e != cudaSuccess) return e;
    const int grid = (A.batch + A.ipc - 1) / A.ipc;
    k<<<grid, 32 * A.ipc, smem, s>>>(P, A);
    return cudaGetLastError();
}

template <typename FT>
cudaError_t launch_solve(const DevPlan& P, const SolveArgs& A, int threads, cudaStream_t s) {
    const KernelSmem& K = A.L.fwd;
    if (K.vec_in_smem && K.fac_in_smem) return launch_solve_cfg<FT, true, true, false>(P, A, threads, s);
    if (K.vec_in_smem) return launch_solve_cfg<FT, true, false, false>(P, A, threads, s);
    if (K.fac_in_smem)
        return K.x_in_smem ? launch_solve_cfg<FT, false, true, true>(P, A, threads, s)
                           : launch_solve_cfg<FT, false, true, false>(P, A, threads, s);
    return K.x_in_smem ? launch_solve_cfg<FT, false, false, true>(P, A, threads, s)
                       : launch_solve_cfg<FT, false, false, false>(P, A, threads, s);
}

template <typename FT>
cudaError_t launch_adjoint(const DevPlan& P, const AdjArgs& A, int threads, cudaStream_t s) {
    const KernelSmem& K = A.L.adj;
    if (K.vec_in_smem && K.fac_in_smem)
        return launch_one(adjoint_kernel<FT, true, true>, P, A, K, threads, s);
    if (K.vec_in_smem) return launch_one(adjoint_kernel<FT, true, false>, P, A, K, threads, s);
    if (K.fac_in_smem) return launch_one(adjoint_kernel<FT, false, true>, P, A, K, threads, s);
    return launch_one(adjoint_kernel<FT, false, false>, P, A, K, threads, s);
}

template <typename FT>
cudaError_t launch_solve_multi(const MultiArgs& M, int threads, int grid, size_t smem, cudaStream_t s) {
    auto k = nr_solve_multi_kernel<FT>;
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(k), smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, s>>>(M);
    return cudaGetLastError();
}

template <typename FT>
cudaError_t multi_blocks_per_sm(int threads, size_t smem, int* out) {
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(nr_solve_multi_kernel<FT>), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, nr_solve_multi_kernel<FT>, threads, smem);
}

cudaError_t launch_export_jacobian(const DevPlan& P, int batch, const double* Vm, const double* Va,
                                   double* values, cudaStream_t s) {
    const size_t smem = sizeof(double2) * (size_t)P.n_bus;
    int optin = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int grid = std::min(batch, 152 * 16);
    if (smem + 1024 <= (size_t)optin) {
        e = ensure_smem_limit(reinterpret_cast<const void*>(export_j1_kernel<true>), smem);
        if (e != cudaSuccess) return e;
        export_j1_kernel<true><<<grid, 256, smem, s>>>(P, batch, Vm, Va, values);
    } else {
        export_j1_kernel<false><<<grid, 256, 0, s>>>(P, batch, Vm, Va, values);
    }
    return cudaGetLastError();
}

cudaError_t launch_bde_pattern(const DevPlan& P, int batch, int* row_ptr, int* col_idx,
                               cudaStream_t s) {
    const long long total = (long long)batch * P.nnz_j1;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 8 * 4);
    bde_pattern_kernel<<<grid, 256, 0, s>>>(P, batch, row_ptr, col_idx);
    return cudaGetLastError();
}

template cudaError_t launch_solve_multi<float>(const MultiArgs&, int, int, size_t, cudaStream_t);
template cudaError_t launch_solve_multi<double>(const MultiArgs&, int, int, size_t, cudaStream_t);
template cudaError_t multi_blocks_per_sm<float>(int, size_t, int*);
template cudaError_t multi_blocks_per_sm<double>(int, size_t, int*);
template cudaError_t launch_solve<float>(const DevPlan&, const SolveArgs&, int, cudaStream_t);
template cudaError_t launch_solve<double>(const DevPlan&, const SolveArgs&, int, cudaStream_t);
template cudaError_t launch_adjoint<float>(const DevPlan&, const AdjArgs&, int, cudaStream_t);
template cudaError_t launch_adjoint<double>(const DevPlan&, const AdjArgs&, int, cudaStream_t);

}  // namespace pf
