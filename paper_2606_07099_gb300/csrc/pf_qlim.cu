// pf_qlim.cu -- the Newton solve under reactive-power limits (pf_solve_qlim) and its
// adjoint (pf_adjoint_qlim): the solve body and the adjoint kernel instantiated with each
// scenario's own bus partition (PV buses switching to PQ),
// in a translation unit of its own so that the plain solve keeps its code and the two
// compile in parallel.
#include "pf_body.cuh"
#include "pf_launch.h"

namespace pf {

namespace {
template <typename FT, bool VSM, bool FSM, bool XSM>
cudaError_t launch_q(const DevPlan& P, const SolveArgs& A, int threads, cudaStream_t s) {
    return launch_one(nr_solve_kernel<FT, VSM, FSM, XSM, true>, P, A, A.L.fwd, threads, s);
}
}  // namespace

// One CTA per scenario (the warp-per-scenario form is not instantiated for this path).
template <typename FT>
cudaError_t launch_solve_qlim(const DevPlan& P, const SolveArgs& A, int threads, cudaStream_t s) {
    const KernelSmem& K = A.L.fwd;
    if (K.vec_in_smem && K.fac_in_smem) return launch_q<FT, true, true, false>(P, A, threads, s);
    if (K.vec_in_smem) return launch_q<FT, true, false, false>(P, A, threads, s);
    if (K.fac_in_smem)
        return K.x_in_smem ? launch_q<FT, false, true, true>(P, A, threads, s)
                           : launch_q<FT, false, true, false>(P, A, threads, s);
    return K.x_in_smem ? launch_q<FT, false, false, true>(P, A, threads, s)
                       : launch_q<FT, false, false, false>(P, A, threads, s);
}

// The adjoint of a solve under reactive limits (one CTA per scenario, as pf_adjoint).
template <typename FT>
cudaError_t launch_adjoint_qlim(const DevPlan& P, const AdjArgs& A, int threads, cudaStream_t s) {
    const KernelSmem& K = A.L.adj;
    if (K.vec_in_smem && K.fac_in_smem)
        return launch_one(adjoint_kernel<FT, true, true, true>, P, A, K, threads, s);
    if (K.vec_in_smem) return launch_one(adjoint_kernel<FT, true, false, true>, P, A, K, threads, s);
    if (K.fac_in_smem) return launch_one(adjoint_kernel<FT, false, true, true>, P, A, K, threads, s);
    return launch_one(adjoint_kernel<FT, false, false, true>, P, A, K, threads, s);
}

template cudaError_t launch_adjoint_qlim<float>(const DevPlan&, const AdjArgs&, int, cudaStream_t);
template cudaError_t launch_adjoint_qlim<double>(const DevPlan&, const AdjArgs&, int, cudaStream_t);
template cudaError_t launch_solve_qlim<float>(const DevPlan&, const SolveArgs&, int, cudaStream_t);
template cudaError_t launch_solve_qlim<double>(const DevPlan&, const SolveArgs&, int, cudaStream_t);

}  // namespace pf
