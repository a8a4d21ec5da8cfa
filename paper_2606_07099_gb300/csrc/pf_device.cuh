// pf_device.cuh -- device-side data structures and small helpers (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

// Read-only plan arrays on the device (see pf_plan.h for their meaning).
struct DevPlan {
    int n_bus, n, nnzb, n_levels;
    // top region (the trailing levels top_l0.. whose pivots are taken one at a time in
    // shared memory; top_R = 0: none): first level and row, rows, blocks, lanes per row of
    // its part left of the region, and the lengths of its staged lists
    int top_l0, top_p0, top_R, top_nblk, top_g, top_nl, top_nfw, top_nbw, top_nints;
    int top_nft, top_nbt, top_nints_fwd;  // transposed rounds; the forward solve's list length
    const int* top_map;    // [top_nblk] fac position of each region block
    const int* top_split;  // [top_R] first entry of each region row inside the region
    const int* top_ints;   // piv | lc_ptr | lc | tr_ptr | fwk | fw | bwk | bw | ftk | ft | btk | bt
    const int2* top_tr;    // Schur triples: (target, L block | U block << 16)
    const int* y_ptr;
    const int* y_idx;
    const double2* y_gb;  // (G, B) of every Ybus entry
    const float2* y_gb32; // the same in FP32 (for the FP32 Jacobian fill)
    const int* bus_type;
    const int* pos2bus;
    const int* bus2pos;
    const int* lev_ptr;
    const int4* lev_g;    // per level: (gL, gU, gS, 0) lanes per gathered row
    const int* lu_ptr;
    const int* lu_row;
    const int* lu_col;
    const int* lu_diag;
    const int* lu_mirror;
    const int* fill_y;
    const int* la_ptr;
    const int2* la;       // (L block, diagonal block)
    const int* sch_tptr;
    const int* sch_tgt;
    const int* sch_cptr;
    const int2* sch;      // (L block, U block)
    const int* yt_ptr;    // transpose of Ybus (column access for the adjoint products)
    const int* yt_idx;
    const double2* yt_gb;
    int n1, nnz_j1;       // scalar J1 template (block-diagonal export)
    const int* j1_ptr;    // its CSR in the paper's ordering
    const int* j1_col;
    const int4* j1_pos;   // per Ybus entry: positions of (dP/dtheta, dP/dVm, dQ/dtheta, dQ/dVm)
};

// Where one kernel keeps the scenario's vectors and factor (shared or global memory).
struct KernelSmem {
    int vec_in_smem;      // vector arena in shared memory
    int fac_in_smem;      // factor staged in shared memory
    size_t smem_bytes;    // dynamic shared memory per CTA
    size_t smem_fac_off;  // factor offset inside the dynamic shared memory
    int x_in_smem;        // the solve vector in shared memory although the vectors are not
    size_t smem_x_off;    // its offset inside the dynamic shared memory
    size_t vec_bytes;     // size of this kernel's vector arena
    size_t smem_top_off;  // the top region's arena (top_arena_bytes), if any
};

// Per-scenario workspace slot (global memory), offsets in bytes from the slot base.
struct SlotLayout {
    size_t slot_bytes;
    size_t off_state;   // doubles [n_bus] each: Vm, Va (and with kept factors u = e^{j Va}
                        // as Uc, Us and I = Y V as Ire, Iim): the solution, for pf_adjoint
    size_t off_flags;   // int status, iters, has_factor, pad
    size_t off_fac;     // factor values (if stored in global memory), or 0
    size_t off_vec;     // vector arena (if a kernel keeps it in global memory), or 0
    size_t off_qlim;    // reactive-limit state (pf_solve_qlim): int8 type[n_bus], then
                        // double qfix[n_bus] at off_qlim + align16(n_bus); 0 = none
    int fac_global;     // factor region present in the slot
    size_t fac_bytes;
    KernelSmem fwd, adj;
};

struct SolveArgs {
    int batch;
    int ipc;         // scenarios per CTA: 1 = the whole CTA per scenario, >1 = one warp each
    double tol;
    int max_iter;
    int ir_steps;
    double ir_rtol;
    double ir_gate;
    int keep_factors;
    const double* Pd;
    const double* Qd;
    const double* Pg;
    const double* Vset;
    double* Vm;
    double* Va;
    double* Pg_out;
    double* Qg_out;
    double* fmis;
    int* iters;
    int* status;
    char* ws;
    SlotLayout L;
    // reactive limits at PV buses (pf_solve_qlim); Qmax == nullptr: no limits
    const double* Qmin;
    const double* Qmax;
    int max_rounds;
    int* types_out;
    int* rounds_out;
};

// Several networks in one launch (pf_solve_multi): per job its plan and solve arguments,
// and the first global work item of each job (jobs are contiguous ranges of items).
constexpr int kMaxJobs = 8;
struct MultiArgs {
    int n_jobs;
    int total;
    unsigned int* counter;  // work counter in the workspace, zeroed before the launch
    int first[kMaxJobs + 1];  // first work item of each job
    int warp_form[kMaxJobs];  // 1: one scenario per warp (blockDim / 32 per item)
    DevPlan plans[kMaxJobs];
    SolveArgs args[kMaxJobs];
};

struct AdjArgs {
    int batch;
    int top_t;  // sweep the plan's top region in shared memory (else walk its levels)
    int ir_max;
    double ir_rtol;
    const double* dVm;
    const double* dVa;
    const double* dPg;
    const double* dQg;
    const double* Pd;     // forward inputs are not needed: gradients depend on V only
    double* dPd;
    double* dQd;
    double* dPg_in;
    double* dVset;
    int* adj_status;
    char* ws;
    SlotLayout L;
    // after a solve under reactive limits: the upper limits (to tell which limit a
    // switched bus sits at) and the gradients with respect to the limits
    const double* Qmax;
    double* dQmin;
    double* dQmax;
};

// Scenario-interleaved packs (placement PF_PLACE_INTERLEAVED): S scenarios share one
// workspace region in which every per-scenario quantity is stored item-major, [item][S],
// so that the S lanes of a slot touch S consecutive elements of each item; one
// thread-block cluster of `cluster` CTAs runs the pack.  Offsets are in bytes from the
// pack's base.
struct SiLayout {
    int S;              // scenarios per pack (2, 4, 8, 16 or 32)
    int cluster;        // CTAs per pack (one thread-block cluster)
    int threads;        // threads per CTA
    size_t pack_bytes;  // workspace bytes per pack
    size_t off_fac;     // factor: float4 [nnzb][S] (FP32) or double2 [nnzb][2][S] (FP64)
    size_t off_V, off_I, off_U, off_M, off_SP, off_DV;  // double2 [n_bus][S] each:
                        // V, I = Y V, u = e^{j theta}, (Vm, theta), (P_spec, Q_spec), dV
    size_t off_FA, off_FB;  // float4 [n_bus][S]: FP32 fill copies (V, u) and (Vm, u conj(I), 0)
    size_t off_F, off_DZ;   // double2 [n][S]: F1 and the accumulated Newton step
    size_t off_X;       // FT2 [n][S]: the triangular-solve vector
    size_t off_ctl;     // reduction buffers (3 x 32 u64) and singular flags (32 u32)
    size_t smem_bytes;  // dynamic shared memory per CTA (lane-group reductions, top region)
    // the top region of the pack's scenarios: scenario s on CTA s mod cluster, in the
    // CTA's arena at smem_top_off of the dynamic shared memory: top_slots slots of
    // top_stride bytes (blocks and solve vector), then the plan's lists once.  A CTA with
    // more scenarios than slots takes them top_slots at a time, keeping the factored
    // regions in the pack's factor between the factorisation and the sweeps
    size_t smem_top_off, top_stride;
    int top_slots;
};

struct SiArgs {
    int batch;
    // packs of the launch: pack k holds scenarios k q + min(k, r) .. of count q + (k < r)
    // (q = batch / npacks, r = batch % npacks; at most S each)
    int npacks, q, r;
    int max_iter;
    int ir_steps;
    double tol;
    double ir_rtol;
    double ir_gate;
    const double* Pd;
    const double* Qd;
    const double* Pg;
    const double* Vset;
    double* Vm;
    double* Va;
    double* Pg_out;
    double* Qg_out;
    double* fmis;
    int* iters;
    int* status;
    char* ws;
    SiLayout L;
};

// Vector arena carved from one base pointer (shared or global memory).
struct Arrays {
    // FP64, one entry per bus; (Uc, Us) = (cos theta, sin theta) is the unit phasor u
    double *Vm, *Va, *Uc, *Us, *Vre, *Vim, *Ire, *Iim, *dVre, *dVim;
    double *Psp, *Qsp, *w0, *w1, *gV;  // adjoint only (null in the forward layout)
    // FP64, two entries per pivot block
    double *F, *dz;
    double* r;                          // adjoint only
    // FP32 copies per bus feeding the FP32 Jacobian fill: V, u, Vm and u conj(I)
    float *fvr, *fvi, *fur, *fui, *fvm, *fpu, *fqu;
    void* x;  // FT[2n], the triangular-solve vector
    // per-scenario partition under reactive limits (null without limits): the current
    // bus type and, for PV buses switched to PQ, the reactive generation fixed at the limit
    signed char* stype;
    double* qfix;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Region rows per lane of the warp that sweeps the top region (its rows' x in registers).
constexpr int kTopSlots = 4;

// The top region's shared-memory arena: its blocks and one scratch block (ft bytes per
// value; idle lanes read and write the scratch block instead of branching), then its
// solve vector (2 values per row), then its staged index lists (nints ints).
__host__ __device__ inline size_t top_ts_off(int nblk, int ft) {
    return align_up((size_t)(nblk + 1) * 4 * ft, 16);
}
__host__ __device__ inline size_t top_ints_off(int nblk, int R, int ft) {
    return top_ts_off(nblk, ft) + align_up((size_t)2 * R * ft, 16);
}
__host__ __device__ inline size_t top_arena_bytes(int nblk, int R, int nints, int ft) {
    return R ? top_ints_off(nblk, R, ft) + align_up((size_t)4 * nints, 16) : 0;
}

// Arena layout shared by host (sizing) and device (carving).  In the forward layout the
// refinement's dV (FP64, two per bus) shares its bytes with the first four FP32 fill
// copies: the copies are written by the mismatch and read by the fill, dV is written and
// read by the refinement residual, later in the same Newton iteration.
__host__ __device__ inline size_t carve(unsigned char* base, int n_bus, int n, int ft_bytes,
                                        bool adjoint, Arrays* out) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + o;
        o = align_up(o + bytes, 16);
        return p;
    };
    const size_t db = sizeof(double) * (size_t)n_bus, fb = sizeof(float) * (size_t)n_bus;
    const size_t pb = sizeof(double) * 2 * (size_t)n;
    Arrays dummy;
    Arrays* a = out ? out : &dummy;
    double** bus_fwd[8] = {&a->Vm, &a->Va, &a->Uc, &a->Us, &a->Vre, &a->Vim, &a->Ire, &a->Iim};
    for (double** d : bus_fwd) *d = reinterpret_cast<double*>(take(db));
    a->F = reinterpret_cast<double*>(take(pb));
    a->dz = reinterpret_cast<double*>(take(pb));
    if (adjoint) {
        double** bus_adj[7] = {&a->dVre, &a->dVim, &a->Psp, &a->Qsp, &a->w0, &a->w1, &a->gV};
        for (double** d : bus_adj) *d = reinterpret_cast<double*>(take(db));
        a->r = reinterpret_cast<double*>(take(pb));
        float** f32[7] = {&a->fvr, &a->fvi, &a->fur, &a->fui, &a->fvm, &a->fpu, &a->fqu};
        for (float** f : f32) *f = reinterpret_cast<float*>(take(fb));
    } else {
        unsigned char* shared = take(2 * db);  // dV (2 x FP64) == fvr, fvi, fur, fui (4 x FP32)
        a->dVre = reinterpret_cast<double*>(shared);
        a->dVim = reinterpret_cast<double*>(shared + db);
        a->fvr = reinterpret_cast<float*>(shared);
        a->fvi = reinterpret_cast<float*>(shared + fb);
        a->fur = reinterpret_cast<float*>(shared + 2 * fb);
        a->fui = reinterpret_cast<float*>(shared + 3 * fb);
        float** f32[3] = {&a->fvm, &a->fpu, &a->fqu};
        for (float** f : f32) *f = reinterpret_cast<float*>(take(fb));
        a->Psp = a->Qsp = a->w0 = a->w1 = a->gV = a->r = nullptr;
    }
    a->x = take((size_t)ft_bytes * 2 * n);
    a->stype = nullptr;
    a->qfix = nullptr;
    return o;
}

}  // namespace pf
