// pf_device.cuh -- device-side data structures and small helpers (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

// Read-only plan arrays on the device (see pf_plan.h for their meaning).
struct DevPlan {
    int n_bus, n, nnzb, n_levels;
    const int* y_ptr;
    const int* y_idx;
    const double2* y_gb;  // (G, B) of every Ybus entry
    const int* bus_type;
    const int* pos2bus;
    const int* bus2pos;
    const int* lev_ptr;
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
};

// Per-scenario workspace slot (global memory), offsets in bytes from the slot base.
struct SlotLayout {
    size_t slot_bytes;
    size_t off_state;   // double Vm[n_bus], Va[n_bus]: the solution, for pf_adjoint
    size_t off_flags;   // int status, iters, has_factor, pad
    size_t off_fac;     // factor values (if stored in global memory), or 0
    size_t off_vec;     // vector arena (if it lives in global memory), or 0
    int fac_global;     // factor region present in the slot
    int fac_in_smem;    // factor staged in shared memory during the solve
    int vec_in_smem;    // vector arena in shared memory
    size_t smem_bytes;  // dynamic shared memory per CTA
    size_t smem_fac_off;
    size_t vec_bytes, fac_bytes;
};

struct SolveArgs {
    int batch;
    double tol;
    int max_iter;
    int ir_steps;
    double ir_rtol;
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
};

struct AdjArgs {
    int batch;
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
};

// Vector arena carved from one base pointer (shared or global memory).
// Per-bus FP64 arrays first, then the position-indexed (2 per pivot block) ones.
struct Arrays {
    double *Vm, *Va, *Psp, *Qsp, *Vre, *Vim, *Ire, *Iim, *dVre, *dVim, *w0, *w1, *gV;
    double *F, *dz, *r;
    void* x;  // FT[2n]
};
constexpr int kBusArrays = 13;
constexpr int kPosArrays = 3;

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Arena layout shared by host (sizing) and device (carving).
__host__ __device__ inline size_t carve(unsigned char* base, int n_bus, int n, int ft_bytes,
                                        Arrays* out) {
    size_t o = 0;
    double** bus_arr[kBusArrays] = {nullptr};
    double** pos_arr[kPosArrays] = {nullptr};
    if (out) {
        double** b[kBusArrays] = {&out->Vm, &out->Va, &out->Psp, &out->Qsp, &out->Vre,
                                  &out->Vim, &out->Ire, &out->Iim, &out->dVre, &out->dVim,
                                  &out->w0, &out->w1, &out->gV};
        double** q[kPosArrays] = {&out->F, &out->dz, &out->r};
        for (int k = 0; k < kBusArrays; ++k) bus_arr[k] = b[k];
        for (int k = 0; k < kPosArrays; ++k) pos_arr[k] = q[k];
    }
    for (int k = 0; k < kBusArrays; ++k) {
        if (out) *bus_arr[k] = reinterpret_cast<double*>(base + o);
        o = align_up(o + sizeof(double) * (size_t)n_bus, 16);
    }
    for (int k = 0; k < kPosArrays; ++k) {
        if (out) *pos_arr[k] = reinterpret_cast<double*>(base + o);
        o = align_up(o + sizeof(double) * 2 * (size_t)n, 16);
    }
    if (out) out->x = base + o;
    o = align_up(o + (size_t)ft_bytes * 2 * n, 16);
    return o;
}

}  // namespace pf
