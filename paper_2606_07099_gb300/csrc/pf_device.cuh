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
};

// Where one kernel keeps the scenario's vectors and factor (shared or global memory).
struct KernelSmem {
    int vec_in_smem;      // vector arena in shared memory
    int fac_in_smem;      // factor staged in shared memory
    size_t smem_bytes;    // dynamic shared memory per CTA
    size_t smem_fac_off;  // factor offset inside the dynamic shared memory
    size_t vec_bytes;     // size of this kernel's vector arena
};

// Per-scenario workspace slot (global memory), offsets in bytes from the slot base.
struct SlotLayout {
    size_t slot_bytes;
    size_t off_state;   // double Vm[n_bus], Va[n_bus]: the solution, for pf_adjoint
    size_t off_flags;   // int status, iters, has_factor, pad
    size_t off_fac;     // factor values (if stored in global memory), or 0
    size_t off_vec;     // vector arena (if a kernel keeps it in global memory), or 0
    int fac_global;     // factor region present in the slot
    size_t fac_bytes;
    KernelSmem fwd, adj;
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
struct Arrays {
    // FP64, one entry per bus; (Uc, Us) = (cos theta, sin theta) is the unit phasor u
    double *Vm, *Va, *Psp, *Qsp, *Uc, *Us, *Vre, *Vim, *Ire, *Iim, *dVre, *dVim;
    double *w0, *w1, *gV;  // adjoint only (null in the forward layout)
    // FP64, two entries per pivot block
    double *F, *dz, *r;
    // FP32 copies per bus feeding the FP32 Jacobian fill: V, u, Vm and u conj(I)
    float *fvr, *fvi, *fur, *fui, *fvm, *fpu, *fqu;
    void* x;  // FT[2n], the triangular-solve vector
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Arena layout shared by host (sizing) and device (carving).
__host__ __device__ inline size_t carve(unsigned char* base, int n_bus, int n, int ft_bytes,
                                        bool adjoint, Arrays* out) {
    size_t o = 0;
    auto d_bus = [&](double** dst) {
        if (out) *dst = reinterpret_cast<double*>(base + o);
        o = align_up(o + sizeof(double) * (size_t)n_bus, 16);
    };
    auto d_pos = [&](double** dst) {
        if (out) *dst = reinterpret_cast<double*>(base + o);
        o = align_up(o + sizeof(double) * 2 * (size_t)n, 16);
    };
    auto f_bus = [&](float** dst) {
        if (out) *dst = reinterpret_cast<float*>(base + o);
        o = align_up(o + sizeof(float) * (size_t)n_bus, 16);
    };
    Arrays dummy;
    Arrays* a = out ? out : &dummy;
    d_bus(&a->Vm); d_bus(&a->Va); d_bus(&a->Psp); d_bus(&a->Qsp); d_bus(&a->Uc); d_bus(&a->Us);
    d_bus(&a->Vre); d_bus(&a->Vim); d_bus(&a->Ire); d_bus(&a->Iim); d_bus(&a->dVre);
    d_bus(&a->dVim);
    if (adjoint) {
        d_bus(&a->w0); d_bus(&a->w1); d_bus(&a->gV);
    } else if (out) {
        out->w0 = out->w1 = out->gV = nullptr;
    }
    d_pos(&a->F); d_pos(&a->dz); d_pos(&a->r);
    f_bus(&a->fvr); f_bus(&a->fvi); f_bus(&a->fur); f_bus(&a->fui); f_bus(&a->fvm);
    f_bus(&a->fpu); f_bus(&a->fqu);
    if (out) out->x = base + o;
    o = align_up(o + (size_t)ft_bytes * 2 * n, 16);
    return o;
}

}  // namespace pf
