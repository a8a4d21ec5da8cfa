// pf_plan.h -- host-side symbolic plan of one network (internal to libpf).
//
// The plan is the "one-time symbolic analysis" of Sec. III-B: everything about
// the Jacobian J1 of Eq. step1_jacobian that does not depend on the operating
// point.  It is built once per (Ybus pattern, bus types) and shared by every
// scenario of every batch.
//
// Unknowns and equations are grouped per non-slack bus into 2x2 blocks:
// unknowns (theta_i, Vm_i), equations (dP_i, dQ_i).  A PV bus has no Vm unknown
// and no dQ equation; its block row/column is padded with the identity
// equation dVm_i = 0, which keeps every block 2x2 and leaves the solution of the
// true unknowns unchanged (the padded row and column stay exactly zero off the
// diagonal through the elimination).
#pragma once

#include <cstdint>
#include <vector>

namespace pf {

struct Plan {
    // network
    int n_bus = 0, n_slack = 0, n_pv = 0, n_pq = 0;
    std::vector<int> y_ptr, y_idx;       // Ybus CSR, sorted columns, duplicates summed
    std::vector<double> y_g, y_b;        // Re / Im of Ybus entries
    std::vector<int> bus_type;           // 0 PQ, 1 PV, 2 slack
    std::vector<int> yt_ptr, yt_idx;     // transpose of Ybus (CSR of the columns)
    std::vector<double> yt_g, yt_b;

    // block ordering: position p in [0, n) <-> non-slack bus
    int n = 0;                           // number of 2x2 pivot blocks = |B \ R|
    std::vector<int> pos2bus, bus2pos;   // bus2pos = -1 for slack buses

    // elimination-tree levels: positions are sorted by level, so level l holds
    // the pivot range [lev_ptr[l], lev_ptr[l+1])
    int n_levels = 0;
    std::vector<int> lev_ptr;
    // lanes per gathered row (a power of two <= 32) for each level: forward (L part),
    // backward (U part) and Schur-target gathers
    std::vector<int> lev_gL, lev_gU, lev_gS;
    // dense tail: the last dense_s levels (from dense_l0 on) hold one row each and the
    // trailing dense_s x dense_s block of the filled pattern is full (0 = none)
    int dense_s = 0, dense_l0 = 0;
    // lanes per tail row for the gather of its part left of the tail (forward sweeps)
    int dense_g = 1;

    // block CSR of the filled L+U pattern in position order
    std::vector<int> lu_ptr, lu_col, lu_row, lu_diag, lu_mirror;
    std::vector<int> fill_y;             // Ybus entry of block (row bus, col bus), -1 = fill-in

    // factorisation schedule, per level l:
    //  phase A: L(i,k) <- A(i,k) * inv(A(k,k)) for the pairs la[la_ptr[l] .. la_ptr[l+1])
    //           stored as (block position of (i,k), block position of (k,k))
    //  phase B: A(i,j) -= L(i,k) * U(k,j) gathered per target block
    std::vector<int> la_ptr, la_L, la_D;
    std::vector<int> sch_tptr, sch_tgt, sch_cptr, sch_L, sch_U;

    // J1 as a scalar CSR in the paper's ordering (rows [dP_{B\R}; dQ_D], columns
    // [Vm_D; theta_{B\R}], each part in bus order; columns sorted within a row), and for
    // every Ybus entry (i, j) the positions of its up to four J1 entries
    // (dP_i/dtheta_j, dP_i/dVm_j, dQ_i/dtheta_j, dQ_i/dVm_j; -1 where absent): the
    // fixed template the block-diagonal export writes into (Sec. III-A, Alg. 1)
    int n1 = 0;
    std::vector<int> j1_ptr, j1_col, j1_pos;

    // statistics
    int nnz_j1 = 0;
    long long schur_ops = 0;
    int nnzb() const { return (int)lu_col.size(); }
};

enum BuildStatus { BUILD_OK = 0, BUILD_EINVAL = 1, BUILD_ESINGULAR = 2 };

// The schedule choices of a plan (none changes what is computed, only the elimination
// order, the levels and how their work is split): the ordering's degree slack, the
// largest dense tail, and the rule that splits a long gather over lane groups (rows
// longer than split_len blocks on levels of at most split_rows rows).
struct PlanParams {
    int order_slack = 1;
    int dense_max = 32;
    int split_len = 8;
    int split_rows = 128;
};

// Validates the inputs, sorts/sums the CSR and builds the whole plan.
BuildStatus build_plan(int n_bus, const int* y_indptr, const int* y_indices,
                       const double* y_re, const double* y_im, const int* bus_type,
                       Plan& plan, const PlanParams& params = PlanParams());

// Minimum-degree elimination order of an undirected graph given by sorted
// adjacency lists; also returns, for every node, its neighbours at the time it
// is eliminated (the row pattern of U in elimination terms).  Among the nodes whose
// degree is within `slack` of the minimum, the one lowest in the elimination tree
// built so far goes first (slack 0: ties only).
void minimum_degree(const std::vector<std::vector<int>>& adj,
                    std::vector<int>& order, std::vector<std::vector<int>>& structs,
                    int slack);

// The ordering's degree slack: 1 gave 24-30 % fewer elimination levels than exact
// minimum degree on the 118- to 2000-bus grids for 1-3 % more fill.
constexpr int kOrderSlack = 1;

// Largest dense tail the factorisation stages in shared memory (32 x 32 blocks: 16 KB in
// FP32, 32 KB in FP64 per scenario), and the smallest worth it.
constexpr int kDenseMax = 32;
constexpr int kDenseMin = 3;

}  // namespace pf
