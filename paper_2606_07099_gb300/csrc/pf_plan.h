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
    // top region: the trailing levels top_l0 .. n_levels - 1 (rows top_p0 .. n - 1, top_R
    // of them; top_R = 0: none).  The factorisation and the sweeps take its pivots one at a
    // time in shared memory instead of level by level (few rows per level there, so a
    // level step is mostly latency).  Its blocks are the region rows' entries from column
    // top_p0 on, numbered row by row (local index r <-> fac position top_map[r]); every
    // list below holds local indices, which fit in 16 bits.
    int top_l0 = 0, top_p0 = 0, top_R = 0;
    int top_g = 1;                       // lanes per region row for its part left of the region
    std::vector<int> top_map;            // [blocks] fac position of each region block
    std::vector<int> top_split;          // [top_R] first entry of each region row inside it
    // staged into shared memory as one array: piv[R] (pivot blocks), lc_ptr[R + 1] and
    // lc[nl] (per pivot k, the L blocks (i, k), i > k), tr_ptr[R + 1] (per pivot, its range
    // of Schur triples), then the sweep rounds: fwk[nfw] and fw[32 nfw] (ascending columns
    // k, their L blocks (i, k), i > k), bwk[nbw] and bw[32 nbw] (descending columns, their
    // U blocks (i, k), i < k).  A round holds one entry per lane: the lane that owns row i
    // (i % 32) gets (i / 32) << 16 | block, the others -1; fwk holds the round's column,
    // bwk its column << 1 | (1 for the column's first round).  The forward solve's lists
    // end at top_nints_fwd; after them, the transposed sweeps' rounds (the adjoint):
    // ftk[nft] and ft[32 nft] (ascending columns j, U's row j: (k, U(j, k)), k > j; ftk
    // j << 1 | first, the first round applying the transposed pivot inverse), btk[nbt]
    // and bt[32 nbt] (descending columns i, L's row i: (k, L(i, k)), k < i; btk i)
    std::vector<int> top_ints;
    int top_nl = 0, top_nfw = 0, top_nbw = 0, top_nft = 0, top_nbt = 0, top_nints_fwd = 0;
    // Schur triples of the region pivots: (target, L block | U block << 16), per pivot
    std::vector<int> top_tr_t, top_tr_lu;
    int top_blocks() const { return (int)top_map.size(); }

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
// top region (trailing levels of at most top_rows rows each, while the region holds at
// most top_blocks blocks; top_rows 0, or fewer than top_min_pivots pivots in the network:
// none), and the rule that splits a long gather over
// lane groups (rows longer than split_len blocks on levels of at most split_rows rows).
struct PlanParams {
    int order_slack = 1;
    int top_rows = 4;
    int top_blocks = 2048;
    int top_min_pivots = 1024;  // smaller networks get no region
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

// Smallest top region worth its pivot-by-pivot schedule (rows), and the largest number of
// blocks a region may hold (its local indices are 16-bit).
constexpr int kTopMin = 3;
constexpr int kTopMaxBlocks = 65534;  // local indices (and the scratch block) in 16 bits
// Largest region in rows: each lane of the sweeping warp holds its rows' x in registers,
// 4 per lane (kTopSlots of the device code).
constexpr int kTopMaxRows = 128;
// Largest shared-memory arena of a region in FP64 (blocks of 32 bytes, the solve vector
// and the lists), so that it fits a CTA with room to spare for the rest of the kernel.
constexpr long long kTopMaxBytes = 160 * 1024;

}  // namespace pf
