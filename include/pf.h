/*
 * pf.h -- C ABI of the batched AC power-flow library (libpf).
 *
 * The library solves many AC power-flow scenarios that share one network
 * (one admittance matrix Ybus and one bus-type partition) with Newton-Raphson
 * on the polar mismatch equations, and differentiates the solution by the
 * implicit-function theorem.  It follows SABLE (arXiv 2606.07099):
 *
 *   - Sec. II-A: bus sets D (PQ), G (PV), R (slack/reference, any number >= 1),
 *     Ybus = G + jB, V_i = Vm_i e^{j theta_i}, dP = P_spec - P, dQ = Q_spec - Q;
 *   - Sec. II-B.1, Eqs. reduced_pf_system .. step1_jacobian: Step 1 solves
 *     F1 = [dP_{B\R}; dQ_D] = 0 for z1 = [Vm_D; theta_{B\R}] by Newton steps
 *     J1 dz = -F1 from the flat start of Sec. IV-A;
 *   - Eq. F2_completion: Step 2 recovers pg_R and qg_{B\D} explicitly;
 *   - Sec. II-B.2: the backward pass solves J1^T lambda = g_z1 and maps lambda to
 *     gradients (Eqs. chain_rule .. Jstep3_impl), here extended to the loads;
 *   - Sec. III-B, Alg. 1: the Jacobian values are refreshed in place on one fixed
 *     sparsity template computed once per network;
 *   - Sec. III-C, Table I: stagewise mixed precision (FP32 factorisation and
 *     triangular solves, FP64 mismatch, residuals and convergence control).
 *
 * Conventions shared by every call
 *   - Bus arrays are row-major [batch][n_bus] float64, bus index fastest.
 *   - bus_type: 0 = PQ (load), 1 = PV (generator), 2 = slack (reference).
 *   - "device" pointers are CUDA device (or managed) memory owned by the caller;
 *     "host" pointers are ordinary host memory owned by the caller and only read
 *     during the call.  The library keeps no pointer the caller passed in.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     pf_solve / pf_adjoint only enqueue work on it and return without waiting.
 *   - A non-PF_OK return code means the call did nothing on the device (argument
 *     or state errors are found before any launch), except PF_ECUDA, which
 *     reports a CUDA error raised by a launch.  Per-scenario numerical failure is
 *     never an error code: it is reported in the per-scenario `status` array.
 */
#ifndef PF_H_
#define PF_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_handle pf_handle; /* opaque; owns the network plan on host and device */

typedef enum {
    PF_OK = 0,
    PF_EINVAL = 1,             /* bad argument (size, pointer, bus types, CSR) */
    PF_ESINGULAR_PATTERN = 2,  /* a bus has no path to a slack bus, or no diagonal */
    PF_ENOMEM = 3,             /* host or device allocation failed (pf_create only) */
    PF_ECUDA = 4,              /* a CUDA runtime call failed */
    PF_ESTATE = 5,             /* pf_adjoint without a matching preceding pf_solve */
    PF_ENOTSUP = 6             /* no device path for this size (reported, not faked) */
} pf_err;

/* Per-scenario outcome, written to status[b]. */
typedef enum {
    PF_CONVERGED = 0, /* ||F1||_inf <= tol */
    PF_MAXITER = 1,   /* max_iter Newton steps done without reaching tol */
    PF_DIVERGED = 2,  /* non-finite mismatch or ||F1||_inf > 1e10 */
    PF_SINGULAR = 3   /* a pivot block of J1 was singular or non-finite */
} pf_status;

typedef enum {
    PF_FP64 = 0,  /* every stage in FP64 */
    PF_MIXED = 1  /* Table I: FP32 factor + solves, FP64 mismatch / residual / update,
                     with `ir_steps` FP64-residual refinement sweeps per Newton step */
} pf_precision;

/* Read-only facts about a network plan (host side). */
typedef struct {
    int n_bus;         /* buses */
    int n_slack;       /* |R| */
    int n_pv;          /* |G| */
    int n_pq;          /* |D| */
    int n_unknowns;    /* |z1| = |B\R| + |D|  (Newton unknowns) */
    int n_block;       /* 2x2 pivot blocks = |B\R| (PV buses padded with an identity row) */
    int nnz_ybus;      /* stored Ybus entries */
    int nnz_j1;        /* scalar nonzeros of J1 (Eq. step1_jacobian) */
    int nnzb_lu;       /* 2x2 blocks in the filled L+U pattern */
    int n_levels;      /* depth of the elimination tree */
    long long schur_block_ops; /* 2x2 multiply-subtracts of one factorisation */
    long long plan_bytes;      /* the network's device plan (shared by every scenario) */
    int top_pivots;            /* pivots of the top region: the trailing top_levels
                                  elimination levels (few rows each), whose pivots the LU
                                  and the sweeps take one at a time in shared memory
                                  instead of level by level (0: none) */
    int top_levels;            /* elimination levels in the top region */
    int top_blocks;            /* 2x2 blocks the top region holds in shared memory */
    int top_arena_bytes;       /* bytes of one scenario's top-region arena in FP64
                                  (blocks, solve vector, index lists), at most 160 KB */
} pf_plan_info;

/* Tunables of a solve; zero-initialise and set what you need. */
typedef struct {
    int precision;     /* pf_precision */
    int ir_steps;      /* PF_MIXED: max refinement sweeps per Newton step (0 = the paper's
                          scheme without refinement); ignored for PF_FP64 */
    double ir_rtol;    /* PF_MIXED: stop refining once ||r||_inf <= eta ||F1||_inf with the
                          forcing term eta = min(ir_rtol, ||F1||_inf) (loose far from the
                          solution, quadratic near it); 0 = always run ir_steps sweeps */
    int group_threads; /* threads per scenario (32..1024, multiple of 32; 0 = auto) */
    int keep_factors;  /* nonzero: store each scenario's last LU factor in the workspace
                          so that pf_adjoint can reuse it (required before pf_adjoint) */
    int placement;     /* pf_placement: where a scenario's vectors and factor live while
                          it is solved (0 = auto: the autotuned choice, else a heuristic) */
    int instances_per_cta; /* 0 = auto; 1 = one scenario per CTA of group_threads threads;
                          2..8 = that many scenarios per CTA, one warp each (group_threads
                          must then be 0 or 32) */
    double ir_gate;    /* PF_MIXED: check and refine a Newton step only once ||F1||_inf <=
                          ir_gate (far from the solution the Newton model error dwarfs the
                          FP32 solve error); 0 = every step */
    int pack;          /* PF_PLACE_INTERLEAVED: scenarios per pack (2, 4, 8, 16 or 32; 0 =
                          auto or the autotuned choice); ignored by the other placements */
    int cluster;       /* PF_PLACE_INTERLEAVED: CTAs per pack, one thread-block cluster
                          (1..16, 1 = a single CTA with CTA barriers; 0 = auto or the autotuned
                          choice); group_threads is then the threads per CTA (group_threads /
                          pack a power of two >= 16) */
} pf_solve_opts;

typedef enum {
    PF_PLACE_AUTO = 0,
    PF_PLACE_ONCHIP = 1,   /* vectors and factor in shared memory (if they fit) */
    PF_PLACE_VECTORS = 2,  /* vectors in shared memory, factor in the global workspace */
    PF_PLACE_GLOBAL = 3,   /* everything in the global workspace (most scenarios per SM) */
    PF_PLACE_FACTOR = 4,   /* factor in shared memory, vectors in the global workspace */
    PF_PLACE_INTERLEAVED = 5  /* scenario-interleaved packs: `pack` scenarios share one
                          workspace region with every quantity stored [item][scenario], and one
                          thread-block cluster of `cluster` CTAs runs the pack, each step of
                          the Newton iteration (and each elimination level) spread over all its
                          CTAs and separated by cluster barriers.  For networks whose factor
                          does not fit on chip.  Forward solves only (pf_solve, pf_solve_host,
                          pf_solve_noalloc): keep_factors and pf_solve_qlim get PF_ENOTSUP
                          when this placement is asked for explicitly; PF_PLACE_AUTO then uses
                          another placement */
} pf_placement;

/* Result of pf_autotune: the fastest launch configuration found for one precision. */
typedef struct {
    int group_threads;
    int placement;
    int instances_per_cta;
    float ms;              /* measured time of one pf_solve with that configuration */
    int pack;              /* PF_PLACE_INTERLEAVED: scenarios per pack and CTAs per cluster */
    int cluster;
} pf_tune_result;

/*
 * pf_build_ybus -- host helper: Ybus of pi-model branches (Sec. II-A's Ybus).
 * Branch k joins f[k] -> t[k] with series impedance r[k] + j x[k], total line
 * charging b[k] and off-nominal tap ratio tap[k] on the from side:
 *   Yff += (ys + j b/2) / tap^2, Ytt += ys + j b/2, Yft += Ytf += -ys / tap,
 * ys = 1 / (r + j x).  Output is CSR with sorted column indices and summed
 * duplicates.  Call once with indices/g/bv = NULL to get *nnz; then call again
 * with arrays of that size (indptr: n_bus + 1).  All pointers are host.
 * Errors: PF_EINVAL for n_bus < 1, n_branch < 0, a bus index out of range, a
 * zero series impedance or a non-positive tap, or *nnz too small on the second call.
 */
pf_err pf_build_ybus(int n_bus, int n_branch, const int* f, const int* t,
                     const double* r, const double* x, const double* b, const double* tap,
                     int* indptr, int* indices, double* g, double* bv, int* nnz);

/*
 * pf_create -- one-time symbolic analysis (Sec. III-B: pattern, indexing metadata
 * and LU analysis built once per topology) and upload of the plan to the current
 * CUDA device.  Host inputs: Ybus in CSR (n_bus x n_bus, y_re = G, y_im = B; any
 * column order; duplicates are summed) and bus_type[n_bus].  The plan holds the
 * fill-reducing ordering of the bus graph, the 2x2-block LU pattern, its
 * elimination-tree level schedule and the Jacobian fill map.  *out receives the
 * handle (NULL on error).  Errors: PF_EINVAL (bad sizes, bus types, no slack
 * bus, CSR out of range), PF_ESINGULAR_PATTERN (an island without a slack bus or
 * a non-slack bus without a diagonal entry), PF_ENOMEM, PF_ECUDA.
 */
pf_err pf_create(int n_bus, const int* y_indptr, const int* y_indices,
                 const double* y_re, const double* y_im, const int* bus_type,
                 pf_handle** out);

/*
 * The schedule choices of a plan (Sec. III-B's one-time analysis leaves them free; none
 * changes what is computed, only the elimination order, the level schedule and how the
 * levels' work is split, hence rounding and speed):
 *   order_slack: the fill-reducing minimum-degree ordering breaks ties, and near-ties up
 *     to this degree slack, towards a shallower elimination tree (0 = ties only);
 *   top_rows, top_blocks: the top region is made of the trailing elimination levels
 *     (from the top of the tree down) that hold at most top_rows rows each, as long as
 *     the region's blocks (its rows' entries from its first row on) number at most
 *     top_blocks (0..65534), its rows at most 128, and its FP64 shared-memory arena
 *     (blocks, solve vector, index lists) at most 160 KB.  The LU and the triangular
 *     sweeps take its pivots one at a time with the blocks in shared memory (16 bytes
 *     per block in the mixed form, 32 in FP64, plus the lists), instead of one
 *     barrier-separated step per level.  top_rows 0 = no region; regions under 3 rows
 *     are not used;
 *   top_min_pivots: networks with fewer pivot blocks get no region (their level steps
 *     are cheap, and a region's shared memory would cost scenarios in flight);
 *   split_len, split_rows: on levels of at most split_rows rows, a gathered row longer
 *     than split_len blocks is split over a power-of-two group of lanes (about four
 *     blocks each, at most 32 lanes), reduced in a fixed order.
 * pf_plan_opts_default writes the defaults pf_create uses (1, 4, 2048, 1024, 8, 128).
 */
typedef struct {
    int order_slack;
    int top_rows;
    int top_blocks;
    int top_min_pivots;
    int split_len;
    int split_rows;
} pf_plan_opts;

void pf_plan_opts_default(pf_plan_opts* opts);

/*
 * pf_create_ex -- pf_create with explicit schedule choices (host, NULL = the defaults).
 * Errors: as pf_create, and PF_EINVAL for order_slack outside 0..8, a negative top_rows,
 * top_min_pivots or split_rows, top_blocks outside 0..65534, or split_len < 1.
 */
pf_err pf_create_ex(int n_bus, const int* y_indptr, const int* y_indices,
                    const double* y_re, const double* y_im, const int* bus_type,
                    const pf_plan_opts* plan_opts, pf_handle** out);

/*
 * pf_analyze -- the host half of pf_create without any device work: validates the
 * network and runs the symbolic analysis, then reports the plan.  Inputs as in
 * pf_create (host).  If pos2bus / lu_ptr / lu_col / lev_ptr are non-NULL they
 * receive the block ordering (pos2bus[n_block]: bus of pivot position p), the
 * filled L+U block pattern in CSR over positions (lu_ptr[n_block + 1],
 * lu_col[nnzb_lu]) and the level ranges (lev_ptr[n_levels + 1]); if j1_ptr / j1_col
 * are non-NULL they receive the scalar J1 template of pf_jacobian_pattern
 * (j1_ptr[n_unknowns + 1], j1_col[nnz_j1]).  Call first with them NULL to learn the
 * sizes from *info.  Errors as pf_create, minus PF_ENOMEM / PF_ECUDA.
 */
pf_err pf_analyze(int n_bus, const int* y_indptr, const int* y_indices,
                  const double* y_re, const double* y_im, const int* bus_type,
                  pf_plan_info* info, int* pos2bus, int* lu_ptr, int* lu_col, int* lev_ptr,
                  int* j1_ptr, int* j1_col);

/*
 * pf_analyze_ex -- pf_analyze with explicit schedule choices (host, NULL = the defaults,
 * as in pf_create_ex): the plan pf_create_ex would build, without any device work.
 * Errors: as pf_analyze, and PF_EINVAL for schedule choices pf_create_ex refuses.
 */
pf_err pf_analyze_ex(int n_bus, const int* y_indptr, const int* y_indices,
                     const double* y_re, const double* y_im, const int* bus_type,
                     const pf_plan_opts* plan_opts, pf_plan_info* info, int* pos2bus,
                     int* lu_ptr, int* lu_col, int* lev_ptr, int* j1_ptr, int* j1_col);

/* Plan facts (host only, no device work).  PF_EINVAL on NULL arguments. */
pf_err pf_get_plan_info(const pf_handle* h, pf_plan_info* info);

/*
 * pf_jacobian_pattern -- the fixed sparse template of J1 (Eq. step1_jacobian) of one
 * scenario as a scalar CSR in the paper's ordering (host output): rows
 * [dP_{B\R}; dQ_D], columns z1 = [Vm_D; theta_{B\R}], each part in bus order, columns
 * ascending within a row; one entry per Ybus entry (i, j) and applicable (row, column)
 * pair.  j1_ptr[n_unknowns + 1], j1_col[nnz_j1] (sizes from pf_plan_info).  This is the
 * per-scenario block of the block-diagonal embedding (BDE) of Sec. III-A.
 * Errors: PF_EINVAL on NULL arguments.
 */
pf_err pf_jacobian_pattern(const pf_handle* h, int* j1_ptr, int* j1_col);

/*
 * pf_bde_pattern -- the index arrays of the block-diagonal embedding (Sec. III-A) of
 * `batch` scenarios, written on the device: one CSR of size (batch n1) x (batch n1)
 * whose diagonal block k is the J1 template shifted by k n1 (n1 = n_unknowns):
 * row_ptr[batch n1 + 1] (device int) and col_idx[batch nnz_j1] (device int).  The
 * pattern is fixed; pf_export_jacobian refreshes only the values.  Asynchronous on
 * `stream`.  Errors: PF_EINVAL (NULL, batch < 1, batch nnz_j1 >= 2^31), PF_ECUDA.
 */
pf_err pf_bde_pattern(const pf_handle* h, int batch, int* row_ptr, int* col_idx, void* stream);

/*
 * pf_export_jacobian -- the values of J1 = dF1/dz1 (Eq. step1_jacobian, element formulas
 * of Alg. 1) of `batch` scenarios at the voltages Vm, Va (device, [batch][n_bus],
 * FP64), written in FP64 into values[batch][nnz_j1] (device) in the order of
 * pf_jacobian_pattern: scenario k's values are the k-th block of the BDE matrix of
 * pf_bde_pattern (an in-place value update of the fixed template, Sec. III-A/III-B).
 * Inputs at slack buses are read for V only.  Asynchronous on `stream`.  For callers
 * that hand the batch to another sparse solver; pf_solve itself never forms this
 * matrix (it fills its factor directly).  Errors: PF_EINVAL, PF_ECUDA.
 */
pf_err pf_export_jacobian(const pf_handle* h, int batch, const double* Vm, const double* Va,
                          double* values, void* stream);

/*
 * pf_workspace_size -- device bytes pf_solve / pf_adjoint need for `batch`
 * scenarios with these options (placement PF_PLACE_AUTO: the placement pf_solve would
 * pick now; PF_PLACE_GLOBAL needs the most and serves every placement).  The caller
 * allocates the workspace (any device allocator, 256-byte alignment) and passes the
 * same buffer to pf_adjoint after pf_solve.  Errors: PF_EINVAL.
 */
pf_err pf_workspace_size(const pf_handle* h, int batch, const pf_solve_opts* opts,
                         size_t* bytes);

/*
 * pf_solve -- batched Newton-Raphson power flow, Step 1 + Step 2 of Sec. II-B.1.
 * Inputs (device, [batch][n_bus]): Pd, Qd loads; Pg generation (read on PV buses
 * only); Vset voltage set points (read on PV and slack buses only).  Flat start:
 * Vm = 1 on PQ buses, Vset elsewhere, theta = 0.  Each scenario iterates until
 * ||F1||_inf <= tol (checked before every Newton step) or max_iter steps.
 * Outputs (device): Vm, Va [batch][n_bus] (the final iterate); Pg_out, Qg_out
 * [batch][n_bus] -- the completed generation of Eq. F2_completion (Pg_out: the
 * input pg on G, the recovered pg_R on R, 0 on D; Qg_out: recovered qg on B\D,
 * 0 on D); iters[batch] (Newton steps taken), status[batch] (pf_status),
 * final_mismatch[batch] (||F1||_inf of the final iterate).  Any output pointer
 * except Vm, Va, status may be NULL.  Errors: PF_EINVAL (batch < 1, tol <= 0,
 * max_iter < 0, NULL input, workspace too small), PF_ENOTSUP, PF_ECUDA.
 */
pf_err pf_solve(pf_handle* h, int batch,
                const double* Pd, const double* Qd, const double* Pg, const double* Vset,
                double tol, int max_iter, const pf_solve_opts* opts,
                double* Vm, double* Va, double* Pg_out, double* Qg_out,
                int* iters, int* status, double* final_mismatch,
                void* workspace, size_t workspace_bytes, void* stream);

/*
 * pf_solve_host -- pf_solve whose per-scenario arrays may live in host memory: each of
 * Pd, Qd, Pg, Vset, Vm, Va, Pg_out, Qg_out, iters, status, final_mismatch (same layouts
 * and NULL rules as pf_solve) may be page-locked host memory (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister) or device memory of the handle's device.  The solve
 * kernel reads and writes them in place through the unified address space: on a
 * coherent CPU-GPU link (NVLink-C2C) every scenario's rows move while other scenarios
 * compute, with no separate copy before or after the launch.  The outputs are complete
 * once `stream` has been synchronised.  Every array (and the device workspace) is checked
 * before anything is launched: it must lie, for all the bytes the call touches, inside
 * one allocation that CUDA knows and that kernels on the handle's device address at the
 * same pointer value; otherwise (pageable memory, a range past the end of an allocation,
 * another device's memory) the call returns PF_EINVAL and does nothing.  With
 * PF_PLACE_AUTO a per-scenario placement serves this call (the fastest per-scenario
 * shape of the last pf_autotune, also when the tuning picked interleaved packs): those
 * kernels read each scenario's host rows over its Newton iterations, while interleaved
 * packs read them in one burst before the solve starts, which measured slower end to end.
 * The workspace must then hold pf_workspace_size for PF_PLACE_GLOBAL (the largest
 * per-scenario slot).  Errors: those of pf_solve.
 */
pf_err pf_solve_host(pf_handle* h, int batch,
                     const double* Pd, const double* Qd, const double* Pg, const double* Vset,
                     double tol, int max_iter, const pf_solve_opts* opts,
                     double* Vm, double* Va, double* Pg_out, double* Qg_out,
                     int* iters, int* status, double* final_mismatch,
                     void* workspace, size_t workspace_bytes, void* stream);

/*
 * pf_addressable -- whether [ptr, ptr + bytes) lies inside one allocation that CUDA knows
 * (page-locked host memory, or device memory of the handle's device) and that kernels
 * on that device address at the same pointer value: the check pf_solve_host applies to
 * each of its arrays.  Writes 1 or 0 to *ok; launches nothing.  Errors: PF_EINVAL (NULL
 * h or ok).
 */
pf_err pf_addressable(const pf_handle* h, const void* ptr, size_t bytes, int* ok);

/*
 * pf_qlim_workspace_size -- device bytes pf_solve_qlim needs for `batch` scenarios with
 * these options (the pf_solve workspace plus the scenario's own bus partition).
 * opts->keep_factors must be 0.  Errors: PF_EINVAL.
 */
pf_err pf_qlim_workspace_size(const pf_handle* h, int batch, const pf_solve_opts* opts,
                              size_t* bytes);

/*
 * pf_solve_qlim -- pf_solve with reactive-power limits at the PV buses.  The paper has
 * no counterpart (its PV buses hold Vm at any reactive output); this is the PV -> PQ
 * switching of production power-flow tools, around the same Step 1 / Step 2.
 * When a scenario has converged, every bus of it that is still PV and whose recovered
 * reactive generation qg = Q + qd lies outside [Qmin, Qmax] becomes a PQ bus of that
 * scenario with qg fixed at the violated limit (all violators at once); Newton then
 * continues from the current voltages on the new partition, with max_iter steps per
 * round.  A switched bus stays PQ.  The symbolic plan is unchanged: every bus already
 * owns a full 2x2 block of the factor pattern (a PV bus's Vm row and column are padded
 * with the identity), so a switch changes values only.
 * Inputs as pf_solve, plus Qmin, Qmax (device, [batch][n_bus], read on PV buses).
 * Outputs as pf_solve (Pg_out and Qg_out on the network's bus sets: a switched bus
 * reports its input pg and its qg, at the limit), plus bus_type_out (device int,
 * [batch][n_bus], nullable: the final partition of each scenario) and rounds (device
 * int [batch], nullable: switching rounds taken); iters counts the Newton steps of all
 * rounds.  status: PF_CONVERGED when a converged round leaves no violator;
 * PF_MAXITER when a round ran out of steps or violators remain after max_rounds rounds
 * (the outputs are then the last converged point, on its partition); PF_DIVERGED /
 * PF_SINGULAR as pf_solve.  With keep_factors the workspace (pf_qlim_workspace_size with
 * the same options) keeps each scenario's factor and final partition for
 * pf_adjoint_qlim (plain pf_adjoint refuses it with PF_ESTATE).
 * Errors: as pf_solve, and PF_EINVAL for NULL limits or max_rounds < 0.
 */
pf_err pf_solve_qlim(pf_handle* h, int batch,
                     const double* Pd, const double* Qd, const double* Pg, const double* Vset,
                     const double* Qmin, const double* Qmax,
                     double tol, int max_iter, int max_rounds, const pf_solve_opts* opts,
                     double* Vm, double* Va, double* Pg_out, double* Qg_out,
                     int* iters, int* status, double* final_mismatch,
                     int* bus_type_out, int* rounds,
                     void* workspace, size_t workspace_bytes, void* stream);

/*
 * pf_bde_workspace_size / pf_solve_bde -- the same Newton-Raphson solve (Step 1 + Step 2,
 * FP64 form: inputs, outputs, flags and iteration semantics as pf_solve) run the way the
 * paper runs a batch: as ONE block-diagonal matrix (Sec. III-A), with one batch-wide
 * kernel per phase and, for the factorisation and the triangular sweeps, one per
 * elimination-tree level, the host checking convergence after every mismatch.  Values are
 * stored scenario-interleaved in the workspace (pf_bde_workspace_size bytes, 256-byte
 * aligned).  It exists to measure that execution model beside the fused one-launch
 * pf_solve on the same plan and arithmetic; it is stream-synchronous (one host read per
 * Newton iteration) and leaves no state for pf_adjoint.  Errors: PF_EINVAL, PF_ECUDA.
 */
pf_err pf_bde_workspace_size(const pf_handle* h, int batch, size_t* bytes);
pf_err pf_solve_bde(pf_handle* h, int batch,
                    const double* Pd, const double* Qd, const double* Pg, const double* Vset,
                    double tol, int max_iter,
                    double* Vm, double* Va, double* Pg_out, double* Qg_out,
                    int* iters, int* status, double* final_mismatch,
                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * pf_adjoint_qlim -- the implicit-differentiation backward pass (Sec. II-B.2) of the
 * preceding pf_solve_qlim with keep_factors on this handle.  At a converged solution a
 * switched bus k is a PQ bus with fixed reactive injection qlim_k - qd_k: the adjoint
 * runs on each scenario's final partition, with qlim an input.  Cotangents and outputs as
 * pf_adjoint, with: dPg_in nonzero on the network's PV buses (switched ones included),
 * dVset zero at switched buses (their Vm is an unknown), and dQmin / dQmax (device,
 * [batch][n_bus]) the gradients with respect to the limit each switched bus sits at
 * (zero elsewhere; Qmax, the limits given to the solve, tells which one).  The paper has
 * no counterpart (it has no reactive limits).  Errors: PF_EINVAL (NULL, sizes),
 * PF_ESTATE (no matching preceding pf_solve_qlim with keep_factors), PF_ECUDA.
 */
pf_err pf_adjoint_qlim(pf_handle* h, int batch,
                       const double* dVm, const double* dVa, const double* dPg, const double* dQg,
                       const double* Qmax,
                       double* dPd, double* dQd, double* dPg_in, double* dVset,
                       double* dQmin, double* dQmax, int* adj_status,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * pf_autotune -- picks the launch configuration (threads per scenario and placement
 * of the scenario data) for this handle, `batch` and opts->precision by timing
 * pf_solve on the given inputs (device, as pf_solve) for every candidate: 32..1024
 * threads per scenario, or 2, 4 or 8 one-warp scenarios per CTA, times every placement
 * that fits; and, without keep_factors, interleaved packs: 2 to 32 scenarios on one CTA
 * of 256, 512 or 1024 threads, or 4 to 16 scenarios on clusters of 2 to 16 CTAs of 512 or
 * 1024 threads, the shapes that occupy at least half of the SMs (or use 16-CTA clusters)
 * and whose workspace fits the one given (the best shape depends on the batch: a few scenarios of a large network
 * want the most threads each, thousands of small ones the most scenarios per SM).  The fastest one is kept in
 * the handle and used by later pf_solve calls with group_threads = 0 and placement =
 * PF_PLACE_AUTO at the same precision; *out (nullable) receives it.  The workspace
 * must hold pf_workspace_size for PF_PLACE_GLOBAL; the call allocates small temporary
 * output buffers of its own.  Not the hot path: it launches every
 * candidate several times and waits for the device (stream-synchronous).
 * Errors: as pf_solve.
 */
pf_err pf_autotune(pf_handle* h, int batch,
                   const double* Pd, const double* Qd, const double* Pg, const double* Vset,
                   double tol, int max_iter, const pf_solve_opts* opts,
                   void* workspace, size_t workspace_bytes, void* stream, pf_tune_result* out);

/*
 * One network's part of a pf_solve_multi call: the handle, its batch and the same
 * device arrays pf_solve takes ([batch][n_bus of h]; Pg_out, Qg_out, iters and
 * final_mismatch may be NULL).
 */
typedef struct {
    pf_handle* h;
    int batch;
    const double *Pd, *Qd, *Pg, *Vset;
    double *Vm, *Va, *Pg_out, *Qg_out;
    int *iters, *status;
    double* final_mismatch;
} pf_job;

#define PF_MAX_JOBS 8

/*
 * pf_multi_workspace_size -- workspace bytes for pf_solve_multi over these jobs, and
 * (job_offsets, nullable, n_jobs entries) where each job's part starts inside it.
 * Errors: PF_EINVAL (n_jobs outside 1..PF_MAX_JOBS, a NULL handle, batch < 1, bad opts).
 */
pf_err pf_multi_workspace_size(int n_jobs, const pf_job* jobs, const pf_solve_opts* opts,
                               size_t* bytes, size_t* job_offsets);

/*
 * pf_solve_multi -- the scenarios of several networks (grids of different sizes, uneven
 * batches) in ONE persistent launch.  CTAs take work items from a device work counter,
 * the most expensive network's first, and run each with its own plan: same Newton
 * iteration, outputs and status as pf_solve per job.  CTAs have group_threads threads
 * (0 = 256; 64 to 512).  opts->placement PF_PLACE_AUTO gives each network its own form:
 * networks of up to 160 buses one scenario per warp (group_threads / 32 per item, data
 * on chip when they fit), larger ones the whole CTA per scenario with the factor in
 * shared memory when it fits; PF_PLACE_GLOBAL runs every network with the whole CTA from
 * the global workspace.  instances_per_cta must be 0 or 1.
 * With keep_factors, each job's handle remembers its part of the workspace, so
 * pf_adjoint(job.h, job.batch, ..., workspace + job_offsets[j], ...) differentiates it.
 * All handles must live on the current device.  Errors: PF_EINVAL, PF_ENOTSUP (the
 * jobs' shared memory does not fit one CTA of this size), PF_ECUDA.
 */
pf_err pf_solve_multi(int n_jobs, const pf_job* jobs, double tol, int max_iter,
                      const pf_solve_opts* opts, void* workspace, size_t workspace_bytes,
                      void* stream);

/*
 * pf_autotune_multi -- picks the launch shape of pf_solve_multi for these jobs by timing
 * it on their inputs (device, as pf_solve_multi) for every candidate: 128, 256 and 512
 * threads per CTA, each with PF_PLACE_AUTO (per-network forms) and PF_PLACE_GLOBAL
 * (every network from the global workspace); shapes whose shared memory does not fit
 * are skipped.  Each candidate runs once to warm up and three times timed (CUDA events
 * on `stream`); *out (host) receives the fastest: group_threads, placement,
 * instances_per_cta = 1 and its best time in ms.  Pass those two fields in the opts of
 * later pf_solve_multi calls.  The workspace must hold pf_multi_workspace_size of every
 * candidate shape (the largest of the six).  Not the hot path: it waits for the
 * device after every trial; the trial solves overwrite the jobs' outputs and leave no
 * adjoint state.  Errors: PF_EINVAL, PF_ENOTSUP (no candidate fits), PF_ECUDA.
 */
pf_err pf_autotune_multi(int n_jobs, const pf_job* jobs, double tol, int max_iter,
                         const pf_solve_opts* opts, void* workspace, size_t workspace_bytes,
                         void* stream, pf_tune_result* out);

/*
 * pf_adjoint -- implicit-differentiation backward pass of Sec. II-B.2 at the
 * solution returned by the preceding pf_solve on this handle (same batch, same
 * workspace, keep_factors set).  Cotangents (device, [batch][n_bus]; dPg and dQg
 * may be NULL = 0): dVm, dVa, dPg, dQg with respect to the pf_solve outputs
 * Vm, Va, Pg_out, Qg_out.  Outputs (device, [batch][n_bus]): gradients with
 * respect to the pf_solve inputs -- dPd, dQd, dPg_in (nonzero on G only), dVset
 * (nonzero on B\D only).  The transposed system J1^T lambda = g_z1 is solved with
 * the stored factors of the last Newton step as preconditioner and FP64-residual
 * refinement against J1 at the solution; a scenario whose refinement stalls is
 * refactored at the solution.  adj_status[batch] (nullable) gets 0 on success,
 * 3 (PF_SINGULAR) if the refactorisation failed, and copies the forward status
 * for scenarios that did not converge (their gradients are written as 0).
 * Errors: PF_EINVAL, PF_ESTATE (no preceding pf_solve with keep_factors, or a
 * different batch), PF_ECUDA.
 */
pf_err pf_adjoint(pf_handle* h, int batch,
                  const double* dVm, const double* dVa, const double* dPg, const double* dQg,
                  double* dPd, double* dQd, double* dPg_in, double* dVset, int* adj_status,
                  void* workspace, size_t workspace_bytes, void* stream);

/*
 * pf_solve_noalloc -- pf_solve for callers that cannot allocate device memory.
 * The paper has no counterpart: this entry point exists for callers that may not
 * call cudaMalloc (code running while another part of the process captures a CUDA
 * graph, plug-ins whose host application owns the device allocator, real-time
 * loops with a memory budget fixed at start-up).  It takes the same arguments as
 * pf_solve minus the workspace: the per-scenario scratch lives in a static device
 * array of PF_NOALLOC_SCRATCH_BYTES that the library holds on every device it is
 * loaded on until the process exits.  No allocation of any kind happens inside.
 *   - pf_create looks the array's device address up on the handle's device and
 *     keeps it on the handle.  Under lazy module loading that lookup may be what
 *     loads the module holding the array and commits its memory, so it happens in
 *     pf_create (which allocates anyway), never in pf_solve_noalloc.  A device reset
 *     ends the handle together with that address.
 *   - All calls share the array: calls whose kernels overlap on the GPU race and
 *     corrupt each other; order them on one stream.  Nothing in it needs clearing.
 *   - keep_factors must be 0 (pf_adjoint needs a caller-owned workspace).
 * Errors: PF_EINVAL when keep_factors is set or when the batch needs more scratch
 * than PF_NOALLOC_SCRATCH_BYTES (pf_workspace_size tells the need); PF_ECUDA when
 * pf_create could not look the array up; plus every error of pf_solve.
 */
#define PF_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
pf_err pf_solve_noalloc(pf_handle* h, int batch,
                        const double* Pd, const double* Qd, const double* Pg, const double* Vset,
                        double tol, int max_iter, const pf_solve_opts* opts,
                        double* Vm, double* Va, double* Pg_out, double* Qg_out,
                        int* iters, int* status, double* final_mismatch, void* stream);

/*
 * pf_measure_fma_peak -- measured fused multiply-add throughput of the current device
 * (not part of the paper's method: the denominator of the ALU roofline that the solve
 * kernels are reported against, taken on the same GPU and at the same clocks).
 * fp64 != 0 measures FP64 FMA, else FP32 FMA: 8 CTAs of 256 threads per SM, each thread
 * running 8 independent FMA chains of `iters` steps (>= 16), timed with CUDA events on
 * `stream` after one shorter warm-up launch.  Writes TFLOP/s (2 flop per FMA) to *tflops
 * (host).  Synchronises on the stream.  Errors: PF_EINVAL, PF_ECUDA.
 */
pf_err pf_measure_fma_peak(int fp64, int iters, double* tflops, void* stream);

/* pf_destroy -- frees the handle's host and device memory (waits for the device). */
void pf_destroy(pf_handle* h);

/* pf_error_string -- static text for an error code. */
const char* pf_error_string(pf_err e);

#ifdef __cplusplus
}
#endif

#endif /* PF_H_ */
