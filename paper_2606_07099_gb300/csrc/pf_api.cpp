// pf_api.cpp -- the C ABI of libpf (declared in include/pf.h).
//
// Host-side responsibilities only: argument checks, the one-time plan
// (pf_plan.cpp), its upload, the shared-memory/workspace layout of a solve, and
// the kernel launches (pf_kernels.cu).  No numerical work runs here.
#include <cuda.h>  // pointer-attribute types only; the driver function is fetched at run time
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pf.h"
#include "pf_launch.h"
#include "pf_plan.h"

struct pf_handle {
    pf::Plan plan;
    int device = 0;
    int smem_optin = 0;
    int num_sms = 0;
    void* d_buf = nullptr;
    pf::DevPlan dp{};
    // autotuned launch configuration per precision (index 0 = FP64, 1 = mixed)
    pf_tune_result tuned[2] = {{0, 0, 0, 0.f}, {0, 0, 0, 0.f}};
    // the fastest per-scenario configuration of the same tuning run: the choice for the
    // calls the interleaved placement does not serve (kept factors, reactive limits)
    pf_tune_result tuned_ps[2] = {{0, 0, 0, 0.f}, {0, 0, 0, 0.f}};
    // state of the last pf_solve (for pf_adjoint)
    int last_batch = -1;
    int last_ft = 0;
    int last_keep = 0;
    int last_threads = 0;
    const void* last_ws = nullptr;
    pf::SlotLayout last_layout{};
    size_t plan_bytes = 0;  // the device plan buffer
    int last_qlim = 0;      // the last solve ran under reactive limits (pf_adjoint_qlim)
    void* noalloc_scratch = nullptr;  // device address of pf_solve_noalloc's static scratch
                                      // array on this handle's device (null: lookup failed)
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

int auto_threads(int n) {
    if (n <= 48) return 32;
    if (n <= 160) return 128;
    if (n <= 400) return 128;
    if (n <= 1600) return 128;
    if (n <= 6000) return 256;
    return 512;
}

// Shared memory reserved for the kernels' static arrays and the runtime.
constexpr size_t kStaticSmemReserve = 1024;

// Shared-memory placement of one kernel (pf_placement): vectors and factor in shared
// memory, vectors only, or neither (everything streams from the global slot).  A
// placement that does not fit falls back to the next one down.
// The triangular-solve vector is the only vector every level of a sweep reads right
// after an earlier level wrote it; when the vectors live in the global workspace it
// still goes to shared memory if it is small (<= 8 KB).
constexpr size_t kXSmemMax = 8 * 1024;

void add_x(pf::KernelSmem& k, size_t x_bytes, size_t budget) {
    if (k.vec_in_smem || x_bytes > kXSmemMax || k.smem_bytes + x_bytes > budget) return;
    k.x_in_smem = 1;
    k.smem_x_off = k.smem_bytes;
    k.smem_bytes += pf::align_up(x_bytes, 16);
}

pf::KernelSmem place(size_t vec_bytes, size_t fac_bytes, size_t budget, int placement,
                     size_t x_bytes = kXSmemMax + 1) {
    pf::KernelSmem k{};
    k.vec_bytes = vec_bytes;
    if (placement == PF_PLACE_FACTOR) {
        if (fac_bytes <= budget) {
            k.fac_in_smem = 1;
            k.smem_fac_off = 0;
            k.smem_bytes = fac_bytes;
        }
        add_x(k, x_bytes, budget);
        return k;
    }
    if (placement <= PF_PLACE_ONCHIP && vec_bytes + fac_bytes <= budget) {
        k.vec_in_smem = 1;
        k.fac_in_smem = 1;
        k.smem_fac_off = vec_bytes;
        k.smem_bytes = vec_bytes + fac_bytes;
    } else if (placement <= PF_PLACE_VECTORS && vec_bytes <= budget) {
        k.vec_in_smem = 1;
        k.smem_bytes = vec_bytes;
    }
    add_x(k, x_bytes, budget);
    return k;
}

size_t smem_budget(const pf_handle* h) {
    return (size_t)h->smem_optin > kStaticSmemReserve ? (size_t)h->smem_optin - kStaticSmemReserve : 0;
}

static_assert(pf::kTopMaxRows == 32 * pf::kTopSlots, "region rows: one register slot per row");

// Shared memory an SM may give the adjoint's top-region arenas (see pf_adjoint).
constexpr size_t kTopAdjSmemPerSm = 128 * 1024;

// Shared memory of the top region's arena (its blocks, solve vector and lists: the
// forward solve's, or with `adj` the adjoint's, which also holds the transposed rounds).
size_t top_bytes(const pf::Plan& P, int ft_bytes, bool adj = false) {
    return pf::top_arena_bytes(P.top_blocks(), P.top_R,
                               adj ? (int)P.top_ints.size() : P.top_nints_fwd, ft_bytes);
}

// Default placement without tuning data: keep a scenario on chip only while at least
// three of them fit on one SM (76 KB each); past that, more scenarios in flight from
// the global workspace beat fewer scenarios in shared memory.
int heuristic_placement(const pf_handle* h, int ft_bytes) {
    const pf::Plan& P = h->plan;
    const size_t vec = pf::carve(nullptr, P.n_bus, P.n, ft_bytes, false, nullptr);
    const size_t fac = pf::align_up((size_t)P.nnzb() * 4 * ft_bytes, 16);
    const size_t lim = std::min<size_t>(smem_budget(h), 76 * 1024);
    if (vec + fac <= lim) return PF_PLACE_ONCHIP;
    if (vec <= lim) return PF_PLACE_VECTORS;
    return PF_PLACE_GLOBAL;
}

pf::SlotLayout make_layout(const pf_handle* h, int ft_bytes, int keep, int placement,
                           bool qlim = false) {
    const pf::Plan& P = h->plan;
    pf::SlotLayout L{};
    L.fac_bytes = pf::align_up((size_t)P.nnzb() * 4 * ft_bytes, 16);
    // the top region's arena comes out of the budget first, then follows the placement's
    // own arrays (a multiple of 16 bytes: warp arenas are laid end to end)
    const size_t top = top_bytes(P, ft_bytes), top_adj = top_bytes(P, ft_bytes, true);
    const size_t full = smem_budget(h);
    L.fwd = place(pf::carve(nullptr, P.n_bus, P.n, ft_bytes, false, nullptr), L.fac_bytes,
                  full > top ? full - top : 0, placement, (size_t)ft_bytes * 2 * (size_t)P.n);
    L.adj = place(pf::carve(nullptr, P.n_bus, P.n, ft_bytes, true, nullptr), L.fac_bytes,
                  full > top_adj ? full - top_adj : 0, placement);
    L.fwd.smem_top_off = pf::align_up(L.fwd.smem_bytes, 16);
    L.fwd.smem_bytes = L.fwd.smem_top_off + top;
    L.adj.smem_top_off = pf::align_up(L.adj.smem_bytes, 16);
    L.adj.smem_bytes = L.adj.smem_top_off + top_adj;
    L.fac_global = (!L.fwd.fac_in_smem || keep) ? 1 : 0;
    size_t vec_global = 0;
    if (!L.fwd.vec_in_smem) vec_global = std::max(vec_global, L.fwd.vec_bytes);
    if (keep && !L.adj.vec_in_smem) vec_global = std::max(vec_global, L.adj.vec_bytes);
    size_t o = 0;
    L.off_state = o;  // kept factors: Vm, Va, Uc, Us, Ire, Iim at the solution; else Vm, Va
    o = pf::align_up(o + sizeof(double) * (keep ? 6 : 2) * (size_t)P.n_bus, 256);
    L.off_flags = o;
    o = pf::align_up(o + 16, 256);
    if (L.fac_global) {
        L.off_fac = o;
        o = pf::align_up(o + L.fac_bytes, 256);
    }
    if (vec_global) {
        L.off_vec = o;
        o = pf::align_up(o + vec_global, 256);
    }
    if (qlim) {  // per-scenario partition: int8 type per bus, then FP64 fixed qg per bus
        L.off_qlim = o;
        o = pf::align_up(o + pf::align_up((size_t)P.n_bus, 16) + sizeof(double) * (size_t)P.n_bus, 256);
    }
    L.slot_bytes = o;
    return L;
}

struct LaunchCfg {
    int threads;
    int placement;   // -1: the interleaved placement was asked for where it does not apply
    int ipc;
    int S, cluster;  // PF_PLACE_INTERLEAVED: scenarios per pack, CTAs per cluster
};

// Interleaved packs without tuning data: 16 scenarios per pack from 256 scenarios up (8
// below), and the largest cluster (at most 16 CTAs) that keeps every pack of the batch
// resident at once.
int auto_pack(int batch) { return batch >= 256 ? 16 : 8; }
int auto_cluster(const pf_handle* h, int batch, int S) {
    const int packs = (batch + S - 1) / S;
    int c = 16;
    while (c > 1 && (long long)packs * c > h->num_sms) c >>= 1;
    return c;
}

pf::SiLayout si_layout(const pf_handle* h, int ft, const LaunchCfg& c);

// The launch configuration of a solve.  `si_ok`: the interleaved placement may serve this
// call (a forward solve without kept factors); where it may not, an automatic choice
// falls back to the heuristic placement and an explicit request is refused (-1).
LaunchCfg resolve(const pf_handle* h, const pf_solve_opts* o, int batch = 0, bool si_ok = true) {
    const int ft = o->precision == PF_MIXED ? 4 : 8;
    const int pi = o->precision == PF_MIXED ? 1 : 0;
    // where the interleaved placement may not serve, the tuned per-scenario shape stands in
    const pf_tune_result& t =
        (!si_ok && h->tuned[pi].placement == PF_PLACE_INTERLEAVED) ? h->tuned_ps[pi] : h->tuned[pi];
    const bool use_tuned = o->group_threads == 0 && o->instances_per_cta == 0 && t.group_threads;
    LaunchCfg c;
    c.threads = o->group_threads ? o->group_threads
                                 : (use_tuned ? t.group_threads : auto_threads(h->plan.n));
    c.ipc = o->instances_per_cta ? o->instances_per_cta
                                 : (use_tuned ? t.instances_per_cta : 1);
    if (c.ipc > 1) c.threads = 32;
    c.placement = o->placement ? o->placement
                               : (t.placement ? t.placement : heuristic_placement(h, ft));
    c.S = c.cluster = 0;
    if (c.placement == PF_PLACE_INTERLEAVED) {
        if (!si_ok) {
            if (o->placement == PF_PLACE_INTERLEAVED) {
                c.placement = -1;
                return c;
            }
            c.placement = heuristic_placement(h, ft);
            c.threads = o->group_threads ? o->group_threads : auto_threads(h->plan.n);
            c.ipc = 1;
            return c;
        }
        const bool tuned_si = t.placement == PF_PLACE_INTERLEAVED;
        c.ipc = 1;
        c.S = o->pack ? o->pack : (tuned_si && t.pack ? t.pack : auto_pack(batch));
        c.cluster = o->cluster ? o->cluster
                               : (tuned_si && t.cluster ? t.cluster : auto_cluster(h, batch, c.S));
        c.threads = o->group_threads ? o->group_threads
                                     : (tuned_si && t.group_threads ? t.group_threads : 1024);
        // an automatic cluster size grows until the pack's top regions fit its CTAs
        if (!o->cluster && !(tuned_si && t.cluster))
            while (c.cluster < 16 && si_layout(h, ft, c).smem_bytes > smem_budget(h)) c.cluster *= 2;
    }
    return c;
}

// Interleaved-pack shape check: threads / S a power of two of at least 16 lane groups (a
// split sweep row's groups then never straddle two rounds), at most 1024 threads.
bool si_shape_ok(int S, int cluster, int threads) {
    if (S != 2 && S != 4 && S != 8 && S != 16 && S != 32) return false;
    if (cluster < 1 || cluster > 16 || threads < 32 || threads > 1024 || threads % S) return false;
    const int ns = threads / S;
    return ns >= 16 && (ns & (ns - 1)) == 0;
}

// Workspace layout of one interleaved pack.
pf::SiLayout si_layout(const pf_handle* h, int ft, const LaunchCfg& c) {
    const pf::Plan& P = h->plan;
    pf::SiLayout L{};
    L.S = c.S;
    L.cluster = c.cluster;
    L.threads = c.threads;
    const size_t S = (size_t)c.S, nb = (size_t)P.n_bus, n = (size_t)P.n;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = pf::align_up(o + bytes, 256);
        return at;
    };
    L.off_fac = take((size_t)P.nnzb() * S * 4 * ft);
    L.off_V = take(nb * S * 16);
    L.off_I = take(nb * S * 16);
    L.off_U = take(nb * S * 16);
    L.off_M = take(nb * S * 16);
    L.off_SP = take(nb * S * 16);
    L.off_DV = take(ft == 4 ? nb * S * 16 : 0);
    L.off_FA = take(ft == 4 ? nb * S * 16 : 0);
    L.off_FB = take(ft == 4 ? nb * S * 16 : 0);
    L.off_F = take(n * S * 16);
    L.off_DZ = take(ft == 4 ? n * S * 16 : 0);
    L.off_X = take(n * S * 2 * ft);
    L.off_ctl = take(3 * 32 * sizeof(unsigned long long) + 32 * sizeof(unsigned int));
    L.pack_bytes = o;
    L.smem_bytes = (size_t)c.threads * 2 * ft;  // one FT2 partial sum per thread
    L.top_slots = 0;
    L.top_stride = 0;
    L.smem_top_off = pf::align_up(L.smem_bytes, 16);
    if (P.top_R > 0) {
        // as many scenarios' regions as fit (a power of two), at most this CTA's share
        const size_t lists = pf::align_up((size_t)4 * P.top_nints_fwd, 16);
        const size_t budget = smem_budget(h);
        L.top_stride = pf::top_ints_off(P.top_blocks(), P.top_R, ft);
        const int share = (c.S + c.cluster - 1) / c.cluster;
        int slots = 1;
        while (slots < share && L.smem_top_off + (size_t)(2 * slots) * L.top_stride + lists <= budget)
            slots *= 2;
        L.top_slots = slots;
        L.smem_bytes = L.smem_top_off + (size_t)L.top_slots * L.top_stride + lists;
    }
    return L;
}

// Packs of an interleaved launch.  With one CTA per pack, a batch whose full packs would
// leave SMs idle is spread over one pack per SM (at least one scenario a pack): 2048
// scenarios in packs of 16 become 152 packs of 13-14 instead of 128.  (Spreading a batch
// that already fills every SM over all resident slots measured slower: 4096 scenarios in
// 304 packs of 13-14 took 0.82 ms against 0.76 ms in 256 packs of 16.)  Which pack holds
// which scenario does not change any result.
int si_npacks(const pf_handle* h, int /*ft*/, const LaunchCfg& c, int batch) {
    const int plain = std::max(1, (batch + c.S - 1) / c.S);
    if (c.cluster != 1 || h->num_sms <= 0 || plain >= h->num_sms) return plain;
    return std::max(plain, std::min(h->num_sms, batch));
}

size_t si_workspace(const pf_handle* h, int ft, const LaunchCfg& c, int batch) {
    return si_layout(h, ft, c).pack_bytes * (size_t)si_npacks(h, ft, c, batch);
}

bool opts_ok(const pf_solve_opts* o) {
    if (!o) return false;
    if (o->precision != PF_FP64 && o->precision != PF_MIXED) return false;
    if (o->ir_steps < 0 || o->ir_steps > 64) return false;
    if (!(o->ir_rtol >= 0.0) || !(o->ir_gate >= 0.0)) return false;
    if (o->group_threads != 0 &&
        (o->group_threads < 32 || o->group_threads > 1024 || o->group_threads % 32)) return false;
    if (o->placement < PF_PLACE_AUTO || o->placement > PF_PLACE_INTERLEAVED) return false;
    if (o->pack != 0 && o->pack != 2 && o->pack != 4 && o->pack != 8 && o->pack != 16 &&
        o->pack != 32)
        return false;
    if (o->cluster < 0 || o->cluster > 16) return false;
    if (o->instances_per_cta < 0 || o->instances_per_cta > 8) return false;
    if (o->instances_per_cta > 1 && o->group_threads != 0 && o->group_threads != 32) return false;
    return true;
}

template <typename T>
size_t push(std::vector<unsigned char>& buf, const std::vector<T>& v) {
    size_t off = pf::align_up(buf.size(), 16);
    buf.resize(off + sizeof(T) * v.size());
    if (!v.empty()) std::memcpy(buf.data() + off, v.data(), sizeof(T) * v.size());
    return off;
}

}  // namespace

namespace {

// Every plan array packed into one buffer (one device allocation per network).
struct PlanOffsets {
    size_t ygb, ytgb, ygb32, yptr, yidx, ytptr, ytidx, bt, p2b, b2p, lev, lup, lur, luc, lud,
        lum, fy, lap, la, stp, stg, scp, sch, levg, j1pos, j1ptr, j1col, tmap, tsplit, tints, ttr;
};

void pack_plan(const pf::Plan& P, std::vector<unsigned char>& buf, PlanOffsets& o) {
    std::vector<double2> ygb(P.y_g.size()), ytgb(P.yt_g.size());
    std::vector<float2> ygb32(P.y_g.size());
    for (size_t k = 0; k < P.y_g.size(); ++k) {
        ygb[k] = make_double2(P.y_g[k], P.y_b[k]);
        ygb32[k] = make_float2((float)P.y_g[k], (float)P.y_b[k]);
    }
    for (size_t k = 0; k < P.yt_g.size(); ++k) ytgb[k] = make_double2(P.yt_g[k], P.yt_b[k]);
    std::vector<int2> la(P.la_L.size()), sch(P.sch_L.size());
    std::vector<int4> levg(P.n_levels), j1pos(P.y_idx.size());
    for (int l = 0; l < P.n_levels; ++l) levg[l] = make_int4(P.lev_gL[l], P.lev_gU[l], P.lev_gS[l], 0);
    for (size_t k = 0; k < la.size(); ++k) la[k] = make_int2(P.la_L[k], P.la_D[k]);
    for (size_t k = 0; k < sch.size(); ++k) sch[k] = make_int2(P.sch_L[k], P.sch_U[k]);
    for (size_t k = 0; k < j1pos.size(); ++k)
        j1pos[k] = make_int4(P.j1_pos[4 * k], P.j1_pos[4 * k + 1], P.j1_pos[4 * k + 2],
                             P.j1_pos[4 * k + 3]);
    o.ygb = push(buf, ygb), o.ytgb = push(buf, ytgb), o.ygb32 = push(buf, ygb32);
    o.yptr = push(buf, P.y_ptr), o.yidx = push(buf, P.y_idx);
    o.ytptr = push(buf, P.yt_ptr), o.ytidx = push(buf, P.yt_idx);
    o.bt = push(buf, P.bus_type), o.p2b = push(buf, P.pos2bus), o.b2p = push(buf, P.bus2pos);
    o.lev = push(buf, P.lev_ptr), o.lup = push(buf, P.lu_ptr), o.lur = push(buf, P.lu_row);
    o.luc = push(buf, P.lu_col), o.lud = push(buf, P.lu_diag), o.lum = push(buf, P.lu_mirror);
    o.fy = push(buf, P.fill_y), o.lap = push(buf, P.la_ptr), o.la = push(buf, la);
    o.stp = push(buf, P.sch_tptr), o.stg = push(buf, P.sch_tgt), o.scp = push(buf, P.sch_cptr);
    o.sch = push(buf, sch), o.levg = push(buf, levg), o.j1pos = push(buf, j1pos);
    o.j1ptr = push(buf, P.j1_ptr), o.j1col = push(buf, P.j1_col);
    std::vector<int2> ttr(P.top_tr_t.size());
    for (size_t k = 0; k < ttr.size(); ++k) ttr[k] = make_int2(P.top_tr_t[k], P.top_tr_lu[k]);
    o.tmap = push(buf, P.top_map), o.tsplit = push(buf, P.top_split);
    o.tints = push(buf, P.top_ints), o.ttr = push(buf, ttr);
}

// Reactive-limit inputs of pf_solve_qlim (null for pf_solve).
struct QlimIn {
    const double* Qmin;
    const double* Qmax;
    int max_rounds;
    int* types_out;
    int* rounds_out;
};

// The interleaved-pack solve (PF_PLACE_INTERLEAVED): one thread-block cluster per pack.
pf_err solve_si(pf_handle* h, int batch, const double* Pd, const double* Qd, const double* Pg,
                const double* Vset, double tol, int max_iter, const pf_solve_opts* opts,
                const LaunchCfg& cfg, double* Vm, double* Va, double* Pg_out, double* Qg_out,
                int* iters, int* status, double* final_mismatch, void* workspace,
                size_t workspace_bytes, void* stream) {
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    if (!si_shape_ok(cfg.S, cfg.cluster, cfg.threads)) return PF_EINVAL;
    const pf::SiLayout L = si_layout(h, ft, cfg);
    if (workspace_bytes < si_workspace(h, ft, cfg, batch)) return PF_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return PF_EINVAL;
    DeviceGuard guard(h->device);
    bool fits = false;
    cudaError_t e = ft == 4 ? pf::si_shape_fits<float>(cfg.S, cfg.cluster, cfg.threads, L.smem_bytes, &fits)
                            : pf::si_shape_fits<double>(cfg.S, cfg.cluster, cfg.threads, L.smem_bytes, &fits);
    if (e != cudaSuccess) return PF_ECUDA;
    if (!fits) return PF_ENOTSUP;  // no cluster of this shape can be resident on this GPU
    pf::SiArgs A{};
    A.batch = batch;
    A.npacks = si_npacks(h, ft, cfg, batch);
    A.q = batch / A.npacks;
    A.r = batch % A.npacks;
    A.max_iter = max_iter;
    A.ir_steps = opts->precision == PF_MIXED ? opts->ir_steps : 0;
    A.tol = tol;
    A.ir_rtol = opts->ir_rtol;
    A.ir_gate = opts->ir_gate;
    A.Pd = Pd;
    A.Qd = Qd;
    A.Pg = Pg;
    A.Vset = Vset;
    A.Vm = Vm;
    A.Va = Va;
    A.Pg_out = Pg_out;
    A.Qg_out = Qg_out;
    A.fmis = final_mismatch;
    A.iters = iters;
    A.status = status;
    A.ws = static_cast<char*>(workspace);
    A.L = L;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = ft == 4 ? pf::launch_solve_si<float>(h->dp, A, s) : pf::launch_solve_si<double>(h->dp, A, s);
    h->last_batch = -1;  // leaves no state for pf_adjoint
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_err solve_impl(pf_handle* h, int batch, const double* Pd, const double* Qd, const double* Pg,
                  const double* Vset, double tol, int max_iter, const pf_solve_opts* opts,
                  double* Vm, double* Va, double* Pg_out, double* Qg_out, int* iters, int* status,
                  double* final_mismatch, void* workspace, size_t workspace_bytes, void* stream,
                  const QlimIn* q, bool si_allowed = true) {
    if (!h || batch < 1 || !Pd || !Qd || !Pg || !Vset || !Vm || !Va || !status || !workspace)
        return PF_EINVAL;
    if (!(tol > 0.0) || max_iter < 0 || !opts_ok(opts)) return PF_EINVAL;
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    LaunchCfg cfg = resolve(h, opts, batch, si_allowed && !opts->keep_factors && !q);
    if (cfg.placement < 0) return PF_ENOTSUP;
    if (cfg.placement == PF_PLACE_INTERLEAVED)
        return solve_si(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, opts, cfg, Vm, Va, Pg_out,
                        Qg_out, iters, status, final_mismatch, workspace, workspace_bytes, stream);
    if (q) cfg.ipc = 1;  // reactive limits: one CTA per scenario (32 threads if tuned to warps)
    pf::SlotLayout L = make_layout(h, ft, opts->keep_factors, cfg.placement, q != nullptr);
    if (workspace_bytes < L.slot_bytes * (size_t)batch) return PF_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return PF_EINVAL;
    const int threads = cfg.threads;
    if (cfg.ipc > 1 && L.fwd.smem_bytes * (size_t)cfg.ipc > smem_budget(h)) return PF_EINVAL;
    DeviceGuard guard(h->device);
    pf::SolveArgs A{};
    A.batch = batch;
    A.ipc = cfg.ipc;
    A.tol = tol;
    A.max_iter = max_iter;
    A.ir_steps = opts->precision == PF_MIXED ? opts->ir_steps : 0;
    A.ir_rtol = opts->ir_rtol;
    A.ir_gate = opts->ir_gate;
    A.keep_factors = opts->keep_factors ? 1 : 0;
    A.Pd = Pd;
    A.Qd = Qd;
    A.Pg = Pg;
    A.Vset = Vset;
    A.Vm = Vm;
    A.Va = Va;
    A.Pg_out = Pg_out;
    A.Qg_out = Qg_out;
    A.fmis = final_mismatch;
    A.iters = iters;
    A.status = status;
    A.ws = static_cast<char*>(workspace);
    A.L = L;
    if (q) {
        A.Qmin = q->Qmin;
        A.Qmax = q->Qmax;
        A.max_rounds = q->max_rounds;
        A.types_out = q->types_out;
        A.rounds_out = q->rounds_out;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (q)  // one CTA per scenario: the warp-per-scenario form has no reactive-limit variant
        e = ft == 4 ? pf::launch_solve_qlim<float>(h->dp, A, threads, s)
                    : pf::launch_solve_qlim<double>(h->dp, A, threads, s);
    else
        e = ft == 4 ? pf::launch_solve<float>(h->dp, A, threads, s)
                    : pf::launch_solve<double>(h->dp, A, threads, s);
    if (e != cudaSuccess) {
        h->last_batch = -1;
        return PF_ECUDA;
    }
    h->last_qlim = q ? 1 : 0;
    h->last_batch = batch;
    h->last_ft = ft;
    h->last_keep = A.keep_factors;
    h->last_threads = threads;
    h->last_ws = workspace;
    h->last_layout = L;
    return PF_OK;
}

// cuPointerGetAttribute, looked up through the runtime (no link-time driver dependency)
using PtrAttrFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
PtrAttrFn ptr_attr_fn() {
    static const PtrAttrFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return static_cast<PtrAttrFn>(nullptr);
        return reinterpret_cast<PtrAttrFn>(f);
    }();
    return fn;
}

// [p, p + bytes) inside one allocation known to CUDA (page-locked host memory, or device
// memory of `device`) that kernels address at the pointer value p itself.  Any query that
// fails counts as "no": nothing unproven is handed to a kernel.
bool addressable(const void* p, size_t bytes, int device) {
    const PtrAttrFn fn = ptr_attr_fn();
    if (!fn || !p) return false;
    const CUdeviceptr d = static_cast<CUdeviceptr>(reinterpret_cast<uintptr_t>(p));
    unsigned int type = 0;
    if (fn(&type, CU_POINTER_ATTRIBUTE_MEMORY_TYPE, d) != CUDA_SUCCESS) return false;
    if (type != CU_MEMORYTYPE_HOST && type != CU_MEMORYTYPE_DEVICE) return false;
    CUdeviceptr dp = 0;
    if (fn(&dp, CU_POINTER_ATTRIBUTE_DEVICE_POINTER, d) != CUDA_SUCCESS || dp != d) return false;
    if (type == CU_MEMORYTYPE_DEVICE) {
        int ord = -1;
        if (fn(&ord, CU_POINTER_ATTRIBUTE_DEVICE_ORDINAL, d) != CUDA_SUCCESS || ord != device)
            return false;
    }
    CUdeviceptr start = 0;
    size_t size = 0;
    if (fn(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, d) != CUDA_SUCCESS) return false;
    if (fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, d) != CUDA_SUCCESS) return false;
    return d >= start && bytes <= size && static_cast<size_t>(d - start) <= size - bytes;
}

}  // namespace

namespace pf {
int handle_device(const pf_handle* h) { return h->device; }
void* handle_noalloc_scratch(const pf_handle* h) { return h->noalloc_scratch; }
}  // namespace pf

namespace {
pf_err adjoint_impl(pf_handle* h, int batch, const double* dVm, const double* dVa,
                    const double* dPg, const double* dQg, double* dPd, double* dQd,
                    double* dPg_in, double* dVset, int* adj_status, void* workspace,
                    size_t workspace_bytes, void* stream, const double* Qmax, double* dQmin,
                    double* dQmax) {
    if (!h || batch < 1 || !dVm || !dVa || !dPd || !dQd || !dPg_in || !dVset || !workspace)
        return PF_EINVAL;
    const bool ql = Qmax != nullptr;
    if (h->last_batch != batch || !h->last_keep || h->last_ws != workspace ||
        h->last_qlim != (ql ? 1 : 0))
        return PF_ESTATE;
    const pf::SlotLayout& L = h->last_layout;
    if (workspace_bytes < L.slot_bytes * (size_t)batch) return PF_EINVAL;
    DeviceGuard guard(h->device);
    pf::AdjArgs A{};
    A.batch = batch;
    A.ir_max = 8;
    A.ir_rtol = 1e-12;
    A.dVm = dVm;
    A.dVa = dVa;
    A.dPg = dPg;
    A.dQg = dQg;
    A.dPd = dPd;
    A.dQd = dQd;
    A.dPg_in = dPg_in;
    A.dVset = dVset;
    A.adj_status = adj_status;
    A.ws = static_cast<char*>(workspace);
    A.L = L;
    // The adjoint takes the top region in shared memory (its transposed sweeps, and a
    // refactorisation) unless the region's arena, over the CTAs one SM holds at this CTA
    // size (64 registers a thread), would take more than kTopAdjSmemPerSm of the SM's
    // L1/shared memory: the adjoint's other phases read the scenario's vectors through
    // L1.  Without it the kernel walks the region's levels like the others and needs no
    // arena.
    {
        const pf::Plan& P = h->plan;
        const int ft = h->last_ft;
        const size_t per_sm = (size_t)std::max(1, 1024 / std::max(32, h->last_threads));
        A.top_t = (P.top_R > 0 && top_bytes(P, ft, true) * per_sm <= kTopAdjSmemPerSm) ? 1 : 0;
        if (!A.top_t) A.L.adj.smem_bytes = A.L.adj.smem_top_off;
    }
    A.Qmax = Qmax;
    A.dQmin = dQmin;
    A.dQmax = dQmax;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (ql)
        e = h->last_ft == 4 ? pf::launch_adjoint_qlim<float>(h->dp, A, h->last_threads, s)
                            : pf::launch_adjoint_qlim<double>(h->dp, A, h->last_threads, s);
    else
        e = h->last_ft == 4 ? pf::launch_adjoint<float>(h->dp, A, h->last_threads, s)
                            : pf::launch_adjoint<double>(h->dp, A, h->last_threads, s);
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}
}  // namespace

extern "C" {

const char* pf_error_string(pf_err e) {
    switch (e) {
        case PF_OK: return "ok";
        case PF_EINVAL: return "invalid argument";
        case PF_ESINGULAR_PATTERN: return "singular network pattern (island without slack or missing diagonal)";
        case PF_ENOMEM: return "out of memory";
        case PF_ECUDA: return "CUDA error";
        case PF_ESTATE: return "no matching pf_solve state for pf_adjoint";
        case PF_ENOTSUP: return "not supported";
    }
    return "unknown error";
}

pf_err pf_build_ybus(int n_bus, int n_branch, const int* f, const int* t, const double* r,
                     const double* x, const double* b, const double* tap, int* indptr,
                     int* indices, double* g, double* bv, int* nnz) {
    if (n_bus < 1 || n_branch < 0 || !nnz || !indptr) return PF_EINVAL;
    if (n_branch > 0 && (!f || !t || !r || !x || !b || !tap)) return PF_EINVAL;
    std::vector<std::vector<std::pair<int, std::complex<double>>>> rows(n_bus);
    for (int k = 0; k < n_branch; ++k) {
        if (f[k] < 0 || f[k] >= n_bus || t[k] < 0 || t[k] >= n_bus) return PF_EINVAL;
        std::complex<double> z(r[k], x[k]);
        if (std::abs(z) == 0.0 || !(tap[k] > 0.0)) return PF_EINVAL;
        const std::complex<double> ys = 1.0 / z, sh(0.0, 0.5 * b[k]);
        const double a = tap[k];
        rows[f[k]].push_back({f[k], (ys + sh) / (a * a)});
        rows[t[k]].push_back({t[k], ys + sh});
        rows[f[k]].push_back({t[k], -ys / a});
        rows[t[k]].push_back({f[k], -ys / a});
    }
    int count = 0;
    indptr[0] = 0;
    std::vector<std::vector<std::pair<int, std::complex<double>>>> merged(n_bus);
    for (int i = 0; i < n_bus; ++i) {
        auto& rw = rows[i];
        std::stable_sort(rw.begin(), rw.end(),
                         [](const auto& p, const auto& q) { return p.first < q.first; });
        for (auto& e : rw) {
            if (!merged[i].empty() && merged[i].back().first == e.first) merged[i].back().second += e.second;
            else merged[i].push_back(e);
        }
        count += (int)merged[i].size();
        indptr[i + 1] = count;
    }
    if (!indices || !g || !bv) {
        *nnz = count;
        return PF_OK;
    }
    if (*nnz < count) return PF_EINVAL;
    int o = 0;
    for (int i = 0; i < n_bus; ++i)
        for (auto& e : merged[i]) {
            indices[o] = e.first;
            g[o] = e.second.real();
            bv[o] = e.second.imag();
            ++o;
        }
    *nnz = count;
    return PF_OK;
}

void pf_plan_opts_default(pf_plan_opts* o) {
    if (!o) return;
    const pf::PlanParams d;
    o->order_slack = d.order_slack;
    o->top_rows = d.top_rows;
    o->top_blocks = d.top_blocks;
    o->top_min_pivots = d.top_min_pivots;
    o->split_len = d.split_len;
    o->split_rows = d.split_rows;
}

pf_err pf_create(int n_bus, const int* y_indptr, const int* y_indices, const double* y_re,
                 const double* y_im, const int* bus_type, pf_handle** out) {
    return pf_create_ex(n_bus, y_indptr, y_indices, y_re, y_im, bus_type, nullptr, out);
}

// The planner's parameters from the caller's schedule choices (NULL: the defaults);
// false if a choice is out of range.
static bool plan_params(const pf_plan_opts* o, pf::PlanParams& pp) {
    pp = pf::PlanParams();
    if (!o) return true;
    if (o->order_slack < 0 || o->order_slack > 8 || o->top_rows < 0 || o->top_blocks < 0 ||
        o->top_blocks > pf::kTopMaxBlocks || o->top_min_pivots < 0 || o->split_len < 1 ||
        o->split_rows < 0)
        return false;
    pp.order_slack = o->order_slack;
    pp.top_rows = o->top_rows;
    pp.top_blocks = o->top_blocks;
    pp.top_min_pivots = o->top_min_pivots;
    pp.split_len = o->split_len;
    pp.split_rows = o->split_rows;
    return true;
}

pf_err pf_create_ex(int n_bus, const int* y_indptr, const int* y_indices, const double* y_re,
                    const double* y_im, const int* bus_type, const pf_plan_opts* plan_opts,
                    pf_handle** out) {
    if (!out) return PF_EINVAL;
    *out = nullptr;
    pf::PlanParams pp;
    if (!plan_params(plan_opts, pp)) return PF_EINVAL;
    pf_handle* h = new (std::nothrow) pf_handle();
    if (!h) return PF_ENOMEM;
    pf::BuildStatus bs = pf::build_plan(n_bus, y_indptr, y_indices, y_re, y_im, bus_type, h->plan, pp);
    if (bs != pf::BUILD_OK) {
        delete h;
        return bs == pf::BUILD_ESINGULAR ? PF_ESINGULAR_PATTERN : PF_EINVAL;
    }
    const pf::Plan& P = h->plan;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return PF_ECUDA;
    }
    std::vector<unsigned char> buf;
    PlanOffsets po;
    pack_plan(P, buf, po);
    if (buf.empty()) buf.resize(16);
    if (cudaMalloc(&h->d_buf, buf.size()) != cudaSuccess) {
        delete h;
        return PF_ENOMEM;
    }
    if (cudaMemcpy(h->d_buf, buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(h->d_buf);
        delete h;
        return PF_ECUDA;
    }
    h->plan_bytes = buf.size();
    // pf_solve_noalloc's scratch address on this device, looked up here (a call that may
    // load the module holding the array), so that the no-allocation entry point itself
    // never does; a failed lookup only disables that entry point
    if (pf::noalloc_lookup(&h->noalloc_scratch) != cudaSuccess) h->noalloc_scratch = nullptr;
    auto* base = static_cast<unsigned char*>(h->d_buf);
    auto I = [&](size_t o) { return reinterpret_cast<const int*>(base + o); };
    pf::DevPlan& d = h->dp;
    d.n_bus = P.n_bus;
    d.n = P.n;
    d.nnzb = P.nnzb();
    d.n_levels = P.n_levels;
    d.top_l0 = P.top_l0;
    d.top_p0 = P.top_p0;
    d.top_R = P.top_R;
    d.top_nblk = P.top_blocks();
    d.top_g = P.top_g;
    d.top_nl = P.top_nl;
    d.top_nfw = P.top_nfw;
    d.top_nbw = P.top_nbw;
    d.top_nints = (int)P.top_ints.size();
    d.top_nft = P.top_nft;
    d.top_nbt = P.top_nbt;
    d.top_nints_fwd = P.top_nints_fwd;
    d.top_map = I(po.tmap);
    d.top_split = I(po.tsplit);
    d.top_ints = I(po.tints);
    d.top_tr = reinterpret_cast<const int2*>(base + po.ttr);
    d.y_ptr = I(po.yptr);
    d.y_idx = I(po.yidx);
    d.y_gb = reinterpret_cast<const double2*>(base + po.ygb);
    d.y_gb32 = reinterpret_cast<const float2*>(base + po.ygb32);
    d.yt_ptr = I(po.ytptr);
    d.yt_idx = I(po.ytidx);
    d.yt_gb = reinterpret_cast<const double2*>(base + po.ytgb);
    d.bus_type = I(po.bt);
    d.pos2bus = I(po.p2b);
    d.bus2pos = I(po.b2p);
    d.lev_ptr = I(po.lev);
    d.lev_g = reinterpret_cast<const int4*>(base + po.levg);
    d.lu_ptr = I(po.lup);
    d.lu_row = I(po.lur);
    d.lu_col = I(po.luc);
    d.lu_diag = I(po.lud);
    d.lu_mirror = I(po.lum);
    d.fill_y = I(po.fy);
    d.la_ptr = I(po.lap);
    d.la = reinterpret_cast<const int2*>(base + po.la);
    d.sch_tptr = I(po.stp);
    d.sch_tgt = I(po.stg);
    d.sch_cptr = I(po.scp);
    d.sch = reinterpret_cast<const int2*>(base + po.sch);
    d.n1 = P.n1;
    d.nnz_j1 = P.nnz_j1;
    d.j1_pos = reinterpret_cast<const int4*>(base + po.j1pos);
    d.j1_ptr = I(po.j1ptr);
    d.j1_col = I(po.j1col);
    *out = h;
    return PF_OK;
}

static void fill_info(const pf::Plan& P, size_t plan_bytes, pf_plan_info* info) {
    info->n_bus = P.n_bus;
    info->n_slack = P.n_slack;
    info->n_pv = P.n_pv;
    info->n_pq = P.n_pq;
    info->n_unknowns = (P.n_bus - P.n_slack) + P.n_pq;
    info->n_block = P.n;
    info->nnz_ybus = (int)P.y_idx.size();
    info->nnz_j1 = P.nnz_j1;
    info->nnzb_lu = P.nnzb();
    info->n_levels = P.n_levels;
    info->schur_block_ops = P.schur_ops;
    info->plan_bytes = (long long)plan_bytes;
    info->top_pivots = P.top_R;
    info->top_levels = P.n_levels - P.top_l0;
    info->top_blocks = P.top_blocks();
    info->top_arena_bytes = (int)top_bytes(P, 8, true);
}

pf_err pf_get_plan_info(const pf_handle* h, pf_plan_info* info) {
    if (!h || !info) return PF_EINVAL;
    fill_info(h->plan, h->plan_bytes, info);
    return PF_OK;
}

pf_err pf_jacobian_pattern(const pf_handle* h, int* j1_ptr, int* j1_col) {
    if (!h || !j1_ptr || !j1_col) return PF_EINVAL;
    std::copy(h->plan.j1_ptr.begin(), h->plan.j1_ptr.end(), j1_ptr);
    std::copy(h->plan.j1_col.begin(), h->plan.j1_col.end(), j1_col);
    return PF_OK;
}

pf_err pf_bde_pattern(const pf_handle* h, int batch, int* row_ptr, int* col_idx, void* stream) {
    if (!h || batch < 1 || !row_ptr || !col_idx) return PF_EINVAL;
    if ((long long)batch * h->plan.nnz_j1 >= (1LL << 31) ||
        (long long)batch * h->plan.n1 >= (1LL << 31)) return PF_EINVAL;
    DeviceGuard guard(h->device);
    return pf::launch_bde_pattern(h->dp, batch, row_ptr, col_idx, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_err pf_export_jacobian(const pf_handle* h, int batch, const double* Vm, const double* Va,
                          double* values, void* stream) {
    if (!h || batch < 1 || !Vm || !Va || !values) return PF_EINVAL;
    DeviceGuard guard(h->device);
    return pf::launch_export_jacobian(h->dp, batch, Vm, Va, values,
                                      static_cast<cudaStream_t>(stream)) == cudaSuccess ? PF_OK
                                                                                        : PF_ECUDA;
}

pf_err pf_analyze(int n_bus, const int* y_indptr, const int* y_indices, const double* y_re,
                  const double* y_im, const int* bus_type, pf_plan_info* info, int* pos2bus,
                  int* lu_ptr, int* lu_col, int* lev_ptr, int* j1_ptr, int* j1_col) {
    return pf_analyze_ex(n_bus, y_indptr, y_indices, y_re, y_im, bus_type, nullptr, info, pos2bus,
                         lu_ptr, lu_col, lev_ptr, j1_ptr, j1_col);
}

pf_err pf_analyze_ex(int n_bus, const int* y_indptr, const int* y_indices, const double* y_re,
                     const double* y_im, const int* bus_type, const pf_plan_opts* plan_opts,
                     pf_plan_info* info, int* pos2bus, int* lu_ptr, int* lu_col, int* lev_ptr,
                     int* j1_ptr, int* j1_col) {
    if (!info) return PF_EINVAL;
    pf::PlanParams pp;
    if (!plan_params(plan_opts, pp)) return PF_EINVAL;
    pf::Plan P;
    pf::BuildStatus bs = pf::build_plan(n_bus, y_indptr, y_indices, y_re, y_im, bus_type, P, pp);
    if (bs != pf::BUILD_OK) return bs == pf::BUILD_ESINGULAR ? PF_ESINGULAR_PATTERN : PF_EINVAL;
    std::vector<unsigned char> buf;
    PlanOffsets po;
    pack_plan(P, buf, po);
    fill_info(P, buf.size(), info);
    if (j1_ptr) std::copy(P.j1_ptr.begin(), P.j1_ptr.end(), j1_ptr);
    if (j1_col) std::copy(P.j1_col.begin(), P.j1_col.end(), j1_col);
    if (pos2bus) std::copy(P.pos2bus.begin(), P.pos2bus.end(), pos2bus);
    if (lu_ptr) std::copy(P.lu_ptr.begin(), P.lu_ptr.end(), lu_ptr);
    if (lu_col) std::copy(P.lu_col.begin(), P.lu_col.end(), lu_col);
    if (lev_ptr) std::copy(P.lev_ptr.begin(), P.lev_ptr.end(), lev_ptr);
    return PF_OK;
}

pf_err pf_workspace_size(const pf_handle* h, int batch, const pf_solve_opts* opts, size_t* bytes) {
    if (!h || !bytes || batch < 1 || !opts_ok(opts)) return PF_EINVAL;
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    const LaunchCfg cfg = resolve(h, opts, batch, !opts->keep_factors);
    if (cfg.placement < 0) return PF_ENOTSUP;
    if (cfg.placement == PF_PLACE_INTERLEAVED) {
        if (!si_shape_ok(cfg.S, cfg.cluster, cfg.threads)) return PF_EINVAL;
        *bytes = si_workspace(h, ft, cfg, batch);
        return PF_OK;
    }
    const size_t slot = make_layout(h, ft, opts->keep_factors, cfg.placement).slot_bytes;
    *bytes = slot * (size_t)batch;
    return PF_OK;
}

pf_err pf_solve(pf_handle* h, int batch, const double* Pd, const double* Qd, const double* Pg,
                const double* Vset, double tol, int max_iter, const pf_solve_opts* opts,
                double* Vm, double* Va, double* Pg_out, double* Qg_out, int* iters, int* status,
                double* final_mismatch, void* workspace, size_t workspace_bytes, void* stream) {
    return solve_impl(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, opts, Vm, Va, Pg_out, Qg_out,
                      iters, status, final_mismatch, workspace, workspace_bytes, stream, nullptr);
}

pf_err pf_addressable(const pf_handle* h, const void* ptr, size_t bytes, int* ok) {
    if (!h || !ok) return PF_EINVAL;
    DeviceGuard guard(h->device);
    *ok = addressable(ptr, bytes, h->device) ? 1 : 0;
    return PF_OK;
}

pf_err pf_solve_host(pf_handle* h, int batch, const double* Pd, const double* Qd,
                     const double* Pg, const double* Vset, double tol, int max_iter,
                     const pf_solve_opts* opts, double* Vm, double* Va, double* Pg_out,
                     double* Qg_out, int* iters, int* status, double* final_mismatch,
                     void* workspace, size_t workspace_bytes, void* stream) {
    if (!h || batch < 1 || !Pd || !Qd || !Pg || !Vset || !Vm || !Va || !status || !workspace)
        return PF_EINVAL;
    if (!opts_ok(opts)) return PF_EINVAL;
    // host buffers: the per-scenario forms read them over the Newton iterations; the
    // interleaved packs read them in one burst before they start (measured slower end to
    // end), so they serve this call only when asked for explicitly
    size_t ws_need = 0;
    {
        const int ft = opts->precision == PF_MIXED ? 4 : 8;
        const LaunchCfg cfg = resolve(h, opts, batch,
                                      opts->placement == PF_PLACE_INTERLEAVED && !opts->keep_factors);
        if (cfg.placement < 0) return PF_ENOTSUP;
        if (cfg.placement == PF_PLACE_INTERLEAVED) {
            if (!si_shape_ok(cfg.S, cfg.cluster, cfg.threads)) return PF_EINVAL;
            ws_need = si_workspace(h, ft, cfg, batch);
        } else {
            ws_need = make_layout(h, ft, opts->keep_factors, cfg.placement).slot_bytes * (size_t)batch;
        }
    }
    const size_t row = sizeof(double) * (size_t)batch * (size_t)h->plan.n_bus;
    DeviceGuard guard(h->device);
    const void* in[] = {Pd, Qd, Pg, Vset, Vm, Va};
    for (const void* p : in)
        if (!addressable(p, row, h->device)) return PF_EINVAL;
    if ((Pg_out && !addressable(Pg_out, row, h->device)) ||
        (Qg_out && !addressable(Qg_out, row, h->device)) ||
        (iters && !addressable(iters, sizeof(int) * (size_t)batch, h->device)) ||
        !addressable(status, sizeof(int) * (size_t)batch, h->device) ||
        (final_mismatch && !addressable(final_mismatch, sizeof(double) * (size_t)batch, h->device)))
        return PF_EINVAL;
    if (workspace_bytes < ws_need || !addressable(workspace, ws_need, h->device)) return PF_EINVAL;
    return solve_impl(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, opts, Vm, Va, Pg_out, Qg_out,
                      iters, status, final_mismatch, workspace, workspace_bytes, stream, nullptr,
                      opts->placement == PF_PLACE_INTERLEAVED);
}

pf_err pf_bde_workspace_size(const pf_handle* h, int batch, size_t* bytes) {
    if (!h || !bytes || batch < 1) return PF_EINVAL;
    *bytes = pf::bde_workspace_bytes(h->dp, batch);
    return PF_OK;
}

pf_err pf_solve_bde(pf_handle* h, int batch, const double* Pd, const double* Qd, const double* Pg,
                    const double* Vset, double tol, int max_iter, double* Vm, double* Va,
                    double* Pg_out, double* Qg_out, int* iters, int* status,
                    double* final_mismatch, void* workspace, size_t workspace_bytes,
                    void* stream) {
    if (!h || batch < 1 || !Pd || !Qd || !Pg || !Vset || !Vm || !Va || !status || !workspace)
        return PF_EINVAL;
    if (!(tol > 0.0) || max_iter < 0) return PF_EINVAL;
    if (workspace_bytes < pf::bde_workspace_bytes(h->dp, batch)) return PF_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return PF_EINVAL;
    DeviceGuard guard(h->device);
    h->last_batch = -1;  // leaves no state for pf_adjoint
    return pf::solve_bde(h->dp, batch, Pd, Qd, Pg, Vset, tol, max_iter, Vm, Va, Pg_out, Qg_out,
                         iters, status, final_mismatch, workspace,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_err pf_qlim_workspace_size(const pf_handle* h, int batch, const pf_solve_opts* opts,
                              size_t* bytes) {
    if (!h || !bytes || batch < 1 || !opts_ok(opts)) return PF_EINVAL;
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    const LaunchCfg cfg = resolve(h, opts, batch, false);
    if (cfg.placement < 0) return PF_ENOTSUP;
    *bytes = make_layout(h, ft, opts->keep_factors, cfg.placement, true).slot_bytes * (size_t)batch;
    return PF_OK;
}

pf_err pf_solve_qlim(pf_handle* h, int batch, const double* Pd, const double* Qd,
                     const double* Pg, const double* Vset, const double* Qmin, const double* Qmax,
                     double tol, int max_iter, int max_rounds, const pf_solve_opts* opts,
                     double* Vm, double* Va, double* Pg_out, double* Qg_out, int* iters,
                     int* status, double* final_mismatch, int* bus_type_out, int* rounds,
                     void* workspace, size_t workspace_bytes, void* stream) {
    if (!Qmin || !Qmax || max_rounds < 0 || !opts) return PF_EINVAL;
    QlimIn q{Qmin, Qmax, max_rounds, bus_type_out, rounds};
    return solve_impl(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, opts, Vm, Va, Pg_out, Qg_out,
                      iters, status, final_mismatch, workspace, workspace_bytes, stream, &q);
}


pf_err pf_adjoint(pf_handle* h, int batch, const double* dVm, const double* dVa, const double* dPg,
                  const double* dQg, double* dPd, double* dQd, double* dPg_in, double* dVset,
                  int* adj_status, void* workspace, size_t workspace_bytes, void* stream) {
    return adjoint_impl(h, batch, dVm, dVa, dPg, dQg, dPd, dQd, dPg_in, dVset, adj_status,
                        workspace, workspace_bytes, stream, nullptr, nullptr, nullptr);
}

pf_err pf_adjoint_qlim(pf_handle* h, int batch, const double* dVm, const double* dVa,
                       const double* dPg, const double* dQg, const double* Qmax, double* dPd,
                       double* dQd, double* dPg_in, double* dVset, double* dQmin, double* dQmax,
                       int* adj_status, void* workspace, size_t workspace_bytes, void* stream) {
    if (!Qmax || !dQmin || !dQmax) return PF_EINVAL;
    return adjoint_impl(h, batch, dVm, dVa, dPg, dQg, dPd, dQd, dPg_in, dVset, adj_status,
                        workspace, workspace_bytes, stream, Qmax, dQmin, dQmax);
}

pf_err pf_autotune(pf_handle* h, int batch, const double* Pd, const double* Qd, const double* Pg,
                   const double* Vset, double tol, int max_iter, const pf_solve_opts* opts,
                   void* workspace, size_t workspace_bytes, void* stream, pf_tune_result* out) {
    if (!h || batch < 1 || !Pd || !Qd || !Pg || !Vset || !workspace || !opts_ok(opts)) return PF_EINVAL;
    {
        pf_solve_opts g = *opts;
        g.placement = PF_PLACE_GLOBAL;  // the largest slot of all placements
        size_t need = 0;
        if (pf_workspace_size(h, batch, &g, &need) != PF_OK || workspace_bytes < need) return PF_EINVAL;
    }
    DeviceGuard guard(h->device);
    const int nb = h->plan.n_bus;
    // temporary outputs of the trial solves
    double* dbuf = nullptr;
    int* ibuf = nullptr;
    const size_t nd = (size_t)batch * nb;
    if (cudaMalloc(&dbuf, sizeof(double) * (2 * nd + (size_t)batch)) != cudaSuccess) return PF_ENOMEM;
    if (cudaMalloc(&ibuf, sizeof(int) * 2 * (size_t)batch) != cudaSuccess) {
        cudaFree(dbuf);
        return PF_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pf_tune_result best{0, 0, 0, 0.f};
    pf_err err = PF_OK;
    // (threads per scenario, scenarios per CTA)
    const int cands[][2] = {{32, 1},  {64, 1}, {128, 1}, {256, 1}, {512, 1},
                            {1024, 1}, {32, 2}, {32, 4},  {32, 8}};
    for (int pl = PF_PLACE_ONCHIP; pl <= PF_PLACE_FACTOR && err == PF_OK; ++pl) {
        // skip placements that fall back to another one (they would time a duplicate)
        const int ft = opts->precision == PF_MIXED ? 4 : 8;
        const pf::SlotLayout L = make_layout(h, ft, opts->keep_factors, pl);
        const int eff = (L.fwd.fac_in_smem && L.fwd.vec_in_smem) ? PF_PLACE_ONCHIP
                        : L.fwd.vec_in_smem ? PF_PLACE_VECTORS
                        : L.fwd.fac_in_smem ? PF_PLACE_FACTOR : PF_PLACE_GLOBAL;
        if (eff != pl) continue;
        for (const auto& cand : cands) {
            const int th = cand[0], ipc = cand[1];
            if (ipc > 1 && L.fwd.smem_bytes * (size_t)ipc > smem_budget(h)) continue;
            pf_solve_opts o = *opts;
            o.group_threads = th;
            o.instances_per_cta = ipc;
            o.placement = pl;
            float ms_best = 0.f;
            for (int rep = 0; rep < 3 && err == PF_OK; ++rep) {
                cudaEventRecord(e0, s);
                err = pf_solve(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, &o, dbuf, dbuf + nd,
                               nullptr, nullptr, ibuf, ibuf + batch, dbuf + 2 * nd, workspace,
                               workspace_bytes, stream);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) err = PF_ECUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && (ms_best == 0.f || ms < ms_best)) ms_best = ms;  // rep 0 warms up
            }
            if (err == PF_OK && (best.group_threads == 0 || ms_best < best.ms)) best = {th, pl, ipc, ms_best};
        }
    }
    const pf_tune_result best_ps = best;
    // interleaved packs on thread-block clusters (forward solves without kept factors, on
    // networks large enough for it): scenarios per pack x CTAs per cluster x threads
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    if (err == PF_OK && !opts->keep_factors) {
        for (int S : {2, 4, 8, 16, 32}) {
            if (S >= 2 * batch && S > 2) continue;  // packs mostly empty
            for (int cl : {1, 2, 4, 8, 16}) {
                if (cl > 1 && (S < 4 || S > 16)) continue;
                // too few SMs for the batch, unless no larger cluster is left to try (a few
                // scenarios of a large network: one pack on the largest cluster)
                if ((long long)((batch + S - 1) / S) * cl < h->num_sms / 2 && cl < 16) continue;
                for (int th : {256, 512, 1024}) {
                    if (cl > 1 && th < 512) continue;
                    const LaunchCfg c{th, PF_PLACE_INTERLEAVED, 1, S, cl};
                    if (!si_shape_ok(S, cl, th) || si_workspace(h, ft, c, batch) > workspace_bytes)
                        continue;
                    bool fits = false;
                    const size_t smem = si_layout(h, ft, c).smem_bytes;
                    if ((ft == 4 ? pf::si_shape_fits<float>(S, cl, th, smem, &fits)
                                 : pf::si_shape_fits<double>(S, cl, th, smem, &fits)) != cudaSuccess) {
                        err = PF_ECUDA;
                        break;
                    }
                    if (!fits) continue;
                    pf_solve_opts o = *opts;
                    o.group_threads = th;
                    o.instances_per_cta = 0;
                    o.placement = PF_PLACE_INTERLEAVED;
                    o.pack = S;
                    o.cluster = cl;
                    float ms_best = 0.f;
                    for (int rep = 0; rep < 3 && err == PF_OK; ++rep) {
                        cudaEventRecord(e0, s);
                        err = pf_solve(h, batch, Pd, Qd, Pg, Vset, tol, max_iter, &o, dbuf,
                                       dbuf + nd, nullptr, nullptr, ibuf, ibuf + batch,
                                       dbuf + 2 * nd, workspace, workspace_bytes, stream);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) err = PF_ECUDA;
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (rep > 0 && (ms_best == 0.f || ms < ms_best)) ms_best = ms;
                    }
                    if (err == PF_OK && ms_best < best.ms)
                        best = {th, PF_PLACE_INTERLEAVED, 1, ms_best, S, cl};
                    if (err != PF_OK) break;
                }
                if (err != PF_OK) break;
            }
            if (err != PF_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dbuf);
    cudaFree(ibuf);
    h->last_batch = -1;  // the trial solves invalidate the adjoint state
    if (err != PF_OK) return err;
    h->tuned[opts->precision == PF_MIXED ? 1 : 0] = best;
    h->tuned_ps[opts->precision == PF_MIXED ? 1 : 0] = best_ps;
    if (out) *out = best;
    return PF_OK;
}

}  // extern "C"

namespace {

bool multi_ok(int n_jobs, const pf_job* jobs, const pf_solve_opts* opts) {
    if (n_jobs < 1 || n_jobs > pf::kMaxJobs || !jobs || !opts_ok(opts)) return false;
    if (opts->placement != PF_PLACE_AUTO && opts->placement != PF_PLACE_GLOBAL) return false;
    if (opts->instances_per_cta > 1) return false;
    if (opts->group_threads != 0 && (opts->group_threads < 64 || opts->group_threads > 512))
        return false;
    for (int j = 0; j < n_jobs; ++j)
        if (!jobs[j].h || jobs[j].batch < 1) return false;
    return true;
}

// Threads per CTA of a multi-network launch.
int multi_threads(const pf_solve_opts* opts) { return opts->group_threads ? opts->group_threads : 256; }

// Networks up to this size run one scenario per warp inside a multi-network launch (the
// launch shape single-network tuning picks for them); larger ones use the whole CTA.
constexpr int kWarpFormBuses = 160;

// The form of one job inside a multi-network launch.  PF_PLACE_GLOBAL: every job in CTA
// form with its data in the global workspace.  PF_PLACE_AUTO: small networks in warp
// form (vectors and factor on chip when blockDim / 32 of them fit, else global), larger
// ones in CTA form with the factor in shared memory when it fits.
struct JobForm {
    int warp;
    int placement;
};

JobForm multi_form(const pf_handle* h, const pf_solve_opts* opts) {
    if (opts->placement == PF_PLACE_GLOBAL) return {0, PF_PLACE_GLOBAL};
    const pf::Plan& P = h->plan;
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    const size_t budget = smem_budget(h);
    const size_t vec = pf::carve(nullptr, P.n_bus, P.n, ft, false, nullptr);
    const size_t fac = pf::align_up((size_t)P.nnzb() * 4 * ft, 16);
    const size_t wpc = (size_t)multi_threads(opts) / 32;
    const size_t top = top_bytes(P, ft);
    if (wpc >= 2 && P.n_bus <= kWarpFormBuses)
        return {1, (vec + fac + top) * wpc <= budget ? PF_PLACE_ONCHIP : PF_PLACE_GLOBAL};
    return {0, fac + (size_t)ft * 2 * P.n + top <= budget ? PF_PLACE_FACTOR : PF_PLACE_GLOBAL};
}

pf::SlotLayout multi_layout(const pf_handle* h, const pf_solve_opts* opts) {
    return make_layout(h, opts->precision == PF_MIXED ? 4 : 8, opts->keep_factors,
                       multi_form(h, opts).placement);
}

// Dynamic shared memory one CTA needs for a job (warp form: one arena per warp).
size_t multi_job_smem(const pf_handle* h, const pf_solve_opts* opts, const pf::SlotLayout& L) {
    const size_t per = L.fwd.smem_bytes;
    return multi_form(h, opts).warp ? per * (size_t)(multi_threads(opts) / 32) : per;
}

// Workspace: a 256-byte header (the work counter), then one region per job.
size_t multi_layout_offsets(int n_jobs, const pf_job* jobs, const pf_solve_opts* opts,
                            size_t* offsets) {
    size_t o = 256;
    for (int j = 0; j < n_jobs; ++j) {
        if (offsets) offsets[j] = o;
        o = pf::align_up(o + multi_layout(jobs[j].h, opts).slot_bytes * (size_t)jobs[j].batch, 256);
    }
    return o;
}

}  // namespace

extern "C" {

pf_err pf_multi_workspace_size(int n_jobs, const pf_job* jobs, const pf_solve_opts* opts,
                               size_t* bytes, size_t* job_offsets) {
    if (!bytes || !multi_ok(n_jobs, jobs, opts)) return PF_EINVAL;
    *bytes = multi_layout_offsets(n_jobs, jobs, opts, job_offsets);
    return PF_OK;
}

pf_err pf_solve_multi(int n_jobs, const pf_job* jobs, double tol, int max_iter,
                      const pf_solve_opts* opts, void* workspace, size_t workspace_bytes,
                      void* stream) {
    if (!multi_ok(n_jobs, jobs, opts) || !workspace || !(tol > 0.0) || max_iter < 0) return PF_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return PF_EINVAL;
    for (int j = 0; j < n_jobs; ++j) {
        const pf_job& J = jobs[j];
        if (!J.Pd || !J.Qd || !J.Pg || !J.Vset || !J.Vm || !J.Va || !J.status) return PF_EINVAL;
        if (J.h->device != jobs[0].h->device) return PF_EINVAL;
    }
    size_t offs[pf::kMaxJobs];
    if (workspace_bytes < multi_layout_offsets(n_jobs, jobs, opts, offs)) return PF_EINVAL;
    const int threads = multi_threads(opts);
    const int wpc = threads / 32;
    const int ft = opts->precision == PF_MIXED ? 4 : 8;
    // most expensive scenarios first (factor blocks x levels as the cost estimate)
    int order[pf::kMaxJobs];
    for (int j = 0; j < n_jobs; ++j) order[j] = j;
    std::stable_sort(order, order + n_jobs, [&](int a, int b) {
        const pf::Plan &pa = jobs[a].h->plan, &pb = jobs[b].h->plan;
        return (long long)pa.nnzb() * pa.n_levels > (long long)pb.nnzb() * pb.n_levels;
    });
    DeviceGuard guard(jobs[0].h->device);
    pf::MultiArgs M{};
    M.n_jobs = n_jobs;
    M.counter = static_cast<unsigned int*>(workspace);
    size_t smem = 0;
    int first = 0;
    for (int k = 0; k < n_jobs; ++k) {
        const pf_job& J = jobs[order[k]];
        pf::SlotLayout L = multi_layout(J.h, opts);
        smem = std::max(smem, multi_job_smem(J.h, opts, L));
        M.warp_form[k] = multi_form(J.h, opts).warp;
        pf::SolveArgs& A = M.args[k];
        A = pf::SolveArgs{};
        A.batch = J.batch;
        A.ipc = 1;
        A.tol = tol;
        A.max_iter = max_iter;
        A.ir_steps = opts->precision == PF_MIXED ? opts->ir_steps : 0;
        A.ir_rtol = opts->ir_rtol;
        A.ir_gate = opts->ir_gate;
        A.keep_factors = opts->keep_factors ? 1 : 0;
        A.Pd = J.Pd;
        A.Qd = J.Qd;
        A.Pg = J.Pg;
        A.Vset = J.Vset;
        A.Vm = J.Vm;
        A.Va = J.Va;
        A.Pg_out = J.Pg_out;
        A.Qg_out = J.Qg_out;
        A.fmis = J.final_mismatch;
        A.iters = J.iters;
        A.status = J.status;
        A.ws = static_cast<char*>(workspace) + offs[order[k]];
        A.L = L;
        M.plans[k] = J.h->dp;
        M.first[k] = first;
        first += M.warp_form[k] ? (J.batch + wpc - 1) / wpc : J.batch;
    }
    M.first[n_jobs] = first;
    M.total = first;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int per_sm = 0;
    cudaError_t e = ft == 4 ? pf::multi_blocks_per_sm<float>(threads, smem, &per_sm)
                            : pf::multi_blocks_per_sm<double>(threads, smem, &per_sm);
    if (e != cudaSuccess) return PF_ECUDA;
    if (per_sm < 1) return PF_ENOTSUP;  // the jobs' shared memory does not fit one CTA
    const int grid = std::min(per_sm * jobs[0].h->num_sms, M.total);
    if (cudaMemsetAsync(M.counter, 0, sizeof(unsigned int), s) != cudaSuccess) return PF_ECUDA;
    e = ft == 4 ? pf::launch_solve_multi<float>(M, threads, grid, smem, s)
                : pf::launch_solve_multi<double>(M, threads, grid, smem, s);
    if (e != cudaSuccess) return PF_ECUDA;
    for (int k = 0; k < n_jobs; ++k) {  // each handle can now run pf_adjoint on its part
        pf_handle* h = jobs[order[k]].h;
        h->last_batch = M.args[k].batch;
        h->last_ft = ft;
        h->last_keep = M.args[k].keep_factors;
        h->last_threads = M.warp_form[k] ? 32 : threads;  // the adjoint: one CTA per scenario
        h->last_qlim = 0;
        h->last_ws = M.args[k].ws;
        h->last_layout = M.args[k].L;
    }
    return PF_OK;
}

pf_err pf_autotune_multi(int n_jobs, const pf_job* jobs, double tol, int max_iter,
                         const pf_solve_opts* opts, void* workspace, size_t workspace_bytes,
                         void* stream, pf_tune_result* out) {
    if (!multi_ok(n_jobs, jobs, opts) || !workspace || !out) return PF_EINVAL;
    // the workspace must hold every candidate's layout
    for (int th : {128, 256, 512}) {
        for (int pl : {PF_PLACE_AUTO, PF_PLACE_GLOBAL}) {
            pf_solve_opts o = *opts;
            o.placement = pl;
            o.group_threads = th;
            if (workspace_bytes < multi_layout_offsets(n_jobs, jobs, &o, nullptr)) return PF_EINVAL;
        }
    }
    DeviceGuard guard(jobs[0].h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PF_ECUDA;
    }
    pf_tune_result best{0, 0, 0, 0.f};
    pf_err err = PF_OK;
    for (int th : {128, 256, 512}) {
        for (int pl : {PF_PLACE_AUTO, PF_PLACE_GLOBAL}) {
            pf_solve_opts o = *opts;
            o.group_threads = th;
            o.placement = pl;
            o.instances_per_cta = 0;
            float ms_best = 0.f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {  // rep 0 warms up
                cudaEventRecord(e0, s);
                const pf_err r = pf_solve_multi(n_jobs, jobs, tol, max_iter, &o, workspace,
                                                workspace_bytes, stream);
                cudaEventRecord(e1, s);
                if (r == PF_ENOTSUP) { ok = false; break; }  // does not fit: not a candidate
                if (r != PF_OK) { err = r; ok = false; break; }
                if (cudaEventSynchronize(e1) != cudaSuccess) { err = PF_ECUDA; ok = false; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && (ms_best == 0.f || ms < ms_best)) ms_best = ms;
            }
            if (err != PF_OK) break;
            if (ok && (best.group_threads == 0 || ms_best < best.ms)) best = {th, pl, 1, ms_best};
        }
        if (err != PF_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int j = 0; j < n_jobs; ++j) jobs[j].h->last_batch = -1;  // trial solves: no adjoint state
    if (err != PF_OK) return err;
    if (best.group_threads == 0) return PF_ENOTSUP;
    *out = best;
    return PF_OK;
}

void pf_destroy(pf_handle* h) {
    if (!h) return;
    if (h->d_buf) {
        DeviceGuard guard(h->device);
        cudaDeviceSynchronize();
        cudaFree(h->d_buf);
    }
    delete h;
}

}  // extern "C"
