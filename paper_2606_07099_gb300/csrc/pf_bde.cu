// pf_bde.cu -- the "one big matrix" execution of the batched Newton-Raphson solve.
//
// The paper solves a batch as one block-diagonal (BDE) sparse system: each step of a
// Newton iteration -- mismatch, Jacobian values, numeric LU, triangular solves, update --
// is one operation over the whole batch matrix, driven from the host, which also checks
// convergence (Sec. III-A, III-B).  This file runs that execution model with this
// library's own kernels, so it can be measured beside the fused solver (pf_solve, one
// persistent launch in which each CTA iterates its own scenario): one kernel per phase
// and, for the factorisation and the sweeps, one kernel per elimination-tree level, each
// spanning every scenario of the batch; the host reads the number of unconverged
// scenarios after every mismatch.  Values are stored scenario-interleaved (entry-major:
// value k of scenario b at k * batch + b), so consecutive threads, which take
// consecutive scenarios of the same entry, access consecutive addresses.  FP64
// throughout (the FP64 form of pf_solve, same symbolic plan, same element formulas).
#include <algorithm>
#include <vector>

#include "pf_body.cuh"
#include "pf_launch.h"

namespace pf {

namespace {

constexpr int kActive = -1;  // status of a scenario still iterating

struct BdeState {
    int batch;
    double *Vm, *Va, *Vre, *Vim, *Ire, *Iim;  // [n_bus][batch]
    double *F, *x;                            // [2n][batch]
    double* fac;                              // [nnzb][4][batch]
    unsigned long long* nkey;                 // [batch] max |F1| as an ordered key
    int *status, *iters, *bad;                // [batch]
    unsigned int* active;                     // unconverged scenarios (one counter)
};

__device__ __forceinline__ unsigned long long mag_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

#define BDE_LOOP(total) \
    for (long long t_ = blockIdx.x * (long long)blockDim.x + threadIdx.x; t_ < (total); \
         t_ += (long long)gridDim.x * blockDim.x)

__global__ void bde_start(DevPlan P, BdeState S, const double* Vset) {
    BDE_LOOP((long long)P.n_bus * S.batch) {
        const int b = (int)(t_ % S.batch), i = (int)(t_ / S.batch);
        const double vm = (__ldg(P.bus_type + i) == 0) ? 1.0 : Vset[(size_t)b * P.n_bus + i];
        S.Vm[t_] = vm;
        S.Va[t_] = 0.0;
        S.Vre[t_] = vm;
        S.Vim[t_] = 0.0;
        if (i == 0) {
            S.status[b] = kActive;
            S.iters[b] = 0;
            S.nkey[b] = 0ull;
            S.bad[b] = 0;
        }
    }
}

// I = Y V, F1 at pivot positions, max |F1| per scenario (active scenarios)
__global__ void bde_mismatch(DevPlan P, BdeState S, const double* Pd, const double* Qd,
                             const double* Pg) {
    BDE_LOOP((long long)P.n_bus * S.batch) {
        const int b = (int)(t_ % S.batch), i = (int)(t_ / S.batch);
        if (S.status[b] != kActive) continue;
        double ir = 0.0, ii = 0.0;
        for (int k = __ldg(P.y_ptr + i); k < __ldg(P.y_ptr + (i + 1)); ++k) {
            const size_t j = (size_t)__ldg(P.y_idx + k) * S.batch + b;
            const double2 y = __ldg(P.y_gb + k);
            ir = fma(y.x, S.Vre[j], fma(-y.y, S.Vim[j], ir));
            ii = fma(y.x, S.Vim[j], fma(y.y, S.Vre[j], ii));
        }
        S.Ire[t_] = ir;
        S.Iim[t_] = ii;
        const int p = __ldg(P.bus2pos + i);
        if (p < 0) continue;
        const double vr = S.Vre[t_], vi = S.Vim[t_];
        const int ty = __ldg(P.bus_type + i);
        const size_t row = (size_t)b * P.n_bus + i;
        const double fP = (ty == 1 ? Pg[row] : 0.0) - Pd[row] - (vr * ir + vi * ii);
        const double fQ = (ty == 0) ? -Qd[row] - (vi * ir - vr * ii) : 0.0;
        S.F[(size_t)(2 * p) * S.batch + b] = fP;
        S.F[(size_t)(2 * p + 1) * S.batch + b] = fQ;
        atomicMax(S.nkey + b, mag_key(fP) > mag_key(fQ) ? mag_key(fP) : mag_key(fQ));
    }
}

// the convergence decision of each scenario after a mismatch; counts the ones that go on
__global__ void bde_decide(BdeState S, double tol, int k, int max_iter, double* fmis) {
    BDE_LOOP(S.batch) {
        const int b = (int)t_;
        if (S.status[b] != kActive) continue;
        const unsigned long long key = S.nkey[b];
        const double norm = key >= 0x7FF0000000000000ull ? INFINITY : __longlong_as_double((long long)key);
        S.nkey[b] = 0ull;
        S.bad[b] = 0;
        if (fmis) fmis[b] = norm;
        if (!(norm <= 1e10)) S.status[b] = 2;
        else if (norm <= tol) S.status[b] = 0;
        else if (k >= max_iter) S.status[b] = 1;
        else atomicAdd(S.active, 1u);
    }
}

// Jacobian blocks (Alg. 1 element formulas, FP64) into the factor template
__global__ void bde_fill(DevPlan P, BdeState S) {
    BDE_LOOP((long long)P.nnzb * S.batch) {
        const int b = (int)(t_ % S.batch), e = (int)(t_ / S.batch);
        if (S.status[b] != kActive) continue;
        const int p = __ldg(P.lu_row + e), q = __ldg(P.lu_col + e);
        const int yi = __ldg(P.fill_y + e);
        const int i = __ldg(P.pos2bus + p), j = __ldg(P.pos2bus + q);
        Blk<double> m{0.0, 0.0, 0.0, 0.0};
        if (yi >= 0) {
            const size_t bi = (size_t)i * S.batch + b, bj = (size_t)j * S.batch + b;
            const double2 y = __ldg(P.y_gb + yi);
            const double vmi = S.Vm[bi], vmj = S.Vm[bj];
            const double c = S.Vre[bi] / vmi, s = S.Vim[bi] / vmi;
            const double ir = S.Ire[bi], ii = S.Iim[bi];
            m = jac_block<double>(p == q, y.x, y.y, S.Vre[bi], S.Vim[bi], S.Vre[bj] / vmj,
                                  S.Vim[bj] / vmj, vmj, vmi, c * ir + s * ii, s * ir - c * ii);
        }
        m = pad_pv(m, p == q, __ldg(P.bus_type + i), __ldg(P.bus_type + j));
        double* f = S.fac + (size_t)e * 4 * S.batch + b;
        f[0] = m.a;
        f[S.batch] = m.b;
        f[2 * (size_t)S.batch] = m.c;
        f[3 * (size_t)S.batch] = m.d;
    }
}

__device__ __forceinline__ Blk<double> bld(const BdeState& S, int e, int b) {
    const double* f = S.fac + (size_t)e * 4 * S.batch + b;
    return {f[0], f[S.batch], f[2 * (size_t)S.batch], f[3 * (size_t)S.batch]};
}
__device__ __forceinline__ void bst(const BdeState& S, int e, int b, Blk<double> m) {
    double* f = S.fac + (size_t)e * 4 * S.batch + b;
    f[0] = m.a;
    f[S.batch] = m.b;
    f[2 * (size_t)S.batch] = m.c;
    f[3 * (size_t)S.batch] = m.d;
}

// LU, level l, phase A: L(i,k) <- A(i,k) inv(A(k,k)) for the level's L columns
__global__ void bde_lu_scale(DevPlan P, BdeState S, int l) {
    const int a0 = __ldg(P.la_ptr + l), na = __ldg(P.la_ptr + l + 1) - a0;
    BDE_LOOP((long long)na * S.batch) {
        const int b = (int)(t_ % S.batch), c = a0 + (int)(t_ / S.batch);
        if (S.status[b] != kActive) continue;
        const int2 ld = __ldg(P.la + c);
        int dummy = 0;
        bst(S, ld.x, b, mul(bld(S, ld.x, b), inv2(bld(S, ld.y, b), &dummy)));
    }
}

// LU, level l, phase B: the Schur updates of every target of the level, and the level's
// pivots replaced by their inverses (a singular pivot marks the scenario)
__global__ void bde_lu_update(DevPlan P, BdeState S, int l) {
    const int t0 = __ldg(P.sch_tptr + l), nt = __ldg(P.sch_tptr + l + 1) - t0;
    const int p0 = __ldg(P.lev_ptr + l), np = __ldg(P.lev_ptr + l + 1) - p0;
    BDE_LOOP((long long)(nt + np) * S.batch) {
        const int b = (int)(t_ % S.batch), w = (int)(t_ / S.batch);
        if (S.status[b] != kActive) continue;
        if (w < nt) {
            const int t = t0 + w;
            Blk<double> acc{0.0, 0.0, 0.0, 0.0};
            for (int c = __ldg(P.sch_cptr + t); c < __ldg(P.sch_cptr + t + 1); ++c) {
                const int2 lu = __ldg(P.sch + c);
                const Blk<double> xl = bld(S, lu.x, b), yu = bld(S, lu.y, b);
                acc.a += xl.a * yu.a + xl.b * yu.c;
                acc.b += xl.a * yu.b + xl.b * yu.d;
                acc.c += xl.c * yu.a + xl.d * yu.c;
                acc.d += xl.c * yu.b + xl.d * yu.d;
            }
            const int tg = __ldg(P.sch_tgt + t);
            const Blk<double> m = bld(S, tg, b);
            bst(S, tg, b, {m.a - acc.a, m.b - acc.b, m.c - acc.c, m.d - acc.d});
        } else {
            const int dk = __ldg(P.lu_diag + p0 + (w - nt));
            int bad = 0;
            bst(S, dk, b, inv2(bld(S, dk, b), &bad));
            if (bad) S.bad[b] = 1;
        }
    }
}

// after the factorisation: a singular scenario stops; the others get x = -F1
__global__ void bde_rhs(DevPlan P, BdeState S) {
    BDE_LOOP((long long)2 * P.n * S.batch) {
        const int b = (int)(t_ % S.batch);
        if (S.status[b] != kActive) continue;
        if (S.bad[b]) {
            if (t_ < S.batch) S.status[b] = 3;  // one thread per scenario decides
            continue;
        }
        S.x[t_] = -S.F[t_];
    }
}

// one level of a triangular sweep: lower (L y = x, unit diagonal) or upper (U x = y,
// pivots stored inverted)
template <bool UPPER>
__global__ void bde_sweep(DevPlan P, BdeState S, int l) {
    const int r0 = __ldg(P.lev_ptr + l), nr = __ldg(P.lev_ptr + l + 1) - r0;
    BDE_LOOP((long long)nr * S.batch) {
        const int b = (int)(t_ % S.batch), p = r0 + (int)(t_ / S.batch);
        if (S.status[b] != kActive || S.bad[b]) continue;
        const int dg = __ldg(P.lu_diag + p);
        const int e0 = UPPER ? dg + 1 : __ldg(P.lu_ptr + p);
        const int e1 = UPPER ? __ldg(P.lu_ptr + p + 1) : dg;
        double s0 = 0.0, s1 = 0.0;
        for (int e = e0; e < e1; ++e) {
            const int q = __ldg(P.lu_col + e);
            const Blk<double> m = bld(S, e, b);
            const double y0 = S.x[(size_t)(2 * q) * S.batch + b];
            const double y1 = S.x[(size_t)(2 * q + 1) * S.batch + b];
            s0 += m.a * y0 + m.b * y1;
            s1 += m.c * y0 + m.d * y1;
        }
        double* x0 = S.x + (size_t)(2 * p) * S.batch + b;
        double* x1 = S.x + (size_t)(2 * p + 1) * S.batch + b;
        const double v0 = *x0 - s0, v1 = *x1 - s1;
        if (UPPER) {
            const Blk<double> d = bld(S, dg, b);
            *x0 = d.a * v0 + d.b * v1;
            *x1 = d.c * v0 + d.d * v1;
        } else {
            *x0 = v0;
            *x1 = v1;
        }
    }
}

// theta_{B\R} += dtheta, Vm_D += dVm, V = Vm e^{j theta}
__global__ void bde_update(DevPlan P, BdeState S) {
    BDE_LOOP((long long)P.n * S.batch) {
        const int b = (int)(t_ % S.batch), p = (int)(t_ / S.batch);
        if (S.status[b] != kActive || S.bad[b]) continue;
        const int i = __ldg(P.pos2bus + p);
        const size_t bi = (size_t)i * S.batch + b;
        const double th = S.Va[bi] + S.x[(size_t)(2 * p) * S.batch + b];
        const double vm = S.Vm[bi] + ((__ldg(P.bus_type + i) == 0) ? S.x[(size_t)(2 * p + 1) * S.batch + b] : 0.0);
        double s, c;
        sincos(th, &s, &c);
        S.Va[bi] = th;
        S.Vm[bi] = vm;
        S.Vre[bi] = vm * c;
        S.Vim[bi] = vm * s;
        if (p == 0) S.iters[b] += 1;
    }
}

// Step 2 (Eq. F2_completion) and the outputs, [batch][n_bus]
__global__ void bde_finish(DevPlan P, BdeState S, const double* Pd, const double* Qd,
                           const double* Pg, double* Vm, double* Va, double* Pg_out,
                           double* Qg_out, int* iters, int* status) {
    BDE_LOOP((long long)P.n_bus * S.batch) {
        const int b = (int)(t_ % S.batch), i = (int)(t_ / S.batch);
        const size_t row = (size_t)b * P.n_bus + i;
        const int ty = __ldg(P.bus_type + i);
        const double vr = S.Vre[t_], vi = S.Vim[t_], ir = S.Ire[t_], ii = S.Iim[t_];
        Vm[row] = S.Vm[t_];
        Va[row] = S.Va[t_];
        if (Pg_out) Pg_out[row] = (ty == 1) ? Pg[row] : (ty == 2 ? vr * ir + vi * ii + Pd[row] : 0.0);
        if (Qg_out) Qg_out[row] = (ty == 0) ? 0.0 : (vi * ir - vr * ii) + Qd[row];
        if (i == 0) {
            status[b] = S.status[b];
            if (iters) iters[b] = S.iters[b];
        }
    }
}

int grid_for(long long threads) {
    return (int)std::min<long long>(std::max<long long>((threads + 255) / 256, 1), 152LL * 64);
}

}  // namespace

size_t bde_workspace_bytes(const DevPlan& P, int batch) {
    const size_t B = (size_t)batch;
    size_t o = 0;
    auto take = [&](size_t bytes) { o = align_up(o + bytes, 256); };
    for (int k = 0; k < 6; ++k) take(8 * B * P.n_bus);
    take(8 * B * 2 * P.n);
    take(8 * B * 2 * P.n);
    take(8 * B * 4 * (size_t)P.nnzb);
    take(8 * B);
    take(4 * B);
    take(4 * B);
    take(4 * B);
    take(4);
    return o;
}

cudaError_t solve_bde(const DevPlan& P, int batch, const double* Pd, const double* Qd,
                      const double* Pg, const double* Vset, double tol, int max_iter, double* Vm,
                      double* Va, double* Pg_out, double* Qg_out, int* iters, int* status,
                      double* fmis, void* ws, cudaStream_t s) {
    BdeState S{};
    S.batch = batch;
    unsigned char* base = static_cast<unsigned char*>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + o;
        o = align_up(o + bytes, 256);
        return p;
    };
    const size_t B = (size_t)batch;
    double** bus[6] = {&S.Vm, &S.Va, &S.Vre, &S.Vim, &S.Ire, &S.Iim};
    for (double** d : bus) *d = reinterpret_cast<double*>(take(8 * B * P.n_bus));
    S.F = reinterpret_cast<double*>(take(8 * B * 2 * P.n));
    S.x = reinterpret_cast<double*>(take(8 * B * 2 * P.n));
    S.fac = reinterpret_cast<double*>(take(8 * B * 4 * (size_t)P.nnzb));
    S.nkey = reinterpret_cast<unsigned long long*>(take(8 * B));
    S.status = reinterpret_cast<int*>(take(4 * B));
    S.iters = reinterpret_cast<int*>(take(4 * B));
    S.bad = reinterpret_cast<int*>(take(4 * B));
    S.active = reinterpret_cast<unsigned int*>(take(4));

    const long long nb = (long long)P.n_bus * batch;
    bde_start<<<grid_for(nb), 256, 0, s>>>(P, S, Vset);
    std::vector<int> h_lev(P.n_levels + 1), h_la(P.n_levels + 1), h_sch(P.n_levels + 1);
    cudaError_t e = cudaMemcpyAsync(h_lev.data(), P.lev_ptr, sizeof(int) * (P.n_levels + 1),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_la.data(), P.la_ptr, sizeof(int) * (P.n_levels + 1),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_sch.data(), P.sch_tptr, sizeof(int) * (P.n_levels + 1),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int k = 0;; ++k) {
        bde_mismatch<<<grid_for(nb), 256, 0, s>>>(P, S, Pd, Qd, Pg);
        if ((e = cudaMemsetAsync(S.active, 0, 4, s)) != cudaSuccess) return e;
        bde_decide<<<grid_for(batch), 256, 0, s>>>(S, tol, k, max_iter, fmis);
        unsigned int active = 0;  // the host's convergence check of this execution model
        if ((e = cudaMemcpyAsync(&active, S.active, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (active == 0) break;
        bde_fill<<<grid_for((long long)P.nnzb * batch), 256, 0, s>>>(P, S);
        for (int l = 0; l < P.n_levels; ++l) {
            const long long na = h_la[l + 1] - h_la[l];
            const long long nt = (h_sch[l + 1] - h_sch[l]) + (h_lev[l + 1] - h_lev[l]);
            if (na) bde_lu_scale<<<grid_for(na * batch), 256, 0, s>>>(P, S, l);
            bde_lu_update<<<grid_for(nt * batch), 256, 0, s>>>(P, S, l);
        }
        bde_rhs<<<grid_for((long long)2 * P.n * batch), 256, 0, s>>>(P, S);
        for (int l = 0; l < P.n_levels; ++l)
            bde_sweep<false><<<grid_for((long long)(h_lev[l + 1] - h_lev[l]) * batch), 256, 0, s>>>(P, S, l);
        for (int l = P.n_levels - 1; l >= 0; --l)
            bde_sweep<true><<<grid_for((long long)(h_lev[l + 1] - h_lev[l]) * batch), 256, 0, s>>>(P, S, l);
        bde_update<<<grid_for((long long)P.n * batch), 256, 0, s>>>(P, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    bde_finish<<<grid_for(nb), 256, 0, s>>>(P, S, Pd, Qd, Pg, Vm, Va, Pg_out, Qg_out, iters, status);
    return cudaGetLastError();
}

}  // namespace pf
