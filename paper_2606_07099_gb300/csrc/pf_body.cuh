// pf_body.cuh -- device code of the batched Newton-Raphson power flow and its adjoint
// on sm_103a (internal; included by the translation units that instantiate kernels).
//
// One CTA owns one scenario at a time (the grid has one CTA per scenario, so the
// hardware block scheduler balances scenarios that need different iteration
// counts).  Every step of a Newton iteration runs inside the same kernel, on the
// scenario's state staged in shared memory when it fits:
//
//   mismatch  I = Y V, S = V conj(I), F1 = spec - S           (Sec. II-A, FP64)
//   fill      polar 2x2 Jacobian blocks on the fixed pattern  (Alg. 1 values, FT)
//   factor    level-scheduled right-looking 2x2-block LU      (FT = float | double)
//   solve     level-scheduled block triangular sweeps         (FT)
//   refine    FP64 residual r = -F1 - J1 dz (matrix-free)     (Table I + refinement)
//   update    theta_{B\R} += dtheta, Vm_D += dVm, u and V     (FP64)
//
// until ||F1||_inf <= tol; then Step 2 (Eq. F2_completion) writes the recovered
// generation.  The convergence decision is taken on the device per scenario;
// the host never waits inside the loop.
#pragma once

#include <cfloat>
#include <cmath>

#include "pf_device.cuh"

namespace pf {

// ---------------------------------------------------------------- small helpers
template <typename T>
struct Blk {
    T a, b, c, d;  // [[a, b], [c, d]]: rows (dP, dQ), columns (theta, Vm)
};

__device__ __forceinline__ Blk<float> ldb(const float* f, int e) {
    float4 v = reinterpret_cast<const float4*>(f)[e];
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Blk<double> ldb(const double* f, int e) {
    const double2* p = reinterpret_cast<const double2*>(f) + 2 * e;
    double2 u = p[0], w = p[1];
    return {u.x, u.y, w.x, w.y};
}
__device__ __forceinline__ void stb(float* f, int e, Blk<float> v) {
    reinterpret_cast<float4*>(f)[e] = make_float4(v.a, v.b, v.c, v.d);
}
__device__ __forceinline__ void stb(double* f, int e, Blk<double> v) {
    double2* p = reinterpret_cast<double2*>(f) + 2 * e;
    p[0] = make_double2(v.a, v.b);
    p[1] = make_double2(v.c, v.d);
}
template <typename T>
__device__ __forceinline__ Blk<T> mul(Blk<T> x, Blk<T> y) {
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c,
            x.c * y.b + x.d * y.d};
}
// x - y*z
template <typename T>
__device__ __forceinline__ Blk<T> msub(Blk<T> x, Blk<T> y, Blk<T> z) {
    return {x.a - (y.a * z.a + y.b * z.c), x.b - (y.a * z.b + y.b * z.d),
            x.c - (y.c * z.a + y.d * z.c), x.d - (y.c * z.b + y.d * z.d)};
}
// inverse of a 2x2 block; *bad = 1 if (numerically) singular or non-finite
template <typename T>
__device__ __forceinline__ Blk<T> inv2(Blk<T> m, int* bad) {
    T det = m.a * m.d - m.b * m.c;
    T amax = fmax(fmax(fabs(m.a), fabs(m.b)), fmax(fabs(m.c), fabs(m.d)));
    if (!(fabs(det) > T(1e-30) * amax * amax) || !(amax < T(INFINITY))) *bad = 1;
    T r = T(1) / det;
    return {m.d * r, -m.b * r, -m.c * r, m.a * r};
}

template <typename T>
__device__ __forceinline__ T* ftptr(void* p) { return reinterpret_cast<T*>(p); }

// A "group" solves one scenario: either the whole CTA (W = false) or one warp of it
// (W = true: several independent scenarios per CTA, one per warp).  GTID / GSZ are the
// thread's rank and the size of its group; gsync<W> is the group barrier.
#define GTID (W ? (int)(threadIdx.x & 31u) : (int)threadIdx.x)
#define GSZ (W ? 32 : (int)blockDim.x)

template <bool W>
__device__ __forceinline__ void gsync() {
    if (W || blockDim.x == 32) __syncwarp();
    else __syncthreads();
}

// |v| as an ordered integer key: for non-negative doubles the IEEE order is the order of
// their bit patterns, so a max over keys is an exact FP64 max done on the integer pipe
// (an FP64 compare costs a warp 64 cycles of this GPU's FP64 pipe).  NaN keys exceed the
// key of +inf; key_to_norm maps them (and +inf) to +inf.
__device__ __forceinline__ unsigned long long abs_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ double key_to_norm(unsigned long long k) {
    return k < 0x7ff0000000000000ULL ? __longlong_as_double((long long)k) : INFINITY;
}
// |v| with non-finite values mapped to +inf (so that max-reductions see them)
__device__ __forceinline__ float absinf(float v) {
    float a = fabsf(v);
    return (a <= FLT_MAX) ? a : INFINITY;
}

// Group-wide max of non-negative, non-NaN values (norms, flags); every thread gets the
// result.  For such values the order of the bit patterns is the order of the values, so
// the max runs on the integer pipe.  `red` holds one double per warp.
template <bool W>
__device__ double group_max(double v, double* red) {
    unsigned long long k = (unsigned long long)__double_as_longlong(v);
    for (int o = 16; o; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
    if (W || blockDim.x == 32) {
        __syncwarp();  // also orders the shared-memory writes of the phase that reduced
        return __longlong_as_double((long long)k);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = __longlong_as_double((long long)k);
    __syncthreads();
    unsigned long long r = (unsigned long long)__double_as_longlong(red[0]);
    for (int i = 1; i < nw; ++i) r = max(r, (unsigned long long)__double_as_longlong(red[i]));
    return __longlong_as_double((long long)r);
}

// ---------------------------------------------------------------- FP64 network kernels
// e^{j d} for a Newton angle step |d| <= 1/8 from the Maclaurin series of sin and cos,
// truncated after d^9 and d^10: the first omitted terms, d^11/11! and d^12/12!, are below
// 2.4e-17 and 3.1e-20 relative.  Horner form in d^2 with the series' own coefficients
// (constants folded at compile time): 11 FP64 operations, each a scarce FP64-pipe slot.
__device__ __forceinline__ void small_angle_phasor(double d, double* c, double* s) {
    const double d2 = d * d;
    const double ps =
        fma(d2, fma(d2, fma(d2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0);
    *s = fma(d * d2, ps, d);
    *c = fma(d2,
             fma(d2,
                 fma(d2, fma(d2, fma(d2, -1.0 / 3628800.0, 1.0 / 40320.0), -1.0 / 720.0),
                     1.0 / 24.0),
                 -0.5),
             1.0);
}

// Newton update of one bus (FP64) that also advances u = e^{j theta} and V = Vm u: small
// angle steps rotate u by e^{j dth}; larger ones recompute it from theta.
__device__ __forceinline__ void update_bus(const Arrays& a, int i, double dth, double dvm, bool pq) {
    const double th = a.Va[i] + dth;
    a.Va[i] = th;
    const double vm = pq ? a.Vm[i] + dvm : a.Vm[i];
    a.Vm[i] = vm;
    double c, s;
    if (abs_key(dth) <= 0x3fc0000000000000ULL) {  // |dth| <= 1/8 (false for NaN)
        double rc, rs;
        small_angle_phasor(dth, &rc, &rs);
        const double uc = a.Uc[i], us = a.Us[i];
        c = uc * rc - us * rs;
        s = us * rc + uc * rs;
    } else {
        sincos(th, &s, &c);
    }
    a.Uc[i] = c;
    a.Us[i] = s;
    a.Vre[i] = vm * c;
    a.Vim[i] = vm * s;
}

// The bus type the Newton equations of this scenario use: the network's, or under
// reactive limits (QL) the scenario's own partition (PV buses may have become PQ).
template <bool QL>
__device__ __forceinline__ int ntype(const DevPlan& P, const Arrays& a, int i) {
    return QL ? (int)a.stype[i] : __ldg(P.bus_type + i);
}

// FP32 copies of the per-bus quantities the FP32 Jacobian fill reads:
// V, u, Vm and (pu, qu) = u conj(I), so that S = Vm (pu + j qu).  Five conversions, the
// products formed in FP32: the FP32 Jacobian is the refinement's preconditioner, and an
// FP64 operation costs a warp 64 cycles of this GPU's FP64 pipe (an FP32 one, 1-2).
__device__ __forceinline__ void store_bus_f32(const Arrays& a, int i, double ir, double ii) {
    const float c = float(a.Uc[i]), s = float(a.Us[i]), vm = float(a.Vm[i]);
    const float fir = float(ir), fii = float(ii);
    a.fvr[i] = vm * c;
    a.fvi[i] = vm * s;
    a.fur[i] = c;
    a.fui[i] = s;
    a.fvm[i] = vm;
    a.fpu[i] = fmaf(c, fir, s * fii);
    a.fqu[i] = fmaf(s, fir, -(c * fii));
}

// I = Y V, S = V conj(I), F1 at pivot positions; returns ||F1||_inf (inf if non-finite).
// The specified injections P_spec = pg - pd (pg on PV buses only) and Q_spec = -qd are
// read from the scenario's input rows.  With F32COPY the FP32 per-bus copies for the
// FP32 Jacobian fill are written too.
template <bool F32COPY, bool W, bool QL = false>
__device__ double phase_mismatch(const DevPlan& P, const Arrays& a, const double* Pd,
                                 const double* Qd, const double* Pg, double* red) {
    unsigned long long kmax = 0;
    for (int i = GTID; i < P.n_bus; i += GSZ) {
        double ir = 0.0, ii = 0.0;
        for (int k = __ldg(P.y_ptr + i); k < __ldg(P.y_ptr + (i + 1)); ++k) {
            const int j = __ldg(P.y_idx + k);
            const double2 y = __ldg(P.y_gb + k);
            const double vr = a.Vre[j], vi = a.Vim[j];
            ir = fma(y.x, vr, fma(-y.y, vi, ir));
            ii = fma(y.x, vi, fma(y.y, vr, ii));
        }
        a.Ire[i] = ir;
        a.Iim[i] = ii;
        if (F32COPY) store_bus_f32(a, i, ir, ii);
        const int p = __ldg(P.bus2pos + i);
        if (p >= 0) {
            const double vr = a.Vre[i], vi = a.Vim[i];
            const int t = ntype<QL>(P, a, i);
            // pg enters at every generator bus that is not a reference bus: PV buses and
            // PV buses switched to PQ under reactive limits (whose network type is still 1)
            const double psp = (__ldg(P.bus_type + i) == 1 ? __ldg(Pg + i) : 0.0) - __ldg(Pd + i);
            const double qsp = (QL ? a.qfix[i] : 0.0) - __ldg(Qd + i);
            // F = spec - S with S = V conj(I) = (vr ir + vi ii) + j (vi ir - vr ii), as FMA
            // chains onto the specified values
            const double fP = fma(-vr, ir, fma(-vi, ii, psp));
            const double fQ = (t == 0) ? fma(-vi, ir, fma(vr, ii, qsp)) : 0.0;
            a.F[2 * p] = fP;
            a.F[2 * p + 1] = fQ;
            kmax = max(kmax, max(abs_key(fP), abs_key(fQ)));
        }
    }
    return group_max<W>(key_to_norm(kmax), red);
}

// G_j = conj(m_j I_j) + sum_i m_i conj(V_i) Y_ij;  w0_j = Re(G_j u_j) = d(m.S)/dVm_j,
// w1_j = -Im(G_j V_j) = d(m.S)/dtheta_j, for the injection weights m = mP + j mQ held in
// (Psp, Qsp).  This is (d[P;Q]/d[Vm;theta])^T [mP; mQ] without forming the Jacobian.
template <bool W>
__device__ void phase_jvt(const DevPlan& P, const Arrays& a) {
    for (int i = GTID; i < P.n_bus; i += GSZ) {
        const double mr = a.Psp[i], mi = a.Qsp[i];
        // h = m conj(V)
        a.dVre[i] = mr * a.Vre[i] + mi * a.Vim[i];
        a.dVim[i] = mi * a.Vre[i] - mr * a.Vim[i];
    }
    gsync<W>();
    for (int j = GTID; j < P.n_bus; j += GSZ) {
        double gr = 0.0, gi = 0.0;
        for (int k = __ldg(P.yt_ptr + j); k < __ldg(P.yt_ptr + (j + 1)); ++k) {
            const int i = __ldg(P.yt_idx + k);
            const double2 y = __ldg(P.yt_gb + k);  // Y_ij
            const double hr = a.dVre[i], hi = a.dVim[i];
            gr = fma(hr, y.x, fma(-hi, y.y, gr));
            gi = fma(hr, y.y, fma(hi, y.x, gi));
        }
        const double mr = a.Psp[j], mi = a.Qsp[j];
        const double Ir = a.Ire[j], Ii = a.Iim[j];
        // conj(m I) = (mr Ir - mi Ii) - j(mr Ii + mi Ir), as FMA chains onto the sums
        gr = fma(mr, Ir, fma(-mi, Ii, gr));
        gi = fma(-mr, Ii, fma(-mi, Ir, gi));
        const double vr = a.Vre[j], vi = a.Vim[j];
        a.w0[j] = gr * a.Uc[j] - gi * a.Us[j];
        a.w1[j] = -(gr * vi + gi * vr);
    }
}

// ---------------------------------------------------------------- Jacobian fill (Alg. 1)
// J1 = dF1/dz1 in 2x2 blocks; F = spec - S, so every entry is minus the derivative of
// the calculated injection.  With u = e^{j theta}, W = V_i conj(Y_ij V_j) and
// W' = V_i conj(Y_ij u_j) = W / Vm_j (i != j):
//   dP_i/dtheta_j = Im W, dQ_i/dtheta_j = -Re W, dP_i/dVm_j = Re W', dQ_i/dVm_j = Im W';
// on the diagonal, with pu + j qu = u_i conj(I_i) (so P_i + j Q_i = Vm_i (pu + j qu)):
//   dP_i/dtheta_i = -Q_i - B_ii Vm_i^2, dQ_i/dtheta_i = P_i - G_ii Vm_i^2,
//   dP_i/dVm_i = pu + G_ii Vm_i,        dQ_i/dVm_i = qu - B_ii Vm_i.
// The values are the same as Alg. 1's; they are computed in the precision of the
// factor they feed (FP32 from FP32 copies of the bus quantities, or FP64).
template <typename T>
__device__ __forceinline__ Blk<T> jac_block(bool diag, T gij, T bij, T vri, T vii, T urj, T uij,
                                            T vmj, T vmi, T pui, T qui) {
    if (diag) {
        const T vm2 = vmi * vmi;
        return {vmi * qui + bij * vm2, -(pui + gij * vmi), -vmi * pui + gij * vm2,
                -(qui - bij * vmi)};
    }
    const T yur = gij * urj - bij * uij, yui = gij * uij + bij * urj;  // Y_ij u_j
    const T wr = vri * yur + vii * yui;                                 // W' = V_i conj(Y_ij u_j)
    const T wi = vii * yur - vri * yui;
    return {-wi * vmj, -wr, wr * vmj, -wi};
}

template <typename T>
__device__ __forceinline__ Blk<T> pad_pv(Blk<T> m, bool diag, int ti, int tj) {
    // PV buses: no dQ row and no Vm column; padded with the identity equation dVm_i = 0
    if (ti == 1) { m.c = T(0); m.d = T(0); }
    if (tj == 1) { m.b = T(0); m.d = T(0); }
    if (diag && ti == 1) m.d = T(1);
    return m;
}

template <bool W, bool QL = false>
__device__ void phase_fill(const DevPlan& P, const Arrays& a, float* fac) {
    // two blocks per thread and round: both blocks' loads are issued before either store
    // (the stores to the factor could otherwise alias the next block's bus reads)
    auto block = [&](int e, int p, int q, int yi, int i, int j) {
        Blk<float> m{0.f, 0.f, 0.f, 0.f};
        if (yi >= 0) {
            const float2 y = __ldg(P.y_gb32 + yi);
            m = jac_block<float>(p == q, y.x, y.y, a.fvr[i], a.fvi[i], a.fur[j], a.fui[j],
                                 a.fvm[j], a.fvm[i], a.fpu[i], a.fqu[i]);
        }
        return pad_pv(m, p == q, ntype<QL>(P, a, i), ntype<QL>(P, a, j));
    };
    for (int e = GTID; e < P.nnzb; e += 2 * GSZ) {
        const int e2 = e + GSZ;
        const bool two = e2 < P.nnzb;
        const int p = __ldg(P.lu_row + e), q = __ldg(P.lu_col + e);
        const int p2 = two ? __ldg(P.lu_row + e2) : p, q2 = two ? __ldg(P.lu_col + e2) : q;
        const int yi = __ldg(P.fill_y + e), yi2 = two ? __ldg(P.fill_y + e2) : -1;
        const int i = __ldg(P.pos2bus + p), j = __ldg(P.pos2bus + q);
        const int i2 = __ldg(P.pos2bus + p2), j2 = __ldg(P.pos2bus + q2);
        const Blk<float> m1 = block(e, p, q, yi, i, j);
        const Blk<float> m2 = block(e2, p2, q2, yi2, i2, j2);
        stb(fac, e, m1);
        if (two) stb(fac, e2, m2);
    }
}

template <bool W, bool QL = false>
__device__ void phase_fill(const DevPlan& P, const Arrays& a, double* fac) {
    for (int e = GTID; e < P.nnzb; e += GSZ) {
        const int p = __ldg(P.lu_row + e), q = __ldg(P.lu_col + e);
        const int yi = __ldg(P.fill_y + e);
        const int i = __ldg(P.pos2bus + p), j = __ldg(P.pos2bus + q);
        Blk<double> m{0.0, 0.0, 0.0, 0.0};
        if (yi >= 0) {
            const double2 y = __ldg(P.y_gb + yi);
            const double c = a.Uc[i], s = a.Us[i], ir = a.Ire[i], ii = a.Iim[i];
            m = jac_block<double>(p == q, y.x, y.y, a.Vre[i], a.Vim[i], a.Uc[j], a.Us[j],
                                  a.Vm[j], a.Vm[i], c * ir + s * ii, s * ir - c * ii);
        }
        stb(fac, e, pad_pv(m, p == q, ntype<QL>(P, a, i), ntype<QL>(P, a, j)));
    }
}

// ---------------------------------------------------------------- block LU
// Gathers (one row of a triangular sweep, or the Schur updates of one target block) run
// on one thread; their indices and operands are loaded kBatch at a time before any
// arithmetic, so the loads of a gather overlap instead of forming one long chain (four
// FP32 blocks, or two FP64 blocks to stay within the register budget).  The summation
// order depends only on the plan, so results do not depend on blockDim.
template <typename FT>
constexpr int kBatch = sizeof(FT) == 4 ? 4 : 2;

// Sum of the Schur contributions L(i,k) U(k,j) of one target over its list entries
// c, c + stride, ... < c1 (kBatch pairs at a time).
template <typename FT>
__device__ __forceinline__ Blk<FT> schur_gather(const DevPlan& P, const FT* fac, int c, int c1,
                                                int stride) {
    Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
    constexpr int NB = kBatch<FT>;
    for (; c < c1; c += NB * stride) {
        int2 lu[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k)
            lu[k] = (c + k * stride < c1) ? __ldg(P.sch + c + k * stride) : make_int2(-1, -1);
        Blk<FT> xl[NB], yu[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (lu[k].x >= 0) {
                xl[k] = ldb(fac, lu[k].x);
                yu[k] = ldb(fac, lu[k].y);
            } else {
                xl[k] = yu[k] = Blk<FT>{FT(0), FT(0), FT(0), FT(0)};
            }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            acc.a += xl[k].a * yu[k].a + xl[k].b * yu[k].c;
            acc.b += xl[k].a * yu[k].b + xl[k].b * yu[k].d;
            acc.c += xl[k].c * yu[k].a + xl[k].d * yu[k].c;
            acc.d += xl[k].c * yu[k].b + xl[k].d * yu[k].d;
        }
    }
    return acc;
}

// Two targets' gathers interleaved (A over ca..ea, B over cb..eb), half a batch of each
// per round so that both chains of loads are in flight at once.  Each target still sums
// its pairs in order from zero, as schur_gather does (the zero blocks of a short round
// add +0, which leaves every partial sum unchanged).
template <typename FT>
__device__ __forceinline__ void schur_gather2(const DevPlan& P, const FT* fac, int ca, int ea,
                                              int cb, int eb, Blk<FT>& A, Blk<FT>& B) {
    A = Blk<FT>{FT(0), FT(0), FT(0), FT(0)};
    B = A;
    constexpr int NB = kBatch<FT> / 2 > 0 ? kBatch<FT> / 2 : 1;
    for (; ca < ea || cb < eb; ca += NB, cb += NB) {
        int2 la[NB], lb[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            la[k] = (ca + k < ea) ? __ldg(P.sch + ca + k) : make_int2(-1, -1);
            lb[k] = (cb + k < eb) ? __ldg(P.sch + cb + k) : make_int2(-1, -1);
        }
        Blk<FT> xa[NB], ya[NB], xb[NB], yb[NB];
        const Blk<FT> z{FT(0), FT(0), FT(0), FT(0)};
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            xa[k] = la[k].x >= 0 ? ldb(fac, la[k].x) : z;
            ya[k] = la[k].x >= 0 ? ldb(fac, la[k].y) : z;
            xb[k] = lb[k].x >= 0 ? ldb(fac, lb[k].x) : z;
            yb[k] = lb[k].x >= 0 ? ldb(fac, lb[k].y) : z;
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            A.a += xa[k].a * ya[k].a + xa[k].b * ya[k].c;
            A.b += xa[k].a * ya[k].b + xa[k].b * ya[k].d;
            A.c += xa[k].c * ya[k].a + xa[k].d * ya[k].c;
            A.d += xa[k].c * ya[k].b + xa[k].d * ya[k].d;
            B.a += xb[k].a * yb[k].a + xb[k].b * yb[k].c;
            B.b += xb[k].a * yb[k].b + xb[k].b * yb[k].d;
            B.c += xb[k].c * yb[k].a + xb[k].d * yb[k].c;
            B.d += xb[k].c * yb[k].b + xb[k].d * yb[k].d;
        }
    }
}

template <typename T>
__device__ __forceinline__ Blk<T> sub_blk(Blk<T> m, Blk<T> s) {
    return {m.a - s.a, m.b - s.b, m.c - s.c, m.d - s.d};
}

// The plan's top region: its trailing elimination levels hold a few rows each, so a level
// step there is mostly the latency of its chain of index and operand loads and of its
// barrier.  Its blocks are staged in shared memory (T, in the plan's local numbering) and
// its pivots are taken one at a time, in pivot order, with the level schedule's own
// steps -- L column scaling by the pivot's inverse, Schur updates, the pivot replaced by
// its inverse -- by at most kTopThreads threads.  Every target block receives one update
// per pivot, in pivot order, so the result does not depend on the number of threads.
template <typename FT>
struct TopArena {
    FT* T;   // the region's blocks
    FT* ts;  // the region rows' part of the solve vector
    int* I;  // the plan's staged lists: piv | lc_ptr | lc | tr_ptr | fwk | fw | bwk | bw, then
             // for the adjoint ftk | ft | btk | bt
};

// The region's arena at byte offset `off` of the kernel's dynamic shared memory (every
// extern __shared__ array starts at that one base), addressed from the shared-memory
// symbol itself so that its loads and stores are shared-memory instructions.
template <typename FT>
__device__ __forceinline__ TopArena<FT> top_arena(const DevPlan& P, size_t off) {
    extern __shared__ __align__(16) unsigned char pf_dyn_smem[];
    unsigned char* a = pf_dyn_smem + off;
    return {reinterpret_cast<FT*>(a),
            reinterpret_cast<FT*>(a + top_ts_off(P.top_nblk, (int)sizeof(FT))),
            reinterpret_cast<int*>(a + top_ints_off(P.top_nblk, P.top_R, (int)sizeof(FT)))};
}

constexpr size_t kNoTop = ~size_t(0);  // no region arena (level sweeps over every level)
constexpr int kTopThreads = 1024;  // threads of a CTA that factor the region
constexpr int kTopPrefetch = 2;    // Schur triples per thread loaded one pivot ahead

// Barrier of the region's factoring threads: the group's warp, or named barrier 1 over the
// first nt threads of the CTA (the others wait at the group barrier that follows).
template <bool W>
__device__ __forceinline__ void top_bar(int nt) {
    if (W)
        __syncwarp();
    else
        asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
}

// The region's pivots on one scenario's arena A, by threads t = 0 .. nt - 1 (each calls it,
// `bar` is their barrier); bk is set if a pivot was singular.
//
// FP32: one barrier per pivot.  Each Schur triple of pivot k scales its L block on the fly,
// L(i,k) = A(i,k) P_k^-1 (the same product the stored L block gets), and the stores of
// column k's L blocks and of the pivot inverse are deferred to pivot k + 1's round, when
// no thread reads those blocks any more (pivot k + 1 reads column k + 1 and row k + 1
// only, and its targets lie beyond both); every thread forms the pivot inverse.
// FP64: two barriers per pivot, as in the level schedule (L column scaling, then the
// Schur triples): a 2x2 inverse formed by every thread, and the scaling repeated in
// every triple, would add instructions on this GPU's narrow FP64 pipe, so only the
// threads that scale an L block (and thread 0) form the inverse.
template <typename FT, typename Bar>
__device__ __forceinline__ void top_factor(const DevPlan& P, const TopArena<FT>& A, int t, int nt,
                                           Bar bar, int& bk) {
    const int R = P.top_R;
    FT* T = A.T;
    const int* piv = A.I;
    const int* lcp = piv + R;
    const int* lc = lcp + R + 1;
    const int* trp = lc + P.top_nl;
    constexpr int PF = kTopPrefetch;
    const int2 idle = make_int2(-1, 0);
    int2 nx[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) {
        const int c = trp[0] + t + j * nt;
        nx[j] = c < trp[1] ? __ldg(P.top_tr + c) : idle;
    }
    Blk<FT> dprev{FT(0), FT(0), FT(0), FT(0)};
    if constexpr (sizeof(FT) == 8) {
        for (int k = 0; k < R; ++k) {
            int2 cur[PF];
#pragma unroll
            for (int j = 0; j < PF; ++j) cur[j] = nx[j];
            if (k + 1 < R) {
                const int d0 = trp[k + 1], d1 = trp[k + 2];
#pragma unroll
                for (int j = 0; j < PF; ++j) {
                    const int c = d0 + t + j * nt;
                    nx[j] = c < d1 ? __ldg(P.top_tr + c) : idle;
                }
            }
            const int l0 = lcp[k], l1 = lcp[k + 1];
            Blk<FT> d = dprev;
            if (t == 0 || l0 + t < l1) d = inv2(ldb(T, piv[k]), &bk);
            for (int c = l0 + t; c < l1; c += nt) {  // L(i, k) <- A(i, k) A(k, k)^-1
                const int li = lc[c] & 0xffff;
                stb(T, li, mul(ldb(T, li), d));
            }
            bar();
            if (t == 0) stb(T, piv[k], d);  // no triple of this pivot reads the pivot block
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                if (cur[j].x >= 0) {
                    const unsigned lu = (unsigned)cur[j].y;
                    const Blk<FT> x = ldb(T, (int)(lu & 0xffffu)), y = ldb(T, (int)(lu >> 16));
                    Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
                    acc.a += x.a * y.a + x.b * y.c;
                    acc.b += x.a * y.b + x.b * y.d;
                    acc.c += x.c * y.a + x.d * y.c;
                    acc.d += x.c * y.b + x.d * y.d;
                    stb(T, cur[j].x, sub_blk(ldb(T, cur[j].x), acc));
                }
            }
            for (int c = trp[k] + t + PF * nt; c < trp[k + 1]; c += nt) {
                const int2 tr = __ldg(P.top_tr + c);
                const unsigned lu = (unsigned)tr.y;
                const Blk<FT> x = ldb(T, (int)(lu & 0xffffu)), y = ldb(T, (int)(lu >> 16));
                Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
                acc.a += x.a * y.a + x.b * y.c;
                acc.b += x.a * y.b + x.b * y.d;
                acc.c += x.c * y.a + x.d * y.c;
                acc.d += x.c * y.b + x.d * y.d;
                stb(T, tr.x, sub_blk(ldb(T, tr.x), acc));
            }
            bar();
        }
        return;
    }
    for (int k = 0; k < R; ++k) {
        int2 cur[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) cur[j] = nx[j];
        if (k + 1 < R) {  // the next pivot's first triples: plan data, loaded ahead
            const int d0 = trp[k + 1], d1 = trp[k + 2];
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                const int c = d0 + t + j * nt;
                nx[j] = c < d1 ? __ldg(P.top_tr + c) : idle;
            }
        }
        const Blk<FT> d = inv2(ldb(T, piv[k]), &bk);
        if (k > 0) {  // deferred: column k - 1's L blocks and its pivot inverse
            for (int c = lcp[k - 1] + t; c < lcp[k]; c += nt) {
                const int li = lc[c] & 0xffff;
                stb(T, li, mul(ldb(T, li), dprev));
            }
            if (t == 0) stb(T, piv[k - 1], dprev);
        }
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            if (cur[j].x >= 0) {
                const unsigned lu = (unsigned)cur[j].y;
                const Blk<FT> x = mul(ldb(T, (int)(lu & 0xffffu)), d);
                const Blk<FT> y = ldb(T, (int)(lu >> 16));
                Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
                acc.a += x.a * y.a + x.b * y.c;
                acc.b += x.a * y.b + x.b * y.d;
                acc.c += x.c * y.a + x.d * y.c;
                acc.d += x.c * y.b + x.d * y.d;
                stb(T, cur[j].x, sub_blk(ldb(T, cur[j].x), acc));
            }
        }
        for (int c = trp[k] + t + PF * nt; c < trp[k + 1]; c += nt) {
            const int2 tr = __ldg(P.top_tr + c);
            const unsigned lu = (unsigned)tr.y;
            const Blk<FT> x = mul(ldb(T, (int)(lu & 0xffffu)), d), y = ldb(T, (int)(lu >> 16));
            Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
            acc.a += x.a * y.a + x.b * y.c;
            acc.b += x.a * y.b + x.b * y.d;
            acc.c += x.c * y.a + x.d * y.c;
            acc.d += x.c * y.b + x.d * y.d;
            stb(T, tr.x, sub_blk(ldb(T, tr.x), acc));
        }
        dprev = d;
        bar();
    }
    if (t == 0) stb(T, piv[R - 1], dprev);  // the last pivot has no L blocks below it
}

// Factors the region in the arena at `arena` (shared memory) after the levels below it;
// with `wb` the factored blocks are also written back into fac (for sweeps or an adjoint
// that read the factor there).  Sets *bad if a pivot was singular.
template <typename FT, bool W>
__device__ void top_lu(const DevPlan& P, FT* fac, size_t arena, int* bad, bool wb) {
    const int nb = P.top_nblk;
    const TopArena<FT> A = top_arena<FT>(P, arena);
    for (int k = GTID; k < P.top_nints_fwd; k += GSZ) A.I[k] = __ldg(P.top_ints + k);
    for (int r = GTID; r < nb; r += GSZ) stb(A.T, r, ldb(fac, __ldg(P.top_map + r)));
    gsync<W>();
    const int nt = W ? 32 : min(GSZ, kTopThreads);
    if (GTID < nt) {
        int bk = 0;
        top_factor<FT>(P, A, GTID, nt, [nt] { top_bar<W>(nt); }, bk);
        if (GTID == 0) *bad |= bk;
    }
    gsync<W>();
    if (wb) {
        for (int r = GTID; r < nb; r += GSZ) stb(fac, __ldg(P.top_map + r), ldb(A.T, r));
        gsync<W>();
    }
}

// Right-looking, one elimination-tree level at a time.  Phase A scales the L columns of
// the level's pivots; phase B gathers every Schur update of the level into its target
// block (no two threads write the same block) and replaces the level's pivot blocks by
// their inverses.  (A variant with one barrier per level, recomputing L(i,k) inside each
// Schur update, measured slower: the extra 2x2 inverse per update costs more than the
// barrier it saves.)  The plan's top region, if any, is factored by top_lu in `top`
// (shared memory; written back into fac with `wb`), or with top == kNoTop by the level
// schedule like the rest.  Returns nonzero if a pivot was singular.
template <typename FT, bool W>
__device__ int phase_lu(const DevPlan& P, FT* fac, int* s_bad, size_t top, bool wb) {
    int bad = 0;
    if (!W && threadIdx.x == 0) *s_bad = 0;
    const bool rg = P.top_R > 0 && top != kNoTop;  // kNoTop: every level by the schedule
    const int n_sparse = rg ? P.top_l0 : P.n_levels;
    for (int l = 0; l < n_sparse; ++l) {
        // FP32 factor: two items per thread and round, so that two chains of loads are in
        // flight (within a level the pivots read, the L blocks scaled and the Schur
        // targets written are disjoint sets of blocks).  The FP64 factor keeps one: its
        // block arithmetic is bound by the FP64 pipe, and the pairing measured slower.
        constexpr int IPT = sizeof(FT) == 4 ? 2 : 1;
        const int a0 = __ldg(P.la_ptr + l), a1 = __ldg(P.la_ptr + l + 1);
        for (int c = a0 + GTID; c < a1; c += IPT * GSZ) {
            const int2 ld = __ldg(P.la + c);
            int dummy = 0;
            if constexpr (IPT == 2) {
                const bool two = c + GSZ < a1;
                const int2 ld2 = two ? __ldg(P.la + c + GSZ) : ld;
                const Blk<FT> m1 = ldb(fac, ld.x), q1 = ldb(fac, ld.y);
                const Blk<FT> m2 = ldb(fac, ld2.x), q2 = ldb(fac, ld2.y);
                stb(fac, ld.x, mul(m1, inv2(q1, &dummy)));
                if (two) stb(fac, ld2.x, mul(m2, inv2(q2, &dummy)));
            } else {
                stb(fac, ld.x, mul(ldb(fac, ld.x), inv2(ldb(fac, ld.y), &dummy)));
            }
        }
        gsync<W>();
        const int t0 = __ldg(P.sch_tptr + l), t1 = __ldg(P.sch_tptr + l + 1);
        const int G = __ldg(P.lev_g + l).z;  // lanes per target (a power of two <= 32; uniform)
        if (G == 1) {  // one thread per target (IPT targets per round)
            for (int t = t0 + GTID; t < t1; t += IPT * GSZ) {
                if constexpr (IPT == 2) {
                    const int t2 = t + GSZ;
                    const bool two = t2 < t1;
                    Blk<FT> acc, acc2;
                    schur_gather2(P, fac, __ldg(P.sch_cptr + t), __ldg(P.sch_cptr + t + 1),
                                  two ? __ldg(P.sch_cptr + t2) : 0,
                                  two ? __ldg(P.sch_cptr + t2 + 1) : 0, acc, acc2);
                    const int tg = __ldg(P.sch_tgt + t);
                    const int tg2 = two ? __ldg(P.sch_tgt + t2) : tg;
                    const Blk<FT> o1 = ldb(fac, tg), o2 = ldb(fac, tg2);
                    stb(fac, tg, sub_blk(o1, acc));
                    if (two) stb(fac, tg2, sub_blk(o2, acc2));
                } else {
                    const Blk<FT> acc = schur_gather(P, fac, __ldg(P.sch_cptr + t),
                                                     __ldg(P.sch_cptr + t + 1), 1);
                    const int tg = __ldg(P.sch_tgt + t);
                    stb(fac, tg, sub_blk(ldb(fac, tg), acc));
                }
            }
        } else {  // G lanes per target; every lane runs the same rounds
            const int sub = GTID & (G - 1), nrg = GSZ / G;
            for (int tb = t0; tb < t1; tb += nrg) {
                const int t = tb + GTID / G;
                const bool act = t < t1;
                Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
                if (act) acc = schur_gather(P, fac, __ldg(P.sch_cptr + t) + sub, __ldg(P.sch_cptr + t + 1), G);
                for (int o = G >> 1; o; o >>= 1) {  // butterfly over the target's lanes
                    acc.a += __shfl_xor_sync(0xffffffffu, acc.a, o);
                    acc.b += __shfl_xor_sync(0xffffffffu, acc.b, o);
                    acc.c += __shfl_xor_sync(0xffffffffu, acc.c, o);
                    acc.d += __shfl_xor_sync(0xffffffffu, acc.d, o);
                }
                if (act && sub == 0) {
                    const int tg = __ldg(P.sch_tgt + t);
                    stb(fac, tg, sub_blk(ldb(fac, tg), acc));
                }
            }
        }
        const int r1 = __ldg(P.lev_ptr + l + 1);
        for (int p = __ldg(P.lev_ptr + l) + GTID; p < r1; p += IPT * GSZ) {
            const int dk = __ldg(P.lu_diag + p);
            if constexpr (IPT == 2) {
                const bool two = p + GSZ < r1;
                const int dk2 = two ? __ldg(P.lu_diag + p + GSZ) : dk;
                const Blk<FT> d1 = ldb(fac, dk), d2 = ldb(fac, dk2);
                stb(fac, dk, inv2(d1, &bad));
                if (two) stb(fac, dk2, inv2(d2, &bad));
            } else {
                stb(fac, dk, inv2(ldb(fac, dk), &bad));
            }
        }
        gsync<W>();
    }
    if (rg) top_lu<FT, W>(P, fac, top, &bad, wb);
    if (W) return __any_sync(0xffffffffu, bad);
    if (bad) *s_bad = 1;
    gsync<W>();
    return *s_bad;
}

// One level of a block triangular sweep: x_p <- op(x_p - sum_e M_e x_q(e)) for the rows p
// of the level, where the gathered entries e of row p are the L part (lower sweeps) or
// the U part (upper sweeps) of row p in the L+U pattern.  TRANS sweeps read the block at
// the mirrored position, transposed (row p of U^T / L^T).  The stored pivot inverse (or
// its transpose) is applied by the upper sweep of LU and by the first sweep of (LU)^T.
// The gathered sum of one row over its entries e0 + first, e0 + first + stride, ... < e1
// (kBatch at a time): s0, s1 += M_e x_q(e) (or M_e^T x_q(e) for the transposed sweeps).
template <typename FT, bool TRANS>
__device__ __forceinline__ void row_gather(const DevPlan& P, const FT* fac, const FT* x, int e,
                                           int e1, int stride, FT& s0, FT& s1) {
    constexpr int NB = kBatch<FT>;
    for (; e < e1; e += NB * stride) {
        int q[NB], pos[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int ek = e + k * stride;
            const bool ok = ek < e1;
            q[k] = ok ? __ldg(P.lu_col + ek) : -1;
            pos[k] = ok ? (TRANS ? __ldg(P.lu_mirror + ek) : ek) : 0;
        }
        Blk<FT> m[NB];
        FT y0[NB], y1[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (q[k] >= 0) {
                m[k] = ldb(fac, pos[k]);
                y0[k] = x[2 * q[k]];
                y1[k] = x[2 * q[k] + 1];
            } else {
                m[k] = Blk<FT>{FT(0), FT(0), FT(0), FT(0)};
                y0[k] = y1[k] = FT(0);
            }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (TRANS) {
                s0 += m[k].a * y0[k] + m[k].c * y1[k];
                s1 += m[k].b * y0[k] + m[k].d * y1[k];
            } else {
                s0 += m[k].a * y0[k] + m[k].b * y1[k];
                s1 += m[k].c * y0[k] + m[k].d * y1[k];
            }
        }
    }
}

// x_p <- op(x_p - s) with the row's pivot (inverted) for the sweeps that divide.
template <typename FT, bool UPPER, bool TRANS>
__device__ __forceinline__ void row_finish(const FT* fac, FT* x, int p, int dg, FT s0, FT s1) {
    constexpr bool DIAG = UPPER != TRANS;
    const FT x0 = x[2 * p] - s0, x1 = x[2 * p + 1] - s1;
    if (DIAG) {
        const Blk<FT> d = ldb(fac, dg);
        if (TRANS) {
            x[2 * p] = d.a * x0 + d.c * x1;
            x[2 * p + 1] = d.b * x0 + d.d * x1;
        } else {
            x[2 * p] = d.a * x0 + d.b * x1;
            x[2 * p + 1] = d.c * x0 + d.d * x1;
        }
    } else {
        x[2 * p] = x0;
        x[2 * p + 1] = x1;
    }
}

template <typename FT, bool UPPER, bool TRANS, bool W>
__device__ __forceinline__ void sweep_level(const DevPlan& P, const FT* fac, FT* x, int l) {
    const int r0 = __ldg(P.lev_ptr + l), r1 = __ldg(P.lev_ptr + l + 1);
    const int4 lg = __ldg(P.lev_g + l);
    const int G = UPPER ? lg.y : lg.x;  // lanes per row (a power of two <= 32; uniform)
    if (G == 1) {  // one thread per row
        for (int p = r0 + GTID; p < r1; p += GSZ) {
            const int dg = __ldg(P.lu_diag + p);
            FT s0 = FT(0), s1 = FT(0);
            row_gather<FT, TRANS>(P, fac, x, UPPER ? dg + 1 : __ldg(P.lu_ptr + p),
                                  UPPER ? __ldg(P.lu_ptr + p + 1) : dg, 1, s0, s1);
            row_finish<FT, UPPER, TRANS>(fac, x, p, dg, s0, s1);
        }
        return;
    }
    // G lanes per row; every lane runs the same rounds (the shuffles need whole warps)
    const int sub = GTID & (G - 1), nrg = GSZ / G;
    for (int pb = r0; pb < r1; pb += nrg) {
        const int p = pb + GTID / G;
        const bool act = p < r1;
        const int dg = act ? __ldg(P.lu_diag + p) : 0;
        FT s0 = FT(0), s1 = FT(0);
        if (act)
            row_gather<FT, TRANS>(P, fac, x, (UPPER ? dg + 1 : __ldg(P.lu_ptr + p)) + sub,
                                  UPPER ? __ldg(P.lu_ptr + p + 1) : dg, G, s0, s1);
        for (int o = G >> 1; o; o >>= 1) {  // butterfly over the row's lanes: a fixed order
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (act && sub == 0) row_finish<FT, UPPER, TRANS>(fac, x, p, dg, s0, s1);
    }
}

// x_q of one register slot (q uniform over the warp).
template <typename FT>
__device__ __forceinline__ FT top_slot(const FT (&v)[kTopSlots], int q) {
    FT r = v[0];
#pragma unroll
    for (int j = 1; j < kTopSlots; ++j) r = q == j ? v[j] : r;
    return r;
}

// v0[q], v1[q] -= M (x0, x1) for this lane's slot q (q < 0: no entry), without branches
// (the other slots subtract zero, which leaves every value unchanged).
template <typename FT>
__device__ __forceinline__ void top_upd(FT (&v0)[kTopSlots], FT (&v1)[kTopSlots], int q,
                                        const Blk<FT>& m, FT x0, FT x1) {
    const FT d0 = m.a * x0 + m.b * x1, d1 = m.c * x0 + m.d * x1;
#pragma unroll
    for (int j = 0; j < kTopSlots; ++j) {
        v0[j] -= q == j ? d0 : FT(0);
        v1[j] -= q == j ? d1 : FT(0);
    }
}

// The region's forward and backward sweeps by one warp, on the region rows' part of the
// solve vector held in registers: lane l owns rows l, l + 32, ... (slot q = row / 32).
// The plan lists the sweeps as rounds of one entry per lane.  A forward round of column
// k: x_k (final) is broadcast by its owner lane and every lane updates its row i > k with
// L(i,k) x_k.  A backward round of column k: its first round forms x_k <- P_k^-1 x_k (the
// owner keeps it in the row's slot), every round updates rows i < k with U(i,k) x_k.
// Each row receives its updates in column order.  No round branches: an empty entry
// (-1) reads block 0 into no slot, and the rounds' loads depend on the plan only, so
// several rounds' loads are in flight together.  Reads ts (the rows after their part
// left of the region), hands row i's solution to out(i, x0, x1).
template <typename FT, typename Out>
__device__ __forceinline__ void top_sweeps(const DevPlan& P, const TopArena<FT>& A, int lane,
                                           const FT* ts, Out out) {
    const int R = P.top_R;
    const int* piv = A.I;
    const int* fwk = piv + R + (R + 1) + P.top_nl + (R + 1);
    const int* fw = fwk + P.top_nfw;
    const int* bwk = fw + 32 * P.top_nfw;
    const int* bw = bwk + P.top_nbw;
    const FT* T = A.T;
    FT v0[kTopSlots], v1[kTopSlots];
#pragma unroll
    for (int j = 0; j < kTopSlots; ++j) {
        const int i = j * 32 + lane;
        v0[j] = i < R ? ts[2 * i] : FT(0);
        v1[j] = i < R ? ts[2 * i + 1] : FT(0);
    }
#pragma unroll 4
    for (int u = 0; u < P.top_nfw; ++u) {
        const int k = fwk[u], e = fw[u * 32 + lane];
        const Blk<FT> m = ldb(T, max(e, 0) & 0xffff);
        const FT x0 = __shfl_sync(0xffffffffu, top_slot(v0, k >> 5), k & 31);
        const FT x1 = __shfl_sync(0xffffffffu, top_slot(v1, k >> 5), k & 31);
        top_upd(v0, v1, e >= 0 ? e >> 16 : -1, m, x0, x1);
    }
#pragma unroll 4
    for (int u = 0; u < P.top_nbw; ++u) {
        const int kf = bwk[u], k = kf >> 1, e = bw[u * 32 + lane];
        const Blk<FT> m = ldb(T, max(e, 0) & 0xffff);
        const Blk<FT> d = ldb(T, piv[k]);
        const FT y0 = __shfl_sync(0xffffffffu, top_slot(v0, k >> 5), k & 31);
        const FT y1 = __shfl_sync(0xffffffffu, top_slot(v1, k >> 5), k & 31);
        const bool first = (kf & 1) != 0;
        const FT x0 = first ? d.a * y0 + d.b * y1 : y0;
        const FT x1 = first ? d.c * y0 + d.d * y1 : y1;
        const bool own = first && (k & 31) == lane;  // the owner keeps x_k in the row's slot
#pragma unroll
        for (int j = 0; j < kTopSlots; ++j) {
            v0[j] = own && (k >> 5) == j ? x0 : v0[j];
            v1[j] = own && (k >> 5) == j ? x1 : v1[j];
        }
        top_upd(v0, v1, e >= 0 ? e >> 16 : -1, m, x0, x1);
    }
#pragma unroll
    for (int j = 0; j < kTopSlots; ++j) {
        const int i = j * 32 + lane;
        if (i < R) out(i, v0[j], v1[j]);
    }
}

// The sweeps over the top region (after the levels below it have been swept forward, so
// the x of every row left of the region is final): first every region row's part left of
// the region (one gather over all region rows, top_g lanes per row) into the region's copy
// of x in shared memory, then the region's columns one at a time by one warp (top_sweeps),
// which writes the region's x back.
template <typename FT, bool W>
__device__ void top_solve(const DevPlan& P, const FT* fac, FT* x, size_t arena) {
    const int p0 = P.top_p0, G = P.top_g;
    const TopArena<FT> A = top_arena<FT>(P, arena);
    if (G == 1) {
        for (int p = p0 + GTID; p < P.n; p += GSZ) {
            FT s0 = FT(0), s1 = FT(0);
            row_gather<FT, false>(P, fac, x, __ldg(P.lu_ptr + p), __ldg(P.top_split + p - p0), 1,
                                  s0, s1);
            A.ts[2 * (p - p0)] = x[2 * p] - s0;
            A.ts[2 * (p - p0) + 1] = x[2 * p + 1] - s1;
        }
    } else {  // G lanes per row; every lane runs the same rounds (the shuffles need whole warps)
        const int sub = GTID & (G - 1), nrg = GSZ / G;
        for (int pb = p0; pb < P.n; pb += nrg) {
            const int p = pb + GTID / G;
            const bool act = p < P.n;
            FT s0 = FT(0), s1 = FT(0);
            if (act)
                row_gather<FT, false>(P, fac, x, __ldg(P.lu_ptr + p) + sub,
                                      __ldg(P.top_split + p - p0), G, s0, s1);
            for (int o = G >> 1; o; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (act && sub == 0) {
                A.ts[2 * (p - p0)] = x[2 * p] - s0;
                A.ts[2 * (p - p0) + 1] = x[2 * p + 1] - s1;
            }
        }
    }
    gsync<W>();
    if (GTID < 32)
        top_sweeps<FT>(P, A, GTID, A.ts, [x, p0](int i, FT x0, FT x1) {
            x[2 * (p0 + i)] = x0;
            x[2 * (p0 + i) + 1] = x1;
        });
    gsync<W>();
}

// The region's transposed sweeps, (L U)^T x = b (the adjoint's solve), by one warp with
// the region rows' x in registers as in top_sweeps.  U^T forward, ascending columns j:
// the column's first round forms x_j <- P_j^-T x_j (the owner keeps it), every round
// updates rows k > j with U(j,k)^T x_j.  L^T backward, descending columns i: rows k < i
// with L(i,k)^T x_i.  Reads ts, hands row i's solution to out(i, x0, x1).
template <typename FT, typename Out>
__device__ __forceinline__ void top_sweeps_t(const DevPlan& P, const TopArena<FT>& A, int lane,
                                             const FT* ts, Out out) {
    const int R = P.top_R;
    const int* piv = A.I;
    const int* ftk = A.I + P.top_nints_fwd;
    const int* ft = ftk + P.top_nft;
    const int* btk = ft + 32 * P.top_nft;
    const int* bt = btk + P.top_nbt;
    const FT* T = A.T;
    FT v0[kTopSlots], v1[kTopSlots];
#pragma unroll
    for (int j = 0; j < kTopSlots; ++j) {
        const int i = j * 32 + lane;
        v0[j] = i < R ? ts[2 * i] : FT(0);
        v1[j] = i < R ? ts[2 * i + 1] : FT(0);
    }
#pragma unroll 4
    for (int u = 0; u < P.top_nft; ++u) {
        const int kf = ftk[u], k = kf >> 1, e = ft[u * 32 + lane];
        const Blk<FT> m = ldb(T, max(e, 0) & 0xffff);
        const Blk<FT> d = ldb(T, piv[k]);
        const FT y0 = __shfl_sync(0xffffffffu, top_slot(v0, k >> 5), k & 31);
        const FT y1 = __shfl_sync(0xffffffffu, top_slot(v1, k >> 5), k & 31);
        const bool first = (kf & 1) != 0;
        const FT x0 = first ? d.a * y0 + d.c * y1 : y0;
        const FT x1 = first ? d.b * y0 + d.d * y1 : y1;
        const bool own = first && (k & 31) == lane;
#pragma unroll
        for (int j = 0; j < kTopSlots; ++j) {
            v0[j] = own && (k >> 5) == j ? x0 : v0[j];
            v1[j] = own && (k >> 5) == j ? x1 : v1[j];
        }
        top_upd(v0, v1, e >= 0 ? e >> 16 : -1, Blk<FT>{m.a, m.c, m.b, m.d}, x0, x1);
    }
#pragma unroll 4
    for (int u = 0; u < P.top_nbt; ++u) {
        const int k = btk[u], e = bt[u * 32 + lane];
        const Blk<FT> m = ldb(T, max(e, 0) & 0xffff);
        const FT x0 = __shfl_sync(0xffffffffu, top_slot(v0, k >> 5), k & 31);
        const FT x1 = __shfl_sync(0xffffffffu, top_slot(v1, k >> 5), k & 31);
        top_upd(v0, v1, e >= 0 ? e >> 16 : -1, Blk<FT>{m.a, m.c, m.b, m.d}, x0, x1);
    }
#pragma unroll
    for (int j = 0; j < kTopSlots; ++j) {
        const int i = j * 32 + lane;
        if (i < R) out(i, v0[j], v1[j]);
    }
}

// The transposed sweeps over the top region (after the U^T levels below it): each region
// row's part left of the region (the mirrors of its L part, transposed; top_g lanes per
// row) into the region's copy of x, then top_sweeps_t by one warp.  The region's blocks
// and all its lists must be staged (top_stage).
template <typename FT, bool W>
__device__ void top_solve_t(const DevPlan& P, const FT* fac, FT* x, size_t arena) {
    const int p0 = P.top_p0, G = P.top_g;
    const TopArena<FT> A = top_arena<FT>(P, arena);
    const int sub = GTID & (G - 1), nrg = GSZ / G;
    for (int pb = p0; pb < P.n; pb += nrg) {  // every lane runs the same rounds
        const int p = pb + GTID / G;
        const bool act = p < P.n;
        FT s0 = FT(0), s1 = FT(0);
        if (act)
            row_gather<FT, true>(P, fac, x, __ldg(P.lu_ptr + p) + sub, __ldg(P.top_split + p - p0),
                                 G, s0, s1);
        for (int o = G >> 1; o; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (act && sub == 0) {
            A.ts[2 * (p - p0)] = x[2 * p] - s0;
            A.ts[2 * (p - p0) + 1] = x[2 * p + 1] - s1;
        }
    }
    gsync<W>();
    if (GTID < 32)
        top_sweeps_t<FT>(P, A, GTID, A.ts, [x, p0](int i, FT x0, FT x1) {
            x[2 * (p0 + i)] = x0;
            x[2 * (p0 + i) + 1] = x1;
        });
    gsync<W>();
}

// Stages the region's factored blocks (from fac) and all its lists, for the transposed
// sweeps.
template <typename FT, bool W>
__device__ void top_stage(const DevPlan& P, const FT* fac, size_t arena) {
    const TopArena<FT> A = top_arena<FT>(P, arena);
    for (int k = GTID; k < P.top_nints; k += GSZ) A.I[k] = __ldg(P.top_ints + k);
    for (int r = GTID; r < P.top_nblk; r += GSZ) stb(A.T, r, ldb(fac, __ldg(P.top_map + r)));
    gsync<W>();
}

// x <- (LU)^{-1} x in place (x holds 2 values per pivot): L y = x by ascending levels,
// then U x = y by descending levels.  With `top` (the top region as phase_lu left it in
// shared memory) the region's levels are swept there, one column at a time.
template <typename FT, bool W>
__device__ void phase_solve(const DevPlan& P, const FT* fac, FT* x, size_t top = kNoTop) {
    const bool dt = top != kNoTop && P.top_R > 0;
    const int nl = dt ? P.top_l0 : P.n_levels;
    for (int l = 0; l < nl; ++l) {
        sweep_level<FT, false, false, W>(P, fac, x, l);
        gsync<W>();
    }
    if (dt) top_solve<FT, W>(P, fac, x, top);
    for (int l = nl - 1; l >= 0; --l) {
        sweep_level<FT, true, false, W>(P, fac, x, l);
        gsync<W>();
    }
}

// x <- (LU)^{-T} x: U^T y = x by ascending levels (row p of U^T = mirrored L-part
// positions of row p), then L^T x = y by descending levels (mirrored U-part positions).
// With `top` (the region staged there by top_stage) the region's levels are swept there.
template <typename FT, bool W>
__device__ void phase_solve_t(const DevPlan& P, const FT* fac, FT* x, size_t top = kNoTop) {
    const bool dt = top != kNoTop && P.top_R > 0;
    const int nl = dt ? P.top_l0 : P.n_levels;
    for (int l = 0; l < nl; ++l) {
        sweep_level<FT, false, true, W>(P, fac, x, l);
        gsync<W>();
    }
    if (dt) top_solve_t<FT, W>(P, fac, x, top);
    for (int l = nl - 1; l >= 0; --l) {
        sweep_level<FT, true, true, W>(P, fac, x, l);
        gsync<W>();
    }
}

// r = -F1 - J1 dz with J1 dz = -[Re dS; Im dS] linearised through Ybus (FP64):
// dV_i = u_i dVm_i + j V_i dtheta_i, dS_i = dV_i conj(I_i) + V_i conj(sum_k Y_ik dV_k).
// r is rounded straight into the solve vector x (the next right-hand side).  Returns
// ||r||_inf over the true (unpadded) rows, of r as rounded into x.
template <typename FT, bool W, bool QL = false>
__device__ double phase_residual(const DevPlan& P, const Arrays& a, FT* x, double* red) {
    for (int i = GTID; i < P.n_bus; i += GSZ) {
        const int p = __ldg(P.bus2pos + i);
        double dr = 0.0, di = 0.0;
        if (p >= 0) {
            const double dth = a.dz[2 * p];
            const double dvm = (ntype<QL>(P, a, i) == 0) ? a.dz[2 * p + 1] : 0.0;
            dr = a.Uc[i] * dvm - a.Vim[i] * dth;  // dV = u dVm + j V dtheta
            di = a.Us[i] * dvm + a.Vre[i] * dth;
        }
        a.dVre[i] = dr;
        a.dVim[i] = di;
    }
    gsync<W>();
    FT lmax = FT(0);
    for (int i = GTID; i < P.n_bus; i += GSZ) {
        const int p = __ldg(P.bus2pos + i);
        if (p < 0) continue;
        double ir = 0.0, ii = 0.0;
        for (int k = __ldg(P.y_ptr + i); k < __ldg(P.y_ptr + (i + 1)); ++k) {
            const int j = __ldg(P.y_idx + k);
            const double2 y = __ldg(P.y_gb + k);
            const double vr = a.dVre[j], vi = a.dVim[j];
            ir = fma(y.x, vr, fma(-y.y, vi, ir));
            ii = fma(y.x, vi, fma(y.y, vr, ii));
        }
        const double vr = a.Vre[i], vi = a.Vim[i], Ir = a.Ire[i], Ii = a.Iim[i];
        const double dvr = a.dVre[i], dvi = a.dVim[i];
        // r = -F + dS, dS = dV conj(I) + V conj(dI), as FMA chains onto -F
        const double rP = fma(dvr, Ir, fma(dvi, Ii, fma(vr, ir, fma(vi, ii, -a.F[2 * p]))));
        const double rQ =
            (ntype<QL>(P, a, i) == 0)
                ? fma(dvi, Ir, fma(-dvr, Ii, fma(vi, ir, fma(-vr, ii, -a.F[2 * p + 1]))))
                : 0.0;
        const FT xr = FT(rP), xq = FT(rQ);
        x[2 * p] = xr;
        x[2 * p + 1] = xq;
        // the refinement's stopping norm is taken on the residual as the solve receives it
        lmax = fmax(lmax, fmax(absinf(xr), absinf(xq)));
    }
    return group_max<W>(double(lmax), red);
}

// Reactive limits at a converged point: every bus still PV whose recovered reactive
// generation qg = Q + qd lies outside [Qmin, Qmax] is a violator.  With ``apply`` the
// violators become PQ buses of this scenario with qg fixed at the violated limit.
// Returns whether there was a violator (group-wide; ends with a barrier).
template <bool W>
__device__ bool phase_q_limits(const DevPlan& P, const Arrays& a, const SolveArgs& A,
                               size_t row, bool apply, double* red) {
    double any = 0.0;
    for (int i = GTID; i < P.n_bus; i += GSZ) {
        if (a.stype[i] != 1) continue;
        const double qg = (a.Vim[i] * a.Ire[i] - a.Vre[i] * a.Iim[i]) + A.Qd[row + i];
        const double qmax = A.Qmax[row + i], qmin = A.Qmin[row + i];
        if (!(qg > qmax) && !(qg < qmin)) continue;
        any = 1.0;
        if (apply) {
            a.qfix[i] = (qg > qmax) ? qmax : qmin;
            a.stype[i] = 0;
        }
    }
    return group_max<W>(any, red) > 0.0;
}

// ---------------------------------------------------------------- forward kernel
// The Newton loop of one scenario, run by one group (see GTID / GSZ).
template <typename FT, bool VSM, bool FSM, bool XSM, bool W, bool QL = false>
__device__ __forceinline__ void solve_body(const DevPlan& P, const SolveArgs& A, const int b,
                                           unsigned char* smem, double* red, int* s_bad_ptr) {
    int& s_bad = *s_bad_ptr;
    if (b >= A.batch) return;
    const SlotLayout& L = A.L;
    const KernelSmem& K = L.fwd;
    unsigned char* slot = reinterpret_cast<unsigned char*>(A.ws) + (size_t)b * L.slot_bytes;
    // VSM / FSM are compile-time so that the compiler sees which pointers address
    // shared memory (plain shared loads instead of generic ones)
    if (W) smem += (threadIdx.x >> 5) * K.smem_bytes;  // this warp's own arena
    unsigned char* vbase = VSM ? smem : slot + L.off_vec;
    FT* fac = FSM ? reinterpret_cast<FT*>(smem + K.smem_fac_off)
                  : reinterpret_cast<FT*>(slot + L.off_fac);
    Arrays a;
    carve(vbase, P.n_bus, P.n, (int)sizeof(FT), false, &a);
    FT* x = XSM ? reinterpret_cast<FT*>(smem + K.smem_x_off) : ftptr<FT>(a.x);
    constexpr bool mixed = sizeof(FT) == 4;
    const size_t row = (size_t)b * P.n_bus;
    if (QL) {  // reactive limits: the scenario's own partition, starting as the network's
        a.stype = reinterpret_cast<signed char*>(slot + L.off_qlim);
        a.qfix = reinterpret_cast<double*>(slot + L.off_qlim + align_up((size_t)P.n_bus, 16));
        for (int i = GTID; i < P.n_bus; i += GSZ) {
            a.stype[i] = (signed char)__ldg(P.bus_type + i);
            a.qfix[i] = 0.0;
        }
    }

    // flat start and specified injections (Sec. II-A, Sec. IV-A)
    for (int i = GTID; i < P.n_bus; i += GSZ) {  // theta = 0: u = 1, V = Vm
        const int t = __ldg(P.bus_type + i);
        const double vm = (t == 0) ? 1.0 : A.Vset[row + i];
        a.Vm[i] = vm;
        a.Va[i] = 0.0;
        a.Uc[i] = 1.0;
        a.Us[i] = 0.0;
        a.Vre[i] = vm;
        a.Vim[i] = 0.0;
    }
    if (!W && GTID == 0) s_bad = 0;
    gsync<W>();

    int it = 0, it_round = 0, rounds = 0, status = 1;
    double norm = 0.0;
    bool factored = false;
    for (;;) {
        norm = phase_mismatch<mixed, W, QL>(P, a, A.Pd + row, A.Qd + row, A.Pg + row, red);
        if (!(norm <= 1e10)) { status = 2; break; }
        if (norm <= A.tol) {
            status = 0;
            if (!QL) break;
            // outer loop of the reactive limits: switch the violators and continue Newton
            // from this point on the new partition (max_iter steps per round)
            const bool more = rounds < A.max_rounds;
            if (!phase_q_limits<W>(P, a, A, row, more, red)) break;
            if (!more) { status = 1; break; }
            ++rounds;
            it_round = 0;
            continue;
        }
        if (it_round >= A.max_iter) { status = 1; break; }
        phase_fill<W, QL>(P, a, fac);
        gsync<W>();
        // the top region, factored by phase_lu, stays in shared memory for this step's
        // sweeps (and goes back into fac too when the factor is kept for the adjoint)
        const size_t top = (W ? (size_t)(threadIdx.x >> 5) * K.smem_bytes : 0) + K.smem_top_off;
        if (phase_lu<FT, W>(P, fac, &s_bad, top, A.keep_factors != 0)) {
            status = 3;
            factored = false;
            break;
        }
        factored = true;
        // first solve with the FT factor
        for (int k = GTID; k < 2 * P.n; k += GSZ) x[k] = FT(-a.F[k]);
        gsync<W>();
        phase_solve<FT, W>(P, fac, x, top);
        if (mixed) {
            for (int k = GTID; k < 2 * P.n; k += GSZ) a.dz[k] = double(x[k]);
            gsync<W>();
            const int sweeps = (A.ir_gate > 0.0 && norm > A.ir_gate) ? 0 : A.ir_steps;
            for (int s = 0; s < sweeps; ++s) {
                const double rmax = phase_residual<FT, W, QL>(P, a, x, red);  // ends with a barrier
                // forcing term min(ir_rtol, ||F1||): loose far from the solution, quadratic
                // near it, so the inexact Newton steps keep the quadratic convergence
                if (A.ir_rtol > 0.0 && rmax <= fmin(A.ir_rtol, norm) * norm) break;
                phase_solve<FT, W>(P, fac, x, top);
                for (int k = GTID; k < 2 * P.n; k += GSZ) a.dz[k] += double(x[k]);
                gsync<W>();
            }
        }
        // update (FP64)
        for (int p = GTID; p < P.n; p += GSZ) {
            const int i = __ldg(P.pos2bus + p);
            const double dth = mixed ? a.dz[2 * p] : double(x[2 * p]);
            const double dvm = mixed ? a.dz[2 * p + 1] : double(x[2 * p + 1]);
            update_bus(a, i, dth, dvm, ntype<QL>(P, a, i) == 0);
        }
        ++it;
        ++it_round;
        gsync<W>();
    }

    // Step 2 and outputs
    double* st = reinterpret_cast<double*>(slot + L.off_state);
    for (int i = GTID; i < P.n_bus; i += GSZ) {
        const int t = __ldg(P.bus_type + i);
        const double vr = a.Vre[i], vi = a.Vim[i], ir = a.Ire[i], ii = a.Iim[i];
        const double Pi = vr * ir + vi * ii, Qi = vi * ir - vr * ii;
        A.Vm[row + i] = a.Vm[i];
        A.Va[row + i] = a.Va[i];
        if (A.keep_factors) {  // the solution the adjoint differentiates at, with its
            st[i] = a.Vm[i];     // phasor and injected current (from the final mismatch)
            st[P.n_bus + i] = a.Va[i];
            st[2 * P.n_bus + i] = a.Uc[i];
            st[3 * P.n_bus + i] = a.Us[i];
            st[4 * P.n_bus + i] = ir;
            st[5 * P.n_bus + i] = ii;
        }
        if (A.Pg_out) A.Pg_out[row + i] = (t == 1) ? A.Pg[row + i] : (t == 2 ? Pi + A.Pd[row + i] : 0.0);
        if (A.Qg_out) A.Qg_out[row + i] = (t == 0) ? 0.0 : Qi + A.Qd[row + i];
        if (QL && A.types_out) A.types_out[row + i] = ntype<QL>(P, a, i);
    }
    if (A.keep_factors && factored && FSM) {
        FT* dst = reinterpret_cast<FT*>(slot + L.off_fac);
        const int nv = P.nnzb * 4;
        for (int k = GTID; k < nv; k += GSZ) dst[k] = fac[k];
    }
    if (GTID == 0) {
        A.status[b] = status;
        if (A.iters) A.iters[b] = it;
        if (A.fmis) A.fmis[b] = norm;
        if (QL && A.rounds_out) A.rounds_out[b] = rounds;
        int* fl = reinterpret_cast<int*>(slot + L.off_flags);
        fl[0] = status;
        fl[1] = it;
        fl[2] = (A.keep_factors && factored) ? 1 : 0;
    }
}

template <typename FT, bool VSM, bool FSM, bool XSM, bool QL = false>
__global__ void __launch_bounds__(1024) nr_solve_kernel(DevPlan P, SolveArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_bad;
    solve_body<FT, VSM, FSM, XSM, false, QL>(P, A, blockIdx.x, smem, red, &s_bad);
}

// Several scenarios per CTA, one per warp; the tighter register budget (42 per thread)
// lets more warps -- more scenarios in flight -- share an SM.
template <typename FT, bool VSM, bool FSM, bool XSM>
__global__ void __launch_bounds__(256, 6) nr_solve_warps_kernel(DevPlan P, SolveArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    int unused = 0;  // the warp groups vote instead of sharing a flag
    const int b = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    solve_body<FT, VSM, FSM, XSM, true>(P, A, b, smem, nullptr, &unused);
}

// Several networks in one persistent launch: CTAs take work items from a counter, jobs in
// the order given (the host puts the most expensive first), and run each with its own
// plan and its own form: a job in CTA form solves one scenario per item with the whole
// CTA (its factor in shared memory, or everything in the global workspace), a job in warp
// form solves one scenario per warp, blockDim / 32 of them per item.
template <typename FT>
__global__ void __launch_bounds__(512, 1) nr_solve_multi_kernel(MultiArgs M) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_bad;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(M.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();  // everyone has read s_item before it is overwritten
        if (item >= M.total) break;
        int j = 0;
        while (j + 1 < M.n_jobs && item >= M.first[j + 1]) ++j;
        const int r = item - M.first[j];
        const KernelSmem& K = M.args[j].L.fwd;
        if (M.warp_form[j]) {
            const int b = r * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
            int unused = 0;
            if (K.vec_in_smem)
                solve_body<FT, true, true, false, true>(M.plans[j], M.args[j], b, smem, nullptr, &unused);
            else if (K.x_in_smem)
                solve_body<FT, false, false, true, true>(M.plans[j], M.args[j], b, smem, nullptr, &unused);
            else
                solve_body<FT, false, false, false, true>(M.plans[j], M.args[j], b, smem, nullptr, &unused);
        } else if (K.fac_in_smem) {
            if (K.x_in_smem)
                solve_body<FT, false, true, true, false>(M.plans[j], M.args[j], r, smem, red, &s_bad);
            else
                solve_body<FT, false, true, false, false>(M.plans[j], M.args[j], r, smem, red, &s_bad);
        } else if (K.x_in_smem) {
            solve_body<FT, false, false, true, false>(M.plans[j], M.args[j], r, smem, red, &s_bad);
        } else {
            solve_body<FT, false, false, false, false>(M.plans[j], M.args[j], r, smem, red, &s_bad);
        }
        __syncthreads();  // the next item reuses the shared arrays
    }
}

// ---------------------------------------------------------------- adjoint kernel
// Sec. II-B.2 at the converged state: v_bar2 = -J2^T c, g_z1, J1^T lambda = g_z1,
// dL/dx = g_x - [lambda_G; J3^T lambda]; loads through dF1/dpd = dF1/dqd = -1.
// All Jacobian-transpose products are taken matrix-free through Ybus^T (phase_jvt);
// the transposed solve uses the stored factor of the last Newton step and refines
// with the FP64 residual of J1 at the solution.
template <typename FT, bool VSM, bool FSM, bool QL = false>
__global__ void __launch_bounds__(1024) adjoint_kernel(DevPlan P, AdjArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_bad;
    const int b = blockIdx.x;
    if (b >= A.batch) return;
    const SlotLayout& L = A.L;
    const KernelSmem& K = L.adj;
    unsigned char* slot = reinterpret_cast<unsigned char*>(A.ws) + (size_t)b * L.slot_bytes;
    unsigned char* vbase = VSM ? smem : slot + L.off_vec;
    FT* gfac = reinterpret_cast<FT*>(slot + L.off_fac);
    FT* fac = FSM ? reinterpret_cast<FT*>(smem + K.smem_fac_off) : gfac;
    Arrays a;
    carve(vbase, P.n_bus, P.n, (int)sizeof(FT), true, &a);
    if (QL) {  // the scenario's final partition under reactive limits (left by the solve)
        a.stype = reinterpret_cast<signed char*>(slot + L.off_qlim);
        a.qfix = reinterpret_cast<double*>(slot + L.off_qlim + align_up((size_t)P.n_bus, 16));
    }
    FT* x = ftptr<FT>(a.x);
    const size_t row = (size_t)b * P.n_bus;
    const int* fl = reinterpret_cast<const int*>(slot + L.off_flags);
    const int fwd_status = fl[0];
    const int has_factor = fl[2];

    if (fwd_status != 0) {
        for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
            A.dPd[row + i] = 0.0;
            A.dQd[row + i] = 0.0;
            A.dPg_in[row + i] = 0.0;
            A.dVset[row + i] = 0.0;
            if (QL) A.dQmin[row + i] = A.dQmax[row + i] = 0.0;
        }
        if (threadIdx.x == 0 && A.adj_status) A.adj_status[b] = fwd_status;
        return;
    }
    // the solution z* with u = e^{j theta} and I = Y V as the forward's final mismatch
    // evaluated them (no FP64 sincos or SpMV here)
    const double* st = reinterpret_cast<const double*>(slot + L.off_state);
    for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
        const double vm = st[i], c = st[2 * P.n_bus + i], s = st[3 * P.n_bus + i];
        a.Vm[i] = vm;
        a.Va[i] = st[P.n_bus + i];
        a.Uc[i] = c;
        a.Us[i] = s;
        a.Vre[i] = vm * c;
        a.Vim[i] = vm * s;
        a.Ire[i] = st[4 * P.n_bus + i];
        a.Iim[i] = st[5 * P.n_bus + i];
    }
    if (threadIdx.x == 0) s_bad = 0;
    // Step-2 weights: c_P on R (dL/dpg_R), c_Q on B\D (dL/dqg; under reactive limits the
    // final B\D: a switched bus's qg is its limit, not a recovered output)
    for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
        const int t = ntype<QL>(P, a, i);
        a.Psp[i] = (t == 2 && A.dPg) ? A.dPg[row + i] : 0.0;
        a.Qsp[i] = (t != 0 && A.dQg) ? A.dQg[row + i] : 0.0;
    }
    gsync<false>();
    phase_jvt<false>(P, a);  // v_bar2 = -J2^T c = (d[P_R; Q_{B\D}]/dv)^T c
    gsync<false>();
    unsigned long long kg = 0;
    for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
        const double gvm = A.dVm[row + i] + a.w0[i];
        const double gva = A.dVa[row + i] + a.w1[i];
        a.gV[i] = gvm;
        const int p = __ldg(P.bus2pos + i);
        if (p >= 0) {
            a.F[2 * p] = gva;                                   // theta component of g_z1
            a.F[2 * p + 1] = (ntype<QL>(P, a, i) == 0) ? gvm : 0.0;  // Vm component (PQ only)
            kg = max(kg, max(abs_key(gva), abs_key(a.F[2 * p + 1])));
        }
    }
    const double gnorm = group_max<false>(key_to_norm(kg), red);

    // stage the stored factor
    bool have = has_factor != 0;
    if (have && FSM) {
        const int nv = P.nnzb * 4;
        for (int k = threadIdx.x; k < nv; k += blockDim.x) fac[k] = gfac[k];
        gsync<false>();
    }
    int astat = 0;
    bool refactored = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (!have) {  // refactor at z*: the FP32 fill copies first
            if (sizeof(FT) == 4) {
                for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x)
                    store_bus_f32(a, i, a.Ire[i], a.Iim[i]);
                gsync<false>();
            }
            phase_fill<false, QL>(P, a, fac);
            gsync<false>();
            if (phase_lu<FT, false>(P, fac, &s_bad, A.top_t ? K.smem_top_off : kNoTop, true)) {
                astat = 3;
                break;
            }
            have = true;
            refactored = true;
        }
        const size_t tt = (P.top_R && A.top_t) ? K.smem_top_off : kNoTop;
        if (tt != kNoTop) top_stage<FT, false>(P, fac, tt);  // the factored region
        for (int k = threadIdx.x; k < 2 * P.n; k += blockDim.x) x[k] = FT(a.F[k]);
        gsync<false>();
        phase_solve_t<FT, false>(P, fac, x, tt);
        for (int k = threadIdx.x; k < 2 * P.n; k += blockDim.x) a.dz[k] = double(x[k]);
        gsync<false>();
        bool conv = false;
        for (int s = 0;; ++s) {
            // m1 = lambda on the F1 rows; r = g_z1 - J1^T lambda = g_z1 + (Jv^T m1)[z1]
            for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
                const int p = __ldg(P.bus2pos + i);
                a.Psp[i] = (p >= 0) ? a.dz[2 * p] : 0.0;
                a.Qsp[i] = (p >= 0 && ntype<QL>(P, a, i) == 0) ? a.dz[2 * p + 1] : 0.0;
            }
            gsync<false>();
            phase_jvt<false>(P, a);
            gsync<false>();
            unsigned long long kr = 0;
            for (int p = threadIdx.x; p < P.n; p += blockDim.x) {
                const int i = __ldg(P.pos2bus + p);
                const double r0 = a.F[2 * p] + a.w1[i];
                const double r1 = (ntype<QL>(P, a, i) == 0) ? a.F[2 * p + 1] + a.w0[i] : 0.0;
                a.r[2 * p] = r0;
                a.r[2 * p + 1] = r1;
                kr = max(kr, max(abs_key(r0), abs_key(r1)));
            }
            const double rmax = group_max<false>(key_to_norm(kr), red);
            if (rmax <= A.ir_rtol * gnorm) { conv = true; break; }
            if (s >= A.ir_max || !(rmax <= 1e300)) break;
            for (int k = threadIdx.x; k < 2 * P.n; k += blockDim.x) x[k] = FT(a.r[k]);
            gsync<false>();
            phase_solve_t<FT, false>(P, fac, x, tt);
            for (int k = threadIdx.x; k < 2 * P.n; k += blockDim.x) a.dz[k] += double(x[k]);
            gsync<false>();
        }
        if (conv) break;
        if (refactored) { astat = 1; break; }
        have = false;  // stale factor did not converge: refactor at the solution
    }
    // gradients; w0 holds (Jv^T m1)_Vm for the final lambda
    for (int i = threadIdx.x; i < P.n_bus; i += blockDim.x) {
        const int t = ntype<QL>(P, a, i);        // the partition of the solution
        const int t0 = __ldg(P.bus_type + i);    // the network's (pg is an input on its G)
        const int p = __ldg(P.bus2pos + i);
        const double lP = (p >= 0) ? a.dz[2 * p] : 0.0;
        const double lQ = (p >= 0 && t == 0) ? a.dz[2 * p + 1] : 0.0;
        const double cP = A.dPg ? A.dPg[row + i] : 0.0;
        const double cQ = A.dQg ? A.dQg[row + i] : 0.0;
        A.dPd[row + i] = (t == 2) ? cP : lP;
        A.dQd[row + i] = (t == 0) ? lQ : cQ;
        A.dPg_in[row + i] = (t0 == 1) ? cP - lP : 0.0;
        A.dVset[row + i] = (t != 0) ? a.gV[i] + a.w0[i] : 0.0;
        if (QL) {  // a switched bus: Qg_out = qlim, and qlim enters F1 like minus a load
            const double dq = (t0 == 1 && t == 0) ? cQ - lQ : 0.0;
            const bool at_max = a.qfix[i] == A.Qmax[row + i];
            A.dQmax[row + i] = at_max ? dq : 0.0;
            A.dQmin[row + i] = at_max ? 0.0 : dq;
        }
    }
    if (threadIdx.x == 0 && A.adj_status) A.adj_status[b] = astat;
}

// ---------------------------------------------------------------- launch helpers
// Raises a kernel's dynamic shared-memory limit (once per device and kernel).
cudaError_t ensure_smem_limit(const void* k, size_t bytes);

template <typename KernelT, typename ArgT>
cudaError_t launch_one(KernelT k, const DevPlan& P, const ArgT& A, const KernelSmem& K,
                       int threads, cudaStream_t s) {
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(k), K.smem_bytes);
    if (e != cudaSuccess) return e;
    k<<<A.batch, threads, K.smem_bytes, s>>>(P, A);
    return cudaGetLastError();
}

}  // namespace pf
