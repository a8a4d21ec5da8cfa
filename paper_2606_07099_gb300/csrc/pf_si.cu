// pf_si.cu -- the Newton-Raphson solve on scenario-interleaved packs, one thread-block
// cluster (or one CTA) per pack (placement PF_PLACE_INTERLEAVED; sm_103a).
//
// The per-scenario form (pf_body.cuh) gives each scenario one CTA.  On large networks
// (thousands of buses) that leaves every elimination-level step of the factorisation
// and of the triangular sweeps as a chain of dependent index -> operand loads run by one
// CTA, with each thread's 16-byte loads scattered over its own scenario's workspace.
// Here S scenarios (a pack) are solved together in the layout the paper's block-diagonal
// execution uses for its batch (Sec. III-A): item k of scenario s of the pack sits at
// [k][s], so a slot of S lanes works on one item (a bus, a factor block, a Schur target,
// a row of a sweep) for all S scenarios at once: the plan's indices are loaded once per
// slot and every operand load is S consecutive elements.  A cluster of C CTAs shares the
// pack: each phase splits its items over all C x (threads / S) slots, and the phases
// (and the levels inside the factorisation and the sweeps) are separated by hardware
// cluster barriers.  Data written by one CTA and read by another goes through L2 only
// (ld.global.cg / st.global.cg): the barrier's release/acquire orders it, and no SM keeps
// a stale L1 copy.  With C = 1 a pack is one CTA: CTA barriers and plain (L1-cached)
// loads, the shape that suits small networks with many scenarios.
//
// The arithmetic is that of the per-scenario form: FP64 mismatch, update, residual and
// convergence test; the factor and the sweeps in FT (float: the mixed form, refined by
// FP64 residuals; double: the all-FP64 form); static 2x2 pivots on the plan's ordering;
// every gather summed in an order fixed by the plan (long sweep rows split over at most
// kGMax lane groups, combined in order), so results do not depend on S, the cluster
// size or the threads per CTA.  Per-scenario decisions (convergence, divergence,
// iteration limit, refinement) are taken from cluster-wide per-scenario maxima that every
// CTA reads after the same barrier, so all CTAs of a cluster take the same control path.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "pf_body.cuh"
#include "pf_launch.h"

namespace pf {
namespace si {

constexpr int kGMax = 16;  // lane groups a long sweep row is split over, at most

template <typename FT>
struct V2;
template <>
struct V2<float> {
    using T = float2;
};
template <>
struct V2<double> {
    using T = double2;
};

__device__ __forceinline__ void cluster_sync() {
    __syncwarp();  // the .aligned barrier wants every lane of the warp at the same instruction
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// The barrier between the phases of a pack: the cluster's, or the CTA's when one CTA runs
// the pack (its global writes are then ordered for its own threads by __syncthreads).
template <bool CL>
__device__ __forceinline__ void pack_sync() {
    if (CL) cluster_sync();
    else __syncthreads();
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_ncta() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_index() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// Loads and stores of pack data: through L2 only (cache-global) when several CTAs share
// the pack, plain (L1-cached) when one CTA runs it -- its own writes are then visible to
// its own later loads after a CTA barrier.
template <bool CL, typename T>
__device__ __forceinline__ T ldm(const T* p) {
    if constexpr (CL) return __ldcg(p);
    else return *p;
}
template <bool CL, typename T>
__device__ __forceinline__ void stm(T* p, T v) {
    if constexpr (CL) __stcg(p, v);
    else *p = v;
}

// One pack's arrays (global memory).
template <typename FT>
struct Pack {
    FT* fac;
    double2 *V, *I, *U, *M, *SP, *DV, *F, *DZ;
    float4 *FA, *FB;
    typename V2<FT>::T* X;
    unsigned long long* red;  // 3 x 32 reduction slots (rotating)
    unsigned int* sing;       // 32 singular flags
};

// factor block e of lane s: float4 [e][S]; FP64 as two double2 rows [e][2][S]
template <int S, bool CL>
__device__ __forceinline__ Blk<float> ldf(const float* fac, int e, int s) {
    const float4 v = ldm<CL>(reinterpret_cast<const float4*>(fac) + ((size_t)e * S + s));
    return {v.x, v.y, v.z, v.w};
}
template <int S, bool CL>
__device__ __forceinline__ Blk<double> ldf(const double* fac, int e, int s) {
    const double2* p = reinterpret_cast<const double2*>(fac) + ((size_t)e * 2 * S + s);
    const double2 u = ldm<CL>(p), w = ldm<CL>(p + S);
    return {u.x, u.y, w.x, w.y};
}
template <int S, bool CL>
__device__ __forceinline__ void stf(float* fac, int e, int s, Blk<float> v) {
    stm<CL>(reinterpret_cast<float4*>(fac) + ((size_t)e * S + s), make_float4(v.a, v.b, v.c, v.d));
}
template <int S, bool CL>
__device__ __forceinline__ void stf(double* fac, int e, int s, Blk<double> v) {
    double2* p = reinterpret_cast<double2*>(fac) + ((size_t)e * 2 * S + s);
    stm<CL>(p, make_double2(v.a, v.b));
    stm<CL>(p + S, make_double2(v.c, v.d));
}
__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

// Cluster-wide maximum, per scenario lane, of a non-negative value given as its ordered
// integer key (abs_key); every thread of every CTA receives its lane's maximum.  Ends
// with a cluster barrier, so it also orders everything written before it.  The three
// global slots rotate: slot r is read right after round r's barrier, and CTA 0 clears
// slot r + 1 during round r, after the barrier that ended every read of its last use.
template <int S, bool CL>
__device__ double cluster_max(unsigned long long k, unsigned long long* red, int& round,
                              unsigned long long* s_red, unsigned rank) {
#pragma unroll
    for (int o = S; o < 32; o <<= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
    if (threadIdx.x < S) s_red[threadIdx.x] = 0ull;
    __syncthreads();
    if ((threadIdx.x & 31u) < (unsigned)S) atomicMax(&s_red[threadIdx.x & (S - 1)], k);
    __syncthreads();
    unsigned long long* slot = red + (round % 3) * 32;
    if (threadIdx.x < S) {
        atomicMax(slot + threadIdx.x, s_red[threadIdx.x]);
        if (rank == 0) atomicExch(red + ((round + 1) % 3) * 32 + threadIdx.x, 0ull);
    }
    pack_sync<CL>();
    const unsigned long long r = __ldcg(slot + (threadIdx.x & (S - 1)));  // set by atomics: L2
    ++round;
    return key_to_norm(r);
}

// The pack's lanes that satisfy `pred` (the same mask in every warp of the cluster, since
// every lane index s appears in every warp and all lanes of one s agree).
template <int S>
__device__ __forceinline__ unsigned lanes_where(bool pred) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    return S == 32 ? m : (m & ((1u << S) - 1u));
}

// ---------------------------------------------------------------- per-bus phases
// I = Y V, S = V conj(I), F1 = spec - S at the pivot positions; with FP32 copies for the
// FP32 fill.  Returns the lane's max |F1| as an ordered key.
template <typename FT, int S, bool CL>
__device__ unsigned long long si_mismatch(const DevPlan& P, const Pack<FT>& k, int gs, int TS,
                                          int s, bool go) {
    unsigned long long kmax = 0;
    if (!go) return kmax;
    for (int i = gs; i < P.n_bus; i += TS) {
        double ir = 0.0, ii = 0.0;
        const int k1 = __ldg(P.y_ptr + i + 1);
        for (int q = __ldg(P.y_ptr + i); q < k1; ++q) {
            const int j = __ldg(P.y_idx + q);
            const double2 y = __ldg(P.y_gb + q);
            const double2 v = ldm<CL>(k.V + ((size_t)j * S + s));
            ir = fma(y.x, v.x, fma(-y.y, v.y, ir));
            ii = fma(y.x, v.y, fma(y.y, v.x, ii));
        }
        const size_t o = (size_t)i * S + s;
        stm<CL>(k.I + o, make_double2(ir, ii));
        if constexpr (sizeof(FT) == 4) {  // FP32 copies of V, u, Vm and u conj(I) for the FP32 fill
            const double2 u = ldm<CL>(k.U + o), m = ldm<CL>(k.M + o);
            const float c = float(u.x), sn = float(u.y), vm = float(m.x);
            const float fir = float(ir), fii = float(ii);
            stm<CL>(k.FA + o, make_float4(vm * c, vm * sn, c, sn));
            stm<CL>(k.FB + o, make_float4(vm, fmaf(c, fir, sn * fii), fmaf(sn, fir, -(c * fii)), 0.f));
        }
        const int p = __ldg(P.bus2pos + i);
        if (p >= 0) {
            const double2 v = ldm<CL>(k.V + o), sp = ldm<CL>(k.SP + o);
            const double fP = fma(-v.x, ir, fma(-v.y, ii, sp.x));
            const double fQ = (__ldg(P.bus_type + i) == 0) ? fma(-v.y, ir, fma(v.x, ii, sp.y)) : 0.0;
            stm<CL>(k.F + ((size_t)p * S + s), make_double2(fP, fQ));
            kmax = max(kmax, max(abs_key(fP), abs_key(fQ)));
        }
    }
    return kmax;
}

// The Jacobian fill (Alg. 1 values, the element formulas of jac_block) into the factor,
// and x = -F1 for the first solve.
template <int S, bool CL>
__device__ void si_fill(const DevPlan& P, const Pack<float>& k, int gs, int TS, int s, bool go) {
    if (!go) return;
    // two blocks per slot and round, both blocks' loads before either store (the stores to
    // the factor could otherwise alias the next block's bus reads for the compiler)
    auto block = [&](int e) {
        const int p = __ldg(P.lu_row + e), q = __ldg(P.lu_col + e), yi = __ldg(P.fill_y + e);
        const int i = __ldg(P.pos2bus + p), j = __ldg(P.pos2bus + q);
        Blk<float> m{0.f, 0.f, 0.f, 0.f};
        if (yi >= 0) {
            const float2 y = __ldg(P.y_gb32 + yi);
            const float4 ai = ldm<CL>(k.FA + ((size_t)i * S + s)), bi = ldm<CL>(k.FB + ((size_t)i * S + s));
            const float4 aj = ldm<CL>(k.FA + ((size_t)j * S + s)), bj = ldm<CL>(k.FB + ((size_t)j * S + s));
            m = jac_block<float>(p == q, y.x, y.y, ai.x, ai.y, aj.z, aj.w, bj.x, bi.x, bi.y, bi.z);
        }
        return pad_pv(m, p == q, __ldg(P.bus_type + i), __ldg(P.bus_type + j));
    };
    for (int e = gs; e < P.nnzb; e += 2 * TS) {
        const int e2 = e + TS;
        const bool two = e2 < P.nnzb;
        const Blk<float> m1 = block(e), m2 = block(two ? e2 : e);
        stf<S, CL>(k.fac, e, s, m1);
        if (two) stf<S, CL>(k.fac, e2, s, m2);
    }
    for (int p = gs; p < P.n; p += TS) {
        const double2 f = ldm<CL>(k.F + ((size_t)p * S + s));
        stm<CL>(k.X + ((size_t)p * S + s), make_float2(float(-f.x), float(-f.y)));
    }
}

template <int S, bool CL>
__device__ void si_fill(const DevPlan& P, const Pack<double>& k, int gs, int TS, int s, bool go) {
    if (!go) return;
    for (int e = gs; e < P.nnzb; e += TS) {
        const int p = __ldg(P.lu_row + e), q = __ldg(P.lu_col + e), yi = __ldg(P.fill_y + e);
        const int i = __ldg(P.pos2bus + p), j = __ldg(P.pos2bus + q);
        Blk<double> m{0.0, 0.0, 0.0, 0.0};
        if (yi >= 0) {
            const double2 y = __ldg(P.y_gb + yi);
            const size_t oi = (size_t)i * S + s, oj = (size_t)j * S + s;
            const double2 ui = ldm<CL>(k.U + oi), Ii = ldm<CL>(k.I + oi), vi = ldm<CL>(k.V + oi);
            const double2 mi = ldm<CL>(k.M + oi), uj = ldm<CL>(k.U + oj), mj = ldm<CL>(k.M + oj);
            m = jac_block<double>(p == q, y.x, y.y, vi.x, vi.y, uj.x, uj.y, mj.x, mi.x,
                                  ui.x * Ii.x + ui.y * Ii.y, ui.y * Ii.x - ui.x * Ii.y);
        }
        stf<S, CL>(k.fac, e, s, pad_pv(m, p == q, __ldg(P.bus_type + i), __ldg(P.bus_type + j)));
    }
    for (int p = gs; p < P.n; p += TS) {
        const double2 f = ldm<CL>(k.F + ((size_t)p * S + s));
        stm<CL>(k.X + ((size_t)p * S + s), make_double2(-f.x, -f.y));
    }
}

// ---------------------------------------------------------------- factorisation
// Sum of the Schur contributions L(i,k) U(k,j) of one target over its pairs c0 .. c1,
// kBatch pairs at a time, in pair order (as schur_gather does per scenario).
template <typename FT, int S, bool CL>
__device__ __forceinline__ Blk<FT> si_schur(const DevPlan& P, const FT* fac, int c, int c1, int s) {
    constexpr int NB = kBatch<FT>;
    Blk<FT> acc{FT(0), FT(0), FT(0), FT(0)};
    for (; c < c1; c += NB) {
        int2 lu[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) lu[q] = (c + q < c1) ? __ldg(P.sch + c + q) : make_int2(-1, -1);
        Blk<FT> xl[NB], yu[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            if (lu[q].x >= 0) {
                xl[q] = ldf<S, CL>(fac, lu[q].x, s);
                yu[q] = ldf<S, CL>(fac, lu[q].y, s);
            } else {
                xl[q] = yu[q] = Blk<FT>{FT(0), FT(0), FT(0), FT(0)};
            }
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            acc.a += xl[q].a * yu[q].a + xl[q].b * yu[q].c;
            acc.b += xl[q].a * yu[q].b + xl[q].b * yu[q].d;
            acc.c += xl[q].c * yu[q].a + xl[q].d * yu[q].c;
            acc.d += xl[q].c * yu[q].b + xl[q].d * yu[q].d;
        }
    }
    return acc;
}

// Two targets' sums interleaved (A over ca..ea, B over cb..eb), half a batch of each per
// round so that both chains of loads are in flight at once; each target still sums its
// pairs in order from zero, as si_schur does.
template <typename FT, int S, bool CL>
__device__ __forceinline__ void si_schur2(const DevPlan& P, const FT* fac, int ca, int ea, int cb,
                                          int eb, int s, Blk<FT>& A, Blk<FT>& B) {
    constexpr int NB = kBatch<FT> / 2 > 0 ? kBatch<FT> / 2 : 1;
    const Blk<FT> z{FT(0), FT(0), FT(0), FT(0)};
    A = z;
    B = z;
    for (; ca < ea || cb < eb; ca += NB, cb += NB) {
        int2 la[NB], lb[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            la[q] = (ca + q < ea) ? __ldg(P.sch + ca + q) : make_int2(-1, -1);
            lb[q] = (cb + q < eb) ? __ldg(P.sch + cb + q) : make_int2(-1, -1);
        }
        Blk<FT> xa[NB], ya[NB], xb[NB], yb[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            xa[q] = la[q].x >= 0 ? ldf<S, CL>(fac, la[q].x, s) : z;
            ya[q] = la[q].x >= 0 ? ldf<S, CL>(fac, la[q].y, s) : z;
            xb[q] = lb[q].x >= 0 ? ldf<S, CL>(fac, lb[q].x, s) : z;
            yb[q] = lb[q].x >= 0 ? ldf<S, CL>(fac, lb[q].y, s) : z;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            A.a += xa[q].a * ya[q].a + xa[q].b * ya[q].c;
            A.b += xa[q].a * ya[q].b + xa[q].b * ya[q].d;
            A.c += xa[q].c * ya[q].a + xa[q].d * ya[q].c;
            A.d += xa[q].c * ya[q].b + xa[q].d * ya[q].d;
            B.a += xb[q].a * yb[q].a + xb[q].b * yb[q].c;
            B.b += xb[q].a * yb[q].b + xb[q].b * yb[q].d;
            B.c += xb[q].c * yb[q].a + xb[q].d * yb[q].c;
            B.d += xb[q].c * yb[q].b + xb[q].d * yb[q].d;
        }
    }
}

// One elimination level: the L-column scalings (phase A), a pack barrier, then the
// level's Schur targets and pivot inversions (phase B), and a pack barrier.  With the
// FP32 factor each slot takes two items per round (their loads in flight together;
// within a level the pivots read, the L blocks scaled and the targets written are
// disjoint).  A singular pivot raises the lane's flag in the pack's `sing` array.
template <typename FT, int S, bool CL>
__device__ void si_lu_level(const DevPlan& P, const Pack<FT>& k, int l, int gs, int TS, int s,
                            bool go) {
    if constexpr (sizeof(FT) == 4) {
        if (go) {
            const int a1 = __ldg(P.la_ptr + l + 1);
            for (int c = __ldg(P.la_ptr + l) + gs; c < a1; c += 2 * TS) {
                const bool two = c + TS < a1;
                const int2 ld = __ldg(P.la + c), ld2 = two ? __ldg(P.la + c + TS) : ld;
                int dummy = 0;
                const Blk<FT> m1 = ldf<S, CL>(k.fac, ld.x, s), q1 = ldf<S, CL>(k.fac, ld.y, s);
                const Blk<FT> m2 = ldf<S, CL>(k.fac, ld2.x, s), q2 = ldf<S, CL>(k.fac, ld2.y, s);
                stf<S, CL>(k.fac, ld.x, s, mul(m1, inv2(q1, &dummy)));
                if (two) stf<S, CL>(k.fac, ld2.x, s, mul(m2, inv2(q2, &dummy)));
            }
        }
        pack_sync<CL>();
        if (go) {
            const int t0 = __ldg(P.sch_tptr + l), t1 = __ldg(P.sch_tptr + l + 1);
            for (int t = t0 + gs; t < t1; t += 2 * TS) {
                const int t2 = t + TS;
                const bool two = t2 < t1;
                Blk<FT> acc, acc2;
                si_schur2<FT, S, CL>(P, k.fac, __ldg(P.sch_cptr + t), __ldg(P.sch_cptr + t + 1),
                                     two ? __ldg(P.sch_cptr + t2) : 0,
                                     two ? __ldg(P.sch_cptr + t2 + 1) : 0, s, acc, acc2);
                const int tg = __ldg(P.sch_tgt + t), tg2 = two ? __ldg(P.sch_tgt + t2) : tg;
                const Blk<FT> o1 = ldf<S, CL>(k.fac, tg, s), o2 = ldf<S, CL>(k.fac, tg2, s);
                stf<S, CL>(k.fac, tg, s, sub_blk(o1, acc));
                if (two) stf<S, CL>(k.fac, tg2, s, sub_blk(o2, acc2));
            }
            int bad = 0;
            const int r1 = __ldg(P.lev_ptr + l + 1);
            for (int p = __ldg(P.lev_ptr + l) + gs; p < r1; p += 2 * TS) {
                const bool two = p + TS < r1;
                const int dk = __ldg(P.lu_diag + p), dk2 = two ? __ldg(P.lu_diag + p + TS) : dk;
                const Blk<FT> d1 = ldf<S, CL>(k.fac, dk, s), d2 = ldf<S, CL>(k.fac, dk2, s);
                stf<S, CL>(k.fac, dk, s, inv2(d1, &bad));
                if (two) stf<S, CL>(k.fac, dk2, s, inv2(d2, &bad));
            }
            if (bad) atomicOr(k.sing + s, 1u);
        }
        pack_sync<CL>();
        return;
    }
    if (go) {
        const int a1 = __ldg(P.la_ptr + l + 1);
        for (int c = __ldg(P.la_ptr + l) + gs; c < a1; c += TS) {
            const int2 ld = __ldg(P.la + c);
            int dummy = 0;
            const Blk<FT> m = ldf<S, CL>(k.fac, ld.x, s), d = ldf<S, CL>(k.fac, ld.y, s);
            stf<S, CL>(k.fac, ld.x, s, mul(m, inv2(d, &dummy)));
        }
    }
    pack_sync<CL>();
    if (go) {
        const int t0 = __ldg(P.sch_tptr + l), nT = __ldg(P.sch_tptr + l + 1) - t0;
        const int r0 = __ldg(P.lev_ptr + l), nI = nT + (__ldg(P.lev_ptr + l + 1) - r0);
        int bad = 0;
        for (int u = gs; u < nI; u += TS) {
            if (u < nT) {
                const int t = t0 + u;
                const int tg = __ldg(P.sch_tgt + t);
                const Blk<FT> acc =
                    si_schur<FT, S, CL>(P, k.fac, __ldg(P.sch_cptr + t), __ldg(P.sch_cptr + t + 1), s);
                stf<S, CL>(k.fac, tg, s, sub_blk(ldf<S, CL>(k.fac, tg, s), acc));
            } else {
                const int dk = __ldg(P.lu_diag + r0 + (u - nT));
                stf<S, CL>(k.fac, dk, s, inv2(ldf<S, CL>(k.fac, dk, s), &bad));
            }
        }
        if (bad) atomicOr(k.sing + s, 1u);
    }
    pack_sync<CL>();
}

// ---------------------------------------------------------------- triangular sweeps
// Gathered sum of one row over its entries e, e + stride, ... < e1 (kBatch at a time):
// s0, s1 += M_e x_q(e).
template <typename FT, int S, bool CL>
__device__ __forceinline__ void si_row_gather(const DevPlan& P, const Pack<FT>& k, int e, int e1,
                                              int stride, int s, FT& s0, FT& s1) {
    constexpr int NB = kBatch<FT>;
    for (; e < e1; e += NB * stride) {
        int q[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) q[b] = (e + b * stride < e1) ? __ldg(P.lu_col + e + b * stride) : -1;
        Blk<FT> m[NB];
        typename V2<FT>::T y[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (q[b] >= 0) {
                m[b] = ldf<S, CL>(k.fac, e + b * stride, s);
                y[b] = ldm<CL>(k.X + ((size_t)q[b] * S + s));
            } else {
                m[b] = Blk<FT>{FT(0), FT(0), FT(0), FT(0)};
                y[b] = mk2(FT(0), FT(0));
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            s0 += m[b].a * y[b].x + m[b].b * y[b].y;
            s1 += m[b].c * y[b].x + m[b].d * y[b].y;
        }
    }
}

// x_p <- x_p - s (lower sweep) or P_p^-1 (x_p - s) (upper sweep; the stored pivot is the
// inverse).
template <typename FT, int S, bool UPPER, bool CL>
__device__ __forceinline__ void si_row_finish(const Pack<FT>& k, int p, int dg, int s, FT s0,
                                              FT s1) {
    typename V2<FT>::T* xp = k.X + ((size_t)p * S + s);
    const typename V2<FT>::T x = ldm<CL>(xp);
    const FT x0 = x.x - s0, x1 = x.y - s1;
    if (UPPER) {
        const Blk<FT> d = ldf<S, CL>(k.fac, dg, s);
        stm<CL>(xp, mk2(d.a * x0 + d.b * x1, d.c * x0 + d.d * x1));
    } else {
        stm<CL>(xp, mk2(x0, x1));
    }
}

// One level of a sweep (lower: L part of each row, ascending levels; upper: U part,
// descending).  Rows whose plan splits the gather (G > 1 lanes) are split into
// min(G, kGMax) lane groups of one CTA (row r of the level belongs to CTA r mod C); the
// groups' partial sums meet in shared memory and are added in group order.  Ends with a
// cluster barrier.
template <typename FT, int S, bool UPPER, bool CL>
__device__ void si_sweep_level(const DevPlan& P, const Pack<FT>& k, int l, int gs, int TS, int s,
                               int slot, int NS, int rank, int C, bool go,
                               typename V2<FT>::T* part) {
    const int r0 = __ldg(P.lev_ptr + l), R = __ldg(P.lev_ptr + l + 1) - r0;
    const int4 lg = __ldg(P.lev_g + l);
    const int G = min(UPPER ? lg.y : lg.x, kGMax);
    if (G == 1) {
        if (go) {
            for (int r = gs; r < R; r += TS) {
                const int p = r0 + r, dg = __ldg(P.lu_diag + p);
                FT s0 = FT(0), s1 = FT(0);
                si_row_gather<FT, S, CL>(P, k, UPPER ? dg + 1 : __ldg(P.lu_ptr + p),
                                     UPPER ? __ldg(P.lu_ptr + p + 1) : dg, 1, s, s0, s1);
                si_row_finish<FT, S, UPPER, CL>(k, p, dg, s, s0, s1);
            }
        }
    } else {
        const int Rc = R > rank ? (R - rank + C - 1) / C : 0;  // this CTA's rows
        const int total = Rc * G;
        for (int base = 0; base < total; base += NS) {  // G divides NS: no row straddles rounds
            const int li = base + slot;
            const bool act = go && li < total;
            const int lr = li / G, g = li - lr * G;
            const int p = r0 + rank + lr * C;
            FT s0 = FT(0), s1 = FT(0);
            int dg = 0;
            if (act) {
                dg = __ldg(P.lu_diag + p);
                si_row_gather<FT, S, CL>(P, k, (UPPER ? dg + 1 : __ldg(P.lu_ptr + p)) + g,
                                     UPPER ? __ldg(P.lu_ptr + p + 1) : dg, G, s, s0, s1);
            }
            part[slot * S + s] = mk2(s0, s1);
            __syncthreads();
            if (act && g == 0) {
                FT t0 = FT(0), t1 = FT(0);
                for (int h = 0; h < G; ++h) {
                    const typename V2<FT>::T v = part[(slot + h) * S + s];
                    t0 += v.x;
                    t1 += v.y;
                }
                si_row_finish<FT, S, UPPER, CL>(k, p, dg, s, t0, t1);
            }
            __syncthreads();
        }
    }
    pack_sync<CL>();
}

// ---------------------------------------------------------------- top region
// The plan's top region (see top_factor / top_sweeps): scenario s of the pack is factored
// and swept by CTA s mod C, in slot s / C of that CTA's arena, with the per-scenario
// form's steps and order.  The levels below the region go as before, over the cluster.
template <typename FT>
__device__ __forceinline__ TopArena<FT> si_top_arena(const DevPlan& P, const SiLayout& L, int j) {
    extern __shared__ __align__(16) unsigned char pf_dyn_smem[];
    unsigned char* a = pf_dyn_smem + L.smem_top_off + (size_t)j * L.top_stride;
    return {reinterpret_cast<FT*>(a),
            reinterpret_cast<FT*>(a + top_ts_off(P.top_nblk, (int)sizeof(FT))),
            reinterpret_cast<int*>(pf_dyn_smem + L.smem_top_off + (size_t)L.top_slots * L.top_stride)};
}

// Scenarios of the pack on this CTA: slot j holds scenario rank + j C.
__device__ __forceinline__ int si_top_nsc(int S, unsigned rank, unsigned C) {
    return (int)rank < S ? (S - 1 - (int)rank) / (int)C + 1 : 0;
}

// The region's factorisation for this CTA's scenarios (after the levels below it and
// their pack barrier); the caller ends it with a pack barrier.  `go` is the thread's own
// lane's flag; a slot's scenario is read from its lane.  With more scenarios than slots
// they go top_slots at a time, each chunk's factored regions written back into the pack's
// factor for the sweeps.
template <typename FT, int S, bool CL>
__device__ void si_top_lu(const DevPlan& P, const SiLayout& L, const Pack<FT>& k, unsigned rank,
                          unsigned C, bool go) {
    const int nsc = si_top_nsc(S, rank, C);
    if (nsc == 0) return;  // uniform over the CTA
    const int nb = P.top_nblk;
    const bool resident = nsc <= L.top_slots;
    int* I = si_top_arena<FT>(P, L, 0).I;
    for (int q = (int)threadIdx.x; q < P.top_nints_fwd; q += (int)blockDim.x) I[q] = __ldg(P.top_ints + q);
    for (int c0 = 0; c0 < nsc; c0 += L.top_slots) {
        const int m = min(L.top_slots, nsc - c0);  // a power of two that divides blockDim
        for (int u = (int)threadIdx.x; u < m * nb; u += (int)blockDim.x) {
            const int j = u / nb, r = u - j * nb;
            stb(si_top_arena<FT>(P, L, j).T, r,
                ldf<S, CL>(k.fac, __ldg(P.top_map + r), (int)rank + (c0 + j) * (int)C));
        }
        __syncthreads();
        const int j = (int)threadIdx.x & (m - 1), sj = (int)rank + (c0 + j) * (int)C;
        const bool gj = __shfl_sync(0xffffffffu, go, sj & 31);
        int bk = 0;
        top_factor<FT>(P, si_top_arena<FT>(P, L, j), (int)threadIdx.x / m, (int)blockDim.x / m,
                       [] { __syncthreads(); }, bk);
        if (gj && bk && (int)threadIdx.x < m) atomicOr(k.sing + sj, 1u);
        __syncthreads();
        if (!resident) {
            for (int u = (int)threadIdx.x; u < m * nb; u += (int)blockDim.x) {
                const int jj = u / nb, r = u - jj * nb;
                stf<S, CL>(k.fac, __ldg(P.top_map + r), (int)rank + (c0 + jj) * (int)C,
                           ldb(si_top_arena<FT>(P, L, jj).T, r));
            }
            __syncthreads();
        }
    }
}

// The region's sweeps for this CTA's scenarios (after the forward levels below it and
// their pack barrier): each region row's part left of the region, gathered from the
// pack's factor and solve vector (top_g lanes per row), then one warp per scenario sweeps
// the region and writes its x back into the pack's solve vector.  The caller ends it with
// a pack barrier.  Scenarios whose regions are not resident are staged again from the
// pack's factor, top_slots at a time.
template <typename FT, int S, bool CL>
__device__ void si_top_solve(const DevPlan& P, const SiLayout& L, const Pack<FT>& k, unsigned rank,
                             unsigned C, bool go) {
    const int nsc = si_top_nsc(S, rank, C);
    if (nsc == 0) return;
    const int R = P.top_R, p0 = P.top_p0, G = P.top_g, nb = P.top_nblk;
    const bool resident = nsc <= L.top_slots;
    for (int c0 = 0; c0 < nsc; c0 += L.top_slots) {
        const int m = min(L.top_slots, nsc - c0);
        if (!resident)
            for (int u = (int)threadIdx.x; u < m * nb; u += (int)blockDim.x) {
                const int j = u / nb, r = u - j * nb;
                stb(si_top_arena<FT>(P, L, j).T, r,
                    ldf<S, CL>(k.fac, __ldg(P.top_map + r), (int)rank + (c0 + j) * (int)C));
            }
        const int items = R * m * G;
        for (int ub = 0; ub < items; ub += (int)blockDim.x) {  // every lane runs the same rounds
            const int u = ub + (int)threadIdx.x;
            const bool act = u < items;
            const int g = u % G, rj = u / G, j = rj % m, r = rj / m;
            const int sj = (int)rank + (c0 + j) * (int)C;
            FT s0 = FT(0), s1 = FT(0);
            if (act)
                si_row_gather<FT, S, CL>(P, k, __ldg(P.lu_ptr + p0 + r) + g, __ldg(P.top_split + r),
                                         G, sj, s0, s1);
            for (int o = G >> 1; o; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (act && g == 0) {
                const typename V2<FT>::T xv = ldm<CL>(k.X + ((size_t)(p0 + r) * S + sj));
                FT* ts = si_top_arena<FT>(P, L, j).ts;
                ts[2 * r] = xv.x - s0;
                ts[2 * r + 1] = xv.y - s1;
            }
        }
        __syncthreads();
        const int nw = (int)blockDim.x >> 5, w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
        for (int j = w; j < m; j += nw) {
            const int sj = (int)rank + (c0 + j) * (int)C;
            const bool gj = __shfl_sync(0xffffffffu, go, sj & 31);
            if (!gj) continue;  // uniform over the warp
            const TopArena<FT> A = si_top_arena<FT>(P, L, j);
            top_sweeps<FT>(P, A, lane, A.ts, [&k, p0, sj](int i, FT x0, FT x1) {
                stm<CL>(k.X + ((size_t)(p0 + i) * S + sj), mk2(x0, x1));
            });
        }
        __syncthreads();
    }
}

template <typename FT, int S, bool CL>
__device__ void si_solve(const DevPlan& P, const SiLayout& L, const Pack<FT>& k, int gs, int TS,
                         int s, int slot, int NS, int rank, int C, bool go,
                         typename V2<FT>::T* part) {
    const int nl = P.top_R ? P.top_l0 : P.n_levels;
    for (int l = 0; l < nl; ++l)
        si_sweep_level<FT, S, false, CL>(P, k, l, gs, TS, s, slot, NS, rank, C, go, part);
    if (P.top_R) {
        si_top_solve<FT, S, CL>(P, L, k, (unsigned)rank, (unsigned)C, go);
        pack_sync<CL>();
    }
    for (int l = nl - 1; l >= 0; --l)
        si_sweep_level<FT, S, true, CL>(P, k, l, gs, TS, s, slot, NS, rank, C, go, part);
}

// ---------------------------------------------------------------- refinement (mixed)
// dz += x (dz = x on the first call), and dV = u dVm + j V dtheta for the residual.
template <int S, bool CL>
__device__ void si_accumulate(const DevPlan& P, const Pack<float>& k, int gs, int TS, int s,
                              bool go, bool first) {
    if (!go) return;
    for (int i = gs; i < P.n_bus; i += TS) {
        const int p = __ldg(P.bus2pos + i);
        double2 dv = make_double2(0.0, 0.0);
        if (p >= 0) {
            const size_t op = (size_t)p * S + s;
            const float2 xv = ldm<CL>(k.X + op);
            double2 dz = make_double2(double(xv.x), double(xv.y));
            if (!first) {
                const double2 d0 = ldm<CL>(k.DZ + op);
                dz.x += d0.x;
                dz.y += d0.y;
            }
            stm<CL>(k.DZ + op, dz);
            const size_t o = (size_t)i * S + s;
            const double dth = dz.x, dvm = (__ldg(P.bus_type + i) == 0) ? dz.y : 0.0;
            const double2 u = ldm<CL>(k.U + o), v = ldm<CL>(k.V + o);
            dv = make_double2(u.x * dvm - v.y * dth, u.y * dvm + v.x * dth);
        }
        stm<CL>(k.DV + ((size_t)i * S + s), dv);
    }
}

// r = -F1 - J1 dz (FP64, linearised through Ybus), rounded into x; returns the lane's
// max |r| (of the rounded values) as an ordered key.
template <int S, bool CL>
__device__ unsigned long long si_residual(const DevPlan& P, const Pack<float>& k, int gs, int TS,
                                          int s, bool go) {
    float lmax = 0.f;
    if (!go) return 0ull;
    for (int i = gs; i < P.n_bus; i += TS) {
        const int p = __ldg(P.bus2pos + i);
        if (p < 0) continue;
        double ir = 0.0, ii = 0.0;
        const int k1 = __ldg(P.y_ptr + i + 1);
        for (int q = __ldg(P.y_ptr + i); q < k1; ++q) {
            const int j = __ldg(P.y_idx + q);
            const double2 y = __ldg(P.y_gb + q);
            const double2 d = ldm<CL>(k.DV + ((size_t)j * S + s));
            ir = fma(y.x, d.x, fma(-y.y, d.y, ir));
            ii = fma(y.x, d.y, fma(y.y, d.x, ii));
        }
        const size_t o = (size_t)i * S + s, op = (size_t)p * S + s;
        const double2 v = ldm<CL>(k.V + o), I = ldm<CL>(k.I + o), dv = ldm<CL>(k.DV + o);
        const double2 F = ldm<CL>(k.F + op);
        const double rP = fma(dv.x, I.x, fma(dv.y, I.y, fma(v.x, ir, fma(v.y, ii, -F.x))));
        const double rQ = (__ldg(P.bus_type + i) == 0)
                              ? fma(dv.y, I.x, fma(-dv.x, I.y, fma(v.y, ir, fma(-v.x, ii, -F.y))))
                              : 0.0;
        const float xr = float(rP), xq = float(rQ);
        stm<CL>(k.X + op, make_float2(xr, xq));
        lmax = fmaxf(lmax, fmaxf(absinf(xr), absinf(xq)));
    }
    return abs_key(double(lmax));
}

// ---------------------------------------------------------------- update
template <typename FT, int S, bool CL>
__device__ void si_update(const DevPlan& P, const Pack<FT>& k, int gs, int TS, int s, bool go) {
    if (!go) return;
    for (int i = gs; i < P.n_bus; i += TS) {
        const int p = __ldg(P.bus2pos + i);
        if (p < 0) continue;
        double dth, dvm;
        if constexpr (sizeof(FT) == 4) {  // the refined step, accumulated in FP64
            const double2 dz = ldm<CL>(k.DZ + ((size_t)p * S + s));
            dth = dz.x;
            dvm = dz.y;
        } else {
            const double2 x = ldm<CL>(k.X + ((size_t)p * S + s));
            dth = x.x;
            dvm = x.y;
        }
        const size_t o = (size_t)i * S + s;
        const double2 m = ldm<CL>(k.M + o);
        const double th = m.y + dth;
        const double vm = (__ldg(P.bus_type + i) == 0) ? m.x + dvm : m.x;
        double c, sn;
        if (abs_key(dth) <= 0x3fc0000000000000ULL) {  // |dth| <= 1/8: rotate u (false for NaN)
            double rc, rs;
            small_angle_phasor(dth, &rc, &rs);
            const double2 u = ldm<CL>(k.U + o);
            c = u.x * rc - u.y * rs;
            sn = u.y * rc + u.x * rs;
        } else {
            sincos(th, &sn, &c);
        }
        stm<CL>(k.M + o, make_double2(vm, th));
        stm<CL>(k.U + o, make_double2(c, sn));
        stm<CL>(k.V + o, make_double2(vm * c, vm * sn));
    }
}

template <typename FT>
__device__ __forceinline__ Pack<FT> carve_pack(const SiArgs& A, unsigned pack) {
    const SiLayout& L = A.L;
    char* base = A.ws + (size_t)pack * L.pack_bytes;
    Pack<FT> k;
    k.fac = reinterpret_cast<FT*>(base + L.off_fac);
    k.V = reinterpret_cast<double2*>(base + L.off_V);
    k.I = reinterpret_cast<double2*>(base + L.off_I);
    k.U = reinterpret_cast<double2*>(base + L.off_U);
    k.M = reinterpret_cast<double2*>(base + L.off_M);
    k.SP = reinterpret_cast<double2*>(base + L.off_SP);
    k.DV = reinterpret_cast<double2*>(base + L.off_DV);
    k.F = reinterpret_cast<double2*>(base + L.off_F);
    k.DZ = reinterpret_cast<double2*>(base + L.off_DZ);
    k.FA = reinterpret_cast<float4*>(base + L.off_FA);
    k.FB = reinterpret_cast<float4*>(base + L.off_FB);
    k.X = reinterpret_cast<typename V2<FT>::T*>(base + L.off_X);
    k.red = reinterpret_cast<unsigned long long*>(base + L.off_ctl);
    k.sing = reinterpret_cast<unsigned int*>(base + L.off_ctl + 3 * 32 * sizeof(unsigned long long));
    return k;
}

// ---------------------------------------------------------------- the kernel
template <typename FT, int S, bool CL>
__global__ void __launch_bounds__(1024, 1) nr_solve_si_kernel(DevPlan P, SiArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_red[32];
    constexpr bool mixed = sizeof(FT) == 4;
    auto* part = reinterpret_cast<typename V2<FT>::T*>(smem);
    const int s = (int)(threadIdx.x & (S - 1)), slot = (int)(threadIdx.x / S);
    const int NS = (int)(blockDim.x / S);
    const unsigned rank = cluster_rank(), C = cluster_ncta(), pack = cluster_index();
    const int gs = (int)rank * NS + slot, TS = (int)C * NS;
    // this pack's scenarios: b0 .. b0 + nb - 1 in lanes 0 .. nb - 1
    const int b0 = (int)pack * A.q + min((int)pack, A.r), nb = A.q + ((int)pack < A.r ? 1 : 0);
    const int b = b0 + s;
    const bool valid = s < nb;
    const Pack<FT> k = carve_pack<FT>(A, pack);
    int round = 0;

    // reduction slots and singular flags start at zero
    if (rank == 0 && threadIdx.x < 3 * 32) atomicExch(k.red + threadIdx.x, 0ull);
    if (rank == 0 && threadIdx.x < 32) atomicExch(k.sing + threadIdx.x, 0u);
    // flat start (Sec. IV-A) and the specified injections, transposed into the pack: the
    // pack's input rows are read in row order (consecutive threads, consecutive buses of
    // one scenario), so that every read is coalesced -- also when the inputs are in host
    // memory and each transaction crosses the chip-to-chip link
    const int nflat = S * P.n_bus;
    for (int f = (int)(rank * blockDim.x + threadIdx.x); f < nflat; f += (int)(C * blockDim.x)) {
        const int sf = f / P.n_bus, i = f - sf * P.n_bus, bf = b0 + sf;
        const int t = __ldg(P.bus_type + i);
        double vm = 1.0, psp = 0.0, qsp = 0.0;
        if (sf < nb) {
            const size_t r = (size_t)bf * P.n_bus + i;
            if (t != 0) vm = A.Vset[r];
            psp = (t == 1 ? A.Pg[r] : 0.0) - A.Pd[r];
            qsp = -A.Qd[r];
        }
        const size_t o = (size_t)i * S + sf;
        stm<CL>(k.M + o, make_double2(vm, 0.0));
        stm<CL>(k.U + o, make_double2(1.0, 0.0));
        stm<CL>(k.V + o, make_double2(vm, 0.0));
        stm<CL>(k.SP + o, make_double2(psp, qsp));
    }
    pack_sync<CL>();

    int status = valid ? -1 : 4;  // -1: still iterating; 4: no scenario in this lane
    int it = 0;
    double norm = 0.0;
    for (;;) {
        const unsigned long long km = si_mismatch<FT, S, CL>(P, k, gs, TS, s, status < 0);
        const double nrm = cluster_max<S, CL>(km, k.red, round, s_red, rank);
        if (status < 0) {
            norm = nrm;
            if (!(norm <= 1e10)) status = 2;
            else if (norm <= A.tol) status = 0;
            else if (it >= A.max_iter) status = 1;
        }
        if (lanes_where<S>(status < 0) == 0u) break;
        const bool go = status < 0;
        si_fill<S, CL>(P, k, gs, TS, s, go);
        pack_sync<CL>();
        const int nl = P.top_R ? P.top_l0 : P.n_levels;
        for (int l = 0; l < nl; ++l) si_lu_level<FT, S, CL>(P, k, l, gs, TS, s, go);
        if (P.top_R) {
            si_top_lu<FT, S, CL>(P, A.L, k, rank, C, go);
            pack_sync<CL>();
        }
        // read after the last level's barrier, through L2 (the flags are set by atomics)
        if (go && __ldcg(k.sing + s) != 0u) status = 3;
        const bool g2 = status < 0;
        if (lanes_where<S>(g2) == 0u) break;
        si_solve<FT, S, CL>(P, A.L, k, gs, TS, s, slot, NS, (int)rank, (int)C, g2, part);
        if constexpr (mixed) {
            si_accumulate<S, CL>(P, k, gs, TS, s, g2, true);
            pack_sync<CL>();
            const int sweeps = (A.ir_gate > 0.0 && norm > A.ir_gate) ? 0 : A.ir_steps;
            bool refine = g2 && sweeps > 0;
            for (int sw = 0; lanes_where<S>(refine) != 0u; ++sw) {
                const unsigned long long kr = si_residual<S, CL>(P, k, gs, TS, s, refine);
                const double rmax = cluster_max<S, CL>(kr, k.red, round, s_red, rank);
                // forcing term min(ir_rtol, ||F1||): see the per-scenario form
                if (refine && A.ir_rtol > 0.0 && rmax <= fmin(A.ir_rtol, norm) * norm) refine = false;
                if (lanes_where<S>(refine) == 0u) break;
                si_solve<FT, S, CL>(P, A.L, k, gs, TS, s, slot, NS, (int)rank, (int)C, refine, part);
                si_accumulate<S, CL>(P, k, gs, TS, s, refine, false);
                pack_sync<CL>();
                if (sw + 1 >= sweeps) refine = false;
            }
        }
        si_update<FT, S, CL>(P, k, gs, TS, s, g2);
        pack_sync<CL>();
        if (g2) ++it;
    }

    // Step 2 (Eq. F2_completion) and outputs, from the state of each scenario's last
    // mismatch evaluation; written in row order, like the inputs were read
    for (int f = (int)(rank * blockDim.x + threadIdx.x); f < nflat; f += (int)(C * blockDim.x)) {
        const int sf = f / P.n_bus, i = f - sf * P.n_bus, bf = b0 + sf;
        if (sf >= nb) continue;
        const size_t o = (size_t)i * S + sf, r = (size_t)bf * P.n_bus + i;
        const int t = __ldg(P.bus_type + i);
        const double2 m = ldm<CL>(k.M + o), v = ldm<CL>(k.V + o), I = ldm<CL>(k.I + o);
        A.Vm[r] = m.x;
        A.Va[r] = m.y;
        if (A.Pg_out) A.Pg_out[r] = (t == 1) ? A.Pg[r] : (t == 2 ? v.x * I.x + v.y * I.y + A.Pd[r] : 0.0);
        if (A.Qg_out) A.Qg_out[r] = (t == 0) ? 0.0 : (v.y * I.x - v.x * I.y) + A.Qd[r];
    }
    if (valid && rank == 0 && slot == 0) {
        A.status[b] = status;
        if (A.iters) A.iters[b] = it;
        if (A.fmis) A.fmis[b] = norm;
    }
}

}  // namespace si

// ---------------------------------------------------------------- launch
// One CTA per pack (cluster 1) runs the single-CTA instantiation: CTA barriers, no cluster
// launch attribute.
template <typename FT, int S, bool CL>
static cudaError_t prepare() {
    static std::mutex mu;
    static std::map<int, bool> done;  // per device: the non-portable cluster size allowed
    if (!CL) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(si::nr_solve_si_kernel<FT, S, CL>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <typename FT, int S, bool CL>
static cudaLaunchConfig_t si_config(int grid, int cluster, int threads, size_t smem,
                                    cudaStream_t st, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = CL ? 1 : 0;
    return cfg;
}

template <typename FT, int S, bool CL>
static cudaError_t launch_s(const DevPlan& P, const SiArgs& A, cudaStream_t st) {
    cudaError_t e = prepare<FT, S, CL>();
    if (e != cudaSuccess) return e;
    e = ensure_smem_limit(reinterpret_cast<const void*>(si::nr_solve_si_kernel<FT, S, CL>),
                          A.L.smem_bytes);
    if (e != cudaSuccess) return e;
    const int packs = A.npacks;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = si_config<FT, S, CL>(packs * A.L.cluster, A.L.cluster,
                                                        A.L.threads, A.L.smem_bytes, st, at);
    e = cudaLaunchKernelEx(&cfg, si::nr_solve_si_kernel<FT, S, CL>, P, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename FT, int S>
static cudaError_t launch_c(const DevPlan& P, const SiArgs& A, cudaStream_t st) {
    return A.L.cluster > 1 ? launch_s<FT, S, true>(P, A, st) : launch_s<FT, S, false>(P, A, st);
}

template <typename FT>
cudaError_t launch_solve_si(const DevPlan& P, const SiArgs& A, cudaStream_t s) {
    switch (A.L.S) {
        case 2: return launch_c<FT, 2>(P, A, s);
        case 4: return launch_c<FT, 4>(P, A, s);
        case 8: return launch_c<FT, 8>(P, A, s);
        case 16: return launch_c<FT, 16>(P, A, s);
        case 32: return launch_c<FT, 32>(P, A, s);
        default: return cudaErrorInvalidValue;
    }
}

// How many of the shape's CTAs one SM holds (one CTA per pack), or how many of its
// clusters the GPU holds (clusters); 0 if the shape cannot run.
template <typename FT, int S, bool CL>
static cudaError_t resident_s(int cluster, int threads, size_t smem, int* n) {
    *n = 0;
    cudaError_t e = prepare<FT, S, CL>();
    if (e != cudaSuccess) return e;
    if (ensure_smem_limit(reinterpret_cast<const void*>(si::nr_solve_si_kernel<FT, S, CL>), smem) !=
        cudaSuccess) {
        cudaGetLastError();  // more shared memory than a CTA may have: the shape does not fit
        return cudaSuccess;
    }
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = si_config<FT, S, CL>(cluster, cluster, threads, smem, 0, at);
    if (CL) {
        e = cudaOccupancyMaxActiveClusters(n, si::nr_solve_si_kernel<FT, S, CL>, &cfg);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, si::nr_solve_si_kernel<FT, S, CL>,
                                                          threads, smem);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();  // a refused shape is an answer, not an error
        *n = 0;
    }
    return cudaSuccess;
}

template <typename FT, int S>
static cudaError_t resident_c(int cluster, int threads, size_t smem, int* n) {
    return cluster > 1 ? resident_s<FT, S, true>(cluster, threads, smem, n)
                       : resident_s<FT, S, false>(cluster, threads, smem, n);
}

template <typename FT>
cudaError_t si_resident(int S, int cluster, int threads, size_t smem, int* n) {
    *n = 0;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, size_t>, int> known;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_tuple(dev, S, cluster, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = known.find(key);
        if (it != known.end()) {
            *n = it->second;
            return cudaSuccess;
        }
    }
    switch (S) {
        case 2: e = resident_c<FT, 2>(cluster, threads, smem, n); break;
        case 4: e = resident_c<FT, 4>(cluster, threads, smem, n); break;
        case 8: e = resident_c<FT, 8>(cluster, threads, smem, n); break;
        case 16: e = resident_c<FT, 16>(cluster, threads, smem, n); break;
        case 32: e = resident_c<FT, 32>(cluster, threads, smem, n); break;
        default: return cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(mu);
        known[key] = *n;
    }
    return e;
}

template <typename FT>
cudaError_t si_shape_fits(int S, int cluster, int threads, size_t smem, bool* fits) {
    int n = 0;
    const cudaError_t e = si_resident<FT>(S, cluster, threads, smem, &n);
    *fits = n > 0;
    return e;
}

template cudaError_t launch_solve_si<float>(const DevPlan&, const SiArgs&, cudaStream_t);
template cudaError_t launch_solve_si<double>(const DevPlan&, const SiArgs&, cudaStream_t);
template cudaError_t si_shape_fits<float>(int, int, int, size_t, bool*);
template cudaError_t si_shape_fits<double>(int, int, int, size_t, bool*);
template cudaError_t si_resident<float>(int, int, int, size_t, int*);
template cudaError_t si_resident<double>(int, int, int, size_t, int*);

}  // namespace pf
