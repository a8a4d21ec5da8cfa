// Host check of the plan's top region (test helper, built and run by test_plan_top.py).
//
// Reads one network (Ybus CSR and bus types, binary), builds the plan with the given
// region options, then on a random diagonally dominant 2x2-block matrix with the plan's
// filled pattern:
//   1. factors it by a plain right-looking block LU in pivot order (the reference), and
//      again by the plan's level schedule below the region followed by the region's own
//      lists (pivots, L columns, Schur triples) on the region's local block numbering;
//   2. checks every list entry against the pattern (the block it names sits at the row
//      and column the list says);
//   3. solves L U x = b with reference sweeps, and with level sweeps below the region plus
//      the region's forward and backward rounds (one entry per lane and round, the row
//      owned by lane i mod 32, slot i / 32);
//   4. solves (L U)^T x = b (the adjoint's solve) both ways, with the region's transposed
//      rounds.
// Prints the region's size and the largest differences; exits 1 if a list entry is wrong
// or a difference exceeds 1e-12.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "pf_plan.h"

using namespace pf;

namespace {

struct B {
    double a, b, c, d;
};
B mul(B x, B y) { return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d}; }
B sub(B x, B y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
B inv(B m) {
    const double det = m.a * m.d - m.b * m.c;
    return {m.d / det, -m.b / det, -m.c / det, m.a / det};
}
void apply(const B& m, double x0, double x1, double* y) {  // y -= M x
    y[0] -= m.a * x0 + m.b * x1;
    y[1] -= m.c * x0 + m.d * x1;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 5) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int nb = 0, nnz = 0;
    if (std::fread(&nb, 4, 1, f) != 1 || std::fread(&nnz, 4, 1, f) != 1) return 2;
    std::vector<int> ptr(nb + 1), idx(nnz), bt(nb);
    std::vector<double> re(nnz), im(nnz);
    if (std::fread(ptr.data(), 4, nb + 1, f) != (size_t)nb + 1 ||
        std::fread(idx.data(), 4, nnz, f) != (size_t)nnz ||
        std::fread(re.data(), 8, nnz, f) != (size_t)nnz ||
        std::fread(im.data(), 8, nnz, f) != (size_t)nnz ||
        std::fread(bt.data(), 4, nb, f) != (size_t)nb)
        return 2;
    std::fclose(f);
    PlanParams pp;
    pp.top_rows = std::atoi(argv[2]);
    pp.top_blocks = std::atoi(argv[3]);
    pp.top_min_pivots = std::atoi(argv[4]);
    Plan P;
    if (build_plan(nb, ptr.data(), idx.data(), re.data(), im.data(), bt.data(), P, pp) != BUILD_OK)
        return 2;
    const int n = P.n, R = P.top_R, p0 = P.top_p0, nnzb = P.nnzb();
    std::printf("pivots %d levels %d region: first level %d, %d pivots, %d blocks, %d triples\n", n,
                P.n_levels, P.top_l0, R, P.top_blocks(), (int)P.top_tr_t.size());

    std::mt19937 rng(7);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::vector<B> A(nnzb);
    for (int p = 0; p < n; ++p)
        for (int e = P.lu_ptr[p]; e < P.lu_ptr[p + 1]; ++e) {
            A[e] = {U(rng), U(rng), U(rng), U(rng)};
            if (e == P.lu_diag[p]) A[e].a += 40.0, A[e].d += 40.0;
        }
    auto find = [&](int i, int j) {
        const auto b = P.lu_col.begin() + P.lu_ptr[i], e = P.lu_col.begin() + P.lu_ptr[i + 1];
        const auto it = std::lower_bound(b, e, j);
        return (it != e && *it == j) ? (int)(it - P.lu_col.begin()) : -1;
    };

    // 1a. reference: right-looking block LU in pivot order (pivots stored inverted)
    std::vector<B> X = A;
    std::vector<std::vector<int>> colL(n);
    for (int i = 0; i < n; ++i)
        for (int e = P.lu_ptr[i]; e < P.lu_diag[i]; ++e) colL[P.lu_col[e]].push_back(e);
    for (int k = 0; k < n; ++k) {
        const B d = inv(X[P.lu_diag[k]]);
        for (int e : colL[k]) X[e] = mul(X[e], d);
        for (int e : colL[k])
            for (int u = P.lu_diag[k] + 1; u < P.lu_ptr[k + 1]; ++u) {
                const int t = find(P.lu_row[e], P.lu_col[u]);
                X[t] = sub(X[t], mul(X[e], X[u]));
            }
        X[P.lu_diag[k]] = d;
    }
    // 1b. the plan: level schedule below the region, then the region's lists
    std::vector<B> Y = A;
    for (int l = 0; l < P.top_l0; ++l) {
        for (int c = P.la_ptr[l]; c < P.la_ptr[l + 1]; ++c) Y[P.la_L[c]] = mul(Y[P.la_L[c]], inv(Y[P.la_D[c]]));
        for (int t = P.sch_tptr[l]; t < P.sch_tptr[l + 1]; ++t) {
            B acc{0, 0, 0, 0};
            for (int c = P.sch_cptr[t]; c < P.sch_cptr[t + 1]; ++c) {
                const B m = mul(Y[P.sch_L[c]], Y[P.sch_U[c]]);
                acc = {acc.a + m.a, acc.b + m.b, acc.c + m.c, acc.d + m.d};
            }
            Y[P.sch_tgt[t]] = sub(Y[P.sch_tgt[t]], acc);
        }
        for (int p = P.lev_ptr[l]; p < P.lev_ptr[l + 1]; ++p) Y[P.lu_diag[p]] = inv(Y[P.lu_diag[p]]);
    }
    long long bad = 0;
    std::vector<B> T;
    const int* I = P.top_ints.data();
    const int *piv = I, *lcp = I + R, *lc = lcp + R + 1, *trp = lc + P.top_nl;
    const int *fwk = trp + R + 1, *fw = fwk + P.top_nfw, *bwk = fw + 32 * P.top_nfw,
              *bw = bwk + P.top_nbw;
    if (R > 0) {
        if ((int)(bw + 32 * P.top_nbw - I) != P.top_nints_fwd) ++bad;
        T.resize(P.top_blocks());
        for (int r = 0; r < P.top_blocks(); ++r) T[r] = Y[P.top_map[r]];
        for (int k = 0; k < R; ++k) {
            const B d = inv(T[piv[k]]);
            for (int c = lcp[k]; c < lcp[k + 1]; ++c) T[lc[c] & 0xffff] = mul(T[lc[c] & 0xffff], d);
            for (int c = trp[k]; c < trp[k + 1]; ++c) {
                const unsigned v = (unsigned)P.top_tr_lu[c];
                T[P.top_tr_t[c]] = sub(T[P.top_tr_t[c]], mul(T[v & 0xffff], T[v >> 16]));
            }
            T[piv[k]] = d;
        }
        for (int r = 0; r < P.top_blocks(); ++r) Y[P.top_map[r]] = T[r];
    }
    double dfac = 0.0;
    for (int e = 0; e < nnzb; ++e)
        dfac = std::max({dfac, std::fabs(X[e].a - Y[e].a), std::fabs(X[e].b - Y[e].b),
                         std::fabs(X[e].c - Y[e].c), std::fabs(X[e].d - Y[e].d)});

    // 2. list entries against the pattern
    auto at = [&](int r, int row, int col) {  // local block r is (row, col) of the region
        const int e = P.top_map[r];
        return P.lu_row[e] == p0 + row && P.lu_col[e] == p0 + col;
    };
    int lastk = R;
    for (int k = 0; k < R; ++k) {
        if (!at(piv[k], k, k)) ++bad;
        for (int c = lcp[k]; c < lcp[k + 1]; ++c) {  // L blocks (i, k) of the region, i > k
            const int e = P.top_map[lc[c]];
            if (P.lu_col[e] != p0 + k || P.lu_row[e] <= p0 + k) ++bad;
        }
    }
    for (int u = 0; u < P.top_nfw; ++u)
        for (int l = 0; l < 32; ++l) {
            const int v = fw[u * 32 + l];
            if (v >= 0 && !(at(v & 0xffff, (v >> 16) * 32 + l, fwk[u]) && (v >> 16) * 32 + l > fwk[u])) ++bad;
        }
    for (int u = 0; u < P.top_nbw; ++u) {
        const int k = bwk[u] >> 1;
        if ((bwk[u] & 1) && k != lastk - 1) ++bad;  // every column, descending
        if (bwk[u] & 1) lastk = k;
        for (int l = 0; l < 32; ++l) {
            const int v = bw[u * 32 + l];
            if (v >= 0 && !(at(v & 0xffff, (v >> 16) * 32 + l, k) && (v >> 16) * 32 + l < k)) ++bad;
        }
    }
    if (R > 0 && lastk != 0) ++bad;

    // 3. L U x = b: reference sweeps against level sweeps plus the region's rounds
    std::vector<double> b0(2 * n);
    for (double& v : b0) v = U(rng);
    std::vector<double> xr = b0, xs = b0;
    for (int p = 0; p < n; ++p)
        for (int e = P.lu_ptr[p]; e < P.lu_diag[p]; ++e) apply(X[e], xr[2 * P.lu_col[e]], xr[2 * P.lu_col[e] + 1], &xr[2 * p]);
    for (int p = n - 1; p >= 0; --p) {
        for (int e = P.lu_diag[p] + 1; e < P.lu_ptr[p + 1]; ++e) apply(X[e], xr[2 * P.lu_col[e]], xr[2 * P.lu_col[e] + 1], &xr[2 * p]);
        const B d = X[P.lu_diag[p]];
        const double y0 = xr[2 * p], y1 = xr[2 * p + 1];
        xr[2 * p] = d.a * y0 + d.b * y1;
        xr[2 * p + 1] = d.c * y0 + d.d * y1;
    }
    for (int p = 0; p < p0; ++p)
        for (int e = P.lu_ptr[p]; e < P.lu_diag[p]; ++e) apply(Y[e], xs[2 * P.lu_col[e]], xs[2 * P.lu_col[e] + 1], &xs[2 * p]);
    if (R > 0) {
        std::vector<double> ts(2 * R);
        for (int p = p0; p < n; ++p) {  // each region row's part left of the region
            double s[2] = {xs[2 * p], xs[2 * p + 1]};
            for (int e = P.lu_ptr[p]; e < P.top_split[p - p0]; ++e) apply(Y[e], xs[2 * P.lu_col[e]], xs[2 * P.lu_col[e] + 1], s);
            ts[2 * (p - p0)] = s[0];
            ts[2 * (p - p0) + 1] = s[1];
        }
        for (int u = 0; u < P.top_nfw; ++u) {
            const int k = fwk[u];
            const double x0 = ts[2 * k], x1 = ts[2 * k + 1];
            for (int l = 0; l < 32; ++l) {
                const int v = fw[u * 32 + l];
                if (v >= 0) apply(T[v & 0xffff], x0, x1, &ts[2 * ((v >> 16) * 32 + l)]);
            }
        }
        for (int u = 0; u < P.top_nbw; ++u) {
            const int k = bwk[u] >> 1;
            double x0 = ts[2 * k], x1 = ts[2 * k + 1];
            if (bwk[u] & 1) {
                const B d = T[piv[k]];
                const double y0 = x0, y1 = x1;
                x0 = d.a * y0 + d.b * y1;
                x1 = d.c * y0 + d.d * y1;
                ts[2 * k] = x0;
                ts[2 * k + 1] = x1;
            }
            for (int l = 0; l < 32; ++l) {
                const int v = bw[u * 32 + l];
                if (v >= 0) apply(T[v & 0xffff], x0, x1, &ts[2 * ((v >> 16) * 32 + l)]);
            }
        }
        for (int k = 0; k < 2 * R; ++k) xs[2 * p0 + k] = ts[k];
    }
    for (int p = p0 - 1; p >= 0; --p) {
        for (int e = P.lu_diag[p] + 1; e < P.lu_ptr[p + 1]; ++e) apply(Y[e], xs[2 * P.lu_col[e]], xs[2 * P.lu_col[e] + 1], &xs[2 * p]);
        const B d = Y[P.lu_diag[p]];
        const double y0 = xs[2 * p], y1 = xs[2 * p + 1];
        xs[2 * p] = d.a * y0 + d.b * y1;
        xs[2 * p + 1] = d.c * y0 + d.d * y1;
    }
    double dsol = 0.0;
    for (int k = 0; k < 2 * n; ++k) dsol = std::max(dsol, std::fabs(xs[k] - xr[k]));

    // 4. (L U)^T x = b (the adjoint's solve): U^T forward then L^T backward, reference
    //    against level sweeps plus the region's transposed rounds
    auto applyT = [](const B& m, double x0, double x1, double* y) {  // y -= M^T x
        y[0] -= m.a * x0 + m.c * x1;
        y[1] -= m.b * x0 + m.d * x1;
    };
    auto pivT = [](const B& d, double* y) {  // y <- Dinv^T y
        const double y0 = y[0], y1 = y[1];
        y[0] = d.a * y0 + d.c * y1;
        y[1] = d.b * y0 + d.d * y1;
    };
    std::vector<double> tr = b0, tp = b0;
    for (int p = 0; p < n; ++p) {  // row p of U^T: the mirrors of row p's L part
        for (int e = P.lu_ptr[p]; e < P.lu_diag[p]; ++e)
            applyT(X[P.lu_mirror[e]], tr[2 * P.lu_col[e]], tr[2 * P.lu_col[e] + 1], &tr[2 * p]);
        pivT(X[P.lu_diag[p]], &tr[2 * p]);
    }
    for (int p = n - 1; p >= 0; --p)  // row p of L^T: the mirrors of row p's U part
        for (int e = P.lu_diag[p] + 1; e < P.lu_ptr[p + 1]; ++e)
            applyT(X[P.lu_mirror[e]], tr[2 * P.lu_col[e]], tr[2 * P.lu_col[e] + 1], &tr[2 * p]);
    for (int p = 0; p < p0; ++p) {
        for (int e = P.lu_ptr[p]; e < P.lu_diag[p]; ++e)
            applyT(Y[P.lu_mirror[e]], tp[2 * P.lu_col[e]], tp[2 * P.lu_col[e] + 1], &tp[2 * p]);
        pivT(Y[P.lu_diag[p]], &tp[2 * p]);
    }
    if (R > 0) {
        const int *ftk = bw + 32 * P.top_nbw, *ft = ftk + P.top_nft, *btk = ft + 32 * P.top_nft,
                  *bt = btk + P.top_nbt;
        if ((int)(ftk - I) != P.top_nints_fwd || (size_t)(bt + 32 * P.top_nbt - I) != P.top_ints.size()) ++bad;
        std::vector<double> ts(2 * R);
        for (int p = p0; p < n; ++p) {
            double s[2] = {tp[2 * p], tp[2 * p + 1]};
            for (int e = P.lu_ptr[p]; e < P.top_split[p - p0]; ++e)
                applyT(Y[P.lu_mirror[e]], tp[2 * P.lu_col[e]], tp[2 * P.lu_col[e] + 1], s);
            ts[2 * (p - p0)] = s[0];
            ts[2 * (p - p0) + 1] = s[1];
        }
        int lastj = -1;
        for (int u = 0; u < P.top_nft; ++u) {
            const int j = ftk[u] >> 1;
            if (ftk[u] & 1) {
                if (j != lastj + 1) ++bad;  // every column, ascending
                lastj = j;
                pivT(T[piv[j]], &ts[2 * j]);
            }
            for (int l = 0; l < 32; ++l) {
                const int v = ft[u * 32 + l];
                if (v < 0) continue;
                const int k = (v >> 16) * 32 + l;
                if (!at(v & 0xffff, j, k) || k <= j) ++bad;  // U(j, k), k > j
                applyT(T[v & 0xffff], ts[2 * j], ts[2 * j + 1], &ts[2 * k]);
            }
        }
        if (lastj != R - 1) ++bad;
        for (int u = 0; u < P.top_nbt; ++u) {
            const int i = btk[u];
            if (u > 0 && i > btk[u - 1]) ++bad;  // descending
            for (int l = 0; l < 32; ++l) {
                const int v = bt[u * 32 + l];
                if (v < 0) continue;
                const int k = (v >> 16) * 32 + l;
                if (!at(v & 0xffff, i, k) || k >= i) ++bad;  // L(i, k), k < i
                applyT(T[v & 0xffff], ts[2 * i], ts[2 * i + 1], &ts[2 * k]);
            }
        }
        for (int k = 0; k < 2 * R; ++k) tp[2 * p0 + k] = ts[k];
    }
    for (int p = p0 - 1; p >= 0; --p)
        for (int e = P.lu_diag[p] + 1; e < P.lu_ptr[p + 1]; ++e)
            applyT(Y[P.lu_mirror[e]], tp[2 * P.lu_col[e]], tp[2 * P.lu_col[e] + 1], &tp[2 * p]);
    double dsolt = 0.0;
    for (int k = 0; k < 2 * n; ++k) dsolt = std::max(dsolt, std::fabs(tp[k] - tr[k]));
    std::printf("list errors %lld, factor max diff %.3e, solution max diff %.3e, transposed %.3e\n",
                bad, dfac, dsol, dsolt);
    return (bad == 0 && dfac <= 1e-12 && dsol <= 1e-12 && dsolt <= 1e-12) ? 0 : 1;
}
