// pf_plan.cpp -- one-time symbolic analysis of a network (Sec. III-B).
//
// Steps, in order:
//   1. validate and canonicalise the Ybus CSR (sorted columns, summed duplicates);
//   2. check that every bus reaches a slack bus through nonzero Ybus entries;
//   3. order the non-slack buses by minimum degree on the bus graph (the J1
//      block pattern inherits the Ybus pattern, Sec. III-B.1), so that the 2x2
//      block LU of J1 has little fill, breaking ties and near-ties (degree within
//      kOrderSlack of the minimum) towards a shallower elimination tree: every tree
//      level is a barrier-separated step of the factorisation and of each sweep;
//   4. build the elimination tree, group the pivots by tree level and renumber
//      them level by level (any topological order of the tree gives the same
//      fill, so this keeps the fill of step 3);
//   5. emit the filled block pattern (CSR), the transpose ("mirror") map, the
//      Ybus index of every block (the cached fill metadata of Alg. 1) and the
//      per-level factorisation schedule.
#include "pf_plan.h"

#include <algorithm>
#include <numeric>
#include <set>
#include <utility>

namespace pf {

namespace {

// merge two sorted vectors, dropping values a and b
void merge_without(const std::vector<int>& x, const std::vector<int>& y, int a, int b,
                   std::vector<int>& out) {
    out.clear();
    out.reserve(x.size() + y.size());
    size_t i = 0, j = 0;
    auto push = [&](int v) {
        if (v != a && v != b && (out.empty() || out.back() != v)) out.push_back(v);
    };
    while (i < x.size() || j < y.size()) {
        if (j >= y.size() || (i < x.size() && x[i] < y[j])) push(x[i++]);
        else if (i >= x.size() || y[j] < x[i]) push(y[j++]);
        else { push(x[i]); ++i; ++j; }
    }
}

int find_in_row(const std::vector<int>& ptr, const std::vector<int>& col, int r, int c) {
    auto b = col.begin() + ptr[r], e = col.begin() + ptr[r + 1];
    auto it = std::lower_bound(b, e, c);
    if (it == e || *it != c) return -1;
    return (int)(it - col.begin());
}

}  // namespace

void minimum_degree(const std::vector<std::vector<int>>& adj0, std::vector<int>& order,
                    std::vector<std::vector<int>>& structs, int slack) {
    const int n = (int)adj0.size();
    std::vector<std::vector<int>> adj = adj0;
    // lvl[v]: a lower bound of v's elimination-tree level (every eliminated neighbour of
    // v is a descendant of v).  The next pivot is, among the nodes whose current degree
    // is within `slack` of the minimum, the one of lowest lvl (then lowest degree, then
    // lowest id): ties, and near-ties, are broken towards a shallower tree.
    std::vector<int> lvl(n, 0);
    std::vector<std::set<std::pair<int, int>>> bucket(n + 1);  // by degree: (lvl, node)
    for (int v = 0; v < n; ++v) bucket[adj[v].size()].insert({0, v});
    order.clear();
    order.reserve(n);
    structs.assign(n, {});
    std::vector<int> tmp;
    int dmin = 0;
    for (int left = n; left > 0; --left) {
        while (bucket[dmin].empty()) ++dmin;
        int v = -1, bd = 0, bl = 0;
        for (int d = dmin; d <= std::min(n, dmin + slack); ++d) {
            if (bucket[d].empty()) continue;
            const auto& c = *bucket[d].begin();
            if (v < 0 || c.first < bl || (c.first == bl && d < bd) ||
                (c.first == bl && d == bd && c.second < v)) {
                v = c.second;
                bd = d;
                bl = c.first;
            }
        }
        bucket[bd].erase({bl, v});
        order.push_back(v);
        const std::vector<int> nb = adj[v];  // all alive (eliminated nodes are removed)
        structs[v] = nb;
        for (int u : nb) {
            bucket[adj[u].size()].erase({lvl[u], u});
            merge_without(adj[u], nb, u, v, tmp);  // u joins the clique of v's neighbours
            adj[u].swap(tmp);
            lvl[u] = std::max(lvl[u], lvl[v] + 1);
            bucket[adj[u].size()].insert({lvl[u], u});
        }
        adj[v].clear();
        dmin = std::max(0, dmin - 1);  // a neighbour's degree drops by at most one (it loses v)
    }
}

// The top region from level l0 on (none if l0 == n_levels): local block numbering, the
// LU lists and the sweep rounds (see Plan).  `lanes` is the plan's gather split rule.
template <typename Lanes>
static BuildStatus build_top(Plan& P, int l0, Lanes lanes) {
    const int n = P.n, p0 = P.lev_ptr[l0], R = n - p0;
    P.top_l0 = l0;
    P.top_p0 = p0;
    P.top_R = R;
    P.top_map.clear();
    P.top_split.assign(R, 0);
    P.top_ints.clear();
    P.top_tr_t.clear();
    P.top_tr_lu.clear();
    P.top_nl = P.top_nfw = P.top_nbw = P.top_nft = P.top_nbt = 0;
    P.top_nints_fwd = 0;
    P.top_g = 1;
    if (R == 0) return BUILD_OK;
    std::vector<int> base(R + 1, 0);
    int mT = 0;  // longest part of a region row left of the region
    for (int p = p0; p < n; ++p) {
        const auto b = P.lu_col.begin() + P.lu_ptr[p], e = P.lu_col.begin() + P.lu_ptr[p + 1];
        const int f = (int)(std::lower_bound(b, e, p0) - P.lu_col.begin());
        P.top_split[p - p0] = f;
        base[p - p0 + 1] = base[p - p0] + (P.lu_ptr[p + 1] - f);
        mT = std::max(mT, f - P.lu_ptr[p]);
    }
    P.top_g = lanes(mT, R);
    P.top_map.resize(base[R]);
    for (int p = p0; p < n; ++p)
        for (int e = P.top_split[p - p0]; e < P.lu_ptr[p + 1]; ++e)
            P.top_map[base[p - p0] + e - P.top_split[p - p0]] = e;
    auto loc = [&](int p, int e) { return base[p - p0] + e - P.top_split[p - p0]; };
    // the region's L columns (rows below the pivot) and U columns (rows above), rows
    // ascending, as (local row, local block)
    std::vector<std::vector<std::pair<int, int>>> lcol(R), ucol(R);
    for (int i = p0; i < n; ++i) {
        for (int e = P.top_split[i - p0]; e < P.lu_diag[i]; ++e)
            lcol[P.lu_col[e] - p0].push_back({i - p0, loc(i, e)});
        for (int e = P.lu_diag[i] + 1; e < P.lu_ptr[i + 1]; ++e)
            ucol[P.lu_col[e] - p0].push_back({i - p0, loc(i, e)});
    }
    std::vector<int>& I = P.top_ints;
    for (int k = p0; k < n; ++k) I.push_back(loc(k, P.lu_diag[k]));  // piv
    I.push_back(0);                                                   // lc_ptr
    for (int k = 0; k < R; ++k) I.push_back(I.back() + (int)lcol[k].size());
    for (int k = 0; k < R; ++k)                                       // lc
        for (const auto& e : lcol[k]) I.push_back(e.second);
    P.top_nl = I[2 * R];
    // Schur triples: for pivot k, every L block (i, k) of the region times every U block
    // (k, j) updates block (i, j), which the filled pattern holds
    I.push_back(0);  // tr_ptr
    for (int k = p0; k < n; ++k) {
        for (const auto& le : lcol[k - p0]) {
            const int i = p0 + le.first;
            for (int e = P.lu_diag[k] + 1; e < P.lu_ptr[k + 1]; ++e) {
                const int j = P.lu_col[e];
                const auto b = P.lu_col.begin() + P.lu_ptr[i], en = P.lu_col.begin() + P.lu_ptr[i + 1];
                const auto it = std::lower_bound(b, en, j);
                if (it == en || *it != j) return BUILD_EINVAL;  // clique property violated: bug
                P.top_tr_t.push_back(loc(i, (int)(it - P.lu_col.begin())));
                P.top_tr_lu.push_back(le.second | (loc(k, e) << 16));
            }
        }
        I.push_back((int)P.top_tr_t.size());
    }
    // sweep rounds: a column's entries go to the lane that owns their row (row i: lane
    // i % 32, register slot i / 32), one entry per lane and round, (slot << 16 | block)
    // or -1.  Per round its column: k for the forward rounds (columns without entries have
    // none), k << 1 | first for the backward rounds (every column has at least one: its
    // first round also applies the pivot inverse)
    auto rounds = [&](const std::vector<std::vector<std::pair<int, int>>>& cols, bool every,
                      int& total) {
        std::vector<int> rk, re;
        for (int k = 0; k < R; ++k) {
            std::vector<std::vector<int>> lane(32);
            for (const auto& e : cols[k]) lane[e.first % 32].push_back(((e.first / 32) << 16) | e.second);
            size_t nr = 0;
            for (const auto& l : lane) nr = std::max(nr, l.size());
            if (every) nr = std::max<size_t>(nr, 1);
            for (size_t r = 0; r < nr; ++r) {
                rk.push_back(every ? (k << 1) | (r == 0 ? 1 : 0) : k);
                for (int l = 0; l < 32; ++l) re.push_back(r < lane[l].size() ? lane[l][r] : -1);
            }
        }
        total = (int)rk.size();
        I.insert(I.end(), rk.begin(), rk.end());
        I.insert(I.end(), re.begin(), re.end());
    };
    rounds(lcol, false, P.top_nfw);
    // the backward sweep takes the columns in descending order
    std::vector<std::vector<std::pair<int, int>>> ucol_desc(ucol.rbegin(), ucol.rend());
    {
        const size_t at = I.size();
        rounds(ucol_desc, true, P.top_nbw);
        // column indices of the reversed list back to the region's own
        for (int u = 0; u < P.top_nbw; ++u) {
            const int v = I[at + u];
            I[at + u] = ((R - 1 - (v >> 1)) << 1) | (v & 1);
        }
    }
    P.top_nints_fwd = (int)I.size();
    // the transposed sweeps of (L U)^T x = b (the adjoint): U^T forward, ascending columns j
    // with U's row j, (k, U(j, k)) for k > j, the first round of each column applying the
    // transposed pivot inverse; then L^T backward, descending columns i with L's row i,
    // (k, L(i, k)) for k < i
    std::vector<std::vector<std::pair<int, int>>> urow(R), lrow_desc(R);
    for (int j = p0; j < n; ++j) {
        for (int e = P.lu_diag[j] + 1; e < P.lu_ptr[j + 1]; ++e)
            urow[j - p0].push_back({P.lu_col[e] - p0, loc(j, e)});
        for (int e = P.top_split[j - p0]; e < P.lu_diag[j]; ++e)
            lrow_desc[n - 1 - j].push_back({P.lu_col[e] - p0, loc(j, e)});
    }
    rounds(urow, true, P.top_nft);
    {
        const size_t at = I.size();
        rounds(lrow_desc, false, P.top_nbt);
        for (int u = 0; u < P.top_nbt; ++u) I[at + u] = R - 1 - I[at + u];
    }
    return BUILD_OK;
}

// Bytes of the region's shared-memory arena in FP64 (blocks, solve vector, lists).
static long long top_arena_fp64(const Plan& P) {
    auto a16 = [](long long v) { return (v + 15) / 16 * 16; };
    return a16((long long)(P.top_blocks() + 1) * 32) + a16((long long)P.top_R * 16) +
           a16((long long)P.top_ints.size() * 4);
}

BuildStatus build_plan(int n_bus, const int* y_indptr, const int* y_indices,
                       const double* y_re, const double* y_im, const int* bus_type,
                       Plan& P, const PlanParams& pp) {
    if (n_bus < 1 || !y_indptr || !y_indices || !y_re || !y_im || !bus_type) return BUILD_EINVAL;
    if (y_indptr[0] != 0) return BUILD_EINVAL;
    for (int i = 0; i < n_bus; ++i)
        if (y_indptr[i + 1] < y_indptr[i]) return BUILD_EINVAL;
    P = Plan();
    P.n_bus = n_bus;
    P.bus_type.assign(bus_type, bus_type + n_bus);
    for (int i = 0; i < n_bus; ++i) {
        int t = bus_type[i];
        if (t < 0 || t > 2) return BUILD_EINVAL;
        if (t == 0) P.n_pq++;
        else if (t == 1) P.n_pv++;
        else P.n_slack++;
    }
    if (P.n_slack < 1) return BUILD_EINVAL;

    // 1. canonical CSR
    P.y_ptr.assign(n_bus + 1, 0);
    std::vector<std::pair<int, std::pair<double, double>>> row;
    for (int i = 0; i < n_bus; ++i) {
        row.clear();
        for (int k = y_indptr[i]; k < y_indptr[i + 1]; ++k) {
            int j = y_indices[k];
            if (j < 0 || j >= n_bus) return BUILD_EINVAL;
            row.push_back({j, {y_re[k], y_im[k]}});
        }
        std::stable_sort(row.begin(), row.end(),
                         [](const auto& a, const auto& b) { return a.first < b.first; });
        for (size_t k = 0; k < row.size(); ++k) {
            if (!P.y_idx.empty() && (int)P.y_idx.size() > P.y_ptr[i] && P.y_idx.back() == row[k].first) {
                P.y_g.back() += row[k].second.first;
                P.y_b.back() += row[k].second.second;
            } else {
                P.y_idx.push_back(row[k].first);
                P.y_g.push_back(row[k].second.first);
                P.y_b.push_back(row[k].second.second);
            }
        }
        P.y_ptr[i + 1] = (int)P.y_idx.size();
    }

    // transpose (the adjoint needs products with Ybus^T; equal to Ybus without phase shifters)
    {
        const int nnz = (int)P.y_idx.size();
        P.yt_ptr.assign(n_bus + 1, 0);
        for (int k = 0; k < nnz; ++k) P.yt_ptr[P.y_idx[k] + 1]++;
        for (int i = 0; i < n_bus; ++i) P.yt_ptr[i + 1] += P.yt_ptr[i];
        P.yt_idx.resize(nnz);
        P.yt_g.resize(nnz);
        P.yt_b.resize(nnz);
        std::vector<int> fill(P.yt_ptr.begin(), P.yt_ptr.end() - 1);
        for (int i = 0; i < n_bus; ++i)
            for (int k = P.y_ptr[i]; k < P.y_ptr[i + 1]; ++k) {
                int d = fill[P.y_idx[k]]++;
                P.yt_idx[d] = i;
                P.yt_g[d] = P.y_g[k];
                P.yt_b[d] = P.y_b[k];
            }
    }

    // 2. every non-slack bus needs a diagonal entry and a path to a slack bus
    for (int i = 0; i < n_bus; ++i)
        if (bus_type[i] != 2 && find_in_row(P.y_ptr, P.y_idx, i, i) < 0) return BUILD_ESINGULAR;
    {
        std::vector<char> seen(n_bus, 0);
        std::vector<int> stack;
        for (int i = 0; i < n_bus; ++i)
            if (bus_type[i] == 2) { seen[i] = 1; stack.push_back(i); }
        while (!stack.empty()) {
            int u = stack.back();
            stack.pop_back();
            for (int k = P.y_ptr[u]; k < P.y_ptr[u + 1]; ++k) {
                int v = P.y_idx[k];
                if (!seen[v] && (P.y_g[k] != 0.0 || P.y_b[k] != 0.0)) { seen[v] = 1; stack.push_back(v); }
            }
        }
        for (int i = 0; i < n_bus; ++i)
            if (!seen[i]) return BUILD_ESINGULAR;
    }

    // 3. bus graph of the non-slack buses and its minimum-degree order
    std::vector<int> nodes;  // node id -> bus
    std::vector<int> bus2node(n_bus, -1);
    for (int i = 0; i < n_bus; ++i)
        if (bus_type[i] != 2) { bus2node[i] = (int)nodes.size(); nodes.push_back(i); }
    const int n = (int)nodes.size();
    P.n = n;
    std::vector<std::vector<int>> adj(n);
    for (int a = 0; a < n; ++a) {
        int i = nodes[a];
        for (int k = P.y_ptr[i]; k < P.y_ptr[i + 1]; ++k) {
            int j = P.y_idx[k];
            int b = bus2node[j];
            if (b >= 0 && b != a) { adj[a].push_back(b); adj[b].push_back(a); }
        }
    }
    for (auto& v : adj) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    std::vector<int> order;
    std::vector<std::vector<int>> structs;
    minimum_degree(adj, order, structs, pp.order_slack);
    std::vector<int> elim(n);  // node -> elimination index
    for (int k = 0; k < n; ++k) elim[order[k]] = k;

    // 4. elimination tree and levels (children are eliminated before parents)
    std::vector<int> level(n, 0);
    for (int k = 0; k < n; ++k) {
        int v = order[k];
        int parent = -1;
        for (int u : structs[v])
            if (parent < 0 || elim[u] < elim[parent]) parent = u;
        if (parent >= 0) level[parent] = std::max(level[parent], level[v] + 1);
    }
    int n_levels = 0;
    for (int v = 0; v < n; ++v) n_levels = std::max(n_levels, level[v] + 1);
    if (n == 0) n_levels = 0;
    std::vector<int> byl(n);
    std::iota(byl.begin(), byl.end(), 0);
    std::sort(byl.begin(), byl.end(), [&](int a, int b) {
        if (level[a] != level[b]) return level[a] < level[b];
        return elim[a] < elim[b];
    });
    std::vector<int> node2pos(n);
    for (int p = 0; p < n; ++p) node2pos[byl[p]] = p;
    P.n_levels = n_levels;
    P.lev_ptr.assign(n_levels + 1, 0);
    for (int v = 0; v < n; ++v) P.lev_ptr[level[v] + 1]++;
    for (int l = 0; l < n_levels; ++l) P.lev_ptr[l + 1] += P.lev_ptr[l];
    P.pos2bus.resize(n);
    P.bus2pos.assign(n_bus, -1);
    for (int p = 0; p < n; ++p) {
        P.pos2bus[p] = nodes[byl[p]];
        P.bus2pos[nodes[byl[p]]] = p;
    }

    // 5. filled block pattern in position order
    std::vector<std::vector<int>> upos(n);  // U(p, .) columns, ascending
    for (int v = 0; v < n; ++v) {
        int p = node2pos[v];
        for (int u : structs[v]) upos[p].push_back(node2pos[u]);
        std::sort(upos[p].begin(), upos[p].end());
    }
    std::vector<std::vector<int>> rows(n);
    for (int p = 0; p < n; ++p) {
        rows[p].push_back(p);
        for (int q : upos[p]) {
            if (q <= p) return BUILD_EINVAL;  // cannot happen: ancestors sit on higher levels
            rows[p].push_back(q);
            rows[q].push_back(p);  // L(q, p)
        }
    }
    P.lu_ptr.assign(n + 1, 0);
    for (int p = 0; p < n; ++p) {
        std::sort(rows[p].begin(), rows[p].end());
        P.lu_ptr[p + 1] = P.lu_ptr[p] + (int)rows[p].size();
    }
    const int nnzb = P.lu_ptr[n];
    P.lu_col.resize(nnzb);
    P.lu_row.resize(nnzb);
    P.lu_diag.resize(n);
    for (int p = 0; p < n; ++p)
        for (size_t k = 0; k < rows[p].size(); ++k) {
            int e = P.lu_ptr[p] + (int)k;
            P.lu_col[e] = rows[p][k];
            P.lu_row[e] = p;
            if (rows[p][k] == p) P.lu_diag[p] = e;
        }
    P.lu_mirror.resize(nnzb);
    P.fill_y.resize(nnzb);
    for (int e = 0; e < nnzb; ++e) {
        int p = P.lu_row[e], q = P.lu_col[e];
        P.lu_mirror[e] = find_in_row(P.lu_ptr, P.lu_col, q, p);
        P.fill_y[e] = find_in_row(P.y_ptr, P.y_idx, P.pos2bus[p], P.pos2bus[q]);
    }

    // factorisation schedule
    P.la_ptr.assign(n_levels + 1, 0);
    P.sch_tptr.assign(n_levels + 1, 0);
    P.sch_cptr.assign(1, 0);
    struct Contrib {
        int t, L, U;
    };
    std::vector<Contrib> contrib;
    for (int l = 0; l < n_levels; ++l) {
        contrib.clear();
        for (int k = P.lev_ptr[l]; k < P.lev_ptr[l + 1]; ++k) {
            const int dk = P.lu_diag[k];
            for (int e = dk + 1; e < P.lu_ptr[k + 1]; ++e) {  // U(k, j), j > k
                P.la_L.push_back(P.lu_mirror[e]);             // L(j, k)
                P.la_D.push_back(dk);
            }
            for (int ei = dk + 1; ei < P.lu_ptr[k + 1]; ++ei) {
                int i = P.lu_col[ei];
                int Lik = P.lu_mirror[ei];
                for (int ej = dk + 1; ej < P.lu_ptr[k + 1]; ++ej) {
                    int j = P.lu_col[ej];
                    int t = find_in_row(P.lu_ptr, P.lu_col, i, j);
                    if (t < 0) return BUILD_EINVAL;  // clique property violated: bug
                    contrib.push_back({t, Lik, ej});
                }
            }
        }
        P.la_ptr[l + 1] = (int)P.la_L.size();
        std::stable_sort(contrib.begin(), contrib.end(),
                         [](const Contrib& a, const Contrib& b) { return a.t < b.t; });
        for (size_t c = 0; c < contrib.size(); ++c) {
            if (c == 0 || contrib[c].t != contrib[c - 1].t) {
                P.sch_tgt.push_back(contrib[c].t);
                P.sch_cptr.push_back(P.sch_cptr.back());
            }
            P.sch_L.push_back(contrib[c].L);
            P.sch_U.push_back(contrib[c].U);
            P.sch_cptr.back()++;
        }
        P.sch_tptr[l + 1] = (int)P.sch_tgt.size();
        P.schur_ops += (long long)contrib.size();
    }

    // lanes per gathered row.  One thread gathers a row, except on levels of few rows
    // (<= 128) whose longest gather exceeds 8 blocks: towards the top of the elimination
    // tree a level is a handful of long, nearly dense rows, and one thread per row would
    // make the whole level wait on one long sequential gather.  There a row is split over
    // a power-of-two group of lanes (about four blocks each) and reduced by shuffles.  The
    // choice depends on the plan only, so the summation order (and every result) is the
    // same for any number of threads per scenario.
    auto lanes = [&pp](int len, int rows) {
        if (len <= pp.split_len || rows > pp.split_rows) return 1;
        int g = 1;
        while (g * 4 < len && g < 32) g <<= 1;
        return g;
    };
    P.lev_gL.assign(n_levels, 1);
    P.lev_gU.assign(n_levels, 1);
    P.lev_gS.assign(n_levels, 1);
    for (int l = 0; l < n_levels; ++l) {
        int mL = 0, mU = 0, mS = 0;
        for (int p = P.lev_ptr[l]; p < P.lev_ptr[l + 1]; ++p) {
            mL = std::max(mL, P.lu_diag[p] - P.lu_ptr[p]);
            mU = std::max(mU, P.lu_ptr[p + 1] - P.lu_diag[p] - 1);
        }
        for (int t = P.sch_tptr[l]; t < P.sch_tptr[l + 1]; ++t)
            mS = std::max(mS, P.sch_cptr[t + 1] - P.sch_cptr[t]);
        const int rows = P.lev_ptr[l + 1] - P.lev_ptr[l];
        const int targets = P.sch_tptr[l + 1] - P.sch_tptr[l];
        P.lev_gL[l] = lanes(mL, rows);
        P.lev_gU[l] = lanes(mU, rows);
        P.lev_gS[l] = lanes(mS, targets);
    }

    // top region: the trailing levels of at most top_rows rows each, taken from the top of
    // the tree down while the region's blocks (its rows' entries from its first row on)
    // stay within top_blocks, its rows within kTopMaxRows and its FP64 arena within
    // kTopMaxBytes.  Its pivots are factored and swept one at a time.
    {
        auto first_in = [&P](int p, int p0) {  // first entry of row p at column >= p0
            const auto b = P.lu_col.begin() + P.lu_ptr[p], e = P.lu_col.begin() + P.lu_ptr[p + 1];
            return (int)(std::lower_bound(b, e, p0) - P.lu_col.begin());
        };
        auto blocks_from = [&](int p0) {
            long long c = 0;
            for (int p = p0; p < n; ++p) c += P.lu_ptr[p + 1] - first_in(p, p0);
            return c;
        };
        const long long cap = std::min(pp.top_blocks, kTopMaxBlocks);
        int l0 = n_levels;
        while (pp.top_rows > 0 && n >= pp.top_min_pivots && l0 > 0 &&
               P.lev_ptr[l0] - P.lev_ptr[l0 - 1] <= pp.top_rows &&
               n - P.lev_ptr[l0 - 1] <= kTopMaxRows && blocks_from(P.lev_ptr[l0 - 1]) <= cap)
            --l0;
        for (;; ++l0) {  // shrink from the bottom of the region until its arena fits
            if (n - P.lev_ptr[l0] < kTopMin) l0 = n_levels;
            if (build_top(P, l0, [&](int len, int rows) { return lanes(len, rows); }) != BUILD_OK)
                return BUILD_EINVAL;
            if (P.top_R == 0 || top_arena_fp64(P) <= kTopMaxBytes) break;
        }
    }

    // scalar nonzeros of J1 (rows dP_{B\R}, dQ_D; columns theta_{B\R}, Vm_D)
    long long nnz = 0;
    for (int i = 0; i < n_bus; ++i) {
        if (bus_type[i] == 2) continue;
        int ri = 1 + (bus_type[i] == 0);
        for (int k = P.y_ptr[i]; k < P.y_ptr[i + 1]; ++k) {
            int j = P.y_idx[k];
            if (bus_type[j] == 2) continue;
            nnz += ri * (1 + (bus_type[j] == 0));
        }
    }
    P.nnz_j1 = (int)nnz;

    // the scalar J1 template in the paper's ordering
    std::vector<int> rowP(n_bus, -1), rowQ(n_bus, -1), colV(n_bus, -1), colT(n_bus, -1);
    int nBR = 0, nD = 0;
    for (int i = 0; i < n_bus; ++i) {
        if (bus_type[i] != 2) colT[i] = nBR, rowP[i] = nBR++;
        if (bus_type[i] == 0) colV[i] = nD++;
    }
    for (int i = 0; i < n_bus; ++i) {
        if (bus_type[i] == 0) rowQ[i] = nBR + colV[i];
        if (bus_type[i] != 2) colT[i] += nD;
    }
    P.n1 = nBR + nD;
    std::vector<int> cntV(n_bus, 0), cntT(n_bus, 0);
    for (int i = 0; i < n_bus; ++i)
        for (int k = P.y_ptr[i]; k < P.y_ptr[i + 1]; ++k) {
            cntV[i] += bus_type[P.y_idx[k]] == 0;
            cntT[i] += bus_type[P.y_idx[k]] != 2;
        }
    P.j1_ptr.assign(P.n1 + 1, 0);
    for (int i = 0; i < n_bus; ++i) {
        if (rowP[i] >= 0) P.j1_ptr[rowP[i] + 1] = cntV[i] + cntT[i];
        if (rowQ[i] >= 0) P.j1_ptr[rowQ[i] + 1] = cntV[i] + cntT[i];
    }
    for (int r = 0; r < P.n1; ++r) P.j1_ptr[r + 1] += P.j1_ptr[r];
    P.j1_col.assign(P.j1_ptr[P.n1], -1);
    P.j1_pos.assign(4 * P.y_idx.size(), -1);
    for (int i = 0; i < n_bus; ++i) {
        const int rows[2] = {rowP[i], rowQ[i]};
        for (int h = 0; h < 2; ++h) {  // h = 0: the dP_i row, h = 1: the dQ_i row
            if (rows[h] < 0) continue;
            int v = P.j1_ptr[rows[h]], t = v + cntV[i];
            for (int k = P.y_ptr[i]; k < P.y_ptr[i + 1]; ++k) {
                const int j = P.y_idx[k];
                if (colV[j] >= 0) {
                    P.j1_col[v] = colV[j];
                    P.j1_pos[4 * k + 2 * h + 1] = v++;
                }
                if (bus_type[j] != 2) {
                    P.j1_col[t] = colT[j];
                    P.j1_pos[4 * k + 2 * h] = t++;
                }
            }
        }
    }
    return BUILD_OK;
}

}  // namespace pf
