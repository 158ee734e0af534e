// Symbolic analysis of the sparse Cholesky factor of Lambda (host code).
//
// Algorithm 2 keeps Lambda sparse; its Armijo step needs log det(Lambda + alpha D) (Section
// 4), which for a sparse Lambda comes from a sparse Cholesky factor.  The structure of
// that factor depends only on the pattern and the pivot order, and is found once per
// pattern before any numeric work:
//
//  1. the pivot order: natural; reverse Cuthill-McKee (breadth-first from a
//     pseudo-peripheral vertex of each component, neighbours by ascending degree, the whole
//     order reversed: a small profile for banded patterns); minimum degree (always
//     eliminate a vertex of least current degree in the elimination graph, whose
//     neighbours then become a clique: no fill at all on a forest, little on a chain with
//     few extra links; once the remaining graph is at least 90 % dense the rest is taken
//     as it stands, order no longer mattering there); or given;
//  2. the elimination tree, by path compression over the ancestors found so far: for each
//     pivot k and each earlier neighbour i, climb from i to the root of its current
//     subtree and hang that root under k;
//  3. column counts from row subtrees: row k of L holds exactly the nodes on the tree
//     paths from each earlier neighbour of k up to k, so marking those paths row by row
//     counts every entry of L once (O(nnz(L)) in all).
//
// Deterministic; no GPU is used.
#include <algorithm>
#include <cstdint>
#include <iterator>
#include <set>
#include <vector>

#include "../../include/cggm.h"
#include "graph_order.hpp"

namespace {

// Symmetric adjacency of the pattern without the diagonal, neighbours ascending, no repeats.
struct Adjacency {
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
    int64_t degree(int64_t v) const { return ptr[v + 1] - ptr[v]; }
};

Adjacency symmetrise(int64_t q, const int64_t *row_ptr, const int32_t *col)
{
    std::vector<int64_t> deg(q + 1, 0);
    for (int64_t i = 0; i < q; i++)
        for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; t++)
            if (col[t] != i) {
                deg[i]++;
                deg[col[t]]++;
            }
    std::vector<int64_t> start(q + 1, 0);
    for (int64_t v = 0; v < q; v++) start[v + 1] = start[v] + deg[v];
    std::vector<int32_t> raw(start[q]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < q; i++)
        for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; t++)
            if (col[t] != i) {
                raw[fill[i]++] = col[t];
                raw[fill[col[t]]++] = (int32_t)i;
            }
    Adjacency a;
    a.ptr.assign(q + 1, 0);
    a.adj.reserve(raw.size());
    for (int64_t v = 0; v < q; v++) {
        auto b = raw.begin() + start[v], e = raw.begin() + start[v + 1];
        std::sort(b, e);
        e = std::unique(b, e);
        a.adj.insert(a.adj.end(), b, e);
        a.ptr[v + 1] = (int64_t)a.adj.size();
    }
    return a;
}

// Reverse Cuthill-McKee order (new -> old): the Cuthill-McKee orders of the components, in
// the order of their lowest vertex, concatenated and reversed.
std::vector<int32_t> rcm_order(const Adjacency &a, int64_t q)
{
    std::vector<int32_t> level(q, -1), perm;
    perm.reserve(q);
    for (int32_t s = 0; s < q; s++) {
        if (level[s] >= 0) continue;
        const std::vector<int32_t> comp = cggm::graph::cuthill_mckee(a, s, level);
        perm.insert(perm.end(), comp.begin(), comp.end());
    }
    std::reverse(perm.begin(), perm.end());
    return perm;
}

// Minimum-degree order (new -> old) on the explicit elimination graph.  Ties go to the
// lower index.  Eliminating v joins its current neighbours into a clique.
std::vector<int32_t> min_degree_order(const Adjacency &a, int64_t q)
{
    constexpr double kDenseRest = 0.9;
    std::vector<std::vector<int32_t>> adj(q);
    for (int64_t v = 0; v < q; v++) adj[v].assign(a.adj.begin() + a.ptr[v], a.adj.begin() + a.ptr[v + 1]);
    std::set<std::pair<int64_t, int32_t>> by_degree;
    for (int32_t v = 0; v < q; v++) by_degree.insert({(int64_t)adj[v].size(), v});
    std::vector<int32_t> perm, merged;
    perm.reserve(q);
    while (!by_degree.empty()) {
        const auto first = *by_degree.begin();
        const int64_t remaining = q - (int64_t)perm.size();
        if (remaining > 64 && (double)(first.first + 1) >= kDenseRest * (double)remaining) {
            for (const auto &e : by_degree) perm.push_back(e.second);
            break;
        }
        by_degree.erase(by_degree.begin());
        const int32_t v = first.second;
        perm.push_back(v);
        const std::vector<int32_t> nb = std::move(adj[v]);
        adj[v].clear();
        for (int32_t u : nb) {
            by_degree.erase({(int64_t)adj[u].size(), u});
            merged.clear();
            std::set_union(adj[u].begin(), adj[u].end(), nb.begin(), nb.end(),
                           std::back_inserter(merged));
            merged.erase(std::remove_if(merged.begin(), merged.end(),
                                        [&](int32_t x) { return x == u || x == v; }),
                         merged.end());
            adj[u].swap(merged);
            by_degree.insert({(int64_t)adj[u].size(), u});
        }
    }
    return perm;
}

// Minimum-degree order with approximate degrees (new -> old), on the quotient graph: an
// eliminated pivot p becomes an element holding the variables of its clique (its own
// variables and those of the elements it absorbs); every variable keeps its original
// edges not yet covered by an element, and its elements.  An element's variables stay
// fixed for its life (a variable is eliminated only by absorbing every element it is in),
// so for the variables i of the new element the exact degree is bounded by
//     |edges of i| + (|L_p| - 1) + sum over i's other elements e of |L_e \ L_p|,
// where |L_e \ L_p| is counted for all of them in one pass over the new element's
// variables; the bound is also capped by the old degree + |L_p| - 1 and by the number of
// other remaining variables.  No union over elements is formed, so the cost follows the
// quotient graph rather than the fill.  Ties go to the lower index; the dense-remainder
// rule is the exact order's.
std::vector<int32_t> approx_min_degree_order(const Adjacency &a, int64_t q)
{
    constexpr double kDenseRest = 0.9;
    enum : char { kVar = 0, kElem = 1, kGone = 2 };
    std::vector<char> status(q, kVar);
    std::vector<std::vector<int32_t>> vadj(q), eadj(q), elem(q);
    std::vector<int64_t> degree(q), outside(q, 0), mark(q, -1);
    std::set<std::pair<int64_t, int32_t>> by_degree;
    for (int32_t v = 0; v < q; v++) {
        vadj[v].assign(a.adj.begin() + a.ptr[v], a.adj.begin() + a.ptr[v + 1]);
        degree[v] = (int64_t)vadj[v].size();
        by_degree.insert({degree[v], v});
    }
    int64_t stamp = 0;
    std::vector<int32_t> perm, lp;
    perm.reserve(q);
    while (!by_degree.empty()) {
        const auto first = *by_degree.begin();
        const int64_t remaining = q - (int64_t)perm.size();
        if (remaining > 64 && (double)(first.first + 1) >= kDenseRest * (double)remaining) {
            for (const auto &e : by_degree) perm.push_back(e.second);
            break;
        }
        by_degree.erase(by_degree.begin());
        const int32_t p = first.second;
        // the new element and the absorption of p's elements
        const int64_t in_lp = ++stamp;
        mark[p] = in_lp;
        lp.clear();
        for (int32_t u : vadj[p])
            if (status[u] == kVar && mark[u] != in_lp) {
                mark[u] = in_lp;
                lp.push_back(u);
            }
        for (int32_t e : eadj[p]) {
            if (status[e] != kElem) continue;
            for (int32_t u : elem[e])
                if (status[u] == kVar && mark[u] != in_lp) {
                    mark[u] = in_lp;
                    lp.push_back(u);
                }
            status[e] = kGone;
            std::vector<int32_t>().swap(elem[e]);
        }
        status[p] = kElem;
        elem[p] = lp;
        std::vector<int32_t>().swap(vadj[p]);
        std::vector<int32_t>().swap(eadj[p]);
        perm.push_back(p);
        for (int32_t i : lp) {
            auto &ea = eadj[i];
            ea.erase(std::remove_if(ea.begin(), ea.end(),
                                    [&](int32_t e) { return status[e] != kElem; }),
                     ea.end());
            auto &va = vadj[i];
            va.erase(std::remove_if(va.begin(), va.end(),
                                    [&](int32_t u) { return status[u] != kVar || mark[u] == in_lp; }),
                     va.end());
        }
        // |L_e \ L_p| for the other elements of the new element's variables
        const int64_t seen = ++stamp;
        for (int32_t i : lp)
            for (int32_t e : eadj[i]) {
                if (mark[e] != seen) {
                    mark[e] = seen;
                    outside[e] = (int64_t)elem[e].size();
                }
                outside[e]--;
            }
        const int64_t lpn = (int64_t)lp.size();
        for (int32_t i : lp) {
            int64_t d = (int64_t)vadj[i].size() + lpn - 1;
            for (int32_t e : eadj[i]) d += outside[e];
            d = std::min(d, std::min(remaining - 2, degree[i] + lpn - 1));
            if (d < 0) d = 0;
            eadj[i].push_back(p);
            by_degree.erase({degree[i], i});
            degree[i] = d;
            by_degree.insert({d, i});
        }
    }
    return perm;
}

}  // namespace

extern "C" cggm_status cggm_chol_symbolic(int64_t q, const int64_t *row_ptr, const int32_t *col,
                                          int ordering, const int32_t *perm_in,
                                          int32_t *perm_out, int32_t *parent_out,
                                          int64_t *colcount_out, int64_t *nnz_L_out)
{
    if (q < 0 || q > INT32_MAX) return CGGM_EINVAL;
    if (q > 0 && (!row_ptr || !col || !perm_out || !parent_out || !colcount_out))
        return CGGM_EINVAL;
    if (ordering != CGGM_ORDER_NATURAL && ordering != CGGM_ORDER_RCM &&
        ordering != CGGM_ORDER_GIVEN && ordering != CGGM_ORDER_MINDEG &&
        ordering != CGGM_ORDER_AMD)
        return CGGM_EINVAL;
    if (q == 0) {
        if (nnz_L_out) *nnz_L_out = 0;
        return CGGM_OK;
    }
    if (row_ptr[0] != 0) return CGGM_EINVAL;
    for (int64_t i = 0; i < q; i++)
        if (row_ptr[i + 1] < row_ptr[i]) return CGGM_EINVAL;
    for (int64_t t = 0; t < row_ptr[q]; t++)
        if (col[t] < 0 || col[t] >= q) return CGGM_EINVAL;
    const Adjacency a = symmetrise(q, row_ptr, col);

    // 1. pivot order (new -> old) and its inverse
    std::vector<int32_t> perm(q), iperm(q, -1);
    if (ordering == CGGM_ORDER_NATURAL) {
        for (int32_t k = 0; k < q; k++) perm[k] = k;
    } else if (ordering == CGGM_ORDER_RCM) {
        perm = rcm_order(a, q);
    } else if (ordering == CGGM_ORDER_MINDEG) {
        perm = min_degree_order(a, q);
    } else if (ordering == CGGM_ORDER_AMD) {
        perm = approx_min_degree_order(a, q);
    } else {
        if (!perm_in) return CGGM_EINVAL;
        for (int64_t k = 0; k < q; k++) perm[k] = perm_in[k];
    }
    for (int32_t k = 0; k < q; k++) {
        const int32_t v = perm[k];
        if (v < 0 || v >= q || iperm[v] >= 0) return CGGM_EINVAL;  // not a permutation
        iperm[v] = k;
    }

    // 2. elimination tree of the permuted pattern
    std::vector<int32_t> parent(q, -1), ancestor(q, -1);
    for (int32_t k = 0; k < q; k++) {
        const int32_t v = perm[k];
        for (int64_t t = a.ptr[v]; t < a.ptr[v + 1]; t++) {
            int32_t r = iperm[a.adj[t]];
            if (r >= k) continue;
            while (ancestor[r] != -1 && ancestor[r] != k) {
                const int32_t up = ancestor[r];
                ancestor[r] = k;
                r = up;
            }
            if (ancestor[r] == -1) {
                ancestor[r] = k;
                parent[r] = k;
            }
        }
    }

    // 3. column counts from the row subtrees
    std::vector<int64_t> count(q, 1);  // the diagonal
    std::vector<int32_t> mark(q, -1);
    for (int32_t k = 0; k < q; k++) {
        mark[k] = k;
        const int32_t v = perm[k];
        for (int64_t t = a.ptr[v]; t < a.ptr[v + 1]; t++) {
            int32_t r = iperm[a.adj[t]];
            if (r >= k) continue;
            while (mark[r] != k) {  // k is an ancestor of r: the walk ends at k
                count[r]++;         // L(k, r) is an entry
                mark[r] = k;
                r = parent[r];
            }
        }
    }
    int64_t nnz = 0;
    for (int32_t k = 0; k < q; k++) {
        perm_out[k] = perm[k];
        parent_out[k] = parent[k];
        colcount_out[k] = count[k];
        nnz += count[k];
    }
    if (nnz_L_out) *nnz_L_out = nnz;
    return CGGM_OK;
}

extern "C" cggm_status cggm_chol_supernodes(int64_t q, const int32_t *parent,
                                            const int64_t *colcount, int64_t *start_out,
                                            int64_t *nsuper_out)
{
    if (q < 0 || q > INT32_MAX || !nsuper_out) return CGGM_EINVAL;
    if (q > 0 && (!parent || !colcount || !start_out)) return CGGM_EINVAL;
    std::vector<int32_t> children(q, 0);
    for (int64_t k = 0; k < q; k++) {
        if (colcount[k] < 1 || colcount[k] > q - k) return CGGM_EINVAL;
        if (parent[k] == -1) continue;
        if (parent[k] <= k || parent[k] >= q) return CGGM_EINVAL;
        children[parent[k]]++;
    }
    int64_t ns = 0;
    if (q > 0) start_out[ns++] = 0;
    for (int64_t k = 0; k + 1 < q; k++) {
        // column k + 1 continues k's supernode when k is its only child and column k below
        // its diagonal holds exactly column k + 1's entries
        const bool joins = parent[k] == k + 1 && children[k + 1] == 1 &&
                           colcount[k] == colcount[k + 1] + 1;
        if (!joins) start_out[ns++] = k + 1;
    }
    start_out[ns] = q;
    *nsuper_out = ns;
    return CGGM_OK;
}

extern "C" cggm_status cggm_permute_csr(int64_t q, const int64_t *row_ptr, const int32_t *col,
                                        const double *val, const int32_t *perm,
                                        int64_t *out_row_ptr, int32_t *out_col,
                                        double *out_val)
{
    if (q < 0 || q > INT32_MAX) return CGGM_EINVAL;
    if (q > 0 && (!row_ptr || !perm || !out_row_ptr)) return CGGM_EINVAL;
    if (q == 0) {
        if (out_row_ptr) out_row_ptr[0] = 0;
        return CGGM_OK;
    }
    if (row_ptr[0] != 0) return CGGM_EINVAL;
    for (int64_t i = 0; i < q; i++)
        if (row_ptr[i + 1] < row_ptr[i]) return CGGM_EINVAL;
    const int64_t nnz = row_ptr[q];
    if (nnz > 0 && (!col || !out_col)) return CGGM_EINVAL;
    std::vector<int32_t> iperm(q, -1);
    for (int32_t k = 0; k < q; k++) {
        if (perm[k] < 0 || perm[k] >= q || iperm[perm[k]] >= 0) return CGGM_EINVAL;
        iperm[perm[k]] = k;
    }
    for (int64_t t = 0; t < nnz; t++)
        if (col[t] < 0 || col[t] >= q) return CGGM_EINVAL;
    // row k of the result is row perm[k] of the input with its columns renamed, sorted
    std::vector<std::pair<int32_t, int64_t>> row;  // (new column, source position)
    int64_t at = 0;
    out_row_ptr[0] = 0;
    for (int32_t k = 0; k < q; k++) {
        const int32_t src = perm[k];
        row.clear();
        for (int64_t t = row_ptr[src]; t < row_ptr[src + 1]; t++) row.push_back({iperm[col[t]], t});
        std::stable_sort(row.begin(), row.end(),
                         [](const auto &x, const auto &y) { return x.first < y.first; });
        for (const auto &e : row) {
            out_col[at] = e.first;
            if (val && out_val) out_val[at] = val[e.second];
            at++;
        }
        out_row_ptr[k + 1] = at;
    }
    return CGGM_OK;
}

// Row structure of every supernode (the sorted rows of its dense block of L, in pivot
// numbering): its own columns, the rows below it where the permuted pattern has an entry
// in one of its columns, and the rows below it of its child supernodes (a child's rows
// past its own columns all lie in its parent's structure), merged in supernode order so
// that every child is done before its parent.
extern "C" cggm_status cggm_chol_structure(int64_t q, const int64_t *row_ptr, const int32_t *col,
                                           const int32_t *perm, const int32_t *parent,
                                           const int64_t *colcount, int64_t nsuper,
                                           const int64_t *super_start, int64_t *rows_ptr_out,
                                           int32_t *rows_out)
{
    if (q < 0 || q > INT32_MAX || nsuper < 0 || nsuper > q || !rows_ptr_out) return CGGM_EINVAL;
    if (q > 0 && (!row_ptr || !col || !perm || !parent || !colcount || !super_start))
        return CGGM_EINVAL;
    if ((q == 0) != (nsuper == 0)) return CGGM_EINVAL;
    rows_ptr_out[0] = 0;
    if (q == 0) return CGGM_OK;
    if (super_start[0] != 0 || super_start[nsuper] != q) return CGGM_EINVAL;
    for (int64_t s = 0; s < nsuper; s++)
        if (super_start[s + 1] <= super_start[s]) return CGGM_EINVAL;
    for (int64_t s = 0; s < nsuper; s++) {
        const int64_t c = colcount[super_start[s]];
        if (c < 1 || c > q - super_start[s]) return CGGM_EINVAL;
        rows_ptr_out[s + 1] = rows_ptr_out[s] + c;
    }
    if (!rows_out) return CGGM_OK;  // sizes only
    if (row_ptr[0] != 0) return CGGM_EINVAL;
    for (int64_t i = 0; i < q; i++)
        if (row_ptr[i + 1] < row_ptr[i]) return CGGM_EINVAL;
    std::vector<int32_t> iperm(q, -1), snode(q);
    for (int32_t k = 0; k < q; k++) {
        if (perm[k] < 0 || perm[k] >= q || iperm[perm[k]] >= 0) return CGGM_EINVAL;
        iperm[perm[k]] = k;
    }
    for (int64_t t = 0; t < row_ptr[q]; t++)
        if (col[t] < 0 || col[t] >= q) return CGGM_EINVAL;
    for (int64_t s = 0; s < nsuper; s++)
        for (int64_t k = super_start[s]; k < super_start[s + 1]; k++) snode[k] = (int32_t)s;
    const Adjacency a = symmetrise(q, row_ptr, col);
    // child supernodes of each supernode (the supernode holding the parent of its last column)
    std::vector<std::vector<int32_t>> kids(nsuper);
    for (int64_t s = 0; s < nsuper; s++) {
        const int32_t last = (int32_t)(super_start[s + 1] - 1);
        if (parent[last] < -1 || parent[last] >= q || (parent[last] >= 0 && parent[last] <= last))
            return CGGM_EINVAL;
        if (parent[last] >= 0) kids[snode[parent[last]]].push_back((int32_t)s);
    }
    std::vector<int64_t> mark(q, -1);
    std::vector<int32_t> rows;
    for (int64_t s = 0; s < nsuper; s++) {
        const int32_t f = (int32_t)super_start[s], l = (int32_t)super_start[s + 1];
        rows.clear();
        for (int32_t k = f; k < l; k++) {
            rows.push_back(k);
            mark[k] = s;
        }
        for (int32_t k = f; k < l; k++) {
            const int32_t v = perm[k];
            for (int64_t t = a.ptr[v]; t < a.ptr[v + 1]; t++) {
                const int32_t r = iperm[a.adj[t]];
                if (r >= l && mark[r] != s) {
                    mark[r] = s;
                    rows.push_back(r);
                }
            }
        }
        for (int32_t c : kids[s])
            for (int64_t t = rows_ptr_out[c]; t < rows_ptr_out[c + 1]; t++) {
                const int32_t r = rows_out[t];
                if (r >= l && mark[r] != s) {
                    mark[r] = s;
                    rows.push_back(r);
                }
            }
        if ((int64_t)rows.size() != rows_ptr_out[s + 1] - rows_ptr_out[s]) return CGGM_EINVAL;
        std::sort(rows.begin(), rows.end());
        std::copy(rows.begin(), rows.end(), rows_out + rows_ptr_out[s]);
    }
    return CGGM_OK;
}
