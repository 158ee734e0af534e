// Column partitions for the block coordinate descent of Algorithm 2 (Section 4).
//
// Section 4 cuts the q output columns into blocks so that the columns of Sigma (and Psi)
// that one block needs fit in memory together, and picks the cut by graph clustering.
// For Lambda the graph is that of its active set: an edge i - j for each active
// off-diagonal coordinate, since an active entry between two blocks costs a cache miss
// (Section 4.1).  For Theta it joins two columns that hold active entries in a common
// row, the pattern of S^T S over the active set, since each block a row touches costs one
// row of S_xx (Section 4.2).  The paper calls METIS; this file is a self-contained host
// partitioner of its own design, which computes three candidate partitions and keeps the
// one of lowest cut:
//
//  1. the weighted graph in CSR form, with self loops dropped and parallel edges merged;
//  2. single level: connected components, each ordered by breadth-first search from a
//     pseudo-peripheral vertex, neighbours taken by ascending degree (Cuthill-McKee
//     order); a component too large for one block is cut along that order into the
//     fewest pieces of equal size up to one;
//  3. multilevel (two candidates): heavy-edge matching coarsens the graph while it is
//     well above the block count; on the coarsest graph pieces are grown greedily around
//     the most strongly connected vertex, either up to the block size or (second
//     candidate) stopping early at a cluster's edge; the blocks are then projected back
//     level by level and refined at each level;
//  4. pieces are joined along their heaviest links while they fit, and packed by
//     first-fit decreasing;
//  5. boundary refinement: passes over the vertices that move a vertex to the adjacent
//     block it is most connected to, when that lowers the cut and the block has room, or
//     else exchange it with a neighbour in that block when the exchange lowers the cut.
//     The cut never grows.
//
// Host code only: no GPU is used.  Deterministic: ties go to the lower index.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <queue>
#include <vector>

#include "../../include/cggm.h"
#include "graph_order.hpp"

namespace {

using namespace cggm;

constexpr int kRefinePasses = 8;
constexpr int64_t kCliqueMaxRow = 16;  // rows with more active columns are joined as a path

struct Graph {
    int64_t n = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
    std::vector<double> w;
    int64_t degree(int64_t v) const { return ptr[v + 1] - ptr[v]; }
};

struct Edge {
    int32_t u, v;
    double w;
};

// CSR of the undirected graph on n vertices: both directions of every edge, self loops
// dropped, parallel edges merged with their weights added, neighbours ascending.
Graph build_graph(int64_t n, const std::vector<Edge> &edges)
{
    Graph g;
    g.n = n;
    std::vector<int64_t> deg(n + 1, 0);
    for (const Edge &e : edges)
        if (e.u != e.v) {
            deg[e.u]++;
            deg[e.v]++;
        }
    std::vector<int64_t> start(n + 1, 0);
    for (int64_t v = 0; v < n; v++) start[v + 1] = start[v] + deg[v];
    std::vector<std::pair<int32_t, double>> raw(start[n]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (const Edge &e : edges)
        if (e.u != e.v) {
            raw[fill[e.u]++] = {e.v, e.w};
            raw[fill[e.v]++] = {e.u, e.w};
        }
    g.ptr.assign(n + 1, 0);
    g.adj.reserve(raw.size());
    g.w.reserve(raw.size());
    for (int64_t v = 0; v < n; v++) {
        auto b = raw.begin() + start[v], e = raw.begin() + start[v + 1];
        std::sort(b, e, [](const auto &x, const auto &y) { return x.first < y.first; });
        for (auto it = b; it != e; ++it) {
            if (!g.adj.empty() && (int64_t)g.adj.size() > g.ptr[v] && g.adj.back() == it->first)
                g.w.back() += it->second;
            else {
                g.adj.push_back(it->first);
                g.w.push_back(it->second);
            }
        }
        g.ptr[v + 1] = (int64_t)g.adj.size();
    }
    return g;
}

// Pieces (vertex lists of weight at most cap) grouped into blocks: pairs of pieces are
// joined in order of the edge weight between them, heaviest first, while the joined
// weight fits in `cap`; the groups are then packed by first-fit decreasing weight (equal
// weights keep their order).  Returns the block of every vertex.
std::vector<int32_t> pack_pieces(const Graph &g, const std::vector<std::vector<int32_t>> &pieces,
                                 const std::vector<int64_t> &piece_w, int64_t cap)
{
    const int64_t n = g.n;
    const int64_t np = (int64_t)pieces.size();
    std::vector<int32_t> of(n, -1);
    for (int64_t k = 0; k < np; k++)
        for (int32_t v : pieces[k]) of[v] = (int32_t)k;
    std::vector<Edge> links;
    for (int32_t v = 0; v < n; v++)
        for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++)
            if (g.adj[t] > v && of[g.adj[t]] != of[v]) links.push_back({of[v], of[g.adj[t]], g.w[t]});
    const Graph pg = build_graph(np, links);
    std::vector<Edge> order;
    for (int32_t a = 0; a < np; a++)
        for (int64_t t = pg.ptr[a]; t < pg.ptr[a + 1]; t++)
            if (pg.adj[t] > a) order.push_back({a, pg.adj[t], pg.w[t]});
    std::stable_sort(order.begin(), order.end(),
                     [](const Edge &x, const Edge &y) { return x.w > y.w; });
    std::vector<int32_t> root(np);
    std::vector<int64_t> gw(piece_w.begin(), piece_w.end());
    for (int32_t k = 0; k < np; k++) root[k] = k;
    auto find = [&](int32_t k) {
        while (root[k] != k) k = root[k] = root[root[k]];
        return k;
    };
    for (const Edge &e : order) {
        const int32_t a = find(e.u), b = find(e.v);
        if (a == b || gw[a] + gw[b] > cap) continue;
        root[std::max(a, b)] = std::min(a, b);
        gw[std::min(a, b)] += gw[std::max(a, b)];
    }
    std::vector<int32_t> groups;
    for (int32_t k = 0; k < np; k++)
        if (find(k) == k) groups.push_back(k);
    std::stable_sort(groups.begin(), groups.end(),
                     [&](int32_t a, int32_t b) { return gw[a] > gw[b]; });
    std::vector<int64_t> room;
    std::vector<int32_t> bin_of(np, -1);
    size_t open = 0;  // bins before it are full
    for (int32_t k : groups) {
        while (open < room.size() && room[open] == 0) open++;
        size_t b = open;
        while (b < room.size() && room[b] < gw[k]) b++;
        if (b == room.size()) room.push_back(cap);
        room[b] -= gw[k];
        bin_of[k] = (int32_t)b;
    }
    std::vector<int32_t> blk(n, -1);
    for (int32_t v = 0; v < n; v++) blk[v] = bin_of[find(of[v])];
    return blk;
}

// Greedy growing: from the unassigned vertex of least degree, a piece takes, one at a time,
// the unassigned vertex most strongly connected to it (ties: lower index) that still fits
// in `cap`, until none is left; then the next piece starts.  With `settle`, a piece that
// is at least half full also stops at a vertex that has less edge weight into the piece
// than out of it, so that a cluster smaller than a block is not topped up from its
// neighbours.  Pieces are then packed.
std::vector<int32_t> grown_blocks(const Graph &g, const std::vector<int64_t> &vw, int64_t cap,
                                  bool settle)
{
    const int64_t n = g.n;
    std::vector<int32_t> seeds(n);
    for (int32_t v = 0; v < n; v++) seeds[v] = v;
    std::stable_sort(seeds.begin(), seeds.end(),
                     [&](int32_t a, int32_t b) { return g.degree(a) < g.degree(b); });
    std::vector<char> taken(n, 0);
    std::vector<double> conn(n, 0.0), wdeg(n, 0.0);
    for (int32_t v = 0; v < n; v++)
        for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++) wdeg[v] += g.w[t];
    std::vector<int32_t> touched;
    std::vector<std::vector<int32_t>> pieces;
    std::vector<int64_t> piece_w;
    using Item = std::pair<double, int32_t>;
    auto lower = [](const Item &a, const Item &b) {
        return a.first != b.first ? a.first < b.first : a.second > b.second;
    };
    for (int32_t seed : seeds) {
        if (taken[seed]) continue;
        pieces.emplace_back();
        piece_w.push_back(0);
        std::priority_queue<Item, std::vector<Item>, decltype(lower)> pq(lower);
        pq.push({0.0, seed});
        touched.clear();
        while (!pq.empty() && piece_w.back() < cap) {
            const Item it = pq.top();
            pq.pop();
            const int32_t v = it.second;
            if (taken[v] || it.first != conn[v] || piece_w.back() + vw[v] > cap) continue;
            if (settle && 2 * piece_w.back() >= cap && 2.0 * conn[v] < wdeg[v]) break;
            taken[v] = 1;
            pieces.back().push_back(v);
            piece_w.back() += vw[v];
            for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++) {
                const int32_t u = g.adj[t];
                if (taken[u]) continue;
                if (conn[u] == 0.0) touched.push_back(u);
                conn[u] += g.w[t];
                pq.push({conn[u], u});
            }
        }
        for (int32_t u : touched) conn[u] = 0.0;
    }
    return pack_pieces(g, pieces, piece_w, cap);
}

// Step 2: an initial assignment of every vertex to a block of at most `cap`
// columns: components in Cuthill-McKee order, a component too large for one block cut
// into the fewest pieces of equal size up to one, pieces packed.
std::vector<int32_t> initial_blocks(const Graph &g, int64_t cap)
{
    const int64_t n = g.n;
    std::vector<int32_t> level(n, -1);
    std::vector<std::vector<int32_t>> pieces;
    std::vector<int64_t> piece_w;
    for (int32_t v = 0; v < n; v++) {
        if (level[v] >= 0) continue;
        std::vector<int32_t> ord = graph::cuthill_mckee(g, v, level);
        const int64_t size = (int64_t)ord.size();
        const int64_t parts = (size + cap - 1) / cap;
        int64_t at = 0;
        for (int64_t k = 0; k < parts; k++) {
            const int64_t len = size / parts + (k < size % parts ? 1 : 0);
            pieces.emplace_back(ord.begin() + at, ord.begin() + at + len);
            piece_w.push_back(len);
            at += len;
        }
    }
    return pack_pieces(g, pieces, piece_w, cap);
}

// Weight from v to each block among its neighbours' blocks, as (block, weight) pairs
// sorted by block.
void block_links(const Graph &g, const std::vector<int32_t> &blk, int32_t v,
                 std::vector<std::pair<int32_t, double>> &out)
{
    out.clear();
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++) out.push_back({blk[g.adj[t]], g.w[t]});
    std::sort(out.begin(), out.end(),
              [](const auto &a, const auto &b) { return a.first < b.first; });
    size_t k = 0;
    for (size_t t = 0; t < out.size(); t++) {
        if (k > 0 && out[k - 1].first == out[t].first)
            out[k - 1].second += out[t].second;
        else
            out[k++] = out[t];
    }
    out.resize(k);
}

double link_to(const std::vector<std::pair<int32_t, double>> &links, int32_t b)
{
    for (const auto &l : links)
        if (l.first == b) return l.second;
    return 0.0;
}

double edge_weight(const Graph &g, int32_t u, int32_t v)
{
    auto b = g.adj.begin() + g.ptr[u], e = g.adj.begin() + g.ptr[u + 1];
    auto it = std::lower_bound(b, e, v);
    return (it != e && *it == v) ? g.w[it - g.adj.begin()] : 0.0;
}

// Step 5.  Every accepted move or exchange lowers the cut by more than a rounding margin
// and keeps every block's vertex weight within `cap`.
void refine(const Graph &g, const std::vector<int64_t> &vw, std::vector<int32_t> &blk,
            int64_t cap)
{
    int32_t nb = 0;
    for (int32_t b : blk) nb = std::max(nb, b + 1);
    std::vector<int64_t> size(nb, 0);
    for (int32_t v = 0; v < g.n; v++) size[blk[v]] += vw[v];
    std::vector<std::pair<int32_t, double>> lv, lu;
    for (int pass = 0; pass < kRefinePasses; pass++) {
        bool changed = false;
        for (int32_t v = 0; v < g.n; v++) {
            block_links(g, blk, v, lv);
            const int32_t own = blk[v];
            const double w_own = link_to(lv, own);
            int32_t best = -1;
            double gain = 0.0;
            for (const auto &l : lv)
                if (l.first != own && l.second - w_own > gain) {
                    gain = l.second - w_own;
                    best = l.first;
                }
            const double margin = 1e-12 * (1.0 + w_own + gain);
            if (best < 0 || gain <= margin) continue;
            if (size[best] + vw[v] <= cap) {
                blk[v] = best;
                size[own] -= vw[v];
                size[best] += vw[v];
                changed = true;
                continue;
            }
            // exchange with the neighbour u in `best` whose swap lowers the cut most
            int32_t partner = -1;
            double total_best = margin;
            for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++) {
                const int32_t u = g.adj[t];
                if (blk[u] != best) continue;
                if (size[own] - vw[v] + vw[u] > cap || size[best] - vw[u] + vw[v] > cap) continue;
                block_links(g, blk, u, lu);
                const double gu = link_to(lu, own) - link_to(lu, best);
                const double total = gain + gu - 2.0 * edge_weight(g, u, v);
                if (total > total_best) {
                    total_best = total;
                    partner = u;
                }
            }
            if (partner >= 0) {
                blk[partner] = own;
                blk[v] = best;
                size[own] += vw[partner] - vw[v];
                size[best] += vw[v] - vw[partner];
                changed = true;
            }
        }
        if (!changed) break;
    }
}

// Block ids renumbered 0..k-1 by the lowest column of each block; returns k.
int64_t renumber(std::vector<int32_t> &blk)
{
    int32_t nb = 0;
    for (int32_t b : blk) nb = std::max(nb, b + 1);
    std::vector<int32_t> map(nb, -1);
    int32_t k = 0;
    for (int32_t &b : blk) {
        if (map[b] < 0) map[b] = k++;
        b = map[b];
    }
    return k;
}

double cut_weight(const Graph &g, const std::vector<int32_t> &blk)
{
    double c = 0.0;
    for (int32_t v = 0; v < g.n; v++)
        for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++)
            if (g.adj[t] > v && blk[g.adj[t]] != blk[v]) c += g.w[t];
    return c;
}

// One level of coarsening by heavy-edge matching: each vertex, in index order, is paired
// with its unmatched neighbour of heaviest edge whose combined weight stays within
// `maxvw`; pairs (and unpaired vertices) become the vertices of the coarse graph, whose
// edges are the fine edges between pairs with their weights added.  Returns false when
// the graph shrinks by less than 5 %.
bool coarsen(const Graph &g, const std::vector<int64_t> &vw, int64_t maxvw, Graph &gc,
             std::vector<int64_t> &vwc, std::vector<int32_t> &cmap)
{
    const int64_t n = g.n;
    std::vector<int32_t> match(n, -1);
    for (int32_t v = 0; v < n; v++) {
        if (match[v] >= 0) continue;
        int32_t best = -1;
        double bw = 0.0;
        for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++) {
            const int32_t u = g.adj[t];
            if (match[u] < 0 && vw[u] + vw[v] <= maxvw && g.w[t] > bw) {
                bw = g.w[t];
                best = u;
            }
        }
        match[v] = best >= 0 ? best : v;
        if (best >= 0) match[best] = v;
    }
    cmap.assign(n, -1);
    int32_t nc = 0;
    for (int32_t v = 0; v < n; v++)
        if (cmap[v] < 0) {
            cmap[v] = nc;
            cmap[match[v]] = nc;
            nc++;
        }
    if (nc > n - n / 20) return false;
    vwc.assign(nc, 0);
    for (int32_t v = 0; v < n; v++) vwc[cmap[v]] += vw[v];
    std::vector<Edge> edges;
    for (int32_t v = 0; v < n; v++)
        for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++)
            if (g.adj[t] > v && cmap[g.adj[t]] != cmap[v])
                edges.push_back({cmap[v], cmap[g.adj[t]], g.w[t]});
    gc = build_graph(nc, edges);
    return true;
}

// Multilevel form: coarsen while the graph is well above the block count (coarse vertices
// hold at most a quarter block), assign blocks on the coarsest graph, then project back
// level by level, refining at each.  Moving a coarse vertex moves a whole cluster, which
// single-vertex refinement on the fine graph cannot do.
std::vector<int32_t> multilevel_blocks(const Graph &g0, int64_t cap, bool settle)
{
    std::vector<Graph> gs{g0};
    std::vector<std::vector<int64_t>> vws{std::vector<int64_t>(g0.n, 1)};
    std::vector<std::vector<int32_t>> maps;
    const int64_t maxvw = std::max<int64_t>(1, cap / 4);
    const int64_t kmin = (g0.n + cap - 1) / cap;
    const int64_t stop = std::max<int64_t>(64, 8 * kmin);
    while (gs.back().n > stop && maps.size() < 40) {
        Graph gc;
        std::vector<int64_t> vwc;
        std::vector<int32_t> cmap;
        if (!coarsen(gs.back(), vws.back(), maxvw, gc, vwc, cmap)) break;
        gs.push_back(std::move(gc));
        vws.push_back(std::move(vwc));
        maps.push_back(std::move(cmap));
    }
    std::vector<int32_t> blk = grown_blocks(gs.back(), vws.back(), cap, settle);
    refine(gs.back(), vws.back(), blk, cap);
    for (size_t l = maps.size(); l-- > 0;) {
        std::vector<int32_t> fine(gs[l].n);
        for (int64_t v = 0; v < gs[l].n; v++) fine[v] = blk[maps[l][v]];
        blk.swap(fine);
        refine(gs[l], vws[l], blk, cap);
    }
    return blk;
}

// Three candidates: the single-level one (steps 2-4 on the graph itself) and the
// multilevel one with either growing rule.  The lowest cut wins, then the fewest blocks,
// then the earlier candidate.
cggm_status partition_graph(int64_t q, const std::vector<Edge> &edges, int64_t max_block,
                            int32_t *block_out, int64_t *nblocks_out, double *cut_out)
{
    const Graph g = build_graph(q, edges);
    const std::vector<int64_t> ones(q, 1);
    std::vector<int32_t> best = initial_blocks(g, max_block);
    refine(g, ones, best, max_block);
    int64_t kbest = renumber(best);
    double cbest = cut_weight(g, best);
    for (bool settle : {false, true}) {
        std::vector<int32_t> c = multilevel_blocks(g, max_block, settle);
        const int64_t kc = renumber(c);
        const double cc = cut_weight(g, c);
        const double tol = 1e-12 * (1.0 + cbest);
        if (cc < cbest - tol || (cc <= cbest + tol && kc < kbest)) {
            best.swap(c);
            kbest = kc;
            cbest = cc;
        }
    }
    std::copy(best.begin(), best.end(), block_out);
    if (nblocks_out) *nblocks_out = kbest;
    if (cut_out) *cut_out = cbest;
    return CGGM_OK;
}

}  // namespace

extern "C" cggm_status cggm_partition_columns(int64_t q, int64_t m, const int32_t *ei,
                                              const int32_t *ej, const double *w,
                                              int64_t max_block, int32_t *block_out,
                                              int64_t *nblocks_out, double *cut_out)
{
    if (q < 0 || q > INT32_MAX || m < 0 || max_block < 1) return CGGM_EINVAL;
    if ((q > 0 && !block_out) || (m > 0 && (!ei || !ej))) return CGGM_EINVAL;
    std::vector<Edge> edges;
    edges.reserve((size_t)m);
    for (int64_t t = 0; t < m; t++) {
        if (ei[t] < 0 || ei[t] >= q || ej[t] < 0 || ej[t] >= q) return CGGM_EINVAL;
        const double wt = w ? w[t] : 1.0;
        if (!std::isfinite(wt) || wt < 0.0) return CGGM_EINVAL;
        edges.push_back({ei[t], ej[t], wt});
    }
    return partition_graph(q, edges, max_block, block_out, nblocks_out, cut_out);
}

extern "C" cggm_status cggm_partition_theta_columns(int64_t p, int64_t q, int64_t m,
                                                    const int32_t *ti, const int32_t *tj,
                                                    int64_t max_block, int32_t *block_out,
                                                    int64_t *nblocks_out,
                                                    int64_t *row_blocks_out)
{
    if (p < 0 || p > INT32_MAX || q < 0 || q > INT32_MAX || m < 0 || max_block < 1)
        return CGGM_EINVAL;
    if ((q > 0 && !block_out) || (m > 0 && (!ti || !tj))) return CGGM_EINVAL;
    // the active columns of every row (counting sort by row, then sorted and unique)
    std::vector<int64_t> rp(p + 1, 0);
    for (int64_t t = 0; t < m; t++) {
        if (ti[t] < 0 || ti[t] >= p || tj[t] < 0 || tj[t] >= q) return CGGM_EINVAL;
        rp[ti[t] + 1]++;
    }
    for (int64_t i = 0; i < p; i++) rp[i + 1] += rp[i];
    std::vector<int32_t> cols(m);
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    for (int64_t t = 0; t < m; t++) cols[fill[ti[t]]++] = tj[t];
    std::vector<int64_t> rlen(p, 0);
    std::vector<Edge> edges;
    for (int64_t i = 0; i < p; i++) {
        auto b = cols.begin() + rp[i], e = cols.begin() + rp[i + 1];
        std::sort(b, e);
        e = std::unique(b, e);
        const int64_t d = e - b;
        rlen[i] = d;
        if (d < 2) continue;
        if (d <= kCliqueMaxRow) {
            // every pair, each of weight 1/(d-1): the row adds d/2 in all
            const double wt = 1.0 / (double)(d - 1);
            for (int64_t a = 0; a < d; a++)
                for (int64_t c = a + 1; c < d; c++) edges.push_back({b[a], b[c], wt});
        } else {
            for (int64_t a = 0; a + 1 < d; a++) edges.push_back({b[a], b[a + 1], 1.0});
        }
    }
    const cggm_status st = partition_graph(q, edges, max_block, block_out, nblocks_out, nullptr);
    if (st != CGGM_OK) return st;
    if (row_blocks_out) {
        // sum over rows of the number of blocks the row's active entries fall in
        int64_t total = 0;
        std::vector<int32_t> seen;
        for (int64_t i = 0; i < p; i++) {
            seen.clear();
            for (int64_t t = rp[i]; t < rp[i] + rlen[i]; t++) seen.push_back(block_out[cols[t]]);
            std::sort(seen.begin(), seen.end());
            total += std::unique(seen.begin(), seen.end()) - seen.begin();
        }
        *row_blocks_out = total;
    }
    return CGGM_OK;
}

// Visiting order of the blocked passes of Algorithm 2 and the cache counts of Section 4.
// Lambda: each coordinate (i, j), i <= j, belongs to the block pair (z, r) of its indices'
// blocks, z <= r, with a the index in block z and b the other; the pass runs by (z, r),
// then a, then b.  It forms the Sigma columns of every block once (as block z) and those
// of block r again for each off-diagonal pair (z, r) holding a coordinate (a miss).
// Theta: by the block r of j, then row i, then j; Sigma is formed once (q columns) and a
// row of S_xx for each non-empty (i, C_r) (a miss).
extern "C" cggm_status cggm_block_order(int kind, int64_t q, int64_t m, const int32_t *ci,
                                        const int32_t *cj, const int32_t *block,
                                        int32_t *order_out, int64_t *columns_out,
                                        int64_t *misses_out)
{
    if ((kind != 0 && kind != 1) || q < 0 || q > INT32_MAX || m < 0 || m > INT32_MAX)
        return CGGM_EINVAL;
    if ((q > 0 && !block) || (m > 0 && (!ci || !cj || !order_out))) return CGGM_EINVAL;
    int32_t nb = 0;
    for (int64_t v = 0; v < q; v++) {
        if (block[v] < 0 || block[v] >= q) return CGGM_EINVAL;
        nb = std::max(nb, block[v] + 1);
    }
    std::vector<int64_t> size(nb, 0);
    for (int64_t v = 0; v < q; v++) size[block[v]]++;
    for (int32_t z = 0; z < nb; z++)
        if (size[z] == 0) return CGGM_EINVAL;  // ids must be 0..k-1 with no empty block
    struct Key {
        int32_t k0, k1, k2, k3;
        int32_t pos;
    };
    std::vector<Key> keys((size_t)m);
    for (int64_t t = 0; t < m; t++) {
        const int32_t i = ci[t], j = cj[t];
        if (kind == 0) {
            if (i < 0 || j < i || j >= q) return CGGM_EINVAL;
            const bool swap = block[i] > block[j];
            const int32_t a = swap ? j : i, b = swap ? i : j;
            keys[t] = {block[a], block[b], a, b, (int32_t)t};
        } else {
            if (i < 0 || j < 0 || j >= q) return CGGM_EINVAL;
            keys[t] = {block[j], i, j, 0, (int32_t)t};
        }
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) {
        if (x.k0 != y.k0) return x.k0 < y.k0;
        if (x.k1 != y.k1) return x.k1 < y.k1;
        if (x.k2 != y.k2) return x.k2 < y.k2;
        return x.k3 < y.k3;
    });
    int64_t columns = 0, misses = 0;
    if (kind == 0) {
        columns = q;  // every block once, as block z
        for (int64_t t = 0; t < m; t++) {
            const Key &k = keys[t];
            const bool first = t == 0 || keys[t - 1].k0 != k.k0 || keys[t - 1].k1 != k.k1;
            if (first && k.k0 != k.k1) {
                misses++;
                columns += size[k.k1];
            }
        }
    } else {
        columns = q;
        for (int64_t t = 0; t < m; t++) {
            const Key &k = keys[t];
            if (t == 0 || keys[t - 1].k0 != k.k0 || keys[t - 1].k1 != k.k1) misses++;
        }
    }
    for (int64_t t = 0; t < m; t++) order_out[t] = keys[t].pos;
    if (columns_out) *columns_out = columns;
    if (misses_out) *misses_out = misses;
    return CGGM_OK;
}

// Section 4's rule for the number of blocks: the smallest k whose blocks' columns fit in the
// budget.  Lambda (Section 4.1) holds 2q/k columns of Sigma and 2q/k of Psi, q entries each,
// so 4 q ceil(q/k) entries; Theta (Section 4.2) holds q/k columns of Sigma, q ceil(q/k).
extern "C" cggm_status cggm_block_count(int kind, int64_t q, int64_t bytes_per_value,
                                        int64_t budget_bytes, int64_t *k_out,
                                        int64_t *max_block_out)
{
    if ((kind != 0 && kind != 1) || q < 1 || bytes_per_value < 1 || budget_bytes < 1 ||
        !k_out || !max_block_out)
        return CGGM_EINVAL;
    const int64_t factor = kind == 0 ? 4 : 1;  // held columns per block column
    // entries one block column costs, q each; a budget below one column is too small
    const double per_col = (double)factor * (double)q * (double)bytes_per_value;
    const int64_t cols = (int64_t)std::floor((double)budget_bytes / per_col);
    if (cols < 1) return CGGM_ENOMEM;
    const int64_t max_block = std::min(cols, q);
    *k_out = (q + max_block - 1) / max_block;
    *max_block_out = (q + *k_out - 1) / *k_out;  // blocks of equal size up to one
    return CGGM_OK;
}
