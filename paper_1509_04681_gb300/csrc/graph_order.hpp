// Breadth-first orders of an undirected graph in CSR form, shared by the column partition
// and the symbolic Cholesky (host code).  G is any type with `ptr` (n + 1 offsets), `adj`
// (neighbour lists, no self loops) and `degree(v)`.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace cggm {
namespace graph {

// Breadth-first search over the component of `root`: `order` receives the visit order and
// `level` the distance from the root (entries of unvisited vertices must be -1 on entry).
// With `by_degree`, each vertex's unvisited neighbours are taken by ascending (degree,
// index); otherwise in adjacency order.
template <class G>
void bfs(const G &g, int32_t root, std::vector<int32_t> &order, std::vector<int32_t> &level,
         bool by_degree)
{
    order.clear();
    order.push_back(root);
    level[root] = 0;
    std::vector<int32_t> nb;
    for (size_t h = 0; h < order.size(); h++) {
        const int32_t v = order[h];
        nb.clear();
        for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; t++)
            if (level[g.adj[t]] < 0) nb.push_back(g.adj[t]);
        if (by_degree)
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                const int64_t da = g.degree(a), db = g.degree(b);
                return da != db ? da < db : a < b;
            });
        for (int32_t u : nb)
            if (level[u] < 0) {
                level[u] = level[v] + 1;
                order.push_back(u);
            }
    }
}

// Cuthill-McKee order of the component of `seed`, from a pseudo-peripheral vertex: start at
// the component's vertex of least degree (ties: lower index), and move to the least-degree
// vertex of the last level while that lengthens the search (at most four searches).  On
// return `level` holds the final search's levels for the component (>= 0), so a caller
// looping over seeds can skip vertices already placed.
template <class G>
std::vector<int32_t> cuthill_mckee(const G &g, int32_t seed, std::vector<int32_t> &level)
{
    constexpr int kSweeps = 4;
    std::vector<int32_t> order;
    bfs(g, seed, order, level, false);
    int32_t root = seed;
    for (int32_t v : order)
        if (g.degree(v) < g.degree(root) || (g.degree(v) == g.degree(root) && v < root)) root = v;
    int32_t depth = -1;
    for (int s = 0; s < kSweeps; s++) {
        for (int32_t v : order) level[v] = -1;
        bfs(g, root, order, level, false);
        const int32_t d = level[order.back()];
        if (d <= depth) break;
        depth = d;
        int32_t next = order.back();
        for (int32_t v : order)
            if (level[v] == d &&
                (g.degree(v) < g.degree(next) || (g.degree(v) == g.degree(next) && v < next)))
                next = v;
        root = next;
    }
    for (int32_t v : order) level[v] = -1;
    bfs(g, root, order, level, true);
    return order;
}

}  // namespace graph
}  // namespace cggm
