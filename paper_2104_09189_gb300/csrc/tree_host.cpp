// tree_host.cpp -- the spanning tree of strategy (c) (Sec. 3).
//
// Strategy (c) starts the walk of node i at the triangle just located for a
// neighbouring node, its parent P_i in a spanning tree of the mesh's node
// graph: the nodes are put in an order in which every node but the root
// comes after its parent (Sec. 3, Algorithm 1).  The tree is built once per
// numbering: breadth-first from the node nearest the centre of the square
// (the root the paper's experiments use, Sec. 4), neighbours taken in the
// order of the triangle list.  A breadth-first tree is shallow, and its
// levels are the parallel rounds the paper suggests: all nodes whose parents
// are on the previous level are located together.
#include <cmath>
#include <vector>

#include "sl_internal.h"

namespace sl {

sl_status build_tree(const sl_mesh *m, std::vector<int32_t> &order, std::vector<int64_t> &level_off,
                     std::vector<int32_t> &parent)
{
    const int64_t N = m->N;
    // node graph of every problem (global ids), CSR over the triangle edges
    std::vector<int64_t> start(N + 1, 0);
    for (int32_t p = 0; p < m->n_problems; ++p)
        for (int64_t j = m->tri_off[p]; j < m->tri_off[p + 1]; ++j)
            for (int k = 0; k < 3; ++k) start[m->node_off[p] + m->tri[3 * j + k] + 1] += 2;
    for (int64_t i = 0; i < N; ++i) start[i + 1] += start[i];
    std::vector<int32_t> adj((size_t)start[N]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int32_t p = 0; p < m->n_problems; ++p) {
        const int64_t n0 = m->node_off[p];
        for (int64_t j = m->tri_off[p]; j < m->tri_off[p + 1]; ++j)
            for (int k = 0; k < 3; ++k) {
                const int64_t a = n0 + m->tri[3 * j + k];
                adj[(size_t)fill[a]++] = (int32_t)(n0 + m->tri[3 * j + (k + 1) % 3]);
                adj[(size_t)fill[a]++] = (int32_t)(n0 + m->tri[3 * j + (k + 2) % 3]);
            }
    }
    parent.assign((size_t)N, -1);
    std::vector<int32_t> level((size_t)N, -1);
    int32_t depth = 0;
    std::vector<int32_t> queue;
    queue.reserve((size_t)N);
    for (int32_t p = 0; p < m->n_problems; ++p) {
        const int64_t lo = m->node_off[p], hi = m->node_off[p + 1];
        if (hi <= lo) continue;
        int64_t root = lo;
        double best = 1e300;
        for (int64_t i = lo; i < hi; ++i) {
            const double dx = m->xy[2 * i] - 0.5, dy = m->xy[2 * i + 1] - 0.5, d = dx * dx + dy * dy;
            if (d < best) {
                best = d;
                root = i;
            }
        }
        queue.clear();
        queue.push_back((int32_t)root);
        parent[(size_t)root] = (int32_t)root;
        level[(size_t)root] = 0;
        for (size_t q = 0; q < queue.size(); ++q) {
            const int32_t u = queue[q];
            for (int64_t e = start[u]; e < start[u + 1]; ++e) {
                const int32_t v = adj[(size_t)e];
                if (level[(size_t)v] >= 0) continue;
                level[(size_t)v] = level[(size_t)u] + 1;
                parent[(size_t)v] = u;
                depth = level[(size_t)v] > depth ? level[(size_t)v] : depth;
                queue.push_back(v);
            }
        }
        if ((int64_t)queue.size() != hi - lo)
            return fail(SL_E_MESH, "strategy (c): the node graph of problem " + std::to_string(p) + " is not connected");
    }
    // all problems' level k together, ascending node index within a level
    level_off.assign((size_t)depth + 2, 0);
    for (int64_t i = 0; i < N; ++i) ++level_off[(size_t)level[(size_t)i] + 1];
    for (int32_t k = 0; k <= depth; ++k) level_off[(size_t)k + 1] += level_off[(size_t)k];
    order.assign((size_t)N, 0);
    std::vector<int64_t> pos(level_off.begin(), level_off.end() - 1);
    for (int64_t i = 0; i < N; ++i) order[(size_t)pos[(size_t)level[(size_t)i]]++] = (int32_t)i;
    return SL_OK;
}

}  // namespace sl
