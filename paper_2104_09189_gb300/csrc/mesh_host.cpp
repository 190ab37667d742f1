// mesh_host.cpp -- host side of the mesh handle: validation, neighbour
// lists, the initial start-triangle list T^0 and space-filling-curve
// renumbering.  The data structures are those of the paper's Sec. 3 (node
// list V, triangle list T, neighbour list N, start list T^0), 0-based.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>

#include "predicates.cuh"
#include "sl_internal.h"

namespace sl {

static thread_local std::string g_err;

sl_status fail(sl_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

// Run f(lo, hi) over [0, n) on the hardware threads.
template <class F>
static void parallel_for(int64_t n, F f)
{
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::max(1u, std::min(hw ? hw : 1u, 64u));
    if (n < 65536) nt = 1;
    if (nt == 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int k = 0; k < nt; ++k) {
        int64_t lo = n * k / nt, hi = n * (k + 1) / nt;
        th.emplace_back([=] { f(lo, hi); });
    }
    for (auto &t : th) t.join();
}

// Vertex -> incident triangles (local indices, ascending triangle index).
struct Incidence {
    std::vector<int64_t> start;
    std::vector<int32_t> items;
};

static void build_incidence(int64_t n, int64_t nt, const int32_t *tri, Incidence &inc)
{
    inc.start.assign(n + 1, 0);
    for (int64_t q = 0; q < 3 * nt; ++q) inc.start[tri[q] + 1]++;
    for (int64_t v = 0; v < n; ++v) inc.start[v + 1] += inc.start[v];
    inc.items.resize(3 * nt);
    std::vector<int64_t> fill(inc.start.begin(), inc.start.end() - 1);
    for (int64_t j = 0; j < nt; ++j)
        for (int k = 0; k < 3; ++k) inc.items[fill[tri[3 * j + k]]++] = (int32_t)j;
}

sl_status build_and_validate(sl_mesh *m, const int32_t *nbr_in)
{
    const int64_t N = m->N, Nt = m->Nt;
    // coordinates
    for (int64_t i = 0; i < 2 * N; ++i) {
        double v = m->xy[i];
        if (!(v >= 0.0 && v <= 1.0))
            return fail(SL_E_MESH, "node " + std::to_string(i / 2) + " lies outside [0,1]^2 or is not finite");
    }
    m->nbr.assign(3 * Nt, -1);
    m->t0.assign(N, -1);
    m->cells.assign(m->n_problems, 1);
    for (int32_t p = 0; p < m->n_problems; ++p) {
        const int64_t n0 = m->node_off[p], n = m->node_off[p + 1] - n0;
        const int64_t j0 = m->tri_off[p], nt = m->tri_off[p + 1] - j0;
        if (n < 3 || nt < 1) return fail(SL_E_MESH, "problem " + std::to_string(p) + " has fewer than 3 nodes or no triangle");
        const int32_t *tri = m->tri.data() + 3 * j0;
        const double *xy = m->xy.data() + 2 * n0;
        int32_t *nbr = m->nbr.data() + 3 * j0;
        for (int64_t q = 0; q < 3 * nt; ++q)
            if (tri[q] < 0 || tri[q] >= n)
                return fail(SL_E_MESH, "problem " + std::to_string(p) + ": vertex index out of range in triangle " +
                                           std::to_string(q / 3));
        // orientation (exact) and area
        std::atomic<int64_t> bad_ccw{-1};
        std::mutex mu;
        double area2 = 0.0;
        parallel_for(nt, [&](int64_t lo, int64_t hi) {
            double s = 0.0;
            for (int64_t j = lo; j < hi; ++j) {
                const int32_t *t = tri + 3 * j;
                double ax = xy[2 * t[0]], ay = xy[2 * t[0] + 1], bx = xy[2 * t[1]], by = xy[2 * t[1] + 1];
                double cx = xy[2 * t[2]], cy = xy[2 * t[2] + 1];
                slp::OrientResult r = slp::orient(ax, ay, bx, by, cx, cy);
                if (r.sign <= 0) bad_ccw.store(j);
                s += r.det;
            }
            std::lock_guard<std::mutex> g(mu);
            area2 += s;
        });
        if (bad_ccw.load() >= 0)
            return fail(SL_E_MESH, "problem " + std::to_string(p) + ": triangle " + std::to_string(bad_ccw.load()) +
                                       " is not strictly counter-clockwise");
        if (std::fabs(0.5 * area2 - 1.0) > 1e-9)
            return fail(SL_E_MESH, "problem " + std::to_string(p) + ": total triangle area is " +
                                       std::to_string(0.5 * area2) + ", not 1 (mesh does not cover the square)");
        Incidence inc;
        build_incidence(n, nt, tri, inc);
        for (int64_t v = 0; v < n; ++v)
            if (inc.start[v + 1] == inc.start[v])
                return fail(SL_E_MESH, "problem " + std::to_string(p) + ": node " + std::to_string(v) + " is in no triangle");
        // neighbours: the triangle across the edge opposite vertex k
        std::atomic<int> err{0};
        std::atomic<int64_t> err_j{-1};
        parallel_for(nt, [&](int64_t lo, int64_t hi) {
            for (int64_t j = lo; j < hi; ++j) {
                const int32_t *t = tri + 3 * j;
                for (int k = 0; k < 3; ++k) {
                    int32_t a = t[(k + 1) % 3], b = t[(k + 2) % 3];   // directed edge a -> b
                    int32_t found = -1;
                    int count = 0;
                    for (int64_t q = inc.start[a]; q < inc.start[a + 1]; ++q) {
                        int32_t o = inc.items[q];
                        if (o == j) continue;
                        const int32_t *u = tri + 3 * (int64_t)o;
                        for (int r = 0; r < 3; ++r) {
                            if (u[r] == b && u[(r + 1) % 3] == a) { found = o; count++; }
                            if (u[r] == a && u[(r + 1) % 3] == b) { err.store(1); err_j.store(j); }
                        }
                    }
                    if (count > 1) { err.store(2); err_j.store(j); }
                    nbr[3 * j + k] = found;
                    if (found < 0) {
                        double xa = xy[2 * a], ya = xy[2 * a + 1], xb = xy[2 * b], yb = xy[2 * b + 1];
                        bool on = (xa == 0.0 && xb == 0.0) || (xa == 1.0 && xb == 1.0) || (ya == 0.0 && yb == 0.0) ||
                                  (ya == 1.0 && yb == 1.0);
                        if (!on) { err.store(3); err_j.store(j); }
                    }
                }
            }
        });
        static const char *what[] = {"", "two triangles share an edge with the same orientation",
                                     "an edge is shared by more than two triangles",
                                     "a boundary edge does not lie on a side of the square"};
        if (err.load())
            return fail(SL_E_MESH, "problem " + std::to_string(p) + ": " + what[err.load()] + " (triangle " +
                                       std::to_string(err_j.load()) + ")");
        if (nbr_in) {
            const int32_t *given = nbr_in + 3 * j0;
            for (int64_t q = 0; q < 3 * nt; ++q)
                if (given[q] != nbr[q])
                    return fail(SL_E_MESH, "problem " + std::to_string(p) + ": supplied neighbour list is inconsistent at triangle " +
                                               std::to_string(q / 3));
        }
        // T^0: a random incident triangle per node (Sec. 3), reproducible from
        // (seed, global node index) and independent of later renumbering.
        for (int64_t v = 0; v < n; ++v) {
            int64_t deg = inc.start[v + 1] - inc.start[v];
            uint64_t h = splitmix_at(m->seed, (uint64_t)(n0 + v));
            m->t0[n0 + v] = (int32_t)(j0 + inc.items[inc.start[v] + (int64_t)(h % (uint64_t)deg)]);
        }
        m->cells[p] = (int32_t)std::max(1.0, std::floor(std::sqrt((double)nt / 2.0) + 0.5));
    }
    m->t0_init = m->t0;
    return SL_OK;
}

// ---------------------------------------------------------------------------
// Space-filling-curve renumbering

static uint32_t quantize(double v)
{
    double s = v * 65536.0;
    if (!(s > 0.0)) return 0;
    if (s >= 65535.0) return 65535;
    return (uint32_t)s;
}

// Position along the Hilbert curve of cell (x, y) of a 2^16 x 2^16 grid.
static uint64_t hilbert_key(uint32_t x, uint32_t y)
{
    uint64_t d = 0;
    for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1u : 0u;
        uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {                       // rotate the quadrant
            if (rx == 1) {
                x = 0xFFFFu - x;
                y = 0xFFFFu - y;
            }
            uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

static uint64_t morton_key(uint32_t x, uint32_t y)
{
    uint64_t d = 0;
    for (int b = 15; b >= 0; --b) d = (d << 2) | ((uint64_t)((y >> b) & 1u) << 1) | ((x >> b) & 1u);
    return d;
}

// Renumber every problem by explicit permutations, new -> old and local to
// the problem (node_perm: N entries, tri_perm: Nt entries): coordinates,
// triangles, neighbours and both T^0 lists follow.
sl_status permute_host(sl_mesh *m, const int32_t *node_perm, const int32_t *tri_perm)
{
    std::vector<double> xy2(m->xy.size());
    std::vector<int32_t> tri2(m->tri.size()), nbr2(m->nbr.size()), t02(m->t0.size()), t0i2(m->t0.size());
    for (int32_t p = 0; p < m->n_problems; ++p) {
        const int64_t n0 = m->node_off[p], n = m->node_off[p + 1] - n0;
        const int64_t j0 = m->tri_off[p], nt = m->tri_off[p + 1] - j0;
        const double *xy = m->xy.data() + 2 * n0;
        const int32_t *tri = m->tri.data() + 3 * j0;
        std::vector<int32_t> inv_n(n, -1), inv_t(nt, -1);
        for (int64_t a = 0; a < n; ++a) {
            const int32_t old = node_perm[n0 + a];
            if (old < 0 || old >= n || inv_n[old] >= 0) return fail(SL_E_ARG, "not a permutation of a problem's nodes");
            inv_n[old] = (int32_t)a;
        }
        for (int64_t a = 0; a < nt; ++a) {
            const int32_t old = tri_perm[j0 + a];
            if (old < 0 || old >= nt || inv_t[old] >= 0) return fail(SL_E_ARG, "not a permutation of a problem's triangles");
            inv_t[old] = (int32_t)a;
        }
        for (int64_t a = 0; a < n; ++a) {
            const int64_t old = node_perm[n0 + a];
            xy2[2 * (n0 + a)] = xy[2 * old];
            xy2[2 * (n0 + a) + 1] = xy[2 * old + 1];
            t02[n0 + a] = (int32_t)j0 + inv_t[m->t0[n0 + old] - (int32_t)j0];
            t0i2[n0 + a] = (int32_t)j0 + inv_t[m->t0_init[n0 + old] - (int32_t)j0];
        }
        for (int64_t a = 0; a < nt; ++a) {
            const int64_t old = tri_perm[j0 + a];
            for (int k = 0; k < 3; ++k) {
                tri2[3 * (j0 + a) + k] = inv_n[tri[3 * old + k]];
                const int32_t nb = m->nbr[3 * (j0 + old) + k];
                nbr2[3 * (j0 + a) + k] = nb < 0 ? -1 : inv_t[nb];
            }
        }
    }
    m->xy.swap(xy2);
    m->tri.swap(tri2);
    m->nbr.swap(nbr2);
    m->t0.swap(t02);
    m->t0_init.swap(t0i2);
    return SL_OK;
}

sl_status reorder_host(sl_mesh *m, int32_t curve, int32_t *node_perm, int32_t *tri_perm)
{
    std::vector<int32_t> np(m->N), tp(m->Nt);
    for (int32_t p = 0; p < m->n_problems; ++p) {
        const int64_t n0 = m->node_off[p], n = m->node_off[p + 1] - n0;
        const int64_t j0 = m->tri_off[p], nt = m->tri_off[p + 1] - j0;
        for (int64_t i = 0; i < n; ++i) np[n0 + i] = (int32_t)i;
        for (int64_t j = 0; j < nt; ++j) tp[j0 + j] = (int32_t)j;
        if (curve == SL_CURVE_NONE) continue;
        auto key = [curve](double x, double y) {
            uint32_t qx = quantize(x), qy = quantize(y);
            return curve == SL_CURVE_HILBERT ? hilbert_key(qx, qy) : morton_key(qx, qy);
        };
        const double *xy = m->xy.data() + 2 * n0;
        const int32_t *tri = m->tri.data() + 3 * j0;
        std::vector<std::pair<uint64_t, int32_t>> nk(n), tk(nt);
        parallel_for(n, [&](int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; ++i) nk[i] = {key(xy[2 * i], xy[2 * i + 1]), (int32_t)i};
        });
        parallel_for(nt, [&](int64_t lo, int64_t hi) {
            for (int64_t j = lo; j < hi; ++j) {
                const int32_t *t = tri + 3 * j;
                double cx = (xy[2 * t[0]] + xy[2 * t[1]] + xy[2 * t[2]]) / 3.0;
                double cy = (xy[2 * t[0] + 1] + xy[2 * t[1] + 1] + xy[2 * t[2] + 1]) / 3.0;
                tk[j] = {key(cx, cy), (int32_t)j};
            }
        });
        std::sort(nk.begin(), nk.end());
        std::sort(tk.begin(), tk.end());
        for (int64_t a = 0; a < n; ++a) np[n0 + a] = nk[a].second;
        for (int64_t a = 0; a < nt; ++a) tp[j0 + a] = tk[a].second;
    }
    if (node_perm) std::copy(np.begin(), np.end(), node_perm);
    if (tri_perm) std::copy(tp.begin(), tp.end(), tri_perm);
    if (curve == SL_CURVE_NONE) return SL_OK;
    return permute_host(m, np.data(), tp.data());
}

}  // namespace sl

// ---------------------------------------------------------------------------
// Host-only entry points

extern "C" const char *sl_last_error(void) { return sl::g_err.c_str(); }

static sl_status check_args(int32_t n_problems, const int64_t *node_off, const int64_t *tri_off, const double *xy,
                           const int32_t *tri)
{
    if (n_problems < 1 || !node_off || !tri_off || !xy || !tri)
        return sl::fail(SL_E_ARG, "n_problems < 1 or a required pointer is NULL");
    if (node_off[0] != 0 || tri_off[0] != 0) return sl::fail(SL_E_ARG, "offsets must start at 0");
    for (int32_t p = 0; p < n_problems; ++p)
        if (node_off[p + 1] < node_off[p] || tri_off[p + 1] < tri_off[p])
            return sl::fail(SL_E_ARG, "offsets must be non-decreasing");
    if (node_off[n_problems] >= ((int64_t)1 << 31))
        return sl::fail(SL_E_ARG, "more than 2^31-1 nodes");
    // the fast kernels number half-edges 3 t + k in int32
    if (3 * tri_off[n_problems] >= ((int64_t)1 << 31))
        return sl::fail(SL_E_ARG, "more than 715827882 triangles");
    return SL_OK;
}

// A host-only handle filled and validated (no device state).
static sl_status make_host_mesh(int32_t n_problems, const int64_t *node_off, const int64_t *tri_off,
                                const double *xy, const int32_t *tri, const int32_t *nbr, int32_t precision,
                                uint64_t seed, sl_mesh **out)
{
    *out = nullptr;
    sl_status st = check_args(n_problems, node_off, tri_off, xy, tri);
    if (st != SL_OK) return st;
    sl_mesh *m = new (std::nothrow) sl_mesh();
    if (!m) return sl::fail(SL_E_NOMEM, "out of host memory");
    try {
        m->n_problems = n_problems;
        m->node_off.assign(node_off, node_off + n_problems + 1);
        m->tri_off.assign(tri_off, tri_off + n_problems + 1);
        m->N = node_off[n_problems];
        m->Nt = tri_off[n_problems];
        m->precision = precision;
        m->seed = seed;
        m->xy.assign(xy, xy + 2 * m->N);
        m->tri.assign(tri, tri + 3 * m->Nt);
    } catch (...) {
        delete m;
        return sl::fail(SL_E_NOMEM, "out of host memory");
    }
    if (precision == SL_FP32)   // the mesh the FP32 path sees: coordinates rounded to float
        for (double &v : m->xy) v = (double)(float)v;
    st = sl::build_and_validate(m, nbr);
    if (st != SL_OK) {
        delete m;
        return st;
    }
    *out = m;
    return SL_OK;
}

extern "C" sl_status sl_mesh_validate(int32_t n_problems, const int64_t *node_off, const int64_t *tri_off,
                                      const double *xy, const int32_t *tri, const int32_t *nbr, uint64_t seed,
                                      int32_t *nbr_out, int32_t *t0_out)
{
    sl_mesh *m = nullptr;
    sl_status st = make_host_mesh(n_problems, node_off, tri_off, xy, tri, nbr, SL_FP64, seed, &m);
    if (st != SL_OK) return st;
    if (nbr_out) std::memcpy(nbr_out, m->nbr.data(), sizeof(int32_t) * m->nbr.size());
    if (t0_out)
        for (int32_t p = 0; p < m->n_problems; ++p)
            for (int64_t i = m->node_off[p]; i < m->node_off[p + 1]; ++i) t0_out[i] = m->t0[i] - (int32_t)m->tri_off[p];
    delete m;
    return SL_OK;
}

extern "C" sl_status sl_mesh_create(int32_t n_problems, const int64_t *node_off, const int64_t *tri_off,
                                    const double *xy, const int32_t *tri, const int32_t *nbr, int32_t precision,
                                    uint64_t seed, sl_mesh **out)
{
    if (!out) return sl::fail(SL_E_ARG, "sl_mesh_create: out is NULL");
    *out = nullptr;
    if (precision != SL_FP64 && precision != SL_FP32) return sl::fail(SL_E_ARG, "sl_mesh_create: unknown precision");
    sl_mesh *m = nullptr;
    sl_status st = make_host_mesh(n_problems, node_off, tri_off, xy, tri, nbr, precision, seed, &m);
    if (st != SL_OK) return st;
    if (st == SL_OK) st = sl::upload(m);
    if (st != SL_OK) {
        sl::free_device(m);
        delete m;
        return st;
    }
    *out = m;
    return SL_OK;
}

extern "C" sl_status sl_mesh_info(const sl_mesh *m, int64_t *n_nodes, int64_t *n_tri, int32_t *n_problems,
                                  int32_t *precision)
{
    if (!m) return sl::fail(SL_E_ARG, "sl_mesh_info: mesh is NULL");
    if (n_nodes) *n_nodes = m->N;
    if (n_tri) *n_tri = m->Nt;
    if (n_problems) *n_problems = m->n_problems;
    if (precision) *precision = m->precision;
    return SL_OK;
}

extern "C" sl_status sl_mesh_export(const sl_mesh *m, double *xy, int32_t *tri, int32_t *nbr)
{
    if (!m) return sl::fail(SL_E_ARG, "sl_mesh_export: mesh is NULL");
    if (xy) std::memcpy(xy, m->xy.data(), sizeof(double) * m->xy.size());
    if (tri) std::memcpy(tri, m->tri.data(), sizeof(int32_t) * m->tri.size());
    if (nbr) std::memcpy(nbr, m->nbr.data(), sizeof(int32_t) * m->nbr.size());
    return SL_OK;
}

// The structured Courant grid of Sec. 4: one problem of M x M square cells
// of [0,1]^2, each split into its upper triangle (l,m), (l+1,m+1), (l,m+1)
// and its lower triangle (l,m), (l+1,m), (l+1,m+1).  Fills slot_tri[2 (M m +
// l) + (upper ? 0 : 1)] with the current index of that triangle, identifying
// every triangle by its vertices (any numbering), or fails.
static sl_status courant_slots(const sl_mesh *m, int32_t &M, std::vector<int32_t> &slot_tri)
{
    if (m->n_problems != 1) return sl::fail(SL_E_ARG, "direct location needs a single-problem mesh");
    M = m->cells.empty() ? 0 : m->cells[0];
    if (M < 1 || m->Nt != 2 * (int64_t)M * M || m->N != (int64_t)(M + 1) * (M + 1))
        return sl::fail(SL_E_ARG, "direct location: the mesh is not a structured Courant grid (sizes)");
    slot_tri.assign((size_t)2 * M * M, -1);
    auto grid = [&](int32_t v, int64_t &gi, int64_t &gj) {
        const double gx = m->xy[2 * (size_t)v] * M, gy = m->xy[2 * (size_t)v + 1] * M;
        gi = std::llround(gx);
        gj = std::llround(gy);
        return std::fabs(gx - (double)gi) <= 1e-3 && std::fabs(gy - (double)gj) <= 1e-3;   // float-rounded meshes too
    };
    for (int64_t t = 0; t < m->Nt; ++t) {
        int64_t gi[3], gj[3];
        for (int k = 0; k < 3; ++k)
            if (!grid(m->tri[3 * t + k], gi[k], gj[k]))
                return sl::fail(SL_E_ARG, "direct location: a node is not a grid point");
        const int64_t l = std::min(std::min(gi[0], gi[1]), gi[2]), mm = std::min(std::min(gj[0], gj[1]), gj[2]);
        if (l < 0 || mm < 0 || l >= M || mm >= M) return sl::fail(SL_E_ARG, "direct location: bad cell");
        // upper: the corner (l+1, m) is missing; lower: the corner (l, m+1)
        bool has10 = false, has01 = false, has00 = false, has11 = false;
        for (int k = 0; k < 3; ++k) {
            const int64_t di = gi[k] - l, dj = gj[k] - mm;
            has00 |= di == 0 && dj == 0;
            has11 |= di == 1 && dj == 1;
            has10 |= di == 1 && dj == 0;
            has01 |= di == 0 && dj == 1;
        }
        if (!(has00 && has11 && (has10 != has01)))
            return sl::fail(SL_E_ARG, "direct location: a triangle is not half of a grid cell split along (l,m)-(l+1,m+1)");
        const size_t slot = 2 * (size_t)(M * mm + l) + (has01 ? 0 : 1);
        if (slot_tri[slot] >= 0) return sl::fail(SL_E_ARG, "direct location: two triangles in one half cell");
        slot_tri[slot] = (int32_t)t;
    }
    return SL_OK;
}

extern "C" sl_status sl_mesh_get_option(const sl_mesh *m, int32_t option, int64_t *value)
{
    if (!m || !value) return sl::fail(SL_E_ARG, "sl_mesh_get_option: NULL argument");
    switch (option) {
    case SL_OPT_STATS: *value = m->opt_stats; break;
    case SL_OPT_WALK_CAP: *value = m->opt_walk_cap; break;
    case SL_OPT_KERNEL: *value = m->opt_kernel; break;
    case SL_OPT_BLOCK: *value = m->opt_block; break;
    case SL_OPT_CONFIG: *value = m->opt_config; break;
    case SL_OPT_CONFIG_FIRST: *value = m->opt_config_first; break;
    case SL_OPT_STRATEGY: *value = m->opt_strategy; break;
    case SL_OPT_OUTSIDE: *value = m->opt_outside; break;
    case SL_OPT_SPLIT: *value = m->opt_split; break;
    case SL_OPT_ASYNC: *value = m->opt_async; break;
    case SL_OPT_PRECISE: *value = m->opt_precise; break;
    case SL_OPT_RECORDS: *value = m->d.he8 ? 8 : 16; break;
    case SL_OPT_L2_WINDOW: *value = m->opt_l2; break;
    case SL_OPT_PDL: *value = m->opt_pdl; break;
    default: return sl::fail(SL_E_ARG, "unknown option");
    }
    return SL_OK;
}

extern "C" sl_status sl_mesh_set_option(sl_mesh *m, int32_t option, int64_t value)
{
    if (!m) return sl::fail(SL_E_ARG, "sl_mesh_set_option: mesh is NULL");
    switch (option) {
    case SL_OPT_STATS: m->opt_stats = value ? 1 : 0; break;
    case SL_OPT_WALK_CAP:
        if (value < 0 || value > (1 << 30)) return sl::fail(SL_E_ARG, "walk cap out of range");
        m->opt_walk_cap = (int32_t)value;
        break;
    case SL_OPT_KERNEL:
        if (value < 0 || value > 2) return sl::fail(SL_E_ARG, "unknown kernel selector");
        m->opt_kernel = (int32_t)value;
        break;
    case SL_OPT_BLOCK:
        if (value != 0 && (value < 32 || value > 1024 || value % 32)) return sl::fail(SL_E_ARG, "block size must be 0 or a multiple of 32 in [32, 1024]");
        m->opt_block = (int32_t)value;
        break;
    case SL_OPT_CONFIG:
        if (value < 0 || value > 5) return sl::fail(SL_E_ARG, "launch configuration must be 0..5");
        m->opt_config = (int32_t)value;
        break;
    case SL_OPT_CONFIG_FIRST:
        if (value < 0 || value > 5) return sl::fail(SL_E_ARG, "launch configuration must be 0..5");
        m->opt_config_first = (int32_t)value;
        break;
    case SL_OPT_STRATEGY: {
        if (value < 0 || value > 3) return sl::fail(SL_E_ARG, "strategy must be 0 (b), 1 (a), 2 (direct) or 3 (c)");
        if (value == 3) {
            std::vector<int32_t> order, parent;
            std::vector<int64_t> level_off;
            sl_status st = sl::build_tree(m, order, level_off, parent);
            if (st == SL_OK) st = sl::upload_tree(m, order, parent);
            if (st != SL_OK) return st;
            m->tree_level_off = level_off;
        }
        if (value == 2) {
            int32_t M = 0;
            std::vector<int32_t> slots;
            sl_status st = courant_slots(m, M, slots);
            if (st == SL_OK) st = sl::upload_grid_table(m, slots);
            if (st != SL_OK) return st;
            m->grid_M = M;
        }
        m->opt_strategy = (int32_t)value;
        sl_status st = sl::reset_t0_sync(m);
        if (st != SL_OK) return st;
        break;
    }
    case SL_OPT_SPLIT:
        if (value != 0 && value != 1) return sl::fail(SL_E_ARG, "split must be 0 or 1");
        m->opt_split = (int32_t)value;
        break;
    case SL_OPT_OUTSIDE:
        if (value != 0 && value != 1) return sl::fail(SL_E_ARG, "outside mode must be 0 (clip) or 1 (exclude)");
        m->opt_outside = (int32_t)value;
        break;
    case SL_OPT_RECORDS: {
        if (value != 0 && value != 1) return sl::fail(SL_E_ARG, "records must be 0 (16 bytes) or 1 (compact where they fit)");
        m->opt_records = (int32_t)value;
        const sl_status st = sl::build_walk_records(m);
        if (st != SL_OK) return st;
        break;
    }
    case SL_OPT_L2_WINDOW:
        if (value != 0 && value != 1) return sl::fail(SL_E_ARG, "L2 window must be 0 or 1");
        m->opt_l2 = (int32_t)value;
        if (!value) sl::release_l2_window(m);
        break;
    case SL_OPT_PDL:
        if (value != 0 && value != 1) return sl::fail(SL_E_ARG, "pdl must be 0 or 1");
        m->opt_pdl = (int32_t)value;
        break;
    case SL_OPT_PRECISE:
        if (value < 0 || value > (1 << 30)) return sl::fail(SL_E_ARG, "precise gradient bound out of range");
        m->opt_precise = (int32_t)value;
        break;
    case SL_OPT_ASYNC:
        if (value != 0 && value != 1) return sl::fail(SL_E_ARG, "async must be 0 or 1");
        m->opt_async = (int32_t)value;
        return SL_OK;   // the recorded launches do not depend on it
    default: return sl::fail(SL_E_ARG, "unknown option");
    }
    m->graph.valid = false;   // recorded launches may depend on options
    return SL_OK;
}
