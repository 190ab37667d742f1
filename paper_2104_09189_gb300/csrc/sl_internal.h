// sl_internal.h -- the mesh handle and helpers shared by the library's
// translation units (host code + CUDA code of the product library only).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sl.h"

namespace sl {

// Set the thread-local error message and return the status.
sl_status fail(sl_status st, const std::string &msg);

// SplitMix64 (Steele, Lea & Flood 2014): the output mix applied to a counter.
inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
inline uint64_t splitmix_at(uint64_t seed, uint64_t i)
{
    const uint64_t g = 0x9E3779B97F4A7C15ULL;
    return mix64(mix64(seed * g) + (i + 1) * g);
}

struct DeviceMesh {
    void *xy = nullptr;               // double2[N] (FP64) or float2[N] (FP32)
    int32_t *tv[3] = {nullptr, nullptr, nullptr};   // vertex k of triangle j (global node index)
    int32_t *tn[3] = {nullptr, nullptr, nullptr};   // neighbour across edge opposite vertex k (global);
                                                    // boundary: -1 - side (0: x=0, 1: x=1, 2: y=0, 3: y=1)
    int32_t *t0 = nullptr;            // start / last foot triangle of node i (global)
    int32_t *t0_init = nullptr;       // the initial start triangles (global)
    void *t0v = nullptr;              // int4 (T^0, its vertex ids) per node
    void *grid_t0v = nullptr;         // int4 start state per structured-grid triangle (strategy 2)
    int32_t *queue = nullptr;         // split steps: nodes left to the finish pass (N)
    uint32_t *queue_count = nullptr;
    int32_t *tree_order = nullptr;    // strategy (c): nodes by spanning-tree level (N)
    int32_t *tree_parent = nullptr;   // strategy (c): parent of every node (N; the root its own)
    int64_t *node_off = nullptr;      // n_problems + 1
    void *chunk_prob = nullptr;       // int2 per 128 nodes: problems of the first and last node (more
                                      // than one problem)
    uint32_t *status = nullptr;       // [0] = OR of (1 << sl_status); others reserved
    unsigned long long *stats = nullptr;   // 8 counters (sl_stats order)
    void *probs = nullptr;            // per-problem step data (device)
    size_t probs_bytes = 0;
    void *fprobs = nullptr;           // per-problem step constants of the fast kernels (device)
    size_t fprobs_bytes = 0;
    void *xyq = nullptr;              // float4 (xh, yh, xl, yl) per node (FP64 meshes)
    void *xyh = nullptr;              // float2 (xh, yh) per node (FP64 meshes): hop tests
    void *g1 = nullptr, *g2 = nullptr;   // field node tables, float4 (hi, lo) per node
    double *tparams = nullptr;        // field parameters the tables were built from (device)
    void *dfa = nullptr, *dfb = nullptr;   // value scratch of sl_step for the fast FP64 kernel
    void *he = nullptr;               // float4 half-edge walk records of the fast kernels (3 Nt), or NULL
    void *he8 = nullptr;              // uint2 compact records (FP64 meshes that fit, 3 Nt), or NULL
};

struct GraphCache {
    bool valid = false;
    void *exec = nullptr;             // cudaGraphExec_t
    int64_t n0 = 0;
    int32_t n_steps = 0;
    const void *v = nullptr, *v_scratch = nullptr;
    std::vector<uint8_t> probs;       // problems the graph was recorded with
    int32_t kernel = 0;
    int32_t stats = 0;
    int32_t config = 0, config_first = 0, split = 0;
    bool t0_initial = false;
};

}  // namespace sl

struct sl_mesh {
    int32_t n_problems = 0;
    int64_t N = 0, Nt = 0;
    int32_t precision = SL_FP64;
    int device = 0;
    uint64_t seed = 1;
    std::vector<int64_t> node_off, tri_off;
    // host copies in the current numbering (local indices per problem)
    std::vector<double> xy;
    std::vector<int32_t> tri, nbr;
    std::vector<int32_t> t0;          // T^0, global triangle indices (host copy)
    std::vector<int32_t> t0_init;     // the initial T^0 chosen at creation
    std::vector<int32_t> cells;       // per problem: sqrt(Nt/2), the M of a grid mesh
    // options
    int32_t opt_stats = 0;
    int32_t opt_walk_cap = 0;         // 0 = default
    int32_t opt_kernel = 0;
    int32_t opt_block = 0;
    int32_t opt_config = 5;           // launch configuration of the fast kernels (later steps)
    int32_t opt_config_first = 0;     // ... for a step whose walks start at the initial triangles
    int32_t opt_strategy = 0;         // 0 = strategy (b), 1 = strategy (a) (T^0 never overwritten),
                                      // 2 = direct location on a structured Courant grid,
                                      // 3 = strategy (c) (spanning-tree parent's triangle)
    int32_t grid_M = 0;               // cells per side when the mesh is a structured Courant grid
    std::vector<int64_t> tree_level_off;   // strategy (c): level k = tree_order[off[k], off[k+1])
    int32_t opt_outside = 0;          // 0 = clip feet that leave the square, 1 = exclude the node
    int32_t opt_split = 0;            // 1 = split steps (settle pass + finish pass), FP64 meshes
    int32_t opt_async = 0;            // 1 = sl_run without stats returns unsynchronised
    int32_t opt_precise = 32;         // gradient bound of the FP64 value path (0 = off)
    int32_t opt_records = 0;          // 0 = 16-byte walk records, 1 = compact records where they fit
    int32_t opt_l2 = 0;               // 1 = persisting L2 window on the walk records in recorded graphs
    int32_t opt_pdl = 1;              // 1 = step kernels after the first of a sequence: programmatic serialization
    bool l2_limit_set = false;        // the context's persisting L2 limit was raised (l2_limit_prev saved)
    size_t l2_limit_prev = 0;
    bool t0_initial = true;           // T^0 holds the initial start triangles
    float hop_L = __builtin_inff();   // FP64 meshes: a bound of every edge's |dx| + |dy| in the hop
                                      // coordinates (upload_arrays)
    int32_t sms = 0;                  // multiprocessors of the device
    bool stepped = false;
    std::vector<double> table_key;    // field parameters of the current node tables
    sl::DeviceMesh d;
    sl::GraphCache graph;
    // device value buffers for sl_run_host
    void *host_v = nullptr, *host_v2 = nullptr;
    void *capture_stream = nullptr;   // cudaStream_t used only to record graphs
};

namespace sl {
struct FastProb;
struct FastArgs;

// Node tables of the trigonometric fields: which tables the problems need
// (need1: g1 for SWIRL, PAPER, FOURIER8; need2: g2 for PAPER, FOURIER8) and
// the key the tables are built for, kTableKeyStride doubles per problem
// (kind, p[0..SL_NPARAMS-1]).
constexpr size_t kTableKeyStride = 1 + SL_NPARAMS;
std::vector<double> field_table_key(int32_t n_problems, const sl_problem *probs, bool &need1, bool &need2);
// host side (mesh_host.cpp)
sl_status build_and_validate(sl_mesh *m, const int32_t *nbr_in);
sl_status reorder_host(sl_mesh *m, int32_t curve, int32_t *node_perm, int32_t *tri_perm);
// renumber by explicit new -> old permutations, local to each problem
sl_status permute_host(sl_mesh *m, const int32_t *node_perm, const int32_t *tri_perm);
// device side (api_device.cu)
sl_status upload(sl_mesh *m);
// (re)build the half-edge walk records in the form opt_records and the mesh allow
sl_status build_walk_records(sl_mesh *m);
// give back the persisting L2 lines and the context's previous limit
void release_l2_window(sl_mesh *m);
// the fast kernels' constants of step n of one problem, validated as sl_step validates them
sl_status fast_constants_one(const sl_problem &q, int64_t n, int32_t p, FastProb &f);
// the arguments of a fast-kernel step of the whole mesh: the step's constants
// on the device (fp) and on the host (fh, or NULL; a single problem's are
// also passed in the kernel parameters), values vin -> vout, debug outputs
// or NULL
void fast_args_for(const sl_mesh *m, const FastProb *fp, const void *vin, void *vout, const sl_debug *dbg,
                   const FastProb *fh, FastArgs &out);
void free_device(sl_mesh *m);
sl_status reset_t0_sync(sl_mesh *m);
sl_status upload_grid_table(sl_mesh *m, const std::vector<int32_t> &slot_tri);
sl_status build_tree(const sl_mesh *m, std::vector<int32_t> &order, std::vector<int64_t> &level_off,
                     std::vector<int32_t> &parent);
sl_status upload_tree(sl_mesh *m, const std::vector<int32_t> &order, const std::vector<int32_t> &parent);
int32_t default_walk_cap(const sl_mesh *m);
}  // namespace sl
