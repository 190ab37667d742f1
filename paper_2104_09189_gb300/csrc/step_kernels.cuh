// step_kernels.cuh -- arguments and helpers of the step kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "predicates.cuh"
#include "step_common.cuh"

namespace sl {

struct StepArgs {
    const void *xy;               // double2[N] or float2[N]
    const int32_t *tv[3];         // triangle vertices (global node indices), SoA
    const int32_t *tn[3];         // neighbours (global triangle indices, -1 = boundary), SoA
    int32_t *t0;                  // start / located triangle per node (in place)
    int4 *t0v;                    // (T^0, its vertex ids) per node, kept in step with t0
    const void *vin;              // V^n
    void *vout;                   // V^{n+1}
    const ProbStep *probs;        // per-problem data of this step (device)
    const int64_t *node_off;      // problem node offsets (device)
    int32_t nprob;
    int32_t walk_cap;
    int64_t N;
    uint32_t *status;             // deferred status bits
    unsigned long long *stats;    // counters in sl_stats order
    sl_debug dbg;                 // optional per-node outputs (device pointers)
    int32_t keep_t0;              // strategy (a) or direct location: T^0 is never overwritten
    int32_t exclude;              // nodes whose foot leaves the square are excluded (Sec. 4)
    int32_t grid_M;               // > 0: start at the direct location on the structured grid (Sec. 4)
    const int4 *grid_t0v;         // start state of structured triangle 2 (M m + l) + (lower ? 1 : 0)
    // strategy (c): the launch covers the nodes order[base, base + count) (one
    // spanning-tree level) and each starts at its parent's T^0; otherwise
    // order is NULL and the launch covers nodes [0, count)
    const int32_t *order;
    const int32_t *parent;
    int64_t base, count;
};

__device__ __forceinline__ uint64_t mix64_dev(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Warp-aggregated counters: one atomic per warp and counter.
__device__ __forceinline__ void warp_stats(unsigned long long *stats, bool active, uint32_t hops,
                                           uint32_t exact_tests, uint32_t clipped, uint32_t fallback,
                                           uint32_t limit, uint32_t filter2 = 0, uint32_t excluded = 0)
{
    const unsigned full = 0xffffffffu;
    unsigned n = __reduce_add_sync(full, active ? 1u : 0u);
    unsigned h = __reduce_add_sync(full, hops);
    unsigned hm = __reduce_max_sync(full, hops);
    unsigned e = __reduce_add_sync(full, exact_tests);
    unsigned f2 = __reduce_add_sync(full, filter2);
    unsigned c = __reduce_add_sync(full, clipped);
    unsigned fb = __reduce_add_sync(full, fallback);
    unsigned l = __reduce_add_sync(full, limit);
    unsigned x = __reduce_add_sync(full, excluded);
    if ((threadIdx.x & 31) == 0) {
        if (n) atomicAdd(&stats[0], (unsigned long long)n);
        if (h) atomicAdd(&stats[1], (unsigned long long)h);
        if (hm) atomicMax(&stats[2], (unsigned long long)hm);
        if (e) atomicAdd(&stats[3], (unsigned long long)e);
        if (f2) atomicAdd(&stats[4], (unsigned long long)f2);
        if (c) atomicAdd(&stats[5], (unsigned long long)c);
        if (fb) atomicAdd(&stats[6], (unsigned long long)fb);
        if (l) atomicAdd(&stats[7], (unsigned long long)l);
        if (x) atomicAdd(&stats[8], (unsigned long long)x);
    }
}

// The triangle of the structured Courant grid (M cells per side of [0,1]^2)
// that the paper's direct formula (Sec. 4) gives for the point (x, y):
// cell (l, m) = (floor(x M), floor(y M)) clamped to the grid, upper triangle
// when x M - l < y M - m.  Returns the slot 2 (M m + l) + (upper ? 0 : 1).
__device__ __forceinline__ int grid_slot(float x, float y, int M)
{
    const float gx = x * (float)M, gy = y * (float)M;
    const int l = min(max((int)floorf(gx), 0), M - 1), m = min(max((int)floorf(gy), 0), M - 1);
    return 2 * (M * m + l) + (gx - (float)l < gy - (float)m ? 0 : 1);
}

// The node a thread of a step kernel works on (-1: none): thread t of the
// launch takes node t, or order[base + t] for a spanning-tree level.
template <class Args>
__device__ __forceinline__ int64_t node_of_thread(const Args &a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.count) return -1;
    return a.order ? (int64_t)a.order[a.base + t] : t;
}

void launch_plain_f64(const StepArgs &a, bool stats, bool debug, int block, cudaStream_t s);

}  // namespace sl
