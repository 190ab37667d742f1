// step_fast.cuh -- arguments of the fast step kernels (FP64-accuracy
// double-float kernel and FP32 kernel) and their launchers.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/sl.h"

namespace sl {

// Per-problem constants of one step, evaluated on the host in double and
// stored as (hi, lo) float pairs.  Foot of node x for each field kind:
//   ZERO      X = x
//   AFFINE    X = x - (c0 + c1 x + c2 y),  Y = y - (c3 + c4 x + c5 y)
//             (c0 = dt (p0 + p3 t), c1 = dt p1, c2 = dt p2, c3..c5 alike)
//   ROTATION  X = x + c0 (y - c2),  Y = y - c0 (x - c1)    (c0 = dt p0, (c1, c2) = centre)
//   SWIRL     X = x - c0 g1(x)                         (c0 = dt cos(pi t / T))
//   PAPER,    X = x - c0 g1(x) - c1 g2(x)              (c0, c1 = dt x time factors)
//   FOURIER8
// g1, g2 are node tables filled once per field (k_field_tables).  A rotation
// centre inside the unit square is stored in (grid, remainder) form instead
// (flag kFastCentreGrid): a node's grid part minus the centre's is then exact
// in float, and x - c costs two additions.
struct FastProb {
    int32_t kind;
    int32_t flags;      // kFastCentreGrid
    double dt;          // only used by the clip path and the debug output
    float2 c[6];        // (hi, lo)
};

constexpr int32_t kFastCentreGrid = 1;

// The six per-step constants of a problem as float pairs: (hi, lo), or for a
// rotation centre in [0, 1]^2 the (grid, remainder) split of the node
// coordinates (g = c rounded to the grid of 2^-24, r = fl32(c - g)).
void pack_fast_constants(int32_t kind, const double c[6], FastProb &f);

struct FastArgs {
    const float4 *xyq;            // FP64 meshes: (xh, yh, xl, yl); FP32 meshes: unused
    const float2 *xyf;            // FP32 meshes: (x, y); FP64 meshes: unused
    const double2 *xyd;           // exact coordinates (FP64 meshes)
    const float2 *xyh;            // FP64 meshes: high parts (xh, yh) for the FP32 hop tests
    const int32_t *tv[3];
    const int32_t *tn[3];         // -1 - side on the boundary (0: x=0, 1: x=1, 2: y=0, 3: y=1)
    const float4 *he;             // half-edge walk records, 3 per triangle (k_build_he), or NULL
    const uint2 *he8;             // FP64 meshes whose records fit in 8 bytes (k_build_he8), or NULL
    int32_t *t0;
    int4 *t0v;                    // per node: (3 T^0, T[0][T^0], T[1][T^0], T[2][T^0]), kept in
                                  // step with t0
    const void *vin;              // FP64: float2 (hi, lo) values; FP32: float values
    void *vout;
    const float4 *g1, *g2;        // field tables (hi, lo) per node (FP64 meshes), or NULL
    const float2 *g1f, *g2f;      // field tables rounded to float (FP32 meshes), or NULL
    const FastProb *probs;
    FastProb prob0;               // single: a copy of probs[0] (kernel parameter space)
    int32_t single;               // one problem, prob0 valid
    const int64_t *node_off;
    const int2 *chunk_prob;       // more than one problem: per 128 nodes, the first and last node's
                                  // problem (chunk_problem); else NULL
    int32_t nprob;
    int32_t walk_cap;
    int64_t N;
    uint32_t *status;
    unsigned long long *stats;
    sl_debug dbg;
    float hop_L;                  // FP64 meshes: an upper bound of every edge's |dx| + |dy| in the hop
                                  // coordinates (the runs of lean hops; +inf: a bound per hop)
    float steep_g2;               // G^2 of SL_OPT_PRECISE (double-float kernel; +inf = off): a value
                                  // with (v_k - v_3)^2 > G^2 den is evaluated in FP64
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
    // split steps: the nodes the settle pass leaves to the finish pass
    int32_t *queue;
    uint32_t *queue_count;
    uint32_t *queue_next;         // split steps: the next step's counter, zeroed by the settle pass (or NULL)
    // host side only: launch with programmatic stream serialization (the
    // kernel before it on the stream is a step kernel of the same sequence of
    // steps; see launch_step_kernel)
    int32_t pdl;
};

// Programmatic dependent launch.  A step kernel launched with programmatic
// stream serialization may be scheduled while the kernel before it on the
// stream is still running: its launch and the start of its blocks overlap
// that kernel's last wave.  Every step kernel signals its dependents as its
// blocks start (pdl_launch_dependents) and then waits (pdl_wait) until the
// kernel before it has completed and its writes are visible, before anything
// else.  (Waiting later, after the foot, which needs no data a step writes,
// stopped the compiler from issuing the start-state load ahead of the foot
// arithmetic and cost more than it hid.)  For a kernel launched without the
// attribute both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename Kernel>
inline void launch_step_kernel(Kernel k, unsigned grid, unsigned block, cudaStream_t s, const FastArgs &a)
{
    if (!a.pdl) {
        k<<<grid, block, 0, s>>>(a);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, a);
}
#endif

// config: launch configuration 0..kFastConfigs-1 (see step_fast.cu)
void launch_fast_df(const FastArgs &a, bool stats, bool debug, int config, cudaStream_t s);
// one launch configuration each (step_fast_c*.cu)
void launch_fast_df_c0(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
void launch_fast_df_c1(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
void launch_fast_df_c2(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
void launch_fast_df_c3(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
void launch_fast_df_c4(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
void launch_fast_df_c5(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
void launch_fast_df_ext(const FastArgs &a, bool stats, bool debug, cudaStream_t s);
// the two passes of a split step: lean settle pass, then the finish pass over
// its queue (reset: zero the queue counter first)
void launch_settle_df(const FastArgs &a, bool stats, bool debug, bool reset, cudaStream_t s);
void launch_finish_df(const FastArgs &a, bool stats, bool debug, int sms, cudaStream_t s);
constexpr int kFastConfigs = 6;
void launch_fast_f32(const FastArgs &a, bool stats, bool debug, int config, cudaStream_t s);

// the memory accesses of a steady step with no arithmetic (sl_probe_gather)
void launch_gather_probe(const float4 *xyq, const int4 *t0v, const float2 *vin, float2 *vout, int64_t N,
                         cudaStream_t s);

// value format conversions for the double-float kernel
void launch_to_df(const double *src, float2 *dst, int64_t n, cudaStream_t s);
void launch_from_df(const float2 *src, double *dst, int64_t n, cudaStream_t s);

// node tables of the fields (double precision, once per field)
struct FieldTableArgs {
    const double2 *xyd;           // node coordinates (FP64 meshes), or NULL
    const float2 *xyf;            // node coordinates (FP32 meshes), or NULL
    const int64_t *node_off;
    int32_t nprob;
    int64_t N;
    const double *params;         // nprob x (kind, p[SL_NPARAMS]) as 1 + SL_NPARAMS doubles
    float4 *g1, *g2;              // FP64 meshes: (hi, lo) pairs
    float2 *g1f, *g2f;            // FP32 meshes: the values rounded to float
};
void launch_field_tables(const FieldTableArgs &a, cudaStream_t s);

// Half-edge walk records, he[3 t + k] for the edge of triangle t opposite its
// vertex k.  Interior edge, u = tn[k][t], k' the slot of t in u's neighbours:
//   (Qx, Qy, e0', e1') with Q = tv[k'][u] (coordinates: xyh for FP64 meshes,
//   the float coordinates for FP32 meshes), e0' = 3u + (k'+1) mod 3 and
//   e1' = 3u + (k'+2) mod 3 as int bits: the walk state of u entered
//   through this edge is (W0, W1, W2) = (T[k'+1][u], T[k'+2][u], Q).
// Boundary edge: (NaN, NaN, 3t + (k+1) mod 3, side code tn[k][t] < 0): NaN
// coordinates end an FP32 hop loop, and the first code still names an edge
// of t, the triangle the walk is in.
void launch_build_he(const int32_t *const tv[3], const int32_t *const tn[3], const float2 *xyc, int64_t nt,
                     float4 *he, cudaStream_t s);

// Compact 8-byte half-edge records of FP64 meshes, he8[3 t + k] for the edge
// of triangle t opposite its vertex T[k][t].  Interior edge, u, k', Q and
// e0' = 3 u + (k'+1) mod 3 as above; (dx, dy) = Q - W0 with W0 = T[k'+1][u],
// the entered triangle's first vertex (Q - W0 is an edge of u), in units of
// 2^-24 (the hop coordinates are on that grid, so the difference is an exact
// integer), stored biased, b = d + 2^17 in [2, 2^18 - 2]:
//   word 0 = bx | (by & 0x3FFF) << 18,
//   word 1 = by >> 14 | f << 4 | e0' << 5,
// f = 1 when e0' is slot 2 of u (the other exit is then e0' - 2, else
// e0' + 1).  The float with bits 0x3F000000 | b is 0.5 + b 2^-24, so Q = W0
// + that - (0.5 + 2^-7), all exact.  Boundary edge: zero offset and e0' = 3 t
// + (k+1) mod 3, an exit of t itself (a walk can never cross it: the foot
// lies in the square).  Sets *overflow to 1 when some |dx| or |dy| exceeds
// 2^17 - 2 (an edge longer than about 2^-7) or e0' reaches 2^27 (more than
// 44.7 M triangles): the mesh then keeps 16-byte records.
void launch_build_he8(const int32_t *const tv[3], const int32_t *const tn[3], const float2 *xyh, int64_t nt,
                      uint2 *he8, uint32_t *overflow, cudaStream_t s);

// t0v[i] = (3 t0[i], its three vertex ids in slot order)
void launch_fill_t0v(const int32_t *t0, const int32_t *tv0, const int32_t *tv1, const int32_t *tv2, int4 *t0v,
                     int64_t n, cudaStream_t s);
// t0 = t0_init and the start-state cache with it, one pass
void launch_reset_t0(const int32_t *t0_init, const int32_t *tv0, const int32_t *tv1, const int32_t *tv2, int32_t *t0,
                     int4 *t0v, int64_t n, cudaStream_t s);

}  // namespace sl
