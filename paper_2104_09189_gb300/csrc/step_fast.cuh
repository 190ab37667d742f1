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
// g1, g2 are node tables filled once per field (k_field_tables).
struct FastProb {
    int32_t kind;
    int32_t pad;
    double dt;          // only used by the clip path and the debug output
    float2 c[6];        // (hi, lo)
};

struct FastArgs {
    const float4 *xyq;            // FP64 meshes: (xh, yh, xl, yl); FP32 meshes: unused
    const float2 *xyf;            // FP32 meshes: (x, y); FP64 meshes: unused
    const double2 *xyd;           // exact coordinates (FP64 meshes)
    const float2 *xyh;            // FP64 meshes: high parts (xh, yh) for the FP32 hop tests
    const int32_t *tv[3];
    const int32_t *tn[3];         // -1 - side on the boundary (0: x=0, 1: x=1, 2: y=0, 3: y=1)
    int32_t *t0;
    int4 *t0v;                    // per node: (T^0, its three vertex ids), kept in step with t0
    const void *vin;              // FP64: float2 (hi, lo) values; FP32: float values
    void *vout;
    const float4 *g1, *g2;        // field tables (hi, lo) per node, or NULL
    const FastProb *probs;
    const int64_t *node_off;
    int32_t nprob;
    int32_t walk_cap;
    int64_t N;
    uint32_t *status;
    unsigned long long *stats;
    sl_debug dbg;
    // walk queue (optional): walks longer than hop_budget FP32 hops are
    // pushed here by the main kernel, continued by the walk kernel and
    // completed by the finish pass
    int32_t *queue;
    uint32_t *queue_hops;
    uint32_t *queue_count;
    int32_t hop_budget;
};

// config: launch configuration 0..3 (see step_fast.cu)
void launch_fast_df(const FastArgs &a, bool stats, bool debug, int config, int sms, cudaStream_t s);
constexpr int kFastConfigs = 6;
void launch_fast_f32(const FastArgs &a, bool stats, bool debug, int config, cudaStream_t s);

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
    const double *params;         // nprob x (kind, p[48]) as 49 doubles
    float4 *g1, *g2;
};
void launch_field_tables(const FieldTableArgs &a, cudaStream_t s);

// t0v[i] = (t0[i], its three vertex ids)
void launch_fill_t0v(const int32_t *t0, const int32_t *tv0, const int32_t *tv1, const int32_t *tv2, int4 *t0v,
                     int64_t n, cudaStream_t s);

}  // namespace sl
