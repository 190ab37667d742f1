// step_common.cuh -- per-step problem data, field evaluation and the Euler
// foot with the boundary clip, shared by the step kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/sl.h"

namespace sl {

// Everything a kernel needs to know about one problem at one step.  The
// time-dependent factors of the fields are evaluated once per step on the
// host (c[]), the node-dependent ones per node on the device.
struct ProbStep {
    int32_t kind;
    int32_t pad;
    double dt;
    double t;              // t_{n+1} = (n+1) dt
    double p[SL_NPARAMS];
    double c[8];           // SWIRL: c0 = cos(pi t / p0); FOURIER8: c[m] = a_m cos(2 pi t + phi_m);
                           // PAPER: c0 = p1 t
};

// Device status word bits and counters
enum { kStatusWords = 4, kStatCounters = 9 };

// f(x, t_{n+1}) at a node, in double precision, in the evaluation order of
// the field definitions listed in sl.h.  Intrinsics with explicit rounding
// keep the compiler from contracting a*b+c into one FMA, so affine and
// rotation fields round exactly like the definition written out.
__device__ __forceinline__ void field_f64(const ProbStep &P, double x, double y, double &fx, double &fy)
{
    const double *p = P.p;
    switch (P.kind) {
    case SL_FIELD_AFFINE:
        fx = __dadd_rn(__dadd_rn(__dadd_rn(p[0], __dmul_rn(p[1], x)), __dmul_rn(p[2], y)), __dmul_rn(p[3], P.t));
        fy = __dadd_rn(__dadd_rn(__dadd_rn(p[4], __dmul_rn(p[5], x)), __dmul_rn(p[6], y)), __dmul_rn(p[7], P.t));
        break;
    case SL_FIELD_ROTATION:
        fx = __dmul_rn(p[0], __dsub_rn(p[2], y));
        fy = __dmul_rn(p[0], __dsub_rn(x, p[1]));
        break;
    case SL_FIELD_SWIRL: {
        double sx, cx, sy, cy;
        sincospi(x, &sx, &cx);
        sincospi(y, &sy, &cy);
        double s2y = 2.0 * sy * cy;       // sin(2 pi y)
        double s2x = 2.0 * sx * cx;       // sin(2 pi x)
        fx = __dmul_rn(__dmul_rn(P.c[0], __dmul_rn(sx, sx)), s2y);
        fy = -__dmul_rn(__dmul_rn(P.c[0], __dmul_rn(sy, sy)), s2x);
        break;
    }
    case SL_FIELD_FOURIER8: {
        double gx = 0.0, gy = 0.0;
        const double pi = 3.14159265358979323846;
        for (int m = 0; m < 8; ++m) {
            double k = p[4 * m], l = p[4 * m + 1];
            double skx, ckx, sly, cly;
            sincospi(k * x, &skx, &ckx);
            sincospi(l * y, &sly, &cly);
            gx += P.c[m] * skx * (l * pi) * cly;
            gy -= P.c[m] * (k * pi) * ckx * sly;
        }
        fx = gx;
        fy = gy;
        break;
    }
    case SL_FIELD_PAPER: {
        double dx = x - p[2], dy = y - p[3];
        double arg = p[0] * sqrt(dx * dx + dy * dy) + P.c[0];
        sincos(arg, &fy, &fx);
        break;
    }
    default:
        fx = 0.0;
        fy = 0.0;
        break;
    }
}

// Boundary clip: if q = (qx, qy) leaves [0,1]^2 the segment x -> q is stopped
// at its first boundary crossing; coordinates that attain the crossing are
// set exactly to 0 or 1, the other one is clamped to [0,1].  Returns true if
// q was outside.
__host__ __device__ __forceinline__ bool clip_to_square(double x, double y, double qx, double qy, double &X,
                                                        double &Y)
{
    if (qx >= 0.0 && qx <= 1.0 && qy >= 0.0 && qy <= 1.0) {
        X = qx;
        Y = qy;
        return false;
    }
#ifdef __CUDA_ARCH__
    double dx = __dsub_rn(qx, x), dy = __dsub_rn(qy, y);
    double sx = 2.0, sy = 2.0, bx = 0.0, by = 0.0;
    if (qx < 0.0) { sx = __ddiv_rn(-x, dx); bx = 0.0; }
    if (qx > 1.0) { sx = __ddiv_rn(__dsub_rn(1.0, x), dx); bx = 1.0; }
    if (qy < 0.0) { sy = __ddiv_rn(-y, dy); by = 0.0; }
    if (qy > 1.0) { sy = __ddiv_rn(__dsub_rn(1.0, y), dy); by = 1.0; }
    double s = sx < sy ? sx : sy;
    double cx = __dadd_rn(x, __dmul_rn(s, dx));
    double cy = __dadd_rn(y, __dmul_rn(s, dy));
#else
    double dx = qx - x, dy = qy - y;
    double sx = 2.0, sy = 2.0, bx = 0.0, by = 0.0;
    if (qx < 0.0) { sx = -x / dx; bx = 0.0; }
    if (qx > 1.0) { sx = (1.0 - x) / dx; bx = 1.0; }
    if (qy < 0.0) { sy = -y / dy; by = 0.0; }
    if (qy > 1.0) { sy = (1.0 - y) / dy; by = 1.0; }
    double s = sx < sy ? sx : sy;
    double cx = x + s * dx;
    double cy = y + s * dy;
#endif
    if (sx == s) cx = bx;
    if (sy == s) cy = by;
    X = fmin(fmax(cx, 0.0), 1.0);
    Y = fmin(fmax(cy, 0.0), 1.0);
    return true;
}

// Euler foot X = x - dt f(x, t_{n+1}) (Eq. 4) followed by clip_to_square.
__device__ __forceinline__ bool foot_clip_f64(double x, double y, double dt, double fx, double fy, double &X,
                                              double &Y)
{
    double qx = __dsub_rn(x, __dmul_rn(dt, fx));
    double qy = __dsub_rn(y, __dmul_rn(dt, fy));
    return clip_to_square(x, y, qx, qy, X, Y);
}

// Problem of a global node index (binary search over the node offsets).
__device__ __forceinline__ int problem_of(const int64_t *node_off, int nprob, int64_t i)
{
    int lo = 0, hi = nprob;     // node_off[lo] <= i < node_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (node_off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Problem of node i < N from the per-chunk table (kChunkShift: chunks of 128
// consecutive nodes; for each, the problems of its first and last node, see
// chunk_problem_table), searching only in a chunk that spans problems.  A
// warp's lanes read the same entry.
constexpr int kChunkShift = 7;

__device__ __forceinline__ int chunk_problem(const int2 *chunk_prob, const int64_t *node_off, int64_t i)
{
    const int2 c = __ldg(&chunk_prob[i >> kChunkShift]);
    if (c.x == c.y) return c.x;
    return c.x + problem_of(node_off + c.x, c.y - c.x + 1, i);
}

}  // namespace sl
