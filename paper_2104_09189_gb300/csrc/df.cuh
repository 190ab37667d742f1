// df.cuh -- double-float arithmetic on the FP32 pipe.
//
// GB300 executes about two FP64 operations per clock per SM against 128 FP32
// ones, and float<->double conversions run at the FP64 rate too.  The fast
// FP64-accuracy kernel therefore keeps values as unevaluated sums hi + lo of
// two floats (48-bit significands) and uses the error-free transformations
// of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA-based exact product:
//   two_sum(a, b)      : s + e = a + b exactly, s = fl(a + b)
//   fast_two_sum(a, b) : the same when |a| >= |b| (or a == 0)
//   two_prod(a, b)     : p + e = a * b exactly (no underflow), p = fl(a * b)
// Intrinsics with explicit rounding stop the compiler from contracting or
// reassociating the error terms.
#pragma once

#include <cuda_runtime.h>

namespace sl {

struct df {
    float h, l;
};

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bv = __fsub_rn(s, a);
    float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

__device__ __forceinline__ void fast_two_sum_f(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_make(float h, float l)
{
    df r;
    r.h = h;
    r.l = l;
    return r;
}

// a + b: exact head sum, tails added in float; absolute error about
// 2^-24 (|a.l| + |b.l|) + 2^-48 |a + b|.
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum_f(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    df r;
    fast_two_sum_f(s, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.h, -a.l); }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b with relative error about 2^-46.
__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    df r;
    fast_two_sum_f(p, e, r.h, r.l);
    return r;
}

// cross(a, b) = a.x b.y - a.y b.x for df vectors
__device__ __forceinline__ df df_cross(df ax, df ay, df bx, df by)
{
    return df_sub(df_mul(ax, by), df_mul(ay, bx));
}

// 1 / a, relative error about 2^-45 (a.h != 0)
__device__ __forceinline__ df df_rcp(df a)
{
    float r = __frcp_rn(a.h);
    // residual 1 - a r, computed with an exact product of the heads
    float e = __fmaf_rn(-a.h, r, 1.0f);
    e = __fmaf_rn(-a.l, r, e);
    df q;
    fast_two_sum_f(r, __fmul_rn(r, e), q.h, q.l);
    return q;
}

// Exact sign of orient(p, q, X) = (qx-px)(Xy-py) - (qy-py)(Xx-px) for double
// vertices p, q and a point X given as the exact sums Xx = xh + xl,
// Xy = yh + yl.  Expanded into ten products, each split without error by an
// FMA, and summed into a nonoverlapping expansion (Shewchuk's
// Grow-Expansion with zero elimination).  Exact while every nonzero input has
// magnitude in [2^-450, 2^450].
__device__ __forceinline__ int orient_exact_split(double px, double py, double qx, double qy, double xh, double xl,
                                                  double yh, double yl)
{
    // det = qx Xy - qx py - px Xy - qy Xx + qy px + py Xx
    const double u[10] = {qx, qx, -qx, -px, -px, -qy, -qy, qy, py, py};
    const double v[10] = {yh, yl, py, yh, yl, xh, xl, px, xh, xl};
    double e[20];
    int n = 0;
    for (int k = 0; k < 10; ++k) {
        double p = u[k] * v[k];
        double r = fma(u[k], v[k], -p);
        n = slp::grow(e, n, r);
        n = slp::grow(e, n, p);
    }
    if (n == 0) return 0;
    return e[n - 1] > 0.0 ? 1 : -1;
}

// h + l == p exactly, for a normalised float pair (h, l) and a double p:
// then h = fl32(p) and p - h is exact (Sterbenz), so the test is exact.
__device__ __forceinline__ bool df_equals(float h, float l, double p)
{
    return h == __double2float_rn(p) && (double)l == p - (double)h;
}

// Exact sign of orient(P, Q, X), X = (xh + xl, yh + yl), in three stages:
//  1. X on an axis-parallel edge line, or X equal to P or Q: exactly 0;
//  2. double evaluation of (Qx-Px)(Xy-Py) - (Qy-Py)(Xx-Px) with the
//     differences X - P formed by an error-free TwoSum (so feet a few ulps
//     from a vertex are still resolved), accepted when it clears its
//     forward error bound;
//  3. the full expansion (orient_exact_split).
// `stage` receives the stage that decided.
__device__ __forceinline__ int orient_exact_df(double2 P, double2 Q, float xh, float xl, float yh, float yl, int &stage)
{
    stage = 1;
    if (P.x == Q.x && df_equals(xh, xl, P.x)) return 0;
    if (P.y == Q.y && df_equals(yh, yl, P.y)) return 0;
    if ((df_equals(xh, xl, P.x) && df_equals(yh, yl, P.y)) || (df_equals(xh, xl, Q.x) && df_equals(yh, yl, Q.y)))
        return 0;                                             // X is an endpoint
    stage = 2;
    const double a = Q.x - P.x, b = Q.y - P.y;
    double s, e, r;
    slp::two_sum((double)xh, -P.x, s, e);
    r = e + (double)xl;
    const double c = s + r;                                   // X.x - P.x
    const double ec = 0x1p-52 * (fabs(c) + fabs(r));
    slp::two_sum((double)yh, -P.y, s, e);
    r = e + (double)yl;
    const double d = s + r;                                   // X.y - P.y
    const double ed = 0x1p-52 * (fabs(d) + fabs(r));
    const double t1 = a * d, t2 = b * c;
    const double det = t1 - t2;
    const double E = fabs(a) * ed + fabs(b) * ec + 0x1p-51 * (fabs(t1) + fabs(t2));
    if (fabs(c) + fabs(d) > 0x1p-900 && fabs(a) + fabs(b) > 0x1p-400) {
        if (det > E) return 1;
        if (det < -E) return -1;
    }
    stage = 3;
    return orient_exact_split(P.x, P.y, Q.x, Q.y, xh, xl, yh, yl);
}

}  // namespace sl
