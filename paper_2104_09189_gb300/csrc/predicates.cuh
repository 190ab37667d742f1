// predicates.cuh -- exact orientation sign for the barycentric walk.
//
// The walk of Algorithm 1 moves across the edge opposite the most negative
// barycentric coordinate and stops when all three are >= 0 (Sec. 2.2).  The
// numerators of Eq. 6 are orientation determinants, so the stopping test is
// three orientation signs; they are computed exactly here so that the
// located triangle is the true one even for feet on or next to an edge.
//
// Stage 1: double evaluation with the forward error bound of Shewchuk,
//          "Adaptive Precision Floating-Point Arithmetic and Fast Robust
//          Geometric Predicates" (1997), bound (3 + 16 eps) eps (|t1| + |t2|).
// Stage 2: exact sum of the six coordinate products.  Each product a*b is
//          split without error into p + e with p = fl(a*b), e = fma(a,b,-p)
//          (exact when no underflow occurs), and the twelve doubles are
//          accumulated into a nonoverlapping expansion with Knuth's
//          error-free TwoSum (Shewchuk's Grow-Expansion); the sign of an
//          expansion is the sign of its largest nonzero component.
// Stage 2 is exact when every nonzero coordinate has magnitude in
// [2^-450, 2^450]; outside that range the result is the stage-1 sign and
// the caller is told (range flag).
#pragma once

#ifndef __CUDACC__
#include <cmath>
#define SL_HD inline
#else
#define SL_HD __host__ __device__ __forceinline__
#endif

namespace slp {

SL_HD void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    double bv = s - a;
    double av = s - bv;
    e = (a - av) + (b - bv);
}

SL_HD void two_prod(double a, double b, double &p, double &e)
{
    p = a * b;
    e = fma(a, b, -p);
}

// Add b to the nonoverlapping, increasing-magnitude expansion e[0..n).
SL_HD int grow(double *e, int n, double b)
{
    double q = b;
    int m = 0;
    for (int k = 0; k < n; ++k) {
        double s, r;
        two_sum(q, e[k], s, r);
        q = s;
        if (r != 0.0) e[m++] = r;      // drop zero components
    }
    if (q != 0.0) e[m++] = q;
    return m;
}

SL_HD bool in_exact_range(double v)
{
    double a = fabs(v);
    return a == 0.0 || (a >= 0x1p-450 && a <= 0x1p+450);
}

// Exact sign of orient(a, b, c) = (bx-ax)(cy-ay) - (by-ay)(cx-ax).
SL_HD int orient_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    // det = bx cy - bx ay - ax cy - by cx + ax by + ay cx
    const double u[6] = {bx, -bx, -ax, -by, ax, ay};
    const double v[6] = {cy, ay, cy, cx, by, cx};
    double e[12];
    int n = 0;
    for (int k = 0; k < 6; ++k) {
        double p, r;
        two_prod(u[k], v[k], p, r);
        n = grow(e, n, r);
        n = grow(e, n, p);
    }
    if (n == 0) return 0;
    return e[n - 1] > 0.0 ? 1 : -1;
}

// Shewchuk's stage-A relative bound for orient2d: (3 + 16 eps) eps, eps = 2^-53.
constexpr double kCcwErr = (3.0 + 16.0 * 0x1p-53) * 0x1p-53;

struct OrientResult {
    int sign;      // -1, 0, +1 (exact)
    double det;    // double-precision estimate of the determinant
    int stage;     // 1 = decided by the double filter, 2 = exact stage
    bool range;    // some coordinate was outside the exact range
};

SL_HD OrientResult orient(double ax, double ay, double bx, double by, double cx, double cy)
{
    OrientResult r;
    double t1 = (bx - ax) * (cy - ay);
    double t2 = (by - ay) * (cx - ax);
    r.det = t1 - t2;
    double mag = fabs(t1) + fabs(t2);
    double bound = kCcwErr * mag;
    r.range = false;
    if (mag > 0x1p-900) {
        if (r.det > bound) { r.sign = 1; r.stage = 1; return r; }
        if (r.det < -bound) { r.sign = -1; r.stage = 1; return r; }
    }
    r.stage = 2;
    r.range = !(in_exact_range(ax) && in_exact_range(ay) && in_exact_range(bx) && in_exact_range(by) &&
                in_exact_range(cx) && in_exact_range(cy));
    r.sign = orient_exact(ax, ay, bx, by, cx, cy);
    return r;
}

}  // namespace slp
