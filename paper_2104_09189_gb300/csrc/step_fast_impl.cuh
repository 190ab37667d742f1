// step_fast_impl.cuh -- device code of the fast FP64-accuracy step kernel
// (included by step_fast.cu and the step_fast_c*.cu files, which
// instantiate its launch configurations in separate translation units).
//
// The same step as step_plain.cu (Euler foot at t_{n+1} with the boundary
// clip, barycentric walk from T^0_i -- strategy (b) of Sec. 3 -- and P1
// interpolation with the barycentric coordinates of Eq. 6), arranged for a
// GPU whose FP64 rate is 1/64 of its FP32 rate:
//
//  * walk hops are decided in FP32 on the high parts of the coordinates:
//    an edge is crossed only when its orientation is negative beyond a
//    certified FP32 error bound, so every hop is a hop of the exact
//    barycentric walk (Algorithm 1, most negative coordinate first);
//  * the stopping test is certified in double-float arithmetic (hi + lo
//    float pairs, ~2^-46 relative) with an error bound, and falls back to an
//    exact expansion-arithmetic sign on the double coordinates when the
//    bound cannot decide -- so the located triangle contains the foot
//    exactly;
//  * the barycentric coordinates theta_1 = n_1 / den, theta_2 = n_2 / den
//    (Eq. 6, numerators relative to vertex 3) and the P1 value
//    v_3 + theta_1 (v_1 - v_3) + theta_2 (v_2 - v_3) (= theta_1 v_1 +
//    theta_2 v_2 + theta_3 v_3 with theta_3 = 1 - theta_1 - theta_2,
//    Remark 1) are evaluated in double-float as well;
//  * node values travel between steps as (hi, lo) float pairs.
#pragma once

#include "predicates.cuh"
#include "df.cuh"
#include "step_common.cuh"
#include "step_fast.cuh"
#include "step_kernels.cuh"

namespace sl {

__device__ __forceinline__ df dfp(float2 v) { return df_make(v.x, v.y); }

__device__ __forceinline__ bool df_lt(df a, df b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ bool df_neg_strict(df a) { return a.h < 0.0f || (a.h == 0.0f && a.l < 0.0f); }
__device__ __forceinline__ bool df_gt1(df a) { return a.h > 1.0f || (a.h == 1.0f && a.l > 0.0f); }
__device__ __forceinline__ bool df_is(df a, float v) { return a.h == v && a.l == 0.0f; }

// a / b in double-float (b.h != 0): relative error about 2^-44.
__device__ __forceinline__ df df_div(df a, df b)
{
    const float q1 = __fdiv_rn(a.h, b.h);
    const df r = df_sub(a, df_mul(b, df_make(q1, 0.0f)));
    const float q2 = __fdiv_rn(r.h, b.h);
    df q;
    fast_two_sum_f(q1, q2, q.h, q.l);
    return q;
}

// The clip and the exclusion decide on the foot rounded to double, the
// precision Eq. 4 is evaluated in: a double-float coordinate above 1 by at
// most half an ulp of 1 in double (2^-53, ties to even) rounds to exactly 1
// and lies on the boundary.  (Below 1 and near 0 the double-float and double
// decisions already agree.)  Without this, a boundary node whose velocity is
// tangent to within 1e-16 could be clipped by one arithmetic and not by the
// other, and the clip moves the foot by a whole step.
__device__ __forceinline__ void round_boundary(df &X)
{
    if (X.h == 1.0f && X.l > 0.0f && X.l <= 0x1p-53f) X.l = 0.0f;
}

// Boundary clip of the Euler foot q of node x, in double-float: if q leaves
// [0,1]^2 the segment x -> q stops at its first boundary crossing; the
// coordinates that attain the crossing become exactly 0 or 1, the other one
// is clamped to [0,1].  Returns true if q was outside.
__device__ __forceinline__ bool clip_df(df x, df y, df &X, df &Y)
{
    const bool xlo = df_neg_strict(X), xhi = df_gt1(X), ylo = df_neg_strict(Y), yhi = df_gt1(Y);
    if (!(xlo || xhi || ylo || yhi)) return false;
    const df dx = df_sub(X, x), dy = df_sub(Y, y);
    const df two = df_make(2.0f, 0.0f);
    df sx = two, sy = two;
    const float bx = xhi ? 1.0f : 0.0f, by = yhi ? 1.0f : 0.0f;
    if (xlo || xhi) sx = df_div(df_sub(df_make(bx, 0.0f), x), dx);
    if (ylo || yhi) sy = df_div(df_sub(df_make(by, 0.0f), y), dy);
    const bool xfirst = !df_lt(sy, sx);       // sx <= sy
    const bool yfirst = !df_lt(sx, sy);       // sy <= sx
    const df s = xfirst ? sx : sy;
    if (s.h == 0.0f) {
        // a node on the side it moves out through: the foot is the node
        // itself, kept as its own coordinate pair
        X = x;
        Y = y;
        return true;
    }
    df cx = df_add(x, df_mul(s, dx)), cy = df_add(y, df_mul(s, dy));
    if (xfirst) cx = df_make(bx, 0.0f);
    if (yfirst) cy = df_make(by, 0.0f);
    if (df_neg_strict(cx)) cx = df_make(0.0f, 0.0f);
    if (df_gt1(cx)) cx = df_make(1.0f, 0.0f);
    if (df_neg_strict(cy)) cy = df_make(0.0f, 0.0f);
    if (df_gt1(cy)) cy = df_make(1.0f, 0.0f);
    X = cx;
    Y = cy;
    return true;
}

// Displacement d = -dt f(x, t_{n+1}) of the Euler foot X = x + d (Eq. 4) in
// double-float, with the field's time factors folded into the per-step
// constants.
template <int kKind>
__device__ __forceinline__ void disp_df_k(const FastProb &P, const FastArgs &a, int64_t i, df x, df y, df &DX,
                                          df &DY)
{
    switch (kKind) {
    case SL_FIELD_AFFINE: {
        DX = df_neg(df_add(df_add(dfp(P.c[0]), df_mul(dfp(P.c[1]), x)), df_mul(dfp(P.c[2]), y)));
        DY = df_neg(df_add(df_add(dfp(P.c[3]), df_mul(dfp(P.c[4]), x)), df_mul(dfp(P.c[5]), y)));
        break;
    }
    case SL_FIELD_ROTATION:
        if (P.flags & kFastCentreGrid) {
            // node and centre in (grid, remainder) form: the grid parts
            // subtract exactly, the remainders with one rounding (2^-49)
            const df dy = df_make(__fsub_rn(y.h, P.c[2].x), __fsub_rn(y.l, P.c[2].y));
            const df dx = df_make(__fsub_rn(x.h, P.c[1].x), __fsub_rn(x.l, P.c[1].y));
            DX = df_mul(dfp(P.c[0]), dy);
            DY = df_neg(df_mul(dfp(P.c[0]), dx));
        } else {
            DX = df_mul(dfp(P.c[0]), df_sub(y, dfp(P.c[2])));
            DY = df_neg(df_mul(dfp(P.c[0]), df_sub(x, dfp(P.c[1]))));
        }
        break;
    case SL_FIELD_SWIRL: {
        const float4 g = a.g1[i];
        const df k = dfp(P.c[0]);
        DX = df_neg(df_mul(k, df_make(g.x, g.z)));
        DY = df_neg(df_mul(k, df_make(g.y, g.w)));
        break;
    }
    case SL_FIELD_PAPER:
    case SL_FIELD_FOURIER8: {
        const float4 g = a.g1[i], q = a.g2[i];
        const df k0 = dfp(P.c[0]), k1 = dfp(P.c[1]);
        DX = df_neg(df_add(df_mul(k0, df_make(g.x, g.z)), df_mul(k1, df_make(q.x, q.z))));
        DY = df_neg(df_add(df_mul(k0, df_make(g.y, g.w)), df_mul(k1, df_make(q.y, q.w))));
        break;
    }
    default:
        DX = df_make(0.0f, 0.0f);
        DY = df_make(0.0f, 0.0f);
        break;
    }
}

// The same for a kind known only at run time.
__device__ __forceinline__ void disp_df(const FastProb &P, const FastArgs &a, int64_t i, df x, df y, df &DX, df &DY)
{
    switch (P.kind) {
    case SL_FIELD_AFFINE: disp_df_k<SL_FIELD_AFFINE>(P, a, i, x, y, DX, DY); break;
    case SL_FIELD_ROTATION: disp_df_k<SL_FIELD_ROTATION>(P, a, i, x, y, DX, DY); break;
    case SL_FIELD_SWIRL: disp_df_k<SL_FIELD_SWIRL>(P, a, i, x, y, DX, DY); break;
    case SL_FIELD_PAPER: disp_df_k<SL_FIELD_PAPER>(P, a, i, x, y, DX, DY); break;
    case SL_FIELD_FOURIER8: disp_df_k<SL_FIELD_FOURIER8>(P, a, i, x, y, DX, DY); break;
    default: disp_df_k<SL_FIELD_ZERO>(P, a, i, x, y, DX, DY); break;
    }
}

// A foot coordinate x + d straight in the (grid, remainder) form of the
// certified test, for a node coordinate x = (grid, remainder) and a
// displacement d = (h, l): dg = d.h rounded to the grid of 2^-24, g = x.g +
// dg (grid values below 1: exact), r = (x.r + (d.h - dg)) + d.l, where d.h -
// dg is exact (a multiple of ulp(d.h) below 2^-25).  |r| <= 2^-24 and a few
// ulps of d, within the margins of hop_bound and cert_bound_g, and the pair
// is within about 2^-48 of x + d.  Returns false unless g lies at least
// 2^-23 inside (0, 1), so that x + d does: the caller then takes the
// double-float sum, the boundary rounding and the clip.
__device__ __forceinline__ bool foot_grid(df x, df d, df &X)
{
    const float dg = __fmul_rn(rintf(__fmul_rn(d.h, 16777216.0f)), 0x1p-24f);
    const float g = __fadd_rn(x.h, dg);
    X = df_make(g, __fadd_rn(__fadd_rn(x.l, __fsub_rn(d.h, dg)), d.l));
    return g >= 0x1p-23f && g <= 1.0f - 0x1p-23f;
}

// Error bound of the FP32 hop test.  Node coordinates are stored as a grid
// part (the coordinate rounded to the grid of 2^-24, also the hop
// coordinate) and a remainder; the foot is exactly X.h + X.l and the hop test
// uses X.h.  Every hop coordinate is within 2^-25 of the exact one, so every
// difference is within 2^-24 + 2^-24 |d| of the exact difference, and a cross
// product of differences whose |.|-sum is at most S is within
// 2^-23 S + 2^-22 S^2 (two-fold margins).
__device__ __forceinline__ float hop_bound(float S) { return S * __fmaf_rn(S, 0x1p-22f, 0x1p-23f) + 0x1p-46f; }

// Coordinates in the certified test are pairs g + r: g on the grid of 2^-24
// (mesh nodes are stored so, the foot is converted by to_grid), |r| <= 2^-24,
// the pair within 2^-49 of the coordinate.  A difference of two such pairs is
// (g1 - g2) + (r1 - r2): the first difference is exact in float, the second
// is rounded once (|r1 - r2| <= 2^-23, error <= 2^-48).
struct gd {
    float g, r;
};

__device__ __forceinline__ gd gd_sub(float g1, float r1, float g2, float r2)
{
    gd d;
    d.g = __fsub_rn(g1, g2);
    d.r = __fsub_rn(r1, r2);
    return d;
}

// x = g + r with g = x rounded to the grid of 2^-24 (x in [0, 1]): the
// scaling by 2^24 and back is exact, and so is x.h - g.
__device__ __forceinline__ void to_grid(df x, float &g, float &r)
{
    g = __fmul_rn(rintf(__fmul_rn(x.h, 16777216.0f)), 0x1p-24f);
    r = __fadd_rn(__fsub_rn(x.h, g), x.l);
}

// u_x v_y - u_y v_x for differences u, v in the pair form, as a normalised
// double-float: the products of the grid parts with their exact FMA
// remainders, the cross terms accumulated by FMA, the two products summed by
// TwoSum.  Error bound (S = |u_x.g| + |u_y.g| + |v_x.g| + |v_y.g|): the input
// pairs are within 3 * 2^-49 of the exact differences (at most 2^-47 S),
// every remainder |r| <= 2^-23 makes each FMA's rounding at most
// 2^-24 (2^-24 |p| + 2^-23 (|u.g| + |v.g|)), and the final additions add
// 2^-47 (|p| + |q| + S); with |p| + |q| <= S^2 / 4 everything stays below
// cert_bound_g(S) = 2^-44 S + 2^-44 S^2 + 2^-64.
__device__ __forceinline__ df cross_gd(gd ux, gd uy, gd vx, gd vy)
{
    const float p = __fmul_rn(ux.g, vy.g);
    float e = __fmaf_rn(ux.g, vy.g, -p);
    e = __fmaf_rn(ux.g, vy.r, e);
    e = __fmaf_rn(ux.r, vy.g, e);
    e = __fmaf_rn(ux.r, vy.r, e);
    const float q = __fmul_rn(uy.g, vx.g);
    float f = __fmaf_rn(uy.g, vx.g, -q);
    f = __fmaf_rn(uy.g, vx.r, f);
    f = __fmaf_rn(uy.r, vx.g, f);
    f = __fmaf_rn(uy.r, vx.r, f);
    float s, t;
    two_sum_f(p, -q, s, t);
    t = __fadd_rn(t, __fsub_rn(e, f));
    df n;
    fast_two_sum_f(s, t, n.h, n.l);
    return n;
}

__device__ __forceinline__ float cert_bound_g(float S) { return S * __fmaf_rn(S, 0x1p-44f, 0x1p-44f) + 0x1p-64f; }

// Exact signs of the edges selected by `need` (bit k: the edge opposite
// W_k) of the triangle (W0, W1, W2), on the double coordinates and the exact
// foot (one inlined copy of the staged predicate for all three edges).
// Packed result: bits 2k..2k+1 the sign of edge k (0: 0, 1: +1, 2: -1),
// bits 8..9 the tests decided by the expansion, bits 10..11 those decided by
// the double filter, bit 12 a coordinate outside the exact range.
__device__ __forceinline__ uint32_t exact_signs(const double2 *xyd, int w0, int w1, int w2, df X, df Y, uint32_t need)
{
    // The foot is loop-invariant: without this barrier the compiler hoists
    // its float -> double conversions (FP64-pipe work) out of the rare branch
    // that calls this function into every node's path.
    asm volatile("" : "+f"(X.h), "+f"(X.l), "+f"(Y.h), "+f"(Y.l));
    const double2 Ad = xyd[w0], Bd = xyd[w1], Cd = xyd[w2];
    uint32_t out = 0, n3 = 0, n2 = 0;
    for (int k = 0; k < 3; ++k) {
        if (!(need >> k & 1u)) continue;
        const double2 P = k == 0 ? Bd : (k == 1 ? Cd : Ad), Q = k == 0 ? Cd : (k == 1 ? Ad : Bd);
        int stg = 0;
        const int sg = orient_exact_df(P, Q, X.h, X.l, Y.h, Y.l, stg);
        out |= (sg > 0 ? 1u : (sg < 0 ? 2u : 0u)) << (2 * k);
        n3 += stg == 3;
        n2 += stg == 2;
    }
    const bool in_range = slp::in_exact_range(Ad.x) && slp::in_exact_range(Ad.y) && slp::in_exact_range(Bd.x) &&
                          slp::in_exact_range(Bd.y) && slp::in_exact_range(Cd.x) && slp::in_exact_range(Cd.y) &&
                          slp::in_exact_range(X.h) && slp::in_exact_range(Y.h) && slp::in_exact_range(X.l) &&
                          slp::in_exact_range(Y.l);
    return out | (n3 << 8) | (n2 << 10) | (in_range ? 0u : 1u << 12);
}

__device__ __forceinline__ int unpack_sign(uint32_t r, int k)
{
    const uint32_t v = (r >> (2 * k)) & 3u;
    return v == 1u ? 1 : (v == 2u ? -1 : 0);
}

// Randomised visibility walk step: a uniformly drawn negative edge (signs
// s1..s3 of the edges opposite W0..W2, at least one negative).
__device__ __forceinline__ int random_negative_edge(int64_t i, uint32_t hops, int s1, int s2, int s3)
{
    const int neg[3] = {s1 < 0, s2 < 0, s3 < 0};
    const int nneg = neg[0] + neg[1] + neg[2];
    int pick = (int)(mix64_dev(((uint64_t)i << 20) ^ (uint64_t)hops) % (uint64_t)nneg);
    int k = -1;
    for (int q = 0; q < 3; ++q)
        if (neg[q] && pick-- == 0) k = q;
    return k;
}

// The three barycentric numerators of the foot X (pair form) in the triangle
// (A, B, C) (vertex pairs (gx, gy, rx, ry)), relative to C, with their
// certification bounds:  n1 = orient(B, C, X) (theta of A), n2 = orient(C, A,
// X) (theta of B), den = orient(A, B, C) > 0, and theta of C's numerator
// den - n1 - n2 from the high parts, n3h, with its bound e3 (the low parts
// and two roundings add at most 2^-22 of the terms).
struct Certified {
    df n1, n2, den;
    float ea, eb, ed, n3h, e3;
};

// The numerators alone, with the |.|-sums of the grid differences of A, B
// and the foot relative to C that their bounds take.
struct Numerators {
    df n1, n2, den;
    float sA, sB, sX;
};

__device__ __forceinline__ Numerators numerators(float4 A, float4 B, float4 C, float Xg, float Xr, float Yg,
                                                 float Yr)
{
    const gd dAx = gd_sub(A.x, A.z, C.x, C.z), dAy = gd_sub(A.y, A.w, C.y, C.w);
    const gd dBx = gd_sub(B.x, B.z, C.x, C.z), dBy = gd_sub(B.y, B.w, C.y, C.w);
    const gd dXx = gd_sub(Xg, Xr, C.x, C.z), dXy = gd_sub(Yg, Yr, C.y, C.w);
    Numerators t;
    t.n1 = cross_gd(dXx, dXy, dBx, dBy);
    t.n2 = cross_gd(dAx, dAy, dXx, dXy);
    t.den = cross_gd(dAx, dAy, dBx, dBy);
    t.sA = fabsf(dAx.g) + fabsf(dAy.g);
    t.sB = fabsf(dBx.g) + fabsf(dBy.g);
    t.sX = fabsf(dXx.g) + fabsf(dXy.g);
    return t;
}

__device__ __forceinline__ Certified certify_bounds(const Numerators &n)
{
    Certified t;
    t.n1 = n.n1;
    t.n2 = n.n2;
    t.den = n.den;
    t.ea = cert_bound_g(n.sX + n.sB);
    t.eb = cert_bound_g(n.sA + n.sX);
    t.ed = cert_bound_g(n.sA + n.sB);
    t.n3h = __fsub_rn(__fsub_rn(t.den.h, t.n1.h), t.n2.h);
    t.e3 = t.ed + t.ea + t.eb + 0x1p-22f * (fabsf(t.den.h) + fabsf(t.n1.h) + fabsf(t.n2.h));
    return t;
}

__device__ __forceinline__ Certified certify(float4 A, float4 B, float4 C, float Xg, float Xr, float Yg, float Yr)
{
    return certify_bounds(numerators(A, B, C, Xg, Xr, Yg, Yr));
}

// 1 / d to about 2^-24 relative: the hardware approximation refined by one
// Newton step.  d is twice a triangle's area, far above the subnormal range
// for any triangle with vertices on the grid of 2^-24.
__device__ __forceinline__ float rcp_refined(float d)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return __fmaf_rn(r, __fmaf_rn(-d, r, 1.0f), r);
}

// The P1 value (Remark 1) with the barycentric coordinates of Eq. 6,
// theta_k = n_k / den:  V = v3 + (n1 (v1 - v3) + n2 (v2 - v3)) / den, in
// double-float: the value differences from a TwoSum of the high parts, the
// products from their exact FMA remainders, and the quotient by one
// correction step (Karp and Markstein's division: q1 = w r, the residual
// w - q1 den from two FMAs, q2 = residual r), about 2^-45 relative.
__device__ __forceinline__ float2 p1_value_of(float2 V1, float2 V2, float2 V3, df n1, df n2, df den)
{
    float d1h, d1l, d2h, d2l;
    two_sum_f(V1.x, -V3.x, d1h, d1l);
    d1l = __fadd_rn(d1l, __fsub_rn(V1.y, V3.y));
    two_sum_f(V2.x, -V3.x, d2h, d2l);
    d2l = __fadd_rn(d2l, __fsub_rn(V2.y, V3.y));
    const float p1 = __fmul_rn(n1.h, d1h), p2 = __fmul_rn(n2.h, d2h);
    float q1 = __fmaf_rn(n1.h, d1h, -p1), q2 = __fmaf_rn(n2.h, d2h, -p2);
    q1 = __fmaf_rn(n1.h, d1l, q1);
    q1 = __fmaf_rn(n1.l, d1h, q1);
    q2 = __fmaf_rn(n2.h, d2l, q2);
    q2 = __fmaf_rn(n2.l, d2h, q2);
    float ws, wt;
    two_sum_f(p1, p2, ws, wt);
    wt = __fadd_rn(wt, __fadd_rn(q1, q2));
    const float r = rcp_refined(den.h);
    const float c1 = __fmul_rn(ws, r);
    const float rho = __fadd_rn(__fmaf_rn(-c1, den.h, ws), __fmaf_rn(-c1, den.l, wt));
    const df v = df_add(dfp(V3), df_make(c1, __fmul_rn(rho, r)));
    return make_float2(v.h, v.l);
}

// V^n is steep in the triangle (SL_OPT_PRECISE): max_k (v_k - v_3)^2 >
// G^2 den on the high parts, den twice the area, so that max |v_k - v_3| / sqrt(den)
// -- about the P1 gradient -- exceeds G.  The double-float value is then off
// by more than about 2^-46 G, and precise_value takes over.
__device__ __forceinline__ bool steep(float2 V1, float2 V2, float2 V3, float den_h, float g2)
{
    const float d1 = __fsub_rn(V1.x, V3.x), d2 = __fsub_rn(V2.x, V3.x);
    return fmaxf(__fmul_rn(d1, d1), __fmul_rn(d2, d2)) > __fmul_rn(g2, den_h);
}

__device__ __forceinline__ double wide(float2 p) { return __dadd_rn((double)p.x, (double)p.y); }

// The P1 value of an unclipped node in FP64, on its located triangle (w0,
// w1, w2): the Euler foot X = x_i - dt f(x_i, t_{n+1}) (Eq. 4) from the
// node's double coordinates, with the step's constants and the node tables
// widened from their float pairs (48 bits of constants whose product with
// the node's velocity, the displacement, is far below 1: within about 2^-52
// of the double foot); then the barycentric coordinates of Eq. 6 on the
// triangle's double vertices and the interpolation of Remark 1, all in
// double.  Returns the value as a (hi, lo) pair.  Rare (steep data only), so
// kept out of line: its double registers do not weigh on the walk.
static __device__ __noinline__ float2 precise_value(const double2 *__restrict__ xyd, const float4 *__restrict__ g1,
                                             const float4 *__restrict__ g2, const FastProb &P, int64_t i, int w0,
                                             int w1, int w2, float2 V1, float2 V2, float2 V3)
{
    const double2 x = xyd[i];
    double X = x.x, Y = x.y;
    const double c0 = wide(P.c[0]), c1 = wide(P.c[1]), c2 = wide(P.c[2]);
    switch (P.kind) {
    case SL_FIELD_AFFINE: {
        const double c3 = wide(P.c[3]), c4 = wide(P.c[4]), c5 = wide(P.c[5]);
        X = x.x - ((c0 + c1 * x.x) + c2 * x.y);
        Y = x.y - ((c3 + c4 * x.x) + c5 * x.y);
        break;
    }
    case SL_FIELD_ROTATION:     // c0 = dt p0, (c1, c2) = centre (either split sums to it)
        X = x.x + c0 * (x.y - c2);
        Y = x.y - c0 * (x.x - c1);
        break;
    case SL_FIELD_SWIRL: {
        const float4 g = g1[i];
        X = x.x - c0 * wide(make_float2(g.x, g.z));
        Y = x.y - c0 * wide(make_float2(g.y, g.w));
        break;
    }
    case SL_FIELD_PAPER:
    case SL_FIELD_FOURIER8: {
        const float4 g = g1[i], q = g2[i];
        X = x.x - (c0 * wide(make_float2(g.x, g.z)) + c1 * wide(make_float2(q.x, q.z)));
        Y = x.y - (c0 * wide(make_float2(g.y, g.w)) + c1 * wide(make_float2(q.y, q.w)));
        break;
    }
    default: break;
    }
    const double2 A = xyd[w0], B = xyd[w1], C = xyd[w2];
    const double den = (B.y - C.y) * (A.x - C.x) + (C.x - B.x) * (A.y - C.y);
    const double t1 = ((B.y - C.y) * (X - C.x) + (C.x - B.x) * (Y - C.y)) / den;
    const double t2 = ((C.y - A.y) * (X - C.x) + (A.x - C.x) * (Y - C.y)) / den;
    const double v3 = wide(V3);
    const double v = v3 + t1 * (wide(V1) - v3) + t2 * (wide(V2) - v3);
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}


// A foot that comes out of the foot arithmetic as its own node's stored
// coordinate pair, bit for bit, is that node (see step_node): a boundary
// node whose velocity points out of the square is clipped at the start of
// its segment, and a node where the field vanishes does not move.
__device__ __forceinline__ bool foot_is_node(df x, df y, df X, df Y)
{
    return X.h == x.h && X.l == x.l && Y.h == y.h && Y.l == y.l;
}

// A foot with both high parts strictly inside (0, 1) needs neither the
// boundary rounding nor the clip (both act only at or beyond a side).
__device__ __forceinline__ bool df_inside(df X, df Y)
{
    return X.h > 0.0f && X.h < 1.0f && Y.h > 0.0f && Y.h < 1.0f;
}

__device__ __forceinline__ void foot_to_grid(df &X, df &Y)
{
    float g, r;
    to_grid(X, g, r);
    X = df_make(g, r);
    to_grid(Y, g, r);
    Y = df_make(g, r);
}

// The foot of node i for this step: Euler (Eq. 4) in double-float, in the
// (grid, remainder) form of the certified test.  A foot well inside the
// square comes straight in that form (foot_grid); any other is summed in
// double-float, decided against the boundary in double rounding, clipped and
// then split.  Returns true when clipped.  at_node: a foot on or beyond a side
// that is the node itself (an outward boundary node); a foot inside the
// square is not reported here.
template <int kKind>
__device__ __forceinline__ bool foot_pair(const FastArgs &a, int64_t i, const FastProb &P, df &X, df &Y,
                                          bool &at_node)
{
    const float4 xq = a.xyq[i];
    const df x = df_make(xq.x, xq.z), y = df_make(xq.y, xq.w);
    df DX, DY;
    if (kKind < 0) disp_df(P, a, i, x, y, DX, DY);
    else disp_df_k<kKind < 0 ? 0 : kKind>(P, a, i, x, y, DX, DY);
    at_node = false;
    if (foot_grid(x, DX, X) & foot_grid(y, DY, Y)) return false;
    X = df_add(x, DX);
    Y = df_add(y, DY);
    const bool inside = df_inside(X, Y);
    bool clipped = false;
    if (!inside) {
        round_boundary(X);
        round_boundary(Y);
        clipped = clip_df(x, y, X, Y);
    }
    at_node = !inside && foot_is_node(x, y, X, Y);
    foot_to_grid(X, Y);
    return clipped;
}

// FP32 hops on the high parts while one of the two exits of the current
// triangle (W0, W1, W2) = (p0, p1, p2), entered through its third edge, is
// certainly negative (hop_bound); e0, e1: the half-edge codes of the edges
// opposite W0 and W1.  One 16-byte half-edge record per hop.
//
// The loop keeps the vertices relative to the foot, a_k = W_k - X: grid
// values minus a grid value, exact in float, so a new vertex costs two
// subtractions and each orientation one product and one FMA:
// orient(W1, W2, X) = a1 x a2, orient(W2, W0, X) = a2 x a0.  Each a_k is
// within 2^-24 of the exact difference, which with the product roundings
// stays below hop_bound(S), S = the sum of the six |a|.  The more negative
// exit is taken (the first on a tie), as in the certified walk.  A boundary
// record carries NaN coordinates: the next test fails and the loop ends, its
// first code naming an edge of the triangle the walk is still in.
//
// A walk that is still going after kLeanPlain hops continues in runs that
// share one bound.  Where the test with the triangle's own bound passes, the
// next kLeanRun hops are tested against hop_bound(3 (M + kLeanRun L)), M the
// largest |a_k|_1 of that triangle and L (FastArgs::hop_L) the longest edge
// of the mesh in the same norm: each hop's new vertex shares an edge with a
// vertex of the triangle before, so after j hops every |a_k|_1 is at most M
// + j L and S at most three times that.  A test that fails against the run's
// bound is taken again with the triangle's own, so the hops, where the loop
// stops and every result are those of a test with S at every hop, at about a
// quarter fewer instructions per hop.  Short walks, most of a steady step's,
// keep the bound per hop and skip the setting up of runs.
constexpr uint32_t kLeanPlain = 4;
constexpr uint32_t kLeanRun = 16;

__device__ __forceinline__ float lean_run_bound(float m0, float m1, float m2, float L)
{
    return hop_bound(__fmul_ru(3.0f, __fmaf_ru((float)kLeanRun, L, fmaxf(fmaxf(m0, m1), m2))));
}

// The lean walk on either record form: Rec::hop(c2) crosses the exit opposite
// W1 (c2) or W0 and returns the new vertex relative to the foot, given the
// kept slot-0 vertex.
template <typename Rec>
__device__ __forceinline__ void lean_walk(Rec &rec, float a0x, float a0y, float a1x, float a1y, float a2x, float a2y,
                                          uint32_t &hops, uint32_t cap, float L)
{
    float o1, o2;
    // the first hops, each on its own bound
    for (uint32_t n = 0;; ++n) {
        if (hops >= cap) return;
        o1 = __fmaf_rn(a1x, a2y, -__fmul_rn(a1y, a2x));    // ~ theta of W0 * den
        o2 = __fmaf_rn(a2x, a0y, -__fmul_rn(a2y, a0x));    // ~ theta of W1 * den
        const float S = fabsf(a0x) + fabsf(a0y) + fabsf(a1x) + fabsf(a1y) + fabsf(a2x) + fabsf(a2y);
        if (!(fminf(o1, o2) < -hop_bound(S))) return;
        if (n == kLeanPlain) break;
        const bool c2 = o2 < o1;
        if (c2) { a1x = a2x; a1y = a2y; }
        else { a0x = a2x; a0y = a2y; }
        rec.hop(c2, a0x, a0y, a2x, a2y);
        ++hops;
    }
    // runs: the test at the current triangle has passed
    for (;;) {
        const float hb = lean_run_bound(fabsf(a0x) + fabsf(a0y), fabsf(a1x) + fabsf(a1y), fabsf(a2x) + fabsf(a2y), L);
        const uint32_t lim = min(cap, hops + kLeanRun);
        for (;;) {
            const bool c2 = o2 < o1;
            if (c2) { a1x = a2x; a1y = a2y; }
            else { a0x = a2x; a0y = a2y; }
            rec.hop(c2, a0x, a0y, a2x, a2y);
            if (++hops >= lim) break;
            o1 = __fmaf_rn(a1x, a2y, -__fmul_rn(a1y, a2x));
            o2 = __fmaf_rn(a2x, a0y, -__fmul_rn(a2y, a0x));
            if (!(fminf(o1, o2) < -hb)) break;
        }
        if (hops >= cap) return;
        o1 = __fmaf_rn(a1x, a2y, -__fmul_rn(a1y, a2x));
        o2 = __fmaf_rn(a2x, a0y, -__fmul_rn(a2y, a0x));
        const float S = fabsf(a0x) + fabsf(a0y) + fabsf(a1x) + fabsf(a1y) + fabsf(a2x) + fabsf(a2y);
        if (!(fminf(o1, o2) < -hop_bound(S))) return;
    }
}

// 16-byte records: the new vertex's hop coordinates and both exit codes.
struct Rec16 {
    const float4 *he;
    float fx, fy;
    int32_t e0, e1;
    __device__ __forceinline__ void hop(bool c2, float, float, float &a2x, float &a2y)
    {
        const float4 Q = __ldg(&he[c2 ? e1 : e0]);
        a2x = __fsub_rn(Q.x, fx);
        a2y = __fsub_rn(Q.y, fy);
        e0 = __float_as_int(Q.z);
        e1 = __float_as_int(Q.w);
    }
};

__device__ __forceinline__ void lean_hops(const FastArgs &a, float fx, float fy, float p0x, float p0y, float p1x,
                                          float p1y, float p2x, float p2y, int32_t &e0, int32_t &e1, uint32_t &hops,
                                          uint32_t cap)
{
    Rec16 r{a.he, fx, fy, e0, e1};
    lean_walk(r, __fsub_rn(p0x, fx), __fsub_rn(p0y, fy), __fsub_rn(p1x, fx), __fsub_rn(p1y, fy), __fsub_rn(p2x, fx),
              __fsub_rn(p2y, fy), hops, cap, a.hop_L);
    e0 = r.e0;
    e1 = r.e1;
}

// Triangle of a half-edge code h = 3 t + k (h >= 0).
__device__ __forceinline__ int32_t tri_of(int32_t h) { return (int32_t)__umulhi((uint32_t)h, 0xAAAAAAABu) >> 1; }

// Fields of a compact record (k_build_he8).  he8_offx / he8_offy: 0.5 + b
// 2^-24 for the biased delta b, by its bits; subtracting kHe8Bias (0.5 +
// 2^-7) leaves d 2^-24 exactly, d = Q - W0 of the entered triangle.  he8_e0:
// the exit code opposite W0 of the entered triangle; he8_d1: the step from
// it to the exit opposite W1.
constexpr float kHe8Bias = 0.5078125f;
__device__ __forceinline__ float he8_offx(uint2 R) { return __uint_as_float((R.x & 0x3FFFFu) | 0x3F000000u); }
__device__ __forceinline__ float he8_offy(uint2 R)
{
    return __uint_as_float((__funnelshift_r(R.x, R.y, 18) & 0x3FFFFu) | 0x3F000000u);
}
__device__ __forceinline__ int32_t he8_e0(uint2 R) { return (int32_t)(R.y >> 5); }
__device__ __forceinline__ int32_t he8_d1(uint2 R) { return 1 - 3 * (int32_t)((R.y >> 4) & 1u); }

// The same FP32 hops on 8-byte half-edge records (k_build_he8), for meshes
// fine enough that every edge is within 2^17 grid units (of 2^-24).  State as
// in lean_hops, with the vertices already relative to the foot, a_k = W_k -
// X, and the exits e0 and e0 + d1.  Crossing the exit opposite W_c loads
// that half-edge's record; the entered triangle's W0 is the vertex the
// current state keeps in slot 0 after the crossing (W0 when c = 1, W2 when c
// = 0), and its new vertex is that W0 + d: a2 = a0 + (he8_off - kHe8Bias),
// exact (multiples of 2^-24 below 1).  A hop is taken only across an edge the
// foot lies certainly beyond, never a boundary edge for a foot in the
// square; a boundary record would decode to the current triangle anyway.
// 8-byte records: the new vertex as an offset from the entered triangle's
// W0, the slot-0 vertex the state keeps after the crossing.
struct Rec8 {
    const uint2 *he8;
    int32_t e0, d1;
    __device__ __forceinline__ void hop(bool c2, float a0x, float a0y, float &a2x, float &a2y)
    {
        const uint2 Q = __ldg(&he8[c2 ? e0 + d1 : e0]);
        a2x = __fadd_rn(__fsub_rn(he8_offx(Q), kHe8Bias), a0x);
        a2y = __fadd_rn(__fsub_rn(he8_offy(Q), kHe8Bias), a0y);
        e0 = he8_e0(Q);
        d1 = he8_d1(Q);
    }
};

__device__ __forceinline__ void lean_hops8(const uint2 *__restrict__ he8, float a0x, float a0y, float a1x, float a1y,
                                           float a2x, float a2y, int32_t &e0, int32_t &d1, uint32_t &hops,
                                           uint32_t cap, float L)
{
    Rec8 r{he8, e0, d1};
    lean_walk(r, a0x, a0y, a1x, a1y, a2x, a2y, hops, cap, L);
    e0 = r.e0;
    d1 = r.d1;
}

// The new vertex of a compact record, W0 + d, with W0 (the entered
// triangle's first vertex) a hop coordinate.
__device__ __forceinline__ float2 he8_vertex(uint2 R, float wx, float wy)
{
    return make_float2(__fadd_rn(__fsub_rn(he8_offx(R), kHe8Bias), wx),
                       __fadd_rn(__fsub_rn(he8_offy(R), kHe8Bias), wy));
}

// Debug output of a foot held as a float pair (h, l): feet receives the sum
// rounded to double and feet_lo the exact rest (Knuth's TwoSum in double), so
// that feet + feet_lo is, exactly, the point the kernel located.  One double
// cannot always hold the pair: a remainder far below the grid part's last bit
// puts more than 53 bits between them.
__device__ __forceinline__ void write_foot(const FastArgs &a, int64_t i, df X, df Y)
{
    const double xh = X.h, xl = X.l, yh = Y.h, yl = Y.l;
    const double sx = __dadd_rn(xh, xl), sy = __dadd_rn(yh, yl);
    if (a.dbg.feet) {
        a.dbg.feet[2 * i] = sx;
        a.dbg.feet[2 * i + 1] = sy;
    }
    if (a.dbg.feet_lo) {
        const double bx = __dsub_rn(sx, xh), by = __dsub_rn(sy, yh);
        a.dbg.feet_lo[2 * i] = __dadd_rn(__dsub_rn(xh, __dsub_rn(sx, bx)), __dsub_rn(xl, bx));
        a.dbg.feet_lo[2 * i + 1] = __dadd_rn(__dsub_rn(yh, __dsub_rn(sy, by)), __dsub_rn(yl, by));
    }
}

// Debug output of a foot that is its own node (see step_node): the point
// located is the node's double coordinate, not the float pair it was found
// equal to.
__device__ __forceinline__ void write_node_foot(const FastArgs &a, int64_t i)
{
    const double2 p = a.xyd[i];
    if (a.dbg.feet) {
        a.dbg.feet[2 * i] = p.x;
        a.dbg.feet[2 * i + 1] = p.y;
    }
    if (a.dbg.feet_lo) {
        a.dbg.feet_lo[2 * i] = 0.0;
        a.dbg.feet_lo[2 * i + 1] = 0.0;
    }
}

struct NodeCounters {
    uint32_t hops = 0, exact = 0, clipped = 0, fallback = 0, limit = 0, filter2 = 0, excluded = 0;
};


// One node of the step.
//
// FP32 walk state: the current triangle as its vertices (W0, W1, W2),
// counter-clockwise, and the half-edge codes e0, e1 of its edges opposite
// W0 and W1 (code 3 j + s: edge s of triangle j, opposite its vertex s).
// Crossing an edge loads one 16-byte half-edge record (the next triangle's
// new vertex and its two exit codes, see k_build_he), so an FP32 hop is a
// single gather.  The edge the walk came through is never a candidate
// again: it was crossed because the foot lies strictly beyond it, so its
// barycentric coordinate in the new triangle is positive.  The certified
// test and the value always take the triangle's vertices in slot order
// (T[0][j], T[1][j], T[2][j]), so the result depends on the located triangle
// and the foot only, not on the path of the walk.
template <bool kDebug, bool kExt, bool kCompact>
__device__ __forceinline__ void step_node(const FastArgs &a, int64_t i, int pi, NodeCounters &c)
{
    const FastProb &P = a.probs[pi];
    const float4 xq = a.xyq[i];
    const df x = df_make(xq.x, xq.z), y = df_make(xq.y, xq.w);
    df DX, DY;
    disp_df(P, a, i, x, y, DX, DY);
    df X, Y;
    uint32_t flags = 0;
    bool at_node;
    // From here on the foot is in its (grid, remainder) form, Xg + Xr
    // exactly, the form the certified test needs (the exact stage takes any
    // float pair).  A foot well inside the square comes straight in that form
    // (foot_grid, as in the settle pass; a node whose field vanishes keeps its
    // own pair there); any other is summed in double-float, decided against
    // the boundary, excluded or clipped, and then split (0 and 1 are grid
    // points, so the split does not move a foot off a side).
    if (foot_grid(x, DX, X) & foot_grid(y, DY, Y)) {
        at_node = foot_is_node(x, y, X, Y);
    } else {
        X = df_add(x, DX);
        Y = df_add(y, DY);
        round_boundary(X);
        round_boundary(Y);
        if (kExt && a.exclude && (df_neg_strict(X) || df_gt1(X) || df_neg_strict(Y) || df_gt1(Y))) {
            // the paper's experiments exclude nodes whose foot leaves the
            // domain (Sec. 4): V unchanged, no walk, T^0 unchanged
            ((float2 *)a.vout)[i] = ((const float2 *)a.vin)[i];
            c.excluded = 1;
            if (a.parent) {
                // strategy (c): the children start where this node would have
                a.t0[i] = a.t0[a.parent[i]];
                a.t0v[i] = a.t0v[a.parent[i]];
            }
            if (kDebug) {
                write_foot(a, i, X, Y);
                if (a.dbg.tri) a.dbg.tri[i] = -1;
                if (a.dbg.moves) a.dbg.moves[i] = 0;
                if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)SL_NODE_EXCLUDED;
            }
            return;
        }
        if (clip_df(x, y, X, Y)) {
            flags |= SL_NODE_CLIPPED;
            c.clipped = 1;
        }
        at_node = foot_is_node(x, y, X, Y);
        float g, r;
        to_grid(X, g, r);
        X = df_make(g, r);
        to_grid(Y, g, r);
        Y = df_make(g, r);
    }
    const float &Xg = X.h, &Xr = X.l, &Yg = Y.h, &Yr = Y.l;

    // start triangle and its vertex ids from the per-node cache (one
    // coalesced 16-byte load), or from the direct location on a structured
    // grid
    const int4 tq = kExt && a.grid_M > 0 ? __ldg(&a.grid_t0v[grid_slot(X.h, Y.h, a.grid_M)])
                                         : a.t0v[kExt && a.parent ? (int64_t)a.parent[i] : i];
    // A foot that is the node itself lies on a vertex: when the start
    // triangle has node i as a vertex it contains the foot (two barycentric
    // coordinates are zero) and the P1 value is the node's own value.  The
    // double-float pair is only within 2^-49 of the node's double
    // coordinate, so without this the exact stage would run on a
    // rounding-sized offset every step.
    if (at_node && (tq.y == (int32_t)i || tq.z == (int32_t)i || tq.w == (int32_t)i)) {
        const int32_t j0 = tri_of(tq.x);
        ((float2 *)a.vout)[i] = ((const float2 *)a.vin)[i];
        if (kExt && a.parent && !a.keep_t0) {
            a.t0[i] = j0;
            a.t0v[i] = tq;
        }
        if (kDebug) {
            write_node_foot(a, i);
            if (a.dbg.tri) a.dbg.tri[i] = j0;
            if (a.dbg.moves) a.dbg.moves[i] = 0;
            if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)(flags | SL_NODE_DEGENERATE);
        }
        return;
    }
    int32_t e0 = tq.x, e1 = 0;
    int32_t j = 0;
    int w0 = tq.y, w1 = tq.z, w2 = tq.w;
    bool ids = true;           // w0..w2 are the vertex ids of the current triangle
    const uint32_t cap = (uint32_t)a.walk_cap;
    uint32_t &hops = c.hops;
    bool found = false;
    int s1 = 0, s2 = 0, s3 = 0;
    df n1, n2, den;
    if (cap > 0) {
        // A foot that moved is usually clear of its start triangle: test the
        // three edges of T^0 in FP32 first and, when one is certainly
        // negative, hop at once (the certified test then runs where the FP32
        // walk stops).  The vertex pairs come through L1, where a certified
        // test of T^0 finds them again.
        const float4 A = a.xyq[w0], B = a.xyq[w1], C = a.xyq[w2];
        const float ax = A.x - C.x, ay = A.y - C.y, bx = B.x - C.x, by = B.y - C.y;
        const float xx = X.h - C.x, xy = Y.h - C.y;
        const float o1 = __fmaf_rn(xx, by, -__fmul_rn(xy, bx));
        const float o2 = __fmaf_rn(ax, xy, -__fmul_rn(ay, xx));
        const float dn = __fmaf_rn(ax, by, -__fmul_rn(ay, bx));
        const float o3 = dn - o1 - o2;
        const float S = fabsf(ax) + fabsf(ay) + fabsf(bx) + fabsf(by) + fabsf(xx) + fabsf(xy);
        const float e = hop_bound(S);
        const float e3 = 3.0f * e + 0x1p-23f * (fabsf(dn) + fabsf(o1) + fabsf(o2));
        int k = -1;
        float best = 0.0f;
        if (o1 < -e) { k = 0; best = o1; }
        if (o2 < -e && (k < 0 || o2 < best)) { k = 1; best = o2; }
        if (o3 < -e3 && (k < 0 || o3 < best)) { k = 2; best = o3; }
        if (kCompact && k >= 0) {
            const uint2 R = __ldg(&a.he8[tq.x + k]);
            if (tri_of(he8_e0(R)) != tri_of(tq.x)) {     // not a boundary edge
                // the next triangle: (W2, W1, Q), (W0, W2, Q) or (W1, W0, Q),
                // Q = its first vertex + the record's offset
                const float p0x = k == 1 ? A.x : (k == 0 ? C.x : B.x), p0y = k == 1 ? A.y : (k == 0 ? C.y : B.y);
                const float p1x = k == 0 ? B.x : (k == 1 ? C.x : A.x), p1y = k == 0 ? B.y : (k == 1 ? C.y : A.y);
                const float2 Q = he8_vertex(R, p0x, p0y);
                e0 = he8_e0(R);
                e1 = he8_d1(R);     // compact records: e1 holds the step to the second exit
                ids = false;
                ++hops;
                lean_hops8(a.he8, __fsub_rn(p0x, X.h), __fsub_rn(p0y, Y.h), __fsub_rn(p1x, X.h), __fsub_rn(p1y, Y.h),
                           __fsub_rn(Q.x, X.h), __fsub_rn(Q.y, Y.h), e0, e1, hops, cap, a.hop_L);
            }
        } else if (k >= 0) {
            const float4 R = __ldg(&a.he[tq.x + k]);
            if (!isnan(R.x)) {
                // the next triangle: (W2, W1, Q), (W0, W2, Q) or (W1, W0, Q)
                float p0x = k == 1 ? A.x : (k == 0 ? C.x : B.x), p0y = k == 1 ? A.y : (k == 0 ? C.y : B.y);
                float p1x = k == 0 ? B.x : (k == 1 ? C.x : A.x), p1y = k == 0 ? B.y : (k == 1 ? C.y : A.y);
                float p2x = R.x, p2y = R.y;
                e0 = __float_as_int(R.z);
                e1 = __float_as_int(R.w);
                ids = false;
                ++hops;
                lean_hops(a, X.h, Y.h, p0x, p0y, p1x, p1y, p2x, p2y, e0, e1, hops, cap);
            }
        }
    }
    for (;;) {
        // certified test in double-float on (W0, W1, W2) = the vertices in
        // slot order, relative to W2
        j = tri_of(e0);
        if (!ids) {
            w0 = a.tv[0][j];
            w1 = a.tv[1][j];
            w2 = a.tv[2][j];
            ids = true;
        }
        // vertices as (grid, remainder) pairs: (gx, gy, rx, ry)
        const float4 A = a.xyq[w0], B = a.xyq[w1], C = a.xyq[w2];
        const Certified t = certify(A, B, C, Xg, Xr, Yg, Yr);
        n1 = t.n1;
        n2 = t.n2;
        den = t.den;
        const float ea = t.ea, eb = t.eb, ed = t.ed;
        s1 = n1.h > ea ? 1 : (n1.h < -ea ? -1 : 2);
        s2 = n2.h > eb ? 1 : (n2.h < -eb ? -1 : 2);
        float n3h = t.n3h;
        s3 = n3h > t.e3 ? 1 : (n3h < -t.e3 ? -1 : 2);
        if (s3 == 2) {
            const df n3 = df_sub(df_sub(den, n1), n2);
            const float ec = ed + ea + eb + 0x1p-45f * (fabsf(den.h) + fabsf(n1.h) + fabsf(n2.h));
            n3h = n3.h;
            s3 = n3.h > ec ? 1 : (n3.h < -ec ? -1 : 2);
        }
        if (s1 == 2 || s2 == 2 || s3 == 2) {
            // a boundary edge with the foot on its side of the square: exactly 0
            // (fside: the sides the foot lies on, bit = boundary side code)
            const uint32_t fside = (df_is(X, 0.0f) ? 1u : 0u) | (df_is(X, 1.0f) ? 2u : 0u) |
                                   (df_is(Y, 0.0f) ? 4u : 0u) | (df_is(Y, 1.0f) ? 8u : 0u);
            if (s1 == 2) { const int32_t nb = a.tn[0][j]; if (nb < 0 && (fside >> (-1 - nb) & 1u)) s1 = 0; }
            if (s2 == 2) { const int32_t nb = a.tn[1][j]; if (nb < 0 && (fside >> (-1 - nb) & 1u)) s2 = 0; }
            if (s3 == 2) { const int32_t nb = a.tn[2][j]; if (nb < 0 && (fside >> (-1 - nb) & 1u)) s3 = 0; }
        }
        if (s1 == 2 || s2 == 2 || s3 == 2) {
            // exact signs on the double coordinates and the exact foot
            const uint32_t r = exact_signs(a.xyd, w0, w1, w2, X, Y, (s1 == 2 ? 1u : 0u) | (s2 == 2 ? 2u : 0u) | (s3 == 2 ? 4u : 0u));
            if (s1 == 2) s1 = unpack_sign(r, 0);
            if (s2 == 2) s2 = unpack_sign(r, 1);
            if (s3 == 2) s3 = unpack_sign(r, 2);
            c.exact += (r >> 8) & 3u;
            c.filter2 += (r >> 10) & 3u;
            flags |= SL_NODE_EXACT;
            if (r & (1u << 12)) flags |= SL_NODE_RANGE;
        }
        if (s1 >= 0 && s2 >= 0 && s3 >= 0) {
            found = true;
            break;
        }
        if (hops >= 2 * cap) break;
        int k;
        if (hops < cap) {
            // the paper's rule: the most negative barycentric coordinate
            k = -1;
            float best = 0.0f;
            if (s1 < 0) { k = 0; best = n1.h; }
            if (s2 < 0 && (k < 0 || n2.h < best)) { k = 1; best = n2.h; }
            if (s3 < 0 && (k < 0 || n3h < best)) { k = 2; best = n3h; }
        } else {
            // after `cap` hops: randomised visibility walk (certified at
            // every triangle), which terminates on any triangulation
            if (hops == cap) {
                c.fallback = 1;
                flags |= SL_NODE_FALLBACK;
            }
            k = random_negative_edge(i, hops, s1, s2, s3);
        }
        if (kCompact) {
            const uint2 R = __ldg(&a.he8[3 * j + k]);
            if (tri_of(he8_e0(R)) == j) break;    // a boundary edge: not for a foot inside a valid mesh
            const float2 P0 = a.xyh[k == 1 ? w0 : (k == 0 ? w2 : w1)], P1 = a.xyh[k == 0 ? w1 : (k == 1 ? w2 : w0)];
            const float2 Q = he8_vertex(R, P0.x, P0.y);
            e0 = he8_e0(R);
            e1 = he8_d1(R);
            ids = false;
            ++hops;
            lean_hops8(a.he8, __fsub_rn(P0.x, X.h), __fsub_rn(P0.y, Y.h), __fsub_rn(P1.x, X.h), __fsub_rn(P1.y, Y.h),
                       __fsub_rn(Q.x, X.h), __fsub_rn(Q.y, Y.h), e0, e1, hops, cap, a.hop_L);
            continue;
        }
        const float4 R = __ldg(&a.he[3 * j + k]);
        if (isnan(R.x)) break;    // a boundary edge: not for a foot inside a valid mesh
        // the next triangle: (W2, W1, Q), (W0, W2, Q) or (W1, W0, Q); the
        // high parts of the kept vertices are reloaded (L1 hits) rather than
        // kept live through the certified test
        const float2 P0 = a.xyh[k == 1 ? w0 : (k == 0 ? w2 : w1)], P1 = a.xyh[k == 0 ? w1 : (k == 1 ? w2 : w0)];
        float p0x = P0.x, p0y = P0.y, p1x = P1.x, p1y = P1.y;
        float p2x = R.x, p2y = R.y;
        e0 = __float_as_int(R.z);
        e1 = __float_as_int(R.w);
        ids = false;
        ++hops;
        // FP32 hops on the high parts while an edge is certainly negative
        lean_hops(a, X.h, Y.h, p0x, p0y, p1x, p1y, p2x, p2y, e0, e1, hops, cap);
    }
    if (!found) {
        flags |= SL_NODE_WALK_LIMIT;
        c.limit = 1;
    }
    if (s1 == 0 || s2 == 0 || s3 == 0) flags |= SL_NODE_DEGENERATE;

    // the P1 value (Remark 1) with the barycentric coordinates of Eq. 6, in
    // FP64 where V^n is steep (SL_OPT_PRECISE)
    {
        const float2 *vin = (const float2 *)a.vin;
        const float2 V1 = vin[w0], V2 = vin[w1], V3 = vin[w2];
        if (!(flags & SL_NODE_CLIPPED) && steep(V1, V2, V3, den.h, a.steep_g2)) {
            ((float2 *)a.vout)[i] = precise_value(a.xyd, a.g1, a.g2, P, i, w0, w1, w2, V1, V2, V3);
            flags |= SL_NODE_PRECISE;
        } else {
            ((float2 *)a.vout)[i] = p1_value_of(V1, V2, V3, n1, n2, den);
        }
    }
    if ((hops > 0 || (kExt && a.parent)) && !(kExt && a.keep_t0)) {
        a.t0[i] = j;
        a.t0v[i] = make_int4(3 * j, w0, w1, w2);
    }
    if (c.limit) atomicOr(a.status, 1u << SL_E_WALK_LIMIT);
    if (flags & SL_NODE_RANGE) atomicOr(a.status, 1u << SL_E_ARG);
    if (kDebug) {
        write_foot(a, i, X, Y);
        if (a.dbg.tri) a.dbg.tri[i] = j;
        if (a.dbg.moves) a.dbg.moves[i] = (int32_t)hops;
        if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)flags;
    }
}

// kExt: the variant with the options of the paper's experiments (exclusion,
// strategies (a), (c) and the direct structured-grid start); the default
// variant compiles them out and keeps its registers for the walk.
template <bool kStats, bool kDebug, int kBlock, int kMinBlocks, bool kExt, bool kCompact>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_step_fast_df(FastArgs a)
{
    const int64_t i = kExt ? node_of_thread(a) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = kExt ? i >= 0 : i < a.N;
    pdl_launch_dependents();
    pdl_wait();
    NodeCounters c;
    // the node's problem: the chunk table, or a search per node in a spanning-tree
    // level (a level mixes problems)
    const int pi = !active || a.nprob == 1 ? 0
                   : (kExt && a.order ? problem_of(a.node_off, a.nprob, i) : chunk_problem(a.chunk_prob, a.node_off, i));
    if (active) step_node<kDebug, kExt, kCompact>(a, i, pi, c);
    if (kStats) warp_stats(a.stats, active, c.hops, c.exact, c.clipped, c.fallback, c.limit, c.filter2, c.excluded);
}

// The settle pass's test: one bound for the three numerators (ea, eb, ed <=
// E), looser than the certified test's, so a node settled here is settled
// there too.
__device__ __forceinline__ bool settle_test(const Numerators &t)
{
    const float E = cert_bound_g(t.sA + t.sB + t.sX);
    const float n3h = __fsub_rn(__fsub_rn(t.den.h, t.n1.h), t.n2.h);
    return fminf(t.n1.h, t.n2.h) > E && n3h > 3.0f * E + 0x1p-22f * (fabsf(t.den.h) + fabsf(t.n1.h) + fabsf(t.n2.h));
}

// A node the settle test left undecided: 0 = to the finish pass, 1 = settled
// in T^0 with the barycentric value and a sign exactly zero (the foot on a
// boundary edge), 2 = settled with the node's own value, 3 = settled in T^0,
// every sign certified positive.
//  * The foot is node i (as in step_node).  When T^0 has node i as a vertex,
//    two of its signs are zero, so the test cannot have passed: settled with
//    the node's value.  (A foot inside the square at its node, f = 0 there,
//    is left to the finish pass, which takes the same decision.)
//  * Otherwise the signs are taken as step_node's certified test takes them
//    at T^0: the per-numerator bounds, the double-float third numerator, and
//    a zero sign for a foot on a side of the square (clipped onto it, or
//    there by itself) across the boundary edge of its triangle on that side
//    (the side codes).  A negative sign, or one those stages leave undecided
//    (the exact stage), leaves the node to the finish pass.
__device__ __forceinline__ int settle_decide(const FastArgs &a, int64_t i, int4 tq, df X, df Y, bool clipped,
                                             bool at_node, const Numerators &t)
{
    if (at_node) return (tq.y == (int32_t)i || tq.z == (int32_t)i || tq.w == (int32_t)i) ? 2 : 0;
    // the signs exactly as step_node's certified test takes them
    const Certified u = certify_bounds(t);
    const int s1 = u.n1.h > u.ea ? 1 : (u.n1.h < -u.ea ? -1 : 2);
    const int s2 = u.n2.h > u.eb ? 1 : (u.n2.h < -u.eb ? -1 : 2);
    int s3 = u.n3h > u.e3 ? 1 : (u.n3h < -u.e3 ? -1 : 2);
    if (s3 == 2) {
        const df n3 = df_sub(df_sub(u.den, u.n1), u.n2);
        const float ec = u.ed + u.ea + u.eb + 0x1p-45f * (fabsf(u.den.h) + fabsf(u.n1.h) + fabsf(u.n2.h));
        s3 = n3.h > ec ? 1 : (n3.h < -ec ? -1 : 2);
    }
    if (s1 < 0 || s2 < 0 || s3 < 0) return 0;
    const uint32_t fside = (df_is(X, 0.0f) ? 1u : 0u) | (df_is(X, 1.0f) ? 2u : 0u) | (df_is(Y, 0.0f) ? 4u : 0u) |
                           (df_is(Y, 1.0f) ? 8u : 0u);
    const int32_t j = tri_of(tq.x);
    const int32_t nb1 = s1 == 2 ? a.tn[0][j] : 0, nb2 = s2 == 2 ? a.tn[1][j] : 0, nb3 = s3 == 2 ? a.tn[2][j] : 0;
    if (s1 == 2 && !(nb1 < 0 && (fside >> (-1 - nb1) & 1u))) return 0;
    if (s2 == 2 && !(nb2 < 0 && (fside >> (-1 - nb2) & 1u))) return 0;
    if (s3 == 2 && !(nb3 < 0 && (fside >> (-1 - nb3) & 1u))) return 0;
    return (s1 == 2 || s2 == 2 || s3 == 2) ? 1 : 3;
}

// Settle pass of a split step: the nodes whose foot is certainly in the
// start triangle (all three signs certified positive, or zero by a boundary
// side code for a clipped foot; no hop, no exact stage) are finished here
// with a lean kernel; every other node is appended
// to the queue for the finish pass, which runs the full node step on it.  The
// foot, the certified test and the value are the same functions as in
// step_node, so the split does not change any result.
template <bool kDebug, int kKind>
__device__ __forceinline__ bool settle_node(const FastArgs &a, int64_t i, int pi, NodeCounters &c)
{
    const FastProb &P = kKind < 0 ? a.probs[pi] : a.prob0;
    df X, Y;
    bool at_node;
    const bool clipped = foot_pair<kKind>(a, i, P, X, Y, at_node);
    const int4 tq = a.t0v[i];
    const float4 A = a.xyq[tq.y], B = a.xyq[tq.z], C = a.xyq[tq.w];
    // the start triangle's values are read together with its vertices, not
    // after the test: most feet stay in it, and the value then costs no
    // further round trip to memory
    const float2 *vin = (const float2 *)a.vin;
    const float2 V1 = vin[tq.y], V2 = vin[tq.z], V3 = vin[tq.w];
    const Numerators t = numerators(A, B, C, X.h, X.l, Y.h, Y.l);
    bool degenerate = false;
    if (!settle_test(t)) {
        const int d = settle_decide(a, i, tq, X, Y, clipped, at_node, t);
        if (d == 0) return false;
        if (d == 2) {
            ((float2 *)a.vout)[i] = vin[i];
            c.clipped = clipped;
            if (kDebug) {
                write_node_foot(a, i);
                if (a.dbg.tri) a.dbg.tri[i] = tri_of(tq.x);
                if (a.dbg.moves) a.dbg.moves[i] = 0;
                if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)((clipped ? SL_NODE_CLIPPED : 0u) | SL_NODE_DEGENERATE);
            }
            return true;
        }
        degenerate = d == 1;
    }
    const float2 val = p1_value_of(V1, V2, V3, t.n1, t.n2, t.den);
    // steep V^n: the finish pass evaluates the value in FP64 (step_node).
    // (Calling that out-of-line path from here put a stack frame and the call
    // convention on this pass, which then ran slower in recorded runs than
    // the finish pass's occasional node costs.)
    if (!clipped && steep(V1, V2, V3, t.den.h, a.steep_g2)) return false;
    ((float2 *)a.vout)[i] = val;
    c.clipped = clipped;
    if (kDebug) {
        write_foot(a, i, X, Y);
        if (a.dbg.tri) a.dbg.tri[i] = tri_of(tq.x);
        if (a.dbg.moves) a.dbg.moves[i] = 0;
        if (a.dbg.flags)
            a.dbg.flags[i] = (uint8_t)((clipped ? SL_NODE_CLIPPED : 0u) | (degenerate ? SL_NODE_DEGENERATE : 0u));
    }
    return true;
}

// kKind >= 0: a single problem of that field kind, whose constants come
// from the kernel parameters (a.prob0); -1: any problems.
template <bool kStats, bool kDebug, int kBlock, int kMinBlocks, int kKind>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_settle_df(FastArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < a.N;
    pdl_launch_dependents();
    pdl_wait();
    NodeCounters c;
    const int pi = kKind < 0 && active && a.nprob > 1 ? chunk_problem(a.chunk_prob, a.node_off, i) : 0;
    // the next step's counter (its previous user, the finish pass of the
    // step before, has completed)
    if (a.queue_next && blockIdx.x == 0 && threadIdx.x == 0) *a.queue_next = 0;
    const bool queued = active && !settle_node<kDebug, kKind>(a, i, pi, c);
    // warp-aggregated append to the queue of the finish pass
    const unsigned mask = __ballot_sync(0xffffffffu, queued);
    if (mask) {
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(a.queue_count, (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (queued) a.queue[base + (uint32_t)__popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
    }
    if (kStats) warp_stats(a.stats, active && !queued, 0u, 0u, active && !queued ? c.clipped : 0u, 0u, 0u);
}

// Finish pass: the full node step (certified walk, exact stage, value) for
// the queued nodes, a persistent grid striding over the queue.
template <bool kStats, bool kDebug, bool kCompact>
__global__ void __launch_bounds__(128, 8) k_finish_df(FastArgs a)
{
    pdl_launch_dependents();
    pdl_wait();
    const uint32_t count = *a.queue_count;
    NodeCounters tot;
    uint32_t done = 0, hmax = 0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        NodeCounters c;
        const int64_t i = a.queue[q];
        step_node<kDebug, false, kCompact>(a, i, a.nprob == 1 ? 0 : chunk_problem(a.chunk_prob, a.node_off, i), c);
        tot.hops += c.hops;
        hmax = c.hops > hmax ? c.hops : hmax;
        tot.exact += c.exact;
        tot.filter2 += c.filter2;
        tot.clipped += c.clipped;
        tot.fallback += c.fallback;
        tot.limit += c.limit;
        ++done;
    }
    if (kStats) {
        // a thread may have finished several nodes: its sums go in whole
        const unsigned full = 0xffffffffu;
        const unsigned n = __reduce_add_sync(full, done), h = __reduce_add_sync(full, tot.hops);
        const unsigned hm = __reduce_max_sync(full, hmax), e = __reduce_add_sync(full, tot.exact);
        const unsigned f2 = __reduce_add_sync(full, tot.filter2), cl = __reduce_add_sync(full, tot.clipped);
        const unsigned fb = __reduce_add_sync(full, tot.fallback), l = __reduce_add_sync(full, tot.limit);
        if ((threadIdx.x & 31) == 0) {
            if (n) atomicAdd(&a.stats[0], (unsigned long long)n);
            if (h) atomicAdd(&a.stats[1], (unsigned long long)h);
            if (hm) atomicMax(&a.stats[2], (unsigned long long)hm);
            if (e) atomicAdd(&a.stats[3], (unsigned long long)e);
            if (f2) atomicAdd(&a.stats[4], (unsigned long long)f2);
            if (cl) atomicAdd(&a.stats[5], (unsigned long long)cl);
            if (fb) atomicAdd(&a.stats[6], (unsigned long long)fb);
            if (l) atomicAdd(&a.stats[7], (unsigned long long)l);
        }
    }
}

template <int kBlock, int kMinBlocks, bool kExt, bool kCompact>
inline void launch_fast_df_form(const FastArgs &a, bool stats, bool debug, unsigned grid, cudaStream_t s)
{
    if (stats) {
        if (debug) launch_step_kernel(k_step_fast_df<true, true, kBlock, kMinBlocks, kExt, kCompact>, grid, kBlock, s, a);
        else launch_step_kernel(k_step_fast_df<true, false, kBlock, kMinBlocks, kExt, kCompact>, grid, kBlock, s, a);
    } else {
        if (debug) launch_step_kernel(k_step_fast_df<false, true, kBlock, kMinBlocks, kExt, kCompact>, grid, kBlock, s, a);
        else launch_step_kernel(k_step_fast_df<false, false, kBlock, kMinBlocks, kExt, kCompact>, grid, kBlock, s, a);
    }
}

// compact 8-byte records when the mesh has them (a.he8), else 16-byte ones
template <int kBlock, int kMinBlocks, bool kExt = false>
inline void launch_fast_df_cfg(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    const unsigned grid = (unsigned)((a.count + kBlock - 1) / kBlock);
    if (grid == 0) return;
    if (a.he8) launch_fast_df_form<kBlock, kMinBlocks, kExt, true>(a, stats, debug, grid, s);
    else launch_fast_df_form<kBlock, kMinBlocks, kExt, false>(a, stats, debug, grid, s);
}

}  // namespace sl
