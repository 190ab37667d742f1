/*
 * sl_oracle.c -- plain CPU oracle for one semi-Lagrangian step
 *                (Euler foot -> boundary clip -> point location -> P1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes, for node x_i of a triangulation of the unit square and a
 * step n -> n+1 (paper: Cacace & Ferretti, "Efficient implementation of
 * characteristic-based schemes on unstructured triangular grids"):
 *
 *   1. t = (n+1) dt and the Euler foot X = x_i - dt f(x_i, t)      (Eq. 4,
 *      "eulero"; restated at the start of Sec. 3).  The paper's Algorithm 2
 *      writes f(x_i, t_n) instead; this oracle follows the equation.
 *   2. Boundary clip: the paper stops characteristics on the boundary
 *      (Sec. 1, text after Eq. 4) without giving the rule.  Reading taken
 *      here: if X leaves [0,1]^2, stop the segment x_i -> X at the first
 *      boundary crossing, put every coordinate that attains that crossing
 *      exactly on 0 or 1, clamp the other coordinate to [0,1].
 *   3. Point location.  The walk of Algorithm 1 reaches a triangle that
 *      contains X; when X is strictly inside a triangle that triangle is
 *      unique, so the oracle does not walk: it finds the containing triangle
 *      directly.  Candidates come from a uniform bin grid (a triangle is
 *      listed in every bin its bounding box touches, the query uses the same
 *      bin map, so every containing triangle is a candidate); containment is
 *      decided with EXACT orientation signs (all three >= 0).  Among several
 *      containing triangles (X on an edge or vertex) the lowest index wins.
 *   4. Barycentric coordinates by Eq. 6 ("barycoords"), theta_3 = 1 -
 *      theta_1 - theta_2, and the P1 value theta_1 v_1 + theta_2 v_2 +
 *      theta_3 v_3 (Remark 1 of Sec. 2.2; Algorithm 2, interpolation loop).
 *
 * Floating point: compiled with -ffp-contract=off, so every operation is one
 * IEEE double operation in the order written.  Fields use the C library's
 * sin/cos/sqrt; sin(k pi x) and cos(k pi x) reduce k x modulo 2 exactly
 * first (sincos_pi), so that they vanish exactly where the definition makes
 * them vanish: the swirl and stream-function fields are then exactly tangent
 * to the sides of the square, as their definitions make them.
 *
 * Exact orientation: a double-precision evaluation with a forward error
 * bound, and, when the bound cannot certify the sign, an exact evaluation
 * with multi-limb integers (each double written as m * 2^e and all six
 * coordinates scaled to a common exponent).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "sl_oracle.h"

/* ------------------------------------------------------------------ */
/* Fields                                                               */
/* ------------------------------------------------------------------ */

static const double PI = 3.14159265358979323846;


/* sin(pi v) and cos(pi v) with the argument reduced exactly: r = v - 2
 * round(v / 2) is exact (for v = 2n + r with n != 0, v and 2n are within a
 * factor of two), so at integer and half-integer v the values are the exact
 * 0 and +-1 of the definition; elsewhere the library's sin and cos of pi r. */
static void sincos_pi(double v, double *s, double *c)
{
    const double r = v - 2.0 * nearbyint(0.5 * v);
    if (r == 0.0) {
        *s = 0.0;
        *c = 1.0;
    } else if (r == 1.0 || r == -1.0) {
        *s = 0.0;
        *c = -1.0;
    } else if (r == 0.5 || r == -0.5) {
        *s = r > 0.0 ? 1.0 : -1.0;
        *c = 0.0;
    } else {
        *s = sin(PI * r);
        *c = cos(PI * r);
    }
}

void orc_field(int kind, const double *p, double x, double y, double t,
               double *fx, double *fy)
{
    switch (kind) {
    case ORC_FIELD_ZERO:
        *fx = 0.0;
        *fy = 0.0;
        return;
    case ORC_FIELD_AFFINE:
        /* f_x = p0 + p1 x + p2 y + p3 t,  f_y = p4 + p5 x + p6 y + p7 t */
        *fx = p[0] + p[1] * x + p[2] * y + p[3] * t;
        *fy = p[4] + p[5] * x + p[6] * y + p[7] * t;
        return;
    case ORC_FIELD_ROTATION:
        /* solid rotation with angular speed p0 about (p1, p2) */
        *fx = p[0] * (p[2] - y);
        *fy = p[0] * (x - p[1]);
        return;
    case ORC_FIELD_SWIRL: {
        /* cos(pi t / T) (sin^2(pi x) sin(2 pi y), -sin^2(pi y) sin(2 pi x)) */
        double c = cos(PI * t / p[0]);
        double sx, cx, sy, cy, s2x, s2y;
        sincos_pi(x, &sx, &cx);
        sincos_pi(y, &sy, &cy);
        sincos_pi(2.0 * x, &s2x, &cx);
        sincos_pi(2.0 * y, &s2y, &cy);
        *fx = c * (sx * sx) * s2y;
        *fy = -c * (sy * sy) * s2x;
        return;
    }
    case ORC_FIELD_FOURIER8: {
        /* psi = sum_m a_m cos(2 pi t + phi_m) sin(k_m pi x) sin(l_m pi y);
         * f = (d psi / dy, -d psi / dx). */
        double gx = 0.0, gy = 0.0;
        for (int m = 0; m < 8; ++m) {
            double k = p[4 * m], l = p[4 * m + 1], a = p[4 * m + 2], phi = p[4 * m + 3];
            double am = a * cos(2.0 * PI * t + phi);
            double skx, ckx, sly, cly;
            sincos_pi(k * x, &skx, &ckx);
            sincos_pi(l * y, &sly, &cly);
            gx += am * skx * (l * PI) * cly;
            gy -= am * (k * PI) * ckx * sly;
        }
        *fx = gx;
        *fy = gy;
        return;
    }
    case ORC_FIELD_PAPER: {
        /* Sec. 4: (cos(C0 |x - c| + C1 t), sin(C0 |x - c| + C1 t)) */
        double dx = x - p[2], dy = y - p[3];
        double arg = p[0] * sqrt(dx * dx + dy * dy) + p[1] * t;
        *fx = cos(arg);
        *fy = sin(arg);
        return;
    }
    default:
        *fx = NAN;
        *fy = NAN;
        return;
    }
}

/* Boundary clip (reading of Sec. 1): if q leaves [0,1]^2, stop the segment
 * x -> q at its first boundary crossing; every coordinate that attains the
 * crossing is set exactly to 0 or 1, the other one is clamped to [0,1].
 * Returns 1 if q was outside. */
static int clip_segment(double x, double y, double qx, double qy, double *X, double *Y)
{
    if (qx >= 0.0 && qx <= 1.0 && qy >= 0.0 && qy <= 1.0) {
        *X = qx;
        *Y = qy;
        return 0;
    }
    double dx = qx - x, dy = qy - y;
    double sx = 2.0, sy = 2.0;         /* > 1 means "this axis is not violated" */
    double bx = 0.0, by = 0.0;
    if (qx < 0.0) { sx = (0.0 - x) / dx; bx = 0.0; }
    if (qx > 1.0) { sx = (1.0 - x) / dx; bx = 1.0; }
    if (qy < 0.0) { sy = (0.0 - y) / dy; by = 0.0; }
    if (qy > 1.0) { sy = (1.0 - y) / dy; by = 1.0; }
    double s = sx < sy ? sx : sy;
    double cx = x + s * dx;
    double cy = y + s * dy;
    if (sx == s) cx = bx;
    if (sy == s) cy = by;
    if (cx < 0.0) cx = 0.0;
    if (cx > 1.0) cx = 1.0;
    if (cy < 0.0) cy = 0.0;
    if (cy > 1.0) cy = 1.0;
    *X = cx;
    *Y = cy;
    return 1;
}

/* Euler foot (Eq. 4) followed by the boundary clip.  Returns 1 if clipped. */
int orc_foot(int kind, const double *p, double dt, double t, double x, double y,
             double *X, double *Y)
{
    double fx, fy;
    orc_field(kind, p, x, y, t, &fx, &fy);
    double qx = x - dt * fx;
    double qy = y - dt * fy;
    return clip_segment(x, y, qx, qy, X, Y);
}

/* ------------------------------------------------------------------ */
/* Exact orientation sign                                               */
/* ------------------------------------------------------------------ */

/* Signed multi-limb integer: value = sign * sum_k d[k] 2^(32 k). */
#define BIG_LIMBS 144           /* 4608 bits: enough for products of any two
                                   finite doubles brought to a common scale */
typedef struct {
    int sign;                   /* -1, 0, +1 */
    int n;                      /* limbs in use */
    uint32_t d[BIG_LIMBS];
} big;

static void big_set_scaled(big *r, int64_t m, int shift)
{
    /* r = m * 2^shift, shift >= 0, |m| < 2^63 */
    memset(r, 0, sizeof(*r));
    if (m == 0) return;
    r->sign = m < 0 ? -1 : 1;
    uint64_t a = (uint64_t)(m < 0 ? -m : m);
    int limb = shift / 32, bit = shift % 32;
    /* a << bit spans at most 3 limbs */
    uint64_t lo = a << bit;                        /* low 64 bits */
    uint64_t hi = bit ? (a >> (64 - bit)) : 0;     /* overflow bits */
    r->d[limb] = (uint32_t)lo;
    r->d[limb + 1] = (uint32_t)(lo >> 32);
    r->d[limb + 2] = (uint32_t)hi;
    r->n = limb + 3;
    while (r->n > 0 && r->d[r->n - 1] == 0) r->n--;
}

static int big_cmp_mag(const big *a, const big *b)
{
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int k = a->n - 1; k >= 0; --k)
        if (a->d[k] != b->d[k]) return a->d[k] < b->d[k] ? -1 : 1;
    return 0;
}

static void mag_add(big *r, const big *a, const big *b)
{
    int n = a->n > b->n ? a->n : b->n;
    uint64_t carry = 0;
    for (int k = 0; k < n; ++k) {
        uint64_t s = carry + (k < a->n ? a->d[k] : 0) + (k < b->n ? b->d[k] : 0);
        r->d[k] = (uint32_t)s;
        carry = s >> 32;
    }
    r->n = n;
    if (carry) r->d[r->n++] = (uint32_t)carry;
}

static void mag_sub(big *r, const big *a, const big *b)   /* |a| >= |b| */
{
    int64_t borrow = 0;
    for (int k = 0; k < a->n; ++k) {
        int64_t s = (int64_t)a->d[k] - (k < b->n ? b->d[k] : 0) - borrow;
        borrow = s < 0;
        r->d[k] = (uint32_t)(s + (borrow ? ((int64_t)1 << 32) : 0));
    }
    r->n = a->n;
    while (r->n > 0 && r->d[r->n - 1] == 0) r->n--;
}

/* r = a + sb * b, sb = +1 or -1 (r may not alias a or b) */
static void big_addsub(big *r, const big *a, const big *b, int sb)
{
    int bs = b->sign * sb;
    memset(r, 0, sizeof(*r));
    if (b->sign == 0) { *r = *a; return; }
    if (a->sign == 0) { *r = *b; r->sign = bs; return; }
    if (a->sign == bs) {
        mag_add(r, a, b);
        r->sign = bs;
        return;
    }
    int c = big_cmp_mag(a, b);
    if (c == 0) return;
    if (c > 0) { mag_sub(r, a, b); r->sign = a->sign; }
    else       { mag_sub(r, b, a); r->sign = bs; }
}

static void big_mul(big *r, const big *a, const big *b)
{
    memset(r, 0, sizeof(*r));
    if (a->sign == 0 || b->sign == 0) return;
    for (int i = 0; i < a->n; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < b->n; ++j) {
            uint64_t cur = (uint64_t)a->d[i] * b->d[j] + r->d[i + j] + carry;
            r->d[i + j] = (uint32_t)cur;
            carry = cur >> 32;
        }
        int k = i + b->n;
        while (carry) {
            uint64_t cur = (uint64_t)r->d[k] + carry;
            r->d[k] = (uint32_t)cur;
            carry = cur >> 32;
            ++k;
        }
    }
    r->n = a->n + b->n;
    while (r->n > 0 && r->d[r->n - 1] == 0) r->n--;
    r->sign = a->sign * b->sign;
}

/* sign of det [bx-ax, cx-ax; by-ay, cy-ay] computed exactly */
static int orient_exact(const double v[6])
{
    /* v = ax, ay, bx, by, cx, cy */
    int64_t m[6];
    int e[6], emin = 1 << 30;
    for (int k = 0; k < 6; ++k) {
        if (v[k] == 0.0) { m[k] = 0; e[k] = 0; continue; }
        int ex;
        double f = frexp(v[k], &ex);        /* v = f 2^ex, 0.5 <= |f| < 1 */
        m[k] = (int64_t)ldexp(f, 53);       /* exact: |m| < 2^53 */
        e[k] = ex - 53;
        if (e[k] < emin) emin = e[k];
    }
    big b[6];
    for (int k = 0; k < 6; ++k) big_set_scaled(&b[k], m[k], m[k] ? e[k] - emin : 0);
    big dbx, dby, dcx, dcy, t1, t2, det;
    big_addsub(&dbx, &b[2], &b[0], -1);
    big_addsub(&dby, &b[3], &b[1], -1);
    big_addsub(&dcx, &b[4], &b[0], -1);
    big_addsub(&dcy, &b[5], &b[1], -1);
    big_mul(&t1, &dbx, &dcy);
    big_mul(&t2, &dby, &dcx);
    big_addsub(&det, &t1, &t2, -1);
    return det.sign;
}

static int g_force_exact = 0;
static long g_exact_calls = 0;     /* statistics only */

void orc_set_force_exact(int on) { g_force_exact = on; }
long orc_exact_calls(void) { return g_exact_calls; }

/* Sign of the orientation of (a, b, c): +1 if counter-clockwise, -1 if
 * clockwise, 0 if collinear.  Exact for all finite inputs. */
int orc_orient_sign(double ax, double ay, double bx, double by, double cx, double cy)
{
    if (!g_force_exact) {
        double t1 = (bx - ax) * (cy - ay);
        double t2 = (by - ay) * (cx - ax);
        double det = t1 - t2;
        double mag = fabs(t1) + fabs(t2);
        /* Each of the two products carries at most 3 roundings (two
         * differences, one product) and the final difference one more, so
         * |det - exact| <= (4u + O(u^2)) * mag with u = 2^-53.  The test
         * below uses 8u (= 2^-50) of margin, and leaves tiny magnitudes,
         * where underflow breaks relative bounds, to the exact path. */
        double bound = 0x1p-50 * mag;
        if (mag > 0x1p-900 && mag < 0x1p+900) {
            if (det > bound) return 1;
            if (det < -bound) return -1;
        }
    }
    __atomic_fetch_add(&g_exact_calls, 1, __ATOMIC_RELAXED);
    double v[6] = {ax, ay, bx, by, cx, cy};
    return orient_exact(v);
}

/* The same sign for a query point given as an unevaluated sum of two
 * doubles per coordinate, q = (qxh + qxl, qyh + qyl), taken exactly (a
 * double-float foot is such a sum, and one double cannot always hold it).
 * The determinant is linear in q:
 *   orient(a, b, q) = orient(a, b, qh) + (bx - ax) qyl - (by - ay) qxl,
 * evaluated exactly with the multi-limb integers on all eight inputs. */
static int orient_exact_pair(const double v[8])
{
    /* v = ax, ay, bx, by, qxh, qyh, qxl, qyl */
    int64_t m[8];
    int e[8], emin = 1 << 30;
    for (int k = 0; k < 8; ++k) {
        if (v[k] == 0.0) { m[k] = 0; e[k] = 0; continue; }
        int ex;
        double f = frexp(v[k], &ex);
        m[k] = (int64_t)ldexp(f, 53);
        e[k] = ex - 53;
        if (e[k] < emin) emin = e[k];
    }
    big b[8];
    for (int k = 0; k < 8; ++k) big_set_scaled(&b[k], m[k], m[k] ? e[k] - emin : 0);
    big dbx, dby, qx, qy, dqx, dqy, t1, t2, det;
    big_addsub(&dbx, &b[2], &b[0], -1);
    big_addsub(&dby, &b[3], &b[1], -1);
    big_addsub(&qx, &b[4], &b[6], 1);          /* qx = qxh + qxl exactly */
    big_addsub(&qy, &b[5], &b[7], 1);
    big_addsub(&dqx, &qx, &b[0], -1);
    big_addsub(&dqy, &qy, &b[1], -1);
    big_mul(&t1, &dbx, &dqy);
    big_mul(&t2, &dby, &dqx);
    big_addsub(&det, &t1, &t2, -1);
    return det.sign;
}

/* Sign of orient(a, b, q) for q = (qxh + qxl, qyh + qyl), exact for all
 * finite inputs.  With qxl = qyl = 0 this is orc_orient_sign(a, b, qh). */
int orc_orient_sign2(double ax, double ay, double bx, double by, double qxh, double qyh, double qxl, double qyl)
{
    if (qxl == 0.0 && qyl == 0.0) return orc_orient_sign(ax, ay, bx, by, qxh, qyh);
    if (!g_force_exact) {
        double ex = bx - ax, ey = by - ay;
        double t1 = ex * (qyh - ay);
        double t2 = ey * (qxh - ax);
        double c1 = ex * qyl;
        double c2 = ey * qxl;
        double det = (t1 - t2) + (c1 - c2);
        double mag = fabs(t1) + fabs(t2) + fabs(c1) + fabs(c2);
        /* t1, t2 carry at most 3 roundings each, c1, c2 at most 2 (the
         * difference ex or ey and the product), and the three additions one
         * each: |det - exact| <= (8u + O(u^2)) mag, u = 2^-53.  2^-49 mag
         * doubles that margin; an underflowed c1 or c2 is off by at most
         * 2^-1074, far below it while mag > 2^-900. */
        double bound = 0x1p-49 * mag;
        if (mag > 0x1p-900 && mag < 0x1p+900) {
            if (det > bound) return 1;
            if (det < -bound) return -1;
        }
    }
    __atomic_fetch_add(&g_exact_calls, 1, __ATOMIC_RELAXED);
    double v[8] = {ax, ay, bx, by, qxh, qyh, qxl, qyl};
    return orient_exact_pair(v);
}

/* ------------------------------------------------------------------ */
/* Mesh with a uniform bin grid                                        */
/* ------------------------------------------------------------------ */

struct orc_mesh {
    int64_t n, nt;
    double *xy;          /* 2n */
    int32_t *tri;        /* 3nt */
    int B;               /* bins per side */
    int64_t *start;      /* B*B+1 offsets into items */
    int32_t *items;      /* triangle indices, ascending within each bin */
};

static int bin_of(double v, int B)
{
    double s = v * (double)B;           /* the same map for triangles and queries */
    if (!(s >= 0.0)) return 0;          /* also catches NaN */
    if (s >= (double)B) return B - 1;
    return (int)s;                      /* floor for s >= 0 */
}

orc_mesh *orc_mesh_create(int64_t n, int64_t nt, const double *xy, const int32_t *tri)
{
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    if (!m) return NULL;
    m->n = n;
    m->nt = nt;
    m->xy = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    m->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nt);
    if (!m->xy || !m->tri) { orc_mesh_destroy(m); return NULL; }
    memcpy(m->xy, xy, sizeof(double) * 2 * (size_t)n);
    memcpy(m->tri, tri, sizeof(int32_t) * 3 * (size_t)nt);
    int B = (int)ceil(sqrt((double)nt / 2.0));
    if (B < 1) B = 1;
    m->B = B;
    size_t nb = (size_t)B * B;
    m->start = (int64_t *)calloc(nb + 1, sizeof(int64_t));
    if (!m->start) { orc_mesh_destroy(m); return NULL; }
    /* two passes: count, then fill in ascending triangle order */
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fill = NULL;
        if (pass == 1) {
            for (size_t b = 0; b < nb; ++b) m->start[b + 1] += m->start[b];
            m->items = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m->start[nb] ? m->start[nb] : 1));
            fill = (int64_t *)malloc(sizeof(int64_t) * nb);
            if (!m->items || !fill) { free(fill); orc_mesh_destroy(m); return NULL; }
            memcpy(fill, m->start, sizeof(int64_t) * nb);
        }
        for (int64_t j = 0; j < nt; ++j) {
            double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
            for (int k = 0; k < 3; ++k) {
                int32_t v = tri[3 * j + k];
                double px = xy[2 * v], py = xy[2 * v + 1];
                if (px < xmin) xmin = px;
                if (px > xmax) xmax = px;
                if (py < ymin) ymin = py;
                if (py > ymax) ymax = py;
            }
            int i0 = bin_of(xmin, B), i1 = bin_of(xmax, B);
            int j0 = bin_of(ymin, B), j1 = bin_of(ymax, B);
            for (int bj = j0; bj <= j1; ++bj)
                for (int bi = i0; bi <= i1; ++bi) {
                    size_t b = (size_t)bj * B + bi;
                    if (pass == 0) m->start[b + 1]++;
                    else m->items[fill[b]++] = (int32_t)j;
                }
        }
        free(fill);
    }
    return m;
}

void orc_mesh_destroy(orc_mesh *m)
{
    if (!m) return;
    free(m->xy);
    free(m->tri);
    free(m->start);
    free(m->items);
    free(m);
}

int orc_mesh_bins(const orc_mesh *m) { return m->B; }

/* The three orientation signs of X against the edges of triangle j: s[k] is
 * the sign of the area of (X, opposite edge of vertex k), i.e. of theta_k. */
static void tri_signs(const orc_mesh *m, int64_t j, double X, double Y, int s[3])
{
    const int32_t *t = m->tri + 3 * j;
    double x1 = m->xy[2 * t[0]], y1 = m->xy[2 * t[0] + 1];
    double x2 = m->xy[2 * t[1]], y2 = m->xy[2 * t[1] + 1];
    double x3 = m->xy[2 * t[2]], y3 = m->xy[2 * t[2] + 1];
    s[0] = orc_orient_sign(x2, y2, x3, y3, X, Y);
    s[1] = orc_orient_sign(x3, y3, x1, y1, X, Y);
    s[2] = orc_orient_sign(x1, y1, x2, y2, X, Y);
}

int orc_locate(const orc_mesh *m, double X, double Y, int32_t *tri_out, int *flags)
{
    int B = m->B;
    size_t b = (size_t)bin_of(Y, B) * B + bin_of(X, B);
    int32_t best = -1;
    int count = 0, degen = 0;
    for (int64_t q = m->start[b]; q < m->start[b + 1]; ++q) {
        int32_t j = m->items[q];
        int s[3];
        tri_signs(m, j, X, Y, s);
        if (s[0] >= 0 && s[1] >= 0 && s[2] >= 0) {
            if (count == 0) {
                best = j;              /* items are ascending: lowest index */
                degen = (s[0] == 0 || s[1] == 0 || s[2] == 0);
            }
            count++;
        }
    }
    *tri_out = best;
    int f = 0;
    if (degen) f |= ORC_FLAG_DEGENERATE;
    if (count > 1) f |= ORC_FLAG_MULTI;
    *flags = f;
    return best >= 0 ? 0 : -1;
}

/* The three signs of tri_signs for a query point q = qh + ql (pair form). */
static void tri_signs2(const orc_mesh *m, int64_t j, double X, double Y, double Xl, double Yl, int s[3])
{
    const int32_t *t = m->tri + 3 * j;
    double x1 = m->xy[2 * t[0]], y1 = m->xy[2 * t[0] + 1];
    double x2 = m->xy[2 * t[1]], y2 = m->xy[2 * t[1] + 1];
    double x3 = m->xy[2 * t[2]], y3 = m->xy[2 * t[2] + 1];
    s[0] = orc_orient_sign2(x2, y2, x3, y3, X, Y, Xl, Yl);
    s[1] = orc_orient_sign2(x3, y3, x1, y1, X, Y, Xl, Yl);
    s[2] = orc_orient_sign2(x1, y1, x2, y2, X, Y, Xl, Yl);
}

/* orc_locate for the point (X + Xl, Y + Yl), taken exactly.  The bin is the
 * one of the rounded sums: a triangle's bins cover its bounding box
 * [bmin, bmax] through the same monotone map, and bmin <= q implies
 * bmin <= fl(q) for a double bmin (rounding to nearest is monotone), so every
 * containing triangle is still a candidate. */
int orc_locate2(const orc_mesh *m, double X, double Y, double Xl, double Yl, int32_t *tri_out, int *flags)
{
    int B = m->B;
    size_t b = (size_t)bin_of(Y + Yl, B) * B + bin_of(X + Xl, B);
    int32_t best = -1;
    int count = 0, degen = 0;
    for (int64_t q = m->start[b]; q < m->start[b + 1]; ++q) {
        int32_t j = m->items[q];
        int s[3];
        tri_signs2(m, j, X, Y, Xl, Yl, s);
        if (s[0] >= 0 && s[1] >= 0 && s[2] >= 0) {
            if (count == 0) {
                best = j;
                degen = (s[0] == 0 || s[1] == 0 || s[2] == 0);
            }
            count++;
        }
    }
    *tri_out = best;
    int f = 0;
    if (degen) f |= ORC_FLAG_DEGENERATE;
    if (count > 1) f |= ORC_FLAG_MULTI;
    *flags = f;
    return best >= 0 ? 0 : -1;
}

/* P1 value at (X, Y) in triangle j, by Eq. 6 and the interpolation formula
 * of Remark 1. */
double orc_interp(const orc_mesh *m, int32_t j, double X, double Y, const double *V)
{
    const int32_t *t = m->tri + 3 * (int64_t)j;
    double xi1 = m->xy[2 * t[0]], eta1 = m->xy[2 * t[0] + 1];
    double xi2 = m->xy[2 * t[1]], eta2 = m->xy[2 * t[1] + 1];
    double xi3 = m->xy[2 * t[2]], eta3 = m->xy[2 * t[2] + 1];
    double den = (eta2 - eta3) * (xi1 - xi3) + (xi3 - xi2) * (eta1 - eta3);
    double th1 = ((eta2 - eta3) * (X - xi3) + (xi3 - xi2) * (Y - eta3)) / den;
    double th2 = ((eta3 - eta1) * (X - xi3) + (xi1 - xi3) * (Y - eta3)) / den;
    double th3 = 1.0 - th1 - th2;
    return th1 * V[t[0]] + th2 * V[t[1]] + th3 * V[t[2]];
}

/* ------------------------------------------------------------------ */
/* One step over all nodes, threaded over contiguous node ranges         */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_mesh *m;
    int kind;
    const double *p;
    double dt, t;
    const double *vin;
    double *vout, *feet;
    int32_t *tri;
    uint8_t *flags;
    int64_t lo, hi;
    int exclude;
    int err;
} step_job;

static void *step_worker(void *arg)
{
    step_job *J = (step_job *)arg;
    const orc_mesh *m = J->m;
    for (int64_t i = J->lo; i < J->hi; ++i) {
        double X, Y;
        if (J->exclude) {
            /* Sec. 4: nodes whose Euler foot leaves the domain are excluded
             * from the computation; V keeps its value there */
            double fx, fy;
            orc_field(J->kind, J->p, m->xy[2 * i], m->xy[2 * i + 1], J->t, &fx, &fy);
            const double qx = m->xy[2 * i] - J->dt * fx, qy = m->xy[2 * i + 1] - J->dt * fy;
            if (!(qx >= 0.0 && qx <= 1.0 && qy >= 0.0 && qy <= 1.0)) {
                if (J->vout) J->vout[i] = J->vin[i];
                if (J->feet) { J->feet[2 * i] = qx; J->feet[2 * i + 1] = qy; }
                if (J->tri) J->tri[i] = -1;
                if (J->flags) J->flags[i] = (uint8_t)ORC_FLAG_EXCLUDED;
                continue;
            }
        }
        int clipped = orc_foot(J->kind, J->p, J->dt, J->t, m->xy[2 * i], m->xy[2 * i + 1], &X, &Y);
        int32_t j;
        int f;
        if (orc_locate(m, X, Y, &j, &f) != 0) { J->err = -1; j = -1; }
        if (clipped) f |= ORC_FLAG_CLIPPED;
        if (J->vout) J->vout[i] = j >= 0 ? orc_interp(m, j, X, Y, J->vin) : NAN;
        if (J->feet) { J->feet[2 * i] = X; J->feet[2 * i + 1] = Y; }
        if (J->tri) J->tri[i] = j;
        if (J->flags) J->flags[i] = (uint8_t)f;
    }
    return NULL;
}

static int run_jobs(step_job *tmpl, int64_t lo, int64_t hi, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int64_t total = hi - lo;
    if (total < (int64_t)nthreads * 64) nthreads = total > 64 ? (int)(total / 64) : 1;
    step_job jobs[256];
    pthread_t th[256];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k] = *tmpl;
        jobs[k].lo = lo + total * k / nthreads;
        jobs[k].hi = lo + total * (k + 1) / nthreads;
        jobs[k].err = 0;
    }
    int started = 0;
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, step_worker, &jobs[k]) != 0) break;
        started = k;
    }
    step_worker(&jobs[0]);
    for (int k = started + 1; k < nthreads; ++k) step_worker(&jobs[k]);   /* threads that failed to start */
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    int err = 0;
    for (int k = 0; k < nthreads; ++k) if (jobs[k].err) err = jobs[k].err;
    return err;
}

int orc_step_range(const orc_mesh *m, int kind, const double *p, double dt, int64_t n,
                   const double *vin, double *vout, double *feet, int32_t *tri, uint8_t *flags,
                   int64_t lo, int64_t hi, int nthreads)
{
    return orc_step_range_x(m, kind, p, dt, n, vin, vout, feet, tri, flags, lo, hi, nthreads, 0);
}

int orc_step_range_x(const orc_mesh *m, int kind, const double *p, double dt, int64_t n,
                     const double *vin, double *vout, double *feet, int32_t *tri, uint8_t *flags,
                     int64_t lo, int64_t hi, int nthreads, int exclude)
{
    step_job J;
    memset(&J, 0, sizeof(J));
    J.exclude = exclude;
    J.m = m;
    J.kind = kind;
    J.p = p;
    J.dt = dt;
    J.t = (double)(n + 1) * dt;        /* t_{n+1} */
    J.vin = vin;
    J.vout = vout;
    J.feet = feet;
    J.tri = tri;
    J.flags = flags;
    if (lo < 0) lo = 0;
    if (hi > m->n) hi = m->n;
    if (hi <= lo) return 0;
    return run_jobs(&J, lo, hi, nthreads);
}

int orc_step(const orc_mesh *m, int kind, const double *p, double dt, int64_t n,
             const double *vin, double *vout, double *feet, int32_t *tri, uint8_t *flags,
             int nthreads)
{
    return orc_step_range(m, kind, p, dt, n, vin, vout, feet, tri, flags, 0, m->n, nthreads);
}

int orc_run(const orc_mesh *m, int kind, const double *p, double dt, int64_t n0, int nsteps,
            double *v, double *scratch, int nthreads)
{
    double *a = v, *b = scratch;
    for (int s = 0; s < nsteps; ++s) {
        int err = orc_step(m, kind, p, dt, n0 + s, a, b, NULL, NULL, NULL, nthreads);
        if (err) return err;
        double *tmp = a; a = b; b = tmp;
    }
    if (a != v) memcpy(v, a, sizeof(double) * (size_t)m->n);
    return 0;
}

/* Batch location and sign triples of query points, threaded over
 * contiguous ranges.  Points are (q[2i] + ql[2i], q[2i+1] + ql[2i+1]),
 * taken exactly; ql may be NULL (points q). */
typedef struct {
    const orc_mesh *m;
    const double *q, *ql;
    const int32_t *tri_in;     /* sign mode: the triangle of each point */
    int32_t *tri;
    uint8_t *flags;
    int8_t *signs;             /* sign mode: 3 per point */
    int64_t lo, hi;
    int err;
} point_job;

static void *point_worker(void *arg)
{
    point_job *J = (point_job *)arg;
    for (int64_t i = J->lo; i < J->hi; ++i) {
        const double X = J->q[2 * i], Y = J->q[2 * i + 1];
        const double Xl = J->ql ? J->ql[2 * i] : 0.0, Yl = J->ql ? J->ql[2 * i + 1] : 0.0;
        if (J->signs) {
            int s[3] = {-2, -2, -2};          /* -2: not a triangle of the mesh */
            const int32_t j = J->tri_in[i];
            if (j >= 0 && j < J->m->nt) tri_signs2(J->m, j, X, Y, Xl, Yl, s);
            for (int k = 0; k < 3; ++k) J->signs[3 * i + k] = (int8_t)s[k];
            continue;
        }
        int32_t j;
        int f;
        if (orc_locate2(J->m, X, Y, Xl, Yl, &j, &f) != 0) J->err = -1;
        J->tri[i] = j;
        if (J->flags) J->flags[i] = (uint8_t)f;
    }
    return NULL;
}

static int run_points(point_job *tmpl, int64_t npts, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (npts < (int64_t)nthreads * 256) nthreads = npts > 256 ? (int)(npts / 256) : 1;
    point_job jobs[256];
    pthread_t th[256];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k] = *tmpl;
        jobs[k].lo = npts * k / nthreads;
        jobs[k].hi = npts * (k + 1) / nthreads;
        jobs[k].err = 0;
    }
    int started = 0;
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, point_worker, &jobs[k]) != 0) break;
        started = k;
    }
    point_worker(&jobs[0]);
    for (int k = started + 1; k < nthreads; ++k) point_worker(&jobs[k]);
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    int err = 0;
    for (int k = 0; k < nthreads; ++k) if (jobs[k].err) err = jobs[k].err;
    return err;
}

/* Locate arbitrary query points (no foot, no clip): the lowest-index
 * containing triangle and the flags of orc_locate.  Returns -1 if some point
 * lies in no triangle (its tri is -1). */
int orc_locate_points(const orc_mesh *m, int64_t npts, const double *q, int32_t *tri, uint8_t *flags)
{
    return orc_locate_points2(m, npts, q, NULL, tri, flags, 1);
}

int orc_locate_points2(const orc_mesh *m, int64_t npts, const double *q, const double *ql, int32_t *tri,
                       uint8_t *flags, int nthreads)
{
    point_job J;
    memset(&J, 0, sizeof(J));
    J.m = m;
    J.q = q;
    J.ql = ql;
    J.tri = tri;
    J.flags = flags;
    return run_points(&J, npts, nthreads);
}

/* Exact signs of each point against the three edges of a given triangle
 * (the edge opposite vertex k first, as tri_signs): the point lies in the
 * closed triangle iff all three are >= 0.  -2 marks an index that is not a
 * triangle of the mesh. */
void orc_tri_signs2(const orc_mesh *m, int64_t npts, const int32_t *tri, const double *q, const double *ql,
                    int8_t *signs, int nthreads)
{
    point_job J;
    memset(&J, 0, sizeof(J));
    J.m = m;
    J.q = q;
    J.ql = ql;
    J.tri_in = tri;
    J.signs = signs;
    run_points(&J, npts, nthreads);
}

void orc_feet(int kind, const double *p, double dt, int64_t n, int64_t npts, const double *xy,
              double *feet, uint8_t *clipped)
{
    double t = (double)(n + 1) * dt;
    for (int64_t i = 0; i < npts; ++i) {
        int c = orc_foot(kind, p, dt, t, xy[2 * i], xy[2 * i + 1], &feet[2 * i], &feet[2 * i + 1]);
        if (clipped) clipped[i] = (uint8_t)c;
    }
}
