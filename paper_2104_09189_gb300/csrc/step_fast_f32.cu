// step_fast_f32.cu -- the FP32 step kernel.
//
// The same step (Euler foot at t_{n+1}, boundary clip, barycentric walk from
// T^0_i -- strategy (b) of Sec. 3 -- and P1 interpolation, Eq. 6 and Remark
// 1) on a mesh whose coordinates are the double coordinates rounded to
// float, with float node values:
//
//  * the foot is evaluated in float with the operation order given below
//    (X = x - k g for table fields, ...); a foot that leaves the square is
//    clipped in double and rounded back to float (the coordinate on the
//    boundary is exactly 0 or 1);
//  * the coordinates are exact floats, so an FP32 orientation has the
//    classic forward error bound (3 + 16 e) e (|t1| + |t2|), e = 2^-24
//    (Shewchuk 1997, stage A, in single precision): each walk decision is
//    certified in FP32 and only undecided signs fall back to the double
//    predicate (a double filter, then an exact expansion) on the floats
//    promoted exactly -- the located triangle contains the float foot
//    exactly;
//  * theta_1, theta_2 (Eq. 6, relative to vertex 3) and the P1 value are
//    evaluated in float.
#include "predicates.cuh"
#include "step_common.cuh"
#include "step_fast.cuh"
#include "step_kernels.cuh"

namespace sl {

// Foot in float.  Operation order (each step one IEEE float operation):
//   AFFINE    f = (c0 + c1 x) + c2 y,  X = x - f   (and c3..c5 for Y)
//   ROTATION  X = x + c0 (y - c2),     Y = y - c0 (x - c1)
//   SWIRL     X = x - c0 g1x
//   PAPER,    X = x - (c0 g1x + c1 g2x)
//   FOURIER8
// with c_k = fl32 of the per-step constants and g = fl32 of the double node
// tables.
__device__ __forceinline__ void foot_f32(const FastProb &P, const FastArgs &a, int64_t i, float x, float y, float &X,
                                         float &Y)
{
    const float c0 = P.c[0].x, c1 = P.c[1].x, c2 = P.c[2].x;
    switch (P.kind) {
    case SL_FIELD_AFFINE: {
        const float c3 = P.c[3].x, c4 = P.c[4].x, c5 = P.c[5].x;
        const float fx = __fadd_rn(__fadd_rn(c0, __fmul_rn(c1, x)), __fmul_rn(c2, y));
        const float fy = __fadd_rn(__fadd_rn(c3, __fmul_rn(c4, x)), __fmul_rn(c5, y));
        X = __fsub_rn(x, fx);
        Y = __fsub_rn(y, fy);
        break;
    }
    case SL_FIELD_ROTATION:
        X = __fadd_rn(x, __fmul_rn(c0, __fsub_rn(y, c2)));
        Y = __fsub_rn(y, __fmul_rn(c0, __fsub_rn(x, c1)));
        break;
    case SL_FIELD_SWIRL: {
        const float2 g = a.g1f[i];
        X = __fsub_rn(x, __fmul_rn(c0, g.x));
        Y = __fsub_rn(y, __fmul_rn(c0, g.y));
        break;
    }
    case SL_FIELD_PAPER:
    case SL_FIELD_FOURIER8: {
        const float2 g = a.g1f[i], q = a.g2f[i];
        X = __fsub_rn(x, __fadd_rn(__fmul_rn(c0, g.x), __fmul_rn(c1, q.x)));
        Y = __fsub_rn(y, __fadd_rn(__fmul_rn(c0, g.y), __fmul_rn(c1, q.y)));
        break;
    }
    default:
        X = x;
        Y = y;
        break;
    }
}

// Stage-A bound of an FP32 cross product of two rounded differences of
// exact floats, with two-fold margin: 2^-22 (|t1| + |t2|).
__device__ __forceinline__ float cross_f32(float ux, float uy, float vx, float vy, float &bound)
{
    const float t2 = __fmul_rn(uy, vx);
    const float t1 = __fmul_rn(ux, vy);
    bound = 0x1p-22f * (fabsf(t1) + fabsf(t2));
    return __fsub_rn(t1, t2);
}

// Triangle of a half-edge code h = 3 t + k (h >= 0).
__device__ __forceinline__ int32_t tri_of_f32(int32_t h) { return (int32_t)__umulhi((uint32_t)h, 0xAAAAAAABu) >> 1; }

// Walk state as in the double-float kernel: the current triangle's vertices
// (W0, W1, W2), counter-clockwise, as float coordinates, and the half-edge
// codes e0, e1, e2 of its edges opposite W0, W1, W2 (code 3 j + s: edge s of
// triangle j).  A hop loads one 16-byte half-edge record (k_build_he).  After
// a hop the edge the walk came through (opposite W2) is not tested: its
// orientation was certified negative from the other side, so here it is
// positive.  The value is evaluated with the located triangle's vertices in
// slot order, so it does not depend on the path of the walk.
// kExt: the variant with the options of the paper's experiments (exclusion,
// strategies (a), (c) and the direct structured-grid start); the default
// variant compiles them out.
template <bool kStats, bool kDebug, int kBlock, int kMinBlocks, bool kExt>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_step_fast_f32(FastArgs a)
{
    const int64_t i = kExt ? node_of_thread(a) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = kExt ? i >= 0 : i < a.N;
    uint32_t hops = 0, exact_tests = 0, clipped_cnt = 0, fallback_cnt = 0, limit_cnt = 0, fp64_tests = 0;
    uint32_t excluded_cnt = 0;
    // the node's problem: the chunk table, or a search per node in a spanning-tree
    // level (a level mixes problems)
    const int pi = !active || a.nprob == 1 ? 0
                   : (kExt && a.order ? problem_of(a.node_off, a.nprob, i) : chunk_problem(a.chunk_prob, a.node_off, i));
    pdl_launch_dependents();
    pdl_wait();
    if (active) {
        const FastProb &P = a.probs[pi];
        const float2 xf = a.xyf[i];
        float X, Y;
        foot_f32(P, a, i, xf.x, xf.y, X, Y);
        uint32_t flags = 0;
        bool excluded = false;
        if (kExt && a.exclude && !(X >= 0.0f && X <= 1.0f && Y >= 0.0f && Y <= 1.0f)) {
            // the paper's experiments exclude nodes whose foot leaves the
            // domain (Sec. 4): V unchanged, no walk, T^0 unchanged
            ((float *)a.vout)[i] = ((const float *)a.vin)[i];
            excluded_cnt = 1;
            excluded = true;
            if (a.parent) {
                // strategy (c): the children start where this node would have
                a.t0[i] = a.t0[a.parent[i]];
                a.t0v[i] = a.t0v[a.parent[i]];
            }
            if (kDebug) {
                if (a.dbg.feet) {
                    a.dbg.feet[2 * i] = (double)X;
                    a.dbg.feet[2 * i + 1] = (double)Y;
                }
                if (a.dbg.feet_lo) {
                    a.dbg.feet_lo[2 * i] = 0.0;
                    a.dbg.feet_lo[2 * i + 1] = 0.0;
                }
                if (a.dbg.tri) a.dbg.tri[i] = -1;
                if (a.dbg.moves) a.dbg.moves[i] = 0;
                if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)SL_NODE_EXCLUDED;
            }
        } else if (!(X >= 0.0f && X <= 1.0f && Y >= 0.0f && Y <= 1.0f)) {
            // boundary clip in double, rounded back to float
            double cx, cy;
            clip_to_square((double)xf.x, (double)xf.y, (double)X, (double)Y, cx, cy);
            X = __double2float_rn(cx);
            Y = __double2float_rn(cy);
            flags |= SL_NODE_CLIPPED;
            clipped_cnt = 1;
        }
        if (!excluded) {
            const uint32_t fside = (X == 0.0f ? 1u : 0u) | (X == 1.0f ? 2u : 0u) | (Y == 0.0f ? 4u : 0u) |
                                   (Y == 1.0f ? 8u : 0u);

            // start state from the per-node cache (T^0 and its vertex ids)
            const int4 tq = kExt && a.grid_M > 0 ? __ldg(&a.grid_t0v[grid_slot(X, Y, a.grid_M)])
                                                 : a.t0v[kExt && a.parent ? (int64_t)a.parent[i] : i];
            int32_t e0 = tq.x, e1, e2;
            {
                const int32_t j0 = tri_of_f32(e0), s0 = e0 - 3 * j0;
                e1 = 3 * j0 + (s0 == 2 ? 0 : s0 + 1);
                e2 = 3 * j0 + (s0 == 0 ? 2 : s0 - 1);
            }
            // the vertices relative to the foot, a_k = W_k - X, rounded once
            float a0x, a0y, a1x, a1y, a2x, a2y;
            {
                const float2 A = a.xyf[tq.y], B = a.xyf[tq.z], C = a.xyf[tq.w];
                a0x = __fsub_rn(A.x, X);
                a0y = __fsub_rn(A.y, Y);
                a1x = __fsub_rn(B.x, X);
                a1y = __fsub_rn(B.y, Y);
                a2x = __fsub_rn(C.x, X);
                a2y = __fsub_rn(C.y, Y);
            }
            bool moved = false;
            const uint32_t cap = (uint32_t)a.walk_cap;
            bool found = false;
            int s1 = 0, s2 = 0, s3 = 0;
            float o1 = 0.0f, o2 = 0.0f, o3 = 0.0f;
            for (;;) {
                float eb1, eb2;
                o1 = cross_f32(a1x, a1y, a2x, a2y, eb1);    // orient(W1, W2, X): theta of W0 * den
                o2 = cross_f32(a2x, a2y, a0x, a0y, eb2);    // orient(W2, W0, X): theta of W1 * den
                s1 = o1 > eb1 ? 1 : (o1 < -eb1 ? -1 : 2);
                s2 = o2 > eb2 ? 1 : (o2 < -eb2 ? -1 : 2);
                s3 = 1;
                if (!moved) {
                    float eb3;
                    o3 = cross_f32(a0x, a0y, a1x, a1y, eb3);    // orient(W0, W1, X): theta of W2 * den
                    s3 = o3 > eb3 ? 1 : (o3 < -eb3 ? -1 : 2);
                }
                if (s1 == 2 || s2 == 2 || s3 == 2) {
                    // boundary edge with the foot on its side: exactly 0 (the
                    // record of a boundary half-edge holds its side code last)
                    if (s1 == 2) {
                        const int nb = __float_as_int(__ldg(&a.he[e0]).w);
                        if (nb < 0 && (fside >> (-1 - nb) & 1u)) s1 = 0;
                    }
                    if (s2 == 2) {
                        const int nb = __float_as_int(__ldg(&a.he[e1]).w);
                        if (nb < 0 && (fside >> (-1 - nb) & 1u)) s2 = 0;
                    }
                    if (s3 == 2) {
                        const int nb = __float_as_int(__ldg(&a.he[e2]).w);
                        if (nb < 0 && (fside >> (-1 - nb) & 1u)) s3 = 0;
                    }
                }
                if (s1 == 2 || s2 == 2 || s3 == 2) {
                    // the foot on a vertex (e.g. a node whose field vanishes): the
                    // two edges through that vertex have orientation exactly 0
                    // (a difference of two floats is zero only when they are equal)
                    const bool onA = a0x == 0.0f && a0y == 0.0f, onB = a1x == 0.0f && a1y == 0.0f;
                    const bool onC = a2x == 0.0f && a2y == 0.0f;
                    if (s1 == 2 && (onB || onC)) s1 = 0;
                    if (s2 == 2 && (onC || onA)) s2 = 0;
                    if (s3 == 2 && (onA || onB)) s3 = 0;
                }
                if (s1 == 2 || s2 == 2 || s3 == 2) {
                    // double predicate on the float coordinates promoted exactly:
                    // the vertices reloaded by slot (W0 is slot e0 - 3 j, W1 slot
                    // e1 - 3 j) in this rare branch; the barrier keeps the
                    // conversions of the loop-invariant foot inside it
                    const int32_t jj = tri_of_f32(e0), sa = e0 - 3 * jj, sb = e1 - 3 * jj, sc = 3 - sa - sb;
                    const float2 A = a.xyf[a.tv[sa][jj]], B = a.xyf[a.tv[sb][jj]], C = a.xyf[a.tv[sc][jj]];
                    float xb = X, yb = Y;
                    asm volatile("" : "+f"(xb), "+f"(yb));
                    const double Xd = xb, Yd = yb;
                    if (s1 == 2) {
                        slp::OrientResult r = slp::orient(B.x, B.y, C.x, C.y, Xd, Yd);
                        s1 = r.sign;
                        fp64_tests += r.stage == 1;
                        exact_tests += r.stage == 2;
                    }
                    if (s2 == 2) {
                        slp::OrientResult r = slp::orient(C.x, C.y, A.x, A.y, Xd, Yd);
                        s2 = r.sign;
                        fp64_tests += r.stage == 1;
                        exact_tests += r.stage == 2;
                    }
                    if (s3 == 2) {
                        slp::OrientResult r = slp::orient(A.x, A.y, B.x, B.y, Xd, Yd);
                        s3 = r.sign;
                        fp64_tests += r.stage == 1;
                        exact_tests += r.stage == 2;
                    }
                    flags |= SL_NODE_EXACT;
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
                    if (s1 < 0) { k = 0; best = o1; }
                    if (s2 < 0 && (k < 0 || o2 < best)) { k = 1; best = o2; }
                    if (s3 < 0 && (k < 0 || o3 < best)) { k = 2; best = o3; }
                } else {
                    if (hops == cap) {
                        fallback_cnt = 1;
                        flags |= SL_NODE_FALLBACK;
                    }
                    const int neg[3] = {s1 < 0, s2 < 0, s3 < 0};
                    const int nneg = neg[0] + neg[1] + neg[2];
                    int pick = (int)(mix64_dev(((uint64_t)i << 20) ^ (uint64_t)hops) % (uint64_t)nneg);
                    k = -1;
                    for (int q = 0; q < 3; ++q)
                        if (neg[q] && pick-- == 0) k = q;
                }
                const float4 R = __ldg(&a.he[k == 0 ? e0 : (k == 1 ? e1 : e2)]);
                if (isnan(R.x)) break;    // a boundary edge: not for a foot inside a valid mesh
                // the next triangle: (W2, W1, Q), (W0, W2, Q) or (W1, W0, Q)
                if (k == 0) {
                    a0x = a2x;
                    a0y = a2y;
                } else if (k == 1) {
                    a1x = a2x;
                    a1y = a2y;
                } else {
                    const float tx = a0x, ty = a0y;
                    a0x = a1x;
                    a0y = a1y;
                    a1x = tx;
                    a1y = ty;
                }
                a2x = __fsub_rn(R.x, X);
                a2y = __fsub_rn(R.y, Y);
                e0 = __float_as_int(R.z);
                e1 = __float_as_int(R.w);
                moved = true;
                ++hops;
                // lean hops: the two exits of the entered triangle, taken while
                // one is certainly negative (the same stage-A bound, on the
                // vertices relative to the foot); the full test above decides
                // where no edge is certainly negative
                while (hops < cap) {
                    float eb1, eb2;
                    const float q1 = cross_f32(a1x, a1y, a2x, a2y, eb1);
                    const float q2 = cross_f32(a2x, a2y, a0x, a0y, eb2);
                    const bool c1 = q1 < -eb1, c2 = q2 < -eb2 && !(c1 && q1 <= q2);
                    if (!(c1 || c2)) break;
                    const float4 Q = __ldg(&a.he[c2 ? e1 : e0]);
                    if (isnan(Q.x)) break;    // a boundary edge: not for a foot inside a valid mesh
                    if (c2) {
                        a1x = a2x;
                        a1y = a2y;
                    } else {
                        a0x = a2x;
                        a0y = a2y;
                    }
                    a2x = __fsub_rn(Q.x, X);
                    a2y = __fsub_rn(Q.y, Y);
                    e0 = __float_as_int(Q.z);
                    e1 = __float_as_int(Q.w);
                    ++hops;
                }
            }
            if (!found) {
                flags |= SL_NODE_WALK_LIMIT;
                limit_cnt = 1;
            }
            if (s1 == 0 || s2 == 0 || s3 == 0) flags |= SL_NODE_DEGENERATE;

            // the located triangle in slot order: its vertex ids and the
            // numerators of Eq. 6, orient(V1, V2, X), orient(V2, V0, X) and
            // orient(V0, V1, X), on the vertices relative to the foot (their
            // sum is twice the triangle's area)
            int w0 = tq.y, w1 = tq.z, w2 = tq.w;
            const int32_t j = tri_of_f32(e0);
            if (moved) {
                w0 = a.tv[0][j];
                w1 = a.tv[1][j];
                w2 = a.tv[2][j];
                // (W0, W1, W2) = slots (s, s+1, s+2)
                const int32_t s = e0 - 3 * j;
                const float v0x = s == 0 ? a0x : (s == 1 ? a2x : a1x), v0y = s == 0 ? a0y : (s == 1 ? a2y : a1y);
                const float v1x = s == 0 ? a1x : (s == 1 ? a0x : a2x), v1y = s == 0 ? a1y : (s == 1 ? a0y : a2y);
                const float v2x = s == 0 ? a2x : (s == 1 ? a1x : a0x), v2y = s == 0 ? a2y : (s == 1 ? a1y : a0y);
                float eb;
                o1 = cross_f32(v1x, v1y, v2x, v2y, eb);
                o2 = cross_f32(v2x, v2y, v0x, v0y, eb);
                o3 = cross_f32(v0x, v0y, v1x, v1y, eb);
            }
            const float dn = __fadd_rn(__fadd_rn(o1, o2), o3);
            // theta of W0, W1 (Eq. 6) and the P1 value (Remark 1) in float
            const float r = __frcp_rn(dn);
            const float th1 = __fmul_rn(o1, r), th2 = __fmul_rn(o2, r);
            const float *vin = (const float *)a.vin;
            const float v1 = vin[w0], v2 = vin[w1], v3 = vin[w2];
            const float v = __fmaf_rn(th1, __fsub_rn(v1, v3), __fmaf_rn(th2, __fsub_rn(v2, v3), v3));
            ((float *)a.vout)[i] = v;
            if ((moved || (kExt && a.parent)) && !(kExt && a.keep_t0)) {
                a.t0[i] = j;
                a.t0v[i] = make_int4(3 * j, w0, w1, w2);
            }
            if (limit_cnt) atomicOr(a.status, 1u << SL_E_WALK_LIMIT);
            if (kDebug) {
                if (a.dbg.feet) {
                    a.dbg.feet[2 * i] = (double)X;
                    a.dbg.feet[2 * i + 1] = (double)Y;
                }
                if (a.dbg.feet_lo) {
                    a.dbg.feet_lo[2 * i] = 0.0;
                    a.dbg.feet_lo[2 * i + 1] = 0.0;
                }
                if (a.dbg.tri) a.dbg.tri[i] = j;
                if (a.dbg.moves) a.dbg.moves[i] = (int32_t)hops;
                if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)flags;
            }
        }
    }
    if (kStats)
        warp_stats(a.stats, active, hops, exact_tests, clipped_cnt, fallback_cnt, limit_cnt, fp64_tests, excluded_cnt);
}

template <int kBlock, int kMinBlocks, bool kExt = false>
static void launch_f32_cfg(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    const unsigned grid = (unsigned)((a.count + kBlock - 1) / kBlock);
    if (grid == 0) return;
    if (stats) {
        if (debug) launch_step_kernel(k_step_fast_f32<true, true, kBlock, kMinBlocks, kExt>, grid, kBlock, s, a);
        else launch_step_kernel(k_step_fast_f32<true, false, kBlock, kMinBlocks, kExt>, grid, kBlock, s, a);
    } else {
        if (debug) launch_step_kernel(k_step_fast_f32<false, true, kBlock, kMinBlocks, kExt>, grid, kBlock, s, a);
        else launch_step_kernel(k_step_fast_f32<false, false, kBlock, kMinBlocks, kExt>, grid, kBlock, s, a);
    }
}

void launch_fast_f32(const FastArgs &a, bool stats, bool debug, int config, cudaStream_t s)
{
    if (a.exclude || a.order || a.grid_M > 0 || a.keep_t0) {
        // the experiment options: one configuration (128 x 8)
        launch_f32_cfg<128, 8, true>(a, stats, debug, s);
        return;
    }
    switch (config) {
    case 1: launch_f32_cfg<256, 3>(a, stats, debug, s); break;
    case 2: launch_f32_cfg<128, 8>(a, stats, debug, s); break;
    case 3: launch_f32_cfg<128, 9>(a, stats, debug, s); break;
    case 4: launch_f32_cfg<256, 5>(a, stats, debug, s); break;
    case 5: launch_f32_cfg<128, 12>(a, stats, debug, s); break;
    default: launch_f32_cfg<256, 4>(a, stats, debug, s); break;
    }
}

}  // namespace sl
