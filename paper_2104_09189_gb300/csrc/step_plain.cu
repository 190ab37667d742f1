// step_plain.cu -- the plain FP64 step: one thread per node, every operation
// in double precision, written as the paper states it.  It is the reference
// point for the optimised kernels and the "plain FP64 GPU step".
//
// Per node i (Algorithm 2, one pass of the time loop, fused):
//   1. Euler foot at t_{n+1} and boundary clip            (Eq. 4)
//   2. start triangle j = T^0_i                           (strategy (b), Sec. 3)
//   3. barycentric walk: stop when all three orientation signs of the foot
//      against the edges of T_j are >= 0, else move to the neighbour across
//      the edge opposite the most negative coordinate      (Sec. 2.2, Alg. 1)
//   4. theta by Eq. 6, theta_3 = 1 - theta_1 - theta_2, and
//      V^{n+1}_i = theta_1 v_1 + theta_2 v_2 + theta_3 v_3 (Remark 1)
//   5. T^0_i <- T^f_i                                      (Alg. 1, strategy (b))
#include "step_kernels.cuh"

namespace sl {

// Walk from triangle j0, Eq. 6 and the P1 value for node i whose clipped foot
// is (X, Y); T^0_i <- the located triangle (unless kept, kExt).
template <bool kDebug, bool kExt>
__device__ __forceinline__ void plain_walk_value(const StepArgs &a, int64_t i, int32_t j0, double X, double Y,
                                                 bool clipped, uint32_t &hops, uint32_t &exact_tests,
                                                 uint32_t &clipped_cnt, uint32_t &fallback_cnt, uint32_t &limit_cnt)
{
    const double2 *xy = (const double2 *)a.xy;
    const double *vin = (const double *)a.vin;
    uint32_t flags = clipped ? SL_NODE_CLIPPED : 0u;
    clipped_cnt = clipped;

    int32_t j = j0;
    int s1 = 0, s2 = 0, s3 = 0;
    bool found = false;
    const uint32_t cap = (uint32_t)a.walk_cap;
    double2 A, B, C;
    for (;;) {
        const int ia = a.tv[0][j], ib = a.tv[1][j], ic = a.tv[2][j];
        A = xy[ia];
        B = xy[ib];
        C = xy[ic];
        slp::OrientResult o1 = slp::orient(B.x, B.y, C.x, C.y, X, Y);
        slp::OrientResult o2 = slp::orient(C.x, C.y, A.x, A.y, X, Y);
        slp::OrientResult o3 = slp::orient(A.x, A.y, B.x, B.y, X, Y);
        s1 = o1.sign;
        s2 = o2.sign;
        s3 = o3.sign;
        exact_tests += (o1.stage == 2) + (o2.stage == 2) + (o3.stage == 2);
        if (o1.stage == 2 || o2.stage == 2 || o3.stage == 2) flags |= SL_NODE_EXACT;
        if (o1.range || o2.range || o3.range) flags |= SL_NODE_RANGE;
        if (s1 >= 0 && s2 >= 0 && s3 >= 0) {
            found = true;
            break;
        }
        if (hops >= 2 * cap) break;
        int k;
        if (hops < cap) {
            // the paper's rule: the most negative barycentric coordinate
            // (theta_k = det_k / area, one positive area for all k);
            // ties go to the lowest k
            double best = 0.0;
            k = -1;
            if (s1 < 0) { k = 0; best = o1.det; }
            if (s2 < 0 && (k < 0 || o2.det < best)) { k = 1; best = o2.det; }
            if (s3 < 0 && (k < 0 || o3.det < best)) { k = 2; best = o3.det; }
        } else {
            // fallback after `cap` hops: a randomised visibility walk
            // (a uniformly drawn negative edge) terminates on any
            // triangulation with probability one
            if (hops == cap) fallback_cnt = 1, flags |= SL_NODE_FALLBACK;
            const int neg[3] = {s1 < 0, s2 < 0, s3 < 0};
            const int nneg = neg[0] + neg[1] + neg[2];
            uint64_t h = mix64_dev(((uint64_t)i << 20) ^ (uint64_t)hops);
            int pick = (int)(h % (uint64_t)nneg);
            k = -1;
            for (int q = 0; q < 3; ++q)
                if (neg[q] && pick-- == 0) k = q;
        }
        const int32_t nj = a.tn[k][j];
        if (nj < 0) break;       // cannot happen for a foot inside a valid mesh
        j = nj;
        ++hops;
    }
    if (!found) {
        flags |= SL_NODE_WALK_LIMIT;
        limit_cnt = 1;
    }
    if (s1 == 0 || s2 == 0 || s3 == 0) flags |= SL_NODE_DEGENERATE;

    // Eq. 6 and the P1 formula of Remark 1, operation by operation
    const double xi1 = A.x, eta1 = A.y, xi2 = B.x, eta2 = B.y, xi3 = C.x, eta3 = C.y;
    const double e23 = __dsub_rn(eta2, eta3), x32 = __dsub_rn(xi3, xi2);
    const double x13 = __dsub_rn(xi1, xi3), e13 = __dsub_rn(eta1, eta3);
    const double e31 = __dsub_rn(eta3, eta1);
    const double dX = __dsub_rn(X, xi3), dY = __dsub_rn(Y, eta3);
    const double den = __dadd_rn(__dmul_rn(e23, x13), __dmul_rn(x32, e13));
    const double th1 = __ddiv_rn(__dadd_rn(__dmul_rn(e23, dX), __dmul_rn(x32, dY)), den);
    const double th2 = __ddiv_rn(__dadd_rn(__dmul_rn(e31, dX), __dmul_rn(x13, dY)), den);
    const double th3 = __dsub_rn(__dsub_rn(1.0, th1), th2);
    const int ia = a.tv[0][j], ib = a.tv[1][j], ic = a.tv[2][j];
    const double v = __dadd_rn(__dadd_rn(__dmul_rn(th1, vin[ia]), __dmul_rn(th2, vin[ib])), __dmul_rn(th3, vin[ic]));
    ((double *)a.vout)[i] = v;
    if (!(kExt && a.keep_t0)) {
        a.t0[i] = j;
        a.t0v[i] = make_int4(3 * j, ia, ib, ic);     // the start state of the fast kernels
    }
    if (limit_cnt) atomicOr(a.status, 1u << SL_E_WALK_LIMIT);
    if (flags & SL_NODE_RANGE) atomicOr(a.status, 1u << SL_E_ARG);
    if (kDebug) {
        if (a.dbg.feet) {
            a.dbg.feet[2 * i] = X;
            a.dbg.feet[2 * i + 1] = Y;
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

// kExt: the variant with the options of the paper's experiments (exclusion,
// strategies (a), (c) and the direct structured-grid start); the default
// variant is the plain step alone.
template <bool kStats, bool kDebug, bool kExt>
__global__ void __launch_bounds__(256) k_step_plain_f64(StepArgs a)
{
    const int64_t i = kExt ? node_of_thread(a) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = kExt ? i >= 0 : i < a.N;
    uint32_t hops = 0, exact_tests = 0, clipped_cnt = 0, fallback_cnt = 0, limit_cnt = 0, excluded_cnt = 0;
    if (active) {
        const int pi = a.nprob == 1 ? 0 : problem_of(a.node_off, a.nprob, i);
        const ProbStep &P = a.probs[pi];
        const double2 xi = ((const double2 *)a.xy)[i];
        double fx, fy;
        field_f64(P, xi.x, xi.y, fx, fy);
        if (!kExt) {
            double X, Y;
            const bool clipped = foot_clip_f64(xi.x, xi.y, P.dt, fx, fy, X, Y);
            plain_walk_value<kDebug, false>(a, i, a.t0[i], X, Y, clipped, hops, exact_tests, clipped_cnt,
                                            fallback_cnt, limit_cnt);
        } else {
            const double qx = __dsub_rn(xi.x, __dmul_rn(P.dt, fx)), qy = __dsub_rn(xi.y, __dmul_rn(P.dt, fy));
            if (a.exclude && !(qx >= 0.0 && qx <= 1.0 && qy >= 0.0 && qy <= 1.0)) {
                // the paper's experiments exclude nodes whose foot leaves the
                // domain (Sec. 4): V unchanged, no walk, T^0 unchanged
                ((double *)a.vout)[i] = ((const double *)a.vin)[i];
                excluded_cnt = 1;
                if (a.parent) {
                    // strategy (c): the children start where this node would have
                    a.t0[i] = a.t0[a.parent[i]];
                    a.t0v[i] = a.t0v[a.parent[i]];
                }
                if (kDebug) {
                    if (a.dbg.feet) {
                        a.dbg.feet[2 * i] = qx;
                        a.dbg.feet[2 * i + 1] = qy;
                    }
                    if (a.dbg.feet_lo) {
                        a.dbg.feet_lo[2 * i] = 0.0;
                        a.dbg.feet_lo[2 * i + 1] = 0.0;
                    }
                    if (a.dbg.tri) a.dbg.tri[i] = -1;
                    if (a.dbg.moves) a.dbg.moves[i] = 0;
                    if (a.dbg.flags) a.dbg.flags[i] = (uint8_t)SL_NODE_EXCLUDED;
                }
            } else {
                double X, Y;
                const bool clipped = clip_to_square(xi.x, xi.y, qx, qy, X, Y);
                const int32_t j0 = a.grid_M > 0 ? a.grid_t0v[grid_slot((float)X, (float)Y, a.grid_M)].x / 3
                                                : a.t0[a.parent ? (int64_t)a.parent[i] : i];
                plain_walk_value<kDebug, true>(a, i, j0, X, Y, clipped, hops, exact_tests, clipped_cnt,
                                               fallback_cnt, limit_cnt);
            }
        }
    }
    if (kStats) warp_stats(a.stats, active, hops, exact_tests, clipped_cnt, fallback_cnt, limit_cnt, 0, excluded_cnt);
}

template <bool kExt>
static void launch_plain_variant(const StepArgs &a, bool stats, bool debug, unsigned grid, int block, cudaStream_t s)
{
    if (stats) {
        if (debug) k_step_plain_f64<true, true, kExt><<<grid, block, 0, s>>>(a);
        else k_step_plain_f64<true, false, kExt><<<grid, block, 0, s>>>(a);
    } else {
        if (debug) k_step_plain_f64<false, true, kExt><<<grid, block, 0, s>>>(a);
        else k_step_plain_f64<false, false, kExt><<<grid, block, 0, s>>>(a);
    }
}

void launch_plain_f64(const StepArgs &a, bool stats, bool debug, int block, cudaStream_t s)
{
    if (block <= 0) block = 256;
    if (block > 256) block = 256;
    const unsigned grid = (unsigned)((a.count + block - 1) / block);
    if (grid == 0) return;
    if (a.exclude || a.order || a.grid_M > 0 || a.keep_t0) launch_plain_variant<true>(a, stats, debug, grid, block, s);
    else launch_plain_variant<false>(a, stats, debug, grid, block, s);
}

}  // namespace sl
