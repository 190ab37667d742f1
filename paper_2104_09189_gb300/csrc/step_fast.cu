// step_fast.cu -- the fast FP64-accuracy step kernel for GB300: launchers of
// the split step, the gather probe, value conversions, field tables and
// the walk records (the step kernels themselves are in step_fast_impl.cuh).
#include "step_fast_impl.cuh"

namespace sl {

template <bool kCompact>
static void launch_finish(const FastArgs &a, bool stats, bool debug, unsigned grid, cudaStream_t s)
{
    if (stats) {
        if (debug) launch_step_kernel(k_finish_df<true, true, kCompact>, grid, 128, s, a);
        else launch_step_kernel(k_finish_df<true, false, kCompact>, grid, 128, s, a);
    } else {
        if (debug) launch_step_kernel(k_finish_df<false, true, kCompact>, grid, 128, s, a);
        else launch_step_kernel(k_finish_df<false, false, kCompact>, grid, 128, s, a);
    }
}

template <int kBlock, int kMinBlocks>
static void launch_settle_cfg(const FastArgs &a, bool stats, bool debug, bool reset, cudaStream_t s)
{
    const unsigned grid = (unsigned)((a.N + kBlock - 1) / kBlock);
    if (grid == 0) return;
    if (reset) cudaMemsetAsync(a.queue_count, 0, sizeof(uint32_t), s);
    if (stats) {
        if (debug) launch_step_kernel(k_settle_df<true, true, kBlock, kMinBlocks, -1>, grid, kBlock, s, a);
        else launch_step_kernel(k_settle_df<true, false, kBlock, kMinBlocks, -1>, grid, kBlock, s, a);
    } else if (debug) {
        launch_step_kernel(k_settle_df<false, true, kBlock, kMinBlocks, -1>, grid, kBlock, s, a);
    } else if (!a.single) {
        launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, -1>, grid, kBlock, s, a);
    } else {
        // the timed path of a single mesh: the field kind compiled in
        switch (a.prob0.kind) {
        case SL_FIELD_AFFINE:
            launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, SL_FIELD_AFFINE>, grid, kBlock, s, a);
            break;
        case SL_FIELD_ROTATION:
            launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, SL_FIELD_ROTATION>, grid, kBlock, s, a);
            break;
        case SL_FIELD_SWIRL:
            launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, SL_FIELD_SWIRL>, grid, kBlock, s, a);
            break;
        case SL_FIELD_PAPER:
            launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, SL_FIELD_PAPER>, grid, kBlock, s, a);
            break;
        case SL_FIELD_FOURIER8:
            launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, SL_FIELD_FOURIER8>, grid, kBlock, s, a);
            break;
        default: launch_step_kernel(k_settle_df<false, false, kBlock, kMinBlocks, SL_FIELD_ZERO>, grid, kBlock, s, a); break;
        }
    }
}

// The settle pass needs 32 registers, so it runs at 128 x 14 (56 resident
// warps per SM): faster than at 48 or 64.  The caller provides a.queue (N
// entries) and a.queue_count (zeroed here when reset, else by the previous
// step's settle pass through its queue_next).
void launch_settle_df(const FastArgs &a, bool stats, bool debug, bool reset, cudaStream_t s)
{
    launch_settle_cfg<128, 14>(a, stats, debug, reset, s);
}

// The finish pass: a persistent grid of 8 blocks of 128 per SM over the queue.
void launch_finish_df(const FastArgs &a, bool stats, bool debug, int sms, cudaStream_t s)
{
    const unsigned g2 = (unsigned)(sms > 0 ? sms : 152) * 8u;
    if (a.he8) launch_finish<true>(a, stats, debug, g2, s);
    else launch_finish<false>(a, stats, debug, g2, s);
}


// Launch configurations (threads per block x resident blocks per SM the
// register budget is sized for): 0 = 256 x 4 (64 registers), 1 = 256 x 3,
// 2 = 128 x 8, 3 = 128 x 9 (56 registers), 4 = 256 x 5, 5 = 128 x 12.  Each
// is instantiated in a translation unit of its own pair (step_fast_c*.cu).
void launch_fast_df(const FastArgs &a, bool stats, bool debug, int config, cudaStream_t s)
{
    if (a.exclude || a.order || a.grid_M > 0 || a.keep_t0) {
        // the experiment options: one configuration (128 x 8, 64 registers)
        launch_fast_df_ext(a, stats, debug, s);
        return;
    }
    switch (config) {
    case 1: launch_fast_df_c1(a, stats, debug, s); break;
    case 2: launch_fast_df_c2(a, stats, debug, s); break;
    case 3: launch_fast_df_c3(a, stats, debug, s); break;
    case 4: launch_fast_df_c4(a, stats, debug, s); break;
    case 5: launch_fast_df_c5(a, stats, debug, s); break;
    default: launch_fast_df_c0(a, stats, debug, s); break;
    }
}

// ---------------------------------------------------------------------------
// Gather probe: the memory accesses of a step whose feet stay in their start
// triangles, with only a sum as arithmetic (sl_probe_gather).

__global__ void __launch_bounds__(128, 14) k_gather_probe(const float4 *xyq, const int4 *t0v, const float2 *vin,
                                                          float2 *vout, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 xq = xyq[i];
    const int4 tq = t0v[i];
    const float4 A = xyq[tq.y], B = xyq[tq.z], C = xyq[tq.w];
    const float2 V1 = vin[tq.y], V2 = vin[tq.z], V3 = vin[tq.w];
    const float s = ((xq.x + xq.y) + (xq.z + xq.w)) + ((A.x + A.y) + (A.z + A.w)) + ((B.x + B.y) + (B.z + B.w)) +
                    ((C.x + C.y) + (C.z + C.w)) + __int_as_float(tq.x & 0x007fffff);
    vout[i] = make_float2((V1.x + V2.x) + (V3.x + s), (V1.y + V2.y) + V3.y);
}

void launch_gather_probe(const float4 *xyq, const int4 *t0v, const float2 *vin, float2 *vout, int64_t N,
                         cudaStream_t s)
{
    if (N > 0) k_gather_probe<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(xyq, t0v, vin, vout, N);
}

// ---------------------------------------------------------------------------
// Value format conversions (once per run, not per step)

// h = v rounded to the nearest float (ties to even) and l = v - h rounded
// to the nearest float, from the bits of v with integer operations, for
// 2^-74 <= |v| < 2^127 (both parts normal floats); false otherwise.  The
// 29 mantissa bits below the float's 23 decide the rounding of h; v - h is
// then the signed integer rem (or rem - 2^29) times 2^(e - 1075), exact, and
// converting that integer to float rounds it once, the scaling by a power of
// two being exact in the normal range.  GB300 converts double to float on its
// slow FP64 pipe, so this keeps the conversion at memory speed.
__device__ __forceinline__ bool split_double_bits(double v, float &h, float &l)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e < 1075 - 126 || e > 1023 + 126) return false;
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t top = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // the float's 23 mantissa bits
    const uint32_t rem = lo & 0x1FFFFFFFu;                       // the 29 bits below them
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (top & 1u));
    const uint32_t fb = (((uint32_t)(e - 1023 + 127) << 23) | top) + (up ? 1u : 0u);   // a carry bumps the exponent
    h = __uint_as_float(sign | fb);
    const int32_t r = up ? (int32_t)rem - 0x20000000 : (int32_t)rem;
    const float scale = __uint_as_float((uint32_t)(e - 1075 + 127) << 23);   // 2^(e - 1075)
    const float m = __fmul_rn(__int2float_rn(r), scale);
    l = sign ? -m : m;
    return true;
}

__global__ void k_to_df(const double *__restrict__ src, float2 *__restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        float h, l;
        if (!split_double_bits(v, h, l)) {
            // zero, tiny, huge or not finite: the FP64 pipe
            h = __double2float_rn(v);
            l = __double2float_rn(v - (double)h);
        }
        dst[i] = make_float2(h, l);
    }
}

// A float as a double from its bits (exact) for zero and normal floats;
// false for subnormal, infinite and NaN ones.
__device__ __forceinline__ bool widen_float_bits(float f, double &d)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t ef = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if ((u & 0x7FFFFFFFu) == 0u) {
        d = __longlong_as_double((long long)sign);
        return true;
    }
    if (ef == 0u || ef == 0xFFu) return false;
    d = __longlong_as_double((long long)(sign | ((unsigned long long)(ef - 127u + 1023u) << 52) |
                                         ((unsigned long long)(u & 0x7FFFFFu) << 29)));
    return true;
}

__global__ void k_from_df(const float2 *src, double *dst, int64_t n)
{
    // may run in place (src and dst alias, same 8-byte slots)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[i];
        double a, b;
        if (!widen_float_bits(v.x, a)) a = (double)v.x;
        if (!widen_float_bits(v.y, b)) b = (double)v.y;
        dst[i] = a + b;
    }
}

static unsigned grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)(g > 0 ? g : 1);
}

void launch_to_df(const double *src, float2 *dst, int64_t n, cudaStream_t s)
{
    if (n > 0) k_to_df<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
}

void launch_from_df(const float2 *src, double *dst, int64_t n, cudaStream_t s)
{
    if (n > 0) k_from_df<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
}

// ---------------------------------------------------------------------------
// Node tables of the fields whose space dependence is costly (trigonometric):
//   SWIRL     g1 = (sin^2(pi x) sin(2 pi y), -sin^2(pi y) sin(2 pi x))
//   PAPER     g1 = (cos a, sin a), g2 = (-sin a, cos a), a = C0 |x - c|
//             (f = cos(C1 t) g1 + sin(C1 t) g2)
//   FOURIER8  g1 = sum_m a_m cos(phi_m) h_m, g2 = -sum_m a_m sin(phi_m) h_m,
//             h_m = (l_m pi sin(k_m pi x) cos(l_m pi y), -k_m pi cos(k_m pi x) sin(l_m pi y))
//             (f = cos(2 pi t) g1 + sin(2 pi t) g2)
// evaluated once per field in double and stored as (hi, lo) floats.

__device__ __forceinline__ float4 pack_df2(double gx, double gy)
{
    const float hx = __double2float_rn(gx), hy = __double2float_rn(gy);
    return make_float4(hx, hy, __double2float_rn(gx - (double)hx), __double2float_rn(gy - (double)hy));
}

__global__ void k_field_tables(FieldTableArgs a)
{
    const double pi = 3.14159265358979323846;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int pidx = a.nprob == 1 ? 0 : problem_of(a.node_off, a.nprob, i);
        const double *q = a.params + (1 + SL_NPARAMS) * (int64_t)pidx;
        const int kind = (int)q[0];
        const double *p = q + 1;
        const double2 xy = a.xyd ? a.xyd[i] : make_double2((double)a.xyf[i].x, (double)a.xyf[i].y);
        double g1x = 0, g1y = 0, g2x = 0, g2y = 0;
        if (kind == SL_FIELD_SWIRL) {
            double sx, cx, sy, cy;
            sincospi(xy.x, &sx, &cx);
            sincospi(xy.y, &sy, &cy);
            g1x = (sx * sx) * (2.0 * sy * cy);
            g1y = -(sy * sy) * (2.0 * sx * cx);
        } else if (kind == SL_FIELD_PAPER) {
            const double dx = xy.x - p[2], dy = xy.y - p[3];
            double s, c;
            sincos(p[0] * sqrt(dx * dx + dy * dy), &s, &c);
            g1x = c;
            g1y = s;
            g2x = -s;
            g2y = c;
        } else if (kind == SL_FIELD_FOURIER8) {
            for (int m = 0; m < 8; ++m) {
                const double k = p[4 * m], l = p[4 * m + 1], am = p[4 * m + 2], ph = p[4 * m + 3];
                double skx, ckx, sly, cly, sph, cph;
                sincospi(k * xy.x, &skx, &ckx);
                sincospi(l * xy.y, &sly, &cly);
                sincos(ph, &sph, &cph);
                const double hx = l * pi * skx * cly, hy = -k * pi * ckx * sly;
                g1x += am * cph * hx;
                g1y += am * cph * hy;
                g2x -= am * sph * hx;
                g2y -= am * sph * hy;
            }
        }
        if (a.g1) a.g1[i] = pack_df2(g1x, g1y);
        if (a.g2) a.g2[i] = pack_df2(g2x, g2y);
        if (a.g1f) a.g1f[i] = make_float2(__double2float_rn(g1x), __double2float_rn(g1y));
        if (a.g2f) a.g2f[i] = make_float2(__double2float_rn(g2x), __double2float_rn(g2y));
    }
}

// T^0 back to its initial triangles and the start-state cache with it, one
// pass (sl_mesh_reset_t0).
__global__ void k_reset_t0(const int32_t *__restrict__ t0_init, const int32_t *__restrict__ tv0,
                           const int32_t *__restrict__ tv1, const int32_t *__restrict__ tv2, int32_t *__restrict__ t0,
                           int4 *__restrict__ t0v, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = t0_init[i];
        t0[i] = j;
        t0v[i] = make_int4(3 * j, tv0[j], tv1[j], tv2[j]);
    }
}

__global__ void k_fill_t0v(const int32_t *__restrict__ t0, const int32_t *__restrict__ tv0,
                           const int32_t *__restrict__ tv1, const int32_t *__restrict__ tv2, int4 *__restrict__ t0v,
                           int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = t0[i];
        t0v[i] = make_int4(3 * j, tv0[j], tv1[j], tv2[j]);
    }
}

struct HalfEdgeArgs {
    const int32_t *tv[3];
    const int32_t *tn[3];
    const float2 *xyc;
    int64_t nt;
    float4 *he;
};

__global__ void k_build_he(HalfEdgeArgs a)
{
    const int64_t nh = 3 * a.nt;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = (int32_t)(h / 3), k = (int32_t)(h - 3 * (int64_t)t);
        const int32_t u = a.tn[k][t];
        float4 r = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                               __int_as_float(3 * t + (k == 2 ? 0 : k + 1)), __int_as_float(u));
        if (u >= 0) {
            int kp = 0;
            if (a.tn[1][u] == t) kp = 1;
            else if (a.tn[2][u] == t) kp = 2;
            const float2 q = a.xyc[a.tv[kp][u]];
            r = make_float4(q.x, q.y, __int_as_float(3 * u + (kp == 2 ? 0 : kp + 1)),
                            __int_as_float(3 * u + (kp == 0 ? 2 : kp - 1)));
        }
        a.he[h] = r;
    }
}

void launch_build_he(const int32_t *const tv[3], const int32_t *const tn[3], const float2 *xyc, int64_t nt,
                     float4 *he, cudaStream_t s)
{
    HalfEdgeArgs a;
    for (int k = 0; k < 3; ++k) {
        a.tv[k] = tv[k];
        a.tn[k] = tn[k];
    }
    a.xyc = xyc;
    a.nt = nt;
    a.he = he;
    if (nt > 0) k_build_he<<<grid_for(3 * nt, 256), 256, 0, s>>>(a);
}

struct HalfEdge8Args {
    const int32_t *tv[3];
    const int32_t *tn[3];
    const float2 *xyh;
    int64_t nt;
    uint2 *he8;
    uint32_t *overflow;
};

__global__ void k_build_he8(HalfEdge8Args a)
{
    const int64_t nh = 3 * a.nt;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = (int32_t)(h / 3), k = (int32_t)(h - 3 * (int64_t)t);
        const int32_t u = a.tn[k][t];
        if (3 * (int64_t)t + 2 >= (1 << 27)) atomicOr(a.overflow, 1u);
        // boundary edge: zero offset, the exits of t itself
        int32_t e0 = 3 * t + (k == 2 ? 0 : k + 1);
        uint32_t bx = 1u << 17, by = 1u << 17;
        if (u >= 0) {
            int kp = 0;
            if (a.tn[1][u] == t) kp = 1;
            else if (a.tn[2][u] == t) kp = 2;
            // Q and the entered triangle's first vertex W0 = T[k'+1][u] (an
            // edge of u)
            const float2 q = a.xyh[a.tv[kp][u]], w = a.xyh[a.tv[kp == 2 ? 0 : kp + 1][u]];
            // grid values: the differences and their scaling by 2^24 are exact
            const float fx = __fmul_rn(__fsub_rn(q.x, w.x), 16777216.0f);
            const float fy = __fmul_rn(__fsub_rn(q.y, w.y), 16777216.0f);
            if (fabsf(fx) > 131070.0f || fabsf(fy) > 131070.0f || 3 * (int64_t)u + 2 >= (1 << 27)) {
                atomicOr(a.overflow, 1u);
            } else {
                bx = (uint32_t)(__float2int_rn(fx) + (1 << 17));
                by = (uint32_t)(__float2int_rn(fy) + (1 << 17));
                e0 = 3 * u + (kp == 2 ? 0 : kp + 1);
            }
        }
        const uint32_t f = (e0 % 3 == 2) ? 1u : 0u;
        const uint2 r = make_uint2(bx | ((by & 0x3FFFu) << 18), (by >> 14) | (f << 4) | ((uint32_t)e0 << 5));
        a.he8[h] = r;
    }
}

void launch_build_he8(const int32_t *const tv[3], const int32_t *const tn[3], const float2 *xyh, int64_t nt,
                      uint2 *he8, uint32_t *overflow, cudaStream_t s)
{
    HalfEdge8Args a;
    for (int k = 0; k < 3; ++k) {
        a.tv[k] = tv[k];
        a.tn[k] = tn[k];
    }
    a.xyh = xyh;
    a.nt = nt;
    a.he8 = he8;
    a.overflow = overflow;
    if (nt > 0) k_build_he8<<<grid_for(3 * nt, 256), 256, 0, s>>>(a);
}

void launch_fill_t0v(const int32_t *t0, const int32_t *tv0, const int32_t *tv1, const int32_t *tv2, int4 *t0v,
                     int64_t n, cudaStream_t s)
{
    if (n > 0) k_fill_t0v<<<grid_for(n, 256), 256, 0, s>>>(t0, tv0, tv1, tv2, t0v, n);
}

void launch_reset_t0(const int32_t *t0_init, const int32_t *tv0, const int32_t *tv1, const int32_t *tv2, int32_t *t0,
                     int4 *t0v, int64_t n, cudaStream_t s)
{
    if (n > 0) k_reset_t0<<<grid_for(n, 256), 256, 0, s>>>(t0_init, tv0, tv1, tv2, t0, t0v, n);
}

void launch_field_tables(const FieldTableArgs &a, cudaStream_t s)
{
    if (a.N > 0) k_field_tables<<<grid_for(a.N, 256), 256, 0, s>>>(a);
}

}  // namespace sl
