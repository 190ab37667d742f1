// noalloc.cu -- sl_step_noalloc: one step of the fast double-float kernel
// that performs no device allocation at all.
//
// Why: sl_step allocates its value scratch and per-step constant buffers
// the first time it needs them (cudaMalloc), which synchronises the device
// and can fail when a host framework's caching allocator already owns the
// memory.  Code that steps a mesh from inside such an application's loop,
// from a callback that must not synchronise, or under a fixed device-memory
// budget reserved up front cannot allocate per step.  This entry point gives
// those callers the same step with all of its scratch in a fixed,
// library-owned static device array.
//
// The scratch: kNoAllocMaxNodes (hi, lo) float pairs (8 MiB) for the step's
// output values and kNoAllocMaxProblems per-problem constant records
// (16 KiB), held by every GPU that loads this library until the process
// exits.  All calls on a device share it and every call overwrites what it
// uses (nothing has to start at zero), so calls that overlap on the GPU --
// two streams, or two meshes stepped concurrently -- race on it and must be
// serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "sl_internal.h"
#include "step_fast.cuh"
#include "step_common.cuh"

namespace sl {
namespace {

constexpr int64_t kNoAllocMaxNodes = SL_NOALLOC_MAX_NODES;
constexpr int32_t kNoAllocMaxProblems = SL_NOALLOC_MAX_PROBLEMS;
constexpr int kMaxDevices = 64;

// File-scope scratch.  In host code these names are only stand-ins for the
// device symbols; their device addresses come from cudaGetSymbolAddress.
static __device__ __align__(256) float2 g_noalloc_values[kNoAllocMaxNodes];
static __device__ __align__(256) FastProb g_noalloc_probs[kNoAllocMaxProblems];

struct DeviceScratch {
    bool ready = false;
    float2 *values = nullptr;
    FastProb *probs = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// Device addresses of the scratch on the current device, looked up once per
// device (the first call on a device does it).
sl_status scratch_for(int dev, DeviceScratch &out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(SL_E_STATE, "sl_step_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch &s = g_scratch[dev];
    if (!s.ready) {
        void *pv = nullptr, *pp = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&pv, g_noalloc_values);
        if (e != cudaSuccess)
            return fail(SL_E_CUDA, std::string("sl_step_noalloc: cudaGetSymbolAddress(values): ") + cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&pp, g_noalloc_probs);
        if (e != cudaSuccess)
            return fail(SL_E_CUDA, std::string("sl_step_noalloc: cudaGetSymbolAddress(constants): ") + cudaGetErrorString(e));
        s.values = (float2 *)pv;
        s.probs = (FastProb *)pp;
        s.ready = true;
    }
    out = s;
    return SL_OK;
}

// Node tables of trigonometric fields must already match these problems
// (building them would allocate).
bool tables_ready(const sl_mesh *m, const sl_problem *probs)
{
    bool need1 = false, need2 = false;
    for (int32_t p = 0; p < m->n_problems; ++p) {
        const int kind = probs[p].kind;
        need1 |= kind == SL_FIELD_SWIRL || kind == SL_FIELD_PAPER || kind == SL_FIELD_FOURIER8;
        need2 |= kind == SL_FIELD_PAPER || kind == SL_FIELD_FOURIER8;
    }
    if (!need1) return true;
    if (!m->d.g1 || (need2 && !m->d.g2)) return false;
    if (m->table_key.size() != (size_t)m->n_problems * 49) return false;
    for (int32_t p = 0; p < m->n_problems; ++p) {
        if (m->table_key[49 * (size_t)p] != (double)probs[p].kind) return false;
        for (int k = 0; k < SL_NPARAMS; ++k)
            if (m->table_key[49 * (size_t)p + 1 + k] != probs[p].p[k]) return false;
    }
    return true;
}

}  // namespace
}  // namespace sl

using namespace sl;

extern "C" sl_status sl_step_noalloc(sl_mesh *m, const sl_problem *probs, int64_t n, const double *v_in,
                                     double *v_out, void *stream)
{
    if (!m || !probs || !v_in || !v_out) return fail(SL_E_ARG, "sl_step_noalloc: NULL argument");
    if ((const void *)v_in == (const void *)v_out) return fail(SL_E_ARG, "sl_step_noalloc: v_in and v_out must not alias");
    if (n < 0) return fail(SL_E_ARG, "sl_step_noalloc: n must be >= 0");
    if (m->precision != SL_FP64) return fail(SL_E_ARG, "sl_step_noalloc: FP64 meshes only");
    if (m->opt_strategy == 3)
        return fail(SL_E_STATE, "sl_step_noalloc: strategy (c) needs one launch per tree level (use sl_step)");
    if (m->N > kNoAllocMaxNodes)
        return fail(SL_E_ARG, "sl_step_noalloc: the mesh has " + std::to_string(m->N) + " nodes; the static scratch holds at most " +
                                  std::to_string(kNoAllocMaxNodes) + " (use sl_step)");
    if (m->n_problems > kNoAllocMaxProblems)
        return fail(SL_E_ARG, "sl_step_noalloc: at most " + std::to_string(kNoAllocMaxProblems) + " problems");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SL_E_CUDA, std::string("sl_step_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != m->device) return fail(SL_E_STATE, "sl_step_noalloc: the current device is not the mesh's device");
    if (!tables_ready(m, probs))
        return fail(SL_E_STATE, "sl_step_noalloc: the node tables of these fields are not built; call sl_step or sl_run "
                                "once with the same problems first (that call allocates them)");
    DeviceScratch sc;
    sl_status st = scratch_for(dev, sc);
    if (st != SL_OK) return st;

    FastProb host[kNoAllocMaxProblems];
    for (int32_t p = 0; p < m->n_problems; ++p) {
        st = fast_constants_one(probs[p], n, p, host[p]);
        if (st != SL_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // pageable source: the copy is staged before the call returns
    e = cudaMemcpyAsync(sc.probs, host, sizeof(FastProb) * m->n_problems, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(SL_E_CUDA, std::string("sl_step_noalloc: constants copy: ") + cudaGetErrorString(e));

    // V^n (double) -> (hi, lo) pairs in the caller's output buffer; the step
    // writes V^{n+1} pairs to the static scratch; then back to double.
    launch_to_df(v_in, (float2 *)v_out, m->N, s);
    FastArgs a;
    std::memset(&a, 0, sizeof(a));
    a.xyq = (const float4 *)m->d.xyq;
    a.xyh = (const float2 *)m->d.xyh;
    a.xyd = (const double2 *)m->d.xy;
    for (int k = 0; k < 3; ++k) {
        a.tv[k] = m->d.tv[k];
        a.tn[k] = m->d.tn[k];
    }
    a.he = (const float4 *)m->d.he;
    a.t0 = m->d.t0;
    a.t0v = (int4 *)m->d.t0v;
    a.vin = v_out;
    a.vout = sc.values;
    a.g1 = (const float4 *)m->d.g1;
    a.g2 = (const float4 *)m->d.g2;
    a.probs = sc.probs;
    a.node_off = m->d.node_off;
    a.nprob = m->n_problems;
    a.walk_cap = m->opt_walk_cap > 0 ? m->opt_walk_cap : default_walk_cap(m);
    a.N = m->N;
    a.status = m->d.status;
    a.stats = m->d.stats;
    a.keep_t0 = m->opt_strategy == 1 || m->opt_strategy == 2;   // (a), direct: T^0 kept
    a.exclude = m->opt_outside == 1;
    a.grid_M = m->opt_strategy == 2 ? m->grid_M : 0;
    a.grid_t0v = (const int4 *)m->d.grid_t0v;
    a.count = m->N;
    launch_fast_df(a, m->opt_stats != 0, false, m->opt_config, s);
    launch_from_df(sc.values, v_out, m->N, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SL_E_CUDA, std::string("sl_step_noalloc: launch: ") + cudaGetErrorString(e));
    m->stepped = true;
    m->t0_initial = false;
    return SL_OK;
}
