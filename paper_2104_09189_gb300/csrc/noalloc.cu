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
// exits.  The constants reach their records through kernel parameters, not
// through a copy from host memory.  All calls on a device share it and every call overwrites what it
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
    const std::vector<double> key = field_table_key(m->n_problems, probs, need1, need2);
    if (!need1) return true;
    if (!m->d.g1 || (need2 && !m->d.g2)) return false;
    return key == m->table_key;
}

// The step's per-problem constants travel to the static array in the
// parameters of a small kernel, kConstChunk problems per launch (4 KiB of
// parameters), so no host buffer has to outlive the call.
constexpr int kConstChunk = 63;
struct ConstChunk {
    int32_t base, count;
    FastProb p[kConstChunk];
};

__global__ void k_noalloc_constants(const ConstChunk c)
{
    const int t = threadIdx.x;
    if (t < c.count) g_noalloc_probs[c.base + t] = c.p[t];
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
    for (int32_t b = 0; b < m->n_problems; b += kConstChunk) {
        ConstChunk c;
        c.base = b;
        c.count = m->n_problems - b < kConstChunk ? m->n_problems - b : kConstChunk;
        std::memcpy(c.p, host + b, sizeof(FastProb) * (size_t)c.count);
        k_noalloc_constants<<<1, kConstChunk, 0, s>>>(c);
    }

    // V^n (double) -> (hi, lo) pairs in the caller's output buffer; the step
    // writes V^{n+1} pairs to the static scratch; then back to double.  The
    // fused kernel in the launch configuration sl_step would take for this
    // step (SL_OPT_KERNEL = 1 and SL_OPT_SPLIT do not apply here).
    launch_to_df(v_in, (float2 *)v_out, m->N, s);
    FastArgs a;
    fast_args_for(m, sc.probs, v_out, sc.values, nullptr, host, a);
    launch_fast_df(a, m->opt_stats != 0, false, m->t0_initial ? m->opt_config_first : m->opt_config, s);
    launch_from_df(sc.values, v_out, m->N, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SL_E_CUDA, std::string("sl_step_noalloc: launch: ") + cudaGetErrorString(e));
    m->stepped = true;
    m->t0_initial = false;
    return SL_OK;
}
