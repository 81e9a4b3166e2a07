// An MPPI solve that allocates nothing.
//
// Some callers cannot allocate device memory at solve time: code that runs where
// cudaMalloc is forbidden or unsafe (a real-time control thread that must not
// block on the allocator, an embedded or plug-in host that owns all device
// memory, or a process that has handed its memory budget to another framework).
// For them the per-solve scratch of the rollout kernel (costs, quantised
// frequencies, sampled deviations, partial sums, completion counters and the
// parameter block) lives in one file-scope device array, sized once for the
// whole process.  The kernel is the library's ordinary rollout kernel; only
// where its scratch lives differs.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "sbs_internal.h"

using namespace sbs;

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  In host code this name is only a stand-in for the device
// variable: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[SBS_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mutex;
struct Cached {
    unsigned long long ctx_id;  // unique id of the context the address belongs to
    void* addr;                 // device address of the array in that context
};
Cached g_scratch[kMaxDevices] = {};

// Unique id of the current context (the driver's cuCtxGetCurrent and cuCtxGetId,
// found once through the runtime, so the library needs no link to the driver
// library); 0 when there is none.  A device reset ends the context that held the
// array, and ids are never reused, so the next call sees a new id and looks the
// address up again instead of using a stale one.
unsigned long long current_context_id()
{
    typedef int (*CtxGetCurrent)(void**);
    typedef int (*CtxGetId)(void*, unsigned long long*);
    static void* fns[2] = {nullptr, nullptr};
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[2] = {"cuCtxGetCurrent", "cuCtxGetId"};
        for (int i = 0; i < 2; ++i) {
            void* f = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion(names[i], &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                fns[i] = f;
            cudaGetLastError();
        }
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!fns[0] || !fns[1] || ((CtxGetCurrent)fns[0])(&ctx) != 0 || !ctx) return 0;
    if (((CtxGetId)fns[1])(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on the current device (looked up once per
// device and context, with that device current).
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SBS_ERR_CUDA;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_mutex);
    Cached& c = g_scratch[dev];
    if (!c.addr || !id || c.ctx_id != id) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return SBS_ERR_CUDA;
        }
        c.addr = p;
        c.ctx_id = current_context_id();  // the lookup made the device's context current
    }
    *out = c.addr;
    return SBS_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int sbs_solve_mppi_static(const sbs_config* cfg, const sbs_problem* prob, const float* state_in,
                                     float* state_out, uint64_t iter, sbs_result* result, void* stream)
{
    int st = validate_config(cfg);
    if (st) return st;
    if (cfg->method != SBS_MPPI || cfg->P != 0 || cfg->iterations != 1) return SBS_ERR_INVALID_ARG;
    if (!prob || prob->host_memory || !prob->x0 || !prob->xref || !state_in || !state_out || !result)
        return SBS_ERR_INVALID_ARG;
    if (cfg->world_feet && !prob->feet) return SBS_ERR_INVALID_ARG;
    if ((const void*)state_in == (const void*)state_out || prob->shift < 0) return SBS_ERR_INVALID_ARG;
    st = validate_gait(&prob->gait);
    if (st) return st;

    InstParams P;
    fill_params(cfg, &P);
    const WsLayout L = ws_layout(P.K, P.H, 0, P.T, 1);
    // scratch layout: parameters | counters | MPPI comparison mean | workspace
    const size_t o_params = 0;
    const size_t o_counters = up256(sizeof(InstParams));
    const size_t o_mppi = o_counters + up256((size_t)L.counters * sizeof(unsigned));
    const size_t o_ws = o_mppi + up256((size_t)P.D * sizeof(float));
    const size_t need = o_ws + L.bytes;
    if (need > SBS_STATIC_SCRATCH_BYTES) return SBS_ERR_BUDGET;

    void* base_v = nullptr;
    st = scratch_address(&base_v);
    if (st) return st;
    char* base = (char*)base_v;
    P.state[0] = const_cast<float*>(state_in);
    P.state[1] = state_out;
    P.mppi_mean = (float*)(base + o_mppi);
    P.Bsp = nullptr;
    P.Ssp = nullptr;

    cudaStream_t s = (cudaStream_t)stream;
    // The parameter block is copied from this call's stack: a captured copy would
    // read a dead frame when replayed, so the call refuses a capturing stream.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return SBS_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return SBS_ERR_INVALID_ARG;
    // the parameter block (from host memory) and zeroed counters, ahead of the kernel
    if (cudaMemcpyAsync(base + o_params, &P, sizeof(P), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SBS_ERR_CUDA;
    unsigned* counters = (unsigned*)(base + o_counters);
    if (cudaMemsetAsync(counters, 0, (size_t)L.counters * sizeof(unsigned), s) != cudaSuccess) return SBS_ERR_CUDA;

    TickArgs t;
    std::memset(&t, 0, sizeof(t));
    t.x0 = prob->x0;
    t.xref = prob->xref;
    t.fext = prob->f_ext;
    t.feet = prob->feet;
    for (int i = 0; i < 4; ++i) t.offset[i] = prob->gait.offset[i];
    t.duty = prob->gait.duty;
    t.phase0 = prob->gait.phase0;
    t.shift = prob->shift;
    t.src = 0;
    t.iter = iter;
    t.partials = 1;
    t.mppi_to_state = 1;
    t.result = result;
    t.ws = ws_at(L, base + o_ws, counters);
    return launch_rollout((const InstParams*)(base + o_params), P, t, stream);
}
