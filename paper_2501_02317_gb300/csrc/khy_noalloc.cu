// khy_noalloc.cu -- khy_step_noalloc: one Heun step on a caller-owned device
// state with no device allocation at all.
//
// Some callers cannot call cudaMalloc when they want to step: a host program
// that reserves all device memory up front for its own pool, a real-time loop
// that cannot afford the implicit device synchronisation cudaMalloc/cudaFree
// may cause, or a plug-in whose host application owns every allocation.  For
// them this entry point keeps its scratch -- the stage-1 state U1 and the step
// clock -- in one file-scope __device__ array of fixed size, which every GPU
// that loads the library holds until the process exits.  The caller passes
// the state (in and out) and a small output buffer; nothing else is needed.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is fetched once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.  The cached address is valid
// while the device's primary context lives: a cudaDeviceReset would reload
// the module and leave it stale, so callers must not reset the device while
// they use this entry point.  All calls share the array and
// it keeps the last call's contents: the clock is re-initialised at the start
// of every call, and U1 is fully rewritten by stage 1 before stage 2 reads it.
// Calls whose work overlaps on the GPU (different streams, or several host
// threads) race on the array.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/khydro.h"
#include "khy_internal.h"

using namespace khy;

namespace {

constexpr size_t kU1Bytes = (size_t)KHY_NOALLOC_SCRATCH_BYTES;
constexpr size_t kClockOffset = kU1Bytes;                    // 256-aligned
constexpr size_t kScratchTotal = kU1Bytes + 256;
static_assert(sizeof(Clock) <= 256, "clock must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchTotal];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

__global__ void noalloc_clock_init(Clock *c, double t, double t_end) {
    c->t = t;
    c->t_end = t_end;
    c->dt = 0.0;
    c->dtdx[0] = c->dtdx[1] = c->dtdx[2] = 0.0;
    c->wmin_bits = kInfBits;
    c->steps = 0;
    c->max_steps = 1;
    c->active = 0;
    c->status = 0;
    c->floor_hits = 0;
}

__global__ void noalloc_export(const Clock *c, double *out) {
    out[0] = c->t;
    out[1] = c->active ? c->dt : 0.0;
    out[2] = (double)c->status;
}

}  // namespace

extern "C" khy_status khy_step_noalloc(const khy_mesh_desc *desc, double *U_dev, double t, double t_end,
                                       double *out_dev, void *cuda_stream) {
    int st = validate_desc(desc);
    if (st != KHY_OK) return (khy_status)st;
    if (!U_dev || !out_dev) return (khy_status)record_error(KHY_ERR_ARG, "khy_step_noalloc: NULL state or output");
    if (desc->prec == KHY_PREC_FP32)
        return (khy_status)record_error(KHY_ERR_ARG, "khy_step_noalloc: FP64 or mixed precision only");
    if (desc->integrator == KHY_INT_VL2)
        return (khy_status)record_error(KHY_ERR_ARG, "khy_step_noalloc: Heun integrator only");
    if (!(t == t) || !(t_end == t_end)) return (khy_status)record_error(KHY_ERR_ARG, "khy_step_noalloc: t or t_end is NaN");
    const Geom g = geom_of_desc(*desc);
    const size_t need = sizeof(double) * (size_t)(2 + desc->ndim) * (size_t)g.ncell;
    if (need > kU1Bytes) {
        char msg[200];
        snprintf(msg, sizeof(msg), "khy_step_noalloc: the state needs %zu bytes of scratch, more than the %zu-byte "
                 "no-allocation limit", need, kU1Bytes);
        return (khy_status)record_error(KHY_ERR_ARG, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return (khy_status)record_error(KHY_ERR_CUDA, "khy_step_noalloc: no usable current device");
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {  // set-up, once per device, with that device current
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                char msg[200];
                snprintf(msg, sizeof(msg), "khy_step_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return (khy_status)record_error(KHY_ERR_CUDA, msg);
            }
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
    }
    double *U1 = reinterpret_cast<double *>(base);
    Clock *clk = reinterpret_cast<Clock *>(base + kClockOffset);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool fp64 = desc->prec == KHY_PREC_FP64;

    e = fp64 ? prepare_fp64(desc->ndim) : prepare_mixed(desc->ndim);
    if (e == cudaSuccess) {
        noalloc_clock_init<<<1, 1, 0, s>>>(clk, t, t_end);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = fp64 ? launch_dt_fp64(g, U_dev, clk, nullptr, 0, s) : launch_dt_mixed(g, U_dev, clk, nullptr, 0, s);
    if (e == cudaSuccess) e = launch_clock_step(clk, g, s);
    StageArgs a;
    a.g = g;
    a.clk = clk;
    a.Win = nullptr;  // stages 1, 2: primitives recovered on the fly
    a.Wout = nullptr;
    a.cubic = 1;
    for (int d = 1; d < g.ndim; ++d)
        if (g.dx[d] != g.dx[0]) a.cubic = 0;
    if (e == cudaSuccess) {
        a.Uin = U_dev;
        a.Ubase = U_dev;
        a.Uout = U1;
        e = fp64 ? launch_stage_fp64(a, 1, s) : launch_stage_mixed(a, 1, s);
    }
    if (e == cudaSuccess) {
        a.Uin = U1;
        a.Ubase = U_dev;
        a.Uout = U_dev;
        e = fp64 ? launch_stage_fp64(a, 2, s) : launch_stage_mixed(a, 2, s);
    }
    if (e == cudaSuccess) {
        noalloc_export<<<1, 1, 0, s>>>(clk, out_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "khy_step_noalloc: %s", cudaGetErrorString(e));
        return (khy_status)record_error(KHY_ERR_CUDA, msg);
    }
    return KHY_OK;
}
