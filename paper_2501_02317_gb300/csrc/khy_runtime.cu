// khy_runtime.cu -- host runtime behind the C ABI of include/khydro.h.
//
// A khy_sim owns U^n and U^1 (FP64, field-major; with the van Leer
// integrator the second array holds the half-step primitives W^{n+1/2} in the
// flux precision instead), for Heun the primitives of U^n and U^1 (flux
// precision; the stage kernels read them instead of recovering halo cells),
// and a device Clock.  Steps are recorded once into a CUDA graph of
// kStepsPerGraph steps and replayed;
// the time step, the clip to t_end and the stop condition live on the device
// (clock_kernel), so the host only polls the clock between graph replays.
//
// Built with -fmad=false: the primitive->conserved conversion here must match
// the CPU reference bit for bit.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/khydro.h"
#include "khy_internal.h"

using namespace khy;

namespace {

thread_local char g_err[512] = "";

khy_status fail(khy_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define KHY_CUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? KHY_ERR_OOM : KHY_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

constexpr int kStepsPerGraph = 16;

// ------------------------------------------------------------ kernels

// Start of a Heun step: dt from the accumulated CFL minimum, clipped to
// t_end (Sec. 3.1, first sub-step only); advances t and the step counter and
// arms the stage kernels; resets the minimum for the stage-2 launch.
__global__ void clock_step_kernel(Clock *c, Geom g) { clock_step(c, g); }

__global__ void clock_target_kernel(Clock *c, double t_end, long long max_steps) {
    c->t_end = t_end;
    c->max_steps = max_steps < 0 ? LLONG_MAX : c->steps + max_steps;
    c->active = 0;
}

__global__ void clock_wmin_reset_kernel(Clock *c) { c->wmin_bits = kInfBits; }

// primitive -> conserved (Eq. 2): m_d = rho v_d, E = p/(gamma-1) + (0.5 rho) |v|^2.
// W may alias U: every cell's fields are read before they are written.
template <int ND>
__global__ void prim_to_cons_kernel(Geom g, const double *W, double *U) {
    constexpr int NV = ND + 2;
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double rho = W[c];
        double v[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) v[d] = W[(long long)(1 + d) * N + c];
        const double p = W[(long long)(NV - 1) * N + c];
        double vsq = v[0] * v[0];
#pragma unroll
        for (int d = 1; d < ND; ++d) vsq = vsq + v[d] * v[d];
        U[c] = rho;
#pragma unroll
        for (int d = 0; d < ND; ++d) U[(long long)(1 + d) * N + c] = rho * v[d];
        U[(long long)(NV - 1) * N + c] = p / g.gm1 + 0.5 * rho * vsq;
    }
}

// all-FP32 path: the state lives in FP32; the API's FP64 arrays are converted
__global__ void to_float_kernel(const double *in, float *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void to_double_kernel(const float *in, double *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// Error-free transformation a + b = s + e (Knuth TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Per-block compensated partial sums of one field: out[2*block] = sum,
// out[2*block+1] = compensation.
__global__ void __launch_bounds__(256) totals_kernel(const double *X, long long N, double *out) {
    double s = 0.0, comp = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double t, e;
        two_sum(s, X[i], t, e);
        s = t;
        comp += e;
    }
    __shared__ double ss[256], sc[256];
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = comp;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            double t, e;
            two_sum(ss[threadIdx.x], ss[threadIdx.x + h], t, e);
            ss[threadIdx.x] = t;
            sc[threadIdx.x] = sc[threadIdx.x] + sc[threadIdx.x + h] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = ss[0];
        out[2 * blockIdx.x + 1] = sc[0];
    }
}

constexpr int kTotalsBlocks = 304;

}  // namespace

// ------------------------------------------------------------ the simulation

struct khy_sim {
    khy_mesh_desc desc;
    Geom geom;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *U = nullptr;   // U^n (FP32 values in the first half for KHY_PREC_FP32)
    double *U1 = nullptr;  // U^1, or W^{n+1/2} (van Leer); also scratch of >= ncell doubles
    void *W0 = nullptr;    // Heun: primitives of U^n (written by the CFL kernel and stage 2)
    void *W1 = nullptr;    // Heun: primitives of U^1 (written by stage 1)
    size_t u_bytes = 0, u1_bytes = 0, w_bytes = 0;
    Clock *clk = nullptr;
    Clock *clk_host = nullptr;  // pinned mirror for polling
    double *red = nullptr;      // totals partials [2*kTotalsBlocks]
    double *red_host = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool wmin_valid = false;
};

namespace {

int nvar_of(const khy_mesh_desc &d) { return 2 + d.ndim; }

khy_status validate(const khy_mesh_desc *d) {
    if (!d) return fail(KHY_ERR_ARG, "desc is NULL");
    if (d->ndim < 1 || d->ndim > 3) return fail(KHY_ERR_ARG, "ndim must be 1, 2 or 3 (got %d)", d->ndim);
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < d->ndim) {
            if (d->n[a] < 2) return fail(KHY_ERR_ARG, "n[%d] = %d: active axes need at least 2 cells", a, d->n[a]);
            if (!(d->hi[a] > d->lo[a]) || !std::isfinite(d->lo[a]) || !std::isfinite(d->hi[a]))
                return fail(KHY_ERR_ARG, "hi[%d] must exceed lo[%d], both finite", a, a);
            for (int s = 0; s < 2; ++s)
                if (d->bc[a][s] < KHY_BC_PERIODIC || d->bc[a][s] > KHY_BC_REFLECT)
                    return fail(KHY_ERR_ARG, "bc[%d][%d] = %d is not a khy_bc", a, s, d->bc[a][s]);
        } else if (d->n[a] != 1) {
            return fail(KHY_ERR_ARG, "n[%d] must be 1 for ndim = %d", a, d->ndim);
        }
        // checked before the product can exceed 2^31 (and long long's range)
        if (ncell > (1LL << 31) / d->n[a]) return fail(KHY_ERR_ARG, "too many cells (more than 2^31)");
        ncell *= d->n[a];
    }
    if (!(d->gamma > 1.0) || !std::isfinite(d->gamma)) return fail(KHY_ERR_ARG, "gamma must be > 1");
    if (!(d->cfl > 0.0 && d->cfl <= 1.0)) return fail(KHY_ERR_ARG, "cfl must be in (0, 1]");
    if (d->prec != KHY_PREC_FP64 && d->prec != KHY_PREC_MIXED && d->prec != KHY_PREC_FP32)
        return fail(KHY_ERR_ARG, "prec must be a khy_prec");
    if (d->integrator != KHY_INT_HEUN && d->integrator != KHY_INT_VL2 && d->integrator != KHY_INT_HEUN_LEAN)
        return fail(KHY_ERR_ARG, "integrator must be a khy_integrator");
    if (!(d->rho_floor >= 0.0) || !(d->p_floor >= 0.0)) return fail(KHY_ERR_ARG, "floors must be >= 0");
    return KHY_OK;
}

khy_status check_periodic_pairs(const khy_mesh_desc &d) {
    for (int a = 0; a < d.ndim; ++a)
        if ((d.bc[a][0] == KHY_BC_PERIODIC) != (d.bc[a][1] == KHY_BC_PERIODIC))
            return fail(KHY_ERR_ARG, "axis %d: periodic must be set on both sides or neither", a);
    return KHY_OK;
}

Geom make_geom(const khy_mesh_desc &d) {
    Geom g;
    memset(&g, 0, sizeof(g));
    g.ndim = d.ndim;
    g.ncell = 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = d.n[a];
        g.bc[a][0] = d.bc[a][0];
        g.bc[a][1] = d.bc[a][1];
        g.dx[a] = (d.hi[a] - d.lo[a]) / (double)d.n[a];
        g.ncell *= d.n[a];
    }
    g.gamma = d.gamma;
    g.gm1 = d.gamma - 1.0;
    g.g1 = (d.gamma + 1.0) / (2.0 * d.gamma);
    g.gp1 = d.gamma + 1.0;
    g.gm1_gp1 = (d.gamma - 1.0) / (d.gamma + 1.0);
    g.cfl = d.cfl;
    g.rho_floor = d.rho_floor;
    g.p_floor = d.p_floor;
    g.f_gamma = (float)g.gamma;
    g.f_gm1 = (float)g.gm1;
    g.f_g1 = (float)g.g1;
    g.f_gp1 = (float)g.gp1;
    g.f_gm1_gp1 = (float)g.gm1_gp1;
    g.f_igm1 = (float)(1.0 / g.gm1);
    g.f_rho_floor = (float)g.rho_floor;
    g.f_p_floor = (float)g.p_floor;
    for (int a = 0; a < 3; ++a) g.f_dx[a] = (float)g.dx[a];
    return g;
}

// Launches sub-step 1 or 2 of the simulation's integrator: Heun stages 5, 6
// (from the stored primitives W0 -> W1 -> W0), lean Heun stages 1, 2, or van
// Leer stages 3 (predictor: U -> W^{n+1/2} in U1) and 4 (corrector:
// W^{n+1/2}, U -> U).
cudaError_t launch_stage(const khy_sim *s, int sub) {
    StageArgs a;
    a.g = s->geom;
    a.clk = s->clk;
    a.cubic = 1;
    for (int d = 1; d < s->geom.ndim; ++d)
        if (s->geom.dx[d] != s->geom.dx[0]) a.cubic = 0;
    a.Win = nullptr;
    a.Wout = nullptr;
    int stage = sub;
    if (s->desc.integrator == KHY_INT_VL2) {
        stage = sub + 2;
        a.Uin = s->U;
        a.Ubase = s->U;
        a.Uout = s->U;
        if (sub == 1) a.Wout = s->U1;
        else a.Win = s->U1;
    } else {
        if (sub == 1) {
            a.Uin = s->U;
            a.Ubase = s->U;
            a.Uout = s->U1;
        } else {
            a.Uin = s->U1;
            a.Ubase = s->U;
            a.Uout = s->U;
        }
        if (s->desc.integrator == KHY_INT_HEUN) {
            stage = sub + 4;
            a.Win = sub == 1 ? s->W0 : s->W1;
            a.Wout = sub == 1 ? s->W1 : s->W0;
        }
    }
    if (s->desc.prec == KHY_PREC_FP32) return launch_stage_single(a, stage, s->stream);
    return s->desc.prec == KHY_PREC_FP64 ? launch_stage_fp64(a, stage, s->stream)
                                         : launch_stage_mixed(a, stage, s->stream);
}

cudaError_t prepare_prec_of(const khy_sim *s) {
    if (s->desc.prec == KHY_PREC_FP32) return prepare_single(s->desc.ndim);
    return s->desc.prec == KHY_PREC_FP64 ? prepare_fp64(s->desc.ndim) : prepare_mixed(s->desc.ndim);
}

bool single_state(const khy_sim *s) { return s->desc.prec == KHY_PREC_FP32; }

int conv_blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 8); }

// FP32 state <-> FP64 values, one field at a time through U1 (>= ncell
// doubles in every configuration).  kind: the cudaMemcpyKind of src.
cudaError_t fields_to_float(khy_sim *s, const double *src, cudaMemcpyKind kind) {
    const long long N = s->geom.ncell;
    float *Uf = reinterpret_cast<float *>(s->U);
    for (int q = 0; q < 2 + s->desc.ndim; ++q) {
        // float field q occupies bytes [4qN, 4(q+1)N) of U: for src == U those
        // belong to FP64 fields < q (already converted) or to field 0 itself
        cudaError_t e = cudaMemcpyAsync(s->U1, src + (long long)q * N, N * sizeof(double), kind, s->stream);
        if (e != cudaSuccess) return e;
        to_float_kernel<<<conv_blocks(N), 256, 0, s->stream>>>(s->U1, Uf + (long long)q * N, N);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// FP64 copy of field q of an FP32 state in U1
cudaError_t field_to_double(khy_sim *s, int q) {
    const long long N = s->geom.ncell;
    to_double_kernel<<<conv_blocks(N), 256, 0, s->stream>>>(reinterpret_cast<const float *>(s->U) + (long long)q * N,
                                                            s->U1, N);
    return cudaGetLastError();
}

cudaError_t enqueue_one_step(const khy_sim *s) {
    clock_step_kernel<<<1, 1, 0, s->stream>>>(s->clk, s->geom);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_stage(s, 1)) != cudaSuccess) return e;
    return launch_stage(s, 2);
}

khy_status ensure_graph(khy_sim *s) {
    if (s->graph) return KHY_OK;
    KHY_CUDA(prepare_prec_of(s));
    cudaGraph_t g = nullptr;
    KHY_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < kStepsPerGraph && err == cudaSuccess; ++i) err = enqueue_one_step(s);
    cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        KHY_CUDA(err);
    }
    KHY_CUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    KHY_CUDA(e3);
    return KHY_OK;
}

void drop_graph(khy_sim *s) {
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
}

khy_status ensure_wmin(khy_sim *s) {
    if (s->wmin_valid) return KHY_OK;
    clock_wmin_reset_kernel<<<1, 1, 0, s->stream>>>(s->clk);
    KHY_CUDA(cudaGetLastError());
    // also stores the primitives of U^n for the Heun stages (W0)
    const int vl = s->desc.integrator == KHY_INT_VL2;
    if (s->desc.prec == KHY_PREC_FP32) KHY_CUDA(launch_dt_single(s->geom, s->U, s->clk, s->W0, vl, s->stream));
    else KHY_CUDA(s->desc.prec == KHY_PREC_FP64 ? launch_dt_fp64(s->geom, s->U, s->clk, s->W0, vl, s->stream)
                                                : launch_dt_mixed(s->geom, s->U, s->clk, s->W0, vl, s->stream));
    s->wmin_valid = true;
    return KHY_OK;
}

khy_status read_clock(khy_sim *s) {
    KHY_CUDA(cudaMemcpyAsync(s->clk_host, s->clk, sizeof(Clock), cudaMemcpyDeviceToHost, s->stream));
    KHY_CUDA(cudaStreamSynchronize(s->stream));
    return KHY_OK;
}

khy_status status_of(const Clock &c) {
    if (c.status & FLAG_NONPHYSICAL)
        return fail(KHY_ERR_NONPHYSICAL, "non-physical state (rho <= 0, E - ke < 0 or NaN) seen by the recovery");
    if (c.status & FLAG_DT_UNDERFLOW) return fail(KHY_ERR_DT_UNDERFLOW, "CFL time step underflow or not finite");
    return KHY_OK;
}

khy_status check_count(const khy_sim *s, size_t count) {
    const size_t want = (size_t)nvar_of(s->desc) * (size_t)s->geom.ncell;
    if (count != want) return fail(KHY_ERR_ARG, "count = %zu, expected nvar*ncell = %zu", count, want);
    return KHY_OK;
}

}  // namespace

// ------------------------------------------------------------ C ABI

extern "C" {

const char *khy_last_error(void) { return g_err; }

int khy_version(void) { return 100; }

khy_status khy_create(const khy_mesh_desc *desc, void *cuda_stream, khy_sim **out) {
    if (!out) return fail(KHY_ERR_ARG, "out is NULL");
    *out = nullptr;
    khy_status st = validate(desc);
    if (st != KHY_OK) return st;
    khy_sim *s = new (std::nothrow) khy_sim();
    if (!s) return fail(KHY_ERR_OOM, "host allocation failed");
    s->desc = *desc;
    s->geom = make_geom(*desc);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            s->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = (e == cudaSuccess);
        }
    }
    const size_t bytes = sizeof(double) * (size_t)nvar_of(*desc) * (size_t)s->geom.ncell;
    s->u_bytes = bytes;
    // van Leer: the primitives W^{n+1/2} in the flux precision (FP32 in the
    // mixed and FP32 paths); >= ncell doubles, which the FP32 conversions need
    s->u1_bytes = (desc->integrator == KHY_INT_VL2 && desc->prec != KHY_PREC_FP64) ? bytes / 2 : bytes;
    if (e == cudaSuccess) e = cudaMalloc(&s->U, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->U1, s->u1_bytes);
    if (desc->integrator == KHY_INT_HEUN) {  // primitives of U^n and U^1 in the flux precision
        s->w_bytes = desc->prec == KHY_PREC_FP64 ? bytes : bytes / 2;
        if (e == cudaSuccess) e = cudaMalloc(&s->W0, s->w_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s->W1, s->w_bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->clk, sizeof(Clock));
    if (e == cudaSuccess) e = cudaMalloc(&s->red, sizeof(double) * 2 * kTotalsBlocks);
    if (e == cudaSuccess) e = cudaMallocHost(&s->clk_host, sizeof(Clock));
    if (e == cudaSuccess) e = cudaMallocHost(&s->red_host, sizeof(double) * 2 * kTotalsBlocks);
    if (e == cudaSuccess) {
        Clock c;
        memset(&c, 0, sizeof(c));
        c.wmin_bits = kInfBits;
        *s->clk_host = c;
        e = cudaMemcpyAsync(s->clk, s->clk_host, sizeof(Clock), cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->U, 0, bytes, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        khy_destroy(s);
        return fail(e == cudaErrorMemoryAllocation ? KHY_ERR_OOM : KHY_ERR_CUDA, "khy_create: %s",
                    cudaGetErrorString(e));
    }
    *out = s;
    return KHY_OK;
}

void khy_destroy(khy_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    cudaFree(s->U);
    cudaFree(s->U1);
    cudaFree(s->W0);
    cudaFree(s->W1);
    cudaFree(s->clk);
    cudaFree(s->red);
    cudaFreeHost(s->clk_host);
    cudaFreeHost(s->red_host);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

khy_status khy_set_boundary(khy_sim *s, int axis, int side, int bc) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    if (axis < 0 || axis >= s->desc.ndim) return fail(KHY_ERR_ARG, "axis %d out of range", axis);
    if (side < 0 || side > 1) return fail(KHY_ERR_ARG, "side must be 0 or 1");
    if (bc < KHY_BC_PERIODIC || bc > KHY_BC_REFLECT) return fail(KHY_ERR_ARG, "bc %d is not a khy_bc", bc);
    if (s->desc.bc[axis][side] == bc) return KHY_OK;
    s->desc.bc[axis][side] = bc;
    s->geom = make_geom(s->desc);
    drop_graph(s);  // kernel parameters changed
    return KHY_OK;
}

khy_status khy_set_conserved_dev(khy_sim *s, const double *U_dev, size_t count) {
    if (!s || !U_dev) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    if (single_state(s)) {
        KHY_CUDA(fields_to_float(s, U_dev, cudaMemcpyDeviceToDevice));
    } else {
        KHY_CUDA(cudaMemcpyAsync(s->U, U_dev, count * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    }
    s->wmin_valid = false;
    return KHY_OK;
}

khy_status khy_set_conserved(khy_sim *s, const double *U, size_t count) {
    if (!s || !U) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    if (single_state(s)) {
        KHY_CUDA(fields_to_float(s, U, cudaMemcpyHostToDevice));
    } else {
        KHY_CUDA(cudaMemcpyAsync(s->U, U, count * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    }
    KHY_CUDA(cudaStreamSynchronize(s->stream));
    s->wmin_valid = false;
    return KHY_OK;
}

// primitive values already copied into U (FP64) -> conserved, in place
static khy_status convert_prim(khy_sim *s) {
    const int blocks = (int)std::min<long long>((s->geom.ncell + 255) / 256, 152 * 8);
    switch (s->desc.ndim) {
        case 1: prim_to_cons_kernel<1><<<blocks, 256, 0, s->stream>>>(s->geom, s->U, s->U); break;
        case 2: prim_to_cons_kernel<2><<<blocks, 256, 0, s->stream>>>(s->geom, s->U, s->U); break;
        default: prim_to_cons_kernel<3><<<blocks, 256, 0, s->stream>>>(s->geom, s->U, s->U); break;
    }
    KHY_CUDA(cudaGetLastError());
    if (single_state(s)) KHY_CUDA(fields_to_float(s, s->U, cudaMemcpyDeviceToDevice));
    s->wmin_valid = false;
    return KHY_OK;
}

khy_status khy_set_primitive(khy_sim *s, const double *W, size_t count) {
    if (!s || !W) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    KHY_CUDA(cudaMemcpyAsync(s->U, W, count * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    st = convert_prim(s);
    if (st != KHY_OK) return st;
    KHY_CUDA(cudaStreamSynchronize(s->stream));
    return KHY_OK;
}

khy_status khy_set_primitive_dev(khy_sim *s, const double *W_dev, size_t count) {
    if (!s || !W_dev) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    KHY_CUDA(cudaMemcpyAsync(s->U, W_dev, count * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    return convert_prim(s);
}

khy_status khy_set_time(khy_sim *s, double t) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    if (!std::isfinite(t)) return fail(KHY_ERR_ARG, "t must be finite");
    khy_status st = read_clock(s);
    if (st != KHY_OK) return st;
    s->clk_host->t = t;
    KHY_CUDA(cudaMemcpyAsync(&s->clk->t, &s->clk_host->t, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    KHY_CUDA(cudaStreamSynchronize(s->stream));
    return KHY_OK;
}

khy_status khy_enqueue_steps(khy_sim *s, double t_end, long nsteps) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    if (nsteps < 0) return fail(KHY_ERR_ARG, "nsteps must be >= 0");
    if (std::isnan(t_end)) return fail(KHY_ERR_ARG, "t_end is NaN");
    khy_status st = check_periodic_pairs(s->desc);
    if (st != KHY_OK) return st;
    if ((st = ensure_graph(s)) != KHY_OK) return st;
    clock_target_kernel<<<1, 1, 0, s->stream>>>(s->clk, t_end, (long long)nsteps);
    KHY_CUDA(cudaGetLastError());
    if ((st = ensure_wmin(s)) != KHY_OK) return st;
    long left = nsteps;
    while (left >= kStepsPerGraph) {
        KHY_CUDA(cudaGraphLaunch(s->graph, s->stream));
        left -= kStepsPerGraph;
    }
    for (; left > 0; --left) KHY_CUDA(enqueue_one_step(s));
    return KHY_OK;
}

khy_status khy_step_to(khy_sim *s, double t_end, long max_steps, long *steps_taken, double *t_out) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    if (std::isnan(t_end)) return fail(KHY_ERR_ARG, "t_end is NaN");
    khy_status st = check_periodic_pairs(s->desc);
    if (st != KHY_OK) return st;
    if ((st = ensure_graph(s)) != KHY_OK) return st;
    if ((st = read_clock(s)) != KHY_OK) return st;
    const long long steps0 = s->clk_host->steps;
    clock_target_kernel<<<1, 1, 0, s->stream>>>(s->clk, t_end, max_steps < 0 ? -1LL : (long long)max_steps);
    KHY_CUDA(cudaGetLastError());
    if ((st = ensure_wmin(s)) != KHY_OK) return st;
    for (;;) {
        KHY_CUDA(cudaGraphLaunch(s->graph, s->stream));
        if ((st = read_clock(s)) != KHY_OK) return st;
        const Clock &c = *s->clk_host;
        if (!(c.t < c.t_end) || c.steps >= c.max_steps || (c.status & FLAG_DT_UNDERFLOW)) break;
    }
    if (steps_taken) *steps_taken = (long)(s->clk_host->steps - steps0);
    if (t_out) *t_out = s->clk_host->t;
    return status_of(*s->clk_host);
}

khy_status khy_profile_steps(khy_sim *s, double t_end, long nsteps, float ms[3]) {
    if (!s || !ms) return fail(KHY_ERR_ARG, "NULL argument");
    if (nsteps < 1) return fail(KHY_ERR_ARG, "nsteps must be >= 1");
    khy_status st = check_periodic_pairs(s->desc);
    if (st != KHY_OK) return st;
    KHY_CUDA(prepare_prec_of(s));
    clock_target_kernel<<<1, 1, 0, s->stream>>>(s->clk, t_end, (long long)nsteps);
    KHY_CUDA(cudaGetLastError());
    if ((st = ensure_wmin(s)) != KHY_OK) return st;
    std::vector<cudaEvent_t> ev(4 * (size_t)nsteps, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    for (long i = 0; i < nsteps && e == cudaSuccess; ++i) {
        cudaEvent_t *E = &ev[4 * (size_t)i];
        e = cudaEventRecord(E[0], s->stream);
        if (e == cudaSuccess) {
            clock_step_kernel<<<1, 1, 0, s->stream>>>(s->clk, s->geom);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(E[1], s->stream);
        if (e == cudaSuccess) e = launch_stage(s, 1);
        if (e == cudaSuccess) e = cudaEventRecord(E[2], s->stream);
        if (e == cudaSuccess) e = launch_stage(s, 2);
        if (e == cudaSuccess) e = cudaEventRecord(E[3], s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    double acc[3] = {0.0, 0.0, 0.0};
    for (long i = 0; i < nsteps && e == cudaSuccess; ++i) {
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[4 * (size_t)i + k], ev[4 * (size_t)i + k + 1]);
            acc[k] += t;
        }
    }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    KHY_CUDA(e);
    for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / (double)nsteps);
    return KHY_OK;
}

khy_status khy_get_conserved(khy_sim *s, double *U, size_t count) {
    if (!s || !U) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    if (single_state(s)) {
        const long long N = s->geom.ncell;
        for (int q = 0; q < nvar_of(s->desc); ++q) {
            KHY_CUDA(field_to_double(s, q));
            KHY_CUDA(cudaMemcpyAsync(U + (long long)q * N, s->U1, N * sizeof(double), cudaMemcpyDeviceToHost,
                                     s->stream));
        }
    } else {
        KHY_CUDA(cudaMemcpyAsync(U, s->U, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    }
    KHY_CUDA(cudaStreamSynchronize(s->stream));
    return KHY_OK;
}

khy_status khy_get_primitive(khy_sim *s, double *W, size_t count) {
    if (!s || !W) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    st = ensure_wmin(s);  // Heun: the primitives of U^n are (now) in W0
    if (st != KHY_OK) return st;
    void *src = s->W0;
    if (!src) {
        // lean Heun and van Leer keep no primitives between steps: recover
        // them into the step's scratch buffer (U1 holds nvar*ncell values of
        // the flux precision).  The CFL minimum this pass contributes is the
        // one already accumulated for the next step (same candidates).
        src = s->U1;
        const int vl = s->desc.integrator == KHY_INT_VL2;
        if (single_state(s)) KHY_CUDA(launch_dt_single(s->geom, s->U, s->clk, src, vl, s->stream));
        else KHY_CUDA(s->desc.prec == KHY_PREC_FP64 ? launch_dt_fp64(s->geom, s->U, s->clk, src, vl, s->stream)
                                                    : launch_dt_mixed(s->geom, s->U, s->clk, src, vl, s->stream));
    }
    if (s->desc.prec == KHY_PREC_FP64) {
        KHY_CUDA(cudaMemcpyAsync(W, src, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        KHY_CUDA(cudaStreamSynchronize(s->stream));
    } else {
        std::vector<float> tmp(count);
        KHY_CUDA(cudaMemcpyAsync(tmp.data(), src, count * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        KHY_CUDA(cudaStreamSynchronize(s->stream));
        for (size_t i = 0; i < count; ++i) W[i] = (double)tmp[i];
    }
    return KHY_OK;
}

khy_status khy_get_conserved_dev(khy_sim *s, double *U_dev, size_t count) {
    if (!s || !U_dev) return fail(KHY_ERR_ARG, "NULL argument");
    khy_status st = check_count(s, count);
    if (st != KHY_OK) return st;
    if (single_state(s)) {
        const long long N = s->geom.ncell;
        for (int q = 0; q < nvar_of(s->desc); ++q) {
            KHY_CUDA(field_to_double(s, q));
            KHY_CUDA(cudaMemcpyAsync(U_dev + (long long)q * N, s->U1, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                     s->stream));
        }
    } else {
        KHY_CUDA(cudaMemcpyAsync(U_dev, s->U, count * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    }
    return KHY_OK;
}

khy_status khy_get_time(khy_sim *s, double *t, long *steps, double *last_dt) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    khy_status st = read_clock(s);
    if (st != KHY_OK) return st;
    if (t) *t = s->clk_host->t;
    if (steps) *steps = (long)s->clk_host->steps;
    if (last_dt) *last_dt = s->clk_host->dt;
    return KHY_OK;
}

khy_status khy_totals(khy_sim *s, double out[5]) {
    if (!s || !out) return fail(KHY_ERR_ARG, "NULL argument");
    const int nv = nvar_of(s->desc);
    const long long N = s->geom.ncell;
    const int blocks = (int)std::min<long long>((N + 255) / 256, kTotalsBlocks);
    for (int q = 0; q < nv; ++q) {
        const double *src = s->U + (long long)q * N;
        if (single_state(s)) {
            KHY_CUDA(field_to_double(s, q));
            src = s->U1;
        }
        totals_kernel<<<blocks, 256, 0, s->stream>>>(src, N, s->red);
        KHY_CUDA(cudaGetLastError());
        KHY_CUDA(cudaMemcpyAsync(s->red_host, s->red, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, s->stream));
        KHY_CUDA(cudaStreamSynchronize(s->stream));
        // Neumaier over the block partials, compensations added at the end
        double sum = 0.0, comp = 0.0;
        for (int b = 0; b < blocks; ++b) {
            const double x = s->red_host[2 * b];
            const double t = sum + x;
            if (std::fabs(sum) >= std::fabs(x)) comp += (sum - t) + x;
            else comp += (x - t) + sum;
            sum = t;
            comp += s->red_host[2 * b + 1];
        }
        out[q] = sum + comp;
    }
    for (int q = nv; q < 5; ++q) out[q] = 0.0;
    return KHY_OK;
}

khy_status khy_get_flags(khy_sim *s, unsigned *flags, unsigned long long *floor_hits, int clear) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    khy_status st = read_clock(s);
    if (st != KHY_OK) return st;
    if (flags) *flags = s->clk_host->status;
    if (floor_hits) *floor_hits = s->clk_host->floor_hits;
    if (clear) {
        s->clk_host->status = 0;
        s->clk_host->floor_hits = 0;
        KHY_CUDA(cudaMemcpyAsync(&s->clk->status, &s->clk_host->status, sizeof(unsigned), cudaMemcpyHostToDevice,
                                 s->stream));
        KHY_CUDA(cudaMemcpyAsync(&s->clk->floor_hits, &s->clk_host->floor_hits, sizeof(unsigned long long),
                                 cudaMemcpyHostToDevice, s->stream));
        KHY_CUDA(cudaStreamSynchronize(s->stream));
    }
    return KHY_OK;
}

khy_status khy_device_bytes(khy_sim *s, size_t *state_bytes, size_t *total_bytes) {
    if (!s) return fail(KHY_ERR_ARG, "sim is NULL");
    const size_t st = s->u_bytes + s->u1_bytes + 2 * s->w_bytes;
    if (state_bytes) *state_bytes = st;
    if (total_bytes) *total_bytes = st + sizeof(Clock) + sizeof(double) * 2 * kTotalsBlocks;
    return KHY_OK;
}

}  // extern "C"

// ------------------------------------------------------------ helpers for khy_noalloc.cu

namespace khy {
int validate_desc(const khy_mesh_desc *d) {
    khy_status st = validate(d);
    if (st != KHY_OK) return st;
    return check_periodic_pairs(*d);
}
Geom geom_of_desc(const khy_mesh_desc &d) { return make_geom(d); }
int record_error(int status, const char *msg) { return fail((khy_status)status, "%s", msg); }
cudaError_t launch_clock_step(Clock *c, const Geom &g, cudaStream_t s) {
    clock_step_kernel<<<1, 1, 0, s>>>(c, g);
    return cudaGetLastError();
}
}  // namespace khy
