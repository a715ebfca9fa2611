// khy_server.cu -- a serving loop for simulation jobs (continuous batching).
//
// Jobs (one grid each: 2D or 3D, any size, own target time) are submitted from
// any host thread and queued.  A server thread owns the GPU work:
//   * admission: a queued job is admitted as soon as a slot and HBM for its
//     state arrays (U and U^1 in FP64, the primitives of both in FP32) are free
//     in the server's arena (one allocation of hbm_budget bytes made at
//     creation, 24 bytes per state element; first-fit with coalescing); its
//     initial state is copied in and converted on the device, its clock set;
//   * stepping: every iteration runs a few Heun steps of every active job of
//     one dimensionality in one persistent launch per stage (the batch engine
//     of khy_batch.cu, rescheduled whenever the active set changes), so the
//     work of jobs that arrived at different times overlaps on the device;
//   * retirement: a job whose clock reached its target is copied back to the
//     host, its slot and memory are freed at once for the next job.
// Every job's result is bitwise equal to the same grid stepped alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/khydro.h"
#include "khy_internal.h"

using namespace khy;

namespace {

constexpr int kStepsPerIteration = 4;
constexpr int kServeCtasPerSlot = 16;  // schedule pieces per resident CTA slot (khy_batch.cu)

khy_status sfail(int st, const char *msg) { return (khy_status)record_error(st, msg); }

__global__ void srv_clock_kernel(const GridDesc *grids, Clock *clocks, const int *slots, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) clock_step(clocks + slots[i], grids[slots[i]].g);
}

__global__ void srv_clock_init_kernel(Clock *c, double t_end) {
    c->t = 0.0;
    c->t_end = t_end;
    c->dt = 0.0;
    c->dtdx[0] = c->dtdx[1] = c->dtdx[2] = 0.0;
    c->wmin_bits = kInfBits;
    c->steps = 0;
    c->max_steps = LLONG_MAX;
    c->active = 0;
    c->status = 0;
    c->floor_hits = 0;
}

template <int ND>
__global__ void srv_prim_to_cons_kernel(Geom g, const double *W, double *U) {
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

// First-fit allocator over [0, size) in units of doubles, 32-double aligned.
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> length
    size_t size = 0;
    void init(size_t n) {
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t n, size_t *off) {
        n = (n + 31) & ~size_t(31);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 31) & ~size_t(31);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum JobState { QUEUED = 0, ACTIVE = 1, DONE = 2, FAILED = 3 };

struct Job {
    long id = 0;
    khy_mesh_desc desc;
    Geom geom;
    std::vector<double> W;       // initial primitive state (host copy)
    std::vector<double> result;  // final conserved state
    double t_end = 0.0;
    int state = QUEUED;
    int slot = -1;
    size_t off = 0, len = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    long steps = 0;
    unsigned status = 0;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct khy_server {
    int device = 0;
    size_t budget = 0;
    int max_slots = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *arena = nullptr;  // [U | U1 (half doubles each) | W0 | W1 (half floats each)]
    size_t half = 0;          // elements per region
    Arena alloc;
    GridDesc *d_grids = nullptr;  // per slot
    Clock *d_clocks = nullptr;    // per slot
    Clock *h_clocks = nullptr;    // pinned, per slot
    std::vector<GridDesc> h_grids;
    std::vector<int> slot_job;    // slot -> job index in jobs (or -1)
    // per-dimensionality schedules (index 2 and 3)
    SegDesc *d_segs[4] = {};
    int *d_cta[4] = {};
    int *d_slots[4] = {};
    size_t cap_segs[4] = {}, cap_cta[4] = {}, cap_slots[4] = {};
    int nblocks[4] = {}, nactive[4] = {};
    int variant[4] = {1, 1, 3, 0};  // tile variants: 2D rows of 124, 3D 32x8
    bool dirty[4] = {true, true, true, true};
    double *h_stage = nullptr;  // pinned staging for W / results
    size_t h_stage_len = 0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<long> queue;
    std::map<long, Job> jobs;
    long next_id = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    unsigned long long cell_updates = 0;
    long completed = 0;
    int error = 0;
    char errmsg[256] = "";
};

namespace {

MultiArgs srv_args(const khy_server *s, int nd, int stage) {
    MultiArgs a;
    a.grids = s->d_grids;
    a.segs = s->d_segs[nd];
    a.cta_seg = s->d_cta[nd];
    a.clocks = s->d_clocks;
    a.queue = nullptr;
    a.nseg = 0;
    double *U = s->arena, *U1 = s->arena + s->half;
    float *W0 = reinterpret_cast<float *>(s->arena + 2 * s->half), *W1 = W0 + s->half;
    if (stage == 1) {
        a.Uin = U;
        a.Ubase = U;
        a.Uout = U1;
        a.Win = W0;
        a.Wout = W1;
    } else {
        a.Uin = U1;
        a.Ubase = U;
        a.Uout = U;
        a.Win = W1;
        a.Wout = W0;
    }
    return a;
}

template <class T>
cudaError_t ensure_cap(T **p, size_t *cap, size_t n) {
    if (n <= *cap && *p) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, sizeof(T) * std::max<size_t>(n, 16));
    if (e == cudaSuccess) *cap = std::max<size_t>(n, 16);
    return e;
}

// Rebuilds the segment schedule of one dimensionality over its active slots.
cudaError_t reschedule(khy_server *s, int nd) {
    int tx = 0, ty = 0;
    multi_variant_tile(nd, s->variant[nd], &tx, &ty);
    const int resident = multi_resident(false, nd, s->variant[nd]);
    std::vector<int> slots;
    std::vector<SegDesc> segs;
    std::vector<int> cta;
    for (int k = 0; k < s->max_slots; ++k) {
        const int j = s->slot_job[k];
        if (j >= 0 && s->h_grids[k].g.ndim == nd) slots.push_back(k);
    }
    s->nactive[nd] = (int)slots.size();
    std::vector<Geom> geoms;
    for (int k : slots) geoms.push_back(s->h_grids[k].g);
    // pieces of equal estimated cost, kServeCtasPerSlot per resident CTA
    // slot (the hardware balances them, as in a batch)
    if (!slots.empty()) build_segments(slots, geoms, nd, tx, ty, kServeCtasPerSlot * std::max(1, resident), segs, cta);
    else cta.assign(1, 0);
    s->nblocks[nd] = (int)cta.size() - 1;
    cudaError_t e = ensure_cap(&s->d_segs[nd], &s->cap_segs[nd], segs.size());
    if (e == cudaSuccess) e = ensure_cap(&s->d_cta[nd], &s->cap_cta[nd], cta.size());
    if (e == cudaSuccess) e = ensure_cap(&s->d_slots[nd], &s->cap_slots[nd], slots.size());
    if (e == cudaSuccess && !segs.empty())
        e = cudaMemcpyAsync(s->d_segs[nd], segs.data(), sizeof(SegDesc) * segs.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_cta[nd], cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && !slots.empty())
        e = cudaMemcpyAsync(s->d_slots[nd], slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // the host vectors die here
    s->dirty[nd] = false;
    return e;
}

cudaError_t stage_host(khy_server *s, size_t n) {
    if (n <= s->h_stage_len) return cudaSuccess;
    cudaFreeHost(s->h_stage);
    s->h_stage = nullptr;
    s->h_stage_len = 0;
    cudaError_t e = cudaMallocHost(&s->h_stage, sizeof(double) * n);
    if (e == cudaSuccess) s->h_stage_len = n;
    return e;
}

// Admits queued jobs that fit (FIFO with backfill).  Called with mu held.
cudaError_t admit(khy_server *s) {
    cudaError_t e = cudaSuccess;
    for (auto it = s->queue.begin(); it != s->queue.end() && e == cudaSuccess;) {
        Job &j = s->jobs[*it];
        int slot = -1;
        for (int k = 0; k < s->max_slots; ++k)
            if (s->slot_job[k] < 0) {
                slot = k;
                break;
            }
        if (slot < 0) break;
        size_t off = 0;
        if (!s->alloc.alloc(j.len / 2, &off)) {
            ++it;
            continue;
        }
        j.slot = slot;
        j.off = off;
        j.state = ACTIVE;
        j.t_admit = now_s(s->t0);
        s->slot_job[slot] = 1;
        GridDesc gd;
        memset(&gd, 0, sizeof(gd));
        gd.g = j.geom;
        gd.off = (long long)off;
        gd.cubic = 1;
        for (int d = 1; d < j.geom.ndim; ++d)
            if (j.geom.dx[d] != j.geom.dx[0]) gd.cubic = 0;
        s->h_grids[slot] = gd;
        // initial state: W -> U1 region (scratch), convert into U, clock, CFL minimum
        e = stage_host(s, j.W.size());
        if (e == cudaSuccess) {
            memcpy(s->h_stage, j.W.data(), sizeof(double) * j.W.size());
            e = cudaMemcpyAsync(s->arena + s->half + off, s->h_stage, sizeof(double) * j.W.size(),
                                cudaMemcpyHostToDevice, s->stream);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_grids + slot, &s->h_grids[slot], sizeof(GridDesc), cudaMemcpyHostToDevice, s->stream);
        const int blocks = (int)std::min<long long>((j.geom.ncell + 255) / 256, 152 * 4);
        if (e == cudaSuccess) {
            if (j.geom.ndim == 2) srv_prim_to_cons_kernel<2><<<blocks, 256, 0, s->stream>>>(j.geom, s->arena + s->half + off, s->arena + off);
            else srv_prim_to_cons_kernel<3><<<blocks, 256, 0, s->stream>>>(j.geom, s->arena + s->half + off, s->arena + off);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            srv_clock_init_kernel<<<1, 1, 0, s->stream>>>(s->d_clocks + slot, j.t_end);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)  // also stores the job's primitives in W0
            e = launch_dt_mixed(j.geom, s->arena + off, s->d_clocks + slot,
                                reinterpret_cast<float *>(s->arena + 2 * s->half) + off, 0, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // staging buffer reuse
        j.W.clear();
        j.W.shrink_to_fit();
        s->dirty[j.geom.ndim] = true;
        it = s->queue.erase(it);
    }
    return e;
}

cudaError_t step_active(khy_server *s) {
    cudaError_t e = cudaSuccess;
    for (int nd = 2; nd <= 3 && e == cudaSuccess; ++nd) {
        if (s->dirty[nd]) e = reschedule(s, nd);
        if (e != cudaSuccess || s->nactive[nd] == 0) continue;
        for (int k = 0; k < kStepsPerIteration && e == cudaSuccess; ++k) {
            srv_clock_kernel<<<(s->nactive[nd] + 127) / 128, 128, 0, s->stream>>>(s->d_grids, s->d_clocks, s->d_slots[nd],
                                                                                  s->nactive[nd]);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_multi_stage(false, srv_args(s, nd, 1), nd, s->variant[nd], 1, s->nblocks[nd], s->stream);
            if (e == cudaSuccess) e = launch_multi_stage(false, srv_args(s, nd, 2), nd, s->variant[nd], 2, s->nblocks[nd], s->stream);
        }
    }
    return e;
}

// Copies back and frees every job whose clock reached its target.
cudaError_t retire(khy_server *s) {
    cudaError_t e = cudaMemcpyAsync(s->h_clocks, s->d_clocks, sizeof(Clock) * s->max_slots, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &kv : s->jobs) {
        Job &j = kv.second;
        if (j.state != ACTIVE) continue;
        const Clock &c = s->h_clocks[j.slot];
        const bool failed = (c.status & (FLAG_NONPHYSICAL | FLAG_DT_UNDERFLOW)) != 0;
        if (!(c.t >= c.t_end) && !failed) continue;
        const size_t n = j.len / 2;
        j.result.resize(n);
        e = stage_host(s, n);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_stage, s->arena + j.off, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return e;
        memcpy(j.result.data(), s->h_stage, sizeof(double) * n);
        j.steps = (long)c.steps;
        j.status = c.status;
        j.t_done = now_s(s->t0);
        j.state = failed ? FAILED : DONE;
        s->cell_updates += (unsigned long long)c.steps * (unsigned long long)j.geom.ncell;
        s->completed += 1;
        s->alloc.release(j.off, j.len / 2);
        s->slot_job[j.slot] = -1;
        s->dirty[j.geom.ndim] = true;
        j.slot = -1;
    }
    s->cv.notify_all();
    return cudaSuccess;
}

void worker_main(khy_server *s) {
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        cudaError_t e;
        bool any_active = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            e = admit(s);
            for (int k = 0; k < s->max_slots; ++k)
                if (s->slot_job[k] >= 0) any_active = true;
            if (e == cudaSuccess && !any_active) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (e == cudaSuccess) e = step_active(s);
        if (e == cudaSuccess) e = retire(s);
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->error = KHY_ERR_CUDA;
            snprintf(s->errmsg, sizeof(s->errmsg), "server: %s", cudaGetErrorString(e));
            s->cv.notify_all();
            return;
        }
    }
}

}  // namespace

extern "C" {

khy_status khy_server_create(size_t hbm_budget_bytes, int max_slots, void *cuda_stream, khy_server **out) {
    if (!out) return sfail(KHY_ERR_ARG, "khy_server_create: out is NULL");
    *out = nullptr;
    if (max_slots < 1 || hbm_budget_bytes < 4096) return sfail(KHY_ERR_ARG, "khy_server_create: need max_slots >= 1 and a budget");
    khy_server *s = new (std::nothrow) khy_server();
    if (!s) return sfail(KHY_ERR_OOM, "khy_server_create: host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    // 2 doubles + 2 floats per state element
    s->half = (hbm_budget_bytes / (2 * sizeof(double) + 2 * sizeof(float))) & ~size_t(31);
    s->alloc.init(s->half);
    s->h_grids.resize(max_slots);
    s->slot_job.assign(max_slots, -1);
    cudaError_t e = cudaSuccess;
    e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) {
        if (cuda_stream) s->stream = (cudaStream_t)cuda_stream;
        else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->arena, (2 * sizeof(double) + 2 * sizeof(float)) * s->half);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_grids, sizeof(GridDesc) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_clocks, sizeof(Clock) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_clocks, sizeof(Clock) * max_slots);
    if (e == cudaSuccess) {
        for (int k = 0; k < max_slots; ++k) {
            memset(&s->h_clocks[k], 0, sizeof(Clock));
            memset(&s->h_grids[k], 0, sizeof(GridDesc));
        }
        e = cudaMemcpyAsync(s->d_clocks, s->h_clocks, sizeof(Clock) * max_slots, cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_grids, s->h_grids.data(), sizeof(GridDesc) * max_slots, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = prepare_mixed(2);
    if (e == cudaSuccess) e = prepare_mixed(3);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        khy_server_destroy(s);
        return sfail(e == cudaErrorMemoryAllocation ? KHY_ERR_OOM : KHY_ERR_CUDA, cudaGetErrorString(e));
    }
    for (int nd = 2; nd <= 3; ++nd)
        if (multi_resident(false, nd, s->variant[nd]) <= 0) {
            khy_server_destroy(s);
            return sfail(KHY_ERR_CUDA, "khy_server_create: kernel occupancy query failed");
        }
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread(worker_main, s);
    *out = s;
    return KHY_OK;
}

void khy_server_destroy(khy_server *s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->arena);
    cudaFree(s->d_grids);
    cudaFree(s->d_clocks);
    for (int nd = 0; nd < 4; ++nd) {
        cudaFree(s->d_segs[nd]);
        cudaFree(s->d_cta[nd]);
        cudaFree(s->d_slots[nd]);
    }
    cudaFreeHost(s->h_clocks);
    cudaFreeHost(s->h_stage);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

khy_status khy_server_submit(khy_server *s, const khy_mesh_desc *desc, const double *W, size_t count, double t_end,
                             long *job_id) {
    if (!s || !desc || !W || !job_id) return sfail(KHY_ERR_ARG, "khy_server_submit: NULL argument");
    int st = validate_desc(desc);
    if (st != KHY_OK) return (khy_status)st;
    if (desc->ndim < 2 || desc->prec != KHY_PREC_MIXED || desc->integrator == KHY_INT_VL2)
        return sfail(KHY_ERR_ARG, "khy_server_submit: the server runs mixed-precision 2D and 3D Heun jobs");
    if (!(t_end > 0.0) || !std::isfinite(t_end)) return sfail(KHY_ERR_ARG, "khy_server_submit: t_end must be > 0");
    Job j;
    j.desc = *desc;
    j.geom = geom_of_desc(*desc);
    const size_t n = (size_t)(2 + desc->ndim) * (size_t)j.geom.ncell;
    if (count != n) return sfail(KHY_ERR_ARG, "khy_server_submit: count must be nvar*ncell");
    j.len = 2 * n;  // U and U^1
    if (((n + 31) & ~size_t(31)) > s->half)
        return sfail(KHY_ERR_BUDGET, "khy_server_submit: the job's state arrays exceed the HBM budget");
    j.W.assign(W, W + n);
    j.t_end = t_end;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return sfail(s->error, s->errmsg);
    j.id = s->next_id++;
    j.t_submit = now_s(s->t0);
    const long id = j.id;
    s->jobs.emplace(id, std::move(j));
    s->queue.push_back(id);
    s->cv.notify_all();
    *job_id = id;
    return KHY_OK;
}

khy_status khy_server_poll(khy_server *s, long job_id, int *state, double times[3], long *steps) {
    if (!s) return sfail(KHY_ERR_ARG, "khy_server_poll: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return sfail(s->error, s->errmsg);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return sfail(KHY_ERR_ARG, "khy_server_poll: unknown job");
    const Job &j = it->second;
    if (state) *state = j.state;
    if (times) {
        times[0] = j.t_submit;
        times[1] = j.t_admit;
        times[2] = j.t_done;
    }
    if (steps) *steps = j.steps;
    return KHY_OK;
}

khy_status khy_server_wait(khy_server *s, long job_id, double timeout_s) {
    if (!s) return sfail(KHY_ERR_ARG, "khy_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        if (s->error) return sfail(s->error, s->errmsg);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return sfail(KHY_ERR_ARG, "khy_server_wait: unknown job");
        if (it->second.state == DONE) return KHY_OK;
        if (it->second.state == FAILED) return sfail(KHY_ERR_NONPHYSICAL, "khy_server_wait: the job failed (status bits set)");
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout)
            return sfail(KHY_ERR_TIMEOUT, "khy_server_wait: timed out");
    }
}

khy_status khy_server_result(khy_server *s, long job_id, double *U, size_t count, int release) {
    if (!s || !U) return sfail(KHY_ERR_ARG, "khy_server_result: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return sfail(KHY_ERR_ARG, "khy_server_result: unknown job");
    Job &j = it->second;
    if (j.state != DONE && j.state != FAILED) return sfail(KHY_ERR_ARG, "khy_server_result: job not finished");
    if (count != j.result.size()) return sfail(KHY_ERR_ARG, "khy_server_result: count must be nvar*ncell");
    memcpy(U, j.result.data(), sizeof(double) * count);
    if (release) s->jobs.erase(it);
    return KHY_OK;
}

khy_status khy_server_stats(khy_server *s, long *completed, int *active, int *queued,
                            unsigned long long *cell_updates, double *elapsed_s) {
    if (!s) return sfail(KHY_ERR_ARG, "khy_server_stats: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (active) {
        int a = 0;
        for (int k = 0; k < s->max_slots; ++k) a += s->slot_job[k] >= 0;
        *active = a;
    }
    if (queued) *queued = (int)s->queue.size();
    if (cell_updates) *cell_updates = s->cell_updates;
    if (elapsed_s) *elapsed_s = now_s(s->t0);
    return KHY_OK;
}

}  // extern "C"
