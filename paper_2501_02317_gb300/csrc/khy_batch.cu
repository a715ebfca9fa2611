// khy_batch.cu -- many independent grids stepped together (batched and
// served workloads).
//
// All grids of a batch share one dimensionality and one precision.  Their
// conserved states share one device pool (grid i at offset off_i, a
// multiple of 32 elements so that every grid's arrays start on 128 bytes;
// each grid field-major as in the single-grid API), U^1 in a second
// pool, and the primitives of U^n and U^1 in two pools of the flux precision
// at the same offsets (the stage kernels read them instead of recovering halo
// cells, as a single grid's Heun step does); every grid has its own clock,
// so its own dt (Sec. 3.1) and its own target time.  One Heun step of the whole batch is three launches: a clock
// launch (one thread per grid), and one launch per stage that covers every
// grid through a precomputed segment schedule (tile runs of planes, cut into
// pieces of equal estimated cost, several per resident CTA slot).  K steps are recorded
// once in a CUDA graph and replayed.
//
// The tile shape is a "variant" and the schedule cuts the work into
// ctas_per_slot pieces per resident CTA slot; khy_batch_autotune times every
// (variant, ctas_per_slot) pair on the batch's own state and keeps the
// fastest, cached per shape class (dimensionality, precision, grid count and
// mean grid side, each to a power of two).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/khydro.h"
#include "khy_internal.h"

using namespace khy;

namespace {

constexpr int kBatchStepsPerGraph = 8;

__global__ void multi_clock_kernel(const GridDesc *grids, Clock *clocks, int ngrids, int *queue) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ngrids) clock_step(clocks + i, grids[i].g);
    if (queue != nullptr && i < 2) queue[i] = 0;  // segment counters of the step's two stage launches
}

__global__ void multi_target_kernel(Clock *clocks, int first, int count, double t_end, long long max_steps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        Clock *c = clocks + first + i;
        c->t_end = t_end;
        c->max_steps = max_steps < 0 ? LLONG_MAX : c->steps + max_steps;
        c->active = 0;
    }
}

__global__ void multi_wmin_reset_kernel(Clock *clocks, int ngrids) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ngrids) clocks[i].wmin_bits = kInfBits;
}

// a state between the host layout and the pool layout: blockIdx.x walks the
// grids, blockIdx.y splits each grid's range (a batch of few large grids
// still spreads over the GPU)
__global__ void multi_relayout_kernel(const GridDesc *grids, const long long *hoff, int ngrids, int nvar,
                                      const double *src, double *dst, int to_pool) {
    for (int gi = blockIdx.x; gi < ngrids; gi += gridDim.x) {
        const long long n = (long long)nvar * grids[gi].g.ncell;
        const double *s = src + (to_pool ? hoff[gi] : grids[gi].off);
        double *d = dst + (to_pool ? grids[gi].off : hoff[gi]);
        for (long long c = threadIdx.x + (long long)blockIdx.y * blockDim.x; c < n; c += (long long)blockDim.x * gridDim.y)
            d[c] = s[c];
    }
}

// launch shape of multi_relayout_kernel: about 2432 blocks in all
dim3 relayout_grid(int ngrids) {
    const int gx = std::min(ngrids, 2432);
    const int gy = std::max(1, std::min(64, 2432 / std::max(1, ngrids)));
    return dim3((unsigned)gx, (unsigned)gy, 1u);
}

// primitive (host layout: grids back to back, grid i at hoff[i]) ->
// conserved (pool layout) for every grid (Eq. 2), one block per grid at a time
template <int ND>
__global__ void multi_prim_to_cons_kernel(const GridDesc *grids, const long long *hoff, int ngrids,
                                          const double *W, double *U) {
    constexpr int NV = ND + 2;
    for (int gi = blockIdx.x; gi < ngrids; gi += gridDim.x) {
        const GridDesc &gd = grids[gi];
        const long long N = gd.g.ncell;
        const double *w = W + hoff[gi];
        double *u = U + gd.off;
        for (long long c = threadIdx.x; c < N; c += blockDim.x) {
            const double rho = w[c];
            double v[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) v[d] = w[(long long)(1 + d) * N + c];
            const double p = w[(long long)(NV - 1) * N + c];
            double vsq = v[0] * v[0];
#pragma unroll
            for (int d = 1; d < ND; ++d) vsq = vsq + v[d] * v[d];
            u[c] = rho;
#pragma unroll
            for (int d = 0; d < ND; ++d) u[(long long)(1 + d) * N + c] = rho * v[d];
            u[(long long)(NV - 1) * N + c] = p / gd.g.gm1 + 0.5 * rho * vsq;
        }
    }
}

struct Schedule {
    std::vector<SegDesc> segs;
    std::vector<int> cta_seg;  // size nblocks + 1
    int nblocks = 0;
};

// nblocks > 0: that many CTAs, each with its own contiguous share of the
// segments; nblocks = 0: the queue schedule for `resident` persistent CTAs
Schedule build_schedule(const std::vector<GridDesc> &gd, int ndim, int TX, int TY, int nblocks, int resident) {
    std::vector<int> ids(gd.size());
    std::vector<Geom> geoms(gd.size());
    for (size_t i = 0; i < gd.size(); ++i) {
        ids[i] = (int)i;
        geoms[i] = gd[i].g;
    }
    Schedule s;
    if (nblocks > 0) build_segments(ids, geoms, ndim, TX, TY, nblocks, s.segs, s.cta_seg);
    else build_segments_queue(ids, geoms, ndim, TX, TY, resident, s.segs, s.cta_seg);
    s.nblocks = (int)s.cta_seg.size() - 1;
    return s;
}

// The schedule of a batch cuts its tile runs into ctas_per_slot x (resident
// CTA slots) pieces of equal estimated cost: more pieces than slots, so the
// hardware hands pieces to slots as they free up and no CTA waits for a
// slower one (the cost model ignores the small grids' fixed overheads).
// 4096-grid 2D batch, mixed, tile rows of 124, cell-updates/s: 1 -> 1.24e10,
// 4 -> 1.32e10, 8 -> 1.38e10, 16 -> 1.44e10, 32 -> 1.45e10, 64 -> 1.33e10.
// ctas_per_slot = 0 is the queue schedule: one persistent CTA per resident
// slot, each taking the next tile run (cut only where the batch has too few
// of them) from a counter, longest first -- each run pays its warm-up
// planes once instead of once per piece.
constexpr int kDefaultCtasPerSlot = 16;
constexpr int kTunedCtasPerSlot[] = {0, 1, 4, 16, 32};

// Tuned (variant, ctas per slot) per batch shape class: dimensionality,
// precision, log2 of the grid count and log2 of the cell-weighted mean grid
// side (so batches of similar grid sizes share a tuning).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune_cache;

}  // namespace

struct khy_batch {
    int ngrids = 0, ndim = 0, prec = 0, nvar = 0;
    std::vector<khy_mesh_desc> desc;
    std::vector<GridDesc> gd;
    size_t pool = 0;   // doubles per state pool (grids at 32-element offsets)
    size_t hpool = 0;  // doubles of a host state array (grids back to back)
    std::vector<long long> hoff;      // grid offsets in a host state array
    long long *d_hoff = nullptr;
    long long cells = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *U = nullptr, *U1 = nullptr;
    void *W0 = nullptr, *W1 = nullptr;  // primitives of U and U1 (flux precision)
    GridDesc *d_grids = nullptr;
    Clock *d_clocks = nullptr;
    Clock *h_clocks = nullptr;  // pinned
    SegDesc *d_segs = nullptr;
    int *d_cta = nullptr;
    int *d_queue = nullptr;  // segment counters of the queue schedule (one per stage launch)
    int nblocks = 0;
    int nseg = 0;
    int variant = -1;
    int ctas_per_slot = kDefaultCtasPerSlot;
    cudaGraphExec_t graph = nullptr;
    bool wmin_valid = false;
};

namespace {

khy_status bfail(int st, const char *msg) { return (khy_status)record_error(st, msg); }

#define KHY_BCUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return bfail(e_ == cudaErrorMemoryAllocation ? KHY_ERR_OOM : KHY_ERR_CUDA,   \
                         cudaGetErrorString(e_));                                        \
    } while (0)

MultiArgs args_of(const khy_batch *b, int stage) {
    MultiArgs a;
    a.grids = b->d_grids;
    a.segs = b->d_segs;
    a.cta_seg = b->d_cta;
    a.clocks = b->d_clocks;
    a.queue = b->ctas_per_slot == 0 ? b->d_queue + (stage - 1) : nullptr;
    a.nseg = b->nseg;
    if (stage == 1) {
        a.Uin = b->U;
        a.Ubase = b->U;
        a.Uout = b->U1;
        a.Win = b->W0;
        a.Wout = b->W1;
    } else {
        a.Uin = b->U1;
        a.Ubase = b->U;
        a.Uout = b->U;
        a.Win = b->W1;
        a.Wout = b->W0;
    }
    return a;
}

// Class of a batch for the tuning cache.
std::tuple<int, int, int, int> shape_class(const khy_batch *b) {
    double side = 0.0;  // cell-weighted mean side
    for (const GridDesc &g : b->gd) side += (double)g.g.ncell * std::pow((double)g.g.ncell, 1.0 / b->ndim);
    side /= (double)std::max<long long>(1, b->cells);
    return std::make_tuple(b->ndim, b->prec, (int)std::floor(std::log2((double)b->ngrids)),
                           (int)std::floor(std::log2(std::max(1.0, side))));
}

khy_status apply_schedule(khy_batch *b, int v, int ctas_per_slot) {
    int tx = 0, ty = 0;
    multi_variant_tile(b->ndim, v, &tx, &ty);
    if (tx == 0) return bfail(KHY_ERR_ARG, "khy_batch: no such tile variant");
    if (ctas_per_slot < 0 || ctas_per_slot > 256) return bfail(KHY_ERR_ARG, "khy_batch: ctas_per_slot must be in [0, 256]");
    const int resident = multi_resident(b->prec == KHY_PREC_FP64, b->ndim, v);
    if (resident <= 0) return bfail(KHY_ERR_CUDA, "khy_batch: kernel occupancy query failed");
    Schedule s = build_schedule(b->gd, b->ndim, tx, ty, ctas_per_slot * resident, resident);
    cudaFree(b->d_segs);
    cudaFree(b->d_cta);
    b->d_segs = nullptr;
    b->d_cta = nullptr;
    KHY_BCUDA(cudaMalloc(&b->d_segs, sizeof(SegDesc) * std::max<size_t>(1, s.segs.size())));
    KHY_BCUDA(cudaMalloc(&b->d_cta, sizeof(int) * s.cta_seg.size()));
    KHY_BCUDA(cudaMemcpyAsync(b->d_segs, s.segs.data(), sizeof(SegDesc) * s.segs.size(), cudaMemcpyHostToDevice,
                              b->stream));
    KHY_BCUDA(cudaMemcpyAsync(b->d_cta, s.cta_seg.data(), sizeof(int) * s.cta_seg.size(), cudaMemcpyHostToDevice,
                              b->stream));
    KHY_BCUDA(cudaStreamSynchronize(b->stream));
    b->nblocks = s.nblocks;
    b->nseg = (int)s.segs.size();
    b->variant = v;
    b->ctas_per_slot = ctas_per_slot;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return KHY_OK;
}

cudaError_t enqueue_batch_step(const khy_batch *b) {
    multi_clock_kernel<<<(b->ngrids + 127) / 128, 128, 0, b->stream>>>(b->d_grids, b->d_clocks, b->ngrids, b->d_queue);
    cudaError_t e = cudaGetLastError();
    const bool fp64 = b->prec == KHY_PREC_FP64;
    if (e == cudaSuccess) e = launch_multi_stage(fp64, args_of(b, 1), b->ndim, b->variant, 1, b->nblocks, b->stream);
    if (e == cudaSuccess) e = launch_multi_stage(fp64, args_of(b, 2), b->ndim, b->variant, 2, b->nblocks, b->stream);
    return e;
}

khy_status ensure_batch_graph(khy_batch *b) {
    if (b->graph) return KHY_OK;
    cudaGraph_t g = nullptr;
    KHY_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < kBatchStepsPerGraph && err == cudaSuccess; ++i) err = enqueue_batch_step(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        KHY_BCUDA(err);
    }
    KHY_BCUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    KHY_BCUDA(e3);
    return KHY_OK;
}

khy_status ensure_batch_wmin(khy_batch *b) {
    if (b->wmin_valid) return KHY_OK;
    multi_wmin_reset_kernel<<<(b->ngrids + 127) / 128, 128, 0, b->stream>>>(b->d_clocks, b->ngrids);
    KHY_BCUDA(cudaGetLastError());
    KHY_BCUDA(launch_multi_dt(b->prec == KHY_PREC_FP64, args_of(b, 1), b->ndim, b->variant, b->nblocks, b->stream));
    b->wmin_valid = true;
    return KHY_OK;
}

khy_status read_clocks(khy_batch *b) {
    KHY_BCUDA(cudaMemcpyAsync(b->h_clocks, b->d_clocks, sizeof(Clock) * b->ngrids, cudaMemcpyDeviceToHost, b->stream));
    KHY_BCUDA(cudaStreamSynchronize(b->stream));
    return KHY_OK;
}

bool all_done(const khy_batch *b) {
    for (int i = 0; i < b->ngrids; ++i) {
        const Clock &c = b->h_clocks[i];
        if (c.t < c.t_end && c.steps < c.max_steps && !(c.status & FLAG_DT_UNDERFLOW)) return false;
    }
    return true;
}

khy_status batch_status(const khy_batch *b) {
    for (int i = 0; i < b->ngrids; ++i) {
        if (b->h_clocks[i].status & FLAG_NONPHYSICAL) return bfail(KHY_ERR_NONPHYSICAL, "khy_batch: non-physical state in a grid");
        if (b->h_clocks[i].status & FLAG_DT_UNDERFLOW) return bfail(KHY_ERR_DT_UNDERFLOW, "khy_batch: CFL step underflow in a grid");
    }
    return KHY_OK;
}

}  // namespace

namespace khy {
// Cost model per plane of a tile run: its active cells plus a fixed part for
// the barriers and index work; every run (and every piece of a split run)
// also pays a warm-up -- its first planes of stored primitives are copied and
// the march faces below its first plane computed -- about one plane of work.  Boundaries between CTAs
// are placed at multiples of total/nblocks of the cumulative cost; the total
// is re-estimated after each pass because splits add warm-up planes.
void build_segments(const std::vector<int> &ids, const std::vector<Geom> &geoms, int ndim, int TX, int TY,
                    int nblocks, std::vector<SegDesc> &segs, std::vector<int> &cta_seg) {
    struct Run { int id, x0, y0, nm; double per; };
    std::vector<Run> runs;
    const double fixed = 0.25 * TX * TY;
    const double warm = ndim >= 2 ? 1.0 : 0.0;
    double W = 0.0;
    for (size_t i = 0; i < geoms.size(); ++i) {
        const Geom &g = geoms[i];
        const int nm = ndim >= 2 ? g.n[ndim - 1] : 1;
        const int nty = ndim == 3 ? (g.n[1] + TY - 1) / TY : 1;
        const int ntx = (g.n[0] + TX - 1) / TX;
        for (int b = 0; b < nty; ++b)
            for (int a = 0; a < ntx; ++a) {
                const int w = std::min(TX, g.n[0] - a * TX);
                const int h = ndim == 3 ? std::min(TY, g.n[1] - b * TY) : 1;
                runs.push_back(Run{ids[i], a * TX, b * TY, nm, (double)w * h + fixed});
                W += runs.back().per * (nm + warm);
            }
    }
    const int min_planes = 8;
    const int G = std::max(1, std::min<int>(nblocks, (int)std::min<size_t>(runs.size() * 64, 1 << 30)));
    for (int pass = 0; pass < 3; ++pass) {
        segs.clear();
        cta_seg.assign(1, 0);
        int cta = 0;
        double C = 0.0, bound = W / G;
        auto close_cta = [&]() {
            if (cta < G - 1) {
                cta_seg.push_back((int)segs.size());
                ++cta;
                bound = (cta + 1) * W / G;
            }
        };
        for (const Run &r : runs) {
            int k = 0;
            while (k < r.nm) {
                const double full = (warm + (r.nm - k)) * r.per;
                if (C + full <= bound || cta == G - 1 || ndim == 1) {
                    segs.push_back(SegDesc{r.id, r.x0, r.y0, k, r.nm});
                    C += full;
                    k = r.nm;
                    if (C >= bound) close_cta();
                    continue;
                }
                int take = (int)std::floor((bound - C) / r.per - warm);
                if (take < min_planes) {
                    if ((int)segs.size() > cta_seg.back()) {  // this CTA has work: start the next one
                        close_cta();
                        continue;
                    }
                    take = min_planes;
                }
                if (r.nm - k - take < min_planes) take = r.nm - k;
                segs.push_back(SegDesc{r.id, r.x0, r.y0, k, k + take});
                C += (warm + take) * r.per;
                k += take;
                close_cta();
            }
        }
        if (cta_seg.back() != (int)segs.size()) cta_seg.push_back((int)segs.size());
        if (C <= W * 1.0001) break;
        W = C;  // splits added warm-up planes: re-cut with the real total
    }
    // drop empty CTAs at the end
    while (cta_seg.size() > 2 && cta_seg[cta_seg.size() - 2] == cta_seg.back()) cta_seg.pop_back();
}

// Queue schedule (persistent CTAs that take segments from a counter): every
// tile run whole, cut into near-equal pieces only where it costs more than
// 1/(4 resident) of the batch (at least 16 planes each), the list ordered
// longest first; cta_seg splits it into min(resident, segments) contiguous
// groups for the kernels that keep a static split (the CFL-minimum kernel).
void build_segments_queue(const std::vector<int> &ids, const std::vector<Geom> &geoms, int ndim, int TX, int TY,
                          int resident, std::vector<SegDesc> &segs, std::vector<int> &cta_seg) {
    struct Piece { SegDesc s; double cost; };
    const double fixed = 0.25 * TX * TY;
    const double warm = ndim >= 2 ? 1.0 : 0.0;
    std::vector<Piece> pieces;
    double W = 0.0;
    for (size_t i = 0; i < geoms.size(); ++i) {
        const Geom &g = geoms[i];
        const int nm = ndim >= 2 ? g.n[ndim - 1] : 1;
        const int nty = ndim == 3 ? (g.n[1] + TY - 1) / TY : 1;
        const int ntx = (g.n[0] + TX - 1) / TX;
        for (int b = 0; b < nty; ++b)
            for (int a = 0; a < ntx; ++a) {
                const int w = std::min(TX, g.n[0] - a * TX);
                const int h = ndim == 3 ? std::min(TY, g.n[1] - b * TY) : 1;
                const double per = (double)w * h + fixed;
                pieces.push_back(Piece{SegDesc{ids[i], a * TX, b * TY, 0, nm}, per});
                W += per * (nm + warm);
            }
    }
    const double cap = W / (4.0 * std::max(1, resident));
    std::vector<Piece> cut;
    for (const Piece &r : pieces) {
        const int nm = r.s.k1;
        const double full = (warm + nm) * r.cost;
        int np = 1;
        if (ndim >= 2 && full > cap) np = std::max(1, std::min((int)std::ceil(full / cap), nm / 16));
        for (int q = 0; q < np; ++q) {
            const int k0 = (int)((long long)nm * q / np), k1 = (int)((long long)nm * (q + 1) / np);
            SegDesc sd = r.s;
            sd.k0 = k0;
            sd.k1 = k1;
            cut.push_back(Piece{sd, (warm + (k1 - k0)) * r.cost});
        }
    }
    std::stable_sort(cut.begin(), cut.end(), [](const Piece &a, const Piece &b) { return a.cost > b.cost; });
    segs.clear();
    for (const Piece &p : cut) segs.push_back(p.s);
    const int G = std::max(1, std::min<int>(resident, (int)segs.size()));
    cta_seg.assign(G + 1, 0);
    for (int c = 0; c <= G; ++c) cta_seg[c] = (int)((long long)segs.size() * c / G);
}

void multi_variant_tile(int ndim, int variant, int *tx, int *ty) {
    // the same shapes as variant_tile() of the kernels (tx = 0: none)
    static const int table[4][kMultiVariants][2] = {{{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
                                                    {{128, 1}, {256, 1}, {0, 0}, {0, 0}, {0, 0}},
                                                    {{64, 1}, {128, 1}, {256, 1}, {124, 1}, {252, 1}},
                                                    {{32, 8}, {32, 16}, {64, 8}, {0, 0}, {0, 0}}};
    *tx = *ty = 0;
    if (ndim < 1 || ndim > 3 || variant < 0 || variant >= kMultiVariants) return;
    *tx = table[ndim][variant][0];
    *ty = table[ndim][variant][1];
}
int multi_resident(bool fp64, int ndim, int variant) {
    return fp64 ? multi_resident_fp64(ndim, variant) : multi_resident_mixed(ndim, variant);
}
cudaError_t launch_multi_stage(bool fp64, const MultiArgs &a, int ndim, int variant, int stage, int nblocks,
                               cudaStream_t s) {
    return fp64 ? launch_multi_stage_fp64(a, ndim, variant, stage, nblocks, s)
                : launch_multi_stage_mixed(a, ndim, variant, stage, nblocks, s);
}
cudaError_t launch_multi_dt(bool fp64, const MultiArgs &a, int ndim, int variant, int nblocks, cudaStream_t s) {
    return fp64 ? launch_multi_dt_fp64(a, ndim, variant, nblocks, s) : launch_multi_dt_mixed(a, ndim, variant, nblocks, s);
}
}  // namespace khy

extern "C" {

khy_status khy_batch_create(const khy_mesh_desc *descs, int ngrids, void *cuda_stream, khy_batch **out) {
    if (!out) return bfail(KHY_ERR_ARG, "khy_batch_create: out is NULL");
    *out = nullptr;
    if (!descs || ngrids < 1) return bfail(KHY_ERR_ARG, "khy_batch_create: need at least one grid");
    for (int i = 0; i < ngrids; ++i) {
        int st = validate_desc(&descs[i]);
        if (st != KHY_OK) return (khy_status)st;
        if (descs[i].ndim != descs[0].ndim || descs[i].prec != descs[0].prec)
            return bfail(KHY_ERR_ARG, "khy_batch_create: all grids must share ndim and prec");
        if (descs[i].prec == KHY_PREC_FP32) return bfail(KHY_ERR_ARG, "khy_batch_create: FP64 or mixed precision only");
        if (descs[i].integrator == KHY_INT_VL2) return bfail(KHY_ERR_ARG, "khy_batch_create: Heun integrator only");
    }
    khy_batch *b = new (std::nothrow) khy_batch();
    if (!b) return bfail(KHY_ERR_OOM, "khy_batch_create: host allocation failed");
    b->ngrids = ngrids;
    b->ndim = descs[0].ndim;
    b->prec = descs[0].prec;
    b->nvar = 2 + b->ndim;
    b->desc.assign(descs, descs + ngrids);
    b->gd.resize(ngrids);
    size_t off = 0, hoff = 0;
    b->hoff.resize(ngrids);
    for (int i = 0; i < ngrids; ++i) {
        GridDesc &g = b->gd[i];
        memset(&g, 0, sizeof(g));
        g.g = geom_of_desc(descs[i]);
        off = (off + 31) & ~size_t(31);
        g.off = (long long)off;
        b->hoff[i] = (long long)hoff;
        hoff += (size_t)b->nvar * (size_t)g.g.ncell;
        g.cubic = 1;
        for (int d = 1; d < b->ndim; ++d)
            if (g.g.dx[d] != g.g.dx[0]) g.cubic = 0;
        off += (size_t)b->nvar * (size_t)g.g.ncell;
        b->cells += g.g.ncell;
    }
    b->pool = off;
    b->hpool = hoff;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    const size_t wsize = b->prec == KHY_PREC_FP64 ? sizeof(double) : sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc(&b->U, sizeof(double) * b->pool);
    if (e == cudaSuccess) e = cudaMalloc(&b->U1, sizeof(double) * b->pool);
    if (e == cudaSuccess) e = cudaMalloc(&b->W0, wsize * b->pool);
    if (e == cudaSuccess) e = cudaMalloc(&b->W1, wsize * b->pool);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_grids, sizeof(GridDesc) * ngrids);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_hoff, sizeof(long long) * ngrids);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_hoff, b->hoff.data(), sizeof(long long) * ngrids, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_clocks, sizeof(Clock) * ngrids);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_clocks, sizeof(Clock) * ngrids);
    if (e == cudaSuccess) {
        for (int i = 0; i < ngrids; ++i) {
            memset(&b->h_clocks[i], 0, sizeof(Clock));
            b->h_clocks[i].wmin_bits = kInfBits;
        }
        e = cudaMemcpyAsync(b->d_clocks, b->h_clocks, sizeof(Clock) * ngrids, cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_grids, b->gd.data(), sizeof(GridDesc) * ngrids, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->U, 0, sizeof(double) * b->pool, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        khy_batch_destroy(b);
        return bfail(e == cudaErrorMemoryAllocation ? KHY_ERR_OOM : KHY_ERR_CUDA, cudaGetErrorString(e));
    }
    int v = 0, cps = kDefaultCtasPerSlot;
    {  // a schedule tuned for the same shape class, else variant 0
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(shape_class(b));
        if (it != g_tune_cache.end()) {
            v = it->second.first;
            cps = it->second.second;
        }
    }
    khy_status st = apply_schedule(b, v, cps);
    if (st != KHY_OK) {
        khy_batch_destroy(b);
        return st;
    }
    *out = b;
    return KHY_OK;
}

void khy_batch_destroy(khy_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->U);
    cudaFree(b->U1);
    cudaFree(b->W0);
    cudaFree(b->W1);
    cudaFree(b->d_grids);
    cudaFree(b->d_hoff);
    cudaFree(b->d_clocks);
    cudaFree(b->d_segs);
    cudaFree(b->d_cta);
    cudaFree(b->d_queue);
    cudaFreeHost(b->h_clocks);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

khy_status khy_batch_set_primitive(khy_batch *b, const double *W, size_t count) {
    if (!b || !W) return bfail(KHY_ERR_ARG, "khy_batch_set_primitive: NULL argument");
    if (count != b->hpool) return bfail(KHY_ERR_ARG, "khy_batch_set_primitive: count must be the sum of nvar*ncell");
    KHY_BCUDA(cudaMemcpyAsync(b->U1, W, sizeof(double) * count, cudaMemcpyHostToDevice, b->stream));
    const int blocks = std::min(b->ngrids, 152 * 8);
    switch (b->ndim) {
        case 1: multi_prim_to_cons_kernel<1><<<blocks, 256, 0, b->stream>>>(b->d_grids, b->d_hoff, b->ngrids, b->U1, b->U); break;
        case 2: multi_prim_to_cons_kernel<2><<<blocks, 256, 0, b->stream>>>(b->d_grids, b->d_hoff, b->ngrids, b->U1, b->U); break;
        default: multi_prim_to_cons_kernel<3><<<blocks, 256, 0, b->stream>>>(b->d_grids, b->d_hoff, b->ngrids, b->U1, b->U); break;
    }
    KHY_BCUDA(cudaGetLastError());
    KHY_BCUDA(cudaStreamSynchronize(b->stream));
    b->wmin_valid = false;
    return KHY_OK;
}

khy_status khy_batch_set_conserved(khy_batch *b, const double *U, size_t count) {
    if (!b || !U) return bfail(KHY_ERR_ARG, "khy_batch_set_conserved: NULL argument");
    if (count != b->hpool) return bfail(KHY_ERR_ARG, "khy_batch_set_conserved: count must be the sum of nvar*ncell");
    KHY_BCUDA(cudaMemcpyAsync(b->U1, U, sizeof(double) * count, cudaMemcpyHostToDevice, b->stream));  // staging
    multi_relayout_kernel<<<relayout_grid(b->ngrids), 256, 0, b->stream>>>(b->d_grids, b->d_hoff, b->ngrids,
                                                                                b->nvar, b->U1, b->U, 1);
    KHY_BCUDA(cudaGetLastError());
    KHY_BCUDA(cudaStreamSynchronize(b->stream));
    b->wmin_valid = false;
    return KHY_OK;
}

khy_status khy_batch_get_conserved(khy_batch *b, double *U, size_t count) {
    if (!b || !U) return bfail(KHY_ERR_ARG, "khy_batch_get_conserved: NULL argument");
    if (count != b->hpool) return bfail(KHY_ERR_ARG, "khy_batch_get_conserved: count must be the sum of nvar*ncell");
    // U1 holds nothing between steps: it stages the host layout
    multi_relayout_kernel<<<relayout_grid(b->ngrids), 256, 0, b->stream>>>(b->d_grids, b->d_hoff, b->ngrids,
                                                                                b->nvar, b->U, b->U1, 0);
    KHY_BCUDA(cudaGetLastError());
    KHY_BCUDA(cudaMemcpyAsync(U, b->U1, sizeof(double) * count, cudaMemcpyDeviceToHost, b->stream));
    KHY_BCUDA(cudaStreamSynchronize(b->stream));
    return KHY_OK;
}

khy_status khy_batch_set_target(khy_batch *b, int grid, double t_end, long max_steps) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_set_target: NULL batch");
    if (grid < -1 || grid >= b->ngrids) return bfail(KHY_ERR_ARG, "khy_batch_set_target: grid out of range");
    if (std::isnan(t_end)) return bfail(KHY_ERR_ARG, "khy_batch_set_target: t_end is NaN");
    const int first = grid < 0 ? 0 : grid, count = grid < 0 ? b->ngrids : 1;
    multi_target_kernel<<<(count + 127) / 128, 128, 0, b->stream>>>(b->d_clocks, first, count, t_end,
                                                                     max_steps < 0 ? -1LL : (long long)max_steps);
    KHY_BCUDA(cudaGetLastError());
    return KHY_OK;
}

khy_status khy_batch_enqueue_steps(khy_batch *b, long nsteps) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_enqueue_steps: NULL batch");
    if (nsteps < 0) return bfail(KHY_ERR_ARG, "khy_batch_enqueue_steps: nsteps must be >= 0");
    khy_status st = ensure_batch_wmin(b);
    if (st != KHY_OK) return st;
    if ((st = ensure_batch_graph(b)) != KHY_OK) return st;
    long left = nsteps;
    for (; left >= kBatchStepsPerGraph; left -= kBatchStepsPerGraph) KHY_BCUDA(cudaGraphLaunch(b->graph, b->stream));
    for (; left > 0; --left) KHY_BCUDA(enqueue_batch_step(b));
    return KHY_OK;
}

khy_status khy_batch_run(khy_batch *b, long *batch_steps) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_run: NULL batch");
    long n = 0;
    khy_status st = read_clocks(b);
    if (st != KHY_OK) return st;
    while (!all_done(b)) {
        if ((st = khy_batch_enqueue_steps(b, kBatchStepsPerGraph)) != KHY_OK) return st;
        n += kBatchStepsPerGraph;
        if ((st = read_clocks(b)) != KHY_OK) return st;
    }
    if (batch_steps) *batch_steps = n;
    return batch_status(b);
}

khy_status khy_batch_get_clock(khy_batch *b, int grid, double *t, long *steps, double *dt) {
    if (!b || grid < 0 || grid >= b->ngrids) return bfail(KHY_ERR_ARG, "khy_batch_get_clock: bad batch or grid");
    khy_status st = read_clocks(b);
    if (st != KHY_OK) return st;
    if (t) *t = b->h_clocks[grid].t;
    if (steps) *steps = (long)b->h_clocks[grid].steps;
    if (dt) *dt = b->h_clocks[grid].dt;
    return KHY_OK;
}

khy_status khy_batch_set_variant(khy_batch *b, int variant) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_set_variant: NULL batch");
    return apply_schedule(b, variant, b->ctas_per_slot);
}

khy_status khy_batch_set_schedule(khy_batch *b, int variant, int ctas_per_slot) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_set_schedule: NULL batch");
    return apply_schedule(b, variant, ctas_per_slot);
}

khy_status khy_batch_get_schedule(khy_batch *b, int *variant, int *ctas_per_slot) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_get_schedule: NULL batch");
    if (variant) *variant = b->variant;
    if (ctas_per_slot) *ctas_per_slot = b->ctas_per_slot;
    return KHY_OK;
}

khy_status khy_batch_profile_steps(khy_batch *b, long nsteps, float ms[3]) {
    if (!b || !ms || nsteps < 1) return bfail(KHY_ERR_ARG, "khy_batch_profile_steps: bad argument");
    khy_status st = ensure_batch_wmin(b);
    if (st != KHY_OK) return st;
    cudaEvent_t ev[4];
    for (auto &x : ev) KHY_BCUDA(cudaEventCreate(&x));
    double acc[3] = {0, 0, 0};
    const bool fp64 = b->prec == KHY_PREC_FP64;
    cudaError_t e = cudaSuccess;
    for (long i = 0; i < nsteps && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ev[0], b->stream);
        if (e == cudaSuccess) {
            multi_clock_kernel<<<(b->ngrids + 127) / 128, 128, 0, b->stream>>>(b->d_grids, b->d_clocks, b->ngrids, b->d_queue);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
        if (e == cudaSuccess) e = launch_multi_stage(fp64, args_of(b, 1), b->ndim, b->variant, 1, b->nblocks, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], b->stream);
        if (e == cudaSuccess) e = launch_multi_stage(fp64, args_of(b, 2), b->ndim, b->variant, 2, b->nblocks, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3], b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    KHY_BCUDA(e);
    for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / nsteps);
    return KHY_OK;
}

khy_status khy_batch_autotune(khy_batch *b, int trial_steps, int *variant, float *ms_per_step) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_autotune: NULL batch");
    if (trial_steps < 1) trial_steps = 2;
    // the trials step a copy; the state and the clocks are put back afterwards
    double *saved = nullptr;
    Clock *saved_clk = nullptr;
    KHY_BCUDA(cudaMalloc(&saved, sizeof(double) * b->pool));
    cudaError_t e = cudaMalloc(&saved_clk, sizeof(Clock) * b->ngrids);
    if (e != cudaSuccess) {
        cudaFree(saved);
        KHY_BCUDA(e);
    }
    e = cudaMemcpyAsync(saved, b->U, sizeof(double) * b->pool, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(saved_clk, b->d_clocks, sizeof(Clock) * b->ngrids, cudaMemcpyDeviceToDevice, b->stream);
    int best = b->variant, best_cps = b->ctas_per_slot;
    float best_ms = 1e30f;
    khy_status st = KHY_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    constexpr int ncps = (int)(sizeof(kTunedCtasPerSlot) / sizeof(kTunedCtasPerSlot[0]));
    for (int trial = 0; trial < kMultiVariants * ncps && e == cudaSuccess && st == KHY_OK; ++trial) {
        const int v = trial / ncps, cps = kTunedCtasPerSlot[trial % ncps];
        int tx = 0, ty = 0;
        multi_variant_tile(b->ndim, v, &tx, &ty);
        if (tx == 0) continue;
        if ((st = apply_schedule(b, v, cps)) != KHY_OK) break;
        multi_target_kernel<<<(b->ngrids + 127) / 128, 128, 0, b->stream>>>(b->d_clocks, 0, b->ngrids, INFINITY,
                                                                             (long long)trial_steps + 1);
        b->wmin_valid = false;
        if ((st = ensure_batch_wmin(b)) != KHY_OK) break;
        e = enqueue_batch_step(b);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int i = 0; i < trial_steps && e == cudaSuccess; ++i) e = enqueue_batch_step(b);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms /= trial_steps;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = v;
            best_cps = cps;
        }
        // restore the state for the next trial
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->U, saved, sizeof(double) * b->pool, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_clocks, saved_clk, sizeof(Clock) * b->ngrids, cudaMemcpyDeviceToDevice, b->stream);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    cudaFree(saved);
    cudaFree(saved_clk);
    b->wmin_valid = false;
    if (st != KHY_OK) return st;
    KHY_BCUDA(e);
    if ((st = apply_schedule(b, best, best_cps)) != KHY_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[shape_class(b)] = std::make_pair(best, best_cps);
    }
    if (variant) *variant = best;
    if (ms_per_step) *ms_per_step = best_ms;
    return KHY_OK;
}

khy_status khy_batch_info(khy_batch *b, long long *cells, size_t *pool_doubles, int *variant, int *nblocks) {
    if (!b) return bfail(KHY_ERR_ARG, "khy_batch_info: NULL batch");
    if (cells) *cells = b->cells;
    if (pool_doubles) *pool_doubles = b->pool;
    if (variant) *variant = b->variant;
    if (nblocks) *nblocks = b->nblocks;
    return KHY_OK;
}

}  // extern "C"
