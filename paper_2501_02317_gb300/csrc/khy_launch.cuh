// khy_launch.cuh -- host-side dispatch of the stage and CFL kernels for one
// reconstruction precision R (included once per precision translation unit).
//
// The stage kernel runs either one CTA per run of planes of a tile column
// (large grids) or one persistent CTA per resident slot, each with a
// contiguous share of the (tile, plane) sequence.
#pragma once

#include "khy_internal.h"

namespace khy {

// Boundaries of the runs of planes a tile column is cut into (kb[0] = 0 ..
// kb[n] = nm), returns n (0: no split fits kMaxChunks): runs of about
// kChunkPlanes planes, then runs that shrink (kChunkTaper, in order) at the
// end of the column, so the last CTAs to start are short and the others do
// not wait long behind them.  Measured on the 256^3 box, mixed Heun,
// cell-updates/s: one contiguous share per resident CTA 9.41e9; runs of 24
// planes (last one 16) 1.02e10; runs of 32 then 24, 16, 12, 8, 4: 1.045e10;
// runs of ~53 then 32, 24, 16, 12, 8, 4: 1.054e10 (kept); DRAM traffic of
// the Heun stage pair 5.55 GB -> 4.12 GB (neighbouring tiles now share their
// halo rows through L2).
inline int chunk_bounds(int nm, int *kb) {
    constexpr int kChunkPlanes = 64;
    constexpr int kChunkTaper[] = {32, 24, 16, 12, 8, 4};
    constexpr int nt = (int)(sizeof(kChunkTaper) / sizeof(kChunkTaper[0]));
    int tsum = 0;
    for (int i = 0; i < nt; ++i) tsum += kChunkTaper[i];
    const int bulk = nm - tsum;
    if (bulk < kChunkPlanes) {  // short column: even runs of about kChunkPlanes
        const int n = (nm + kChunkPlanes - 1) / kChunkPlanes;
        if (n > kMaxChunks) return 0;
        for (int c = 0; c <= n; ++c) kb[c] = (int)((long long)c * nm / n);
        return n;
    }
    const int nb = (bulk + kChunkPlanes - 1) / kChunkPlanes;
    if (nb + nt > kMaxChunks) return 0;
    for (int c = 0; c <= nb; ++c) kb[c] = (int)((long long)c * bulk / nb);
    for (int i = 0; i < nt; ++i) kb[nb + 1 + i] = kb[nb + i] + kChunkTaper[i];
    return nb + nt;
}

template <class R, int ND, int STAGE, int TX, int TY, class S = double>
struct StageLaunch {
    static int &resident() {  // resident CTAs on the device, 0 until prepared
        static int r = 0;
        return r;
    }
    static cudaError_t prepare() {
        constexpr size_t smem = Tile<ND, TX, TY>::template smem_bytes<R>();
        auto kern = stage_kernel<R, ND, STAGE, TX, TY, S>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cta_threads<R, ND, TX, TY>(), smem)) != cudaSuccess) return e;
        resident() = sms * (per_sm > 0 ? per_sm : 1);
        return cudaSuccess;
    }
    static cudaError_t launch(const StageArgs &a, cudaStream_t s) {
        if (resident() == 0) {
            cudaError_t e = prepare();
            if (e != cudaSuccess) return e;
        }
        constexpr size_t smem = Tile<ND, TX, TY>::template smem_bytes<R>();
        const long long ntx = (a.g.n[0] + TX - 1) / TX;
        const long long nty = (ND == 3) ? (a.g.n[1] + TY - 1) / TY : 1;
        const long long nm = (ND >= 2) ? a.g.n[ND - 1] : 1;
        // Large grids: each tile column cut into runs of planes (chunk_bounds),
        // one run per CTA, as many CTAs as runs (the hardware balances
        // them).  Grids with fewer runs than three CTA waves keep one
        // contiguous share per resident CTA (their state fits in L2, and a
        // persistent CTA pays fewer warm-up planes).
        StageArgs b = a;
        long long total;
        const int nch = (ND >= 2) ? chunk_bounds((int)nm, b.kb) : 0;
        if (nch > 0 && ntx * nty * nch >= 3LL * resident()) {
            b.nchunk = nch;
            total = ntx * nty * nch;
        } else {
            b.nchunk = 0;
            total = ntx * nty * nm;
            if (total > resident()) total = resident();
        }
        stage_kernel<R, ND, STAGE, TX, TY, S><<<(int)total, cta_threads<R, ND, TX, TY>(), smem, s>>>(b);
        return cudaGetLastError();
    }
};

// tile shapes per precision and dimensionality
template <class R, int ND> struct TileOf;
template <> struct TileOf<double, 1> { static constexpr int TX = 128, TY = 1; };
template <> struct TileOf<double, 2> { static constexpr int TX = 128, TY = 1; };
template <> struct TileOf<double, 3> { static constexpr int TX = 32, TY = 8; };
template <> struct TileOf<float, 1> { static constexpr int TX = 256, TY = 1; };
template <> struct TileOf<float, 2> { static constexpr int TX = 124, TY = 1; };  // 125 face-pair tasks: 4 whole warps
template <> struct TileOf<float, 3> { static constexpr int TX = 32, TY = 8; };

template <class R, int ND, int STAGE, class S = double>
using StageOf = StageLaunch<R, ND, STAGE, TileOf<R, ND>::TX, TileOf<R, ND>::TY, S>;

template <class R, int ND, class S>
static cudaError_t launch_stage_nd(const StageArgs &a, int stage, cudaStream_t s) {
    switch (stage) {
        case 1: return StageOf<R, ND, 1, S>::launch(a, s);
        case 2: return StageOf<R, ND, 2, S>::launch(a, s);
        case 3: return StageOf<R, ND, 3, S>::launch(a, s);
        case 4: return StageOf<R, ND, 4, S>::launch(a, s);
        case 5: return StageOf<R, ND, 5, S>::launch(a, s);
        case 6: return StageOf<R, ND, 6, S>::launch(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// stage 1, 2: Heun; 3, 4: van Leer predictor and corrector; 5, 6: Heun from
// stored primitives
template <class R, class S = double>
static cudaError_t launch_stage_prec(const StageArgs &a, int stage, cudaStream_t s) {
    switch (a.g.ndim) {
        case 1: return launch_stage_nd<R, 1, S>(a, stage, s);
        case 2: return launch_stage_nd<R, 2, S>(a, stage, s);
        case 3: return launch_stage_nd<R, 3, S>(a, stage, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class R, int ND, class S>
static cudaError_t prepare_nd() {
    cudaError_t e;
    if ((e = StageOf<R, ND, 1, S>::prepare()) != cudaSuccess) return e;
    if ((e = StageOf<R, ND, 2, S>::prepare()) != cudaSuccess) return e;
    if ((e = StageOf<R, ND, 3, S>::prepare()) != cudaSuccess) return e;
    if ((e = StageOf<R, ND, 4, S>::prepare()) != cudaSuccess) return e;
    if ((e = StageOf<R, ND, 5, S>::prepare()) != cudaSuccess) return e;
    return StageOf<R, ND, 6, S>::prepare();
}

template <class R, class S = double>
static cudaError_t prepare_prec(int ndim) {
    switch (ndim) {
        case 1: return prepare_nd<R, 1, S>();
        case 2: return prepare_nd<R, 2, S>();
        case 3: return prepare_nd<R, 3, S>();
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- many grids

template <class R, int ND, int STAGE, int TX, int TY>
struct MultiLaunch {
    static int &resident() {
        static int r = 0;
        return r;
    }
    static cudaError_t prepare() {
        constexpr size_t smem = Tile<ND, TX, TY>::template smem_bytes<R>();
        auto kern = multi_stage_kernel<R, ND, STAGE, TX, TY>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cta_threads<R, ND, TX, TY>(), smem)) != cudaSuccess) return e;
        resident() = sms * (per_sm > 0 ? per_sm : 1);
        return cudaSuccess;
    }
    static cudaError_t launch(const MultiArgs &a, int nblocks, cudaStream_t s) {
        if (resident() == 0) {
            cudaError_t e = prepare();
            if (e != cudaSuccess) return e;
        }
        constexpr size_t smem = Tile<ND, TX, TY>::template smem_bytes<R>();
        if (nblocks <= 0) return cudaSuccess;
        multi_stage_kernel<R, ND, STAGE, TX, TY><<<nblocks, cta_threads<R, ND, TX, TY>(), smem, s>>>(a);
        return cudaGetLastError();
    }
};

// variant table: tile shapes per dimensionality.  The 2D widths 124 and 252
// give the FP32 face loop 125 and 253 face-pair tasks per row (TX/2 march,
// TX/2 + 1 x) -- 4 and 8 whole warps -- where 128 and 256 give 129 and 257
// and one more warp-round of flux code for a single task.
struct VariantTile { int tx, ty; };
__host__ __device__ constexpr VariantTile variant_tile(int ndim, int v) {
    return ndim == 1 ? (v == 0 ? VariantTile{128, 1} : v == 1 ? VariantTile{256, 1} : VariantTile{0, 0})
         : ndim == 2 ? (v == 0 ? VariantTile{64, 1} : v == 1 ? VariantTile{128, 1} : v == 2 ? VariantTile{256, 1}
                      : v == 3 ? VariantTile{124, 1} : v == 4 ? VariantTile{252, 1} : VariantTile{0, 0})
         : ndim == 3 ? (v == 0 ? VariantTile{32, 8} : v == 1 ? VariantTile{32, 16} : v == 2 ? VariantTile{64, 8} : VariantTile{0, 0})
                     : VariantTile{0, 0};
}

template <int ND, int V>
struct VT {
    static constexpr int tx = (variant_tile(ND, V).tx > 0) ? variant_tile(ND, V).tx : 32;
    static constexpr int ty = (variant_tile(ND, V).tx > 0) ? variant_tile(ND, V).ty : 1;
};

template <class R, int ND, int V, int STAGE>
using MultiOf = MultiLaunch<R, ND, STAGE, VT<ND, V>::tx, VT<ND, V>::ty>;

// batch stage 1 / 2: the Heun stages that read stored primitives (5, 6)
template <class R, int ND, int V>
static cudaError_t multi_stage_v(const MultiArgs &a, int stage, int nblocks, cudaStream_t s) {
    return stage == 1 ? MultiOf<R, ND, V, 5>::launch(a, nblocks, s) : MultiOf<R, ND, V, 6>::launch(a, nblocks, s);
}

template <class R>
static cudaError_t launch_multi_stage_prec(const MultiArgs &a, int ndim, int v, int stage, int nblocks, cudaStream_t s) {
    if (variant_tile(ndim, v).tx == 0) return cudaErrorInvalidValue;
    switch (ndim * 10 + v) {
        case 10: return multi_stage_v<R, 1, 0>(a, stage, nblocks, s);
        case 11: return multi_stage_v<R, 1, 1>(a, stage, nblocks, s);
        case 20: return multi_stage_v<R, 2, 0>(a, stage, nblocks, s);
        case 21: return multi_stage_v<R, 2, 1>(a, stage, nblocks, s);
        case 22: return multi_stage_v<R, 2, 2>(a, stage, nblocks, s);
        case 23: return multi_stage_v<R, 2, 3>(a, stage, nblocks, s);
        case 24: return multi_stage_v<R, 2, 4>(a, stage, nblocks, s);
        case 30: return multi_stage_v<R, 3, 0>(a, stage, nblocks, s);
        case 31: return multi_stage_v<R, 3, 1>(a, stage, nblocks, s);
        case 32: return multi_stage_v<R, 3, 2>(a, stage, nblocks, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class R, int ND, int V>
static int multi_resident_v() {
    using L1 = MultiOf<R, ND, V, 5>;
    using L2 = MultiOf<R, ND, V, 6>;
    if (L1::resident() == 0 && L1::prepare() != cudaSuccess) return 0;
    if (L2::resident() == 0 && L2::prepare() != cudaSuccess) return 0;
    return L1::resident() < L2::resident() ? L1::resident() : L2::resident();
}

template <class R>
static int multi_resident_prec(int ndim, int v) {
    switch (ndim * 10 + v) {
        case 10: return multi_resident_v<R, 1, 0>();
        case 11: return multi_resident_v<R, 1, 1>();
        case 20: return multi_resident_v<R, 2, 0>();
        case 21: return multi_resident_v<R, 2, 1>();
        case 22: return multi_resident_v<R, 2, 2>();
        case 23: return multi_resident_v<R, 2, 3>();
        case 24: return multi_resident_v<R, 2, 4>();
        case 30: return multi_resident_v<R, 3, 0>();
        case 31: return multi_resident_v<R, 3, 1>();
        case 32: return multi_resident_v<R, 3, 2>();
        default: return 0;
    }
}

// CFL minimum of every grid; stores the primitives of a.Uin into the pool a.Win
template <class R>
static cudaError_t launch_multi_dt_prec(const MultiArgs &a, int ndim, int v, int nblocks, cudaStream_t s) {
    const VariantTile t = variant_tile(ndim, v);
    if (t.tx == 0) return cudaErrorInvalidValue;
    if (nblocks <= 0) return cudaSuccess;
    R *W = reinterpret_cast<R *>(const_cast<void *>(a.Win));
    switch (ndim) {
        case 1: multi_dt_kernel<R, 1><<<nblocks, 256, 0, s>>>(a, t.tx, t.ty, W); break;
        case 2: multi_dt_kernel<R, 2><<<nblocks, 256, 0, s>>>(a, t.tx, t.ty, W); break;
        case 3: multi_dt_kernel<R, 3><<<nblocks, 256, 0, s>>>(a, t.tx, t.ty, W); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class R, class S = double>
static cudaError_t launch_dt_prec(const Geom &g, const double *U, Clock *clk, void *W, int from_state,
                                  cudaStream_t s) {
    const long long blocks_needed = (g.ncell + 255) / 256;
    const int blocks = (int)(blocks_needed < 152 * 8 ? blocks_needed : 152 * 8);
    R *Wr = reinterpret_cast<R *>(W);
    switch (g.ndim) {
        case 1: dt_kernel<R, 1, S><<<blocks, 256, 0, s>>>(g, U, clk, Wr, from_state); break;
        case 2: dt_kernel<R, 2, S><<<blocks, 256, 0, s>>>(g, U, clk, Wr, from_state); break;
        case 3: dt_kernel<R, 3, S><<<blocks, 256, 0, s>>>(g, U, clk, Wr, from_state); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace khy
