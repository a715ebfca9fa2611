// khy_launch.cuh -- host-side dispatch of the stage and CFL kernels for one
// reconstruction precision R (included once per precision translation unit).
#pragma once

#include "khy_internal.h"

namespace khy {

template <int ND, class R, int STAGE, int TX, int TY>
static cudaError_t configure_stage_tile() {
    constexpr size_t smem = Tile<ND, TX, TY>::template smem_bytes<R>();
    return cudaFuncSetAttribute(stage_kernel<ND, R, STAGE, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <int ND, class R, int STAGE, int TX, int TY>
static cudaError_t launch_stage_tile(const StageArgs &a, cudaStream_t s) {
    using T = Tile<ND, TX, TY>;
    constexpr size_t smem = T::template smem_bytes<R>();
    dim3 grid;
    const int nxt = (a.g.n[0] + TX - 1) / TX;
    if (ND == 1) {
        grid = dim3(nxt, 1, 1);
    } else if (ND == 2) {
        grid = dim3(nxt, (a.g.n[1] + a.kchunk - 1) / a.kchunk, 1);
    } else {
        grid = dim3(nxt, (a.g.n[1] + TY - 1) / TY, (a.g.n[2] + a.kchunk - 1) / a.kchunk);
    }
    stage_kernel<ND, R, STAGE, TX, TY><<<grid, TX * TY, smem, s>>>(a);
    return cudaGetLastError();
}

template <class R>
static cudaError_t launch_stage_prec(const StageArgs &a, int stage, cudaStream_t s) {
    switch (a.g.ndim) {
        case 1: return stage == 1 ? launch_stage_tile<1, R, 1, 128, 1>(a, s) : launch_stage_tile<1, R, 2, 128, 1>(a, s);
        case 2: return stage == 1 ? launch_stage_tile<2, R, 1, 128, 1>(a, s) : launch_stage_tile<2, R, 2, 128, 1>(a, s);
        case 3: return stage == 1 ? launch_stage_tile<3, R, 1, 32, 8>(a, s) : launch_stage_tile<3, R, 2, 32, 8>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class R>
static cudaError_t prepare_prec(int ndim) {
    cudaError_t e;
    switch (ndim) {
        case 1:
            if ((e = configure_stage_tile<1, R, 1, 128, 1>()) != cudaSuccess) return e;
            return configure_stage_tile<1, R, 2, 128, 1>();
        case 2:
            if ((e = configure_stage_tile<2, R, 1, 128, 1>()) != cudaSuccess) return e;
            return configure_stage_tile<2, R, 2, 128, 1>();
        case 3:
            if ((e = configure_stage_tile<3, R, 1, 32, 8>()) != cudaSuccess) return e;
            return configure_stage_tile<3, R, 2, 32, 8>();
        default: return cudaErrorInvalidValue;
    }
}

static inline cudaError_t launch_dt_any(const Geom &g, const double *U, Clock *clk, cudaStream_t s) {
    const long long blocks_needed = (g.ncell + 255) / 256;
    const int blocks = (int)(blocks_needed < 152 * 8 ? blocks_needed : 152 * 8);
    switch (g.ndim) {
        case 1: dt_kernel<1><<<blocks, 256, 0, s>>>(g, U, clk); break;
        case 2: dt_kernel<2><<<blocks, 256, 0, s>>>(g, U, clk); break;
        case 3: dt_kernel<3><<<blocks, 256, 0, s>>>(g, U, clk); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace khy
