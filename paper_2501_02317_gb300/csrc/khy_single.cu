// khy_single.cu -- all-FP32 instantiation of the hydro kernels: FP32 state,
// FP32 reconstruction and fluxes (the paper's "Single" configuration,
// Sec. 3.2.2 with float2_t mapped to single precision).
#include "khy_launch.cuh"

namespace khy {

cudaError_t launch_stage_single(const StageArgs &a, int stage, cudaStream_t s) {
    return launch_stage_prec<float, float>(a, stage, s);
}

cudaError_t launch_dt_single(const Geom &g, const double *U, Clock *clk, void *W, int from_state, cudaStream_t s) {
    return launch_dt_prec<float, float>(g, U, clk, W, from_state, s);
}

cudaError_t prepare_single(int ndim) { return prepare_prec<float, float>(ndim); }

}  // namespace khy
