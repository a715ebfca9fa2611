// khy_fp64.cu -- all-FP64 instantiation of the hydro kernels.  Built with
// -fmad=false: every double operation rounds on its own, in the order the
// CPU reference uses, so results match it bit for bit.
#include "khy_launch.cuh"

namespace khy {

cudaError_t launch_stage_fp64(const StageArgs &a, int stage, cudaStream_t s) {
    return launch_stage_prec<double>(a, stage, s);
}

cudaError_t launch_dt_fp64(const Geom &g, const double *U, Clock *clk, void *W, int from_state, cudaStream_t s) {
    return launch_dt_prec<double>(g, U, clk, W, from_state, s);
}

cudaError_t prepare_fp64(int ndim) { return prepare_prec<double>(ndim); }

cudaError_t launch_multi_stage_fp64(const MultiArgs &a, int ndim, int variant, int stage, int nblocks,
                                  cudaStream_t s) {
    return launch_multi_stage_prec<double>(a, ndim, variant, stage, nblocks, s);
}

cudaError_t launch_multi_dt_fp64(const MultiArgs &a, int ndim, int variant, int nblocks, cudaStream_t s) {
    return launch_multi_dt_prec<double>(a, ndim, variant, nblocks, s);
}

int multi_resident_fp64(int ndim, int variant) { return multi_resident_prec<double>(ndim, variant); }

}  // namespace khy
