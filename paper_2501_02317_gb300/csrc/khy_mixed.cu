// khy_mixed.cu -- mixed-precision instantiation of the hydro kernels
// (Sec. 3.2.2): PLM reconstruction and the HLLC flux in FP32; conserved state,
// the internal energy of the recovery and the flux-difference accumulation in
// FP64 (see khy_mixed_kernels.cuh for how the FP64 work is kept small).
#include "khy_launch.cuh"

namespace khy {

cudaError_t launch_stage_mixed(const StageArgs &a, int stage, cudaStream_t s) {
    return launch_stage_prec<float>(a, stage, s);
}

cudaError_t launch_dt_mixed(const Geom &g, const double *U, Clock *clk, void *W, int from_state, cudaStream_t s) {
    return launch_dt_prec<float>(g, U, clk, W, from_state, s);
}

cudaError_t prepare_mixed(int ndim) { return prepare_prec<float>(ndim); }

cudaError_t launch_multi_stage_mixed(const MultiArgs &a, int ndim, int variant, int stage, int nblocks,
                                  cudaStream_t s) {
    return launch_multi_stage_prec<float>(a, ndim, variant, stage, nblocks, s);
}

cudaError_t launch_multi_dt_mixed(const MultiArgs &a, int ndim, int variant, int nblocks, cudaStream_t s) {
    return launch_multi_dt_prec<float>(a, ndim, variant, nblocks, s);
}

int multi_resident_mixed(int ndim, int variant) { return multi_resident_prec<float>(ndim, variant); }

}  // namespace khy
