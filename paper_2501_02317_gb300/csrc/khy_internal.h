// khy_internal.h -- launchers shared between the translation units of
// libkhydro.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include "khy_stage.cuh"

namespace khy {

// Stage kernel (stage = 1 or 2) and CFL-minimum kernel for each precision.
// khy_fp64.cu builds the double instantiations with -fmad=false; khy_mixed.cu
// builds the float (mixed) instantiations.
cudaError_t launch_stage_fp64(const StageArgs &a, int stage, cudaStream_t s);
cudaError_t launch_dt_fp64(const Geom &g, const double *U, Clock *clk, cudaStream_t s);
cudaError_t launch_stage_mixed(const StageArgs &a, int stage, cudaStream_t s);
cudaError_t launch_dt_mixed(const Geom &g, const double *U, Clock *clk, cudaStream_t s);

// Sets the shared-memory limits of the stage kernels of one dimensionality
// and caches their persistent grid sizes; call before the first launch (in
// particular before a stream capture).
cudaError_t prepare_fp64(int ndim);
cudaError_t prepare_mixed(int ndim);

}  // namespace khy

// Runtime helpers shared with khy_noalloc.cu (implemented in khy_runtime.cu).

struct khy_mesh_desc;

namespace khy {
int validate_desc(const khy_mesh_desc *d);             // khy_status of the descriptor check
Geom geom_of_desc(const khy_mesh_desc &d);
int record_error(int status, const char *msg);         // sets khy_last_error(), returns status
cudaError_t launch_clock_step(Clock *c, const Geom &g, cudaStream_t s);
}  // namespace khy
