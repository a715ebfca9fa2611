// khy_internal.h -- launchers shared between the translation units of
// libkhydro.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "khy_stage.cuh"

namespace khy {

// Stage kernel (stage 1, 2: Heun; 3, 4: van Leer predictor and corrector;
// 5, 6: Heun from stored primitives) and CFL-minimum kernel for each
// precision; the CFL kernel also stores the primitives when W is not null,
// and with from_state uses the van Leer corrector's estimate (mixed / FP32).
// khy_fp64.cu builds the double instantiations with -fmad=false; khy_mixed.cu
// builds the float (mixed) instantiations.
cudaError_t launch_stage_fp64(const StageArgs &a, int stage, cudaStream_t s);
cudaError_t launch_dt_fp64(const Geom &g, const double *U, Clock *clk, void *W, int from_state, cudaStream_t s);
cudaError_t launch_stage_mixed(const StageArgs &a, int stage, cudaStream_t s);
cudaError_t launch_dt_mixed(const Geom &g, const double *U, Clock *clk, void *W, int from_state, cudaStream_t s);
// all-FP32 path (khy_single.cu): the state pointers in StageArgs and U point
// to FP32 arrays (the buffers are reinterpreted)
cudaError_t launch_stage_single(const StageArgs &a, int stage, cudaStream_t s);
cudaError_t launch_dt_single(const Geom &g, const double *U, Clock *clk, void *W, int from_state, cudaStream_t s);
cudaError_t prepare_single(int ndim);

// Many-grid (batched / served) launches.  A variant is a tile shape; the
// variants of each dimensionality are listed by multi_variant_tile (the
// autotuner times them and picks one).  nblocks is the CTA count of the
// segment schedule (at most multi_resident).
constexpr int kMultiVariants = 5;
void multi_variant_tile(int ndim, int variant, int *tx, int *ty);  // tx = 0: no such variant
int multi_resident(bool fp64, int ndim, int variant);              // resident CTAs, 0 on error
cudaError_t launch_multi_stage(bool fp64, const MultiArgs &a, int ndim, int variant, int stage, int nblocks,
                               cudaStream_t s);
cudaError_t launch_multi_dt(bool fp64, const MultiArgs &a, int ndim, int variant, int nblocks, cudaStream_t s);
cudaError_t launch_multi_stage_fp64(const MultiArgs &a, int ndim, int variant, int stage, int nblocks, cudaStream_t s);
cudaError_t launch_multi_stage_mixed(const MultiArgs &a, int ndim, int variant, int stage, int nblocks, cudaStream_t s);
cudaError_t launch_multi_dt_fp64(const MultiArgs &a, int ndim, int variant, int nblocks, cudaStream_t s);
cudaError_t launch_multi_dt_mixed(const MultiArgs &a, int ndim, int variant, int nblocks, cudaStream_t s);
int multi_resident_fp64(int ndim, int variant);
int multi_resident_mixed(int ndim, int variant);

// Segment schedule for many grids (khy_batch.cu): every tile of every grid
// (ids[i] names grid i in the SegDesc) is a run of planes along its march
// axis; the runs are cut at nblocks equal shares of the estimated cost.
void build_segments(const std::vector<int> &ids, const std::vector<Geom> &geoms, int ndim, int TX, int TY,
                    int nblocks, std::vector<SegDesc> &segs, std::vector<int> &cta_seg);
void build_segments_queue(const std::vector<int> &ids, const std::vector<Geom> &geoms, int ndim, int TX, int TY,
                          int resident, std::vector<SegDesc> &segs, std::vector<int> &cta_seg);

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
