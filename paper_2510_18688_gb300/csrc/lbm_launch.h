// lbm_launch.h -- host-side launchers of the sm_103a kernels (internal to
// the library; the public interface is include/lbm.h).
#pragma once

#include <cuda_runtime.h>

#include "lbm_kernels.cuh"
#include "lbm_step.cuh"
#include "lbm_split.cuh"
#include "lbm_tile.cuh"

namespace lbmk {

inline dim3 block_dims(int ty = TY) { return dim3(TX, (unsigned)ty, 1); }
inline dim3 grid_dims(const Geom& g, int ty = TY) {
  return dim3((unsigned)((g.nx + TX - 1) / TX), (unsigned)tiles_y(g.ny, ty), 1);
}

// MODE_STEP or MODE_READ, with or without the fused diagnostics; MODE_STEP
// on 32 x ty tiles (ty = 4, 8 or 16), MODE_READ on 32 x 8.
cudaError_t launch_step_f32(const Args<float>& a, int mode, bool diag, cudaStream_t s,
                            int ty = TY);
cudaError_t launch_step_f64(const Args<double>& a, int mode, bool diag, cudaStream_t s,
                            int ty = TY);
// Two-kernel form of MODE_STEP (macro pass, then collide pass).
cudaError_t launch_split_f64(const SplitArgs<double>& a, bool diag, cudaStream_t s);
cudaError_t launch_init_f32(const InitArgs<float>& a, cudaStream_t s);
// The float step as the TMA-staged tile kernel (lbm_tile.cuh) with 1 or 2
// shared-memory stages on `grid` CTAs (persistent when grid < tiles);
// prepare_tile_* sets its shared-memory sizes once (call before the first
// launch, outside stream capture).
cudaError_t prepare_tile_f32();  // also the batched tile kernel
cudaError_t prepare_tile_f16s();
cudaError_t launch_tile_f32(const TileArgs<float>& t, bool diag, int stages, int grid,
                            cudaStream_t s);
cudaError_t launch_tile_f16s(const TileArgs<__half>& t, bool diag, int stages, int grid,
                             cudaStream_t s);
// Up to BATCH_MAX_GRIDS FP32 grids in one launch of the one-stage tile
// kernel, one CTA per 32 x 8 tile.
cudaError_t launch_tile_batch_f32(const TileBatch<float>& b, bool diag, bool all,
                                  cudaStream_t s);
// FP16 population storage, FP32 arithmetic.
cudaError_t launch_step_f16s(const Args<float, __half>& a, int mode, bool diag, cudaStream_t s,
                             int ty = TY);
cudaError_t launch_init_f16s(const InitArgs<float, __half>& a, cudaStream_t s);
// Reverse mode of the enthalpy-lattice step (lbm_adjoint.cuh).
struct AdjArgs;
cudaError_t launch_adjoint_seed(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_step(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_init(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_reduce(const double* acc, const Geom& g, double* out, cudaStream_t s);
// Forward-mode tangent (FP64 value and derivative).
cudaError_t launch_step_tan(const Args<Dual>& a, int mode, bool diag, cudaStream_t s);
cudaError_t launch_init_tan(const InitArgs<Dual>& a, cudaStream_t s);
// Up to BATCH_MAX_GRIDS grids in one launch, one CTA per tile.
cudaError_t launch_batch_f32(const BatchTable<float>& b, bool diag, bool all, cudaStream_t s);
cudaError_t launch_batch_f64(const BatchTable<double>& b, bool diag, bool all, cudaStream_t s);
// Grid-wide diagnostics from the per-CTA partials (one CTA).
cudaError_t launch_diag_finalize(const double* partial, int nb, double* out, long long step,
                                 cudaStream_t s);
cudaError_t launch_init_f64(const InitArgs<double>& a, cudaStream_t s);
// Interface crossings along one line of dense FP64 fields (one CTA); out: 2
// device doubles, or 4 with the derivative fields (else null).
cudaError_t launch_crossings(const double* phi, const double* w, const double* fl,
                             const double* dphi, const double* dw, const double* dfl, int nx,
                             int ny, int axis, int index, double* out, cudaStream_t s);

}  // namespace lbmk
