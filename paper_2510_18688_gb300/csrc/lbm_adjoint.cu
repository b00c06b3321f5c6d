// lbm_adjoint.cu -- the reverse-mode (adjoint) kernels and their launchers: enthalpy lattice,
// phase field, the two coupled, and the whole step (lbm_adjoint.cuh, lbm_adjoint_full.cuh).
// the kernels of the adjoint headers are compiled in this unit only
#define LBM_ADJOINT_KERNELS
#include "lbm_adjoint.cuh"
#include "lbm_adjoint_full.cuh"
#include "lbm_launch.h"

namespace lbmk {

cudaError_t launch_adjoint_seed(const AdjArgs& a, cudaStream_t s) {
  lbm_adjoint_seed_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const AdjArgs& a, cudaStream_t s) {
  lbm_adjoint_step_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const AdjArgs& a, cudaStream_t s) {
  lbm_adjoint_init_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_reduce(const double* acc, const Geom& g, double* out, cudaStream_t s) {
  lbm_adjoint_reduce_kernel<<<1, NT, 0, s>>>(acc, g, out);
  return cudaGetLastError();
}

cudaError_t launch_phase_adjoint_fields(const PhaseAdjArgs& a, cudaStream_t s) {
  lbm_phase_fields_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_phase_adjoint_seed(const PhaseAdjArgs& a, cudaStream_t s) {
  lbm_phase_seed_kernel<<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

// one reverse step: the node's own terms, then the gather of the stencil
// transposes and the local chain
cudaError_t launch_phase_adjoint_step(const PhaseAdjArgs& a, cudaStream_t s) {
  lbm_phase_adjoint1_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  lbm_phase_adjoint2_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_phase_adjoint_init(const PhaseAdjArgs& a, cudaStream_t s) {
  lbm_phase_init_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_frz_fields(const FrzArgs& a, cudaStream_t s) {
  lbm_frz_fields_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_frz_mub(const FrzArgs& a, cudaStream_t s) {
  lbm_frz_mub_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_frz_step(const FrzArgs& a, cudaStream_t s) {
  lbm_frz_step_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_frz_seed_ff(const FrzArgs& a, cudaStream_t s) {
  lbm_frz_seed_ff_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_frz_seed_crossing(const FrzArgs& a, double* phib, cudaStream_t s) {
  lbm_frz_seed_crossing_kernel<<<1, 32, 0, s>>>(a, phib);
  return cudaGetLastError();
}

cudaError_t launch_full_fields(const FullArgs& a, cudaStream_t s) {
  lbm_full_fields_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_full_k1(const FullArgs& a, cudaStream_t s) {
  lbm_full_k1_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_full_k2(const FullArgs& a, cudaStream_t s) {
  lbm_full_k2_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_full_seed_ff(const FullArgs& a, double* llag, cudaStream_t s) {
  lbm_full_seed_ff_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a, llag);
  return cudaGetLastError();
}

cudaError_t launch_full_seed_crossing(const FullArgs& a, double* phib, cudaStream_t s) {
  lbm_full_seed_crossing_kernel<<<1, 32, 0, s>>>(a, phib);
  return cudaGetLastError();
}

cudaError_t launch_full_dT0(const FullArgs& a, const double* lam, double* out, cudaStream_t s) {
  lbm_full_dT0_kernel<<<grid_dims(a.g), block_dims(), 0, s>>>(a, lam, out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_init_fields(const Geom& g, const double* gpop, const double* lag,
                                       const double* phi0, double* phi, double* fs,
                                       cudaStream_t s) {
  lbm_adjoint_init_fields_kernel<<<grid_dims(g), block_dims(), 0, s>>>(g, gpop, lag, phi0, phi, fs);
  return cudaGetLastError();
}

}  // namespace lbmk
