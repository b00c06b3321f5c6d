// lbm_adjoint.cu -- launchers of the enthalpy-lattice adjoint kernels.
#include "lbm_adjoint.cuh"
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

}  // namespace lbmk
