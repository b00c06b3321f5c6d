// lbm_f64.cu -- instantiation of the fused step, read-out and init kernels
// for double arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

cudaError_t launch_step_f64(const Args<double>& a, int mode, bool diag, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g), block = block_dims();
  if (mode == MODE_STEP) {
    if (diag) lbm_step_kernel<double, MODE_STEP, true><<<grid, block, 0, s>>>(a);
    else lbm_step_kernel<double, MODE_STEP, false><<<grid, block, 0, s>>>(a);
  } else {
    if (diag) lbm_step_kernel<double, MODE_READ, true><<<grid, block, 0, s>>>(a);
    else lbm_step_kernel<double, MODE_READ, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_f64(const InitArgs<double>& a, cudaStream_t s) {
  lbm_init_kernel<double><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lbmk
