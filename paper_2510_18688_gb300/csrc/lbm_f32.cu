// lbm_f32.cu -- instantiation of the fused step, read-out and init kernels
// for float arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

cudaError_t launch_step_f32(const Args<float>& a, int mode, bool diag, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g), block = block_dims();
  if (mode == MODE_STEP) {
    if (diag) lbm_step_kernel<float, MODE_STEP, true><<<grid, block, 0, s>>>(a);
    else lbm_step_kernel<float, MODE_STEP, false><<<grid, block, 0, s>>>(a);
  } else {
    if (diag) lbm_step_kernel<float, MODE_READ, true><<<grid, block, 0, s>>>(a);
    else lbm_step_kernel<float, MODE_READ, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_f32(const InitArgs<float>& a, cudaStream_t s) {
  lbm_init_kernel<float><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lbmk
