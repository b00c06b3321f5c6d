// lbm_f16.cu -- instantiation of the fused step, read-out and init kernels
// with FP16 population storage and FP32 arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

template <int MODE, bool DIAG>
static void launch_one(const Args<float, __half>& a, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g), block = block_dims();
  if (a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT))
    lbm_step_kernel<float, MODE, DIAG, 7, __half><<<grid, block, 0, s>>>(a);
  else
    lbm_step_kernel<float, MODE, DIAG, 0, __half><<<grid, block, 0, s>>>(a);
}

cudaError_t launch_step_f16s(const Args<float, __half>& a, int mode, bool diag, cudaStream_t s) {
  if (mode == MODE_STEP) {
    if (diag) launch_one<MODE_STEP, true>(a, s);
    else launch_one<MODE_STEP, false>(a, s);
  } else {
    if (diag) launch_one<MODE_READ, true>(a, s);
    else launch_one<MODE_READ, false>(a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_f16s(const InitArgs<float, __half>& a, cudaStream_t s) {
  lbm_init_kernel<float, __half><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lbmk
