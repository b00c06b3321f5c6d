// lbm_f32.cu -- instantiation of the fused step, read-out and init kernels
// for float arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

template <int MODE, bool DIAG>
static void launch_one(const Args<float>& a, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g), block = block_dims();
  // the all-lattices case is specialised at compile time
  if (a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT))
    lbm_step_kernel<float, MODE, DIAG, 7><<<grid, block, 0, s>>>(a);
  else
    lbm_step_kernel<float, MODE, DIAG, 0><<<grid, block, 0, s>>>(a);
}

cudaError_t launch_step_f32(const Args<float>& a, int mode, bool diag, cudaStream_t s) {
  if (mode == MODE_STEP) {
    if (diag) launch_one<MODE_STEP, true>(a, s);
    else launch_one<MODE_STEP, false>(a, s);
  } else {
    if (diag) launch_one<MODE_READ, true>(a, s);
    else launch_one<MODE_READ, false>(a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_f32(const BatchTable<float>& b, bool diag, bool all, cudaStream_t s) {
  const dim3 block = block_dims();
  const int ctas = b.tile_base[b.ngrids];
  if (all) {
    if (diag) lbm_batch_kernel<float, true, 7><<<ctas, block, 0, s>>>(b);
    else lbm_batch_kernel<float, false, 7><<<ctas, block, 0, s>>>(b);
  } else {
    if (diag) lbm_batch_kernel<float, true, 0><<<ctas, block, 0, s>>>(b);
    else lbm_batch_kernel<float, false, 0><<<ctas, block, 0, s>>>(b);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_f32(const InitArgs<float>& a, cudaStream_t s) {
  lbm_init_kernel<float><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lbmk
