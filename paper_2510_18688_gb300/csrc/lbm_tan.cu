// lbm_tan.cu -- instantiation of the step, read-out and init kernels with
// forward-mode tangent arithmetic (FP64 value and derivative, sm_103a).
#include "lbm_launch.h"

namespace lbmk {

// the lattice set is read at run time (no compile-time specialisation)
template <int MODE, bool DIAG>
static void launch_one(const Args<Dual>& a, cudaStream_t s) {
  lbm_step_kernel<Dual, MODE, DIAG, 0, Dual><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
}

cudaError_t launch_step_tan(const Args<Dual>& a, int mode, bool diag, cudaStream_t s) {
  if (mode == MODE_STEP) {
    if (diag) launch_one<MODE_STEP, true>(a, s);
    else launch_one<MODE_STEP, false>(a, s);
  } else {
    if (diag) launch_one<MODE_READ, true>(a, s);
    else launch_one<MODE_READ, false>(a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_tan(const InitArgs<Dual>& a, cudaStream_t s) {
  lbm_init_kernel<Dual, Dual><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lbmk
