// lbm_f16.cu -- instantiation of the fused step, read-out and init kernels
// with FP16 population storage and FP32 arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

template <int MODE, bool DIAG, int TYS = TY>
static void launch_one(const Args<float, __half>& a, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g, TYS), block = block_dims(TYS);
  // the all-lattices case is specialised at compile time
  if (a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT))
    lbm_step_kernel<float, MODE, DIAG, 7, __half, TYS><<<grid, block, 0, s>>>(a);
  else
    lbm_step_kernel<float, MODE, DIAG, 0, __half, TYS><<<grid, block, 0, s>>>(a);
}

template <bool DIAG>
static void launch_shape(const Args<float, __half>& a, int ty, cudaStream_t s) {
  if (ty == 4) launch_one<MODE_STEP, DIAG, 4>(a, s);
  else if (ty == 16) launch_one<MODE_STEP, DIAG, 16>(a, s);
  else launch_one<MODE_STEP, DIAG>(a, s);
}

cudaError_t launch_step_f16s(const Args<float, __half>& a, int mode, bool diag, cudaStream_t s, int ty) {
  if (mode == MODE_STEP) {
    if (diag) launch_shape<true>(a, ty, s);
    else launch_shape<false>(a, ty, s);
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


template <bool DIAG, int LATC, int NST>
static cudaError_t prepare_tile_one() {
  return cudaFuncSetAttribute(lbm_tile_kernel<__half, DIAG, LATC, NST>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tile_smem_bytes<__half>(NST));
}

template <int NST>
static cudaError_t prepare_tile_nst() {
  cudaError_t e = prepare_tile_one<false, 7, NST>();
  if (e == cudaSuccess) e = prepare_tile_one<true, 7, NST>();
  if (e == cudaSuccess) e = prepare_tile_one<false, 0, NST>();
  if (e == cudaSuccess) e = prepare_tile_one<true, 0, NST>();
  return e;
}

static cudaError_t prepare_tile1();

cudaError_t prepare_tile_f16s() {
  cudaError_t e = prepare_tile_nst<1>();
  if (e == cudaSuccess) e = prepare_tile1();
  if (e == cudaSuccess) e = prepare_tile_nst<2>();
  return e;
}

template <int NST>
static void tile_launch(const TileArgs<__half>& t, bool diag, int grid, cudaStream_t s) {
  const size_t smem = tile_smem_bytes<__half>(NST);
  const bool all = t.a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT);
  if (all) {
    if (diag) lbm_tile_kernel<__half, true, 7, NST><<<grid, block_dims(), smem, s>>>(t);
    else lbm_tile_kernel<__half, false, 7, NST><<<grid, block_dims(), smem, s>>>(t);
  } else {
    if (diag) lbm_tile_kernel<__half, true, 0, NST><<<grid, block_dims(), smem, s>>>(t);
    else lbm_tile_kernel<__half, false, 0, NST><<<grid, block_dims(), smem, s>>>(t);
  }
}

template <bool DIAG, int LATC>
static cudaError_t prepare_tile1_one() {
  cudaError_t e = cudaFuncSetAttribute(lbm_tile1_kernel<__half, DIAG, LATC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tile_smem_bytes<__half>(1));
  // all of the unified L1/shared storage as shared memory: four CTAs per SM
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lbm_tile1_kernel<__half, DIAG, LATC>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

static cudaError_t prepare_tile1() {
  cudaError_t e = prepare_tile1_one<false, 7>();
  if (e == cudaSuccess) e = prepare_tile1_one<true, 7>();
  if (e == cudaSuccess) e = prepare_tile1_one<false, 0>();
  if (e == cudaSuccess) e = prepare_tile1_one<true, 0>();
  return e;
}

// One CTA per tile, one stage: the kernel without the persistent loop.
static void tile1_launch(const TileArgs<__half>& t, bool diag, cudaStream_t s) {
  const size_t smem = tile_smem_bytes<__half>(1);
  if (t.a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT)) {
    if (diag) lbm_tile1_kernel<__half, true, 7><<<t.ntiles, block_dims(), smem, s>>>(t);
    else lbm_tile1_kernel<__half, false, 7><<<t.ntiles, block_dims(), smem, s>>>(t);
  } else {
    if (diag) lbm_tile1_kernel<__half, true, 0><<<t.ntiles, block_dims(), smem, s>>>(t);
    else lbm_tile1_kernel<__half, false, 0><<<t.ntiles, block_dims(), smem, s>>>(t);
  }
}

cudaError_t launch_tile_f16s(const TileArgs<__half>& t, bool diag, int stages, int grid, cudaStream_t s) {
  if (stages == 2) tile_launch<2>(t, diag, grid, s);
  else if (grid >= t.ntiles) tile1_launch(t, diag, s);
  else tile_launch<1>(t, diag, grid, s);
  return cudaGetLastError();
}

}  // namespace lbmk
