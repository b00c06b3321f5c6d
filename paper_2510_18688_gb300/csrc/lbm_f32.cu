// lbm_f32.cu -- instantiation of the fused step, read-out and init kernels
// for float arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

template <int MODE, bool DIAG, int TYS = TY>
static void launch_one(const Args<float>& a, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g, TYS), block = block_dims(TYS);
  // the all-lattices case is specialised at compile time
  if (a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT))
    lbm_step_kernel<float, MODE, DIAG, 7, float, TYS><<<grid, block, 0, s>>>(a);
  else
    lbm_step_kernel<float, MODE, DIAG, 0, float, TYS><<<grid, block, 0, s>>>(a);
}

template <bool DIAG>
static void launch_shape(const Args<float>& a, int ty, cudaStream_t s) {
  if (ty == 4) launch_one<MODE_STEP, DIAG, 4>(a, s);
  else if (ty == 16) launch_one<MODE_STEP, DIAG, 16>(a, s);
  else launch_one<MODE_STEP, DIAG>(a, s);
}

cudaError_t launch_step_f32(const Args<float>& a, int mode, bool diag, cudaStream_t s, int ty) {
  if (mode == MODE_STEP) {
    if (diag) launch_shape<true>(a, ty, s);
    else launch_shape<false>(a, ty, s);
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


template <bool DIAG, int LATC, int NST>
static cudaError_t prepare_tile_one() {
  return cudaFuncSetAttribute(lbm_tile_kernel<float, DIAG, LATC, NST>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tile_smem_bytes<float>(NST));
}

template <int NST>
static cudaError_t prepare_tile_nst() {
  cudaError_t e = prepare_tile_one<false, 7, NST>();
  if (e == cudaSuccess) e = prepare_tile_one<true, 7, NST>();
  if (e == cudaSuccess) e = prepare_tile_one<false, 0, NST>();
  if (e == cudaSuccess) e = prepare_tile_one<true, 0, NST>();
  return e;
}

template <bool DIAG, int LATC>
static cudaError_t prepare_tile_batch_one() {
  return cudaFuncSetAttribute(lbm_tile_batch_kernel<float, DIAG, LATC>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tile_smem_bytes<float>(1));
}

static cudaError_t prepare_tile1();

cudaError_t prepare_tile_f32() {
  cudaError_t e = prepare_tile_nst<1>();
  if (e == cudaSuccess) e = prepare_tile1();
  if (e == cudaSuccess) e = prepare_tile_nst<2>();
  if (e == cudaSuccess) e = prepare_tile_batch_one<false, 7>();
  if (e == cudaSuccess) e = prepare_tile_batch_one<true, 7>();
  if (e == cudaSuccess) e = prepare_tile_batch_one<false, 0>();
  if (e == cudaSuccess) e = prepare_tile_batch_one<true, 0>();
  return e;
}

template <int NST>
static void tile_launch(const TileArgs<float>& t, bool diag, int grid, cudaStream_t s) {
  const size_t smem = tile_smem_bytes<float>(NST);
  const bool all = t.a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT);
  if (all) {
    if (diag) lbm_tile_kernel<float, true, 7, NST><<<grid, block_dims(), smem, s>>>(t);
    else lbm_tile_kernel<float, false, 7, NST><<<grid, block_dims(), smem, s>>>(t);
  } else {
    if (diag) lbm_tile_kernel<float, true, 0, NST><<<grid, block_dims(), smem, s>>>(t);
    else lbm_tile_kernel<float, false, 0, NST><<<grid, block_dims(), smem, s>>>(t);
  }
}

template <bool DIAG, int LATC>
static cudaError_t prepare_tile1_one() {
  cudaError_t e = cudaFuncSetAttribute(lbm_tile1_kernel<float, DIAG, LATC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tile_smem_bytes<float>(1));
  // all of the unified L1/shared storage as shared memory: four CTAs per SM
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lbm_tile1_kernel<float, DIAG, LATC>,
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
static void tile1_launch(const TileArgs<float>& t, bool diag, cudaStream_t s) {
  const size_t smem = tile_smem_bytes<float>(1);
  if (t.a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT)) {
    if (diag) lbm_tile1_kernel<float, true, 7><<<t.ntiles, block_dims(), smem, s>>>(t);
    else lbm_tile1_kernel<float, false, 7><<<t.ntiles, block_dims(), smem, s>>>(t);
  } else {
    if (diag) lbm_tile1_kernel<float, true, 0><<<t.ntiles, block_dims(), smem, s>>>(t);
    else lbm_tile1_kernel<float, false, 0><<<t.ntiles, block_dims(), smem, s>>>(t);
  }
}

cudaError_t launch_tile_f32(const TileArgs<float>& t, bool diag, int stages, int grid, cudaStream_t s) {
  if (stages == 2) tile_launch<2>(t, diag, grid, s);
  else if (grid >= t.ntiles) tile1_launch(t, diag, s);
  else tile_launch<1>(t, diag, grid, s);
  return cudaGetLastError();
}

cudaError_t launch_tile_batch_f32(const TileBatch<float>& b, bool diag, bool all, cudaStream_t s) {
  const size_t smem = tile_smem_bytes<float>(1);
  const int ctas = b.tile_base[b.ngrids];
  if (all) {
    if (diag) lbm_tile_batch_kernel<float, true, 7><<<ctas, block_dims(), smem, s>>>(b);
    else lbm_tile_batch_kernel<float, false, 7><<<ctas, block_dims(), smem, s>>>(b);
  } else {
    if (diag) lbm_tile_batch_kernel<float, true, 0><<<ctas, block_dims(), smem, s>>>(b);
    else lbm_tile_batch_kernel<float, false, 0><<<ctas, block_dims(), smem, s>>>(b);
  }
  return cudaGetLastError();
}

}  // namespace lbmk
