// lbm_f64.cu -- instantiation of the fused step, read-out and init kernels
// for double arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

template <int MODE, bool DIAG>
static void launch_one(const Args<double>& a, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g), block = block_dims();
  // the all-lattices case is specialised at compile time
  if (a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT))
    lbm_step_kernel<double, MODE, DIAG, 7><<<grid, block, 0, s>>>(a);
  else
    lbm_step_kernel<double, MODE, DIAG, 0><<<grid, block, 0, s>>>(a);
}

cudaError_t launch_step_f64(const Args<double>& a, int mode, bool diag, cudaStream_t s) {
  if (mode == MODE_STEP) {
    if (diag) launch_one<MODE_STEP, true>(a, s);
    else launch_one<MODE_STEP, false>(a, s);
  } else {
    if (diag) launch_one<MODE_READ, true>(a, s);
    else launch_one<MODE_READ, false>(a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_f64(const SplitArgs<double>& a, bool diag, cudaStream_t s) {
  const dim3 grid = grid_dims(a.a.g), block = block_dims();
  const bool all = a.a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT);
  if (all) lbm_macro_kernel<double, 7><<<grid, block, 0, s>>>(a);
  else lbm_macro_kernel<double, 0><<<grid, block, 0, s>>>(a);
  if (all) {
    if (diag) lbm_collide_kernel<double, true, 7><<<grid, block, 0, s>>>(a);
    else lbm_collide_kernel<double, false, 7><<<grid, block, 0, s>>>(a);
  } else {
    if (diag) lbm_collide_kernel<double, true, 0><<<grid, block, 0, s>>>(a);
    else lbm_collide_kernel<double, false, 0><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_f64(const BatchTable<double>& b, bool diag, bool all, cudaStream_t s) {
  const dim3 block = block_dims();
  const int ctas = b.tile_base[b.ngrids];
  if (all) {
    if (diag) lbm_batch_kernel<double, true, 7><<<ctas, block, 0, s>>>(b);
    else lbm_batch_kernel<double, false, 7><<<ctas, block, 0, s>>>(b);
  } else {
    if (diag) lbm_batch_kernel<double, true, 0><<<ctas, block, 0, s>>>(b);
    else lbm_batch_kernel<double, false, 0><<<ctas, block, 0, s>>>(b);
  }
  return cudaGetLastError();
}

// One CTA: along one grid line of dense [ny][nx] fields, the largest
// coordinate where phi crosses 0 and where s = w (1 - fl) crosses 1/2, by
// linear interpolation between neighbouring nodes (NaN if none).
static __global__ void __launch_bounds__(NT) lbm_crossings_kernel(const double* __restrict__ phi,
                                                                  const double* __restrict__ w,
                                                                  const double* __restrict__ fl,
                                                                  int nx, int ny, int axis,
                                                                  int index,
                                                                  double* __restrict__ out) {
  __shared__ double s_best[2][NT / 32];
  const int len = axis == 0 ? nx : ny;
  const long long stride = axis == 0 ? 1 : nx;
  const long long base = axis == 0 ? (long long)index * nx : index;
  double best0 = -1.0, best1 = -1.0;  // coordinates are >= 0
  for (int k = threadIdx.x; k + 1 < len; k += blockDim.x) {
    const long long i0 = base + k * stride, i1 = i0 + stride;
    const double a = phi[i0], b = phi[i1];
    if ((a <= 0.0) != (b <= 0.0)) best0 = fmax(best0, k + a / (a - b));
    const double sa = w[i0] * (1.0 - fl[i0]) - 0.5, sb = w[i1] * (1.0 - fl[i1]) - 0.5;
    if ((sa <= 0.0) != (sb <= 0.0)) best1 = fmax(best1, k + sa / (sa - sb));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    best0 = fmax(best0, __shfl_xor_sync(0xffffffffu, best0, o));
    best1 = fmax(best1, __shfl_xor_sync(0xffffffffu, best1, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_best[0][warp] = best0;
    s_best[1][warp] = best1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double b = -1.0;
    for (int v = 0; v < NT / 32; v++) b = fmax(b, s_best[threadIdx.x][v]);
    out[threadIdx.x] = b < 0.0 ? __longlong_as_double(0x7ff8000000000000ULL) : b;
  }
}

cudaError_t launch_crossings(const double* phi, const double* w, const double* fl, int nx, int ny,
                             int axis, int index, double* out, cudaStream_t s) {
  lbm_crossings_kernel<<<1, NT, 0, s>>>(phi, w, fl, nx, ny, axis, index, out);
  return cudaGetLastError();
}

cudaError_t launch_init_f64(const InitArgs<double>& a, cudaStream_t s) {
  lbm_init_kernel<double><<<grid_dims(a.g), block_dims(), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diag_finalize(const double* partial, int nb, double* out, long long step,
                                 cudaStream_t s) {
  lbm_diag_finalize_kernel<<<1, NT, 0, s>>>(partial, nb, out, step);
  return cudaGetLastError();
}

}  // namespace lbmk
