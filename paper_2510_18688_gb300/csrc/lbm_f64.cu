// lbm_f64.cu -- instantiation of the fused step, read-out and init kernels
// for double arithmetic (sm_103a).
#include "lbm_launch.h"

namespace lbmk {

template <int MODE, bool DIAG, int TYS = TY>
static void launch_one(const Args<double>& a, cudaStream_t s) {
  const dim3 grid = grid_dims(a.g, TYS), block = block_dims(TYS);
  // the all-lattices case is specialised at compile time
  if (a.g.lattices == (LAT_FLOW | LAT_PHASE | LAT_HEAT))
    lbm_step_kernel<double, MODE, DIAG, 7, double, TYS><<<grid, block, 0, s>>>(a);
  else
    lbm_step_kernel<double, MODE, DIAG, 0, double, TYS><<<grid, block, 0, s>>>(a);
}

template <bool DIAG>
static void launch_shape(const Args<double>& a, int ty, cudaStream_t s) {
  if (ty == 4) launch_one<MODE_STEP, DIAG, 4>(a, s);
  else if (ty == 16) launch_one<MODE_STEP, DIAG, 16>(a, s);
  else launch_one<MODE_STEP, DIAG>(a, s);
}

cudaError_t launch_step_f64(const Args<double>& a, int mode, bool diag, cudaStream_t s, int ty) {
  if (mode == MODE_STEP) {
    if (diag) launch_shape<true>(a, ty, s);
    else launch_shape<false>(a, ty, s);
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
// linear interpolation between neighbouring nodes (NaN if none).  With the
// derivative fields dphi, dw, dfl (else null) also the derivatives of the
// two positions: (a b' - b a') / (a - b)^2 at the crossing that is kept.
static __global__ void __launch_bounds__(NT) lbm_crossings_kernel(
    const double* __restrict__ phi, const double* __restrict__ w, const double* __restrict__ fl,
    const double* __restrict__ dphi, const double* __restrict__ dw,
    const double* __restrict__ dfl, int nx, int ny, int axis, int index,
    double* __restrict__ out) {
  __shared__ double s_best[2][2][NT / 32];
  const int len = axis == 0 ? nx : ny;
  const long long stride = axis == 0 ? 1 : nx;
  const long long base = axis == 0 ? (long long)index * nx : index;
  const bool tan = dphi != nullptr;
  double best[2] = {-1.0, -1.0}, dbest[2] = {0.0, 0.0};  // coordinates are >= 0
  for (int k = threadIdx.x; k + 1 < len; k += blockDim.x) {
    const long long i0 = base + k * stride, i1 = i0 + stride;
    {
      const double a = phi[i0], b = phi[i1];
      if ((a <= 0.0) != (b <= 0.0)) {
        const double x = k + a / (a - b);
        if (x > best[0]) {
          best[0] = x;
          if (tan) dbest[0] = (a * dphi[i1] - b * dphi[i0]) / ((a - b) * (a - b));
        }
      }
    }
    {
      const double a = w[i0] * (1.0 - fl[i0]) - 0.5, b = w[i1] * (1.0 - fl[i1]) - 0.5;
      if ((a <= 0.0) != (b <= 0.0)) {
        const double x = k + a / (a - b);
        if (x > best[1]) {
          best[1] = x;
          if (tan) {
            const double da = dw[i0] * (1.0 - fl[i0]) - w[i0] * dfl[i0];
            const double db = dw[i1] * (1.0 - fl[i1]) - w[i1] * dfl[i1];
            dbest[1] = (a * db - b * da) / ((a - b) * (a - b));
          }
        }
      }
    }
  }
  // keep the larger position and its derivative (ties: the first operand)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const double x = __shfl_xor_sync(0xffffffffu, best[q], o);
      const double dx = __shfl_xor_sync(0xffffffffu, dbest[q], o);
      if (x > best[q] || (x == best[q] && dx < dbest[q])) {
        best[q] = x;
        dbest[q] = dx;
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
      s_best[q][0][warp] = best[q];
      s_best[q][1][warp] = dbest[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int q = threadIdx.x;
    double b = -1.0, db = 0.0;
    for (int v = 0; v < NT / 32; v++) {
      if (s_best[q][0][v] > b) {
        b = s_best[q][0][v];
        db = s_best[q][1][v];
      }
    }
    const double nan = __longlong_as_double(0x7ff8000000000000ULL);
    out[q] = b < 0.0 ? nan : b;
    if (tan) out[2 + q] = b < 0.0 ? nan : db;
  }
}

cudaError_t launch_crossings(const double* phi, const double* w, const double* fl,
                             const double* dphi, const double* dw, const double* dfl, int nx,
                             int ny, int axis, int index, double* out, cudaStream_t s) {
  lbm_crossings_kernel<<<1, NT, 0, s>>>(phi, w, fl, dphi, dw, dfl, nx, ny, axis, index, out);
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
