// lbm_static.cu -- the allocation-free entry point lbm_diagnostics_noalloc.
//
// It runs the same read-out kernel with fused diagnostics as
// lbm_compute_diagnostics, and the same one-CTA finalize kernel, on a state
// the caller already holds in device memory, with the scratch (one FP64
// partial per diagnostic per CTA) in a file-scope device array instead of
// context-owned memory.  Nothing here calls cudaMalloc, cudaFree or any
// allocating routine.
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_host.h"
#include "lbm_launch.h"

namespace {

// Largest grid the static scratch serves: 4096 CTAs of 32 x 8 nodes
// (1,048,576 nodes, e.g. 1024 x 1024).
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_BLOCKS;
constexpr size_t kPartials = (size_t)lbmk::NDIAG * kMaxBlocks;
// per-CTA partial sums; every launch overwrites the slots it uses, so
// nothing has to be cleared between calls
static __device__ __align__(256) double g_noalloc_scratch[kPartials];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device; in host code g_noalloc_scratch only names a host-side stand-in).
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int lbm_diagnostics_noalloc(const lbm_params* params, const void* pops,
                                       const void* lags, const void* phi0,
                                       const uint8_t* cold_mask, double* out, void* stream) {
  char err[512] = {0};
  if (!params || !pops || !lags || !phi0 || !out) return LBM_ERR_ARG;
  int st = lbmh::validate(params, err, sizeof(err));
  if (st != LBM_OK) {
    std::fprintf(stderr, "lbm_diagnostics_noalloc: %s\n", err);
    return st;
  }
  if (params->precision == LBM_FP16S || params->precision == LBM_FP64_TANGENT) {
    std::fprintf(stderr, "lbm_diagnostics_noalloc: only LBM_FP32 and LBM_FP64 states\n");
    return LBM_ERR_UNSUPPORTED;
  }
  lbmk::Geom g = lbmh::make_geom(*params);
  g.has_mask = cold_mask ? 1 : 0;
  const dim3 grid = lbmk::grid_dims(g);
  const long long nb = (long long)grid.x * grid.y;
  if (nb > kMaxBlocks) {
    std::fprintf(stderr,
                 "lbm_diagnostics_noalloc: a %d x %d grid needs %lld tiles of 32 x 8 nodes; the "
                 "static scratch holds at most %d (about 1M nodes)\n",
                 params->nx, params->ny, nb, kMaxBlocks);
    return LBM_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "lbm_diagnostics_noalloc: scratch lookup failed: %s\n",
                 cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  {
    if (params->precision == LBM_FP32) {
      lbmk::Args<float> a;
      std::memset(&a, 0, sizeof(a));
      a.g = g;
      a.c = lbmh::make_coef<float>(*params);
      a.pin = (const float*)pops;
      a.lin = (const float*)lags;
      a.phi0 = (const float*)phi0;
      a.mask = cold_mask;
      a.diag_partial = scratch;
      e = lbmk::launch_step_f32(a, lbmk::MODE_READ, true, s);
    } else {
      lbmk::Args<double> a;
      std::memset(&a, 0, sizeof(a));
      a.g = g;
      a.c = lbmh::make_coef<double>(*params);
      a.pin = (const double*)pops;
      a.lin = (const double*)lags;
      a.phi0 = (const double*)phi0;
      a.mask = cold_mask;
      a.diag_partial = scratch;
      e = lbmk::launch_step_f64(a, lbmk::MODE_READ, true, s);
    }
  }
  if (e == cudaSuccess) e = lbmk::launch_diag_finalize(scratch, (int)nb, out, 0, s);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "lbm_diagnostics_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
