// lbm_static.cu -- the allocation-free entry point lbm_diagnostics_noalloc.
//
// It runs the same read-out kernel with fused diagnostics as
// lbm_compute_diagnostics, and the same one-CTA finalize kernel, on a state
// the caller already holds in device memory, with the scratch (one FP64
// partial per diagnostic per CTA) in a file-scope device array instead of
// context-owned memory.  Nothing here calls cudaMalloc, cudaFree or any
// allocating routine.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

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
// Device address of the scratch, looked up once per device (first call with
// that device current) under a lock, so that host threads making their first
// calls at the same time agree on it.  In host code g_noalloc_scratch only
// names a host-side stand-in, never the device memory itself.
std::atomic<double*> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_lock;

cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  double* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> guard(g_scratch_lock);
    p = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (!p) {
      void* q = nullptr;
      e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
      if (e != cudaSuccess) return e;
      p = (double*)q;
      g_scratch_addr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
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
