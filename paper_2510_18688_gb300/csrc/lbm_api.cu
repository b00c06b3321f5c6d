// lbm_api.cu -- host implementation of the C ABI declared in include/lbm.h.
//
// The context owns every device buffer of one grid: two population buffers
// (27 planes each, A/B), two lag-field buffers (6 planes each), the static
// phi0 plane and the cold-mask byte plane, the diagnostic partial sums and
// result, and staging buffers for host transfers.  All work is enqueued on
// the caller's stream; nothing here computes physics on the host beyond the
// derived constants of the parameter set.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <memory>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_host.h"
#include <nvtx3/nvToolsExt.h>
#include <atomic>

#include "lbm_adjoint.cuh"
#include "lbm_adjoint_full.cuh"
#include "lbm_launch.h"

using lbmk::Args;
using lbmk::Coef;
using lbmk::Geom;
using lbmk::InitArgs;

struct lbm_ctx {
  lbm_params p;
  Geom g;
  Coef<float> cf;
  Coef<double> cd;
  Coef<lbmk::Dual> ct;   // LBM_FP64_TANGENT: constants with their derivatives
  bool tangent;          // precision LBM_FP64_TANGENT
  size_t esize;          // bytes per real of the lag fields and phi0
  size_t pop_esize;      // bytes per stored population
  void* pop[2];
  void* lag[2];
  void* phi0;
  uint8_t* mask;
  double* diag_partial;
  double* diag_out;      // NDIAG + 1
  double* staging;       // NFIELD * nx * ny doubles, for host reads (lazy)
  void* in_stage;        // 4 * nx * ny doubles + nx * ny bytes, for host inputs (lazy)
  double* h_diag;        // pinned, NDIAG + 1
  void* scratch;         // NSCRATCH planes (phi, fs, rho) of the two-kernel step
  bool split;            // step as macro + collide kernels, or fused (default)
  int nlag;              // lag planes per buffer: NLAG, plus T for float arithmetic
  // float contexts: the step as the TMA-staged tile kernel (lbm_tile.cuh)
  bool tile;
  bool tile_ok;          // the tile kernel's tensor maps exist (float contexts)
  int form;              // kernel form (form_available, set_kernel_form)
  int ty;                // tile height of the one-CTA-per-tile step (4, 8 or 16)
  int tile_stages;       // shared-memory stages of the tile kernel (1 or 2)
  int tile_grid;         // its CTAs (persistent when fewer than the tiles)
  int sms;               // multiprocessors of the context's device
  CUtensorMap tm_f[2], tm_gh[2], tm_lag[2], tm_phi0;  // per A/B buffer
  lbmk::TileMaps* d_maps;  // device copy of the maps by parity (FP32: for batches)
  unsigned* status;      // device word: a tile's copies did not arrive in time
  int cur;
  int64_t step;
  bool have_geometry;
  bool have_diag;
  bool diag_pending;     // partials written, grid-wide sum not yet taken
  int64_t diag_step;     // state index of the pending partials
  cudaStream_t last_stream;
  int nblocks;            // 32 x 8 tiles of the grid
  int diag_nb;            // per-CTA diagnostic partials written by the last diagnosed launch
  int diag_cap;           // partials the array holds (the most any tile shape writes)
  // captured steps: one period of the step sequence, replayed whole
  bool graphs;           // replay captured periods (default; LBM_STEP_GRAPHS=0 disables)
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;
  int graph_cur;         // buffer parity the graph starts from
  int64_t graph_phase;   // step index modulo the period it starts from
  uint64_t gen;          // bumped when geometry or state is replaced
  uint64_t graph_gen;
  int graph_min;         // shortest captured period (32; lbm_autotune may change it)
  int graph_len;         // steps in the captured graph
  char err[512];
};

namespace {

const uint32_t kMagic = 0x4c424d46u;  // "LBMF"
constexpr int kForms = 6;              // kernel form ids (form_available)
constexpr int kAutotuneVariants = 2 * kForms;  // kernel forms x 2 captured periods
const uint32_t kVersion = 2u;  // 2: float states keep g0, h0 relative to references

struct StateHeader {
  uint32_t magic, version;
  int32_t nx, ny, precision, lattices;
  int64_t step;
};

// Testing hook for the failure paths of lbm_create: when armed with n >= 0,
// the (n + 1)-th device or pinned allocation made by lbm_create fails as if
// the device were out of memory (then the hook disarms itself).
std::atomic<int> g_alloc_countdown{-1};

// Testing hook for the bounded waits of the tile kernel: while armed, every
// tile kernel launched expects 16 bytes more than its copies deliver, so its
// first wait runs out (no copy is left in flight).
std::atomic<int> g_tile_timeout{0};

bool injected_alloc_failure() {
  int n = g_alloc_countdown.load();
  while (n >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(n, n - 1)) return n == 0;
  }
  return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc(void** p, size_t bytes) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, 0);
}

// NVTX range for the duration of a scope (a no-op unless a tool listens)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(lbm_ctx* c, int code, const char* fmt, const char* detail = "") {
  if (c) std::snprintf(c->err, sizeof(c->err), fmt, detail);
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not offer it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// A 3-D tiled map over `planes` planes of a grid in the library's layout
// (x fastest, rows of pitch elements, planes of `plane` elements); cells
// outside nx x ny read as zero.
bool encode_map(CUtensorMap* m, CUtensorMapDataType dt, size_t esize, void* base,
                const lbmk::Geom& g, int planes, unsigned bx, unsigned by, unsigned bz) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * esize, (cuuint64_t)g.plane * esize};
  const cuuint32_t box[3] = {bx, by, bz};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor maps of a float context's tile kernel (both A/B buffers).
template <typename S>
bool make_tile_maps(lbm_ctx* c, CUtensorMapDataType dt) {
  using St = lbmk::TileStage<S>;
  bool ok = true;
  for (int b = 0; b < 2; b++) {
    ok = ok && encode_map(&c->tm_f[b], dt, sizeof(S), c->pop[b], c->g, 27, lbmk::TX, lbmk::TY, 9);
    ok = ok && encode_map(&c->tm_gh[b], dt, sizeof(S), c->pop[b], c->g, 27, St::WG, lbmk::TY + 2, 18);
    ok = ok && encode_map(&c->tm_lag[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), c->lag[b],
                          c->g, lbmk::NLAG + 1, St::WL, lbmk::TY + 2, lbmk::NLAG + 1);
  }
  ok = ok && encode_map(&c->tm_phi0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), c->phi0, c->g,
                        1, St::WL, lbmk::TY + 2, 1);
  return ok;
}

template <typename S>
lbmk::TileArgs<S> tile_args(lbm_ctx* c, const lbmk::Args<float, S>& a) {
  lbmk::TileArgs<S> t;
  std::memset(&t, 0, sizeof(t));
  t.a = a;
  t.map_f = c->tm_f[c->cur];
  t.map_gh = c->tm_gh[c->cur];
  t.map_lag = c->tm_lag[c->cur];
  t.map_phi0 = c->tm_phi0;
  t.tiles_x = (c->g.nx + lbmk::TX - 1) / lbmk::TX;
  t.ntiles = c->nblocks;
  t.status = c->status;
  t.extra_tx = g_tile_timeout.load() ? 16u : 0u;
  return t;
}

// Tile kernel configuration: `stages` shared-memory stages and `per_sm`
// persistent CTAs per multiprocessor (0: one CTA per tile).
void set_tile_config(lbm_ctx* c, int stages, int per_sm) {
  c->tile_stages = stages;
  c->tile_grid = per_sm > 0 ? std::max(1, std::min(c->nblocks, per_sm * c->sms)) : c->nblocks;
}

// Kernel forms of the step (lbm_autotune): 0 one CTA per 32 x 8 tile;
// 1 float: TMA-staged, one stage, one CTA per tile / FP64: the two-kernel
// split; 2 TMA-staged, two stages, two persistent CTAs per SM (float);
// 3 TMA-staged, one stage, three persistent CTAs per SM (float); 4 one CTA
// per 32 x 4 tile; 5 one CTA per 32 x 16 tile.  Tangent contexts: 0.
bool form_available(const lbm_ctx* c, int form) {
  if (form < 0 || form >= kForms) return false;
  if (c->tangent) return form == 0;
  if (form == 0 || form >= 4) return true;
  if (c->p.precision == LBM_FP64) return form == 1;
  return c->tile_ok;
}

// Tiles (CTAs, partials) of a one-CTA-per-tile launch with tiles of height ty.
int tiles_of(const lbm_ctx* c, int ty) {
  return ((c->g.nx + lbmk::TX - 1) / lbmk::TX) * lbmk::tiles_y(c->g.ny, ty);
}

void set_kernel_form(lbm_ctx* c, int form) {
  c->form = form;
  c->ty = form == 4 ? 4 : (form == 5 ? 16 : lbmk::TY);
  if (c->p.precision == LBM_FP64 && !c->tangent) {
    c->split = form == 1;
    return;
  }
  c->split = false;
  c->tile = c->tile_ok && form >= 1 && form <= 3;
  if (form == 1) set_tile_config(c, 1, 0);
  else if (form == 2) set_tile_config(c, 2, 2);
  else if (form == 3) set_tile_config(c, 1, 3);
}

// A tile kernel whose copies did not arrive within its bounded wait sets
// c->status; the next synchronising read reports it (once).
int check_timeout(lbm_ctx* c, cudaStream_t s) {
  if (!c->status) return LBM_OK;
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, c->status, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "status download");
  if (v) {
    cudaMemsetAsync(c->status, 0, sizeof(unsigned), s);
    return fail(c, LBM_ERR_TIMEOUT,
                "a step's tile copies did not arrive in time; the state is undefined%s");
  }
  return LBM_OK;
}

template <typename R, typename S = R>
Args<R, S> step_args(lbm_ctx* c, const Coef<R>& coef) {
  Args<R, S> a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.c = coef;
  a.pin = (const S*)c->pop[c->cur];
  a.pout = (S*)c->pop[c->cur ^ 1];
  a.lin = (const R*)c->lag[c->cur];
  a.lout = (R*)c->lag[c->cur ^ 1];
  a.phi0 = (const R*)c->phi0;
  a.mask = c->mask;
  a.diag_partial = c->diag_partial;
  return a;
}

cudaError_t launch(lbm_ctx* c, int mode, bool diag, double* const* outs, cudaStream_t s) {
  // the step launches one CTA per 32 x ty tile (other forms and the
  // read-out: per 32 x 8 tile), each writing one set of diagnostic partials
  const bool shaped = mode == lbmk::MODE_STEP && !c->split && !c->tile;
  const int ty = shaped ? c->ty : lbmk::TY;
  if (diag) c->diag_nb = tiles_of(c, ty);
  if (mode == lbmk::MODE_STEP && c->split) {  // FP64 only
    lbmk::SplitArgs<double> a;
    a.a = step_args<double>(c, c->cd);
    a.sc = (double*)c->scratch;
    return lbmk::launch_split_f64(a, diag, s);
  }
  if (c->p.precision == LBM_FP32) {
    Args<float> a = step_args<float>(c, c->cf);
    if (mode == lbmk::MODE_STEP && c->tile)
      return lbmk::launch_tile_f32(tile_args<float>(c, a), diag, c->tile_stages, c->tile_grid, s);
    if (outs)
      for (int k = 0; k < lbmk::NFIELD; k++) a.out[k] = outs[k];
    return lbmk::launch_step_f32(a, mode, diag, s, ty);
  }
  if (c->tangent) {
    Args<lbmk::Dual> a = step_args<lbmk::Dual>(c, c->ct);
    if (outs)
      for (int k = 0; k < lbmk::NFIELD; k++) a.out[k] = outs[k];
    return lbmk::launch_step_tan(a, mode, diag, s);
  }
  if (c->p.precision == LBM_FP16S) {
    Args<float, __half> a = step_args<float, __half>(c, c->cf);
    if (mode == lbmk::MODE_STEP && c->tile)
      return lbmk::launch_tile_f16s(tile_args<__half>(c, a), diag, c->tile_stages, c->tile_grid,
                                    s);
    if (outs)
      for (int k = 0; k < lbmk::NFIELD; k++) a.out[k] = outs[k];
    return lbmk::launch_step_f16s(a, mode, diag, s, ty);
  }
  Args<double> a = step_args<double>(c, c->cd);
  if (outs)
    for (int k = 0; k < lbmk::NFIELD; k++) a.out[k] = outs[k];
  return lbmk::launch_step_f64(a, mode, diag, s, ty);
}

// Steps of one captured period: the buffer parity repeats every two steps
// and the diagnostic schedule every diag_every steps; short periods are
// repeated up to at least 32 steps so that one graph launch covers many
// kernels.
int graph_period(int diag_every, int min_steps = 32) {
  const int base = diag_every <= 0 ? 2 : (diag_every % 2 == 0 ? diag_every : 2 * diag_every);
  return base >= min_steps ? base : base * ((min_steps + base - 1) / base);
}
constexpr int kMaxGraphSteps = 256;

// True when `s` is not being captured by the caller (a captured replay
// inside a caller's capture is left to plain launches).
bool stream_free(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}

// Records, after a span of steps [first, end) with diagnostics every d > 0
// steps, that the last diagnosed state is pending.
void note_diag_span(lbm_ctx* c, int64_t first, int64_t end) {
  const int64_t d = c->p.diag_every;
  if (d <= 0 || end <= first) return;
  const int64_t last = (end - 1) - ((end - 1) % d);
  if (last < first) return;
  c->have_diag = true;
  c->diag_pending = true;
  c->diag_step = last;
}

cudaError_t step_launches(lbm_ctx* c, int64_t nsteps, cudaStream_t s) {
  for (int64_t k = 0; k < nsteps; k++) {
    const bool diag = c->p.diag_every > 0 && (c->step % c->p.diag_every) == 0;
    cudaError_t e = launch(c, lbmk::MODE_STEP, diag, nullptr, s);
    if (e != cudaSuccess) return e;
    note_diag_span(c, c->step, c->step + 1);
    c->cur ^= 1;
    c->step++;
  }
  return cudaSuccess;
}

// The captured period that starts from the context's current parity and
// phase, captured on a private stream the first time it is needed.
cudaError_t step_graph(lbm_ctx* c, int period, cudaGraphExec_t* out) {
  const int64_t phase = c->step % period;
  if (c->graph && c->graph_cur == c->cur && c->graph_phase == phase && c->graph_gen == c->gen &&
      c->graph_len == period) {
    *out = c->graph;
    return cudaSuccess;
  }
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  const int cur = c->cur;
  const int64_t step = c->step, diag_step = c->diag_step;
  const bool have_diag = c->have_diag, pending = c->diag_pending;
  e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = step_launches(c, period, c->cap_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->cap_stream, &g);
  // capture enqueues nothing: the host-side state goes back to the start
  c->cur = cur;
  c->step = step;
  c->diag_step = diag_step;
  c->have_diag = have_diag;
  c->diag_pending = pending;
  if (el != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return el != cudaSuccess ? el : e;
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return e;
  }
  c->graph_cur = cur;
  c->graph_phase = phase;
  c->graph_gen = c->gen;
  c->graph_len = period;
  *out = c->graph;
  return cudaSuccess;
}

void free_all(lbm_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* dev[] = {c->pop[0], c->pop[1], c->lag[0],     c->lag[1],    c->phi0,   c->mask,
                 c->diag_partial, c->diag_out, c->staging, c->in_stage,
                 c->scratch, c->status, c->d_maps};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (c->h_diag) cudaFreeHost(c->h_diag);
}

}  // namespace

extern "C" {

const char* lbm_status_string(int status) {
  switch (status) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_PARAM: return "invalid physical parameter";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_NONFINITE: return "non-finite state";
    case LBM_ERR_UNSUPPORTED: return "unsupported";
    case LBM_ERR_STATE: return "call out of order";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : "null context"; }

#ifndef LBM_SOURCE_HASH
#define LBM_SOURCE_HASH "unknown"
#endif
const char* lbm_source_hash(void) { return LBM_SOURCE_HASH; }

int64_t lbm_step_count(const lbm_ctx* c) { return c ? c->step : -1; }

int lbm_create(const lbm_params* params, lbm_ctx** out) {
  if (!params || !out) return LBM_ERR_ARG;
  *out = nullptr;
  char err[512] = {0};
  int st = lbmh::validate(params, err, sizeof(err));
  if (st != LBM_OK) {
    std::fprintf(stderr, "lbm_create: %s\n", err);
    return st;
  }
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  std::memset(c, 0, sizeof(*c));
  c->p = *params;
  c->tangent = params->precision == LBM_FP64_TANGENT;
  c->esize = c->tangent ? sizeof(lbmk::Dual)
                        : (params->precision == LBM_FP64 ? sizeof(double) : sizeof(float));
  c->pop_esize = params->precision == LBM_FP16S ? sizeof(__half) : c->esize;
  c->nlag = (params->precision == LBM_FP32 || params->precision == LBM_FP16S) ? lbmk::NLAG + 1
                                                                              : lbmk::NLAG;
  c->g = lbmh::make_geom(*params);
  {
    // LBM_STEP_KERNEL=split selects the two-kernel step (macro pass +
    // collide pass); the default is the fused one-kernel step
    const char* k = std::getenv("LBM_STEP_KERNEL");
    c->split = k && std::strcmp(k, "split") == 0 && params->precision == LBM_FP64;
    // LBM_STEP_GRAPHS=0 launches every step on its own instead of
    // replaying captured periods
    const char* gr = std::getenv("LBM_STEP_GRAPHS");
    c->graphs = !(gr && std::strcmp(gr, "0") == 0);
    c->graph_min = 32;
  }
  c->cf = lbmh::make_coef<float>(*params);
  c->cd = lbmh::make_coef<double>(*params);
  if (c->tangent) c->ct = lbmh::make_coef_tangent(*params);
  const size_t dmul = c->tangent ? 2 : 1;  // tangent: values, then derivatives
  const dim3 gd = lbmk::grid_dims(c->g);
  c->nblocks = (int)(gd.x * gd.y);
  c->ty = lbmk::TY;
  c->diag_nb = c->nblocks;
  c->diag_cap = std::max(c->nblocks, tiles_of(c, 4));  // 32 x 4 tiles write the most
  const size_t P = (size_t)c->g.plane;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; b++) {
    e = dev_malloc(&c->pop[b], 27 * P * c->pop_esize);
    if (e == cudaSuccess) e = dev_malloc(&c->lag[b], c->nlag * P * c->esize);
  }
  if (e == cudaSuccess) e = dev_malloc(&c->phi0, P * c->esize);
  if (e == cudaSuccess) e = dev_malloc(&c->scratch, lbmk::NSCRATCH * P * c->esize);
  if (e == cudaSuccess) e = dev_malloc((void**)&c->mask, P);
  if (e == cudaSuccess)
    e = dev_malloc((void**)&c->diag_partial, dmul * lbmk::NDIAG * c->diag_cap * sizeof(double));
  if (e == cudaSuccess) e = dev_malloc((void**)&c->diag_out, dmul * (lbmk::NDIAG + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->mask, 0, P);
  if (e == cudaSuccess) e = dev_malloc((void**)&c->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(unsigned));
  if (e == cudaSuccess && (params->precision == LBM_FP32 || params->precision == LBM_FP16S)) {
    // the TMA-staged tile kernel needs its tensor maps and shared-memory sizes
    const bool maps = params->precision == LBM_FP32
                          ? make_tile_maps<float>(c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32)
                          : make_tile_maps<__half>(c, CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->sms = std::max(1, sms);
    if (e == cudaSuccess && maps)
      e = params->precision == LBM_FP32 ? lbmk::prepare_tile_f32() : lbmk::prepare_tile_f16s();
    c->tile_ok = e == cudaSuccess && maps;
    if (c->tile_ok && params->precision == LBM_FP32) {
      // the maps by parity in device memory, for the batched tile kernel
      lbmk::TileMaps hm[2];
      for (int b = 0; b < 2; b++) {
        hm[b].f = c->tm_f[b];
        hm[b].gh = c->tm_gh[b];
        hm[b].lag = c->tm_lag[b];
        hm[b].phi0 = c->tm_phi0;
      }
      e = dev_malloc((void**)&c->d_maps, sizeof(hm));
      if (e == cudaSuccess) e = cudaMemcpy(c->d_maps, hm, sizeof(hm), cudaMemcpyHostToDevice);
    }
    // Default kernel form (lbm_autotune measures them all): one CTA per
    // tile from global loads on grids of fewer than eight tiles per
    // multiprocessor, where every tile's loads and compute overlap with
    // the other resident CTAs'; the TMA-staged form with one CTA per tile on
    // larger grids.  LBM_STEP_KERNEL=fused forces the first,
    // LBM_TILE=<stages>:<CTAs per SM> (0: one CTA per tile) a tile kernel.
    int form = (c->tile_ok && c->nblocks >= 8 * c->sms) ? 1 : 0;
    if (const char* v = std::getenv("LBM_TILE")) {
      int a = 0, b = 0;
      if (c->tile_ok && std::sscanf(v, "%d:%d", &a, &b) == 2 && (a == 1 || a == 2) && b >= 0 &&
          b <= 4) {
        set_kernel_form(c, 1);
        set_tile_config(c, a, b);
        form = -1;
      }
    }
    if (const char* k = std::getenv("LBM_STEP_KERNEL"))
      if (std::strcmp(k, "fused") == 0) form = 0;
    if (form >= 0) set_kernel_form(c, form);
  }
  // LBM_KERNEL_FORM=<form id> forces one kernel form where the context has it
  if (const char* f = std::getenv("LBM_KERNEL_FORM")) {
    char* end = nullptr;
    const long v = std::strtol(f, &end, 10);
    if (end != f && form_available(c, (int)v)) set_kernel_form(c, (int)v);
  }
  if (e == cudaSuccess)
    e = host_alloc((void**)&c->h_diag, dmul * (lbmk::NDIAG + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    int code = cuda_fail(c, e, "lbm_create allocation");
    std::fprintf(stderr, "lbm_create: %s\n", c->err);
    free_all(c);
    delete c;
    return code;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  free_all(c);
  delete c;
}

int lbm_set_geometry(lbm_ctx* c, const double* phi0, const uint8_t* cold_mask,
                     const double* phi, const double* T, const double* fl, int where,
                     void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!phi0 || !phi || !T || !fl) return fail(c, LBM_ERR_ARG, "null input array%s");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(c, LBM_ERR_ARG, "bad `where`%s");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)c->g.nx * c->g.ny;
  const double* d_phi0 = phi0;
  const double* d_phi = phi;
  const double* d_T = T;
  const double* d_fl = fl;
  const uint8_t* d_mask = cold_mask;
  cudaError_t e;
  if (where == LBM_HOST) {
    if (!c->in_stage) {
      e = cudaMalloc(&c->in_stage, 4 * N * sizeof(double) + N);
      if (e != cudaSuccess) return cuda_fail(c, e, "input staging allocation");
    }
    double* base = (double*)c->in_stage;
    const double* src[4] = {phi0, phi, T, fl};
    for (int k = 0; k < 4; k++) {
      e = cudaMemcpyAsync(base + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "input upload");
    }
    d_phi0 = base;
    d_phi = base + N;
    d_T = base + 2 * N;
    d_fl = base + 3 * N;
    if (cold_mask) {
      uint8_t* mb = (uint8_t*)(base + 4 * N);
      e = cudaMemcpyAsync(mb, cold_mask, N, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "mask upload");
      d_mask = mb;
    }
  }
  c->g.has_mask = cold_mask ? 1 : 0;
  c->cur = 0;
  if (c->p.precision == LBM_FP32) {
    InitArgs<float> a;
    std::memset(&a, 0, sizeof(a));
    a.g = c->g; a.c = c->cf;
    a.pout = (float*)c->pop[0]; a.lout = (float*)c->lag[0]; a.phi0_out = (float*)c->phi0;
    a.mask_out = c->mask; a.phi0 = d_phi0; a.mask = d_mask; a.phi = d_phi; a.T = d_T; a.fl = d_fl;
    e = lbmk::launch_init_f32(a, s);
  } else if (c->tangent) {
    InitArgs<lbmk::Dual> a;
    std::memset(&a, 0, sizeof(a));
    a.g = c->g; a.c = c->ct;
    a.pout = (lbmk::Dual*)c->pop[0]; a.lout = (lbmk::Dual*)c->lag[0];
    a.phi0_out = (lbmk::Dual*)c->phi0;
    a.mask_out = c->mask; a.phi0 = d_phi0; a.mask = d_mask; a.phi = d_phi; a.T = d_T; a.fl = d_fl;
    e = lbmk::launch_init_tan(a, s);
  } else if (c->p.precision == LBM_FP16S) {
    InitArgs<float, __half> a;
    std::memset(&a, 0, sizeof(a));
    a.g = c->g; a.c = c->cf;
    a.pout = (__half*)c->pop[0]; a.lout = (float*)c->lag[0]; a.phi0_out = (float*)c->phi0;
    a.mask_out = c->mask; a.phi0 = d_phi0; a.mask = d_mask; a.phi = d_phi; a.T = d_T; a.fl = d_fl;
    e = lbmk::launch_init_f16s(a, s);
  } else {
    InitArgs<double> a;
    std::memset(&a, 0, sizeof(a));
    a.g = c->g; a.c = c->cd;
    a.pout = (double*)c->pop[0]; a.lout = (double*)c->lag[0]; a.phi0_out = (double*)c->phi0;
    a.mask_out = c->mask; a.phi0 = d_phi0; a.mask = d_mask; a.phi = d_phi; a.T = d_T; a.fl = d_fl;
    e = lbmk::launch_init_f64(a, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel launch");
  if (where == LBM_HOST) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_geometry synchronisation");
  }
  c->step = 0;
  c->gen++;  // captured steps of the old geometry are stale
  c->have_geometry = true;
  c->have_diag = false;
  c->diag_pending = false;
  c->last_stream = s;
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t nsteps, void* stream) {
  Range nvtx_range("lbm_step");
  if (!c) return LBM_ERR_ARG;
  if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps must be >= 0%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_set_geometry%s");
  cudaStream_t s = (cudaStream_t)stream;
  int64_t left = nsteps;
  const int period = graph_period(c->p.diag_every, c->graph_min);
  if (c->graphs && period <= kMaxGraphSteps && left >= period && stream_free(s)) {
    // whole periods replay one captured graph (same kernels, same order)
    cudaGraphExec_t g = nullptr;
    cudaError_t e = step_graph(c, period, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "step graph capture");
    const int64_t reps = left / period;
    for (int64_t r = 0; r < reps; r++) {
      e = cudaGraphLaunch(g, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "step graph launch");
    }
    note_diag_span(c, c->step, c->step + reps * period);
    c->step += reps * period;  // the period is even: the parity is unchanged
    left -= reps * period;
  }
  cudaError_t e = step_launches(c, left, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  c->last_stream = s;
  return LBM_OK;
}

}  // extern "C"

namespace {

// Field read-out; `deriv` selects the derivative half of a tangent context.
// Tangent read-outs write value and derivative (2 N doubles per field) and
// always go through the staging memory.
int read_fields_impl(lbm_ctx* c, uint32_t field_mask, double* const* out, int where,
                     cudaStream_t s, bool deriv) {
  if (!out) return fail(c, LBM_ERR_ARG, "null output table%s");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(c, LBM_ERR_ARG, "bad `where`%s");
  if (field_mask >> lbmk::NFIELD) return fail(c, LBM_ERR_ARG, "unknown field bits%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "read before lbm_set_geometry%s");
  for (int k = 0; k < lbmk::NFIELD; k++)
    if ((field_mask >> k & 1u) && !out[k]) return fail(c, LBM_ERR_ARG, "selected field has null output%s");
  const size_t N = (size_t)c->g.nx * c->g.ny;
  const size_t fstride = c->tangent ? 2 * N : N;
  const bool staged = where == LBM_HOST || c->tangent;
  double* outs[lbmk::NFIELD] = {nullptr};
  cudaError_t e;
  if (staged) {
    if (!c->staging) {
      e = cudaMalloc(&c->staging, lbmk::NFIELD * fstride * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(c, e, "read-out staging allocation");
    }
    for (int k = 0; k < lbmk::NFIELD; k++)
      if (field_mask >> k & 1u) outs[k] = c->staging + k * fstride;
  } else {
    for (int k = 0; k < lbmk::NFIELD; k++)
      if (field_mask >> k & 1u) outs[k] = out[k];
  }
  e = launch(c, lbmk::MODE_READ, false, outs, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "read-out kernel launch");
  if (staged) {
    const cudaMemcpyKind kind = where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int k = 0; k < lbmk::NFIELD; k++) {
      if (!(field_mask >> k & 1u)) continue;
      e = cudaMemcpyAsync(out[k], outs[k] + (deriv ? N : 0), N * sizeof(double), kind, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "field download");
    }
    if (where == LBM_HOST) {
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(c, e, "read_fields synchronisation");
    }
  }
  c->last_stream = s;
  return LBM_OK;
}

int read_crossings_impl(lbm_ctx* c, int axis, int index, double* out, cudaStream_t s, bool deriv) {
  if (!out) return fail(c, LBM_ERR_ARG, "null output%s");
  if (axis != 0 && axis != 1) return fail(c, LBM_ERR_ARG, "axis must be 0 (x) or 1 (y)%s");
  if (index < 0 || index >= (axis == 0 ? c->g.ny : c->g.nx))
    return fail(c, LBM_ERR_ARG, "line index outside the grid%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "read before lbm_set_geometry%s");
  const size_t N = (size_t)c->g.nx * c->g.ny;
  const size_t fstride = c->tangent ? 2 * N : N;
  cudaError_t e;
  if (!c->staging) {
    e = cudaMalloc(&c->staging, lbmk::NFIELD * fstride * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e, "read-out staging allocation");
  }
  double* outs[lbmk::NFIELD] = {nullptr};
  outs[lbmk::F_PHI] = c->staging + lbmk::F_PHI * fstride;
  outs[lbmk::F_W] = c->staging + lbmk::F_W * fstride;
  outs[lbmk::F_FL] = c->staging + lbmk::F_FL * fstride;
  double* d_out = c->staging + lbmk::F_T * fstride;  // an unused staging plane
  e = launch(c, lbmk::MODE_READ, false, outs, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "read-out kernel launch");
  const double* dphi = deriv ? outs[lbmk::F_PHI] + N : nullptr;
  const double* dw = deriv ? outs[lbmk::F_W] + N : nullptr;
  const double* dfl = deriv ? outs[lbmk::F_FL] + N : nullptr;
  e = lbmk::launch_crossings(outs[lbmk::F_PHI], outs[lbmk::F_W], outs[lbmk::F_FL], dphi, dw, dfl,
                             c->g.nx, c->g.ny, axis, index, d_out, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "crossings kernel launch");
  e = cudaMemcpyAsync(out, d_out, (deriv ? 4 : 2) * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "crossings download");
  c->last_stream = s;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_read_fields(lbm_ctx* c, uint32_t field_mask, double* const* out, int where,
                    void* stream) {
  if (!c) return LBM_ERR_ARG;
  const int st = read_fields_impl(c, field_mask, out, where, (cudaStream_t)stream, false);
  if (st != LBM_OK) return st;
  return check_timeout(c, (cudaStream_t)stream);
}

int lbm_read_tangent_fields(lbm_ctx* c, uint32_t field_mask, double* const* out, int where,
                            void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!c->tangent) return fail(c, LBM_ERR_UNSUPPORTED, "not a tangent context%s");
  return read_fields_impl(c, field_mask, out, where, (cudaStream_t)stream, true);
}

int lbm_read_crossings(lbm_ctx* c, int axis, int index, double* out, void* stream) {
  if (!c) return LBM_ERR_ARG;
  return read_crossings_impl(c, axis, index, out, (cudaStream_t)stream, false);
}

int lbm_read_crossings_tangent(lbm_ctx* c, int axis, int index, double* out, void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!c->tangent) return fail(c, LBM_ERR_UNSUPPORTED, "not a tangent context%s");
  return read_crossings_impl(c, axis, index, out, (cudaStream_t)stream, true);
}

int lbm_compute_diagnostics(lbm_ctx* c, void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "diagnostics before lbm_set_geometry%s");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch(c, lbmk::MODE_READ, true, nullptr, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics kernel launch");
  c->have_diag = true;
  c->diag_pending = true;
  c->diag_step = c->step;
  c->last_stream = s;
  return LBM_OK;
}

int lbm_read_diagnostics(lbm_ctx* c, lbm_diag* out) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->have_diag) return fail(c, LBM_ERR_STATE, "no diagnostics computed yet%s");
  cudaError_t e = cudaSuccess;
  if (c->diag_pending) {
    e = lbmk::launch_diag_finalize(c->diag_partial, c->diag_nb, c->diag_out, c->diag_step,
                                   c->last_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics finalize launch");
    c->diag_pending = false;
  }
  e = cudaMemcpyAsync(c->h_diag, c->diag_out, (lbmk::NDIAG + 1) * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics download");
  const int st = check_timeout(c, c->last_stream);
  if (st != LBM_OK) return st;
  const double* d = c->h_diag;
  out->mass = d[0];
  out->material_mass = d[1];
  out->rhoH = d[2];
  out->liquid_volume = d[3];
  out->material_volume = d[4];
  out->frozen_volume = d[5];
  out->phi_sum = d[6];
  out->kinetic = d[7];
  out->nonfinite = d[8];
  out->step = (int64_t)d[9];
  if (d[8] != 0.0) return fail(c, LBM_ERR_NONFINITE, "non-finite populations in the state%s");
  return LBM_OK;
}

int lbm_read_tangent_diagnostics(lbm_ctx* c, lbm_diag* out) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->tangent) return fail(c, LBM_ERR_UNSUPPORTED, "not a tangent context%s");
  if (!c->have_diag) return fail(c, LBM_ERR_STATE, "no diagnostics computed yet%s");
  // the derivative partials follow the value partials
  double* dout = c->diag_out + (lbmk::NDIAG + 1);
  double* hd = c->h_diag + (lbmk::NDIAG + 1);
  cudaError_t e = lbmk::launch_diag_finalize(c->diag_partial + (size_t)lbmk::NDIAG * c->diag_nb,
                                             c->diag_nb, dout, c->diag_step, c->last_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hd, dout, (lbmk::NDIAG + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                        c->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "tangent diagnostics");
  out->mass = hd[0];
  out->material_mass = hd[1];
  out->rhoH = hd[2];
  out->liquid_volume = hd[3];
  out->material_volume = hd[4];
  out->frozen_volume = hd[5];
  out->phi_sum = hd[6];
  out->kinetic = hd[7];
  out->nonfinite = 0.0;
  out->step = (int64_t)hd[9];
  return LBM_OK;
}

int lbm_state_size(const lbm_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LBM_ERR_ARG;
  *bytes = sizeof(StateHeader) + (27 * c->pop_esize + c->nlag * c->esize) * (size_t)c->g.plane;
  return LBM_OK;
}

int lbm_save_state(lbm_ctx* c, void* host_buf, size_t capacity, void* stream) {
  if (!c || !host_buf) return LBM_ERR_ARG;
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "save before lbm_set_geometry%s");
  size_t need;
  lbm_state_size(c, &need);
  if (capacity < need) return fail(c, LBM_ERR_ARG, "state buffer too small%s");
  cudaStream_t s = (cudaStream_t)stream;
  StateHeader h = {kMagic, kVersion, c->g.nx, c->g.ny, c->p.precision, (int32_t)c->p.lattices,
                   c->step};
  std::memcpy(host_buf, &h, sizeof(h));
  char* dst = (char*)host_buf + sizeof(h);
  const size_t pb = 27 * (size_t)c->g.plane * c->pop_esize;
  cudaError_t e = cudaMemcpyAsync(dst, c->pop[c->cur], pb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + pb, c->lag[c->cur], c->nlag * (size_t)c->g.plane * c->esize,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "state download");
  return LBM_OK;
}

int lbm_load_state(lbm_ctx* c, const void* host_buf, size_t size, void* stream) {
  if (!c || !host_buf) return LBM_ERR_ARG;
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "load before lbm_set_geometry%s");
  size_t need;
  lbm_state_size(c, &need);
  if (size < need) return fail(c, LBM_ERR_ARG, "state buffer too small%s");
  StateHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (h.magic != kMagic || h.version != kVersion || h.nx != c->g.nx || h.ny != c->g.ny ||
      h.precision != c->p.precision || h.lattices != (int32_t)c->p.lattices)
    return fail(c, LBM_ERR_ARG, "state does not match this context%s");
  cudaStream_t s = (cudaStream_t)stream;
  const char* src = (const char*)host_buf + sizeof(h);
  const size_t pb = 27 * (size_t)c->g.plane * c->pop_esize;
  cudaError_t e = cudaMemcpyAsync(c->pop[c->cur], src, pb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->lag[c->cur], src + pb, c->nlag * (size_t)c->g.plane * c->esize,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "state upload");
  c->step = h.step;
  c->gen++;  // captured steps start from another parity or phase
  c->have_diag = false;
  c->diag_pending = false;
  c->last_stream = s;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// reverse mode: frozen fraction of an enthalpy-lattice run and its gradient
// ---------------------------------------------------------------------------

extern "C" void lbm_debug_fail_allocation(int after) {
  g_alloc_countdown.store(after < 0 ? -1 : after);
}

void lbm_debug_tile_timeout(int on) { g_tile_timeout.store(on ? 1 : 0); }

extern "C" int lbm_adjoint_frozen_fraction(lbm_ctx* c, int64_t nsteps, int every, double* ff_out,
                                           double* grad, void* stream) {
  Range nvtx_range("lbm_adjoint_frozen_fraction");
  if (!c) return LBM_ERR_ARG;
  if (!ff_out || !grad) return fail(c, LBM_ERR_ARG, "null output%s");
  if (nsteps < 1 || every < 1) return fail(c, LBM_ERR_ARG, "nsteps and the checkpoint interval must be >= 1%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "adjoint before lbm_set_geometry%s");
  // the enthalpy lattice alone, or with a flow lattice that stays exactly at
  // rest (no mass source: rho_s = rho_l; no body force)
  const bool resting_flow = c->p.lattices == (LBM_LAT_FLOW | LBM_LAT_HEAT) &&
                            c->p.rho_s == c->p.rho_l && c->p.gx == 0.0 && c->p.gy == 0.0;
  if (c->p.precision != LBM_FP64 || !(c->p.lattices == LBM_LAT_HEAT || resting_flow))
    return fail(c, LBM_ERR_UNSUPPORTED,
                "the adjoint covers FP64 contexts with the enthalpy lattice (alone, or with a flow "
                "lattice that stays at rest: rho_s = rho_l, no body force)%s");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)c->g.plane;
  const size_t hN = 9 * P, lN = lbmk::NLAG * P, stN = hN + lN;  // doubles per stored state
  const int64_t nck = (nsteps + every - 1) / every;
  const int64_t seglen = std::min<int64_t>(every, nsteps);
  double *ck = nullptr, *seg = nullptr, *lam = nullptr, *acc = nullptr, *dout = nullptr, *fin = nullptr;
  cudaError_t e = cudaMalloc(&ck, nck * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&seg, seglen * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&lam, 2 * (9 + 2) * P * sizeof(double));
  // accumulators: T_wall[0..3], L, T_cold, padded for two 5-plane reductions
  const int nacc = 10;
  if (e == cudaSuccess) e = cudaMalloc(&acc, nacc * P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, nacc * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&fin, (27 + lbmk::NLAG) * P * sizeof(double));
  auto release = [&]() {
    for (double* p : {ck, seg, lam, acc, dout, fin})
      if (p) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "adjoint allocation");
  }
  auto hplanes = [&](int par) { return (double*)c->pop[par] + 18 * P; };
  auto save = [&](double* dst) {
    cudaError_t r = cudaMemcpyAsync(dst, hplanes(c->cur), hN * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(dst + hN, c->lag[c->cur], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return r;
  };
  int st = LBM_OK;
  const int64_t step0 = c->step;
  std::vector<int> ckpar((size_t)nck);
  // forward, keeping every `every`-th state
  for (int64_t k = 0; k < nsteps && e == cudaSuccess && st == LBM_OK; k++) {
    if (k % every == 0) {
      ckpar[(size_t)(k / every)] = c->cur;
      e = save(ck + (k / every) * stN);
    }
    if (e == cudaSuccess) st = lbm_step(c, 1, s);
  }
  double ffv = 0.0, inv_sum_w = 0.0;
  if (e == cudaSuccess && st == LBM_OK) st = lbm_compute_diagnostics(c, s);
  if (e == cudaSuccess && st == LBM_OK) {
    lbm_diag d;
    st = lbm_read_diagnostics(c, &d);
    if (st == LBM_OK) {
      ffv = d.frozen_volume / d.material_volume;
      inv_sum_w = 1.0 / d.material_volume;
    }
  }
  const int parN = c->cur;
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(fin, c->pop[parN], 27 * P * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fin + 27 * P, c->lag[parN], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, nacc * P * sizeof(double), s);
  // adjoint buffers: two sets of (9 population planes, lag fl, lag Q)
  double* lb[2] = {lam, lam + (9 + 2) * P};
  lbmk::AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.c = c->cd;
  a.mask = (const unsigned char*)c->mask;
  a.has_mask = c->g.has_mask;
  a.phi0 = (const double*)c->phi0;
  a.acc = acc;
  a.inv_sum_w = inv_sum_w;
  int cur_adj = 0;
  if (e == cudaSuccess && st == LBM_OK) {
    a.h = hplanes(parN);
    a.lag = (const double*)c->lag[parN];
    a.lam_out = lb[0];
    a.lfl_out = lb[0] + 9 * P;
    a.lq_out = lb[0] + 10 * P;
    e = lbmk::launch_adjoint_seed(a, s);
  }
  // reverse sweep: recompute each segment from its checkpoint, then step back
  for (int64_t sg = nck - 1; sg >= 0 && e == cudaSuccess && st == LBM_OK; sg--) {
    const int64_t k0 = sg * every, k1 = std::min<int64_t>(k0 + every, nsteps);
    const int par = ckpar[(size_t)sg];
    e = cudaMemcpyAsync(hplanes(par), ck + sg * stN, hN * sizeof(double),
                        cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->lag[par], ck + sg * stN + hN, lN * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    c->cur = par;
    c->step = step0 + k0;
    c->gen++;
    for (int64_t j = 0; j < k1 - k0 && e == cudaSuccess && st == LBM_OK; j++) {
      e = save(seg + j * stN);
      if (e == cudaSuccess) st = lbm_step(c, 1, s);
    }
    for (int64_t j = k1 - k0 - 1; j >= 0 && e == cudaSuccess && st == LBM_OK; j--) {
      a.h = seg + j * stN;
      a.lag = seg + j * stN + hN;
      a.lam_in = lb[cur_adj];
      a.lfl_in = lb[cur_adj] + 9 * P;
      a.lq_in = lb[cur_adj] + 10 * P;
      a.lam_out = lb[cur_adj ^ 1];
      a.lfl_out = lb[cur_adj ^ 1] + 9 * P;
      a.lq_out = lb[cur_adj ^ 1] + 10 * P;
      e = lbmk::launch_adjoint_step(a, s);
      cur_adj ^= 1;
    }
  }
  // a run from set_geometry's state: add that state's dependence on L
  if (e == cudaSuccess && st == LBM_OK && step0 == 0) {
    a.lam_in = lb[cur_adj];
    a.lag = ck + hN;  // checkpoint 0 holds the initial lags
    e = lbmk::launch_adjoint_init(a, s);
  }
  double hg[10] = {0};
  if (e == cudaSuccess && st == LBM_OK) e = lbmk::launch_adjoint_reduce(acc, c->g, dout, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = lbmk::launch_adjoint_reduce(acc + 5 * P, c->g, dout + 5, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(hg, dout, sizeof(hg), cudaMemcpyDeviceToHost, s);
  // the context ends at the final state, as after lbm_step(nsteps)
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->pop[parN], fin, 27 * P * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->lag[parN], fin + 27 * P, lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  c->cur = parN;
  c->step = step0 + nsteps;
  c->gen++;
  if (e == cudaSuccess && st == LBM_OK) st = lbm_compute_diagnostics(c, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
  if (st != LBM_OK) return st;
  *ff_out = ffv;
  for (int k = 0; k < 6; k++) grad[k] = hg[k];
  c->last_stream = s;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// reverse mode: an interface crossing of a phase-field run and its gradient
// ---------------------------------------------------------------------------

extern "C" int lbm_adjoint_crossing(lbm_ctx* c, int64_t nsteps, int every, int axis, int index,
                                    double* pos_out, double* grad, void* stream) {
  Range nvtx_range("lbm_adjoint_crossing");
  if (!c) return LBM_ERR_ARG;
  if (!pos_out || !grad) return fail(c, LBM_ERR_ARG, "null output%s");
  if (nsteps < 1 || every < 1) return fail(c, LBM_ERR_ARG, "nsteps and the checkpoint interval must be >= 1%s");
  if ((axis != 0 && axis != 1) || index < 0 || index >= (axis == 0 ? c->p.ny : c->p.nx))
    return fail(c, LBM_ERR_ARG, "axis must be 0 or 1 and index a line of the grid%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "adjoint before lbm_set_geometry%s");
  if (c->p.precision != LBM_FP64 || c->p.lattices != LBM_LAT_PHASE || !(c->p.sigma > 0.0))
    return fail(c, LBM_ERR_UNSUPPORTED,
                "the phase-field adjoint covers FP64 contexts with the phase-field lattice alone "
                "and sigma > 0%s");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)c->g.plane;
  const size_t gN = 9 * P, lN = lbmk::NLAG * P, stN = gN + lN;  // doubles per stored state
  const int64_t nck = (nsteps + every - 1) / every;
  const int64_t seglen = std::min<int64_t>(every, nsteps);
  // work planes: phi, fs, phib, fsb, mub, 9 gs, 2 x 9 adjoint populations
  const size_t wN = (5 + 9 + 18) * P;
  double *ck = nullptr, *seg = nullptr, *wk = nullptr, *acc = nullptr, *dout = nullptr,
         *fin = nullptr;
  cudaError_t e = cudaMalloc(&ck, nck * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&seg, seglen * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&wk, wN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&acc, lbmk::ADJ_NACC * P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, (lbmk::ADJ_NACC + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&fin, (27 + lbmk::NLAG) * P * sizeof(double));
  auto release = [&]() {
    for (double* p : {ck, seg, wk, acc, dout, fin})
      if (p) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "adjoint allocation");
  }
  auto gplanes = [&](int par) { return (double*)c->pop[par] + 9 * P; };
  auto save = [&](double* dst) {
    cudaError_t r = cudaMemcpyAsync(dst, gplanes(c->cur), gN * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(dst + gN, c->lag[c->cur], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return r;
  };
  int st = LBM_OK;
  const int64_t step0 = c->step;
  std::vector<int> ckpar((size_t)nck);
  for (int64_t k = 0; k < nsteps && e == cudaSuccess && st == LBM_OK; k++) {
    if (k % every == 0) {
      ckpar[(size_t)(k / every)] = c->cur;
      e = save(ck + (k / every) * stN);
    }
    if (e == cudaSuccess) st = lbm_step(c, 1, s);
  }
  const int parN = c->cur;
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(fin, c->pop[parN], 27 * P * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fin + 27 * P, c->lag[parN], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, lbmk::ADJ_NACC * P * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(wk, 0, wN * sizeof(double), s);
  const double pi = 3.14159265358979323846;
  double* lb[2] = {wk + 14 * P, wk + 23 * P};
  lbmk::PhaseAdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.c = c->cd;
  a.phi0 = (const double*)c->phi0;
  a.phi = wk;
  a.fs = wk + P;
  a.phib = wk + 2 * P;
  a.fsb = wk + 3 * P;
  a.mub = wk + 4 * P;
  a.gs = wk + 5 * P;
  a.acc = acc;
  a.dcos_dtheta = -std::sin(c->p.theta_deg * pi / 180.0) * (pi / 180.0);
  a.axis = axis;
  a.index = index;
  a.out = dout + lbmk::ADJ_NACC;
  int cur_adj = 0;
  // seed: the crossing on the final state
  if (e == cudaSuccess && st == LBM_OK) {
    a.gpop = gplanes(parN);
    a.lag = (const double*)c->lag[parN];
    a.lam_out = lb[0];
    e = lbmk::launch_phase_adjoint_fields(a, s);
    if (e == cudaSuccess) e = lbmk::launch_phase_adjoint_seed(a, s);
  }
  // reverse sweep: recompute each segment from its checkpoint, then step back
  for (int64_t sg = nck - 1; sg >= 0 && e == cudaSuccess && st == LBM_OK; sg--) {
    const int64_t k0 = sg * every, k1 = std::min<int64_t>(k0 + every, nsteps);
    const int par = ckpar[(size_t)sg];
    e = cudaMemcpyAsync(gplanes(par), ck + sg * stN, gN * sizeof(double),
                        cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->lag[par], ck + sg * stN + gN, lN * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    c->cur = par;
    c->step = step0 + k0;
    c->gen++;
    for (int64_t j = 0; j < k1 - k0 && e == cudaSuccess && st == LBM_OK; j++) {
      e = save(seg + j * stN);
      if (e == cudaSuccess) st = lbm_step(c, 1, s);
    }
    for (int64_t j = k1 - k0 - 1; j >= 0 && e == cudaSuccess && st == LBM_OK; j--) {
      a.gpop = seg + j * stN;
      a.lag = seg + j * stN + gN;
      a.lam_in = lb[cur_adj];
      a.lam_out = lb[cur_adj ^ 1];
      e = lbmk::launch_phase_adjoint_fields(a, s);
      if (e == cudaSuccess) e = lbmk::launch_phase_adjoint_step(a, s);
      cur_adj ^= 1;
    }
  }
  // a run from set_geometry's state: add that state's dependence on theta
  // and sigma (phi and fs of checkpoint 0 are still in the work planes)
  if (e == cudaSuccess && st == LBM_OK && step0 == 0) {
    a.lam_in = lb[cur_adj];
    e = lbmk::launch_phase_adjoint_init(a, s);
  }
  double hg[lbmk::ADJ_NACC + 1] = {0};
  if (e == cudaSuccess && st == LBM_OK) e = lbmk::launch_adjoint_reduce(acc, c->g, dout, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(hg, dout, sizeof(hg), cudaMemcpyDeviceToHost, s);
  // the context ends at the final state, as after lbm_step(nsteps)
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->pop[parN], fin, 27 * P * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->lag[parN], fin + 27 * P, lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  c->cur = parN;
  c->step = step0 + nsteps;
  c->gen++;
  if (e == cudaSuccess && st == LBM_OK) st = lbm_compute_diagnostics(c, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
  if (st != LBM_OK) return st;
  *pos_out = hg[lbmk::ADJ_NACC];
  grad[0] = hg[0];
  grad[1] = hg[1];
  c->last_stream = s;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// reverse mode: the coupled phase-field and enthalpy step (freezing, fluid at
// rest)
// ---------------------------------------------------------------------------

extern "C" int lbm_adjoint_freezing(lbm_ctx* c, int64_t nsteps, int every, int observable,
                                    int axis, int index, double* value_out, double* grad,
                                    void* stream) {
  Range nvtx_range("lbm_adjoint_freezing");
  if (!c) return LBM_ERR_ARG;
  if (!value_out || !grad) return fail(c, LBM_ERR_ARG, "null output%s");
  if (nsteps < 1 || every < 1) return fail(c, LBM_ERR_ARG, "nsteps and the checkpoint interval must be >= 1%s");
  if (observable != 0 && observable != 1) return fail(c, LBM_ERR_ARG, "observable must be 0 or 1%s");
  if (observable == 1 &&
      ((axis != 0 && axis != 1) || index < 0 || index >= (axis == 0 ? c->p.ny : c->p.nx)))
    return fail(c, LBM_ERR_ARG, "axis must be 0 or 1 and index a line of the grid%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "adjoint before lbm_set_geometry%s");
  if (c->p.precision != LBM_FP64 || c->p.lattices != (LBM_LAT_PHASE | LBM_LAT_HEAT) ||
      !(c->p.sigma > 0.0))
    return fail(c, LBM_ERR_UNSUPPORTED,
                "the coupled adjoint covers FP64 contexts with the phase-field and enthalpy "
                "lattices (no flow lattice) and sigma > 0%s");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)c->g.plane;
  const size_t pN = 18 * P, lN = lbmk::NLAG * P, stN = pN + lN;
  const int64_t nck = (nsteps + every - 1) / every;
  const int64_t seglen = std::min<int64_t>(every, nsteps);
  // work planes: two adjoint sets of (18 populations, fl, w, Q); phi, fs,
  // mub, the seed's phi adjoint and lag adjoints (fl, w)
  const size_t setN = 21 * P;
  const size_t wN = 2 * setN + 6 * P;
  const int nacc = 10;  // FRZ_NACC planes, padded for two 5-plane reductions
  double *ck = nullptr, *seg = nullptr, *wk = nullptr, *acc = nullptr, *dout = nullptr,
         *fin = nullptr;
  cudaError_t e = cudaMalloc(&ck, nck * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&seg, seglen * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&wk, wN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&acc, nacc * P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, 11 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&fin, (27 + lbmk::NLAG) * P * sizeof(double));
  auto release = [&]() {
    for (double* p : {ck, seg, wk, acc, dout, fin})
      if (p) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "adjoint allocation");
  }
  auto gh = [&](int par) { return (double*)c->pop[par] + 9 * P; };
  auto save = [&](double* dst) {
    cudaError_t r = cudaMemcpyAsync(dst, gh(c->cur), pN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(dst + pN, c->lag[c->cur], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return r;
  };
  int st = LBM_OK;
  const int64_t step0 = c->step;
  std::vector<int> ckpar((size_t)nck);
  for (int64_t k = 0; k < nsteps && e == cudaSuccess && st == LBM_OK; k++) {
    if (k % every == 0) {
      ckpar[(size_t)(k / every)] = c->cur;
      e = save(ck + (k / every) * stN);
    }
    if (e == cudaSuccess) st = lbm_step(c, 1, s);
  }
  double ffv = 0.0, inv_sum_w = 0.0;
  if (e == cudaSuccess && st == LBM_OK && observable == 0) {
    st = lbm_compute_diagnostics(c, s);
    lbm_diag d;
    if (st == LBM_OK) st = lbm_read_diagnostics(c, &d);
    if (st == LBM_OK) {
      ffv = d.frozen_volume / d.material_volume;
      inv_sum_w = 1.0 / d.material_volume;
    }
  }
  const int parN = c->cur;
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(fin, c->pop[parN], 27 * P * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fin + 27 * P, c->lag[parN], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, nacc * P * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(wk, 0, wN * sizeof(double), s);
  const double pi = 3.14159265358979323846;
  double* lb[2] = {wk, wk + setN};
  double* phi = wk + 2 * setN;
  double* fsp = phi + P;
  double* mub = phi + 2 * P;
  double* phib_seed = phi + 3 * P;
  double* seed_fl = phi + 4 * P;
  double* seed_w = phi + 5 * P;
  lbmk::FrzArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.c = c->cd;
  a.mask = (const unsigned char*)c->mask;
  a.has_mask = c->g.has_mask;
  a.phi0 = (const double*)c->phi0;
  a.phi = phi;
  a.fs = fsp;
  a.mub = mub;
  a.acc = acc;
  a.dcos_dtheta = -std::sin(c->p.theta_deg * pi / 180.0) * (pi / 180.0);
  a.inv_sum_w = inv_sum_w;
  a.ff = ffv;
  a.axis = axis;
  a.index = index;
  a.out = dout + 10;
  auto set_io = [&](int in, int out) {
    a.lam_in = lb[in];
    a.lfl_in = lb[in] + 18 * P;
    a.lw_in = lb[in] + 19 * P;
    a.lq_in = lb[in] + 20 * P;
    a.lam_out = lb[out];
    a.lfl_out = lb[out] + 18 * P;
    a.lw_out = lb[out] + 19 * P;
    a.lq_out = lb[out] + 20 * P;
  };
  int cur_adj = 0;
  // seed on the final state: the step kernel with zero pulled adjoints and
  // the observable's adjoints as inputs
  if (e == cudaSuccess && st == LBM_OK) {
    a.pop = gh(parN);
    a.lag = (const double*)c->lag[parN];
    e = lbmk::launch_frz_fields(a, s);
    set_io(1, 0);
    if (observable == 0) {
      a.lfl_out = seed_fl;
      a.lw_out = seed_w;
      if (e == cudaSuccess) e = lbmk::launch_frz_seed_ff(a, s);
      set_io(1, 0);
      a.lfl_in = seed_fl;
      a.lw_in = seed_w;
    } else {
      if (e == cudaSuccess) e = lbmk::launch_frz_seed_crossing(a, phib_seed, s);
      a.phib_seed = phib_seed;
    }
    if (e == cudaSuccess) e = lbmk::launch_frz_step(a, s);
    a.phib_seed = nullptr;
  }
  // reverse sweep: recompute each segment from its checkpoint, then step back
  for (int64_t sg = nck - 1; sg >= 0 && e == cudaSuccess && st == LBM_OK; sg--) {
    const int64_t k0 = sg * every, k1 = std::min<int64_t>(k0 + every, nsteps);
    const int par = ckpar[(size_t)sg];
    e = cudaMemcpyAsync(gh(par), ck + sg * stN, pN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->lag[par], ck + sg * stN + pN, lN * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    c->cur = par;
    c->step = step0 + k0;
    c->gen++;
    for (int64_t j = 0; j < k1 - k0 && e == cudaSuccess && st == LBM_OK; j++) {
      e = save(seg + j * stN);
      if (e == cudaSuccess) st = lbm_step(c, 1, s);
    }
    for (int64_t j = k1 - k0 - 1; j >= 0 && e == cudaSuccess && st == LBM_OK; j--) {
      a.pop = seg + j * stN;
      a.lag = seg + j * stN + pN;
      set_io(cur_adj, cur_adj ^ 1);
      e = lbmk::launch_frz_fields(a, s);
      if (e == cudaSuccess) e = lbmk::launch_frz_mub(a, s);
      if (e == cudaSuccess) e = lbmk::launch_frz_step(a, s);
      cur_adj ^= 1;
    }
  }
  // a run from set_geometry's state: the initial populations' dependence on
  // L (rest enthalpy population) and on theta and sigma (phase equilibrium,
  // with the phi and fs set_geometry used, rebuilt from checkpoint 0)
  if (e == cudaSuccess && st == LBM_OK && step0 == 0) {
    lbmk::AdjArgs ha;
    std::memset(&ha, 0, sizeof(ha));
    ha.g = c->g;
    ha.c = c->cd;
    ha.lam_in = lb[cur_adj] + 9 * P;
    ha.lag = ck + pN;
    ha.acc = acc;
    e = lbmk::launch_adjoint_init(ha, s);
    if (e == cudaSuccess)
      e = lbmk::launch_adjoint_init_fields(c->g, ck, ck + pN, (const double*)c->phi0, phi, fsp, s);
    lbmk::PhaseAdjArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.g = c->g;
    pa.c = c->cd;
    pa.lam_in = lb[cur_adj];
    pa.phi = phi;
    pa.fs = fsp;
    pa.phi0 = (const double*)c->phi0;
    pa.acc = acc + 5 * P;
    pa.dcos_dtheta = a.dcos_dtheta;
    if (e == cudaSuccess) e = lbmk::launch_phase_adjoint_init(pa, s);
  }
  double hg[11] = {0};
  if (e == cudaSuccess && st == LBM_OK) e = lbmk::launch_adjoint_reduce(acc, c->g, dout, s);
  if (e == cudaSuccess && st == LBM_OK) e = lbmk::launch_adjoint_reduce(acc + 5 * P, c->g, dout + 5, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(hg, dout, sizeof(hg), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->pop[parN], fin, 27 * P * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->lag[parN], fin + 27 * P, lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  c->cur = parN;
  c->step = step0 + nsteps;
  c->gen++;
  if (e == cudaSuccess && st == LBM_OK) st = lbm_compute_diagnostics(c, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
  if (st != LBM_OK) return st;
  *value_out = observable == 0 ? ffv : hg[10];
  for (int k = 0; k < lbmk::FRZ_NACC; k++) grad[k] = hg[k];
  c->last_stream = s;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// reverse mode: the whole coupled step (flow, phase field, enthalpy)
// ---------------------------------------------------------------------------

extern "C" int lbm_adjoint_coupled(lbm_ctx* c, int64_t nsteps, int every, int observable,
                                   int axis, int index, double* value_out, double* grad,
                                   double* dT0, void* stream) {
  Range nvtx_range("lbm_adjoint_coupled");
  if (!c) return LBM_ERR_ARG;
  if (!value_out || !grad) return fail(c, LBM_ERR_ARG, "null output%s");
  if (nsteps < 1 || every < 1) return fail(c, LBM_ERR_ARG, "nsteps and the checkpoint interval must be >= 1%s");
  if (observable != 0 && observable != 1) return fail(c, LBM_ERR_ARG, "observable must be 0 or 1%s");
  if (observable == 1 &&
      ((axis != 0 && axis != 1) || index < 0 || index >= (axis == 0 ? c->p.ny : c->p.nx)))
    return fail(c, LBM_ERR_ARG, "axis must be 0 or 1 and index a line of the grid%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "adjoint before lbm_set_geometry%s");
  if (dT0 && c->step != 0)
    return fail(c, LBM_ERR_STATE, "the initial-temperature gradient needs a run from lbm_set_geometry%s");
  if (c->p.precision != LBM_FP64 || c->p.lattices != (LBM_LAT_FLOW | LBM_LAT_PHASE | LBM_LAT_HEAT) ||
      c->p.readings != 0 || !(c->p.sigma > 0.0))
    return fail(c, LBM_ERR_UNSUPPORTED,
                "the coupled-step adjoint covers FP64 contexts with all three lattices, "
                "readings == 0 and sigma > 0%s");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)c->g.plane;
  const size_t pN = 27 * P, lN = lbmk::NLAG * P, stN = pN + lN;
  const int64_t nck = (nsteps + every - 1) / every;
  const int64_t seglen = std::min<int64_t>(every, nsteps);
  // work planes: two adjoint sets of (27 populations, NLAG lags); phi, fs,
  // rho; 7 stencil adjoints; the seed's phi adjoint and lag adjoints
  const size_t setN = (27 + lbmk::NLAG) * P;
  const size_t wN = 2 * setN + (3 + 7 + 1 + lbmk::NLAG) * P;
  const int nacc = 10;
  double *ck = nullptr, *seg = nullptr, *wk = nullptr, *acc = nullptr, *dout = nullptr,
         *fin = nullptr;
  cudaError_t e = cudaMalloc(&ck, nck * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&seg, seglen * stN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&wk, wN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&acc, nacc * P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, 11 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&fin, stN * sizeof(double));
  auto release = [&]() {
    for (double* p : {ck, seg, wk, acc, dout, fin})
      if (p) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "adjoint allocation");
  }
  auto save = [&](double* dst) {
    cudaError_t r = cudaMemcpyAsync(dst, c->pop[c->cur], pN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(dst + pN, c->lag[c->cur], lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return r;
  };
  int st = LBM_OK;
  const int64_t step0 = c->step;
  std::vector<int> ckpar((size_t)nck);
  for (int64_t k = 0; k < nsteps && e == cudaSuccess && st == LBM_OK; k++) {
    if (k % every == 0) {
      ckpar[(size_t)(k / every)] = c->cur;
      e = save(ck + (k / every) * stN);
    }
    if (e == cudaSuccess) st = lbm_step(c, 1, s);
  }
  double ffv = 0.0, inv_sum_w = 0.0;
  if (e == cudaSuccess && st == LBM_OK && observable == 0) {
    st = lbm_compute_diagnostics(c, s);
    lbm_diag d;
    if (st == LBM_OK) st = lbm_read_diagnostics(c, &d);
    if (st == LBM_OK) {
      ffv = d.frozen_volume / d.material_volume;
      inv_sum_w = 1.0 / d.material_volume;
    }
  }
  const int parN = c->cur;
  if (e == cudaSuccess && st == LBM_OK) e = save(fin);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, nacc * P * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(wk, 0, wN * sizeof(double), s);
  const double pi = 3.14159265358979323846;
  double* lb[2] = {wk, wk + setN};
  double* fld = wk + 2 * setN;
  double* sbp = fld + 3 * P;
  double* phib_seed = sbp + 7 * P;
  double* seed_lag = phib_seed + P;
  lbmk::FullArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.c = c->cd;
  a.phi0 = (const double*)c->phi0;
  a.mask = (const unsigned char*)c->mask;
  a.has_mask = c->g.has_mask;
  a.phi = fld;
  a.fs = fld + P;
  a.rho = fld + 2 * P;
  a.sb = sbp;
  a.acc = acc;
  a.dcos_dtheta = -std::sin(c->p.theta_deg * pi / 180.0) * (pi / 180.0);
  a.inv_sum_w = inv_sum_w;
  a.ff = ffv;
  a.axis = axis;
  a.index = index;
  a.out = dout + 10;
  auto set_io = [&](int in, int out) {
    a.lam_in = lb[in];
    a.llag_in = lb[in] + pN;
    a.lam_out = lb[out];
    a.llag_out = lb[out] + pN;
  };
  int cur_adj = 0;
  if (e == cudaSuccess && st == LBM_OK) {
    a.pop = (const double*)c->pop[parN];
    a.lag = (const double*)c->lag[parN];
    e = lbmk::launch_full_fields(a, s);
    set_io(1, 0);
    if (observable == 0) {
      if (e == cudaSuccess) e = lbmk::launch_full_seed_ff(a, seed_lag, s);
      a.llag_in = seed_lag;
    } else {
      if (e == cudaSuccess) e = lbmk::launch_full_seed_crossing(a, phib_seed, s);
      a.phib_seed = phib_seed;
    }
    if (e == cudaSuccess) e = lbmk::launch_full_k2(a, s);
    a.phib_seed = nullptr;
  }
  for (int64_t sg = nck - 1; sg >= 0 && e == cudaSuccess && st == LBM_OK; sg--) {
    const int64_t k0 = sg * every, k1 = std::min<int64_t>(k0 + every, nsteps);
    const int par = ckpar[(size_t)sg];
    e = cudaMemcpyAsync(c->pop[par], ck + sg * stN, pN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->lag[par], ck + sg * stN + pN, lN * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    c->cur = par;
    c->step = step0 + k0;
    c->gen++;
    for (int64_t j = 0; j < k1 - k0 && e == cudaSuccess && st == LBM_OK; j++) {
      e = save(seg + j * stN);
      if (e == cudaSuccess) st = lbm_step(c, 1, s);
    }
    for (int64_t j = k1 - k0 - 1; j >= 0 && e == cudaSuccess && st == LBM_OK; j--) {
      a.pop = seg + j * stN;
      a.lag = seg + j * stN + pN;
      set_io(cur_adj, cur_adj ^ 1);
      e = lbmk::launch_full_fields(a, s);
      if (e == cudaSuccess) e = lbmk::launch_full_k1(a, s);
      if (e == cudaSuccess) e = lbmk::launch_full_k2(a, s);
      cur_adj ^= 1;
    }
  }
  if (e == cudaSuccess && st == LBM_OK && step0 == 0) {
    lbmk::AdjArgs ha;
    std::memset(&ha, 0, sizeof(ha));
    ha.g = c->g;
    ha.c = c->cd;
    ha.lam_in = lb[cur_adj] + 18 * P;
    ha.lag = ck + pN;
    ha.acc = acc;
    e = lbmk::launch_adjoint_init(ha, s);
    if (e == cudaSuccess)
      e = lbmk::launch_adjoint_init_fields(c->g, ck + 9 * P, ck + pN, (const double*)c->phi0, fld,
                                           fld + P, s);
    lbmk::PhaseAdjArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.g = c->g;
    pa.c = c->cd;
    pa.lam_in = lb[cur_adj] + 9 * P;
    pa.phi = fld;
    pa.fs = fld + P;
    pa.phi0 = (const double*)c->phi0;
    pa.acc = acc + 5 * P;
    pa.dcos_dtheta = a.dcos_dtheta;
    if (e == cudaSuccess) e = lbmk::launch_phase_adjoint_init(pa, s);
    if (e == cudaSuccess && dT0) {
      // the checkpoint-0 state (initial populations and lags) in the
      // reverse sweep's last recomputed slot; the field planes are reused
      a.pop = ck;
      a.lag = ck + pN;
      e = lbmk::launch_full_dT0(a, lb[cur_adj] + 18 * P, fld, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dT0, fld, (size_t)c->p.nx * c->p.ny * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    }
  }
  double hg[11] = {0};
  if (e == cudaSuccess && st == LBM_OK) e = lbmk::launch_adjoint_reduce(acc, c->g, dout, s);
  if (e == cudaSuccess && st == LBM_OK) e = lbmk::launch_adjoint_reduce(acc + 5 * P, c->g, dout + 5, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(hg, dout, sizeof(hg), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->pop[parN], fin, pN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && st == LBM_OK)
    e = cudaMemcpyAsync(c->lag[parN], fin + pN, lN * sizeof(double), cudaMemcpyDeviceToDevice, s);
  c->cur = parN;
  c->step = step0 + nsteps;
  c->gen++;
  if (e == cudaSuccess && st == LBM_OK) st = lbm_compute_diagnostics(c, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
  if (st != LBM_OK) return st;
  *value_out = observable == 0 ? ffv : hg[10];
  for (int k = 0; k < lbmk::FULL_NACC; k++) grad[k] = hg[k];
  c->last_stream = s;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// autotuning of the step form on the context's own grid
// ---------------------------------------------------------------------------

extern "C" int lbm_autotune(lbm_ctx* c, int steps_per_trial, void* stream, double* out_us,
                            int* chosen) {
  Range nvtx_range("lbm_autotune");
  if (!c) return LBM_ERR_ARG;
  if (steps_per_trial < 2) return fail(c, LBM_ERR_ARG, "steps_per_trial must be >= 2%s");
  if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "autotune before lbm_set_geometry%s");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)c->g.plane;
  const size_t pb = 27 * P * c->pop_esize, lb = c->nlag * P * c->esize;
  // the diagnostic partials too: trial steps overwrite them
  const size_t db = (c->tangent ? 2 : 1) * (size_t)lbmk::NDIAG * c->diag_cap * sizeof(double);
  void* backup = nullptr;
  cudaError_t e = cudaMalloc(&backup, pb + lb + db);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune backup allocation");
  // the state the trials start from, and the host-side step bookkeeping
  const int cur = c->cur;
  const int64_t step = c->step, diag_step = c->diag_step;
  const bool have_diag = c->have_diag, pending = c->diag_pending;
  const bool graphs0 = c->graphs;
  const int gmin0 = c->graph_min, form0 = c->form, diag_nb0 = c->diag_nb;
  e = cudaMemcpyAsync(backup, c->pop[cur], pb, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((char*)backup + pb, c->lag[cur], lb, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((char*)backup + pb + lb, c->diag_partial, db, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  // variants: kernel form (v / 2) x shortest captured period (32, 256)
  double us[kAutotuneVariants];
  for (int v = 0; v < kAutotuneVariants; v++) us[v] = -1.0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  for (int v = 0; v < kAutotuneVariants && e == cudaSuccess; v++) {
    if (!form_available(c, v / 2)) continue;
    set_kernel_form(c, v / 2);
    c->graphs = graphs0;
    c->graph_min = (v & 1) ? 256 : 32;
    c->gen++;  // another kernel form: nothing captured before applies
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // rep 0 warms up and captures
      e = cudaMemcpyAsync(c->pop[cur], backup, pb, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lag[cur], (char*)backup + pb, lb, cudaMemcpyDeviceToDevice, s);
      c->cur = cur;
      c->step = step;
      if (e != cudaSuccess) break;
      e = cudaEventRecord(t0, s);
      if (e == cudaSuccess && lbm_step(c, steps_per_trial, s) != LBM_OK) e = cudaErrorUnknown;
      if (e == cudaSuccess) e = cudaEventRecord(t1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e == cudaSuccess && rep == 1) us[v] = 1e3 * ms / steps_per_trial;
    }
  }
  // the fastest variant replaces the context's current one only when it is
  // faster by more than 2 % (the run-to-run spread of these timings), so
  // that near ties keep the default form
  int best = -1;
  for (int v = 0; v < kAutotuneVariants; v++)
    if (us[v] > 0.0 && (best < 0 || us[v] < us[best])) best = v;
  const int cur0 = 2 * form0 + (gmin0 >= 256 ? 1 : 0);
  if (best >= 0 && cur0 < kAutotuneVariants && us[cur0] > 0.0 && us[cur0] <= 1.02 * us[best])
    best = cur0;
  if (best < 0) best = 0;
  // restore the state, keep the fastest variant
  cudaError_t er = cudaMemcpyAsync(c->pop[cur], backup, pb, cudaMemcpyDeviceToDevice, s);
  if (er == cudaSuccess)
    er = cudaMemcpyAsync(c->lag[cur], (char*)backup + pb, lb, cudaMemcpyDeviceToDevice, s);
  if (er == cudaSuccess)
    er = cudaMemcpyAsync(c->diag_partial, (char*)backup + pb + lb, db, cudaMemcpyDeviceToDevice, s);
  if (er == cudaSuccess) er = cudaStreamSynchronize(s);
  c->cur = cur;
  c->step = step;
  c->diag_step = diag_step;
  c->diag_nb = diag_nb0;
  c->have_diag = have_diag;
  c->diag_pending = pending;
  c->gen++;
  c->graphs = graphs0;
  if (e == cudaSuccess && er == cudaSuccess) {
    set_kernel_form(c, best / 2);
    c->graph_min = (best & 1) ? 256 : 32;
  } else {
    set_kernel_form(c, form0);
    c->graph_min = gmin0;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(backup);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune trial");
  if (er != cudaSuccess) return cuda_fail(c, er, "autotune restore");
  if (out_us)
    for (int v = 0; v < kAutotuneVariants; v++) out_us[v] = us[v];
  if (chosen) *chosen = best;
  c->last_stream = s;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// batches: several contexts advanced by one persistent launch per step
// ---------------------------------------------------------------------------

struct lbm_batch {
  std::vector<lbm_ctx*> ctx;
  int precision;
  // FP32 batches step as the batched TMA-staged tile kernel (one stage, one
  // CTA per tile) unless LBM_BATCH_KERNEL=fused; its argument table
  bool tile;
  lbmk::TileBatch<float>* ttab;
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;               // one captured period of batch steps
  std::vector<uint64_t> graph_key;     // (parity, generation) per context, phase
  char err[512];
};

namespace {

// One launch covers up to BATCH_MAX_GRIDS consecutive contexts; the table
// holds each one's step arguments (buffers by its current parity).
template <typename R>
bool fill_table(lbm_batch* b, int first, int count, lbmk::BatchTable<R>& t) {
  bool all = true;
  t.ngrids = count;
  t.tile_base[0] = 0;
  for (int i = 0; i < count; i++) {
    lbm_ctx* c = b->ctx[first + i];
    const Coef<R>* coef;
    if (sizeof(R) == 4) coef = (const Coef<R>*)(const void*)&c->cf;
    else coef = (const Coef<R>*)(const void*)&c->cd;
    t.args[i] = step_args<R>(c, *coef);
    t.tile_base[i + 1] = t.tile_base[i] + c->nblocks;
    if (c->p.lattices != 7u) all = false;
  }
  return all;
}

// The batched tile kernel's table for contexts [first, first + count).
bool fill_tile_table(lbm_batch* b, int first, int count, lbmk::TileBatch<float>& t) {
  bool all = true;
  t.ngrids = count;
  t.tile_base[0] = 0;
  t.extra_tx = g_tile_timeout.load() ? 16u : 0u;
  for (int i = 0; i < count; i++) {
    lbm_ctx* c = b->ctx[first + i];
    t.args[i] = step_args<float>(c, c->cf);
    t.tile_base[i + 1] = t.tile_base[i] + c->nblocks;
    t.tiles_x[i] = (c->g.nx + lbmk::TX - 1) / lbmk::TX;
    t.maps[i] = c->d_maps + c->cur;
    t.status[i] = c->status;
    if (c->p.lattices != 7u) all = false;
  }
  return all;
}

// Marks, for every context, the state of the batch's last diagnosed step in
// a span of `n` steps that starts at the first context's step `first0`.
void note_batch_diag(lbm_batch* b, int64_t first0, int64_t n) {
  lbm_ctx* c0 = b->ctx[0];
  const int64_t d = c0->p.diag_every;
  if (d <= 0 || n <= 0) return;
  const int64_t end = first0 + n;
  const int64_t last = (end - 1) - ((end - 1) % d);
  if (last < first0) return;
  for (lbm_ctx* c : b->ctx) {
    c->have_diag = true;
    c->diag_pending = true;
    c->diag_nb = c->nblocks;  // the batch kernel's 32 x 8 tiles
    c->diag_step = c->step + (last - first0);
  }
}

template <typename R>
cudaError_t batch_launches(lbm_batch* b, int64_t nsteps, cudaStream_t s,
                           lbmk::BatchTable<R>& t) {
  const int n = (int)b->ctx.size();
  lbm_ctx* c0 = b->ctx[0];
  for (int64_t k = 0; k < nsteps; k++) {
    const bool diag = c0->p.diag_every > 0 && (c0->step % c0->p.diag_every) == 0;
    for (int first = 0; first < n; first += lbmk::BATCH_MAX_GRIDS) {
      const int count = std::min(n - first, lbmk::BATCH_MAX_GRIDS);
      cudaError_t e;
      if (sizeof(R) == 4 && b->tile) {
        const bool all = fill_tile_table(b, first, count, *b->ttab);
        e = lbmk::launch_tile_batch_f32(*b->ttab, diag, all, s);
        if (e != cudaSuccess) return e;
        continue;
      }
      const bool all = fill_table<R>(b, first, count, t);
      if (sizeof(R) == 4)
        e = lbmk::launch_batch_f32(*(const lbmk::BatchTable<float>*)(const void*)&t, diag, all, s);
      else
        e = lbmk::launch_batch_f64(*(const lbmk::BatchTable<double>*)(const void*)&t, diag, all,
                                   s);
      if (e != cudaSuccess) return e;
    }
    note_batch_diag(b, c0->step, 1);
    for (lbm_ctx* c : b->ctx) {
      c->cur ^= 1;
      c->step++;
    }
  }
  return cudaSuccess;
}

std::vector<uint64_t> batch_key(const lbm_batch* b, int period) {
  std::vector<uint64_t> k;
  k.reserve(2 * b->ctx.size() + 1);
  for (const lbm_ctx* c : b->ctx) {
    k.push_back((uint64_t)c->cur);
    k.push_back(c->gen);
  }
  k.push_back((uint64_t)(b->ctx[0]->step % period));
  k.push_back((uint64_t)period);
  return k;
}

// The captured period of batch steps from the contexts' current parities
// and phase (captured on a private stream when first needed).
template <typename R>
cudaError_t batch_graph(lbm_batch* b, int period, lbmk::BatchTable<R>& t, cudaGraphExec_t* out) {
  std::vector<uint64_t> key = batch_key(b, period);
  if (b->graph && key == b->graph_key) {
    *out = b->graph;
    return cudaSuccess;
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  struct Saved {
    int cur;
    int64_t step, diag_step;
    bool have_diag, pending;
  };
  std::vector<Saved> saved;
  for (const lbm_ctx* c : b->ctx)
    saved.push_back({c->cur, c->step, c->diag_step, c->have_diag, c->diag_pending});
  e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = batch_launches<R>(b, period, b->cap_stream, t);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap_stream, &g);
  for (size_t i = 0; i < b->ctx.size(); i++) {
    lbm_ctx* c = b->ctx[i];
    c->cur = saved[i].cur;
    c->step = saved[i].step;
    c->diag_step = saved[i].diag_step;
    c->have_diag = saved[i].have_diag;
    c->diag_pending = saved[i].pending;
  }
  if (el != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return el != cudaSuccess ? el : e;
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return e;
  }
  b->graph_key.swap(key);
  *out = b->graph;
  return cudaSuccess;
}

template <typename R>
int batch_step_impl(lbm_batch* b, int64_t nsteps, cudaStream_t s) {
  std::unique_ptr<lbmk::BatchTable<R>> t(new (std::nothrow) lbmk::BatchTable<R>());
  if (!t) return LBM_ERR_OOM;
  lbm_ctx* c0 = b->ctx[0];
  int64_t left = nsteps;
  const int period = graph_period(c0->p.diag_every, c0->graph_min);
  cudaError_t e = cudaSuccess;
  if (c0->graphs && period <= kMaxGraphSteps && left >= period && stream_free(s)) {
    cudaGraphExec_t g = nullptr;
    e = batch_graph<R>(b, period, *t, &g);
    if (e != cudaSuccess) {
      std::snprintf(b->err, sizeof(b->err), "batch graph capture: %s", cudaGetErrorString(e));
      return LBM_ERR_CUDA;
    }
    const int64_t reps = left / period;
    for (int64_t r = 0; r < reps && e == cudaSuccess; r++) e = cudaGraphLaunch(g, s);
    if (e != cudaSuccess) {
      std::snprintf(b->err, sizeof(b->err), "batch graph launch: %s", cudaGetErrorString(e));
      return LBM_ERR_CUDA;
    }
    note_batch_diag(b, c0->step, reps * period);
    for (lbm_ctx* c : b->ctx) c->step += reps * period;  // even period: parities unchanged
    left -= reps * period;
  }
  e = batch_launches<R>(b, left, s, *t);
  for (lbm_ctx* c : b->ctx) c->last_stream = s;
  if (e != cudaSuccess) {
    std::snprintf(b->err, sizeof(b->err), "batch kernel launch: %s", cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_ctx* const* ctxs, int count, lbm_batch** out) {
  if (!ctxs || !out || count < 1) return LBM_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; i++) {
    if (!ctxs[i]) return LBM_ERR_ARG;
    if (ctxs[i]->p.precision != ctxs[0]->p.precision) return LBM_ERR_ARG;
    if (ctxs[i]->p.precision == LBM_FP16S || ctxs[i]->tangent) return LBM_ERR_UNSUPPORTED;
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) return LBM_ERR_ARG;
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->ctx.assign(ctxs, ctxs + count);
  b->precision = ctxs[0]->p.precision;
  b->tile = b->precision == LBM_FP32;
  for (int i = 0; i < count; i++) b->tile = b->tile && ctxs[i]->tile_ok && ctxs[i]->d_maps;
  if (const char* k = std::getenv("LBM_BATCH_KERNEL"))
    if (std::strcmp(k, "fused") == 0) b->tile = false;
  if (b->tile) {
    b->ttab = new (std::nothrow) lbmk::TileBatch<float>();
    if (!b->ttab) {
      delete b;
      return LBM_ERR_OOM;
    }
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps, void* stream) {
  Range nvtx_range("lbm_batch_step");
  if (!b) return LBM_ERR_ARG;
  if (nsteps < 0) return LBM_ERR_ARG;
  for (lbm_ctx* c : b->ctx) {
    if (!c->have_geometry) {
      std::snprintf(b->err, sizeof(b->err), "a context of the batch has no geometry");
      return LBM_ERR_STATE;
    }
  }
  if (nsteps == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return b->precision == LBM_FP32 ? batch_step_impl<float>(b, nsteps, s)
                                  : batch_step_impl<double>(b, nsteps, s);
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b->ttab;
  delete b;
}

}  // extern "C"
