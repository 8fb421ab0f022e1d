// C ABI of the MLS library (include/mls.h): argument validation, ownership,
// device memory, launches and the host-pointer copy paths.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define MLS_HAVE_NVTX 1
#endif

#include "mls_internal.h"

namespace mlsi {

// A named NVTX range around each public call, for profilers and timeline
// tools (header-only NVTX: with no tool attached the calls do nothing; a
// toolkit without the NVTX headers builds the ranges as no-ops).
struct NvtxRange {
#ifdef MLS_HAVE_NVTX
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char *) {}
#endif
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

static thread_local std::string g_err;

mls_status fail(mls_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

mls_status cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky-free error so the handle stays usable
  return e == cudaErrorMemoryAllocation ? MLS_E_NOMEM : MLS_E_CUDA;
}

// Host-side fault injection for tests: while MLS_INJECT_NOMEM is set to a
// nonzero value every device allocation of the library fails with
// MLS_E_NOMEM before any CUDA call is made.
static bool inject_nomem() {
  const char *e = getenv("MLS_INJECT_NOMEM");
  return e && atoi(e) != 0;
}

// Device memory of handles and render contexts comes from one stream-ordered
// pool per device that keeps freed memory for reuse (release threshold at
// its maximum).  A pool that gives memory back to the system at every
// synchronisation (the default pool's behaviour) maps it again at the next
// allocation, and a render's scratch of tens of MB then costs more host time
// than its kernels take on the device.  The pool holds at most the largest
// working set the process has had, until the process exits.
constexpr int kPoolDevices = 64;
static cudaMemPool_t g_pool[kPoolDevices];
static std::mutex g_pool_mu;

static cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kPoolDevices) return cudaMallocAsync(p, bytes, st);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props;
      memset(&props, 0, sizeof props);
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np;
      if ((e = cudaMemPoolCreate(&np, &props)) != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      if ((e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
        cudaMemPoolDestroy(np);
        return e;
      }
      g_pool[dev] = np;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

mls_status dev_alloc(mls_handle *h, void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (inject_nomem()) return fail(MLS_E_NOMEM, "device allocation failed (MLS_INJECT_NOMEM)");
  cudaError_t e = pool_alloc(p, bytes ? bytes : 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  h->owned.push_back(*p);
  return MLS_OK;
}

static mls_status ctx_alloc(RenderCtx *c, void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (inject_nomem()) return fail(MLS_E_NOMEM, "device allocation failed (MLS_INJECT_NOMEM)");
  cudaError_t e = pool_alloc(p, bytes ? bytes : 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  c->owned.push_back(*p);
  return MLS_OK;
}

static void ctx_release(RenderCtx *c, void *p, cudaStream_t st) {
  if (!p) return;
  for (size_t i = 0; i < c->owned.size(); ++i)
    if (c->owned[i] == p) {
      c->owned.erase(c->owned.begin() + i);
      break;
    }
  cudaFreeAsync(p, st);
}

// Free every allocation of a context (stream-ordered on st).
static void ctx_free_all(RenderCtx *c, cudaStream_t st) {
  for (void *p : c->owned) cudaFreeAsync(p, st);
  *c = RenderCtx();
}

static void release(mls_handle *h, void *p, cudaStream_t st) {
  if (!p) return;
  for (size_t i = 0; i < h->owned.size(); ++i)
    if (h->owned[i] == p) {
      h->owned.erase(h->owned.begin() + i);
      break;
    }
  cudaFreeAsync(p, st);
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static mls_status check_view(const mls_view *v) {
  if (!v) return fail(MLS_E_INVAL, "view is NULL");
  if (v->W < 1 || v->H < 1) return fail(MLS_E_INVAL, "view W and H must be >= 1");
  if ((int64_t)v->W * v->H > (int64_t)1 << 30) return fail(MLS_E_INVAL, "view has more than 2^30 pixels");
  if (!std::isfinite(v->x0) || !std::isfinite(v->x1) || !std::isfinite(v->y0) || !std::isfinite(v->y1) ||
      !(v->x1 > v->x0) || !(v->y1 > v->y0))
    return fail(MLS_E_INVAL, "view rectangle must be finite with x1 > x0 and y1 > y0");
  return MLS_OK;
}

static mls_status check_levels(const double *levels, int L, int D) {
  if (L < 0 || L > 254) return fail(MLS_E_INVAL, "L must be in [0, 254]");
  if (L > 0 && !levels) return fail(MLS_E_INVAL, "levels is NULL");
  for (int d = 0; d < D && L > 0; ++d)
    for (int j = 0; j < L; ++j) {
      const double t = levels[(size_t)d * L + j];
      if (!std::isfinite(t)) return fail(MLS_E_INVAL, "levels must be finite");
      if (j > 0 && !(t >= levels[(size_t)d * L + j - 1])) return fail(MLS_E_INVAL, "levels must ascend");
    }
  return MLS_OK;
}

size_t scratch_bytes_for(int W, int H) {
  const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
  const size_t padded = (size_t)tx * kTile * ty * kTile;
  const size_t ntile = (size_t)tx * ty;
  return 256 + padded * sizeof(float) + padded * sizeof(int) + 2 * (size_t)W * H * sizeof(int) +
         3 * ntile * sizeof(float) + 4 * ntile * sizeof(int) + 256 +
         (size_t)handover_split_cap((int64_t)W * H) * handover_entry_bytes();
}

// Grow a render context's scratch to fit a view.
static mls_status ensure_scratch(RenderCtx *c, int W, int H, cudaStream_t st) {
  const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
  const size_t padded = (size_t)tx * kTile * ty * kTile;
  const size_t ntile = (size_t)tx * ty;
  const size_t need = scratch_bytes_for(W, H);
  if (need > c->scratch_bytes) {
    ctx_release(c, c->scratch, st);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    void *p;
    mls_status s = ctx_alloc(c, &p, need, st);
    if (s != MLS_OK) return s;
    c->scratch = p;
    c->scratch_bytes = need;
  }
  char *b = (char *)c->scratch;
  c->counters = (unsigned int *)b;           // [0] hand-over count, [1] FP64 count, [2] retried half tiles
  c->visited = (unsigned long long *)(b + 16);
  c->err = (int *)(b + 64);
  c->mstab = (float *)(b + 256);
  c->cnt = (int *)(b + 256 + padded * sizeof(float));
  c->relist = (int *)(b + 256 + padded * (sizeof(float) + sizeof(int)));
  c->relist2 = c->relist + (size_t)W * H;
  c->tcen = (float *)(c->relist2 + (size_t)W * H);
  c->tile_mark = (int *)(c->tcen + 2 * ntile);
  c->retry_tiles = c->tile_mark + 2 * ntile;   // both indexed by half tile
  c->tmax = (float *)(c->retry_tiles + 2 * ntile);
  c->ho_claims = (unsigned int *)(b + 32);  // in the header zeroed before every render
  // the split hand-over's entries, 256-byte aligned past the per-tile arrays
  const size_t ho_off = ((size_t)((char *)(c->tmax + ntile) - b) + 255) / 256 * 256;
  c->ho_state = b + ho_off;
  c->ho_cap = handover_split_cap((int64_t)W * H);
  return MLS_OK;
}

// Pinned host staging of the level uploads, per device and shared by every
// handle on it, so that a render enqueues its level copies without waiting
// for its stream (a copy from pageable memory would need the stream drained
// before the source could be reused).  Uploads take the slots of a small
// ring in turn; a slot is refilled only after the copy that last read it has
// completed.
namespace {
constexpr int kStageSlots = 8;
constexpr int kStageDevices = 64;
struct LevelStage {
  std::mutex mu;
  int next = 0;
  void *buf[kStageSlots] = {};
  size_t cap[kStageSlots] = {};
  cudaEvent_t done[kStageSlots] = {};
  bool pending[kStageSlots] = {};
};
LevelStage g_level_stage[kStageDevices];
}  // namespace

static mls_status upload_levels(mls_handle *h, RenderCtx *c, const double *levels, int L, cudaStream_t st) {
  const int D = h->desc.D;
  const size_t cnt = (size_t)D * L;
  if (cnt == 0) return MLS_OK;
  if (h->device < 0 || h->device >= kStageDevices) return fail(MLS_E_UNSUPPORTED, "device ordinal out of range");
  if (cnt > c->lev_cap) {
    ctx_release(c, c->lev64, st);
    ctx_release(c, c->lev32, st);
    c->lev64 = nullptr;
    c->lev32 = nullptr;
    c->lev_cap = 0;
    void *p;
    mls_status s;
    if ((s = ctx_alloc(c, &p, cnt * sizeof(double), st)) != MLS_OK) return s;
    c->lev64 = (double *)p;
    if ((s = ctx_alloc(c, &p, cnt * sizeof(float), st)) != MLS_OK) return s;
    c->lev32 = (float *)p;
    c->lev_cap = cnt;
  }
  LevelStage &g = g_level_stage[h->device];
  std::lock_guard<std::mutex> lock(g.mu);
  const int k = g.next;
  g.next = (g.next + 1) % kStageSlots;
  if (g.pending[k]) {
    MLS_CUDA_TRY(cudaEventSynchronize(g.done[k]));
    g.pending[k] = false;
  }
  if (!g.done[k]) MLS_CUDA_TRY(cudaEventCreateWithFlags(&g.done[k], cudaEventDisableTiming));
  const size_t bytes = cnt * (sizeof(double) + sizeof(float));
  if (g.cap[k] < bytes) {
    if (g.buf[k]) cudaFreeHost(g.buf[k]);
    g.buf[k] = nullptr;
    g.cap[k] = 0;
    MLS_CUDA_TRY(cudaMallocHost(&g.buf[k], bytes));
    g.cap[k] = bytes;
  }
  double *dn = (double *)g.buf[k];
  float *up = (float *)(dn + cnt);
  // float copies rounded up: for a float f, f >= t exactly when f >= t_up
  for (size_t i = 0; i < cnt; ++i) {
    dn[i] = levels[i];
    float f = (float)levels[i];
    if ((double)f < levels[i]) f = nextafterf(f, INFINITY);
    up[i] = f;
  }
  MLS_CUDA_TRY(cudaMemcpyAsync(c->lev64, dn, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
  MLS_CUDA_TRY(cudaMemcpyAsync(c->lev32, up, cnt * sizeof(float), cudaMemcpyHostToDevice, st));
  MLS_CUDA_TRY(cudaEventRecord(g.done[k], st));
  g.pending[k] = true;
  return MLS_OK;
}

static mls_status ensure_stage(RenderCtx *c, size_t bytes, cudaStream_t st) {
  if (bytes <= c->stage_bytes) return MLS_OK;
  ctx_release(c, c->stage, st);
  c->stage = nullptr;
  c->stage_bytes = 0;
  void *p;
  mls_status s = ctx_alloc(c, &p, bytes, st);
  if (s != MLS_OK) return s;
  c->stage = p;
  c->stage_bytes = bytes;
  return MLS_OK;
}

// Largest rhs amplification accepted with split FP16 weights: the noisy,
// sparse wine-shaped data (178 points, linear basis) reach the 1e-3 bound
// near lambda 1000, smooth and rough Fourier fields do not.  Single FP16
// weights (scaled by 2^14 in the tensor kernel) are accepted up to 60.
constexpr float kLambdaSplitFp16 = 200.f;
// Tile width (16 pixels) in units of h above which the tile frame is not used.
constexpr double kTileFrameMaxH = 4.0;

static mlsk::KParams base_params(const mls_handle *h, const RenderCtx *c, const mls_view *v) {
  const PointSet &P = h->P;
  const mls_desc &d = h->desc;
  mlsk::KParams p;
  memset(&p, 0, sizeof p);
  p.n = P.n;
  p.n_pad = P.n_pad;
  p.D = P.D;
  p.D_pad = P.D_pad;
  p.xs = P.xs;
  p.ys = P.ys;
  p.xs_lo = P.xs_lo;
  p.ys_lo = P.ys_lo;
  p.FT32 = P.FT32;
  p.FR32 = P.FR32;
  p.FR32lo = P.FR32lo;
  p.fcen32 = P.fcen32;
  p.fscl32 = P.fscl32;
  p.fcen64 = P.fcen;
  p.fscl64 = P.fscl;
  p.x64 = P.x64;
  p.y64 = P.y64;
  p.FT64 = P.FT64;
  p.xyb = P.xyb;
  p.fb = P.fb;
  p.fb_dc = P.fb_dc;
  p.cell_start = P.cell_start;
  p.gx = P.gx;
  p.gy = P.gy;
  p.gx0 = P.gx0;
  p.gy0 = P.gy0;
  p.cell = P.cell;
  p.inv_cell = P.cell > 0.0 ? 1.0 / P.cell : 0.0;
  p.degree = d.variant != MLS_V_POLY ? 1 : d.degree;   // the mappings use the linear moments
  p.variant = d.variant;
  p.trunc = d.support;
  p.weight = d.weight;
  p.h = d.h;
  p.alpha = d.alpha;
  p.cond_fp64 = d.cond_fp64;
  p.rcond_min = d.rcond_degenerate;
  p.cond_recompute = d.cond_recompute;
  p.cond_fp64_f = (float)d.cond_fp64;
  p.cond_recompute_f = (float)d.cond_recompute;
  p.inv_rcond_min_f = (float)(1.0 / d.rcond_degenerate);
  p.trunc_f = (float)d.support;
  p.trunc_on = d.support > 0.0 ? 1 : 0;
  // amplification of right-hand-side rounding the fast path accepts, from the
  // precision of its weights and operands (calibrated against the FP64 oracle)
  p.lambda_max = d.precision == MLS_P_FP32 ? 1000.f
               : d.precision == MLS_P_FP16 ? (d.weight_split == 1 ? kLambdaSplitFp16 : 60.f)
               : (d.weight_split == 1 ? 50.f : 10.f);
  p.W = v->W;
  p.H = v->H;
  p.x0 = v->x0;
  p.y0 = v->y0;
  p.sx = (v->x1 - v->x0) / (double)v->W;
  p.sy = (v->y1 - v->y0) / (double)v->H;
  p.ctr_x = P.ctr_x;
  p.ctr_y = P.ctr_y;
  p.inv_s = 1.0 / P.s;
  p.tiles_x = (v->W + kTile - 1) / kTile;
  p.tiles_y = (v->H + kTile - 1) / kTile;
  p.mstab = c->mstab;
  p.cnt = c->cnt;
  p.tcen = c->tcen;
  p.tmax = c->tmax;
  p.gcut = (h->operand_cut && !field_is_fp64(d.precision) && d.weight == MLS_W_GAUSS && !(d.support > 0.0) &&
            d.variant == MLS_V_POLY)
               ? mlsk::kGaussOperandCut
               : 0.f;
  p.relist = c->relist;
  p.relist_count = c->counters;
  p.err = c->err;
  p.f32_shape = (d.weight == MLS_W_GAUSS) ? h->f32_shape : 0;
  p.lev64 = c->lev64;
  p.lev32 = c->lev32;
  return p;
}

}  // namespace mlsi

using namespace mlsi;

extern "C" {

int32_t mls_abi_version(void) { return MLS_ABI_VERSION; }

const char *mls_last_error(void) { return g_err.c_str(); }

mls_status mls_desc_default(mls_desc *desc) {
  if (!desc) return fail(MLS_E_INVAL, "desc is NULL");
  memset(desc, 0, sizeof *desc);
  desc->n = 0;
  desc->D = 1;
  desc->degree = 1;
  desc->weight = MLS_W_GAUSS;
  desc->precision = MLS_P_FP32;
  desc->h = 0.05;
  desc->alpha = 1.0;
  desc->cond_fp64 = 1e6;
  desc->rcond_degenerate = 1e-12;
  desc->cond_recompute = 0.0;
  desc->weight_split = -1;
  return MLS_OK;
}

mls_status mls_create(const mls_desc *desc, const double *xy, const double *F, int32_t on_device, void *stream,
                      mls_handle **out) {
  mlsi::NvtxRange nvtx_range("mls_create");
  g_err.clear();
  if (!out) return fail(MLS_E_INVAL, "out is NULL");
  *out = nullptr;
  if (!desc || !xy || !F) return fail(MLS_E_INVAL, "desc, xy and F must not be NULL");
  const mls_desc &d = *desc;
  if (d.n < 1 || d.n > ((int64_t)1 << 31) - 1024) return fail(MLS_E_INVAL, "n must be in [1, 2^31 - 1024]");
  if (d.D < 1 || d.D > 256) return fail(MLS_E_INVAL, "D must be in [1, 256]");
  if (d.degree < 0 || d.degree > 2) return fail(MLS_E_INVAL, "degree must be 0, 1 or 2");
  if (d.weight < MLS_W_GAUSS || d.weight > MLS_W_INVDIST) return fail(MLS_E_INVAL, "unknown weight");
  if (d.precision < MLS_P_FP64 || d.precision > MLS_P_FP64_TC) return fail(MLS_E_INVAL, "unknown precision");
  if (!finite_pos(d.h)) return fail(MLS_E_INVAL, "h must be finite and > 0");
  if (d.weight == MLS_W_INVDIST && !finite_pos(d.alpha)) return fail(MLS_E_INVAL, "alpha must be finite and > 0");
  if (!finite_pos(d.cond_fp64)) return fail(MLS_E_INVAL, "cond_fp64 must be > 0");
  if (!(d.rcond_degenerate >= 0.0) || !(d.rcond_degenerate < 1.0))
    return fail(MLS_E_INVAL, "rcond_degenerate must be in [0, 1)");
  if (!(d.cond_recompute >= 0.0)) return fail(MLS_E_INVAL, "cond_recompute must be >= 0");
  if (d.weight_split < -1 || d.weight_split > 2) return fail(MLS_E_INVAL, "weight_split must be -1, 0, 1 or 2");
  if (d.variant < MLS_V_POLY || d.variant > MLS_V_MEAN) return fail(MLS_E_INVAL, "unknown variant");
  if (d.variant != MLS_V_POLY && d.D != 2) return fail(MLS_E_INVAL, "the rigid and mean mappings take D = 2");
  if (!(d.support >= 0.0 && d.support <= 1e6)) return fail(MLS_E_INVAL, "support must be 0 or in (0, 1e6]");
  if (d.support > 0.0 && d.weight != MLS_W_GAUSS)
    return fail(MLS_E_INVAL, "support (the truncated Gaussian) applies to the Gaussian weight only");
  if (d.precision == MLS_P_FP64_TC &&
      (d.weight == MLS_W_INVDIST || d.support > 0.0 || d.variant != MLS_V_POLY))
    return fail(MLS_E_UNSUPPORTED, "MLS_P_FP64_TC takes the full-sum Gaussian and the Wendland weight, "
                                   "polynomial fit only");

  mls_handle *h = new mls_handle();
  h->desc = d;
  if (h->desc.cond_recompute == 0.0) h->desc.cond_recompute = d.precision == MLS_P_BF16 ? 1e2 : 1e3;
  if (h->desc.weight_split < 0) h->desc.weight_split = d.precision == MLS_P_BF16 ? 1 : 2;
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  mls_status s = MLS_OK;
  const double *xy_d = xy, *F_d = F;
  if (!on_device) {
    // one staging block for both inputs
    void *p;
    if ((s = dev_alloc(h, &p, sizeof(double) * d.n * (2 + d.D), st)) != MLS_OK) goto bad;
    xy_d = (const double *)p;
    F_d = xy_d + 2 * d.n;
    {
      cudaError_t e = cudaMemcpyAsync((void *)xy_d, xy, sizeof(double) * 2 * d.n, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)F_d, F, sizeof(double) * d.n * d.D, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) {
        s = cuda_fail(e, "cudaMemcpyAsync (points)");
        goto bad;
      }
    }
  }
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    s = cuda_fail(cudaGetLastError(), "cudaGetDevice");
    goto bad;
  }
  // the events first: prep_points waits once for the device (the point
  // ranges), and host work after that wait leaves the device idle
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaEventCreate(&h->evk0) != cudaSuccess || cudaEventCreate(&h->evk1) != cudaSuccess) {
    s = cuda_fail(cudaGetLastError(), "cudaEventCreate");
    goto bad;
  }
  if ((s = prep_points(h, xy_d, F_d, st)) != MLS_OK) goto bad;
  if (!on_device) {
    // the staging copies of the inputs are not needed once prepared
    release(h, (void *)xy_d, st);
  }
  // host inputs: the copies above have completed, since prep_points waited
  // for the stream after them (the point ranges), so the caller may reuse
  // its buffers without another wait here
  *out = h;
  return MLS_OK;
bad:
  for (void *p : h->owned) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
  cudaGetLastError();
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->evk0) cudaEventDestroy(h->evk0);
  if (h->evk1) cudaEventDestroy(h->evk1);
  delete h;
  return s;
}

}  // extern "C"

namespace mlsi {

// Where a host output of `bytes` bytes lives: page-locked and mapped for the
// handle's device as one range (the kernels may write it directly through
// *dev), pageable (staged in device memory and copied back), or neither: a
// buffer whose first byte is page-locked but whose extent runs past that
// mapped range.  The kernels could reach only the mapped part of such a
// buffer and the copy engines refuse it, so it is rejected.
enum HostKind { HOST_PAGEABLE, HOST_MAPPED, HOST_STRADDLES };

// Largest field written into page-locked host memory by the kernels
// themselves (256 MiB; above it the render is staged and copied).
constexpr size_t kDirectOutMaxBytes = (size_t)256 << 20;

static HostKind host_kind(void *ptr, size_t bytes, int device, void **dev) {
  *dev = nullptr;
  if (!ptr || bytes == 0) return HOST_PAGEABLE;
  cudaPointerAttributes a{}, e{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return HOST_PAGEABLE;
  }
  if (a.type != cudaMemoryTypeHost) return HOST_PAGEABLE;
  const char *last = (const char *)ptr + (bytes - 1);
  if (cudaPointerGetAttributes(&e, last) != cudaSuccess) {
    cudaGetLastError();
    return HOST_STRADDLES;
  }
  if (e.type != cudaMemoryTypeHost || !a.devicePointer || !e.devicePointer ||
      (const char *)e.devicePointer != (const char *)a.devicePointer + (bytes - 1))
    return HOST_STRADDLES;
  if (a.device != device || e.device != device) return HOST_PAGEABLE;   // another device's mapping: stage
  *dev = a.devicePointer;
  return HOST_MAPPED;
}

// Host-side part of a render: validation, scratch, level upload, staging;
// fills the kernel parameters.  Everything here may allocate or synchronise,
// so none of it runs inside a stream capture.
static mls_status render_prepare(mls_handle *h, RenderCtx *c, const mls_view *view, void *field,
                                 uint8_t *status, const double *levels, int32_t L, uint8_t *bands,
                                 int32_t on_device, cudaStream_t st, mlsk::KParams *out) {
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  mls_status s = check_view(view);
  if (s != MLS_OK) return s;
  if (!field) return fail(MLS_E_INVAL, "field is NULL");
  if (bands && (!levels || L < 1) && L != 0) return fail(MLS_E_INVAL, "bands need levels");
  if ((s = check_levels(levels, bands ? L : 0, h->desc.D)) != MLS_OK) return s;
  const int W = view->W, H = view->H;
  const size_t plane = (size_t)W * H;
  const bool fp64 = field_is_fp64(h->desc.precision);
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  if ((s = ensure_scratch(c, W, H, st)) != MLS_OK) return s;
  if (bands && L > 0 && (s = upload_levels(h, c, levels, L, st)) != MLS_OK) return s;
  void *field_d = field;
  uint8_t *status_d = status, *bands_d = bands;
  c->direct_out = false;
  c->copy_out = false;
  if (!on_device) {
    // Page-locked host outputs are written by the kernels directly (over
    // NVLink-C2C on GB300, overlapped with the render); other host memory is
    // staged in device memory and copied back after the render.
    void *fm = nullptr, *sm = nullptr, *bm = nullptr;
    const HostKind fk = host_kind(field, plane * h->desc.D * esz, h->device, &fm);
    const HostKind sk = status ? host_kind(status, plane, h->device, &sm) : HOST_PAGEABLE;
    const HostKind bk = bands ? host_kind(bands, plane * h->desc.D, h->device, &bm) : HOST_PAGEABLE;
    if (fk == HOST_STRADDLES || sk == HOST_STRADDLES || bk == HOST_STRADDLES)
      return fail(MLS_E_INVAL, "a host output starts in page-locked memory but runs past its page-locked "
                               "block; pass it wholly inside one page-locked block, or in pageable memory");
    // Page-locked outputs (all those given).  Small ones are written by the
    // kernels directly, overlapped with the render.  Large ones are rendered
    // into device staging and copied afterwards by a kernel through their
    // device addresses: the hand-over's writes are scattered (one pixel of
    // every dimension plane at a time), and over NVLink-C2C scattered writes
    // of a large render cost more than one coalesced copy.
    const bool mapped = fm && (!status || sm) && (!bands || bm);
    const size_t fbytes = plane * h->desc.D * esz;
    const bool large = h->out_mode == 1 || (h->out_mode == 0 && fbytes > kDirectOutMaxBytes);
    c->direct_out = mapped && !large;
    c->copy_out = mapped && large;
    if (c->direct_out) {
      field_d = fm;
      status_d = (uint8_t *)sm;
      bands_d = (uint8_t *)bm;
    }
    c->out_dev[0] = fm;
    c->out_dev[1] = sm;
    c->out_dev[2] = bm;
  }
  if (!on_device && !c->direct_out) {
    const size_t fbytes = (plane * h->desc.D * esz + 255) / 256 * 256;
    const size_t sbytes = (plane + 255) / 256 * 256;
    const size_t bbytes = bands ? plane * h->desc.D : 0;
    if ((s = ensure_stage(c, fbytes + sbytes + bbytes, st)) != MLS_OK) return s;
    field_d = c->stage;
    status_d = status ? (uint8_t *)c->stage + fbytes : nullptr;
    bands_d = bands ? (uint8_t *)c->stage + fbytes + sbytes : nullptr;
  }
  mlsk::KParams p = base_params(h, c, view);
  p.field = field_d;
  p.field_fp64 = fp64 ? 1 : 0;
  p.status = status_d;
  p.bands = bands_d;
  p.L = bands ? L : 0;
  *out = p;
  return MLS_OK;
}

// Device part of a render: memsets and kernel launches only (capturable in
// a CUDA graph).  With `timing` the handle's events bracket the render and
// its main kernel.  *nlaunch receives the kernels launched.
static mls_status render_enqueue(mls_handle *h, RenderCtx *c, const mlsk::KParams &p, cudaStream_t st,
                                 bool timing, int64_t *nlaunch) {
  mls_status s;
  const size_t plane = (size_t)p.W * p.H;
  const bool fp64 = h->desc.precision == MLS_P_FP64;
  int64_t launches = 0;
  MLS_CUDA_TRY(cudaMemsetAsync(c->scratch, 0, 256, st));
  if (timing) MLS_CUDA_TRY(cudaEventRecord(h->ev0, st));
  if (h->desc.variant != MLS_V_POLY) {
    // the rigid and mean-displacement mappings: one kernel, FP64 for FP64
    // renders and FP32 otherwise
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk0, st));
    launch_variant(p, fp64, st);
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));
    launches += 1;
    h->last_path = MLS_PATH_VARIANT;
  } else if (h->desc.precision == MLS_P_FP64_TC &&
             kTile * fmax(fabs(p.sx), fabs(p.sy)) / h->desc.h > kTileFrameMaxH) {
    // tiles too wide for one moment frame: the FP64 kernel (each pixel in
    // its own frame)
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk0, st));
    h->last_path = MLS_PATH_FP64;
    launch_f64(p, (int64_t)plane, st);
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));
    launches += 1;
  } else if (h->desc.precision == MLS_P_FP64_TC) {
    // FP64-equivalent moments on the tensor cores; pixels whose support count
    // could cross a degree threshold are finished by the FP64 kernel
    launch_prepass(p, st);
    launches += 1;
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk0, st));
    h->last_path = MLS_PATH_FP64_TC;
    int nl = 0;
    mlsk::KParams pt = p;
    pt.visited = c->visited;
    if ((s = launch_tc64(pt, st, &nl)) != MLS_OK) return s;
    launches += nl;
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));
    mlsk::KParams q = p;
    q.list = c->relist;
    q.list_count = c->counters;
    q.list_cap = (int64_t)plane;
    launch_f64(q, 0, st);
    launches += 1;
  } else if (fp64) {
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk0, st));
    h->last_path = MLS_PATH_FP64;
    launch_f64(p, (int64_t)plane, st);
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));
    launches += 1;
  } else {
    launch_prepass(p, st);
    if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk0, st));
    // A 16 x 16 tile much wider than h has no moment frame that suits all
    // its pixels (the tensor path shares one per tile): such renders use the
    // CUDA-core kernel with each pixel in its own frame, at FP32 limits.
    // The inverse-distance weight (Eq. eq-weights) has no finite support or
    // scale for the tile operand's range clip: it also takes this path.
    const double tile_h = kTile * fmax(fabs(p.sx), fabs(p.sy)) / h->desc.h;
    if (tile_h > kTileFrameMaxH || h->desc.precision == MLS_P_FP32 || h->desc.weight == MLS_W_INVDIST) {
      mlsk::KParams pf = p;
      pf.visited = c->visited;
      pf.pixel_frame = tile_h > kTileFrameMaxH ? 1 : 0;
      pf.lambda_max = 1000.f;
      h->last_path = MLS_PATH_FP32;
      launch_f32(pf, st);
      launches += 2;
      if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));
    } else {
      const bool fp16 = h->desc.precision == MLS_P_FP16;
      int nl = 0;
      h->last_path = MLS_PATH_TENSOR;
      if (h->desc.weight_split == 2) {
        // single weights everywhere; the 8-row halves of tiles with a
        // failing pixel are queued and rendered again with split weights
        const int ntile = p.tiles_x * p.tiles_y;
        MLS_CUDA_TRY(cudaMemsetAsync(c->tile_mark, 0, sizeof(int) * 2 * ntile, st));
        mlsk::KParams p1 = p;
        p1.visited = c->visited;
        p1.retry_tiles = c->retry_tiles;
        p1.retry_count = c->counters + 2;
        p1.tile_mark = c->tile_mark;
        if ((s = launch_tc(p1, fp16, 0, st, &nl)) != MLS_OK) return s;
        launches += 1 + nl;
        if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));   // main kernel: the pass over every tile
        mlsk::KParams p2 = p;
        p2.lambda_max = fp16 ? kLambdaSplitFp16 : 50.f;
        p2.tile_list = c->retry_tiles;
        p2.tile_count = c->counters + 2;
        if ((s = launch_tc(p2, fp16, 1, st, &nl)) != MLS_OK) return s;
        launches += nl;
      } else {
        mlsk::KParams p1 = p;
        p1.visited = c->visited;
        if ((s = launch_tc(p1, fp16, h->desc.weight_split, st, &nl)) != MLS_OK) return s;
        launches += 1 + nl;
        if (timing) MLS_CUDA_TRY(cudaEventRecord(h->evk1, st));
      }
    }
    // pixels handed over by the reduced-precision path: centroid-frame
    // recompute, and the FP64 tier for what is left
    const int64_t split_cap = h->ho_cap_limit >= 0 && h->ho_cap_limit < c->ho_cap ? h->ho_cap_limit : c->ho_cap;
    const int64_t least = h->ho_least >= 0 ? h->ho_least : kHandoverSplitLeast;
    launches += launch_handover(p, c->relist, c->counters, (int64_t)plane, split_cap, least, c->ho_state,
                                c->ho_claims, c->relist2, c->counters + 1, st) +
                1;
    mlsk::KParams q = p;
    q.list = c->relist2;
    q.list_count = c->counters + 1;
    q.list_cap = (int64_t)plane;
    q.field_fp64 = 0;
    launch_f64(q, 0, st);
  }
  MLS_CUDA_TRY(cudaGetLastError());
  if (timing) MLS_CUDA_TRY(cudaEventRecord(h->ev1, st));
  h->timed = timing;
  h->last_pairs = (h->desc.weight == MLS_W_WENDLAND) ? 0 : (int64_t)plane * h->desc.n;
  *nlaunch = launches;
  return MLS_OK;
}

}  // namespace mlsi

extern "C" {

mls_status mls_render(mls_handle *h, const mls_view *view, void *field, uint8_t *status, const double *levels,
                      int32_t L, uint8_t *bands, int32_t on_device, void *stream) {
  mlsi::NvtxRange nvtx_range("mls_render");
  g_err.clear();
  cudaStream_t st = (cudaStream_t)stream;
  mlsk::KParams p;
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  mls_status s = render_prepare(h, &h->ctx, view, field, status, levels, L, bands, on_device, st, &p);
  if (s != MLS_OK) return s;
  h->stream = st;
  int64_t nl = 0;
  if ((s = render_enqueue(h, &h->ctx, p, st, true, &nl)) != MLS_OK) return s;
  h->launches += nl;
  if (!on_device) {
    const size_t plane = (size_t)view->W * view->H;
    const size_t esz = field_is_fp64(h->desc.precision) ? sizeof(double) : sizeof(float);
    if (h->ctx.copy_out) {
      launch_copy(h->ctx.out_dev[0], p.field, plane * h->desc.D * esz, st);
      if (status) launch_copy(h->ctx.out_dev[1], p.status, plane, st);
      if (bands) launch_copy(h->ctx.out_dev[2], p.bands, plane * h->desc.D, st);
      MLS_CUDA_TRY(cudaGetLastError());
    } else if (!h->ctx.direct_out) {
      MLS_CUDA_TRY(cudaMemcpyAsync(field, p.field, plane * h->desc.D * esz, cudaMemcpyDeviceToHost, st));
      if (status) MLS_CUDA_TRY(cudaMemcpyAsync(status, p.status, plane, cudaMemcpyDeviceToHost, st));
      if (bands) MLS_CUDA_TRY(cudaMemcpyAsync(bands, p.bands, plane * h->desc.D, cudaMemcpyDeviceToHost, st));
    }
    MLS_CUDA_TRY(cudaStreamSynchronize(st));
    int err = 0;
    MLS_CUDA_TRY(cudaMemcpy(&err, h->ctx.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err >= mlsk::ERR_INDEX)
      return fail(MLS_E_CUDA, "checked build: a kernel index lay outside its array (site " +
                                  std::to_string(err - mlsk::ERR_INDEX) + ")");
    if (err) return fail(MLS_E_TIMEOUT, "a bounded device wait gave up (error word " + std::to_string(err) + ")");
  }
  return MLS_OK;
}

mls_status mls_bands(mls_handle *h, const mls_view *view, const void *field, const double *levels, int32_t L,
                     uint8_t *bands, int32_t on_device, void *stream) {
  mlsi::NvtxRange nvtx_range("mls_bands");
  g_err.clear();
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  mls_status s = check_view(view);
  if (s != MLS_OK) return s;
  if (!field || !bands) return fail(MLS_E_INVAL, "field and bands must not be NULL");
  if ((s = check_levels(levels, L, h->desc.D)) != MLS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  const size_t plane = (size_t)view->W * view->H;
  const bool fp64 = field_is_fp64(h->desc.precision);
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  if ((s = ensure_scratch(&h->ctx, view->W, view->H, st)) != MLS_OK) return s;
  if (L > 0 && (s = upload_levels(h, &h->ctx, levels, L, st)) != MLS_OK) return s;
  const void *field_d = field;
  uint8_t *bands_d = bands;
  if (!on_device) {
    const size_t fbytes = (plane * h->desc.D * esz + 255) / 256 * 256;
    if ((s = ensure_stage(&h->ctx, fbytes + plane * h->desc.D, st)) != MLS_OK) return s;
    field_d = h->ctx.stage;
    bands_d = (uint8_t *)h->ctx.stage + fbytes;
    MLS_CUDA_TRY(cudaMemcpyAsync((void *)field_d, field, plane * h->desc.D * esz, cudaMemcpyHostToDevice, st));
  }
  mlsk::KParams p = base_params(h, &h->ctx, view);
  p.field = (void *)field_d;
  p.field_fp64 = fp64 ? 1 : 0;
  p.bands = bands_d;
  p.L = L;
  launch_bands(p, fp64, st);
  MLS_CUDA_TRY(cudaGetLastError());
  if (!on_device) {
    MLS_CUDA_TRY(cudaMemcpyAsync(bands, bands_d, plane * h->desc.D, cudaMemcpyDeviceToHost, st));
    MLS_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return MLS_OK;
}

mls_status mls_sync(mls_handle *h, double timeout_s, mls_stats *stats) {
  mlsi::NvtxRange nvtx_range("mls_sync");
  g_err.clear();
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  if (!(timeout_s > 0.0)) return fail(MLS_E_INVAL, "timeout_s must be > 0");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(h->stream);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_s) return fail(MLS_E_TIMEOUT, "stream did not finish within the watchdog time");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  unsigned int cnt[3] = {0, 0, 0};
  unsigned long long visited = 0;
  int err = 0;
  if (h->ctx.scratch) {
    MLS_CUDA_TRY(cudaMemcpy(cnt, h->ctx.counters, sizeof cnt, cudaMemcpyDeviceToHost));
    MLS_CUDA_TRY(cudaMemcpy(&visited, h->ctx.visited, sizeof visited, cudaMemcpyDeviceToHost));
    MLS_CUDA_TRY(cudaMemcpy(&err, h->ctx.err, sizeof err, cudaMemcpyDeviceToHost));
  }
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->pairs = visited ? (int64_t)visited : h->last_pairs;
    stats->recomputed = cnt[0];
    stats->recomputed_fp64 = cnt[1];
    stats->retried_tiles = cnt[2];
    stats->device_error = err;
    float ms = 0.f;
    if (h->timed && cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) stats->last_render_ms = ms;
    if (h->timed && cudaEventElapsedTime(&ms, h->evk0, h->evk1) == cudaSuccess) stats->main_kernel_ms = ms;
    stats->launches = h->launches;
    stats->main_path = h->last_path;
    cudaGetLastError();
  }
  if (err >= mlsk::ERR_INDEX)
    return fail(MLS_E_CUDA, "checked build: a kernel index lay outside its array (site " +
                                std::to_string(err - mlsk::ERR_INDEX) + ")");
  if (err) return fail(MLS_E_TIMEOUT, "a bounded device wait gave up (error word " + std::to_string(err) + ")");
  return MLS_OK;
}

int mls_debug_operand_cut(mls_handle *h, int32_t on) {
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  h->operand_cut = on != 0;
  return MLS_OK;
}

int mls_debug_host_output(mls_handle *h, int32_t mode) {
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  if (mode < 0 || mode > 2) return fail(MLS_E_INVAL, "mode must be 0, 1 or 2");
  h->out_mode = mode;
  return MLS_OK;
}

int mls_debug_handover_split(mls_handle *h, int64_t cap, int64_t least) {
  if (!h) return fail(MLS_E_INVAL, "handle is NULL");
  if (cap < -1 || least < -1) return fail(MLS_E_INVAL, "cap and least must be -1 or >= 0");
  h->ho_cap_limit = cap;
  h->ho_least = least;
  return MLS_OK;
}

mls_status mls_destroy(mls_handle *h) {
  mlsi::NvtxRange nvtx_range("mls_destroy");
  g_err.clear();
  if (!h) return MLS_OK;
  cudaStream_t st = h->stream;
  cudaStreamSynchronize(st);
  for (void *p : h->owned) cudaFreeAsync(p, st);
  ctx_free_all(&h->ctx, st);
  cudaStreamSynchronize(st);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->evk0) cudaEventDestroy(h->evk0);
  if (h->evk1) cudaEventDestroy(h->evk1);
  cudaGetLastError();
  delete h;
  return MLS_OK;
}


// ---------------------------------------------------------------------------
// Batches: many resident datasets rendered by one CUDA graph.

}  // extern "C"

struct mls_batch {
  std::vector<mls_handle *> hs;
  int flags = 0;
  cudaStream_t origin = nullptr;          // capture origin, level uploads
  std::vector<cudaStream_t> child;        // one branch per dataset
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> sig;              // what the captured graph was built for
  std::vector<int64_t> nl;                // kernels per dataset per render
  cudaStream_t last = nullptr;
  bool timed = false, tuned = false;
  int64_t captures = 0, replays = 0;
};

namespace mlsi {

static void batch_free(mls_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t c : b->child)
    if (c) cudaStreamDestroy(c);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->origin) cudaStreamDestroy(b->origin);
  cudaGetLastError();
  delete b;
}

static void sig_push(std::vector<uint64_t> &v, const void *p) { v.push_back((uint64_t)(uintptr_t)p); }
static void sig_push(std::vector<uint64_t> &v, double d) {
  uint64_t u;
  memcpy(&u, &d, sizeof u);
  v.push_back(u);
}

// Autotuner: for each tensor-precision dataset, time split weights everywhere
// (1) against the two-pass scheme (2) on the actual view and keep the faster.
// Both meet the same error bound; which is faster depends on how many tiles
// the single-weight pass queues.
static mls_status batch_tune(mls_batch *b, const mls_view *views, void *const *fields, uint8_t *const *status,
                             const double *const *levels, const int32_t *L, uint8_t *const *bands) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  mls_status s = MLS_OK;
  // time one render of dataset k as it is configured now (the first run warms up)
  auto time_render = [&](size_t k, float *ms) -> mls_status {
    mls_handle *h = b->hs[k];
    mlsk::KParams p;
    mls_status r = render_prepare(h, &h->ctx, &views[k], fields[k], status ? status[k] : nullptr,
                                  levels ? levels[k] : nullptr, L ? L[k] : 0, bands ? bands[k] : nullptr, 1,
                                  b->origin, &p);
    float t = 0.f;
    for (int rep = 0; rep < 2 && r == MLS_OK; ++rep) {
      int64_t nl = 0;
      if (cudaEventRecord(e0, b->origin) != cudaSuccess) r = cuda_fail(cudaGetLastError(), "cudaEventRecord");
      if (r == MLS_OK) r = render_enqueue(h, &h->ctx, p, b->origin, false, &nl);
      if (r == MLS_OK && cudaEventRecord(e1, b->origin) != cudaSuccess)
        r = cuda_fail(cudaGetLastError(), "cudaEventRecord");
      if (r == MLS_OK && cudaEventSynchronize(e1) != cudaSuccess)
        r = cuda_fail(cudaGetLastError(), "cudaEventSynchronize");
      if (r == MLS_OK) cudaEventElapsedTime(&t, e0, e1);
      h->launches += nl;
    }
    *ms = t;
    return r;
  };
  for (size_t k = 0; k < b->hs.size() && s == MLS_OK; ++k) {
    // renders on the FP32 kernel (FP32 precision, tiles wider than 4 h): its
    // block shape, for the Gaussian
    mls_handle *h = b->hs[k];
    const mls_view &v = views[k];
    const double tile_h = kTile * fmax(fabs((v.x1 - v.x0) / v.W), fabs((v.y1 - v.y0) / v.H)) / h->desc.h;
    const bool f32_route = h->desc.variant == MLS_V_POLY && h->desc.weight == MLS_W_GAUSS &&
                           (h->desc.precision == MLS_P_FP32 ||
                            ((h->desc.precision == MLS_P_FP16 || h->desc.precision == MLS_P_BF16) &&
                             tile_h > kTileFrameMaxH));
    if (!f32_route) continue;
    float best = 1e30f;
    int best_shape = 0;
    for (int shape = 0; shape <= 2 && s == MLS_OK; ++shape) {
      h->f32_shape = shape;
      float t = 0.f;
      s = time_render(k, &t);
      if (s == MLS_OK && t < best) {
        best = t;
        best_shape = shape;
      }
    }
    h->f32_shape = best_shape;
  }
  for (size_t k = 0; k < b->hs.size() && s == MLS_OK; ++k) {
    mls_handle *h = b->hs[k];
    if (h->desc.precision != MLS_P_FP16 && h->desc.precision != MLS_P_BF16) continue;
    float best = 1e30f;
    int best_ws = h->desc.weight_split;
    for (int ws = 1; ws <= 2 && s == MLS_OK; ++ws) {
      h->desc.weight_split = ws;
      mlsk::KParams p;
      s = render_prepare(h, &h->ctx, &views[k], fields[k], status ? status[k] : nullptr, levels ? levels[k] : nullptr,
                         L ? L[k] : 0, bands ? bands[k] : nullptr, 1, b->origin, &p);
      float t = 0.f;
      for (int rep = 0; rep < 2 && s == MLS_OK; ++rep) {   // the first run warms up
        int64_t nl = 0;
        if (cudaEventRecord(e0, b->origin) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
        if (s == MLS_OK) s = render_enqueue(h, &h->ctx, p, b->origin, false, &nl);
        if (s == MLS_OK && cudaEventRecord(e1, b->origin) != cudaSuccess)
          s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
        if (s == MLS_OK && cudaEventSynchronize(e1) != cudaSuccess)
          s = cuda_fail(cudaGetLastError(), "cudaEventSynchronize");
        if (s == MLS_OK) cudaEventElapsedTime(&t, e0, e1);
        h->launches += nl;
      }
      if (s == MLS_OK && t < best) {
        best = t;
        best_ws = ws;
      }
    }
    h->desc.weight_split = best_ws;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // namespace mlsi

extern "C" {

mls_status mls_batch_create(int32_t count, mls_handle *const *handles, int32_t flags, mls_batch **out) {
  mlsi::NvtxRange nvtx_range("mls_batch_create");
  g_err.clear();
  if (!out) return fail(MLS_E_INVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || count > 4096 || !handles) return fail(MLS_E_INVAL, "count must be in [1, 4096] with handles");
  if (flags & ~MLS_BATCH_AUTOTUNE) return fail(MLS_E_INVAL, "unknown batch flags");
  int dev = -1;
  for (int k = 0; k < count; ++k) {
    if (!handles[k]) return fail(MLS_E_INVAL, "a handle is NULL");
    for (int j = 0; j < k; ++j)
      if (handles[j] == handles[k]) return fail(MLS_E_INVAL, "a handle appears twice in the batch");
    if (dev >= 0 && handles[k]->device != dev) return fail(MLS_E_INVAL, "handles live on different devices");
    dev = handles[k]->device;
  }
  mls_batch *b = new mls_batch;
  b->hs.assign(handles, handles + count);
  b->flags = flags;
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreate(&b->ev0) == cudaSuccess && cudaEventCreate(&b->ev1) == cudaSuccess;
  b->child.assign(count, nullptr);
  b->join.assign(count, nullptr);
  for (int k = 0; k < count && ok; ++k)
    ok = cudaStreamCreateWithFlags(&b->child[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    mls_status s = cuda_fail(cudaGetLastError(), "batch streams and events");
    batch_free(b);
    return s;
  }
  *out = b;
  return MLS_OK;
}

mls_status mls_batch_render(mls_batch *b, const mls_view *views, void *const *fields, uint8_t *const *status,
                            const double *const *levels, const int32_t *L, uint8_t *const *bands, void *stream) {
  mlsi::NvtxRange nvtx_range("mls_batch_render");
  g_err.clear();
  if (!b || !views || !fields) return fail(MLS_E_INVAL, "batch, views and fields must not be NULL");
  const size_t n = b->hs.size();
  cudaStream_t st = (cudaStream_t)stream;
  // host preparation is ordered after the previous batch render
  if (b->timed) MLS_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev1, 0));
  mls_status s;
  if ((b->flags & MLS_BATCH_AUTOTUNE) && !b->tuned) {
    if ((s = batch_tune(b, views, fields, status, levels, L, bands)) != MLS_OK) return s;
    b->tuned = true;
  }
  std::vector<mlsk::KParams> ps(n);
  std::vector<uint64_t> sig;
  for (size_t k = 0; k < n; ++k) {
    mls_handle *h = b->hs[k];
    s = render_prepare(h, &h->ctx, &views[k], fields[k], status ? status[k] : nullptr, levels ? levels[k] : nullptr,
                       L ? L[k] : 0, bands ? bands[k] : nullptr, 1, b->origin, &ps[k]);
    if (s != MLS_OK) return fail(s, "dataset " + std::to_string(k) + ": " + g_err);
    const mls_view &v = views[k];
    sig.push_back(((uint64_t)(uint32_t)v.W << 32) | (uint32_t)v.H);
    sig_push(sig, v.x0);
    sig_push(sig, v.y0);
    sig_push(sig, v.x1);
    sig_push(sig, v.y1);
    sig_push(sig, ps[k].field);
    sig_push(sig, (const void *)ps[k].status);
    sig_push(sig, (const void *)ps[k].bands);
    sig.push_back((uint64_t)ps[k].L);
    sig_push(sig, h->ctx.scratch);
    sig_push(sig, (const void *)h->ctx.lev64);
    sig_push(sig, (const void *)h->ctx.lev32);
    sig.push_back((uint64_t)h->desc.weight_split);
  }
  // every upload has landed before the graph reads it
  MLS_CUDA_TRY(cudaStreamSynchronize(b->origin));
  if (!b->exec || sig != b->sig) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->nl.assign(n, 0);
    MLS_CUDA_TRY(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
    mls_status cs = MLS_OK;
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) cs = cuda_fail(cudaGetLastError(), "fork");
    for (size_t k = 0; k < n && cs == MLS_OK; ++k) {
      if (cudaStreamWaitEvent(b->child[k], b->fork, 0) != cudaSuccess) {
        cs = cuda_fail(cudaGetLastError(), "branch");
        break;
      }
      cs = render_enqueue(b->hs[k], &b->hs[k]->ctx, ps[k], b->child[k], false, &b->nl[k]);
      if (cs == MLS_OK && (cudaEventRecord(b->join[k], b->child[k]) != cudaSuccess ||
                           cudaStreamWaitEvent(b->origin, b->join[k], 0) != cudaSuccess))
        cs = cuda_fail(cudaGetLastError(), "join");
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->origin, &g);
    if (cs != MLS_OK) {
      if (g) cudaGraphDestroy(g);
      return cs;
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
    b->graph = g;
    MLS_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->sig = sig;
    ++b->captures;
  }
  MLS_CUDA_TRY(cudaEventRecord(b->ev0, st));
  MLS_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  MLS_CUDA_TRY(cudaEventRecord(b->ev1, st));
  ++b->replays;
  b->last = st;
  b->timed = true;
  for (size_t k = 0; k < n; ++k) {
    b->hs[k]->stream = st;
    b->hs[k]->launches += b->nl[k];
  }
  return MLS_OK;
}

mls_status mls_batch_sync(mls_batch *b, double timeout_s, mls_batch_stats *stats) {
  mlsi::NvtxRange nvtx_range("mls_batch_sync");
  g_err.clear();
  if (!b) return fail(MLS_E_INVAL, "batch is NULL");
  const auto t0 = std::chrono::steady_clock::now();
  if (b->timed) {
    for (;;) {
      const cudaError_t e = cudaEventQuery(b->ev1);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return fail(MLS_E_TIMEOUT, "batch did not finish within the watchdog time");
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  mls_batch_stats bs;
  memset(&bs, 0, sizeof bs);
  bs.datasets = (int64_t)b->hs.size();
  int first_err = 0;
  for (size_t k = 0; k < b->hs.size(); ++k) {
    mls_handle *h = b->hs[k];
    unsigned int cnt[3] = {0, 0, 0};
    int err = 0;
    if (h->ctx.scratch) {
      MLS_CUDA_TRY(cudaMemcpy(cnt, h->ctx.counters, sizeof cnt, cudaMemcpyDeviceToHost));
      MLS_CUDA_TRY(cudaMemcpy(&err, h->ctx.err, sizeof err, cudaMemcpyDeviceToHost));
    }
    bs.pairs += h->last_pairs;
    bs.recomputed += cnt[0];
    if (err && !first_err) first_err = err;
    if (k < b->nl.size()) bs.launches += b->nl[k];
  }
  bs.device_error = first_err;
  bs.captures = b->captures;
  bs.replays = b->replays;
  float ms = 0.f;
  if (b->timed && cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) bs.last_render_ms = ms;
  cudaGetLastError();
  if (stats) *stats = bs;
  if (first_err) return fail(MLS_E_TIMEOUT, "a bounded device wait gave up in the batch");
  return MLS_OK;
}

mls_status mls_batch_destroy(mls_batch *b) {
  mlsi::NvtxRange nvtx_range("mls_batch_destroy");
  g_err.clear();
  if (!b) return MLS_OK;
  if (b->timed) cudaEventSynchronize(b->ev1);
  cudaStreamSynchronize(b->origin);
  batch_free(b);
  return MLS_OK;
}


// ---------------------------------------------------------------------------
// Serving: a worker thread, a FIFO of requests, a pool of stream slots and a
// device-memory budget.

}  // extern "C"

namespace mlsi {

using Clock = std::chrono::steady_clock;

struct ServeReq {
  int64_t id;
  mls_request r;
  std::vector<double> levels;        // copied at submit
  int64_t footprint;
  Clock::time_point t_submit, t_admit;
};

struct ServeSlot {
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool busy = false;
  ServeReq req;
  RenderCtx ctx;
  void *out = nullptr;               // device outputs of the request
};

}  // namespace mlsi

struct mls_server {
  mls_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<mlsi::ServeReq> queue;
  std::vector<mlsi::ServeSlot> slots;
  std::vector<mls_request_done> done;
  int64_t next_id = 1, submitted = 0, completed = 0, failed = 0;
  int64_t inflight = 0, bytes = 0, peak_inflight = 0, peak_bytes = 0;
  bool stop = false;
  std::thread worker;
};

namespace mlsi {

static size_t out_bytes(const mls_handle *h, const mls_view &v, size_t *fbytes, size_t *sbytes) {
  const size_t plane = (size_t)v.W * v.H;
  const size_t esz = field_is_fp64(h->desc.precision) ? sizeof(double) : sizeof(float);
  *fbytes = (plane * h->desc.D * esz + 255) / 256 * 256;
  *sbytes = (plane + 255) / 256 * 256;
  return *fbytes + *sbytes + plane * h->desc.D;
}

static int64_t footprint(const mls_request &r) {
  size_t fb, sb;
  return (int64_t)(scratch_bytes_for(r.view.W, r.view.H) + out_bytes(r.dataset, r.view, &fb, &sb) +
                   (size_t)r.dataset->desc.D * r.L * (sizeof(double) + sizeof(float)) + 4096);
}

// Start an admitted request on its slot (worker thread).
static mls_status serve_start(ServeSlot &sl) {
  mls_request &r = sl.req.r;
  mls_handle *h = r.dataset;
  size_t fbytes, sbytes;
  const size_t ob = out_bytes(h, r.view, &fbytes, &sbytes);
  mls_status s = ctx_alloc(&sl.ctx, &sl.out, ob, sl.st);
  if (s != MLS_OK) return s;
  char *o = (char *)sl.out;
  void *field_d = o;
  uint8_t *status_d = (uint8_t *)(o + fbytes);
  uint8_t *bands_d = r.L > 0 ? (uint8_t *)(o + fbytes + sbytes) : nullptr;
  mlsk::KParams p;
  s = render_prepare(h, &sl.ctx, &r.view, field_d, status_d, r.L > 0 ? sl.req.levels.data() : nullptr, r.L,
                     bands_d, 1, sl.st, &p);
  if (s != MLS_OK) return s;
  MLS_CUDA_TRY(cudaEventRecord(sl.e0, sl.st));
  int64_t nl = 0;
  if ((s = render_enqueue(h, &sl.ctx, p, sl.st, false, &nl)) != MLS_OK) return s;
  const size_t plane = (size_t)r.view.W * r.view.H;
  const size_t esz = field_is_fp64(h->desc.precision) ? sizeof(double) : sizeof(float);
  if (r.field) MLS_CUDA_TRY(cudaMemcpyAsync(r.field, field_d, plane * h->desc.D * esz, cudaMemcpyDeviceToHost, sl.st));
  if (r.status) MLS_CUDA_TRY(cudaMemcpyAsync(r.status, status_d, plane, cudaMemcpyDeviceToHost, sl.st));
  if (r.bands && bands_d)
    MLS_CUDA_TRY(cudaMemcpyAsync(r.bands, bands_d, plane * h->desc.D, cudaMemcpyDeviceToHost, sl.st));
  MLS_CUDA_TRY(cudaEventRecord(sl.e1, sl.st));
  return MLS_OK;
}

static void serve_finish(mls_server *sv, ServeSlot &sl, mls_status st) {
  mls_request_done d;
  memset(&d, 0, sizeof d);
  d.id = sl.req.id;
  int err = 0;
  if (st == MLS_OK && sl.ctx.err && cudaMemcpy(&err, sl.ctx.err, sizeof err, cudaMemcpyDeviceToHost) == cudaSuccess &&
      err)
    st = MLS_E_TIMEOUT;
  float ms = 0.f;
  if (st == MLS_OK && cudaEventElapsedTime(&ms, sl.e0, sl.e1) == cudaSuccess) d.device_ms = ms;
  const auto now = Clock::now();
  d.status = st;
  d.latency_ms = std::chrono::duration<double, std::milli>(now - sl.req.t_submit).count();
  d.queued_ms = std::chrono::duration<double, std::milli>(sl.req.t_admit - sl.req.t_submit).count();
  d.footprint = sl.req.footprint;
  ctx_free_all(&sl.ctx, sl.st);
  sl.out = nullptr;
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->done.push_back(d);
  ++sv->completed;
  if (st != MLS_OK) ++sv->failed;
  --sv->inflight;
  sv->bytes -= sl.req.footprint;
  sl.busy = false;
  sv->cv.notify_all();
}

static void serve_loop(mls_server *sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    // completions
    bool any_busy = false;
    for (ServeSlot &sl : sv->slots) {
      if (!sl.busy) continue;
      const cudaError_t e = cudaEventQuery(sl.e1);
      if (e == cudaSuccess) serve_finish(sv, sl, MLS_OK);
      else if (e != cudaErrorNotReady) serve_finish(sv, sl, cuda_fail(e, "request"));
      else any_busy = true;
    }
    // admissions: FIFO head while a slot and the memory budget allow
    for (;;) {
      ServeSlot *free_slot = nullptr;
      ServeReq req;
      {
        std::unique_lock<std::mutex> lk(sv->mu);
        if (sv->queue.empty()) break;
        for (ServeSlot &sl : sv->slots)
          if (!sl.busy) {
            free_slot = &sl;
            break;
          }
        if (!free_slot || sv->bytes + sv->queue.front().footprint > sv->cfg.mem_budget) break;
        req = std::move(sv->queue.front());
        sv->queue.pop_front();
        ++sv->inflight;
        sv->bytes += req.footprint;
        sv->peak_inflight = std::max(sv->peak_inflight, sv->inflight);
        sv->peak_bytes = std::max(sv->peak_bytes, sv->bytes);
        free_slot->busy = true;
      }
      req.t_admit = Clock::now();
      free_slot->req = std::move(req);
      const mls_status st = serve_start(*free_slot);
      if (st != MLS_OK) {
        cudaStreamSynchronize(free_slot->st);
        serve_finish(sv, *free_slot, st);
      } else {
        any_busy = true;
      }
    }
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (sv->stop && sv->queue.empty() && sv->inflight == 0) break;
      if (!any_busy && sv->queue.empty() && !sv->stop) {
        sv->cv.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace mlsi

extern "C" {

mls_status mls_server_create(const mls_server_config *cfg, mls_server **out) {
  mlsi::NvtxRange nvtx_range("mls_server_create");
  g_err.clear();
  if (!out || !cfg) return fail(MLS_E_INVAL, "cfg and out must not be NULL");
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 64) return fail(MLS_E_INVAL, "slots must be in [1, 64]");
  if (cfg->mem_budget < (1 << 20)) return fail(MLS_E_INVAL, "mem_budget must be at least 1 MiB");
  mls_server *sv = new mls_server;
  sv->cfg = *cfg;
  MLS_CUDA_TRY(cudaGetDevice(&sv->device));
  sv->slots.resize(cfg->slots);
  bool ok = true;
  for (ServeSlot &sl : sv->slots)
    ok = ok && cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&sl.e0) == cudaSuccess && cudaEventCreate(&sl.e1) == cudaSuccess;
  if (!ok) {
    mls_status s = cuda_fail(cudaGetLastError(), "server streams");
    for (ServeSlot &sl : sv->slots) {
      if (sl.st) cudaStreamDestroy(sl.st);
      if (sl.e0) cudaEventDestroy(sl.e0);
      if (sl.e1) cudaEventDestroy(sl.e1);
    }
    delete sv;
    return s;
  }
  // freed request memory stays in the stream-ordered pool for the next one
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
    uint64_t keep = (uint64_t)cfg->mem_budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  sv->worker = std::thread(serve_loop, sv);
  *out = sv;
  return MLS_OK;
}

mls_status mls_server_submit(mls_server *sv, const mls_request *req, int64_t *id) {
  mlsi::NvtxRange nvtx_range("mls_server_submit");
  g_err.clear();
  if (!sv || !req || !id) return fail(MLS_E_INVAL, "server, request and id must not be NULL");
  if (!req->dataset) return fail(MLS_E_INVAL, "request has no dataset");
  mls_status s = check_view(&req->view);
  if (s != MLS_OK) return s;
  if ((s = check_levels(req->levels, req->L, req->dataset->desc.D)) != MLS_OK) return s;
  if (req->bands && req->L < 1) return fail(MLS_E_INVAL, "bands need levels");
  ServeReq q;
  q.r = *req;
  if (req->L > 0) q.levels.assign(req->levels, req->levels + (size_t)req->dataset->desc.D * req->L);
  q.r.levels = nullptr;
  q.footprint = footprint(*req);
  if (q.footprint > sv->cfg.mem_budget)
    return fail(MLS_E_NOMEM, "request needs " + std::to_string(q.footprint) + " device bytes, more than the budget");
  q.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    q.id = sv->next_id++;
    *id = q.id;
    ++sv->submitted;
    sv->queue.push_back(std::move(q));
  }
  sv->cv.notify_all();
  return MLS_OK;
}

mls_status mls_server_poll(mls_server *sv, mls_request_done *done, int32_t cap, int32_t *n) {
  g_err.clear();
  if (!sv || !n || (cap > 0 && !done)) return fail(MLS_E_INVAL, "server, done and n must not be NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  const int32_t k = (int32_t)std::min<size_t>((size_t)std::max(cap, 0), sv->done.size());
  for (int32_t i = 0; i < k; ++i) done[i] = sv->done[i];
  sv->done.erase(sv->done.begin(), sv->done.begin() + k);
  *n = k;
  return MLS_OK;
}

mls_status mls_server_drain(mls_server *sv, double timeout_s, mls_server_stats *stats) {
  mlsi::NvtxRange nvtx_range("mls_server_drain");
  g_err.clear();
  if (!sv) return fail(MLS_E_INVAL, "server is NULL");
  const auto t0 = Clock::now();
  std::unique_lock<std::mutex> lk(sv->mu);
  while (sv->completed < sv->submitted) {
    if (std::chrono::duration<double>(Clock::now() - t0).count() > timeout_s)
      return fail(MLS_E_TIMEOUT, "requests did not complete within the watchdog time");
    sv->cv.wait_for(lk, std::chrono::milliseconds(2));
  }
  if (stats) {
    stats->submitted = sv->submitted;
    stats->completed = sv->completed;
    stats->failed = sv->failed;
    stats->peak_inflight = sv->peak_inflight;
    stats->peak_bytes = sv->peak_bytes;
  }
  return MLS_OK;
}

mls_status mls_server_destroy(mls_server *sv) {
  mlsi::NvtxRange nvtx_range("mls_server_destroy");
  g_err.clear();
  if (!sv) return MLS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (ServeSlot &sl : sv->slots) {
    cudaStreamSynchronize(sl.st);
    ctx_free_all(&sl.ctx, sl.st);
    cudaStreamSynchronize(sl.st);
    cudaStreamDestroy(sl.st);
    cudaEventDestroy(sl.e0);
    cudaEventDestroy(sl.e1);
  }
  cudaGetLastError();
  delete sv;
  return MLS_OK;
}

}  // extern "C"
