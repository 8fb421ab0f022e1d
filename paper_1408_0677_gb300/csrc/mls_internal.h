// Host-side internals of the MLS library: the handle and the launchers that
// each CUDA translation unit exports to the C ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dev_common.cuh"
#include "mls.h"

namespace mlsi {

constexpr int kTile = 16;            // tensor / prepass tile side (pixels)
constexpr int kPointPad = 64;        // points are padded to a multiple of this

struct PointSet {
  int64_t n = 0, n_pad = 0;
  int D = 0, D_pad = 0;
  double s = 1.0, ctr_x = 0.0, ctr_y = 0.0;
  double bbox[4] = {0, 0, 0, 0};     // xmin, ymin, xmax, ymax
  double *x64 = nullptr, *y64 = nullptr, *FT64 = nullptr;
  float *xs = nullptr, *ys = nullptr, *FT32 = nullptr;
  float *FR32 = nullptr;             // point-major normalised values (reduced-precision renders)
  float *FR32lo = nullptr;           // their low parts (FR32 + FR32lo: the values to ~48 bits)
  float *xs_lo = nullptr, *ys_lo = nullptr;
  double *fcen = nullptr, *fscl = nullptr;
  float *fcen32 = nullptr, *fscl32 = nullptr;
  float *xyb = nullptr, *fb = nullptr;   // point-blocked layouts of the tensor path
  int fb_dc = 0;
  int *cell_start = nullptr;
  int gx = 0, gy = 0;
  double gx0 = 0, gy0 = 0, cell = 0;
};

// Per-render device scratch: the stabiliser and counts of the padded tile
// grid, hand-over lists, tile frames and queue, counters and error word, the
// uploaded levels and a staging area for host-pointer calls.  A handle owns
// one for its own renders; the server gives every request in flight its own,
// so renders of one resident dataset can overlap.
struct RenderCtx {
  std::vector<void *> owned;         // allocations of this context
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  float *mstab = nullptr;
  int *cnt = nullptr;
  int *relist = nullptr;
  int *relist2 = nullptr;            // pixels the hand-over path passes to FP64
  float *tcen = nullptr;             // per-tile moment frame centres
  unsigned int *counters = nullptr;  // [0] recompute count, [1] FP64 count, [2] retried half tiles
  unsigned int *ho_claims = nullptr; // [0], [1]: entries claimed by the split hand-over's warp kernels
  void *ho_state = nullptr;          // per-entry state of the split hand-over
  int64_t ho_cap = 0;                // its capacity in entries
  int *tile_mark = nullptr;          // per half tile: queued for the split-weight pass
  int *retry_tiles = nullptr;
  float *tmax = nullptr;             // per-tile largest stabiliser (Gaussian)
  unsigned long long *visited = nullptr;   // pixel-point pairs the main kernel visited
  int *err = nullptr;
  double *lev64 = nullptr;
  float *lev32 = nullptr;
  size_t lev_cap = 0;
  void *stage = nullptr;             // staging for host-pointer calls
  size_t stage_bytes = 0;
  bool direct_out = false;           // host outputs written by the kernels themselves
  bool copy_out = false;             // page-locked host outputs filled from the staging by a copy kernel
  void *out_dev[3] = {nullptr, nullptr, nullptr};   // their device addresses (field, status, bands)
};

// Bytes of the scratch a W x H render needs (see ensure_scratch).
size_t scratch_bytes_for(int W, int H);

}  // namespace mlsi

struct mls_handle {
  mls_desc desc;
  int device = 0;
  cudaStream_t stream = nullptr;     // stream of the last call
  mlsi::PointSet P;
  std::vector<void *> owned;         // handle-lifetime device allocations
  mlsi::RenderCtx ctx;               // scratch of mls_render / mls_bands on this handle
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk0 = nullptr, evk1 = nullptr;
  int64_t launches = 0;              // kernels launched by this handle
  int64_t last_pairs = 0;
  int32_t last_path = 0;   // MLS_PATH_* of the last render's main pass
  int32_t f32_shape = 0;   // FP32 kernel block shape (the batch autotuner may change it)
  bool timed = false;
  bool operand_cut = true;           // reduced-precision Gaussian: skip pairs whose weight rounds to zero
  int64_t ho_cap_limit = -1;         // test hooks: split hand-over capacity limit (-1: none)
  int64_t ho_least = -1;             // and shortest list it takes (-1: kHandoverSplitLeast)
  int32_t out_mode = 0;              // test hook: page-locked outputs 0 by size, 1 staged + copy, 2 direct
};

namespace mlsi {

// prep.cu
mls_status prep_points(mls_handle *h, const double *xy_dev, const double *F_dev, cudaStream_t st);
// prepass.cu: stabiliser m = min r^2 (Gaussian, inverse distance) or support
// counts (Wendland) over the padded tile grid
void launch_prepass(const mlsk::KParams &p, cudaStream_t st);
// plain.cu
void launch_f32(const mlsk::KParams &p, cudaStream_t st);
void launch_f64(const mlsk::KParams &p, int64_t npix, cudaStream_t st);
void launch_bands(const mlsk::KParams &p, bool fp64, cudaStream_t st);
// device-to-host copy by a kernel (dst: page-locked host memory's device address)
void launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st);
// rigid / mean-displacement mappings (KParams.variant), FP64 or FP32
void launch_variant(const mlsk::KParams &p, bool fp64, cudaStream_t st);
// handover.cu: ill-conditioned pixels of the reduced-precision renders
// (a list of at least `least` entries: its first min(count, split_cap)
// entries through four kernels whose per-entry state, handover_entry_bytes()
// each, is at `state`, with two zeroed claim counters at `claims`; shorter
// lists and the rest through one fused kernel)
// Returns the kernels launched.
int launch_handover(const mlsk::KParams &p, const int *list, const unsigned int *cnt, int64_t cap,
                    int64_t split_cap, int64_t least, void *state, unsigned int *claims, int *list2,
                    unsigned int *cnt2, cudaStream_t st);
// the shortest list the split kernels take: one chunk of 32 pixels for each
// of the fused kernel's 608 blocks (below it the fused kernel is faster)
constexpr int64_t kHandoverSplitLeast = 608 * 32;
size_t handover_entry_bytes();
// state capacity of the split hand-over kernels for a plane of `plane`
// pixels: an eighth of the plane (at least 1024 entries, at most 2^19)
inline int64_t handover_split_cap(int64_t plane) {
  int64_t c = plane >> 3;
  if (c < 1024) c = 1024;
  if (c > (1 << 19)) c = 1 << 19;
  return c < plane ? c : plane;
}
// tc.cu
mls_status launch_tc(const mlsk::KParams &p, int fp16, int wsplit, cudaStream_t st, int *nlaunch);
int tc_dims_per_pass(int D, int degree);
// tc64.cu: FP64-equivalent moments on the tensor cores (MLS_P_FP64_TC)
mls_status launch_tc64(const mlsk::KParams &p, cudaStream_t st, int *nlaunch);

// Renders whose field is double: FP64 and its tensor-core emulation.
inline bool field_is_fp64(int precision) { return precision == MLS_P_FP64 || precision == MLS_P_FP64_TC; }

// errors (mls_api.cu)
mls_status fail(mls_status s, const std::string &msg);
mls_status cuda_fail(cudaError_t e, const char *what);
mls_status dev_alloc(mls_handle *h, void **p, size_t bytes, cudaStream_t st);

}  // namespace mlsi

#define MLS_CUDA_TRY(expr)                                        \
  do {                                                            \
    cudaError_t e__ = (expr);                                     \
    if (e__ != cudaSuccess) return mlsi::cuda_fail(e__, #expr);   \
  } while (0)
