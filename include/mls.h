/*
 * mls.h -- C ABI of the GB300 (sm_103a) moving-least-squares field library.
 *
 * For every pixel p of a W x H grid the library evaluates the weighted
 * least-squares polynomial fit of the data values f_i at the given 2D points
 * x_i, with weights w_i = w(|x_i - p|), and then labels each data dimension
 * with its iso-band index.  This is the per-pixel MLS evaluation of Section
 * 3.3 of Muelder, Leaf, Sigovan and Ma, "A Moving Least Squares Based
 * Approach for Contour Visualization of Multi-Dimensional Data"
 * (arXiv:1408.0677): Eq. eq-weights (weights), Eq. eq-affinemls with Eqs.
 * eq-pstar / eq-qstar (the linear-basis fit is the paper's affine MLS),
 * Eq. eq-meanmls (the constant-basis fit is its weighted mean), Section 3.4
 * (discrete colours = iso-band labels) and Section 4.5 (O(whn): every pixel
 * is independent and depends on every point).
 *
 * Conventions shared by every entry point
 *  - Pixel (u, v) has centre (x0 + (u + 1/2)(x1 - x0)/W,
 *    y0 + (v + 1/2)(y1 - y0)/H); images are row-major with v = 0 at y0.
 *  - Fields and bands are planar: element (d, v, u) at d*W*H + v*W + u.
 *  - Basis b(d) = (1, d_x, d_y [, d_x^2, d_x d_y, d_y^2]) of degree 0, 1 or
 *    2; the fit's value at p is the constant coefficient.
 *  - Calls are asynchronous on the CUDA stream passed as `stream`
 *    (a cudaStream_t; NULL means the legacy default stream) when every
 *    buffer is on the device; with host buffers the call copies through the
 *    device and returns after the stream has finished.
 *  - The caller owns every input and output buffer.  The handle owns its
 *    device copies of the points and values and its scratch memory.
 *  - Errors are returned as an mls_status before any launch when they are
 *    argument errors; nothing is written then.  mls_last_error() gives a
 *    thread-local message for the last failure.
 *  - A handle is not thread safe; different handles are independent.
 */
#ifndef MLS_H
#define MLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLS_ABI_VERSION 5

typedef enum mls_status {
    MLS_OK = 0,
    MLS_E_INVAL = 1,       /* bad argument; nothing launched or written */
    MLS_E_NOMEM = 2,       /* device allocation failed; the handle stays usable */
    MLS_E_CUDA = 3,        /* a CUDA runtime call failed */
    MLS_E_TIMEOUT = 4,     /* a bounded device wait or host watchdog expired */
    MLS_E_UNSUPPORTED = 5  /* valid request this build does not implement */
} mls_status;

/* Weight functions w(r) (Section 3.3). */
typedef enum mls_weight {
    MLS_W_GAUSS = 0,       /* exp(-r^2 / h^2), all points */
    MLS_W_WENDLAND = 1,    /* (1 - q)^4 (4 q + 1), q = r / h < 1; compact, binned */
    MLS_W_INVDIST = 2      /* 1 / r^(2 alpha) (Eq. eq-weights), all points */
} mls_weight;

/* Arithmetic of the moment accumulation. */
typedef enum mls_precision {
    MLS_P_FP64 = 0,        /* FP64 on CUDA cores; field is double */
    MLS_P_FP32 = 1,        /* FP32 on CUDA cores; field is float */
    MLS_P_BF16 = 2,        /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
    MLS_P_FP16 = 3,        /* FP16 operands on tcgen05 tensor cores, FP32 accumulate */
    MLS_P_FP64_TC = 4      /* FP64-equivalent on tcgen05 tensor cores (weights and operands split
                              into ten exact FP16 digits, exact FP32 partial sums, FP64 solve);
                              field is double.  Gaussian (full sum) and Wendland weights, the
                              polynomial fit (no truncated Gaussian, inverse distance or mappings);
                              views whose 16-pixel tile spans more than 4 h take the FP64 kernel */
} mls_precision;

/* Per-pixel status bits (status image, one byte per pixel). */
#define MLS_ST_DEGREE_MASK 0x03u  /* basis degree used (0, 1, 2) */
#define MLS_ST_NO_SUPPORT  0x04u  /* no point with positive weight: value NaN, band 255 */
#define MLS_ST_FP64_SOLVE  0x08u  /* condition estimate above cond_fp64: FP64 factorisation */
#define MLS_ST_RECOMPUTED  0x10u  /* pixel handed to the recompute path (FP64 decisions) */
#define MLS_ST_DEGRADED    0x20u  /* degree lowered by the degenerate-pixel policy */
#define MLS_ST_COINCIDENT  0x40u  /* inverse distance: pixel centre on a data point */

/*
 * Problem description.  Fill with mls_desc_default() and override.
 *   n, D        number of points and data dimensions (1 <= D <= 256)
 *   degree      basis degree 0, 1 or 2
 *   weight      mls_weight
 *   precision   mls_precision
 *   h           Gaussian h, Wendland support radius, or inverse-distance
 *               basis scale (> 0); the basis is scaled by h
 *   alpha       inverse-distance exponent (Eq. eq-weights); > 0
 *   cond_fp64   condition estimate above which the per-pixel factorisation
 *               runs in FP64 (default 1e6)
 *   rcond_degenerate  reciprocal condition (1-norm, diagonally equilibrated
 *               moment matrix) below which the degree is lowered (1e-12)
 *   cond_recompute    condition estimate (pixel frame) above which a
 *               reduced-precision pixel is handed to the recompute path:
 *               FP64 moments for the degree policy, the fit solved in the
 *               frame of the weighted centroid, and FP64 throughout where
 *               even that frame is ill conditioned (0 = default for the
 *               precision: FP32 1e3, FP16 1e3, BF16 1e2)
 *   weight_split      tensor-core precisions: 1 stores each weight as a hi +
 *               lo pair of 16-bit values (three products per point tile);
 *               0 rounds each weight once (two products); 2 renders with
 *               single weights first and renders again, with split weights,
 *               the 16 x 16 tiles where a pixel fails the single-weight
 *               checks; -1 (default) picks 2 for FP16 and 1 for BF16
 *   variant     MLS_V_POLY: the polynomial fit of the given degree (Section
 *               3.3.2 affine MLS for degree 1, the weighted mean for 0);
 *               MLS_V_RIGID (Section 3.3.3, Eqs. eq-rigidmls and
 *               eq-rigidmlspartial) or MLS_V_MEAN (Section 3.3.1, Eq.
 *               eq-meanmls: v + sum w (q - p) / sum w): the paper's mappings
 *               of 2-D values q_i (D must be 2; degree is ignored).  These
 *               run on the CUDA-core kernels (FP32 limits for FP16/BF16).
 *   support     MLS_W_GAUSS only: 0 (default) sums every point; c > 0 is
 *               the truncated Gaussian, whose weight is zero unless
 *               |x_i - p_x| < c h and |y_i - p_y| < c h (a box of
 *               half-width c h around the pixel; every pair left out has
 *               weight below exp(-c^2) of the kernel's peak, e.g. 2.3e-16
 *               for c = 6).  Points are then visited through the uniform
 *               grid, and a pixel's support count (the degree policy's
 *               "points with non-zero weight") is the number of points in
 *               its box: a pixel with an empty box is NaN.  Must be finite,
 *               0 or in (0, 1e6].
 */
typedef struct mls_desc {
    int64_t n;
    int32_t D;
    int32_t degree;
    int32_t weight;
    int32_t precision;
    double h;
    double alpha;
    double cond_fp64;
    double rcond_degenerate;
    double cond_recompute;
    int32_t weight_split;
    int32_t variant;
    double support;
} mls_desc;

/* Mappings (mls_desc.variant). */
#define MLS_V_POLY 0
#define MLS_V_RIGID 1
#define MLS_V_MEAN 2

/* Output grid: W x H pixels over [x0, x1] x [y0, y1]. */
typedef struct mls_view {
    int32_t W, H;
    double x0, y0, x1, y1;
} mls_view;

/* Counters of the last completed render (see mls_sync). */
typedef struct mls_stats {
    int64_t pairs;            /* pixel-point pairs the main kernel visited */
    int64_t recomputed;       /* pixels handed to the recompute path */
    int64_t recomputed_fp64;  /* of those, pixels finished by the pure FP64 kernel */
    int64_t device_error;     /* device error word (0 = none; timeouts set it) */
    int64_t launches;         /* kernels this handle has launched since mls_create */
    double last_render_ms;    /* device time of the last render (CUDA events) */
    double main_kernel_ms;    /* device time of its main MLS kernel(s) over every tile, events on the
                                 same stream (weight_split 2: the single-weight pass only) */
    int64_t retried_tiles;    /* half tiles (16 x 8 pixels) rendered again with split weights
                                 (weight_split 2) */
    int32_t main_path;        /* kernel family of the last render's main pass (MLS_PATH_*) */
    int32_t reserved;
} mls_stats;

/* mls_stats.main_path: which kernels computed the moments of the last render. */
enum {
    MLS_PATH_NONE = 0,        /* no render yet */
    MLS_PATH_TENSOR = 1,      /* tcgen05 tensor-core kernel (FP16/BF16 operands, FP32 accumulators) */
    MLS_PATH_FP32 = 2,        /* FP32 CUDA-core kernel (FP32 renders, wide tiles, inverse distance) */
    MLS_PATH_FP64 = 3,        /* FP64 kernel (FP64 renders) */
    MLS_PATH_VARIANT = 4,     /* rigid / mean-displacement mapping kernel */
    MLS_PATH_FP64_TC = 5      /* FP64-equivalent tensor-core kernel (MLS_P_FP64_TC) */
};

typedef struct mls_handle mls_handle;

/* Fill *desc with defaults (Gaussian, linear basis, FP32, h = 0.05). */
mls_status mls_desc_default(mls_desc *desc);

/*
 * Create a handle holding a resident copy of the points (Section 3.3: the
 * control points p_i with values q_i, read as data values).
 *   xy        n x 2 float64, row-major (x_i, y_i)
 *   F         n x D float64, row-major values
 *   on_device nonzero: xy and F are device pointers read on `stream`
 *             (keep them alive until the stream reaches this call);
 *             zero: host pointers, copied before return
 *   out       receives the handle
 * Converts the values to the layouts the kernels read, normalises them per
 * dimension and, for the Wendland weight, bins the points on a uniform grid
 * of cell size h (counting sort; deterministic order).
 * Device memory of handles, renders, batches and server requests comes from
 * one stream-ordered memory pool per device, created by the library on first
 * use.  It keeps freed memory for reuse instead of returning it to the
 * system: the pool holds up to the largest working set the process has had
 * until the process exits.
 * Errors: MLS_E_INVAL (desc, pointers), MLS_E_NOMEM, MLS_E_CUDA.
 */
mls_status mls_create(const mls_desc *desc, const double *xy, const double *F,
                      int32_t on_device, void *stream, mls_handle **out);

/*
 * Render the MLS field over `view` (Section 3.3, the first pass of the
 * paper's two-pass renderer, into a headless buffer).
 *   field   D x H x W; double for MLS_P_FP64, float otherwise (required)
 *   status  H x W bytes of MLS_ST_* bits, or NULL
 *   levels  D x L float64 ascending iso-levels (host memory), or NULL
 *   L       number of levels per dimension (0..254)
 *   bands   D x H x W bytes, iso-band labels fused into the render
 *           (Section 3.4: band = #{j : t_dj <= f_d}, 255 for NaN), or NULL
 *   on_device  nonzero: field/status/bands are device pointers, and the
 *           call returns once the work is enqueued on `stream`.  Zero: they
 *           are host pointers and the call returns when the results are in
 *           them.  Page-locked host buffers registered with the handle's
 *           device (all three of those given) are written by the kernels
 *           directly; other host memory is staged in device memory and
 *           copied back.  A host output whose first byte is page-locked
 *           but whose extent runs past that page-locked block is rejected
 *           (MLS_E_INVAL) before any launch.
 * Precision routing: FP16/BF16 renders use the tensor-core kernel, except
 * with the inverse-distance weight (no finite support for the tile operand's
 * range clip) and when a 16-pixel tile spans more than 4 h (no moment frame
 * suits all its pixels); those use the CUDA-core kernel with FP32 limits.
 * Errors: MLS_E_INVAL, MLS_E_NOMEM, MLS_E_CUDA, MLS_E_UNSUPPORTED.
 */
mls_status mls_render(mls_handle *h, const mls_view *view, void *field, uint8_t *status,
                      const double *levels, int32_t L, uint8_t *bands,
                      int32_t on_device, void *stream);

/*
 * Iso-band labels of an existing field (Section 3.4, discrete colours).
 *   field   D x H x W in the handle's field type (device or host per on_device)
 *   levels  D x L float64 ascending (host memory)
 *   bands   D x H x W bytes out
 * Errors: MLS_E_INVAL, MLS_E_NOMEM, MLS_E_CUDA.
 */
mls_status mls_bands(mls_handle *h, const mls_view *view, const void *field,
                     const double *levels, int32_t L, uint8_t *bands,
                     int32_t on_device, void *stream);

/* ---------------------------------------------------------------------------
 * Batches (no counterpart in the paper, which renders one dataset per frame,
 * Section 4 Performance): many resident datasets rendered together.
 * mls_batch_render prepares every dataset (scratch, level uploads: these
 * may allocate and synchronise), then launches ONE CUDA graph in which each
 * dataset's kernels run on their own branch, so small datasets fill the GPU
 * together.  The graph is captured on the first call and replayed while the
 * views, buffers and level counts stay the same (a change re-captures).
 * With MLS_BATCH_AUTOTUNE the first call times, per FP16/BF16 dataset, split
 * weights everywhere against the two-pass scheme (weight_split 1 and 2) on
 * the actual view and keeps the faster; both meet the same error bound.
 */
typedef struct mls_batch mls_batch;

#define MLS_BATCH_AUTOTUNE 1

typedef struct mls_batch_stats {
    int64_t datasets;
    int64_t pairs;            /* pixel-point pairs of the last render (full-sum datasets) */
    int64_t recomputed;       /* pixels handed to the recompute path, all datasets */
    int64_t device_error;     /* first non-zero device error word (0 = none) */
    int64_t launches;         /* kernels per batch render */
    int64_t captures;         /* graph captures so far */
    int64_t replays;          /* graph launches so far */
    double last_render_ms;    /* device time of the last batch render (events around the graph) */
} mls_batch_stats;

/*
 * Group `count` handles (distinct, same device; the caller keeps ownership
 * and must not destroy them before the batch) into a batch.
 * Errors: MLS_E_INVAL, MLS_E_CUDA.
 */
mls_status mls_batch_create(int32_t count, mls_handle *const *handles, int32_t flags,
                            mls_batch **out);

/*
 * Render every dataset k of the batch over views[k] into device buffers
 * fields[k] (D_k x H_k x W_k, float or double per its precision), status[k]
 * and bands[k] (each array or entry may be NULL), with levels[k] (host, D_k x
 * L[k] doubles; NULL / L[k] = 0 for no bands).  Asynchronous on `stream`;
 * the buffers must stay valid until mls_batch_sync returns.  Render calls on
 * one batch must not overlap (the datasets' scratch is reused).
 * Errors: MLS_E_INVAL (naming the dataset), MLS_E_NOMEM, MLS_E_CUDA.
 */
mls_status mls_batch_render(mls_batch *b, const mls_view *views, void *const *fields,
                            uint8_t *const *status, const double *const *levels,
                            const int32_t *L, uint8_t *const *bands, void *stream);

/* Wait for the last batch render (host watchdog of timeout_s) and fill *stats. */
mls_status mls_batch_sync(mls_batch *b, double timeout_s, mls_batch_stats *stats);

/* Release the batch (waits for its last render; the handles stay alive). */
mls_status mls_batch_destroy(mls_batch *b);

/* ---------------------------------------------------------------------------
 * Serving (no counterpart in the paper, whose renders follow user
 * interaction one at a time, Section 3.5): a worker thread admits render
 * requests on resident datasets into a pool of stream slots while the
 * requests already admitted hold less device memory than a budget.  Each
 * admitted request gets its own scratch and outputs (stream-ordered
 * allocations, freed when it completes), so requests on the same dataset
 * overlap on the device and a request that arrives while others run starts
 * as soon as a slot and memory are free (continuous batching).
 */
typedef struct mls_server mls_server;

typedef struct mls_server_config {
    int32_t slots;          /* requests in flight at most, 1 .. 64 */
    int32_t reserved;
    int64_t mem_budget;     /* device bytes the requests in flight may hold */
} mls_server_config;

typedef struct mls_request {
    mls_handle *dataset;    /* resident dataset (mls_create), alive until the request completes */
    mls_view view;
    const double *levels;   /* host D x L doubles, copied at submit; NULL when L = 0 */
    int32_t L;              /* 0 .. 254 */
    int32_t reserved;
    uint8_t *bands;         /* host D x H x W out (page-locked for overlap), or NULL */
    uint8_t *status;        /* host H x W out, or NULL */
    void *field;            /* host D x H x W float (double for FP64 datasets), or NULL */
} mls_request;

typedef struct mls_request_done {
    int64_t id;
    int32_t status;         /* mls_status of the request */
    int32_t reserved;
    double latency_ms;      /* submit to completion seen by the worker (host clock) */
    double queued_ms;       /* submit to admission */
    double device_ms;       /* its kernels and copies (events on its slot stream) */
    int64_t footprint;      /* device bytes it held */
} mls_request_done;

typedef struct mls_server_stats {
    int64_t submitted, completed, failed;
    int64_t peak_inflight;  /* most requests in flight at once */
    int64_t peak_bytes;     /* most device bytes held by requests in flight */
} mls_server_stats;

/* Start a server (worker thread on the current device).  Errors: MLS_E_INVAL, MLS_E_CUDA. */
mls_status mls_server_create(const mls_server_config *cfg, mls_server **out);

/* Queue a request (thread-safe, returns at once) and give its id.  The host
 * output buffers must stay valid until it completes.  Errors: MLS_E_INVAL
 * (bad view, levels or buffers), MLS_E_NOMEM (its footprint exceeds the
 * whole budget). */
mls_status mls_server_submit(mls_server *s, const mls_request *req, int64_t *id);

/* Move up to `cap` completion records into done[] (*n receives the count). */
mls_status mls_server_poll(mls_server *s, mls_request_done *done, int32_t cap, int32_t *n);

/* Wait until every submitted request has completed (watchdog timeout_s). */
mls_status mls_server_drain(mls_server *s, double timeout_s, mls_server_stats *stats);

/* Drain, stop the worker and release the server. */
mls_status mls_server_destroy(mls_server *s);

/* Most levels (D * L) that mls_bands_noalloc accepts. */
#define MLS_NOALLOC_MAX_LEVELS 4096

/*
 * Iso-band labels without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory, such
 * as an application whose device memory belongs to its own pool allocator
 * (a cudaMalloc here could fail or fragment that pool) or a frame loop that
 * must not stall in cudaMalloc / cudaFree (both may synchronise the device).
 * The labels are those of mls_bands: band = #{j : t_dj <= f_d}, 255 for NaN.
 *
 *   D, W, H     dimensions and raster size; D * L <= MLS_NOALLOC_MAX_LEVELS
 *   field       device, D x H x W, float (field_fp64 = 0) or double (1)
 *   levels      host, D x L doubles, ascending per dimension, finite
 *   L           1 .. 254
 *   bands       device, D x H x W bytes out
 *   stream      CUDA stream of the work (NULL: the legacy default stream)
 *
 * The levels are kept in a fixed array of the library's device data
 * (MLS_NOALLOC_MAX_LEVELS x 12 bytes = 48 KiB), which every device that
 * loads the library holds until the process exits.  The first call on a
 * device looks up that array's device address (loading the library's module
 * on the device), so make the first call before any stream capture.  Every
 * call on a device shares the array and leaves its levels there; calls whose
 * work overlaps on the GPU race on it, so order them on one stream.  Nothing
 * in the array needs to start at zero.  Pageable host levels (ordinary
 * malloc or numpy memory) have been copied when the call returns and may be
 * reused at once; page-locked levels are read when the stream reaches the
 * copy, so keep them unchanged until then.  The labels are ready when the
 * stream reaches them.
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * Errors: MLS_E_INVAL (bad sizes, D * L above the maximum, NULL pointers,
 * levels not ascending or not finite), MLS_E_UNSUPPORTED (device ordinal
 * above 63), MLS_E_CUDA.
 */
mls_status mls_bands_noalloc(int32_t D, int32_t W, int32_t H, const void *field,
                             int32_t field_fp64, const double *levels, int32_t L,
                             uint8_t *bands, void *stream);

/*
 * Wait for the handle's last stream with a host-side watchdog of
 * `timeout_s` seconds, then read the device error word and counters into
 * *stats (may be NULL).  Returns MLS_E_TIMEOUT when the watchdog expires or
 * a bounded device wait gave up.
 */
mls_status mls_sync(mls_handle *h, double timeout_s, mls_stats *stats);

/* Release the handle and its device memory (waits for its stream). */
mls_status mls_destroy(mls_handle *h);

/*
 * Space mappings (Section 3.4): the field rendered as an RGBA8 image.  The
 * paper describes the renderings in words; the definitions taken, per pixel
 * and shown plane f (one or two of the field's D planes):
 *   grad   |(f_x, f_y)| in value units per pixel: central differences,
 *          one-sided at the image edge or next to a NaN neighbour
 *   band   b = #{j : t_j <= f} (as mls_bands)
 *   lines  coverage clamp(w/2 + 1/2 - d, 0, 1), d = the pixel distance
 *          min |f - t| / grad to the band's bounding levels; black
 *   colours a three-anchor ramp (blue, grey, red) for one plane, or four
 *          corners (blue; pink along the first plane; cyan along the
 *          second) for two
 *
 *   MLS_MAP_LINES          contour lines, black on white
 *   MLS_MAP_DISCRETE       one colour per band, sampled at (b + 1/2) / (L + 1)
 *   MLS_MAP_DISCRETE_LINES both
 *   MLS_MAP_ADAPTIVE       contour lines plus sub-levels: the band spacing
 *                          halved k = 1..sublevels times, depth-k levels at
 *                          odd multiples of spacing / 2^k above the band's
 *                          lower level, faded in by their pixel spacing
 *                          (spacing / 2^k / grad) between fade_lo and fade_hi:
 *                          more lines where space is expanded, fewer where
 *                          it is compressed
 *   MLS_MAP_GRADIENT       colours at clamp((f - lo) / (hi - lo), 0, 1), with
 *                          the contour lines over them
 *   MLS_MAP_TEXTURE        a texture looked up (bilinear, clamp to edge) at
 *                          those coordinates (the second 1/2 for one plane)
 * A pixel where a shown plane is NaN is transparent (0, 0, 0, 0); others
 * have alpha 255 (the texture's own alpha for MLS_MAP_TEXTURE).  Every step
 * is IEEE float arithmetic in a fixed order: the bytes do not depend on the
 * device.
 */
#define MLS_MAP_LINES 0
#define MLS_MAP_DISCRETE 1
#define MLS_MAP_DISCRETE_LINES 2
#define MLS_MAP_ADAPTIVE 3
#define MLS_MAP_GRADIENT 4
#define MLS_MAP_TEXTURE 5

typedef struct mls_map_desc {
    int32_t mode;            /* MLS_MAP_* */
    int32_t ndim;            /* planes shown: 1 or 2 */
    int32_t dim[2];          /* their indices in [0, D) */
    float line_width;        /* pixels, in [0, 1e4] */
    float fade_lo, fade_hi;  /* MLS_MAP_ADAPTIVE: 0 <= fade_lo < fade_hi (pixels) */
    int32_t sublevels;       /* MLS_MAP_ADAPTIVE: halvings, 0 .. 16 */
    int32_t reserved;
    double lo[2], hi[2];     /* MLS_MAP_GRADIENT / _TEXTURE: value range per shown plane (lo != hi) */
    const uint8_t *texture;  /* MLS_MAP_TEXTURE: device, tex_h rows of tex_w RGBA8 texels */
    int32_t tex_w, tex_h;    /* 1 .. 65536 */
} mls_map_desc;

/*
 * Render the mapping of a field into rgba.
 *   D, W, H     planes and raster of the field
 *   field       device, D x H x W, float (field_fp64 = 0) or double (1)
 *   levels      host, D x L doubles, ascending per plane, finite (rows of
 *               the shown planes are read); L in [0, 254] (0: no lines, one
 *               band)
 *   rgba        device, H x W x 4 bytes out (row 0 at y0, like the field)
 *   stream      CUDA stream of the work (NULL: the legacy default stream)
 * No device allocation; the levels travel with the launch, so the call
 * returns as soon as the kernel is queued.  Errors: MLS_E_INVAL (bad
 * description, sizes, levels or pointers, before any launch),
 * MLS_E_UNSUPPORTED (more than 2,097,120 rows), MLS_E_CUDA.
 */
mls_status mls_space_map(const mls_map_desc *m, int32_t D, int32_t W, int32_t H, const void *field,
                         int32_t field_fp64, const double *levels, int32_t L, uint8_t *rgba, void *stream);

/* Thread-local message of the last error ("" when none). */
const char *mls_last_error(void);

/* ABI version of the loaded library (MLS_ABI_VERSION). */
int32_t mls_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLS_H */
