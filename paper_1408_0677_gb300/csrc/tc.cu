// Tensor-core MLS (tcgen05 + TMEM, sm_103a).
//
// For a 16 x 16 pixel tile with centre c and points x_i, write x~_i =
// (x_i - c)/h and delta_p = (p - c)/h.  The weighted least-squares fit at p
// (Section 3.3 of the paper) does not depend on where the polynomial basis
// is centred, so the moments can be taken in the tile frame:
//   S~_a(p) = sum_i w_pi x~_i^a           (|a| <= 2 deg: the matrix M)
//   R~_ad(p) = sum_i w_pi b_a(x~_i) f_id  (the right-hand sides)
// Both are one product  W[pixels x points] . G[points x (16 + K D)]  whose
// operand G depends only on the tile and the points; only w is generated per
// (pixel, point) pair.  This is the P.V product of attention with
// P = exp(...):
//   - warps 0-7 generate the weights in registers (FP32; separable factors
//     for the Gaussian, one approximate square root per pair for Wendland)
//     and store them as FP16/BF16 into a 128B-swizzled K-major A tile;
//   - warps 8-15 build G for the point tile as a hi + lo pair of FP16/BF16
//     operands (G = G_hi + G_lo to ~22 / 16 bits: the moment matrix needs more
//     than one 16-bit rounding, the weights do not);
//   - one thread of warp 16 issues tcgen05.mma (kind::f16, FP32 accumulate in
//     TMEM) for two 128-pixel accumulators, D += A.G_hi + A.G_lo;
//   - warp 17 walks the point cells and stages the point tiles by TMA bulk
//     copies;
//   - the epilogue (warps 0-15) reads the moments back with tcgen05.ld, shifts
//     M to the pixel frame, solves (FP32 Cholesky + refinement, FP64 above
//     cond_fp64), evaluates the fit, labels the iso-bands and stores.
// Pixels whose condition estimate exceeds cond_recompute, whose support count
// sits near a degree threshold, or whose nearest point is so far that range
// clipping of G could matter, are handed to the FP64 path.
//
// Every mbarrier wait is bounded (globaltimer); on expiry the kernel records
// an error word, skips the remaining work, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mls_internal.h"
#include "tcgen05.cuh"

namespace mlsi {
namespace {

using namespace mlsk;
using namespace tcx;

constexpr int kM = 128;           // pixels per accumulator (TMEM lanes)
constexpr int kKT = 64;           // points per stage = one 128-byte row of 16-bit values
constexpr int kStages = 2;
constexpr int kNMax = 256;        // operand columns per accumulator (TMEM budget 2 x 256)
// 18 warps: 8 weight producers (each half of a stage's points for one pixel
// row of both accumulators; the epilogue's warps too), 8 operand builders,
// the MMA issuer and the point-tile loader
constexpr int kWeightWarps = 8;
constexpr int kBuildWarps = 8;
constexpr int kMmaWarp = kWeightWarps + kBuildWarps;
constexpr int kLoadWarp = kMmaWarp + 1;
constexpr int kThreads = 32 * (kLoadWarp + 1);
static_assert(kWeightWarps == 8 && kBuildWarps == 8, "the weight warps cover 256 pixels; the epilogue pairs each with a builder warp");
constexpr int kDcMax = 40;        // value dimensions per pass (bounds the staged point tile)
constexpr float kRMax = 15.f;     // |x~|_inf clip of the operand (FP16 range of x~^4)
constexpr float kLog2e = 1.4426950408889634f;
// staged point tile: per 8-point block (x[8], y[8], pad[4]) and (Dc x 8 + 4) values
constexpr int kXB = 20;                     // floats per position block
constexpr int kPosFloats = (kKT / 8) * kXB; // 160 floats of positions per stage
// separable Gaussian weights: per stage buffer of 16 column and 16 row factor
// rows of 64 points (row stride 68 floats: rows fall on distinct banks)
constexpr int kEXS = 68;
// The 16 row-factor rows start 16 floats past the column-factor rows
// (kRowOff): 16 kEXS is a multiple of 32 banks, so without the shift a point's
// column and row factors land on the same bank and every store pair conflicts.
constexpr int kRowOff = 16 * kEXS + 16;
constexpr int kExyFloats = 32 * kEXS + 16;
constexpr int kGaussHdr = kWeightWarps * 32 * 4;   // per weight warp: alpha[16], beta[16]
constexpr int kPrmBytes = kGaussHdr + 2 * kExyFloats * 4;   // >= the Wendland point parameters (8 KB)
// Common factor of all FP16 weights (the fit does not depend on it): the
// largest weight becomes 2^14, so the low half of a split weight stays in
// the FP16 normal range for weights down to 2^-17 of the largest (unscaled,
// weights below 1/8 had subnormal low halves and only ~2^-24 absolute
// precision).  BF16 has the FP32 exponent range and needs no factor.
template <bool FP16>
__device__ __forceinline__ float weight_scale() { return FP16 ? 16384.f : 1.f; }
// largest log2 of (stabiliser / tile-split stabiliser): the factor products
// of a pixel's largest weights stay in the FP32 normal range
constexpr float kResMax = 96.f;

constexpr int kABytes = kM * 128;                  // 16 KB per A tile
// Two kernel shapes share one layout: two 128-pixel accumulators with single
// 16-bit weights, or one accumulator with weights split hi + lo; either way
// a stage holds two A tiles.
constexpr int kOffA = 0;                           // A[stage][acc or part]
constexpr int kOffB = kOffA + kStages * 2 * kABytes;      // 64 KB: B[stage][part]
constexpr int kSmemLimit = 232448;                        // 227 KB per CTA

// Shared-memory layout, sized for the operand width N and the dimensions per
// pass Dc: A tiles, B tiles (2 x N rows of 128 B per stage), per-warp point
// parameters, a ring of staged point tiles (x, y and Dc value rows of 64
// floats each, filled by TMA bulk copies), barriers.
// bytes past offBar: barriers, TMEM slot and tile geometry (512), then the
// slot table of the staged point tiles (4 stages x 8 slots x 16 bytes)
constexpr int kMisc = 1024;
// epilogue: each pixel's z and keep flag (8 floats) at the end of the 64 KB
// of A tiles, past the staged levels (Dc (P + 2) floats: Dc <= 40 and P <= 256
// for L <= 254 levels, so below 41 KB)
constexpr int kZOff = 56 * 1024;
constexpr int kOffSlots = 512;

struct TcLayout {
  int offB, bpart;          // B tiles: offset, bytes per tile
  int offPrm;
  int offData, dstage, dstages;
  int offBar;
  int total;
};

TcLayout make_layout(int N, int Dc) {
  TcLayout L;
  L.offB = kOffB;
  L.bpart = N * 128;
  L.offPrm = L.offB + kStages * 2 * L.bpart;
  L.offData = L.offPrm + kPrmBytes;
  L.dstage = (kKT / 8) * (kXB + Dc * 8 + 4) * 4;
  const int fixed = L.offData + kMisc + 1024;
  int ds = (kSmemLimit - fixed) / L.dstage;
  L.dstages = ds > 4 ? 4 : ds;
  // barriers, TMEM slot, the tile geometry (+256), the stage slot table (+512)
  L.offBar = L.offData + L.dstages * L.dstage;
  L.total = L.offBar + kMisc + 1024;
  return L;
}

// Iso-band label #{j : t_j <= f} over ascending levels (rounded up to float,
// so the float comparison equals the double one), by binary search; 255 for NaN.
// Iso-band labels #{t <= f} of G values, value g against the level row
// lev + row[g] * P: the L ascending levels, then NaN up to P (a power of two
// >= L; NaN <= f is false).  Steps of P/2, ..., 1 find how many of the first
// P - 1 entries are <= f, one more comparison takes the last entry.  Every
// load is unconditional and every step a select, so there are no branches
// and the G searches' shared-memory loads run side by side (a loop per value
// would wait out each load in turn).  NaN values get 255.
template <int G>
__device__ __forceinline__ void band_labels(const float (&f)[G], const int (&row)[G], const float *lev, int P,
                                            int (&band)[G]) {
#pragma unroll
  for (int g = 0; g < G; ++g) band[g] = 0;
  for (int step = P >> 1; step > 0; step >>= 1) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float t = lev[row[g] * P + band[g] + step - 1];
      band[g] = (t <= f[g]) ? band[g] + step : band[g];
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const float t = lev[row[g] * P + band[g]];
    band[g] = (f[g] != f[g]) ? 255 : band[g] + (t <= f[g] ? 1 : 0);
  }
}

// Two FP32 lanes in one 64-bit register pair: sm_100-family cores execute
// add / mul / fma on both halves in one instruction (IEEE round to nearest
// per half, the same results as two scalar operations).
__device__ __forceinline__ uint64_t f2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 f2_get(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// Eight operand values -> hi and lo 16-byte chunks (G = hi + lo).
template <bool FP16>
__device__ __forceinline__ void split8(const float (&x)[8], uint4 &hi, uint4 &lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = pack2<FP16>(x[2 * q], x[2 * q + 1]);
    const float2 b = unpack2<FP16>(h[q]);
    const float2 r = f2_get(f2_sub(f2(x[2 * q], x[2 * q + 1]), f2(b.x, b.y)));
    l[q] = pack2<FP16>(r.x, r.y);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Four operand values, as two lane pairs, -> hi and lo 8-byte chunks (as split4).
template <bool FP16>
__device__ __forceinline__ void split4p(uint64_t v01, uint64_t v23, uint2 &hi, uint2 &lo) {
  const float2 a = f2_get(v01), b = f2_get(v23);
  const uint32_t h0 = pack2<FP16>(a.x, a.y), h1 = pack2<FP16>(b.x, b.y);
  const float2 ua = unpack2<FP16>(h0), ub = unpack2<FP16>(h1);
  const float2 ra = f2_get(f2_sub(v01, f2(ua.x, ua.y))), rb = f2_get(f2_sub(v23, f2(ub.x, ub.y)));
  hi = make_uint2(h0, h1);
  lo = make_uint2(pack2<FP16>(ra.x, ra.y), pack2<FP16>(rb.x, rb.y));
}

// Four operand values -> hi and lo 8-byte chunks (G = hi + lo).
template <bool FP16>
__device__ __forceinline__ void split4(const float (&x)[4], uint2 &hi, uint2 &lo) {
  uint32_t h[2], l[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    h[q] = pack2<FP16>(x[2 * q], x[2 * q + 1]);
    const float2 b = unpack2<FP16>(h[q]);
    l[q] = pack2<FP16>(x[2 * q] - b.x, x[2 * q + 1] - b.y);
  }
  hi = make_uint2(h[0], h[1]);
  lo = make_uint2(l[0], l[1]);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// the products x_k y_k g of four lanes, two at a time
__device__ __forceinline__ void prod4(const float4 &x, const float4 &y, uint64_t g, float *w) {
  const float2 a = f2_get(f2_mul(f2_mul(f2(x.x, x.y), f2(y.x, y.y)), g));
  const float2 b = f2_get(f2_mul(f2_mul(f2(x.z, x.w), f2(y.z, y.w)), g));
  w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}

// Wendland weight S (1 - q)^4 (4 q + 1) of a pair with q^2 = t, zero for
// t >= 1.  The weight is rounded to a 16-bit operand next, so the square root
// is the approximate one (relative error near 2^-23, far below that
// rounding); S is the common factor of all weights (a power of two, exact).
template <bool FP16>
__device__ __forceinline__ float wendland_weight(float t) {
  const float S = weight_scale<FP16>();
  const float q = sqrt_approx(fmaxf(t, 0.f));
  const float o = 1.f - q;
  const float o2 = o * o;
  return (t < 1.f) ? o2 * o2 * fmaf(4.f * S, q, S) : 0.f;
}

// wendland_weight of two pairs (q^2 = t.x and t.y) with two-lane arithmetic:
// the same operations, so the same results
template <bool FP16>
__device__ __forceinline__ float2 wendland_weight2(uint64_t t2) {
  const float S = weight_scale<FP16>();
  const float2 t = f2_get(t2);
  const float qa = sqrt_approx(fmaxf(t.x, 0.f)), qb = sqrt_approx(fmaxf(t.y, 0.f));
  const uint64_t q = f2(qa, qb);
  const uint64_t o = f2_sub(f2(1.f, 1.f), q);
  const uint64_t o2 = f2_mul(o, o);
  const float2 w = f2_get(f2_mul(f2_mul(o2, o2), f2_fma(f2(4.f * S, 4.f * S), q, f2(S, S))));
  return make_float2(t.x < 1.f ? w.x : 0.f, t.y < 1.f ? w.y : 0.f);
}

// The sequence of point tiles a CTA visits: all points, or the cell rows of
// the uniform grid overlapping the CTA's pixels +- r: r = h for the Wendland
// weight, c h for the truncated Gaussian, h sqrt(max_p m_p + gcut) for the
// Gaussian (beyond it every weight rounds to zero in the 16-bit operand).
// Tile starts are rounded down to 8 points; indices outside [lo, hi) are
// masked.  One thread (the loader) walks them; the other roles read each
// stage's slots from shared memory.
// Per-CTA geometry, computed once in FP64 by one warp (GB300's FP64 rate is a
// small fraction of FP32's: every thread evaluating these cost more than the
// contraction on short point ranges): the tile-frame offsets of the 16 pixel
// columns and rows, and the cell range the CTA visits.
struct TileGeo {
  float col[16], row[16];
  int cr[4];                // cx0, cx1, cy0, cy1
  // trimming of the cell rows to the reach of the tile's pixels (the tile's
  // pixel-centre extent and the reach, in cells relative to (cx0, cy0))
  float tx0, tx1, ty0, ty1, rc;
  int trim;
};

__device__ __forceinline__ bool ranges_all(const KParams &p) {
  return p.weight != MLS_W_WENDLAND && !p.trunc_on && !(p.gcut > 0.f);
}

// One warp: lane k < 16 column k, lane 16 + k row k; lanes 0..3 the cell range.
__device__ void tile_geometry(const KParams &p, int u0, int v0, int hgt, float cxs, float cys, int lane,
                              TileGeo *g) {
  if (lane < 16) g->col[lane] = (float)((p.x0 + (u0 + lane + 0.5) * p.sx - p.ctr_x) * p.inv_s - (double)cxs);
  else g->row[lane - 16] = (float)((p.y0 + (v0 + lane - 16 + 0.5) * p.sy - p.ctr_y) * p.inv_s - (double)cys);
  if (lane < 4 && !ranges_all(p)) {
    // r = h (Wendland), c h (truncated Gaussian), h sqrt(max m + gcut) (Gaussian)
    const float rs = p.weight == MLS_W_WENDLAND ? 1.f
                     : p.trunc > 0.0            ? (float)p.trunc
                                                : sqrtf(p.tmax[tile_i(p, (v0 >> 4) * p.tiles_x + (u0 >> 4))] + p.gcut);
    const double rad = p.h * (double)rs * (1.0 + 1e-5);
    const bool ax = lane < 2, upper = lane & 1;
    const double s = ax ? p.sx : p.sy, o = ax ? p.x0 : p.y0, g0 = ax ? p.gx0 : p.gy0;
    const int n0 = ax ? u0 : v0, n1 = ax ? u0 + 15 : v0 + hgt - 1, ng = ax ? p.gx : p.gy;
    const double a = o + (n0 + 0.5) * s, b = o + (n1 + 0.5) * s;
    const double e = upper ? fmax(a, b) + rad : fmin(a, b) - rad;
    const int c = (int)floor((e - g0) * p.inv_cell);   // the binning's expression
    g->cr[lane] = upper ? min(c, ng - 1) : max(c, 0);
  }
  __syncwarp();
  if (lane == 0) {
    // The points within reach of some pixel of the tile lie in the tile's
    // pixel-centre rectangle widened by the disc of radius r (the box of the
    // truncated Gaussian widens it to a rectangle: no trimming there).  A
    // cell row at distance dy from the rectangle needs only the columns
    // within sqrt(r^2 - dy^2) of it; the other cells hold points whose
    // weight is zero at every pixel of the tile.
    g->trim = (!ranges_all(p) && !p.trunc_on) ? 1 : 0;
    if (g->trim) {
      const float rs = p.weight == MLS_W_WENDLAND ? 1.f
                                                  : sqrtf(p.tmax[tile_i(p, (v0 >> 4) * p.tiles_x + (u0 >> 4))] + p.gcut);
      const double rad = p.h * (double)rs * (1.0 + 1e-5);
      const double xa = p.x0 + (u0 + 0.5) * p.sx, xb = p.x0 + (u0 + 15 + 0.5) * p.sx;
      const double ya = p.y0 + (v0 + 0.5) * p.sy, yb = p.y0 + (v0 + hgt - 1 + 0.5) * p.sy;
      g->tx0 = (float)((fmin(xa, xb) - p.gx0) * p.inv_cell - g->cr[0]);
      g->tx1 = (float)((fmax(xa, xb) - p.gx0) * p.inv_cell - g->cr[0]);
      g->ty0 = (float)((fmin(ya, yb) - p.gy0) * p.inv_cell - g->cr[2]);
      g->ty1 = (float)((fmax(ya, yb) - p.gy0) * p.inv_cell - g->cr[2]);
      g->rc = (float)(rad * p.inv_cell);
    }
  }
}

// The 8-point blocks of the visited ranges, packed densely into stages of 8
// blocks (64 points): slot after slot takes the next block of the current
// cell row and moves on to the next non-empty row when the row ends (a row
// of ~50 points would otherwise start a half-empty stage of its own).
struct Slot {
  int gb;       // 8-point block index (points 8 gb .. 8 gb + 7), < 0: empty slot
  int lo, hi;   // point range of its row: points outside are masked
};

// The walk is warp-collective.  A window of 32 cell rows is loaded at once
// (lane k: the k-th row of the window, one round trip of parallel loads); each row's
// 8-point blocks get consecutive global slot numbers, starting at S_k (a
// prefix sum over the window, continuing the previous windows).  Stage kt
// holds the global slots 8 kt .. 8 kt + 7; lane q < 8 finds the row of slot
// 8 kt + q as the last row k with S_k <= 8 kt + q (a ballot per slot) and
// forms its slot from that row's range, so no thread walks slot by slot.
struct PackW {
  int cx0, cx1, cy0, cy1;
  bool trim;                    // rows trimmed to the reach (TileGeo)
  float tx0, tx1, ty0, ty1, rc;
  int rnext;          // first row not yet loaded
  int W0, T;          // global slots [W0, T) belong to the loaded window
  int J;              // first global slot of the next stage
  bool all;           // every point (one row [0, n))
  int rlo, rhi, S;    // this lane's row of the window: point range, first slot
};

__device__ __forceinline__ void packw_load(const KParams &p, PackW &w) {
  const int lane = threadIdx.x & 31;
  const int r = w.rnext + lane;
  w.rlo = w.rhi = 0;
  if (r <= w.cy1) {
    int c0 = w.cx0, c1 = w.cx1;
    if (w.trim) {
      // the row's distance from the tile's rectangle and the columns within
      // reach, widened by 0.01 cell against the FP32 rounding of the
      // (small, tile-relative) coordinates
      const float rr = (float)(r - w.cy0);
      const float dy = fmaxf(0.f, fmaxf(rr - w.ty1, w.ty0 - (rr + 1.f)));
      const float h2 = w.rc * w.rc - dy * dy;
      const float hw = sqrtf(fmaxf(h2, 0.f)) + 0.01f;
      if (dy > w.rc + 0.01f) {
        c1 = c0 - 1;   // no point of the row is within reach
      } else {
        c0 = w.cx0 + max(0, (int)floorf(w.tx0 - hw));
        c1 = w.cx0 + min(w.cx1 - w.cx0, (int)floorf(w.tx1 + hw));
      }
    }
    if (c0 <= c1) {
      w.rlo = cell_at(p, (int64_t)r * p.gx + c0);
      w.rhi = cell_at(p, (int64_t)r * p.gx + c1 + 1);
    }
  }
  const int nb = (w.rhi > w.rlo) ? ((w.rhi - 1) >> 3) - (w.rlo >> 3) + 1 : 0;
  int inc = nb;   // inclusive prefix sum over the lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  w.W0 = w.T;
  w.S = w.W0 + inc - nb;
  w.T = w.W0 + __shfl_sync(0xffffffffu, inc, 31);
  w.rnext += 32;
}

__device__ __forceinline__ void packw_init(const KParams &p, const TileGeo *g, PackW &w) {
  w.all = ranges_all(p);
  w.J = 0;
  w.W0 = 0;
  w.rlo = w.rhi = w.S = 0;
  w.cx0 = w.cx1 = w.cy0 = w.cy1 = 0;
  w.trim = false;
  w.tx0 = w.tx1 = w.ty0 = w.ty1 = w.rc = 0.f;
  if (w.all) {
    w.T = (int)((p.n + 7) >> 3);   // blocks of [0, n)
    w.rnext = 1;
    w.cy1 = 0;
    return;
  }
  w.cx0 = g->cr[0];
  w.cx1 = g->cr[1];
  w.cy0 = g->cr[2];
  w.cy1 = g->cr[3];
  w.rnext = g->cr[2];
  w.trim = g->trim != 0;
  w.tx0 = g->tx0;
  w.tx1 = g->tx1;
  w.ty0 = g->ty0;
  w.ty1 = g->ty1;
  w.rc = g->rc;
  w.T = 0;
  if (w.cx0 > w.cx1) w.rnext = w.cy1 + 1;   // no cells: nothing to visit
}

// Make the window hold slot J (load windows while it lies past them and rows
// remain); returns whether the stage starting at J exists.
__device__ __forceinline__ bool packw_valid(const KParams &p, PackW &w) {
  while (w.J >= w.T && w.rnext <= w.cy1) packw_load(p, w);
  return w.J < w.T;
}

// The stage starting at J: lane q < 8 returns slot q (gb < 0: empty), J
// advances by 8.  Requires packw_valid.
__device__ __forceinline__ Slot packw_stage(const KParams &p, PackW &w) {
  const int lane = threadIdx.x & 31;
  Slot mine{-1, 0, 0};
  if (w.all) {
    const int j = w.J + lane;
    if (lane < kKT / 8 && j < w.T) mine = Slot{j, 0, (int)p.n};
    w.J += kKT / 8;
    return mine;
  }
  for (;;) {
    // slots of this stage inside the loaded window
    uint32_t m[kKT / 8];
#pragma unroll
    for (int q = 0; q < kKT / 8; ++q) m[q] = __ballot_sync(0xffffffffu, w.S <= w.J + q);
    uint32_t mq = m[0];
#pragma unroll
    for (int q = 1; q < kKT / 8; ++q) mq = (lane == q) ? m[q] : mq;
    const int j = w.J + lane;
    const int k = mq ? 31 - __clz(mq) : 0;
    const int lo = __shfl_sync(0xffffffffu, w.rlo, k);
    const int hi = __shfl_sync(0xffffffffu, w.rhi, k);
    const int S0 = __shfl_sync(0xffffffffu, w.S, k);
    if (lane < kKT / 8 && j >= w.W0 && j < w.T) mine = Slot{(lo >> 3) + (j - S0), lo, hi};
    if (w.J + kKT / 8 <= w.T || w.rnext > w.cy1) break;
    packw_load(p, w);   // the stage continues into the next window
  }
  w.J += kKT / 8;
  return mine;
}

__device__ __forceinline__ bool slot_has(const Slot &s, int i) { return s.gb >= 0 && i >= s.lo && i < s.hi; }

// Slot q of staged point tile ds, as the loader wrote it.
__device__ __forceinline__ Slot slot_read(const int4 *tab, int ds, int q) {
  const int4 e = tab[ds * 8 + q];
  return Slot{e.x, e.y, e.z};
}

template <int DEG, int WK, bool FP16, int NACC, bool WSPLIT>
__global__ void __launch_bounds__(kThreads, 1) k_mls_tc(KParams p, int d0, int Dc, int N, uint32_t idesc,
                                                         TcLayout lay, int pass) {
  static_assert(NACC * (WSPLIT ? 2 : 1) == 2, "a stage holds two A tiles");
  constexpr int K = n_terms(DEG), NM = n_moments(DEG);
  constexpr int TH = 8 * NACC;          // tile height in pixels (width 16)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // align to 1024 B by offsetting the shared array itself (not through an
  // integer cast), so every access below stays a shared-memory access
  unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t *bars = (uint64_t *)(smem + lay.offBar);
  const uint32_t bar_full0 = smem_u32(&bars[0]);    // full[s] at +8 s
  const uint32_t bar_empty0 = smem_u32(&bars[2]);   // empty[s]
  const uint32_t bar_acc = smem_u32(&bars[4]);
  const uint32_t bar_dfull0 = smem_u32(&bars[5]);   // staged point tile ready [ds]
  const uint32_t bar_dempty0 = smem_u32(&bars[9]);  // staged point tile consumed [ds]
  const uint32_t bar_exy0 = smem_u32(&bars[13]);    // Gaussian factor table [kt & 1] written
  uint32_t *tmem_slot = (uint32_t *)(smem + lay.offBar + 128);
  TileGeo *geo = (TileGeo *)(smem + lay.offBar + 256);
  const int DST = lay.dstages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int u0, v0;
  if (p.tile_list) {
    // second pass over listed half tiles (2 tile + the 8-row half): one CTA
    // per entry, the rest exit.  An 8-row CTA (NACC == 1) takes its half; a
    // 16-row CTA would take the whole tile.
    const int slot = blockIdx.x;
    if (slot >= (int)*p.tile_count) return;
    const int ht = (int)queue_i(p, p.tile_list[queue_i(p, slot)]), tl = ht >> 1;
    u0 = (tl % p.tiles_x) * 16;
    v0 = (tl / p.tiles_x) * 16 + (NACC == 1 ? (ht & 1) * 8 : 0);
  } else {
    u0 = blockIdx.x * 16;
    v0 = blockIdx.y * TH;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar_full0 + 8 * s, kWeightWarps + kBuildWarps);
      mbar_init(bar_empty0 + 8 * s, 1);
    }
    mbar_init(bar_acc, 1);
    for (int ds = 0; ds < DST; ++ds) {
      mbar_init(bar_dfull0 + 8 * ds, 1);
      mbar_init(bar_dempty0 + 8 * ds, kWeightWarps + kBuildWarps + 1);   // the producer warps and the MMA issuer
    }
    mbar_init(bar_exy0, kWeightWarps);
    mbar_init(bar_exy0 + 8, kWeightWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // moment frame of the tile: the weighted centroid of the points near its
  // centre (from the prepass); the fit is solved in this frame
  const int tile = (v0 >> 4) * p.tiles_x + (u0 >> 4);
  const float cxs = p.tcen[2 * tile_i(p, tile)], cys = p.tcen[2 * tile_i(p, tile) + 1];
  if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), 512);
  if (warp == kLoadWarp) tile_geometry(p, u0, v0, TH, cxs, cys, lane, geo);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t limit = kWaitLimitNs;
  bool alive = true;

  // The loader walks the cell rows and writes each staged point tile's slots
  // {8-point block, row range} into the slot table beside it; the other roles
  // read them there.  A stage whose first slot is empty ends the tile.
  int4 *slot_tab = (int4 *)(smem + lay.offBar + kOffSlots);
  int nst = 0;   // point tiles this thread consumed (the epilogue reads whether any)

  if (warp < kWeightWarps && WK == MLS_W_GAUSS) {
    // ------------------------------------------------ weight producers (Gaussian, separable)
    // w = exp2(L_p - log2e |x~ - delta_p|^2) with L_p = log2e m_p.  The tile's
    // pixels lie on 16 columns dx_c and 16 rows dy_r, so with the stabiliser
    // split as alpha_c + beta_r <= L_p (beta_r = min_c L, alpha_c =
    // min_r (L - beta_r)) every weight is a product of a column factor
    // exp2(alpha_c - log2e (dx_c - x)^2) and a row factor
    // exp2(beta_r - log2e (dy_r - y)^2): 32 exp2 per point instead of 256,
    // and one multiply per weight.  A per-point exponent shift balances the
    // two factors (neither overflows).  The product carries the factor
    // 2^(alpha_c + beta_r - L_p) <= 1, which one more multiply by its inverse
    // removes, so every pixel's largest weight is 1 as with the per-pixel
    // stabiliser (pixels whose factor would leave the FP32 range are handed over).
    // The truncated Gaussian's box |dx|, |dy| < c is separable too: a column
    // (row) factor is zero where the point is c or more away along x (y).
    // thread t: pixel row m = t mod 128 of both accumulators, chunks (8
    // points each) 4 hh .. 4 hh + 3 of every stage
    const int t = threadIdx.x;
    const int m = t & 127, hh = t >> 7;
    const bool boxed = p.trunc_on;
    const float cbox = p.trunc_f;
    float *sAB = (float *)(smem + lay.offPrm) + 32 * warp;     // this warp's alpha[16], beta[16]
    float *exy = (float *)(smem + lay.offPrm + kGaussHdr);     // [2][16 column rows, 16 row rows at kRowOff]
    {
      const int stride = p.tiles_x * 16;
      const int r = lane & 15, c = lane & 15;
      float b = INFINITY;
      if (r < TH)
        for (int cc = 0; cc < 16; ++cc) b = fminf(b, kLog2e * p.mstab[pix_i(p, (int64_t)(v0 + r) * stride + u0 + cc)]);
      float a = INFINITY;
      for (int rr = 0; rr < TH; ++rr) {
        const float br = __shfl_sync(0xffffffffu, b, rr);
        a = fminf(a, kLog2e * p.mstab[pix_i(p, (int64_t)(v0 + rr) * stride + u0 + c)] - br);
      }
      sAB[lane] = (lane < 16) ? a : ((r < TH) ? b : 0.f);
      __syncwarp();
    }
    // this thread's factor rows: point jp, columns (half 0) or rows (half 1),
    // entries fk(kk) = 4 (kk >> 1) + (kk & 1) + 2 kh, kk = 0..7, of the 16
    // (the partners of a point are lanes ^ 1, the other half, and ^ 2, the
    // other entries; with entries 2 rows apart the 32 lanes' stores fall on
    // distinct banks)
    const int jp = t >> 2, kh = (t >> 1) & 1, half = t & 1;
    auto fk = [&](int kk) { return 4 * (kk >> 1) + (kk & 1) + 2 * kh; };
    float off[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) off[kk] = half ? geo->row[fk(kk)] : geo->col[fk(kk)];
    // this thread's pixels: column c, rows r0 (and r0 + 8), and their
    // corrections 2^(L_p - alpha_c - beta_r)
    const int cown = m & 15, r0 = m >> 4;
    float gcor[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int rr = r0 + 8 * a;
      const float res = (rr < TH) ? kLog2e * p.mstab[pix_i(p, (int64_t)(v0 + rr) * (p.tiles_x * 16) + u0 + cown)] -
                                        sAB[cown] - sAB[16 + rr]
                                  : 0.f;
      gcor[a] = ex2_approx(fminf(res, kResMax)) * weight_scale<FP16>();
    }
    const uint64_t g0x2 = f2(gcor[0], gcor[0]), g1x2 = f2(gcor[1], gcor[1]);
    int kt = 0;
    for (; alive; ++kt) {
      const int s = kt & 1;
      const int ds = kt % DST;
      if (!mbar_wait(bar_dfull0 + 8 * ds, (kt / DST) & 1, p.err, ERR_WAIT_FULL, limit)) {
        alive = false;
        break;
      }
      if (slot_tab[ds * 8].x < 0) break;
      const Slot mine = slot_read(slot_tab, ds, jp >> 3);
      const float *dxs = (const float *)(smem + lay.offData + ds * lay.dstage);
      float *tab = exy + s * kExyFloats;
      {
        float pos = 0.f;
        bool ok = slot_has(mine, mine.gb * 8 + (jp & 7));
        if (ok) {
          const float x = dxs[(jp >> 3) * kXB + (jp & 7)] - cxs;
          const float y = dxs[(jp >> 3) * kXB + 8 + (jp & 7)] - cys;
          ok = fmaxf(fabsf(x), fabsf(y)) <= kRMax;
          pos = half ? y : x;
        }
        float e[8];
        float mx = -INFINITY;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float d = off[kk] - pos;
          e[kk] = fmaf(-kLog2e * d, d, sAB[16 * half + fk(kk)]);
          if (half == 0 || fk(kk) < TH) mx = fmaxf(mx, e[kk]);
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        const float other = __shfl_xor_sync(0xffffffffu, mx, 1);
        const float sh = half ? 0.5f * (mx - other) : 0.5f * (other - mx);   // Y' = Y - sh, X' = X + sh
        float *dst = tab + half * kRowOff + jp;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          // the truncated Gaussian's box (uniform over the grid)
          const bool in = ok && (!boxed || fabsf(off[kk] - pos) < cbox);
          dst[fk(kk) * kEXS] = in ? ex2_approx(half ? e[kk] - sh : e[kk] + sh) : 0.f;
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar_dempty0 + 8 * ds);
        mbar_arrive(bar_exy0 + 8 * s);
      }
      if (!mbar_wait(bar_exy0 + 8 * s, (kt >> 1) & 1, p.err, ERR_WAIT_FULL, limit) ||
          !mbar_wait(bar_empty0 + 8 * s, ((kt >> 1) & 1) ^ 1, p.err, ERR_WAIT_EMPTY, limit)) {
        alive = false;
        break;
      }
      unsigned char *A0 = smem + kOffA + (s * 2 + 0) * kABytes;
      unsigned char *A1 = smem + kOffA + (s * 2 + 1) * kABytes;
      const float *fx = tab + cown * kEXS;
      const float *fy0 = tab + kRowOff + r0 * kEXS;
      const float *fy1 = tab + kRowOff + (r0 + 8) * kEXS;
#pragma unroll 2
      for (int c = 4 * hh; c < 4 * hh + 4; ++c) {
        const float4 xa = *(const float4 *)(fx + 8 * c), xb = *(const float4 *)(fx + 8 * c + 4);
        const float4 ya = *(const float4 *)(fy0 + 8 * c), yb = *(const float4 *)(fy0 + 8 * c + 4);
        // w = (column factor x row factor) x correction, two lanes per instruction
        float w0[8];
        prod4(xa, ya, g0x2, w0);
        prod4(xb, yb, g0x2, w0 + 4);
        uint4 q0, q1;
        if (WSPLIT) {
          split8<FP16>(w0, q0, q1);          // A0 = hi, A1 = lo of accumulator 0
        } else {
          const float4 za = *(const float4 *)(fy1 + 8 * c), zb = *(const float4 *)(fy1 + 8 * c + 4);
          float w1[8];
          prod4(xa, za, g1x2, w1);
          prod4(xb, zb, g1x2, w1 + 4);
          q0.x = pack2<FP16>(w0[0], w0[1]); q0.y = pack2<FP16>(w0[2], w0[3]);
          q0.z = pack2<FP16>(w0[4], w0[5]); q0.w = pack2<FP16>(w0[6], w0[7]);
          q1.x = pack2<FP16>(w1[0], w1[1]); q1.y = pack2<FP16>(w1[2], w1[3]);
          q1.z = pack2<FP16>(w1[4], w1[5]); q1.w = pack2<FP16>(w1[6], w1[7]);
        }
        *(uint4 *)(A0 + sw128_off(m, c)) = q0;
        *(uint4 *)(A1 + sw128_off(m, c)) = q1;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_full0 + 8 * s);
    }
    nst = kt;
  } else if (warp < kWeightWarps) {
    // ------------------------------------------------ weight producers (Wendland)
    // thread t: row m = t mod 128 of every accumulator, the stage's points
    // 32 hh .. 32 hh + 31 (this warp's point parameters)
    const int t = threadIdx.x;
    const int m = t & 127, hh = t >> 7;
    float dx[NACC], dy[NACC], E[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
      const int q = a * 128 + m;
      const int u = u0 + (q & 15), v = v0 + (q >> 4);
      dx[a] = geo->col[q & 15];
      dy[a] = geo->row[q >> 4];
      const size_t pi = (size_t)v * (p.tiles_x * 16) + u;
      if (WK == MLS_W_GAUSS)
        E[a] = kLog2e * (p.mstab[pix_i(p, pi)] - (dx[a] * dx[a] + dy[a] * dy[a]));
      else
        E[a] = dx[a] * dx[a] + dy[a] * dy[a];
    }
    // the pixel parts as lane pairs: both accumulators' pixels, or one twice
    const uint64_t E2 = f2(E[0], E[NACC - 1]), dx2 = f2(dx[0], dx[NACC - 1]), dy2 = f2(dy[0], dy[NACC - 1]);
    float4 *prm = (float4 *)(smem + lay.offPrm) + warp * kKT;
    int kt = 0;
    for (; alive; ++kt) {
      const int s = kt & 1;
      const int ds = kt % DST;
      if (!mbar_wait(bar_dfull0 + 8 * ds, (kt / DST) & 1, p.err, ERR_WAIT_FULL, limit)) {
        alive = false;
        break;
      }
      if (slot_tab[ds * 8].x < 0) break;
      const float *dxs = (const float *)(smem + lay.offData + ds * lay.dstage);
      __syncwarp();
      {
        const int j = 32 * hh + lane;
        const Slot sl = slot_read(slot_tab, ds, j >> 3);
        float x = 0.f, y = 0.f;
        bool ok = slot_has(sl, sl.gb * 8 + (j & 7));
        if (ok) {
          // blocked tile: 8-point blocks of (x[8], y[8])
          x = dxs[(j >> 3) * kXB + (j & 7)] - cxs;
          y = dxs[(j >> 3) * kXB + 8 + (j & 7)] - cys;
          ok = fmaxf(fabsf(x), fabsf(y)) <= kRMax;
        }
        float4 v;
        if (WK == MLS_W_GAUSS)
          v = ok ? make_float4(-kLog2e * (x * x + y * y), 2.f * kLog2e * x, 2.f * kLog2e * y, 0.f)
                 : make_float4(-INFINITY, 0.f, 0.f, 0.f);
        else
          v = ok ? make_float4(x * x + y * y, -2.f * x, -2.f * y, 0.f) : make_float4(INFINITY, 0.f, 0.f, 0.f);
        prm[j] = v;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_dempty0 + 8 * ds);
      if (!mbar_wait(bar_empty0 + 8 * s, ((kt >> 1) & 1) ^ 1, p.err, ERR_WAIT_EMPTY, limit)) {
        alive = false;
        break;
      }
      unsigned char *A0 = smem + kOffA + (s * 2 + 0) * kABytes;
      unsigned char *A1 = smem + kOffA + (s * 2 + 1) * kABytes;
#pragma unroll 1
      for (int c = 4 * hh; c < 4 * hh + 4; ++c) {
        float w0[8], w1[8];
        // q^2 = |x~|^2 - 2 x~ . delta + |delta|^2 (the point's and the pixel's
        // parts), two lanes per instruction: the two accumulators' pixels of
        // one point, or (one accumulator) two points
        if (NACC == 2) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 pr = prm[8 * c + j];
            uint64_t t2 = f2_add(f2(pr.x, pr.x), E2);
            t2 = f2_fma(f2(pr.z, pr.z), dy2, t2);
            t2 = f2_fma(f2(pr.y, pr.y), dx2, t2);
            const float2 w = wendland_weight2<FP16>(t2);
            w0[j] = w.x;
            w1[j] = w.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const float4 pa = prm[8 * c + j], pb = prm[8 * c + j + 1];
            uint64_t t2 = f2_add(f2(pa.x, pb.x), E2);
            t2 = f2_fma(f2(pa.z, pb.z), dy2, t2);
            t2 = f2_fma(f2(pa.y, pb.y), dx2, t2);
            const float2 w = wendland_weight2<FP16>(t2);
            w0[j] = w.x;
            w0[j + 1] = w.y;
          }
        }
        uint4 q0, q1;
        if (WSPLIT) {
          split8<FP16>(w0, q0, q1);          // A0 = hi, A1 = lo of accumulator 0
        } else {
          q0.x = pack2<FP16>(w0[0], w0[1]); q0.y = pack2<FP16>(w0[2], w0[3]);
          q0.z = pack2<FP16>(w0[4], w0[5]); q0.w = pack2<FP16>(w0[6], w0[7]);
          q1.x = pack2<FP16>(w1[0], w1[1]); q1.y = pack2<FP16>(w1[2], w1[3]);
          q1.z = pack2<FP16>(w1[4], w1[5]); q1.w = pack2<FP16>(w1[6], w1[7]);
        }
        *(uint4 *)(A0 + sw128_off(m, c)) = q0;
        *(uint4 *)(A1 + sw128_off(m, c)) = q1;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_full0 + 8 * s);
    }
    nst = kt;
  } else if (warp < kMmaWarp) {
    // ------------------------------------------------ operand builders
    // thread: points 4 hp .. 4 hp + 3 of the 8-point group g, the moment row
    // rr and the value rows of dimensions rr, rr + 16, ...  (a warp writes two
    // whole 128-byte rows per store; the per-point masking and basis values
    // are shared by the rows of a thread)
    const int tt = threadIdx.x - 32 * kWeightWarps;
    const int hp = tt & 1, g = (tt >> 1) & 7;
    const int rr = tt >> 4;        // row class 0..15
    // exponents of this thread's monomial row (fixed for the whole kernel)
    const int mex = mono_ex(rr < 15 ? rr : 0), mey = mono_ey(rr < 15 ? rr : 0);
    const float mrow = (rr < NM) ? 1.f : 0.f;
    int kt = 0;
    for (; alive; ++kt) {
      const int s = kt & 1;
      const int ds = kt % DST;
      float xv[4], yv[4], msk[4];
      if (!mbar_wait(bar_dfull0 + 8 * ds, (kt / DST) & 1, p.err, ERR_WAIT_FULL, limit)) {
        alive = false;
        break;
      }
      if (slot_tab[ds * 8].x < 0) break;
      const Slot mine = slot_read(slot_tab, ds, g);
      const int i0 = mine.gb * 8 + 4 * hp;
      const float *dsm = (const float *)(smem + lay.offData + ds * lay.dstage);
      if (mine.gb >= 0) {
        const float4 xa = *(const float4 *)(dsm + kXB * g + 4 * hp);
        const float4 ya = *(const float4 *)(dsm + kXB * g + 8 + 4 * hp);
        xv[0] = xa.x; xv[1] = xa.y; xv[2] = xa.z; xv[3] = xa.w;
        yv[0] = ya.x; yv[1] = ya.y; yv[2] = ya.z; yv[3] = ya.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) xv[j] = yv[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j;
        xv[j] -= cxs;
        yv[j] -= cys;
        const bool ok = slot_has(mine, i) && fmaxf(fabsf(xv[j]), fabsf(yv[j])) <= kRMax;
        msk[j] = ok ? 1.f : 0.f;
        if (!ok) { xv[j] = 0.f; yv[j] = 0.f; }
      }
      if (!mbar_wait(bar_empty0 + 8 * s, ((kt >> 1) & 1) ^ 1, p.err, ERR_WAIT_EMPTY, limit)) {
        alive = false;
        break;
      }
      unsigned char *Bh = smem + lay.offB + (s * 2 + 0) * lay.bpart + 8 * hp;
      unsigned char *Bl = smem + lay.offB + (s * 2 + 1) * lay.bpart + 8 * hp;
      // monomial row rr of the moment part (rows 0..15; rows >= NM are zero),
      // branch-free: x^ex = (x or 1)(x^2 or 1)(x^4 or 1) by the bits of ex
      {
        float val[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float x1 = xv[j], x2 = x1 * x1, y1 = yv[j], y2 = y1 * y1;
          const float px = ((mex & 1) ? x1 : 1.f) * ((mex & 2) ? x2 : 1.f) * ((mex & 4) ? x2 * x2 : 1.f);
          const float py = ((mey & 1) ? y1 : 1.f) * ((mey & 2) ? y2 : 1.f) * ((mey & 4) ? y2 * y2 : 1.f);
          val[j] = mrow * msk[j] * px * py;
        }
        uint2 hi, lo;
        split4<FP16>(val, hi, lo);
        *(uint2 *)(Bh + sw128_off(rr, g)) = hi;
        *(uint2 *)(Bl + sw128_off(rr, g)) = lo;
      }
      // value rows 16 + d K + a, dimensions d = rr, rr + 16, ...: basis values
      // b_a of points (0, 1) and (2, 3) as lane pairs (a masked point has
      // x = y = 0 and a zero value, so its products are zero without the mask)
      uint64_t bas[K][2];
#pragma unroll
      for (int hq = 0; hq < 2; ++hq) {
        const uint64_t x = f2(xv[2 * hq], xv[2 * hq + 1]), y = f2(yv[2 * hq], yv[2 * hq + 1]);
        bas[0][hq] = f2(msk[2 * hq], msk[2 * hq + 1]);
        if (K > 1) { bas[1][hq] = x; bas[2][hq] = y; }
        if (K > 3) {
          bas[3][hq] = f2_mul(x, x);
          bas[4][hq] = f2_mul(x, y);
          bas[5][hq] = f2_mul(y, y);
        }
      }
      for (int d = rr; d < Dc; d += 16) {
        float fv[4];
        if (mine.gb >= 0) {
          const float4 fa = *(const float4 *)(dsm + kPosFloats + g * (Dc * 8 + 4) + d * 8 + 4 * hp);
          fv[0] = fa.x; fv[1] = fa.y; fv[2] = fa.z; fv[3] = fa.w;
          // slots past the copied tile hold stale shared memory: never multiply them
#pragma unroll
          for (int j = 0; j < 4; ++j) fv[j] = (msk[j] != 0.f) ? fv[j] : 0.f;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) fv[j] = 0.f;
        }
        const uint64_t fp0 = f2(fv[0], fv[1]), fp1 = f2(fv[2], fv[3]);
#pragma unroll
        for (int a = 0; a < K; ++a) {
          // b_0 f = f (the value is zero where the mask is)
          const uint64_t v0 = a == 0 ? fp0 : f2_mul(bas[a][0], fp0);
          const uint64_t v1 = a == 0 ? fp1 : f2_mul(bas[a][1], fp1);
          uint2 hi, lo;
          split4p<FP16>(v0, v1, hi, lo);
          const int row = 16 + d * K + a;
          *(uint2 *)(Bh + sw128_off(row, g)) = hi;
          *(uint2 *)(Bl + sw128_off(row, g)) = lo;
        }
      }
      // zero rows that pad N to a multiple of 16
      for (int row = 16 + Dc * K + rr; row < N; row += 16) {
        const uint2 z = make_uint2(0, 0);
        *(uint2 *)(Bh + sw128_off(row, g)) = z;
        *(uint2 *)(Bl + sw128_off(row, g)) = z;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar_dempty0 + 8 * ds);
        mbar_arrive(bar_full0 + 8 * s);
      }
    }
    nst = kt;
  } else if (warp == kLoadWarp) {
    // ------------------------------------------------ point-tile loader (TMA bulk copies)
    // The whole warp walks the cell rows (collectively, see PackW); lane q
    // keeps slot q, lanes 0-7 write the slot table, lane 0 waits and arms the
    // barrier, and the first slot of each run of consecutive blocks copies it.
    {
      PackW it;
      packw_init(p, geo, it);
      int kt = 0;
      unsigned long long visited = 0;
      for (; alive && packw_valid(p, it); ++kt) {
        const int ds = kt % DST;
        // lane q keeps slot q of the stage
        const Slot mine = packw_stage(p, it);
        int ok = 1;
        if (lane == 0) ok = mbar_wait(bar_dempty0 + 8 * ds, ((kt / DST) & 1) ^ 1, p.err, ERR_WAIT_EMPTY, limit);
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          alive = false;
          break;
        }
        // the slots travel with the copies: the arrive below releases them
        if (lane < kKT / 8) slot_tab[ds * 8 + lane] = make_int4(mine.gb, mine.lo, mine.hi, 0);
        const bool valid = lane < kKT / 8 && mine.gb >= 0;
        // points of this tile inside the visited ranges
        if (valid) visited += (unsigned long long)max(0, min(mine.hi, mine.gb * 8 + 8) - max(mine.lo, mine.gb * 8));
        // point-blocked layouts: slot q of the stage holds block gb_q
        // (positions 80 bytes, values 32 Dc + 16 bytes: every copy stays
        // 16-byte aligned); the filled slots are a prefix of the stage
        const int64_t nblk = p.n_pad >> 3;
        const uint32_t fbb = (uint32_t)(Dc * 8 + 4) * 4;
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        const int prev = __shfl_up_sync(0xffffffffu, mine.gb, 1);
        // one copy per run of consecutive blocks, issued by its first slot
        const bool start = valid && (lane == 0 || prev + 1 != mine.gb);
        const uint32_t smask = __ballot_sync(0xffffffffu, start);
        const uint32_t dst = sbase + lay.offData + ds * lay.dstage;
        const uint32_t bar = bar_dfull0 + 8 * ds;
        if (lane == 0) mbar_expect_tx(bar, (uint32_t)__popc(vmask) * (kXB * 4 + fbb));
        __syncwarp();
        if (start) {
          const uint32_t above = smask & ~((2u << lane) - 1u);    // later run starts
          const int end = above ? __ffs(above) - 1 : __popc(vmask);
          const uint32_t nb = (uint32_t)(end - lane);
          // checked build: the copied blocks lie inside the point arrays
          const int64_t blk = chk(p.err, mine.gb, nblk - nb + 1, SITE_BLOCK);
          bulk_g2s(dst + lane * kXB * 4, p.xyb + blk * kXB, nb * kXB * 4, bar);
          bulk_g2s(dst + kPosFloats * 4 + lane * fbb, p.fb + ((size_t)pass * nblk + blk) * (Dc * 8 + 4), nb * fbb, bar);
        }
        __syncwarp();
      }
      __syncwarp();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) visited += __shfl_xor_sync(0xffffffffu, visited, o);
      if (lane == 0 && p.visited && d0 == 0 && visited) atomicAdd(p.visited, visited * (unsigned long long)(16 * TH));
      // every issued copy has landed before the CTA may exit (waited before
      // the end marker below completes one of these barriers once more)
      const int first = kt > DST ? kt - DST : 0;
      for (int k2 = first; k2 < kt && lane == 0; ++k2)
        mbar_wait(bar_dfull0 + 8 * (k2 % DST), (k2 / DST) & 1, p.err, ERR_WAIT_FULL, limit);
      // end marker: stage kt with an empty first slot and no copies
      if (alive && lane == 0) {
        const int ds = kt % DST;
        if (mbar_wait(bar_dempty0 + 8 * ds, ((kt / DST) & 1) ^ 1, p.err, ERR_WAIT_EMPTY, limit)) {
          slot_tab[ds * 8] = make_int4(-1, 0, 0, 0);
          mbar_arrive(bar_dfull0 + 8 * ds);
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int kt = 0;
      for (; alive; ++kt) {
        const int s = kt & 1;
        const int ds = kt % DST;
        // the staged tile's first slot says whether stage kt exists; this
        // thread is the ninth consumer of the staged tile, so the loader
        // cannot reuse the slot table before it is read
        if (!mbar_wait(bar_dfull0 + 8 * ds, (kt / DST) & 1, p.err, ERR_WAIT_FULL, limit)) {
          alive = false;
          break;
        }
        const bool last = slot_tab[ds * 8].x < 0;
        mbar_arrive(bar_dempty0 + 8 * ds);
        if (last) break;
        if (!mbar_wait(bar_full0 + 8 * s, (kt >> 1) & 1, p.err, ERR_WAIT_FULL, limit)) {
          alive = false;
          break;
        }
        tc_fence_after();
        // products per accumulator: A.G_hi + A.G_lo, or with split weights
        // A_hi.G_hi + A_hi.G_lo + A_lo.G_hi (A_lo.G_lo is below FP32 rounding)
        constexpr int NT = WSPLIT ? 3 : 2;
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
#pragma unroll
          for (int k = 0; k < kKT / 16; ++k) {
#pragma unroll
            for (int term = 0; term < NT; ++term) {
              const int ap = WSPLIT ? (term == 2 ? 1 : 0) : a;
              const int bp = (term == 1) ? 1 : 0;
              const uint32_t abase = sbase + kOffA + (s * 2 + ap) * kABytes;
              const uint32_t bbase = sbase + lay.offB + (s * 2 + bp) * lay.bpart;
              mma_f16(tmem + a * 256, desc_sw128(abase + 32 * k), desc_sw128(bbase + 32 * k), idesc,
                      (kt | k | term) != 0 ? 1u : 0u);
            }
          }
        }
        mma_commit(bar_empty0 + 8 * s);
      }
      mma_commit(bar_acc);
    }
    __syncwarp();
  }

  __syncthreads();   // every role has left its loop (the stabiliser split is read below)

  // ------------------------------------------------ epilogue (the 16 producer warps)
  // has any point tile been visited?
  const bool any_tile = nst > 0;
  if (warp < kMmaWarp) {
    // weight warp w and builder warp w + 8 read the same TMEM lanes (pixels):
    // both solve the pixel's system, and they take alternate groups of value
    // columns; the weight warps (eh = 0) write the pixel's status
    const int eh = warp / kWeightWarps;
    const int wg = (warp >> 2) & 1;
    // two accumulators: one warpgroup of each half each; one accumulator: the
    // four warpgroups share it
    const int a = (NACC == 2) ? wg : 0;
    const bool primary = eh == 0 && ((NACC == 2) || wg == 0);
    const int gfirst = (NACC == 2) ? eh : (warp >> 2), gstep = (NACC == 2) ? 2 : 4;
    const int m = 32 * (warp & 3) + lane;
    const int q = a * 128 + m;
    const int u = u0 + (q & 15), v = v0 + (q >> 4);
    const bool inside = (u < p.W) && (v < p.H);
    const size_t pi = (size_t)v * (p.tiles_x * 16) + u;
    // the pixel's stabiliser (Gaussian) and support count (Wendland,
    // truncated Gaussian), and the first staged levels and scales (below),
    // are fetched while the last MMAs drain
    const float mst = (WK == MLS_W_WENDLAND) ? 0.f : p.mstab[pix_i(p, pi)];
    const int cflag = (WK == MLS_W_WENDLAND || p.trunc_on) ? p.cnt[pix_i(p, pi)] : 0;
    // level rows padded with NaN to P entries, a power of two >= L
    int P = 1;
    while (P < p.L) P *= 2;
    const int nstage = Dc * (P + 2);
    auto staged = [&](int e) -> float {
      if (e < Dc * P) {
        const int d = e / P, j = e - d * P;
        if (j >= p.L) return __int_as_float(0x7fc00000);
        return (d0 + d < p.D) ? p.lev32[(size_t)(d0 + d) * p.L + j] : 0.f;
      }
      const int d = e - Dc * P, g = d0 + d % Dc;
      return (g < p.D) ? (d < Dc ? p.fscl32[g] : p.fcen32[g]) : 0.f;
    };
    constexpr int kPre = 4;
    float pre[kPre];
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int e = threadIdx.x + 256 * k;
      pre[k] = (eh == 0 && e < nstage) ? staged(e) : 0.f;
    }
    const bool acc_ok = __all_sync(0xffffffffu, mbar_wait(bar_acc, 0, p.err, ERR_WAIT_ACC, limit));
    tc_fence_after();
    // every MMA has completed: the operand tiles' shared memory now holds this
    // pass's levels (rounded up to float) and value scales, read per dimension
    // below (levels [Dc][P], then scl[Dc], cen[Dc])
    float *s_lev = (float *)(smem + kOffA);
    float *s_scl = s_lev + Dc * P, *s_cen = s_scl + Dc;
    // s_lev, s_scl and s_cen are consecutive: element e of the staging order
    // sits at s_lev[e]
    if (eh == 0) {
#pragma unroll
      for (int k = 0; k < kPre; ++k) {
        const int e = threadIdx.x + 256 * k;
        if (e < nstage) s_lev[e] = pre[k];
      }
      for (int e = threadIdx.x + 256 * kPre; e < nstage; e += 256) s_lev[e] = staged(e);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kMmaWarp) : "memory");   // the sixteen epilogue warps
    const float dxp = geo->col[q & 15];
    const float dyp = geo->row[q >> 4];
    const uint32_t tbase = tmem + a * 256 + ((uint32_t)(32 * (warp & 3)) << 16);
    const bool read = acc_ok && any_tile;   // warp-uniform
    // The primary thread of each pixel solves and publishes z and whether the
    // value is kept ([q][0..K-1], [q][7]) past the end of the staged levels
    // (the operand tiles are free now); the other threads of the pixel read it.
    float *s_z = (float *)(smem + kOffA + kZOff);
    float z[K];
#pragma unroll
    for (int b2 = 0; b2 < K; ++b2) z[b2] = 0.f;
    int outcome = SOLVE_RECOMPUTE;
    int degu = DEG;
    bool nosup = false;
    if (primary) {
      float St[16];
      if (read) tmem_ld16(tbase, St);
      else
  #pragma unroll
        for (int j = 0; j < 16; ++j) St[j] = 0.f;
      int count;
      bool handover = false;
      bool cuncertain = false;
      if (WK == MLS_W_WENDLAND) {
        count = cflag & kCntMask;
        handover = cuncertain = count_uncertain<K>(cflag);
      } else {
        count = (int)(p.n < (1 << 30) ? p.n : (1 << 30));
        if (p.trunc_on) {
          // truncated Gaussian: the points in the pixel's box
          count = cflag & kCntMask;
          cuncertain = count_uncertain<K>(cflag);
        }
        // clipping |x~|_inf <= kRMax is exact in 16-bit arithmetic only when the
        // pixel has a point within (kRMax - |delta|_inf - 4.2) h
        const float reach = kRMax - fmaxf(fabsf(dxp), fabsf(dyp));
        handover = cuncertain || !(mst <= reach * reach - 18.f) || !read;
        {
          // the weight producers undo the split stabiliser's factor 2^-res up to kResMax
          const float *sAB0 = (const float *)(smem + lay.offPrm);
          const float res = kLog2e * mst - sAB0[q & 15] - sAB0[16 + (q >> 4)];
          handover = handover || !(res <= kResMax);
        }
      }
      nosup = (count == 0) && !cuncertain;
      if (!nosup && !handover) outcome = solve_by_count<K>(count, St, dxp, dyp, z, p, &degu);
#pragma unroll
      for (int b2 = 0; b2 < K; ++b2) s_z[q * 8 + b2] = z[b2];
      s_z[q * 8 + 7] = (!nosup && outcome != SOLVE_RECOMPUTE) ? 1.f : 0.f;
    }
    asm volatile("bar.sync 2, %0;" ::"n"(32 * kMmaWarp) : "memory");   // z published
    bool done;
    if (primary) {
      done = !nosup && outcome != SOLVE_RECOMPUTE;
    } else {
#pragma unroll
      for (int b2 = 0; b2 < K; ++b2) z[b2] = s_z[q * 8 + b2];
      done = s_z[q * 8 + 7] != 0.f;
    }
    const bool give = primary && !nosup && outcome == SOLVE_RECOMPUTE;
    const size_t plane = (size_t)p.W * p.H;
    const size_t pix = (size_t)v * p.W + u;
    float *field = (float *)p.field;
    if (primary && inside && give && d0 == 0) {
      if (p.retry_tiles) {
        // first of two passes: queue the pixel's 8-row half of the tile once
        // for the split-weight pass (the other half keeps this pass's values)
        const int ht = 2 * tile + ((v >> 3) & 1);
        if (atomicExch(&p.tile_mark[queue_i(p, ht)], 1) == 0) {
          const unsigned int k = atomicAdd(p.retry_count, 1u);
          p.retry_tiles[queue_i(p, k)] = ht;
        }
      } else {
        const unsigned int k = atomicAdd(p.relist_count, 1u);
        p.relist[list_i(p, k)] = (int)pix;
      }
    }
    if (primary && inside && nosup) {
      for (int d = d0; d < d0 + Dc && d < p.D; ++d) {
        field[(size_t)d * plane + pix] = __int_as_float(0x7fc00000);
        if (p.bands) p.bands[(size_t)d * plane + pix] = 255;
      }
    }
    // value columns in groups of 24 (K = 3, 6) or 16 (K = 1)
    constexpr int GC = (K == 1) ? 16 : 24;
    constexpr int GD = GC / K;
    for (int gbase = gfirst * GD; gbase < Dc; gbase += gstep * GD) {
      float rv[GC];
      if (read) {
        if (GC == 24) {
          float t24[24];
          tmem_ld24(tbase + 16 + gbase * K, t24);
#pragma unroll
          for (int j = 0; j < 24; ++j) rv[j] = t24[j];
        } else {
#pragma unroll
          for (int c = 0; c < GC / 16; ++c) {
            float tmp[16];
            tmem_ld16(tbase + 16 + gbase * K + 16 * c, tmp);
#pragma unroll
            for (int j = 0; j < 16; ++j) rv[16 * c + j] = tmp[j];
          }
        }
      }
      if (done && inside && read) {
        // the group's values (a column past the pass's last dimension reads
        // that dimension's scales and is not stored)
        float fv[GD];
        int row[GD];
#pragma unroll
        for (int dd = 0; dd < GD; ++dd) {
          const int d = min(gbase + dd, Dc - 1);
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < K; ++b) acc = fmaf(z[b], rv[dd * K + b], acc);
          fv[dd] = fmaf(acc, s_scl[d], s_cen[d]);
          row[dd] = d;
        }
        int band[GD];
        if (p.bands) band_labels<GD>(fv, row, s_lev, P, band);
#pragma unroll
        for (int dd = 0; dd < GD; ++dd) {
          const int d = gbase + dd;
          if (d < Dc && d0 + d < p.D) {
            const size_t o = (size_t)(d0 + d) * plane + pix;
            field[o] = fv[dd];
            if (p.bands) p.bands[o] = (uint8_t)band[dd];
          }
        }
      }
    }
    if (primary && inside && p.status && d0 == 0 && !give)
      p.status[pix] = nosup ? (uint8_t)MLS_ST_NO_SUPPORT
                            : (uint8_t)(degu | (outcome == SOLVE_FP64 ? MLS_ST_FP64_SOLVE : 0) |
                                        (degu < DEG ? MLS_ST_DEGRADED : 0));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Bounded-wait self test: waits on an mbarrier phase that nothing completes
// and reports the error code the kernel leaves behind.
__global__ void k_wait_selftest(int *err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(b, 0, err, ERR_WAIT_FULL, limit_ns);
}

template <int DEG, int WK, bool FP16, int NACC, bool WSPLIT>
void launch_one(const KParams &p, int d0, int Dc, int N, uint32_t idesc, cudaStream_t st) {
  // all tiles, or (list of half tiles) one slot per half tile of which the
  // listed ones work
  const dim3 grid = p.tile_list ? dim3((unsigned)(2 * p.tiles_x * p.tiles_y))
                                : dim3(p.tiles_x, p.tiles_y * (2 / NACC));
  auto k = k_mls_tc<DEG, WK, FP16, NACC, WSPLIT>;
  const TcLayout lay = make_layout(N, Dc);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
  k<<<grid, kThreads, lay.total, st>>>(p, d0, Dc, N, idesc, lay, d0 / Dc);
}

template <int DEG, int WK>
void launch_deg_w(const KParams &p, int fp16, int wsplit, int d0, int Dc, int N, uint32_t idesc,
                  cudaStream_t st) {
  if (fp16) {
    if (wsplit) launch_one<DEG, WK, true, 1, true>(p, d0, Dc, N, idesc, st);
    else launch_one<DEG, WK, true, 2, false>(p, d0, Dc, N, idesc, st);
  } else {
    if (wsplit) launch_one<DEG, WK, false, 1, true>(p, d0, Dc, N, idesc, st);
    else launch_one<DEG, WK, false, 2, false>(p, d0, Dc, N, idesc, st);
  }
}

}  // namespace

// Dimensions per pass so that 16 + K Dc columns fit one 256-column accumulator.
int dims_per_pass(int degree) {
  const int K = mlsk::n_terms(degree);
  const int group = (K == 1) ? 16 : 24 / K;   // the epilogue reads whole groups
  int dc = (kNMax - 16) / K;
  if (dc > kDcMax) dc = kDcMax;
  dc -= dc % group;
  return dc;
}

int tc_dims_per_pass(int D, int degree) {
  const int dmax = dims_per_pass(degree);
  const int passes = (D + dmax - 1) / dmax;
  return (D + passes - 1) / passes;   // balanced passes
}

mls_status launch_tc(const KParams &p, int fp16, int wsplit, cudaStream_t st, int *nlaunch) {
  *nlaunch = 0;
  const int K = mlsk::n_terms(p.degree);
  const int per = tc_dims_per_pass(p.D, p.degree);
  if (per != p.fb_dc) return fail(MLS_E_INVAL, "blocked value layout does not match the pass split");
  for (int d0 = 0; d0 < p.D; d0 += per) {
    const int Dc = per;   // the last pass reads zero-padded dimensions
    const int group = (K == 1) ? 16 : 24 / K;
    const int Dg = (Dc + group - 1) / group * group;    // columns the epilogue reads
    int N = 16 + Dg * K;
    N = (N + 15) / 16 * 16;
    if (N > kNMax) return fail(MLS_E_UNSUPPORTED, "operand wider than one accumulator");
    if (make_layout(N, Dc).dstages < 1) return fail(MLS_E_UNSUPPORTED, "point tile does not fit shared memory");
    const uint32_t fmt = fp16 ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
                           ((uint32_t)(kM >> 4) << 24);
    if (p.weight == MLS_W_GAUSS) {
      if (p.degree == 0) launch_deg_w<0, MLS_W_GAUSS>(p, fp16, wsplit, d0, Dc, N, idesc, st);
      else if (p.degree == 1) launch_deg_w<1, MLS_W_GAUSS>(p, fp16, wsplit, d0, Dc, N, idesc, st);
      else launch_deg_w<2, MLS_W_GAUSS>(p, fp16, wsplit, d0, Dc, N, idesc, st);
    } else if (p.weight == MLS_W_WENDLAND) {
      if (p.degree == 0) launch_deg_w<0, MLS_W_WENDLAND>(p, fp16, wsplit, d0, Dc, N, idesc, st);
      else if (p.degree == 1) launch_deg_w<1, MLS_W_WENDLAND>(p, fp16, wsplit, d0, Dc, N, idesc, st);
      else launch_deg_w<2, MLS_W_WENDLAND>(p, fp16, wsplit, d0, Dc, N, idesc, st);
    } else {
      return fail(MLS_E_UNSUPPORTED, "tensor-core path takes the Gaussian and Wendland weights");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mls_tc launch");
    ++*nlaunch;
  }
  return MLS_OK;
}

}  // namespace mlsi

extern "C" int mls_debug_wait_selftest(int64_t limit_ns, int *code_out) {
  int *d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return MLS_E_CUDA;
  cudaMemset(d, 0, sizeof(int));
  mlsi::k_wait_selftest<<<1, 32>>>(d, (uint64_t)limit_ns);
  cudaError_t e = cudaDeviceSynchronize();
  int code = 0;
  cudaMemcpy(&code, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (code_out) *code_out = code;
  return e == cudaSuccess ? MLS_OK : MLS_E_CUDA;
}
