// Device-side definitions shared by the CUDA translation units of the MLS
// library: the kernel parameter block, error words, bounded waits and the
// per-pixel moment solve (Section 3.3 of the paper: the weighted
// least-squares fit at the pixel, read off as the constant coefficient).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mls.h"

namespace mlsk {

// Device error word values (written with atomicExch, read by mls_sync).
enum : int {
  ERR_NONE = 0,
  ERR_WAIT_FULL = 1,      // MMA issuer gave up waiting for a filled stage
  ERR_WAIT_EMPTY = 2,     // producer gave up waiting for a drained stage
  ERR_WAIT_ACC = 3,       // epilogue gave up waiting for the accumulator
  ERR_CAND_OVERFLOW = 4,  // (informational) candidate list overflowed, brute force used
  ERR_INDEX = 0x100,      // checked build: ERR_INDEX + site, an index outside its array
};

// Index sites of the checked build (ERR_INDEX + site).
enum : int {
  SITE_CELL = 1,     // cell_start of the uniform grid: [gx gy + 1]
  SITE_PIXEL = 2,    // per-pixel scratch of the padded tile grid (stabiliser, counts)
  SITE_TILE = 3,     // per-tile scratch (frames, largest stabiliser): [tiles_x tiles_y]
  SITE_LIST = 4,     // hand-over lists and their pixel ids: [W H]
  SITE_QUEUE = 5,    // half-tile queue and marks: [2 tiles_x tiles_y]
  SITE_BLOCK = 6,    // 8-point blocks of the tensor path's staged copies: [n_pad / 8]
};

#ifdef MLS_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// Checked build (-DMLS_CHECKED): an index outside [0, n) records
// ERR_INDEX + site in the error word (no trap: mls_sync reports it and the
// context stays usable) and is clamped into the array, so the access itself
// stays in bounds.  In the normal build this is the index itself.
__device__ __forceinline__ int64_t chk(int *err, int64_t i, int64_t n, int site) {
  if (kChecked && (i < 0 || i >= n)) {
    if (err) atomicCAS(err, 0, ERR_INDEX + site);
    return i < 0 || n <= 0 ? 0 : n - 1;
  }
  return i;
}

// One nanosecond-resolution global timer read.
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Every bounded spin gives up after this long (the host watchdog is longer).
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Wendland support counts (prepass): bit kCntBoundary marks a pixel with a
// point whose squared distance (units of the radius) lies within
// kCntEdgeTol of 1, where FP32 and FP64 may count it differently.
constexpr int kCntBoundary = 1 << 30;
constexpr int kCntMask = kCntBoundary - 1;
constexpr float kCntEdgeTol = 4e-6f;
// Reduced-precision Gaussian renders visit, per tile, only the points within
// h sqrt(max_p m_p + kGaussOperandCut) of its pixels.  Every pair left out has
// weight below e^-28 < 2^-40 of its pixel's largest: FP16 weights (largest
// scaled to 2^14) round such a weight to exactly zero (below 2^-25), and in
// BF16 or FP32 it lies below the FP32 resolution of the sums (at most n
// e^-28 of the largest weight's share for n < 2^16 points).  FP64 renders sum
// every pair.
constexpr float kGaussOperandCut = 28.f;

// Monomials of degree <= 4 in (x, y), the entries of the moment matrix:
// 0:1 1:x 2:y 3:xx 4:xy 5:yy 6:xxx 7:xxy 8:xyy 9:yyy 10:xxxx 11:xxxy 12:xxyy 13:xyyy 14:yyyy
// Exponents (ex, ey) of monomial j.
__host__ __device__ constexpr int mono_ex(int j) {
  return j == 0 ? 0 : j == 1 ? 1 : j == 2 ? 0 : j == 3 ? 2 : j == 4 ? 1 : j == 5 ? 0
       : j == 6 ? 3 : j == 7 ? 2 : j == 8 ? 1 : j == 9 ? 0 : j == 10 ? 4 : j == 11 ? 3
       : j == 12 ? 2 : j == 13 ? 1 : 0;
}
__host__ __device__ constexpr int mono_ey(int j) {
  return j == 0 ? 0 : j == 1 ? 0 : j == 2 ? 1 : j == 3 ? 0 : j == 4 ? 1 : j == 5 ? 2
       : j == 6 ? 0 : j == 7 ? 1 : j == 8 ? 2 : j == 9 ? 3 : j == 10 ? 0 : j == 11 ? 1
       : j == 12 ? 2 : j == 13 ? 3 : 4;
}
__host__ __device__ constexpr int mono_index(int ex, int ey) {
  // inverse of (mono_ex, mono_ey) for ex + ey <= 4
  return (ex + ey) == 0 ? 0 : (ex + ey) == 1 ? 1 + ey : (ex + ey) == 2 ? 3 + ey
       : (ex + ey) == 3 ? 6 + ey : 10 + ey;
}
// Basis terms b_a (a < 6): 1, x, y, xx, xy, yy.  M_ab = S[midx(a, b)], the
// moment of the product monomial; in unrolled loops the index folds to a
// constant, so a moment array held in registers stays there.
__host__ __device__ constexpr int midx(int a, int b) {
  return mono_index(mono_ex(a) + mono_ex(b), mono_ey(a) + mono_ey(b));
}
__host__ __device__ constexpr int n_terms(int deg) { return (deg + 1) * (deg + 2) / 2; }
// number of moment monomials needed by a degree-deg basis (degree <= 2 deg)
__host__ __device__ constexpr int n_moments(int deg) { return (2 * deg + 1) * (2 * deg + 2) / 2; }
__host__ __device__ constexpr int binom(int n, int k) {
  return (k == 0 || k == n) ? 1 : (n == 2 ? 2 : n == 3 ? 3 : n == 4 ? (k == 2 ? 6 : 4) : 1);
}

// Parameters every kernel receives by value.
struct KParams {
  // points (binned order for the Wendland weight)
  int64_t n, n_pad;
  int D, D_pad;
  const float *xs, *ys;        // (x - ctr) / s, FP32, [n_pad]
  const float *xs_lo, *ys_lo;  // low parts: xs + xs_lo = (x - ctr) / s to ~48 bits
  const float *FT32;           // normalised values (f - cen) / scl, [D_pad][n_pad]
  const float *FR32;           // the same values point-major, [n_pad][D] (hand-over path)
  const float *FR32lo;         // their low parts: FR32 + FR32lo = the value to ~48 bits
  const float *fcen32, *fscl32;
  const double *fcen64, *fscl64;   // value centre and half range per dimension (FP64)
  const double *x64, *y64;     // raw positions [n]
  const double *FT64;          // raw values [D][n]
  const float *xyb;            // tensor path: (x[8], y[8], pad[4]) per 8-point block, [n_pad/8][20]
  const float *fb;             // tensor path: values per pass, [passes][n_pad/8][fb_dc * 8 + 4]
  int fb_dc;                   // dimensions per pass of fb
  const int *cell_start;       // [gx * gy + 1] (Wendland)
  int gx, gy;
  double gx0, gy0, cell;       // grid origin and cell size in raw coordinates
  double inv_cell;             // 1 / cell, formed on the host as the binning forms it
  // method
  int degree, weight;
  double h, alpha;
  double cond_fp64, rcond_min, cond_recompute;
  // the same thresholds rounded to float on the host ((float)cond_fp64,
  // (float)cond_recompute, (float)(1 / rcond_min)): GB300's FP64 pipe is a
  // small fraction of its FP32 rate, and every conversion or division of a
  // double in a per-pixel solve costs the whole warp that fraction
  float cond_fp64_f, cond_recompute_f, inv_rcond_min_f;
  float lambda_max;            // bound on sum_a |z_a| sqrt(M_00 M_aa) kept on the fast path
  // view
  int W, H;
  double x0, y0, sx, sy;       // pixel (u,v) centre = (x0 + (u+.5) sx, y0 + (v+.5) sy)
  double ctr_x, ctr_y, inv_s;  // scaled coordinate frame of xs/ys
  int tiles_x, tiles_y;        // 16 x 16 pixel tiles covering the view
  // iso-levels
  int L;
  const double *lev64;         // [D][L]
  const float *lev32;          // [D][L] rounded up to float (exact float-vs-double test)
  // outputs
  void *field;                 // [D][H][W] float or double
  int field_fp64;              // 1: field is double
  uint8_t *status;             // [H][W] or null
  uint8_t *bands;              // [D][H][W] or null
  // scratch
  const float *mstab;          // [tiles_y*16][tiles_x*16] stabiliser min r^2 / s^2
  const int *cnt;              // same shape, Wendland in-support counts
  const float *tcen;           // [tiles_y][tiles_x][2] moment frame centre of each tile (scaled)
  const float *tmax;           // [tiles_y][tiles_x] largest stabiliser of the tile's pixels (units of h^2)
  float gcut;                  // > 0: Gaussian tiles visit points within h sqrt(tmax + gcut) only
  unsigned long long *visited; // non-null: the tensor kernel adds the pixel-point pairs it visits
  int *relist;                 // pixels handed to the FP64 path
  unsigned int *relist_count;
  int *err;
  // FP64 list mode
  int *retry_tiles;            // tensor path, first of two passes: tiles to render again
  unsigned int *retry_count;   //   (appended once per tile, guarded by tile_mark)
  int *tile_mark;
  const int *tile_list;        // tensor path, second pass: the tiles to render, or null
  const unsigned int *tile_count;
  int pixel_frame;             // FP32 kernel: moments in each pixel's own frame (not the tile's)
  int f32_shape;               // FP32 kernel block shape: 0 16 x 8, 1 8 x 8, 2 8 x 4 (Gaussian)
  int variant;                 // MLS_V_*: the polynomial fit, or the rigid / mean mapping of 2-D values
  double trunc;                // truncated Gaussian: box half-width in units of h (0: full sum)
  float trunc_f;               // (float)trunc
  int trunc_on;                // trunc > 0
  const int *list;             // pixel indices, or null for all pixels
  const unsigned int *list_count;  // device count for list mode, or null
  int64_t list_cap;
};

// Indices of the library's scratch arrays, checked in the checked build.
__device__ __forceinline__ int cell_at(const KParams &p, int64_t i) {
  return p.cell_start[chk(p.err, i, (int64_t)p.gx * p.gy + 1, SITE_CELL)];
}
__device__ __forceinline__ int64_t pix_i(const KParams &p, int64_t i) {
  return chk(p.err, i, (int64_t)p.tiles_x * p.tiles_y * 256, SITE_PIXEL);
}
__device__ __forceinline__ int64_t tile_i(const KParams &p, int64_t i) {
  return chk(p.err, i, (int64_t)p.tiles_x * p.tiles_y, SITE_TILE);
}
__device__ __forceinline__ int64_t list_i(const KParams &p, int64_t i) {
  return chk(p.err, i, (int64_t)p.W * p.H, SITE_LIST);
}
__device__ __forceinline__ int64_t queue_i(const KParams &p, int64_t i) {
  return chk(p.err, i, 2 * (int64_t)p.tiles_x * p.tiles_y, SITE_QUEUE);
}

__device__ __forceinline__ void set_error(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Pixel centre in the scaled frame (FP64 arithmetic, rounded once to float).
__device__ __forceinline__ float scaled_px(const KParams &p, int u) {
  return (float)((p.x0 + ((double)u + 0.5) * p.sx - p.ctr_x) * p.inv_s);
}
__device__ __forceinline__ float scaled_py(const KParams &p, int v) {
  return (float)((p.y0 + ((double)v + 0.5) * p.sy - p.ctr_y) * p.inv_s);
}

// Iso-band label: #{j : t_j <= f}; levels rounded up to float make the float
// comparison equal to the double one.
__device__ __forceinline__ uint8_t band_of(float f, const float *lev, int L) {
  if (f != f) return 255;
  int c = 0;
  for (int j = 0; j < L; ++j) c += (lev[j] <= f) ? 1 : 0;
  return (uint8_t)c;
}
__device__ __forceinline__ uint8_t band_of(double f, const double *lev, int L) {
  if (f != f) return 255;
  int c = 0;
  for (int j = 0; j < L; ++j) c += (lev[j] <= f) ? 1 : 0;
  return (uint8_t)c;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits).  Error-free transformations
// (Knuth's two-sum; the FMA two-product), so no step relies on FP64 units.
struct df32 {
  float hi, lo;
};
__device__ __forceinline__ df32 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df32 df_quick(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  df32 s = df_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_quick(s.hi, s.lo);
}
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return df_quick(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.hi, b, -p);
  return df_quick(p, fmaf(a.lo, b, e));
}
// Double-float helpers without renormalisation, for long accumulations.
// a * b as an unevaluated pair (p, e)
__device__ __forceinline__ df32 df_prod(df32 a, df32 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return {p, e};
}
__device__ __forceinline__ df32 df_prod_f(df32 a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return {p, e};
}
// s += x (two-sum on the high parts, low parts summed)
__device__ __forceinline__ void df_acc(df32 &s, df32 x) {
  const float t = s.hi + x.hi;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (x.hi - bb);
  s.lo += err + x.lo;
  s.hi = t;
}
// (ahi + alo) - (bhi + blo)
__device__ __forceinline__ df32 df_diff(float ahi, float alo, float bhi, float blo) {
  df32 s = df_two_sum(ahi, -bhi);
  s.lo += alo - blo;
  return df_quick(s.hi, s.lo);
}

// Table of 2^(j/64), j = 0..63, as double-float pairs, for df_exp.  Filled
// once per block (FP64 exp2 of 64 arguments) by df_exp_table_init.
__device__ __forceinline__ void df_exp_table_init(float2 *tab) {
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    const double v = exp2((double)j / 64.0);
    tab[j] = make_float2((float)v, (float)(v - (double)(float)v));
  }
}

// exp(a) of a double-float argument, -70 <= a <= 1, in FP32 arithmetic, to
// about 1e-14 relative (below -70 the low part of the result is subnormal).  Table-driven method of P. T. P. Tang (ACM TOMS
// 15(2), 1989): a = (64 k + j) ln2/64 + r with |r| <= ln2/128, so that
// exp(a) = 2^k 2^(j/64) exp(r); exp(r) - 1 from its Taylor series, the
// first two terms in double-float and the rest (below 3e-8) in FP32.
// ln2/64 = C1 + C2 + C3 with C1 of 10 significant bits, so that N C1 is
// exact for |N| < 2^14 and a - N C1 is exact.
__device__ __forceinline__ df32 df_exp(df32 a, const float2 *tab) {
  constexpr float kInvC = 92.332481384277344f;        // 64 / ln 2 (rounded)
  constexpr float C1 = 0.010833740234375f;           // 710 / 2^16
  constexpr float C2 = -3.3155381515825866e-06f;
  constexpr float C3 = 2.5727683872212026e-14f;
  const float N = rintf(a.hi * kInvC);
  const float t = fmaf(-N, C1, a.hi);                // exact
  df32 r = df_two_sum(t, a.lo);
  const float p2 = N * C2, e2 = fmaf(N, C2, -p2);    // N C2 exactly
  r = df_add(r, {-p2, -e2});
  r = df_add(r, {-N * C3, 0.f});
  const df32 r2 = df_mul(r, r);
  const float q = r.hi;
  const float tail = q * q * q * fmaf(q, fmaf(q, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f);
  df32 e = df_add(r, {0.5f * r2.hi, 0.5f * r2.lo});
  e = df_add(e, {tail, 0.f});
  const df32 one_e = df_add({1.f, 0.f}, e);
  const int Ni = (int)N;
  const int j = Ni & 63, k = Ni >> 6;                // N = 64 k + j, 0 <= j < 64
  const float2 T = tab[j];
  const df32 w = df_mul({T.x, T.y}, one_e);
  const float scale = __int_as_float((k + 127) << 23);   // 2^k, normal for k >= -126
  return {w.hi * scale, w.lo * scale};
}

// sqrt of a double-float r >= 0: the FP32 root corrected by one Newton step
// on the residual (Karp and Markstein, ACM TOMS 23(4), 1997).
__device__ __forceinline__ df32 df_sqrt(df32 r) {
  if (!(r.hi > 0.f)) return {0.f, 0.f};
  const float s = sqrtf(r.hi);
  const float res = fmaf(-s, s, r.hi) + r.lo;        // r - s^2
  return df_quick(s, res / (2.f * s));
}

// Wendland C2 weight (1 - q)^4 (4 q + 1) at q = sqrt(r2) < 1, double-float.
__device__ __forceinline__ df32 df_wendland(df32 r2) {
  const df32 q = df_sqrt(r2);
  const df32 o = df_add({1.f, 0.f}, {-q.hi, -q.lo});
  const df32 o2 = df_mul(o, o);
  const df32 q4 = df_add({1.f, 0.f}, {4.f * q.hi, 4.f * q.lo});
  return df_mul(df_mul(o2, o2), q4);
}

// ---------------------------------------------------------------------------
// Small dense linear algebra on the K x K moment matrix (K = 1, 3, 6).

// Cholesky factor L of the SPD matrix A, and the reciprocals of its pivots
// (the triangular solves multiply by them instead of dividing).
template <int K, typename T>
__device__ __forceinline__ bool cholesky(const T (&A)[K][K], T (&L)[K][K], T (&dinv)[K]) {
#pragma unroll
  for (int j = 0; j < K; ++j) {
    T s = A[j][j];
#pragma unroll
    for (int t = 0; t < j; ++t) s -= L[j][t] * L[j][t];
    if (!(s > T(0))) return false;
    const T ljj = sqrt(s);
    const T inv = T(1) / ljj;
    L[j][j] = ljj;
    dinv[j] = inv;
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      T v = A[i][j];
#pragma unroll
      for (int t = 0; t < j; ++t) v -= L[i][t] * L[j][t];
      L[i][j] = v * inv;
    }
#pragma unroll
    for (int i = 0; i < j; ++i) L[i][j] = T(0);
  }
  return true;
}

template <int K, typename T>
__device__ __forceinline__ void chol_solve(const T (&L)[K][K], const T (&dinv)[K], T (&x)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T v = x[i];
#pragma unroll
    for (int t = 0; t < i; ++t) v -= L[i][t] * x[t];
    x[i] = v * dinv[i];
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
    T v = x[i];
#pragma unroll
    for (int t = i + 1; t < K; ++t) v -= L[t][i] * x[t];
    x[i] = v * dinv[i];
  }
}

// 1-norm condition number of the SPD matrix A from its Cholesky factor.
template <int K, typename T>
__device__ __forceinline__ T cond1(const T (&A)[K][K], const T (&L)[K][K], const T (&dinv)[K]) {
  T nA = 0, nI = 0;
#pragma unroll
  for (int c = 0; c < K; ++c) {
    T col[K];
#pragma unroll
    for (int a = 0; a < K; ++a) col[a] = (a == c) ? T(1) : T(0);
    chol_solve<K, T>(L, dinv, col);
    T s = 0, sa = 0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      s += fabs(col[a]);
      sa += fabs(A[a][c]);
    }
    nI = s > nI ? s : nI;
    nA = sa > nA ? sa : nA;
  }
  return nA * nI;
}

// Outcome of the reduced-precision per-pixel solve.
enum SolveOutcome : int { SOLVE_OK = 0, SOLVE_FP64 = 1, SOLVE_RECOMPUTE = 2 };

// Solve M z = b for the moment matrix given by its distinct moments S in a
// frame whose origin is offset from the pixel by -delta, with b = b(delta) the
// basis at the pixel: the fit's value is then z . R for the right-hand sides
// R taken in the same frame.  FP32 equilibrated Cholesky, a 1-norm condition
// estimate, one step of iterative refinement; FP64 factorisation when the
// estimate exceeds cond_fp64; SOLVE_RECOMPUTE when it exceeds cond_recompute,
// when the factorisation fails, or when the pixel-frame condition (bounded by
// the frame condition times the growth of the basis under the shift) could
// come near the degeneracy threshold.  Recomputed pixels go to the hand-over
// path, which applies the full degree policy.
template <int K>
__device__ __forceinline__ int solve_pixel_fp32(const float *S, float dx, float dy, float (&z)[K],
                                                const KParams &p) {
  float M[K][K];
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b < K; ++b) M[a][b] = S[midx(a, b)];
  float bv[6] = {1.f, dx, dy, dx * dx, dx * dy, dy * dy};
  float sd[K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    if (!(M[a][a] > 0.f)) return SOLVE_RECOMPUTE;
    sd[a] = rsqrtf(M[a][a]);
  }
  float Me[K][K], Lf[K][K], df[K];
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b < K; ++b) Me[a][b] = M[a][b] * sd[a] * sd[b];
  if (!cholesky<K, float>(Me, Lf, df)) return SOLVE_RECOMPUTE;
  // a pivot this small means a condition beyond what FP32 can estimate
#pragma unroll
  for (int a = 0; a < K; ++a)
    if (!(Lf[a][a] * Lf[a][a] > 1e-6f)) return SOLVE_RECOMPUTE;
  const float cnd = (K == 1) ? 1.f : cond1<K, float>(Me, Lf, df);
  if (!(cnd <= p.cond_recompute_f)) return SOLVE_RECOMPUTE;
  if (K > 1) {
    const float gr = 1.f + fmaxf(fabsf(dx), fabsf(dy));
    const float g2 = gr * gr;
    const float growth = (K == 3) ? g2 : g2 * g2;
    if (!(cnd * growth * 100.f < p.inv_rcond_min_f)) return SOLVE_RECOMPUTE;
  }
  if (cnd > p.cond_fp64_f) {
    // FP64 factorisation of the same moments
    double Md[K][K], sdd[K], Med[K][K], Ld[K][K], dd[K];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = 0; b < K; ++b) Md[a][b] = (double)M[a][b];
#pragma unroll
    for (int a = 0; a < K; ++a) sdd[a] = 1.0 / sqrt(Md[a][a]);
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = 0; b < K; ++b) Med[a][b] = Md[a][b] * sdd[a] * sdd[b];
    if (!cholesky<K, double>(Med, Ld, dd)) return SOLVE_RECOMPUTE;
    double y[K];
#pragma unroll
    for (int a = 0; a < K; ++a) y[a] = (double)bv[a] * sdd[a];
    chol_solve<K, double>(Ld, dd, y);
#pragma unroll
    for (int a = 0; a < K; ++a) z[a] = (float)(y[a] * sdd[a]);
    return SOLVE_FP64;
  }
  // z = S Me^{-1} S b
  float y[K];
#pragma unroll
  for (int a = 0; a < K; ++a) y[a] = bv[a] * sd[a];
  chol_solve<K, float>(Lf, df, y);
#pragma unroll
  for (int a = 0; a < K; ++a) z[a] = y[a] * sd[a];
  // one refinement step: r = b - M z, z += M^{-1} r
  float r[K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    float acc = bv[a];
#pragma unroll
    for (int b = 0; b < K; ++b) acc = fmaf(-M[a][b], z[b], acc);
    r[a] = acc * sd[a];
  }
  chol_solve<K, float>(Lf, df, r);
#pragma unroll
  for (int a = 0; a < K; ++a) z[a] = fmaf(r[a], sd[a], z[a]);
  // rounding of each right-hand side R_a moves the value by at most about
  // eps * sqrt(M_00 M_aa) |z_a| (Cauchy-Schwarz): keep the pixel only when
  // that amplification is small
  float lambda = 0.f;
#pragma unroll
  for (int a = 0; a < K; ++a) lambda = fmaf(fabsf(z[a]), sqrtf(M[0][0] * M[a][a]), lambda);
  if (!(lambda <= p.lambda_max)) return SOLVE_RECOMPUTE;
  return SOLVE_OK;
}

// Degree policy by support count (Wendland), then the FP32 solve: the highest
// degree whose n_terms fits the count, using the leading block of the same
// moments; z is zero past that degree's terms.  Returns the solve outcome and
// the degree in *deg (the count is exact unless the boundary flag is set).
template <int K>
__device__ __forceinline__ int solve_by_count(int count, const float *S, float dx, float dy, float (&z)[K],
                                              const KParams &p, int *deg) {
#pragma unroll
  for (int a = 0; a < K; ++a) z[a] = 0.f;
  if (count >= K) {
    *deg = (K == 6) ? 2 : (K == 3) ? 1 : 0;
    return solve_pixel_fp32<K>(S, dx, dy, z, p);
  }
  if (K == 6 && count >= 3) {
    float z3[3];
    *deg = 1;
    const int o = solve_pixel_fp32<3>(S, dx, dy, z3, p);
#pragma unroll
    for (int a = 0; a < 3; ++a) z[a] = z3[a];
    return o;
  }
  float z1[1];
  *deg = 0;
  const int o = solve_pixel_fp32<1>(S, dx, dy, z1, p);
  z[0] = z1[0];
  return o;
}

// Whether a boundary-flagged count could cross a degree threshold (count
// within one of n_terms for some degree <= DEG): such pixels go to the FP64
// definition.
template <int K>
__device__ __forceinline__ bool count_uncertain(int cflag) {
  if (!(cflag & kCntBoundary)) return false;
  const int c = cflag & kCntMask;
  return (c >= 0 && c <= 2) || (K >= 3 && c >= 2 && c <= 4) || (K >= 6 && c >= 5 && c <= 7);
}

}  // namespace mlsk
