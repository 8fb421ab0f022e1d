// CUDA-core MLS kernels: the plain FP32 form (one thread per pixel, points
// staged through shared memory), the FP64 form (one warp per pixel, used for
// FP64 renders and for the pixels the reduced-precision paths hand over),
// and the standalone iso-band labelling.
//
// Per pixel p and point x_i (Section 3.3 of the paper, generalised to D data
// dimensions): w_i = w(|x_i - p|); with d_i = (x_i - p)/h and basis
// b = (1, d_x, d_y, d_x^2, d_x d_y, d_y^2) truncated to the degree,
// M = sum w b b^T is held as its distinct moments sum w d^a (|a| <= 2 deg)
// and R = sum w b f^T; the fit's value is e0 . M^{-1} R.
#include <float.h>
#include <string.h>

#include <algorithm>

#include "mls_internal.h"

namespace mlsi {
namespace {

using namespace mlsk;

constexpr float kLog2e = 1.4426950408889634f;

// Monomials of degree <= 4 of (dx, dy) (the moment index order of midx).
template <int NM>
__device__ __forceinline__ void monomials(float dx, float dy, float (&m)[15]) {
  m[0] = 1.f;
  if (NM > 1) {
    m[1] = dx; m[2] = dy;
    m[3] = dx * dx; m[4] = dx * dy; m[5] = dy * dy;
  }
  if (NM > 6) {
    m[6] = m[3] * dx; m[7] = m[3] * dy; m[8] = m[5] * dx; m[9] = m[5] * dy;
    m[10] = m[3] * m[3]; m[11] = m[3] * m[4]; m[12] = m[3] * m[5]; m[13] = m[4] * m[5]; m[14] = m[5] * m[5];
  }
}

__device__ __forceinline__ void cell_range_d(double lo, double hi, double r, double g0, double inv_cell, int g,
                                             int &c0, int &c1) {
  c0 = (int)floor((lo - r - g0) * inv_cell);
  c1 = (int)floor((hi + r - g0) * inv_cell);
  c0 = max(c0, 0);
  c1 = min(c1, g - 1);
}

// ---------------------------------------------------------------------------
// Plain FP32: one thread per pixel, 16 x 8 pixels per block.
constexpr int kF32Chunk = 128;
constexpr int kF32DC = 16;

// Block shapes of the FP32 kernel (KParams.f32_shape): BW x BH pixels, one
// thread each.  A block visits the points within reach of all its pixels, so
// where the reach is a few pixels a smaller block visits fewer points per
// pixel, while a larger one reuses each staged point over more threads; the
// batch autotuner times the shapes per dataset.
template <int DEG, int WK, int BW, int BH>
__global__ __launch_bounds__(BW * BH) void k_mls_f32(KParams p) {
  constexpr int K = n_terms(DEG), NM = n_moments(DEG), DC = kF32DC;
  constexpr int NT = BW * BH;
  __shared__ float sx[kF32Chunk], sy[kF32Chunk];
  __shared__ float sf[DC][kF32Chunk];
  // block geometry, formed once in FP64 (GB300's FP64 rate is a small
  // fraction of FP32's): frame offsets of the BW columns and BH rows, cell range
  __shared__ float s_col[BW], s_row[BH];
  __shared__ int s_rng[4];
  const int t = threadIdx.x;
  const int bu0 = blockIdx.x * BW, bv0 = blockIdx.y * BH;
  const int u = bu0 + t % BW, v = bv0 + t / BW;
  const bool inside = (u < p.W) && (v < p.H);
  // moments in the frame of the tile's weighted centroid (see the prepass),
  // (dpx, dpy) = pixel minus frame origin; or, when the tile is large
  // compared with h (p.pixel_frame), in each pixel's own frame
  const int tile = (bv0 >> 4) * p.tiles_x + (bu0 >> 4);
  const float cxs = p.tcen[2 * tile_i(p, tile)], cys = p.tcen[2 * tile_i(p, tile) + 1];
  if (t < BW) s_col[t] = (float)((p.x0 + (bu0 + t + 0.5) * p.sx - p.ctr_x) * p.inv_s - (double)cxs);
  else if (t < BW + BH) s_row[t - BW] = (float)((p.y0 + (bv0 + t - BW + 0.5) * p.sy - p.ctr_y) * p.inv_s - (double)cys);
  const size_t pstride = (size_t)p.tiles_x * 16;
  // compact support: the Wendland weight, or the truncated Gaussian's box |dx|, |dy| < c
  const bool binned = (WK == MLS_W_WENDLAND) || (WK == MLS_W_GAUSS && p.trunc > 0.0);
  const float cbox = (WK == MLS_W_GAUSS && p.trunc > 0.0) ? (float)p.trunc : INFINITY;
  const float m = (WK == MLS_W_WENDLAND) ? 0.f : p.mstab[pix_i(p, (int64_t)v * pstride + u)];
  const int cflag = binned ? p.cnt[pix_i(p, (int64_t)v * pstride + u)] : 0;
  const int count = binned ? (cflag & kCntMask) : (int)(p.n < (1 << 30) ? p.n : (1 << 30));
  const float alpha = (float)p.alpha;
  // point ranges: all points, or the cell rows overlapping the block's pixels
  // +- h (+- c h; Gaussian: +- h sqrt(max m + gcut), beyond which every weight
  // is below FP32 resolution of the sums)
  const bool cut = (WK == MLS_W_GAUSS) && !binned && p.gcut > 0.f;
  if ((binned || cut) && t == BW + BH) {
    const double rad = (WK == MLS_W_WENDLAND) ? p.h
                       : binned ? p.trunc * p.h * (1.0 + 1e-5)
                                : p.h * (double)sqrtf(p.tmax[tile_i(p, tile)] + p.gcut) * (1.0 + 1e-5);
    const double xa = p.x0 + (bu0 + 0.5) * p.sx, xb = p.x0 + (bu0 + BW - 0.5) * p.sx;
    const double ya = p.y0 + (bv0 + 0.5) * p.sy, yb = p.y0 + (bv0 + BH - 0.5) * p.sy;
    cell_range_d(fmin(xa, xb), fmax(xa, xb), rad, p.gx0, p.inv_cell, p.gx, s_rng[0], s_rng[1]);
    cell_range_d(fmin(ya, yb), fmax(ya, yb), rad, p.gy0, p.inv_cell, p.gy, s_rng[2], s_rng[3]);
  }
  __syncthreads();
  const float dpx = s_col[t % BW], dpy = s_row[t / BW];
  int nr = 1, cx0 = 0, cx1 = 0, cy0 = 0;
  if (binned || cut) {
    cx0 = s_rng[0];
    cx1 = s_rng[1];
    cy0 = s_rng[2];
    nr = (cx0 <= cx1) ? max(s_rng[3] - cy0 + 1, 0) : 0;
  }
  const size_t plane = (size_t)p.W * p.H;
  const size_t pix = (size_t)v * p.W + u;
  float *field = (float *)p.field;
  bool handed_over = false;
  uint8_t st = 0;

  for (int d0 = 0; d0 < p.D; d0 += DC) {
    float S[15], R[K][DC];
#pragma unroll
    for (int j = 0; j < 15; ++j) S[j] = 0.f;
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int dd = 0; dd < DC; ++dd) R[a][dd] = 0.f;
    float csum[DC];
    int ccnt = 0;
#pragma unroll
    for (int dd = 0; dd < DC; ++dd) csum[dd] = 0.f;
    for (int r = 0; r < nr; ++r) {
      int a0, a1;
      if (binned || cut) {
        a0 = cell_at(p, (int64_t)(cy0 + r) * p.gx + cx0);
        a1 = cell_at(p, (int64_t)(cy0 + r) * p.gx + cx1 + 1);
      } else {
        a0 = 0;
        a1 = (int)p.n;
      }
      for (int base = a0; base < a1; base += kF32Chunk) {
        __syncthreads();
        const int cnt = min(kF32Chunk, a1 - base);
        for (int j = t; j < cnt; j += NT) {
          sx[j] = p.xs[base + j] - cxs;
          sy[j] = p.ys[base + j] - cys;
        }
        for (int e = t; e < DC * kF32Chunk; e += NT) {
          const int dd = e / kF32Chunk, j = e % kF32Chunk;
          sf[dd][j] = (j < cnt) ? p.FT32[(size_t)(d0 + dd) * p.n_pad + base + j] : 0.f;
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
          const float dx = sx[j], dy = sy[j];               // frame coordinates
          const float qx = dx - dpx, qy = dy - dpy;         // from the pixel
          const float r2 = fmaf(qx, qx, qy * qy);
          float w;
          if (WK == MLS_W_GAUSS) {
            w = (fabsf(qx) < cbox && fabsf(qy) < cbox) ? exp2f((m - r2) * kLog2e) : 0.f;
          } else if (WK == MLS_W_WENDLAND) {
            const float q = sqrtf(r2);
            const float o = 1.f - q;
            const float o2 = o * o;
            w = (q < 1.f) ? o2 * o2 * fmaf(4.f, q, 1.f) : 0.f;
          } else {
            if (r2 == 0.f) {
              ++ccnt;
#pragma unroll
              for (int dd = 0; dd < DC; ++dd) csum[dd] += sf[dd][j];
              w = 0.f;
            } else {
              w = exp2f(alpha * __log2f(m / r2));
            }
          }
          float mo[15];
          if (p.pixel_frame) monomials<NM>(qx, qy, mo);
          else monomials<NM>(dx, dy, mo);
#pragma unroll
          for (int q = 0; q < NM; ++q) S[q] = fmaf(w, mo[q], S[q]);
#pragma unroll
          for (int a = 0; a < K; ++a) {
            const float wb = w * mo[a];
#pragma unroll
            for (int dd = 0; dd < DC; ++dd) R[a][dd] = fmaf(wb, sf[dd][j], R[a][dd]);
          }
        }
      }
    }
    if (p.visited && d0 == 0 && t == 0) {
      // pixel-point pairs of this block (points in its ranges x its pixels)
      unsigned long long npts = 0;
      for (int r = 0; r < nr; ++r)
        npts += (binned || cut) ? (unsigned long long)(cell_at(p, (int64_t)(cy0 + r) * p.gx + cx1 + 1) -
                                                       cell_at(p, (int64_t)(cy0 + r) * p.gx + cx0))
                                : (unsigned long long)p.n;
      if (npts) atomicAdd(p.visited, npts * (unsigned long long)NT);
    }
    // --- per-pixel solve
    if (!inside) continue;
    float z[K];
    bool write = true;
    if (WK == MLS_W_INVDIST && ccnt > 0) {
      st = MLS_ST_COINCIDENT;
#pragma unroll
      for (int dd = 0; dd < DC; ++dd) {
        const int d = d0 + dd;
        if (d < p.D) {
          const float f = fmaf(csum[dd] / (float)ccnt, p.fscl32[d], p.fcen32[d]);
          field[(size_t)d * plane + pix] = f;
          if (p.bands) p.bands[(size_t)d * plane + pix] = band_of(f, p.lev32 + (size_t)d * p.L, p.L);
        }
      }
      continue;
    }
    const bool uncertain = binned && count_uncertain<K>(cflag);
    if (count == 0 && !uncertain) {
      st = MLS_ST_NO_SUPPORT;
#pragma unroll
      for (int dd = 0; dd < DC; ++dd) {
        const int d = d0 + dd;
        if (d < p.D) {
          field[(size_t)d * plane + pix] = __int_as_float(0x7fc00000);
          if (p.bands) p.bands[(size_t)d * plane + pix] = 255;
        }
      }
      continue;
    }
    int outcome = SOLVE_RECOMPUTE;
    int degu = DEG;
    // the count rule of the degree policy; pixels whose count could differ
    // from the FP64 count at a degree threshold go to the FP64 path
    if (!uncertain)
      outcome = solve_by_count<K>(count, S, p.pixel_frame ? 0.f : dpx, p.pixel_frame ? 0.f : dpy, z, p, &degu);
    if (outcome == SOLVE_RECOMPUTE) {
      write = false;
      if (d0 == 0) {
        const unsigned int k = atomicAdd(p.relist_count, 1u);
        p.relist[list_i(p, k)] = (int)pix;
      }
      handed_over = true;
    } else {
      st = (uint8_t)(degu | (outcome == SOLVE_FP64 ? MLS_ST_FP64_SOLVE : 0) | (degu < DEG ? MLS_ST_DEGRADED : 0));
    }
    if (write) {
#pragma unroll
      for (int dd = 0; dd < DC; ++dd) {
        const int d = d0 + dd;
        if (d < p.D) {
          float acc = 0.f;
#pragma unroll
          for (int a = 0; a < K; ++a) acc = fmaf(z[a], R[a][dd], acc);
          const float f = fmaf(acc, p.fscl32[d], p.fcen32[d]);
          field[(size_t)d * plane + pix] = f;
          if (p.bands) p.bands[(size_t)d * plane + pix] = band_of(f, p.lev32 + (size_t)d * p.L, p.L);
        }
      }
    }
  }
  if (inside && !handed_over && p.status) p.status[pix] = st;
}

// ---------------------------------------------------------------------------
// FP64: one warp per pixel; lanes split the points, moments are summed by a
// butterfly reduction, every lane applies the full degree policy.
constexpr int kF64DC = 8;
// On the hand-over path (pixels recomputed for a reduced-precision render)
// Gaussian pairs with (r^2 - m)/h^2 above this are not accumulated: their
// weight is below e^-60 of the largest, which leaves every moment unchanged
// at FP64 rounding unless the significant points alone are degenerate for
// the basis.  FP64 renders sum every pair.
constexpr double kGaussCut = 60.0;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-lane cache of the points with a positive weight (index and weight),
// filled while the first DC dimensions are summed: the later dimension
// chunks of the same pixel read it instead of recomputing every candidate's
// distance and weight (the moments and the degree policy do not change with
// the dimensions).  Bit-identical: each lane sums its points in the same order.
constexpr int kF64Slots = 24;                  // cache entries per lane
constexpr int kF64SmemBytes = 8 * kF64Slots * 32 * (4 + 8);

// Degree policy of the FP64 definition on the distinct moments S (every lane
// of a warp, identical arithmetic): the highest degree whose support count
// suffices, whose equilibrated matrix factorises and whose rcond_1 reaches
// rcond_min.  Returns the degree (-1: none) and, with k its basis terms, the
// fit's weights on the right-hand sides, zc_c = s_0 (Me^-1)_c0 s_c with s
// the equilibration (the value is sum_c zc_c R_c: column 0 of the inverse,
// the one solve Me z = e_0, whose rounding grows with the condition once).
template <int DEG>
__device__ __forceinline__ int f64_policy(const double (&S)[15], int64_t count, double rcond_min, double (&zc)[6],
                                          int &k_out) {
  int used = -1;
  for (int deg = DEG; deg >= 0 && used < 0; --deg) {
    const int k = n_terms(deg);
    if (count < k) continue;
    double Mm[6][6], sdg[6], Me[6][6], Lm[6][6];
    bool ok = true;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) Mm[a][b] = S[midx(a, b)];
    for (int a = 0; a < k && ok; ++a) {
      if (!(Mm[a][a] > 0.0)) ok = false;
      else sdg[a] = 1.0 / sqrt(Mm[a][a]);
    }
    if (!ok) continue;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) Me[a][b] = Mm[a][b] * sdg[a] * sdg[b];
    // Cholesky
    for (int j = 0; j < k && ok; ++j) {
      double s = Me[j][j];
      for (int tt = 0; tt < j; ++tt) s -= Lm[j][tt] * Lm[j][tt];
      if (!(s > 0.0)) { ok = false; break; }
      const double ljj = sqrt(s);
      Lm[j][j] = ljj;
      for (int i2 = j + 1; i2 < k; ++i2) {
        double vv = Me[i2][j];
        for (int tt = 0; tt < j; ++tt) vv -= Lm[i2][tt] * Lm[j][tt];
        Lm[i2][j] = vv / ljj;
      }
    }
    if (!ok) continue;
    // inverse, rcond_1
    double Inv[6][6];
    for (int c = 0; c < k; ++c) {
      double col[6];
      for (int a = 0; a < k; ++a) col[a] = (a == c) ? 1.0 : 0.0;
      for (int i2 = 0; i2 < k; ++i2) {
        double vv = col[i2];
        for (int tt = 0; tt < i2; ++tt) vv -= Lm[i2][tt] * col[tt];
        col[i2] = vv / Lm[i2][i2];
      }
      for (int i2 = k - 1; i2 >= 0; --i2) {
        double vv = col[i2];
        for (int tt = i2 + 1; tt < k; ++tt) vv -= Lm[tt][i2] * col[tt];
        col[i2] = vv / Lm[i2][i2];
      }
      for (int a = 0; a < k; ++a) Inv[a][c] = col[a];
    }
    double nA = 0.0, nI = 0.0;
    for (int c = 0; c < k; ++c) {
      double sa = 0.0, si = 0.0;
      for (int a = 0; a < k; ++a) { sa += fabs(Me[a][c]); si += fabs(Inv[a][c]); }
      nA = fmax(nA, sa);
      nI = fmax(nI, si);
    }
    const double rc = 1.0 / (nA * nI);
    if (!(rc >= rcond_min)) continue;
    for (int c = 0; c < k; ++c) zc[c] = sdg[0] * Inv[c][0] * sdg[c];
    used = deg;
    k_out = k;
  }
  return used;
}

template <int DEG, int WK, typename OutT>
__global__ __launch_bounds__(256) void k_mls_f64(KParams p, int64_t npix_all) {
  constexpr int NM = n_moments(DEG), DC = kF64DC;
  const int lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char f64_smem[];
  double *c_w = (double *)f64_smem + (size_t)(threadIdx.x >> 5) * kF64Slots * 32;            // [slot][lane]
  int *c_i = (int *)(f64_smem + (size_t)8 * kF64Slots * 32 * 8) + (size_t)(threadIdx.x >> 5) * kF64Slots * 32;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t npix = p.list ? (int64_t)((int64_t)*p.list_count < p.list_cap ? (int64_t)*p.list_count : p.list_cap)
                              : npix_all;
  const size_t plane = (size_t)p.W * p.H;
  const double inv_s = 1.0 / p.h;
  const double h2 = p.h * p.h;
  const int64_t n = p.n;
  OutT *field = (OutT *)p.field;
  // compact support: the Wendland weight, or the truncated Gaussian's box
  // |x_i - p_x|, |y_i - p_y| < rho = c h
  const bool binned = (WK == MLS_W_WENDLAND) || (WK == MLS_W_GAUSS && p.trunc > 0.0);
  const double rho = p.trunc * p.h;

  for (int64_t q = warp0; q < npix; q += nwarps) {
    const int64_t id = p.list ? list_i(p, p.list[list_i(p, q)]) : q;
    const int u = (int)(id % p.W), v = (int)(id / p.W);
    // the same expression order as the FP64 definition, without contraction
    const double px = __dadd_rn(p.x0, __dmul_rn(__dadd_rn((double)u, 0.5), p.sx));
    const double py = __dadd_rn(p.y0, __dmul_rn(__dadd_rn((double)v, 0.5), p.sy));
    // candidate ranges: all points, or the cell rows cy0..cy0+nr-1 (columns
    // cx0..cx1) covering the support (Wendland), the box (truncated Gaussian),
    // or, for listed pixels of the Gaussian, the reach r^2 <= m + kGaussCut h^2
    // of the pairs the list tier sums (the others are skipped below anyway)
    const float mlist = (p.list && WK == MLS_W_GAUSS) ? p.mstab[pix_i(p, (int64_t)v * (p.tiles_x * 16) + u)] : 0.f;
    const bool reach = (WK == MLS_W_GAUSS) && p.list && !binned && p.cell_start != nullptr;
    int nr = 1, cx0 = 0, cx1 = 0, cy0 = 0;
    if (binned || reach) {
      const double inv_cell = p.inv_cell;
      const double rad = (WK == MLS_W_WENDLAND) ? p.h
                         : binned ? rho * (1.0 + 1e-5)
                                  : p.h * sqrt(fmax((double)mlist, 0.0) + kGaussCut + 1.0) * (1.0 + 1e-5);
      int cy1;
      cell_range_d(px, px, rad, p.gx0, inv_cell, p.gx, cx0, cx1);
      cell_range_d(py, py, rad, p.gy0, inv_cell, p.gy, cy0, cy1);
      nr = (cx0 <= cx1) ? max(cy1 - cy0 + 1, 0) : 0;
    }
    // stabiliser m = min r^2 (Gaussian, inverse distance); hand-over lists
    // take the prepass value (any common weight factor leaves the fit unchanged)
    double m = 0.0;
    const float mhat = (p.list && WK != MLS_W_WENDLAND) ? p.mstab[pix_i(p, (int64_t)v * (p.tiles_x * 16) + u)] : 0.f;
    const float pxs = scaled_px(p, u), pys = scaled_py(p, v);
    if (p.list && WK != MLS_W_WENDLAND) {
      m = (double)mhat * h2;
    } else if (WK != MLS_W_WENDLAND) {
      double mm = DBL_MAX;
      for (int64_t i = lane; i < n; i += 32) {
        const double dx = __dadd_rn(p.x64[i], -px), dy = __dadd_rn(p.y64[i], -py);
        mm = fmin(mm, __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mm = fmin(mm, __shfl_xor_sync(0xffffffffu, mm, o));
      m = mm;
    }
    const bool coincident = (WK == MLS_W_INVDIST) && (m == 0.0);
    uint8_t st = MLS_ST_RECOMPUTED;
    // moments, count and policy of the first chunk, reused by the later ones
    // when every lane's positive-weight points fit its cache (not for the
    // inverse distance, whose coincident points take the other branch)
    double S[15];
    int64_t count = 0;
    int ncache = 0;
    bool cached = false;
    int used_saved = -1, k_saved = 1;
    double zc_saved[6];
    for (int d0 = 0; d0 < p.D; d0 += DC) {
      double R[6][DC], csum[DC];
      int64_t ccnt = 0;
      const bool fresh = !cached;
      if (fresh) {
        count = 0;
        ncache = 0;
#pragma unroll
        for (int j = 0; j < 15; ++j) S[j] = 0.0;
      }
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int dd = 0; dd < DC; ++dd) R[a][dd] = 0.0;
#pragma unroll
      for (int dd = 0; dd < DC; ++dd) csum[dd] = 0.0;
      if (!fresh) {
        // the cached points: same order, same weights and basis terms
        for (int k = 0; k < ncache; ++k) {
          const double w = c_w[k * 32 + lane];
          const int64_t i = c_i[k * 32 + lane];
          const double dx = __dadd_rn(p.x64[i], -px), dy = __dadd_rn(p.y64[i], -py);
          const double ddx = dx * inv_s, ddy = dy * inv_s;
          double mo[6];
          mo[0] = 1.0;
          if (NM > 1) {
            mo[1] = ddx; mo[2] = ddy; mo[3] = ddx * ddx; mo[4] = ddx * ddy; mo[5] = ddy * ddy;
          }
          double fv[DC];
#pragma unroll
          for (int dd = 0; dd < DC; ++dd) fv[dd] = (d0 + dd < p.D) ? p.FT64[(size_t)(d0 + dd) * n + i] : 0.0;
#pragma unroll
          for (int a = 0; a < n_terms(DEG); ++a) {
            const double wb = w * mo[a];
#pragma unroll
            for (int dd = 0; dd < DC; ++dd) R[a][dd] += wb * fv[dd];
          }
        }
      }
      for (int r = 0; r < nr && fresh; ++r) {
        const int64_t a0 = (binned || reach) ? cell_at(p, (int64_t)(cy0 + r) * p.gx + cx0) : 0;
        const int64_t a1 = (binned || reach) ? cell_at(p, (int64_t)(cy0 + r) * p.gx + cx1 + 1) : n;
        for (int64_t i = a0 + lane; i < a1; i += 32) {
          if (WK == MLS_W_GAUSS && p.list && !binned) {
            // conservative FP32 test before any FP64 work on far pairs
            const float dxs = p.xs[i] - pxs, dys = p.ys[i] - pys;
            if (fmaf(dxs, dxs, dys * dys) - mhat > (float)kGaussCut + 1.f) {
              ++count;
              continue;
            }
          }
          const double dx = __dadd_rn(p.x64[i], -px), dy = __dadd_rn(p.y64[i], -py);
          const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
          double w;
          if (WK == MLS_W_GAUSS) {
            if (binned && !(fabs(dx) < rho && fabs(dy) < rho)) continue;
            ++count;
            if (p.list && r2 - m > kGaussCut * h2) continue;
            w = exp(-(r2 - m) / h2);
          } else if (WK == MLS_W_WENDLAND) {
            if (r2 < h2) {
              const double qd = sqrt(r2) / p.h;
              const double o = 1.0 - qd;
              w = o * o * o * o * (4.0 * qd + 1.0);
              ++count;
            } else {
              w = 0.0;
            }
          } else {
            ++count;
            if (coincident) {
              w = 0.0;
              if (r2 == 0.0) {
                ++ccnt;
#pragma unroll
                for (int dd = 0; dd < DC; ++dd)
                  if (d0 + dd < p.D) csum[dd] += p.FT64[(size_t)(d0 + dd) * n + i];
              }
            } else {
              w = pow(m / r2, p.alpha);
            }
          }
          if (w == 0.0) continue;
          if (ncache < kF64Slots) {
            c_w[ncache * 32 + lane] = w;
            c_i[ncache * 32 + lane] = (int)i;
          }
          ++ncache;
          const double ddx = dx * inv_s, ddy = dy * inv_s;
          double mo[15];
          mo[0] = 1.0;
          if (NM > 1) {
            mo[1] = ddx; mo[2] = ddy; mo[3] = ddx * ddx; mo[4] = ddx * ddy; mo[5] = ddy * ddy;
          }
          if (NM > 6) {
            mo[6] = mo[3] * ddx; mo[7] = mo[3] * ddy; mo[8] = mo[5] * ddx; mo[9] = mo[5] * ddy;
            mo[10] = mo[3] * mo[3]; mo[11] = mo[3] * mo[4]; mo[12] = mo[3] * mo[5];
            mo[13] = mo[4] * mo[5]; mo[14] = mo[5] * mo[5];
          }
#pragma unroll
          for (int j = 0; j < NM; ++j) S[j] += w * mo[j];
          double fv[DC];
#pragma unroll
          for (int dd = 0; dd < DC; ++dd) fv[dd] = (d0 + dd < p.D) ? p.FT64[(size_t)(d0 + dd) * n + i] : 0.0;
#pragma unroll
          for (int a = 0; a < n_terms(DEG); ++a) {
            const double wb = w * mo[a];
#pragma unroll
            for (int dd = 0; dd < DC; ++dd) R[a][dd] += wb * fv[dd];
          }
        }
      }
      if (fresh) {
#pragma unroll
        for (int j = 0; j < NM; ++j) S[j] = warp_sum(S[j]);
        count = warp_sum(count);
        if (WK == MLS_W_GAUSS && !binned) count = n;   // every point has positive weight
      }
#pragma unroll
      for (int a = 0; a < n_terms(DEG); ++a)
#pragma unroll
        for (int dd = 0; dd < DC; ++dd) R[a][dd] = warp_sum(R[a][dd]);
      if (WK == MLS_W_INVDIST) {
        ccnt = warp_sum(ccnt);
#pragma unroll
        for (int dd = 0; dd < DC; ++dd) csum[dd] = warp_sum(csum[dd]);
      }
      // degree policy (every lane, identical arithmetic)
      double out[DC];
      int used = -1;
      if (coincident) {
#pragma unroll
        for (int dd = 0; dd < DC; ++dd) out[dd] = csum[dd] / (double)ccnt;
        used = 0;
        st |= MLS_ST_COINCIDENT;
      } else if (!fresh) {
        used = used_saved;
        if (used >= 0) {
#pragma unroll
          for (int dd = 0; dd < DC; ++dd) {
            double acc = 0.0;
            for (int c = 0; c < k_saved; ++c) acc += zc_saved[c] * R[c][dd];
            out[dd] = acc;
          }
        }
      } else {
        double zc[6];
        used = f64_policy<DEG>(S, count, p.rcond_min, zc, k_saved);
        if (used >= 0) {
#pragma unroll
          for (int dd = 0; dd < DC; ++dd) {
            double acc = 0.0;
            for (int c = 0; c < k_saved; ++c) acc += zc[c] * R[c][dd];
            out[dd] = acc;
          }
          for (int c = 0; c < k_saved; ++c) zc_saved[c] = zc[c];
        }
        used_saved = used;
      }
      // the later chunks may read the cache when no lane overflowed it
      if (fresh && WK != MLS_W_INVDIST) cached = __all_sync(0xffffffffu, ncache <= kF64Slots);
      if (used < 0) {
        st |= MLS_ST_NO_SUPPORT;
#pragma unroll
        for (int dd = 0; dd < DC; ++dd) out[dd] = __longlong_as_double(0x7ff8000000000000ll);
      } else {
        st = (uint8_t)((st & ~MLS_ST_DEGREE_MASK) | used | (used < DEG ? MLS_ST_DEGRADED : 0));
      }
      // lane dd writes dimension d0 + dd
#pragma unroll
      for (int dd = 0; dd < DC; ++dd) {
        const int d = d0 + dd;
        if (lane == dd && d < p.D) {
          const OutT f = (OutT)out[dd];
          field[(size_t)d * plane + id] = f;
          if (p.bands) {
            if (sizeof(OutT) == 8)
              p.bands[(size_t)d * plane + id] = band_of((double)f, p.lev64 + (size_t)d * p.L, p.L);
            else
              p.bands[(size_t)d * plane + id] = band_of((float)f, p.lev32 + (size_t)d * p.L, p.L);
          }
        }
      }
    }
    if (lane == 0 && p.status) {
      if (!p.list) st &= ~MLS_ST_RECOMPUTED;
      p.status[id] = st;
    }
  }
}

// ---------------------------------------------------------------------------
// Standalone labels: 16 consecutive pixels of one dimension per thread.
template <typename T>
__global__ void k_bands(const T *field, const double *lev64, const float *lev32, int L, int64_t plane, int D,
                        uint8_t *bands) {
  extern __shared__ unsigned char smem_raw[];
  const int d = blockIdx.y;
  if (sizeof(T) == 8) {
    double *lv = (double *)smem_raw;
    for (int j = threadIdx.x; j < L; j += blockDim.x) lv[j] = lev64[(size_t)d * L + j];
  } else {
    float *lv = (float *)smem_raw;
    for (int j = threadIdx.x; j < L; j += blockDim.x) lv[j] = lev32[(size_t)d * L + j];
  }
  __syncthreads();
  const T *f = field + (size_t)d * plane;
  uint8_t *b = bands + (size_t)d * plane;
  // four consecutive values per thread, neighbouring threads on neighbouring
  // values: one 16-byte load and one 4-byte store per thread where aligned
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); i0 < plane; i0 += 4 * nthreads) {
    T x[4];
    const bool full = i0 + 4 <= plane;
    if (sizeof(T) == 4 && full && ((((uintptr_t)(f + i0)) & 15) == 0)) {
      const float4 v = *(const float4 *)(f + i0);
      x[0] = (T)v.x; x[1] = (T)v.y; x[2] = (T)v.z; x[3] = (T)v.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = (i0 + k < plane) ? f[i0 + k] : T(0);
    }
    uint8_t out[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      out[k] = (sizeof(T) == 8) ? band_of((double)x[k], (const double *)smem_raw, L)
                                : band_of((float)x[k], (const float *)smem_raw, L);
    if (full && (((uintptr_t)(b + i0)) & 3) == 0) {
      *(uchar4 *)(b + i0) = make_uchar4(out[0], out[1], out[2], out[3]);
    } else {
      for (int k = 0; k < 4 && i0 + k < plane; ++k) b[i0 + k] = out[k];
    }
  }
}

// FP64 monomials of degree <= 4 of (dx, dy) in the moment index order, as
// k_mls_f64 forms them.
template <int NM>
__device__ __forceinline__ void monomials64(double dx, double dy, double (&mo)[15]) {
  mo[0] = 1.0;
  if (NM > 1) {
    mo[1] = dx; mo[2] = dy; mo[3] = dx * dx; mo[4] = dx * dy; mo[5] = dy * dy;
  }
  if (NM > 6) {
    mo[6] = mo[3] * dx; mo[7] = mo[3] * dy; mo[8] = mo[5] * dx; mo[9] = mo[5] * dy;
    mo[10] = mo[3] * mo[3]; mo[11] = mo[3] * mo[4]; mo[12] = mo[3] * mo[5];
    mo[13] = mo[4] * mo[5]; mo[14] = mo[5] * mo[5];
  }
}

// ---------------------------------------------------------------------------
// The last tier of a reduced-precision render's hand-over (the pixels still
// ill conditioned in the centroid frame, or whose support count is in doubt):
// the weights, support count, moments and degree policy of the FP64
// definition as k_mls_f64 forms them, then the value as sum_i phi_i f_id
// with the shape functions phi_i = w_i (zc . b(x_i)) formed in FP64 and the
// sums over the points in double-float on the FP32 pipes, lanes over the
// dimensions.  k_mls_f64 instead accumulates every right-hand side
// R_ad = sum w_i b_a f_id in FP64: six FP64 multiply-adds per point and
// dimension, which took this tier a sixth of the 200k-point render on
// GB300's FP64 units.  The sums here carry about 2^-46 of sum |phi_i f_id|
// (the fit's Lebesgue sum, in units of the value range), the values
// (FR32 + FR32lo) about 2^-48 each: far inside the reduced precisions'
// tolerance.  Gaussian and Wendland weights (inverse-distance pixels on a
// data point take k_mls_f64).
template <int DEG, int WK>
__global__ __launch_bounds__(256) void k_mls_f64v(KParams p) {
  constexpr int NM = n_moments(DEG);
  constexpr int kVL = 2;   // value dimensions per lane per sweep
  static_assert(WK != MLS_W_INVDIST, "inverse distance takes k_mls_f64");
  const int lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char f64_smem[];
  double *c_w = (double *)f64_smem + (size_t)(threadIdx.x >> 5) * kF64Slots * 32;            // [slot][lane]
  int *c_i = (int *)(f64_smem + (size_t)8 * kF64Slots * 32 * 8) + (size_t)(threadIdx.x >> 5) * kF64Slots * 32;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t npix = (int64_t)*p.list_count < p.list_cap ? (int64_t)*p.list_count : p.list_cap;
  const size_t plane = (size_t)p.W * p.H;
  const double inv_s = 1.0 / p.h;
  const double h2 = p.h * p.h;
  const int64_t n = p.n;
  float *field = (float *)p.field;
  const bool binned = (WK == MLS_W_WENDLAND) || (WK == MLS_W_GAUSS && p.trunc > 0.0);
  const double rho = p.trunc * p.h;
  const bool reach = (WK == MLS_W_GAUSS) && !binned && p.cell_start != nullptr;

  for (int64_t q = warp0; q < npix; q += nwarps) {
    const int64_t id = list_i(p, p.list[list_i(p, q)]);
    const int u = (int)(id % p.W), v = (int)(id / p.W);
    // the same expression order as the FP64 definition, without contraction
    const double px = __dadd_rn(p.x0, __dmul_rn(__dadd_rn((double)u, 0.5), p.sx));
    const double py = __dadd_rn(p.y0, __dmul_rn(__dadd_rn((double)v, 0.5), p.sy));
    const float mhat = (WK == MLS_W_GAUSS) ? p.mstab[pix_i(p, (int64_t)v * (p.tiles_x * 16) + u)] : 0.f;
    int nr = 1, cx0 = 0, cx1 = 0, cy0 = 0;
    if (binned || reach) {
      const double rad = (WK == MLS_W_WENDLAND) ? p.h
                         : binned ? rho * (1.0 + 1e-5)
                                  : p.h * sqrt(fmax((double)mhat, 0.0) + kGaussCut + 1.0) * (1.0 + 1e-5);
      int cy1;
      cell_range_d(px, px, rad, p.gx0, p.inv_cell, p.gx, cx0, cx1);
      cell_range_d(py, py, rad, p.gy0, p.inv_cell, p.gy, cy0, cy1);
      nr = (cx0 <= cx1) ? max(cy1 - cy0 + 1, 0) : 0;
    }
    const double m = (WK == MLS_W_GAUSS) ? (double)mhat * h2 : 0.0;
    const float pxs = scaled_px(p, u), pys = scaled_py(p, v);
    // the weight of candidate i (0: outside the support or the sums), with
    // its scaled offsets; *counted when it enters the support count
    auto weight = [&](int64_t i, bool *counted, double *ddx, double *ddy) -> double {
      *counted = false;
      if (WK == MLS_W_GAUSS && !binned) {
        // conservative FP32 test before any FP64 work on far pairs
        const float dxs = p.xs[i] - pxs, dys = p.ys[i] - pys;
        if (fmaf(dxs, dxs, dys * dys) - mhat > (float)kGaussCut + 1.f) {
          *counted = true;
          return 0.0;
        }
      }
      const double dx = __dadd_rn(p.x64[i], -px), dy = __dadd_rn(p.y64[i], -py);
      const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      *ddx = dx * inv_s;
      *ddy = dy * inv_s;
      if (WK == MLS_W_GAUSS) {
        if (binned && !(fabs(dx) < rho && fabs(dy) < rho)) return 0.0;
        *counted = true;
        if (r2 - m > kGaussCut * h2) return 0.0;
        return exp(-(r2 - m) / h2);
      }
      if (r2 < h2) {
        const double qd = sqrt(r2) / p.h;
        const double o = 1.0 - qd;
        *counted = true;
        return o * o * o * o * (4.0 * qd + 1.0);
      }
      return 0.0;
    };
    // ---- weights, support count and moments (FP64, lanes over the points);
    // the lane's positive-weight points are cached for the value sweeps
    double S[15];
#pragma unroll
    for (int j = 0; j < 15; ++j) S[j] = 0.0;
    int64_t count = 0;
    int ncache = 0;
    for (int r = 0; r < nr; ++r) {
      const int64_t a0 = (binned || reach) ? cell_at(p, (int64_t)(cy0 + r) * p.gx + cx0) : 0;
      const int64_t a1 = (binned || reach) ? cell_at(p, (int64_t)(cy0 + r) * p.gx + cx1 + 1) : n;
      for (int64_t i = a0 + lane; i < a1; i += 32) {
        bool counted;
        double ddx = 0.0, ddy = 0.0;
        const double w = weight(i, &counted, &ddx, &ddy);
        if (counted) ++count;
        if (w == 0.0) continue;
        if (ncache < kF64Slots) {
          c_w[ncache * 32 + lane] = w;
          c_i[ncache * 32 + lane] = (int)i;
        }
        ++ncache;
        double mo[15];
        monomials64<NM>(ddx, ddy, mo);
#pragma unroll
        for (int j = 0; j < NM; ++j) S[j] += w * mo[j];
      }
    }
#pragma unroll
    for (int j = 0; j < NM; ++j) S[j] = warp_sum(S[j]);
    count = warp_sum(count);
    if (WK == MLS_W_GAUSS && !binned) count = n;   // every point has positive weight
    double zc[6];
    int k = 1;
    const int used = f64_policy<DEG>(S, count, p.rcond_min, zc, k);
    if (used < 0) {
      for (int d = lane; d < p.D; d += 32) {
        field[(size_t)d * plane + id] = __int_as_float(0x7fc00000);
        if (p.bands) p.bands[(size_t)d * plane + id] = 255;
      }
      if (lane == 0 && p.status) p.status[id] = MLS_ST_NO_SUPPORT | MLS_ST_RECOMPUTED;
      continue;
    }
    const bool cached = __all_sync(0xffffffffu, ncache <= kF64Slots);
    int nbatch = ncache;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nbatch = max(nbatch, __shfl_xor_sync(0xffffffffu, nbatch, o));
    // phi of a point with weight w at scaled offset (ddx, ddy), double-float
    auto phi_of = [&](double w, double ddx, double ddy) -> df32 {
      double mo[15];
      monomials64<NM>(ddx, ddy, mo);
      double zb = 0.0;
      for (int c = 0; c < k; ++c) zb += zc[c] * mo[c];
      const double ph = w * zb;
      const float hi = (float)ph;
      return {hi, (float)(ph - (double)hi)};
    };
    // one batch of up to 32 points (lane j's point, valid), summed into the
    // lanes' dimensions
    auto sum_batch = [&](bool valid, int idx, df32 phi, int d0, df32 (&acc)[kVL]) {
      const unsigned int vm = __ballot_sync(0xffffffffu, valid);
      for (unsigned int mm = vm; mm; mm &= mm - 1) {
        const int jj = __ffs(mm) - 1;
        const df32 ph = {__shfl_sync(0xffffffffu, phi.hi, jj), __shfl_sync(0xffffffffu, phi.lo, jj)};
        const int ij = __shfl_sync(0xffffffffu, idx, jj);
        const float *fh = p.FR32 + (size_t)ij * p.D + d0 + lane;
        const float *fl = p.FR32lo + (size_t)ij * p.D + d0 + lane;
#pragma unroll
        for (int t = 0; t < kVL; ++t)
          if (d0 + lane + 32 * t < p.D) df_acc(acc[t], df_prod(ph, {fh[32 * t], fl[32 * t]}));
      }
    };
    // ---- values (lanes over the dimensions)
    for (int d0 = 0; d0 < p.D; d0 += 32 * kVL) {
      df32 acc[kVL];
#pragma unroll
      for (int t = 0; t < kVL; ++t) acc[t] = {0.f, 0.f};
      if (cached) {
        for (int b = 0; b < nbatch; ++b) {
          const bool valid = b < ncache;
          df32 phi = {0.f, 0.f};
          int idx = 0;
          if (valid) {
            idx = c_i[b * 32 + lane];
            const double dx = __dadd_rn(p.x64[idx], -px), dy = __dadd_rn(p.y64[idx], -py);
            phi = phi_of(c_w[b * 32 + lane], dx * inv_s, dy * inv_s);
          }
          sum_batch(valid, idx, phi, d0, acc);
        }
      } else {
        for (int r = 0; r < nr; ++r) {
          const int64_t a0 = (binned || reach) ? cell_at(p, (int64_t)(cy0 + r) * p.gx + cx0) : 0;
          const int64_t a1 = (binned || reach) ? cell_at(p, (int64_t)(cy0 + r) * p.gx + cx1 + 1) : n;
          for (int64_t base = a0; base < a1; base += 32) {
            const int64_t i = base + lane;
            bool valid = false;
            df32 phi = {0.f, 0.f};
            if (i < a1) {
              bool counted;
              double ddx = 0.0, ddy = 0.0;
              const double w = weight(i, &counted, &ddx, &ddy);
              if (w != 0.0) {
                valid = true;
                phi = phi_of(w, ddx, ddy);
              }
            }
            sum_batch(valid, (int)i, phi, d0, acc);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < kVL; ++t) {
        const int d = d0 + lane + 32 * t;
        if (d < p.D) {
          // fcen + fscl acc in double-float, rounded to float at the end
          const df32 sv = df_prod_f(df_two_sum(acc[t].hi, acc[t].lo), p.fscl32[d]);
          const df32 fs = df_add({p.fcen32[d], 0.f}, sv);
          const float f = fs.hi + fs.lo;
          field[(size_t)d * plane + id] = f;
          if (p.bands) p.bands[(size_t)d * plane + id] = band_of(f, p.lev32 + (size_t)d * p.L, p.L);
        }
      }
    }
    if (lane == 0 && p.status)
      p.status[id] = (uint8_t)(used | MLS_ST_RECOMPUTED | (used < DEG ? MLS_ST_DEGRADED : 0));
  }
}

template <int DEG>
void f32_dispatch_w(const KParams &p, cudaStream_t st) {
  // block shapes 16 x 8 (every weight), 8 x 8 and 8 x 4 (the Gaussian)
  if (p.weight == MLS_W_GAUSS && p.f32_shape == 1) {
    k_mls_f32<DEG, MLS_W_GAUSS, 8, 8><<<dim3(p.tiles_x * 2, p.tiles_y * 2), 64, 0, st>>>(p);
    return;
  }
  if (p.weight == MLS_W_GAUSS && p.f32_shape == 2) {
    k_mls_f32<DEG, MLS_W_GAUSS, 8, 4><<<dim3(p.tiles_x * 2, p.tiles_y * 4), 32, 0, st>>>(p);
    return;
  }
  dim3 grid(p.tiles_x, p.tiles_y * 2);
  if (p.weight == MLS_W_GAUSS) k_mls_f32<DEG, MLS_W_GAUSS, 16, 8><<<grid, 128, 0, st>>>(p);
  else if (p.weight == MLS_W_WENDLAND) k_mls_f32<DEG, MLS_W_WENDLAND, 16, 8><<<grid, 128, 0, st>>>(p);
  else k_mls_f32<DEG, MLS_W_INVDIST, 16, 8><<<grid, 128, 0, st>>>(p);
}

template <int DEG, typename OutT>
void f64_dispatch_w(const KParams &p, int64_t npix, cudaStream_t st) {
  int grid;
  if (p.list) grid = 152 * 8;
  else grid = (int)std::min<int64_t>((npix + 7) / 8, 152 * 64);
  if (grid < 1) grid = 1;
  // a reduced-precision render's last hand-over tier: FP64 moments and
  // policy, double-float value sums (inverse distance keeps k_mls_f64)
  if (p.list && sizeof(OutT) == 4 && p.FR32 && p.FR32lo && p.weight != MLS_W_INVDIST) {
    if (p.weight == MLS_W_GAUSS) {
      cudaFuncSetAttribute(k_mls_f64v<DEG, MLS_W_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kF64SmemBytes);
      k_mls_f64v<DEG, MLS_W_GAUSS><<<grid, 256, kF64SmemBytes, st>>>(p);
    } else {
      cudaFuncSetAttribute(k_mls_f64v<DEG, MLS_W_WENDLAND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kF64SmemBytes);
      k_mls_f64v<DEG, MLS_W_WENDLAND><<<grid, 256, kF64SmemBytes, st>>>(p);
    }
    return;
  }
  if (p.weight == MLS_W_GAUSS) {
    cudaFuncSetAttribute(k_mls_f64<DEG, MLS_W_GAUSS, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kF64SmemBytes);
    k_mls_f64<DEG, MLS_W_GAUSS, OutT><<<grid, 256, kF64SmemBytes, st>>>(p, npix);
  } else if (p.weight == MLS_W_WENDLAND) {
    cudaFuncSetAttribute(k_mls_f64<DEG, MLS_W_WENDLAND, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kF64SmemBytes);
    k_mls_f64<DEG, MLS_W_WENDLAND, OutT><<<grid, 256, kF64SmemBytes, st>>>(p, npix);
  } else {
    cudaFuncSetAttribute(k_mls_f64<DEG, MLS_W_INVDIST, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kF64SmemBytes);
    k_mls_f64<DEG, MLS_W_INVDIST, OutT><<<grid, 256, kF64SmemBytes, st>>>(p, npix);
  }
}

}  // namespace

void launch_f32(const KParams &p, cudaStream_t st) {
  if (p.degree == 0) f32_dispatch_w<0>(p, st);
  else if (p.degree == 1) f32_dispatch_w<1>(p, st);
  else f32_dispatch_w<2>(p, st);
}

void launch_f64(const KParams &p, int64_t npix, cudaStream_t st) {
  // FP64 renders write double; hand-over lists from the reduced paths write float
  if (p.field_fp64) {
    if (p.degree == 0) f64_dispatch_w<0, double>(p, npix, st);
    else if (p.degree == 1) f64_dispatch_w<1, double>(p, npix, st);
    else f64_dispatch_w<2, double>(p, npix, st);
  } else {
    if (p.degree == 0) f64_dispatch_w<0, float>(p, npix, st);
    else if (p.degree == 1) f64_dispatch_w<1, float>(p, npix, st);
    else f64_dispatch_w<2, float>(p, npix, st);
  }
}

// Device-to-host copy by the SMs (the destination is page-locked host memory
// through its device address): 16-byte loads and stores when both ends are
// 16-byte aligned, 4-byte ones when both are 4-byte aligned, else bytes.
__global__ void k_copy(void *dst, const void *src, size_t bytes) {
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
  const uintptr_t a = (uintptr_t)dst | (uintptr_t)src;
  if ((a & 15) == 0) {
    const size_t nv = bytes / 16;
    uint4 *d = (uint4 *)dst;
    const uint4 *s = (const uint4 *)src;
    for (size_t k = tid; k < nv; k += nt) d[k] = s[k];
    for (size_t k = nv * 16 + tid; k < bytes; k += nt) ((char *)dst)[k] = ((const char *)src)[k];
  } else if ((a & 3) == 0) {
    const size_t nv = bytes / 4;
    for (size_t k = tid; k < nv; k += nt) ((unsigned *)dst)[k] = ((const unsigned *)src)[k];
    for (size_t k = nv * 4 + tid; k < bytes; k += nt) ((char *)dst)[k] = ((const char *)src)[k];
  } else {
    for (size_t k = tid; k < bytes; k += nt) ((char *)dst)[k] = ((const char *)src)[k];
  }
}

void launch_bands(const KParams &p, bool fp64, cudaStream_t st) {
  const int64_t plane = (int64_t)p.W * p.H;
  // blocks of 256 threads, four values per thread and pass, at most 1024
  // blocks per dimension (the loop strides over the rest)
  const int64_t need = (plane + 4 * 256 - 1) / (4 * 256);
  dim3 grid((unsigned)(need < 1024 ? (need < 1 ? 1 : need) : 1024), (unsigned)p.D);
  const size_t sm = (size_t)p.L * (fp64 ? 8 : 4) + 16;
  if (fp64) k_bands<double><<<grid, 256, sm, st>>>((const double *)p.field, p.lev64, p.lev32, p.L, plane, p.D, p.bands);
  else k_bands<float><<<grid, 256, sm, st>>>((const float *)p.field, p.lev64, p.lev32, p.L, plane, p.D, p.bands);
}

void launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return;
  const size_t chunks = (bytes + 15) / 16;
  const size_t blocks = (chunks + 255) / 256;
  k_copy<<<(unsigned)(blocks < 152 * 8 ? (blocks < 1 ? 1 : blocks) : 152 * 8), 256, 0, st>>>(dst, src, bytes);
}

}  // namespace mlsi
