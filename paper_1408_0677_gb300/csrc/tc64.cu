// FP64-equivalent MLS moments on the tensor cores (tcgen05 + TMEM, sm_103a).
//
// GB300's FP64 units run at a small fraction of its FP32 rate, so the plain
// FP64 kernel (plain.cu) takes seconds on the full-sum workloads.  This kernel
// reaches FP64-level moments through the FP16 tensor-core path instead, by
// the splitting idea of Ozaki et al. (error-free transformation of a product
// into exactly computed products of narrow slices):
//
//   - for a 16 x 8 tile in a common tile frame, the moments and right-hand
//     sides are one product W[128 pixels x points] . G[points x 48 columns]
//     (16 monomials of the moment matrix, then the basis times Dc values);
//   - every entry of W (the weight, in double-float, scaled by 1/2) and of G
//     (scaled by its column's power-of-two bound) is rounded to a 60-bit
//     fixed-point integer and written as ten balanced base-64 digits
//     d_0..d_9, |d| <= 32:  v = sum_i d_i 2^(-5-6i);
//   - a digit is an integer held exactly in FP16, a product of two digits is
//     at most 2^10, and the products of the pairs with i + j = t all carry
//     the same scale 2^(-10-6t): one TMEM accumulator per diagonal t = 0..9
//     (the pairs with i + j >= 10 are below 2^-56 of the entries' scales and
//     are left out) sums them exactly in FP32 as long as its integer stays
//     below 2^24, that is for up to 1536 points (10 pairs x 1536 points x
//     33 x 32 < 2^24);
//   - after every 1536 points (and at the end) each thread reads its pixel's
//     ten diagonals and adds them, scaled by 2^(-6t), into FP64 registers;
//   - the epilogue shifts the FP64 moments to the pixel frame and applies the
//     FP64 degree policy and solve of the definition (Section 3.3: the
//     weighted least-squares fit evaluated at the pixel).
//
// The tile frame is shared by the 16 x 8 pixels, so the tile must be narrow
// compared with h: renders whose 16-pixel tile spans more than 4 h take the
// FP64 kernel instead (the same rule as the reduced-precision path).
//
// One CTA of 256 threads (two per pixel) works one tile, stage by stage:
// digits of 64 points are written to shared memory (each pixel's two threads
// take half the points each; Gaussian weights are a column factor times a
// row factor times the pixel's correction, 24 double-float exps per point
// instead of 128), one thread issues the MMAs of the first five weight
// digits, then of the last five (the weight digit tiles are reused), and
// every wait is bounded (globaltimer).  The
// Wendland support count comes from the prepass; pixels whose count could
// cross a degree threshold go to the FP64 kernel.
#include "mls_internal.h"
#include "tcgen05.cuh"

namespace mlsi {
namespace {

using namespace mlsk;
using namespace tcx;

constexpr int kThr64 = 256;                    // two threads per pixel of a 16 x 8 tile
constexpr int kPix = 128;                      // pixels per tile (TMEM lanes)
constexpr int kN64 = 48;                       // operand columns
constexpr int kDig = 10;                       // digits per entry
constexpr int kHalfDig = 5;                    // weight digit tiles resident at once
constexpr int kKP = 64;                        // points per stage
constexpr int kChunkStages = 24;               // stages between drains (1536 points)
constexpr float kReach64 = 45.f;               // Gaussian: points with r^2 - m <= 45 h^2
constexpr int kMaxRows = 96;                   // cell rows a tile may visit
constexpr int kVS = 33;                        // value row stride (float2): rows on distinct banks
constexpr int kADig = 128 * 128;               // 16 KB per weight digit tile
constexpr int kBDig = kN64 * 128;              // 6 KB per operand digit tile
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kHalfDig * kADig;           // 80 KB
constexpr int kOffRem = kOffB + kDig * kBDig;              // 140 KB: weight remainders [64][128] int32
constexpr int kOffPt = kOffRem + kKP * kPix * 4;           // 172 KB: x~ (hi, lo), y~ (hi, lo) per point
constexpr int kOffVal = kOffPt + kKP * 16;                 // values (hi, lo) [64][kVS]
constexpr int kOffFac = kOffVal + kKP * kVS * 8;           // Gaussian factors [24][64] (hi, lo)
constexpr int kOffTab = kOffFac + 24 * kKP * 8;            // exp table (64 float2)
constexpr int kOffRow = kOffTab + 64 * 8;                  // row start[kMaxRows], prefix[kMaxRows + 1]
constexpr int kOffMisc = kOffRow + (2 * kMaxRows + 1) * 4 + 12;
constexpr int kSmem64 = kOffMisc + 2048 + 1024;            // misc (2 KB) + alignment slack

// v in [-1, 1] (double-float) as a 60-bit fixed-point integer round(v 2^59).
__device__ __forceinline__ long long fixed59(df32 v) {
  return __float2ll_rn(v.hi * 576460752303423488.f) + __float2ll_rn(v.lo * 576460752303423488.f);
}

// The first five balanced base-64 digits of V (|V| <= 2^59 + small): V =
// sum_{i<5} d_i 2^(54 - 6i) + rem with |rem| <= 2^29.
__device__ __forceinline__ int top5(long long &V, int (&d)[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int sh = 54 - 6 * i;
    const long long q = (V + (1ll << (sh - 1))) >> sh;
    d[i] = (int)q;
    V -= q << sh;
  }
  return (int)V;
}

// The last five digits of the remainder: rem = sum_{i<5} e_i 2^(24 - 6i).
__device__ __forceinline__ void low5(int R, int (&d)[5]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int sh = 24 - 6 * i;
    const int q = (R + (1 << (sh - 1))) >> sh;
    d[i] = q;
    R -= q << sh;
  }
  d[4] = R;
}

__device__ __forceinline__ uint32_t h2pack(int a, int b) {
  const __half2 h = __halves2half2(__int2half_rn(a), __int2half_rn(b));
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Monomial x^ex y^ey (ex + ey <= 4) in double-float.
__device__ __forceinline__ df32 df_mono(df32 x, df32 y, int ex, int ey) {
  df32 r{1.f, 0.f};
  for (int k = 0; k < ex; ++k) r = df_mul(r, x);
  for (int k = 0; k < ey; ++k) r = df_mul(r, y);
  return r;
}

// FP64 degree policy and value of one pixel from its pixel-frame moment
// matrix M (K x K, basis (1, x, y, x^2, xy, y^2) truncated) and right-hand
// sides R (K x Dc): the definition's equilibrated Cholesky, rcond_1 by the
// explicit inverse, lower degree when a test fails; the value through the
// one solve Me z = e_0 (column 0 of the inverse).  Returns the degree used,
// -1 without support.
template <int K, int DCM>
__device__ int policy_value_f64(const double (&M)[6][6], const double (&R)[K][DCM], int Dc, int count,
                                double rcond_min, double (&out)[DCM]) {
  for (int deg = (K == 6 ? 2 : K == 3 ? 1 : 0); deg >= 0; --deg) {
    const int k = n_terms(deg);
    if (count < k) continue;
    double sd[6], Me[6][6], Lm[6][6], Inv[6][6];
    bool ok = true;
    for (int a = 0; a < k && ok; ++a) {
      if (!(M[a][a] > 0.0)) ok = false;
      else sd[a] = 1.0 / sqrt(M[a][a]);
    }
    if (!ok) continue;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) Me[a][b] = M[a][b] * sd[a] * sd[b];
    for (int j = 0; j < k && ok; ++j) {
      double s = Me[j][j];
      for (int t = 0; t < j; ++t) s -= Lm[j][t] * Lm[j][t];
      if (!(s > 0.0)) { ok = false; break; }
      const double ljj = sqrt(s);
      Lm[j][j] = ljj;
      for (int i = j + 1; i < k; ++i) {
        double v = Me[i][j];
        for (int t = 0; t < j; ++t) v -= Lm[i][t] * Lm[j][t];
        Lm[i][j] = v / ljj;
      }
    }
    if (!ok) continue;
    for (int c = 0; c < k; ++c) {
      double col[6];
      for (int a = 0; a < k; ++a) col[a] = (a == c) ? 1.0 : 0.0;
      for (int i = 0; i < k; ++i) {
        double v = col[i];
        for (int t = 0; t < i; ++t) v -= Lm[i][t] * col[t];
        col[i] = v / Lm[i][i];
      }
      for (int i = k - 1; i >= 0; --i) {
        double v = col[i];
        for (int t = i + 1; t < k; ++t) v -= Lm[t][i] * col[t];
        col[i] = v / Lm[i][i];
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
    if (!(1.0 / (nA * nI) >= rcond_min)) continue;
    for (int dd = 0; dd < Dc; ++dd) {
      double acc = 0.0;
      for (int c = 0; c < k; ++c) acc += sd[0] * Inv[c][0] * sd[c] * R[c][dd];
      out[dd] = acc;
    }
    return deg;
  }
  return -1;
}

template <int DEG, int WK>
__global__ void __launch_bounds__(kThr64, 1) k_mls_tc64(KParams p, int d0, int Dc, uint32_t idesc) {
  constexpr int K = n_terms(DEG);
  constexpr int DCM = (kN64 - 16) / K;   // value dimensions per pass at most
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  const int t = threadIdx.x, warp = t >> 5;
  const int pp = t & (kPix - 1), hf = t >> 7;      // pixel, and which half of its points / columns
  float4 *s_pt = (float4 *)(smem + kOffPt);
  float2 *s_val = (float2 *)(smem + kOffVal);
  float2 *s_fac = (float2 *)(smem + kOffFac);        // [16 columns + 8 rows][64 points]
  float2 *s_tab = (float2 *)(smem + kOffTab);
  int *s_rstart = (int *)(smem + kOffRow);
  int *s_rpre = s_rstart + kMaxRows;
  unsigned char *misc = smem + kOffMisc;
  int *s_misc = (int *)misc;                          // [0] rows, [1] total points
  uint64_t *bar = (uint64_t *)(misc + 16);
  uint32_t *tmem_slot = (uint32_t *)(misc + 24);
  double *s_bound = (double *)(misc + 32);            // |x~|, |y~| bounds of the visited cells
  float *s_ab = (float *)(misc + 48);                 // alpha[16], beta[8]: split stabiliser
  float *s_sh = (float *)(misc + 160);                // per-point exponent shift [64]
  float *s_m = (float *)(misc + 416);                 // stabiliser of each pixel [128]
  double *s_inv = (double *)(misc + 928);             // 1 / value scale of the pass's dimensions (<= 32)
  float2 *s_off = (float2 *)(misc + 1184);            // offsets of the 16 columns, then 8 rows (hi, lo)
  const uint32_t bar_mma = smem_u32(bar);

  const int u0 = blockIdx.x * 16, v0 = blockIdx.y * 8;
  const int tile = (v0 >> 4) * p.tiles_x + (u0 >> 4);
  // the moment frame: the tile's geometric centre, which keeps every pixel's
  // offset |delta| at most half the tile (the shift to the pixel frame
  // cancels terms of size |delta|^4 times the moments)
  const double ox = p.x0 + (u0 + 8) * p.sx, oy = p.y0 + (v0 + 4) * p.sy;
  const int u = u0 + (pp & 15), v = v0 + (pp >> 4);
  const bool inside = (u < p.W) && (v < p.H);
  const size_t pi = (size_t)pix_i(p, (int64_t)v * (p.tiles_x * 16) + u);

  if (t == 0) {
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), 512);
  df_exp_table_init(s_tab);
  if (hf == 0) s_m[pp] = (WK == MLS_W_WENDLAND) ? 0.f : p.mstab[pi];
  for (int dd = t; dd < Dc; dd += kThr64) s_inv[dd] = (d0 + dd < p.D) ? 1.0 / p.fscl64[d0 + dd] : 0.0;
  if (t < 24) {
    // the tile's column (row) centres from the frame origin, scaled by 1/h
    const double o = (t < 16) ? (p.x0 + (u0 + t + 0.5) * p.sx - ox) * p.inv_s
                              : (p.y0 + (v0 + t - 16 + 0.5) * p.sy - oy) * p.inv_s;
    s_off[t] = make_float2((float)o, (float)(o - (double)(float)o));
  }
  // cell rows visited: the pixels' extent +- r (Wendland r = h; Gaussian
  // r = h sqrt(max m + 45), beyond which every weight is below e^-45)
  if (t == 0) {
    const double rs = (WK == MLS_W_WENDLAND) ? 1.0 : sqrt((double)p.tmax[tile_i(p, tile)] + (double)kReach64);
    const double rad = p.h * rs * (1.0 + 1e-5);
    const double xa = p.x0 + (u0 + 0.5) * p.sx, xb = p.x0 + (u0 + 15.5) * p.sx;
    const double ya = p.y0 + (v0 + 0.5) * p.sy, yb = p.y0 + (v0 + 7.5) * p.sy;
    int cx0 = (int)floor((fmin(xa, xb) - rad - p.gx0) * p.inv_cell);
    int cx1 = (int)floor((fmax(xa, xb) + rad - p.gx0) * p.inv_cell);
    int cy0 = (int)floor((fmin(ya, yb) - rad - p.gy0) * p.inv_cell);
    int cy1 = (int)floor((fmax(ya, yb) + rad - p.gy0) * p.inv_cell);
    cx0 = max(cx0, 0);
    cy0 = max(cy0, 0);
    cx1 = min(cx1, p.gx - 1);
    cy1 = min(cy1, p.gy - 1);
    int nrow = 0, total = 0;
    if (cx0 <= cx1) {
      for (int cy = cy0; cy <= cy1 && nrow < kMaxRows; ++cy) {
        const int a = cell_at(p, (int64_t)cy * p.gx + cx0), b = cell_at(p, (int64_t)cy * p.gx + cx1 + 1);
        if (b <= a) continue;
        s_rstart[nrow] = a;
        s_rpre[nrow] = total;
        total += b - a;
        ++nrow;
      }
    }
    if (cx0 <= cx1 && cy1 - cy0 + 1 > kMaxRows) set_error(p.err, ERR_INDEX + SITE_CELL);
    s_rpre[nrow] = total;
    s_misc[0] = nrow;
    s_misc[1] = total;
    // pixel-point pairs this tile visits (once, in the first value pass)
    if (p.visited && d0 == 0 && total) atomicAdd(p.visited, (unsigned long long)total * 128ull);
    // tile-frame extent of the visited cells (scaled by 1/h), with a margin
    const double ex0 = (p.gx0 + cx0 * p.cell - ox) * p.inv_s;
    const double ex1 = (p.gx0 + (cx1 + 1) * p.cell - ox) * p.inv_s;
    const double ey0 = (p.gy0 + cy0 * p.cell - oy) * p.inv_s;
    const double ey1 = (p.gy0 + (cy1 + 1) * p.cell - oy) * p.inv_s;
    s_bound[0] = fmax(fabs(ex0), fabs(ex1)) * (1.0 + 1e-6) + 1e-6;
    s_bound[1] = fmax(fabs(ey0), fabs(ey1)) * (1.0 + 1e-6) + 1e-6;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // the Gaussian stabiliser split alpha_c + beta_r <= m_p over the tile's
  // 16 columns and 8 rows (beta_r = min over the row, alpha_c = min over the
  // column of m - beta), so that each weight is a column factor times a row
  // factor times the pixel's correction exp(m_p - alpha_c - beta_r) >= 1
  if (WK == MLS_W_GAUSS && t < 8) {
    float b = INFINITY;
    for (int c = 0; c < 16; ++c) b = fminf(b, s_m[t * 16 + c]);
    s_ab[16 + t] = b;
  }
  __syncthreads();
  if (WK == MLS_W_GAUSS && t < 16) {
    float a = INFINITY;
    for (int r = 0; r < 8; ++r) a = fminf(a, s_m[r * 16 + t] - s_ab[16 + r]);
    s_ab[t] = a;
  }
  __syncthreads();
  const uint32_t tmem = *tmem_slot;
  const int total = s_misc[1], nrow = s_misc[0];
  const double bx = s_bound[0], by = s_bound[1];

  // this thread's pixel offset from the frame origin (scaled by 1/h)
  const double dpx = (p.x0 + (u + 0.5) * p.sx - ox) * p.inv_s;
  const double dpy = (p.y0 + (v + 0.5) * p.sy - oy) * p.inv_s;
  const df32 dpx32{(float)dpx, (float)(dpx - (double)(float)dpx)};
  const df32 dpy32{(float)dpy, (float)(dpy - (double)(float)dpy)};
  const int cflag = (WK == MLS_W_WENDLAND) ? p.cnt[pi] : 0;
  // Gaussian: the pixel's correction factor exp(m - alpha_c - beta_r)
  // (every offset enters the double-float exponent on its own, exactly, so
  // that alpha, beta and the point shift cancel in the product to the
  // double-float rounding of the exponents)
  df32 corr{1.f, 0.f};
  if (WK == MLS_W_GAUSS) {
    const df32 res = df_add(df_add({s_m[pp], 0.f}, {-s_ab[pp & 15], 0.f}), {-s_ab[16 + (pp >> 4)], 0.f});
    corr = df_exp(res, s_tab);
  }

  // power-of-two bound of each operand column (exponent e: |g| <= 2^e);
  // this thread builds columns rr and rr + 32 (below 48) for points 8 g .. 8 g + 7
  const int g8 = t & 7, rr = t >> 3;
  int cole[2], colkind[2], colm[2], cold[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int c = rr + 32 * q;
    double bound = 0.0;
    colm[q] = cold[q] = 0;
    if (c >= kN64) {
      colkind[q] = 3;                         // not built by this thread
    } else if (c < 15) {
      colkind[q] = (c < n_moments(DEG)) ? 0 : 2;
      colm[q] = c;
      bound = pow(bx, mono_ex(c)) * pow(by, mono_ey(c));
    } else if (c >= 16 && c < 16 + Dc * K && d0 + (c - 16) / K < p.D) {
      colkind[q] = 1;
      colm[q] = (c - 16) % K;
      cold[q] = (c - 16) / K;
      bound = pow(bx, mono_ex(colm[q])) * pow(by, mono_ey(colm[q]));   // |value| <= 1
    } else {
      colkind[q] = 2;
    }
    cole[q] = bound > 0.0 ? (int)ceil(log2(bound * 1.001)) : 0;
  }

  double acc[24];                              // this thread's 24 columns: 24 hf .. 24 hf + 23
#pragma unroll
  for (int c = 0; c < 24; ++c) acc[c] = 0.0;
  const uint64_t limit = kWaitLimitNs;
  bool alive = true;
  uint32_t phase = 0;
  const int nstages = (total + kKP - 1) / kKP;
  int *s_rem = (int *)(smem + kOffRem);

  for (int s = 0; s < nstages && alive; ++s) {
    const int sc = s % kChunkStages;
    // ---- point data of this stage (threads 0..63 a point each, 64..255 its values)
    if (t < kKP) {
      const int kidx = s * kKP + t;
      float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
      float sh = 0.f;
      if (kidx < total) {
        int r = 0;
        while (r + 1 < nrow && s_rpre[r + 1] <= kidx) ++r;
        const int i = s_rstart[r] + (kidx - s_rpre[r]);
        // offset from the frame's origin in FP64, then double-float
        const double xd = (p.x64[i] - ox) * p.inv_s, yd = (p.y64[i] - oy) * p.inv_s;
        pt = make_float4((float)xd, (float)(xd - (double)(float)xd), (float)yd, (float)(yd - (double)(float)yd));
        if (WK == MLS_W_GAUSS) {
          // exponent shift balancing the point's largest column and row factors
          float ex = -INFINITY, ey = -INFINITY;
          for (int c = 0; c < 16; ++c) {
            const float d = (float)xd - s_off[c].x;
            ex = fmaxf(ex, s_ab[c] - d * d);
          }
          for (int r2 = 0; r2 < 8; ++r2) {
            const float d = (float)yd - s_off[16 + r2].x;
            ey = fmaxf(ey, s_ab[16 + r2] - d * d);
          }
          sh = 0.5f * (ex - ey);
        }
      }
      s_pt[t] = pt;
      s_sh[t] = sh;
    }
    for (int e = t; e < kKP * Dc; e += kThr64) {
      const int j = e / Dc, dd = e - j * Dc;
      const int kidx = s * kKP + j;
      float2 fv = make_float2(0.f, 0.f);
      if (kidx < total && d0 + dd < p.D) {
        int r = 0;
        while (r + 1 < nrow && s_rpre[r + 1] <= kidx) ++r;
        const int i = s_rstart[r] + (kidx - s_rpre[r]);
        const int d = d0 + dd;
        const double val = (p.FT64[(size_t)d * p.n + i] - p.fcen64[d]) * s_inv[dd];
        fv = make_float2((float)val, (float)(val - (double)(float)val));
      }
      s_val[j * kVS + dd] = fv;
    }
    __syncthreads();
    // ---- Gaussian factors: 16 column and 8 row factors per point
    if (WK == MLS_W_GAUSS) {
      for (int e = t; e < 24 * kKP; e += kThr64) {
        const int f = e / kKP, j = e - f * kKP;
        const float4 pt = s_pt[j];
        df32 d, arg;
        const float2 o = s_off[f];
        if (f < 16) {
          d = df_add({pt.x, pt.y}, {-o.x, -o.y});
          arg = df_add(df_add(df_mul(d, d), {-s_ab[f], 0.f}), {s_sh[j], 0.f});
        } else {
          d = df_add({pt.z, pt.w}, {-o.x, -o.y});
          arg = df_add(df_add(df_mul(d, d), {-s_ab[f], 0.f}), {-s_sh[j], 0.f});
        }
        df32 w{0.f, 0.f};
        if (s * kKP + j < total && -arg.hi > -70.f) w = df_exp({-arg.hi, -arg.lo}, s_tab);
        s_fac[f * kKP + j] = make_float2(w.hi, w.lo);
      }
      __syncthreads();
    }
    // ---- operand digits: this thread's columns for its eight points
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (colkind[q] == 3) continue;
      const int c = rr + 32 * q;
      uint32_t w[kDig][4];
#pragma unroll
      for (int jj = 0; jj < 8; jj += 2) {
        int dg[2][kDig];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int j = 8 * g8 + jj + h2;
          const float4 pt = s_pt[j];
          df32 gval{0.f, 0.f};
          if (colkind[q] == 0) {
            gval = df_mono({pt.x, pt.y}, {pt.z, pt.w}, mono_ex(colm[q]), mono_ey(colm[q]));
          } else if (colkind[q] == 1) {
            const float2 fv = s_val[j * kVS + cold[q]];
            gval = df_mul(df_mono({pt.x, pt.y}, {pt.z, pt.w}, mono_ex(colm[q]), mono_ey(colm[q])), {fv.x, fv.y});
          }
          if (s * kKP + j >= total) gval = {0.f, 0.f};
          const float sc2 = ldexpf(1.f, -cole[q]);
          long long V = fixed59({gval.hi * sc2, gval.lo * sc2});
          int hi5[5], lo5[5];
          const int rem = top5(V, hi5);
          low5(rem, lo5);
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            dg[h2][i] = hi5[i];
            dg[h2][5 + i] = lo5[i];
          }
        }
#pragma unroll
        for (int i = 0; i < kDig; ++i) w[i][jj >> 1] = h2pack(dg[0][i], dg[1][i]);
      }
#pragma unroll
      for (int i = 0; i < kDig; ++i)
        *(uint4 *)(smem + kOffB + i * kBDig + sw128_off(c, g8)) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    }
    // ---- weight digits 0-4 of this thread's pixel, its half of the 64 points
#pragma unroll 1
    for (int c8 = 4 * hf; c8 < 4 * hf + 4; ++c8) {
      uint32_t w[kHalfDig][4];
#pragma unroll
      for (int jj = 0; jj < 8; jj += 2) {
        int dg[2][kHalfDig];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int j = 8 * c8 + jj + h2;
          df32 wt{0.f, 0.f};
          if (s * kKP + j < total) {
            if (WK == MLS_W_GAUSS) {
              const float2 X = s_fac[(pp & 15) * kKP + j], Y = s_fac[(16 + (pp >> 4)) * kKP + j];
              wt = df_mul(df_mul({X.x, X.y}, {Y.x, Y.y}), corr);
            } else {
              const float4 pt = s_pt[j];
              const df32 dx = df_add({pt.x, pt.y}, {-dpx32.hi, -dpx32.lo});
              const df32 dy = df_add({pt.z, pt.w}, {-dpy32.hi, -dpy32.lo});
              const df32 r2 = df_add(df_mul(dx, dx), df_mul(dy, dy));
              if (r2.hi < 1.f) wt = df_wendland(r2);
            }
          }
          long long V = fixed59({0.5f * wt.hi, 0.5f * wt.lo});
          int hi5[5];
          s_rem[j * kPix + pp] = top5(V, hi5);
#pragma unroll
          for (int i = 0; i < kHalfDig; ++i) dg[h2][i] = hi5[i];
        }
#pragma unroll
        for (int i = 0; i < kHalfDig; ++i) w[i][jj >> 1] = h2pack(dg[0][i], dg[1][i]);
      }
#pragma unroll
      for (int i = 0; i < kHalfDig; ++i)
        *(uint4 *)(smem + kOffA + i * kADig + sw128_off(pp, c8)) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- MMAs of weight digits 0-4 (every operand digit j <= 9 - i)
    if (t == 0) {
      for (int i = 0; i < kHalfDig; ++i)
        for (int j = 0; j + i < kDig; ++j)
#pragma unroll
          for (int k = 0; k < kKP / 16; ++k) {
            const uint64_t ad = desc_sw128(sbase + kOffA + i * kADig + 32 * k);
            const uint64_t bd = desc_sw128(sbase + kOffB + j * kBDig + 32 * k);
            const bool first = (sc == 0) && (i == 0) && (k == 0);
            mma_f16(tmem + (uint32_t)((i + j) * kN64), ad, bd, idesc, first ? 0u : 1u);
          }
      mma_commit(bar_mma);
    }
    bool ok = mbar_wait(bar_mma, phase, p.err, ERR_WAIT_FULL, limit);
    phase ^= 1u;
    tc_fence_after();
    if (!__syncthreads_and(ok)) {
      alive = false;
      break;
    }
    // ---- weight digits 5-9 from the remainders
#pragma unroll 1
    for (int c8 = 4 * hf; c8 < 4 * hf + 4; ++c8) {
      uint32_t w[kHalfDig][4];
#pragma unroll
      for (int jj = 0; jj < 8; jj += 2) {
        int lo0[5], lo1[5];
        low5(s_rem[(8 * c8 + jj) * kPix + pp], lo0);
        low5(s_rem[(8 * c8 + jj + 1) * kPix + pp], lo1);
#pragma unroll
        for (int i = 0; i < kHalfDig; ++i) w[i][jj >> 1] = h2pack(lo0[i], lo1[i]);
      }
#pragma unroll
      for (int i = 0; i < kHalfDig; ++i)
        *(uint4 *)(smem + kOffA + i * kADig + sw128_off(pp, c8)) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) {
      for (int i = kHalfDig; i < kDig; ++i)
        for (int j = 0; j + i < kDig; ++j)
#pragma unroll
          for (int k = 0; k < kKP / 16; ++k) {
            const uint64_t ad = desc_sw128(sbase + kOffA + (i - kHalfDig) * kADig + 32 * k);
            const uint64_t bd = desc_sw128(sbase + kOffB + j * kBDig + 32 * k);
            mma_f16(tmem + (uint32_t)((i + j) * kN64), ad, bd, idesc, 1u);
          }
      mma_commit(bar_mma);
    }
    ok = mbar_wait(bar_mma, phase, p.err, ERR_WAIT_FULL, limit);
    phase ^= 1u;
    tc_fence_after();
    if (!__syncthreads_and(ok)) {
      alive = false;
      break;
    }
    // ---- drain: after every kChunkStages stages and after the last; this
    // thread reads its pixel's columns 24 hf .. 24 hf + 23 of every diagonal
    if (sc == kChunkStages - 1 || s == nstages - 1) {
      const uint32_t tb = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
      for (int dg = 0; dg < kDig; ++dg) {
        float v16[16], v8[8];
        const uint32_t base = tb + (uint32_t)(dg * kN64);
        if (hf == 0) {
          tmem_ld16(base, v16);
          tmem_ld8(base + 16, v8);
        } else {
          tmem_ld8(base + 24, v8);
          tmem_ld16(base + 32, v16);
        }
        const double sc6 = ldexp(1.0, -6 * dg);
#pragma unroll
        for (int c = 0; c < 24; ++c) {
          const float x = (hf == 0) ? (c < 16 ? v16[c] : v8[c - 16]) : (c < 8 ? v8[c] : v16[c - 8]);
          acc[c] = fma((double)x, sc6, acc[c]);
        }
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }

  // ---- epilogue: the second half of every pixel's columns to shared memory
  // (the digit tiles are free now), then FP64 moments in the tile frame ->
  // pixel frame -> policy, one thread per pixel
  double *s_acc = (double *)(smem + kOffA);          // [128][24]
  if (hf == 1) {
#pragma unroll
    for (int c = 0; c < 24; ++c) s_acc[pp * 24 + c] = acc[c];
  }
  __syncthreads();
  const size_t plane = (size_t)p.W * p.H;
  const size_t pix = (size_t)v * p.W + u;
  double *field = (double *)p.field;
  if (alive && inside && hf == 0) {
    auto col = [&](int c) -> double { return c < 24 ? acc[c] : s_acc[pp * 24 + c - 24]; };
    // column scales: weights carry 2, operand columns 2^e, digit products 2^-10
    double S[15];
#pragma unroll
    for (int c = 0; c < 15; ++c) {
      const double bound = pow(bx, mono_ex(c)) * pow(by, mono_ey(c));
      const int e = bound > 0.0 ? (int)ceil(log2(bound * 1.001)) : 0;
      S[c] = (c < n_moments(DEG)) ? ldexp(col(c), e + 1 - 10) : 0.0;
    }
    double Mt[6][6], Rt[K][DCM];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b) Mt[a][b] = (a < K && b < K) ? S[midx(a, b)] : 0.0;
    for (int a = 0; a < K; ++a) {
      const double bound = pow(bx, mono_ex(a)) * pow(by, mono_ey(a));
      const int e = bound > 0.0 ? (int)ceil(log2(bound * 1.001)) : 0;
      for (int dd = 0; dd < Dc; ++dd) Rt[a][dd] = ldexp(col(16 + dd * K + a), e + 1 - 10);
    }
    // basis shift b(x~ - delta) = T b(x~): pixel-frame M = T Mt T^T, R = T Rt
    double T[6][6];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b) T[a][b] = (a == b) ? 1.0 : 0.0;
    const double ax = -dpx, ay = -dpy;   // x~ - delta = x~ + a
    if (K > 1) {
      T[1][0] = ax;
      T[2][0] = ay;
    }
    if (K > 3) {
      T[3][0] = ax * ax; T[3][1] = 2.0 * ax;
      T[4][0] = ax * ay; T[4][1] = ay; T[4][2] = ax;
      T[5][0] = ay * ay; T[5][2] = 2.0 * ay;
    }
    double TM[6][6], M[6][6], R[K][DCM];
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) {
        double s2 = 0.0;
        for (int c = 0; c < K; ++c) s2 += T[a][c] * Mt[c][b];
        TM[a][b] = s2;
      }
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) {
        double s2 = 0.0;
        for (int c = 0; c < K; ++c) s2 += TM[a][c] * T[b][c];
        M[a][b] = s2;
      }
    for (int a = 0; a < K; ++a)
      for (int dd = 0; dd < Dc; ++dd) {
        double s2 = 0.0;
        for (int c = 0; c < K; ++c) s2 += T[a][c] * Rt[c][dd];
        R[a][dd] = s2;
      }
    int count;
    bool give = false;
    if (WK == MLS_W_WENDLAND) {
      count = cflag & kCntMask;
      give = count_uncertain<K>(cflag);
    } else {
      count = (int)(p.n < (1 << 30) ? p.n : (1 << 30));
    }
    if (give) {
      if (d0 == 0) {
        const unsigned int kq = atomicAdd(p.relist_count, 1u);
        p.relist[list_i(p, kq)] = (int)pix;
      }
    } else {
      double out[DCM];
      const int used = policy_value_f64<K, DCM>(M, R, Dc, count, p.rcond_min, out);
      for (int dd = 0; dd < Dc; ++dd) {
        const int d = d0 + dd;
        if (d >= p.D) break;
        const double f = (used >= 0) ? fma(out[dd], p.fscl64[d], p.fcen64[d]) : __longlong_as_double(0x7ff8000000000000ll);
        field[(size_t)d * plane + pix] = f;
        if (p.bands) p.bands[(size_t)d * plane + pix] = band_of(f, p.lev64 + (size_t)d * p.L, p.L);
      }
      if (p.status && d0 == 0)
        p.status[pix] = used < 0 ? (uint8_t)MLS_ST_NO_SUPPORT
                                 : (uint8_t)(used | (used < DEG ? MLS_ST_DEGRADED : 0));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}


template <int DEG, int WK>
void launch_one64(const KParams &p, int d0, int Dc, uint32_t idesc, cudaStream_t st) {
  const dim3 grid(p.tiles_x, p.tiles_y * 2);
  auto k = k_mls_tc64<DEG, WK>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem64);
  k<<<grid, kThr64, kSmem64, st>>>(p, d0, Dc, idesc);
}

}  // namespace

int tc64_dims_per_pass(int degree) { return (kN64 - 16) / mlsk::n_terms(degree); }

mls_status launch_tc64(const KParams &p, cudaStream_t st, int *nlaunch) {
  *nlaunch = 0;
  if (p.weight != MLS_W_GAUSS && p.weight != MLS_W_WENDLAND)
    return fail(MLS_E_UNSUPPORTED, "FP64 emulation takes the Gaussian and Wendland weights");
  if (!p.cell_start) return fail(MLS_E_UNSUPPORTED, "FP64 emulation needs the binned points");
  const int dmax = tc64_dims_per_pass(p.degree);
  const int passes = (p.D + dmax - 1) / dmax;
  const int Dc = (p.D + passes - 1) / passes;
  // kind::f16 with FP16 A and B, FP32 accumulators, M = 128, N = 48
  const uint32_t idesc = (1u << 4) | ((uint32_t)(kN64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  for (int d0 = 0; d0 < p.D; d0 += Dc) {
    if (p.weight == MLS_W_GAUSS) {
      if (p.degree == 0) launch_one64<0, MLS_W_GAUSS>(p, d0, Dc, idesc, st);
      else if (p.degree == 1) launch_one64<1, MLS_W_GAUSS>(p, d0, Dc, idesc, st);
      else launch_one64<2, MLS_W_GAUSS>(p, d0, Dc, idesc, st);
    } else {
      if (p.degree == 0) launch_one64<0, MLS_W_WENDLAND>(p, d0, Dc, idesc, st);
      else if (p.degree == 1) launch_one64<1, MLS_W_WENDLAND>(p, d0, Dc, idesc, st);
      else launch_one64<2, MLS_W_WENDLAND>(p, d0, Dc, idesc, st);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mls_tc64 launch");
    ++*nlaunch;
  }
  return MLS_OK;
}

}  // namespace mlsi
