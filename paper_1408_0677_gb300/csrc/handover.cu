// Hand-over path of the reduced-precision renders: pixels whose moment
// matrix is ill conditioned in the pixel frame (one warp per pixel).
//
// The value of the weighted least-squares fit does not depend on the frame
// of the polynomial basis, but the rounding error of moments accumulated in
// FP32 / tensor-core arithmetic grows with the condition number of the frame
// they are accumulated in.  For a pixel whose weighted points lie to one
// side (the usual cause), the pixel frame is badly conditioned while a frame
// centred on the weighted centroid of the points and scaled by their spread
// is not.  So, per listed pixel:
//   pass 1 (FP64): the distinct moments of the pixel-centred, h-scaled basis
//          and the support count -- the degree policy is decided on these
//          exactly as the FP64 definition does (equilibrated Cholesky,
//          rcond_1 threshold, support count);
//   solve  (FP64): the moments are moved to the centroid frame, where the
//          normal matrix is factorised and z = M_c^{-1} b(p) is formed;
//   pass 2 (FP32): the right-hand sides R_c = sum w b_c(x) f are accumulated
//          in the centroid frame, lane-parallel with a tree reduction, and
//          the value is z . R_c.
// Pixels still ill conditioned in the centroid frame, and inverse-distance
// pixels whose centre lies on a data point, go on to the pure FP64 kernel.
#include <float.h>

#include "mls_internal.h"

namespace mlsi {
namespace {

using namespace mlsk;

constexpr int kDC = 16;                 // value dimensions per pass 2 sweep
constexpr double kCut = 60.0;           // Gaussian pairs with (r^2 - m)/h^2 above: weight < e^-60
constexpr double kKappaCentroid = 3e3;  // above: the pixel goes to the FP64 kernel
// FP32 rounding of the right-hand sides moves the value by at most about
// eps32 * lambda * (summation growth) of the normalised data range, with
// lambda = sum_a |z_a| sqrt(M_00 M_aa) (Cauchy-Schwarz on each R_a); above
// this bound the pixel goes to the FP64 kernel.
constexpr double kLambdaMax = 2e3;
constexpr double kLog2e = 1.4426950408889634;

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Equilibrated Cholesky of the k x k matrix from distinct moments (runtime k);
// returns rcond_1 (0 on failure).  Lm receives the factor of the equilibrated
// matrix, sd the equilibration.
__device__ double factor_moments(const double *S, int k, double (&Lm)[6][6], double (&sd)[6]) {
  double Me[6][6];
  for (int a = 0; a < k; ++a) {
    const double d = S[kMIdx[a][a]];
    if (!(d > 0.0)) return 0.0;
    sd[a] = 1.0 / sqrt(d);
  }
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) Me[a][b] = S[kMIdx[a][b]] * sd[a] * sd[b];
  for (int j = 0; j < k; ++j) {
    double s = Me[j][j];
    for (int t = 0; t < j; ++t) s -= Lm[j][t] * Lm[j][t];
    if (!(s > 0.0)) return 0.0;
    const double ljj = sqrt(s);
    Lm[j][j] = ljj;
    for (int i = j + 1; i < k; ++i) {
      double v = Me[i][j];
      for (int t = 0; t < j; ++t) v -= Lm[i][t] * Lm[j][t];
      Lm[i][j] = v / ljj;
    }
  }
  double nA = 0.0, nI = 0.0;
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
    double sa = 0.0, si = 0.0;
    for (int a = 0; a < k; ++a) {
      sa += fabs(Me[a][c]);
      si += fabs(col[a]);
    }
    nA = fmax(nA, sa);
    nI = fmax(nI, si);
  }
  return 1.0 / (nA * nI);
}

// The weight of one pair as used by both passes: FP64 distance, FP32 rounding
// of the weight (its relative error ~1e-7 acts as a common perturbation of
// the least-squares weights, far below the tolerance of these paths).
template <int WK>
__device__ __forceinline__ float pair_w(double r2, double m, double h, double h2, float alpha) {
  if (WK == MLS_W_GAUSS) {
    return exp2f((float)(-(r2 - m) / h2 * kLog2e));
  } else if (WK == MLS_W_WENDLAND) {
    const float q = (float)(sqrt(r2) / h), o = 1.f - q, o2 = o * o;
    return o2 * o2 * fmaf(4.f, q, 1.f);
  } else {
    return exp2f(alpha * log2f((float)(m / r2)));
  }
}

__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

template <int DEG, int WK>
__global__ __launch_bounds__(256) void k_handover(KParams p, const int *list, const unsigned int *list_count,
                                                  int64_t cap, int *list2, unsigned int *list2_count) {
  constexpr int K = n_terms(DEG), NM = n_moments(DEG);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t npix = (int64_t)*list_count < cap ? (int64_t)*list_count : cap;
  const size_t plane = (size_t)p.W * p.H;
  const double h = p.h, h2 = h * h, inv_s = 1.0 / h;
  float *field = (float *)p.field;

  for (int64_t qi = warp0; qi < npix; qi += nwarps) {
    const int id = list[qi];
    const int u = id % p.W, v = id / p.W;
    const double px = __dadd_rn(p.x0, __dmul_rn(__dadd_rn((double)u, 0.5), p.sx));
    const double py = __dadd_rn(p.y0, __dmul_rn(__dadd_rn((double)v, 0.5), p.sy));
    const float pxs = scaled_px(p, u), pys = scaled_py(p, v);
    const size_t pi = (size_t)v * (p.tiles_x * 16) + u;
    const float mhat = (WK == MLS_W_WENDLAND) ? 0.f : p.mstab[pi];
    const double m = (double)mhat * h2;
    int a0s[3] = {0, 0, 0}, a1s[3] = {0, 0, 0}, nr = 1;
    if (WK == MLS_W_WENDLAND) {
      const double inv_cell = 1.0 / p.cell;
      const int cx0 = max((int)floor((px - h - p.gx0) * inv_cell), 0);
      const int cx1 = min((int)floor((px + h - p.gx0) * inv_cell), p.gx - 1);
      const int cy0 = max((int)floor((py - h - p.gy0) * inv_cell), 0);
      const int cy1 = min((int)floor((py + h - p.gy0) * inv_cell), p.gy - 1);
      nr = 0;
      for (int cy = cy0; cy <= cy1 && cx0 <= cx1 && nr < 3; ++cy, ++nr) {
        a0s[nr] = p.cell_start[cy * p.gx + cx0];
        a1s[nr] = p.cell_start[cy * p.gx + cx1 + 1];
      }
    } else {
      a1s[0] = (int)p.n;
    }

    // ---- pass 1: FP64 pixel-frame moments and support count
    double S[15];
#pragma unroll
    for (int j = 0; j < 15; ++j) S[j] = 0.0;
    long long count = 0;
    int coincident = 0;
    for (int r = 0; r < nr; ++r) {
      for (int i = a0s[r] + lane; i < a1s[r]; i += 32) {
        if (WK == MLS_W_GAUSS) {
          ++count;
          const float dxs = p.xs[i] - pxs, dys = p.ys[i] - pys;
          if (fmaf(dxs, dxs, dys * dys) - mhat > (float)kCut + 1.f) continue;
        }
        const double dx = __dadd_rn(p.x64[i], -px), dy = __dadd_rn(p.y64[i], -py);
        const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        if (WK == MLS_W_GAUSS) {
          if (r2 - m > kCut * h2) continue;
        } else if (WK == MLS_W_WENDLAND) {
          if (!(r2 < h2)) continue;
          ++count;
        } else {
          ++count;
          if (r2 == 0.0) {
            coincident = 1;
            continue;
          }
        }
        const double w = (double)pair_w<WK>(r2, m, h, h2, (float)p.alpha);
        const double ex = dx * inv_s, ey = dy * inv_s;
        double mo[15];
        mo[0] = 1.0;
        if (NM > 1) { mo[1] = ex; mo[2] = ey; mo[3] = ex * ex; mo[4] = ex * ey; mo[5] = ey * ey; }
        if (NM > 6) {
          mo[6] = mo[3] * ex; mo[7] = mo[3] * ey; mo[8] = mo[5] * ex; mo[9] = mo[5] * ey;
          mo[10] = mo[3] * mo[3]; mo[11] = mo[3] * mo[4]; mo[12] = mo[3] * mo[5]; mo[13] = mo[4] * mo[5];
          mo[14] = mo[5] * mo[5];
        }
#pragma unroll
        for (int j = 0; j < NM; ++j) S[j] += w * mo[j];
      }
    }
#pragma unroll
    for (int j = 0; j < NM; ++j) S[j] = wsum(S[j]);
    count = wsum(count);
    const bool to_fp64 = (WK == MLS_W_INVDIST) && __any_sync(0xffffffffu, coincident);

    // ---- degree policy on the pixel-frame moments (FP64)
    int used = -1;
    double Lm[6][6], sd[6];
    if (!to_fp64) {
      for (int deg = DEG; deg >= 0 && used < 0; --deg) {
        const int k = n_terms(deg);
        if (count < k) continue;
        const double rc = factor_moments(S, k, Lm, sd);
        if (rc >= p.rcond_min) used = deg;
      }
    }
    // ---- centroid frame and the solve for z
    double z[6] = {0, 0, 0, 0, 0, 0};
    double cxh = 0.0, cyh = 0.0, isg = 1.0;    // centroid offset (raw units) and 1/(h sigma)
    bool bad = to_fp64;
    if (!bad && used == 0) {
      z[0] = 1.0 / S[0];
    } else if (!bad && used > 0) {
      const int k = n_terms(used);
      const double cx = S[1] / S[0], cy = S[2] / S[0];
      const double var = (S[3] + S[5]) / S[0] - cx * cx - cy * cy;
      if (!(var > 0.0)) {
        bad = true;
      } else {
        const double sg = sqrt(var);
        double Sc[15];
        const int nm = n_moments(used);
        for (int j = 0; j < nm; ++j) {
          const int bx = mono_ex(j), by = mono_ey(j);
          double acc = 0.0;
          for (int jx = 0; jx <= bx; ++jx)
            for (int jy = 0; jy <= by; ++jy)
              acc += binom(bx, jx) * binom(by, jy) * ipow(-cx, bx - jx) * ipow(-cy, by - jy) *
                     S[mono_index(jx, jy)];
          Sc[j] = acc / ipow(sg, bx + by);
        }
        double Lc[6][6], sdc[6];
        const double rcc = factor_moments(Sc, k, Lc, sdc);
        if (!(rcc > 1.0 / kKappaCentroid)) {
          bad = true;
        } else {
          // z = M_c^{-1} b_c(pixel), b_c(pixel) at (-cx, -cy)/sg
          const double ex = -cx / sg, ey = -cy / sg;
          double b[6] = {1.0, ex, ey, ex * ex, ex * ey, ey * ey};
          for (int a = 0; a < k; ++a) b[a] *= sdc[a];
          for (int i = 0; i < k; ++i) {
            double vv = b[i];
            for (int t = 0; t < i; ++t) vv -= Lc[i][t] * b[t];
            b[i] = vv / Lc[i][i];
          }
          for (int i = k - 1; i >= 0; --i) {
            double vv = b[i];
            for (int t = i + 1; t < k; ++t) vv -= Lc[t][i] * b[t];
            b[i] = vv / Lc[i][i];
          }
          double lambda = 0.0;
          for (int a = 0; a < k; ++a) {
            z[a] = b[a] * sdc[a];
            lambda += fabs(z[a]) * sqrt(Sc[0] * Sc[kMIdx[a][a]]);
          }
          if (!(lambda <= kLambdaMax)) bad = true;
          cxh = cx * h;
          cyh = cy * h;
          isg = inv_s / sg;
        }
      }
    }
    if (bad) {
      if (lane == 0) {
        const unsigned int k2 = atomicAdd(list2_count, 1u);
        list2[k2] = id;
      }
      continue;
    }
    if (used < 0) {
      for (int d = lane; d < p.D; d += 32) {
        field[(size_t)d * plane + id] = __int_as_float(0x7fc00000);
        if (p.bands) p.bands[(size_t)d * plane + id] = 255;
      }
      if (lane == 0 && p.status) p.status[id] = MLS_ST_NO_SUPPORT | MLS_ST_RECOMPUTED;
      continue;
    }
    const int ku = n_terms(used);

    // ---- pass 2: FP32 right-hand sides in the centroid frame
    for (int d0 = 0; d0 < p.D; d0 += kDC) {
      float R[K][kDC];
#pragma unroll
      for (int a = 0; a < K; ++a)
#pragma unroll
        for (int dd = 0; dd < kDC; ++dd) R[a][dd] = 0.f;
      for (int r = 0; r < nr; ++r) {
        for (int i = a0s[r] + lane; i < a1s[r]; i += 32) {
          if (WK == MLS_W_GAUSS) {
            const float dxs = p.xs[i] - pxs, dys = p.ys[i] - pys;
            if (fmaf(dxs, dxs, dys * dys) - mhat > (float)kCut + 1.f) continue;
          }
          const double dx = __dadd_rn(p.x64[i], -px), dy = __dadd_rn(p.y64[i], -py);
          const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
          if (WK == MLS_W_GAUSS) {
            if (r2 - m > kCut * h2) continue;
          } else if (WK == MLS_W_WENDLAND) {
            if (!(r2 < h2)) continue;
          }
          const float w = pair_w<WK>(r2, m, h, h2, (float)p.alpha);
          // centroid-frame coordinates formed in FP64 (no cancellation in FP32)
          const float ex = (float)((dx - cxh) * isg), ey = (float)((dy - cyh) * isg);
          float b[6];
          b[0] = w;
          if (K > 1) { b[1] = w * ex; b[2] = w * ey; }
          if (K > 3) { b[3] = w * ex * ex; b[4] = w * ex * ey; b[5] = w * ey * ey; }
#pragma unroll
          for (int dd = 0; dd < kDC; ++dd) {
            const float f = (d0 + dd < p.D) ? p.FT32[(size_t)(d0 + dd) * p.n_pad + i] : 0.f;
#pragma unroll
            for (int a = 0; a < K; ++a) R[a][dd] = fmaf(b[a], f, R[a][dd]);
          }
        }
      }
#pragma unroll
      for (int a = 0; a < K; ++a)
#pragma unroll
        for (int dd = 0; dd < kDC; ++dd) R[a][dd] = wsum(R[a][dd]);
#pragma unroll
      for (int dd = 0; dd < kDC; ++dd) {
        const int d = d0 + dd;
        if (lane == dd && d < p.D) {
          double acc = 0.0;
          for (int a = 0; a < ku; ++a) acc += z[a] * (double)R[a][dd];
          const float f = (float)((double)p.fcen32[d] + (double)p.fscl32[d] * acc);
          field[(size_t)d * plane + id] = f;
          if (p.bands) p.bands[(size_t)d * plane + id] = band_of(f, p.lev32 + (size_t)d * p.L, p.L);
        }
      }
    }
    if (lane == 0 && p.status)
      p.status[id] = (uint8_t)(used | MLS_ST_RECOMPUTED | (used < DEG ? MLS_ST_DEGRADED : 0));
  }
}

template <int WK>
void launch_w(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int *list2,
              unsigned int *cnt2, cudaStream_t st) {
  const int grid = 152 * 8;
  if (p.degree == 0) k_handover<0, WK><<<grid, 256, 0, st>>>(p, list, cnt, cap, list2, cnt2);
  else if (p.degree == 1) k_handover<1, WK><<<grid, 256, 0, st>>>(p, list, cnt, cap, list2, cnt2);
  else k_handover<2, WK><<<grid, 256, 0, st>>>(p, list, cnt, cap, list2, cnt2);
}

}  // namespace

void launch_handover(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int *list2,
                     unsigned int *cnt2, cudaStream_t st) {
  if (p.weight == MLS_W_GAUSS) launch_w<MLS_W_GAUSS>(p, list, cnt, cap, list2, cnt2, st);
  else if (p.weight == MLS_W_WENDLAND) launch_w<MLS_W_WENDLAND>(p, list, cnt, cap, list2, cnt2, st);
  else launch_w<MLS_W_INVDIST>(p, list, cnt, cap, list2, cnt2, st);
}

}  // namespace mlsi
