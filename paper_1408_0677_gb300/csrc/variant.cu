// The paper's other two MLS mappings of 2-D values (D = 2): the rigid form
// (Section 3.3.3, Eqs. eq-rigidmls and eq-rigidmlspartial) and the mean
// displacement (Section 3.3.1, Eq. eq-meanmls).  Point i sits at p_i (the
// distorted position) and carries q_i (its original position); with the
// weights w_i of the polynomial fit (same stabiliser and support):
//
//   p* = sum w p / sum w, q* = sum w q / sum w, u = v - p*,
//   mu1 = sum w dq . dp, mu2 = sum w (dq_x dp_y - dq_y dp_x)
//         (dp = p - p*, dq = q - q*),
//   rigid: f(v) = q* + |u| (mu1 u_x + mu2 u_y, mu1 u_y - mu2 u_x) / |.|,
//   mean:  f(v) = q* + u.
//
// The rigid quotient is undefined where every point of positive weight sits
// at one position (one point in a Wendland support, duplicates): no
// rotation is taken there, f(v) = q* + u.
//
// One thread per pixel, 16 x 8 pixels per block, points staged through
// shared memory.  The centroids and the cross moments are accumulated by
// weighted Welford updates (each point moves the running means by
// w / W of its offset and adds W_old w / W times the product of its offsets
// to the co-moments), so the moments are centred as they are summed: raw
// sums about the pixel lose the angle to cancellation when one weight
// dominates the rest by orders of magnitude, which is common near the edge
// of a compact support.  FP64 renders run it in double on the raw
// coordinates and values; FP32 and FP16 renders in float on the h-scaled
// frame and the normalised values.
#include <float.h>

#include "mls_internal.h"

namespace mlsi {
namespace {

using namespace mlsk;

constexpr int kVChunk = 128;

// pixel centre: FP64 in raw coordinates, in the FP64 definition's expression
// order; FP32 in the h-scaled frame of xs/ys
__device__ __forceinline__ void centre(const KParams &p, int u, int v, double &px, double &py) {
  px = __dadd_rn(p.x0, __dmul_rn(__dadd_rn((double)u, 0.5), p.sx));
  py = __dadd_rn(p.y0, __dmul_rn(__dadd_rn((double)v, 0.5), p.sy));
}
__device__ __forceinline__ void centre(const KParams &p, int u, int v, float &px, float &py) {
  px = scaled_px(p, u);
  py = scaled_py(p, v);
}

__device__ __forceinline__ void load_pos(const KParams &p, int64_t i, double &x, double &y) {
  x = p.x64[i];
  y = p.y64[i];
}
__device__ __forceinline__ void load_pos(const KParams &p, int64_t i, float &x, float &y) {
  x = p.xs[i];
  y = p.ys[i];
}
__device__ __forceinline__ void load_val(const KParams &p, int64_t i, double &a, double &b) {
  a = p.FT64[i];
  b = p.FT64[p.n + i];
}
__device__ __forceinline__ void load_val(const KParams &p, int64_t i, float &a, float &b) {
  a = p.FT32[i];
  b = p.FT32[p.n_pad + i];
}

__device__ __forceinline__ double sub(double a, double b) { return __dadd_rn(a, -b); }
__device__ __forceinline__ float sub(float a, float b) { return a - b; }
__device__ __forceinline__ double dist2(double dx, double dy) { return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)); }
__device__ __forceinline__ float dist2(float dx, float dy) { return fmaf(dx, dx, dy * dy); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
// w / W of the Welford update: exact in FP64; in FP32 the fast quotient (a
// relative error of a few ulp in one point's share moves the means and
// co-moments far less than the FP32 rounding of the sums themselves)
__device__ __forceinline__ double share(double w, double W) { return w / W; }
__device__ __forceinline__ float share(float w, float W) { return __fdividef(w, W); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }

// w for a pair at offset (dx, dy), squared distance r2 (raw units in double,
// units of h in float), m the stabiliser min r^2 (Eq. eq-weights; the
// Wendland kernel; the truncated Gaussian's box |dx|, |dy| < c h)
template <int WK>
__device__ __forceinline__ double pair_weight(double dx, double dy, double r2, double m, const KParams &p) {
  const double h2 = p.h * p.h;
  if (WK == MLS_W_GAUSS && p.trunc > 0.0 && !(fabs(dx) < p.trunc * p.h && fabs(dy) < p.trunc * p.h)) return 0.0;
  if (WK == MLS_W_GAUSS) return exp(-(r2 - m) / h2);
  if (WK == MLS_W_WENDLAND) {
    if (!(r2 < h2)) return 0.0;
    const double qd = sqrt(r2) / p.h, o = 1.0 - qd;
    return o * o * o * o * (4.0 * qd + 1.0);
  }
  return pow(m / r2, p.alpha);
}
template <int WK>
__device__ __forceinline__ float pair_weight(float dx, float dy, float r2, float m, const KParams &p) {
  if (WK == MLS_W_GAUSS && p.trunc > 0.0 && !(fabsf(dx) < (float)p.trunc && fabsf(dy) < (float)p.trunc)) return 0.f;
  if (WK == MLS_W_GAUSS) return exp2f((m - r2) * 1.4426950408889634f);
  if (WK == MLS_W_WENDLAND) {
    const float q = sqrtf(r2), o = 1.f - q, o2 = o * o;
    return (q < 1.f) ? o2 * o2 * fmaf(4.f, q, 1.f) : 0.f;
  }
  return exp2f((float)p.alpha * __log2f(m / r2));
}

template <typename T, int WK>
__global__ __launch_bounds__(128) void k_mls_variant(KParams p, int tiles_x) {
  constexpr bool kF64 = sizeof(T) == 8;
  __shared__ T sx[kVChunk], sy[kVChunk], sa[kVChunk], sb[kVChunk];
  const int t = threadIdx.x;
  const int bx = (int)(blockIdx.x % (unsigned)tiles_x), by = (int)(blockIdx.x / (unsigned)tiles_x);
  const int u = bx * 16 + (t & 15), v = by * 8 + (t >> 4);
  const bool inside = (u < p.W) && (v < p.H);
  T px, py;
  centre(p, u, v, px, py);
  // point ranges: all points, or the cell rows overlapping the block's pixels
  // +- h (Wendland) or +- c h (the truncated Gaussian's box)
  const bool binned = (WK == MLS_W_WENDLAND) || (WK == MLS_W_GAUSS && p.trunc > 0.0);
  const double rad = (WK == MLS_W_WENDLAND) ? p.h : p.trunc * p.h * (1.0 + 1e-5);
  int nr = 1, cx0 = 0, cx1 = 0, cy0 = 0;
  if (binned) {
    const double xa = p.x0 + (bx * 16 + 0.5) * p.sx, xb = p.x0 + (bx * 16 + 15.5) * p.sx;
    const double ya = p.y0 + (by * 8 + 0.5) * p.sy, yb = p.y0 + (by * 8 + 7.5) * p.sy;
    const double inv_cell = p.inv_cell;
    int cy1;
    cx0 = max((int)floor((fmin(xa, xb) - rad - p.gx0) * inv_cell), 0);
    cx1 = min((int)floor((fmax(xa, xb) + rad - p.gx0) * inv_cell), p.gx - 1);
    cy0 = max((int)floor((fmin(ya, yb) - rad - p.gy0) * inv_cell), 0);
    cy1 = min((int)floor((fmax(ya, yb) + rad - p.gy0) * inv_cell), p.gy - 1);
    nr = (cx0 <= cx1) ? max(cy1 - cy0 + 1, 0) : 0;
  }
  // stabiliser (Gaussian, inverse distance): m = min r^2 over all points
  T m = 0;
  if (WK != MLS_W_WENDLAND) {
    T mm = kF64 ? (T)DBL_MAX : (T)FLT_MAX;
    for (int64_t base = 0; base < p.n; base += kVChunk) {
      const int cnt = (int)min((int64_t)kVChunk, p.n - base);
      __syncthreads();
      if (t < cnt) load_pos(p, base + t, sx[t], sy[t]);
      __syncthreads();
      for (int j = 0; j < cnt; ++j) mm = vmin(mm, dist2(sub(sx[j], px), sub(sy[j], py)));
    }
    m = mm;
  }
  // Welford pass: sum of weights, running means of the offsets from the
  // pixel and of the values, co-moments of value and offset
  T W = 0, mpx = 0, mpy = 0, mqa = 0, mqb = 0, cxx = 0, cyy = 0, cxy = 0, cyx = 0, csa = 0, csb = 0;
  int ccnt = 0;
  for (int r = 0; r < nr; ++r) {
    int64_t a0 = 0, a1 = p.n;
    if (binned) {
      a0 = cell_at(p, (int64_t)(cy0 + r) * p.gx + cx0);
      a1 = cell_at(p, (int64_t)(cy0 + r) * p.gx + cx1 + 1);
    }
    for (int64_t base = a0; base < a1; base += kVChunk) {
      const int cnt = (int)min((int64_t)kVChunk, a1 - base);
      __syncthreads();
      if (t < cnt) {
        load_pos(p, base + t, sx[t], sy[t]);
        load_val(p, base + t, sa[t], sb[t]);
      }
      __syncthreads();
      for (int j = 0; j < cnt; ++j) {
        const T dx = sub(sx[j], px), dy = sub(sy[j], py);
        const T r2 = dist2(dx, dy);
        if (WK == MLS_W_INVDIST && r2 == (T)0) {
          ++ccnt;
          csa += sa[j];
          csb += sb[j];
          continue;
        }
        const T w = pair_weight<WK>(dx, dy, r2, m, p);
        if (!(w > (T)0)) continue;
        const T Wn = W + w, rr = share(w, Wn), g = W * rr;   // g = W_old w / W_new
        const T dpx = dx - mpx, dpy = dy - mpy, dqa = sa[j] - mqa, dqb = sb[j] - mqb;
        mpx += rr * dpx;
        mpy += rr * dpy;
        mqa += rr * dqa;
        mqb += rr * dqb;
        cxx += g * dqa * dpx;
        cyy += g * dqb * dpy;
        cxy += g * dqa * dpy;
        cyx += g * dqb * dpx;
        W = Wn;
      }
    }
  }
  if (!inside) return;
  // values: raw in double; (f - cen) / scl in float
  const T sca = kF64 ? (T)1 : (T)p.fscl32[0], scb = kF64 ? (T)1 : (T)p.fscl32[1];
  const T cna = kF64 ? (T)0 : (T)p.fcen32[0], cnb = kF64 ? (T)0 : (T)p.fcen32[1];
  const T hs = kF64 ? (T)1 : (T)p.h;   // offsets: raw in double, units of h in float
  T fa, fb;
  uint8_t st;
  if (ccnt > 0) {
    fa = cna + sca * (csa / (T)ccnt);
    fb = cnb + scb * (csb / (T)ccnt);
    st = MLS_ST_COINCIDENT;
  } else if (!(W > (T)0)) {
    fa = fb = kF64 ? (T)__longlong_as_double(0x7ff8000000000000ll) : (T)__int_as_float(0x7fc00000);
    st = MLS_ST_NO_SUPPORT;
  } else {
    const T qa = cna + sca * mqa, qb = cnb + scb * mqb;
    const T ux = -hs * mpx, uy = -hs * mpy;
    fa = qa + ux;
    fb = qb + uy;
    if (p.variant == MLS_V_RIGID) {
      T mu1 = sca * cxx + scb * cyy, mu2 = sca * cxy - scb * cyx;
      const T big = fmax(fabs(mu1), fabs(mu2));
      const T nu = sqrt(ux * ux + uy * uy);
      if (nu == (T)0) {
        fa = qa;
        fb = qb;
      } else if (big > (T)0) {
        mu1 /= big;
        mu2 /= big;
        const T ra = mu1 * ux + mu2 * uy, rb = mu1 * uy - mu2 * ux;
        const T s = nu / sqrt(ra * ra + rb * rb);
        fa = qa + s * ra;
        fb = qb + s * rb;
      }
    }
    st = 1;
  }
  const size_t plane = (size_t)p.W * p.H, pix = (size_t)v * p.W + u;
  T *field = (T *)p.field;
  field[pix] = fa;
  field[plane + pix] = fb;
  if (p.bands) {
    if (kF64) {
      p.bands[pix] = band_of((double)fa, p.lev64, p.L);
      p.bands[plane + pix] = band_of((double)fb, p.lev64 + p.L, p.L);
    } else {
      p.bands[pix] = band_of((float)fa, p.lev32, p.L);
      p.bands[plane + pix] = band_of((float)fb, p.lev32 + p.L, p.L);
    }
  }
  if (p.status) p.status[pix] = st;
}

template <typename T>
void variant_dispatch(const KParams &p, cudaStream_t st) {
  const int tiles_x = (p.W + 15) / 16, tiles_y = (p.H + 7) / 8;
  const unsigned grid = (unsigned)((int64_t)tiles_x * tiles_y);
  if (p.weight == MLS_W_GAUSS) k_mls_variant<T, MLS_W_GAUSS><<<grid, 128, 0, st>>>(p, tiles_x);
  else if (p.weight == MLS_W_WENDLAND) k_mls_variant<T, MLS_W_WENDLAND><<<grid, 128, 0, st>>>(p, tiles_x);
  else k_mls_variant<T, MLS_W_INVDIST><<<grid, 128, 0, st>>>(p, tiles_x);
}

}  // namespace

void launch_variant(const KParams &p, bool fp64, cudaStream_t st) {
  if (fp64) variant_dispatch<double>(p, st);
  else variant_dispatch<float>(p, st);
}

}  // namespace mlsi
