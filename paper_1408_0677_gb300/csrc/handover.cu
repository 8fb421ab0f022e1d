// Hand-over path of the reduced-precision renders: pixels whose moment
// matrix is ill conditioned in the frame the fast kernels use (one warp per
// pixel).
//
// The value of the weighted least-squares fit (Section 3.3) does not depend
// on the frame of the polynomial basis, but the rounding error of moments
// accumulated in FP32 / tensor-core arithmetic grows with the condition
// number of the frame they are accumulated in.  For a pixel whose weighted
// points lie to one side (the usual cause), the pixel frame is badly
// conditioned while a frame centred on the weighted centroid of the points
// and scaled by their spread is not.  So, per listed pixel:
//   pass 1 (double-float, ~48 bits, on the FP32 units): the distinct moments
//          of the pixel-centred, h-scaled basis and the support count; the
//          degree policy is decided on these as the FP64 definition does
//          (equilibrated factorisation, rcond_1 threshold, support count);
//   solve  (FP64, one lane per pixel for a chunk of 32 pixels): the moments
//          are moved to the centroid frame, where the normal matrix is
//          factorised and z = M_c^{-1} b_c(p) is formed;
//   pass 2 (double-float): the value is sum_i phi_i f_i with the MLS shape
//          functions phi_i = w_i z . b_c(x_i) -- equal to z . R_c -- so each
//          (point, dimension) pair costs one multiply-add; the lanes hold one
//          dimension each and read the values point-major.
// Both passes walk the candidate points 32 at a time, compact the near ones
// (Gaussian weight above e^-40 of the largest, inside the Wendland support)
// into a per-warp ring in shared memory, and process them in dense batches of
// 32 so that no lane idles on a far point.  Weights are double-float too
// (exp and sqrt in FP32 arithmetic: FP64 throughput is low on this part).
// Pixels still ill conditioned in the centroid frame, and inverse-distance
// pixels whose centre lies on a data point, go on to the pure FP64 kernel.
#include <float.h>

#include "mls_internal.h"

namespace mlsi {
namespace {

using namespace mlsk;

constexpr int kWarps = 4;               // warps per block (each owns chunks of 32 pixels)
constexpr int kRing = 64;               // ring of compacted near points per warp
constexpr int kDL = 2;                  // value dimensions per lane per sweep
constexpr float kCut = 40.f;            // Gaussian pairs with (r^2 - m)/h^2 above: weight < e^-40
// centroid-frame condition above which the pixel goes to the FP64 kernel
// (moments and right-hand sides are double-float accurate, ~1e-14)
constexpr double kKappaCentroid = 1e8;

// ---------------------------------------------------------------------------
// Normalised warp-wide double-float sum (the accumulation helpers df_prod,
// df_prod_f and df_acc are shared with the FP64 tier's value sums).
__device__ __forceinline__ df32 df_warp_sum(df32 v) {
  v = df_two_sum(v.hi, v.lo);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df32 t = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, t);
  }
  return v;
}

// ---------------------------------------------------------------------------
// Near points and their weights.

// Whether a point enters the sums: Gaussian weight above e^-kCut of the
// largest, or for the truncated Gaussian (boxed: cbox = c > 0) inside the box
// |dx|, |dy| < c, every point of which counts (double-float offsets); inside
// the Wendland support (double-float distance); any point but a coincident
// one for inverse distance.  `boxed` is decided once per walk: a comparison
// of doubles per candidate took GB300's FP64 pipe a tenth busy.
template <int WK>
__device__ __forceinline__ bool near_test(df32 ex, df32 ey, float mhat, double cbox, bool boxed) {
  if (WK == MLS_W_GAUSS && boxed)
    return fabs((double)ex.hi + (double)ex.lo) < cbox && fabs((double)ey.hi + (double)ey.lo) < cbox;
  if (WK == MLS_W_GAUSS) return fmaf(ex.hi, ex.hi, ey.hi * ey.hi) - mhat <= kCut;
  if (WK == MLS_W_WENDLAND) {
    const df32 r2d = df_add(df_mul(ex, ex), df_mul(ey, ey));
    return (r2d.hi < 1.f) || (r2d.hi == 1.f && r2d.lo < 0.f);
  }
  return !(ex.hi == 0.f && ex.lo == 0.f && ey.hi == 0.f && ey.lo == 0.f);
}

// Weight of one pair, double-float, from the double-float offset (units of
// h): Gaussian relative to the stabiliser (exp(m - r^2)), Wendland in units
// of the radius, inverse distance (m / r^2)^alpha (FP64 pow).
template <int WK>
__device__ __forceinline__ df32 pair_wdf(df32 ex, df32 ey, float mhat, double alpha, const float2 *tab) {
  const df32 r2 = df_add(df_mul(ex, ex), df_mul(ey, ey));
  if (WK == MLS_W_GAUSS) {
    // below e^-87 of the largest weight (possible only in a wide truncation
    // box) the pair adds nothing at FP64 rounding; df_exp's scale needs a >= -87
    const df32 a = df_add({mhat, 0.f}, {-r2.hi, -r2.lo});
    return a.hi < -87.f ? df32{0.f, 0.f} : df_exp(a, tab);
  }
  if (WK == MLS_W_WENDLAND) return df_wendland(r2);
  const double w = pow((double)mhat / ((double)r2.hi + (double)r2.lo), alpha);
  return {(float)w, (float)(w - (double)(float)w)};
}

// Candidate points of one pixel: all points (all_n > 0), or the cells
// [cx0, cx1] x [cy0, cy1] of the uniform grid that cover its near radius.
struct Ranges {
  int cx0, cx1, cy0, cy1, all_n;
};

// Walk the candidates 32 at a time, compact the near ones into the warp's
// ring and call body(valid, i, ex, ey) on dense batches, one point per lane
// (only the last batch has lanes with valid == false).  The whole warp calls
// body.  Returns the number of near points; *coincident is set when a
// candidate lies exactly on the pixel centre (inverse distance).
template <int WK, typename Body>
__device__ __forceinline__ int for_near(const KParams &p, const Ranges &R, float pxh, float pxl, float pyh,
                                        float pyl, float mhat, int lane, int *ri, float4 *rx, int *coincident,
                                        Body body) {
  const unsigned int lt = (1u << lane) - 1u;
  const bool boxed = WK == MLS_W_GAUSS && p.trunc > 0.0;
  int head = 0, total = 0, coin = 0;
  const int nrow = R.all_n > 0 ? 1 : (R.cx0 <= R.cx1 ? R.cy1 - R.cy0 + 1 : 0);
  // the lanes fetch the index ranges of up to 32 cell rows at once
  int my0 = 0, my1 = 0;
  for (int r = 0; r < nrow; ++r) {
    if ((r & 31) == 0) {
      const int rr = r + lane;
      if (R.all_n > 0) {
        my0 = 0;
        my1 = R.all_n;
      } else if (rr < nrow) {
        my0 = cell_at(p, (int64_t)(R.cy0 + rr) * p.gx + R.cx0);
        my1 = cell_at(p, (int64_t)(R.cy0 + rr) * p.gx + R.cx1 + 1);
      }
    }
    const int a0 = __shfl_sync(0xffffffffu, my0, r & 31);
    const int a1 = __shfl_sync(0xffffffffu, my1, r & 31);
    for (int base = a0; base < a1; base += 32) {
      const int i = base + lane;
      bool nr = false;
      df32 ex = {0.f, 0.f}, ey = {0.f, 0.f};
      if (i < a1) {
        ex = df_diff(p.xs[i], p.xs_lo[i], pxh, pxl);
        ey = df_diff(p.ys[i], p.ys_lo[i], pyh, pyl);
        nr = near_test<WK>(ex, ey, mhat, p.trunc, boxed);
        if (WK == MLS_W_INVDIST && !nr) coin = 1;
      }
      const unsigned int bal = __ballot_sync(0xffffffffu, nr);
      if (nr) {
        const int s = head + __popc(bal & lt);   // < 64: head < 32 here
        ri[s] = i;
        rx[s] = make_float4(ex.hi, ex.lo, ey.hi, ey.lo);
      }
      head += __popc(bal);
      total += __popc(bal);
      __syncwarp();
      if (head >= 32) {
        const float4 e = rx[lane];
        const int ii = ri[lane];
        __syncwarp();
        if (lane < head - 32) {
          ri[lane] = ri[lane + 32];
          rx[lane] = rx[lane + 32];
        }
        __syncwarp();
        head -= 32;
        body(true, ii, df32{e.x, e.y}, df32{e.z, e.w});
      }
    }
  }
  if (head > 0) {
    const bool v = lane < head;
    const float4 e = v ? rx[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ii = v ? ri[lane] : 0;
    body(v, ii, df32{e.x, e.y}, df32{e.z, e.w});
  }
  __syncwarp();
  *coincident = __any_sync(0xffffffffu, coin);
  return total;
}

// ---------------------------------------------------------------------------
// Degree policy and centroid-frame solve, one lane per pixel, in a scalar
// type T: FP64 (double), or double-float (dd: hi + lo pairs of FP32, about
// 46 significant bits) on the FP32 pipes.  GB300 runs FP64 at a small
// fraction of its FP32 rate: the split kernels' policy kernel, which has the
// SM to itself, runs in double-float; the fused kernel, whose blocks overlap
// one block's policy warp with the other blocks' double-float phases, in
// FP64 (fewer instructions and registers on its one policy warp).  46 bits
// resolve the rcond_1 threshold test of the definition with room to spare
// (the decision is ambiguous only within a factor around the threshold, far
// wider than the rounding here), and z carries a relative error of about
// 2^-46 times the centroid-frame condition (<= 1e8).

struct dd {
  float hi, lo;
};
__device__ __forceinline__ dd ddf(float a) { return {a, 0.f}; }
__device__ __forceinline__ dd ddd(double a) {
  const float h = (float)a;
  return {h, (float)(a - (double)h)};
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const df32 r = df_add({a.hi, a.lo}, {b.hi, b.lo});
  return {r.hi, r.lo};
}
__device__ __forceinline__ dd operator-(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const df32 r = df_mul({a.hi, a.lo}, {b.hi, b.lo});
  return {r.hi, r.lo};
}
__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
// the sign is that of hi (a normalised pair has |lo| <= ulp(hi) / 2)
__device__ __forceinline__ bool operator>(dd a, dd b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator>=(dd a, dd b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
// a / b: the FP32 quotient q1, then the quotient of the remainder a - q1 b
__device__ __forceinline__ dd ddiv(dd a, dd b) {
  const float q1 = a.hi / b.hi;
  const df32 qb = df_mul_f({b.hi, b.lo}, q1);
  const dd r = a - dd{qb.hi, qb.lo};
  const float q2 = r.hi / b.hi;
  const df32 q = df_two_sum(q1, q2);
  return {q.hi, q.lo};
}

// The operations the policy needs, for both scalar types.
template <typename T> __device__ __forceinline__ T tc_(float a);
template <> __device__ __forceinline__ double tc_<double>(float a) { return (double)a; }
template <> __device__ __forceinline__ dd tc_<dd>(float a) { return ddf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ dd tabs(dd a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ dd tmax(dd a, dd b) { return b > a ? b : a; }
// 1/d for a positive normal d: FP32 seed and two Newton steps in FP64 (each
// doubles the number of correct bits: 2^-23 -> 2^-46 -> FP64 rounding)
__device__ __forceinline__ double trcp(double d) {
  double r = (double)__frcp_rn((float)d);
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}
__device__ __forceinline__ dd trcp(dd b) { return ddiv(ddf(1.f), b); }
__device__ __forceinline__ double trsqrt(double b) { return rsqrt(b); }
// 1/sqrt(b), b > 0: the FP32 estimate r and one Newton step in double-float,
// r + r (1 - b r^2) / 2 (the step doubles the correct bits, 2^-22 -> 2^-44)
__device__ __forceinline__ dd trsqrt(dd b) {
  const float r = rsqrtf(b.hi);
  const dd e = ddf(1.f) - b * (ddf(r) * ddf(r));
  return ddf(r) + ddf(0.5f * r) * e;
}
// v as a pair of floats hi + lo (the form the value phase reads)
__device__ __forceinline__ void tsplit(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}
__device__ __forceinline__ void tsplit(dd v, float &hi, float &lo) {
  hi = v.hi;
  lo = v.lo;
}
__device__ __forceinline__ void tjoin(float hi, float lo, double &v) { v = (double)hi + (double)lo; }
__device__ __forceinline__ void tjoin(float hi, float lo, dd &v) {
  const df32 t = df_two_sum(hi, lo);
  v = {t.hi, t.lo};
}
__device__ __forceinline__ void tfrom(double a, double &v) { v = a; }
__device__ __forceinline__ void tfrom(double a, dd &v) { v = ddd(a); }

// Equilibrated LDL^T factorisation of the K x K moment matrix S[midx(a, b)]
// and rcond_1 = 1 / (|Me|_1 |Me^-1|_1) of the equilibrated matrix Me.
// Returns 0 when a diagonal entry or a pivot is not positive.  L (unit
// lower), dinv (inverse pivots) and sd (equilibration 1/sqrt(M_aa)) receive
// the factorisation.
template <int K, typename T>
__device__ T ldl_rcond(const T (&S)[15], T (&L)[6][6], T (&dinv)[6], T (&sd)[6]) {
  const T zero = tc_<T>(0.f);
  T Me[K][K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    const T d = S[midx(a, a)];
    if (!(d > zero)) return zero;
    sd[a] = trsqrt(d);
  }
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) Me[a][b] = Me[b][a] = S[midx(a, b)] * sd[a] * sd[b];
  // LDL^T (no square roots): D_j = Me_jj - sum_t L_jt (L_jt D_t),
  // L_ij = (Me_ij - sum_t L_it (L_jt D_t)) / D_j, with LD_jt = L_jt D_t kept
  // (it is the numerator of L_jt before the division)
  T LD[K][K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    T dj = Me[j][j];
#pragma unroll
    for (int t = 0; t < j; ++t) dj -= L[j][t] * LD[j][t];
    if (!(dj > zero)) return zero;
    dinv[j] = trcp(dj);
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      T v = Me[i][j];
#pragma unroll
      for (int t = 0; t < j; ++t) v -= L[i][t] * LD[j][t];
      LD[i][j] = v;
      L[i][j] = v * dinv[j];
    }
  }
  // 1-norms of Me and of its inverse.  Me^-1 = L^-T D^-1 L^-1 is symmetric:
  // with Li = L^-1 (unit lower) and G_kj = dinv_k Li_kj, its entry (i, j),
  // i <= j, is sum_{k >= j} Li_ki G_kj (about a third of the operations of K
  // forward and back substitutions)
  T Li[K][K], G[K][K];
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      T v = -L[i][j];
#pragma unroll
      for (int t = j + 1; t < i; ++t) v -= L[i][t] * Li[t][j];
      Li[i][j] = v;
    }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    G[k][k] = dinv[k];
#pragma unroll
    for (int j = 0; j < k; ++j) G[k][j] = dinv[k] * Li[k][j];
  }
  T cI[K], cA[K];
#pragma unroll
  for (int c = 0; c < K; ++c) cI[c] = cA[c] = zero;
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int i = 0; i <= j; ++i) {
      T v = G[j][j] * (j == i ? tc_<T>(1.f) : Li[j][i]);
#pragma unroll
      for (int k = j + 1; k < K; ++k) v += Li[k][i] * G[k][j];
      const T av = tabs(v), am = tabs(Me[i][j]);
      cI[j] += av;
      cA[j] += am;
      if (i != j) {
        cI[i] += av;
        cA[i] += am;
      }
    }
  T nI = zero, nA = zero;
#pragma unroll
  for (int c = 0; c < K; ++c) {
    nI = tmax(nI, cI[c]);
    nA = tmax(nA, cA[c]);
  }
  return trcp(nA * nI);
}

// b <- M^-1 b with M = S^-1 Me S^-1 factorised as above: S Me^-1 S b.
template <int K, typename T>
__device__ __forceinline__ void ldl_solve(const T (&L)[6][6], const T (&dinv)[6], const T (&sd)[6], T (&b)[6]) {
#pragma unroll
  for (int a = 0; a < K; ++a) b[a] = b[a] * sd[a];
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int t = 0; t < i; ++t) b[i] -= L[i][t] * b[t];
#pragma unroll
  for (int i = 0; i < K; ++i) b[i] = b[i] * dinv[i];
#pragma unroll
  for (int i = K - 1; i >= 0; --i)
#pragma unroll
    for (int t = i + 1; t < K; ++t) b[i] -= L[t][i] * b[t];
#pragma unroll
  for (int a = 0; a < K; ++a) b[a] = b[a] * sd[a];
}

// Moments of the frame centred on (cx, cy) and scaled by isg, from the
// pixel-frame moments: sum_i w_i (x_i - cx)^bx (y_i - cy)^by, by binomial
// expansion.  The expansion is separable: a shift in x of every row of equal
// y exponent, then a shift in y of every column.  A 1-D shift of moments
// a_0..a_m by c is the Taylor shift: m passes, pass i replacing a_k by
// a_k - c a_(k-1) for k = m down to i (m (m + 1) / 2 multiply-adds).
template <int NM, typename T>
__device__ __forceinline__ void centroid_moments(const T (&S)[15], T cx, T cy, T isg, T (&Sc)[15]) {
  constexpr int DM = NM == 15 ? 4 : NM == 6 ? 2 : 0;   // total degree of the moments
  T a[15];
#pragma unroll
  for (int j = 0; j < 15; ++j) a[j] = (j < NM) ? S[j] : tc_<T>(0.f);
#pragma unroll
  for (int ey = 0; ey <= DM; ++ey)
#pragma unroll
    for (int i = 1; i <= DM - ey; ++i)
#pragma unroll
      for (int k = DM - ey; k >= i; --k) a[mono_index(k, ey)] -= cx * a[mono_index(k - 1, ey)];
#pragma unroll
  for (int ex = 0; ex <= DM; ++ex)
#pragma unroll
    for (int i = 1; i <= DM - ex; ++i)
#pragma unroll
      for (int k = DM - ex; k >= i; --k) a[mono_index(ex, k)] -= cy * a[mono_index(ex, k - 1)];
  T ps[5];
  ps[0] = tc_<T>(1.f);
#pragma unroll
  for (int e = 1; e < 5; ++e) ps[e] = ps[e - 1] * isg;
#pragma unroll
  for (int j = 0; j < 15; ++j) Sc[j] = (j < NM) ? a[j] * ps[mono_ex(j) + mono_ey(j)] : tc_<T>(0.f);
}

// z = M_c^-1 b_c(pixel) in the frame of the weighted centroid (degree of K
// terms); fr receives that frame as pass 2 applies it (centre hi, lo in x
// and y; 1/sigma).  Returns false when the centroid frame is degenerate or
// still ill conditioned.
template <int K, typename T>
__device__ bool centroid_solve(const T (&Sd)[15], T (&z)[6], float (&fr)[5]) {
  constexpr int DEGK = K == 6 ? 2 : 1;
  const T i0 = trcp(Sd[0]);
  const T cx0 = Sd[1] * i0, cy0 = Sd[2] * i0;
  const T var = (Sd[3] + Sd[5]) * i0 - cx0 * cx0 - cy0 * cy0;
  if (!(var > tc_<T>(0.f))) return false;
  tsplit(cx0, fr[0], fr[1]);
  tsplit(cy0, fr[2], fr[3]);
  float isg_lo;
  tsplit(trsqrt(var), fr[4], isg_lo);
  T cx, cy;
  tjoin(fr[0], fr[1], cx);
  tjoin(fr[2], fr[3], cy);
  const T isg = tc_<T>(fr[4]);
  T Sc[15];
  centroid_moments<n_moments(DEGK), T>(Sd, cx, cy, isg, Sc);
  T L[6][6], dinv[6], sd[6];
  const T rcc = ldl_rcond<K>(Sc, L, dinv, sd);
  T rmin;
  tfrom(1.0 / kKappaCentroid, rmin);
  if (!(rcc > rmin)) return false;
  const T ex = -(cx * isg), ey = -(cy * isg);
  T b[6] = {tc_<T>(1.f), ex, ey, ex * ex, ex * ey, ey * ey};
  ldl_solve<K>(L, dinv, sd, b);
#pragma unroll
  for (int a = 0; a < 6; ++a) z[a] = (a < K) ? b[a] : tc_<T>(0.f);
  return true;
}

// Degree policy on the pixel-frame moments (support count, then rcond_1 of
// the equilibrated matrix against rcond_min, highest degree first), then z.
// Returns the degree used (-1: no degree qualifies); *bad is set when the
// pixel needs the FP64 kernel.
template <int DEG, typename T>
__device__ int pixel_policy(const T (&Sd)[15], long long count, T rcond_min, T (&z)[6], float (&fr)[5], bool *bad) {
  T L[6][6], dinv[6], sd[6];
  int used = -1;
  if (DEG >= 2 && count >= 6 && ldl_rcond<6>(Sd, L, dinv, sd) >= rcond_min) used = 2;
  else if (DEG >= 1 && count >= 3 && ldl_rcond<3>(Sd, L, dinv, sd) >= rcond_min) used = 1;
  else if (count >= 1 && Sd[0] > tc_<T>(0.f)) used = 0;
  for (int a = 0; a < 6; ++a) z[a] = tc_<T>(0.f);
  fr[0] = fr[1] = fr[2] = fr[3] = 0.f;
  fr[4] = 1.f;
  *bad = false;
  if (used == 0) z[0] = trcp(Sd[0]);
  else if (used == 1) *bad = !centroid_solve<3, T>(Sd, z, fr);
  else if (used == 2) *bad = !centroid_solve<6, T>(Sd, z, fr);
  return used;
}

// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// The phases of one listed pixel, shared by the split kernels and the fused
// kernel below.

// Everything the moment and value phases need about pixel `id`: its
// candidate cells, stabiliser and scaled position (hi + lo).  FP64 and
// warp-uniform per pixel: run it one lane per pixel.
template <int WK>
__device__ void pixel_setup(const KParams &p, int id, Ranges &R, float &mhat, float &pxh, float &pxl, float &pyh,
                            float &pyl) {
  const int u = id % p.W, v = id / p.W;
  const double px = __dadd_rn(p.x0, __dmul_rn(__dadd_rn((double)u, 0.5), p.sx));
  const double py = __dadd_rn(p.y0, __dmul_rn(__dadd_rn((double)v, 0.5), p.sy));
  mhat = (WK == MLS_W_WENDLAND) ? 0.f : p.mstab[pix_i(p, (int64_t)v * (p.tiles_x * 16) + u)];
  if (WK == MLS_W_INVDIST) {
    R.all_n = (int)p.n;
    R.cx0 = R.cx1 = R.cy0 = R.cy1 = 0;
  } else {
    // near radius: the support (Wendland), the box (truncated Gaussian), or
    // r^2 <= m + kCut (Gaussian), widened by a relative 1e-5 against rounding
    const double rad = (WK == MLS_W_WENDLAND ? 1.0
                        : p.trunc > 0.0      ? p.trunc
                                             : (double)sqrtf(fmaxf(mhat, 0.f) + kCut)) *
                       p.h * (1.0 + 1e-5);
    const double inv_cell = p.inv_cell;
    R.all_n = 0;
    R.cx0 = max((int)floor((px - rad - p.gx0) * inv_cell), 0);
    R.cx1 = min((int)floor((px + rad - p.gx0) * inv_cell), p.gx - 1);
    R.cy0 = max((int)floor((py - rad - p.gy0) * inv_cell), 0);
    R.cy1 = min((int)floor((py + rad - p.gy0) * inv_cell), p.gy - 1);
  }
  // pixel position in the scaled frame as hi + lo
  const double inv_s = 1.0 / p.h;
  const double pxs64 = (px - p.ctr_x) * inv_s, pys64 = (py - p.ctr_y) * inv_s;
  pxh = (float)pxs64;
  pxl = (float)(pxs64 - (double)pxh);
  pyh = (float)pys64;
  pyl = (float)(pys64 - (double)pyh);
}

// Double-float pixel-frame moments of one pixel, a warp per pixel.  store(k,
// t) is called on every lane with the warp's total t of moment k < NM.
// Returns the near points; *coincident as for_near.
template <int DEG, int WK, typename Store>
__device__ __forceinline__ int pixel_moments(const KParams &p, const Ranges &R, float mhat, float pxh, float pxl,
                                             float pyh, float pyl, int lane, int *ri, float4 *rx,
                                             const float2 *s_tab, int *coincident, Store store) {
  constexpr int NM = n_moments(DEG);
  df32 S[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) S[k] = {0.f, 0.f};
  const int nnear = for_near<WK>(p, R, pxh, pxl, pyh, pyl, mhat, lane, ri, rx, coincident,
                                 [&](bool valid, int, df32 ex, df32 ey) {
    if (!valid) return;
    const df32 w = pair_wdf<WK>(ex, ey, mhat, p.alpha, s_tab);
    df_acc(S[0], w);
    if (NM > 1) {
      const df32 wx = df_prod(w, ex), wy = df_prod(w, ey);
      const df32 wxx = df_prod(wx, ex), wxy = df_prod(wx, ey), wyy = df_prod(wy, ey);
      df_acc(S[1], wx);
      df_acc(S[2], wy);
      df_acc(S[3], wxx);
      df_acc(S[4], wxy);
      df_acc(S[5], wyy);
      if (NM > 6) {
        const df32 wxxx = df_prod(wxx, ex), wxxy = df_prod(wxx, ey);
        const df32 wxyy = df_prod(wyy, ex), wyyy = df_prod(wyy, ey);
        df_acc(S[6], wxxx);
        df_acc(S[7], wxxy);
        df_acc(S[8], wxyy);
        df_acc(S[9], wyyy);
        df_acc(S[10], df_prod(wxxx, ex));
        df_acc(S[11], df_prod(wxxx, ey));
        df_acc(S[12], df_prod(wxxy, ey));
        df_acc(S[13], df_prod(wxyy, ey));
        df_acc(S[14], df_prod(wyyy, ey));
      }
    }
  });
#pragma unroll
  for (int k = 0; k < NM; ++k) store(k, df_warp_sum(S[k]));
  return nnear;
}

// Field values (and bands, status) of one pixel whose policy chose degree
// `used` >= 0, a warp per pixel: value_d = sum_i phi_i f_id with the shape
// functions phi_i = w_i z . b_c(x_i) in the centroid frame fr (centre hi,
// lo in x and y; 1/sigma), z as double-float.
template <int DEG, int WK>
__device__ __forceinline__ void pixel_values(const KParams &p, int id, int used, const Ranges &R, float mhat,
                                             float pxh, float pxl, float pyh, float pyl, const df32 (&zd)[6],
                                             const float (&fr)[5], int lane, int *ri, float4 *rx,
                                             const float2 *s_tab) {
  const size_t plane = (size_t)p.W * p.H;
  float *field = (float *)p.field;
  const int ku = n_terms(used);
  const float cxh = fr[0], cxl = fr[1], cyh = fr[2], cyl = fr[3], isg = fr[4];
  for (int d0 = 0; d0 < p.D; d0 += 32 * kDL) {
    df32 acc[kDL];
#pragma unroll
    for (int t = 0; t < kDL; ++t) acc[t] = {0.f, 0.f};
    int unused;
    for_near<WK>(p, R, pxh, pxl, pyh, pyl, mhat, lane, ri, rx, &unused, [&](bool valid, int i, df32 ex, df32 ey) {
      df32 phi = {0.f, 0.f};
      if (valid) {
        const df32 w = pair_wdf<WK>(ex, ey, mhat, p.alpha, s_tab);
        df32 zb = zd[0];
        if (ku > 1) {
          const df32 cxe = df_mul_f(df_diff(ex.hi, ex.lo, cxh, cxl), isg);
          const df32 cye = df_mul_f(df_diff(ey.hi, ey.lo, cyh, cyl), isg);
          zb = df_add(zb, df_add(df_mul(zd[1], cxe), df_mul(zd[2], cye)));
          if (ku > 3) {
            const df32 t = df_add(df_mul(zd[3], cxe), df_mul(zd[4], cye));
            zb = df_add(zb, df_add(df_mul(t, cxe), df_mul(df_mul(zd[5], cye), cye)));
          }
        }
        phi = df_mul(w, zb);
      }
      const int nb = __popc(__ballot_sync(0xffffffffu, valid));
#pragma unroll 4
      for (int jj = 0; jj < nb; ++jj) {
        const df32 ph = {__shfl_sync(0xffffffffu, phi.hi, jj), __shfl_sync(0xffffffffu, phi.lo, jj)};
        const int ij = __shfl_sync(0xffffffffu, i, jj);
        const float *fp = p.FR32 + (size_t)ij * p.D + d0 + lane;
#pragma unroll
        for (int t = 0; t < kDL; ++t)
          if (d0 + lane + 32 * t < p.D) df_acc(acc[t], df_prod_f(ph, fp[32 * t]));
      }
    });
#pragma unroll
    for (int t = 0; t < kDL; ++t) {
      const int d = d0 + lane + 32 * t;
      if (d < p.D) {
        // fcen + fscl (hi + lo) in double-float, rounded to float at the
        // end (FP32 arithmetic: per-lane FP64 here cost a warp
        // instruction per pixel and dimension sweep)
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

// A pixel without a qualifying degree (no support): NaN and band 255.
__device__ __forceinline__ void pixel_nosupport(const KParams &p, int id, int lane) {
  const size_t plane = (size_t)p.W * p.H;
  float *field = (float *)p.field;
  for (int d = lane; d < p.D; d += 32) {
    field[(size_t)d * plane + id] = __int_as_float(0x7fc00000);
    if (p.bands) p.bands[(size_t)d * plane + id] = 255;
  }
  if (lane == 0 && p.status) p.status[id] = MLS_ST_NO_SUPPORT | MLS_ST_RECOMPUTED;
}

// Policy of one pixel (lane per pixel) from its double-float moments, in
// scalar type T: degree used (-1: none) in bits 8.., bit 0 when the pixel
// needs the FP64 kernel; z as double-float pairs and the centroid frame.
template <int DEG, typename T>
__device__ __forceinline__ int pixel_decide(const float *Sh, const float *Sl, long long count, double rcond_min,
                                            float (&zh)[6], float (&zl)[6], float (&fr)[5]) {
  T Sd[15], z[6], rmin;
#pragma unroll
  for (int k = 0; k < 15; ++k) tjoin(Sh[k], Sl[k], Sd[k]);
  tfrom(rcond_min, rmin);
  bool bad = false;
  const int used = pixel_policy<DEG, T>(Sd, count, rmin, z, fr, &bad);
#pragma unroll
  for (int a = 0; a < 6; ++a) tsplit(z[a], zh[a], zl[a]);
  return (bad ? 1 : 0) | ((used + 1) << 8);
}

// ---------------------------------------------------------------------------
// Split hand-over: the list's first entries (up to the state capacity) in
// four kernels, so that the warp-per-pixel phases run at the occupancy
// their registers allow and wait on no block barrier, and the FP64 phases
// run one lane per pixel over full warps:
//   k_ho_setup    lane per entry: the pixel's setup
//   k_ho_moments  warp per entry (claimed from a counter): moments
//   k_ho_policy   lane per entry: FP64 degree policy and centroid solve
//   k_ho_values   warp per entry: values, bands, status; FP64-tier list
// The entries' state lives in global memory between the kernels.

// State of one list entry between the split kernels (48 words).  The
// moments (S, hi and lo interleaved) are replaced by the solution (zh[6],
// zl[6], fr[5]) once the policy has read them.
struct HoEntry {
  float S[30];
  int count, nnear, flags, id;
  int cx0, cx1, cy0, cy1;
  float mhat, pxh, pxl, pyh, pyl;
  int pad[5];
};
static_assert(sizeof(HoEntry) == 192, "hand-over entry layout");

// Entries the split kernels take: the list's first min(count, cap), when the
// list holds at least `least` entries (shorter lists go to the fused kernel
// whole: a block per chunk of them, with its FP64 policy overlapping the
// other blocks' double-float phases, is faster there than four launches
// with a policy kernel that occupies few warps).
__device__ __forceinline__ int64_t split_count(const unsigned int *list_count, int64_t cap, int64_t least) {
  const int64_t n = (int64_t)*list_count;
  if (n < least) return 0;
  return n < cap ? n : cap;
}

template <int WK>
__global__ __launch_bounds__(128) void k_ho_setup(KParams p, const int *list, const unsigned int *list_count,
                                                  int64_t cap, int64_t least, HoEntry *E) {
  const int64_t n = split_count(list_count, cap, least);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    HoEntry &e = E[k];
    const int id = (int)list_i(p, list[list_i(p, k)]);
    Ranges R;
    float mhat, pxh, pxl, pyh, pyl;
    pixel_setup<WK>(p, id, R, mhat, pxh, pxl, pyh, pyl);
    e.id = id;
    e.cx0 = R.cx0;
    e.cx1 = R.cx1;
    e.cy0 = R.cy0;
    e.cy1 = R.cy1;
    e.mhat = mhat;
    e.pxh = pxh;
    e.pxl = pxl;
    e.pyh = pyh;
    e.pyl = pyl;
  }
}

__device__ __forceinline__ Ranges entry_ranges(const KParams &p, const HoEntry &e, int wk) {
  Ranges R;
  R.cx0 = e.cx0;
  R.cx1 = e.cx1;
  R.cy0 = e.cy0;
  R.cy1 = e.cy1;
  R.all_n = (wk == MLS_W_INVDIST) ? (int)p.n : 0;
  return R;
}

// warps take entries one at a time from *claim
__device__ __forceinline__ int64_t claim_next(unsigned int *claim, int lane) {
  unsigned int k = 0;
  if (lane == 0) k = atomicAdd(claim, 1u);
  return (int64_t)__shfl_sync(0xffffffffu, k, 0);
}

template <int DEG, int WK>
__global__ __launch_bounds__(kWarps * 32, 8) void k_ho_moments(KParams p, const unsigned int *list_count,
                                                               int64_t cap, int64_t least, HoEntry *E,
                                                               unsigned int *claim) {
  __shared__ int s_ri[kWarps][kRing];
  __shared__ float4 s_rx[kWarps][kRing];
  __shared__ float2 s_tab[64];
  const int64_t n = split_count(list_count, cap, least);
  if (n == 0) return;   // uniform over the grid: a short list goes to the fused kernel
  if (WK == MLS_W_GAUSS) df_exp_table_init(s_tab);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int64_t k = claim_next(claim, lane); k < n; k = claim_next(claim, lane)) {
    HoEntry &e = E[k];
    const Ranges R = entry_ranges(p, e, WK);
    int coincident = 0;
    const float mhat = e.mhat;
    const int nnear = pixel_moments<DEG, WK>(p, R, mhat, e.pxh, e.pxl, e.pyh, e.pyl, lane, s_ri[wib], s_rx[wib], s_tab,
                                             &coincident, [&](int q, df32 t) {
      if (lane == q) {
        e.S[2 * q] = t.hi;
        e.S[2 * q + 1] = t.lo;
      }
    });
    if (lane == 0) {
      e.count = (WK == MLS_W_WENDLAND || p.trunc > 0.0) ? nnear : (int)(p.n < (1 << 30) ? p.n : (1 << 30));
      e.nnear = nnear;
      // inverse distance: a coincident point (or a zero stabiliser) goes to
      // the FP64 kernel, which gives the pixel that point's value
      e.flags = (WK == MLS_W_INVDIST && (coincident || !(mhat > 0.f))) ? 1 : 0;
    }
  }
}

// The policy is a long chain of dependent double-float operations per lane:
// a short list is spread over more warps (fewer lanes each, down to 4) so
// that the warp schedulers have other warps to issue while one waits.
template <int DEG>
__global__ __launch_bounds__(32) void k_ho_policy(KParams p, const unsigned int *list_count, int64_t cap,
                                                   int64_t least, HoEntry *E) {
  constexpr int NM = n_moments(DEG);
  const int64_t n = split_count(list_count, cap, least);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  int lpw = 32;
  while (lpw > 4 && (n + lpw - 1) / lpw < nw) lpw >>= 1;
  for (int64_t base = gw * lpw; base < n; base += nw * lpw) {
    const int64_t k = base + lane;
    if (lane >= lpw || k >= n) continue;
    HoEntry &e = E[k];
    if (e.flags & 1) continue;
    float Sh[15], Sl[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) {
      Sh[q] = q < NM ? e.S[2 * q] : 0.f;
      Sl[q] = q < NM ? e.S[2 * q + 1] : 0.f;
    }
    float zh[6], zl[6], fr[5];
    const int flags = pixel_decide<DEG, dd>(Sh, Sl, e.count, p.rcond_min, zh, zl, fr);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      e.S[a] = zh[a];
      e.S[6 + a] = zl[a];
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) e.S[12 + a] = fr[a];
    e.flags = flags;
  }
}

template <int DEG, int WK>
__global__ __launch_bounds__(kWarps * 32, 8) void k_ho_values(KParams p, const unsigned int *list_count,
                                                              int64_t cap, int64_t least, HoEntry *E,
                                                              unsigned int *claim, int *list2,
                                                              unsigned int *list2_count) {
  __shared__ int s_ri[kWarps][kRing];
  __shared__ float4 s_rx[kWarps][kRing];
  __shared__ float2 s_tab[64];
  const int64_t n = split_count(list_count, cap, least);
  if (n == 0) return;   // uniform over the grid: a short list goes to the fused kernel
  if (WK == MLS_W_GAUSS) df_exp_table_init(s_tab);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int64_t k = claim_next(claim, lane); k < n; k = claim_next(claim, lane)) {
    const HoEntry &e = E[k];
    const int id = e.id, flags = e.flags;
    if (flags & 1) {
      if (lane == 0) {
        const unsigned int k2 = atomicAdd(list2_count, 1u);
        list2[list_i(p, k2)] = id;
      }
      continue;
    }
    const int used = (flags >> 8) - 1;
    if (used < 0) {
      pixel_nosupport(p, id, lane);
      continue;
    }
    df32 zd[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) zd[a] = {e.S[a], e.S[6 + a]};
    float fr[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) fr[a] = e.S[12 + a];
    pixel_values<DEG, WK>(p, id, used, entry_ranges(p, e, WK), e.mhat, e.pxh, e.pxl, e.pyh, e.pyl, zd, fr, lane,
                          s_ri[wib], s_rx[wib], s_tab);
  }
}

// ---------------------------------------------------------------------------
// Fused hand-over of the list entries from `first` on (those past the split
// kernels' state capacity): one block per chunk of up to 32 pixels, its
// phases separated by block barriers with the chunk's state in shared memory.

// Per-block state of a chunk of up to 32 pixels between its phases.
struct ChunkSlot {
  float zh[6], zl[6];     // solution in the centroid frame, double-float
  float Sh[15], Sl[15];   // pixel-frame moments, double-float
  float fr[5];     // centroid frame
  long long count;
  int flags;       // bit 0: needs the FP64 kernel; bits 8..: degree used + 1
  int nnear;       // near points (the cost of the pixel's value phase)
  // the pixel's setup (formed once per chunk, one lane per pixel)
  int id;
  Ranges R;
  float mhat, pxh, pxl, pyh, pyl;
};

template <int DEG, int WK>
__global__ __launch_bounds__(kWarps * 32, 4) void k_handover(KParams p, const int *list,
                                                          const unsigned int *list_count, int64_t split_cap,
                                                          int64_t least, int64_t cap, int *list2,
                                                          unsigned int *list2_count) {
  __shared__ int s_ri[kWarps][kRing];
  __shared__ float4 s_rx[kWarps][kRing];
  __shared__ ChunkSlot s_chunk[32];
  __shared__ float2 s_tab[64];
  // the chunk's pixels are claimed one at a time by the warps (counters of
  // the moment and value phases); the value phase takes them in decreasing
  // order of their near points (longest first), so the warps finish together
  __shared__ int s_next[2];
  __shared__ int s_order[32];
  const int64_t total = (int64_t)*list_count < cap ? (int64_t)*list_count : cap;
  const int64_t first = split_count(list_count, split_cap, least);   // taken by the split kernels
  const int64_t npix = total - first;
  if (npix <= 0) return;   // uniform over the grid: nothing past the split kernels
  list += first;
  if (WK == MLS_W_GAUSS) df_exp_table_init(s_tab);
  if (threadIdx.x == 0) s_next[0] = s_next[1] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the warp of the lane-per-pixel phases (setup, FP64 policy) rotates with
  // the block, so that the blocks sharing an SM run those phases on
  // different warp schedulers; the next warp forms the value-phase order
  const int wpol = (int)(blockIdx.x % kWarps), word = (wpol + 1) % kWarps;
  int *ri = s_ri[wib];
  float4 *rx = s_rx[wib];
  ChunkSlot *slots = s_chunk;
  // pixels per block chunk: up to 32 (one per lane of the policy warp), fewer
  // when there are too few pixels to give every block a full chunk.  The
  // block's warps share the moment and value phases (warp per pixel); one
  // warp runs the FP64 policy of all the chunk's pixels, one per lane (GB300's
  // FP64 pipe takes a warp instruction's full cost however few lanes are active)
  const int64_t per = (npix + gridDim.x - 1) / gridDim.x;
  const int csz = per >= 32 ? 32 : (per < 1 ? 1 : (int)per);
  const int64_t nchunks = (npix + csz - 1) / csz;

  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    // Neighbouring list entries are often neighbouring pixels of one tile,
    // with similar costs and shared near points.  With at most one chunk per
    // block, chunk ch takes every nchunks-th entry from ch on, which spreads
    // the expensive pixels (many near points) over the blocks.  With more
    // chunks than blocks, the blocks balance over their several chunks, and
    // a chunk takes a contiguous run, whose pixels share near points in cache.
    const bool strided = nchunks <= (int64_t)gridDim.x;
    const int64_t firstk = strided ? ch : ch * csz, step = strided ? nchunks : 1;
    const int nq = strided ? (int)((npix - ch + nchunks - 1) / nchunks)
                           : (int)((npix - firstk) < csz ? (npix - firstk) : csz);

    // ---- phase 0 (lane per pixel): each pixel's setup, once.  Its FP64
    // arithmetic is warp-uniform per pixel; GB300 charges an FP64 warp
    // instruction in full however few lanes need it, so 32 pixels a lane
    // each cost what one pixel on a whole warp did (twice, for the moment and
    // value phases)
    if (wib == wpol && lane < nq) {
      ChunkSlot &sl = slots[lane];
      const int id = (int)list_i(p, list[list_i(p, firstk + (int64_t)lane * step)]);
      sl.id = id;
      pixel_setup<WK>(p, id, sl.R, sl.mhat, sl.pxh, sl.pxl, sl.pyh, sl.pyl);
    }
    __syncthreads();

    // ---- phase 1 (warp per pixel): double-float pixel-frame moments
    for (;;) {
      int j = 0;
      if (lane == 0) j = atomicAdd(&s_next[0], 1);
      j = __shfl_sync(0xffffffffu, j, 0);
      if (j >= nq) break;
      ChunkSlot &sl = slots[j];
      int coincident = 0;
      const float mhat = sl.mhat;
      const int nnear = pixel_moments<DEG, WK>(p, sl.R, mhat, sl.pxh, sl.pxl, sl.pyh, sl.pyl, lane, ri, rx, s_tab,
                                               &coincident, [&](int q, df32 t) {
        if (lane == q) {
          sl.Sh[q] = t.hi;
          sl.Sl[q] = t.lo;
        }
      });
      if (lane < 15 && lane >= n_moments(DEG)) {
        sl.Sh[lane] = 0.f;
        sl.Sl[lane] = 0.f;
      }
      if (lane == 0) {
        sl.count = (WK == MLS_W_WENDLAND || p.trunc > 0.0) ? nnear : p.n;
        sl.nnear = nnear;
        // inverse distance: a coincident point (or a zero stabiliser) goes to
        // the FP64 kernel, which gives the pixel that point's value
        sl.flags = (WK == MLS_W_INVDIST && (coincident || !(mhat > 0.f))) ? 1 : 0;
      }
      __syncwarp();
    }

    __syncthreads();
    // ---- phase 2 (lane per pixel): degree policy and centroid-frame solve in FP64
    if (wib == word) {
      // value-phase order and counters; the moment counter is reset for the
      // next chunk (every warp has left this chunk's moment phase)
      if (lane < nq) {
        const int c = slots[lane].nnear;
        int rank = 0;
        for (int k = 0; k < nq; ++k) {
          const int ck = slots[k].nnear;
          rank += (ck > c || (ck == c && k < lane)) ? 1 : 0;
        }
        s_order[rank] = lane;
      }
      if (lane == 0) s_next[0] = s_next[1] = 0;
    }
    if (wib == wpol && lane < nq) {
      ChunkSlot &sl = slots[lane];
      if (!(sl.flags & 1)) sl.flags = pixel_decide<DEG, double>(sl.Sh, sl.Sl, sl.count, p.rcond_min, sl.zh, sl.zl, sl.fr);
    }
    __syncthreads();

    // ---- phase 3 (warp per pixel): value = sum_i phi_i f_i, phi_i = w_i z . b_c(x_i)
    for (;;) {
      int k = 0;
      if (lane == 0) k = atomicAdd(&s_next[1], 1);
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k >= nq) break;
      const int j = s_order[k];
      const int id = slots[j].id;
      const int flags = slots[j].flags;
      if (flags & 1) {
        if (lane == 0) {
          const unsigned int k2 = atomicAdd(list2_count, 1u);
          list2[list_i(p, k2)] = id;
        }
        continue;
      }
      const int used = (flags >> 8) - 1;
      if (used < 0) {
        pixel_nosupport(p, id, lane);
        continue;
      }
      df32 zd[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) zd[a] = {slots[j].zh[a], slots[j].zl[a]};
      float fr[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) fr[a] = slots[j].fr[a];
      pixel_values<DEG, WK>(p, id, used, slots[j].R, slots[j].mhat, slots[j].pxh, slots[j].pxl, slots[j].pyh,
                            slots[j].pyl, zd, fr, lane, ri, rx, s_tab);
    }
    __syncthreads();   // the slots are refilled by the next chunk
  }
}

template <int DEG, int WK>
int launch_dw(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int64_t split_cap,
              int64_t least, void *state, unsigned int *claims, int *list2, unsigned int *cnt2, cudaStream_t st) {
  const int64_t sc = state ? (split_cap < cap ? split_cap : cap) : 0;
  int launches = 1;
  if (sc > 0) {
    launches += 4;
    HoEntry *E = (HoEntry *)state;
    // one resident wave each: 4 blocks of 128 threads per SM for the setup,
    // 8 for the warp phases (entries claimed dynamically), 16 one-warp
    // blocks for the policy
    k_ho_setup<WK><<<152 * 4, 128, 0, st>>>(p, list, cnt, sc, least, E);
    k_ho_moments<DEG, WK><<<152 * 8, kWarps * 32, 0, st>>>(p, cnt, sc, least, E, claims);
    k_ho_policy<DEG><<<152 * 16, 32, 0, st>>>(p, cnt, sc, least, E);
    k_ho_values<DEG, WK><<<152 * 8, kWarps * 32, 0, st>>>(p, cnt, sc, least, E, claims + 1, list2, cnt2);
  }
  // lists shorter than `least`, and entries past the split kernels'
  // capacity (one resident wave: 4 blocks of 4 warps per SM; every block
  // returns at once when there are none)
  k_handover<DEG, WK><<<152 * 4, kWarps * 32, 0, st>>>(p, list, cnt, sc, least, cap, list2, cnt2);
  return launches;
}

template <int WK>
int launch_w(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int64_t split_cap,
             int64_t least, void *state, unsigned int *claims, int *list2, unsigned int *cnt2, cudaStream_t st) {
  if (p.degree == 0) return launch_dw<0, WK>(p, list, cnt, cap, split_cap, least, state, claims, list2, cnt2, st);
  if (p.degree == 1) return launch_dw<1, WK>(p, list, cnt, cap, split_cap, least, state, claims, list2, cnt2, st);
  return launch_dw<2, WK>(p, list, cnt, cap, split_cap, least, state, claims, list2, cnt2, st);
}

}  // namespace

size_t handover_entry_bytes() { return sizeof(HoEntry); }

int launch_handover(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int64_t split_cap,
                    int64_t least, void *state, unsigned int *claims, int *list2, unsigned int *cnt2,
                    cudaStream_t st) {
  if (p.weight == MLS_W_GAUSS)
    return launch_w<MLS_W_GAUSS>(p, list, cnt, cap, split_cap, least, state, claims, list2, cnt2, st);
  if (p.weight == MLS_W_WENDLAND)
    return launch_w<MLS_W_WENDLAND>(p, list, cnt, cap, split_cap, least, state, claims, list2, cnt2, st);
  return launch_w<MLS_W_INVDIST>(p, list, cnt, cap, split_cap, least, state, claims, list2, cnt2, st);
}

// Test hook: the double-float weight functions on given arguments.
__global__ void k_debug_df_weight(int kind, const float *ahi, const float *alo, int64_t n, double *out) {
  __shared__ float2 tab[64];
  mlsk::df_exp_table_init(tab);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const mlsk::df32 a = {ahi[i], alo[i]};
    const mlsk::df32 w = kind == 0 ? mlsk::df_exp(a, tab) : kind == 1 ? mlsk::df_wendland(a) : mlsk::df_sqrt(a);
    out[i] = (double)w.hi + (double)w.lo;
  }
}

}  // namespace mlsi

extern "C" int mls_debug_df_weight(int kind, const float *arg_hi, const float *arg_lo, int64_t n, double *out) {
  if (kind < 0 || kind > 2 || n < 0 || (n > 0 && (!arg_hi || !arg_lo || !out))) return MLS_E_INVAL;
  if (n == 0) return MLS_OK;
  float *d = nullptr;
  double *o = nullptr;
  if (cudaMalloc(&d, sizeof(float) * 2 * n) != cudaSuccess) return MLS_E_NOMEM;
  if (cudaMalloc(&o, sizeof(double) * n) != cudaSuccess) {
    cudaFree(d);
    return MLS_E_NOMEM;
  }
  cudaError_t e = cudaMemcpy(d, arg_hi, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + n, arg_lo, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    mlsi::k_debug_df_weight<<<152, 256>>>(kind, d, d + n, n, o);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, o, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(o);
  return e == cudaSuccess ? MLS_OK : MLS_E_CUDA;
}
