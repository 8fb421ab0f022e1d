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
// normalised warp-wide sum
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
// largest, or for the truncated Gaussian (cbox = c > 0) inside the box
// |dx|, |dy| < c, every point of which counts (double-float offsets); inside
// the Wendland support (double-float distance); any point but a coincident
// one for inverse distance.
template <int WK>
__device__ __forceinline__ bool near_test(df32 ex, df32 ey, float mhat, double cbox) {
  if (WK == MLS_W_GAUSS && cbox > 0.0)
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
        nr = near_test<WK>(ex, ey, mhat, p.trunc);
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
// FP64 degree policy and centroid-frame solve, one lane per pixel (GB300's
// FP64 units are few: running the policy once per lane for 32 pixels instead
// of redundantly on every lane of a warp cuts its FP64 instructions 32-fold).

// 1/d for a positive normal d: FP32 seed and two Newton steps (each doubles
// the number of correct bits: 2^-23 -> 2^-46 -> FP64 rounding).
__device__ __forceinline__ double rcp64(double d) {
  double r = (double)__frcp_rn((float)d);
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}

// Equilibrated LDL^T factorisation of the K x K moment matrix S[midx(a, b)]
// and rcond_1 = 1 / (|Me|_1 |Me^-1|_1) of the equilibrated matrix Me.
// Returns 0 when a diagonal entry or a pivot is not positive.  L (unit
// lower), dinv (inverse pivots) and sd (equilibration 1/sqrt(M_aa)) receive
// the factorisation.
template <int K>
__device__ double ldl_rcond(const double (&S)[15], double (&L)[6][6], double (&dinv)[6], double (&sd)[6]) {
  double Me[K][K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    const double d = S[midx(a, a)];
    if (!(d > 0.0)) return 0.0;
    sd[a] = rsqrt(d);
  }
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) Me[a][b] = Me[b][a] = S[midx(a, b)] * sd[a] * sd[b];
  // LDL^T (no square roots): D_j = Me_jj - sum_t L_jt (L_jt D_t),
  // L_ij = (Me_ij - sum_t L_it (L_jt D_t)) / D_j, with LD_jt = L_jt D_t kept
  // (it is the numerator of L_jt before the division)
  double LD[K][K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double dj = Me[j][j];
#pragma unroll
    for (int t = 0; t < j; ++t) dj -= L[j][t] * LD[j][t];
    if (!(dj > 0.0)) return 0.0;
    dinv[j] = rcp64(dj);
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      double v = Me[i][j];
#pragma unroll
      for (int t = 0; t < j; ++t) v -= L[i][t] * LD[j][t];
      LD[i][j] = v;
      L[i][j] = v * dinv[j];
    }
  }
  // 1-norms of Me and of its inverse.  Me^-1 = L^-T D^-1 L^-1 is symmetric:
  // with Li = L^-1 (unit lower) and G_kj = dinv_k Li_kj, its entry (i, j),
  // i <= j, is sum_{k >= j} Li_ki G_kj (about a third of the FP64 operations
  // of K forward and back substitutions)
  double Li[K][K], G[K][K];
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      double v = -L[i][j];
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
  double cI[K], cA[K];
#pragma unroll
  for (int c = 0; c < K; ++c) cI[c] = cA[c] = 0.0;
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int i = 0; i <= j; ++i) {
      double v = 0.0;
#pragma unroll
      for (int k = j; k < K; ++k) v += (k == i ? 1.0 : Li[k][i]) * G[k][j];
      const double av = fabs(v), am = fabs(Me[i][j]);
      cI[j] += av;
      cA[j] += am;
      if (i != j) {
        cI[i] += av;
        cA[i] += am;
      }
    }
  double nI = 0.0, nA = 0.0;
#pragma unroll
  for (int c = 0; c < K; ++c) {
    nI = fmax(nI, cI[c]);
    nA = fmax(nA, cA[c]);
  }
  return 1.0 / (nA * nI);
}

// b <- M^-1 b with M = S^-1 Me S^-1 factorised as above: S Me^-1 S b.
template <int K>
__device__ __forceinline__ void ldl_solve(const double (&L)[6][6], const double (&dinv)[6], const double (&sd)[6],
                                          double (&b)[6]) {
#pragma unroll
  for (int a = 0; a < K; ++a) b[a] *= sd[a];
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int t = 0; t < i; ++t) b[i] -= L[i][t] * b[t];
#pragma unroll
  for (int i = 0; i < K; ++i) b[i] *= dinv[i];
#pragma unroll
  for (int i = K - 1; i >= 0; --i)
#pragma unroll
    for (int t = i + 1; t < K; ++t) b[i] -= L[t][i] * b[t];
#pragma unroll
  for (int a = 0; a < K; ++a) b[a] *= sd[a];
}

// Moments of the frame centred on (cx, cy) and scaled by isg, from the
// pixel-frame moments: sum_i w_i (x_i - cx)^bx (y_i - cy)^by, by binomial
// expansion.  The expansion is separable: a shift in x of every row of equal
// y exponent, then a shift in y of every column.  A 1-D shift of moments
// a_0..a_m by c is the Taylor shift: m passes, pass i replacing a_k by
// a_k - c a_(k-1) for k = m down to i (m (m + 1) / 2 multiply-adds).
template <int NM>
__device__ __forceinline__ void centroid_moments(const double (&S)[15], double cx, double cy, double isg,
                                                 double (&Sc)[15]) {
  constexpr int DM = NM == 15 ? 4 : NM == 6 ? 2 : 0;   // total degree of the moments
  double a[15];
#pragma unroll
  for (int j = 0; j < 15; ++j) a[j] = (j < NM) ? S[j] : 0.0;
#pragma unroll
  for (int ey = 0; ey <= DM; ++ey)
#pragma unroll
    for (int i = 1; i <= DM - ey; ++i)
#pragma unroll
      for (int k = DM - ey; k >= i; --k) a[mono_index(k, ey)] = fma(-cx, a[mono_index(k - 1, ey)], a[mono_index(k, ey)]);
#pragma unroll
  for (int ex = 0; ex <= DM; ++ex)
#pragma unroll
    for (int i = 1; i <= DM - ex; ++i)
#pragma unroll
      for (int k = DM - ex; k >= i; --k) a[mono_index(ex, k)] = fma(-cy, a[mono_index(ex, k - 1)], a[mono_index(ex, k)]);
  double ps[5];
  ps[0] = 1.0;
#pragma unroll
  for (int e = 1; e < 5; ++e) ps[e] = ps[e - 1] * isg;
#pragma unroll
  for (int j = 0; j < 15; ++j) Sc[j] = (j < NM) ? a[j] * ps[mono_ex(j) + mono_ey(j)] : 0.0;
}

// z = M_c^-1 b_c(pixel) in the frame of the weighted centroid (degree of K
// terms); fr receives that frame as pass 2 applies it (centre hi, lo in x
// and y; 1/sigma).  Returns false when the centroid frame is degenerate or
// still ill conditioned.
template <int K>
__device__ bool centroid_solve(const double (&Sd)[15], double (&z)[6], float (&fr)[5]) {
  constexpr int DEGK = K == 6 ? 2 : 1;
  const double cx0 = Sd[1] / Sd[0], cy0 = Sd[2] / Sd[0];
  const double var = (Sd[3] + Sd[5]) / Sd[0] - cx0 * cx0 - cy0 * cy0;
  if (!(var > 0.0)) return false;
  fr[0] = (float)cx0;
  fr[1] = (float)(cx0 - (double)fr[0]);
  fr[2] = (float)cy0;
  fr[3] = (float)(cy0 - (double)fr[2]);
  fr[4] = (float)rsqrt(var);
  const double cx = (double)fr[0] + (double)fr[1], cy = (double)fr[2] + (double)fr[3];
  const double isg = (double)fr[4];
  double Sc[15];
  centroid_moments<n_moments(DEGK)>(Sd, cx, cy, isg, Sc);
  double L[6][6], dinv[6], sd[6];
  const double rcc = ldl_rcond<K>(Sc, L, dinv, sd);
  if (!(rcc > 1.0 / kKappaCentroid)) return false;
  const double ex = -cx * isg, ey = -cy * isg;
  double b[6] = {1.0, ex, ey, ex * ex, ex * ey, ey * ey};
  ldl_solve<K>(L, dinv, sd, b);
#pragma unroll
  for (int a = 0; a < 6; ++a) z[a] = (a < K) ? b[a] : 0.0;
  return true;
}

// Degree policy on the pixel-frame moments (support count, then rcond_1 of
// the equilibrated matrix against rcond_min, highest degree first), then z.
// Returns the degree used (-1: no degree qualifies); *bad is set when the
// pixel needs the FP64 kernel.
template <int DEG>
__device__ int pixel_policy(const double (&Sd)[15], long long count, double rcond_min, double (&z)[6],
                            float (&fr)[5], bool *bad) {
  double L[6][6], dinv[6], sd[6];
  int used = -1;
  if (DEG >= 2 && count >= 6 && ldl_rcond<6>(Sd, L, dinv, sd) >= rcond_min) used = 2;
  else if (DEG >= 1 && count >= 3 && ldl_rcond<3>(Sd, L, dinv, sd) >= rcond_min) used = 1;
  else if (count >= 1 && Sd[0] > 0.0) used = 0;
  for (int a = 0; a < 6; ++a) z[a] = 0.0;
  fr[0] = fr[1] = fr[2] = fr[3] = 0.f;
  fr[4] = 1.f;
  *bad = false;
  if (used == 0) z[0] = 1.0 / Sd[0];
  else if (used == 1) *bad = !centroid_solve<3>(Sd, z, fr);
  else if (used == 2) *bad = !centroid_solve<6>(Sd, z, fr);
  return used;
}

// ---------------------------------------------------------------------------

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
                                                          const unsigned int *list_count, int64_t cap, int *list2,
                                                          unsigned int *list2_count) {
  constexpr int NM = n_moments(DEG);
  __shared__ int s_ri[kWarps][kRing];
  __shared__ float4 s_rx[kWarps][kRing];
  __shared__ ChunkSlot s_chunk[32];
  __shared__ float2 s_tab[64];
  // the chunk's pixels are claimed one at a time by the warps (counters of
  // the moment and value phases); the value phase takes them in decreasing
  // order of their near points (longest first), so the warps finish together
  __shared__ int s_next[2];
  __shared__ int s_order[32];
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
  const int64_t npix = (int64_t)*list_count < cap ? (int64_t)*list_count : cap;
  // pixels per block chunk: up to 32 (one per lane of the policy warp), fewer
  // when there are too few pixels to give every block a full chunk.  The
  // block's warps share the moment and value phases (warp per pixel); one
  // warp runs the FP64 policy of all the chunk's pixels, one per lane (GB300's
  // FP64 pipe takes a warp instruction's full cost however few lanes are active)
  const int64_t per = (npix + gridDim.x - 1) / gridDim.x;
  const int csz = per >= 32 ? 32 : (per < 1 ? 1 : (int)per);
  const int64_t nchunks = (npix + csz - 1) / csz;
  const size_t plane = (size_t)p.W * p.H;
  const double inv_s = 1.0 / p.h;
  float *field = (float *)p.field;

  // everything pass 1 and pass 2 need about pixel `id`
  auto setup = [&](int id, Ranges &R, float &mhat, float &pxh, float &pxl, float &pyh, float &pyl) {
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
    const double pxs64 = (px - p.ctr_x) * inv_s, pys64 = (py - p.ctr_y) * inv_s;
    pxh = (float)pxs64;
    pxl = (float)(pxs64 - (double)pxh);
    pyh = (float)pys64;
    pyl = (float)(pys64 - (double)pyh);
  };

  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    // Neighbouring list entries are often neighbouring pixels of one tile,
    // with similar costs and shared near points.  With at most one chunk per
    // block, chunk ch takes every nchunks-th entry from ch on, which spreads
    // the expensive pixels (many near points) over the blocks.  With more
    // chunks than blocks, the blocks balance over their several chunks, and
    // a chunk takes a contiguous run, whose pixels share near points in cache.
    const bool strided = nchunks <= (int64_t)gridDim.x;
    const int64_t first = strided ? ch : ch * csz, step = strided ? nchunks : 1;
    const int nq = strided ? (int)((npix - ch + nchunks - 1) / nchunks)
                           : (int)((npix - first) < csz ? (npix - first) : csz);

    // ---- phase 0 (lane per pixel): each pixel's setup, once.  Its FP64
    // arithmetic is warp-uniform per pixel; GB300 charges an FP64 warp
    // instruction in full however few lanes need it, so 32 pixels a lane
    // each cost what one pixel on a whole warp did (twice, for the moment and
    // value phases)
    if (wib == wpol && lane < nq) {
      ChunkSlot &sl = slots[lane];
      const int id = (int)list_i(p, list[list_i(p, first + (int64_t)lane * step)]);
      sl.id = id;
      setup(id, sl.R, sl.mhat, sl.pxh, sl.pxl, sl.pyh, sl.pyl);
    }
    __syncthreads();

    // ---- phase 1 (warp per pixel): double-float pixel-frame moments
    for (;;) {
      int j = 0;
      if (lane == 0) j = atomicAdd(&s_next[0], 1);
      j = __shfl_sync(0xffffffffu, j, 0);
      if (j >= nq) break;
      const Ranges R = slots[j].R;
      const float mhat = slots[j].mhat, pxh = slots[j].pxh, pxl = slots[j].pxl, pyh = slots[j].pyh,
                  pyl = slots[j].pyl;
      df32 S[NM];
#pragma unroll
      for (int k = 0; k < NM; ++k) S[k] = {0.f, 0.f};
      int coincident = 0;
      const int nnear = for_near<WK>(p, R, pxh, pxl, pyh, pyl, mhat, lane, ri, rx, &coincident,
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
      // the sums as double-float (the policy lane forms the doubles)
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        df32 t = {0.f, 0.f};
        if (k < NM) t = df_warp_sum(S[k]);
        if (lane == k) {
          slots[j].Sh[k] = t.hi;
          slots[j].Sl[k] = t.lo;
        }
      }
      if (lane == 0) {
        slots[j].count = (WK == MLS_W_WENDLAND || p.trunc > 0.0) ? nnear : p.n;
        slots[j].nnear = nnear;
        // inverse distance: a coincident point (or a zero stabiliser) goes to
        // the FP64 kernel, which gives the pixel that point's value
        slots[j].flags = (WK == MLS_W_INVDIST && (coincident || !(mhat > 0.f))) ? 1 : 0;
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
      if (!(sl.flags & 1)) {
        double Sd[15], z[6];
        float fr[5];
#pragma unroll
        for (int k = 0; k < 15; ++k) Sd[k] = (double)sl.Sh[k] + (double)sl.Sl[k];
        bool bad = false;
        const int used = pixel_policy<DEG>(Sd, sl.count, p.rcond_min, z, fr, &bad);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          sl.zh[a] = (float)z[a];
          sl.zl[a] = (float)(z[a] - (double)sl.zh[a]);
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) sl.fr[a] = fr[a];
        sl.flags = (bad ? 1 : 0) | ((used + 1) << 8);
      }
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
        for (int d = lane; d < p.D; d += 32) {
          field[(size_t)d * plane + id] = __int_as_float(0x7fc00000);
          if (p.bands) p.bands[(size_t)d * plane + id] = 255;
        }
        if (lane == 0 && p.status) p.status[id] = MLS_ST_NO_SUPPORT | MLS_ST_RECOMPUTED;
        continue;
      }
      const Ranges R = slots[j].R;
      const float mhat = slots[j].mhat, pxh = slots[j].pxh, pxl = slots[j].pxl, pyh = slots[j].pyh,
                  pyl = slots[j].pyl;
      const int ku = n_terms(used);
      df32 zd[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        zd[a] = {slots[j].zh[a], slots[j].zl[a]};
      }
      const float cxh = slots[j].fr[0], cxl = slots[j].fr[1], cyh = slots[j].fr[2], cyl = slots[j].fr[3],
                  isg = slots[j].fr[4];
      for (int d0 = 0; d0 < p.D; d0 += 32 * kDL) {
        df32 acc[kDL];
#pragma unroll
        for (int t = 0; t < kDL; ++t) acc[t] = {0.f, 0.f};
        int unused;
        for_near<WK>(p, R, pxh, pxl, pyh, pyl, mhat, lane, ri, rx, &unused,
                     [&](bool valid, int i, df32 ex, df32 ey) {
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
    __syncthreads();   // the slots are refilled by the next chunk
  }
}

template <int WK>
void launch_w(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int *list2,
              unsigned int *cnt2, cudaStream_t st) {
  const int grid = 152 * 4;   // one resident wave (4 blocks of 4 warps per SM)
  if (p.degree == 0) k_handover<0, WK><<<grid, kWarps * 32, 0, st>>>(p, list, cnt, cap, list2, cnt2);
  else if (p.degree == 1) k_handover<1, WK><<<grid, kWarps * 32, 0, st>>>(p, list, cnt, cap, list2, cnt2);
  else k_handover<2, WK><<<grid, kWarps * 32, 0, st>>>(p, list, cnt, cap, list2, cnt2);
}

}  // namespace

void launch_handover(const KParams &p, const int *list, const unsigned int *cnt, int64_t cap, int *list2,
                     unsigned int *cnt2, cudaStream_t st) {
  if (p.weight == MLS_W_GAUSS) launch_w<MLS_W_GAUSS>(p, list, cnt, cap, list2, cnt2, st);
  else if (p.weight == MLS_W_WENDLAND) launch_w<MLS_W_WENDLAND>(p, list, cnt, cap, list2, cnt2, st);
  else launch_w<MLS_W_INVDIST>(p, list, cnt, cap, list2, cnt2, st);
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
