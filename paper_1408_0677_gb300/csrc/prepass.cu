// Per-pixel prepass over the padded 16 x 16 tile grid.
//
// Gaussian and inverse-distance weights: the stabiliser m(p) = min_i
// |x_i - p|^2 (in units of h^2).  Multiplying every weight of a pixel by the
// same positive factor leaves the fit unchanged, so the kernels use
// exp(-(r^2 - m)/h^2) and (m / r^2)^alpha, whose largest value is 1: no
// underflow of the reduced-precision weights.  The search is culled per tile:
// a bound B = min_i (largest squared distance from x_i to the tile's pixel
// centres) is found first; only points whose smallest squared distance to
// the tile is <= B can be nearest to one of its pixels.
//
// Wendland weight: the number of points within the support radius of each
// pixel, from the cells of the uniform grid that overlap the tile, with a
// flag (kCntBoundary) when a point lies so close to the support boundary that
// FP32 and FP64 could count it differently.
//
// Truncated Gaussian: the stabiliser as for the Gaussian, and the number of
// points in each pixel's box |dx|, |dy| < c (units of h), with the same flag
// for a point whose |dx| or |dy| lies within a relative kCntEdgeTol of c.
//
// Both also give each tile the frame its moments are accumulated in: the
// weighted centroid of the points around the tile centre (Gaussian weights of
// scale h, or the Wendland weights).  A pixel whose points lie to one side is
// badly conditioned in its own frame but not in this one, so far fewer pixels
// need the hand-over path; the fit itself does not depend on the frame.
#include <float.h>

#include "mls_internal.h"

namespace mlsi {
namespace {

using mlsk::KParams;

__device__ __forceinline__ float block_sum(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float r = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  return r;
}

__device__ __forceinline__ float block_min(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float r = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fminf(r, red[i]);
  return r;
}

__device__ __forceinline__ float block_max(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float r = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, red[i]);
  return r;
}

__global__ __launch_bounds__(256) void k_prepass_min(KParams p) {
  __shared__ float red[8];
  __shared__ float cx[256], cy[256];
  __shared__ int ccount;
  const int t = threadIdx.x;
  const int u0 = blockIdx.x * 16, v0 = blockIdx.y * 16;
  const int u = u0 + (t & 15), v = v0 + (t >> 4);
  const float px = mlsk::scaled_px(p, u), py = mlsk::scaled_py(p, v);
  const float X0 = mlsk::scaled_px(p, u0), X1 = mlsk::scaled_px(p, u0 + 15);
  const float Y0 = mlsk::scaled_py(p, v0), Y1 = mlsk::scaled_py(p, v0 + 15);
  const int n = (int)p.n;
  // bound on every tile pixel's nearest squared distance
  float b = FLT_MAX;
  for (int i = t; i < n; i += 256) {
    const float x = p.xs[i], y = p.ys[i];
    const float fx = fmaxf(fabsf(x - X0), fabsf(x - X1));
    const float fy = fmaxf(fabsf(y - Y0), fabsf(y - Y1));
    b = fminf(b, fx * fx + fy * fy);
  }
  const float bound = block_min(b, red) * 1.0001f + 1e-30f;
  // stream the points in chunks, keep those that may be nearest
  float m = FLT_MAX;
  for (int base = 0; base < n; base += 256) {
    if (t == 0) ccount = 0;
    __syncthreads();
    const int i = base + t;
    if (i < n) {
      const float x = p.xs[i], y = p.ys[i];
      const float ox = fmaxf(fmaxf(X0 - x, x - X1), 0.f);
      const float oy = fmaxf(fmaxf(Y0 - y, y - Y1), 0.f);
      if (ox * ox + oy * oy <= bound) {
        const int k = atomicAdd(&ccount, 1);
        cx[k] = x;
        cy[k] = y;
      }
    }
    __syncthreads();
    const int c = ccount;
    for (int k = 0; k < c; ++k) {
      const float dx = cx[k] - px, dy = cy[k] - py;
      m = fminf(m, dx * dx + dy * dy);
    }
    __syncthreads();
  }
  const int stride = p.tiles_x * 16;
  const_cast<float *>(p.mstab)[(size_t)v * stride + u] = m;
  // the tile's largest stabiliser bounds the reach of its weights above e^-gcut
  const float mx = block_max(m, red);
  if (t == 0) const_cast<float *>(p.tmax)[blockIdx.y * p.tiles_x + blockIdx.x] = mx;

  // frame of the tile: Gaussian-weighted centroid of the points around its centre
  const float Cx = mlsk::scaled_px(p, u0 + 8) - 0.5f * (mlsk::scaled_px(p, u0 + 8) - mlsk::scaled_px(p, u0 + 7));
  const float Cy = mlsk::scaled_py(p, v0 + 8) - 0.5f * (mlsk::scaled_py(p, v0 + 8) - mlsk::scaled_py(p, v0 + 7));
  float mc = FLT_MAX;
  for (int i = t; i < n; i += 256) {
    const float dx = p.xs[i] - Cx, dy = p.ys[i] - Cy;
    mc = fminf(mc, dx * dx + dy * dy);
  }
  mc = block_min(mc, red);
  float sw = 0.f, swx = 0.f, swy = 0.f;
  for (int i = t; i < n; i += 256) {
    const float dx = p.xs[i] - Cx, dy = p.ys[i] - Cy;
    const float w = exp2f((mc - (dx * dx + dy * dy)) * 1.4426950408889634f);
    sw += w;
    swx = fmaf(w, dx, swx);
    swy = fmaf(w, dy, swy);
  }
  sw = block_sum(sw, red);
  swx = block_sum(swx, red);
  swy = block_sum(swy, red);
  if (t == 0) {
    float *tc = const_cast<float *>(p.tcen) + 2 * (blockIdx.y * p.tiles_x + blockIdx.x);
    tc[0] = (sw > 0.f) ? Cx + swx / sw : Cx;
    tc[1] = (sw > 0.f) ? Cy + swy / sw : Cy;
  }
}

// Inclusive cell range [c0, c1] covering [lo - r, hi + r] along one axis.
__device__ __forceinline__ void cell_range(double lo, double hi, double r, double g0, double inv_cell, int g,
                                           int &c0, int &c1) {
  c0 = (int)floor((lo - r - g0) * inv_cell);
  c1 = (int)floor((hi + r - g0) * inv_cell);
  c0 = max(c0, 0);
  c1 = min(c1, g - 1);
}

// Tile geometry computed once per block (GB300's FP64 rate is a small
// fraction of FP32's: per-thread FP64 set-up cost more than the search):
// scaled pixel-centre coordinates of the 16 columns and rows, and the cell
// window covering the tile's pixel centres +- r (raw units).
struct PreGeo {
  float col[16], row[16];
  int win[4];   // c0, c1, d0, d1
};

__device__ __forceinline__ void pre_geometry(const KParams &p, int u0, int v0, PreGeo *g) {
  const int t = threadIdx.x;
  if (t < 16) g->col[t] = mlsk::scaled_px(p, u0 + t);
  else if (t < 32) g->row[t - 16] = mlsk::scaled_py(p, v0 + t - 16);
}

// Thread 0 sets the window for radius r, or, with bound >= 0, for radius
// max(h sqrt(bound) (1 + 1e-5), rmin); the caller synchronises.
__device__ __forceinline__ void pre_window(const KParams &p, int u0, int v0, double r, PreGeo *g,
                                           float bound = -1.f, double rmin = 0.0) {
  if (threadIdx.x == 0) {
    if (bound >= 0.f) r = fmax(sqrt((double)bound) * p.h * (1.0 + 1e-5) + 1e-12, rmin);
    const double inv_cell = p.inv_cell;
    const double xa = p.x0 + (u0 + 0.5) * p.sx, xb = p.x0 + (u0 + 15.5) * p.sx;
    const double ya = p.y0 + (v0 + 0.5) * p.sy, yb = p.y0 + (v0 + 15.5) * p.sy;
    cell_range(fmin(xa, xb), fmax(xa, xb), r, p.gx0, inv_cell, p.gx, g->win[0], g->win[1]);
    cell_range(fmin(ya, yb), fmax(ya, yb), r, p.gy0, inv_cell, p.gy, g->win[2], g->win[3]);
  }
}

// Gaussian weight (points binned on the uniform grid): the same stabiliser
// and tile frame from the cells near the tile instead of all n points.  A
// window of cells around the tile is grown until it holds a point; the bound
// B = min over its points of the squared distance to the farthest tile corner
// is at least every pixel's nearest squared distance, so every pixel's
// nearest point lies in the cells within sqrt(B) of the tile, which are then
// scanned exactly.  The frame (it only conditions the fit) is the Gaussian-
// weighted centroid, around the tile centre, of the points in the cells within
// 4 h of the tile (weights below e^-16 of the largest are left out).
// The index ranges [a, e) of the cell rows d0 .. d0 + nr - 1 of a window
// (columns c0 .. c1), fetched by the first nr threads at once (one round
// trip for the rows instead of one per row); the caller synchronises.
__device__ __forceinline__ void pre_rows(const KParams &p, int c0, int c1, int d0, int nr, int *ra, int *re) {
  const int t = threadIdx.x;
  if (t < nr) {
    const int64_t row = (int64_t)(d0 + t) * p.gx;
    ra[t] = cell_at(p, row + c0);
    re[t] = cell_at(p, row + c1 + 1);
  }
}

__global__ __launch_bounds__(256) void k_prepass_min_cells(KParams p) {
  __shared__ float red[8];
  __shared__ float cx[256], cy[256];
  __shared__ int ra[256], re[256];
  __shared__ PreGeo G;
  const int t = threadIdx.x;
  const int u0 = blockIdx.x * 16, v0 = blockIdx.y * 16;
  pre_geometry(p, u0, v0, &G);
  __syncthreads();
  const float px = G.col[t & 15], py = G.row[t >> 4];
  const float X0 = G.col[0], X1 = G.col[15], Y0 = G.row[0], Y1 = G.row[15];
  // 1) bound from the first non-empty window of cells around the tile
  float b = FLT_MAX;
  double r = p.cell;
  for (int round = 0; round < 40; ++round) {
    __syncthreads();
    pre_window(p, u0, v0, r, &G);
    __syncthreads();
    const int c0 = G.win[0], c1 = G.win[1], d0 = G.win[2], d1 = G.win[3];
    for (int rb = d0; rb <= d1 && c0 <= c1; rb += 256) {
      const int nr = min(256, d1 - rb + 1);
      __syncthreads();
      pre_rows(p, c0, c1, rb, nr, ra, re);
      __syncthreads();
      for (int k = 0; k < nr; ++k)
        for (int i = ra[k] + t; i < re[k]; i += 256) {
          const float x = p.xs[i], y = p.ys[i];
          const float fx = fmaxf(fabsf(x - X0), fabsf(x - X1));
          const float fy = fmaxf(fabsf(y - Y0), fabsf(y - Y1));
          b = fminf(b, fx * fx + fy * fy);
        }
    }
    if (block_min(b, red) < FLT_MAX) break;   // uniform: every thread sees the same minimum
    r *= 2.0;
  }
  const float bound = block_min(b, red) * 1.0001f + 1e-30f;
  // 2) exact nearest squared distance of each pixel over the cells within sqrt(bound)
  __syncthreads();
  pre_window(p, u0, v0, 0.0, &G, bound);
  __syncthreads();
  int c0 = G.win[0], c1 = G.win[1], d0 = G.win[2], d1 = G.win[3];
  float m = FLT_MAX;
  for (int rb = d0; rb <= d1 && c0 <= c1; rb += 256) {
    const int nr = min(256, d1 - rb + 1);
    __syncthreads();
    pre_rows(p, c0, c1, rb, nr, ra, re);
    __syncthreads();
    for (int k = 0; k < nr; ++k) {
      const int a = ra[k], e = re[k];
      for (int base = a; base < e; base += 256) {
        __syncthreads();
        if (base + t < e) {
          cx[t] = p.xs[base + t];
          cy[t] = p.ys[base + t];
        }
        __syncthreads();
        const int c = min(256, e - base);
        for (int q = 0; q < c; ++q) {
          const float dx = cx[q] - px, dy = cy[q] - py;
          m = fminf(m, dx * dx + dy * dy);
        }
      }
    }
  }
  const int stride = p.tiles_x * 16;
  const_cast<float *>(p.mstab)[(size_t)(v0 + (t >> 4)) * stride + u0 + (t & 15)] = m;
  const float mx = block_max(m, red);
  if (t == 0) const_cast<float *>(p.tmax)[blockIdx.y * p.tiles_x + blockIdx.x] = mx;
  // 3) frame: Gaussian-weighted centroid of the points within 4 h of the
  // tile, in one pass: each thread keeps the sums relative to the smallest
  // squared distance it has seen so far (rescaling them when a nearer point
  // comes), and the block combines them relative to the overall smallest
  const float Cx = G.col[8] - 0.5f * (G.col[8] - G.col[7]);
  const float Cy = G.row[8] - 0.5f * (G.row[8] - G.row[7]);
  constexpr float kL2e = 1.4426950408889634f;
  __syncthreads();
  pre_window(p, u0, v0, 0.0, &G, bound, 4.0 * p.h);
  __syncthreads();
  c0 = G.win[0]; c1 = G.win[1]; d0 = G.win[2]; d1 = G.win[3];
  float ml = FLT_MAX, sw = 0.f, swx = 0.f, swy = 0.f;
  for (int rb = d0; rb <= d1 && c0 <= c1; rb += 256) {
    const int nr = min(256, d1 - rb + 1);
    __syncthreads();
    pre_rows(p, c0, c1, rb, nr, ra, re);
    __syncthreads();
    for (int k = 0; k < nr; ++k)
      for (int i = ra[k] + t; i < re[k]; i += 256) {
        const float dx = p.xs[i] - Cx, dy = p.ys[i] - Cy;
        const float d2 = dx * dx + dy * dy;
        if (d2 < ml) {
          const float sc = (ml == FLT_MAX) ? 0.f : exp2f((d2 - ml) * kL2e);
          sw *= sc;
          swx *= sc;
          swy *= sc;
          ml = d2;
        }
        const float w = exp2f((ml - d2) * kL2e);
        sw += w;
        swx = fmaf(w, dx, swx);
        swy = fmaf(w, dy, swy);
      }
  }
  const float mc = block_min(ml, red);
  const float sc = (ml == FLT_MAX) ? 0.f : exp2f((mc - ml) * kL2e);
  sw = block_sum(sw * sc, red);
  swx = block_sum(swx * sc, red);
  swy = block_sum(swy * sc, red);
  if (t == 0) {
    float *tc = const_cast<float *>(p.tcen) + 2 * (blockIdx.y * p.tiles_x + blockIdx.x);
    tc[0] = (sw > 0.f) ? Cx + swx / sw : Cx;
    tc[1] = (sw > 0.f) ? Cy + swy / sw : Cy;
  }
}

__global__ __launch_bounds__(256) void k_prepass_count(KParams p) {
  __shared__ float cx[256], cy[256];
  __shared__ PreGeo G;
  const int t = threadIdx.x;
  const int u0 = blockIdx.x * 16, v0 = blockIdx.y * 16;
  const int u = u0 + (t & 15), v = v0 + (t >> 4);
  pre_geometry(p, u0, v0, &G);
  pre_window(p, u0, v0, p.h, &G);   // the cells within the support radius of the tile's pixels
  __syncthreads();
  const float px = G.col[t & 15], py = G.row[t >> 4];
  const int cx0 = G.win[0], cx1 = G.win[1], cy0 = G.win[2], cy1 = G.win[3];
  int count = 0;
  bool edge = false;
  for (int cyy = cy0; cyy <= cy1 && cx0 <= cx1; ++cyy) {
    const int a = cell_at(p, (int64_t)cyy * p.gx + cx0);
    const int e = cell_at(p, (int64_t)cyy * p.gx + cx1 + 1);
    for (int base = a; base < e; base += 256) {
      __syncthreads();
      if (base + t < e) {
        cx[t] = p.xs[base + t];
        cy[t] = p.ys[base + t];
      }
      __syncthreads();
      const int c = min(256, e - base);
      for (int k = 0; k < c; ++k) {
        const float dx = cx[k] - px, dy = cy[k] - py;
        const float q2 = dx * dx + dy * dy;
        count += (q2 < 1.f) ? 1 : 0;
        edge = edge || fabsf(q2 - 1.f) < mlsk::kCntEdgeTol;
      }
    }
  }
  const int stride = p.tiles_x * 16;
  const_cast<int *>(p.cnt)[(size_t)v * stride + u] = count | (edge ? mlsk::kCntBoundary : 0);

  // frame of the tile: Wendland-weighted centroid around its centre
  __shared__ float red[8];
  const float Cx = 0.5f * (G.col[7] + G.col[8]);
  const float Cy = 0.5f * (G.row[7] + G.row[8]);
  float sw = 0.f, swx = 0.f, swy = 0.f;
  for (int cyy = cy0; cyy <= cy1 && cx0 <= cx1; ++cyy) {
    const int a = cell_at(p, (int64_t)cyy * p.gx + cx0);
    const int e = cell_at(p, (int64_t)cyy * p.gx + cx1 + 1);
    for (int i = a + t; i < e; i += 256) {
      const float dx = p.xs[i] - Cx, dy = p.ys[i] - Cy;
      const float q = sqrtf(dx * dx + dy * dy);
      const float o = 1.f - q, o2 = o * o;
      const float w = (q < 1.f) ? o2 * o2 * fmaf(4.f, q, 1.f) : 0.f;
      sw += w;
      swx = fmaf(w, dx, swx);
      swy = fmaf(w, dy, swy);
    }
  }
  sw = block_sum(sw, red);
  swx = block_sum(swx, red);
  swy = block_sum(swy, red);
  if (t == 0) {
    float *tc = const_cast<float *>(p.tcen) + 2 * (blockIdx.y * p.tiles_x + blockIdx.x);
    tc[0] = (sw > 0.f) ? Cx + swx / sw : Cx;
    tc[1] = (sw > 0.f) ? Cy + swy / sw : Cy;
  }
}

__global__ __launch_bounds__(256) void k_prepass_box(KParams p) {
  __shared__ float cx[256], cy[256];
  __shared__ PreGeo G;
  const int t = threadIdx.x;
  const int u0 = blockIdx.x * 16, v0 = blockIdx.y * 16;
  const int u = u0 + (t & 15), v = v0 + (t >> 4);
  pre_geometry(p, u0, v0, &G);
  pre_window(p, u0, v0, p.trunc * p.h * (1.0 + 1e-5), &G);   // the cells within the box of the tile's pixels
  __syncthreads();
  const float px = G.col[t & 15], py = G.row[t >> 4];
  const float c = (float)p.trunc;
  // rounding of the scaled offsets grows with the coordinates' magnitude
  const float tx = mlsk::kCntEdgeTol * (c + fabsf(px)), ty = mlsk::kCntEdgeTol * (c + fabsf(py));
  const int cx0 = G.win[0], cx1 = G.win[1], cy0 = G.win[2], cy1 = G.win[3];
  int count = 0;
  bool edge = false;
  for (int cyy = cy0; cyy <= cy1 && cx0 <= cx1; ++cyy) {
    const int a = cell_at(p, (int64_t)cyy * p.gx + cx0);
    const int e = cell_at(p, (int64_t)cyy * p.gx + cx1 + 1);
    for (int base = a; base < e; base += 256) {
      __syncthreads();
      if (base + t < e) {
        cx[t] = p.xs[base + t];
        cy[t] = p.ys[base + t];
      }
      __syncthreads();
      const int n = min(256, e - base);
      for (int k = 0; k < n; ++k) {
        const float ax = fabsf(cx[k] - px), ay = fabsf(cy[k] - py);
        count += (ax < c && ay < c) ? 1 : 0;
        edge = edge || fabsf(ax - c) < tx || fabsf(ay - c) < ty;
      }
    }
  }
  const int stride = p.tiles_x * 16;
  const_cast<int *>(p.cnt)[(size_t)v * stride + u] = count | (edge ? mlsk::kCntBoundary : 0);
}

}  // namespace

void launch_prepass(const KParams &p, cudaStream_t st) {
  dim3 grid(p.tiles_x, p.tiles_y);
  if (p.weight == MLS_W_WENDLAND) {
    k_prepass_count<<<grid, 256, 0, st>>>(p);
  } else {
    if (p.weight == MLS_W_GAUSS && p.cell_start) k_prepass_min_cells<<<grid, 256, 0, st>>>(p);
    else k_prepass_min<<<grid, 256, 0, st>>>(p);
    if (p.trunc > 0.0) k_prepass_box<<<grid, 256, 0, st>>>(p);
  }
}

}  // namespace mlsi
