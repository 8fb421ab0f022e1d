// Space mappings of Section 3.4: the field rendered as an RGBA8 image.
//
// The paper describes the renderings in words; the definitions taken here,
// per pixel and shown field plane (one or two planes):
//   g      the value rounded to float
//   grad   |(g_x, g_y)| per pixel: central differences, one-sided at the image
//          edge or next to a NaN neighbour, 0 with no neighbour
//   b      the band #{t_j <= f} (in the field's own precision, as mls_bands)
//   delta  min |g - t| * (1 / grad) over the band's bounding levels (0 on a
//          level, infinite where grad = 0), in pixels
//   cov    line coverage clamp(w/2 + 1/2 - delta, 0, 1)
//   adaptive lines: the band spacing halved k = 1..K times; depth-k levels
//          (odd multiples of spacing / 2^k above the band's lower level) drawn
//          with the same rule, faded by clamp((spacing / 2^k / grad - fade_lo)
//          / (fade_hi - fade_lo), 0, 1)
//   colours: three-anchor ramp (one plane) or four corner colours (two
//          planes), sampled at (b + 1/2) / (L + 1) for the band colours or at
//          clamp((g - lo) / (hi - lo), 0, 1) for the gradients; the texture
//          mapping looks an RGBA8 texture up bilinearly at those coordinates
//          (clamp to edge); lines black over white or over the colours; NaN
//          transparent.
// Every float operation is a round-to-nearest intrinsic (no contraction), in
// a fixed order, so the bytes are reproducible on any IEEE float machine.
// Quotients are products with a reciprocal formed once: 1/grad and 1/spacing
// per pixel and plane, 1/(L + 1), 1/(hi - lo) and 1/(fade_hi - fade_lo) per
// image (on the host, in float).
//
// 32 x 8 threads per block, each mapping four pixels of a 32 x 32 tile; the
// shown planes are staged as floats with a one-pixel halo in shared memory
// for the differences (all loads of a block in flight before its barrier).  The
// levels travel in the kernel's parameter block (no device allocation) and
// are copied to shared memory, where the per-pixel lookups (different
// indices across a warp) do not serialise as they would in constant memory.
#include <cmath>
#include <cstring>

#include "mls_internal.h"

namespace mlsi {
namespace {

constexpr int kMapMaxL = 254;
constexpr int kBX = 32, kBY = 8, kTH = 32;   // threads 32 x 8, tile 32 x 32 pixels

struct MapParams {
  int mode, ndim, W, H, L, fp64, K;
  const void *plane[2];
  float w, fade_lo, fade_hi;
  float inv_den, inv_l1;        // 1 / (fade_hi - fade_lo), 1 / (L + 1)
  float lo[2], inv_rng[2];      // lo, 1 / (hi - lo)
  const uint8_t *tex;
  int tw, th;
  uint8_t *rgba;
  double lev64[2][kMapMaxL];    // the levels (band decisions on FP64 fields)
  float levru[2][kMapMaxL];     // rounded up (band decisions on FP32 fields)
  float levrn[2][kMapMaxL];     // rounded to nearest (distances)
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }
__device__ __forceinline__ float lerp(float a, float b, float t) { return fadd(a, fmul(fsub(b, a), t)); }

// #{j : t_j <= f} over ascending levels (upper bound)
template <typename T>
__device__ __forceinline__ int band_count(T f, const T *lev, int L) {
  int lo = 0, hi = L;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lev[mid] <= f) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float px_distance(float dv, float grad, float inv_grad) {
  return dv == 0.f ? 0.f : (grad > 0.f ? fmul(dv, inv_grad) : INFINITY);
}

__device__ __forceinline__ float coverage(float delta, float w) {
  return clamp01(fsub(fadd(fmul(w, 0.5f), 0.5f), delta));
}

struct Levels {
  double lev64[2][kMapMaxL];
  float levru[2][kMapMaxL];
  float levrn[2][kMapMaxL];
};

// band and line coverage of one plane at one pixel
__device__ void plane_terms(const MapParams &p, const Levels &S, int k, float g, double f64, float gl, float gr,
                            float gd, float gu, float &cov, int &b) {
  const int L = p.L;
  // gradient
  const bool hl = !isnan(gl), hr = !isnan(gr), hd = !isnan(gd), hu = !isnan(gu);
  const float gx = (hl && hr) ? fmul(fsub(gr, gl), 0.5f) : hr ? fsub(gr, g) : hl ? fsub(g, gl) : 0.f;
  const float gy = (hd && hu) ? fmul(fsub(gu, gd), 0.5f) : hu ? fsub(gu, g) : hd ? fsub(g, gd) : 0.f;
  const float grad = __fsqrt_rn(fadd(fmul(gx, gx), fmul(gy, gy)));
  const float inv_grad = __frcp_rn(grad);
  b = p.fp64 ? band_count(f64, S.lev64[k], L) : band_count(g, S.levru[k], L);
  float dv = INFINITY;
  if (b >= 1) dv = fabsf(fsub(g, S.levrn[k][b - 1]));
  if (b < L) dv = fminf(dv, fabsf(fsub(g, S.levrn[k][b])));
  cov = coverage(px_distance(dv, grad, inv_grad), p.w);
  if (p.mode != MLS_MAP_ADAPTIVE || L < 2) return;
  const float *t = S.levrn[k];
  float spacing, base;
  if (b >= 1 && b <= L - 1) {
    spacing = fsub(t[b], t[b - 1]);
    base = t[b - 1];
  } else if (b == 0) {
    spacing = fsub(t[1], t[0]);
    base = fsub(t[0], spacing);
  } else {
    spacing = fsub(t[L - 1], t[L - 2]);
    base = t[L - 1];
  }
  const float inv_spacing = __frcp_rn(spacing);
  if (!(spacing > 0.f) || isinf(inv_spacing)) return;
  float scale = 0.5f, up = 2.f;
  for (int d = 1; d <= p.K; ++d, scale *= 0.5f, up *= 2.f) {
    const float dk = fmul(spacing, scale), inv_dk = fmul(inv_spacing, up);
    const float sp = grad > 0.f ? fmul(dk, inv_grad) : INFINITY;
    const float alpha = clamp01(fmul(fsub(sp, p.fade_lo), p.inv_den));
    if (!(alpha > 0.f)) break;   // spacing halves with each depth: no deeper level shows either
    const float r = fmul(fsub(g, base), inv_dk);
    const float m = fadd(fmul(2.f, floorf(fmul(r, 0.5f))), 1.f);
    const float dist = fmul(fabsf(fsub(r, m)), dk);
    cov = fmaxf(cov, fmul(coverage(px_distance(dist, grad, inv_grad), p.w), alpha));
  }
}

__device__ __forceinline__ void ramp(float s, float *c) {
  const float A[3][3] = {{0.16f, 0.29f, 0.78f}, {0.93f, 0.93f, 0.93f}, {0.78f, 0.16f, 0.16f}};
  const bool low = s <= 0.5f;
  const float t = low ? fmul(s, 2.f) : fmul(fsub(s, 0.5f), 2.f);
#pragma unroll
  for (int i = 0; i < 3; ++i) c[i] = low ? lerp(A[0][i], A[1][i], t) : lerp(A[1][i], A[2][i], t);
}

__device__ __forceinline__ void corner(float s, float t, float *c) {
  const float B[3] = {0.10f, 0.20f, 0.90f}, P[3] = {0.95f, 0.35f, 0.75f};
  const float C[3] = {0.10f, 0.85f, 0.90f}, Y[3] = {0.95f, 0.95f, 0.75f};
#pragma unroll
  for (int i = 0; i < 3; ++i) c[i] = lerp(lerp(B[i], P[i], s), lerp(C[i], Y[i], s), t);
}

__device__ __forceinline__ uint8_t to_byte(float c) {
  const float q = floorf(fadd(fmul(c, 255.f), 0.5f));
  return (uint8_t)fminf(fmaxf(q, 0.f), 255.f);
}

// The mapping of one pixel from its staged value and neighbours.
__device__ __forceinline__ void map_pixel(const MapParams &p, const Levels &S, const float (*tile)[kTH + 2][kBX + 2],
                                          int ty, int tx, size_t pix) {
  uint8_t *out = p.rgba + 4 * pix;
  float g[2] = {0.f, 0.f}, cov = 0.f;
  int b[2] = {0, 0};
  bool valid = true;
  for (int k = 0; k < p.ndim; ++k) {
    g[k] = tile[k][ty + 1][tx + 1];
    valid = valid && !isnan(g[k]);
  }
  if (!valid) {
    *(uchar4 *)out = make_uchar4(0, 0, 0, 0);
    return;
  }
  for (int k = 0; k < p.ndim; ++k) {
    const double f64 = p.fp64 ? ((const double *)p.plane[k])[pix] : 0.0;
    float ck;
    plane_terms(p, S, k, g[k], f64, tile[k][ty + 1][tx], tile[k][ty + 1][tx + 2], tile[k][ty][tx + 1],
                tile[k][ty + 2][tx + 1], ck, b[k]);
    cov = fmaxf(cov, ck);
  }
  float col[3] = {1.f, 1.f, 1.f};
  const bool lines = p.mode == MLS_MAP_LINES || p.mode == MLS_MAP_DISCRETE_LINES || p.mode == MLS_MAP_ADAPTIVE ||
                     p.mode == MLS_MAP_GRADIENT;
  if (p.mode == MLS_MAP_DISCRETE || p.mode == MLS_MAP_DISCRETE_LINES) {
    const float s0 = fmul(fadd((float)b[0], 0.5f), p.inv_l1);
    const float s1 = fmul(fadd((float)b[1], 0.5f), p.inv_l1);
    if (p.ndim == 1) ramp(s0, col);
    else corner(s0, s1, col);
  } else if (p.mode == MLS_MAP_GRADIENT || p.mode == MLS_MAP_TEXTURE) {
    const float s0 = clamp01(fmul(fsub(g[0], p.lo[0]), p.inv_rng[0]));
    const float s1 = p.ndim == 2 ? clamp01(fmul(fsub(g[1], p.lo[1]), p.inv_rng[1])) : 0.5f;
    if (p.mode == MLS_MAP_TEXTURE) {
      const float x = fsub(fmul(s0, (float)p.tw), 0.5f), y = fsub(fmul(s1, (float)p.th), 0.5f);
      const float x0 = floorf(x), y0 = floorf(y);
      const float fx = fsub(x, x0), fy = fsub(y, y0);
      const int ix0 = min(max((int)x0, 0), p.tw - 1), ix1 = min(max((int)x0 + 1, 0), p.tw - 1);
      const int iy0 = min(max((int)y0, 0), p.th - 1), iy1 = min(max((int)y0 + 1, 0), p.th - 1);
      const uchar4 a = *(const uchar4 *)(p.tex + 4 * ((size_t)iy0 * p.tw + ix0));
      const uchar4 bb = *(const uchar4 *)(p.tex + 4 * ((size_t)iy0 * p.tw + ix1));
      const uchar4 c = *(const uchar4 *)(p.tex + 4 * ((size_t)iy1 * p.tw + ix0));
      const uchar4 d = *(const uchar4 *)(p.tex + 4 * ((size_t)iy1 * p.tw + ix1));
      const float ta[4] = {(float)a.x, (float)a.y, (float)a.z, (float)a.w};
      const float tb[4] = {(float)bb.x, (float)bb.y, (float)bb.z, (float)bb.w};
      const float tc[4] = {(float)c.x, (float)c.y, (float)c.z, (float)c.w};
      const float td[4] = {(float)d.x, (float)d.y, (float)d.z, (float)d.w};
      uint8_t q[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float val = lerp(lerp(ta[i], tb[i], fx), lerp(tc[i], td[i], fx), fy);
        q[i] = (uint8_t)fminf(fmaxf(floorf(fadd(val, 0.5f)), 0.f), 255.f);
      }
      *(uchar4 *)out = make_uchar4(q[0], q[1], q[2], q[3]);
      return;
    }
    if (p.ndim == 1) ramp(s0, col);
    else corner(s0, s1, col);
  }
  if (lines) {
#pragma unroll
    for (int i = 0; i < 3; ++i) col[i] = lerp(col[i], 0.f, cov);
  }
  *(uchar4 *)out = make_uchar4(to_byte(col[0]), to_byte(col[1]), to_byte(col[2]), 255);
}

__global__ __launch_bounds__(kBX * kBY) void k_space_map(const __grid_constant__ MapParams p) {
  __shared__ float tile[2][kTH + 2][kBX + 2];
  __shared__ Levels S;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int u0 = blockIdx.x * kBX, v0 = blockIdx.y * kTH;
  const int t = ty * kBX + tx;
  for (int k = 0; k < p.ndim; ++k)
    for (int j = t; j < p.L; j += kBX * kBY) {
      S.lev64[k][j] = p.lev64[k][j];
      S.levru[k][j] = p.levru[k][j];
      S.levrn[k][j] = p.levrn[k][j];
    }
  // stage the planes with a one-pixel halo (NaN outside the image); every
  // thread issues all of its loads before the barrier
  for (int k = 0; k < p.ndim; ++k) {
    for (int e = t; e < (kTH + 2) * (kBX + 2); e += kBX * kBY) {
      const int yy = e / (kBX + 2), xx = e - yy * (kBX + 2);
      const int u = u0 + xx - 1, v = v0 + yy - 1;
      float val = __int_as_float(0x7fc00000);
      if (u >= 0 && u < p.W && v >= 0 && v < p.H) {
        const size_t i = (size_t)v * p.W + u;
        val = p.fp64 ? __double2float_rn(((const double *)p.plane[k])[i]) : ((const float *)p.plane[k])[i];
      }
      tile[k][yy][xx] = val;
    }
  }
  __syncthreads();
  const int u = u0 + tx;
  if (u >= p.W) return;
#pragma unroll 1
  for (int r = 0; r < kTH / kBY; ++r) {
    const int yy = ty + r * kBY, v = v0 + yy;
    if (v >= p.H) break;
    map_pixel(p, S, tile, yy, tx, (size_t)v * p.W + u);
  }
}

bool finite_d(double x) { return std::isfinite(x); }

}  // namespace
}  // namespace mlsi

mls_status mls_space_map(const mls_map_desc *m, int32_t D, int32_t W, int32_t H, const void *field,
                         int32_t field_fp64, const double *levels, int32_t L, uint8_t *rgba, void *stream) {
  using namespace mlsi;
  if (!m) return fail(MLS_E_INVAL, "map description is NULL");
  if (!field || !rgba) return fail(MLS_E_INVAL, "field and rgba must not be NULL");
  if (D < 1 || W < 1 || H < 1) return fail(MLS_E_INVAL, "D, W and H must be >= 1");
  if ((int64_t)W * H > (int64_t)1 << 30) return fail(MLS_E_INVAL, "more than 2^30 pixels");
  if (field_fp64 != 0 && field_fp64 != 1) return fail(MLS_E_INVAL, "field_fp64 must be 0 or 1");
  if (m->mode < MLS_MAP_LINES || m->mode > MLS_MAP_TEXTURE) return fail(MLS_E_INVAL, "unknown mode");
  if (m->ndim != 1 && m->ndim != 2) return fail(MLS_E_INVAL, "ndim must be 1 or 2");
  for (int k = 0; k < m->ndim; ++k)
    if (m->dim[k] < 0 || m->dim[k] >= D) return fail(MLS_E_INVAL, "dim out of range");
  if (L < 0 || L > kMapMaxL) return fail(MLS_E_INVAL, "L must be in [0, 254]");
  if (L > 0 && !levels) return fail(MLS_E_INVAL, "levels must not be NULL when L > 0");
  if (!(finite_d(m->line_width) && m->line_width >= 0.f && m->line_width <= 1e4f))
    return fail(MLS_E_INVAL, "line_width must be in [0, 1e4]");
  if (m->mode == MLS_MAP_ADAPTIVE) {
    if (!(finite_d(m->fade_lo) && finite_d(m->fade_hi) && m->fade_lo >= 0.f && m->fade_lo < m->fade_hi))
      return fail(MLS_E_INVAL, "fade_lo and fade_hi must satisfy 0 <= fade_lo < fade_hi");
    if (m->sublevels < 0 || m->sublevels > 16) return fail(MLS_E_INVAL, "sublevels must be in [0, 16]");
  }
  if (m->mode == MLS_MAP_GRADIENT || m->mode == MLS_MAP_TEXTURE) {
    for (int k = 0; k < m->ndim; ++k) {
      const float lo = (float)m->lo[k], hi = (float)m->hi[k];
      const float rng = hi - lo;
      if (!(finite_d(m->lo[k]) && finite_d(m->hi[k]) && std::isfinite(lo) && std::isfinite(hi) && rng != 0.f &&
            std::isfinite(rng) && std::isfinite(1.0f / rng)))
        return fail(MLS_E_INVAL, "lo and hi must be finite and differ in float (with a finite 1 / (hi - lo))");
    }
  }
  if (m->mode == MLS_MAP_TEXTURE) {
    if (!m->texture) return fail(MLS_E_INVAL, "texture must not be NULL");
    if (m->tex_w < 1 || m->tex_h < 1 || m->tex_w > 65536 || m->tex_h > 65536)
      return fail(MLS_E_INVAL, "texture size must be in [1, 65536]");
  }
  MapParams p;
  memset(&p, 0, sizeof p);
  p.mode = m->mode;
  p.ndim = m->ndim;
  p.W = W;
  p.H = H;
  p.L = L;
  p.fp64 = field_fp64;
  p.K = m->mode == MLS_MAP_ADAPTIVE ? m->sublevels : 0;
  p.w = m->line_width;
  p.fade_lo = m->fade_lo;
  p.fade_hi = m->fade_hi;
  if (m->mode == MLS_MAP_ADAPTIVE) {
    const float den = m->fade_hi - m->fade_lo;
    p.inv_den = 1.0f / den;
  }
  p.inv_l1 = 1.0f / (float)(L + 1);
  p.tex = m->texture;
  p.tw = m->tex_w;
  p.th = m->tex_h;
  p.rgba = rgba;
  const size_t esz = field_fp64 ? sizeof(double) : sizeof(float);
  for (int k = 0; k < m->ndim; ++k) {
    p.plane[k] = (const unsigned char *)field + (size_t)m->dim[k] * W * H * esz;
    p.lo[k] = (float)m->lo[k];
    {
      const float rng = (float)m->hi[k] - (float)m->lo[k];
      p.inv_rng[k] = 1.0f / rng;
    }
    for (int j = 0; j < L; ++j) {
      const double t = levels[(size_t)m->dim[k] * L + j];
      if (!std::isfinite(t)) return fail(MLS_E_INVAL, "levels must be finite");
      if (j > 0 && !(t >= levels[(size_t)m->dim[k] * L + j - 1])) return fail(MLS_E_INVAL, "levels must ascend");
      float ru = (float)t;
      if ((double)ru < t) ru = std::nextafter(ru, INFINITY);
      p.lev64[k][j] = t;
      p.levru[k][j] = ru;
      p.levrn[k][j] = (float)t;
    }
  }
  dim3 grid((unsigned)((W + kBX - 1) / kBX), (unsigned)((H + kTH - 1) / kTH));
  if (grid.y > 65535u) return fail(MLS_E_UNSUPPORTED, "image taller than 2,097,120 rows");
  k_space_map<<<grid, dim3(kBX, kBY), 0, (cudaStream_t)stream>>>(p);
  MLS_CUDA_TRY(cudaGetLastError());
  return MLS_OK;
}
