// Point preparation (the upload step of mls_create): value ranges and the
// point bounding box, uniform-grid binning for compact-support weights
// (histogram, exclusive scan, scatter, deterministic in-cell order), and the
// conversion of the positions and values to the layouts the kernels read.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mls_internal.h"

namespace mlsi {

namespace {

__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

double host_from_key(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double d;
  memcpy(&d, &u, sizeof d);
  return d;
}

// Column min / max of a rows x cols row-major matrix as order-preserving keys.
__global__ void k_colminmax(const double *A, int64_t rows, int cols, unsigned long long *gmin,
                            unsigned long long *gmax) {
  extern __shared__ unsigned long long sm[];
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    sm[c] = ~0ull;
    sm[cols + c] = 0ull;
  }
  __syncthreads();
  const int64_t total = rows * (int64_t)cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % cols);
    const unsigned long long k = order_key(A[e]);
    atomicMin(&sm[c], k);
    atomicMax(&sm[cols + c], k);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    atomicMin(&gmin[c], sm[c]);
    atomicMax(&gmax[c], sm[cols + c]);
  }
}

// Centre and half-range of every value column from its range keys (the
// values are normalised to [-1, 1] by these; a constant column keeps scale 1).
__global__ void k_value_frames(const unsigned long long *kmin, const unsigned long long *kmax, int D, double *cen,
                               double *scl, float *cen32, float *scl32) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D) return;
  const unsigned long long a = kmin[c], b = kmax[c];
  const double lo = __longlong_as_double((long long)((a >> 63) ? (a & 0x7fffffffffffffffull) : ~a));
  const double hi = __longlong_as_double((long long)((b >> 63) ? (b & 0x7fffffffffffffffull) : ~b));
  const double ce = 0.5 * (lo + hi);
  double sc = 0.5 * (hi - lo);
  if (!(sc > 0.0)) sc = 1.0;
  cen[c] = ce;
  scl[c] = sc;
  cen32[c] = (float)ce;
  scl32[c] = (float)sc;
}

// Range keys before the reduction: m minima at the largest key, then m
// maxima at the smallest.
__global__ void k_init_keys(unsigned long long *p, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * m) p[i] = i < m ? ~0ull : 0ull;
}

// Cell of each point on the uniform grid (the same expression is used by
// every kernel that looks cells up).
__global__ void k_bin_count(const double *xy, int64_t n, double gx0, double gy0, double inv_cell, int gx,
                            int gy, int *key, int *counts) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx = (int)floor((xy[2 * i] - gx0) * inv_cell);
  int cy = (int)floor((xy[2 * i + 1] - gy0) * inv_cell);
  cx = min(max(cx, 0), gx - 1);
  cy = min(max(cy, 0), gy - 1);
  const int c = cy * gx + cx;
  key[i] = c;
  atomicAdd(&counts[c], 1);
}

// Exclusive scan, three passes: per-block scan of 1024 elements, a serial
// scan of the block totals in one block, then the add-back.
__global__ void k_scan_blocks(const int *in, int n, int *out, int *totals) {
  __shared__ int s[1024];
  const int base = blockIdx.x * 1024;
  const int t = threadIdx.x;  // 512 threads, two elements each
  s[2 * t] = (base + 2 * t < n) ? in[base + 2 * t] : 0;
  s[2 * t + 1] = (base + 2 * t + 1 < n) ? in[base + 2 * t + 1] : 0;
  __syncthreads();
  // Hillis-Steele inclusive scan over 1024 entries
  for (int off = 1; off < 1024; off <<= 1) {
    const int a = (2 * t >= off) ? s[2 * t - off] : 0;
    const int b = (2 * t + 1 >= off) ? s[2 * t + 1 - off] : 0;
    __syncthreads();
    s[2 * t] += a;
    s[2 * t + 1] += b;
    __syncthreads();
  }
  if (base + 2 * t < n) out[base + 2 * t] = s[2 * t] - in[base + 2 * t];
  if (base + 2 * t + 1 < n) out[base + 2 * t + 1] = s[2 * t + 1] - in[base + 2 * t + 1];
  if (t == 511) totals[blockIdx.x] = s[1023];
}

__global__ void k_scan_totals(int *totals, int nb, int *grand) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int run = 0;
  for (int b = 0; b < nb; ++b) {
    const int v = totals[b];
    totals[b] = run;
    run += v;
  }
  *grand = run;
}

__global__ void k_scan_add(int *out, int n, const int *totals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += totals[i / 1024];
}

__global__ void k_bin_scatter(const int *key, int64_t n, const int *start, int *cursor, int *perm_tmp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = key[i];
  const int pos = start[c] + atomicAdd(&cursor[c], 1);
  perm_tmp[pos] = (int)i;
}

// Deterministic order inside each cell: rank of each original index among the
// cell's indices (indices are distinct, so the ranks are a permutation).
__global__ void k_bin_rank(const int *start, int ncell, const int *perm_tmp, int *perm) {
  const int c = blockIdx.x;
  if (c >= ncell) return;
  const int s0 = start[c], s1 = start[c + 1], m = s1 - s0;
  if (m == 0) return;
  __shared__ int idx[2048];
  const bool in_smem = m <= 2048;
  if (in_smem)
    for (int e = threadIdx.x; e < m; e += blockDim.x) idx[e] = perm_tmp[s0 + e];
  __syncthreads();
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const int me = in_smem ? idx[e] : perm_tmp[s0 + e];
    int r = 0;
    for (int j = 0; j < m; ++j) r += ((in_smem ? idx[j] : perm_tmp[s0 + j]) < me) ? 1 : 0;
    perm[s0 + r] = me;
  }
}

// Gather by perm and transpose the values: FT64[d][i] = F[perm[i]][d].
__global__ void k_gather_transpose(const double *xy, const double *F, int64_t n, int D, const int *perm,
                                   double *x64, double *y64, double *FT64) {
  __shared__ double tile[32][33];
  const int64_t i0 = blockIdx.x * 32ll;
  const int d0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k;
    const int d = d0 + threadIdx.x;
    if (i < n && d < D) {
      const int64_t src = perm ? perm[i] : i;
      tile[k][threadIdx.x] = F[src * D + d];
    }
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int d = d0 + k;
    const int64_t i = i0 + threadIdx.x;
    if (i < n && d < D) FT64[(int64_t)d * n + i] = tile[threadIdx.x][k];
  }
  if (blockIdx.y == 0 && threadIdx.y == 0) {
    const int64_t i = i0 + threadIdx.x;
    if (i < n) {
      const int64_t src = perm ? perm[i] : i;
      x64[i] = xy[2 * src];
      y64[i] = xy[2 * src + 1];
    }
  }
}

// FP32 layouts: scaled positions and normalised values (f - cen) / scl,
// zero padded, dimension-major [D_pad][n_pad]; for the reduced precisions
// the same values point-major [n_pad][D] as hi + lo floats as well (the
// hand-over paths read all dimensions of one point at a time).  A block
// takes 32 points x 32 dimensions: the dimension-major reads and writes are
// coalesced along the points, the point-major writes along the dimensions
// through a transpose in shared memory.  The block forms 1/scl once per
// dimension (GB300's FP64 divisions are slow: one per value bound the
// kernel).
__global__ void k_finish(const double *x64, const double *y64, const double *FT64, int64_t n, int64_t n_pad,
                         int D, int D_pad, double ctr_x, double ctr_y, double inv_s, const double *cen,
                         const double *scl, float *xs, float *ys, float *FT32, float *xs_lo, float *ys_lo,
                         float *FR32, float *FR32lo) {
  __shared__ double tile[32][33];
  __shared__ double s_cen[32], s_rs[32];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int d0 = blockIdx.y * 32;
  const int tx = threadIdx.x;
  if (threadIdx.y == 0) {
    const int d = d0 + tx;
    s_cen[tx] = d < D ? cen[d] : 0.0;
    s_rs[tx] = d < D ? 1.0 / scl[d] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {   // tile rows: dimensions
    const int d = d0 + k;
    const int64_t i = i0 + tx;
    double v = 0.0;
    if (d < D && i < n) v = (FT64[(int64_t)d * n + i] - s_cen[k]) * s_rs[k];
    if (d < D_pad && i < n_pad) FT32[(int64_t)d * n_pad + i] = (float)v;
    tile[k][tx] = v;
  }
  if (blockIdx.y == 0 && threadIdx.y == 0) {
    const int64_t i = i0 + tx;
    if (i < n_pad) {
      const double X = (i < n) ? (x64[i] - ctr_x) * inv_s : 0.0;
      const double Y = (i < n) ? (y64[i] - ctr_y) * inv_s : 0.0;
      xs[i] = (float)X;
      ys[i] = (float)Y;
      xs_lo[i] = (float)(X - (double)(float)X);
      ys_lo[i] = (float)(Y - (double)(float)Y);
    }
  }
  if (FR32) {
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {   // tile rows: points
      const int64_t i = i0 + k;
      const int d = d0 + tx;
      if (i < n_pad && d < D) {
        const double v = tile[tx][k];
        const float h = (float)v;
        FR32[i * D + d] = h;
        FR32lo[i * D + d] = (float)(v - (double)h);
      }
    }
  }
}

// Point-blocked copies for the tensor path: positions as (x[8], y[8], 4 pad)
// per block of 8 points, values per pass of dc dimensions as
// [block][dc * 8 + 4 pad].  The 16-byte pad per block spreads the blocks of a
// staged tile over the shared-memory banks (the operand builders read 8
// blocks at once).
__global__ void k_block(const float *xs, const float *ys, const float *FT32, int64_t n_pad, int D, int dc,
                        int passes, float *xyb, float *fb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const int64_t b = i >> 3;
  const int j = (int)(i & 7);
  const int64_t fstride = (int64_t)dc * 8 + 4;
  const int64_t nblk = n_pad >> 3;
  // grid row 0: the positions; row 1 + pass dc + dd: value column dd of pass
  // `pass` (one column per grid row, so that small point sets still fill
  // the GPU)
  for (int y = blockIdx.y; y < 1 + passes * dc; y += gridDim.y) {
    if (y == 0) {
      xyb[b * 20 + j] = xs[i];
      xyb[b * 20 + 8 + j] = ys[i];
      if (j < 4) xyb[b * 20 + 16 + j] = 0.f;
    } else {
      const int pass = (y - 1) / dc, dd = (y - 1) % dc;
      const int d = pass * dc + dd;
      float *blk = fb + (pass * nblk + b) * fstride;
      blk[dd * 8 + j] = (d < D) ? FT32[(int64_t)d * n_pad + i] : 0.f;
      if (dd == 0 && j < 4) blk[dc * 8 + j] = 0.f;
    }
  }
}

}  // namespace

// Offsets of the arrays carved out of one device block (each 256-byte
// aligned): a handle's arrays cost one stream-ordered allocation instead of
// one each (every allocation is a driver call on the host, and create's host
// time is device idle time after its one wait for the point ranges).
struct Carve {
  size_t bytes = 0;
  size_t add(size_t nbytes) {
    const size_t o = bytes;
    bytes += (nbytes + 255) / 256 * 256;
    return o;
  }
};

mls_status prep_points(mls_handle *h, const double *xy, const double *F, cudaStream_t st) {
  PointSet &P = h->P;
  const mls_desc &d = h->desc;
  P.n = d.n;
  P.D = d.D;
  P.n_pad = (d.n + kPointPad - 1) / kPointPad * kPointPad;
  P.D_pad = (d.D + 15) / 16 * 16;
  P.s = d.h;
  const int64_t n = P.n;
  const int D = P.D;

  // --- one block for the range keys and every array whose size depends
  // only on n and D
  const bool binned = d.weight != MLS_W_INVDIST;
  const bool blocked = d.precision == MLS_P_FP16 || d.precision == MLS_P_BF16;
  int dc = 0, passes = 0;
  if (blocked) {
    dc = tc_dims_per_pass(D, d.degree);
    passes = (D + dc - 1) / dc;
    P.fb_dc = dc;
  }
  Carve cv;
  const size_t o_keys = cv.add(sizeof(unsigned long long) * 2 * (D + 2));
  const size_t o_x64 = cv.add(sizeof(double) * n), o_y64 = cv.add(sizeof(double) * n);
  const size_t o_FT64 = cv.add(sizeof(double) * n * D);
  const size_t o_xs = cv.add(sizeof(float) * P.n_pad), o_ys = cv.add(sizeof(float) * P.n_pad);
  const size_t o_xs_lo = cv.add(sizeof(float) * P.n_pad), o_ys_lo = cv.add(sizeof(float) * P.n_pad);
  const size_t o_FT32 = cv.add(sizeof(float) * P.n_pad * P.D_pad);
  const size_t o_FR32 = d.precision != MLS_P_FP64 ? cv.add(sizeof(float) * P.n_pad * D) : 0;
  const size_t o_FR32lo = d.precision != MLS_P_FP64 ? cv.add(sizeof(float) * P.n_pad * D) : 0;
  const size_t o_fcen = cv.add(sizeof(double) * D), o_fscl = cv.add(sizeof(double) * D);
  const size_t o_fcen32 = cv.add(sizeof(float) * D), o_fscl32 = cv.add(sizeof(float) * D);
  const size_t o_key = binned ? cv.add(sizeof(int) * n) : 0;
  const size_t o_perm_tmp = binned ? cv.add(sizeof(int) * n) : 0;
  const size_t o_perm = binned ? cv.add(sizeof(int) * n) : 0;
  const size_t o_xyb = blocked ? cv.add(sizeof(float) * (P.n_pad / 8) * 20) : 0;
  const size_t o_fb = blocked ? cv.add(sizeof(float) * (P.n_pad / 8) * ((size_t)dc * 8 + 4) * passes) : 0;
  mls_status ms;
  char *blk = nullptr;
  if ((ms = dev_alloc(h, (void **)&blk, cv.bytes, st)) != MLS_OK) return ms;
  unsigned long long *keys = (unsigned long long *)(blk + o_keys);
  P.x64 = (double *)(blk + o_x64);
  P.y64 = (double *)(blk + o_y64);
  P.FT64 = (double *)(blk + o_FT64);
  P.xs = (float *)(blk + o_xs);
  P.ys = (float *)(blk + o_ys);
  P.xs_lo = (float *)(blk + o_xs_lo);
  P.ys_lo = (float *)(blk + o_ys_lo);
  P.FT32 = (float *)(blk + o_FT32);
  if (d.precision != MLS_P_FP64) {
    P.FR32 = (float *)(blk + o_FR32);
    P.FR32lo = (float *)(blk + o_FR32lo);
  }
  P.fcen = (double *)(blk + o_fcen);
  P.fscl = (double *)(blk + o_fscl);
  P.fcen32 = (float *)(blk + o_fcen32);
  P.fscl32 = (float *)(blk + o_fscl32);
  int *perm = binned ? (int *)(blk + o_perm) : nullptr;
  int *key = binned ? (int *)(blk + o_key) : nullptr;
  int *perm_tmp = binned ? (int *)(blk + o_perm_tmp) : nullptr;
  if (blocked) {
    P.xyb = (float *)(blk + o_xyb);
    P.fb = (float *)(blk + o_fb);
  }

  // --- ranges of x, y and every value column
  k_init_keys<<<(2 * (D + 2) + 255) / 256, 256, 0, st>>>(keys, D + 2);
  ++h->launches;
  {
    const int64_t tot = n * 2;
    const int grid = (int)std::min<int64_t>((tot + 255) / 256, 1216);
    k_colminmax<<<grid, 256, 2 * 2 * sizeof(unsigned long long), st>>>(xy, n, 2, keys, keys + D + 2);
    ++h->launches;
    const int64_t totF = n * D;
    const int gridF = (int)std::min<int64_t>((totF + 255) / 256, 1216);
    k_colminmax<<<gridF, 256, 2 * D * sizeof(unsigned long long), st>>>(F, n, D, keys + 2, keys + D + 4);
    ++h->launches;
  }
  MLS_CUDA_TRY(cudaGetLastError());

  // --- the value frames, formed on the device while the host waits for
  // the ranges below (only the bounding box and the grid need them there)
  k_value_frames<<<(D + 127) / 128, 128, 0, st>>>(keys + 2, keys + D + 4, D, P.fcen, P.fscl, P.fcen32, P.fscl32);
  ++h->launches;
  MLS_CUDA_TRY(cudaGetLastError());
  // --- the ranges on the host: finiteness, the bounding box and the grid
  std::vector<unsigned long long> hk(2 * (D + 2));
  MLS_CUDA_TRY(cudaMemcpyAsync(hk.data(), keys, hk.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  MLS_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> lo(D + 2), hi(D + 2);
  for (int c = 0; c < D + 2; ++c) {
    lo[c] = host_from_key(hk[c]);
    hi[c] = host_from_key(hk[D + 2 + c]);
    if (!std::isfinite(lo[c]) || !std::isfinite(hi[c]))
      return fail(MLS_E_INVAL, "points and values must be finite");
  }
  P.bbox[0] = lo[0];
  P.bbox[1] = lo[1];
  P.bbox[2] = hi[0];
  P.bbox[3] = hi[1];
  P.ctr_x = 0.5 * (lo[0] + hi[0]);
  P.ctr_y = 0.5 * (lo[1] + hi[1]);

  // --- binning for the compact-support weight, and for the Gaussian (the
  // hand-over path visits only the cells within its cut radius; the full-sum
  // kernels read every point and do not depend on the order)
  if (binned) {
    // cells of h; for the Wendland weight h/2: a tile and the pixels it
    // holds visit the cells within h of them, and half-size cells follow
    // the union of their support discs more closely (fewer zero weights)
    double cell = d.weight == MLS_W_WENDLAND ? 0.5 * d.h : d.h;
    const double ex = hi[0] - lo[0], ey = hi[1] - lo[1];
    // keep the grid below 16M cells
    while ((floor(ex / cell) + 1) * (floor(ey / cell) + 1) > 16.0e6) cell *= 2.0;
    P.cell = cell;
    P.gx0 = lo[0];
    P.gy0 = lo[1];
    P.gx = (int)floor(ex / cell) + 1;
    P.gy = (int)floor(ey / cell) + 1;
    const int ncell = P.gx * P.gy;
    const int nb = (ncell + 1 + 1023) / 1024;
    Carve cc;
    const size_t o_start = cc.add(sizeof(int) * (ncell + 1)), o_counts = cc.add(sizeof(int) * (ncell + 1));
    const size_t o_cursor = cc.add(sizeof(int) * ncell), o_totals = cc.add(sizeof(int) * nb);
    const size_t o_grand = cc.add(sizeof(int));
    char *cb = nullptr;
    if ((ms = dev_alloc(h, (void **)&cb, cc.bytes, st)) != MLS_OK) return ms;
    P.cell_start = (int *)(cb + o_start);
    int *counts = (int *)(cb + o_counts), *cursor = (int *)(cb + o_cursor);
    int *totals = (int *)(cb + o_totals), *grand = (int *)(cb + o_grand);
    MLS_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (ncell + 1), st));
    MLS_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, st));
    const int nbk = (int)((n + 255) / 256);
    k_bin_count<<<nbk, 256, 0, st>>>(xy, n, P.gx0, P.gy0, 1.0 / P.cell, P.gx, P.gy, key, counts);
    ++h->launches;
    k_scan_blocks<<<nb, 512, 0, st>>>(counts, ncell + 1, P.cell_start, totals);
    ++h->launches;
    k_scan_totals<<<1, 32, 0, st>>>(totals, nb, grand);
    ++h->launches;
    k_scan_add<<<(ncell + 1 + 255) / 256, 256, 0, st>>>(P.cell_start, ncell + 1, totals);
    ++h->launches;
    k_bin_scatter<<<nbk, 256, 0, st>>>(key, n, P.cell_start, cursor, perm_tmp);
    ++h->launches;
    k_bin_rank<<<ncell, 128, 0, st>>>(P.cell_start, ncell, perm_tmp, perm);
    ++h->launches;
    MLS_CUDA_TRY(cudaGetLastError());
  }

  // --- gather / transpose / normalise
  {
    dim3 g((unsigned)((n + 31) / 32), (unsigned)((D + 31) / 32));
    k_gather_transpose<<<g, dim3(32, 8), 0, st>>>(xy, F, n, D, perm, P.x64, P.y64, P.FT64);
    ++h->launches;
    dim3 g2((unsigned)((P.n_pad + 31) / 32), (unsigned)((P.D_pad + 31) / 32));
    k_finish<<<g2, dim3(32, 8), 0, st>>>(P.x64, P.y64, P.FT64, n, P.n_pad, D, P.D_pad, P.ctr_x, P.ctr_y,
                                         1.0 / P.s, P.fcen, P.fscl, P.xs, P.ys, P.FT32, P.xs_lo, P.ys_lo, P.FR32,
                                         P.FR32lo);
    ++h->launches;
    MLS_CUDA_TRY(cudaGetLastError());
  }
  if (blocked) {
    const int rows = 1 + passes * dc;
    dim3 g3((unsigned)((P.n_pad + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
    k_block<<<g3, 256, 0, st>>>(P.xs, P.ys, P.FT32, P.n_pad, D, dc, passes, P.xyb, P.fb);
    ++h->launches;
    MLS_CUDA_TRY(cudaGetLastError());
  }
  return MLS_OK;
}

}  // namespace mlsi
