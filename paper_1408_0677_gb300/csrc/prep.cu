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

__global__ void k_fill_u64(unsigned long long *p, int n, unsigned long long v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
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

// FP32 layouts: scaled positions and normalised values, zero padded;
// optionally the values point-major as well.
__global__ void k_finish(const double *x64, const double *y64, const double *FT64, int64_t n, int64_t n_pad,
                         int D, int D_pad, double ctr_x, double ctr_y, double inv_s, const double *cen,
                         const double *scl, float *xs, float *ys, float *FT32, float *xs_lo, float *ys_lo,
                         float *FR32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (i >= n_pad) return;
  float v = 0.f;
  if (d < D && i < n) v = (float)((FT64[(int64_t)d * n + i] - cen[d]) / scl[d]);
  FT32[(int64_t)d * n_pad + i] = v;
  if (FR32 && d < D) FR32[i * D + d] = v;
  if (d == 0) {
    const double X = (i < n) ? (x64[i] - ctr_x) * inv_s : 0.0;
    const double Y = (i < n) ? (y64[i] - ctr_y) * inv_s : 0.0;
    xs[i] = (float)X;
    ys[i] = (float)Y;
    xs_lo[i] = (float)(X - (double)(float)X);
    ys_lo[i] = (float)(Y - (double)(float)Y);
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
  if (blockIdx.y == 0) {
    xyb[b * 20 + j] = xs[i];
    xyb[b * 20 + 8 + j] = ys[i];
    if (j < 4) xyb[b * 20 + 16 + j] = 0.f;
  }
  const int64_t nblk = n_pad >> 3;
  for (int pass = blockIdx.y; pass < passes; pass += gridDim.y) {
    float *blk = fb + (pass * nblk + b) * fstride;
    for (int dd = 0; dd < dc; ++dd) {
      const int d = pass * dc + dd;
      blk[dd * 8 + j] = (d < D) ? FT32[(int64_t)d * n_pad + i] : 0.f;
    }
    if (j < 4) blk[dc * 8 + j] = 0.f;
  }
}

}  // namespace

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

  // --- ranges of x, y and every value column
  unsigned long long *keys = nullptr;
  mls_status ms;
  if ((ms = dev_alloc(h, (void **)&keys, sizeof(unsigned long long) * 2 * (D + 2), st)) != MLS_OK) return ms;
  k_fill_u64<<<(D + 2 + 255) / 256, 256, 0, st>>>(keys, D + 2, ~0ull);
  ++h->launches;
  k_fill_u64<<<(D + 2 + 255) / 256, 256, 0, st>>>(keys + D + 2, D + 2, 0ull);
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
  std::vector<double> cen(D), scl(D);
  std::vector<float> cen32(D), scl32(D);
  for (int c = 0; c < D; ++c) {
    cen[c] = 0.5 * (lo[c + 2] + hi[c + 2]);
    scl[c] = 0.5 * (hi[c + 2] - lo[c + 2]);
    if (!(scl[c] > 0.0)) scl[c] = 1.0;
    cen32[c] = (float)cen[c];
    scl32[c] = (float)scl[c];
  }

  // --- device arrays
  void *p;
#define ALLOC(ptr, bytes)                                                   \
  do {                                                                      \
    if ((ms = dev_alloc(h, &p, (bytes), st)) != MLS_OK) return ms;          \
    ptr = (decltype(ptr))p;                                                 \
  } while (0)
  ALLOC(P.x64, sizeof(double) * n);
  ALLOC(P.y64, sizeof(double) * n);
  ALLOC(P.FT64, sizeof(double) * n * D);
  ALLOC(P.xs, sizeof(float) * P.n_pad);
  ALLOC(P.ys, sizeof(float) * P.n_pad);
  ALLOC(P.xs_lo, sizeof(float) * P.n_pad);
  ALLOC(P.ys_lo, sizeof(float) * P.n_pad);
  ALLOC(P.FT32, sizeof(float) * P.n_pad * P.D_pad);
  if (d.precision != MLS_P_FP64) ALLOC(P.FR32, sizeof(float) * P.n_pad * D);
  ALLOC(P.fcen, sizeof(double) * D);
  ALLOC(P.fscl, sizeof(double) * D);
  ALLOC(P.fcen32, sizeof(float) * D);
  ALLOC(P.fscl32, sizeof(float) * D);
  MLS_CUDA_TRY(cudaMemcpyAsync(P.fcen, cen.data(), sizeof(double) * D, cudaMemcpyHostToDevice, st));
  MLS_CUDA_TRY(cudaMemcpyAsync(P.fscl, scl.data(), sizeof(double) * D, cudaMemcpyHostToDevice, st));
  MLS_CUDA_TRY(cudaMemcpyAsync(P.fcen32, cen32.data(), sizeof(float) * D, cudaMemcpyHostToDevice, st));
  MLS_CUDA_TRY(cudaMemcpyAsync(P.fscl32, scl32.data(), sizeof(float) * D, cudaMemcpyHostToDevice, st));

  // --- binning for the compact-support weight
  int *perm = nullptr;
  // binning for the compact-support weight, and for the Gaussian (the
  // hand-over path visits only the cells within its cut radius; the full-sum
  // kernels read every point and do not depend on the order)
  if (d.weight != MLS_W_INVDIST) {
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
    int *key, *counts, *cursor, *perm_tmp, *totals, *grand;
    const int nb = (ncell + 1 + 1023) / 1024;
    ALLOC(P.cell_start, sizeof(int) * (ncell + 1));
    ALLOC(key, sizeof(int) * n);
    ALLOC(counts, sizeof(int) * (ncell + 1));
    ALLOC(cursor, sizeof(int) * ncell);
    ALLOC(perm_tmp, sizeof(int) * n);
    ALLOC(perm, sizeof(int) * n);
    ALLOC(totals, sizeof(int) * nb);
    ALLOC(grand, sizeof(int));
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
    dim3 g2((unsigned)((P.n_pad + 255) / 256), (unsigned)P.D_pad);
    k_finish<<<g2, 256, 0, st>>>(P.x64, P.y64, P.FT64, n, P.n_pad, D, P.D_pad, P.ctr_x, P.ctr_y, 1.0 / P.s,
                                 P.fcen, P.fscl, P.xs, P.ys, P.FT32, P.xs_lo, P.ys_lo, P.FR32);
    ++h->launches;
    MLS_CUDA_TRY(cudaGetLastError());
  }
  if (d.precision == MLS_P_FP16 || d.precision == MLS_P_BF16) {
    const int dc = tc_dims_per_pass(D, d.degree);
    const int passes = (D + dc - 1) / dc;
    P.fb_dc = dc;
    ALLOC(P.xyb, sizeof(float) * (P.n_pad / 8) * 20);
    ALLOC(P.fb, sizeof(float) * (P.n_pad / 8) * ((size_t)dc * 8 + 4) * passes);
    dim3 g3((unsigned)((P.n_pad + 255) / 256), (unsigned)(passes < 8 ? passes : 8));
    k_block<<<g3, 256, 0, st>>>(P.xs, P.ys, P.FT32, P.n_pad, D, dc, passes, P.xyb, P.fb);
    ++h->launches;
    MLS_CUDA_TRY(cudaGetLastError());
  }
#undef ALLOC
  return MLS_OK;
}

}  // namespace mlsi
