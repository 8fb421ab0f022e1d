// Iso-band labelling for callers that cannot allocate device memory.
//
// mls_bands needs a handle, and the handle keeps its device copy of the
// iso-levels in memory it allocates.  Some callers cannot allocate: an
// application whose device memory is owned by its own pool allocator (which
// may have reserved the free memory, so that a cudaMalloc here would fail or
// fragment it), or a frame loop that must not stall in cudaMalloc/cudaFree,
// both of which may synchronise the device.  mls_bands_noalloc takes the
// caller's field and band buffers and keeps the only memory it needs beyond
// them -- the FP64 levels and their rounded-up FP32 copies -- in a
// fixed-size array in the library's own device data segment.
//
// That array exists once per device that loads the library and stays until
// the process exits.  Every call on a device uses the same array and leaves
// its levels there; no part of it has to start at zero, because each call
// writes all of the D x L entries it reads before its kernels read them.
// Calls whose work overlaps on the GPU (different streams, or host threads
// without ordering) race on the array and may label with each other's
// levels: order them on one stream.
#include <cmath>
#include <mutex>

#include "mls_internal.h"

namespace mlsi {
namespace {

// FP64 levels, then their FP32 copies rounded up.
static __device__ __align__(256) unsigned char g_level_scratch[MLS_NOALLOC_MAX_LEVELS * (sizeof(double) + sizeof(float))];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_level_scratch on the current device.  The first call
// on a device looks it up (this loads the library's module on that device).
mls_status scratch_address(void **out) {
  int dev = -1;
  MLS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MLS_E_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_level_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(level scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MLS_OK;
}

// lev32[i] = smallest float >= lev64[i] (for a float f: f >= t exactly when f >= lev32)
__global__ void k_levels_round_up(const double *lev64, float *lev32, int cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) lev32[i] = __double2float_ru(lev64[i]);
}

}  // namespace
}  // namespace mlsi

mls_status mls_bands_noalloc(int32_t D, int32_t W, int32_t H, const void *field, int32_t field_fp64,
                             const double *levels, int32_t L, uint8_t *bands, void *stream) {
  using namespace mlsi;
  if (D < 1 || W < 1 || H < 1) return fail(MLS_E_INVAL, "D, W and H must be >= 1");
  if ((int64_t)W * H > (int64_t)1 << 30) return fail(MLS_E_INVAL, "more than 2^30 pixels");
  if (L < 1 || L > 254) return fail(MLS_E_INVAL, "L must be in [1, 254]");
  if ((int64_t)D * L > MLS_NOALLOC_MAX_LEVELS)
    return fail(MLS_E_INVAL, "D * L = " + std::to_string((int64_t)D * L) +
                                 " exceeds the static level storage of mls_bands_noalloc (" +
                                 std::to_string(MLS_NOALLOC_MAX_LEVELS) + " levels); use mls_bands");
  if (!field || !bands || !levels) return fail(MLS_E_INVAL, "field, levels and bands must not be NULL");
  if (field_fp64 != 0 && field_fp64 != 1) return fail(MLS_E_INVAL, "field_fp64 must be 0 or 1");
  for (int d = 0; d < D; ++d) {
    for (int j = 0; j < L; ++j) {
      const double t = levels[(size_t)d * L + j];
      if (!std::isfinite(t)) return fail(MLS_E_INVAL, "levels must be finite");
      if (j > 0 && !(t >= levels[(size_t)d * L + j - 1])) return fail(MLS_E_INVAL, "levels must ascend");
    }
  }
  void *base = nullptr;
  mls_status s = scratch_address(&base);
  if (s != MLS_OK) return s;
  const int cnt = D * L;
  double *lev64 = (double *)base;
  float *lev32 = (float *)((unsigned char *)base + (size_t)MLS_NOALLOC_MAX_LEVELS * sizeof(double));
  cudaStream_t st = (cudaStream_t)stream;
  // from pageable memory the copy has taken the levels when the call
  // returns; page-locked levels are read when the stream reaches the copy
  MLS_CUDA_TRY(cudaMemcpyAsync(lev64, levels, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
  k_levels_round_up<<<(cnt + 255) / 256, 256, 0, st>>>(lev64, lev32, cnt);
  MLS_CUDA_TRY(cudaGetLastError());
  mlsk::KParams p{};
  p.D = D;
  p.W = W;
  p.H = H;
  p.L = L;
  p.field = (void *)field;
  p.field_fp64 = field_fp64;
  p.bands = bands;
  p.lev64 = lev64;
  p.lev32 = lev32;
  launch_bands(p, field_fp64 != 0, st);
  MLS_CUDA_TRY(cudaGetLastError());
  return MLS_OK;
}
