// Allocation-free Gershgorin bounds: gsp2_bounds_noalloc.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool, a plugin that must not grow the process's device
// footprint, or a library whose users forbid allocation after start-up.  For them
// this entry point computes the spectral bounds of a CSR matrix with its scratch
// (one partial per block plus a ticket counter) in a fixed file-scope device array,
// so the call allocates nothing.  The caller still passes the inputs and the output.
//
// The array is `kMaxBlocks` partials of 16 bytes plus a counter (about 64 KB); every
// GPU that loads the library holds it until the process exits.  Rows are handled in
// blocks of 256, so at most kMaxBlocks * 256 rows are accepted.
#include <mutex>

#include "../../include/gsp2.h"
#include "gsp2_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerBlock = 256;  // 8 warps x 32 rows
constexpr int kMaxBlocks = 4096;
constexpr int kMaxDevices = 64;

struct NoallocScratch {
  double2 slots[kMaxBlocks];
  unsigned int counter;
};

// Shared by every call on a device; a call leaves its partials behind.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// min / max that return NaN when either operand is NaN (fmin and fmax return the other
// operand), so that a NaN in the matrix, or an Inf - Inf radius, reaches the bounds
__device__ __forceinline__ double nan_min(double a, double b) { return (a != a || b != b) ? NAN : fmin(a, b); }
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }

// Same per-row arithmetic as the bounds step of gsp2_density (one warp per row,
// lanes striding over the row), with the scratch passed in explicitly.
__global__ void __launch_bounds__(kThreads) bounds_noalloc_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ colind,
                                                                  const double* __restrict__ vals,
                                                                  double* __restrict__ out,
                                                                  NoallocScratch* scratch) {
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  double lo = INFINITY, hi = -INFINITY;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock + (int64_t)w * 32;
  for (int64_t i = r0; i < r0 + 32 && i < n; ++i) {
    double rad = 0.0, dia = 0.0;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
      const double v = vals[p];
      if (colind[p] == i) dia = v; else rad += fabs(v);
    }
    rad = gsp2::warp_sum(rad);
    dia = gsp2::warp_sum(dia);
    lo = nan_min(lo, dia - rad);
    hi = nan_max(hi, dia + rad);
  }
  __shared__ double s_lo[kThreads / 32], s_hi[kThreads / 32];
  if (lane == 0) { s_lo[w] = lo; s_hi[w] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kThreads / 32; ++k) { lo = nan_min(lo, s_lo[k]); hi = nan_max(hi, s_hi[k]); }
    scratch->slots[blockIdx.x] = make_double2(lo, hi);
  }
  if (gsp2::last_block_ticket(&scratch->counter)) {
    if (threadIdx.x == 0) {
      double a = INFINITY, b = -INFINITY;
      for (unsigned int k = 0; k < gridDim.x; ++k) {
        a = nan_min(a, gsp2::ld_cg(&scratch->slots[k].x));
        b = nan_max(b, gsp2::ld_cg(&scratch->slots[k].y));
      }
      out[0] = a;
      out[1] = b;
      scratch->counter = 0;
    }
  }
}

std::mutex g_addr_mutex;
NoallocScratch* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" gsp2_status gsp2_bounds_noalloc(int64_t n, const int64_t* d_rowptr, const int32_t* d_colind,
                                           const double* d_vals, double* d_bounds, void* stream) {
  if (n < 1 || n > (int64_t)kMaxBlocks * kRowsPerBlock) return GSP2_E_ARG;
  if (!d_rowptr || !d_colind || !d_vals || !d_bounds) return GSP2_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSP2_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  NoallocScratch* scratch = nullptr;
  {
    // The host-side name of the array is not a device address: its address on this device
    // is looked up with the device current.  Outside a stream capture the lookup is
    // repeated on every call (it allocates nothing), so a context re-created after
    // cudaDeviceReset is picked up; inside a capture the address found by an earlier call
    // on this device is used, so the first call on a device must come before any capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return GSP2_E_CUDA;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GSP2_E_CUDA;
      g_addr[dev] = static_cast<NoallocScratch*>(p);
    }
    scratch = g_addr[dev];
    if (!scratch) return GSP2_E_CUDA;
  }
  // the ticket counter must start at zero; the partials are overwritten
  if (cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned int), s) != cudaSuccess) return GSP2_E_CUDA;
  const int blocks = (int)((n + kRowsPerBlock - 1) / kRowsPerBlock);
  bounds_noalloc_kernel<<<blocks, kThreads, 0, s>>>(n, d_rowptr, d_colind, d_vals, d_bounds, scratch);
  return cudaGetLastError() == cudaSuccess ? GSP2_OK : GSP2_E_CUDA;
}
