// lbm_flux_noalloc: the mass / flux reduction of lbm_flux for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc or cudaFree at all: a serving loop or
// a host application that has handed the device's memory to its own pool (for
// example PyTorch's caching allocator) cannot get more without synchronising
// the whole device or failing, and code that runs between the steps of a
// latency-bound loop cannot afford the implicit device synchronisation of
// cudaFree.  This entry point takes the caller's PDF array and output buffer
// and keeps its only scratch, the per-block partial sums, in a fixed array
// compiled into the library.
//
// The scratch array below lives in every GPU that loads the library, for the
// life of the process (LBM_NOALLOC_MAX_BLOCKS x 2 doubles = 256 KiB).  Every
// call shares it, so calls that overlap on the GPU (on two streams, or two
// threads) race on it and must be serialised by the caller.  Each call
// rewrites the partials it reads, so nothing carries over between calls.
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_core.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_BLOCKS;

// Partial (mass, flux) of each block; see the header comment.
static __device__ __align__(256) double g_noalloc_partials[2 * kMaxBlocks];

// Device address of g_noalloc_partials, per device (host code may not use the
// symbol itself as an address).  Looked up again on every call made outside
// a stream capture, so a new context on the device (after cudaDeviceReset,
// which reloads the module) never meets a stale address; a call under
// capture uses the address of the last call on the device.
std::mutex g_mutex;
constexpr int kMaxDevices = 64;
double *g_scratch[kMaxDevices] = {nullptr};

template <class C, int AOS>
__global__ void __launch_bounds__(kThreads) k_noalloc_partials(const typename C::S *f, int64_t n, int64_t npad,
                                                                int64_t chunk, float inv_scale, double gx,
                                                                double *partials) {
  using namespace lbmk;
  // block b sums nodes [b * chunk, (b + 1) * chunk): a fixed assignment, so
  // the result depends only on n and the chunk size
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;  // the last block's chunk may be partial
  double m = 0.0, j = 0.0;
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    double rho = 0.0, jx = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const typename C::S v = AOS ? f[k * Q + i] : f[(int64_t)i * npad + k];
      const double fi = WD(i) + (double)C::dec(v, inv_scale);
      rho += fi;
      jx += CX(i) * fi;
    }
    m += rho;
    j += jx + 0.5 * rho * gx;
  }
  block_reduce_store(m, j, partials);
}

__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double *partials, int nblocks, double *out) {
  double m = 0.0, j = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    m += partials[2 * b];
    j += partials[2 * b + 1];
  }
  __shared__ double sm[kThreads / 32], sj[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    j += __shfl_xor_sync(0xffffffffu, j, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = m;
    sj[threadIdx.x >> 5] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a += sm[w];
      b += sj[w];
    }
    out[0] = a;
    out[1] = b;
  }
}

// The device address of the scratch on the current device: queried with the
// device current when the stream is not capturing (and cached), taken from
// the cache under capture (cudaErrorStreamCaptureUnsupported when no call
// outside a capture came first on this device).
cudaError_t scratch_for_current_device(cudaStream_t s, double **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = static_cast<double *>(p);
  } else if (!g_scratch[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *ptr = g_scratch[dev];
  return cudaSuccess;
}

// Nodes per block: at least LBM_NOALLOC_MIN_CHUNK, at most
// LBM_NOALLOC_MAX_BLOCKS blocks, a multiple of the block size.  A function
// of n alone, so the summation order (and the result's bits) is too.
int64_t chunk_of(int64_t n) {
  int64_t c = (n + kMaxBlocks - 1) / kMaxBlocks;
  c = (c + kThreads - 1) / kThreads * kThreads;
  return c > LBM_NOALLOC_MIN_CHUNK ? c : LBM_NOALLOC_MIN_CHUNK;
}

template <class C>
void launch(int layout, const void *f, int64_t n, int64_t npad, int64_t chunk, int nblocks, float inv_scale,
            double gx, double *scratch, double *out, cudaStream_t s) {
  const auto *fp = static_cast<const typename C::S *>(f);
  if (layout == LBM_AOS)
    k_noalloc_partials<C, 1><<<nblocks, kThreads, 0, s>>>(fp, n, npad, chunk, inv_scale, gx, scratch);
  else
    k_noalloc_partials<C, 0><<<nblocks, kThreads, 0, s>>>(fp, n, npad, chunk, inv_scale, gx, scratch);
  k_noalloc_final<<<1, kThreads, 0, s>>>(scratch, nblocks, out);
}

}  // namespace

extern "C" lbm_status lbm_flux_noalloc(const void *f_dev, int32_t precision, int32_t layout, int64_t n,
                                       int64_t npad, double f16_scale, double gx, double *out_dev,
                                       void *stream) {
  if (!f_dev || !out_dev || n < 1) return LBM_ERR_INVALID_ARG;
  if (precision < LBM_F64 || precision > LBM_F16S || (layout != LBM_SOA && layout != LBM_AOS))
    return LBM_ERR_INVALID_ARG;
  if (layout == LBM_SOA && npad < n) return LBM_ERR_INVALID_ARG;
  if (precision == LBM_F16S && !(f16_scale > 0.0)) return LBM_ERR_INVALID_ARG;
  if (n > LBM_NOALLOC_MAX_NODES) return LBM_ERR_INVALID_ARG;  // beyond the scratch
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *scratch = nullptr;
  if (scratch_for_current_device(s, &scratch) != cudaSuccess) return LBM_ERR_CUDA;
  const int64_t chunk = chunk_of(n);
  const int nblocks = (int)((n + chunk - 1) / chunk);
  const float inv = precision == LBM_F16S ? (float)(1.0 / f16_scale) : 1.0f;
  if (precision == LBM_F64)
    launch<lbmk::CodecF64>(layout, f_dev, n, npad, chunk, nblocks, inv, gx, scratch, out_dev, s);
  else if (precision == LBM_F32)
    launch<lbmk::CodecF32>(layout, f_dev, n, npad, chunk, nblocks, inv, gx, scratch, out_dev, s);
  else
    launch<lbmk::CodecF16S>(layout, f_dev, n, npad, chunk, nblocks, inv, gx, scratch, out_dev, s);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
