// Allocation-free float64 2-norm (no counterpart in the paper; the solver's
// own reductions use context-owned scratch).
//
// For callers that must not allocate device memory once set up: a host that
// reserves the device memory up front (a pool sized at start, nothing left
// for cudaMalloc), or a time-critical loop that cannot afford cudaMalloc,
// which synchronises the device and can fail under memory pressure.  Scratch
// lives in file-scope __device__ arrays; their addresses are looked up once
// per device by cudaGetSymbolAddress on the first call, which is the set-up:
// make that first call before any stream capture begins, and serialise the
// first calls of host threads on one device.  Nothing has to start at zero:
// every block overwrites its own partial sum and the last pass overwrites the
// result.  All callers on a device share the scratch, so calls that can
// overlap (other streams, other host threads) race: serialise them.  Every
// call synchronises its stream before it returns.
#include <math.h>

#include "internal.h"

namespace wsi {

static constexpr int NA_THREADS = 256;
static constexpr int NA_PER_BLOCK = 16384;   // elements summed by one block
static constexpr int NA_MAX_PARTIALS = 8192;  // 64 KiB of partial sums
static constexpr size_t NA_MAX_N = (size_t)NA_PER_BLOCK * NA_MAX_PARTIALS;  // 2^27 elements
static constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_na_partials[NA_MAX_PARTIALS];
static __device__ __align__(256) double g_na_result[1];

// sum of squares of one block's chunk, fixed tree: deterministic
__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const double* __restrict__ x, size_t n, double* part) {
  __shared__ double sh[NA_THREADS / 32];
  const size_t base = (size_t)blockIdx.x * NA_PER_BLOCK;
  const size_t end = base + NA_PER_BLOCK < n ? base + NA_PER_BLOCK : n;
  double s = 0.0;
  for (size_t t = base + threadIdx.x; t < end; t += NA_THREADS) s = fma(x[t], x[t], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// sqrt of the sum of the partials, one block, fixed tree
__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double* __restrict__ part, int np, double* out) {
  __shared__ double sh[NA_THREADS / 32];
  double s = 0.0;
  for (int t = threadIdx.x; t < np; t += NA_THREADS) s += part[t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w];
    out[0] = sqrt(t);
  }
}

struct NaScratch {
  double* partials = nullptr;
  double* result = nullptr;
};
static NaScratch g_na_dev[NA_MAX_DEVICES];

}  // namespace wsi

using namespace wsi;

extern "C" int wsi_norm2_noalloc(const double* x, size_t n, double* out, void* stream) {
  if (!out || (n > 0 && !x)) return WSI_ERR_INVALID_ARG;
  if (n > NA_MAX_N) return WSI_ERR_INVALID_ARG;  // more than 2^27 elements: the partials would not fit
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return WSI_ERR_CUDA;
  NaScratch& S = g_na_dev[dev];
  if (!S.partials) {  // set-up, once per device: addresses of the static scratch
    double* part = nullptr;
    double* res = nullptr;
    if (cudaGetSymbolAddress((void**)&part, g_na_partials) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&res, g_na_result) != cudaSuccess)
      return WSI_ERR_CUDA;
    S.result = res;     // published before partials, which is the "set up" test above
    S.partials = part;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    *out = 0.0;
    return WSI_OK;
  }
  // x must be device (or managed) memory of the current device: a host
  // pointer or another device's memory would fault in the kernel.
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, x) != cudaSuccess) {
    (void)cudaGetLastError();  // clear the error this query just raised
    return WSI_ERR_INVALID_ARG;
  }
  if (!(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) || attr.device != dev)
    return WSI_ERR_INVALID_ARG;
  const int np = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
  // cudaLaunchKernel returns this launch's own error, so an error left by an
  // unrelated earlier call is neither reported here nor cleared
  double* part = S.partials;
  double* res = S.result;
  void* a1[] = {(void*)&x, (void*)&n, (void*)&part};
  if (cudaLaunchKernel((const void*)k_na_partial, dim3(np), dim3(NA_THREADS), a1, 0, st) != cudaSuccess)
    return WSI_ERR_CUDA;
  WSI_COUNT();
  void* a2[] = {(void*)&part, (void*)&np, (void*)&res};
  if (cudaLaunchKernel((const void*)k_na_final, dim3(1), dim3(NA_THREADS), a2, 0, st) != cudaSuccess)
    return WSI_ERR_CUDA;
  WSI_COUNT();
  if (cudaMemcpyAsync(out, S.result, sizeof(double), cudaMemcpyDefault, st) != cudaSuccess) return WSI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return WSI_ERR_CUDA;
  return WSI_OK;
}
