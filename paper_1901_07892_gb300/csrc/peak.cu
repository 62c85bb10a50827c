// Measured fused multiply-add issue rate of the current GPU (no counterpart in
// the paper): the denominator of the "alu" roofline of kernels bound by the
// float64 pipe (the plain float64 Stokes matvec) or by float32 issue (the
// double-float matvec).  Every thread runs eight independent FMA chains
// x <- x a + b in registers (0 < a < 1, so the values stay near b / (1 - a)
// and never become subnormal); one launch fills every SM with 8 blocks of 256
// threads.  Nothing is read from memory; one store that never happens for
// these inputs (the sum of the chains is compared with a negative value)
// keeps the chains live.  Clocks are not touched: the rate is whatever the
// GPU runs at during the call.
#include "internal.h"

namespace wsi {

static constexpr int PK_THREADS = 256;
static constexpr int PK_CHAINS = 8;
static constexpr int PK_UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_peak(T a, T b, int iters, T* sink) {
  T x[PK_CHAINS];
#pragma unroll
  for (int j = 0; j < PK_CHAINS; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PK_UNROLL; ++u) {
#pragma unroll
      for (int j = 0; j < PK_CHAINS; ++j) x[j] = fma(x[j], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < PK_CHAINS; ++j) s += x[j];
  if (s < (T)-1) sink[blockIdx.x] = s;  // all chains stay positive: never taken
}

// the same with packed float32 pairs (one fma.rn.f32x2 per two FMAs)
__global__ void __launch_bounds__(PK_THREADS) k_fma2_peak(float a, float b, int iters, float* sink) {
  float2 x[PK_CHAINS / 2];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int j = 0; j < PK_CHAINS / 2; ++j)
    x[j] = make_float2((float)(threadIdx.x + 2 * j) * 1e-3f, (float)(threadIdx.x + 2 * j + 1) * 1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PK_UNROLL; ++u) {
#pragma unroll
      for (int j = 0; j < PK_CHAINS / 2; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    }
  }
  float s = 0;
#pragma unroll
  for (int j = 0; j < PK_CHAINS / 2; ++j) s += x[j].x + x[j].y;
  if (s < -1.0f) sink[blockIdx.x] = s;
}

}  // namespace wsi

using namespace wsi;

extern "C" int wsi_fma_peak(int fp64, void* stream, double* gflops) {
  if (!gflops || fp64 < 0 || fp64 > 2) return WSI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WSI_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WSI_ERR_CUDA;
  const int blocks = nsm * 8;
  // about 60 ms per launch at the nominal rates (float64 ~1.3 TFLOP/s, float32 ~80)
  const int iters = fp64 == 1 ? 1000 : 40000;
  void* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * sizeof(double)) != cudaSuccess) return WSI_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(e0, st);
    if (fp64 == 1)
      k_fma_peak<double><<<blocks, PK_THREADS, 0, st>>>(0.999, 1e-3, iters, (double*)sink);
    else if (fp64 == 2)
      k_fma2_peak<<<blocks, PK_THREADS, 0, st>>>(0.999f, 1e-3f, iters, (float*)sink);
    else
      k_fma_peak<float><<<blocks, PK_THREADS, 0, st>>>(0.999f, 1e-3f, iters, (float*)sink);
    WSI_COUNT();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return WSI_ERR_CUDA;
  const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * (double)blocks * PK_THREADS;
  *gflops = flops / (best * 1e-3) / 1e9;
  return WSI_OK;
}
