// Float64 Krylov kernels for FGMRES (Sec. 4.2.4): block dot products against
// the Arnoldi basis, multi-axpy updates, norms and type casts.
//
// Reductions are deterministic: a fixed grid of RB blocks walks the vector
// with a grid stride, each block reduces its partial sums in shared memory
// in a fixed order, and one block adds the RB partials in block order.
#include <algorithm>

#include "internal.h"

namespace wsi {

static constexpr int RB = 152 * 4;  // reduction blocks (4 per SM)
static constexpr int RT = 256;      // threads per reduction block
static constexpr int NV = 8;        // basis vectors per pass

template <int M>
__global__ void k_mdot(const double* __restrict__ V, size_t ldv, int m, const double* __restrict__ w, size_t n,
                       double* part) {
  double acc[M];
#pragma unroll
  for (int t = 0; t < M; ++t) acc[t] = 0.0;
  // four independent elements per iteration keep enough loads in flight
  // to cover HBM latency
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
    double wi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) wi[u] = (i + u * stride < n) ? w[i + u * stride] : 0.0;
#pragma unroll
    for (int t = 0; t < M; ++t)
      if (t < m) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i + u * stride < n) acc[t] += V[(size_t)t * ldv + i + u * stride] * wi[u];
      }
  }
  __shared__ double sh[RT / 32][M];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < M; ++t) {
    double v = acc[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double s = 0.0;
    for (int q = 0; q < RT / 32; ++q) s += sh[q][threadIdx.x];
    part[(size_t)blockIdx.x * M + threadIdx.x] = s;
  }
}

// one block per output t < m: the block's threads stride over the nblocks
// partials in a fixed pattern and combine them with a fixed tree
__global__ void k_reduce_parts(const double* __restrict__ part, int nblocks, int M, int m, double* out) {
  int t = blockIdx.x;
  if (t >= m) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(size_t)b * M + t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double sh[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sh[q];
    out[t] = a;
  }
}

void launch_mdot(const double* V, size_t ldv, int m, const double* w, size_t n, double* out, double* scratch,
                 cudaStream_t st) {
  for (int t0 = 0; t0 < m; t0 += NV) {
    int mm = std::min(NV, m - t0);
    ktimer_begin(KC_MDOT, st);
    // each distinct array read once: w is often the last basis row itself
    const bool w_in_v = w == V + (size_t)(t0 + mm - 1) * ldv;
    ktimer_bytes(KC_MDOT, 8.0 * (double)n * (mm + (w_in_v ? 0 : 1)));
    { k_mdot<NV><<<RB, RT, 0, st>>>(V + (size_t)t0 * ldv, ldv, mm, w, n, scratch); WSI_COUNT(); }
    ktimer_end(KC_MDOT, st);
    { k_reduce_parts<<<mm, 256, 0, st>>>(scratch, RB, NV, mm, out + t0); WSI_COUNT(); }
  }
}

// w = (w - sign * sum_t h[t] V_t) * scale[0]   (scale may be null: 1)
__global__ void k_maxpy(const double* __restrict__ V, size_t ldv, int m, const double* __restrict__ h, double* w,
                        size_t n, double sign, const double* __restrict__ scale) {
  __shared__ double hs[64];
  if (threadIdx.x < m && threadIdx.x < 64) hs[threadIdx.x] = sign * h[threadIdx.x];
  __syncthreads();
  const double f = scale ? scale[0] : 1.0;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
    double s[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] = (i + u * stride < n) ? w[i + u * stride] : 0.0;
    for (int t = 0; t < m; ++t) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u * stride < n) s[u] -= hs[t] * V[(size_t)t * ldv + i + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i + u * stride < n) w[i + u * stride] = scale ? s[u] * f : s[u];
  }
}

void launch_maxpy(const double* V, size_t ldv, int m, const double* h, double* w, size_t n, double sign,
                  cudaStream_t st, const double* scale_dev) {
  for (int t0 = 0; t0 < m; t0 += 64) {
    int mm = std::min(64, m - t0);
    const double* sc = (t0 + 64 >= m) ? scale_dev : nullptr;
    ktimer_begin(KC_MAXPY, st);
    ktimer_bytes(KC_MAXPY, 8.0 * (double)n * (mm + 2));  // mm rows and w read, w written
    { k_maxpy<<<RB, RT, 0, st>>>(V + (size_t)t0 * ldv, ldv, mm, h + t0, w, n, sign, sc); WSI_COUNT(); }
    ktimer_end(KC_MAXPY, st);
  }
}

__global__ void k_scale(double* x, size_t n, const double* __restrict__ s, bool inverse) {
  double f = inverse ? 1.0 / s[0] : s[0];
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] *= f;
}

void launch_scale(double* x, size_t n, const double* s_dev, bool inverse, cudaStream_t st) {
  { k_scale<<<RB, RT, 0, st>>>(x, n, s_dev, inverse); WSI_COUNT(); }
}

template <typename T>
__global__ void k_sum(const T* __restrict__ x, size_t n, double* part) {
  double acc = 0.0;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc += cvt<double, T>(x[i]);
  __shared__ double sh[RT / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) sh[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < RT / 32; ++q) s += sh[q];
    part[blockIdx.x] = s;
  }
}

template <typename T>
void launch_sum(const T* x, size_t n, double* out_dev, double* scratch, cudaStream_t st) {
  { k_sum<T><<<RB, RT, 0, st>>>(x, n, scratch); WSI_COUNT(); }
  { k_reduce_parts<<<1, 256, 0, st>>>(scratch, RB, 1, 1, out_dev); WSI_COUNT(); }
}

double host_norm2(const double* x, size_t n, double* scratch, cudaStream_t st) {
  // scratch: RB + 1 doubles on the device
  { k_mdot<1><<<RB, RT, 0, st>>>(x, 0, 1, x, n, scratch); WSI_COUNT(); }
  { k_reduce_parts<<<1, 256, 0, st>>>(scratch, RB, 1, 1, scratch + RB); WSI_COUNT(); }
  double h = 0.0;
  cudaMemcpyAsync(&h, scratch + RB, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return sqrt(h);
}

// max |x_i|: per-block maxima, then one block over the RB partials (max is
// order-independent, so the result is exact and deterministic).  A NaN
// anywhere makes the result NaN (fmax alone would drop it and hide a blown-up
// field).
__device__ __forceinline__ double nanmax(double m, double a) { return (a != a || m != m) ? a + m : fmax(m, a); }

__global__ void k_maxabs_part(const double* __restrict__ x, size_t n, double* part) {
  double m = 0.0;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) m = nanmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = nanmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double sh[RT / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < RT / 32; ++q) a = nanmax(a, sh[q]);
    part[blockIdx.x] = a;
  }
}

__global__ void k_max_parts(const double* __restrict__ part, int nb, double* out) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = nanmax(m, part[b]);
  for (int o = 16; o > 0; o >>= 1) m = nanmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double sh[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a = nanmax(a, sh[q]);
    out[0] = a;
  }
}

double host_maxabs(const double* x, size_t n, double* scratch, cudaStream_t st) {
  // scratch: RB + 1 doubles on the device
  { k_maxabs_part<<<RB, RT, 0, st>>>(x, n, scratch); WSI_COUNT(); }
  { k_max_parts<<<1, 256, 0, st>>>(scratch, RB, scratch + RB); WSI_COUNT(); }
  double h = 0.0;
  cudaMemcpyAsync(&h, scratch + RB, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return h;
}

template <typename T>
__global__ void k_add_scalar(T* x, size_t n, const double* __restrict__ s, double factor) {
  T a = (T)(s[0] * factor);
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] += a;
}

template <typename T>
void launch_add_scalar_from(T* x, size_t n, const double* s_dev, double factor, cudaStream_t st) {
  { k_add_scalar<T><<<RB, RT, 0, st>>>(x, n, s_dev, factor); WSI_COUNT(); }
}

template void launch_sum<double>(const double*, size_t, double*, double*, cudaStream_t);
template void launch_sum<float>(const float*, size_t, double*, double*, cudaStream_t);
template void launch_add_scalar_from<double>(double*, size_t, const double*, double, cudaStream_t);
template void launch_add_scalar_from<float>(float*, size_t, const double*, double, cudaStream_t);

}  // namespace wsi
