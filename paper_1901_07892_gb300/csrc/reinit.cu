// Reinitialisation of the flow level set (Sec. 4.1, the eikonal equation
// d phi/d tau + sgn(phi~)(|grad phi| - 1) = 0 marched to steady state).
//
// Per pseudo-time stage every cell evaluates, along each axis with more than
// one cell, the second-order ENO one-sided differences of phi; where phi~
// changes sign towards a neighbour the difference is taken across the
// interface instead (subcell fix of Min 2010: the interface sits at the zero
// of the quadratic through phi~ with the minmod second difference, and phi
// is 0 there).  The Godunov Hamiltonian of sgn(phi~) gives |grad phi|; the
// local step is cfl * min(h, subcell distances).  Two stages form one TVD
// Runge-Kutta step.  sgn(phi~) and the subcell distances come from phi~
// throughout (immobile interface, Son 2005).  Neumann mirror ghosts.
//
// Layout: one thread per (x, y) column, marching a z-chunk; per z-plane the
// block's tile of phi with a two-cell halo is staged in shared memory (ghosts
// mirrored while staging), the z taps come from a five-entry register window,
// and the loads of the next plane are in flight while a plane is computed.
// phi~ enters through a one-byte code per cell (its sign and the axes along
// which it changes sign), made once per call; its values are read only for
// the subcell distances next to the interface.  Per stage phi is read once
// and written once (plus phi^m in the second stage) with the code byte: 9 or
// 13 bytes per cell in float32.  The arithmetic per cell (three axes of ENO2
// differences and minmod limiters) keeps the issue slots busier than HBM.
#include "internal.h"

namespace wsi {

static constexpr int RX = 32, RY = 8;

__device__ __forceinline__ int mirror_cell(int m, int n) {
  if (m < 0) m = -m - 1;
  else if (m >= n) m = 2 * n - 1 - m;
  return clampi(m, 0, n - 1);
}

template <typename T>
struct ReinitAxes {
  T h[3], ih[3];
  int active[3];  // axis has more than one cell
  T cfl;
};

template <typename T>
__device__ __forceinline__ T minmod_(T a, T b) {
  return a * b > T(0) ? (fabs(a) < fabs(b) ? a : b) : T(0);
}

// fraction of the cell spacing from the centre holding a to the zero of the
// quadratic through a (at 0) and b (at 1) with second difference c, a*b < 0:
// local coordinate t = xi - 1/2, quadratic c0 + c1 t + c2 t^2; the zero in
// [-1/2, 1/2] is the root of smaller magnitude (stable form, linear limit
// for c = 0)
template <typename T>
__device__ __forceinline__ T iface_frac(T a, T b, T c) {
  const T c2 = T(0.5) * c, c1 = b - a, c0 = T(0.5) * (a + b) - T(0.125) * c;
  const T disc = fmax(c1 * c1 - T(4) * c2 * c0, T(0));
  return T(0.5) - T(2) * c0 / (c1 + copysign(sqrt(disc), c1));
}

template <typename T>
__device__ __forceinline__ double widen(T v);
template <>
__device__ __forceinline__ double widen<double>(double v) { return v; }
template <>
__device__ __forceinline__ double widen<float>(float v) { return f2d_fast(v); }

// Per-cell code of phi~, computed once per call (phi~ is fixed): bits 0-1
// the sign (0 zero, 1 positive, 2 negative); bit 2 + 2d (3 + 2d) set when
// phi~ changes sign towards the lower (upper) neighbour along axis d.  A
// mirror ghost equals its cell, so no crossing is flagged across a wall.
template <typename T>
__global__ void k_reinit_code(GridDev g, const T* __restrict__ q0, unsigned char* __restrict__ code) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const size_t plane = (size_t)n0 * n1, n = plane * n2;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(id / plane);
    const size_t r = id - (size_t)k * plane;
    const int j = (int)(r / n0), i = (int)(r - (size_t)j * n0);
    const T q = q0[id];
    unsigned c = q > T(0) ? 1u : (q < T(0) ? 2u : 0u);
    const int cc[3] = {i, j, k}, nn[3] = {n0, n1, n2};
    const size_t sd[3] = {1, (size_t)n0, plane};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (cc[d] > 0 && q * q0[id - sd[d]] < T(0)) c |= 4u << (2 * d);
      if (cc[d] + 1 < nn[d] && q * q0[id + sd[d]] < T(0)) c |= 8u << (2 * d);
    }
    code[id] = (unsigned char)c;
  }
}

// subcell distances of one axis (rare path: the cell is next to the
// interface along this axis); taps of phi~ from global memory
template <typename T>
__device__ __forceinline__ void subcell_axis(const T* __restrict__ q0, size_t id, int c, int n, size_t stride,
                                             unsigned bits, const T p[5], T h, T ih, T mp, T mm, T& Dm, T& Dp,
                                             T& hloc) {
  T q[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) q[m] = q0[id + (ptrdiff_t)(mirror_cell(c - 2 + m, n) - c) * (ptrdiff_t)stride];
  const T qc = q[1] - T(2) * q[2] + q[3];
  if (bits & 2u) {
    const T qp = q[2] - T(2) * q[3] + q[4];
    const T hp = fmin(fmax(h * iface_frac(q[2], q[3], minmod_(qc, qp)), T(1e-10) * h), h);
    Dp = -p[2] / hp - T(0.5) * hp * mp * ih * ih;
    hloc = fmin(hloc, hp);
  }
  if (bits & 1u) {
    const T qm = q[0] - T(2) * q[1] + q[2];
    const T hm = fmin(fmax(h * iface_frac(q[2], q[1], minmod_(qc, qm)), T(1e-10) * h), h);
    Dm = p[2] / hm + T(0.5) * hm * mm * ih * ih;
    hloc = fmin(hloc, hm);
  }
}

// One stage: v = pin + dtau L(pin);  with pavg:  v = (pavg + v) / 2.
// Written to pout, or with out64 (float32 path, last stage) as the change
// v - phi~ added to the float64 level set in out64.
template <typename T>
__global__ void __launch_bounds__(RX* RY) k_reinit(GridDev g, ReinitAxes<T> ax,
                                                   const unsigned char* __restrict__ code,
                                                   const T* __restrict__ q0, const T* __restrict__ pin,
                                                   const T* pavg, T* pout, double* out64, int zchunk) {
  constexpr int HX = RX + 4, HY = RY + 4, NS = (HX * HY + RX * RY - 1) / (RX * RY);
  __shared__ T sP[HY * HX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RX + tx;
  const int x0 = blockIdx.x * RX, y0 = blockIdx.y * RY;
  const int i = x0 + tx, j = y0 + ty;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const bool inside = i < n0 && j < n1;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(k0 + zchunk, n2);
  const size_t plane = (size_t)n0 * n1;
  int soff[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    const int t = tid + r * RX * RY;
    soff[r] = -1;
    if (t < HX * HY) {
      const int hy = t / HX, hx = t - hy * HX;
      soff[r] = mirror_cell(y0 - 2 + hy, n1) * n0 + mirror_cell(x0 - 2 + hx, n0);
    }
  }
  const size_t col = (size_t)min(j, n1 - 1) * n0 + min(i, n0 - 1);
  T zp[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) zp[m] = pin[(size_t)mirror_cell(k0 - 2 + m, n2) * plane + col];
  // software pipeline: the tile, code byte and next z tap of plane k + 1
  // are loaded while plane k is computed
  T nxt[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) nxt[r] = soff[r] >= 0 ? pin[(size_t)k0 * plane + soff[r]] : T(0);
  unsigned cd_next = inside && k0 < k1 ? code[(size_t)k0 * plane + col] : 0u;
  for (int k = k0; k < k1; ++k) {
    const size_t id = (size_t)k * plane + col;
    const unsigned cd = cd_next;
#pragma unroll
    for (int r = 0; r < NS; ++r)
      if (soff[r] >= 0) sP[tid + r * RX * RY] = nxt[r];
    __syncthreads();
    if (k + 1 < k1) {
#pragma unroll
      for (int r = 0; r < NS; ++r)
        if (soff[r] >= 0) nxt[r] = pin[(size_t)(k + 1) * plane + soff[r]];
      cd_next = inside ? code[id + plane] : 0u;
    }
    const T z_in = pin[(size_t)mirror_cell(k + 3, n2) * plane + col];
    if (inside) {
      const T s = (cd & 3u) == 1u ? T(1) : ((cd & 3u) == 2u ? T(-1) : T(0));
      T g2 = T(0), hmin = T(0);
      bool any = false;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!ax.active[d]) continue;
        T p[5];
#pragma unroll
        for (int m = 0; m < 5; ++m)
          p[m] = d == 2 ? zp[m] : (d == 0 ? sP[(ty + 2) * HX + tx + m] : sP[(ty + m) * HX + tx + 2]);
        const T pm = p[0] - T(2) * p[1] + p[2], pc = p[1] - T(2) * p[2] + p[3], pp = p[2] - T(2) * p[3] + p[4];
        const T mp = minmod_(pc, pp), mm = minmod_(pc, pm);
        T Dp = (p[3] - p[2]) * ax.ih[d] - T(0.5) * mp * ax.ih[d];
        T Dm = (p[2] - p[1]) * ax.ih[d] + T(0.5) * mm * ax.ih[d];
        T hloc = ax.h[d];
        const unsigned bits = (cd >> (2 + 2 * d)) & 3u;
        if (bits) {
          const int c = d == 0 ? i : (d == 1 ? j : k);
          const size_t stride = d == 0 ? 1 : (d == 1 ? (size_t)n0 : plane);
          subcell_axis(q0, id, c, g.n[d], stride, bits, p, ax.h[d], ax.ih[d], mp, mm, Dm, Dp, hloc);
        }
        // Godunov: s > 0 takes max(D-, 0) and min(D+, 0), s < 0 min(D-, 0)
        // and max(D+, 0); both are max(s D-, -s D+, 0) in magnitude
        const T t = fmax(fmax(s * Dm, -s * Dp), T(0));
        g2 += t * t;
        hmin = any ? fmin(hmin, hloc) : hloc;
        any = true;
      }
      const T dtau = any ? ax.cfl * hmin : T(0);
      T v = zp[2] + dtau * (-s * (sqrt(g2) - T(1)));
      if (pavg) v = T(0.5) * pavg[id] + T(0.5) * v;
      if (out64) out64[id] = out64[id] + widen<T>(v - q0[id]);
      else pout[id] = v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 4; ++m) zp[m] = zp[m + 1];
    zp[4] = z_in;
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = d2f_fast(a[t]);
}

template <typename T>
static void stage(const GridDev& g, const ReinitAxes<T>& ax, const unsigned char* code, const T* q0, const T* pin,
                  const T* pavg, T* pout, double* out64, cudaStream_t st) {
  const int zc = transport_chunk(g.n[0], g.n[1], g.n[2]);
  dim3 grid(cdiv(g.n[0], RX), cdiv(g.n[1], RY), cdiv(g.n[2], zc));
  ktimer_begin(KC_REINIT, st);
  { k_reinit<T><<<grid, dim3(RX, RY), 0, st>>>(g, ax, code, q0, pin, pavg, pout, out64, zc); WSI_COUNT(); }
  ktimer_end(KC_REINIT, st);
}

template <typename T>
void reinit_levelset(const GridDev& g, double* phi, int iters, double cfl, void* scratch, cudaStream_t st) {
  if (iters <= 0) return;
  const size_t n = (size_t)g.n[0] * g.n[1] * g.n[2];
  ReinitAxes<T> ax;
  for (int d = 0; d < 3; ++d) {
    ax.h[d] = (T)g.h[d];
    ax.ih[d] = (T)g.ih[d];
    ax.active[d] = g.n[d] > 1;
  }
  ax.cfl = (T)cfl;
  T* q0 = (T*)scratch;  // phi~, fixed for the whole iteration
  T* B = q0 + n;        // first-stage result
  T* A = B + n;         // iterate (float32 path; the float64 path iterates in phi)
  // the per-cell code of phi~ after the three arrays (scratch: 3 n doubles;
  // the float64 path uses the third array's space, which it does not need)
  unsigned char* code = sizeof(T) == sizeof(double) ? (unsigned char*)A : (unsigned char*)(A + n);
  const int blocks = std::max((int)std::min<size_t>((n + 255) / 256, 152 * 16), 1);
  if constexpr (sizeof(T) == sizeof(double)) {
    cudaMemcpyAsync(q0, phi, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  } else {
    { k_to_f32<<<blocks, 256, 0, st>>>(phi, (float*)q0, n); WSI_COUNT(); }
  }
  { k_reinit_code<T><<<blocks, 256, 0, st>>>(g, q0, code); WSI_COUNT(); }
  const T* cur = q0;
  for (int m = 0; m < iters; ++m) {
    stage<T>(g, ax, code, q0, cur, nullptr, B, nullptr, st);
    if constexpr (sizeof(T) == sizeof(double)) {
      stage<T>(g, ax, code, q0, B, cur, (T*)phi, nullptr, st);
      cur = (const T*)phi;
    } else if (m + 1 == iters) {
      stage<T>(g, ax, code, q0, B, cur, nullptr, phi, st);
    } else {
      stage<T>(g, ax, code, q0, B, cur, A, nullptr, st);
      cur = A;
    }
  }
}
template void reinit_levelset<double>(const GridDev&, double*, int, double, void*, cudaStream_t);
template void reinit_levelset<float>(const GridDev&, double*, int, double, void*, cudaStream_t);

}  // namespace wsi
