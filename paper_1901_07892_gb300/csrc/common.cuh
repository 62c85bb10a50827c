// Shared device-side definitions of libwsi: grid geometry, index maps of the
// staggered (MAC) arrays, ghost rules at walls, launch helpers.
//
// Layout (Sec. 3.1): x fastest, unghosted.  Component c of the velocity lives
// on c-faces with extents n + e_c; edges in the (c,d) plane have extents
// n + e_c + e_d.  Tangential ghosts across a wall are s * (adjacent value),
// s = -1 no-slip, +1 free-slip; faces on walls hold the zero normal velocity.
// Open top (Sec. 7.1: zero tangential velocity and zero pressure on the top
// plane): the z-faces of the top plane are unknowns, the pressure ghost above
// it is -p of the cell below, the ghost of w above it mirrors w evenly
// (dw/dz = 0) and tangential ghosts take s = -1.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

namespace wsi {

// process-wide count of kernel launches made by the library
extern std::atomic<long long> g_launches;
#define WSI_COUNT() (::wsi::g_launches.fetch_add(1, std::memory_order_relaxed))

// Optional per-kernel timing: when kernel class `id` is enabled, its launches
// are bracketed by CUDA events on their own stream.
enum KernelClass {
  KC_STOKES = 0,     // float64 Stokes matvec (momentum rows + continuity)
  KC_RBGS_P = 1,     // pressure red-black Gauss-Seidel half sweep
  KC_RBGS_V = 2,     // viscous red-black Gauss-Seidel half sweep
  KC_TRANSPORT = 3,  // consistent transport flux divergence
  KC_MDOT = 4,       // Gram-Schmidt block dot products
  KC_MAXPY = 5,      // Gram-Schmidt multi-axpy
  KC_RESTRICT = 6,   // residual + restriction
  KC_PROLONG = 7,    // prolongation + correction
  KC_REINIT = 8,     // level-set reinitialisation stage
  KC_COUNT = 9
};
void ktimer_begin(int id, cudaStream_t st);
void ktimer_end(int id, cudaStream_t st);
// algorithmic bytes of the launch being bracketed (classes whose launches
// differ in size report them; the sum is read by wsi_ktimer_bytes)
void ktimer_bytes(int id, double bytes);

struct GridDev {
  int n[3];       // cells per axis
  double h[3];    // spacing
  double ih[3];   // 1/h (set by grid_finalize)
  double ih2[3];  // 1/h^2
  double bc[6];   // tangential ghost sign per wall (x-, x+, y-, y+, z-, z+)
  int open_top;   // 1: the z+ side is open (zero tangential velocity, zero pressure)
  // float32 copies for float32 kernels (a float64->float32 conversion issues
  // on the narrow float64 pipe, so kernels never convert these per thread)
  float ihf[3], ih2f[3], bcf[6];
};
template <typename T>
__host__ __device__ __forceinline__ T ginv(const GridDev& g, int a);
template <>
__host__ __device__ __forceinline__ double ginv<double>(const GridDev& g, int a) { return g.ih[a]; }
template <>
__host__ __device__ __forceinline__ float ginv<float>(const GridDev& g, int a) { return g.ihf[a]; }
template <typename T>
__host__ __device__ __forceinline__ T ginv2(const GridDev& g, int a);
template <>
__host__ __device__ __forceinline__ double ginv2<double>(const GridDev& g, int a) { return g.ih2[a]; }
template <>
__host__ __device__ __forceinline__ float ginv2<float>(const GridDev& g, int a) { return g.ih2f[a]; }
template <typename T>
__host__ __device__ __forceinline__ T gbc(const GridDev& g, int a);
template <>
__host__ __device__ __forceinline__ double gbc<double>(const GridDev& g, int a) { return g.bc[a]; }
template <>
__host__ __device__ __forceinline__ float gbc<float>(const GridDev& g, int a) { return g.bcf[a]; }

inline void grid_finalize(GridDev& g) {
  for (int a = 0; a < 3; ++a) {
    g.ih[a] = 1.0 / g.h[a];
    g.ih2[a] = 1.0 / (g.h[a] * g.h[a]);
    g.ihf[a] = (float)g.ih[a];
    g.ih2f[a] = (float)g.ih2[a];
  }
  for (int a = 0; a < 6; ++a) g.bcf[a] = (float)g.bc[a];
}

__host__ __device__ __forceinline__ int ext(const GridDev& g, int c, int a) {
  return g.n[a] + (a == c ? 1 : 0);
}
// a C-face with index a along C is an unknown (a row of the momentum
// equation): not on a wall; with an open top the top z-faces are rows
__host__ __device__ __forceinline__ bool face_row(const GridDev& g, int C, int a) {
  return a > 0 && (a < g.n[C] || (C == 2 && g.open_top));
}
// c = 0,1,2 velocity components; c = 3 cell-centred
__host__ __device__ __forceinline__ size_t fsize(const GridDev& g, int c) {
  return (size_t)(g.n[0] + (c == 0)) * (g.n[1] + (c == 1)) * (g.n[2] + (c == 2));
}
__host__ __device__ __forceinline__ size_t fidx(const GridDev& g, int c, int i, int j, int k) {
  return ((size_t)k * (g.n[1] + (c == 1)) + j) * (g.n[0] + (c == 0)) + i;
}
// edge arrays: e = 0 xy (along z), 1 xz (along y), 2 yz (along x)
__host__ __device__ __forceinline__ int edge_id(int c, int d) {
  int a = c < d ? c : d, b = c < d ? d : c;
  return (a == 0 && b == 1) ? 0 : (a == 0 ? 1 : 2);
}
__host__ __device__ __forceinline__ size_t esize(const GridDev& g, int e) {
  int ax = (e == 0 || e == 1) ? 1 : 0, ay = (e == 0 || e == 2) ? 1 : 0, az = (e == 1 || e == 2) ? 1 : 0;
  return (size_t)(g.n[0] + ax) * (g.n[1] + ay) * (g.n[2] + az);
}
__host__ __device__ __forceinline__ size_t eidx(const GridDev& g, int e, int i, int j, int k) {
  int ax = (e == 0 || e == 1) ? 1 : 0, ay = (e == 0 || e == 2) ? 1 : 0;
  return ((size_t)k * (g.n[1] + ay) + j) * (g.n[0] + ax) + i;
}

// offsets of the packed Stokes vector (u, v, w, p)
struct Packing {
  size_t off[5];
};
inline Packing packing(const GridDev& g) {
  Packing p;
  p.off[0] = 0;
  for (int c = 0; c < 4; ++c) p.off[c + 1] = p.off[c] + fsize(g, c);
  return p;
}

template <typename T>
struct Vel {
  T* q[3];
};
template <typename T>
struct CVel {
  const T* q[3];
};

// Read component C at face (i,j,k), with one ghost layer along the two
// tangential axes (mirror with the wall's sign).
template <int C, typename T>
__device__ __forceinline__ T qget(const GridDev& g, const T* __restrict__ q, int i, int j, int k) {
  T s = T(1);
  int idx3[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == C) continue;
    if (idx3[a] < 0) { idx3[a] = 0; s *= (T)g.bc[2 * a]; }
    else if (idx3[a] >= g.n[a]) { idx3[a] = g.n[a] - 1; s *= (T)g.bc[2 * a + 1]; }
  }
  return s * q[fidx(g, C, idx3[0], idx3[1], idx3[2])];
}

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }


// float64 -> float32 by integer operations on the IEEE-754 bit patterns:
// sign, exponent rebiased by 1023 - 127, top 23 significand bits, rounded
// half-up on the 24th dropped bit (a carry may move into the exponent, which
// is the correct rounding).  |a| < 2^-126 flushes to signed zero; overflow,
// infinities and NaN become infinity.  The hardware conversion issues on
// the float64 pipe, which on GB300 runs at 1/64 of the float32 rate; this
// one runs on the integer pipes.
__device__ __forceinline__ float d2f_fast(double a) {
  unsigned long long b = (unsigned long long)__double_as_longlong(a);
  unsigned int hi = (unsigned int)(b >> 32);
  unsigned int sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  unsigned int f = ((unsigned int)e << 23) | (unsigned int)(m >> 29);
  f += (unsigned int)(m >> 28) & 1u;
  if (f >= 0x7F800000u) f = 0x7F800000u;
  return __uint_as_float(sign | f);
}

// float32 -> float64 exactly, by integer operations (normal numbers and
// zero; float32 subnormals become zero)
__device__ __forceinline__ double f2d_fast(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long ed = (unsigned long long)(e == 255u ? 2047u : e - 127u + 1023u) << 52;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | ed | m));
}

template <typename To, typename Ti>
__device__ __forceinline__ To cvt(Ti a) {
  return (To)a;
}
template <>
__device__ __forceinline__ float cvt<float, double>(double a) {
  return d2f_fast(a);
}
template <>
__device__ __forceinline__ double cvt<double, float>(float a) {
  return f2d_fast(a);
}


inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace wsi
