// DLM rigidity step (Sec. 4.2.5) and the IB4 Lagrangian-Eulerian transfers
// (Sec. 3.3) with the wall-adjoint forms J_BC / S_BC (Sec. 3.3.2).
//
// Interpolation is a gather (one thread per marker: the kernel weights of
// each axis are shared by the three components, 64 taps each); spreading
// scatters with float64 atomicAdd into the face arrays.  Weights and sums are
// double-float (float64 accuracy on the float32 pipes; GB300's float64 rate
// is 1/64 of its float32 rate).  Taps that
// fall beyond a wall are folded onto their mirror image with the ghost sign
// (tangential: the wall's sign; normal: odd about the wall face, whose own
// value is zero so taps landing on it drop out), which makes S_BC the exact
// adjoint of J_BC.  Rigid-body sums are deterministic two-stage reductions.
#include <math.h>

#include "df.cuh"
#include "internal.h"

namespace wsi {

// Peskin's four-point kernel (the published formula; Sec. 3.3.1 cites it),
// evaluated in double-float arithmetic (float64 accuracy on the float32
// pipes): r = |r|; (3 - 2r + sqrt(1 + 4r - 4r^2))/8 for r <= 1,
// (5 - 2r - sqrt(-7 + 12r - 4r^2))/8 for 1 < r <= 2, 0 beyond.  The branch
// is chosen on the leading part of r; the branches agree in value and slope
// at r = 1 and r = 2, so the choice at a tie costs O(lo^2).
__device__ __forceinline__ dfl phi4_df(dfl r) {
  if (r.h < 0.0f) r = df_neg(r);
  if (r.h > 2.0f) return df_from_float(0.0f);
  const dfl r2 = df_mul(r, r);
  const dfl two_r = df_scale(r, 2.0f);
  if (r.h <= 1.0f) {
    // 1 + 4r - 4r^2
    const dfl u = df_add(df_from_float(1.0f), df_scale(df_sub(r, r2), 4.0f));
    return df_scale(df_add(df_sub(df_from_float(3.0f), two_r), df_sqrt(u)), 0.125f);
  }
  // -7 + 12r - 4r^2
  const dfl u = df_sub(df_sub(df_mul(r, df_from_float(12.0f)), df_scale(r2, 4.0f)), df_from_float(7.0f));
  return df_scale(df_sub(df_sub(df_from_float(5.0f), two_r), df_sqrt(u)), 0.125f);
}

struct Tap {
  int idx[4];
  dfl w[4];  // kernel weight times ghost sign; 0 for dropped taps
};

// the four taps along axis d of a marker at coordinate Xd, for a component
// normal to d (normal = true: faces at integer positions) or tangential
// (cell centres, offset by half a cell); positions in double-float
__device__ __forceinline__ void taps_axis(const GridDev& g, bool normal, int d, dfl Xd, dfl ih, Tap& t) {
  const int n = g.n[d];
  dfl xs = df_mul(Xd, ih);
  if (!normal) xs = df_sub(xs, df_from_float(0.5f));
  const int base = df_floor(xs) - 1;
  const float s_lo = g.bcf[2 * d], s_hi = g.bcf[2 * d + 1];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int i = base + q;
    const dfl r = df_sub(df_from_float((float)i), xs);
    float sg = 1.0f;
    for (int it = 0; it < 8; ++it) {
      if (normal) {
        if (i < 0) { i = -i; sg = -sg; }
        if (i > n) { i = 2 * n - i; sg = -sg; }
      } else {
        if (i < 0) { i = -1 - i; sg *= s_lo; }
        if (i >= n) { i = 2 * n - 1 - i; sg *= s_hi; }
      }
    }
    const bool valid = normal ? (i > 0 && i < n) : (i >= 0 && i < n);
    t.idx[q] = valid ? i : 0;
    const dfl w = phi4_df(r);
    t.w[q] = valid ? (sg < 0.0f ? df_neg(w) : w) : df_from_float(0.0f);
  }
}

// per marker: the normal and tangential taps of each axis (components share
// them: component c uses the normal taps on axis c, tangential elsewhere)
struct MarkerTaps {
  Tap tn[3], tt[3];
};

__device__ __forceinline__ void marker_taps(const GridDev& g, const double* __restrict__ X, int m, MarkerTaps& T) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const dfl xd = df_split(X[3 * m + d]);
    const dfl ih = df_split(g.ih[d]);
    taps_axis(g, true, d, xd, ih, T.tn[d]);
    taps_axis(g, false, d, xd, ih, T.tt[d]);
  }
}

// one thread per marker, all three components; separable sums
// sum_z w_z sum_y w_y sum_x w_x q in double-float, one float64 addition per
// component at the end
__global__ void __launch_bounds__(128) k_interp(GridDev g, CVel<double> vel, const double* __restrict__ X, int n,
                                                double* U) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  MarkerTaps T;
  marker_taps(g, X, m, T);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Tap& tx = c == 0 ? T.tn[0] : T.tt[0];
    const Tap& ty = c == 1 ? T.tn[1] : T.tt[1];
    const Tap& tz = c == 2 ? T.tn[2] : T.tt[2];
    const double* __restrict__ q = vel.q[c];
    const size_t sx = (size_t)(g.n[0] + (c == 0)), sy = sx * (size_t)(g.n[1] + (c == 1));
    dfl s = df_from_float(0.0f);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
      if (tz.w[kz].h == 0.0f) continue;
      dfl sz = df_from_float(0.0f);
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        if (ty.w[ky].h == 0.0f) continue;
        const double* row = q + (size_t)tz.idx[kz] * sy + (size_t)ty.idx[ky] * sx;
        dfl sr = df_from_float(0.0f);
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) sr = df_add(sr, df_mul(tx.w[kx], df_split(row[tx.idx[kx]])));
        sz = df_add(sz, df_mul(ty.w[ky], sr));
      }
      s = df_add(s, df_mul(tz.w[kz], sz));
    }
    U[3 * m + c] = df_to_double(s);
  }
}

// Deterministic spreading.  Float64 atomics would sum each face's
// contributions in a varying order; instead every contribution is rounded to
// a multiple of a power-of-two quantum 2^-E and added as a 64-bit integer,
// whose sum does not depend on the order.  E is chosen on the device per call
// from a bound on any face's sum: at most 5 cells per axis hold markers whose
// taps reach a face (twice that count where taps fold at a wall), each tap
// weight is at most phi4(0)^3 = 1/8, so |sum| <= 128 c_max max|F| scale with
// c_max the most markers in one cell; E puts that bound below 2^61.  The
// quantum is then ~2^-50 of the largest contribution.

// integer nearest to f 2^E for a float f with |f 2^E| < 2^62 (integer
// operations on the bit pattern; ties away from zero)
__device__ __forceinline__ long long fixed_of(float f, int E) {
  const unsigned u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 0xFFu);
  if (ex == 0) return 0;  // zero (and subnormals, < 2^-126)
  const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 150 + E;  // f 2^E = m 2^sh
  long long v;
  if (sh >= 0) v = m << sh;
  else if (sh > -25) v = (m + (1LL << (-sh - 1))) >> (-sh);
  else v = 0;
  return (u & 0x80000000u) ? -v : v;
}

__global__ void __launch_bounds__(128) k_spread(GridDev g, const double* __restrict__ F,
                                                const double* __restrict__ X, int n, double scale,
                                                unsigned long long* acc0, unsigned long long* acc1,
                                                unsigned long long* acc2, const int* __restrict__ qexp) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const int E = qexp[0];
  MarkerTaps T;
  marker_taps(g, X, m, T);
  const dfl sc = df_split(scale);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Tap& tx = c == 0 ? T.tn[0] : T.tt[0];
    const Tap& ty = c == 1 ? T.tn[1] : T.tt[1];
    const Tap& tz = c == 2 ? T.tn[2] : T.tt[2];
    unsigned long long* q = c == 0 ? acc0 : (c == 1 ? acc1 : acc2);
    const size_t sx = (size_t)(g.n[0] + (c == 0)), sy = sx * (size_t)(g.n[1] + (c == 1));
    const dfl f = df_mul(df_split(F[3 * m + c]), sc);
    dfl fx[4];
#pragma unroll
    for (int kx = 0; kx < 4; ++kx) fx[kx] = df_mul(f, tx.w[kx]);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
      if (tz.w[kz].h == 0.0f) continue;
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        if (ty.w[ky].h == 0.0f) continue;
        const dfl wyz = df_mul(tz.w[kz], ty.w[ky]);
        unsigned long long* row = q + (size_t)tz.idx[kz] * sy + (size_t)ty.idx[ky] * sx;
#pragma unroll
        for (int kx = 0; kx < 4; ++kx)
          if (tx.w[kx].h != 0.0f) {
            const dfl v = df_mul(wyz, fx[kx]);
            atomicAdd(&row[tx.idx[kx]], (unsigned long long)(fixed_of(v.h, E) + fixed_of(v.l, E)));
          }
      }
    }
  }
}

// markers per cell (the cell holding each marker, clamped into the grid)
__global__ void k_marker_count(GridDev g, const double* __restrict__ X, int n, int* cnt) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  int c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) c[d] = clampi((int)floor(X[3 * m + d] * g.ih[d]), 0, g.n[d] - 1);
  atomicAdd(&cnt[fidx(g, 3, c[0], c[1], c[2])], 1);
}

// Per-block maxima of the box's cell counts and of |F| (partials: two per
// block), then one small block turns them into E; maxima do not depend on
// the order in which they are taken.
static constexpr int XB = 152;  // blocks of the partial maxima

__global__ void k_spread_max_part(GridDev g, SpreadBox b, const int* __restrict__ cnt, const double* __restrict__ F,
                                  int n3, double* part) {
  __shared__ int shc[32];
  __shared__ double shf[32];
  const int ex = b.hi[0] - b.lo[0] + 1, ey = b.hi[1] - b.lo[1] + 1, ez = b.hi[2] - b.lo[2] + 1;
  const long long nb = (long long)ex * ey * ez;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int cm = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += stride) {
    const int i = b.lo[0] + (int)(t % ex), j = b.lo[1] + (int)((t / ex) % ey), k = b.lo[2] + (int)(t / ((long long)ex * ey));
    cm = max(cm, cnt[fidx(g, 3, i, j, k)]);
  }
  double fm = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += stride) fm = fmax(fm, fabs(F[t]));
  for (int o = 16; o > 0; o >>= 1) {
    cm = max(cm, __shfl_down_sync(0xffffffffu, cm, o));
    fm = fmax(fm, __shfl_down_sync(0xffffffffu, fm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    shc[threadIdx.x >> 5] = cm;
    shf[threadIdx.x >> 5] = fm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    double f = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      c = max(c, shc[w]);
      f = fmax(f, shf[w]);
    }
    part[2 * blockIdx.x] = (double)c;
    part[2 * blockIdx.x + 1] = f;
  }
}

__global__ void k_spread_exponent(const double* __restrict__ part, int nparts, double scale, int* qexp) {
  if (threadIdx.x != 0) return;
  double c = 0.0, f = 0.0;
  for (int q = 0; q < nparts; ++q) {
    c = fmax(c, part[2 * q]);
    f = fmax(f, part[2 * q + 1]);
  }
  const double B = 128.0 * c * f * scale;
  int e = 0;
  const bool pos = B > 0.0 && B < 1e300;
  if (pos) frexp(B, &e);  // B < 2^e
  qexp[0] = pos ? 61 - e : 0;
}

// counts of the box's cells back to zero for the next call
__global__ void k_clear_box(GridDev g, SpreadBox b, int* cnt) {
  const int ex = b.hi[0] - b.lo[0] + 1, ey = b.hi[1] - b.lo[1] + 1, ez = b.hi[2] - b.lo[2] + 1;
  const long long nb = (long long)ex * ey * ez;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += (long long)gridDim.x * blockDim.x) {
    const int i = b.lo[0] + (int)(t % ex), j = b.lo[1] + (int)((t / ex) % ey), k = b.lo[2] + (int)(t / ((long long)ex * ey));
    cnt[fidx(g, 3, i, j, k)] = 0;
  }
}

// vel += acc 2^-E on the box's faces of component C; acc cleared
template <int C>
__global__ void k_unfix(GridDev g, SpreadBox b, unsigned long long* acc, const int* __restrict__ qexp, double* vel) {
  const int ex = b.hi[0] - b.lo[0] + 1 + (C == 0), ey = b.hi[1] - b.lo[1] + 1 + (C == 1);
  const int ez = b.hi[2] - b.lo[2] + 1 + (C == 2);
  const long long nb = (long long)ex * ey * ez;
  const double q = ldexp(1.0, -qexp[0]);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += (long long)gridDim.x * blockDim.x) {
    const int i = b.lo[0] + (int)(t % ex), j = b.lo[1] + (int)((t / ex) % ey), k = b.lo[2] + (int)(t / ((long long)ex * ey));
    const size_t id = fidx(g, C, i, j, k);
    const long long a = (long long)acc[id];
    if (a != 0) {
      vel[id] += (double)a * q;
      acc[id] = 0ull;
    }
  }
}

void launch_ib_interp(const GridDev& g, const double* const vel[3], const double* X, int n, double* U,
                      cudaStream_t st) {
  if (n <= 0) return;
  CVel<double> v{{vel[0], vel[1], vel[2]}};
  { k_interp<<<cdiv(n, 128), 128, 0, st>>>(g, v, X, n, U); WSI_COUNT(); }
}

SpreadBox spread_box(const GridDev& g, const double mm[6]) {
  SpreadBox b;
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = std::max(0, (int)std::floor(mm[d] * g.ih[d] - 0.5) - 3);
    b.hi[d] = std::min(g.n[d] - 1, (int)std::floor(mm[3 + d] * g.ih[d]) + 3);
    if (b.hi[d] < b.lo[d]) b.hi[d] = b.lo[d];
  }
  return b;
}

void launch_ib_spread(const GridDev& g, const double* F, const double* X, int n, double dV, double* const vel[3],
                      const SpreadWork& w, const SpreadBox& b, cudaStream_t st) {
  if (n <= 0) return;
  const double scale = dV / (g.h[0] * g.h[1] * g.h[2]);
  unsigned long long* acc[3] = {w.acc, w.acc + fsize(g, 0), w.acc + fsize(g, 0) + fsize(g, 1)};
  const long long nb = (long long)(b.hi[0] - b.lo[0] + 2) * (b.hi[1] - b.lo[1] + 2) * (b.hi[2] - b.lo[2] + 2);
  const int blocks = (int)std::min<long long>((nb + 255) / 256, 152 * 8);
  { k_marker_count<<<cdiv(n, 256), 256, 0, st>>>(g, X, n, w.cnt); WSI_COUNT(); }
  { k_spread_max_part<<<XB, 256, 0, st>>>(g, b, w.cnt, F, 3 * n, w.part); WSI_COUNT(); }
  { k_spread_exponent<<<1, 32, 0, st>>>(w.part, XB, scale, w.qexp); WSI_COUNT(); }
  { k_clear_box<<<blocks, 256, 0, st>>>(g, b, w.cnt); WSI_COUNT(); }
  { k_spread<<<cdiv(n, 128), 128, 0, st>>>(g, F, X, n, scale, acc[0], acc[1], acc[2], w.qexp); WSI_COUNT(); }
  { k_unfix<0><<<blocks, 256, 0, st>>>(g, b, acc[0], w.qexp, vel[0]); WSI_COUNT(); }
  { k_unfix<1><<<blocks, 256, 0, st>>>(g, b, acc[1], w.qexp, vel[1]); WSI_COUNT(); }
  { k_unfix<2><<<blocks, 256, 0, st>>>(g, b, acc[2], w.qexp, vel[2]); WSI_COUNT(); }
}

// min (0..2) and max (3..5) of the marker positions: per-block extrema,
// then one small block over the partials
__global__ void k_marker_box_part(const double* __restrict__ X, int n, double* part) {
  __shared__ double sh[6][32];
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      mn[d] = fmin(mn[d], X[3 * m + d]);
      mx[d] = fmax(mx[d], X[3 * m + d]);
    }
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o > 0; o >>= 1) {
      mn[d] = fmin(mn[d], __shfl_down_sync(0xffffffffu, mn[d], o));
      mx[d] = fmax(mx[d], __shfl_down_sync(0xffffffffu, mx[d], o));
    }
  if ((threadIdx.x & 31) == 0)
    for (int d = 0; d < 3; ++d) {
      sh[d][threadIdx.x >> 5] = mn[d];
      sh[3 + d][threadIdx.x >> 5] = mx[d];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = sh[threadIdx.x][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      v = threadIdx.x < 3 ? fmin(v, sh[threadIdx.x][w]) : fmax(v, sh[threadIdx.x][w]);
    part[6 * blockIdx.x + threadIdx.x] = v;
  }
}

__global__ void k_marker_box_final(const double* __restrict__ part, int nparts, double* out) {
  const int q = threadIdx.x;
  if (q >= 6) return;
  double v = part[q];
  for (int b = 1; b < nparts; ++b) v = q < 3 ? fmin(v, part[6 * b + q]) : fmax(v, part[6 * b + q]);
  out[q] = v;
}

void launch_marker_box(const double* X, int n, double* out6, double* scratch, cudaStream_t st) {
  if (n <= 0) return;
  { k_marker_box_part<<<XB, 256, 0, st>>>(X, n, scratch); WSI_COUNT(); }
  { k_marker_box_final<<<1, 32, 0, st>>>(scratch, XB, out6); WSI_COUNT(); }
}

// ---------------------------------------------------------------- rigid sums
static constexpr int SB = 152;  // reduction blocks
static constexpr int ST = 256;
static constexpr int NS = 15;   // sums per marker

__global__ void k_rigid_part(const double* __restrict__ X, const double* __restrict__ U, int n,
                             const double* __restrict__ xc, double* part) {
  double acc[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) acc[q] = 0.0;
  double cx = xc ? xc[0] : 0.0, cy = xc ? xc[1] : 0.0, cz = xc ? xc[2] : 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double x = X[3 * m], y = X[3 * m + 1], z = X[3 * m + 2];
    double rx = x - cx, ry = y - cy, rz = z - cz;
    double ux = U ? U[3 * m] : 0.0, uy = U ? U[3 * m + 1] : 0.0, uz = U ? U[3 * m + 2] : 0.0;
    acc[0] += ux;
    acc[1] += uy;
    acc[2] += uz;
    acc[3] += ry * uz - rz * uy;
    acc[4] += rz * ux - rx * uz;
    acc[5] += rx * uy - ry * ux;
    double rr = rx * rx + ry * ry + rz * rz;
    acc[6] += rr - rx * rx;
    acc[7] += rr - ry * ry;
    acc[8] += rr - rz * rz;
    acc[9] += -rx * ry;
    acc[10] += -rx * rz;
    acc[11] += -ry * rz;
    acc[12] += x;
    acc[13] += y;
    acc[14] += z;
  }
  __shared__ double sh[ST / 32][NS];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double s = 0.0;
    for (int w = 0; w < ST / 32; ++w) s += sh[w][threadIdx.x];
    part[blockIdx.x * NS + threadIdx.x] = s;
  }
}

__global__ void k_rigid_final(const double* __restrict__ part, double* out) {
  int q = threadIdx.x;
  if (q >= NS) return;
  double s = 0.0;
  for (int b = 0; b < SB; ++b) s += part[b * NS + q];
  out[q] = s;
}

void launch_rigid_sums(const double* X, const double* U, int n, const double* xc_dev, double* out, double* scratch,
                       cudaStream_t st) {
  { k_rigid_part<<<SB, ST, 0, st>>>(X, U, n, xc_dev, scratch); WSI_COUNT(); }
  { k_rigid_final<<<1, 32, 0, st>>>(scratch, out); WSI_COUNT(); }
}

__global__ void k_mean3(const double* __restrict__ sums, int n, double* xc) {
  if (threadIdx.x < 3) xc[threadIdx.x] = sums[12 + threadIdx.x] / (double)n;
}

void launch_marker_mean(const double* X, int n, double* xc_dev, double* scratch, cudaStream_t st) {
  // scratch: SB*NS partials followed by NS sums
  { k_rigid_part<<<SB, ST, 0, st>>>(X, nullptr, n, nullptr, scratch); WSI_COUNT(); }
  { k_rigid_final<<<1, 32, 0, st>>>(scratch, scratch + SB * NS); WSI_COUNT(); }
  { k_mean3<<<1, 32, 0, st>>>(scratch + SB * NS, n, xc_dev); WSI_COUNT(); }
}

__global__ void k_body_vel(const double* __restrict__ X, const double* __restrict__ U, int n,
                           const double* __restrict__ rg, const double* __restrict__ xc, double* Ub, double* F) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double rx = X[3 * m] - xc[0], ry = X[3 * m + 1] - xc[1], rz = X[3 * m + 2] - xc[2];
  double wx = rg[3], wy = rg[4], wz = rg[5];
  double bx = rg[0] + (wy * rz - wz * ry);
  double by = rg[1] + (wz * rx - wx * rz);
  double bz = rg[2] + (wx * ry - wy * rx);
  Ub[3 * m] = bx;
  Ub[3 * m + 1] = by;
  Ub[3 * m + 2] = bz;
  if (F) {
    F[3 * m] = bx - U[3 * m];
    F[3 * m + 1] = by - U[3 * m + 1];
    F[3 * m + 2] = bz - U[3 * m + 2];
  }
}

void launch_body_velocity(const double* X, const double* U, int n, const double* rigid_dev, const double* xc_dev,
                          double* Ub, double* F, cudaStream_t st) {
  if (n <= 0) return;
  { k_body_vel<<<cdiv(n, 128), 128, 0, st>>>(X, U, n, rigid_dev, xc_dev, Ub, F); WSI_COUNT(); }
}

// X = X^n + dt (U_b^{n+1} + U_b^n) / 2 (Sec. 4.2.5).  Device bound check: a
// position that is not finite or lies outside the box by more than half a
// cell sets *flag (the step then reports WSI_ERR_DEVICE); nothing traps.
__global__ void k_marker_update(GridDev g, const double* __restrict__ Xn, const double* __restrict__ Ub1,
                                const double* __restrict__ Ub0, int n3, double dt, double* X, int* flag) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  const double v = Xn[t] + dt * 0.5 * (Ub1[t] + Ub0[t]);
  X[t] = v;
  const int d = t % 3;
  const double tol = 0.5 * g.h[d];
  if (flag && !(v >= -tol && v <= g.n[d] * g.h[d] + tol)) atomicOr(flag, 1);
}

void launch_marker_update(const GridDev& g, const double* Xn, const double* Ub_new, const double* Ub_old, int n,
                          double dt, double* X, int* flag, cudaStream_t st) {
  if (n <= 0) return;
  { k_marker_update<<<cdiv(3LL * n, 256), 256, 0, st>>>(g, Xn, Ub_new, Ub_old, 3 * n, dt, X, flag); WSI_COUNT(); }
}

}  // namespace wsi
