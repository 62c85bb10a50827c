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

__global__ void __launch_bounds__(128) k_spread(GridDev g, const double* __restrict__ F,
                                                const double* __restrict__ X, int n, double scale, Vel<double> vel) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  MarkerTaps T;
  marker_taps(g, X, m, T);
  const dfl sc = df_split(scale);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Tap& tx = c == 0 ? T.tn[0] : T.tt[0];
    const Tap& ty = c == 1 ? T.tn[1] : T.tt[1];
    const Tap& tz = c == 2 ? T.tn[2] : T.tt[2];
    double* q = vel.q[c];
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
        double* row = q + (size_t)tz.idx[kz] * sy + (size_t)ty.idx[ky] * sx;
#pragma unroll
        for (int kx = 0; kx < 4; ++kx)
          if (tx.w[kx].h != 0.0f) atomicAdd(&row[tx.idx[kx]], df_to_double(df_mul(wyz, fx[kx])));
      }
    }
  }
}

void launch_ib_interp(const GridDev& g, const double* const vel[3], const double* X, int n, double* U,
                      cudaStream_t st) {
  if (n <= 0) return;
  CVel<double> v{{vel[0], vel[1], vel[2]}};
  { k_interp<<<cdiv(n, 128), 128, 0, st>>>(g, v, X, n, U); WSI_COUNT(); }
}

void launch_ib_spread(const GridDev& g, const double* F, const double* X, int n, double dV, double* const vel[3],
                      cudaStream_t st) {
  if (n <= 0) return;
  Vel<double> v{{vel[0], vel[1], vel[2]}};
  double scale = dV / (g.h[0] * g.h[1] * g.h[2]);
  { k_spread<<<cdiv(n, 128), 128, 0, st>>>(g, F, X, n, scale, v); WSI_COUNT(); }
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
