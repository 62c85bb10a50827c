// Stokes matvec of the mixed path with the strain-rate term in double-float
// arithmetic.
//
// GB300 issues float64 arithmetic at 1/64 of its float32 rate, and the
// float64 Stokes matvec (about 130 float64 operations per cell) is the
// largest single kernel of a time step.  Here each momentum row
//     y = (rho/dt) q + G p - theta L_mu q
// keeps the short terms in float64 and evaluates L_mu q -- about 35
// operations -- with unevaluated float32 pairs (hi + lo, a 48-bit
// significand): Dekker's exact product via fused multiply-add, Knuth's
// error-free two-sum, renormalised after every operation.  Inputs stay
// float64 in memory and are split into (hi, lo) by integer operations on
// their bit patterns, so the float64 pipe only sees the final combination.
// Relative error of L_mu q ~1e-14, far below what the float64 residual of
// FGMRES needs; magnitudes below 2^-126 ~ 1.2e-38 are flushed to zero.
#include <math.h>

#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;

struct dfl {
  float h, l;
};

// exact truncation of a float64 to its leading 24 significand bits (hi) and
// the next 29 bits rounded to a float (lo); a = hi + lo to ~2^-47 relative
__device__ __forceinline__ dfl df_split(double a) {
  unsigned long long b = (unsigned long long)__double_as_longlong(a);
  unsigned int hw = (unsigned int)(b >> 32);
  unsigned int sign = hw & 0x80000000u;
  int e = (int)((hw >> 20) & 0x7FFu);
  int ef = e - 1023 + 127;
  dfl r;
  if (ef <= 0 || e == 0) {
    r.h = 0.0f;
    r.l = 0.0f;
    return r;
  }
  if (ef >= 255) {
    r.h = __uint_as_float(sign | 0x7F800000u);
    r.l = 0.0f;
    return r;
  }
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  r.h = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)(m >> 29));
  unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);  // 29 bits, weight 2^(e-1075)
  float lo = ldexpf((float)rem, e - 1075);
  r.l = sign ? -lo : lo;
  return r;
}

__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
  float s = a + b;
  dfl r;
  r.h = s;
  r.l = b - (s - a);
  return r;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float v = s - a;
  e = (a - (s - v)) + (b - v);
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  float s, e, t, f;
  two_sum(x.h, y.h, s, e);
  two_sum(x.l, y.l, t, f);
  e += t;
  dfl r = quick_two_sum(s, e);
  r.l += f;
  return quick_two_sum(r.h, r.l);
}

__device__ __forceinline__ dfl df_neg(dfl x) {
  x.h = -x.h;
  x.l = -x.l;
  return x;
}

__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return quick_two_sum(p, e);
}

// exact float32 -> float64 by integer operations (normal floats and zero)
__device__ __forceinline__ double f2d_exact(float f) {
  unsigned int u = __float_as_uint(f);
  unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long ed = (unsigned long long)(e - 127 + 1023) << 52;
  unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | ed | m));
}

__device__ __forceinline__ double df_to_double(dfl x) { return f2d_exact(x.h) + f2d_exact(x.l); }

struct DfConst {
  dfl ih[3];     // 1/h
  dfl two_ih2[3];  // 2/h^2
};

// L_mu q at the interior C-face (i,j,k) in double-float
template <int C>
__device__ __forceinline__ dfl strain_df(const GridDev& g, const DfConst& k, const Coef<double>& cf,
                                         const double* const* q, int i, int j, int kk) {
  const double* qc = q[C];
  int id3[3] = {i, j, kk};
  int lo3[3] = {i, j, kk};
  lo3[C] -= 1;
  int hi3[3] = {i, j, kk};
  hi3[C] += 1;
  dfl q0 = df_split(qc[fidx(g, C, i, j, kk)]);
  dfl qp = df_split(qc[fidx(g, C, hi3[0], hi3[1], hi3[2])]);
  dfl qm = df_split(qc[fidx(g, C, lo3[0], lo3[1], lo3[2])]);
  dfl mu_hi = df_split(cf.mu_cc[fidx(g, 3, i, j, kk)]);
  dfl mu_lo = df_split(cf.mu_cc[fidx(g, 3, lo3[0], lo3[1], lo3[2])]);
  dfl L = df_mul(k.two_ih2[C], df_sub(df_mul(mu_hi, df_sub(qp, q0)), df_mul(mu_lo, df_sub(q0, qm))));
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    if (D == C) continue;
    const int E = edge_id(C, D);
    const double* qd = q[D];
    int a3[3] = {id3[0], id3[1], id3[2]};
    int b3[3] = {id3[0], id3[1], id3[2]};
    a3[D] += 1;
    b3[D] -= 1;
    dfl q_hi, q_lo;
    if (a3[D] >= g.n[D]) {
      q_hi = g.bc[2 * D + 1] < 0.0 ? df_neg(q0) : q0;
    } else {
      q_hi = df_split(qc[fidx(g, C, a3[0], a3[1], a3[2])]);
    }
    if (b3[D] < 0) {
      q_lo = g.bc[2 * D] < 0.0 ? df_neg(q0) : q0;
    } else {
      q_lo = df_split(qc[fidx(g, C, b3[0], b3[1], b3[2])]);
    }
    int eh[3] = {id3[0], id3[1], id3[2]};
    eh[D] += 1;
    dfl mue_hi = df_split(cf.mu_e[E][eidx(g, E, eh[0], eh[1], eh[2])]);
    dfl mue_lo = df_split(cf.mu_e[E][eidx(g, E, id3[0], id3[1], id3[2])]);
    int d1[3] = {id3[0], id3[1], id3[2]};
    d1[D] += 1;
    int d0[3] = {d1[0], d1[1], d1[2]};
    d0[C] -= 1;
    int c0[3] = {id3[0], id3[1], id3[2]};
    c0[C] -= 1;
    dfl dqd_hi = df_mul(df_sub(df_split(qd[fidx(g, D, d1[0], d1[1], d1[2])]),
                               df_split(qd[fidx(g, D, d0[0], d0[1], d0[2])])), k.ih[C]);
    dfl dqd_lo = df_mul(df_sub(df_split(qd[fidx(g, D, id3[0], id3[1], id3[2])]),
                               df_split(qd[fidx(g, D, c0[0], c0[1], c0[2])])), k.ih[C]);
    dfl f_hi = df_mul(mue_hi, df_add(df_mul(df_sub(q_hi, q0), k.ih[D]), dqd_hi));
    dfl f_lo = df_mul(mue_lo, df_add(df_mul(df_sub(q0, q_lo), k.ih[D]), dqd_lo));
    L = df_add(L, df_mul(df_sub(f_hi, f_lo), k.ih[D]));
  }
  return L;
}

template <int C>
__device__ __forceinline__ void stokes_row_df(const GridDev& g, const DfConst& k, const Coef<double>& cf,
                                              double inv_dt, double theta, const CVel<double>& q,
                                              const double* __restrict__ p, double* out, int i, int j, int kk) {
  int id3[3] = {i, j, kk};
  size_t id = fidx(g, C, i, j, kk);
  if (id3[C] == 0 || id3[C] == g.n[C]) {
    out[id] = 0.0;
    return;
  }
  double L = df_to_double(strain_df<C>(g, k, cf, q.q, i, j, kk));
  int lo3[3] = {i, j, kk};
  lo3[C] -= 1;
  double gp = (p[fidx(g, 3, i, j, kk)] - p[fidx(g, 3, lo3[0], lo3[1], lo3[2])]) * g.ih[C];
  out[id] = fma(-theta, L, cf.rho_face[C][id] * inv_dt * q.q[C][id] + gp);
}

__global__ void k_stokes_df(GridDev g, DfConst k, Coef<double> cf, double inv_dt, double theta, CVel<double> q,
                            const double* __restrict__ p, double* yu, double* yv, double* yw, double* yp) {
  int z = blockIdx.z;
  int nz = g.n[2];
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (z < nz) {
    if (i < g.n[0] + 1 && j < g.n[1]) stokes_row_df<0>(g, k, cf, inv_dt, theta, q, p, yu, i, j, z);
  } else if (z < 2 * nz) {
    if (i < g.n[0] && j < g.n[1] + 1) stokes_row_df<1>(g, k, cf, inv_dt, theta, q, p, yv, i, j, z - nz);
  } else if (z < 3 * nz + 1) {
    if (i < g.n[0] && j < g.n[1]) stokes_row_df<2>(g, k, cf, inv_dt, theta, q, p, yw, i, j, z - 2 * nz);
  } else {
    int kk = z - (3 * nz + 1);
    if (i < g.n[0] && j < g.n[1]) {
      double d = (q.q[0][fidx(g, 0, i + 1, j, kk)] - q.q[0][fidx(g, 0, i, j, kk)]) * g.ih[0] +
                 (q.q[1][fidx(g, 1, i, j + 1, kk)] - q.q[1][fidx(g, 1, i, j, kk)]) * g.ih[1] +
                 (q.q[2][fidx(g, 2, i, j, kk + 1)] - q.q[2][fidx(g, 2, i, j, kk)]) * g.ih[2];
      yp[fidx(g, 3, i, j, kk)] = -d;
    }
  }
}

static dfl host_split(double a) {
  dfl r;
  r.h = (float)a;
  r.l = (float)(a - (double)r.h);
  return r;
}

void launch_stokes_df(const GridDev& g, const Coef<double>& cf, double inv_dt, double theta, const double* x,
                      double* y, cudaStream_t st) {
  Packing pk = packing(g);
  CVel<double> q{{x + pk.off[0], x + pk.off[1], x + pk.off[2]}};
  const double* p = x + pk.off[3];
  DfConst k;
  for (int a = 0; a < 3; ++a) {
    k.ih[a] = host_split(g.ih[a]);
    k.two_ih2[a] = host_split(2.0 * g.ih2[a]);
  }
  dim3 grid(cdiv(g.n[0] + 1, BX), cdiv(g.n[1] + 1, BY), 4 * g.n[2] + 1);
  ktimer_begin(KC_STOKES, st);
  { k_stokes_df<<<grid, dim3(BX, BY), 0, st>>>(g, k, cf, inv_dt, theta, q, p, y + pk.off[0], y + pk.off[1],
                                               y + pk.off[2], y + pk.off[3]); WSI_COUNT(); }
  ktimer_end(KC_STOKES, st);
}

}  // namespace wsi
