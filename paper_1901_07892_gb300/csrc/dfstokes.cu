// Stokes matvec of the mixed path in double-float arithmetic.
//
// GB300 issues float64 arithmetic at about 1/64 of its float32 rate, and the
// float64 Stokes matvec (about 130 float64 operations per cell) is the
// largest single kernel of a time step.  Here every row
//     y_u = (rho/dt) q + G p - theta L_mu q,    y_p = -D q
// is evaluated with unevaluated float32 pairs (hi + lo): Dekker's exact
// product via fused multiply-add and Knuth's error-free sum of the leading
// parts (the trailing parts are added plainly, an error of ~2^-46 of the
// operands' magnitude, the class of a float64 operation on rounded inputs).
// The operands are split into (hi, lo) float32 pairs by integer operations
// on their bit patterns (47 significant bits kept) in separate streaming
// passes: the coefficients once per solve, the input vector once per
// matvec; the matvec then reads pairs (8 bytes, as many as a float64) and
// issues no split.  The float64 pipe sees one addition per row, which forms
// the float64 result.
// Magnitudes below 2^-126 ~ 1.2e-38 are flushed to zero, and below 2^-103
// only their leading 24 bits are kept.  Array offsets are 32-bit: every
// array holds fewer than 2^31 elements (checked when the grid is created).
#include <math.h>

#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;

struct DfConst {
  dfl ih[3];       // 1/h
  dfl two_ih2[3];  // 2/h^2
  dfl inv_dt;
  dfl mtheta;      // -theta
  unsigned pw;     // bit set: that constant is a power of two (bits 0-2 ih, 3-5 two_ih2, 6 mtheta, 7 inv_dt)
  float bcs[6];    // tangential ghost sign per wall
  int fs[3][3];    // strides of face array C along each axis
  int cs[3];       // strides of the cell arrays
  int es[3][3];    // strides of edge array E
};

__device__ __forceinline__ dfl ldp(const float2* __restrict__ a, int i) {
  const float2 v = __ldg(a + i);
  dfl r;
  r.h = v.x;
  r.l = v.y;
  return r;
}

// momentum row C at the interior C-face (i, j, kk); all operands pre-split
template <int C>
__device__ __forceinline__ double row_df(const GridDev& g, const DfConst& k, const DfCoef& cf, const DfVec& x, int i,
                                         int j, int kk) {
  const int id3[3] = {i, j, kk};
  const int fb = i + j * k.fs[C][1] + kk * k.fs[C][2];
  const int cb = i + j * k.cs[1] + kk * k.cs[2];  // the cell on the + side of the face
  const float2* __restrict__ qc = x.q[C];
  const int sC = k.fs[C][C];
  const dfl q0 = ldp(qc, fb);
  const dfl qp = ldp(qc, fb + sC), qm = ldp(qc, fb - sC);
  const dfl muh = ldp(cf.mu_cc, cb), mul = ldp(cf.mu_cc, cb - k.cs[C]);
  dfl L = df_mulc(df_sub(df_mul(muh, df_sub(qp, q0)), df_mul(mul, df_sub(q0, qm))), k.two_ih2[C], (k.pw >> (3 + C)) & 1);
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    if (D == C) continue;
    const int E = edge_id(C, D);
    const int sD = k.fs[C][D];
    dfl qh, ql;
    if (id3[D] + 1 < g.n[D]) {
      qh = ldp(qc, fb + sD);
    } else {
      qh = k.bcs[2 * D + 1] < 0.0f ? df_neg(q0) : q0;
    }
    if (id3[D] > 0) {
      ql = ldp(qc, fb - sD);
    } else {
      ql = k.bcs[2 * D] < 0.0f ? df_neg(q0) : q0;
    }
    const int eb = i + j * k.es[E][1] + kk * k.es[E][2];
    const dfl meh = ldp(cf.mu_e[E], eb + k.es[E][D]), mel = ldp(cf.mu_e[E], eb);
    const float2* __restrict__ qd = x.q[D];
    const int db = i + j * k.fs[D][1] + kk * k.fs[D][2];
    const int dD = k.fs[D][D], dC = k.fs[D][C];
    const dfl a1 = ldp(qd, db + dD), a0 = ldp(qd, db + dD - dC);
    const dfl b1 = ldp(qd, db), b0 = ldp(qd, db - dC);
    const bool pD = (k.pw >> D) & 1, pC = (k.pw >> C) & 1;
    const dfl fh = df_mul(meh, df_add(df_mulc(df_sub(qh, q0), k.ih[D], pD), df_mulc(df_sub(a1, a0), k.ih[C], pC)));
    const dfl fl = df_mul(mel, df_add(df_mulc(df_sub(q0, ql), k.ih[D], pD), df_mulc(df_sub(b1, b0), k.ih[C], pC)));
    L = df_add(L, df_mulc(df_sub(fh, fl), k.ih[D], pD));
  }
  const dfl rq = df_mul(df_mulc(ldp(cf.rho_face[C], fb), k.inv_dt, (k.pw >> 7) & 1), q0);
  const dfl gp = df_mulc(df_sub(ldp(x.p, cb), ldp(x.p, cb - k.cs[C])), k.ih[C], (k.pw >> C) & 1);
  return df_to_double(df_add(df_add(rq, gp), df_mulc(L, k.mtheta, (k.pw >> 6) & 1)));
}

template <int C>
__device__ __forceinline__ void stokes_row_df(const GridDev& g, const DfConst& k, const DfCoef& cf, const DfVec& x,
                                              double* out, int i, int j, int kk) {
  const int id3[3] = {i, j, kk};
  const int fb = i + j * k.fs[C][1] + kk * k.fs[C][2];
  out[fb] = (id3[C] == 0 || id3[C] == g.n[C]) ? 0.0 : row_df<C>(g, k, cf, x, i, j, kk);
}

// One thread per (i, j, k) evaluates the u-, v-, w- and p-rows there, so the
// blocks resident at a time work on the same few z-planes of every array and
// each array comes from DRAM about once.
__global__ void __launch_bounds__(256) k_stokes_df(GridDev g, DfConst k, DfCoef cf, DfVec x, double* yu, double* yv,
                                                   double* yw, double* yp) {
  const int kk = blockIdx.z;
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  if (i <= n0 && j < n1 && kk < n2) stokes_row_df<0>(g, k, cf, x, yu, i, j, kk);
  if (i < n0 && j <= n1 && kk < n2) stokes_row_df<1>(g, k, cf, x, yv, i, j, kk);
  if (i < n0 && j < n1 && kk <= n2) stokes_row_df<2>(g, k, cf, x, yw, i, j, kk);
  if (i < n0 && j < n1 && kk < n2) {
    const int f0 = i + j * k.fs[0][1] + kk * k.fs[0][2];
    const int f1 = i + j * k.fs[1][1] + kk * k.fs[1][2];
    const int f2 = i + j * k.fs[2][1] + kk * k.fs[2][2];
    const dfl dx = df_mulc(df_sub(ldp(x.q[0], f0 + 1), ldp(x.q[0], f0)), k.ih[0], k.pw & 1);
    const dfl dy = df_mulc(df_sub(ldp(x.q[1], f1 + k.fs[1][1]), ldp(x.q[1], f1)), k.ih[1], (k.pw >> 1) & 1);
    const dfl dz = df_mulc(df_sub(ldp(x.q[2], f2 + k.fs[2][2]), ldp(x.q[2], f2)), k.ih[2], (k.pw >> 2) & 1);
    yp[i + j * k.cs[1] + kk * k.cs[2]] = -df_to_double(df_add(df_add(dx, dy), dz));
  }
}

// x (float64) -> (hi, lo) pairs, n elements; four per thread
__global__ void k_df_split(const double* __restrict__ x, float2* out, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const dfl d = df_split(x[t]);
    out[t] = make_float2(d.h, d.l);
  }
}

void launch_df_split(const double* x, float2* out, size_t n, cudaStream_t st) {
  if (!n) return;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  { k_df_split<<<blocks, 256, 0, st>>>(x, out, n); WSI_COUNT(); }
}

static dfl host_split(double a) {
  dfl r;
  r.h = (float)a;
  r.l = (float)(a - (double)r.h);
  return r;
}

static bool host_pow2(const dfl& c) {
  int e = 0;
  return c.l == 0.0f && c.h != 0.0f && std::fabs(std::frexp((double)c.h, &e)) == 0.5;
}

void launch_stokes_df(const GridDev& g, const DfCoef& cf, double inv_dt, double theta, const float2* x, double* y,
                      cudaStream_t st) {
  Packing pk = packing(g);
  DfVec xv{{x + pk.off[0], x + pk.off[1], x + pk.off[2]}, x + pk.off[3]};
  DfConst k;
  for (int a = 0; a < 3; ++a) {
    k.ih[a] = host_split(g.ih[a]);
    k.two_ih2[a] = host_split(2.0 * g.ih2[a]);
  }
  k.inv_dt = host_split(inv_dt);
  k.mtheta = host_split(-theta);
  k.pw = 0;
  for (int a = 0; a < 3; ++a) {
    if (host_pow2(k.ih[a])) k.pw |= 1u << a;
    if (host_pow2(k.two_ih2[a])) k.pw |= 1u << (3 + a);
  }
  if (host_pow2(k.mtheta)) k.pw |= 1u << 6;
  if (host_pow2(k.inv_dt)) k.pw |= 1u << 7;
  for (int w = 0; w < 6; ++w) k.bcs[w] = (float)g.bc[w];
  const int n0 = g.n[0], n1 = g.n[1];
  for (int c = 0; c < 3; ++c) {
    const int fx = n0 + (c == 0), fy = n1 + (c == 1);
    k.fs[c][0] = 1;
    k.fs[c][1] = fx;
    k.fs[c][2] = fx * fy;
    const int ax = (c == 0 || c == 1) ? 1 : 0, ay = (c == 0 || c == 2) ? 1 : 0;
    k.es[c][0] = 1;
    k.es[c][1] = n0 + ax;
    k.es[c][2] = (n0 + ax) * (n1 + ay);
  }
  k.cs[0] = 1;
  k.cs[1] = n0;
  k.cs[2] = n0 * n1;
  dim3 grid(cdiv(g.n[0] + 1, BX), cdiv(g.n[1] + 1, BY), g.n[2] + 1);
  ktimer_begin(KC_STOKES, st);
  { k_stokes_df<<<grid, dim3(BX, BY), 0, st>>>(g, k, cf, xv, y + pk.off[0], y + pk.off[1], y + pk.off[2],
                                               y + pk.off[3]); WSI_COUNT(); }
  ktimer_end(KC_STOKES, st);
}

}  // namespace wsi
