// Stokes matvec of the mixed path in double-float arithmetic.
//
// GB300 issues float64 arithmetic at about 1/64 of its float32 rate, so
//     y_u = (rho/dt) q + G p - theta L_mu q,    y_p = -D q
// (Sec. 4.2.2) is evaluated on unnormalised float32 head/tail pairs
// (df.cuh: exact head differences and products, tails in plain float32;
// ~2^-46 of the operands' magnitude per operation), from operands split
// into (hi, lo) pairs by integer operations in streaming passes: the
// coefficients once per solve (with 1/dt folded into the face density), the
// input vector once per matvec.  One float64 addition per row forms the
// result.
//
// Flux form, marched along z.  L_mu q is the divergence of the stress:
// normal stresses 2 mu_cc dq_c/dx_c at cells and shear stresses
// mu_e (dq_c/dx_d + dq_d/dx_c) on edges.  Each is formed once per cell by one
// thread and shared: with the x-neighbours of its warp by shuffles (a warp
// covers 32 consecutive x-positions and writes the rows of the 30 inner
// ones), with the next z-level by keeping it in registers while the thread
// marches up its column of KC cells.  Only the y-neighbours' stresses are
// formed twice.  Compared with evaluating every row on its own (each shear
// stress four times), this is about half the float32 instructions.
// Tangential ghosts across walls follow the wall's sign; faces on walls hold
// zero and their rows are written as zero.
// Magnitudes below 2^-126 ~ 1.2e-38 are flushed to zero, and below 2^-103
// only their leading 24 bits are kept.  Array offsets are 32-bit: every
// array holds fewer than 2^31 elements (checked when the grid is created).
#include <math.h>

#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "internal.h"

namespace wsi {

static constexpr int FX = 30;  // x-positions written per warp (32 lanes, one halo lane each side)
static constexpr int FBY = 4;  // warps (y-rows) per block
static constexpr int FKC = 16; // z-levels per thread
// planes ahead whose operands each thread asks L2 to fetch (measured at
// 256^3: 711 us per launch at 2 against 930 us without; 1 and 3 are slower)
static constexpr int FPD = 2;

struct HtConst {
  ht ih[3];       // 1/h
  ht two_ih2[3];  // 2/h^2
  ht mtheta;      // -theta
  unsigned pw;    // power-of-two flags: bits 0-2 ih, 3-5 two_ih2, 6 mtheta
  float bcs[6];   // tangential ghost sign per wall (x-, x+, y-, y+, z-, z+)
  int n[3];
};

__device__ __forceinline__ ht ldh(const float2* __restrict__ a, int i) { return ht_of(__ldg(a + i)); }
__device__ __forceinline__ void pf_l2(const float2* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ ht shfl_up1(ht a) {
  return ht{__shfl_up_sync(0xffffffffu, a.h, 1), __shfl_up_sync(0xffffffffu, a.t, 1)};
}
__device__ __forceinline__ ht shfl_down1(ht a) {
  return ht{__shfl_down_sync(0xffffffffu, a.h, 1), __shfl_down_sync(0xffffffffu, a.t, 1)};
}

// rho/dt q + G p - theta L as a float64
__device__ __forceinline__ double row_out(const HtConst& K, ht rq, ht gp, ht L) {
  return ht_dbl(ht_add(ht_add(rq, gp), ht_k(L, K.mtheta, (K.pw >> 6) & 1)));
}

__global__ void __launch_bounds__(32 * FBY) k_stokes_df(HtConst K, DfCoef cf, DfVec x, double* yu, double* yv,
                                                        double* yw, double* yp) {
  const int nx = K.n[0], ny = K.n[1], nz = K.n[2];
  const int lane = threadIdx.x;
  const int i = blockIdx.x * FX + lane - 1;
  const int j = blockIdx.y * FBY + threadIdx.y;
  if (j >= ny) return;  // uniform over the warp
  const int k0 = blockIdx.z * FKC;
  const int k1 = min(k0 + FKC, nz);
  const bool cI = i >= 0 && i < nx;  // a cell column
  const bool fI = i >= 0 && i <= nx; // an x-face / x-edge column
  const bool lane_rows = lane >= 1 && lane <= FX;
  const int ic = clampi(i, 0, nx - 1), iff = clampi(i, 0, nx), icm = clampi(i - 1, 0, nx - 1);
  const bool hiX = i >= nx, loX = i - 1 < 0;  // column i / i-1 outside the cells: x-ghost
  // strides
  const int su1 = nx + 1, su2 = (nx + 1) * ny;  // u faces
  const int sv1 = nx, sv2 = nx * (ny + 1);      // v faces
  const int sc1 = nx, sc2 = nx * ny;            // cells, w faces
  const int sxy1 = nx + 1, sxy2 = (nx + 1) * (ny + 1);
  const int sxz1 = nx + 1, sxz2 = (nx + 1) * ny;
  const int syz1 = nx, syz2 = nx * (ny + 1);
  const float bxl = K.bcs[0], bxh = K.bcs[1], byl = K.bcs[2], byh = K.bcs[3], bzl = K.bcs[4], bzh = K.bcs[5];
  const bool pxk = K.pw & 1, pyk = (K.pw >> 1) & 1, pzk = (K.pw >> 2) & 1;
  const float2* __restrict__ U = x.q[0];
  const float2* __restrict__ V = x.q[1];
  const float2* __restrict__ W = x.q[2];
  const float2* __restrict__ P = x.p;
  const ht ihx = K.ih[0], ihy = K.ih[1], ihz = K.ih[2];

  // w at (column i or its x-ghost, row jj or its y-ghost, level kk in 0..nz)
  auto w_at = [&](int col_i, bool xghost, float xs, int jj, int kk) -> ht {
    float s = xghost ? xs : 1.f;
    if (jj < 0) { jj = 0; s *= byl; } else if (jj >= ny) { jj = ny - 1; s *= byh; }
    return ht_sgn(ldh(W, col_i + jj * sc1 + kk * sc2), s);
  };
  // shear stresses on the z-level kk edges (0 <= kk <= nz) from the fields at
  // levels kk - 1 (lo) and kk (hi), ghosts already applied:
  // xz at (i, j), yz at (i, j) and at (i, j + 1)
  auto zedges = [&](int kk, ht u_lo, ht u_hi, ht v_lo, ht v_hi, ht vj_lo, ht vj_hi, ht& txz, ht& tyz, ht& tyzj) {
    const ht wc = w_at(ic, hiX, bxh, j, kk);      // w at column i (x-edge column; ghost at i = nx)
    const ht wm = w_at(icm, loX, bxl, j, kk);     // w at column i - 1
    const ht wjm = w_at(ic, false, 1.f, j - 1, kk);
    const ht wjp = w_at(ic, false, 1.f, j + 1, kk);
    const ht w0 = ldh(W, ic + j * sc1 + kk * sc2);
    txz = ht_mul(ldh(cf.mu_e[1], iff + j * sxz1 + kk * sxz2),
                 ht_add(ht_k(ht_sub(u_hi, u_lo), ihz, pzk), ht_k(ht_sub(wc, wm), ihx, pxk)));
    tyz = ht_mul(ldh(cf.mu_e[2], ic + j * syz1 + kk * syz2),
                 ht_add(ht_k(ht_sub(v_hi, v_lo), ihz, pzk), ht_k(ht_sub(w0, wjm), ihy, pyk)));
    tyzj = ht_mul(ldh(cf.mu_e[2], ic + (j + 1) * syz1 + kk * syz2),
                  ht_add(ht_k(ht_sub(vj_hi, vj_lo), ihz, pzk), ht_k(ht_sub(wjp, w0), ihy, pyk)));
  };

  // ---- prologue: fields at level k0, z-edges at level k0, stresses of k0 - 1
  ht u_k = ldh(U, iff + j * su1 + k0 * su2);
  ht v_k = ldh(V, ic + j * sv1 + k0 * sv2);
  ht vj_k = ldh(V, ic + (j + 1) * sv1 + k0 * sv2);
  ht w_k = ldh(W, ic + j * sc1 + k0 * sc2);
  ht txz_k, tyz_k, tyzj_k;
  ht nzz_km1{0.f, 0.f}, p_km1{0.f, 0.f};
  {
    ht u_m, v_m, vj_m;
    if (k0 > 0) {
      u_m = ldh(U, iff + j * su1 + (k0 - 1) * su2);
      v_m = ldh(V, ic + j * sv1 + (k0 - 1) * sv2);
      vj_m = ldh(V, ic + (j + 1) * sv1 + (k0 - 1) * sv2);
      const ht w_m = ldh(W, ic + j * sc1 + (k0 - 1) * sc2);
      nzz_km1 = ht_mul(ldh(cf.mu_cc, ic + j * sc1 + (k0 - 1) * sc2), ht_sub(w_k, w_m));
      p_km1 = ldh(P, ic + j * sc1 + (k0 - 1) * sc2);
    } else {
      u_m = ht_sgn(u_k, bzl);
      v_m = ht_sgn(v_k, bzl);
      vj_m = ht_sgn(vj_k, bzl);
    }
    zedges(k0, u_m, u_k, v_m, v_k, vj_m, vj_k, txz_k, tyz_k, tyzj_k);
  }

  for (int k = k0; k < k1; ++k) {
    const int kp = k + 1;
    {
      // bring this thread's operands FPD levels ahead into L2: the loads of
      // that level then hit L2 instead of DRAM (no register, no wait)
      const int kq = k + FPD;
      if (kq < nz) {
        pf_l2(U + iff + j * su1 + kq * su2);
        pf_l2(V + ic + j * sv1 + kq * sv2);
        pf_l2(W + ic + j * sc1 + kq * sc2);
        pf_l2(P + ic + j * sc1 + kq * sc2);
        pf_l2(cf.mu_cc + ic + j * sc1 + kq * sc2);
        pf_l2(cf.mu_e[0] + iff + j * sxy1 + kq * sxy2);
        pf_l2(cf.mu_e[1] + iff + j * sxz1 + kq * sxz2);
        pf_l2(cf.mu_e[2] + ic + j * syz1 + kq * syz2);
        pf_l2(cf.rho_face[0] + iff + j * su1 + kq * su2);
        pf_l2(cf.rho_face[1] + ic + j * sv1 + kq * sv2);
        pf_l2(cf.rho_face[2] + ic + j * sc1 + kq * sc2);
      }
    }
    // ---- level k + 1: fields and z-edge shear stresses
    ht u_kp, v_kp, vj_kp;
    if (kp < nz) {
      u_kp = ldh(U, iff + j * su1 + kp * su2);
      v_kp = ldh(V, ic + j * sv1 + kp * sv2);
      vj_kp = ldh(V, ic + (j + 1) * sv1 + kp * sv2);
    } else {
      u_kp = ht_sgn(u_k, bzh);
      v_kp = ht_sgn(v_k, bzh);
      vj_kp = ht_sgn(vj_k, bzh);
    }
    const ht w_kp = ldh(W, ic + j * sc1 + kp * sc2);
    ht txz_kp, tyz_kp, tyzj_kp;
    zedges(kp, u_k, u_kp, v_k, v_kp, vj_k, vj_kp, txz_kp, tyz_kp, tyzj_kp);

    // ---- level k: normal stresses and the xy shear stresses at rows j, j + 1
    const int cb = ic + j * sc1 + k * sc2;
    const ht mu_c = ldh(cf.mu_cc, cb);
    const ht u_ip = ldh(U, clampi(i + 1, 0, nx) + j * su1 + k * su2);
    const ht nxx = ht_mul(mu_c, ht_sub(u_ip, u_k));
    const ht nyy = ht_mul(mu_c, ht_sub(vj_k, v_k));
    const ht nzz = ht_mul(mu_c, ht_sub(w_kp, w_k));
    ht nyy_m{0.f, 0.f};
    if (j > 0) nyy_m = ht_mul(ldh(cf.mu_cc, cb - sc1), ht_sub(v_k, ldh(V, ic + (j - 1) * sv1 + k * sv2)));
    // u at rows j - 1, j + 1 of column i (y-ghosts)
    const ht u_jm = j > 0 ? ldh(U, iff + (j - 1) * su1 + k * su2) : ht_sgn(u_k, byl);
    const ht u_jp = j + 1 < ny ? ldh(U, iff + (j + 1) * su1 + k * su2) : ht_sgn(u_k, byh);
    // v at columns i, i - 1 of rows j, j + 1 (x-ghosts)
    const ht vx = hiX ? ht_sgn(v_k, bxh) : v_k;
    const ht vjx = hiX ? ht_sgn(vj_k, bxh) : vj_k;
    const ht vm = ht_sgn(ldh(V, icm + j * sv1 + k * sv2), loX ? bxl : 1.f);
    const ht vjm = ht_sgn(ldh(V, icm + (j + 1) * sv1 + k * sv2), loX ? bxl : 1.f);
    const int eb = iff + j * sxy1 + k * sxy2;
    const ht txy = ht_mul(ldh(cf.mu_e[0], eb), ht_add(ht_k(ht_sub(u_k, u_jm), ihy, pyk), ht_k(ht_sub(vx, vm), ihx, pxk)));
    const ht txyj =
        ht_mul(ldh(cf.mu_e[0], eb + sxy1), ht_add(ht_k(ht_sub(u_jp, u_k), ihy, pyk), ht_k(ht_sub(vjx, vjm), ihx, pxk)));

    // ---- neighbours along x from the adjacent lanes
    const ht nxx_im = shfl_up1(nxx);
    const ht txy_ip = shfl_down1(txy);
    const ht txz_ip = shfl_down1(txz_k);

    const ht p_k = ldh(P, cb);
    if (lane_rows && fI) {
      // u-row at x-face i
      double out = 0.0;
      if (i > 0 && i < nx) {
        const ht L = ht_add(ht_add(ht_k(ht_sub(nxx, nxx_im), K.two_ih2[0], (K.pw >> 3) & 1),
                                   ht_k(ht_sub(txyj, txy), ihy, pyk)),
                            ht_k(ht_sub(txz_kp, txz_k), ihz, pzk));
        const ht rq = ht_mul(ldh(cf.rho_face[0], iff + j * su1 + k * su2), u_k);
        const ht gp = ht_k(ht_sub(p_k, ldh(P, cb - 1)), ihx, pxk);
        out = row_out(K, rq, gp, L);
      }
      yu[iff + j * su1 + k * su2] = out;
    }
    if (lane_rows && cI) {
      // v-row at y-face j (face 0 and face ny are walls)
      double out = 0.0;
      if (j > 0) {
        const ht L = ht_add(ht_add(ht_k(ht_sub(nyy, nyy_m), K.two_ih2[1], (K.pw >> 4) & 1),
                                   ht_k(ht_sub(txy_ip, txy), ihx, pxk)),
                            ht_k(ht_sub(tyz_kp, tyz_k), ihz, pzk));
        const ht rq = ht_mul(ldh(cf.rho_face[1], ic + j * sv1 + k * sv2), v_k);
        const ht gp = ht_k(ht_sub(p_k, ldh(P, cb - sc1)), ihy, pyk);
        out = row_out(K, rq, gp, L);
      }
      yv[ic + j * sv1 + k * sv2] = out;
      if (j == ny - 1) yv[ic + ny * sv1 + k * sv2] = 0.0;
      // w-row at z-face k (face 0 and face nz are walls)
      out = 0.0;
      if (k > 0) {
        const ht L = ht_add(ht_add(ht_k(ht_sub(nzz, nzz_km1), K.two_ih2[2], (K.pw >> 5) & 1),
                                   ht_k(ht_sub(txz_ip, txz_k), ihx, pxk)),
                            ht_k(ht_sub(tyzj_k, tyz_k), ihy, pyk));
        const ht rq = ht_mul(ldh(cf.rho_face[2], cb), w_k);
        const ht gp = ht_k(ht_sub(p_k, p_km1), ihz, pzk);
        out = row_out(K, rq, gp, L);
      }
      yw[cb] = out;
      if (k == nz - 1) yw[cb + sc2] = 0.0;
      // continuity row at the cell
      const ht dq = ht_add(ht_add(ht_k(ht_sub(u_ip, u_k), ihx, pxk), ht_k(ht_sub(vj_k, v_k), ihy, pyk)),
                           ht_k(ht_sub(w_kp, w_k), ihz, pzk));
      yp[cb] = -ht_dbl(dq);
    }
    // ---- carry to level k + 1
    u_k = u_kp;
    v_k = v_kp;
    vj_k = vj_kp;
    w_k = w_kp;
    txz_k = txz_kp;
    tyz_k = tyz_kp;
    tyzj_k = tyzj_kp;
    nzz_km1 = nzz;
    p_km1 = p_k;
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

// up to eight arrays split in one launch: (scale_k x_k) -> (hi, lo) pairs;
// blockIdx.y selects the array
struct SplitSet {
  const double* x[8];
  float2* out[8];
  size_t n[8];
  double scale[8];
  int count;
};

__global__ void k_df_split_set(SplitSet s) {
  const int a = blockIdx.y;
  if (a >= s.count) return;
  const double* __restrict__ x = s.x[a];
  float2* out = s.out[a];
  const size_t n = s.n[a];
  const double sc = s.scale[a];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const dfl d = df_split(sc == 1.0 ? x[t] : sc * x[t]);
    out[t] = make_float2(d.h, d.l);
  }
}

void launch_df_split_set(const double* const* x, float2* const* out, const size_t* n, const double* scale, int count,
                         cudaStream_t st) {
  SplitSet s;
  size_t nmax = 0;
  s.count = count < 8 ? count : 8;
  for (int a = 0; a < s.count; ++a) {
    s.x[a] = x[a];
    s.out[a] = out[a];
    s.n[a] = n[a];
    s.scale[a] = scale[a];
    nmax = std::max(nmax, n[a]);
  }
  if (!nmax) return;
  const int blocks = (int)std::min<size_t>((nmax + 255) / 256, 152 * 4);
  { k_df_split_set<<<dim3(blocks, s.count), 256, 0, st>>>(s); WSI_COUNT(); }
}

// (s x) (float64 product, one rounding) -> (hi, lo) pairs
__global__ void k_df_split_scaled(const double* __restrict__ x, double s, float2* out, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const dfl d = df_split(s * x[t]);
    out[t] = make_float2(d.h, d.l);
  }
}

void launch_df_split_scaled(const double* x, double s, float2* out, size_t n, cudaStream_t st) {
  if (!n) return;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  { k_df_split_scaled<<<blocks, 256, 0, st>>>(x, s, out, n); WSI_COUNT(); }
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

void launch_stokes_df(const GridDev& g, const DfCoef& cf, double theta, const float2* x, double* y,
                      cudaStream_t st) {
  Packing pk = packing(g);
  DfVec xv{{x + pk.off[0], x + pk.off[1], x + pk.off[2]}, x + pk.off[3]};
  HtConst k;
  k.pw = 0;
  for (int a = 0; a < 3; ++a) {
    const dfl ih = host_split(g.ih[a]), t2 = host_split(2.0 * g.ih2[a]);
    k.ih[a] = ht{ih.h, ih.l};
    k.two_ih2[a] = ht{t2.h, t2.l};
    if (host_pow2(ih)) k.pw |= 1u << a;
    if (host_pow2(t2)) k.pw |= 1u << (3 + a);
    k.n[a] = g.n[a];
  }
  const dfl mt = host_split(-theta);
  k.mtheta = ht{mt.h, mt.l};
  if (host_pow2(mt)) k.pw |= 1u << 6;
  for (int w = 0; w < 6; ++w) k.bcs[w] = (float)g.bc[w];
  dim3 grid(cdiv(g.n[0] + 1, FX), cdiv(g.n[1], FBY), cdiv(g.n[2], FKC));
  ktimer_begin(KC_STOKES, st);
  { k_stokes_df<<<grid, dim3(32, FBY), 0, st>>>(k, cf, xv, y + pk.off[0], y + pk.off[1], y + pk.off[2],
                                                y + pk.off[3]); WSI_COUNT(); }
  ktimer_end(KC_STOKES, st);
}

}  // namespace wsi
