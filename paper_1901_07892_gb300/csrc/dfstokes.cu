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
// marches up its column of FKC cells.  Only the y-neighbours' stresses are
// formed twice.
//
// Operand staging.  The eleven split arrays (u, v, w, p; rho_x, rho_y,
// rho_z, mu_cc, mu_xy, mu_xz, mu_yz) are stored with an even row pitch so
// that every row starts on a 16-byte boundary, and a block of FBY warps
// copies, level by level, the 34 x (FBY + 2) tile of each array that its
// rows and their neighbours read into shared memory with tensor-memory-access
// (TMA) copies: one thread issues the eleven copies of a level, an mbarrier
// counts their bytes, and a ring of NST levels keeps the copies of the next
// level in flight while the current two are read.  The x origin of every
// tile is even (2 elements of 8 bytes), as TMA requires; rows and levels
// outside an array read as zero and are never used unghosted.
//
// Tangential ghosts across walls follow the wall's sign; faces on walls hold
// zero and their rows are written as zero.  With an open top the top w-row is
// formed too: the ghost cell above takes minus the normal stress below, the
// pressure ghost is -p, the top edges' shear stresses come from the z-edge
// pass of the last level.  Magnitudes below 2^-126 ~ 1.2e-38
// are flushed to zero, and below 2^-103 only their leading 24 bits are kept.
// Array offsets are 32-bit: every array holds fewer than 2^31 elements
// (checked when the grid is created).
#include <cuda.h>
#include <math.h>

#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "internal.h"

namespace wsi {

static constexpr int FX = 30;    // x-positions written per warp (32 lanes, one halo lane each side)
static constexpr int FBY = 4;    // warps (y-rows) per block
static constexpr int FKC = 16;   // z-levels per block
static constexpr int TX = 34;    // tile columns: x = FX bx - 2 .. FX bx + 31
static constexpr int TY = FBY + 2;  // tile rows: y = FBY by - 1 .. FBY by + FBY
static constexpr int TILE = 208;    // float2 slots per tile (TX TY = 204, padded to a multiple of 128 bytes)
static constexpr int NST = 3;       // levels in the ring: two read, one in flight
static constexpr int STAGE = DF_NARR * TILE;
static constexpr int SMEM_BYTES = NST * STAGE * 8 + NST * 8;
static constexpr uint32_t STAGE_TX = DF_NARR * TX * TY * 8;  // bytes the copies of one level deliver

struct HtConst {
  ht ih[3];       // 1/h
  ht two_ih2[3];  // 2/h^2
  ht mtheta;      // -theta
  unsigned pw;    // power-of-two flags: bits 0-2 ih, 3-5 two_ih2, 6 mtheta
  float bcs[6];   // tangential ghost sign per wall (x-, x+, y-, y+, z-, z+)
  int n[3];
  int open_top;
};

struct DfMaps {
  CUtensorMap m[DF_NARR];
};

namespace tma {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// wait for phase `parity` of the barrier; false after about 2^22 polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 3-D tile copy global -> shared, completion counted on `bar`
__device__ __forceinline__ void load3(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

}  // namespace tma

__device__ __forceinline__ ht shfl_up1(ht a) {
  return ht{__shfl_up_sync(0xffffffffu, a.h, 1), __shfl_up_sync(0xffffffffu, a.t, 1)};
}
__device__ __forceinline__ ht shfl_down1(ht a) {
  return ht{__shfl_down_sync(0xffffffffu, a.h, 1), __shfl_down_sync(0xffffffffu, a.t, 1)};
}

// a * c for a grid constant c: P2 (every constant a power of two, known at
// compile time) scales both parts exactly; otherwise the constant's own flag
template <bool P2>
__device__ __forceinline__ ht hk(ht a, ht c, bool pow2) {
  return P2 ? ht{a.h * c.h, a.t * c.h} : ht_k(a, c, pow2);
}

// rho/dt q + G p - theta L as a float64
template <bool P2>
__device__ __forceinline__ double row_out(const HtConst& K, ht rq, ht gp, ht L) {
  return ht_dbl(ht_add(ht_add(rq, gp), hk<P2>(L, K.mtheta, (K.pw >> 6) & 1)));
}

// P2: 1/h, 2/h^2 and theta are all powers of two (uniform power-of-two
// spacings), so that every multiplication by a grid constant is an exact
// scaling
template <bool P2>
__global__ void __launch_bounds__(32 * FBY) k_stokes_df(const __grid_constant__ DfMaps maps, const HtConst K,
                                                        double* yu, double* yv, double* yw, double* yp, int* err) {
  extern __shared__ __align__(128) float2 dsm[];
  const int nx = K.n[0], ny = K.n[1], nz = K.n[2];
  const int lane = threadIdx.x, tid = threadIdx.y * 32 + lane;
  const int xs = blockIdx.x * FX - 2, ys = blockIdx.y * FBY - 1;  // tile origin (x even)
  const int i = xs + 1 + lane;
  const int j = blockIdx.y * FBY + threadIdx.y;
  const bool jrow = j < ny;  // warp-uniform; warps past the last row only take part in the staging
  const int k0 = blockIdx.z * FKC;
  const int k1 = min(k0 + FKC, nz);
  const int tmax = k1 - k0 + 1;  // ring levels t = 0 .. tmax hold z-levels k0 - 1 .. k1
  const uint32_t sm0 = tma::saddr(dsm), bar0 = sm0 + NST * STAGE * 8;

  // (thread 0) the eleven copies of ring level t into slot t % NST
  auto issue = [&](int t) {
    const int s = t % NST;
    const uint32_t bar = bar0 + 8 * s;
    tma::mbar_expect_tx(bar, STAGE_TX);
    for (int a = 0; a < DF_NARR; ++a)
      tma::load3(sm0 + (uint32_t)((s * DF_NARR + a) * TILE * 8), &maps.m[a], bar, xs, ys, k0 - 1 + t);
  };
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) tma::mbar_init(bar0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int t = 0; t < NST && t <= tmax; ++t) issue(t);
  }
  __syncthreads();
  bool ok = true;
  auto wait = [&](int t) {
    if (!tma::mbar_wait(bar0 + 8 * (t % NST), (t / NST) & 1)) ok = false;
  };
  // slot of ring level t, tile of array a in it, and its element at grid row jj, column ii
  auto slot = [&](int t) -> const float2* { return dsm + (t % NST) * STAGE; };
  auto tile = [&](const float2* S, int a) -> const float2* { return S + a * TILE; };
  auto at = [&](const float2* T, int jj, int ii) -> ht { return ht_of(T[(jj - ys) * TX + (ii - xs)]); };

  const bool cI = i >= 0 && i < nx;  // a cell column
  const bool fI = i >= 0 && i <= nx; // an x-face / x-edge column
  const bool lane_rows = lane >= 1 && lane <= FX;
  const int ic = clampi(i, 0, nx - 1), iff = clampi(i, 0, nx), icm = clampi(i - 1, 0, nx - 1);
  const int ifp = clampi(i + 1, 0, nx);
  const bool hiX = i >= nx, loX = i - 1 < 0;  // column i / i-1 outside the cells: x-ghost
  // output strides (unpadded float64 rows)
  const int su1 = nx + 1, su2 = (nx + 1) * ny;  // u faces
  const int sv1 = nx, sv2 = nx * (ny + 1);      // v faces
  const int sc1 = nx, sc2 = nx * ny;            // cells, w faces
  const float bxl = K.bcs[0], bxh = K.bcs[1], byl = K.bcs[2], byh = K.bcs[3], bzl = K.bcs[4], bzh = K.bcs[5];
  const bool pxk = K.pw & 1, pyk = (K.pw >> 1) & 1, pzk = (K.pw >> 2) & 1;
  const ht ihx = K.ih[0], ihy = K.ih[1], ihz = K.ih[2];

  // w of a level's tile at (column col_i or its x-ghost, row jj or its y-ghost)
  auto w_at = [&](const float2* Tw, int col_i, bool xghost, float xsg, int jj) -> ht {
    float s = xghost ? xsg : 1.f;
    if (jj < 0) { jj = 0; s *= byl; } else if (jj >= ny) { jj = ny - 1; s *= byh; }
    return ht_sgn(at(Tw, jj, col_i), s);
  };
  // shear stresses on the z-level edges of ring level t from the fields at the
  // level below (lo) and at it (hi), ghosts already applied:
  // xz at (i, j), yz at (i, j) and at (i, j + 1)
  auto zedges = [&](const float2* S, ht u_lo, ht u_hi, ht v_lo, ht v_hi, ht vj_lo, ht vj_hi, ht& txz, ht& tyz,
                    ht& tyzj) {
    const float2* Tw = tile(S, DF_W);
    const float2* Te = tile(S, DF_MU_YZ);
    const ht wc = w_at(Tw, ic, hiX, bxh, j);   // w at column i (x-edge column; ghost at i = nx)
    const ht wm = w_at(Tw, icm, loX, bxl, j);  // w at column i - 1
    const ht wjm = w_at(Tw, ic, false, 1.f, j - 1);
    const ht wjp = w_at(Tw, ic, false, 1.f, j + 1);
    const ht w0 = at(Tw, j, ic);
    txz = ht_mul(at(tile(S, DF_MU_XZ), j, iff),
                 ht_add(hk<P2>(ht_sub(u_hi, u_lo), ihz, pzk), hk<P2>(ht_sub(wc, wm), ihx, pxk)));
    tyz = ht_mul(at(Te, j, ic), ht_add(hk<P2>(ht_sub(v_hi, v_lo), ihz, pzk), hk<P2>(ht_sub(w0, wjm), ihy, pyk)));
    tyzj = ht_mul(at(Te, j + 1, ic), ht_add(hk<P2>(ht_sub(vj_hi, vj_lo), ihz, pzk), hk<P2>(ht_sub(wjp, w0), ihy, pyk)));
  };

  // ---- prologue: fields at level k0 (ring 1), z-edges at level k0, stresses of k0 - 1 (ring 0)
  wait(0);
  wait(1);
  const float2* S0 = slot(0);
  const float2* S1 = slot(1);
  ht u_k = at(tile(S1, DF_U), j, iff);
  ht v_k = at(tile(S1, DF_V), j, ic);
  ht vj_k = at(tile(S1, DF_V), j + 1, ic);
  ht w_k = at(tile(S1, DF_W), j, ic);
  ht txz_k, tyz_k, tyzj_k;
  ht nzz_km1{0.f, 0.f}, p_km1{0.f, 0.f};
  {
    ht u_m, v_m, vj_m;
    if (k0 > 0) {
      u_m = at(tile(S0, DF_U), j, iff);
      v_m = at(tile(S0, DF_V), j, ic);
      vj_m = at(tile(S0, DF_V), j + 1, ic);
      const ht w_m = at(tile(S0, DF_W), j, ic);
      nzz_km1 = ht_mul(at(tile(S0, DF_MU_CC), j, ic), ht_sub(w_k, w_m));
      p_km1 = at(tile(S0, DF_P), j, ic);
    } else {
      u_m = ht_sgn(u_k, bzl);
      v_m = ht_sgn(v_k, bzl);
      vj_m = ht_sgn(vj_k, bzl);
    }
    zedges(S1, u_m, u_k, v_m, v_k, vj_m, vj_k, txz_k, tyz_k, tyzj_k);
  }
  __syncthreads();  // ring slot 0 is free
  if (tid == 0 && NST <= tmax) issue(NST);

  for (int k = k0; k < k1; ++k) {
    const int t = k - k0 + 1, tp = t + 1;  // ring levels of k and k + 1
    const float2* Sk = slot(t);
    const float2* Sp = slot(tp);
    wait(tp);
    // ---- level k + 1: fields and z-edge shear stresses
    ht u_kp, v_kp, vj_kp;
    if (k + 1 < nz) {
      u_kp = at(tile(Sp, DF_U), j, iff);
      v_kp = at(tile(Sp, DF_V), j, ic);
      vj_kp = at(tile(Sp, DF_V), j + 1, ic);
    } else {
      u_kp = ht_sgn(u_k, bzh);
      v_kp = ht_sgn(v_k, bzh);
      vj_kp = ht_sgn(vj_k, bzh);
    }
    const ht w_kp = at(tile(Sp, DF_W), j, ic);
    ht txz_kp, tyz_kp, tyzj_kp;
    zedges(Sp, u_k, u_kp, v_k, v_kp, vj_k, vj_kp, txz_kp, tyz_kp, tyzj_kp);

    // ---- level k: normal stresses and the xy shear stresses at rows j, j + 1
    const float2* TU = tile(Sk, DF_U);
    const float2* TV = tile(Sk, DF_V);
    const float2* TP = tile(Sk, DF_P);
    const float2* TM = tile(Sk, DF_MU_CC);
    const float2* TE = tile(Sk, DF_MU_XY);
    const ht mu_c = at(TM, j, ic);
    const ht u_ip = at(TU, j, ifp);
    const ht nxx = ht_mul(mu_c, ht_sub(u_ip, u_k));
    const ht nyy = ht_mul(mu_c, ht_sub(vj_k, v_k));
    const ht nzz = ht_mul(mu_c, ht_sub(w_kp, w_k));
    ht nyy_m{0.f, 0.f};
    if (j > 0) nyy_m = ht_mul(at(TM, j - 1, ic), ht_sub(v_k, at(TV, j - 1, ic)));
    // u at rows j - 1, j + 1 of column i (y-ghosts)
    const ht u_jm = j > 0 ? at(TU, j - 1, iff) : ht_sgn(u_k, byl);
    const ht u_jp = j + 1 < ny ? at(TU, j + 1, iff) : ht_sgn(u_k, byh);
    // v at columns i, i - 1 of rows j, j + 1 (x-ghosts)
    const ht vx = hiX ? ht_sgn(v_k, bxh) : v_k;
    const ht vjx = hiX ? ht_sgn(vj_k, bxh) : vj_k;
    const ht vm = ht_sgn(at(TV, j, icm), loX ? bxl : 1.f);
    const ht vjm = ht_sgn(at(TV, j + 1, icm), loX ? bxl : 1.f);
    const ht txy = ht_mul(at(TE, j, iff), ht_add(hk<P2>(ht_sub(u_k, u_jm), ihy, pyk), hk<P2>(ht_sub(vx, vm), ihx, pxk)));
    const ht txyj =
        ht_mul(at(TE, j + 1, iff), ht_add(hk<P2>(ht_sub(u_jp, u_k), ihy, pyk), hk<P2>(ht_sub(vjx, vjm), ihx, pxk)));
    // ---- neighbours along x from the adjacent lanes
    const ht nxx_im = shfl_up1(nxx);
    const ht txy_ip = shfl_down1(txy);
    const ht txz_ip = shfl_down1(txz_k);

    const ht p_k = at(TP, j, ic);
    if (jrow && lane_rows && fI) {
      // u-row at x-face i
      double out = 0.0;
      if (i > 0 && i < nx) {
        const ht L = ht_add(ht_add(hk<P2>(ht_sub(nxx, nxx_im), K.two_ih2[0], (K.pw >> 3) & 1),
                                   hk<P2>(ht_sub(txyj, txy), ihy, pyk)),
                            hk<P2>(ht_sub(txz_kp, txz_k), ihz, pzk));
        const ht rq = ht_mul(at(tile(Sk, DF_RHO_X), j, iff), u_k);
        const ht gp = hk<P2>(ht_sub(p_k, at(TP, j, ic - 1)), ihx, pxk);
        out = row_out<P2>(K, rq, gp, L);
      }
      yu[iff + j * su1 + k * su2] = out;
    }
    if (jrow && lane_rows && cI) {
      const int cb = ic + j * sc1 + k * sc2;
      // v-row at y-face j (face 0 and face ny are walls)
      double out = 0.0;
      if (j > 0) {
        const ht L = ht_add(ht_add(hk<P2>(ht_sub(nyy, nyy_m), K.two_ih2[1], (K.pw >> 4) & 1),
                                   hk<P2>(ht_sub(txy_ip, txy), ihx, pxk)),
                            hk<P2>(ht_sub(tyz_kp, tyz_k), ihz, pzk));
        const ht rq = ht_mul(at(tile(Sk, DF_RHO_Y), j, ic), v_k);
        const ht gp = hk<P2>(ht_sub(p_k, at(TP, j - 1, ic)), ihy, pyk);
        out = row_out<P2>(K, rq, gp, L);
      }
      yv[ic + j * sv1 + k * sv2] = out;
      if (j == ny - 1) yv[ic + ny * sv1 + k * sv2] = 0.0;
      // w-row at z-face k (face 0 and face nz are walls)
      out = 0.0;
      if (k > 0) {
        const ht L = ht_add(ht_add(hk<P2>(ht_sub(nzz, nzz_km1), K.two_ih2[2], (K.pw >> 5) & 1),
                                   hk<P2>(ht_sub(txz_ip, txz_k), ihx, pxk)),
                            hk<P2>(ht_sub(tyzj_k, tyz_k), ihy, pyk));
        const ht rq = ht_mul(at(tile(Sk, DF_RHO_Z), j, ic), w_k);
        const ht gp = hk<P2>(ht_sub(p_k, p_km1), ihz, pzk);
        out = row_out<P2>(K, rq, gp, L);
      }
      yw[cb] = out;
      if (k == nz - 1 && !K.open_top) yw[cb + sc2] = 0.0;
      // continuity row at the cell
      const ht dq = ht_add(ht_add(hk<P2>(ht_sub(u_ip, u_k), ihx, pxk), hk<P2>(ht_sub(vj_k, v_k), ihy, pyk)),
                           hk<P2>(ht_sub(w_kp, w_k), ihz, pzk));
      yp[cb] = -ht_dbl(dq);
    }
    if (k == nz - 1 && K.open_top) {
      // w-row at the open top's face nz (warp-uniform branch: all lanes shuffle)
      const ht txz_kp_ip = shfl_down1(txz_kp);
      if (jrow && lane_rows && cI) {
        const ht L = ht_add(ht_add(hk<P2>(ht_sub(ht_sgn(nzz, -1.f), nzz), K.two_ih2[2], (K.pw >> 5) & 1),
                                   hk<P2>(ht_sub(txz_kp_ip, txz_kp), ihx, pxk)),
                            hk<P2>(ht_sub(tyzj_kp, tyz_kp), ihy, pyk));
        const ht rq = ht_mul(at(tile(Sp, DF_RHO_Z), j, ic), w_kp);
        const ht gp = hk<P2>(ht_sub(ht_sgn(p_k, -1.f), p_k), ihz, pzk);
        yw[ic + j * sc1 + nz * sc2] = row_out<P2>(K, rq, gp, L);
      }
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
    __syncthreads();  // ring slot of level k is free
    if (tid == 0 && t + NST <= tmax) issue(t + NST);
  }
  if (!ok) {
    atomicExch(err, 1);
    // a wait gave up: give the copies still in flight time to land before the
    // block's shared memory is released
    if (tid == 0)
      for (int t = (tmax + 1 > NST ? tmax + 1 - NST : 0); t <= tmax; ++t) tma::mbar_wait(bar0 + 8 * (t % NST), (t / NST) & 1);
  }
}

// Split of up to DF_NARR float64 arrays into (hi, lo) pairs with padded rows:
// row r of array a (cols[a] elements) goes to out[a] + r pitch[a], the padding
// is written as zero; one warp per row, the rows of every array in one launch
// (blockIdx.y selects the array).
struct PadSplit {
  const double* x[DF_NARR];
  float2* out[DF_NARR];
  double scale[DF_NARR];
  int cols[DF_NARR], pitch[DF_NARR], nrows[DF_NARR];
  int count;
};

__global__ void __launch_bounds__(256) k_df_split_pad(PadSplit s) {
  const int a = blockIdx.y;
  if (a >= s.count) return;
  const int cols = s.cols[a], pitch = s.pitch[a], nr = s.nrows[a];
  const double sc = s.scale[a];
  const int lane = threadIdx.x & 31;
  const int wstride = gridDim.x * (blockDim.x >> 5);
  for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nr; r += wstride) {
    const double* __restrict__ xr = s.x[a] + (size_t)r * cols;
    float2* orow = s.out[a] + (size_t)r * pitch;
    // four loads in flight per lane before the splits and stores
    for (int c0 = lane; c0 < pitch; c0 += 128) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + 32 * u;
        v[u] = c < cols ? __ldg(xr + c) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + 32 * u;
        if (c < pitch) {
          const dfl d = df_split(sc == 1.0 ? v[u] : sc * v[u]);
          orow[c] = make_float2(d.h, d.l);
        }
      }
    }
  }
}

static void split_pad(const DfOperands& o, const int* which, const double* const* x, const double* scale, int count,
                      cudaStream_t st) {
  PadSplit s;
  int rmax = 0;
  s.count = count;
  for (int q = 0; q < count; ++q) {
    const int a = which[q];
    s.x[q] = x[q];
    s.out[q] = o.a[a];
    s.scale[q] = scale[q];
    s.cols[q] = o.cols[a];
    s.pitch[q] = o.pitch[a];
    s.nrows[q] = o.rows[a] * o.levels[a];
    rmax = std::max(rmax, s.nrows[q]);
  }
  if (!rmax) return;
  const int blocks = std::min(cdiv(rmax, 8), 152 * 8);
  { k_df_split_pad<<<dim3(blocks, count), 256, 0, st>>>(s); WSI_COUNT(); }
}

void df_operands_shape(const GridDev& g, DfOperands& o) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  // (columns, rows, levels) of each array: faces of component c have one
  // more along c, edges in the (c, d) plane one more along c and d
  const int dims[DF_NARR][3] = {
      {nx + 1, ny, nz},      {nx, ny + 1, nz},     {nx, ny, nz + 1},     {nx, ny, nz},
      {nx + 1, ny, nz},      {nx, ny + 1, nz},     {nx, ny, nz + 1},     {nx, ny, nz},
      {nx + 1, ny + 1, nz},  {nx + 1, ny, nz + 1}, {nx, ny + 1, nz + 1}};
  for (int a = 0; a < DF_NARR; ++a) {
    o.cols[a] = dims[a][0];
    o.rows[a] = dims[a][1];
    o.levels[a] = dims[a][2];
    o.pitch[a] = (dims[a][0] + 1) & ~1;  // 16-byte rows
  }
}

size_t df_operand_elems(const DfOperands& o, int a) { return (size_t)o.pitch[a] * o.rows[a] * o.levels[a]; }

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int df_operands_encode(DfOperands& o) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return WSI_ERR_CUDA;
    encode = (EncodeTiledFn)fn;
  }
  DfMaps* m = new DfMaps;
  for (int a = 0; a < DF_NARR; ++a) {
    const cuuint64_t dim[3] = {(cuuint64_t)o.cols[a], (cuuint64_t)o.rows[a], (cuuint64_t)o.levels[a]};
    const cuuint64_t stride[2] = {(cuuint64_t)o.pitch[a] * 8, (cuuint64_t)o.pitch[a] * o.rows[a] * 8};
    const cuuint32_t box[3] = {TX, TY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&m->m[a], CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)o.a[a], dim, stride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      delete m;
      return WSI_ERR_CUDA;
    }
  }
  o.maps = m;
  return WSI_OK;
}

void df_operands_release(DfOperands& o) {
  delete static_cast<DfMaps*>(o.maps);
  o.maps = nullptr;
}

void df_split_coefs(const DfOperands& o, const double* const rho[3], const double* const mu_e[3], const double* mu_cc,
                    double inv_dt, cudaStream_t st) {
  const int which[7] = {DF_RHO_X, DF_RHO_Y, DF_RHO_Z, DF_MU_CC, DF_MU_XY, DF_MU_XZ, DF_MU_YZ};
  const double* x[7] = {rho[0], rho[1], rho[2], mu_cc, mu_e[0], mu_e[1], mu_e[2]};
  const double sc[7] = {inv_dt, inv_dt, inv_dt, 1.0, 1.0, 1.0, 1.0};
  split_pad(o, which, x, sc, 7, st);
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

void launch_stokes_df(const GridDev& g, const DfOperands& o, double theta, const double* x, double* y, int* err,
                      cudaStream_t st) {
  Packing pk = packing(g);
  {
    const int which[4] = {DF_U, DF_V, DF_W, DF_P};
    const double* xs[4] = {x + pk.off[0], x + pk.off[1], x + pk.off[2], x + pk.off[3]};
    const double sc[4] = {1.0, 1.0, 1.0, 1.0};
    split_pad(o, which, xs, sc, 4, st);
  }
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
  k.open_top = g.open_top;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_stokes_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    cudaFuncSetAttribute(k_stokes_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  dim3 grid(cdiv(g.n[0] + 1, FX), cdiv(g.n[1], FBY), cdiv(g.n[2], FKC));
  const DfMaps& m = *static_cast<const DfMaps*>(o.maps);
  ktimer_begin(KC_STOKES, st);
  if (k.pw == 0x7Fu)
    k_stokes_df<true><<<grid, dim3(32, FBY), SMEM_BYTES, st>>>(m, k, y + pk.off[0], y + pk.off[1], y + pk.off[2],
                                                               y + pk.off[3], err);
  else
    k_stokes_df<false><<<grid, dim3(32, FBY), SMEM_BYTES, st>>>(m, k, y + pk.off[0], y + pk.off[1], y + pk.off[2],
                                                                y + pk.off[3], err);
  WSI_COUNT();
  ktimer_end(KC_STOKES, st);
}

}  // namespace wsi
