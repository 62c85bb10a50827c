// Consistent mass/momentum transport (Sec. 4.2.2) and level-set advection
// (Sec. 4.2.1), with the bounded cubic-upwind (CUI) limiter.
//
// Transport of the C-face density (and, for the convective term, of the C
// momentum) is a divergence over face-centred control volumes.  Each flux
// through a control-volume face is shared by the two C-faces on either side
// of it, so the kernel computes it once: a 32 x 8 block owns a tile of
// C-faces in (x, y) and marches up a chunk of z-planes; x- and y-fluxes of a
// plane go through shared memory (one halo column / row computed by the edge
// threads), the z-flux of the plane below is kept in a register.  The
// limiter's inputs are staged per plane in shared memory (see k_transport).
//
// Storage and arithmetic type T: float64 on the plain path; float32 on the
// mixed path, where the step keeps float32 shadow copies of the transported
// fields (an explicit stencil apply; reading float32 avoids a float64->float32
// conversion per load, which issues on GB300's narrow float64 pipe).
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;

// Division-free bounded CUI: with num = qC - qU and den = qD - qU,
// t = num/den lies in a branch interval iff num*sign(den) lies in den-scaled
// bounds, and qU + t_f den = qU + {3 num, 5 num/6 + den/3, den, num}.
template <typename T>
__device__ __forceinline__ T cui(T qU, T qC, T qD) {
  T den = qD - qU;
  T num = qC - qU;
  if (den == T(0)) return qC;
  T a = den > T(0) ? num : -num;  // num * sign(den)
  T D = den > T(0) ? den : -den;  // t = a / D
  T f;
  if (a > T(0) && T(13) * a <= T(2) * D)
    f = T(3) * num;
  else if (T(13) * a > T(2) * D && T(5) * a <= T(4) * D)
    f = num * T(5.0 / 6.0) + den * T(1.0 / 3.0);
  else if (T(5) * a > T(4) * D && a <= D)
    f = den;
  else
    f = num;
  return qU + f;
}

// Entry m of the C-face array along axis D extended by two ghost layers: the
// stored index it maps to and the velocity ghost sign.  Density ghosts are
// even mirrors; velocity ghosts are odd about wall faces when C == D (the wall
// face itself is zero; even about an open top, where dw/dz = 0) and take the
// wall's tangential sign across D != C.
template <int C, int D, typename T>
__device__ __forceinline__ int mirror_index(const GridDev& g, int m, T& s) {
  const int n = g.n[D] + (C == D ? 1 : 0);
  int mm = m;
  s = T(1);
  if (m < 0) {
    const int gl = -m;
    if (C == D) {
      mm = gl;
      s = T(-1);
    } else {
      mm = gl - 1;
      s = gbc<T>(g, 2 * D);
    }
  } else if (m >= n) {
    const int gl = m - (n - 1);
    if (C == D) {
      mm = (n - 1) - gl;
      s = (D == 2 && g.open_top) ? T(1) : T(-1);
    } else {
      mm = n - gl;
      s = gbc<T>(g, 2 * D + 1);
    }
  }
  return clampi(mm, 0, n - 1);
}

// limited value from the four taps for advective velocity adv
template <typename T>
__device__ __forceinline__ T lim4(T t0, T t1, T t2, T t3, T adv) {
  return adv > T(0) ? cui<T>(t0, t1, t2) : cui<T>(t3, t2, t1);
}

// advective velocity at the D-direction CV face at position m of the C-face
// column through (i, j, k): C == D: mean of C-faces m and m+1; else mean of
// the two D-faces at D-index m adjacent along C
template <int C, int D, typename T>
__device__ __forceinline__ T adv_at(const GridDev& g, const CVel<T>& vel, int i, int j, int k, int m) {
  int a[3] = {i, j, k};
  a[D] = m;
  if (C == D) {
    const size_t id = fidx(g, C, a[0], a[1], a[2]);
    const size_t st = C == 0 ? 1 : (C == 1 ? (size_t)g.n[0] : (size_t)g.n[0] * g.n[1]);
    return T(0.5) * (vel.q[C][id] + vel.q[C][id + st]);
  }
  const size_t id1 = fidx(g, D, a[0], a[1], a[2]);
  const size_t sc = C == 0 ? 1 : (C == 1 ? (size_t)(g.n[0] + (D == 0)) : (size_t)(g.n[0] + (D == 0)) * (g.n[1] + (D == 1)));
  return T(0.5) * (vel.q[D][id1 - sc] + vel.q[D][id1]);
}

// Asynchronous 4- or 8-byte copies global -> shared (cp.async), grouped per
// staged plane
template <typename T>
__device__ __forceinline__ void cpa(T* dst, const T* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Per z-plane the block stages the transported field (and, for C, the
// velocity component) of its tile with a two-entry halo in x and y into a
// ring of NPL plane slots in shared memory, by asynchronous copies issued
// three planes ahead (the ghosts beyond walls are mirrored through the copies'
// source addresses; the velocity ghosts' signs, and the inlet data across a
// Dirichlet inlet, are applied by the staging thread once its copies have
// landed).  The four limiter taps of every x- and y-flux then come from plane
// k's slot, the z taps of a thread's own column from the slots of planes
// k-1 .. k+2 (a plane beyond a wall reads its mirror image's slot with the
// mirror's sign).  Advective velocities are loaded one plane ahead into
// registers.  Two block barriers per plane: one publishes the plane, one the
// x- and y-fluxes.
static constexpr int NPL = 6;  // planes k-2 .. k+3

// inl (C == 2 with the velocity only, else null): tangential data of w on
// the x- plane of a Dirichlet inlet, (nz+1) x ny; the ghosts of w across it
// are then 2 inl - (mirror image)
template <int C, bool WITHV, typename T>
__global__ void __launch_bounds__(BX* BY) k_transport(GridDev g, CVel<T> vel, const T* __restrict__ rho, T* out,
                                                      int zchunk, const T* __restrict__ inl) {
  constexpr int HX = BX + 4, HY = BY + 4, NS = (HX * HY + BX * BY - 1) / (BX * BY);
  constexpr int PL = HX * HY;
  __shared__ __align__(16) T sR[NPL][PL];
  __shared__ __align__(16) T sQ[WITHV ? NPL : 1][WITHV ? PL : 1];
  __shared__ T sFx[BY][BX + 1];
  __shared__ T sFy[BY + 1][BX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int i = x0 + tx, j = y0 + ty;
  const int e0 = ext(g, C, 0), e1 = ext(g, C, 1), e2 = ext(g, C, 2);
  const bool inside = i < e0 && j < e1;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(k0 + zchunk, e2);
  const int ox = (C == 0) ? -1 : 0, oy = (C == 1) ? -1 : 0, oz = (C == 2) ? -1 : 0;
  const size_t plane = (size_t)e0 * e1;
  const T* __restrict__ qc = vel.q[C];
  // staged entries of this thread: in-plane offset (mirrored) and velocity sign
  int soff[NS];
  T ssg[NS];
  constexpr bool INL = C == 2 && WITHV;
  int sinl[INL ? NS : 1];  // inlet data row of an x-ghost entry, else -1
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    const int t = tid + r * BX * BY;
    soff[r] = -1;
    ssg[r] = T(1);
    if (INL) sinl[r] = -1;
    if (t < PL) {
      const int hy = t / HX, hx = t - hy * HX;
      T sx, sy;
      const int mx = mirror_index<C, 0, T>(g, x0 - 2 + hx, sx);
      const int my = mirror_index<C, 1, T>(g, y0 - 2 + hy, sy);
      soff[r] = my * e0 + mx;
      ssg[r] = sx * sy;
      if (INL && inl && x0 - 2 + hx < 0) sinl[r] = my;
    }
  }
  // ring slot of plane p (k0 - 2 <= p; planes k - 2 .. k + 3 are distinct)
  auto slot = [&](int p) { return (p - k0 + 2) % NPL; };
  // copies of plane p into its slot (planes outside the array: none); one
  // group per call
  auto issue = [&](int p) {
    if (p >= 0 && p < e2) {
      const int s = slot(p);
#pragma unroll
      for (int r = 0; r < NS; ++r) {
        const int t = tid + r * BX * BY;
        if (soff[r] >= 0) {
          const size_t a = (size_t)p * plane + soff[r];
          cpa<T>(&sR[s][t], rho + a);
          if (WITHV) cpa<T>(&sQ[WITHV ? s : 0][WITHV ? t : 0], qc + a);
        }
      }
    }
    cpa_commit();
  };
  // signs and inlet data of this thread's entries of plane p, once landed
  auto fix = [&](int p) {
    if (!WITHV || p < 0 || p >= e2) return;
    const int s = slot(p);
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      const int t = tid + r * BX * BY;
      if (soff[r] < 0) continue;
      const bool inl_here = INL && sinl[INL ? r : 0] >= 0;
      if (ssg[r] == T(1) && !inl_here) continue;
      T q = ssg[r] * sQ[WITHV ? s : 0][WITHV ? t : 0];
      if (inl_here) q += T(2) * inl[(size_t)p * e1 + sinl[INL ? r : 0]];
      sQ[WITHV ? s : 0][WITHV ? t : 0] = q;
    }
  };
  // z taps of this thread's column at plane m (mirrored beyond the walls)
  const int own = (ty + 2) * HX + (tx + 2);
  auto ztap = [&](int m, T& r_, T& q_) {
    T sz;
    const int mm = mirror_index<C, 2, T>(g, m, sz);
    const int s = slot(mm);
    r_ = sR[s][own];
    q_ = WITHV ? sz * sQ[WITHV ? s : 0][WITHV ? own : 0] : T(0);
  };
  // fluxes this thread forms at plane k, and their advective velocities: the
  // two entries of each are found at offsets that move by one z-level of
  // their array per plane (computed once; 32-bit, every array holds fewer
  // than 2^31 entries)
  struct Adv {
    T xh, xl, yh, yl, zh;
  };
  const int mxh = i + ox + 1, mxl = i + ox, myh = j + oy + 1, myl = j + oy;
  const bool fxh0 = inside && (C != 0 || mxh <= g.n[0] - 1), fxl0 = inside && tx == 0 && (C != 0 || mxl >= 0);
  const bool fyh0 = inside && (C != 1 || myh <= g.n[1] - 1), fyl0 = inside && ty == 0 && (C != 1 || myl >= 0);
  // offset at level k0 of the first entry, and the distance to the second
  auto adv_off = [&](int D, int m, int& d) -> int {
    int a[3] = {clampi(i, 0, g.n[0]), clampi(j, 0, g.n[1]), k0};
    a[D] = m;
    if (C == D) {
      d = C == 0 ? 1 : (C == 1 ? g.n[0] : g.n[0] * g.n[1]);
      return (int)fidx(g, C, a[0], a[1], a[2]);
    }
    d = -(C == 0 ? 1 : (C == 1 ? (g.n[0] + (D == 0)) : (g.n[0] + (D == 0)) * (g.n[1] + (D == 1))));
    return (int)fidx(g, D, a[0], a[1], a[2]);
  };
  int dxh = 0, dxl = 0, dyh = 0, dyl = 0, dzh = 0;
  const int oxh = fxh0 ? adv_off(0, mxh, dxh) : 0, oxl = fxl0 ? adv_off(0, mxl, dxl) : 0;
  const int oyh = fyh0 ? adv_off(1, myh, dyh) : 0, oyl = fyl0 ? adv_off(1, myl, dyl) : 0;
  const int ozh = inside ? adv_off(2, k0 + oz + 1, dzh) : 0;
  // one z-level of the u, v, w arrays
  const int lx = (g.n[0] + 1) * g.n[1], ly = g.n[0] * (g.n[1] + 1), lz = g.n[0] * g.n[1];
  const T* __restrict__ U_ = vel.q[0];
  const T* __restrict__ V_ = vel.q[1];
  const T* __restrict__ W_ = vel.q[2];
  auto adv_load = [&](int k) {
    Adv a{T(0), T(0), T(0), T(0), T(0)};
    const int idC = (C == 0) ? i : ((C == 1) ? j : k);
    const bool wall = idC == 0 || idC == g.n[C];
    const int dk = k - k0;
    if ((C == 0) || !wall) {
      if (fxh0) { const int o = oxh + dk * lx; a.xh = T(0.5) * (U_[o] + U_[o + dxh]); }
      if (fxl0) { const int o = oxl + dk * lx; a.xl = T(0.5) * (U_[o] + U_[o + dxl]); }
    }
    if ((C == 1) || !wall) {
      if (fyh0) { const int o = oyh + dk * ly; a.yh = T(0.5) * (V_[o] + V_[o + dyh]); }
      if (fyl0) { const int o = oyl + dk * ly; a.yl = T(0.5) * (V_[o] + V_[o + dyl]); }
    }
    if (inside && ((C == 2) || !wall) && (C != 2 || k + oz + 1 <= g.n[2] - 1)) {
      const int o = ozh + dk * lz;
      a.zh = T(0.5) * (W_[o] + W_[o + dzh]);
    }
    return a;
  };

  // prologue: planes k0-2 .. k0+2 in flight, advective velocities of plane k0
#pragma unroll 1
  for (int p = k0 - 2; p <= k0 + 2; ++p) issue(p);
  Adv cur = adv_load(k0);
  T Fz_lo = T(0);
  for (int k = k0; k < k1; ++k) {
    issue(k + 3);
    const Adv nxt = k + 1 < k1 ? adv_load(k + 1) : Adv{T(0), T(0), T(0), T(0), T(0)};
    cpa_wait<1>();  // planes up to k + 2 have landed (this thread's copies)
    if (k == k0) {
#pragma unroll 1
      for (int p = k0 - 2; p <= k0 + 2; ++p) fix(p);
    } else {
      fix(k + 2);
    }
    __syncthreads();  // plane k + 2 published
    const int s = slot(k);
    const int idC = (C == 0) ? i : ((C == 1) ? j : k);
    const bool wall = idC == 0 || idC == g.n[C];
    T Fz_hi = T(0);
    if (inside) {
      const T* R_ = sR[s];
      const T* Q_ = sQ[WITHV ? s : 0];
      // x-fluxes: hi through the CV face above i (taps i-1 .. i+2), lo below (taps i-2 .. i+1)
      T hi = T(0), lo = T(0);
      const int hr = (ty + 2) * HX;
      if (cur.xh != T(0)) {
        hi = cur.xh * lim4<T>(R_[hr + tx + 1], R_[hr + tx + 2], R_[hr + tx + 3], R_[hr + tx + 4], cur.xh);
        if (WITHV) hi *= lim4<T>(Q_[hr + tx + 1], Q_[hr + tx + 2], Q_[hr + tx + 3], Q_[hr + tx + 4], cur.xh);
      }
      if (cur.xl != T(0)) {
        lo = cur.xl * lim4<T>(R_[hr + tx], R_[hr + tx + 1], R_[hr + tx + 2], R_[hr + tx + 3], cur.xl);
        if (WITHV) lo *= lim4<T>(Q_[hr + tx], Q_[hr + tx + 1], Q_[hr + tx + 2], Q_[hr + tx + 3], cur.xl);
      }
      sFx[ty][tx + 1] = hi;
      if (tx == 0) sFx[ty][0] = lo;
      // y-fluxes
      hi = T(0);
      lo = T(0);
      const int hc = tx + 2;
      if (cur.yh != T(0)) {
        hi = cur.yh * lim4<T>(R_[(ty + 1) * HX + hc], R_[(ty + 2) * HX + hc], R_[(ty + 3) * HX + hc],
                              R_[(ty + 4) * HX + hc], cur.yh);
        if (WITHV)
          hi *= lim4<T>(Q_[(ty + 1) * HX + hc], Q_[(ty + 2) * HX + hc], Q_[(ty + 3) * HX + hc],
                        Q_[(ty + 4) * HX + hc], cur.yh);
      }
      if (cur.yl != T(0)) {
        lo = cur.yl * lim4<T>(R_[ty * HX + hc], R_[(ty + 1) * HX + hc], R_[(ty + 2) * HX + hc],
                              R_[(ty + 3) * HX + hc], cur.yl);
        if (WITHV)
          lo *= lim4<T>(Q_[ty * HX + hc], Q_[(ty + 1) * HX + hc], Q_[(ty + 2) * HX + hc],
                        Q_[(ty + 3) * HX + hc], cur.yl);
      }
      sFy[ty + 1][tx] = hi;
      if (ty == 0) sFy[0][tx] = lo;
      // z-fluxes through the CV faces above (taps k-1 .. k+2) and, at the
      // chunk start, below (taps k-2 .. k+1)
      if (k == k0) {
        Fz_lo = T(0);
        const int mzl = k + oz;
        if (((C == 2) || !wall) && (C != 2 || mzl >= 0)) {
          const T adv = adv_at<C, 2, T>(g, vel, i, j, k, mzl);
          T r4[4], q4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) ztap(k - 2 + q, r4[q], q4[q]);
          Fz_lo = adv * lim4<T>(r4[0], r4[1], r4[2], r4[3], adv);
          if (WITHV) Fz_lo *= lim4<T>(q4[0], q4[1], q4[2], q4[3], adv);
        }
      }
      if (cur.zh != T(0)) {
        T r4[4], q4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) ztap(k - 1 + q, r4[q], q4[q]);
        Fz_hi = cur.zh * lim4<T>(r4[0], r4[1], r4[2], r4[3], cur.zh);
        if (WITHV) Fz_hi *= lim4<T>(q4[0], q4[1], q4[2], q4[3], cur.zh);
      }
    }
    __syncthreads();  // x- and y-fluxes published
    if (inside) {
      const T r = (sFx[ty][tx + 1] - sFx[ty][tx]) * ginv<T>(g, 0) + (sFy[ty + 1][tx] - sFy[ty][tx]) * ginv<T>(g, 1) +
                  (Fz_hi - Fz_lo) * ginv<T>(g, 2);
      out[(size_t)k * plane + (size_t)j * e0 + i] = wall ? T(0) : r;
      Fz_lo = Fz_hi;
    }
    cur = nxt;
  }
  cpa_wait<0>();  // no copies in flight when the block ends
}

// z-chunk of the transport kernels: long marches amortise the chunk start,
// but the grid must still fill the GPU (about 8 blocks per SM)
int transport_chunk(int ex, int ey, int ez) {
  const long long base = (long long)cdiv(ex, BX) * cdiv(ey, BY);
  int c = 32;
  while (c > 4 && base * cdiv(ez, c) < 152LL * 8) c /= 2;
  return c;
}

template <bool WITHV, typename T>
static void transport_all(const GridDev& g, const CVel<T>& v, const T* const rho[3], T* const out[3],
                          const T* inlet_w, cudaStream_t st) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  int zc = transport_chunk(n0 + 1, n1, n2);
  { k_transport<0, WITHV, T><<<dim3(cdiv(n0 + 1, BX), cdiv(n1, BY), cdiv(n2, zc)), dim3(BX, BY), 0, st>>>(
      g, v, rho[0], out[0], zc, nullptr); WSI_COUNT(); }
  zc = transport_chunk(n0, n1 + 1, n2);
  { k_transport<1, WITHV, T><<<dim3(cdiv(n0, BX), cdiv(n1 + 1, BY), cdiv(n2, zc)), dim3(BX, BY), 0, st>>>(
      g, v, rho[1], out[1], zc, nullptr); WSI_COUNT(); }
  zc = transport_chunk(n0, n1, n2 + 1);
  { k_transport<2, WITHV, T><<<dim3(cdiv(n0, BX), cdiv(n1, BY), cdiv(n2 + 1, zc)), dim3(BX, BY), 0, st>>>(
      g, v, rho[2], out[2], zc, WITHV ? inlet_w : nullptr); WSI_COUNT(); }
}

template <typename T>
void launch_transport_flux(const GridDev& g, const T* const vel[3], const T* const rho[3], bool with_velocity,
                           T* const out[3], cudaStream_t st, const T* inlet_w) {
  CVel<T> v{{vel[0], vel[1], vel[2]}};
  ktimer_begin(KC_TRANSPORT, st);
  {
    // algorithmic bytes: per component rho_C, u, v, w (advective
    // velocities), q_C with the velocity, the result
    const double F = (double)(fsize(g, 0) + fsize(g, 1) + fsize(g, 2));
    ktimer_bytes(KC_TRANSPORT, sizeof(T) * F * (with_velocity ? 6.0 : 5.0));
  }
  if (with_velocity)
    transport_all<true, T>(g, v, rho, out, inlet_w, st);
  else
    transport_all<false, T>(g, v, rho, out, nullptr, st);
  ktimer_end(KC_TRANSPORT, st);
}
template void launch_transport_flux<double>(const GridDev&, const double* const[3], const double* const[3], bool,
                                            double* const[3], cudaStream_t, const double*);
template void launch_transport_flux<float>(const GridDev&, const float* const[3], const float* const[3], bool,
                                           float* const[3], cudaStream_t, const float*);

template <typename Ti, typename To>
__global__ void k_lincomb(size_t n, double a, const Ti* __restrict__ x, double b, const Ti* __restrict__ y, double c,
                          const Ti* __restrict__ z, To* out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  // coefficients of +-1 and 0 skip their multiplication (float64 operations
  // are scarce); the common forms are x - y and x + c z
  const bool a1 = a == 1.0, b1 = b == 1.0, bm1 = b == -1.0, c1 = c == 1.0, cm1 = c == -1.0;
  for (; t < n; t += stride) {
    double s = a1 ? (double)x[t] : a * (double)x[t];
    if (y) s = b1 ? s + (double)y[t] : (bm1 ? s - (double)y[t] : fma(b, (double)y[t], s));
    if (z) s = c1 ? s + (double)z[t] : (cm1 ? s - (double)z[t] : fma(c, (double)z[t], s));
    out[t] = (To)s;
  }
}

// float64 inputs, float32 arithmetic and output: the inputs are rounded by
// integer operations (d2f_fast), keeping the float64 pipe idle
__global__ void k_lincomb_tof(size_t n, float a, const double* __restrict__ x, float b, const double* __restrict__ y,
                              float c, const double* __restrict__ z, float* out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; t < n; t += stride) {
    float s = a * d2f_fast(x[t]);
    if (y) s += b * d2f_fast(y[t]);
    if (z) s += c * d2f_fast(z[t]);
    out[t] = s;
  }
}

// the two SSP-RK3 stage velocities of Sec. 4.2.2 in float32 from one pass over
// u^n, u^{n-1} (and u^{n+1,k} in later cycles), and optionally the float32
// copy of u^n; the same arithmetic as k_lincomb_tof for each output
__global__ void k_rk_vel_tof(size_t n, const double* __restrict__ un, const double* __restrict__ unm1,
                             const double* __restrict__ uk, float* u1, float* u2, float* un32) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const float a = d2f_fast(un[t]), b = d2f_fast(unm1[t]);
    if (uk) {
      const float q = d2f_fast(uk[t]);
      u1[t] = 1.0f * q;
      u2[t] = 0.375f * q + 0.75f * a + -0.125f * b;
    } else {
      u1[t] = 2.0f * a + -1.0f * b;
      u2[t] = 1.5f * a + -0.5f * b;
    }
    if (un32) un32[t] = 1.0f * a;
  }
}

// same in float32 arithmetic (float32 inputs and outputs)
__global__ void k_lincomb_f(size_t n, float a, const float* __restrict__ x, float b, const float* __restrict__ y,
                            float c, const float* __restrict__ z, float* out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; t < n; t += stride) {
    float s = a * x[t];
    if (y) s += b * y[t];
    if (z) s += c * z[t];
    out[t] = s;
  }
}

static int lc_blocks(size_t n) {
  int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  return blocks < 1 ? 1 : blocks;
}

void launch_rk_velocities_f32(size_t n, const double* un, const double* unm1, const double* uk, float* u1, float* u2,
                              float* un32, cudaStream_t st) {
  { k_rk_vel_tof<<<lc_blocks(n), 256, 0, st>>>(n, un, unm1, uk, u1, u2, un32); WSI_COUNT(); }
}

void launch_lincomb(size_t n, double a, const double* x, double b, const double* y, double c, const double* z,
                    double* out, cudaStream_t st) {
  { k_lincomb<double, double><<<lc_blocks(n), 256, 0, st>>>(n, a, x, b, y, c, z, out); WSI_COUNT(); }
}
void launch_lincomb_to_f32(size_t n, double a, const double* x, double b, const double* y, double c,
                           const double* z, float* out, cudaStream_t st) {
  { k_lincomb_tof<<<lc_blocks(n), 256, 0, st>>>(n, (float)a, x, (float)b, y, (float)c, z, out); WSI_COUNT(); }
}
void launch_lincomb_f32(size_t n, float a, const float* x, float b, const float* y, float c, const float* z,
                        float* out, cudaStream_t st) {
  { k_lincomb_f<<<lc_blocks(n), 256, 0, st>>>(n, a, x, b, y, c, z, out); WSI_COUNT(); }
}
// out = a*x64 + b*y32 + c*z32 in float64
__global__ void k_lincomb_mix(size_t n, double a, const double* __restrict__ x, double b, const float* __restrict__ y,
                              double c, const float* __restrict__ z, double* out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; t < n; t += stride) out[t] = a * x[t] + b * f2d_fast(y[t]) + c * f2d_fast(z[t]);
}
void launch_lincomb_mix(size_t n, double a, const double* x, double b, const float* y, double c, const float* z,
                        double* out, cudaStream_t st) {
  { k_lincomb_mix<<<lc_blocks(n), 256, 0, st>>>(n, a, x, b, y, c, z, out); WSI_COUNT(); }
}

// ================================================================ level set
// Same staging as k_transport: per z-plane the tile of phi^{n+1/2} with a
// halo of H cells (Neumann mirror ghosts applied while staging) in shared
// memory, the z taps in a 2H-entry register window, the face velocities
// loaded before the staging barrier.  H = 2 for the CUI limiter, 4 for
// xsPPM7 (seven-cell upwind-biased stencils).
template <typename T>
__device__ __forceinline__ int ls_mirror(int m, int n) {
  // repeated even reflection (grids thinner than the halo reflect again)
  for (int it = 0; it < 8; ++it) {
    if (m < 0) m = -m - 1;
    else if (m >= n) m = 2 * n - 1 - m;
  }
  return clampi(m, 0, n - 1);
}

template <typename T>
__device__ __forceinline__ T mm2(T a, T b) {
  return (a > T(0) && b > T(0)) ? fmin(a, b) : ((a < T(0) && b < T(0)) ? fmax(a, b) : T(0));
}
template <typename T>
__device__ __forceinline__ T mm4(T a, T b, T c, T d) {
  if (a > T(0) && b > T(0) && c > T(0) && d > T(0)) return fmin(fmin(a, b), fmin(c, d));
  if (a < T(0) && b < T(0) && c < T(0) && d < T(0)) return fmax(fmax(a, b), fmax(c, d));
  return T(0);
}

// xsPPM7 face value between q0 and p1 (cells ordered along the flow): the
// seventh-order upwind-biased interpolant, accepted when it lies between q0
// and the monotonicity-preserving value, otherwise moved into the
// curvature-widened bounds of Suresh and Huynh (alpha = 4)
template <typename T>
__device__ __forceinline__ T xsppm7_face(T m3, T m2, T m1, T q0, T p1, T p2, T p3) {
  const T u7 = (T(-3) * m3 + T(25) * m2 - T(101) * m1 + T(319) * q0 + T(214) * p1 - T(38) * p2 + T(4) * p3) *
               T(1.0 / 420.0);
  const T alpha = T(4);
  const T ump = q0 + mm2<T>(p1 - q0, alpha * (q0 - m1));
  if ((u7 - q0) * (u7 - ump) <= T(0)) return u7;
  const T dm1 = m2 - T(2) * m1 + q0, d0 = m1 - T(2) * q0 + p1, dp1 = q0 - T(2) * p1 + p2;
  const T dp = mm4<T>(T(4) * d0 - dp1, T(4) * dp1 - d0, d0, dp1);
  const T dm = mm4<T>(T(4) * dm1 - d0, T(4) * d0 - dm1, dm1, d0);
  const T uul = q0 + alpha * (q0 - m1);
  const T umd = T(0.5) * (q0 + p1) - T(0.5) * dp;
  const T ulc = q0 + T(0.5) * (q0 - m1) + T(4.0 / 3.0) * dm;
  const T umin = fmax(fmin(fmin(q0, p1), umd), fmin(fmin(q0, uul), ulc));
  const T umax = fmin(fmax(fmax(q0, p1), umd), fmax(fmax(q0, uul), ulc));
  return u7 + mm2<T>(umin - u7, umax - u7);
}

// upwind face value from the 2H cells around the face (c[H-1] | c[H])
template <typename T, int H>
struct LsLim;
template <typename T>
struct LsLim<T, 2> {
  static __device__ __forceinline__ T face(const T* c, T adv) { return lim4<T>(c[0], c[1], c[2], c[3], adv); }
};
template <typename T>
struct LsLim<T, 4> {
  static __device__ __forceinline__ T face(const T* c, T adv) {
    return adv > T(0) ? xsppm7_face<T>(c[0], c[1], c[2], c[3], c[4], c[5], c[6])
                      : xsppm7_face<T>(c[7], c[6], c[5], c[4], c[3], c[2], c[1]);
  }
};

template <typename T, int H>
__global__ void __launch_bounds__(BX* BY) k_ls_advect(GridDev g, CVel<T> vel,
                                                      const double* __restrict__ phi_n, const T* __restrict__ phi_h,
                                                      double dt, double* out, int zchunk) {
  constexpr int HX = BX + 2 * H, HY = BY + 2 * H, NS = (HX * HY + BX * BY - 1) / (BX * BY);
  __shared__ T sP[HY][HX];
  __shared__ T sFx[BY][BX + 1];
  __shared__ T sFy[BY + 1][BX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int i = x0 + tx, j = y0 + ty;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const bool inside = i < n0 && j < n1;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(k0 + zchunk, n2);
  const size_t plane = (size_t)n0 * n1;
  int soff[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    const int t = tid + r * BX * BY;
    soff[r] = -1;
    if (t < HX * HY) {
      const int hy = t / HX, hx = t - hy * HX;
      soff[r] = ls_mirror<T>(y0 - H + hy, n1) * n0 + ls_mirror<T>(x0 - H + hx, n0);
    }
  }
  const size_t col = (size_t)min(j, n1 - 1) * n0 + min(i, n0 - 1);
  // z window: the 2H cells around the current bottom face (k - H .. k + H - 1)
  T zp[2 * H];
#pragma unroll
  for (int q = 0; q < 2 * H; ++q) zp[q] = phi_h[(size_t)ls_mirror<T>(k0 - H + q, n2) * plane + col];
  T Fz_lo = T(0);
  for (int k = k0; k < k1; ++k) {
    T ux = T(0), uxl = T(0), vy = T(0), vyl = T(0), wz = T(0), wzl = T(0);
    if (inside) {
      ux = vel.q[0][fidx(g, 0, i + 1, j, k)];
      if (tx == 0) uxl = vel.q[0][fidx(g, 0, i, j, k)];
      vy = vel.q[1][fidx(g, 1, i, j + 1, k)];
      if (ty == 0) vyl = vel.q[1][fidx(g, 1, i, j, k)];
      wz = vel.q[2][fidx(g, 2, i, j, k + 1)];
      if (k == k0) wzl = vel.q[2][fidx(g, 2, i, j, k)];
    }
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      const int t = tid + r * BX * BY;
      if (soff[r] >= 0) {
        const int hy = t / HX, hx = t - hy * HX;
        sP[hy][hx] = phi_h[(size_t)k * plane + soff[r]];
      }
    }
    __syncthreads();
    if (inside) {
      const int hy = ty + H, hx = tx + H;
      T c[2 * H];
      // right x-face of cell i: cells i + 1 - H .. i + H
#pragma unroll
      for (int q = 0; q < 2 * H; ++q) c[q] = sP[hy][tx + 1 + q];
      sFx[ty][tx + 1] = ux * LsLim<T, H>::face(c, ux);
      if (tx == 0) {
#pragma unroll
        for (int q = 0; q < 2 * H; ++q) c[q] = sP[hy][tx + q];
        sFx[ty][0] = uxl * LsLim<T, H>::face(c, uxl);
      }
#pragma unroll
      for (int q = 0; q < 2 * H; ++q) c[q] = sP[ty + 1 + q][hx];
      sFy[ty + 1][tx] = vy * LsLim<T, H>::face(c, vy);
      if (ty == 0) {
#pragma unroll
        for (int q = 0; q < 2 * H; ++q) c[q] = sP[ty + q][hx];
        sFy[0][tx] = vyl * LsLim<T, H>::face(c, vyl);
      }
    }
    __syncthreads();
    if (k == k0) Fz_lo = wzl * LsLim<T, H>::face(zp, wzl);
#pragma unroll
    for (int q = 0; q < 2 * H - 1; ++q) zp[q] = zp[q + 1];
    zp[2 * H - 1] = phi_h[(size_t)ls_mirror<T>(k + H, n2) * plane + col];
    if (inside) {
      const T Fz_hi = wz * LsLim<T, H>::face(zp, wz);
      const T Q = (sFx[ty][tx + 1] - sFx[ty][tx]) * ginv<T>(g, 0) + (sFy[ty + 1][tx] - sFy[ty][tx]) * ginv<T>(g, 1) +
                  (Fz_hi - Fz_lo) * ginv<T>(g, 2);
      const size_t id = (size_t)k * plane + (size_t)j * n0 + i;
      out[id] = phi_n[id] - dt * cvt<double, T>(Q);
      Fz_lo = Fz_hi;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_levelset_advect(const GridDev& g, const T* const vel[3], const double* phi_n, const T* phi_half, double dt,
                            double* out, cudaStream_t st, int limiter) {
  CVel<T> v{{vel[0], vel[1], vel[2]}};
  const int zc = transport_chunk(g.n[0], g.n[1], g.n[2]);
  dim3 grid(cdiv(g.n[0], BX), cdiv(g.n[1], BY), cdiv(g.n[2], zc));
  if (limiter == WSI_LIMIT_XSPPM7) {
    k_ls_advect<T, 4><<<grid, dim3(BX, BY), 0, st>>>(g, v, phi_n, phi_half, dt, out, zc);
  } else {
    k_ls_advect<T, 2><<<grid, dim3(BX, BY), 0, st>>>(g, v, phi_n, phi_half, dt, out, zc);
  }
  WSI_COUNT();
}
template void launch_levelset_advect<double>(const GridDev&, const double* const[3], const double*, const double*,
                                             double, double*, cudaStream_t, int);
template void launch_levelset_advect<float>(const GridDev&, const float* const[3], const double*, const float*,
                                            double, double*, cudaStream_t, int);

__global__ void k_box_sdf(GridDev g, const double* __restrict__ xc, double hx_, double hy_, double hz_, double* psi) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  double x = (i + 0.5) * g.h[0], y = (j + 0.5) * g.h[1], z = (k + 0.5) * g.h[2];
  double qx = fabs(x - xc[0]) - hx_, qy = fabs(y - xc[1]) - hy_, qz = fabs(z - xc[2]) - hz_;
  double ox = fmax(qx, 0.0), oy = fmax(qy, 0.0), oz = fmax(qz, 0.0);
  double outside = sqrt(ox * ox + oy * oy + oz * oz);
  double inside = fmin(fmax(fmax(qx, qy), qz), 0.0);
  psi[fidx(g, 3, i, j, k)] = outside + inside;
}

// capped cylinder with its axis along y (radius r, half length hl) about xc
__global__ void k_cyl_sdf(GridDev g, const double* __restrict__ xc, double r, double hl, double* psi) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  double x = (i + 0.5) * g.h[0], y = (j + 0.5) * g.h[1], z = (k + 0.5) * g.h[2];
  double dx = x - xc[0], dz = z - xc[2];
  double qr = sqrt(dx * dx + dz * dz) - r, qy = fabs(y - xc[1]) - hl;
  double or_ = fmax(qr, 0.0), oy = fmax(qy, 0.0);
  psi[fidx(g, 3, i, j, k)] = sqrt(or_ * or_ + oy * oy) + fmin(fmax(qr, qy), 0.0);
}

void launch_cyl_sdf(const GridDev& g, const double* xcom_dev, double radius, double half_length, double* psi,
                    cudaStream_t st) {
  { k_cyl_sdf<<<dim3(cdiv(g.n[0], BX), cdiv(g.n[1], BY), g.n[2]), dim3(BX, BY), 0, st>>>(g, xcom_dev, radius,
                                                                                          half_length, psi); WSI_COUNT(); }
}

void launch_box_sdf(const GridDev& g, const double* xcom_dev, const double half[3], double* psi, cudaStream_t st) {
  { k_box_sdf<<<dim3(cdiv(g.n[0], BX), cdiv(g.n[1], BY), g.n[2]), dim3(BX, BY), 0, st>>>(g, xcom_dev, half[0], half[1],
                                                                                         half[2], psi); WSI_COUNT(); }
}

}  // namespace wsi
