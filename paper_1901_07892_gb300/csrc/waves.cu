// Numerical wave tank (Sec. 7.1): second-order Stokes wave and the
// relaxation zones applied at the end of each time step,
//   q <- alpha q + (1 - alpha) q_target,  alpha = 1 - (exp(xb^3.5) - 1)/(e - 1),
// with a generation zone [0, x_gen] relaxing towards the Stokes wave
// (level set y - eta, liquid-only velocity (1 - H~) (u_w, v_w)) and a damping
// zone [x_damp, lx] relaxing towards still water (phi = y, u = 0).  y is the
// height above the still-water level along the vertical axis.  Cells and
// faces outside both zones are untouched.
#include <math.h>

#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;

__device__ __forceinline__ double wv_eta(const WaveDev& w, double x, double t) {
  double th = w.k * x - w.omega * t;
  return 0.5 * w.H * cos(th) + w.c2 * cos(2.0 * th);
}

__device__ __forceinline__ void wv_vel(const WaveDev& w, double x, double y, double t, double& u, double& v) {
  double th = w.k * x - w.omega * t;
  double s1 = w.k * (w.d + y), s2 = 2.0 * s1;
  u = w.a1 * cosh(s1) * cos(th) + w.a2 * cosh(s2) * cos(2.0 * th);
  v = w.a1 * sinh(s1) * sin(th) + w.a2 * sinh(s2) * sin(2.0 * th);
}

__device__ __forceinline__ double wv_alpha(double xb) {
  xb = fmin(fmax(xb, 0.0), 1.0);
  return 1.0 - (exp(pow(xb, 3.5)) - 1.0) / (M_E - 1.0);
}

__device__ __forceinline__ double wv_heaviside(double phi, double eps) {
  if (phi < -eps) return 0.0;
  if (phi > eps) return 1.0;
  return 0.5 * (1.0 + phi / eps + sin(M_PI * phi / eps) / M_PI);
}

// zone weight at x; returns false outside both zones (x_gen = 0: no
// generation zone, as with a Dirichlet inlet)
__device__ __forceinline__ bool wv_zone(const WaveDev& w, double x, double& a, bool& gen) {
  gen = x < w.x_gen;
  bool dmp = x > w.x_damp;
  if (!gen && !dmp) return false;
  a = gen ? wv_alpha((w.x_gen - x) / w.x_gen) : wv_alpha((x - w.x_damp) / (w.lx - w.x_damp));
  return true;
}

template <int C>
__global__ void k_relax_faces(GridDev g, WaveDev w, double t, double* q) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(g, C, 0) || j >= ext(g, C, 1)) return;
  int id3[3] = {i, j, k};
  if (!face_row(g, C, id3[C])) return;  // faces on walls and the inlet keep their values
  double pos[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] = (a == C ? (double)id3[a] : id3[a] + 0.5) * g.h[a];
  double a, tgt = 0.0;
  bool gen;
  if (!wv_zone(w, pos[0], a, gen)) return;
  if (gen && (C == 0 || C == w.vert)) {
    double y = pos[w.vert] - w.d;
    double phit = y - wv_eta(w, pos[0], t);
    double uw, vw;
    wv_vel(w, pos[0], y, t, uw, vw);
    tgt = (1.0 - wv_heaviside(phit, w.eps)) * (C == 0 ? uw : vw);
  }
  size_t id = fidx(g, C, i, j, k);
  q[id] = a * q[id] + (1.0 - a) * tgt;
}

__global__ void k_relax_cells(GridDev g, WaveDev w, double t, double* phi) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  int id3[3] = {i, j, k};
  double x = (i + 0.5) * g.h[0];
  double a;
  bool gen;
  if (!wv_zone(w, x, a, gen)) return;
  double y = (id3[w.vert] + 0.5) * g.h[w.vert] - w.d;
  double tgt = gen ? y - wv_eta(w, x, t) : y;
  size_t id = fidx(g, 3, i, j, k);
  phi[id] = a * phi[id] + (1.0 - a) * tgt;
}

void launch_wave_relax(const GridDev& g, const WaveDev& w, double t, double* const vel[3], double* phi,
                       cudaStream_t st) {
  { k_relax_faces<0><<<dim3(cdiv(g.n[0] + 1, BX), cdiv(g.n[1], BY), g.n[2]), dim3(BX, BY), 0, st>>>(g, w, t, vel[0]); WSI_COUNT(); }
  { k_relax_faces<1><<<dim3(cdiv(g.n[0], BX), cdiv(g.n[1] + 1, BY), g.n[2]), dim3(BX, BY), 0, st>>>(g, w, t, vel[1]); WSI_COUNT(); }
  { k_relax_faces<2><<<dim3(cdiv(g.n[0], BX), cdiv(g.n[1], BY), g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, w, t, vel[2]); WSI_COUNT(); }
  if (phi) { k_relax_cells<<<dim3(cdiv(g.n[0], BX), cdiv(g.n[1], BY), g.n[2]), dim3(BX, BY), 0, st>>>(g, w, t, phi); WSI_COUNT(); }
}

// ---------------------------------------------------------- Dirichlet inlet
// Inlet data at time t (Sec. 7.1, the inlet's boundary-Heaviside equation),
// x- plane, vertical axis z: normal velocity of face (j, k),
//   gn[k ny + j] = (1 - H~(phi_b)) u_w(0, z_k - d, t),  z_k = (k + 1/2) hz,
// and tangential (vertical) velocity of the x- edge at height z_k = k hz,
//   gw[k ny + j] = (1 - H~(phi_b)) v_w(0, z_k - d, t),  k = 0 .. nz,
// with phi_b = z_k - d - eta(0, t).  Uniform along y.
__global__ void k_inlet_data(GridDev g, WaveDev w, double t, double* gn, double* gw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (j >= g.n[1]) return;
  const double eta = wv_eta(w, 0.0, t);
  double u, v;
  if (k < g.n[2]) {
    const double y = (k + 0.5) * g.h[2] - w.d;
    wv_vel(w, 0.0, y, t, u, v);
    gn[(size_t)k * g.n[1] + j] = (1.0 - wv_heaviside(y - eta, w.eps)) * u;
  }
  const double ye = k * g.h[2] - w.d;
  wv_vel(w, 0.0, ye, t, u, v);
  gw[(size_t)k * g.n[1] + j] = (1.0 - wv_heaviside(ye - eta, w.eps)) * v;
}

void launch_inlet_data(const GridDev& g, const WaveDev& w, double t, double* gn, double* gw, cudaStream_t st) {
  { k_inlet_data<<<dim3(cdiv(g.n[1], 64), g.n[2] + 1), 64, 0, st>>>(g, w, t, gn, gw); WSI_COUNT(); }
}

// The inlet's data lifted to the right-hand side of the implicit solve: the
// rows the data reach, through the operator of Sec. 4.2.2 with the inlet's
// affine ghosts (normal velocity gn on the x- faces, tangential velocity gw
// on the x- edges: ghost 2 gw - w), get b -= K_in x_b:
//   continuity of cells i = 0:   b_p -= gn / hx
//   u at faces i = 1:             b_u += 2 theta mu_cc(0) gn / hx^2
//   v at faces (0, j), 0<j<ny:    b_v -= theta mu_xy (gn(j) - gn(j-1)) / (hy hx)
//   w at faces (0, k) (rows):     b_w -= theta mu_xz (-2 gw / hx + (gn(k) - gn(k-1)) / hz) / hx
// (at an open top's row gn(nz) is the tangential ghost -gn(nz-1)); and the
// explicit viscous term of u^n gets the part of its tangential data gw_n that
// the homogeneous ghost leaves out: b_w += (1 - theta) 2 mu_xz^n gw_n / hx^2.
// One thread per (j, k) of the x- plane, k = 0 .. nz.
__global__ void k_inlet_lift(GridDev g, const double* __restrict__ mu_cc, const double* __restrict__ mu_xy,
                             const double* __restrict__ mu_xz, const double* __restrict__ mu_xz_n,
                             const double* __restrict__ gn, const double* __restrict__ gw,
                             const double* __restrict__ gw_n, double theta, double* bu, double* bv, double* bw,
                             double* bp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  if (j >= ny) return;
  const double ihx = g.ih[0], ihy = g.ih[1], ihz = g.ih[2];
  auto gn_at = [&](int kk, int jj) { return gn[(size_t)kk * ny + jj]; };
  if (k < nz) {
    const double gnv = gn_at(k, j);
    bp[fidx(g, 3, 0, j, k)] -= gnv * ihx;
    if (nx >= 2) bu[fidx(g, 0, 1, j, k)] += 2.0 * theta * mu_cc[fidx(g, 3, 0, j, k)] * gnv * ihx * ihx;
    if (j > 0)
      bv[fidx(g, 1, 0, j, k)] -= theta * mu_xy[eidx(g, 0, 0, j, k)] * (gnv - gn_at(k, j - 1)) * ihy * ihx;
  }
  if (face_row(g, 2, k)) {
    const double gn_hi = k < nz ? gn_at(k, j) : g.bc[5] * gn_at(nz - 1, j);
    const double gwv = gw[(size_t)k * ny + j];
    const size_t e = eidx(g, 1, 0, j, k);
    bw[fidx(g, 2, 0, j, k)] -= theta * mu_xz[e] * (-2.0 * gwv * ihx + (gn_hi - gn_at(k - 1, j)) * ihz) * ihx;
    bw[fidx(g, 2, 0, j, k)] += (1.0 - theta) * 2.0 * mu_xz_n[e] * gw_n[(size_t)k * ny + j] * ihx * ihx;
  }
}

void launch_inlet_lift(const GridDev& g, const double* mu_cc, const double* mu_xy, const double* mu_xz,
                       const double* mu_xz_n, const double* gn, const double* gw, const double* gw_n, double theta,
                       double* b, cudaStream_t st) {
  Packing pk = packing(g);
  { k_inlet_lift<<<dim3(cdiv(g.n[1], 64), g.n[2] + 1), 64, 0, st>>>(g, mu_cc, mu_xy, mu_xz, mu_xz_n, gn, gw, gw_n,
                                                                    theta, b + pk.off[0], b + pk.off[1],
                                                                    b + pk.off[2], b + pk.off[3]); WSI_COUNT(); }
}

// u on the x- faces of a velocity vector <- gn
__global__ void k_inlet_set(GridDev g, const double* __restrict__ gn, double* u) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (j >= g.n[1]) return;
  u[fidx(g, 0, 0, j, k)] = gn[(size_t)k * g.n[1] + j];
}

void launch_inlet_set(const GridDev& g, const double* gn, double* u, cudaStream_t st) {
  { k_inlet_set<<<dim3(cdiv(g.n[1], 64), g.n[2]), 64, 0, st>>>(g, gn, u); WSI_COUNT(); }
}

// omega^2 = g k tanh(k d) by Newton's method from the deep-water guess
WaveDev wave_setup(double H, double T, double d, double x_gen, double x_damp, double lx, int vert, double eps,
                   double grav) {
  WaveDev w;
  w.H = H;
  w.d = d;
  w.omega = 2.0 * M_PI / T;
  double k = w.omega * w.omega / grav;
  for (int it = 0; it < 100; ++it) {
    double f = grav * k * tanh(k * d) - w.omega * w.omega;
    double df = grav * tanh(k * d) + grav * k * d / (cosh(k * d) * cosh(k * d));
    double dk = f / df;
    k -= dk;
    if (fabs(dk) < 1e-15 * k) break;
  }
  w.k = k;
  double lam = 2.0 * M_PI / k;
  w.a1 = H * grav * k / (2.0 * w.omega) / cosh(k * d);
  w.a2 = 3.0 * H * H * w.omega * k / 16.0 / pow(sinh(k * d), 4.0);
  w.c2 = M_PI * H * H / (8.0 * lam) * cosh(k * d) * (2.0 + cosh(2.0 * k * d)) / pow(sinh(k * d), 3.0);
  w.x_gen = x_gen;
  w.x_damp = x_damp;
  w.lx = lx;
  w.vert = vert;
  w.eps = eps;
  return w;
}

}  // namespace wsi
