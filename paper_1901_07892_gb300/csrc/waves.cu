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

// zone weight at x; returns false outside both zones
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
  if (id3[C] == 0 || id3[C] == g.n[C]) return;  // wall faces keep their zero
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
