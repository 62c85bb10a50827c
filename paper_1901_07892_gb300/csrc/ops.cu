// Field kernels of libwsi: material coefficients (Sec. 4.1) and the staggered
// operators of the implicit Stokes system (Sec. 3.1, 4.2.2); transport and
// level-set advection live in transport.cu.
//
// Every kernel walks its output array in x-fastest order with one thread per
// entry (blocks of 32 x 8 in x, y; one z-plane per grid row), so warps read
// and write contiguous rows of the unghosted MAC arrays.
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;

static inline dim3 grid3(int nx, int ny, int nz) { return dim3(cdiv(nx, BX), cdiv(ny, BY), nz); }

// =========================================================== materials
// Smoothed Heaviside of Sec. 2 with t = phi / eps: 0 for t <= -1, 1 for
// t >= 1, the sine ramp between.  The band test runs on a float32 copy of t
// made by integer operations (float64 comparisons issue on GB300's narrow
// float64 pipe); where that copy is ambiguous, |t| within 2^-24 of 1, the
// ramp differs from its limit by ~(1 - |t|)^3, far below float64 resolution.
// code: 0 or 1 away from the band (value exactly 0 or 1), 2 inside.
// Float32 pre-test: tf, a float32 estimate of t = phi/eps whose error is at
// most `bound` (a few units in the last float32 place of the magnitudes that
// formed it), decides the code without any float64 operation when it lies
// beyond the band edges by more than that bound; otherwise 2 (undecided:
// the float64 path runs).
__device__ __forceinline__ int band_code_f(float tf, float bound) {
  if (tf < -1.0f - bound) return 0;
  if (tf > 1.0f + bound) return 1;
  return 2;
}

__device__ __forceinline__ double heav(double phi, double inv_eps, int& code) {
  const double t = phi * inv_eps;
  const float tf = d2f_fast(t);
  if (tf <= -1.0f) {
    code = 0;
    return 0.0;
  }
  if (tf >= 1.0f) {
    code = 1;
    return 1.0;
  }
  code = 2;
  return 0.5 * (1.0 + t + sin(M_PI * t) / M_PI);
}

// two-stage blend (Sec. 2): fluid value from phi, then solid from psi; away
// from both bands the value comes from the table (same expression, host)
__device__ __forceinline__ double two_stage(double h1, int c1, double h2, int c2, double zl, double zg, double zs,
                                            const double* tab) {
  if (c1 < 2 && c2 < 2) return tab[c1 + 2 * c2];
  const double zf = zl + (zg - zl) * h1;
  return zs + (zf - zs) * h2;
}

__device__ __forceinline__ double cell_at(const GridDev& g, const double* a, int i, int j, int k) {
  i = clampi(i, 0, g.n[0] - 1);
  j = clampi(j, 0, g.n[1] - 1);
  k = clampi(k, 0, g.n[2] - 1);
  return a[fidx(g, 3, i, j, k)];
}

__global__ void k_mat_cells(GridDev g, PhaseConst pc, const double* __restrict__ phi, const double* __restrict__ psi,
                            double* rho_cc, double* mu_cc) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  size_t id = fidx(g, 3, i, j, k);
  const double a = phi[id], b = psi[id];
  const float ie = pc.inv_eps_f;
  const float af = d2f_fast(a), bf = d2f_fast(b);
  // bound: 2^-20 |t|, far above the float32 rounding of phi and of phi/eps
  int c1 = band_code_f(af * ie, 9.5367431640625e-07f * fabsf(af * ie)),
      c2 = band_code_f(bf * ie, 9.5367431640625e-07f * fabsf(bf * ie));
  if (c1 < 2 && c2 < 2) {
    if (rho_cc) rho_cc[id] = pc.rho_tab[c1 + 2 * c2];
    mu_cc[id] = pc.mu_tab[c1 + 2 * c2];
    if (pc.inv_mu) pc.inv_mu[id] = pc.imu_tab[c1 + 2 * c2];
    return;
  }
  const double h1 = heav(a, pc.inv_eps, c1), h2 = heav(b, pc.inv_eps, c2);
  if (rho_cc) rho_cc[id] = two_stage(h1, c1, h2, c2, pc.rho_l, pc.rho_g, pc.rho_s, pc.rho_tab);
  const double mu = two_stage(h1, c1, h2, c2, pc.mu_l, pc.mu_g, pc.mu_s, pc.mu_tab);
  mu_cc[id] = mu;
  if (pc.inv_mu) pc.inv_mu[id] = (c1 < 2 && c2 < 2) ? pc.imu_tab[c1 + 2 * c2] : 1.0 / mu;
}

// face density from face-averaged level sets (wall faces: the interior cell)
template <int C>
__global__ void k_mat_faces(GridDev g, PhaseConst pc, const double* __restrict__ phi, const double* __restrict__ psi,
                            double* rho_face, double* beta, double* rho_flow) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(g, C, 0) || j >= ext(g, C, 1)) return;
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  lo[C] -= 1;
  const double pl = cell_at(g, phi, lo[0], lo[1], lo[2]), ph = cell_at(g, phi, hi[0], hi[1], hi[2]);
  size_t id = fidx(g, C, i, j, k);
  const float ie = pc.inv_eps_f;
  // bound: 2^-20 (|phi_lo| + |phi_hi|)/eps, far above the float32 rounding of
  // the two values, their mean and the scaling
  const float plf = d2f_fast(pl), phf = d2f_fast(ph);
  int c1 = band_code_f(0.5f * (plf + phf) * ie, 9.5367431640625e-07f * (fabsf(plf) + fabsf(phf)) * ie);
  double sl = 0.0, sh = 0.0;
  int c2 = 0;
  if (rho_face) {
    sl = cell_at(g, psi, lo[0], lo[1], lo[2]);
    sh = cell_at(g, psi, hi[0], hi[1], hi[2]);
    const float slf = d2f_fast(sl), shf = d2f_fast(sh);
    c2 = band_code_f(0.5f * (slf + shf) * ie, 9.5367431640625e-07f * (fabsf(slf) + fabsf(shf)) * ie);
  }
  if (c1 < 2 && c2 < 2) {  // away from both bands: table values only
    if (rho_face) {
      rho_face[id] = pc.rho_tab[c1 + 2 * c2];
      if (beta) beta[id] = pc.beta_tab[c1 + 2 * c2];
    }
    if (rho_flow) rho_flow[id] = pc.flow_tab[c1];
    return;
  }
  const double pa = 0.5 * (pl + ph);
  const double h1 = heav(pa, pc.inv_eps, c1);
  if (rho_face) {
    const double sa = 0.5 * (sl + sh);
    const double h2 = heav(sa, pc.inv_eps, c2);
    const double r = two_stage(h1, c1, h2, c2, pc.rho_l, pc.rho_g, pc.rho_s, pc.rho_tab);
    rho_face[id] = r;
    if (beta) beta[id] = (c1 < 2 && c2 < 2) ? pc.beta_tab[c1 + 2 * c2] : 1.0 / r;
  }
  if (rho_flow) rho_flow[id] = c1 < 2 ? pc.flow_tab[c1] : pc.rho_l + (pc.rho_g - pc.rho_l) * h1;
}

// Harmonic mean 4 / sum(1/mu) of the 4 cells around an edge (mirror ghosts
// at walls).  The reciprocals come precomputed once per cell when inv_mu is
// given: a float64 division costs tens of instructions at GB300's float64
// rate, and each cell feeds twelve edges.  Where the four reciprocals are
// bit-identical table values the mean comes from the table as well.
template <int E>
__global__ void k_mat_edges(GridDev g, PhaseConst pc, const double* __restrict__ mu_cc,
                            const double* __restrict__ inv_mu, double* mu_e) {
  // E = 0: xy edges, 1: xz, 2: yz
  constexpr int A1 = (E == 2) ? 1 : 0;
  constexpr int A2 = (E == 0) ? 1 : 2;
  int ex = g.n[0] + (A1 == 0 || A2 == 0), ey = g.n[1] + (A1 == 1 || A2 == 1);
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ex || j >= ey) return;
  double v[4];
#pragma unroll
  for (int o1 = 0; o1 < 2; ++o1)
#pragma unroll
    for (int o2 = 0; o2 < 2; ++o2) {
      int c[3] = {i, j, k};
      c[A1] -= o1;
      c[A2] -= o2;
      v[2 * o1 + o2] = inv_mu ? cell_at(g, inv_mu, c[0], c[1], c[2]) : 1.0 / cell_at(g, mu_cc, c[0], c[1], c[2]);
    }
  const long long b0 = __double_as_longlong(v[0]);
  if (b0 == __double_as_longlong(v[1]) && b0 == __double_as_longlong(v[2]) && b0 == __double_as_longlong(v[3])) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (b0 == __double_as_longlong(pc.imu_tab[t])) {
        mu_e[eidx(g, E, i, j, k)] = pc.mue_tab[t];
        return;
      }
  }
  mu_e[eidx(g, E, i, j, k)] = 4.0 / (((v[0] + v[1]) + v[2]) + v[3]);
}

void phase_tables(PhaseConst& pc) {
  pc.inv_eps = 1.0 / pc.eps;
  pc.inv_eps_f = (float)pc.inv_eps;
  for (int h2 = 0; h2 < 2; ++h2)
    for (int h1 = 0; h1 < 2; ++h1) {
      const int t = h1 + 2 * h2;
      const double rf = pc.rho_l + (pc.rho_g - pc.rho_l) * (double)h1;
      pc.rho_tab[t] = pc.rho_s + (rf - pc.rho_s) * (double)h2;
      pc.beta_tab[t] = 1.0 / pc.rho_tab[t];
      const double mf = pc.mu_l + (pc.mu_g - pc.mu_l) * (double)h1;
      pc.mu_tab[t] = pc.mu_s + (mf - pc.mu_s) * (double)h2;
      pc.imu_tab[t] = 1.0 / pc.mu_tab[t];
      const double x = pc.imu_tab[t];
      pc.mue_tab[t] = 4.0 / (((x + x) + x) + x);
    }
  for (int h1 = 0; h1 < 2; ++h1) pc.flow_tab[h1] = pc.rho_l + (pc.rho_g - pc.rho_l) * (double)h1;
}

void launch_materials(const GridDev& g, const PhaseConst& pc, const double* phi, const double* psi, double* rho_cc,
                      double* mu_cc, double* const rho_face[3], double* const beta[3], double* const rho_flow[3],
                      double* const mu_e[3], cudaStream_t st) {
  { k_mat_cells<<<grid3(g.n[0], g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_cc, mu_cc); WSI_COUNT(); }
  { k_mat_faces<0><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_face[0], beta[0],
                                                                             rho_flow[0]); WSI_COUNT(); }
  { k_mat_faces<1><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_face[1], beta[1],
                                                                             rho_flow[1]); WSI_COUNT(); }
  { k_mat_faces<2><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_face[2], beta[2],
                                                                             rho_flow[2]); WSI_COUNT(); }
  { k_mat_edges<0><<<grid3(g.n[0] + 1, g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, pc, mu_cc, pc.inv_mu, mu_e[0]); WSI_COUNT(); }
  { k_mat_edges<1><<<grid3(g.n[0] + 1, g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, pc, mu_cc, pc.inv_mu, mu_e[1]); WSI_COUNT(); }
  { k_mat_edges<2><<<grid3(g.n[0], g.n[1] + 1, g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, pc, mu_cc, pc.inv_mu, mu_e[2]); WSI_COUNT(); }
}

void launch_face_density(const GridDev& g, const PhaseConst& pc, const double* phi, const double* psi,
                         double* const rho_face[3], cudaStream_t st) {
  { k_mat_faces<0><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_face[0], nullptr,
                                                                             nullptr); WSI_COUNT(); }
  { k_mat_faces<1><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_face[1], nullptr,
                                                                             nullptr); WSI_COUNT(); }
  { k_mat_faces<2><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, pc, phi, psi, rho_face[2], nullptr,
                                                                             nullptr); WSI_COUNT(); }
}

// =========================================================== strain-rate operator
// (L_mu q)_C at the interior C-face (i,j,k):
//   d/dx_C (2 mu dq_C/dx_C) + sum_{D != C} d/dx_D [ mu_e (dq_C/dx_D + dq_D/dx_C) ]
// diag (optional): coefficient of q_C(i,j,k) itself in L_mu q.
template <int C, typename T>
__device__ __forceinline__ T strain_at(const GridDev& g, const Coef<T>& cf, const T* const* q, int i, int j, int k,
                                       T* diag) {
  const T* qc = q[C];
  const T ihC = ginv<T>(g, C);
  int id3[3] = {i, j, k};
  T q0 = qc[fidx(g, C, i, j, k)];
  // the top row of an open top: the cell above is a ghost whose normal stress
  // is minus the one below (w mirrors evenly) and whose tangential
  // velocities are -1 times those below
  const bool top = C == 2 && k == g.n[2];
  // normal stress: cells hi = face index along C, lo = index - 1
  int lo3[3] = {i, j, k};
  lo3[C] -= 1;
  int hi3[3] = {i, j, k};
  hi3[C] += 1;
  T mu_lo = cf.mu_cc[fidx(g, 3, lo3[0], lo3[1], lo3[2])];
  T qm = qc[fidx(g, C, lo3[0], lo3[1], lo3[2])];
  T mu_hi = top ? mu_lo : cf.mu_cc[fidx(g, 3, i, j, k)];
  T qp = top ? qm : qc[fidx(g, C, hi3[0], hi3[1], hi3[2])];
  T L = T(2) * ihC * ihC * (mu_hi * (qp - q0) - mu_lo * (q0 - qm));
  T dg = -T(2) * ihC * ihC * (mu_hi + mu_lo);
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    if (D == C) continue;
    const int E = edge_id(C, D);
    const T ihD = ginv<T>(g, D);
    const T* qd = q[D];
    // neighbours along D (ghosts beyond walls mirror with the wall sign)
    int a3[3] = {id3[0], id3[1], id3[2]};
    int b3[3] = {id3[0], id3[1], id3[2]};
    a3[D] += 1;
    b3[D] -= 1;
    T q_hi, q_lo, s_hi = T(0), s_lo = T(0);
    if (a3[D] >= g.n[D]) {
      s_hi = gbc<T>(g, 2 * D + 1);
      q_hi = s_hi * q0;
    } else {
      q_hi = qc[fidx(g, C, a3[0], a3[1], a3[2])];
    }
    if (b3[D] < 0) {
      s_lo = gbc<T>(g, 2 * D);
      q_lo = s_lo * q0;
    } else {
      q_lo = qc[fidx(g, C, b3[0], b3[1], b3[2])];
    }
    // edges: along C at the face index, along D at j_D (lo) and j_D + 1 (hi)
    int eh[3] = {id3[0], id3[1], id3[2]};
    eh[D] += 1;
    T mue_hi = cf.mu_e[E][eidx(g, E, eh[0], eh[1], eh[2])];
    T mue_lo = cf.mu_e[E][eidx(g, E, id3[0], id3[1], id3[2])];
    // q_D on D-faces adjacent along C: cells (index along C) id-1 and id
    int d1[3] = {id3[0], id3[1], id3[2]};  // hi edge, cell id
    d1[D] += 1;
    int d0[3] = {d1[0], d1[1], d1[2]};
    d0[C] -= 1;
    const T qd_d0 = qd[fidx(g, D, d0[0], d0[1], d0[2])];
    const T qd_d1 = top ? gbc<T>(g, 5) * qd_d0 : qd[fidx(g, D, d1[0], d1[1], d1[2])];
    T dqd_hi = (qd_d1 - qd_d0) * ihC;
    int c1[3] = {id3[0], id3[1], id3[2]};  // lo edge
    int c0[3] = {id3[0], id3[1], id3[2]};
    c0[C] -= 1;
    const T qd_c0 = qd[fidx(g, D, c0[0], c0[1], c0[2])];
    const T qd_c1 = top ? gbc<T>(g, 5) * qd_c0 : qd[fidx(g, D, c1[0], c1[1], c1[2])];
    T dqd_lo = (qd_c1 - qd_c0) * ihC;
    T f_hi = mue_hi * ((q_hi - q0) * ihD + dqd_hi);
    T f_lo = mue_lo * ((q0 - q_lo) * ihD + dqd_lo);
    L += (f_hi - f_lo) * ihD;
    dg += (mue_hi * (s_hi - T(1)) - mue_lo * (T(1) - s_lo)) * ihD * ihD;
  }
  if (diag) *diag = dg;
  return L;
}

template <int C, typename T>
__global__ void k_viscous(GridDev g, Coef<T> cf, T inv_dt, T theta, CVel<T> q, T* out, const T* b, bool strain_only) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  int e0 = ext(g, C, 0), e1 = ext(g, C, 1);
  if (i >= e0 || j >= e1) return;
  int id3[3] = {i, j, k};
  size_t id = fidx(g, C, i, j, k);
  if (!face_row(g, C, id3[C])) {
    out[id] = T(0);
    return;
  }
  T L = strain_at<C, T>(g, cf, q.q, i, j, k, nullptr);
  T a;
  if (strain_only)
    a = L;
  else
    a = cf.rho_face[C][id] * inv_dt * q.q[C][id] - theta * L;
  out[id] = b ? b[id] - a : a;
}

template <typename T>
void launch_viscous(const GridDev& g, const Coef<T>& cf, T inv_dt, T theta, const T* const q[3], T* const out[3],
                    cudaStream_t st, bool strain_only) {
  CVel<T> cq{{q[0], q[1], q[2]}};
  { k_viscous<0, T><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, cq, out[0],
                                                                              nullptr, strain_only); WSI_COUNT(); }
  { k_viscous<1, T><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, cq, out[1],
                                                                              nullptr, strain_only); WSI_COUNT(); }
  { k_viscous<2, T><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, cq, out[2],
                                                                              nullptr, strain_only); WSI_COUNT(); }
}

template <typename T>
void launch_viscous_residual(const GridDev& g, const Coef<T>& cf, T inv_dt, T theta, const T* const q[3],
                             const T* const b[3], T* const r[3], cudaStream_t st) {
  CVel<T> cq{{q[0], q[1], q[2]}};
  { k_viscous<0, T><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, cq, r[0], b[0],
                                                                              false); WSI_COUNT(); }
  { k_viscous<1, T><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, cq, r[1], b[1],
                                                                              false); WSI_COUNT(); }
  { k_viscous<2, T><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, cq, r[2], b[2],
                                                                              false); WSI_COUNT(); }
}

// red-black Gauss-Seidel on component C of the viscous block: the other
// components and the other colour are read as they stand.
template <int C, typename T>
__global__ void k_viscous_rbgs(GridDev g, Coef<T> cf, T inv_dt, T theta, Vel<T> q, const T* __restrict__ b,
                               int color) {
  // thread t of a row owns the t-th face of the colour: i = 2t + ((j + k + color) & 1)
  const int j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k + color) & 1);
  int e0 = ext(g, C, 0), e1 = ext(g, C, 1);
  if (i >= e0 || j >= e1) return;
  int id3[3] = {i, j, k};
  if (!face_row(g, C, id3[C])) return;
  size_t id = fidx(g, C, i, j, k);
  T dg;
  const T* cq[3] = {q.q[0], q.q[1], q.q[2]};
  T L = strain_at<C, T>(g, cf, cq, i, j, k, &dg);
  T rf = cf.rho_face[C][id] * inv_dt;
  T a = rf * q.q[C][id] - theta * L;
  T d = rf - theta * dg;
  q.q[C][id] += (b[id] - a) / d;
}

template <typename T>
void launch_viscous_rbgs(const GridDev& g, const Coef<T>& cf, T inv_dt, T theta, T* const q[3], const T* const b[3],
                         int color, cudaStream_t st) {
  Vel<T> vq{{q[0], q[1], q[2]}};
  ktimer_begin(KC_RBGS_V, st);
  { k_viscous_rbgs<0, T><<<grid3((g.n[0] + 2) / 2, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, vq,
                                                                                         b[0], color); WSI_COUNT(); }
  { k_viscous_rbgs<1, T><<<grid3((g.n[0] + 1) / 2, g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta,
                                                                                           vq, b[1], color); WSI_COUNT(); }
  if (g.n[2] > 1)
    { k_viscous_rbgs<2, T><<<grid3((g.n[0] + 1) / 2, g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta,
                                                                                             vq, b[2], color); WSI_COUNT(); }
  ktimer_end(KC_RBGS_V, st);
}

// =========================================================== pressure, grad, div
template <typename T>
__global__ void k_pressure(GridDev g, const T* __restrict__ bx, const T* __restrict__ by, const T* __restrict__ bz,
                           const T* __restrict__ p, T* out) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  size_t id = fidx(g, 3, i, j, k);
  T pc = p[id];
  T s = T(0);
  T ihx2 = ginv2<T>(g, 0), ihy2 = ginv2<T>(g, 1), ihz2 = ginv2<T>(g, 2);
  if (i + 1 < g.n[0]) s += bx[fidx(g, 0, i + 1, j, k)] * (p[id + 1] - pc) * ihx2;
  if (i > 0) s -= bx[fidx(g, 0, i, j, k)] * (pc - p[id - 1]) * ihx2;
  if (j + 1 < g.n[1]) s += by[fidx(g, 1, i, j + 1, k)] * (p[id + g.n[0]] - pc) * ihy2;
  if (j > 0) s -= by[fidx(g, 1, i, j, k)] * (pc - p[id - g.n[0]]) * ihy2;
  size_t pl = (size_t)g.n[0] * g.n[1];
  if (k + 1 < g.n[2]) s += bz[fidx(g, 2, i, j, k + 1)] * (p[id + pl] - pc) * ihz2;
  else if (g.open_top) s -= T(2) * bz[fidx(g, 2, i, j, k + 1)] * pc * ihz2;  // ghost -p above the open top
  if (k > 0) s -= bz[fidx(g, 2, i, j, k)] * (pc - p[id - pl]) * ihz2;
  out[id] = s;
}

template <typename T>
void launch_pressure(const GridDev& g, const T* const beta[3], const T* p, T* out, cudaStream_t st) {
  { k_pressure<T><<<grid3(g.n[0], g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, beta[0], beta[1], beta[2], p, out); WSI_COUNT(); }
}

template <int C, typename T>
__global__ void k_grad(GridDev g, const T* __restrict__ p, T* out) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(g, C, 0) || j >= ext(g, C, 1)) return;
  int id3[3] = {i, j, k};
  size_t id = fidx(g, C, i, j, k);
  if (!face_row(g, C, id3[C])) {
    out[id] = T(0);
    return;
  }
  int lo3[3] = {i, j, k};
  lo3[C] -= 1;
  const T plo = p[fidx(g, 3, lo3[0], lo3[1], lo3[2])];
  const T phi = (C == 2 && k == g.n[2]) ? -plo : p[fidx(g, 3, i, j, k)];  // open top: ghost -p
  out[id] = (phi - plo) * ginv<T>(g, C);
}

template <typename T>
void launch_grad(const GridDev& g, const T* p, T* const out[3], cudaStream_t st) {
  { k_grad<0, T><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, p, out[0]); WSI_COUNT(); }
  { k_grad<1, T><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, p, out[1]); WSI_COUNT(); }
  { k_grad<2, T><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, p, out[2]); WSI_COUNT(); }
}

template <typename T>
__global__ void k_div(GridDev g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w, T* out,
                      T scale) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  T d = (u[fidx(g, 0, i + 1, j, k)] - u[fidx(g, 0, i, j, k)]) * ginv<T>(g, 0) +
        (v[fidx(g, 1, i, j + 1, k)] - v[fidx(g, 1, i, j, k)]) * ginv<T>(g, 1) +
        (w[fidx(g, 2, i, j, k + 1)] - w[fidx(g, 2, i, j, k)]) * ginv<T>(g, 2);
  out[fidx(g, 3, i, j, k)] = scale * d;
}

template <typename T>
void launch_div(const GridDev& g, const T* const q[3], T* out, T scale, cudaStream_t st) {
  { k_div<T><<<grid3(g.n[0], g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, q[0], q[1], q[2], out, scale); WSI_COUNT(); }
}

// packed Stokes matvec: momentum rows A u + G p (zero on wall faces)
template <int C>
__device__ __forceinline__ void stokes_row(const GridDev& g, const Coef<double>& cf, double inv_dt, double theta,
                                           const CVel<double>& q, const double* __restrict__ p, double* out, int i,
                                           int j, int k) {
  int id3[3] = {i, j, k};
  size_t id = fidx(g, C, i, j, k);
  if (!face_row(g, C, id3[C])) {
    out[id] = 0.0;
    return;
  }
  double L = strain_at<C, double>(g, cf, q.q, i, j, k, nullptr);
  int lo3[3] = {i, j, k};
  lo3[C] -= 1;
  const double plo = p[fidx(g, 3, lo3[0], lo3[1], lo3[2])];
  const double phi = (C == 2 && k == g.n[2]) ? -plo : p[fidx(g, 3, i, j, k)];  // open top: ghost -p
  double gp = (phi - plo) * g.ih[C];
  out[id] = cf.rho_face[C][id] * inv_dt * q.q[C][id] - theta * L + gp;
}

// One launch covers the whole packed vector: blockIdx.z walks the z-planes of
// the u, v and w momentum rows, then the continuity rows.
__global__ void k_stokes(GridDev g, Coef<double> cf, double inv_dt, double theta, CVel<double> q,
                         const double* __restrict__ p, double* yu, double* yv, double* yw, double* yp) {
  int z = blockIdx.z;
  int nz = g.n[2];
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (z < nz) {
    if (i < g.n[0] + 1 && j < g.n[1]) stokes_row<0>(g, cf, inv_dt, theta, q, p, yu, i, j, z);
  } else if (z < 2 * nz) {
    if (i < g.n[0] && j < g.n[1] + 1) stokes_row<1>(g, cf, inv_dt, theta, q, p, yv, i, j, z - nz);
  } else if (z < 3 * nz + 1) {
    if (i < g.n[0] && j < g.n[1]) stokes_row<2>(g, cf, inv_dt, theta, q, p, yw, i, j, z - 2 * nz);
  } else {
    int k = z - (3 * nz + 1);
    if (i < g.n[0] && j < g.n[1]) {
      double d = (q.q[0][fidx(g, 0, i + 1, j, k)] - q.q[0][fidx(g, 0, i, j, k)]) * g.ih[0] +
                 (q.q[1][fidx(g, 1, i, j + 1, k)] - q.q[1][fidx(g, 1, i, j, k)]) * g.ih[1] +
                 (q.q[2][fidx(g, 2, i, j, k + 1)] - q.q[2][fidx(g, 2, i, j, k)]) * g.ih[2];
      yp[fidx(g, 3, i, j, k)] = -d;
    }
  }
}

void launch_stokes(const GridDev& g, const Coef<double>& cf, double inv_dt, double theta, const double* x, double* y,
                   cudaStream_t st) {
  Packing pk = packing(g);
  CVel<double> q{{x + pk.off[0], x + pk.off[1], x + pk.off[2]}};
  const double* p = x + pk.off[3];
  dim3 grid(cdiv(g.n[0] + 1, BX), cdiv(g.n[1] + 1, BY), 4 * g.n[2] + 1);
  ktimer_begin(KC_STOKES, st);
  { k_stokes<<<grid, dim3(BX, BY), 0, st>>>(g, cf, inv_dt, theta, q, p, y + pk.off[0], y + pk.off[1],
                                            y + pk.off[2], y + pk.off[3]); WSI_COUNT(); }
  ktimer_end(KC_STOKES, st);
}

template <int C>
__global__ void k_zero_walls(GridDev g, double* q) {
  // walls normal to C: planes index 0 and n along C
  int a = blockIdx.x * BX + threadIdx.x, b = blockIdx.y * BY + threadIdx.y, side = blockIdx.z;
  constexpr int A = (C == 0) ? 1 : 0;
  constexpr int B = (C == 2) ? 1 : 2;
  if (a >= g.n[A] || b >= g.n[B]) return;
  if (C == 2 && side && g.open_top) return;  // the open top's faces are unknowns
  int c3[3];
  c3[C] = side ? g.n[C] : 0;
  c3[A] = a;
  c3[B] = b;
  q[fidx(g, C, c3[0], c3[1], c3[2])] = 0.0;
}

void launch_zero_walls(const GridDev& g, double* const q[3], cudaStream_t st) {
  { k_zero_walls<0><<<dim3(cdiv(g.n[1], BX), cdiv(g.n[2], BY), 2), dim3(BX, BY), 0, st>>>(g, q[0]); WSI_COUNT(); }
  { k_zero_walls<1><<<dim3(cdiv(g.n[0], BX), cdiv(g.n[2], BY), 2), dim3(BX, BY), 0, st>>>(g, q[1]); WSI_COUNT(); }
  { k_zero_walls<2><<<dim3(cdiv(g.n[0], BX), cdiv(g.n[1], BY), 2), dim3(BX, BY), 0, st>>>(g, q[2]); WSI_COUNT(); }
}

// =========================================================== momentum RHS
template <int C, typename T>
__global__ void k_rhs_base(GridDev g, Coef<T> cf_n, CVel<T> uT, const double* __restrict__ rho_n,
                           const double* __restrict__ un, double inv_dt, double theta, double* b0) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(g, C, 0) || j >= ext(g, C, 1)) return;
  int id3[3] = {i, j, k};
  size_t id = fidx(g, C, i, j, k);
  if (!face_row(g, C, id3[C])) {
    b0[id] = 0.0;
    return;
  }
  T L = strain_at<C, T>(g, cf_n, uT.q, i, j, k, nullptr);
  b0[id] = rho_n[id] * un[id] * inv_dt + (1.0 - theta) * (double)L;
}

template <typename T>
void launch_rhs_base(const GridDev& g, const Coef<T>& cf_n, const T* const uT[3], const double* const rho_n[3],
                     const double* const u_n[3], double inv_dt, double theta, double* const b0[3], cudaStream_t st) {
  CVel<T> u{{uT[0], uT[1], uT[2]}};
  { k_rhs_base<0, T><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, cf_n, u, rho_n[0], u_n[0], inv_dt,
                                                                               theta, b0[0]); WSI_COUNT(); }
  { k_rhs_base<1, T><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, cf_n, u, rho_n[1], u_n[1], inv_dt,
                                                                               theta, b0[1]); WSI_COUNT(); }
  { k_rhs_base<2, T><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, cf_n, u, rho_n[2], u_n[2], inv_dt,
                                                                               theta, b0[2]); WSI_COUNT(); }
}

// b = b0 - C + rho_g g over the packed velocity vector; wall faces are zero
// in b0, C and on output
template <typename TC>
__global__ void k_rhs_cycle(size_t n0, size_t n1, size_t n2, const double* __restrict__ b0, const TC* __restrict__ Cc,
                            const double* __restrict__ rg0, const double* __restrict__ rg1,
                            const double* __restrict__ rg2, double g0, double g1, double g2, double* b) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t n = n0 + n1 + n2;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    // components without gravity skip the density load and the product
    double grav = 0.0;
    if (t < n0) {
      if (g0 != 0.0) grav = rg0[t] * g0;
    } else if (t < n0 + n1) {
      if (g1 != 0.0) grav = rg1[t - n0] * g1;
    } else if (g2 != 0.0) {
      grav = rg2[t - n0 - n1] * g2;
    }
    b[t] = b0[t] - cvt<double, TC>(Cc[t]) + grav;
  }
}

template <typename TC>
void launch_rhs_cycle(const GridDev& g, const double* b0, const TC* C, const double* const rho_g[3],
                      const double grav[3], double* b, cudaStream_t st) {
  size_t n0 = fsize(g, 0), n1 = fsize(g, 1), n2 = fsize(g, 2);
  int blocks = (int)std::min<size_t>((n0 + n1 + n2 + 255) / 256, 152 * 16);
  { k_rhs_cycle<TC><<<blocks, 256, 0, st>>>(n0, n1, n2, b0, C, rho_g[0], rho_g[1], rho_g[2], grav[0], grav[1],
                                            grav[2], b); WSI_COUNT(); }
  double* q[3] = {b, b + n0, b + n0 + n1};
  launch_zero_walls(g, q, st);
}

// Non-conservative form (Sec. 4.2.3): b = b0 + rho (u^n/dt - N) + rho_g g with
// b0 = (1 - theta) L_mu^n u^n and rho = rho^{n+1,k+1} the face density of the
// level sets; wall faces are zero on output
template <typename TN>
__global__ void k_rhs_nc(size_t n0, size_t n1, size_t n2, const double* __restrict__ b0, const TN* __restrict__ N,
                         const double* __restrict__ r0, const double* __restrict__ r1, const double* __restrict__ r2,
                         const double* __restrict__ un, double inv_dt, const double* __restrict__ rg0,
                         const double* __restrict__ rg1, const double* __restrict__ rg2, double g0, double g1,
                         double g2, double* b) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t n = n0 + n1 + n2;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    double rho, grav = 0.0;
    if (t < n0) {
      rho = r0[t];
      if (g0 != 0.0) grav = rg0[t] * g0;
    } else if (t < n0 + n1) {
      rho = r1[t - n0];
      if (g1 != 0.0) grav = rg1[t - n0] * g1;
    } else {
      rho = r2[t - n0 - n1];
      if (g2 != 0.0) grav = rg2[t - n0 - n1] * g2;
    }
    b[t] = b0[t] + rho * (un[t] * inv_dt - cvt<double, TN>(N[t])) + grav;
  }
}

template <typename TN>
void launch_rhs_nc(const GridDev& g, const double* b0, const TN* N, const double* const rho[3], const double* u_n,
                   double inv_dt, const double* const rho_g[3], const double grav[3], double* b, cudaStream_t st) {
  size_t n0 = fsize(g, 0), n1 = fsize(g, 1), n2 = fsize(g, 2);
  int blocks = (int)std::min<size_t>((n0 + n1 + n2 + 255) / 256, 152 * 16);
  { k_rhs_nc<TN><<<blocks, 256, 0, st>>>(n0, n1, n2, b0, N, rho[0], rho[1], rho[2], u_n, inv_dt, rho_g[0], rho_g[1],
                                         rho_g[2], grav[0], grav[1], grav[2], b); WSI_COUNT(); }
  double* q[3] = {b, b + n0, b + n0 + n1};
  launch_zero_walls(g, q, st);
}
template void launch_rhs_nc<double>(const GridDev&, const double*, const double*, const double* const[3],
                                    const double*, double, const double* const[3], const double[3], double*,
                                    cudaStream_t);
template void launch_rhs_nc<float>(const GridDev&, const double*, const float*, const double* const[3],
                                   const double*, double, const double* const[3], const double[3], double*,
                                   cudaStream_t);

template void launch_rhs_base<double>(const GridDev&, const Coef<double>&, const double* const[3],
                                      const double* const[3], const double* const[3], double, double,
                                      double* const[3], cudaStream_t);
template void launch_rhs_base<float>(const GridDev&, const Coef<float>&, const float* const[3],
                                     const double* const[3], const double* const[3], double, double,
                                     double* const[3], cudaStream_t);
template void launch_rhs_cycle<double>(const GridDev&, const double*, const double*, const double* const[3],
                                       const double[3], double*, cudaStream_t);
template void launch_rhs_cycle<float>(const GridDev&, const double*, const float*, const double* const[3],
                                      const double[3], double*, cudaStream_t);

// explicit instantiations
template void launch_viscous<double>(const GridDev&, const Coef<double>&, double, double, const double* const[3],
                                     double* const[3], cudaStream_t, bool);
template void launch_viscous<float>(const GridDev&, const Coef<float>&, float, float, const float* const[3],
                                    float* const[3], cudaStream_t, bool);
template void launch_viscous_residual<double>(const GridDev&, const Coef<double>&, double, double,
                                              const double* const[3], const double* const[3], double* const[3],
                                              cudaStream_t);
template void launch_viscous_residual<float>(const GridDev&, const Coef<float>&, float, float, const float* const[3],
                                             const float* const[3], float* const[3], cudaStream_t);
template void launch_viscous_rbgs<double>(const GridDev&, const Coef<double>&, double, double, double* const[3],
                                          const double* const[3], int, cudaStream_t);
template void launch_viscous_rbgs<float>(const GridDev&, const Coef<float>&, float, float, float* const[3],
                                         const float* const[3], int, cudaStream_t);
template void launch_pressure<double>(const GridDev&, const double* const[3], const double*, double*, cudaStream_t);
template void launch_pressure<float>(const GridDev&, const float* const[3], const float*, float*, cudaStream_t);
template void launch_grad<double>(const GridDev&, const double*, double* const[3], cudaStream_t);
template void launch_grad<float>(const GridDev&, const float*, float* const[3], cudaStream_t);
template void launch_div<double>(const GridDev&, const double* const[3], double*, double, cudaStream_t);
template void launch_div<float>(const GridDev&, const float* const[3], float*, float, cudaStream_t);

}  // namespace wsi
