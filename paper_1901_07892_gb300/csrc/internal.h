// Host-side internals of libwsi shared by the translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/wsi.h"
#include "common.cuh"

namespace wsi {

// Coefficients of the Stokes operator on one grid (Sec. 4.1, 4.2.2).
template <typename T>
struct Coef {
  const T* rho_face[3];  // face density of the viscous block (rho breve)
  const T* beta[3];      // 1 / face density, pressure operator
  const T* mu_cc;        // cell viscosity (normal stresses)
  const T* mu_e[3];      // harmonic edge viscosity: xy, xz, yz
};

// ---------------------------------------------------------------- ops.cu
struct PhaseConst {
  double rho_l, rho_g, rho_s, mu_l, mu_g, mu_s, eps;
  double* inv_mu;  // scratch of one cell field for 1/mu (null: edges divide per access)
  // filled by phase_tables(): 1/eps, and the values a cell, face or edge
  // takes away from both smoothing bands, indexed h1 + 2 h2 with h1, h2 in
  // {0, 1} the two Heavisides, each computed by the same expression as inside
  // the bands so that both give identical results there
  double inv_eps;
  float inv_eps_f;
  double rho_tab[4], beta_tab[4], flow_tab[2], mu_tab[4], imu_tab[4], mue_tab[4];
};
// fill the derived fields of pc from its properties (host)
void phase_tables(PhaseConst& pc);
void launch_materials(const GridDev& g, const PhaseConst& pc, const double* phi, const double* psi,
                      double* rho_cc, double* mu_cc, double* const rho_face[3], double* const beta[3],
                      double* const rho_flow[3], double* const mu_e[3], cudaStream_t st);
// level-set face density only (Sec. 4.2.2: rho^n from phi^n, psi^n on faces)
void launch_face_density(const GridDev& g, const PhaseConst& pc, const double* phi, const double* psi,
                         double* const rho_face[3], cudaStream_t st);

// out = alpha * (rho/dt q - theta L_mu q) + beta_in * (G p)  (any of p, rho may be null)
template <typename T>
void launch_viscous(const GridDev& g, const Coef<T>& cf, T inv_dt, T theta, const T* const q[3], T* const out[3],
                    cudaStream_t st, bool strain_only = false);
// r = b - A q (viscous block)
template <typename T>
void launch_viscous_residual(const GridDev& g, const Coef<T>& cf, T inv_dt, T theta, const T* const q[3],
                             const T* const b[3], T* const r[3], cudaStream_t st);
template <typename T>
void launch_pressure(const GridDev& g, const T* const beta[3], const T* p, T* out, cudaStream_t st);
template <typename T>
void launch_grad(const GridDev& g, const T* p, T* const out[3], cudaStream_t st);
template <typename T>
void launch_div(const GridDev& g, const T* const q[3], T* out, T scale, cudaStream_t st);
// packed Stokes matvec in float64: y = K x
void launch_stokes(const GridDev& g, const Coef<double>& cf, double inv_dt, double theta, const double* x, double* y,
                   cudaStream_t st);
// Operands of the double-float Stokes matvec (dfstokes.cu): (hi, lo) float32
// pairs of the input vector and of the coefficients, each array with an even
// row pitch (rows start on 16-byte boundaries, as the tile copies need)
enum DfArray {
  DF_U = 0, DF_V, DF_W, DF_P,           // input vector
  DF_RHO_X, DF_RHO_Y, DF_RHO_Z,        // face density times 1/dt
  DF_MU_CC, DF_MU_XY, DF_MU_XZ, DF_MU_YZ,  // cell and edge viscosity
  DF_NARR
};
struct DfOperands {
  float2* a[DF_NARR] = {};
  int cols[DF_NARR], rows[DF_NARR], levels[DF_NARR], pitch[DF_NARR];
  void* maps = nullptr;  // host copy of the arrays' tile-copy descriptors
};
// extents and pitches of the arrays for grid g
void df_operands_shape(const GridDev& g, DfOperands& o);
// float2 elements array a takes (pitch x rows x levels)
size_t df_operand_elems(const DfOperands& o, int a);
// the tile-copy descriptors of the allocated arrays (WSI_OK or WSI_ERR_CUDA)
int df_operands_encode(DfOperands& o);
void df_operands_release(DfOperands& o);
// split the seven coefficient arrays, the face density times inv_dt
void df_split_coefs(const DfOperands& o, const double* const rho[3], const double* const mu_e[3], const double* mu_cc,
                    double inv_dt, cudaStream_t st);
// y = K x in double-float arithmetic: x split into the operands, then the
// matvec from the coefficients split by the last df_split_coefs; *err is set
// to 1 when a wait for a tile copy gave up
void launch_stokes_df(const GridDev& g, const DfOperands& o, double theta, const double* x, double* y, int* err,
                      cudaStream_t st);
// red-black Gauss-Seidel half sweep on the viscous block for component c
template <typename T>
void launch_viscous_rbgs(const GridDev& g, const Coef<T>& cf, T inv_dt, T theta, T* const q[3], const T* const b[3],
                         int color, cudaStream_t st);

// transport.cu (Sec. 4.2.2): R or C on all three face arrays, storage and
// arithmetic in T; inlet_w: the tangential data of vel's w on a Dirichlet
// inlet's x- plane ((nz+1) x ny, used for C), or null
template <typename T>
void launch_transport_flux(const GridDev& g, const T* const vel[3], const T* const rho[3], bool with_velocity,
                           T* const out[3], cudaStream_t st, const T* inlet_w = nullptr);
// out = a*x + b*y + c*z elementwise over n (any of y, z may be null)
void launch_lincomb(size_t n, double a, const double* x, double b, const double* y, double c, const double* z,
                    double* out, cudaStream_t st);
void launch_lincomb_to_f32(size_t n, double a, const double* x, double b, const double* y, double c,
                           const double* z, float* out, cudaStream_t st);
void launch_lincomb_f32(size_t n, float a, const float* x, float b, const float* y, float c, const float* z,
                        float* out, cudaStream_t st);
// float32 SSP-RK3 stage velocities (first cycle: uk null) and, with un32, the
// float32 copy of u^n, in one pass
void launch_rk_velocities_f32(size_t n, const double* un, const double* unm1, const double* uk, float* u1, float* u2,
                              float* un32, cudaStream_t st);
void launch_lincomb_mix(size_t n, double a, const double* x, double b, const float* y, double c, const float* z,
                        double* out, cudaStream_t st);
// z-chunk of the plane-marching stencil kernels for an ex x ey x ez box of
// points (32 x 8 tiles): long marches, yet about 8 blocks per SM
int transport_chunk(int ex, int ey, int ez);

// ---------------------------------------------------------------- reinit.cu
// iters pseudo-time steps of the level-set reinitialisation (Sec. 4.1) on
// the device level set phi (cells, in place), arithmetic in T; scratch holds
// 3 cells x ncell doubles
template <typename T>
void reinit_levelset(const GridDev& g, double* phi, int iters, double cfl, void* scratch, cudaStream_t st);

template <typename T>
void launch_levelset_advect(const GridDev& g, const T* const vel[3], const double* phi_n, const T* phi_half, double dt,
                            double* out, cudaStream_t st, int limiter);
void launch_box_sdf(const GridDev& g, const double* xcom_dev, const double half[3], double* psi, cudaStream_t st);
void launch_cyl_sdf(const GridDev& g, const double* xcom_dev, double radius, double half_length, double* psi,
                    cudaStream_t st);
// part of the momentum right-hand side fixed over the cycles of a step:
// b0 = rho_n u_n / dt + (1-theta) L_mu^n u_n, the strain term in T from
// T copies of u_n and mu^n (zero on wall faces)
template <typename T>
void launch_rhs_base(const GridDev& g, const Coef<T>& cf_n, const T* const uT[3], const double* const rho_n[3],
                     const double* const u_n[3], double inv_dt, double theta, double* const b0[3], cudaStream_t st);
// b = b0 - C + rho_g g on every face of the packed velocity vector (walls 0)
template <typename TC>
void launch_rhs_cycle(const GridDev& g, const double* b0, const TC* C, const double* const rho_g[3],
                      const double grav[3], double* b, cudaStream_t st);
void launch_zero_walls(const GridDev& g, double* const q[3], cudaStream_t st);
// non-conservative form: b = b0 + rho (u^n/dt - N) + rho_g g (walls 0)
template <typename TN>
void launch_rhs_nc(const GridDev& g, const double* b0, const TN* N, const double* const rho[3], const double* u_n,
                   double inv_dt, const double* const rho_g[3], const double grav[3], double* b, cudaStream_t st);

// ---------------------------------------------------------------- krylov.cu
// deterministic reductions: out[t] = <V_t, w> for t < m (V row-major m x n)
void launch_mdot(const double* V, size_t ldv, int m, const double* w, size_t n, double* out, double* scratch,
                 cudaStream_t st);
// w = (w - sign * sum_t h[t] V_t) * scale  (h and scale on device; scale
// null = 1)
void launch_maxpy(const double* V, size_t ldv, int m, const double* h, double* w, size_t n, double sign,
                  cudaStream_t st, const double* scale_dev = nullptr);
void launch_scale(double* x, size_t n, const double* s_dev, bool inverse, cudaStream_t st);
double host_norm2(const double* x, size_t n, double* scratch, cudaStream_t st);
// max |x_i| read back to the host (scratch: RB + 1 doubles)
double host_maxabs(const double* x, size_t n, double* scratch, cudaStream_t st);
template <typename T>
void launch_sum(const T* x, size_t n, double* out_dev, double* scratch, cudaStream_t st);
template <typename T>
void launch_add_scalar_from(T* x, size_t n, const double* s_dev, double factor, cudaStream_t st);

// ---------------------------------------------------------------- unet.cu
struct UNetImpl;
UNetImpl* unet_create(int Z, int Y, int X, int c0, int c1, int c2);
void unet_destroy(UNetImpl* u);
void unet_pack(UNetImpl* u, cudaStream_t st);  // float32 master weights -> bf16 kernel layouts
void unet_forward(UNetImpl* u, cudaStream_t st);
void unet_backward(UNetImpl* u, cudaStream_t st);
void unet_adam(UNetImpl* u, double lr, cudaStream_t st);
int unet_dim(const UNetImpl* u, int axis);  // 0: Z, 1: Y, 2: X
void unet_set_input3(UNetImpl* u, const float* x3, cudaStream_t st);  // device float [V][3]
size_t unet_nparam(const UNetImpl* u);
float* unet_params(UNetImpl* u);
float* unet_grads(UNetImpl* u);
__nv_bfloat16* unet_input(UNetImpl* u);  // [V][16]
float* unet_output(UNetImpl* u);         // [V]
float* unet_target(UNetImpl* u);         // [V]
double* unet_loss(UNetImpl* u);          // device scalar
float* unet_moment(UNetImpl* u, int which);  // Adam first (0) / second (1) moments
int* unet_step_count(UNetImpl* u);           // Adam steps taken
int unet_width(const UNetImpl* u, int level);  // c0, c1, c2
// reads and clears the flag a tensor-core convolution sets when one of its
// bounded waits ran out (the outputs of that launch are then not valid)
bool unet_take_error(UNetImpl* u);

// learned correction state inside the float32 multigrid (learned.cu)
struct LearnState {
  UNetImpl* net = nullptr;
  int level = 0;
  bool on = false;     // use the correction in V-cycles
  int mode = 1;        // WSI_LEARN_REPLACE or WSI_LEARN_AUGMENT
  bool ready = false;  // inputs restricted for the current coefficients
  std::vector<float*> lrho, phi;  // per level (index = level), restricted inputs
  float* diag = nullptr;
  float* e = nullptr;  // training field on the level
  float* t1 = nullptr;  // training scratch on the level: error, L error, L L error
  float* t2 = nullptr;
  float* t3 = nullptr;
  double* ss = nullptr;  // [0] sum of squares of the network input, [1] training loss
  // initial-guess network: the level-g solution from the restricted right-hand side
  UNetImpl* gnet = nullptr;
  int glevel = 0;
  float* gdiag = nullptr;
  double* gss = nullptr;  // [0] sum of squares of the guess network's input
};

// ---------------------------------------------------------------- mg.cu
template <typename T>
struct MGLevel {
  GridDev g;
  int r[3];         // coarsening ratio to the next level (1 or 2)
  T* beta[3];
  T* x;
  T* b;
  T* res;
  T* cd;            // Chebyshev smoother: direction, and the second buffer pair
  T* cx2;
  T* cd2;
};

// one level of the viscous multigrid (levels >= 1; level 0 uses the fine
// coefficients and the preconditioner's work arrays)
template <typename T>
struct VLevel {
  T* rho_face[3];
  T* mu_cc;
  T* mu_e[3];
  T* u[3];
  T* b[3];
  T* res[3];
};

template <typename T>
struct Precond {
  // pressure multigrid hierarchy
  std::vector<MGLevel<T>> lev;
  double* coarse_inv = nullptr;  // dense float64 inverse of the regularised coarsest operator
  int ncoarse = 0;
  // fine-level viscous coefficients in T
  T* rho_face[3] = {nullptr, nullptr, nullptr};
  T* mu_cc = nullptr;
  T* mu_e[3] = {nullptr, nullptr, nullptr};
  // work
  T* ru[3] = {nullptr, nullptr, nullptr};
  T* ut[3] = {nullptr, nullptr, nullptr};
  T* rp = nullptr;
  T* y = nullptr;
  T* gp[3] = {nullptr, nullptr, nullptr};
  double* dscratch = nullptr;  // reductions
  double* dsum = nullptr;
  bool built = false;
  std::vector<void*> allocs;
  LearnState learn;  // float32 hierarchy only
  std::vector<VLevel<T>> vlev;  // viscous multigrid, index = level (entry 0 unused)
  T* vres0[3] = {nullptr, nullptr, nullptr};  // fine-level viscous residual
};

struct Opts {
  int mg_pre = 2, mg_post = 2, mg_cycles = 1, visc_sweeps = 2;
  int mg_smoother = 0;  // WSI_SMOOTH_RBGS or WSI_SMOOTH_CHEBYSHEV (pressure multigrid)
  int visc_mg = 0;  // > 0: that many viscous V-cycles (visc_sweeps pre and post) instead of plain sweeps
  double theta = 0.5;
};

template <typename T>
int precond_alloc(Precond<T>& P, const GridDev& g, std::string& err);
template <typename T>
void precond_free(Precond<T>& P);
// rebuild level coefficients from the float64 fine coefficients
template <typename T>
int precond_setup(Precond<T>& P, const GridDev& g, const Coef<double>& fine, cudaStream_t st, std::string& err);
// z = P^{-1} v  (packed float64 Stokes vectors)
template <typename T>
void precond_apply(Precond<T>& P, const GridDev& g, const Opts& o, double dt, const double* v, double* z,
                   cudaStream_t st);

// ---------------------------------------------------------------- waves.cu
struct WaveDev {
  double H, d, omega, k, a1, a2, c2, x_gen, x_damp, lx, eps;
  int vert;
};
WaveDev wave_setup(double H, double T, double d, double x_gen, double x_damp, double lx, int vert, double eps,
                   double grav);
// Dirichlet inlet on the x- plane (waves.cu): data at time t (gn: nz x ny
// normal velocities, gw: (nz+1) x ny tangential velocities of the x- edges),
// their lifting into the right-hand side b of the implicit solve (with the
// explicit viscous term's tangential data gw_n), and u's x- faces <- gn
void launch_inlet_data(const GridDev& g, const WaveDev& w, double t, double* gn, double* gw, cudaStream_t st);
void launch_inlet_lift(const GridDev& g, const double* mu_cc, const double* mu_xy, const double* mu_xz,
                       const double* mu_xz_n, const double* gn, const double* gw, const double* gw_n, double theta,
                       double* b, cudaStream_t st);
void launch_inlet_set(const GridDev& g, const double* gn, double* u, cudaStream_t st);
void launch_wave_relax(const GridDev& g, const WaveDev& w, double t, double* const vel[3], double* phi,
                       cudaStream_t st);

// learned.cu
int learned_setup(Precond<float>& P, const double* rho_cc, const double* phi, cudaStream_t st, std::string& err);
// x_level (+)= network correction for rhs (the level's b, or a residual)
void learned_correction(Precond<float>& P, int level, const float* rhs, bool add, cudaStream_t st);
// one training step on the exact pair of a smooth field e (device float on
// the level); for the augmenting mode the pair is taken after the plain
// coarse-grid correction of r = L e.  The loss (device scalar: learned_loss)
// is the residual norm of the correction plus a small error term.
void learned_train(Precond<float>& P, const Opts& o, const float* e, double lr, cudaStream_t st);
const double* learned_loss(const Precond<float>& P);
int learned_alloc(Precond<float>& P, UNetImpl* net, int level, UNetImpl* gnet, int glevel, std::string& err);
// initial guess: P.lev[0].x = prolongation of the guess network's level-g
// solution for the fine right-hand side b0 (float, the level-0 grid)
void learned_guess(Precond<float>& P, const float* b0, cudaStream_t st);
// one Adam step of the guess network on a solver-generated pair (fine
// right-hand side y and its solution x, float on the level-0 grid): both
// averaged down to level g; loss 1/2 mean((o - d x_g / s)^2)
void learned_train_guess(Precond<float>& P, const float* y, const float* x, double lr, cudaStream_t st);
const double* learned_guess_loss(const Precond<float>& P);
// lev[from].x carried to level 0: each finer x set to the prolongation
template <typename T>
void precond_prolong_chain(Precond<T>& P, int from, cudaStream_t st);
// one V-cycle on level 0 of the hierarchy (x, b of level 0)
template <typename T>
void precond_vcycle(Precond<T>& P, const Opts& o, cudaStream_t st);
// everything of a V-cycle on level l but the post-smoothing (x, b of level l)
template <typename T>
void precond_coarse_part(Precond<T>& P, const Opts& o, int l, cudaStream_t st);

// ---------------------------------------------------------------- dlm.cu
void launch_ib_interp(const GridDev& g, const double* const vel[3], const double* X, int n, double* U,
                      cudaStream_t st);
// deterministic spreading (fixed-point integer sums): work arrays that stay
// zero between calls, and the box of cells the markers' taps can reach
struct SpreadWork {
  unsigned long long* acc = nullptr;  // one per face of the packed velocity
  int* cnt = nullptr;                 // one per cell
  int* qexp = nullptr;                // quantum exponent of the current call
  double* part = nullptr;             // reduction partials (6 x 152 doubles)
};
struct SpreadBox {
  int lo[3], hi[3];  // cells, inclusive
};
// box from the marker extent mm = (min x, y, z, max x, y, z)
SpreadBox spread_box(const GridDev& g, const double mm[6]);
void launch_marker_box(const double* X, int n, double* out6, double* scratch, cudaStream_t st);
void launch_ib_spread(const GridDev& g, const double* F, const double* X, int n, double dV, double* const vel[3],
                      const SpreadWork& w, const SpreadBox& b, cudaStream_t st);
// rigid sums: out[0..2] sum U, [3..5] sum R x U, [6..11] sum of R.R I - R (x) R (xx,yy,zz,xy,xz,yz),
// [12..14] sum X; R relative to xc_dev
void launch_rigid_sums(const double* X, const double* U, int n, const double* xc_dev, double* out, double* scratch,
                       cudaStream_t st);
void launch_marker_mean(const double* X, int n, double* xc_dev, double* scratch, cudaStream_t st);
// F = U_r + W_r x (X - xc) - U   (body velocity minus interpolated); Ub also stored
void launch_body_velocity(const double* X, const double* U, int n, const double* rigid_dev, const double* xc_dev,
                          double* Ub, double* F, cudaStream_t st);
// X = X^n + dt (U_b^{n+1} + U_b^n) / 2; *flag |= 1 when a marker leaves the box
// (by more than half a cell) or is not finite (flag may be null)
void launch_marker_update(const GridDev& g, const double* Xn, const double* Ub_new, const double* Ub_old, int n,
                          double dt, double* X, int* flag, cudaStream_t st);

}  // namespace wsi
