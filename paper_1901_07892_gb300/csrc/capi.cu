// C ABI of libwsi (include/wsi.h): context management, the FGMRES driver of
// the implicit Stokes solve (Sec. 4.2.4), the rigidity step (Sec. 4.2.5) and
// the two-cycle time step (Sec. 4.2).  All compute runs in the kernels of
// ops.cu, mg.cu, krylov.cu and dlm.cu; the host only sequences launches,
// runs the (m+1) x m Hessenberg least-squares update of FGMRES and solves the
// 3 x 3 inertia system of a free body.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <random>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "df.cuh"
#include "internal.h"

using namespace wsi;

std::atomic<long long> wsi::g_launches{0};

namespace {
// per-kernel-class event timer (one class enabled at a time, process-wide)
struct KTimer {
  int enabled = -1;
  std::vector<cudaEvent_t> start, stop;
  size_t used = 0;
  bool open = false;
  double bytes = 0.0;  // algorithmic bytes reported by launchers of the enabled class
};
KTimer g_kt;
constexpr size_t KT_MAX = 1 << 16;
}  // namespace

void wsi::ktimer_begin(int id, cudaStream_t st) {
  if (id != g_kt.enabled || g_kt.used >= KT_MAX) return;
  if (g_kt.used == g_kt.start.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    g_kt.start.push_back(a);
    g_kt.stop.push_back(b);
  }
  cudaEventRecord(g_kt.start[g_kt.used], st);
  g_kt.open = true;
}

void wsi::ktimer_bytes(int id, double bytes) {
  if (id == g_kt.enabled && g_kt.used < KT_MAX) g_kt.bytes += bytes;
}

void wsi::ktimer_end(int id, cudaStream_t st) {
  if (id != g_kt.enabled || !g_kt.open) return;
  cudaEventRecord(g_kt.stop[g_kt.used], st);
  ++g_kt.used;
  g_kt.open = false;
}

struct Body {
  int n = 0;
  double dV = 0.0;
  int lock[6] = {1, 1, 1, 1, 1, 1};
  double U_pres[3] = {0, 0, 0}, W_pres[3] = {0, 0, 0};
  int shape = 0;
  double half[3] = {0, 0, 0};
  double *X = nullptr, *Xn = nullptr, *Xh = nullptr, *Ub = nullptr, *Ub_n = nullptr, *U = nullptr, *F = nullptr;
  double* xc = nullptr;       // 3 doubles: centre of mass used for R
  double* rig = nullptr;      // 6 doubles: U_r, W_r
  int* flag = nullptr;        // device bound check of the marker update
  double* sums = nullptr;     // 15 doubles
  double* scratch = nullptr;  // reduction partials
  double U_r[3] = {0, 0, 0}, W_r[3] = {0, 0, 0}, X_com[3] = {0, 0, 0};
};

struct wsi_ctx {
  GridDev g;
  Packing pk;
  cudaStream_t st = nullptr;
  wsi_grid_desc desc;
  wsi_phase_props props;
  bool have_phases = false;
  std::string err;
  std::vector<void*> allocs;
  size_t nvel = 0, nstk = 0, ncell = 0;
  // float64 coefficients of the current operator
  double *rho_cc = nullptr, *mu_cc = nullptr, *rho_face[3], *beta[3], *rho_flow[3], *mu_e[3];
  // time-n coefficients (right-hand side)
  double *mu_cc_n = nullptr, *mu_e_n[3], *rho_n[3], *beta_n[3], *rho_flow_n[3];
  // state
  double *vel = nullptr, *vel_old = nullptr, *p = nullptr, *phi = nullptr, *psi = nullptr;
  // step scratch
  double *vel_k = nullptr, *vel_half = nullptr, *u1 = nullptr, *u2 = nullptr, *rs1 = nullptr, *rs2 = nullptr,
         *R = nullptr, *Cc = nullptr, *phi_k = nullptr, *phi_new = nullptr, *phi_half = nullptr, *psi_k = nullptr,
         *psi_new = nullptr, *b = nullptr, *x = nullptr, *rho_cc_tmp = nullptr;
  // Krylov
  int m = 20;
  double *V = nullptr, *Z = nullptr, *hdev = nullptr, *red = nullptr;
  Precond<double> P64;
  Precond<float> P32;
  bool pc_dirty = true;
  bool pc_alloc = false;
  Opts opts;
  Body body;
  bool has_body = false;
  // float64 part of the momentum right-hand side fixed over a step's cycles
  double* b0 = nullptr;
  double* inv_mu = nullptr;  // materials scratch: 1/mu per cell
  // mixed path: split (hi, lo) copies of the operator coefficients (refreshed
  // at the start of every solve) and of the matvec input
  DfOperands df;
  int* df_err = nullptr;  // set by the matvec when a wait for a tile copy gave up
  // a fully locked body at rest never moves: psi is rebuilt once, then kept
  bool psi_static_done = false;
  // mu_cc / mu_e hold mu(phi^n, psi^n) (true right after a step)
  bool mat_n_valid = false;
  double* ri_scratch = nullptr;  // reinitialisation: 3 x ncell doubles, on first use
  void* ones = nullptr;          // unit face density of the non-conservative convection, on first use
  // learned coarse correction of the float32 pressure multigrid
  wsi_unet* unet = nullptr;
  UNetImpl* unet_impl = nullptr;
  int unet_level = 0;
  bool unet_on = false;
  SpreadWork sw;                  // deterministic spreading work arrays (allocated on first use)
  double* mbox = nullptr;         // 6 doubles: marker extent
  UNetImpl* gunet_impl = nullptr;  // initial-guess network (wsi_attach_unet_guess)
  int gunet_level = 0;
  const double* phi_cur = nullptr;  // level set behind the current coefficients
  // wave tank relaxation zones (Sec. 7.1) and the time of the state
  bool has_waves = false;
  WaveDev wave;
  double time = 0.0;
  // Dirichlet wave inlet on the x- plane (Sec. 7.1): normal data at t^{n+1}
  // (nz x ny) and tangential data of u^{n-1}, u^n, u^{n+1} ((nz+1) x ny),
  // with the combination of a stage velocity (float64 and float32)
  bool inlet = false;
  double *in_gn = nullptr, *in_gw_nm1 = nullptr, *in_gw_n = nullptr, *in_gw_np1 = nullptr, *in_gs = nullptr;
  float* in_gs32 = nullptr;
  // float32 shadows of the explicitly transported fields (mixed path)
  float *vn32 = nullptr, *u1_32 = nullptr, *u2_32 = nullptr, *rn32 = nullptr, *r1_32 = nullptr, *r2_32 = nullptr,
        *R32 = nullptr, *C32 = nullptr, *vh32 = nullptr, *phih32 = nullptr, *mu_cc_n32 = nullptr,
        *mu_e_n32[3] = {nullptr, nullptr, nullptr};
  bool mixed() const { return desc.precision == WSI_PREC_MIXED; }
};

namespace {

int fail(wsi_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(wsi_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(c, WSI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return WSI_OK;
}

double* dalloc(wsi_ctx* c, size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) return nullptr;
  cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(double), c->st);
  c->allocs.push_back(p);
  return (double*)p;
}

// deterministic spreading work arrays (zero-filled; they are left zero by
// every spreading call)
bool ensure_spread_work(wsi_ctx* c) {
  if (c->sw.acc) return true;
  c->sw.acc = (unsigned long long*)dalloc(c, c->nvel);
  c->sw.cnt = (int*)dalloc(c, c->ncell / 2 + 1);
  c->sw.qexp = (int*)dalloc(c, 1);
  c->sw.part = dalloc(c, 6 * 152);
  c->mbox = dalloc(c, 6);
  return c->sw.acc && c->sw.cnt && c->sw.qexp && c->sw.part && c->mbox;
}

void vel_parts(wsi_ctx* c, double* base, double* out[3]) {
  for (int d = 0; d < 3; ++d) out[d] = base + c->pk.off[d];
}
void vel_parts(wsi_ctx* c, const double* base, const double* out[3]) {
  for (int d = 0; d < 3; ++d) out[d] = base + c->pk.off[d];
}

Coef<double> coef_now(wsi_ctx* c) {
  Coef<double> cf;
  for (int d = 0; d < 3; ++d) {
    cf.rho_face[d] = c->rho_face[d];
    cf.beta[d] = c->beta[d];
    cf.mu_e[d] = c->mu_e[d];
  }
  cf.mu_cc = c->mu_cc;
  return cf;
}

Coef<double> coef_n(wsi_ctx* c) {
  Coef<double> cf;
  for (int d = 0; d < 3; ++d) {
    cf.rho_face[d] = c->rho_n[d];
    cf.beta[d] = c->beta_n[d];
    cf.mu_e[d] = c->mu_e_n[d];
  }
  cf.mu_cc = c->mu_cc_n;
  return cf;
}

PhaseConst phase_const(wsi_ctx* c) {
  PhaseConst pc;
  pc.rho_l = c->props.rho_l;
  pc.rho_g = c->props.rho_g;
  pc.rho_s = c->props.rho_s;
  pc.mu_l = c->props.mu_l;
  pc.mu_g = c->props.mu_g;
  pc.mu_s = c->props.mu_s;
  double hc = c->g.n[2] == 1 ? sqrt(c->g.h[0] * c->g.h[1]) : cbrt(c->g.h[0] * c->g.h[1] * c->g.h[2]);
  pc.eps = c->desc.n_cells * hc;
  pc.inv_mu = c->inv_mu;
  phase_tables(pc);
  return pc;
}

// 1/a in double-float arithmetic: float32 reciprocal r, residual 1 - a r
// formed with a split into (hi, lo) and fused multiply-adds, one Newton step;
// one float64 addition forms the result (~1e-14 relative).  Zero,
// subnormal-range and non-finite a take the float64 division.
__global__ void k_recip(size_t n, const double* __restrict__ a, double* b) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double v = a[t];
  const dfl x = df_split(v);
  if (!(fabsf(x.h) > 1e-30f) || !(fabsf(x.h) < 1e30f)) {
    b[t] = 1.0 / v;
    return;
  }
  const float r = 1.0f / x.h;
  // e = 1 - x r, exactly enough: fma for the leading product, lo part plainly
  const float e = fmaf(-x.h, r, 1.0f) - x.l * r;
  b[t] = df_to_double(quick_two_sum(r, r * e));
}

void recip(wsi_ctx* c, const double* a, double* b, size_t n) {
  if (n) { k_recip<<<cdiv(n, 256), 256, 0, c->st>>>(n, a, b); WSI_COUNT(); }
}

int copy_in(wsi_ctx* c, double* dst, const double* src, size_t n) {
  if (!src) return fail(c, WSI_ERR_INVALID_ARG, "null input pointer");
  if (cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->st) != cudaSuccess)
    return fail(c, WSI_ERR_CUDA, "copy in failed");
  return WSI_OK;
}
int copy_out(wsi_ctx* c, double* dst, const double* src, size_t n) {
  if (!dst) return fail(c, WSI_ERR_INVALID_ARG, "null output pointer");
  if (cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->st) != cudaSuccess)
    return fail(c, WSI_ERR_CUDA, "copy out failed");
  return WSI_OK;
}

int ensure_pc(wsi_ctx* c) {
  if (!c->pc_alloc) {
    // allocated on first use: grids that are only used for operator applies
    // need no multigrid hierarchy
    int rc = c->desc.precision == WSI_PREC_MIXED ? precond_alloc<float>(c->P32, c->g, c->err)
                                                 : precond_alloc<double>(c->P64, c->g, c->err);
    if (rc) return rc;
    c->pc_alloc = true;
  }
  if (!c->pc_dirty) return WSI_OK;
  Coef<double> cf = coef_now(c);
  int rc = c->desc.precision == WSI_PREC_MIXED ? precond_setup<float>(c->P32, c->g, cf, c->st, c->err)
                                               : precond_setup<double>(c->P64, c->g, cf, c->st, c->err);
  if (rc == WSI_OK && c->mixed()) {
    rc = learned_alloc(c->P32, c->unet_impl, c->unet_level, c->gunet_impl, c->gunet_level, c->err);
    if (rc == WSI_OK && (c->unet_impl || c->gunet_impl))
      rc = learned_setup(c->P32, c->rho_cc, c->phi_cur ? c->phi_cur : c->phi, c->st, c->err);
    c->P32.learn.on = c->unet_on;
  }
  if (rc == WSI_OK) c->pc_dirty = false;
  return rc;
}

void pc_apply(wsi_ctx* c, double dt, const double* v, double* z) {
  if (c->desc.precision == WSI_PREC_MIXED)
    precond_apply<float>(c->P32, c->g, c->opts, dt, v, z, c->st);
  else
    precond_apply<double>(c->P64, c->g, c->opts, dt, v, z, c->st);
}

// split copies of the coefficients for the double-float matvec (mixed path);
// the face density is stored times 1/dt
void df_coef_refresh(wsi_ctx* c, const Coef<double>& cf, double inv_dt) {
  if (!c->mixed()) return;
  df_split_coefs(c->df, cf.rho_face, cf.mu_e, cf.mu_cc, inv_dt, c->st);  // one launch for the seven arrays
}

// K x: float64 on the plain path; on the mixed path in double-float
// arithmetic (same accuracy class, a fraction of the float64 instructions)
// from the coefficients split by the last df_coef_refresh
void stokes_mv(wsi_ctx* c, const Coef<double>& cf, double inv_dt, double theta, const double* x, double* y,
               cudaStream_t st) {
  if (c->mixed()) {
    (void)inv_dt;  // folded into the split face density by df_coef_refresh
    launch_stokes_df(c->g, c->df, theta, x, y, c->df_err, st);
  } else {
    launch_stokes(c->g, cf, inv_dt, theta, x, y, st);
  }
}

// reads and clears the matvec's device error flag (synchronises the stream)
int df_check(wsi_ctx* c) {
  if (!c->mixed() || !c->df_err) return WSI_OK;
  int h = 0;
  cudaMemcpyAsync(&h, c->df_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "matvec");
  if (!h) return WSI_OK;
  cudaMemsetAsync(c->df_err, 0, sizeof(int), c->st);
  return fail(c, WSI_ERR_DEVICE, "the double-float matvec gave up waiting for a tile copy");
}

// FGMRES(m), right preconditioned by the projection method; float64 Arnoldi
// with classical Gram-Schmidt (see the iteration for the re-orthogonalisation
// rule).
int fgmres(wsi_ctx* c, const double* b, double* x, double dt, const wsi_solve_opts* o, wsi_solve_stats* s) {
  int rc = ensure_pc(c);
  if (rc) return rc;
  const size_t n = c->nstk;
  const int m = c->m;
  const double inv_dt = 1.0 / dt, theta = c->desc.theta;
  Coef<double> cf = coef_now(c);
  df_coef_refresh(c, cf, inv_dt);
  double* V = c->V;
  double* Z = c->Z;
  double* hd = c->hdev;
  double* red = c->red;
  auto Vj = [&](int j) { return V + (size_t)j * n; };
  auto Zj = [&](int j) { return Z + (size_t)j * n; };
  double bnorm = host_norm2(b, n, red, c->st);
  int iters = 0;
  s->iters = 0;
  s->learned_rejected = -1;
  s->rel_residual = 0.0;
  if (!std::isfinite(bnorm)) return fail(c, WSI_ERR_NAN, "non-finite right-hand side");
  if (bnorm == 0.0) {
    cudaMemsetAsync(x, 0, n * sizeof(double), c->st);
    return cuda_check(c, "fgmres");
  }
  if (!o->use_x0) cudaMemsetAsync(x, 0, n * sizeof(double), c->st);
  // r = b - K x  into V_0
  stokes_mv(c, cf, inv_dt, theta, x, Vj(0), c->st);
  launch_lincomb(n, 1.0, b, -1.0, Vj(0), 0.0, nullptr, Vj(0), c->st);
  double beta = host_norm2(Vj(0), n, red, c->st);
  const double tol = o->rtol * bnorm;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1), hcol(2 * (m + 1) + 1);
  int result = WSI_OK;
  while (true) {
    if (!std::isfinite(beta)) return fail(c, WSI_ERR_NAN, "non-finite residual");
    if (beta <= tol) break;
    if (iters >= o->max_iters) {
      result = WSI_ERR_NOT_CONVERGED;
      break;
    }
    double ib = 1.0 / beta;
    cudaMemcpyAsync(hd, &ib, sizeof(double), cudaMemcpyHostToDevice, c->st);
    launch_scale(Vj(0), n, hd, false, c->st);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m; ++j) {
      pc_apply(c, dt, Vj(j), Zj(j));
      double* w = Vj(j + 1);
      stokes_mv(c, cf, inv_dt, theta, Zj(j), w, c->st);
      // Classical Gram-Schmidt.  One pass gives h = V^T w together with w.w
      // (w is V_{j+1}, the last row), so ||w - V h||^2 = w.w - |h|^2 needs no
      // second pass; when that cancels by more than half (the DGKS test) the
      // vector is orthogonalised a second time.  The final axpy also
      // normalises.
      const size_t o2 = (size_t)m + 2, osc = 2 * (size_t)m + 4;
      launch_mdot(V, n, j + 2, w, n, hd, red, c->st);
      cudaMemcpyAsync(hcol.data(), hd, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, c->st);
      if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "fgmres iteration");
      ++iters;
      double ww = hcol[j + 1], hh = 0.0;
      for (int i = 0; i <= j; ++i) hh += hcol[i] * hcol[i];
      double hn2 = ww - hh;
      std::vector<double> hsum(hcol.begin(), hcol.begin() + (j + 1));
      const double* hcoef = hd;
      if (!(hn2 >= 0.5 * ww)) {
        launch_maxpy(V, n, j + 1, hd, w, n, 1.0, c->st);
        launch_mdot(V, n, j + 2, w, n, hd + o2, red, c->st);
        cudaMemcpyAsync(hcol.data(), hd + o2, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, c->st);
        if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "fgmres reorthogonalisation");
        double ww2 = hcol[j + 1], hh2 = 0.0;
        for (int i = 0; i <= j; ++i) {
          hh2 += hcol[i] * hcol[i];
          hsum[i] += hcol[i];
        }
        hn2 = ww2 - hh2;
        hcoef = hd + o2;
      }
      double hn = sqrt(std::max(hn2, 0.0));
      if (!std::isfinite(hn)) return fail(c, WSI_ERR_NAN, "non-finite Krylov vector");
      double ihn = hn > 0.0 ? 1.0 / hn : 0.0;
      cudaMemcpyAsync(hd + osc, &ihn, sizeof(double), cudaMemcpyHostToDevice, c->st);
      launch_maxpy(V, n, j + 1, hcoef, w, n, 1.0, c->st, hd + osc);
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hsum[i];
      H[(size_t)(j + 1) * m + j] = hn;
      // previous rotations
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      double r = hypot(a, bb);
      cs[j] = r == 0.0 ? 1.0 : a / r;
      sn[j] = r == 0.0 ? 0.0 : bb / r;
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      double res = fabs(gv[j + 1]);
      if (res <= tol || iters >= o->max_iters || hn == 0.0) {
        ++j;
        done = true;
        break;
      }
    }
    if (!done) j = m;
    // y = H^{-1} g (upper triangular j x j)
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double sacc = gv[i];
      for (int k = i + 1; k < j; ++k) sacc -= H[(size_t)i * m + k] * y[k];
      y[i] = sacc / H[(size_t)i * m + i];
    }
    cudaMemcpyAsync(hd, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, c->st);
    launch_maxpy(Z, n, j, hd, x, n, -1.0, c->st);
    // true residual
    stokes_mv(c, cf, inv_dt, theta, x, Vj(0), c->st);
    launch_lincomb(n, 1.0, b, -1.0, Vj(0), 0.0, nullptr, Vj(0), c->st);
    beta = host_norm2(Vj(0), n, red, c->st);
  }
  // zero-mean pressure in a closed box (an open top fixes the pressure)
  if (!c->g.open_top) {
    launch_sum<double>(x + c->pk.off[3], c->ncell, hd, red, c->st);
    launch_add_scalar_from<double>(x + c->pk.off[3], c->ncell, hd, -1.0 / (double)c->ncell, c->st);
  }
  s->iters = iters;
  s->rel_residual = beta / bnorm;
  int crc = cuda_check(c, "fgmres");
  if (crc) return crc;
  crc = df_check(c);
  if (crc) return crc;
  if (result == WSI_ERR_NOT_CONVERGED) c->err = "FGMRES reached max_iters";
  return result;
}

// 3x3 solve with partial pivoting; returns false if singular
bool solve3(double A[3][3], const double b[3], double x[3]) {
  double M[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
    M[i][3] = b[i];
  }
  double scale = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) scale = std::max(scale, fabs(A[i][j]));
  for (int p = 0; p < 3; ++p) {
    int piv = p;
    for (int r = p + 1; r < 3; ++r)
      if (fabs(M[r][p]) > fabs(M[piv][p])) piv = r;
    if (fabs(M[piv][p]) <= 1e-300 + 1e-14 * scale) return false;
    for (int k = 0; k < 4; ++k) std::swap(M[p][k], M[piv][k]);
    for (int r = 0; r < 3; ++r) {
      if (r == p) continue;
      double f = M[r][p] / M[p][p];
      for (int k = p; k < 4; ++k) M[r][k] -= f * M[p][k];
    }
  }
  for (int i = 0; i < 3; ++i) x[i] = M[i][3] / M[i][i];
  return true;
}

// Rigidity projection at marker positions Xuse: vel += S(U_b - J vel).
int dlm_project(wsi_ctx* c, double* velv, const double* Xuse) {
  Body& B = c->body;
  double* vq[3];
  vel_parts(c, velv, vq);
  const double* cq[3] = {vq[0], vq[1], vq[2]};
  if (!ensure_spread_work(c)) return fail(c, WSI_ERR_OOM, "out of device memory for spreading");
  launch_marker_mean(Xuse, B.n, B.xc, B.scratch, c->st);
  launch_ib_interp(c->g, cq, Xuse, B.n, B.U, c->st);
  launch_rigid_sums(Xuse, B.U, B.n, B.xc, B.sums, B.scratch, c->st);
  launch_marker_box(Xuse, B.n, c->mbox, c->sw.part, c->st);
  double hs[15], xc[3], mm[6];
  cudaMemcpyAsync(hs, B.sums, sizeof(hs), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(xc, B.xc, sizeof(xc), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(mm, c->mbox, sizeof(mm), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "dlm sums");
  double Ur[3], Wr[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) Ur[d] = hs[d] / (double)B.n;
  double I[3][3] = {{hs[6], hs[9], hs[10]}, {hs[9], hs[7], hs[11]}, {hs[10], hs[11], hs[8]}};
  double L[3] = {hs[3], hs[4], hs[5]};
  if (!solve3(I, L, Wr)) {
    // planar body: rotation only about the normal of its plane
    for (int d = 0; d < 3; ++d) Wr[d] = (I[d][d] > 0.0 && L[d] != 0.0) ? L[d] / I[d][d] : 0.0;
  }
  for (int d = 0; d < 3; ++d) {
    if (B.lock[d]) Ur[d] = B.U_pres[d];
    if (B.lock[3 + d]) Wr[d] = B.W_pres[d];
  }
  double rg[6] = {Ur[0], Ur[1], Ur[2], Wr[0], Wr[1], Wr[2]};
  cudaMemcpyAsync(B.rig, rg, sizeof(rg), cudaMemcpyHostToDevice, c->st);
  launch_body_velocity(Xuse, B.U, B.n, B.rig, B.xc, B.Ub, B.F, c->st);
  launch_ib_spread(c->g, B.F, Xuse, B.n, B.dV, vq, c->sw, spread_box(c->g, mm), c->st);
  for (int d = 0; d < 3; ++d) {
    B.U_r[d] = Ur[d];
    B.W_r[d] = Wr[d];
    B.X_com[d] = xc[d];
  }
  return cuda_check(c, "dlm project");
}


template <typename T>
void parts(wsi_ctx* c, T* base, T* out[3]) {
  for (int d = 0; d < 3; ++d) out[d] = base + c->pk.off[d];
}
template <typename T>
void cparts(wsi_ctx* c, const T* base, const T* out[3]) {
  for (int d = 0; d < 3; ++d) out[d] = base + c->pk.off[d];
}

// SSP-RK3 face density and the consistent convective term (Sec. 4.2.2):
// rho_face <- rho^{n+1,k+1} (beta <- 1/rho), C into c->Cc (plain) or
// c->C32 (mixed).  Stage 1 depends on (u^n, rho^n) only; with reuse_stage1
// its result from an earlier cycle of the same step is kept.
// tangential inlet data of a stage velocity a u_k + b u_n + c u_{n-1}: the
// same combination of the data (u_k's data: at t^{n+1}), into in_gs (and its
// float32 copy on the mixed path); null without an inlet
const void* inlet_stage_data(wsi_ctx* c, double a, double b, double cc) {
  if (!c->inlet) return nullptr;
  const size_t n = (size_t)(c->g.n[2] + 1) * c->g.n[1];
  launch_lincomb(n, a, c->in_gw_np1, b, c->in_gw_n, cc, c->in_gw_nm1, c->in_gs, c->st);
  if (!c->mixed()) return c->in_gs;
  launch_lincomb_to_f32(n, 1.0, c->in_gs, 0.0, nullptr, 0.0, nullptr, c->in_gs32, c->st);
  return c->in_gs32;
}

void transport_stage(wsi_ctx* c, int k, double dt, const double* un, const double* unm1, const double* uk,
                     bool reuse_stage1) {
  const GridDev& g = c->g;
  cudaStream_t st = c->st;
  const size_t nv = c->nvel;
  // the convective term's velocity is u^(2): its inlet data likewise
  const void* g2 = k == 0 ? inlet_stage_data(c, 0.0, 1.5, -0.5) : inlet_stage_data(c, 0.375, 0.75, -0.125);
  if (!c->mixed()) {
    if (k == 0) {
      launch_lincomb(nv, 2.0, un, -1.0, unm1, 0.0, nullptr, c->u1, st);
      launch_lincomb(nv, 1.5, un, -0.5, unm1, 0.0, nullptr, c->u2, st);
    } else {
      launch_lincomb(nv, 1.0, uk, 0.0, nullptr, 0.0, nullptr, c->u1, st);
      launch_lincomb(nv, 0.375, uk, 0.75, un, -0.125, unm1, c->u2, st);
    }
    double *R[3], *Cq[3], *r1[3], *r2[3];
    parts(c, c->R, R);
    parts(c, c->Cc, Cq);
    parts(c, c->rs1, r1);
    parts(c, c->rs2, r2);
    const double *cun[3], *cu1[3], *cu2[3];
    cparts(c, un, cun);
    cparts(c, (const double*)c->u1, cu1);
    cparts(c, (const double*)c->u2, cu2);
    const double* crn[3] = {c->rho_n[0], c->rho_n[1], c->rho_n[2]};
    if (!reuse_stage1) {
      launch_transport_flux<double>(g, cun, crn, false, R, st);
      for (int d = 0; d < 3; ++d) launch_lincomb(fsize(g, d), 1.0, c->rho_n[d], -dt, R[d], 0.0, nullptr, r1[d], st);
    }
    const double* cr1[3] = {r1[0], r1[1], r1[2]};
    launch_transport_flux<double>(g, cu1, cr1, false, R, st);
    for (int d = 0; d < 3; ++d)
      launch_lincomb(fsize(g, d), 0.75, c->rho_n[d], 0.25, r1[d], -0.25 * dt, R[d], r2[d], st);
    const double* cr2[3] = {r2[0], r2[1], r2[2]};
    launch_transport_flux<double>(g, cu2, cr2, false, R, st);
    for (int d = 0; d < 3; ++d)
      launch_lincomb(fsize(g, d), 1.0 / 3.0, c->rho_n[d], 2.0 / 3.0, r2[d], -2.0 / 3.0 * dt, R[d], c->rho_face[d],
                     st);
    launch_transport_flux<double>(g, cu2, cr2, true, Cq, st, (const double*)g2);
  } else {
    float *R[3], *Cq[3], *r1[3], *r2[3], *rn[3];
    parts(c, c->R32, R);
    parts(c, c->C32, Cq);
    parts(c, c->r1_32, r1);
    parts(c, c->r2_32, r2);
    parts(c, c->rn32, rn);
    // stage velocities (and the float32 u^n when stage 1 is formed afresh)
    launch_rk_velocities_f32(nv, un, unm1, k == 0 ? nullptr : uk, c->u1_32, c->u2_32,
                             reuse_stage1 ? nullptr : c->vn32, st);
    const float *cvn[3], *cu1[3], *cu2[3], *crn[3];
    cparts(c, (const float*)c->vn32, cvn);
    cparts(c, (const float*)c->u1_32, cu1);
    cparts(c, (const float*)c->u2_32, cu2);
    cparts(c, (const float*)c->rn32, crn);
    if (!reuse_stage1) {
      for (int d = 0; d < 3; ++d)
        launch_lincomb_to_f32(fsize(g, d), 1.0, c->rho_n[d], 0.0, nullptr, 0.0, nullptr, rn[d], st);
      launch_transport_flux<float>(g, cvn, crn, false, R, st);
      launch_lincomb_f32(nv, 1.0f, c->rn32, (float)-dt, c->R32, 0.0f, nullptr, c->r1_32, st);
    }
    const float* cr1[3] = {r1[0], r1[1], r1[2]};
    launch_transport_flux<float>(g, cu1, cr1, false, R, st);
    launch_lincomb_f32(nv, 0.75f, c->rn32, 0.25f, c->r1_32, (float)(-0.25 * dt), c->R32, c->r2_32, st);
    const float* cr2[3] = {r2[0], r2[1], r2[2]};
    launch_transport_flux<float>(g, cu2, cr2, false, R, st);
    for (int d = 0; d < 3; ++d)
      launch_lincomb_mix(fsize(g, d), 1.0 / 3.0, c->rho_n[d], 2.0 / 3.0, r2[d], -2.0 / 3.0 * dt, R[d],
                         c->rho_face[d], st);
    launch_transport_flux<float>(g, cu2, cr2, true, Cq, st, (const float*)g2);
  }
  for (int d = 0; d < 3; ++d) recip(c, c->rho_face[d], c->beta[d], fsize(g, d));
}

// phi_out = phi_n - dt Q(u_half, phi_half) with u_half = (vk + vn)/2 and
// phi_half = (phik + phin)/2 (Sec. 4.2.1)
void levelset_stage(wsi_ctx* c, const double* vk, const double* vn, const double* phik, const double* phin,
                    double dt, double* phi_out) {
  const GridDev& g = c->g;
  cudaStream_t st = c->st;
  if (!c->mixed()) {
    launch_lincomb(c->nvel, 0.5, vk, 0.5, vn, 0.0, nullptr, c->vel_half, st);
    launch_lincomb(c->ncell, 0.5, phik, 0.5, phin, 0.0, nullptr, c->phi_half, st);
    const double* vh[3];
    cparts(c, (const double*)c->vel_half, vh);
    launch_levelset_advect<double>(g, vh, phin, c->phi_half, dt, phi_out, st, c->desc.ls_limiter);
  } else {
    launch_lincomb_to_f32(c->nvel, 0.5, vk, 0.5, vn, 0.0, nullptr, c->vh32, st);
    launch_lincomb_to_f32(c->ncell, 0.5, phik, 0.5, phin, 0.0, nullptr, c->phih32, st);
    const float* vh[3];
    cparts(c, (const float*)c->vh32, vh);
    launch_levelset_advect<float>(g, vh, phin, c->phih32, dt, phi_out, st, c->desc.ls_limiter);
  }
}

// b0 = rho^n u^n/dt + (1-theta) L_mu^n u^n  (needs transport_stage's float32
// copy of u^n on the mixed path)
// b0 = rho^n u^n w + (1 - theta) L_mu^n u^n; w = 1/dt for the consistent
// form, 0 for the non-conservative one (its mass term uses rho^{n+1,k+1})
void rhs_base(wsi_ctx* c, double w) {
  const GridDev& g = c->g;
  cudaStream_t st = c->st;
  double* b0[3];
  parts(c, c->b0, b0);
  const double* un[3];
  cparts(c, (const double*)c->vel, un);
  const double* crn[3] = {c->rho_n[0], c->rho_n[1], c->rho_n[2]};
  if (!c->mixed()) {
    launch_rhs_base<double>(g, coef_n(c), un, crn, un, w, c->desc.theta, b0, st);
  } else {
    launch_lincomb_to_f32(c->ncell, 1.0, c->mu_cc_n, 0.0, nullptr, 0.0, nullptr, c->mu_cc_n32, st);
    for (int e = 0; e < 3; ++e)
      launch_lincomb_to_f32(esize(g, e), 1.0, c->mu_e_n[e], 0.0, nullptr, 0.0, nullptr, c->mu_e_n32[e], st);
    Coef<float> cf;
    for (int d = 0; d < 3; ++d) {
      cf.rho_face[d] = nullptr;
      cf.beta[d] = nullptr;
      cf.mu_e[d] = c->mu_e_n32[d];
    }
    cf.mu_cc = c->mu_cc_n32;
    const float* u32[3];
    cparts(c, (const float*)c->vn32, u32);
    launch_rhs_base<float>(g, cf, u32, crn, un, w, c->desc.theta, b0, st);
  }
}

int valid_ctx(wsi_ctx* c) { return c ? WSI_OK : WSI_ERR_INVALID_ARG; }

}  // namespace

__global__ void k_fill_one(double* a, float* f, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    if (a) a[t] = 1.0;
    if (f) f[t] = 1.0f;
  }
}

// Non-conservative convection (Sec. 4.2.3): N = div(u^{n+1/2,k} u_lim) with
// the CUI-limited velocity on the face control volumes, i.e. the momentum
// flux of the consistent scheme at unit density, from the half-step velocity
// the level-set stage of this cycle formed (vel_half, or vh32 on the mixed
// path).  Result in Cc (float64) or C32 (float32).
int nc_convection(wsi_ctx* c, int k) {
  const GridDev& g = c->g;
  cudaStream_t st = c->st;
  const size_t nv = c->nvel;
  // inlet data of the half-step velocity (u_k + u_n) / 2
  const void* gh = k == 0 ? inlet_stage_data(c, 0.0, 1.0, 0.0) : inlet_stage_data(c, 0.5, 0.5, 0.0);
  if (!c->ones) {
    c->ones = dalloc(c, nv);
    if (!c->ones) return fail(c, WSI_ERR_OOM, "unit density");
    const int blocks = (int)std::min<size_t>((nv + 255) / 256, 152 * 16);
    if (c->mixed())
      k_fill_one<<<blocks, 256, 0, st>>>(nullptr, (float*)c->ones, nv);
    else
      k_fill_one<<<blocks, 256, 0, st>>>((double*)c->ones, nullptr, nv);
    WSI_COUNT();
  }
  if (c->mixed()) {
    const float *vh[3], *one[3];
    float* N[3];
    cparts(c, (const float*)c->vh32, vh);
    cparts(c, (const float*)c->ones, one);
    parts(c, c->C32, N);
    launch_transport_flux<float>(g, vh, one, true, N, st, (const float*)gh);
  } else {
    const double *vh[3], *one[3];
    double* N[3];
    cparts(c, (const double*)c->vel_half, vh);
    cparts(c, (const double*)c->ones, one);
    parts(c, c->Cc, N);
    launch_transport_flux<double>(g, vh, one, true, N, st, (const double*)gh);
  }
  return WSI_OK;
}

// pseudo-time CFL number of the reinitialisation (local step cfl * h_min)
constexpr double kReinitCfl = 0.3;

int reinit_phi(wsi_ctx* c, double* phi, int iters) {
  if (iters <= 0) return WSI_OK;
  if (!c->ri_scratch) {
    c->ri_scratch = dalloc(c, 3 * c->ncell);
    if (!c->ri_scratch) return fail(c, WSI_ERR_OOM, "reinitialisation scratch");
  }
  if (c->mixed())
    reinit_levelset<float>(c->g, phi, iters, kReinitCfl, c->ri_scratch, c->st);
  else
    reinit_levelset<double>(c->g, phi, iters, kReinitCfl, c->ri_scratch, c->st);
  return WSI_OK;
}

extern "C" {

long long wsi_launch_count(void) { return g_launches.load(); }

int wsi_ktimer_enable(int kernel_class) {
  if (kernel_class < -1 || kernel_class >= KC_COUNT) return WSI_ERR_INVALID_ARG;
  g_kt.enabled = kernel_class;
  g_kt.used = 0;
  g_kt.open = false;
  g_kt.bytes = 0.0;
  return WSI_OK;
}

int wsi_ktimer_bytes(double* bytes) {
  if (!bytes) return WSI_ERR_INVALID_ARG;
  *bytes = g_kt.bytes;
  return WSI_OK;
}

int wsi_ktimer_read(double* total_ms, long long* launches) {
  if (!total_ms || !launches) return WSI_ERR_INVALID_ARG;
  double t = 0.0;
  for (size_t i = 0; i < g_kt.used; ++i) {
    if (cudaEventSynchronize(g_kt.stop[i]) != cudaSuccess) return WSI_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_kt.start[i], g_kt.stop[i]) != cudaSuccess) return WSI_ERR_CUDA;
    t += ms;
  }
  *total_ms = t;
  *launches = (long long)g_kt.used;
  return WSI_OK;
}

size_t wsi_stokes_size(const wsi_ctx* c) { return c ? c->nstk : 0; }
size_t wsi_velocity_size(const wsi_ctx* c) { return c ? c->nvel : 0; }
const char* wsi_last_error(const wsi_ctx* c) { return c ? c->err.c_str() : "null context"; }

int wsi_create_grid(const wsi_grid_desc* d, void* stream, wsi_ctx** out) {
  if (!d || !out) return WSI_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->nx < 2 || d->ny < 2 || d->nz < 1 || !(d->lx > 0) || !(d->ly > 0) || !(d->lz > 0)) return WSI_ERR_INVALID_ARG;
  for (int i = 0; i < 6; ++i)
    if (d->bc[i] != WSI_NO_SLIP && d->bc[i] != WSI_FREE_SLIP) return WSI_ERR_INVALID_ARG;
  if (d->nz == 1 && (d->bc[4] != WSI_FREE_SLIP || d->bc[5] != WSI_FREE_SLIP)) return WSI_ERR_INVALID_ARG;
  if (d->precision != WSI_PREC_FP64 && d->precision != WSI_PREC_MIXED) return WSI_ERR_INVALID_ARG;
  if (d->reinit_iters < 0) return WSI_ERR_INVALID_ARG;
  if (d->transport_form != WSI_FORM_CONSISTENT && d->transport_form != WSI_FORM_NONCONSERVATIVE)
    return WSI_ERR_INVALID_ARG;
  if (d->mg_smoother != WSI_SMOOTH_RBGS && d->mg_smoother != WSI_SMOOTH_CHEBYSHEV) return WSI_ERR_INVALID_ARG;
  if (d->ls_limiter != WSI_LIMIT_CUI && d->ls_limiter != WSI_LIMIT_XSPPM7) return WSI_ERR_INVALID_ARG;
  if ((double)(d->nx + 1) * (d->ny + 1) * (d->nz + 1) >= 2147483648.0) return WSI_ERR_INVALID_ARG;
  if (d->open_top != 0 && d->open_top != 1) return WSI_ERR_INVALID_ARG;
  if (d->open_top && (d->bc[5] != WSI_NO_SLIP || d->nz < 2 || d->visc_mg > 0)) return WSI_ERR_INVALID_ARG;
  wsi_ctx* c = new wsi_ctx();
  c->desc = *d;
  c->st = (cudaStream_t)stream;
  c->g.n[0] = d->nx;
  c->g.n[1] = d->ny;
  c->g.n[2] = d->nz;
  c->g.h[0] = d->lx / d->nx;
  c->g.h[1] = d->ly / d->ny;
  c->g.h[2] = d->lz / d->nz;
  for (int i = 0; i < 6; ++i) c->g.bc[i] = d->bc[i];
  c->g.open_top = d->open_top;
  grid_finalize(c->g);
  c->pk = packing(c->g);
  c->nvel = c->pk.off[3];
  c->nstk = c->pk.off[4];
  c->ncell = fsize(c->g, 3);
  c->m = d->restart > 0 ? std::min(d->restart, 60) : 20;
  c->opts.mg_pre = d->mg_pre > 0 ? d->mg_pre : 2;
  c->opts.mg_post = d->mg_post > 0 ? d->mg_post : 2;
  c->opts.mg_cycles = d->mg_cycles > 0 ? d->mg_cycles : 1;
  c->opts.visc_sweeps = d->visc_sweeps > 0 ? d->visc_sweeps : 2;
  c->opts.visc_mg = d->visc_mg > 0 ? d->visc_mg : 0;
  c->opts.mg_smoother = d->mg_smoother;
  c->opts.theta = d->theta;
  const GridDev& g = c->g;
  bool ok = true;
  auto A = [&](size_t n) {
    double* p = dalloc(c, n);
    ok &= p != nullptr;
    return p;
  };
  c->rho_cc = A(c->ncell);
  c->mu_cc = A(c->ncell);
  c->mu_cc_n = A(c->ncell);
  c->rho_cc_tmp = A(c->ncell);
  for (int k = 0; k < 3; ++k) {
    c->rho_face[k] = A(fsize(g, k));
    c->beta[k] = A(fsize(g, k));
    c->rho_flow[k] = A(fsize(g, k));
    c->rho_n[k] = A(fsize(g, k));
    c->beta_n[k] = A(fsize(g, k));
    c->rho_flow_n[k] = A(fsize(g, k));
    c->mu_e[k] = A(esize(g, k));
    c->mu_e_n[k] = A(esize(g, k));
  }
  c->vel = A(c->nvel);
  c->vel_old = A(c->nvel);
  c->p = A(c->ncell);
  c->phi = A(c->ncell);
  c->psi = A(c->ncell);
  c->vel_k = A(c->nvel);
  c->vel_half = A(c->nvel);
  c->u1 = A(c->nvel);
  c->u2 = A(c->nvel);
  c->rs1 = A(c->nvel);
  c->rs2 = A(c->nvel);
  c->R = A(c->nvel);
  c->Cc = A(c->nvel);
  c->phi_k = A(c->ncell);
  c->phi_new = A(c->ncell);
  c->phi_half = A(c->ncell);
  c->psi_k = A(c->ncell);
  c->psi_new = A(c->ncell);
  c->b = A(c->nstk);
  c->x = A(c->nstk);
  c->V = A(c->nstk * (size_t)(c->m + 1));
  c->Z = A(c->nstk * (size_t)c->m);
  c->hdev = A(4 * (c->m + 2) + 8);
  c->b0 = A(c->nvel);
  c->inv_mu = A(c->ncell);
  if (d->precision == WSI_PREC_MIXED) {
    // float32 shadows: half-size double allocations reinterpreted
    auto F = [&](size_t n) { return (float*)A((n + 1) / 2); };
    c->vn32 = F(c->nvel);
    c->u1_32 = F(c->nvel);
    c->u2_32 = F(c->nvel);
    c->rn32 = F(c->nvel);
    c->r1_32 = F(c->nvel);
    c->r2_32 = F(c->nvel);
    c->R32 = F(c->nvel);
    c->C32 = F(c->nvel);
    c->vh32 = F(c->nvel);
    c->phih32 = F(c->ncell);
    c->mu_cc_n32 = F(c->ncell);
    for (int e = 0; e < 3; ++e) c->mu_e_n32[e] = F(esize(g, e));
    // double-float operands: one float2 per element, the size of a double
    df_operands_shape(g, c->df);
    for (int a = 0; a < DF_NARR; ++a) c->df.a[a] = (float2*)A(df_operand_elems(c->df, a));
    c->df_err = (int*)A(1);
    if (ok) {
      cudaMemsetAsync(c->df_err, 0, sizeof(int), c->st);
      if (df_operands_encode(c->df) != WSI_OK) {
        c->err = "tile-copy descriptors of the matvec operands could not be encoded";
        wsi_destroy(c);
        return WSI_ERR_CUDA;
      }
    }
  }
  c->red = A(8192);
  if (!ok) {
    c->err = "out of device memory";
    wsi_destroy(c);
    return WSI_ERR_OOM;
  }
  if (cuda_check(c, "create")) {
    wsi_destroy(c);
    return WSI_ERR_CUDA;
  }
  *out = c;
  return WSI_OK;
}

void wsi_destroy(wsi_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  precond_free<double>(c->P64);
  precond_free<float>(c->P32);
  df_operands_release(c->df);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

int wsi_set_phases(wsi_ctx* c, const double* phi, const double* psi, const wsi_phase_props* pr,
                   const wsi_body_desc* bodies, int n_bodies) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!pr) return fail(c, WSI_ERR_INVALID_ARG, "null phase properties");
  const double vals[6] = {pr->rho_l, pr->rho_g, pr->rho_s, pr->mu_l, pr->mu_g, pr->mu_s};
  for (double v : vals)
    if (!(v > 0.0) || !std::isfinite(v)) return fail(c, WSI_ERR_INVALID_ARG, "material constants must be positive");
  if (n_bodies < 0 || n_bodies > 1) return fail(c, WSI_ERR_INVALID_ARG, "at most one body per context");
  c->props = *pr;
  int rc = copy_in(c, c->phi, phi, c->ncell);
  if (!rc) rc = copy_in(c, c->psi, psi, c->ncell);
  if (rc) return rc;
  // bodies
  Body& B = c->body;
  c->has_body = n_bodies == 1 && bodies[0].n_markers > 0;
  if (c->has_body) {
    const wsi_body_desc& bd = bodies[0];
    if (!bd.X || !(bd.dV > 0.0)) return fail(c, WSI_ERR_INVALID_ARG, "body needs markers and dV > 0");
    // host-side range check of the markers
    std::vector<double> hx((size_t)bd.n_markers * 3);
    cudaMemcpyAsync(hx.data(), bd.X, hx.size() * sizeof(double), cudaMemcpyDefault, c->st);
    cudaStreamSynchronize(c->st);
    const double L[3] = {c->desc.lx, c->desc.ly, c->desc.lz};
    for (size_t t = 0; t < hx.size(); ++t)
      if (!(hx[t] >= 0.0 && hx[t] <= L[t % 3])) return fail(c, WSI_ERR_INVALID_ARG, "marker outside the box");
    if (bd.n_markers != B.n) {
      size_t n3 = (size_t)bd.n_markers * 3;
      B.X = dalloc(c, n3);
      B.Xn = dalloc(c, n3);
      B.Xh = dalloc(c, n3);
      B.Ub = dalloc(c, n3);
      B.Ub_n = dalloc(c, n3);
      B.U = dalloc(c, n3);
      B.F = dalloc(c, n3);
      B.xc = dalloc(c, 4);
      B.rig = dalloc(c, 8);
      B.flag = (int*)dalloc(c, 1);
      B.sums = dalloc(c, 16);
      B.scratch = dalloc(c, 152 * 16 + 32);
      if (!B.X || !B.scratch) return fail(c, WSI_ERR_OOM, "out of device memory for markers");
    }
    B.n = bd.n_markers;
    B.dV = bd.dV;
    for (int d = 0; d < 6; ++d) B.lock[d] = bd.lock[d];
    for (int d = 0; d < 3; ++d) {
      B.U_pres[d] = bd.U_pres[d];
      B.W_pres[d] = bd.W_pres[d];
      B.half[d] = bd.half[d];
    }
    if (bd.shape < 0 || bd.shape > 2) return fail(c, WSI_ERR_INVALID_ARG, "unknown body shape");
    B.shape = bd.shape;
    cudaMemcpyAsync(B.X, hx.data(), hx.size() * sizeof(double), cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(B.Ub_n, 0, hx.size() * sizeof(double), c->st);
  }
  PhaseConst pc = phase_const(c);
  launch_materials(c->g, pc, c->phi, c->psi, c->rho_cc, c->mu_cc, c->rho_face, c->beta, c->rho_flow, c->mu_e, c->st);
  cudaMemsetAsync(c->vel, 0, c->nvel * sizeof(double), c->st);
  cudaMemsetAsync(c->vel_old, 0, c->nvel * sizeof(double), c->st);
  cudaMemsetAsync(c->p, 0, c->ncell * sizeof(double), c->st);
  c->have_phases = true;
  c->phi_cur = c->phi;
  c->psi_static_done = false;
  c->mat_n_valid = false;
  c->pc_dirty = true;
  return cuda_check(c, "set_phases");
}

int wsi_stokes_solve(wsi_ctx* c, const double* rhs, double* x, double dt, const wsi_solve_opts* o,
                     wsi_solve_stats* s) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "wsi_set_phases must come first");
  if (!o || !s || !(dt > 0.0) || !(o->rtol > 0.0) || o->max_iters < 1) return fail(c, WSI_ERR_INVALID_ARG, "bad options");
  auto t0 = std::chrono::steady_clock::now();
  int rc = copy_in(c, c->b, rhs, c->nstk);
  if (rc) return rc;
  if (o->use_x0) {
    rc = copy_in(c, c->x, x, c->nstk);
    if (rc) return rc;
  }
  // wall-face entries of the right-hand side are not equations
  double* bq[3];
  vel_parts(c, c->b, bq);
  launch_zero_walls(c->g, bq, c->st);
  if (o->use_x0) {
    double* xq[3];
    vel_parts(c, c->x, xq);
    launch_zero_walls(c->g, xq, c->st);
  }
  rc = fgmres(c, c->b, c->x, dt, o, s);
  if (rc != WSI_OK && rc != WSI_ERR_NOT_CONVERGED) return rc;
  int rc2 = copy_out(c, x, c->x, c->nstk);
  if (rc2) return rc2;
  int rc3 = cuda_check(c, "stokes_solve");
  if (rc3) return rc3;
  s->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

int wsi_dlm_constrain(wsi_ctx* c, double* vel, wsi_body_state* out) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->has_body) return fail(c, WSI_ERR_INVALID_ARG, "no body set");
  int rc = copy_in(c, c->vel_k, vel, c->nvel);
  if (rc) return rc;
  rc = dlm_project(c, c->vel_k, c->body.X);
  if (rc) return rc;
  rc = copy_out(c, vel, c->vel_k, c->nvel);
  if (rc) return rc;
  if (out) {
    for (int d = 0; d < 3; ++d) {
      out->U_r[d] = c->body.U_r[d];
      out->W_r[d] = c->body.W_r[d];
      out->X_com[d] = c->body.X_com[d];
    }
  }
  return cuda_check(c, "dlm_constrain");
}

int wsi_step(wsi_ctx* c, double dt, const wsi_solve_opts* o, wsi_step_stats* s) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "wsi_set_phases must come first");
  if (!o || !(dt > 0.0)) return fail(c, WSI_ERR_INVALID_ARG, "bad options");
  auto t0 = std::chrono::steady_clock::now();
  const GridDev& g = c->g;
  cudaStream_t st = c->st;
  PhaseConst pc = phase_const(c);
  Body& B = c->body;
  const size_t nv = c->nvel, nc = c->ncell;
  // time-n coefficients: face density rho^n and mu^n from (phi^n, psi^n).
  // After a step, the viscosity of its last cycle is already mu^n.
  if (c->mat_n_valid) {
    std::swap(c->mu_cc, c->mu_cc_n);
    for (int e = 0; e < 3; ++e) std::swap(c->mu_e[e], c->mu_e_n[e]);
    launch_face_density(g, pc, c->phi, c->psi, c->rho_n, st);
  } else {
    launch_materials(g, pc, c->phi, c->psi, c->rho_cc_tmp, c->mu_cc_n, c->rho_n, c->beta_n, c->rho_flow_n, c->mu_e_n,
                     st);
  }
  c->mat_n_valid = false;
  if (c->inlet) launch_inlet_data(g, c->wave, c->time + dt, c->in_gn, c->in_gw_np1, st);
  // the velocity iterate u^{n+1,k} lives in the velocity part of the solve's
  // packed vector, so that the solves start from it and leave their result
  // in place (no copies between the cycles)
  double* const vk = c->x;
  cudaMemcpyAsync(vk, c->vel, nv * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->phi_k, c->phi, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->psi_k, c->psi, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (c->has_body) cudaMemcpyAsync(B.Xn, B.X, (size_t)B.n * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->x + c->pk.off[3], c->p, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  const int ncyc = 2;
  for (int k = 0; k < ncyc; ++k) {
    // 1. level sets and viscosity at (n+1, k+1)
    levelset_stage(c, vk, c->vel, c->phi_k, c->phi, dt, c->phi_new);
    const double* psi_use = c->psi_k;
    const bool at_rest = B.lock[0] && B.lock[1] && B.lock[2] && B.lock[3] && B.lock[4] && B.lock[5] &&
                         B.U_pres[0] == 0.0 && B.U_pres[1] == 0.0 && B.U_pres[2] == 0.0 && B.W_pres[0] == 0.0 &&
                         B.W_pres[1] == 0.0 && B.W_pres[2] == 0.0;
    if (c->has_body && (B.shape == 1 || B.shape == 2) && !(at_rest && c->psi_static_done)) {
      launch_marker_mean(B.X, B.n, B.xc, B.scratch, st);
      if (B.shape == 1)
        launch_box_sdf(g, B.xc, B.half, c->psi_new, st);
      else
        launch_cyl_sdf(g, B.xc, B.half[0], B.half[1], c->psi_new, st);
      psi_use = c->psi_new;
      if (at_rest && k + 1 == ncyc) c->psi_static_done = true;
    }
    c->phi_cur = c->phi_new;
    launch_materials(g, pc, c->phi_new, psi_use, c->rho_cc, c->mu_cc, c->rho_face, c->beta, c->rho_flow, c->mu_e,
                     st);
    // 2. SSP-RK3 face density and consistent convection; right-hand side.
    //    Non-conservative form (Sec. 4.2.3): the level sets' face density
    //    rho^{n+1,k+1} stays in the operator, N from the half-step velocity.
    const bool nonconservative = c->desc.transport_form == WSI_FORM_NONCONSERVATIVE;
    if (nonconservative) {
      int rn = nc_convection(c, k);
      if (rn) return rn;
      if (k == 0) {
        if (c->mixed()) launch_lincomb_to_f32(nv, 1.0, c->vel, 0.0, nullptr, 0.0, nullptr, c->vn32, st);
        rhs_base(c, 0.0);
      }
    } else {
      transport_stage(c, k, dt, c->vel, c->vel_old, vk, k > 0);
      if (k == 0) rhs_base(c, 1.0 / dt);
    }
    const double* rg[3];
    for (int d = 0; d < 3; ++d) rg[d] = c->props.gravity_mode == WSI_GRAVITY_FLOW ? c->rho_flow[d] : c->rho_face[d];
    if (nonconservative) {
      const double* rf[3] = {c->rho_face[0], c->rho_face[1], c->rho_face[2]};
      if (c->mixed())
        launch_rhs_nc<float>(g, c->b0, c->C32, rf, c->vel, 1.0 / dt, rg, c->desc.gravity, c->b, st);
      else
        launch_rhs_nc<double>(g, c->b0, c->Cc, rf, c->vel, 1.0 / dt, rg, c->desc.gravity, c->b, st);
    } else if (c->mixed()) {
      launch_rhs_cycle<float>(g, c->b0, c->C32, rg, c->desc.gravity, c->b, st);
    } else {
      launch_rhs_cycle<double>(g, c->b0, c->Cc, rg, c->desc.gravity, c->b, st);
    }
    cudaMemsetAsync(c->b + c->pk.off[3], 0, nc * sizeof(double), st);
    // the inlet's data at t^{n+1} lifted into b; the solve is for the
    // velocity with zero x- faces, which then take the data
    if (c->inlet)
      launch_inlet_lift(g, c->mu_cc, c->mu_e[0], c->mu_e[1], c->mu_e_n[1], c->in_gn, c->in_gw_np1, c->in_gw_n,
                        c->desc.theta, c->b, st);
    // 3. Stokes solve from (u^{n+1,k}, p^{n+1/2,k}), in place
    if (c->inlet) {
      double* xq[3];
      parts(c, c->x, xq);
      launch_zero_walls(g, xq, st);
    }
    c->pc_dirty = true;
    wsi_solve_stats ss;
    wsi_solve_opts so = *o;
    so.use_x0 = 1;
    int rc = fgmres(c, c->b, c->x, dt, &so, &ss);
    if (rc != WSI_OK && rc != WSI_ERR_NOT_CONVERGED) return rc;
    if (c->inlet) launch_inlet_set(g, c->in_gn, c->x + c->pk.off[0], st);
    if (s && k < 4) {
      s->iters[k] = ss.iters;
      s->rel_residual[k] = ss.rel_residual;
    }
    // 4. rigidity projection at X^{n+1/2,k}, then positions
    if (c->has_body) {
      launch_lincomb((size_t)B.n * 3, 0.5, B.X, 0.5, B.Xn, 0.0, nullptr, B.Xh, st);
      rc = dlm_project(c, vk, B.Xh);
      if (rc) return rc;
      launch_marker_update(g, B.Xn, B.Ub, B.Ub_n, B.n, dt, B.X, B.flag, st);
    }
    cudaMemcpyAsync(c->phi_k, c->phi_new, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->psi_k, psi_use, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  // wave generation / damping zones relax u^{n+1} and phi^{n+1} (Sec. 7.1)
  if (c->has_waves) {
    double* vq[3];
    parts(c, vk, vq);
    launch_wave_relax(g, c->wave, c->time + dt, vq, c->phi_k, st);
  }
  // phi^{n+1} brought back to a signed distance (Sec. 4.1)
  if (c->desc.reinit_iters > 0) {
    int rr = reinit_phi(c, c->phi_k, c->desc.reinit_iters);
    if (rr) return rr;
  }
  c->time += dt;
  if (c->inlet) {  // the tangential data move on with the velocities
    std::swap(c->in_gw_nm1, c->in_gw_n);
    std::swap(c->in_gw_n, c->in_gw_np1);
  }
  // commit the step: u^n becomes u^{n-1} by exchanging the two buffers
  std::swap(c->vel_old, c->vel);
  cudaMemcpyAsync(c->vel, vk, nv * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->p, c->x + c->pk.off[3], nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->phi, c->phi_k, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->psi, c->psi_k, nc * sizeof(double), cudaMemcpyDeviceToDevice, st);
  // Lagrange-multiplier force (Sec. 8): F = sum_l rho_s [(U_b^{n+1} - U_b^n)
  // - (U_b^{n+1} - J u~)] dV / dt with the last cycle's J u~ (B.U); the two
  // U_b^{n+1} sums cancel, so one reduction of J u~ - U_b^n is taken (B.F is
  // free once the last spreading has run)
  double fsum[3] = {0.0, 0.0, 0.0};
  if (c->has_body) {
    launch_lincomb((size_t)B.n * 3, 1.0, B.U, -1.0, B.Ub_n, 0.0, nullptr, B.F, st);
    launch_rigid_sums(B.X, B.F, B.n, nullptr, B.sums, B.scratch, st);
    cudaMemcpyAsync(fsum, B.sums, sizeof(fsum), cudaMemcpyDeviceToHost, st);
  }
  if (c->has_body) cudaMemcpyAsync(B.Ub_n, B.Ub, (size_t)B.n * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  int hflag = 0;
  if (c->has_body && B.flag) cudaMemcpyAsync(&hflag, B.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  int rc = cuda_check(c, "step");
  if (rc) return rc;
  if (hflag) {
    cudaMemsetAsync(B.flag, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return fail(c, WSI_ERR_DEVICE, "a marker left the box or is not finite (device bound check of the marker update)");
  }
  // the last cycle's viscosity is mu(phi^{n+1}) unless the zones relaxed phi
  c->mat_n_valid = !c->has_waves && c->desc.reinit_iters == 0;
  if (s) {
    s->umax = host_maxabs(c->vel, nv, c->red, st);
    const double f = c->has_body ? c->props.rho_s * B.dV / dt : 0.0;
    for (int d = 0; d < 3; ++d) s->F_lm[d] = f * fsum[d];
    int rs = cuda_check(c, "step stats");
    if (rs) return rs;
    s->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return WSI_OK;
}

int wsi_get_field(wsi_ctx* c, int which, double* dst) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  int rc;
  switch (which) {
    case WSI_F_VEL: rc = copy_out(c, dst, c->vel, c->nvel); break;
    case WSI_F_VEL_OLD: rc = copy_out(c, dst, c->vel_old, c->nvel); break;
    case WSI_F_P: rc = copy_out(c, dst, c->p, c->ncell); break;
    case WSI_F_PHI: rc = copy_out(c, dst, c->phi, c->ncell); break;
    case WSI_F_PSI: rc = copy_out(c, dst, c->psi, c->ncell); break;
    case WSI_F_MARKERS:
      if (!c->has_body) return fail(c, WSI_ERR_INVALID_ARG, "no body");
      rc = copy_out(c, dst, c->body.X, (size_t)c->body.n * 3);
      break;
    default: return fail(c, WSI_ERR_INVALID_ARG, "unknown field");
  }
  if (rc) return rc;
  return cuda_check(c, "get_field");
}

int wsi_set_field(wsi_ctx* c, int which, const double* src) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  int rc;
  switch (which) {
    case WSI_F_VEL:
      rc = copy_in(c, c->vel, src, c->nvel);
      if (!rc) cudaMemcpyAsync(c->vel_old, c->vel, c->nvel * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      break;
    case WSI_F_VEL_OLD: rc = copy_in(c, c->vel_old, src, c->nvel); break;
    case WSI_F_P: rc = copy_in(c, c->p, src, c->ncell); break;
    case WSI_F_PHI:
      rc = copy_in(c, c->phi, src, c->ncell);
      c->mat_n_valid = false;
      break;
    case WSI_F_PSI:
      rc = copy_in(c, c->psi, src, c->ncell);
      c->psi_static_done = false;
      c->mat_n_valid = false;
      break;
    default: return fail(c, WSI_ERR_INVALID_ARG, "unknown field");
  }
  if (rc) return rc;
  return cuda_check(c, "set_field");
}

int wsi_get_coeff(wsi_ctx* c, int which, double* dst) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "no phases set");
  int rc = WSI_OK;
  switch (which) {
    case WSI_C_RHO_CC: rc = copy_out(c, dst, c->rho_cc, c->ncell); break;
    case WSI_C_MU_CC: rc = copy_out(c, dst, c->mu_cc, c->ncell); break;
    case WSI_C_RHO_FACE:
      for (int d = 0; d < 3 && !rc; ++d) rc = copy_out(c, dst + c->pk.off[d], c->rho_face[d], fsize(c->g, d));
      break;
    case WSI_C_RHO_FLOW_FACE:
      for (int d = 0; d < 3 && !rc; ++d) rc = copy_out(c, dst + c->pk.off[d], c->rho_flow[d], fsize(c->g, d));
      break;
    case WSI_C_MU_EDGE: {
      size_t o = 0;
      for (int e = 0; e < 3 && !rc; ++e) {
        rc = copy_out(c, dst + o, c->mu_e[e], esize(c->g, e));
        o += esize(c->g, e);
      }
      break;
    }
    default: return fail(c, WSI_ERR_INVALID_ARG, "unknown coefficient");
  }
  if (rc) return rc;
  return cuda_check(c, "get_coeff");
}

int wsi_apply(wsi_ctx* c, int op, const double* in, double* out, double dt) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "no phases set");
  if (!(dt > 0.0)) return fail(c, WSI_ERR_INVALID_ARG, "dt must be positive");
  Coef<double> cf = coef_now(c);
  double* xin = c->b;
  double* xout = c->x;
  size_t nin = 0, nout = 0;
  switch (op) {
    case WSI_OP_STOKES: nin = c->nstk; nout = c->nstk; break;
    case WSI_OP_VISCOUS:
    case WSI_OP_STRAIN: nin = c->nvel; nout = c->nvel; break;
    case WSI_OP_PRESSURE: nin = c->ncell; nout = c->ncell; break;
    case WSI_OP_GRAD: nin = c->ncell; nout = c->nvel; break;
    case WSI_OP_DIV: nin = c->nvel; nout = c->ncell; break;
    default: return fail(c, WSI_ERR_INVALID_ARG, "unknown operator");
  }
  int rc = copy_in(c, xin, in, nin);
  if (rc) return rc;
  const double* qi[3];
  double* qo[3];
  vel_parts(c, (const double*)xin, qi);
  vel_parts(c, xout, qo);
  switch (op) {
    case WSI_OP_STOKES:
      df_coef_refresh(c, cf, 1.0 / dt);
      stokes_mv(c, cf, 1.0 / dt, c->desc.theta, xin, xout, c->st);
      break;
    case WSI_OP_VISCOUS: launch_viscous<double>(c->g, cf, 1.0 / dt, c->desc.theta, qi, qo, c->st, false); break;
    case WSI_OP_STRAIN: launch_viscous<double>(c->g, cf, 1.0 / dt, c->desc.theta, qi, qo, c->st, true); break;
    case WSI_OP_PRESSURE: {
      const double* bt[3] = {c->beta[0], c->beta[1], c->beta[2]};
      launch_pressure<double>(c->g, bt, xin, xout, c->st);
      break;
    }
    case WSI_OP_GRAD: launch_grad<double>(c->g, xin, qo, c->st); break;
    case WSI_OP_DIV: launch_div<double>(c->g, qi, xout, 1.0, c->st); break;
  }
  rc = copy_out(c, out, xout, nout);
  if (rc) return rc;
  rc = cuda_check(c, "apply");
  if (rc == WSI_OK && op == WSI_OP_STOKES) rc = df_check(c);
  return rc;
}

int wsi_transport(wsi_ctx* c, const double* u_n, const double* u_nm1, const double* u_k, int k, double dt,
                  double* rho_out, double* C_out) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "no phases set");
  size_t nv = c->nvel;
  // u_n -> vel_half, u^{n-1} -> u1 scratch copy, u_k -> vel_k
  int rc = copy_in(c, c->vel_half, u_n, nv);
  if (!rc) rc = copy_in(c, c->rs2, u_nm1, nv);
  if (!rc && k > 0) rc = copy_in(c, c->vel_k, u_k, nv);
  if (rc) return rc;
  PhaseConst pc = phase_const(c);
  launch_materials(c->g, pc, c->phi, c->psi, c->rho_cc_tmp, c->mu_cc_n, c->rho_n, c->beta_n, c->rho_flow_n,
                   c->mu_e_n, c->st);
  // the stage buffers of the plain path alias rs2 only after u^(1), u^(2)
  // are formed, so copy u^{n-1} aside first
  cudaMemcpyAsync(c->vel_old, c->rs2, nv * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  transport_stage(c, k, dt, c->vel_half, c->vel_old, c->vel_k, false);
  c->mat_n_valid = false;  // the operator coefficients now hold the transported density
  c->pc_dirty = true;
  double* rq[3];
  parts(c, c->b, rq);
  for (int d = 0; d < 3; ++d)
    cudaMemcpyAsync(rq[d], c->rho_face[d], fsize(c->g, d) * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  if (c->mixed())
    launch_lincomb_mix(nv, 0.0, c->Cc, 1.0, c->C32, 0.0, c->C32, c->x, c->st);
  else
    cudaMemcpyAsync(c->x, c->Cc, nv * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  rc = copy_out(c, rho_out, c->b, nv);
  if (!rc) rc = copy_out(c, C_out, c->x, nv);
  if (rc) return rc;
  return cuda_check(c, "transport");
}

int wsi_set_waves(wsi_ctx* c, const wsi_wave_desc* w) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!w) {
    c->has_waves = false;
    return WSI_OK;
  }
  const double L[3] = {c->desc.lx, c->desc.ly, c->desc.lz};
  if (!(w->H > 0.0) || !(w->T > 0.0) || !(w->depth > 0.0) || w->vertical < 1 || w->vertical > 2 ||
      !(w->inlet ? w->x_gen >= 0.0 : w->x_gen > 0.0) || !(w->x_damp > w->x_gen) || !(w->x_damp < c->desc.lx) ||
      !(w->depth < L[w->vertical]) || (w->inlet != 0 && w->inlet != 1))
    return fail(c, WSI_ERR_INVALID_ARG, "bad wave description");
  if (w->inlet && (w->vertical != 2 || c->desc.bc[0] != WSI_NO_SLIP))
    return fail(c, WSI_ERR_INVALID_ARG, "the inlet needs vertical = 2 and a no-slip x- side");
  const double* gv = c->desc.gravity;
  double gmag = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
  if (!(gmag > 0.0)) return fail(c, WSI_ERR_INVALID_ARG, "waves need gravity");
  PhaseConst pc = phase_const(c);
  c->wave = wave_setup(w->H, w->T, w->depth, w->x_gen, w->x_damp, c->desc.lx, w->vertical, pc.eps, gmag);
  c->has_waves = true;
  c->time = w->t0;
  c->inlet = w->inlet != 0;
  if (c->inlet) {
    const size_t ne = (size_t)(c->g.n[2] + 1) * c->g.n[1];
    if (!c->in_gn) {
      c->in_gn = dalloc(c, (size_t)c->g.n[2] * c->g.n[1]);
      c->in_gw_nm1 = dalloc(c, ne);
      c->in_gw_n = dalloc(c, ne);
      c->in_gw_np1 = dalloc(c, ne);
      c->in_gs = dalloc(c, ne);
      c->in_gs32 = (float*)dalloc(c, (ne + 1) / 2);
      if (!c->in_gn || !c->in_gw_nm1 || !c->in_gw_n || !c->in_gw_np1 || !c->in_gs || !c->in_gs32)
        return fail(c, WSI_ERR_OOM, "inlet data");
    }
    // the state's x- faces take the data at t0, for u^n and u^{n-1} alike
    launch_inlet_data(c->g, c->wave, c->time, c->in_gn, c->in_gw_n, c->st);
    cudaMemcpyAsync(c->in_gw_nm1, c->in_gw_n, ne * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    launch_inlet_set(c->g, c->in_gn, c->vel, c->st);
    launch_inlet_set(c->g, c->in_gn, c->vel_old, c->st);
  }
  return cuda_check(c, "set_waves");
}

int wsi_wave_relax(wsi_ctx* c, double t, double* vel, double* phi) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->has_waves) return fail(c, WSI_ERR_INVALID_ARG, "wsi_set_waves must come first");
  int rc = copy_in(c, c->vel_half, vel, c->nvel);
  if (!rc && phi) rc = copy_in(c, c->phi_half, phi, c->ncell);
  if (rc) return rc;
  double* vq[3];
  parts(c, c->vel_half, vq);
  launch_wave_relax(c->g, c->wave, t, vq, phi ? c->phi_half : nullptr, c->st);
  rc = copy_out(c, vel, c->vel_half, c->nvel);
  if (!rc && phi) rc = copy_out(c, phi, c->phi_half, c->ncell);
  if (rc) return rc;
  return cuda_check(c, "wave_relax");
}

int wsi_advect_levelset(wsi_ctx* c, const double* vel, const double* phi_n, const double* phi_half, double dt,
                        double* phi_out) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  // phi_half = (phi_k + phi_n)/2 with phi_k = 2 phi_half - phi_n; likewise the
  // velocity is passed as u_half = (u_half + u_half)/2
  // (scratch buffers only: the stored level sets are left untouched)
  int rc = copy_in(c, c->vel_k, vel, c->nvel);
  if (!rc) rc = copy_in(c, c->psi_new, phi_n, c->ncell);
  if (!rc) rc = copy_in(c, c->phi_half, phi_half, c->ncell);
  if (rc) return rc;
  launch_lincomb(c->ncell, 2.0, c->phi_half, -1.0, c->psi_new, 0.0, nullptr, c->phi_k, c->st);
  levelset_stage(c, c->vel_k, c->vel_k, c->phi_k, c->psi_new, dt, c->phi_new);
  rc = copy_out(c, phi_out, c->phi_new, c->ncell);
  if (rc) return rc;
  return cuda_check(c, "advect_levelset");
}

int wsi_reinit(wsi_ctx* c, double* phi, int iters) {
  if (valid_ctx(c) || !phi || iters < 0) return WSI_ERR_INVALID_ARG;
  int rc = copy_in(c, c->phi_new, phi, c->ncell);
  if (!rc) rc = reinit_phi(c, c->phi_new, iters);
  if (!rc) rc = copy_out(c, phi, c->phi_new, c->ncell);
  if (rc) return rc;
  return cuda_check(c, "reinit");
}

int wsi_interp(wsi_ctx* c, const double* vel, const double* X, int n, double* U) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (n <= 0) return WSI_OK;
  double* dX = dalloc(c, (size_t)n * 3);
  double* dU = dalloc(c, (size_t)n * 3);
  if (!dX || !dU) return fail(c, WSI_ERR_OOM, "out of device memory");
  int rc = copy_in(c, c->vel_half, vel, c->nvel);
  if (!rc) rc = copy_in(c, dX, X, (size_t)n * 3);
  if (rc) return rc;
  const double* vh[3];
  vel_parts(c, (const double*)c->vel_half, vh);
  launch_ib_interp(c->g, vh, dX, n, dU, c->st);
  rc = copy_out(c, U, dU, (size_t)n * 3);
  cudaStreamSynchronize(c->st);
  // release the temporaries (last two allocations)
  cudaFree(dX);
  cudaFree(dU);
  c->allocs.resize(c->allocs.size() - 2);
  if (rc) return rc;
  return cuda_check(c, "interp");
}

int wsi_spread(wsi_ctx* c, const double* F, const double* X, int n, double dV, double* vel) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  // the work arrays first: the two staging buffers below must stay the last
  // two allocations (they are released at the end)
  if (!ensure_spread_work(c)) return fail(c, WSI_ERR_OOM, "out of device memory for spreading");
  double* dX = dalloc(c, (size_t)std::max(n, 1) * 3);
  double* dF = dalloc(c, (size_t)std::max(n, 1) * 3);
  if (!dX || !dF) return fail(c, WSI_ERR_OOM, "out of device memory");
  int rc = WSI_OK;
  if (n > 0) {
    rc = copy_in(c, dX, X, (size_t)n * 3);
    if (!rc) rc = copy_in(c, dF, F, (size_t)n * 3);
  }
  if (!rc) {
    cudaMemsetAsync(c->vel_half, 0, c->nvel * sizeof(double), c->st);
    double* vq[3];
    vel_parts(c, c->vel_half, vq);
    double mm[6];
    launch_marker_box(dX, n, c->mbox, c->sw.part, c->st);
    cudaMemcpyAsync(mm, c->mbox, sizeof(mm), cudaMemcpyDeviceToHost, c->st);
    cudaStreamSynchronize(c->st);
    launch_ib_spread(c->g, dF, dX, n, dV, vq, c->sw, spread_box(c->g, mm), c->st);
    rc = copy_out(c, vel, c->vel_half, c->nvel);
  }
  cudaStreamSynchronize(c->st);
  cudaFree(dX);
  cudaFree(dF);
  c->allocs.resize(c->allocs.size() - 2);
  if (rc) return rc;
  return cuda_check(c, "spread");
}

// ------------------------------------------------------------------ learned correction
// ------------------------------------------------------------ checkpoint
namespace {
const char kCkptMagic[8] = {'W', 'S', 'I', 'C', 'K', 'P', 'T', '1'};

struct CkptHeader {
  char magic[8];
  int nx, ny, nz, precision, n_markers, psi_static_done;
  double time;
  double U_r[3], W_r[3], X_com[3];
  int inlet, pad;  // 1: the inlet's tangential data of u^n and u^{n-1} follow the state
};

bool write_dev(FILE* f, const double* d, size_t n, std::vector<double>& h) {
  h.resize(n);
  if (n && cudaMemcpy(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  return fwrite(h.data(), sizeof(double), n, f) == n;
}
bool read_dev(FILE* f, double* d, size_t n, std::vector<double>& h) {
  h.resize(n);
  if (fread(h.data(), sizeof(double), n, f) != n) return false;
  return !n || cudaMemcpy(d, h.data(), n * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
}
}  // namespace

int wsi_checkpoint(wsi_ctx* c, const char* path) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases || !path) return fail(c, WSI_ERR_INVALID_ARG, "checkpoint needs phases and a path");
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail(c, WSI_ERR_CUDA, "checkpoint: stream error");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, WSI_ERR_INVALID_ARG, "checkpoint: cannot open file");
  CkptHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kCkptMagic, 8);
  hd.nx = c->g.n[0];
  hd.ny = c->g.n[1];
  hd.nz = c->g.n[2];
  hd.precision = c->desc.precision;
  hd.n_markers = c->has_body ? c->body.n : 0;
  hd.psi_static_done = c->psi_static_done ? 1 : 0;
  hd.time = c->time;
  hd.inlet = c->inlet ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    hd.U_r[a] = c->body.U_r[a];
    hd.W_r[a] = c->body.W_r[a];
    hd.X_com[a] = c->body.X_com[a];
  }
  std::vector<double> h;
  bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1;
  ok = ok && write_dev(f, c->vel, c->nvel, h) && write_dev(f, c->vel_old, c->nvel, h) &&
       write_dev(f, c->p, c->ncell, h) && write_dev(f, c->phi, c->ncell, h) && write_dev(f, c->psi, c->ncell, h);
  const size_t ne = (size_t)(c->g.n[2] + 1) * c->g.n[1];
  if (ok && c->inlet) ok = write_dev(f, c->in_gw_n, ne, h) && write_dev(f, c->in_gw_nm1, ne, h);
  if (ok && c->has_body) {
    const size_t nm = (size_t)c->body.n * 3;
    ok = write_dev(f, c->body.X, nm, h) && write_dev(f, c->body.Ub_n, nm, h) && write_dev(f, c->body.xc, 3, h);
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? WSI_OK : fail(c, WSI_ERR_CUDA, "checkpoint: write failed");
}

int wsi_restore(wsi_ctx* c, const char* path) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases || !path) return fail(c, WSI_ERR_INVALID_ARG, "restore needs phases and a path");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, WSI_ERR_INVALID_ARG, "restore: cannot open file");
  CkptHeader hd;
  if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kCkptMagic, 8) != 0) {
    fclose(f);
    return fail(c, WSI_ERR_INVALID_ARG, "restore: not a checkpoint");
  }
  if (hd.nx != c->g.n[0] || hd.ny != c->g.n[1] || hd.nz != c->g.n[2] || hd.precision != c->desc.precision ||
      hd.n_markers != (c->has_body ? c->body.n : 0) || hd.inlet != (c->inlet ? 1 : 0)) {
    fclose(f);
    return fail(c, WSI_ERR_INVALID_ARG, "restore: grid, precision, marker count or inlet differ");
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) {
    fclose(f);
    return fail(c, WSI_ERR_CUDA, "restore: stream error");
  }
  std::vector<double> h;
  bool ok = read_dev(f, c->vel, c->nvel, h) && read_dev(f, c->vel_old, c->nvel, h) && read_dev(f, c->p, c->ncell, h) &&
            read_dev(f, c->phi, c->ncell, h) && read_dev(f, c->psi, c->ncell, h);
  const size_t ne = (size_t)(c->g.n[2] + 1) * c->g.n[1];
  if (ok && c->inlet) ok = read_dev(f, c->in_gw_n, ne, h) && read_dev(f, c->in_gw_nm1, ne, h);
  if (ok && c->has_body) {
    const size_t nm = (size_t)c->body.n * 3;
    ok = read_dev(f, c->body.X, nm, h) && read_dev(f, c->body.Ub_n, nm, h) && read_dev(f, c->body.xc, 3, h);
  }
  fclose(f);
  if (!ok) return fail(c, WSI_ERR_INVALID_ARG, "restore: truncated file");
  c->time = hd.time;
  c->psi_static_done = hd.psi_static_done != 0;
  for (int a = 0; a < 3; ++a) {
    c->body.U_r[a] = hd.U_r[a];
    c->body.W_r[a] = hd.W_r[a];
    c->body.X_com[a] = hd.X_com[a];
  }
  // operator coefficients follow from the restored level sets
  PhaseConst pc = phase_const(c);
  launch_materials(c->g, pc, c->phi, c->psi, c->rho_cc, c->mu_cc, c->rho_face, c->beta, c->rho_flow, c->mu_e, c->st);
  c->phi_cur = c->phi;
  c->mat_n_valid = false;
  c->pc_dirty = true;
  return cuda_check(c, "restore");
}

struct wsi_unet {
  UNetImpl* u = nullptr;
  float* x3 = nullptr;  // staging for [V][3] inputs
};

int wsi_unet_create(int nz, int ny, int nx, int c0, int c1, int c2, unsigned long long seed, wsi_unet** out) {
  if (!out) return WSI_ERR_INVALID_ARG;
  *out = nullptr;
  UNetImpl* u = unet_create(nz, ny, nx, c0, c1, c2);
  if (!u) return WSI_ERR_INVALID_ARG;
  wsi_unet* n = new wsi_unet();
  n->u = u;
  size_t V = (size_t)nz * ny * nx;
  if (cudaMalloc(&n->x3, V * 3 * sizeof(float)) != cudaSuccess) {
    unet_destroy(u);
    delete n;
    return WSI_ERR_OOM;
  }
  // He-normal initialisation from the seed (host), zero biases
  std::vector<float> p(unet_nparam(u), 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.0f, 1.0f);
  const int spec[10][3] = {{c0, 3, 16}, {c0, c0, c0}, {c1, c0, c0}, {c1, c1, c1}, {c2, c1, c1},
                           {c2, c2, c2}, {c1, c2 + c1, c2 + c1}, {c1, c1, c1}, {c0, c1 + c0, c1 + c0}, {c0, c0, c0}};
  size_t off = 0;
  for (int l = 0; l < 10; ++l) {
    int co = spec[l][0], ci_real = spec[l][1], ci = spec[l][2];
    float sd = sqrtf(2.0f / (27.0f * ci_real));
    for (int tap = 0; tap < 27; ++tap)
      for (int o = 0; o < co; ++o)
        for (int ci_ = 0; ci_ < ci; ++ci_) p[off + ((size_t)tap * co + o) * ci + ci_] = ci_ < ci_real ? sd * nd(rng) : 0.f;
    off += (size_t)27 * co * ci + co;
  }
  for (int cc = 0; cc < c0; ++cc) p[off + cc] = sqrtf(2.0f / c0) * nd(rng);
  cudaMemcpy(unet_params(u), p.data(), p.size() * sizeof(float), cudaMemcpyHostToDevice);
  unet_pack(u, 0);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    wsi_unet_destroy(n);
    return WSI_ERR_CUDA;
  }
  *out = n;
  return WSI_OK;
}

void wsi_unet_destroy(wsi_unet* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  unet_destroy(n->u);
  cudaFree(n->x3);
  delete n;
}

size_t wsi_unet_num_params(const wsi_unet* n) { return n ? unet_nparam(n->u) : 0; }

int wsi_unet_set_params(wsi_unet* n, const float* p) {
  if (!n || !p) return WSI_ERR_INVALID_ARG;
  if (cudaMemcpy(unet_params(n->u), p, unet_nparam(n->u) * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
    return WSI_ERR_CUDA;
  unet_pack(n->u, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? WSI_OK : WSI_ERR_CUDA;
}

int wsi_unet_get_params(wsi_unet* n, float* p) {
  if (!n || !p) return WSI_ERR_INVALID_ARG;
  return cudaMemcpy(p, unet_params(n->u), unet_nparam(n->u) * sizeof(float), cudaMemcpyDefault) == cudaSuccess
             ? WSI_OK
             : WSI_ERR_CUDA;
}

int wsi_unet_get_grads(wsi_unet* n, float* g) {
  if (!n || !g) return WSI_ERR_INVALID_ARG;
  return cudaMemcpy(g, unet_grads(n->u), unet_nparam(n->u) * sizeof(float), cudaMemcpyDefault) == cudaSuccess
             ? WSI_OK
             : WSI_ERR_CUDA;
}

int wsi_unet_forward(wsi_unet* n, const float* x, float* out) {
  if (!n || !x || !out) return WSI_ERR_INVALID_ARG;
  size_t V = (size_t)unet_dim(n->u, 0) * unet_dim(n->u, 1) * unet_dim(n->u, 2);
  if (cudaMemcpy(n->x3, x, V * 3 * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return WSI_ERR_CUDA;
  unet_set_input3(n->u, n->x3, 0);
  unet_forward(n->u, 0);
  if (cudaMemcpy(out, unet_output(n->u), V * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return WSI_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return WSI_ERR_CUDA;
  return unet_take_error(n->u) ? WSI_ERR_DEVICE : WSI_OK;
}

int wsi_unet_backward(wsi_unet* n, const float* target, double* loss) {
  if (!n || !target) return WSI_ERR_INVALID_ARG;
  size_t V = (size_t)unet_dim(n->u, 0) * unet_dim(n->u, 1) * unet_dim(n->u, 2);
  if (cudaMemcpy(unet_target(n->u), target, V * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return WSI_ERR_CUDA;
  unet_backward(n->u, 0);
  if (loss && cudaMemcpy(loss, unet_loss(n->u), sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return WSI_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return WSI_ERR_CUDA;
  return unet_take_error(n->u) ? WSI_ERR_DEVICE : WSI_OK;
}

int wsi_unet_adam(wsi_unet* n, double lr) {
  if (!n || !(lr >= 0.0)) return WSI_ERR_INVALID_ARG;
  unet_adam(n->u, lr, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? WSI_OK : WSI_ERR_CUDA;
}

namespace {
const char kNetMagic[8] = {'W', 'S', 'I', 'U', 'N', 'E', 'T', '1'};
struct NetHeader {
  char magic[8];
  int c0, c1, c2, step;
  unsigned long long nparam;
};
}  // namespace

int wsi_unet_save(wsi_unet* n, const char* path) {
  if (!n || !path) return WSI_ERR_INVALID_ARG;
  const size_t np = unet_nparam(n->u);
  std::vector<float> h(np * 3);
  if (cudaDeviceSynchronize() != cudaSuccess) return WSI_ERR_CUDA;
  const float* src[3] = {unet_params(n->u), unet_moment(n->u, 0), unet_moment(n->u, 1)};
  for (int a = 0; a < 3; ++a)
    if (cudaMemcpy(h.data() + a * np, src[a], np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      return WSI_ERR_CUDA;
  NetHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kNetMagic, 8);
  hd.c0 = unet_width(n->u, 0);
  hd.c1 = unet_width(n->u, 1);
  hd.c2 = unet_width(n->u, 2);
  hd.step = *unet_step_count(n->u);
  hd.nparam = np;
  FILE* f = fopen(path, "wb");
  if (!f) return WSI_ERR_INVALID_ARG;
  bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? WSI_OK : WSI_ERR_CUDA;
}

int wsi_unet_load(wsi_unet* n, const char* path) {
  if (!n || !path) return WSI_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return WSI_ERR_INVALID_ARG;
  NetHeader hd;
  const size_t np = unet_nparam(n->u);
  if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kNetMagic, 8) != 0 || hd.nparam != np ||
      hd.c0 != unet_width(n->u, 0) || hd.c1 != unet_width(n->u, 1) || hd.c2 != unet_width(n->u, 2)) {
    fclose(f);
    return WSI_ERR_INVALID_ARG;
  }
  std::vector<float> h(np * 3);
  const bool ok = fread(h.data(), sizeof(float), h.size(), f) == h.size();
  fclose(f);
  if (!ok) return WSI_ERR_INVALID_ARG;
  float* dst[3] = {unet_params(n->u), unet_moment(n->u, 0), unet_moment(n->u, 1)};
  for (int a = 0; a < 3; ++a)
    if (cudaMemcpy(dst[a], h.data() + a * np, np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return WSI_ERR_CUDA;
  *unet_step_count(n->u) = hd.step;
  unet_pack(n->u, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? WSI_OK : WSI_ERR_CUDA;
}

int wsi_attach_unet(wsi_ctx* c, wsi_unet* n, int level, int enable) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->mixed()) return fail(c, WSI_ERR_INVALID_ARG, "the learned correction needs a WSI_PREC_MIXED context");
  c->unet = n;
  c->unet_impl = n ? n->u : nullptr;
  c->unet_level = level;
  if (enable < WSI_LEARN_OFF || enable > WSI_LEARN_AUGMENT) return fail(c, WSI_ERR_INVALID_ARG, "bad learned mode");
  c->unet_on = n && enable != WSI_LEARN_OFF;
  c->P32.learn.mode = enable == WSI_LEARN_AUGMENT ? WSI_LEARN_AUGMENT : WSI_LEARN_REPLACE;
  c->pc_dirty = true;
  return WSI_OK;
}

int wsi_attach_unet_guess(wsi_ctx* c, wsi_unet* n, int level) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->mixed()) return fail(c, WSI_ERR_INVALID_ARG, "the learned guess needs a WSI_PREC_MIXED context");
  c->gunet_impl = n ? n->u : nullptr;
  c->gunet_level = level;
  c->pc_dirty = true;
  return WSI_OK;
}

int wsi_unet_train_guess(wsi_ctx* c, const double* y, const double* x, double lr, double* loss) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->gunet_impl || !c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "attach a guess network and set phases first");
  int rc = ensure_pc(c);
  if (rc) return rc;
  Precond<float>& P = c->P32;
  const size_t n = c->ncell;
  // float64 staging in the Krylov work space, then float32 on the level-0 grid
  double* ys = c->V;
  double* xs = c->V + n;
  rc = copy_in(c, ys, y, n);
  if (!rc) rc = copy_in(c, xs, x, n);
  if (rc) return rc;
  launch_lincomb_to_f32(n, 1.0, ys, 0.0, nullptr, 0.0, nullptr, P.lev[0].b, c->st);
  launch_lincomb_to_f32(n, 1.0, xs, 0.0, nullptr, 0.0, nullptr, P.lev[0].x, c->st);
  learned_train_guess(P, P.lev[0].b, P.lev[0].x, lr, c->st);
  if (loss) cudaMemcpyAsync(loss, learned_guess_loss(P), sizeof(double), cudaMemcpyDeviceToHost, c->st);
  return cuda_check(c, "unet_train_guess");
}

int wsi_unet_train_sample(wsi_ctx* c, const double* e, double lr, double* loss) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->unet || !c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "attach a network and set phases first");
  int rc = ensure_pc(c);
  if (rc) return rc;
  Precond<float>& P = c->P32;
  size_t n = fsize(P.lev[c->unet_level].g, 3);
  // the level's residual buffer of level 0 (fine) serves as float64 staging
  double* stage = c->V;
  rc = copy_in(c, stage, e, n);
  if (rc) return rc;
  float* e32 = P.learn.e;
  launch_lincomb_to_f32(n, 1.0, stage, 0.0, nullptr, 0.0, nullptr, e32, c->st);
  learned_train(P, c->opts, e32, lr, c->st);
  if (loss) cudaMemcpyAsync(loss, learned_loss(P), sizeof(double), cudaMemcpyDeviceToHost, c->st);
  return cuda_check(c, "unet_train_sample");
}

int wsi_pressure_solve(wsi_ctx* c, const double* y, double* x, double rtol, int max_cycles, wsi_solve_stats* s) {
  if (valid_ctx(c)) return WSI_ERR_INVALID_ARG;
  if (!c->have_phases) return fail(c, WSI_ERR_INVALID_ARG, "wsi_set_phases must come first");
  if (!(rtol > 0.0) || max_cycles < 1 || !s) return fail(c, WSI_ERR_INVALID_ARG, "bad options");
  s->learned_rejected = -1;
  s->guess = -1;
  auto t0 = std::chrono::steady_clock::now();
  int rc = ensure_pc(c);
  if (rc) return rc;
  const GridDev& g = c->g;
  cudaStream_t st = c->st;
  const size_t n = c->ncell;
  double* yv = c->b + c->pk.off[3];
  double* xv = c->x + c->pk.off[3];
  double* r = c->V;  // scratch
  // constants are in the null space of a closed box's pressure operator
  auto demean = [&](double* a) {
    if (g.open_top) return;
    launch_sum<double>(a, n, c->hdev, c->red, st);
    launch_add_scalar_from<double>(a, n, c->hdev, -1.0 / (double)n, st);
  };
  rc = copy_in(c, yv, y, n);
  if (rc) return rc;
  demean(yv);
  cudaMemsetAsync(xv, 0, n * sizeof(double), st);
  const double ynorm = host_norm2(yv, n, c->red, st);
  const double* bt[3] = {c->beta[0], c->beta[1], c->beta[2]};
  if (c->mixed() && c->gunet_impl && ynorm > 0.0) {
    // learned initial guess: the guess network's coarse solution of the
    // restricted right-hand side, prolongated; kept only if its residual is
    // below that of the zero guess
    MGLevel<float>& L0 = c->P32.lev[0];
    launch_lincomb_to_f32(n, 1.0 / ynorm, yv, 0.0, nullptr, 0.0, nullptr, L0.b, st);
    learned_guess(c->P32, L0.b, st);
    launch_lincomb_mix(n, 0.0, xv, ynorm, L0.x, 0.0, L0.x, xv, st);
    demean(xv);
    launch_pressure<double>(g, bt, xv, r, st);
    launch_lincomb(n, 1.0, yv, -1.0, r, 0.0, nullptr, r, st);
    const double r0 = host_norm2(r, n, c->red, st);
    s->guess = (std::isfinite(r0) && r0 < ynorm) ? 1 : 0;
    if (!s->guess) cudaMemsetAsync(xv, 0, n * sizeof(double), st);
  }
  // The plain V-cycle judges the network: the first two cycles are plain and
  // the second one's residual reduction is the bar; a learned cycle that
  // reduces the residual less is undone and the solve continues plain.
  const int plain_cycles = 2;
  bool learned = c->mixed() && c->unet_on;
  bool last_learned = false;
  double* xb = c->Z;  // iterate before a learned cycle
  double rn = ynorm, prev = ynorm, rho_plain = 1.0;
  int cycles = 0;
  while (true) {
    launch_pressure<double>(g, bt, xv, r, st);
    launch_lincomb(n, 1.0, yv, -1.0, r, 0.0, nullptr, r, st);
    demean(r);
    rn = host_norm2(r, n, c->red, st);
    if (!std::isfinite(rn) && !last_learned) return fail(c, WSI_ERR_NAN, "non-finite pressure residual");
    if (last_learned && !(rn <= rho_plain * prev)) {
      cudaMemcpyAsync(xv, xb, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
      learned = last_learned = false;
      s->learned_rejected = cycles;
      continue;  // residual of the restored iterate
    }
    if (cycles == plain_cycles && prev > 0.0) rho_plain = rn / prev;
    if (rn <= rtol * ynorm || cycles >= max_cycles || ynorm == 0.0) break;
    prev = rn;
    const bool use = learned && cycles >= plain_cycles;
    c->P32.learn.on = use;
    if (use) cudaMemcpyAsync(xb, xv, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (c->mixed()) {
      MGLevel<float>& L0 = c->P32.lev[0];
      launch_lincomb_to_f32(n, 1.0 / rn, r, 0.0, nullptr, 0.0, nullptr, L0.b, st);
      cudaMemsetAsync(L0.x, 0, n * sizeof(float), st);
      precond_vcycle<float>(c->P32, c->opts, st);
      launch_lincomb_mix(n, 1.0, xv, rn, L0.x, 0.0, L0.x, xv, st);
    } else {
      MGLevel<double>& L0 = c->P64.lev[0];
      cudaMemcpyAsync(L0.b, r, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
      cudaMemsetAsync(L0.x, 0, n * sizeof(double), st);
      precond_vcycle<double>(c->P64, c->opts, st);
      launch_lincomb(n, 1.0, xv, 1.0, L0.x, 0.0, nullptr, xv, st);
    }
    last_learned = use;
    ++cycles;
  }
  c->P32.learn.on = c->unet_on;
  demean(xv);
  rc = copy_out(c, x, xv, n);
  if (rc) return rc;
  rc = cuda_check(c, "pressure_solve");
  if (rc) return rc;
  s->iters = cycles;
  s->rel_residual = ynorm > 0.0 ? rn / ynorm : 0.0;
  s->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rn <= rtol * ynorm ? WSI_OK : WSI_ERR_NOT_CONVERGED;
}

}  // extern "C"
