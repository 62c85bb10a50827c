// The learned pressure correction inside the float32 multigrid, its training
// on data the solver generates, and the standalone pressure solve used to
// measure it.  No counterpart in the paper (it extends the pressure solve).
//
// Network input at multigrid level l (3 channels, bf16): log(rho)/7 and the
// level set, both averaged down the hierarchy from the fine cells, and the
// level's right-hand side (or residual) r divided by its RMS s.  Output o
// (float32).  The correction is e = s o / d with d the diagonal of the
// level's operator (sum of beta/h^2 over the cell's faces), so that o = r/s
// reproduces one Jacobi step and the network learns the rest.  Training
// pairs are exact by construction: a seeded smooth field e and r = L_l e;
// the loss is the residual the correction leaves, the quantity the plain
// cycle judges it by.
#include <math.h>

#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;
static inline dim3 grid3(int nx, int ny, int nz) { return dim3(cdiv(nx, BX), cdiv(ny, BY), nz); }
static int nb(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8)); }

// coarse cell = mean of its children (ratios r0, r1, r2)
template <typename Ts>
__global__ void k_avg_down(GridDev gf, GridDev gc, int r0, int r1, int r2, const Ts* __restrict__ f, float* c,
                           int take_log) {
  int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (I >= gc.n[0] || J >= gc.n[1]) return;
  float s = 0.f;
  for (int a = 0; a < r2; ++a)
    for (int b = 0; b < r1; ++b)
      for (int q = 0; q < r0; ++q) {
        float v = (float)f[fidx(gf, 3, I * r0 + q, J * r1 + b, K * r2 + a)];
        s += take_log ? logf(v) : v;
      }
  c[fidx(gc, 3, I, J, K)] = s / (float)(r0 * r1 * r2);
}

// d = sum over interior faces of beta/h^2 (the diagonal of the level operator)
__global__ void k_diag(GridDev g, const float* __restrict__ bx, const float* __restrict__ by,
                       const float* __restrict__ bz, float* d) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  float s = 0.f;
  if (i + 1 < g.n[0]) s += bx[fidx(g, 0, i + 1, j, k)] * g.ih2f[0];
  if (i > 0) s += bx[fidx(g, 0, i, j, k)] * g.ih2f[0];
  if (j + 1 < g.n[1]) s += by[fidx(g, 1, i, j + 1, k)] * g.ih2f[1];
  if (j > 0) s += by[fidx(g, 1, i, j, k)] * g.ih2f[1];
  if (k + 1 < g.n[2]) s += bz[fidx(g, 2, i, j, k + 1)] * g.ih2f[2];
  else if (g.open_top) s += 2.f * bz[fidx(g, 2, i, j, k + 1)] * g.ih2f[2];  // ghost -p above the open top
  if (k > 0) s += bz[fidx(g, 2, i, j, k)] * g.ih2f[2];
  d[fidx(g, 3, i, j, k)] = s > 0.f ? s : 1.f;
}

__global__ void k_sumsq(const float* __restrict__ r, size_t n, double* out) {
  double s = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    s += (double)r[t] * (double)r[t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// x[v] = (lrho/7, phi, r/s, 0...) as bf16 with 16 channels
__global__ void k_assemble(const float* __restrict__ lrho, const float* __restrict__ phi, const float* __restrict__ r,
                           const double* __restrict__ ss, size_t n, __nv_bfloat16* x) {
  float inv = (float)(1.0 / sqrt(fmax(ss[0] / (double)n, 1e-300)));
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    __nv_bfloat16* p = x + v * 16;
    p[0] = __float2bfloat16(lrho[v] * (1.0f / 7.0f));
    p[1] = __float2bfloat16(fminf(fmaxf(phi[v] * 10.0f, -4.0f), 4.0f));
    p[2] = __float2bfloat16(r[v] * inv);
    for (int c = 3; c < 16; ++c) p[c] = __float2bfloat16(0.f);
  }
}

// error of the network's correction: t1 = s o / d - (e - x)   (x null: 0)
__global__ void k_corr_error(const float* __restrict__ o, const float* __restrict__ e, const float* __restrict__ x,
                             const float* __restrict__ d, const double* __restrict__ ss, size_t n, float* t1) {
  const float s = (float)sqrt(fmax(ss[0] / (double)n, 1e-300));
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    t1[v] = o[v] * s / d[v] - (x ? e[v] - x[v] : e[v]);
}

// Gradient of the loss
//   J = 1/2 mean((L t1)^2) / s^2 + lambda/2 mean((d t1)^2) / s^2
// (residual left by the correction, in units of the input's RMS s, plus a
// small error term) with respect to the network output o (t1 = s o/d - e):
//   dJ/do = (L L t1 / (s d) + lambda d t1 / s) / n,
// handed to the network's backward pass as the target tgt = o - n dJ/do
// (its output gradient is (o - tgt) / n).  t3 = L L t1 (L symmetric).
__global__ void k_resid_target(const float* __restrict__ o, const float* __restrict__ t1, const float* __restrict__ t3,
                               const float* __restrict__ d, const double* __restrict__ ss, size_t n, float lambda,
                               float* tgt) {
  const float s = (float)sqrt(fmax(ss[0] / (double)n, 1e-300));
  const float is = 1.0f / s;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    tgt[v] = o[v] - (t3[v] * is / d[v] + lambda * d[v] * t1[v] * is);
}

// loss = 1/2 mean(t2^2)/s^2 + lambda/2 mean((d t1)^2)/s^2, one block
__global__ void k_resid_loss(const float* __restrict__ t1, const float* __restrict__ t2, const float* __restrict__ d,
                             size_t n, float lambda, double* ss) {
  __shared__ double sh[32];
  double a = 0.0;
  for (size_t v = threadIdx.x; v < n; v += blockDim.x) {
    const double r = t2[v], q = (double)d[v] * t1[v];
    a += r * r + lambda * q * q;
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    ss[1] = 0.5 * t / (double)n / fmax(ss[0] / (double)n, 1e-300);
  }
}

// x = s o / d, or x += s o / d
__global__ void k_apply_out(const float* __restrict__ o, const float* __restrict__ d, const double* __restrict__ ss,
                            size_t n, int add, float* x) {
  float s = (float)sqrt(fmax(ss[0] / (double)n, 0.0));
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    float e = o[v] * s / d[v];
    x[v] = add ? x[v] + e : e;
  }
}

// restricted network inputs and the level diagonal; needs the fine rho_cc and
// phi and a built hierarchy
int learned_setup(Precond<float>& P, const double* rho_cc, const double* phi, cudaStream_t st, std::string& err) {
  LearnState& S = P.learn;
  if (!S.net && !S.gnet) return WSI_OK;
  const int top = std::max(S.net ? S.level : 0, S.gnet ? S.glevel : 0);
  if (top < 1 || top >= (int)P.lev.size()) {
    err = "learned correction level outside the multigrid hierarchy";
    return WSI_ERR_INVALID_ARG;
  }
  auto fits = [&](UNetImpl* net, int l) {
    const GridDev& gg = P.lev[l].g;
    return gg.n[0] == unet_dim(net, 2) && gg.n[1] == unet_dim(net, 1) && gg.n[2] == unet_dim(net, 0);
  };
  if ((S.net && !fits(S.net, S.level)) || (S.gnet && !fits(S.gnet, S.glevel))) {
    err = "network dimensions differ from the multigrid level";
    return WSI_ERR_INVALID_ARG;
  }
  // average log(rho) and phi down to the deepest level a network uses
  const GridDev& g0 = P.lev[0].g;
  for (int l = 1; l <= top; ++l) {
    const MGLevel<float>& F = P.lev[l - 1];
    const GridDev& gc = P.lev[l].g;
    dim3 gr = grid3(gc.n[0], gc.n[1], gc.n[2]);
    if (l == 1) {
      { k_avg_down<double><<<gr, dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1], F.r[2], rho_cc, S.lrho[l], 1); WSI_COUNT(); }
      { k_avg_down<double><<<gr, dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1], F.r[2], phi, S.phi[l], 0); WSI_COUNT(); }
    } else {
      { k_avg_down<float><<<gr, dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1], F.r[2], S.lrho[l - 1], S.lrho[l], 0); WSI_COUNT(); }
      { k_avg_down<float><<<gr, dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1], F.r[2], S.phi[l - 1], S.phi[l], 0); WSI_COUNT(); }
    }
  }
  (void)g0;
  if (S.net) {
    const MGLevel<float>& Lc = P.lev[S.level];
    { k_diag<<<grid3(Lc.g.n[0], Lc.g.n[1], Lc.g.n[2]), dim3(BX, BY), 0, st>>>(Lc.g, Lc.beta[0], Lc.beta[1],
                                                                              Lc.beta[2], S.diag); WSI_COUNT(); }
  }
  if (S.gnet) {
    const MGLevel<float>& Lg = P.lev[S.glevel];
    { k_diag<<<grid3(Lg.g.n[0], Lg.g.n[1], Lg.g.n[2]), dim3(BX, BY), 0, st>>>(Lg.g, Lg.beta[0], Lg.beta[1],
                                                                              Lg.beta[2], S.gdiag); WSI_COUNT(); }
  }
  S.ready = true;
  return WSI_OK;
}

// fine field f (level 0) averaged down to level top, into buf[l] (l >= 1)
static void avg_chain(Precond<float>& P, const float* f, int top, float* const* buf, cudaStream_t st) {
  const float* src = f;
  for (int l = 1; l <= top; ++l) {
    const MGLevel<float>& F = P.lev[l - 1];
    const GridDev& gc = P.lev[l].g;
    { k_avg_down<float><<<grid3(gc.n[0], gc.n[1], gc.n[2]), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1], F.r[2],
                                                                                  src, buf[l], 0); WSI_COUNT(); }
    src = buf[l];
  }
}

// The solution of L x = r exceeds the Jacobi estimate r / d by up to the
// ratio of the diagonal to the lowest eigenvalue, about (n_max / pi)^2 on a
// level with n_max cells along its longest axis; the guess network's output
// is taken in those units (x = G s o / d), so that its targets are O(1).
static float guess_gain(const GridDev& g) {
  const double nm = std::max(g.n[0], std::max(g.n[1], g.n[2]));
  return (float)(nm * nm / (M_PI * M_PI));
}

// x = G s o / d
__global__ void k_apply_guess(const float* __restrict__ o, const float* __restrict__ d,
                              const double* __restrict__ ss, size_t n, float gain, float* x) {
  const float s = (float)sqrt(fmax(ss[0] / (double)n, 0.0)) * gain;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    x[v] = o[v] * s / d[v];
}

void learned_guess(Precond<float>& P, const float* b0, cudaStream_t st) {
  LearnState& S = P.learn;
  const int lg = S.glevel;
  std::vector<float*> bb(P.lev.size());
  for (size_t l = 0; l < P.lev.size(); ++l) bb[l] = P.lev[l].b;
  avg_chain(P, b0, lg, bb.data(), st);  // the right-hand side of x = 0 restricts to its average
  MGLevel<float>& L = P.lev[lg];
  const size_t n = fsize(L.g, 3);
  cudaMemsetAsync(S.gss, 0, sizeof(double), st);
  { k_sumsq<<<nb(n), 256, 0, st>>>(L.b, n, S.gss); WSI_COUNT(); }
  { k_assemble<<<nb(n), 256, 0, st>>>(S.lrho[lg], S.phi[lg], L.b, S.gss, n, unet_input(S.gnet)); WSI_COUNT(); }
  unet_forward(S.gnet, st);
  { k_apply_guess<<<nb(n), 256, 0, st>>>(unet_output(S.gnet), S.gdiag, S.gss, n, guess_gain(L.g), L.x); WSI_COUNT(); }
  precond_prolong_chain<float>(P, lg, st);
}

// target d x / (G s) of the guess network (its output o gives x = G s o / d)
__global__ void k_guess_target(const float* __restrict__ x, const float* __restrict__ d,
                               const double* __restrict__ ss, size_t n, float gain, float* tgt) {
  const float is = (float)(1.0 / sqrt(fmax(ss[0] / (double)n, 1e-300))) / gain;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    tgt[v] = d[v] * x[v] * is;
}

void learned_train_guess(Precond<float>& P, const float* y, const float* x, double lr, cudaStream_t st) {
  LearnState& S = P.learn;
  const int lg = S.glevel;
  std::vector<float*> bb(P.lev.size()), xx(P.lev.size());
  for (size_t l = 0; l < P.lev.size(); ++l) {
    bb[l] = P.lev[l].b;
    xx[l] = P.lev[l].res;
  }
  avg_chain(P, y, lg, bb.data(), st);
  avg_chain(P, x, lg, xx.data(), st);
  MGLevel<float>& L = P.lev[lg];
  const size_t n = fsize(L.g, 3);
  cudaMemsetAsync(S.gss, 0, sizeof(double), st);
  { k_sumsq<<<nb(n), 256, 0, st>>>(L.b, n, S.gss); WSI_COUNT(); }
  { k_assemble<<<nb(n), 256, 0, st>>>(S.lrho[lg], S.phi[lg], L.b, S.gss, n, unet_input(S.gnet)); WSI_COUNT(); }
  unet_forward(S.gnet, st);
  { k_guess_target<<<nb(n), 256, 0, st>>>(L.res, S.gdiag, S.gss, n, guess_gain(L.g), unet_target(S.gnet)); WSI_COUNT(); }
  unet_backward(S.gnet, st);
  if (lr > 0.0) unet_adam(S.gnet, lr, st);
}

const double* learned_guess_loss(const Precond<float>& P) { return unet_loss(P.learn.gnet); }

// x_level = (or +=) network correction for rhs on level l
void learned_correction(Precond<float>& P, int l, const float* rhs, bool add, cudaStream_t st) {
  LearnState& S = P.learn;
  MGLevel<float>& L = P.lev[l];
  size_t n = fsize(L.g, 3);
  cudaMemsetAsync(S.ss, 0, sizeof(double), st);
  { k_sumsq<<<nb(n), 256, 0, st>>>(rhs, n, S.ss); WSI_COUNT(); }
  { k_assemble<<<nb(n), 256, 0, st>>>(S.lrho[l], S.phi[l], rhs, S.ss, n, unet_input(S.net)); WSI_COUNT(); }
  unet_forward(S.net, st);
  { k_apply_out<<<nb(n), 256, 0, st>>>(unet_output(S.net), S.diag, S.ss, n, add ? 1 : 0, L.x); WSI_COUNT(); }
}

// one training step on a seeded field e at the level.  Replacing mode: the
// network sees r = L e and corrects toward e.  Augmenting mode: the plain
// coarse-grid correction of r (pre-smoothing, coarser cycle, prolongation)
// gives x1; the network sees the residual r - L x1 and corrects toward the
// error e - x1 it leaves, exact because e is known.  The loss is the
// residual the correction leaves (what the plain cycle judges it by) plus a
// small error term; then backward and Adam.
void learned_train(Precond<float>& P, const Opts& o, const float* e, double lr, cudaStream_t st) {
  LearnState& S = P.learn;
  const int l = S.level;
  MGLevel<float>& L = P.lev[l];
  const size_t n = fsize(L.g, 3);
  const float lambda = 0.1f;
  const float* bt[3] = {L.beta[0], L.beta[1], L.beta[2]};
  launch_pressure<float>(L.g, bt, e, L.res, st);
  const float* x1 = nullptr;
  if (S.mode == WSI_LEARN_AUGMENT) {
    cudaMemcpyAsync(L.b, L.res, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(L.x, 0, n * sizeof(float), st);
    precond_coarse_part<float>(P, o, l, st);
    launch_pressure<float>(L.g, bt, L.x, L.res, st);
    launch_lincomb_f32(n, 1.f, L.b, -1.f, L.res, 0.f, nullptr, L.res, st);
    x1 = L.x;
  }
  cudaMemsetAsync(S.ss, 0, 2 * sizeof(double), st);
  { k_sumsq<<<nb(n), 256, 0, st>>>(L.res, n, S.ss); WSI_COUNT(); }
  { k_assemble<<<nb(n), 256, 0, st>>>(S.lrho[l], S.phi[l], L.res, S.ss, n, unet_input(S.net)); WSI_COUNT(); }
  unet_forward(S.net, st);
  const float* out = unet_output(S.net);
  { k_corr_error<<<nb(n), 256, 0, st>>>(out, e, x1, S.diag, S.ss, n, S.t1); WSI_COUNT(); }
  launch_pressure<float>(L.g, bt, S.t1, S.t2, st);
  launch_pressure<float>(L.g, bt, S.t2, S.t3, st);
  { k_resid_loss<<<1, 1024, 0, st>>>(S.t1, S.t2, S.diag, n, lambda, S.ss); WSI_COUNT(); }
  { k_resid_target<<<nb(n), 256, 0, st>>>(out, S.t1, S.t3, S.diag, S.ss, n, lambda, unet_target(S.net)); WSI_COUNT(); }
  unet_backward(S.net, st);
  if (lr > 0.0) unet_adam(S.net, lr, st);
}

const double* learned_loss(const Precond<float>& P) { return P.learn.ss + 1; }

}  // namespace wsi
