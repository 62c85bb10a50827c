// Projection preconditioner of the implicit Stokes system (Sec. 4.2.4; the
// paper cites the variable-coefficient projection method without printing
// it) with a cell-centred geometric multigrid for the pressure operator
// D(beta G).  Templated on the arithmetic type T: float64 for the plain
// path, float32 inside float64 FGMRES for the mixed path.
//
// One application  z = P^{-1} r  (r = (r_u, r_p)):
//   u~ = A^{-1} r_u      by red-black Gauss-Seidel sweeps on the viscous block
//   y  = r_p + D u~      (mean removed: closed box)
//   phi = L_beta^{-1} y   by V-cycles
//   p  = phi/dt - theta mu y,    u = u~ - beta G phi
// which is the block factorisation of K with the Schur complement
// D A^{-1} G approximated by dt D beta G plus the local-viscosity term.
//
// Multigrid: coarsening by 2 along every axis whose extent is even and >= 4,
// until <= 64 cells; coarse face beta = mean of the coplanar fine faces;
// restriction = mean of the 2^d children (fused with the residual);
// prolongation = (bi/tri)linear on cell centres (fused with the correction);
// smoother = red-black Gauss-Seidel; coarsest = dense float64 inverse of the
// operator regularised on its constant null space.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "internal.h"

namespace wsi {

static constexpr int BX = 32, BY = 8;
static inline dim3 grid3(int nx, int ny, int nz) { return dim3(cdiv(nx, BX), cdiv(ny, BY), nz); }

template <typename T>
static T* dalloc(std::vector<void*>& allocs, size_t n, std::string& err) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    err = "cudaMalloc failed in preconditioner";
    return nullptr;
  }
  allocs.push_back(p);
  return (T*)p;
}

template <typename T>
static int vlev_alloc(Precond<T>& P, std::string& err) {
  P.vlev.assign(P.lev.size(), VLevel<T>{});
  for (int c = 0; c < 3; ++c) {
    P.vres0[c] = dalloc<T>(P.allocs, fsize(P.lev[0].g, c), err);
    if (!P.vres0[c]) return WSI_ERR_OOM;
  }
  for (size_t l = 1; l < P.lev.size(); ++l) {
    const GridDev& g = P.lev[l].g;
    VLevel<T>& V = P.vlev[l];
    for (int c = 0; c < 3; ++c) {
      V.rho_face[c] = dalloc<T>(P.allocs, fsize(g, c), err);
      V.u[c] = dalloc<T>(P.allocs, fsize(g, c), err);
      V.b[c] = dalloc<T>(P.allocs, fsize(g, c), err);
      V.res[c] = dalloc<T>(P.allocs, fsize(g, c), err);
      V.mu_e[c] = dalloc<T>(P.allocs, esize(g, c), err);
      if (!V.rho_face[c] || !V.u[c] || !V.b[c] || !V.res[c] || !V.mu_e[c]) return WSI_ERR_OOM;
    }
    V.mu_cc = dalloc<T>(P.allocs, fsize(g, 3), err);
    if (!V.mu_cc) return WSI_ERR_OOM;
  }
  return WSI_OK;
}

template <typename T>
int precond_alloc(Precond<T>& P, const GridDev& g0, std::string& err) {
  precond_free(P);
  GridDev g = g0;
  for (;;) {
    MGLevel<T> L;
    L.g = g;
    for (int c = 0; c < 3; ++c) {
      L.beta[c] = dalloc<T>(P.allocs, fsize(g, c), err);
      if (!L.beta[c]) return WSI_ERR_OOM;
    }
    size_t nc = fsize(g, 3);
    L.x = dalloc<T>(P.allocs, nc, err);
    L.b = dalloc<T>(P.allocs, nc, err);
    L.res = dalloc<T>(P.allocs, nc, err);
    L.cd = dalloc<T>(P.allocs, nc, err);
    L.cx2 = dalloc<T>(P.allocs, nc, err);
    L.cd2 = dalloc<T>(P.allocs, nc, err);
    if (!L.x || !L.b || !L.res || !L.cd || !L.cx2 || !L.cd2) return WSI_ERR_OOM;
    // Semi-coarsening on anisotropic grids: an axis coarsens only while its
    // spacing is within 1.5x of the finest active spacing, so a grid with
    // hx = 2 hy = 2 hz first coarsens y and z and then all three (point
    // smoothers damp the weakly coupled direction poorly).
    double hmin = 1e300;
    for (int a = 0; a < 3; ++a)
      if (g.n[a] > 1) hmin = std::min(hmin, g.h[a]);
    bool any = false;
    for (int a = 0; a < 3; ++a) {
      L.r[a] = (g.n[a] % 2 == 0 && g.n[a] >= 4 && g.h[a] <= 1.5 * hmin) ? 2 : 1;
      any |= L.r[a] == 2;
    }
    if (!any && nc > 64) {
      // strongly anisotropic grids whose fine axes can no longer coarsen
      // (wave tanks with long cells): coarsen every axis that still can
      for (int a = 0; a < 3; ++a) {
        L.r[a] = (g.n[a] % 2 == 0 && g.n[a] >= 4) ? 2 : 1;
        any |= L.r[a] == 2;
      }
    }
    if (nc <= 64 || !any) {
      for (int a = 0; a < 3; ++a) L.r[a] = 1;
      P.lev.push_back(L);
      break;
    }
    P.lev.push_back(L);
    for (int a = 0; a < 3; ++a) {
      g.n[a] /= L.r[a];
      g.h[a] *= L.r[a];
    }
    grid_finalize(g);
  }
  P.ncoarse = (int)fsize(P.lev.back().g, 3);
  if (P.ncoarse > 1024) {
    err = "coarsest multigrid level too large (grid extents need more factors of 2)";
    return WSI_ERR_INVALID_ARG;
  }
  P.coarse_inv = dalloc<double>(P.allocs, (size_t)P.ncoarse * P.ncoarse, err);
  for (int c = 0; c < 3; ++c) {
    P.rho_face[c] = dalloc<T>(P.allocs, fsize(g0, c), err);
    P.ru[c] = dalloc<T>(P.allocs, fsize(g0, c), err);
    P.ut[c] = dalloc<T>(P.allocs, fsize(g0, c), err);
    P.gp[c] = dalloc<T>(P.allocs, fsize(g0, c), err);
  }
  P.mu_cc = dalloc<T>(P.allocs, fsize(g0, 3), err);
  for (int e = 0; e < 3; ++e) P.mu_e[e] = dalloc<T>(P.allocs, esize(g0, e), err);
  P.rp = dalloc<T>(P.allocs, fsize(g0, 3), err);
  P.y = dalloc<T>(P.allocs, fsize(g0, 3), err);
  P.dscratch = dalloc<double>(P.allocs, 4096, err);
  P.dsum = dalloc<double>(P.allocs, 8, err);
  if (!P.coarse_inv || !P.mu_cc || !P.rp || !P.y || !P.dscratch || !P.dsum) return WSI_ERR_OOM;
  return vlev_alloc(P, err);
}

template <typename T>
void precond_free(Precond<T>& P) {
  for (void* p : P.allocs) cudaFree(p);
  P.allocs.clear();
  P.lev.clear();
  P.built = false;
  P.learn.lrho.clear();
  P.learn.phi.clear();
  P.learn.diag = nullptr;
  P.learn.e = nullptr;
  P.learn.t1 = P.learn.t2 = P.learn.t3 = nullptr;
  P.learn.ss = nullptr;
  P.learn.ready = false;
}

// ------------------------------------------------------------ coefficients
template <int C, typename T>
__global__ void k_coarsen_beta(GridDev gf, GridDev gc, int r0, int r1, int r2, const T* __restrict__ bf, T* bc) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(gc, C, 0) || j >= ext(gc, C, 1)) return;
  int r[3] = {r0, r1, r2};
  int base[3] = {i * r[0], j * r[1], k * r[2]};
  int span[3] = {r[0], r[1], r[2]};
  span[C] = 1;  // the coplanar block only
  T s = T(0);
  for (int c = 0; c < span[2]; ++c)
    for (int b = 0; b < span[1]; ++b)
      for (int a = 0; a < span[0]; ++a) s += bf[fidx(gf, C, base[0] + a, base[1] + b, base[2] + c)];
  bc[fidx(gc, C, i, j, k)] = s / T(span[0] * span[1] * span[2]);
}

// coarse cell viscosity: mean of the children
template <typename T>
__global__ void k_vmu_down(GridDev gf, GridDev gc, int r0, int r1, int r2, const T* __restrict__ mf, T* mc) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= gc.n[0] || j >= gc.n[1]) return;
  T s = T(0);
  for (int c = 0; c < r2; ++c)
    for (int b = 0; b < r1; ++b)
      for (int a = 0; a < r0; ++a) s += mf[fidx(gf, 3, i * r0 + a, j * r1 + b, k * r2 + c)];
  mc[fidx(gc, 3, i, j, k)] = s / T(r0 * r1 * r2);
}

// coarse edge viscosity: harmonic mean of the four coarse cells around the
// edge (indices clamped at walls), the fine-grid rule on the coarse grid
template <int E, typename T>
__global__ void k_vedges(GridDev g, const T* __restrict__ mu, T* mu_e) {
  constexpr int A1 = (E == 2) ? 1 : 0;
  constexpr int A2 = (E == 0) ? 1 : 2;
  const int ex = g.n[0] + (A1 == 0 || A2 == 0), ey = g.n[1] + (A1 == 1 || A2 == 1);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ex || j >= ey) return;
  T s = T(0);
  for (int o1 = 0; o1 < 2; ++o1)
    for (int o2 = 0; o2 < 2; ++o2) {
      int c[3] = {i, j, k};
      c[A1] -= o1;
      c[A2] -= o2;
      for (int a = 0; a < 3; ++a) c[a] = clampi(c[a], 0, g.n[a] - 1);
      s += T(1) / mu[fidx(g, 3, c[0], c[1], c[2])];
    }
  mu_e[eidx(g, E, i, j, k)] = T(4) / s;
}

// Face restriction of component C: full weighting (1/4, 1/2, 1/4) across the
// coarse face along C where that axis coarsens, the mean of the children
// across it; wall faces of the coarse grid are not unknowns (0)
template <int C, typename T>
__global__ void k_vrestrict(GridDev gf, GridDev gc, int r0, int r1, int r2, const T* __restrict__ rf, T* bc) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(gc, C, 0) || j >= ext(gc, C, 1)) return;
  const int I3[3] = {i, j, k};
  const size_t id = fidx(gc, C, i, j, k);
  if (I3[C] == 0 || I3[C] == gc.n[C]) {
    bc[id] = T(0);
    return;
  }
  const int r[3] = {r0, r1, r2};
  int span[3] = {r0, r1, r2};
  span[C] = 1;
  T s = T(0);
  for (int c = 0; c < span[2]; ++c)
    for (int b = 0; b < span[1]; ++b)
      for (int a = 0; a < span[0]; ++a) {
        int f[3] = {i * r[0] + a, j * r[1] + b, k * r[2] + c};
        if (r[C] == 2) {
          f[C] = 2 * I3[C];
          T v = T(0.5) * rf[fidx(gf, C, f[0], f[1], f[2])];
          f[C] -= 1;
          v += T(0.25) * rf[fidx(gf, C, f[0], f[1], f[2])];
          f[C] += 2;
          v += T(0.25) * rf[fidx(gf, C, f[0], f[1], f[2])];
          s += v;
        } else {
          f[C] = I3[C];
          s += rf[fidx(gf, C, f[0], f[1], f[2])];
        }
      }
  bc[id] = s / T(span[0] * span[1] * span[2]);
}

// Face prolongation of component C, added to the fine iterate: linear along
// C where that axis coarsens (coincident faces take the coarse value, the
// faces between two coarse faces their mean), constant across it
template <int C, typename T>
__global__ void k_vprolong(GridDev gf, GridDev gc, int r0, int r1, int r2, const T* __restrict__ uc, T* uf) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(gf, C, 0) || j >= ext(gf, C, 1)) return;
  const int i3[3] = {i, j, k};
  if (i3[C] == 0 || i3[C] == gf.n[C]) return;
  const int r[3] = {r0, r1, r2};
  int I[3];
  for (int a = 0; a < 3; ++a) I[a] = a == C ? i3[a] : i3[a] / r[a];
  T v;
  if (r[C] == 2) {
    if ((i3[C] & 1) == 0) {
      I[C] = i3[C] / 2;
      v = uc[fidx(gc, C, I[0], I[1], I[2])];
    } else {
      I[C] = (i3[C] - 1) / 2;
      v = uc[fidx(gc, C, I[0], I[1], I[2])];
      I[C] += 1;
      v = T(0.5) * (v + uc[fidx(gc, C, I[0], I[1], I[2])]);
    }
  } else {
    v = uc[fidx(gc, C, I[0], I[1], I[2])];
  }
  uf[fidx(gf, C, i, j, k)] += v;
}

// up to sixteen arrays cast in one launch (blockIdx.y selects the array)
template <typename Ts, typename Td>
struct CastSet {
  const Ts* a[16];
  Td* b[16];
  size_t n[16];
  int count;
};

template <typename Ts, typename Td>
__global__ void k_cast_set(CastSet<Ts, Td> s) {
  const int q = blockIdx.y;
  if (q >= s.count) return;
  const Ts* __restrict__ a = s.a[q];
  Td* b = s.b[q];
  const size_t n = s.n[q];
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = cvt<Td, Ts>(a[t]);
}

template <typename Ts, typename Td>
static void cast_set(const CastSet<Ts, Td>& s, cudaStream_t st) {
  size_t nmax = 0;
  for (int q = 0; q < s.count; ++q) nmax = std::max(nmax, s.n[q]);
  if (!nmax) return;
  const int blocks = (int)std::min<size_t>((nmax + 255) / 256, 152 * 4);
  { k_cast_set<Ts, Td><<<dim3(blocks, s.count), 256, 0, st>>>(s); WSI_COUNT(); }
}

// Gauss-Jordan inverse (host, float64) of an SPD matrix, no pivoting needed
static void spd_inverse(std::vector<double>& A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int p = 0; p < n; ++p) {
    double d = A[(size_t)p * n + p];
    double id = 1.0 / d;
    for (int c = 0; c < n; ++c) {
      A[(size_t)p * n + c] *= id;
      I[(size_t)p * n + c] *= id;
    }
    for (int r = 0; r < n; ++r) {
      if (r == p) continue;
      double f = A[(size_t)r * n + p];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)r * n + c] -= f * A[(size_t)p * n + c];
        I[(size_t)r * n + c] -= f * I[(size_t)p * n + c];
      }
    }
  }
  A.swap(I);
}

template <typename T>
int precond_setup(Precond<T>& P, const GridDev& g, const Coef<double>& fine, cudaStream_t st, std::string& err) {
  // fine coefficients in T (one launch for the ten arrays)
  {
    CastSet<double, T> cs;
    cs.count = 0;
    auto add = [&](const double* a, T* b, size_t n) {
      cs.a[cs.count] = a;
      cs.b[cs.count] = b;
      cs.n[cs.count] = n;
      ++cs.count;
    };
    for (int c = 0; c < 3; ++c) {
      add(fine.rho_face[c], P.rho_face[c], fsize(g, c));
      add(fine.beta[c], P.lev[0].beta[c], fsize(g, c));
    }
    add(fine.mu_cc, P.mu_cc, fsize(g, 3));
    for (int e = 0; e < 3; ++e) add(fine.mu_e[e], P.mu_e[e], esize(g, e));
    cast_set(cs, st);
  }
  for (size_t l = 0; l + 1 < P.lev.size(); ++l) {
    MGLevel<T>& F = P.lev[l];
    MGLevel<T>& Cl = P.lev[l + 1];
    const GridDev& gc = Cl.g;
    { k_coarsen_beta<0, T><<<grid3(gc.n[0] + 1, gc.n[1], gc.n[2]), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1],
                                                                                        F.r[2], F.beta[0], Cl.beta[0]); WSI_COUNT(); }
    { k_coarsen_beta<1, T><<<grid3(gc.n[0], gc.n[1] + 1, gc.n[2]), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1],
                                                                                        F.r[2], F.beta[1], Cl.beta[1]); WSI_COUNT(); }
    { k_coarsen_beta<2, T><<<grid3(gc.n[0], gc.n[1], gc.n[2] + 1), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1],
                                                                                        F.r[2], F.beta[2], Cl.beta[2]); WSI_COUNT(); }
    // viscous coefficients: face density like beta (coplanar mean), cell
    // viscosity the mean of the children, edge viscosity harmonic again
    const T* rf[3] = {l == 0 ? P.rho_face[0] : P.vlev[l].rho_face[0], l == 0 ? P.rho_face[1] : P.vlev[l].rho_face[1],
                      l == 0 ? P.rho_face[2] : P.vlev[l].rho_face[2]};
    const T* mf = l == 0 ? P.mu_cc : P.vlev[l].mu_cc;
    VLevel<T>& VC = P.vlev[l + 1];
    { k_coarsen_beta<0, T><<<grid3(gc.n[0] + 1, gc.n[1], gc.n[2]), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1],
                                                                                        F.r[2], rf[0], VC.rho_face[0]); WSI_COUNT(); }
    { k_coarsen_beta<1, T><<<grid3(gc.n[0], gc.n[1] + 1, gc.n[2]), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1],
                                                                                        F.r[2], rf[1], VC.rho_face[1]); WSI_COUNT(); }
    { k_coarsen_beta<2, T><<<grid3(gc.n[0], gc.n[1], gc.n[2] + 1), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1],
                                                                                        F.r[2], rf[2], VC.rho_face[2]); WSI_COUNT(); }
    { k_vmu_down<T><<<grid3(gc.n[0], gc.n[1], gc.n[2]), dim3(BX, BY), 0, st>>>(F.g, gc, F.r[0], F.r[1], F.r[2], mf,
                                                                             VC.mu_cc); WSI_COUNT(); }
    { k_vedges<0, T><<<grid3(gc.n[0] + 1, gc.n[1] + 1, gc.n[2]), dim3(BX, BY), 0, st>>>(gc, VC.mu_cc, VC.mu_e[0]); WSI_COUNT(); }
    { k_vedges<1, T><<<grid3(gc.n[0] + 1, gc.n[1], gc.n[2] + 1), dim3(BX, BY), 0, st>>>(gc, VC.mu_cc, VC.mu_e[1]); WSI_COUNT(); }
    { k_vedges<2, T><<<grid3(gc.n[0], gc.n[1] + 1, gc.n[2] + 1), dim3(BX, BY), 0, st>>>(gc, VC.mu_cc, VC.mu_e[2]); WSI_COUNT(); }
  }
  // dense coarsest operator: M = -L + c 1 1^T (SPD), inverted in float64
  const MGLevel<T>& Lc = P.lev.back();
  const GridDev& gc = Lc.g;
  int n = P.ncoarse;
  std::vector<T> hb[3];
  for (int c = 0; c < 3; ++c) {
    hb[c].resize(fsize(gc, c));
    cudaMemcpyAsync(hb[c].data(), Lc.beta[c], fsize(gc, c) * sizeof(T), cudaMemcpyDeviceToHost, st);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    err = "CUDA error while building the coarse operator";
    return WSI_ERR_CUDA;
  }
  std::vector<double> M((size_t)n * n, 0.0);
  double dmax = 0.0;
  for (int k = 0; k < gc.n[2]; ++k)
    for (int j = 0; j < gc.n[1]; ++j)
      for (int i = 0; i < gc.n[0]; ++i) {
        int row = (int)fidx(gc, 3, i, j, k);
        int c3[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          double ih2 = 1.0 / (gc.h[a] * gc.h[a]);
          // face hi
          if (c3[a] + 1 < gc.n[a]) {
            int f3[3] = {i, j, k};
            f3[a] += 1;
            double b = (double)hb[a][fidx(gc, a, f3[0], f3[1], f3[2])] * ih2;
            int nb3[3] = {i, j, k};
            nb3[a] += 1;
            int col = (int)fidx(gc, 3, nb3[0], nb3[1], nb3[2]);
            M[(size_t)row * n + col] -= b;
            M[(size_t)row * n + row] += b;
          }
          if (c3[a] > 0) {
            double b = (double)hb[a][fidx(gc, a, i, j, k)] * ih2;
            int nb3[3] = {i, j, k};
            nb3[a] -= 1;
            int col = (int)fidx(gc, 3, nb3[0], nb3[1], nb3[2]);
            M[(size_t)row * n + col] -= b;
            M[(size_t)row * n + row] += b;
          }
          if (a == 2 && k + 1 == gc.n[2] && gc.open_top)  // p = 0 on the open top: ghost -p
            M[(size_t)row * n + row] += 2.0 * (double)hb[2][fidx(gc, 2, i, j, k + 1)] * ih2;
        }
        dmax = std::max(dmax, M[(size_t)row * n + row]);
      }
  // a closed box leaves constants in the null space: M = -L + c 1 1^T is SPD
  // and its inverse gives the mean-free solution; with an open top -L is SPD
  const double creg = gc.open_top ? 0.0 : dmax / n;
  for (size_t t = 0; t < M.size(); ++t) M[t] += creg;
  spd_inverse(M, n);
  cudaMemcpyAsync(P.coarse_inv, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    err = "CUDA error in preconditioner setup";
    return WSI_ERR_CUDA;
  }
  P.built = true;
  return WSI_OK;
}

// ------------------------------------------------------------ V-cycle kernels
static inline dim3 grid_rb(const GridDev& g) { return dim3(cdiv(cdiv(g.n[0], 2), BX), cdiv(g.n[1], BY), g.n[2]); }

// one colour of a red-black Gauss-Seidel sweep: thread t of a row owns the
// t-th cell of that colour, i = 2t + ((j + k + color) & 1)
template <typename T>
__global__ void k_rbgs_p(GridDev g, const T* __restrict__ bx, const T* __restrict__ by, const T* __restrict__ bz,
                         T* x, const T* __restrict__ b, int color) {
  const int j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k + color) & 1);
  if (i >= g.n[0] || j >= g.n[1]) return;
  size_t id = fidx(g, 3, i, j, k);
  T ihx2 = ginv2<T>(g, 0), ihy2 = ginv2<T>(g, 1), ihz2 = ginv2<T>(g, 2);
  T s = T(0), d = T(0);
  if (i + 1 < g.n[0]) { T c = bx[fidx(g, 0, i + 1, j, k)] * ihx2; s += c * x[id + 1]; d += c; }
  if (i > 0) { T c = bx[fidx(g, 0, i, j, k)] * ihx2; s += c * x[id - 1]; d += c; }
  if (j + 1 < g.n[1]) { T c = by[fidx(g, 1, i, j + 1, k)] * ihy2; s += c * x[id + g.n[0]]; d += c; }
  if (j > 0) { T c = by[fidx(g, 1, i, j, k)] * ihy2; s += c * x[id - g.n[0]]; d += c; }
  size_t pl = (size_t)g.n[0] * g.n[1];
  if (k + 1 < g.n[2]) { T c = bz[fidx(g, 2, i, j, k + 1)] * ihz2; s += c * x[id + pl]; d += c; }
  else if (g.open_top) d += T(2) * bz[fidx(g, 2, i, j, k + 1)] * ihz2;  // ghost -x above the open top
  if (k > 0) { T c = bz[fidx(g, 2, i, j, k)] * ihz2; s += c * x[id - pl]; d += c; }
  if (d > T(0)) x[id] = (s - b[id]) / d;
}

template <typename T>
__device__ __forceinline__ T lap_at(const GridDev& g, const T* __restrict__ bx, const T* __restrict__ by,
                                    const T* __restrict__ bz, const T* __restrict__ x, int i, int j, int k) {
  size_t id = fidx(g, 3, i, j, k);
  T xc = x[id];
  T ihx2 = ginv2<T>(g, 0), ihy2 = ginv2<T>(g, 1), ihz2 = ginv2<T>(g, 2);
  T s = T(0);
  if (i + 1 < g.n[0]) s += bx[fidx(g, 0, i + 1, j, k)] * (x[id + 1] - xc) * ihx2;
  if (i > 0) s -= bx[fidx(g, 0, i, j, k)] * (xc - x[id - 1]) * ihx2;
  if (j + 1 < g.n[1]) s += by[fidx(g, 1, i, j + 1, k)] * (x[id + g.n[0]] - xc) * ihy2;
  if (j > 0) s -= by[fidx(g, 1, i, j, k)] * (xc - x[id - g.n[0]]) * ihy2;
  size_t pl = (size_t)g.n[0] * g.n[1];
  if (k + 1 < g.n[2]) s += bz[fidx(g, 2, i, j, k + 1)] * (x[id + pl] - xc) * ihz2;
  else if (g.open_top) s -= T(2) * bz[fidx(g, 2, i, j, k + 1)] * xc * ihz2;
  if (k > 0) s -= bz[fidx(g, 2, i, j, k)] * (xc - x[id - pl]) * ihz2;
  return s;
}

// coarse b = mean over children of (b - L x) on the fine grid
template <typename T>
__global__ void k_restrict_res(GridDev gf, GridDev gc, int r0, int r1, int r2, const T* __restrict__ bx,
                               const T* __restrict__ by, const T* __restrict__ bz, const T* __restrict__ x,
                               const T* __restrict__ b, T* bcoarse) {
  int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (I >= gc.n[0] || J >= gc.n[1]) return;
  T s = T(0);
  for (int c = 0; c < r2; ++c)
    for (int bb = 0; bb < r1; ++bb)
      for (int a = 0; a < r0; ++a) {
        int i = I * r0 + a, j = J * r1 + bb, k = K * r2 + c;
        s += b[fidx(gf, 3, i, j, k)] - lap_at<T>(gf, bx, by, bz, x, i, j, k);
      }
  bcoarse[fidx(gc, 3, I, J, K)] = s / T(r0 * r1 * r2);
}

// x_fine += P x_coarse (linear in cell centres along coarsened axes)
template <typename T>
__global__ void k_prolong_add(GridDev gf, GridDev gc, int r0, int r1, int r2, const T* __restrict__ xc, T* xf) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= gf.n[0] || j >= gf.n[1]) return;
  int r[3] = {r0, r1, r2};
  int f3[3] = {i, j, k};
  int c0[3], c1[3];
  T w0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (r[a] == 2) {
      c0[a] = f3[a] >> 1;
      int nb = (f3[a] & 1) ? c0[a] + 1 : c0[a] - 1;
      c1[a] = clampi(nb, 0, gc.n[a] - 1);
      w0[a] = T(0.75);
    } else {
      c0[a] = f3[a];
      c1[a] = f3[a];
      w0[a] = T(1);
    }
  }
  T s = T(0);
#pragma unroll
  for (int cz = 0; cz < 2; ++cz)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        T wx = cx ? T(1) - w0[0] : w0[0];
        T wy = cy ? T(1) - w0[1] : w0[1];
        T wz = cz ? T(1) - w0[2] : w0[2];
        T w = wx * wy * wz;
        if (w == T(0)) continue;
        int a = cx ? c1[0] : c0[0], b = cy ? c1[1] : c0[1], c = cz ? c1[2] : c0[2];
        s += w * xc[fidx(gc, 3, a, b, c)];
      }
  xf[fidx(gf, 3, i, j, k)] += s;
}

// x = Minv (-b), one block
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ Minv, const T* __restrict__ b, T* x) {
  extern __shared__ double sb[];
  for (int t = threadIdx.x; t < n; t += blockDim.x) sb[t] = -(double)b[t];
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += Minv[(size_t)r * n + c] * sb[c];
    x[r] = (T)s;
  }
}

// One pass of the Chebyshev smoother on A = -L (positive semi-definite)
// with Jacobi preconditioning D = diag(A): with x' = x + d (d = 0 on the
// first pass), r = L x' - b = -b - A x' (the residual of A x = -b), and
//     x_out = x',  d_out = alpha d + c r / D.
// Every cell of the level in one coalesced pass (no colouring); the caller
// alternates two buffer pairs and finishes with x += d.
template <typename T>
__global__ void k_cheb_p(GridDev g, const T* __restrict__ bx, const T* __restrict__ by, const T* __restrict__ bz,
                         const T* __restrict__ x, const T* __restrict__ d, const T* __restrict__ b, T* xo, T* dout,
                         T alpha, T c, int first) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  const size_t id = fidx(g, 3, i, j, k);
  const size_t pl = (size_t)g.n[0] * g.n[1];
  auto xv = [&](size_t q) { return first ? x[q] : x[q] + d[q]; };
  const T ihx2 = ginv2<T>(g, 0), ihy2 = ginv2<T>(g, 1), ihz2 = ginv2<T>(g, 2);
  const T xc = xv(id);
  T s = T(0), dg = T(0);
  if (i + 1 < g.n[0]) { T w = bx[fidx(g, 0, i + 1, j, k)] * ihx2; s += w * (xv(id + 1) - xc); dg += w; }
  if (i > 0) { T w = bx[fidx(g, 0, i, j, k)] * ihx2; s += w * (xv(id - 1) - xc); dg += w; }
  if (j + 1 < g.n[1]) { T w = by[fidx(g, 1, i, j + 1, k)] * ihy2; s += w * (xv(id + g.n[0]) - xc); dg += w; }
  if (j > 0) { T w = by[fidx(g, 1, i, j, k)] * ihy2; s += w * (xv(id - g.n[0]) - xc); dg += w; }
  if (k + 1 < g.n[2]) { T w = bz[fidx(g, 2, i, j, k + 1)] * ihz2; s += w * (xv(id + pl) - xc); dg += w; }
  else if (g.open_top) { T w = T(2) * bz[fidx(g, 2, i, j, k + 1)] * ihz2; s -= w * xc; dg += w; }
  if (k > 0) { T w = bz[fidx(g, 2, i, j, k)] * ihz2; s += w * (xv(id - pl) - xc); dg += w; }
  const T r = s - b[id];
  xo[id] = xc;
  dout[id] = (first ? T(0) : alpha * d[id]) + (dg > T(0) ? c * r / dg : T(0));
}

template <typename T>
__global__ void k_cheb_finish(size_t n, const T* __restrict__ x, const T* __restrict__ d, T* out) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    out[t] = x[t] + d[t];
}

// Chebyshev interval of the Jacobi-preconditioned level operator: Gershgorin
// bounds its spectrum by 2 (diagonally dominant, zero row sums away from
// walls); the smoother targets [2/8, 2], the upper part that the coarse grid
// cannot represent.
static constexpr double CHEB_HI = 2.0, CHEB_LO = 0.25;

// m passes of smoothing on level l: red-black Gauss-Seidel sweeps (pre: red
// then black; post: black then red) or a degree-m Chebyshev polynomial
template <typename T>
static void smooth(Precond<T>& P, const Opts& o, size_t l, int m, bool pre, cudaStream_t st) {
  MGLevel<T>& L = P.lev[l];
  const GridDev& g = L.g;
  if (m <= 0) return;
  if (o.mg_smoother != WSI_SMOOTH_CHEBYSHEV) {
    for (int s = 0; s < m; ++s)
      for (int q = 0; q < 2; ++q) {
        const int c = pre ? q : 1 - q;
        ktimer_begin(KC_RBGS_P, st);
        { k_rbgs_p<T><<<grid_rb(g), dim3(BX, BY), 0, st>>>(g, L.beta[0], L.beta[1], L.beta[2], L.x, L.b, c); WSI_COUNT(); }
        ktimer_end(KC_RBGS_P, st);
      }
    return;
  }
  const double theta = 0.5 * (CHEB_HI + CHEB_LO), delta = 0.5 * (CHEB_HI - CHEB_LO), sigma = theta / delta;
  double rho_prev = 1.0 / sigma;
  T* xs[2] = {L.x, L.cx2};
  T* ds[2] = {L.cd, L.cd2};
  const dim3 gr = grid3(g.n[0], g.n[1], g.n[2]);
  int cur = 0;
  for (int k = 0; k < m; ++k) {
    double alpha = 0.0, c = 1.0 / theta;
    if (k > 0) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      alpha = rho * rho_prev;
      c = 2.0 * rho / delta;
      rho_prev = rho;
    }
    ktimer_begin(KC_RBGS_P, st);
    { k_cheb_p<T><<<gr, dim3(BX, BY), 0, st>>>(g, L.beta[0], L.beta[1], L.beta[2], xs[cur], ds[cur], L.b,
                                               xs[1 - cur], ds[1 - cur], (T)alpha, (T)c, k == 0 ? 1 : 0); WSI_COUNT(); }
    ktimer_end(KC_RBGS_P, st);
    cur = 1 - cur;
  }
  const size_t n = fsize(g, 3);
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  { k_cheb_finish<T><<<std::max(blocks, 1), 256, 0, st>>>(n, xs[cur], ds[cur], L.x); WSI_COUNT(); }
}

template <typename T>
static void vcycle(Precond<T>& P, const Opts& o, size_t l, cudaStream_t st);

// pre-smoothing, residual restriction, the coarser cycle and prolongation on
// level l (everything of a V-cycle at l but the post-smoothing)
template <typename T>
static void coarse_part(Precond<T>& P, const Opts& o, size_t l, cudaStream_t st) {
  MGLevel<T>& L = P.lev[l];
  const GridDev& g = L.g;
  dim3 gr = grid3(g.n[0], g.n[1], g.n[2]);
  smooth(P, o, l, o.mg_pre, true, st);
  MGLevel<T>& Cl = P.lev[l + 1];
  const GridDev& gc = Cl.g;
  ktimer_begin(KC_RESTRICT, st);
  { k_restrict_res<T><<<grid3(gc.n[0], gc.n[1], gc.n[2]), dim3(BX, BY), 0, st>>>(
      g, gc, L.r[0], L.r[1], L.r[2], L.beta[0], L.beta[1], L.beta[2], L.x, L.b, Cl.b); WSI_COUNT(); }
  ktimer_end(KC_RESTRICT, st);
  cudaMemsetAsync(Cl.x, 0, fsize(gc, 3) * sizeof(T), st);
  vcycle(P, o, l + 1, st);
  ktimer_begin(KC_PROLONG, st);
  { k_prolong_add<T><<<gr, dim3(BX, BY), 0, st>>>(g, gc, L.r[0], L.r[1], L.r[2], Cl.x, L.x); WSI_COUNT(); }
  ktimer_end(KC_PROLONG, st);
}

template <typename T>
void precond_coarse_part(Precond<T>& P, const Opts& o, int l, cudaStream_t st) {
  coarse_part(P, o, (size_t)l, st);
}
template void precond_coarse_part<float>(Precond<float>&, const Opts&, int, cudaStream_t);

template <typename T>
static void vcycle(Precond<T>& P, const Opts& o, size_t l, cudaStream_t st) {
  MGLevel<T>& L = P.lev[l];
  const GridDev& g = L.g;
  if (l + 1 == P.lev.size()) {
    { k_coarse_solve<T><<<1, 256, P.ncoarse * sizeof(double), st>>>(P.ncoarse, P.coarse_inv, L.b, L.x); WSI_COUNT(); }
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    // learned coarse-grid correction: the network replaces everything below
    // this level, then the usual post-smoothing
    if (P.learn.on && P.learn.ready && (int)l == P.learn.level && P.learn.mode == WSI_LEARN_REPLACE) {
      learned_correction(P, (int)l, L.b, false, st);
      smooth(P, o, l, o.mg_post, false, st);
      return;
    }
  }
  coarse_part(P, o, l, st);
  if constexpr (std::is_same<T, float>::value) {
    // learned augmentation: the network's correction of the residual left
    // by the plain coarse-grid correction
    if (P.learn.on && P.learn.ready && (int)l == P.learn.level && P.learn.mode == WSI_LEARN_AUGMENT) {
      const size_t n = fsize(g, 3);
      const T* bt[3] = {L.beta[0], L.beta[1], L.beta[2]};
      launch_pressure<T>(g, bt, L.x, L.res, st);
      launch_lincomb_f32(n, 1.f, L.b, -1.f, L.res, 0.f, nullptr, L.res, st);
      learned_correction(P, (int)l, L.res, true, st);
    }
  }
  smooth(P, o, l, o.mg_post, false, st);
}

template <typename T>
void precond_vcycle(Precond<T>& P, const Opts& o, cudaStream_t st) {
  vcycle(P, o, 0, st);
}
template void precond_vcycle<double>(Precond<double>&, const Opts&, cudaStream_t);
template void precond_vcycle<float>(Precond<float>&, const Opts&, cudaStream_t);

template <typename T>
void precond_prolong_chain(Precond<T>& P, int from, cudaStream_t st) {
  for (int l = from - 1; l >= 0; --l) {
    MGLevel<T>& L = P.lev[l];
    const GridDev& g = L.g;
    cudaMemsetAsync(L.x, 0, fsize(g, 3) * sizeof(T), st);
    { k_prolong_add<T><<<grid3(g.n[0], g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, P.lev[l + 1].g, L.r[0], L.r[1],
                                                                              L.r[2], P.lev[l + 1].x, L.x); WSI_COUNT(); }
  }
}
template void precond_prolong_chain<float>(Precond<float>&, int, cudaStream_t);

int learned_alloc(Precond<float>& P, UNetImpl* net, int level, UNetImpl* gnet, int glevel, std::string& err) {
  LearnState& S = P.learn;
  S.net = net;
  S.level = level;
  S.gnet = gnet;
  S.glevel = glevel;
  S.ready = false;
  if (!net && !gnet) return WSI_OK;
  if ((net && (level < 1 || level >= (int)P.lev.size())) || (gnet && (glevel < 1 || glevel >= (int)P.lev.size()))) {
    err = "learned correction level outside the multigrid hierarchy";
    return WSI_ERR_INVALID_ARG;
  }
  if (S.lrho.empty()) {
    S.lrho.assign(P.lev.size(), nullptr);
    S.phi.assign(P.lev.size(), nullptr);
    for (size_t l = 1; l < P.lev.size(); ++l) {
      S.lrho[l] = dalloc<float>(P.allocs, fsize(P.lev[l].g, 3), err);
      S.phi[l] = dalloc<float>(P.allocs, fsize(P.lev[l].g, 3), err);
      if (!S.lrho[l] || !S.phi[l]) return WSI_ERR_OOM;
    }
    size_t nmax = fsize(P.lev[1].g, 3);
    S.diag = dalloc<float>(P.allocs, nmax, err);
    S.e = dalloc<float>(P.allocs, nmax, err);
    S.t1 = dalloc<float>(P.allocs, nmax, err);
    S.t2 = dalloc<float>(P.allocs, nmax, err);
    S.t3 = dalloc<float>(P.allocs, nmax, err);
    S.ss = dalloc<double>(P.allocs, 4, err);
    S.gdiag = dalloc<float>(P.allocs, nmax, err);
    S.gss = dalloc<double>(P.allocs, 4, err);
    if (!S.diag || !S.e || !S.t1 || !S.t2 || !S.t3 || !S.ss || !S.gdiag || !S.gss) return WSI_ERR_OOM;
  }
  return WSI_OK;
}

// ------------------------------------------------------------ PC glue kernels
template <typename T>
__global__ void k_div_add(GridDev g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
                          const T* __restrict__ rp, T* y) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  T d = (u[fidx(g, 0, i + 1, j, k)] - u[fidx(g, 0, i, j, k)]) * ginv<T>(g, 0) +
        (v[fidx(g, 1, i, j + 1, k)] - v[fidx(g, 1, i, j, k)]) * ginv<T>(g, 1) +
        (w[fidx(g, 2, i, j, k + 1)] - w[fidx(g, 2, i, j, k)]) * ginv<T>(g, 2);
  size_t id = fidx(g, 3, i, j, k);
  y[id] = rp[id] + d;
}

// u = u~ - beta G phi on C-faces, written as float64 into z
template <int C, typename T>
__global__ void k_vel_update(GridDev g, const T* __restrict__ ut, const T* __restrict__ beta,
                             const T* __restrict__ phi, double* z) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= ext(g, C, 0) || j >= ext(g, C, 1)) return;
  int id3[3] = {i, j, k};
  size_t id = fidx(g, C, i, j, k);
  if (!face_row(g, C, id3[C])) {
    z[id] = 0.0;
    return;
  }
  int lo[3] = {i, j, k};
  lo[C] -= 1;
  const T plo = phi[fidx(g, 3, lo[0], lo[1], lo[2])];
  const T phi_hi = (C == 2 && k == g.n[2]) ? -plo : phi[fidx(g, 3, i, j, k)];  // open top: ghost -phi
  T gphi = (phi_hi - plo) * ginv<T>(g, C);
  z[id] = cvt<double, T>(ut[id] - beta[id] * gphi);
}

// p = phi/dt - theta mu y - mean (mean subtracted with the sum in s_dev)
template <typename T>
__global__ void k_p_update(size_t n, const T* __restrict__ phi, const T* __restrict__ mu, const T* __restrict__ y,
                           double inv_dt, double theta, double* z) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  if constexpr (std::is_same<T, float>::value) {
    // float32 preconditioner: float32 arithmetic, exact widening by integer operations
    const float fi = (float)inv_dt, ft = (float)theta;
    for (; t < n; t += stride) z[t] = f2d_fast(phi[t] * fi - ft * mu[t] * y[t]);
  } else {
    for (; t < n; t += stride) z[t] = (double)phi[t] * inv_dt - theta * (double)mu[t] * (double)y[t];
  }
}

template <typename T>
__global__ void k_sub_mean(T* x, size_t n, const double* __restrict__ sum) {
  T m = (T)(sum[0] / (double)n);
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; t < n; t += stride) x[t] -= m;
}

template <typename T>
static void sub_mean(T* x, size_t n, double* dsum, double* scratch, cudaStream_t st) {
  launch_sum<T>(x, n, dsum, scratch, st);
  int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  { k_sub_mean<T><<<std::max(blocks, 1), 256, 0, st>>>(x, n, dsum); WSI_COUNT(); }
}

// Viscous V-cycle on level l for A u = b, A = rho/dt - theta L_mu on that
// level's grid and coefficients: sweeps, face-residual restriction, the
// coarser cycle (sweeps alone on the coarsest level), prolongation, sweeps.
template <typename T>
static void vcycle_visc(Precond<T>& P, const Opts& o, size_t l, const Coef<T>& cf0, T* const u0[3],
                        const T* const b0[3], T inv_dt, T theta, cudaStream_t st) {
  const GridDev& g = P.lev[l].g;
  Coef<T> cf = cf0;
  T* const* u = u0;
  const T* const* b = b0;
  VLevel<T>& V = P.vlev[l];
  if (l > 0) {
    for (int c = 0; c < 3; ++c) {
      cf.rho_face[c] = V.rho_face[c];
      cf.mu_e[c] = V.mu_e[c];
      cf.beta[c] = nullptr;
    }
    cf.mu_cc = V.mu_cc;
    u = V.u;
    b = V.b;
  }
  const bool coarsest = l + 1 == P.lev.size();
  const int nsw = coarsest ? 4 * o.visc_sweeps : o.visc_sweeps;
  for (int s = 0; s < nsw; ++s)
    for (int c = 0; c < 2; ++c) launch_viscous_rbgs<T>(g, cf, inv_dt, theta, u, b, c, st);
  if (coarsest) return;
  T* res[3];
  for (int c = 0; c < 3; ++c) res[c] = l == 0 ? P.vres0[c] : V.res[c];
  const T* uc[3] = {u[0], u[1], u[2]};
  launch_viscous_residual<T>(g, cf, inv_dt, theta, uc, b, res, st);
  const MGLevel<T>& F = P.lev[l];
  const GridDev& gc = P.lev[l + 1].g;
  VLevel<T>& VC = P.vlev[l + 1];
  const int r0 = F.r[0], r1 = F.r[1], r2 = F.r[2];
  { k_vrestrict<0, T><<<grid3(gc.n[0] + 1, gc.n[1], gc.n[2]), dim3(BX, BY), 0, st>>>(g, gc, r0, r1, r2, res[0], VC.b[0]); WSI_COUNT(); }
  { k_vrestrict<1, T><<<grid3(gc.n[0], gc.n[1] + 1, gc.n[2]), dim3(BX, BY), 0, st>>>(g, gc, r0, r1, r2, res[1], VC.b[1]); WSI_COUNT(); }
  { k_vrestrict<2, T><<<grid3(gc.n[0], gc.n[1], gc.n[2] + 1), dim3(BX, BY), 0, st>>>(g, gc, r0, r1, r2, res[2], VC.b[2]); WSI_COUNT(); }
  for (int c = 0; c < 3; ++c) cudaMemsetAsync(VC.u[c], 0, fsize(gc, c) * sizeof(T), st);
  vcycle_visc<T>(P, o, l + 1, cf0, u0, b0, inv_dt, theta, st);
  { k_vprolong<0, T><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, gc, r0, r1, r2, VC.u[0], u[0]); WSI_COUNT(); }
  { k_vprolong<1, T><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, gc, r0, r1, r2, VC.u[1], u[1]); WSI_COUNT(); }
  { k_vprolong<2, T><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, gc, r0, r1, r2, VC.u[2], u[2]); WSI_COUNT(); }
  for (int s = 0; s < o.visc_sweeps; ++s)
    for (int c = 1; c >= 0; --c) launch_viscous_rbgs<T>(g, cf, inv_dt, theta, u, b, c, st);
}

template <typename T>
void precond_apply(Precond<T>& P, const GridDev& g, const Opts& o, double dt, const double* v, double* z,
                   cudaStream_t st) {
  Packing pk = packing(g);
  {
    CastSet<double, T> cs;
    cs.count = 4;
    for (int c = 0; c < 3; ++c) {
      cs.a[c] = v + pk.off[c];
      cs.b[c] = P.ru[c];
      cs.n[c] = fsize(g, c);
      cudaMemsetAsync(P.ut[c], 0, fsize(g, c) * sizeof(T), st);
    }
    cs.a[3] = v + pk.off[3];
    cs.b[3] = P.rp;
    cs.n[3] = fsize(g, 3);
    cast_set(cs, st);  // one launch for the four parts
  }
  Coef<T> cf;
  for (int c = 0; c < 3; ++c) {
    cf.rho_face[c] = P.rho_face[c];
    cf.beta[c] = P.lev[0].beta[c];
    cf.mu_e[c] = P.mu_e[c];
  }
  cf.mu_cc = P.mu_cc;
  T inv_dt = (T)(1.0 / dt), theta = (T)o.theta;
  // u~ = A^{-1} r_u (approximately): red-black sweeps, or viscous V-cycles
  if (o.visc_mg > 0) {
    for (int c = 0; c < o.visc_mg; ++c) vcycle_visc<T>(P, o, 0, cf, P.ut, P.ru, inv_dt, theta, st);
  } else {
    for (int s = 0; s < o.visc_sweeps; ++s)
      for (int c = 0; c < 2; ++c) launch_viscous_rbgs<T>(g, cf, inv_dt, theta, P.ut, P.ru, c, st);
  }
  // y = r_p + D u~, mean-free in a closed box (the pressure problem's
  // compatibility condition; an open top fixes the pressure instead)
  dim3 gr = grid3(g.n[0], g.n[1], g.n[2]);
  { k_div_add<T><<<gr, dim3(BX, BY), 0, st>>>(g, P.ut[0], P.ut[1], P.ut[2], P.rp, P.y); WSI_COUNT(); }
  size_t ncell = fsize(g, 3);
  if (!g.open_top) sub_mean<T>(P.y, ncell, P.dsum, P.dscratch, st);
  // phi = L^{-1} y
  MGLevel<T>& L0 = P.lev[0];
  cudaMemcpyAsync(L0.b, P.y, ncell * sizeof(T), cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(L0.x, 0, ncell * sizeof(T), st);
  for (int c = 0; c < o.mg_cycles; ++c) vcycle(P, o, 0, st);
  // velocity and pressure updates
  { k_vel_update<0, T><<<grid3(g.n[0] + 1, g.n[1], g.n[2]), dim3(BX, BY), 0, st>>>(g, P.ut[0], L0.beta[0], L0.x,
                                                                                 z + pk.off[0]); WSI_COUNT(); }
  { k_vel_update<1, T><<<grid3(g.n[0], g.n[1] + 1, g.n[2]), dim3(BX, BY), 0, st>>>(g, P.ut[1], L0.beta[1], L0.x,
                                                                                 z + pk.off[1]); WSI_COUNT(); }
  { k_vel_update<2, T><<<grid3(g.n[0], g.n[1], g.n[2] + 1), dim3(BX, BY), 0, st>>>(g, P.ut[2], L0.beta[2], L0.x,
                                                                                 z + pk.off[2]); WSI_COUNT(); }
  int blocks = (int)std::min<size_t>((ncell + 255) / 256, 152 * 16);
  { k_p_update<T><<<std::max(blocks, 1), 256, 0, st>>>(ncell, L0.x, P.mu_cc, P.y, 1.0 / dt, o.theta, z + pk.off[3]); WSI_COUNT(); }
  if (!g.open_top) sub_mean<double>(z + pk.off[3], ncell, P.dsum, P.dscratch, st);
}

template int precond_alloc<double>(Precond<double>&, const GridDev&, std::string&);
template int precond_alloc<float>(Precond<float>&, const GridDev&, std::string&);
template void precond_free<double>(Precond<double>&);
template void precond_free<float>(Precond<float>&);
template int precond_setup<double>(Precond<double>&, const GridDev&, const Coef<double>&, cudaStream_t, std::string&);
template int precond_setup<float>(Precond<float>&, const GridDev&, const Coef<double>&, cudaStream_t, std::string&);
template void precond_apply<double>(Precond<double>&, const GridDev&, const Opts&, double, const double*, double*,
                                    cudaStream_t);
template void precond_apply<float>(Precond<float>&, const GridDev&, const Opts&, double, const double*, double*,
                                   cudaStream_t);

}  // namespace wsi
