// Geometric multigrid preconditioner on the structured Q1 grid (pf_gmg.cu).
//
// Hierarchy: level 0 is the fine grid (nx, ny); level l+1 has ceil(nx_l/2) x ceil(ny_l/2)
// elements, coarse node I sitting on fine node 2I.  Prolongation P is bilinear
// interpolation with the rows of constrained fine DOFs removed; restriction is P^T.
// Coarse operators are Galerkin products A_{l+1} = P^T A_l P, stored as 9-point
// stencils of B x B blocks (B = 2 for displacement, 1 for the phase field).  The fine
// operator is assembled as a stencil only to form A_1 and the smoother bound; the fine
// level itself is applied matrix-free.  Smoother: Chebyshev on D^-1 A over
// [lmax/10, lmax], lmax the Gershgorin bound of D^-1 A (device scalar).  Coarsest level:
// dense inverse, factorised on the host in FP64 at setup.  The V-cycle is a fixed,
// symmetric linear operator, so it preconditions CG.
#pragma once
#include "pf_internal.cuh"

namespace pf {

constexpr int GMG_MAX_LEVELS = 16;
constexpr int GMG_COARSE_MAX = 8;   // coarsen while max(nx, ny) > this
constexpr int CHEB_DEGREE = 2;
constexpr int COARSE_THREADS = 1024;  // threads of the single-CTA coarse cycle
constexpr int GMG_CTA_NODES = 300;    // levels with at most this many nodes run in that CTA

template <class T>
struct GmgLevel {
  int nx = 0, ny = 0;
  size_t nn = 0;
  T *S = nullptr;       // 9*B*B*nn stencil (SoA: entry-major), levels >= 0
  T *invd = nullptr;    // B*nn inverse diagonal (0 on constrained / empty DOFs)
  T *x = nullptr, *b = nullptr, *r = nullptr, *dv = nullptr, *dv2 = nullptr, *y = nullptr;
  uint8_t *fm = nullptr;   // nn bytes, bit c: component c free on this level
  double *lmax = nullptr;  // device scalar
  T *coef = nullptr;       // Chebyshev coefficients in T (see k_cheb_coef)
};

template <class T>
struct Gmg {
  int B = 1;
  int nl = 0;
  int lc = 0;               // first level handled by the single-CTA coarse cycle
  GmgLevel<T> lv[GMG_MAX_LEVELS];
  int ncoarse = 0;          // DOFs of the coarsest level
  T *cinv = nullptr;        // ncoarse^2 dense inverse
  double *hA = nullptr;     // host scratch for the coarse factorisation
  T *hS = nullptr;          // host copy of the coarsest stencil
  T *hInv = nullptr;
  RedWs ws{};
  bool ready = false;
};

// Allocate the hierarchy for a fine grid (device memory owned by the Gmg object).
template <class T>
cudaError_t gmg_alloc(Gmg<T> &G, int nx, int ny, int B, const RedWs &ws);
template <class T>
void gmg_free(Gmg<T> &G);
// Device bytes gmg_alloc takes for an nx x ny grid with B components of tsize bytes.
size_t gmg_bytes(int nx, int ny, int B, size_t tsize);

// Setup from the fine operator.  Elasticity: fine tangent with d (type T) and tension
// bits; damage: per-Gauss-point coefficient c (type T), kappa.  dofm: fine mask.
template <class T>
cudaError_t gmg_setup_elas(Gmg<T> &G, const GridD &g, const MatD &m, const T *d,
                           const uint8_t *tens, cudaStream_t st);
template <class T>
cudaError_t gmg_setup_damage(Gmg<T> &G, const GridD &g, const T *c, double kappa,
                             cudaStream_t st);

// Launchers of the V-cycle building blocks (pf_gmg.cu).
template <class T>
void gmg_sten_apply(const Gmg<T> &G, int l, const T *x, const T *b, T *y, int mode,
                    cudaStream_t st);
template <class T>
void gmg_cheb_first(const Gmg<T> &G, int l, const T *b, T *x, T *d, T *r, cudaStream_t st);
template <class T>
void gmg_cheb_first_x(const Gmg<T> &G, int l, const T *b, const T *y, T *x, T *d, T *r,
                      cudaStream_t st);
template <class T>
void gmg_cheb_step(const Gmg<T> &G, int l, const T *y, T *x, T *d, T *r, cudaStream_t st);
template <class T>
void gmg_sub(size_t n, const T *b, const T *y, T *r, cudaStream_t st);
template <class T>
void gmg_restrict(const Gmg<T> &G, int l, const T *rf, T *bc, cudaStream_t st);
template <class T>
void gmg_prolong_add(const Gmg<T> &G, int l, const T *xc, T *xf, cudaStream_t st);
template <class T>
void gmg_dense(const Gmg<T> &G, const T *b, T *x, cudaStream_t st);
template <class T>
void gmg_sten_cheb(const Gmg<T> &G, int l, const T *din, T *dout, T *x, T *r, cudaStream_t st);
template <class T>
void gmg_coarse_cycle(const Gmg<T> &G, int lc, const T *b0, T *x0, cudaStream_t st);

// z = V(r): one V-cycle (Chebyshev degree 2 pre and post) on the fine residual r.
// fine_apply(x, y) must compute y = A_0 x with constrained rows/columns zeroed.  Levels
// below G.lc run as separate grid-wide kernels; levels from G.lc down to the dense
// solve run in one single-CTA kernel.  Returns the number of kernel launches issued.
template <class T, class FineApply>
int gmg_vcycle(Gmg<T> &G, FineApply fine_apply, const T *r, T *z, cudaStream_t st) {
  int launches = 0;
  const int lc = G.lc;
  for (int l = 0; l < lc; ++l) {
    GmgLevel<T> &L = G.lv[l];
    const T *b = (l == 0) ? r : L.b;
    T *x = (l == 0) ? z : L.x;
    gmg_cheb_first<T>(G, l, b, x, L.dv, L.r, st);
    if (l == 0) {
      fine_apply(L.dv, L.y);
      gmg_cheb_step<T>(G, 0, L.y, x, L.dv, L.r, st);
      fine_apply(x, L.y);
      gmg_sub<T>((size_t)G.B * L.nn, b, L.y, L.r, st);
      launches += 5;
    } else {
      gmg_sten_cheb<T>(G, l, L.dv, L.dv2, x, L.r, st);
      gmg_sten_apply<T>(G, l, x, b, L.r, 1, st);
      launches += 3;
    }
    gmg_restrict<T>(G, l, L.r, G.lv[l + 1].b, st);
    ++launches;
  }
  {
    const T *b0 = lc == 0 ? r : G.lv[lc].b;
    T *x0 = lc == 0 ? z : G.lv[lc].x;
    gmg_coarse_cycle<T>(G, lc, b0, x0, st);
    ++launches;
  }
  for (int l = lc - 1; l >= 0; --l) {
    GmgLevel<T> &L = G.lv[l];
    const T *b = (l == 0) ? r : L.b;
    T *x = (l == 0) ? z : L.x;
    gmg_prolong_add<T>(G, l, G.lv[l + 1].x, x, st);
    if (l == 0) {
      fine_apply(x, L.y);
      gmg_cheb_first_x<T>(G, 0, b, L.y, x, L.dv, L.r, st);
      fine_apply(L.dv, L.y);
      gmg_cheb_step<T>(G, 0, L.y, x, L.dv, L.r, st);
      launches += 5;
    } else {
      gmg_sten_apply<T>(G, l, x, nullptr, L.y, 0, st);
      gmg_cheb_first_x<T>(G, l, b, L.y, x, L.dv, L.r, st);
      gmg_sten_cheb<T>(G, l, L.dv, L.dv2, x, L.r, st);
      launches += 4;
    }
  }
  return launches;
}

}  // namespace pf
