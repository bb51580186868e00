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
// dense inverse, computed on the device in FP64 at setup (k_coarse_inverse).  The
// V-cycle is a fixed, symmetric linear operator, so it preconditions CG.
#pragma once
#include "pf_internal.cuh"

namespace pf {

constexpr int GMG_MAX_LEVELS = 16;
constexpr int GMG_COARSE_MAX = 8;   // coarsen while max(nx, ny) > this
constexpr int CHEB_DEGREE = 2;
constexpr int COARSE_THREADS = 1024;  // threads of the single-CTA coarse cycle
constexpr int GMG_CTA_NODES = 1100;   // levels with at most this many nodes run in that CTA

// Stencil entry index: neighbour k = (dj+1)*3 + (di+1), block (r, c), node; entry-major so
// that consecutive nodes of one entry are contiguous.
template <int B>
__host__ __device__ __forceinline__ size_t sten_idx(int k, int r, int c, size_t node, size_t nn) {
  return ((size_t)(k * B * B + r * B + c)) * nn + node;
}

template <class T>
struct GmgLevel {
  int nx = 0, ny = 0;
  size_t nn = 0;
  T *S = nullptr;       // 9*B*B*nn stencil (SoA: entry-major), levels >= 0
  T *invd = nullptr;    // B*nn inverse diagonal (0 on constrained / empty DOFs)
  T *x = nullptr, *b = nullptr, *r = nullptr, *dv = nullptr, *y = nullptr;
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
  double *cwork = nullptr;  // ncoarse^2 FP64 work array of its factorisation (device)
  RedWs ws{};
  bool ready = false;
  void *dca = nullptr;      // device copy of the coarse-cycle arguments (batched launches)
};

// Lay out the hierarchy for a fine grid in arena A (counting only when A has no base).
template <class T>
cudaError_t gmg_alloc(Gmg<T> &G, int nx, int ny, int B, const RedWs &ws, Arena &A);
template <class T>
void gmg_free(Gmg<T> &G);

// Setup from the fine operator.  Elasticity: fine tangent with d (type T) and tension
// bits; damage: per-Gauss-point coefficient c (type T), kappa.  dofm: fine mask.
template <class T>
cudaError_t gmg_setup_elas(Gmg<T> &G, const GridD &g, const MatD &m, const T *d,
                           const uint8_t *tens, cudaStream_t st);
template <class T>
cudaError_t gmg_setup_damage(Gmg<T> &G, const GridD &g, const T *c, double kappa,
                             cudaStream_t st);
// Elasticity setup from per-point tangents Dq (6 x Q, FP64; spectral split), see sp_points.
template <class T>
cudaError_t gmg_setup_elas_qp(Gmg<T> &G, const GridD &g, const double *Dq, cudaStream_t st);

// Batched V-cycle below level 0 for n hierarchies of one kind (same B, each with
// lc >= 1): the restriction of level 0's residual (lv[0].r -> lv[1].b), and gmg_mid(G, 1)
// of every hierarchy with one launch per kernel and level for all of them.  done[i]: stop
// flag of hierarchy i's Krylov solve (its CTAs skip the launch once it is set).
// gmg_batch_prepare writes the device copy of the coarse-cycle arguments; it allocates,
// so it runs outside stream capture, once per hierarchy.  n <= PF_MAXB.
template <class T>
cudaError_t gmg_batch_prepare(Gmg<T> &G);
template <class T>
int gmg_restrict0_batch(int n, Gmg<T> *const *G, const int *const *done, cudaStream_t st);
template <class T>
int gmg_mid_batch(int n, Gmg<T> *const *G, const int *const *done, cudaStream_t st);

// First level handled by the single-CTA coarse cycle: the first with at most `nodes`
// nodes (GMG_CTA_NODES at allocation).  Returns the new lc.
template <class T>
int gmg_set_coarse_nodes(Gmg<T> &G, int nodes);

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
void gmg_coarse_cycle(const Gmg<T> &G, int lc, const T *b0, T *x0, cudaStream_t st);
// Fused smoothing passes of a stencil level l (see pf_gmg.cu): pre-smoothing from zero
// (x = S_pre b), coarse-grid correction plus first post step (reads lv[l+1].x, writes
// lv[l].r and lv[l].dv), second post step on lv[l].dv and lv[l].r.
template <class T>
void gmg_pre(const Gmg<T> &G, int l, const T *b, T *x, cudaStream_t st);
template <class T>
void gmg_prolong_first(const Gmg<T> &G, int l, const T *xin, T *xout, cudaStream_t st);
template <class T>
void gmg_post(const Gmg<T> &G, int l, T *x, cudaStream_t st);

// lv[l0].x = V_l0(lv[l0].b) for l0 >= 1: the V-cycle below level l0 - 1 on stencil
// levels.  Levels l0 .. G.lc - 1 run as separate grid-wide kernels; levels from G.lc down
// to the dense solve run in one single-CTA kernel.  Returns the kernel launches issued.
template <class T>
int gmg_mid(Gmg<T> &G, int l0, cudaStream_t st) {
  int launches = 0;
  const int lc = G.lc > l0 ? G.lc : l0;
  // down: pre-smoothed iterate in lv[l].y, residual restricted to lv[l+1].b
  for (int l = l0; l < lc; ++l) {
    GmgLevel<T> &L = G.lv[l];
    gmg_pre<T>(G, l, L.b, L.y, st);
    gmg_sten_apply<T>(G, l, L.y, L.b, L.r, 1, st);
    gmg_restrict<T>(G, l, L.r, G.lv[l + 1].b, st);
    launches += 3;
  }
  gmg_coarse_cycle<T>(G, lc, G.lv[lc].b, G.lv[lc].x, st);
  ++launches;
  // up: corrected and post-smoothed iterate in lv[l].x
  for (int l = lc - 1; l >= l0; --l) {
    gmg_prolong_first<T>(G, l, G.lv[l].y, G.lv[l].x, st);
    gmg_post<T>(G, l, G.lv[l].x, st);
    launches += 2;
  }
  return launches;
}

// z = V(r): one V-cycle (Chebyshev degree 2 pre and post) on the fine residual r.
// fine_apply(x, y) must compute y = A_0 x with constrained rows/columns zeroed; level 0 is
// applied matrix-free, coarser levels through gmg_mid.  Returns the kernel launches issued.
template <class T, class FineApply>
int gmg_vcycle(Gmg<T> &G, FineApply fine_apply, const T *r, T *z, cudaStream_t st) {
  if (G.lc == 0) {
    gmg_coarse_cycle<T>(G, 0, r, z, st);
    return 1;
  }
  GmgLevel<T> &L = G.lv[0];
  gmg_cheb_first<T>(G, 0, r, z, L.dv, L.r, st);
  fine_apply(L.dv, L.y);
  gmg_cheb_step<T>(G, 0, L.y, z, L.dv, L.r, st);
  fine_apply(z, L.y);
  gmg_sub<T>((size_t)G.B * L.nn, r, L.y, L.r, st);
  gmg_restrict<T>(G, 0, L.r, G.lv[1].b, st);
  int launches = 6 + gmg_mid<T>(G, 1, st);
  gmg_prolong_add<T>(G, 0, G.lv[1].x, z, st);
  fine_apply(z, L.y);
  gmg_cheb_first_x<T>(G, 0, r, L.y, z, L.dv, L.r, st);
  fine_apply(L.dv, L.y);
  gmg_cheb_step<T>(G, 0, L.y, z, L.dv, L.r, st);
  return launches + 5;
}

}  // namespace pf
