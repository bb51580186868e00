// Internal declarations shared by the libpf translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pf.h"

namespace pf {

// Element tile owned by one 256-thread CTA: TX x TY nodes; the CTA computes the
// (TX+1) x (TY+1) elements touching them (the one-element halo is recomputed by the
// neighbouring CTA as well), so the nodal gather needs no atomics.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int TILE_THREADS = 256;
// Thread count of the element-wise and vector kernels.
constexpr int VEC_THREADS = 256;

struct GridD {
  int nx, ny;
  double hx, hy;
  const uint8_t *active;  // ne bytes or nullptr
  const uint8_t *dofm;    // N bytes (bit0 ux, bit1 uy, bit2 d constrained) or nullptr
};

struct MatD {
  double mu, K, cdim, eta, Gc, l;
};

// Device scalars of one Krylov solve.  The last CTA of each fused reduction updates
// them, so the host never sits between iterations.
struct KrylovScal {
  double rz;       // CG: r.z ;  MINRES: gamma_j
  double pq;       // CG: p.q ;  MINRES: delta_j
  double alpha;    // CG step
  double beta;     // CG direction update
  double rr;       // ||r||^2 (CG) or eta^2 (MINRES)
  double rz_new;
  // MINRES recurrences
  double gam_old, c, c_old, s, s_old, eta, a1, a2, a3, cn;
  int breakdown;
  int pad;
};

// Reduction workspace: per-CTA partials (up to 4 values each) and arrival counters
// (counter[0] for groups, counter[1 + g] for the CTAs of group g), all kept at zero
// between launches.
struct RedWs {
  double *partials;   // 4 * max_blocks doubles
  unsigned *counter;  // red_counters(max_blocks) counters
  int max_blocks;
};
constexpr int RED_GROUP = 64;
inline size_t red_counters(int max_blocks) { return 2 + (size_t)max_blocks / RED_GROUP; }

#ifdef __CUDACC__
// Arrival of CTA `bid` of `nblk` after it published its partials (thread 0 only).  CTAs
// arrive in groups of RED_GROUP; the last CTA of a group arrives at the top counter, so
// no single counter takes more than RED_GROUP atomics.  Returns true in exactly one CTA,
// the last to arrive overall; counters are reset for the next launch.
__device__ __forceinline__ bool red_arrive(unsigned *counter, unsigned bid, unsigned nblk) {
  const unsigned g = bid / RED_GROUP;
  const unsigned ng = (nblk + RED_GROUP - 1) / RED_GROUP;
  const unsigned gsize = (g + 1) * RED_GROUP <= nblk ? RED_GROUP : nblk - g * RED_GROUP;
  __threadfence();
  if (atomicAdd(counter + 1 + g, 1u) != gsize - 1) return false;
  counter[1 + g] = 0u;
  __threadfence();
  if (atomicAdd(counter, 1u) != ng - 1) return false;
  counter[0] = 0u;
  return true;
}
#endif

// CTAs of a grid-wide reduction: two per SM of the current device (set once per
// process from the device attributes).
int red_blocks();

inline unsigned tile_blocks_x(int nx) { return (unsigned)((nx + 1 + TX - 1) / TX); }
inline unsigned tile_blocks_y(int ny) { return (unsigned)((ny + 1 + TY - 1) / TY); }

// ---- operator kernels (pf_ops.cu) ---------------------------------------------------
template <class T>
void elas_apply(const GridD &g, const MatD &m, const T *d, const uint8_t *tens, const T *x,
                T *y, cudaStream_t st, KrylovScal *sc = nullptr, const RedWs *ws = nullptr,
                int epi = 0);
template <class T>
void elas_diag(const GridD &g, const MatD &m, const T *d, const uint8_t *tens, T *diag,
               cudaStream_t st);
void elas_residual(const GridD &g, const MatD &m, const double *u, const double *d, double *F,
                   uint8_t *tens, cudaStream_t st);
template <class T>
void damage_apply(const GridD &g, const T *c, double kappa, const T *x, T *y, cudaStream_t st,
                  KrylovScal *sc = nullptr, const RedWs *ws = nullptr, int epi = 0);
template <class T>
void damage_diag(const GridD &g, const T *c, double kappa, T *diag, cudaStream_t st);
void damage_rhs(const GridD &g, const double *H, double *b, cudaStream_t st);
void qp_energy(const GridD &g, const MatD &m, const double *u, const double *Hprev,
               double *psi, double *Hout, cudaStream_t st);
void fs_coeff(const GridD &g, const MatD &m, int scheme, double psi_crit, const double *u,
              const double *d, const double *Hprev, double *c_aug, uint8_t *active,
              cudaStream_t st);
void fs_predict(const GridD &g, const MatD &m, int scheme, const double *u, const double *d,
                const double *dd, const double *Hprev, const uint8_t *active, double *Hhalf,
                cudaStream_t st);
void dof_mask(int nx, int ny, const uint8_t *flags, const uint8_t *active, uint8_t *mask,
              cudaStream_t st);

// Epilogues of the fused operator + reduction kernels.
enum { EPI_NONE = 0, EPI_CG_ALPHA = 1, EPI_MINRES_DELTA = 2 };

}  // namespace pf
