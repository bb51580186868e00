// Energy-split dispatch of the per-point kernels and the spectral split's assembled
// elasticity tangent (pf_spectral.cu).
#pragma once
#include "pf_internal.cuh"

namespace pf {

// Per-point kernels for the material's split: VD runs the pf_ops.cu kernels, SPECTRAL the
// pf_spectral.cu ones (same arguments and outputs as qp_energy / fs_coeff / fs_predict).
void point_energy(const GridD &g, const MatD &m, const double *u, const double *Hprev,
                  double *psi, double *Hout, cudaStream_t st);
void point_fs_coeff(const GridD &g, const MatD &m, int scheme, double psi_crit,
                    const double *u, const double *d, const double *Hprev, double *c_aug,
                    uint8_t *active, cudaStream_t st, const At1D &at1 = At1D());
void point_fs_predict(const GridD &g, const MatD &m, int scheme, const double *u,
                      const double *d, const double *dd, const double *Hprev,
                      const uint8_t *active, double *Hhalf, cudaStream_t st, int at1 = 0);

// Per-point stress Sq (3 x Q: sxx, syy, sxy) and Newton tangent Dq (6 x Q: D00, D01, D02,
// D11, D12, D22 in Voigt form with engineering shear), FP64, entry-major (k * Q + 4e + q),
// for the material's split; either output may be NULL.  Masked elements get 0.
void sp_points(const GridD &g, const MatD &m, const double *u, const double *d, double *Sq,
               double *Dq, cudaStream_t st);
// F = sum_e sum_q w B^T sigma_q over all 2N DOFs from Sq (one thread per node, no atomics).
void sp_force(const GridD &g, const double *Sq, double *F, cudaStream_t st);
// Nodal stencil of K(Dq) = sum_e sum_q w B^T D_q B in the multigrid layout (9 neighbours x
// 2 x 2 blocks per node, entry-major; stencil index in pf_gmg.cuh), unmasked.
template <class T>
void sp_stencil(const GridD &g, const double *Dq, T *S, cudaStream_t st);
// y = K x through the stencil with rows and columns of constrained DOFs (g.dofm) zeroed;
// with sc/ws and epi != EPI_NONE also x.y and the Krylov epilogue (as elas_apply).
template <class T>
void sp_apply(const GridD &g, const T *S, const T *x, T *y, cudaStream_t st,
              KrylovScal *sc = nullptr, const RedWs *ws = nullptr, int epi = EPI_NONE);
// diag = diagonal of the stencil, 0 on constrained DOFs.
template <class T>
void sp_diag(const GridD &g, const T *S, T *diag, cudaStream_t st);

}  // namespace pf
