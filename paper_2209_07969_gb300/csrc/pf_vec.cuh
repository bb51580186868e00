// Launchers of the vector kernels (pf_vec.cu).
#pragma once
#include "pf_internal.cuh"

namespace pf {
template <class T>
void cg_init(size_t n, const T *b, T *x, T *r, T *z, T *p, const T *invd, KrylovScal *sc,
             const RedWs &ws, cudaStream_t st);
template <class T>
void cg_update(size_t n, T *x, T *r, T *z, const T *p, const T *q, const T *invd,
               KrylovScal *sc, const RedWs &ws, cudaStream_t st);
template <class T>
void cg_dir(size_t n, const T *z, T *p, const KrylovScal *sc, cudaStream_t st);
template <class T>
void invert(size_t n, const T *diag, T *inv, cudaStream_t st);
template <class T>
void pcg_init(size_t n, const T *b, T *x, T *r, KrylovScal *sc, const RedWs &ws, cudaStream_t st);
template <class T>
void pcg_update(size_t n, T *x, T *r, const T *p, const T *q, KrylovScal *sc, const RedWs &ws,
                cudaStream_t st);
template <class T>
void pcg_rz(size_t n, const T *r, const T *z, T *p, int first, KrylovScal *sc, const RedWs &ws,
            cudaStream_t st);
void fill(size_t n, double v, double *y, cudaStream_t st);
// Condition kernel ending each pass of a device-side Krylov loop (k_krylov_while).
void krylov_while(cudaGraphConditionalHandle h, KrylovScal *sc, cudaStream_t st);
void masked_comb(size_t n, int ncomp, const uint8_t *dofm, double s, const double *a, double t,
                 const double *b, double *out, cudaStream_t st);
void add(size_t n, const double *x, double *y, cudaStream_t st);
template <class A, class B>
void convert(size_t n, const A *a, B *b, cudaStream_t st);
// b = (float)(s a) and x += s (double)e: the FP32 side of iterative refinement works on a
// right-hand side scaled to unit size (s a power of two, so the scaling is exact).
void scale_to_f32(size_t n, double s, const double *a, float *b, cudaStream_t st);
// x[i]: a fixed pattern in [0, 1e-3) (operand of launch-shape timings)
void fill_ramp_f32(size_t n, float *x, cudaStream_t st);
void add_scaled_f32(size_t n, double s, const float *e, double *x, cudaStream_t st);
template <class T>
void coef(size_t n, double gcl, const double *H, T *c, cudaStream_t st);
void lift(size_t nn, const uint8_t *flags, const uint8_t *dofm, double ubar, double *u,
          cudaStream_t st);
void norms(size_t n, int ncomp, const uint8_t *dofm, const double *v, double *out,
           const RedWs &ws, cudaStream_t st);
void stag_max(size_t n, const uint8_t *dofm, const double *Kd, const double *b,
              const double *diag, double *out, const RedWs &ws, cudaStream_t st);
void reaction(size_t nn, const uint8_t *flags, int dir, const double *F, double *out,
              const RedWs &ws, cudaStream_t st);
void project(size_t n, const uint8_t *dofm, const double *dlo, double *d, cudaStream_t st);
}  // namespace pf
