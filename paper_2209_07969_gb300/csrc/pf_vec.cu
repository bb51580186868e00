// Vector kernels of the Krylov solvers and the FP64 reductions of the staggered loop.
// Dot products accumulate in FP64 whatever the vector type; the last CTA of each
// reduction updates the solver scalars on the device (no host round trip per step).
#include <math.h>
#include <stdlib.h>

#include "pf_internal.cuh"
#include "pf_vec.cuh"
#include "pf_batch.cuh"

namespace pf {


template <int NV>
__device__ __forceinline__ bool vgrid_reduce(double (&v)[NV], const RedWs ws, double (&tot)[NV],
                                             bool is_max) {
  return red_grid<NV>(v, ws, tot, is_max);
}

// DOF constrained?  ncomp = 2 (u: bit = component) or 1 (d: bit 2).
__device__ __forceinline__ bool constrained(const uint8_t *dofm, size_t i, int ncomp) {
  if (!dofm) return false;
  if (ncomp == 2) return (dofm[i >> 1] >> (i & 1)) & 1;
  return (dofm[i] >> 2) & 1;
}

// ---- CG ------------------------------------------------------------------------------
// Each thread sums its few entries in the vector type; the cross-thread tree (warp,
// CTA, grid) runs in FP64.
// x = 0, r = b, z = M^-1 r, p = z; rz = r.z, rr = r.r -> sc.
template <class T>
__global__ void k_cg_init(size_t n, const T *__restrict__ b, T *__restrict__ x,
                          T *__restrict__ r, T *__restrict__ z, T *__restrict__ p,
                          const T *__restrict__ invd, KrylovScal *sc, RedWs ws) {
  T rz = T(0), rr = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T ri = b[i];
    const T zi = invd[i] * ri;
    x[i] = T(0);
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  double v[2] = {(double)rz, (double)rr}, tot[2];
  if (vgrid_reduce<2>(v, ws, tot, false)) {
    sc->rz = tot[0];
    sc->rr = tot[1];
    sc->rr0 = tot[1];
    sc->it = 0;
    sc->breakdown = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
  }
}

// x += alpha p; r -= alpha q; z = M^-1 r; beta = r.z / rz_old.
template <class T>
__global__ void k_cg_update(size_t n, T *__restrict__ x, T *__restrict__ r, T *__restrict__ z,
                            const T *__restrict__ p, const T *__restrict__ q,
                            const T *__restrict__ invd, KrylovScal *sc, RedWs ws) {
  const T a = (T)sc->alpha;
  T rz = T(0), rr = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    const T zi = invd[i] * ri;
    z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  double v[2] = {(double)rz, (double)rr}, tot[2];
  if (vgrid_reduce<2>(v, ws, tot, false)) {
    const double old = sc->rz;
    sc->beta = (old > 0.0 && isfinite(tot[0])) ? tot[0] / old : 0.0;
    sc->rz = tot[0];
    sc->rr = tot[1];
  }
}

// p = z + beta p.
template <class T>
__global__ void k_cg_dir(size_t n, const T *__restrict__ z, T *__restrict__ p,
                         const KrylovScal *sc) {
  const T bt = (T)sc->beta;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = z[i] + bt * p[i];
}

// ---- CG with an external preconditioner (multigrid) --------------------------------------
// x = 0, r = b; rr = r.r
template <class T>
__global__ void k_pcg_init(size_t n, const T *__restrict__ b, T *__restrict__ x,
                           T *__restrict__ r, KrylovScal *sc, RedWs ws) {
  T rr = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T ri = b[i];
    x[i] = T(0);
    r[i] = ri;
    rr += ri * ri;
  }
  double v[1] = {(double)rr}, tot[1];
  if (vgrid_reduce<1>(v, ws, tot, false)) {
    sc->rr = tot[0];
    sc->rr0 = tot[0];
    sc->it = 0;
    sc->rz = 0.0;
    sc->breakdown = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
  }
}

// x += alpha p; r -= alpha q; rr = r.r
template <class T>
__global__ void k_pcg_update(size_t n, T *__restrict__ x, T *__restrict__ r,
                             const T *__restrict__ p, const T *__restrict__ q, KrylovScal *sc,
                             RedWs ws) {
  const T a = (T)sc->alpha;
  T rr = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    rr += ri * ri;
  }
  double v[1] = {(double)rr}, tot[1];
  if (vgrid_reduce<1>(v, ws, tot, false)) sc->rr = tot[0];
}

// rz_new = r.z; beta = rz_new / rz (0 on the first call, flagged by rz == 0); p = z + beta p
// is left to k_cg_dir.  first != 0: p = z is written here directly.
template <class T>
__global__ void k_pcg_rz(size_t n, const T *__restrict__ r, const T *__restrict__ z,
                         T *__restrict__ p, int first, KrylovScal *sc, RedWs ws) {
  T rz = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T zi = z[i];
    rz += r[i] * zi;
    if (first) p[i] = zi;
  }
  double v[1] = {(double)rz}, tot[1];
  if (vgrid_reduce<1>(v, ws, tot, false)) {
    const double old = sc->rz;
    sc->beta = (!first && old > 0.0 && isfinite(tot[0])) ? tot[0] / old : 0.0;
    sc->rz = tot[0];
    if (!(tot[0] > 0.0)) sc->breakdown = 1;
  }
}

// End of one pass of a device-side Krylov loop (a conditional WHILE node of a CUDA graph):
// count the iteration and keep looping while ||r||^2 > rtol2 ||r0||^2, without breakdown,
// for fewer than maxit iterations.  A NaN residual ends the loop (the comparison fails).
bool pdl_enabled() {
  static const bool on = [] {
    const char *e = getenv("PF_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

__global__ void k_krylov_while(cudaGraphConditionalHandle h, KrylovScal *sc) {
  pdl_enter();
  const int it = sc->it + 1;
  sc->it = it;
  const bool more = sc->rr > sc->rtol2 * sc->rr0 && !sc->breakdown && it < sc->maxit;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Batched form: each simulation that has not stopped counts its iteration and stops on the
// single solve's test (so it runs exactly the iterations it runs alone); the loop goes on
// while any simulation has not stopped.
struct ScalSet {
  int n;
  KrylovScal *sc[PF_MAXB];
};
__global__ void k_krylov_while_batch(cudaGraphConditionalHandle h, ScalSet s) {
  pdl_enter();
  bool any = false;
  for (int i = 0; i < s.n; ++i) {
    KrylovScal *k = s.sc[i];
    if (k->done) continue;
    const int it = k->it + 1;
    k->it = it;
    const bool more = k->rr > k->rtol2 * k->rr0 && !k->breakdown && it < k->maxit;
    if (more)
      any = true;
    else
      k->done = 1;
  }
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

// ---- helpers ---------------------------------------------------------------------------
// inv[i] = free && diag > 0 ? 1/diag : 0.
template <class T>
__global__ void k_invert(size_t n, const T *__restrict__ diag, T *__restrict__ inv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T dv = diag[i];
    inv[i] = dv > T(0) ? T(1) / dv : T(0);
  }
}

// out = free ? s * a - t * b : 0  (b may be null)
__global__ void k_masked_comb(size_t n, int ncomp, const uint8_t *__restrict__ dofm, double s,
                              const double *__restrict__ a, double t,
                              const double *__restrict__ b, double *__restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = s * a[i];
    if (b) v -= t * b[i];
    out[i] = constrained(dofm, i, ncomp) ? 0.0 : v;
  }
}

__global__ void k_fill(size_t n, double v, double *__restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = v;
}

// y += x
__global__ void k_add(size_t n, const double *__restrict__ x, double *__restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

template <class A, class B>
__global__ void k_convert(size_t n, const A *__restrict__ a, B *__restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (B)a[i];
}

__global__ void k_scale_to_f32(size_t n, double s, const double *__restrict__ a,
                               float *__restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)(s * a[i]);
}

__global__ void k_add_scaled_f32(size_t n, double s, const float *__restrict__ e,
                                 double *__restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] += s * (double)e[i];
}

// c = G_c/l + 2 H (AT2 coefficient of the evolution-equation tangent)
template <class T>
__global__ void k_coef(size_t n, double gcl, const double *__restrict__ H, T *__restrict__ c) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    c[i] = (T)(gcl + 2.0 * H[i]);
}

// Lift: u = ubar on LOAD components, 0 on FIX components and fully constrained nodes.
__global__ void k_lift(size_t nn, const uint8_t *__restrict__ flags,
                       const uint8_t *__restrict__ dofm, double ubar, double *__restrict__ u) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const uint8_t f = flags[n], m = dofm[n];
    const bool orphan = (m & 8) != 0;
    if (m & 1) u[2 * n] = (!orphan && (f & PF_LOAD_X)) ? ubar : 0.0;
    if (m & 2) u[2 * n + 1] = (!orphan && (f & PF_LOAD_Y)) ? ubar : 0.0;
  }
}

// sums of squares over free / constrained DOFs
__global__ void k_norms(size_t n, int ncomp, const uint8_t *__restrict__ dofm,
                        const double *__restrict__ v, double *out, RedWs ws) {
  double a = 0.0, b = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double x = v[i];
    if (constrained(dofm, i, ncomp)) b += x * x; else a += x * x;
  }
  double vv[2] = {a, b}, tot[2];
  if (vgrid_reduce<2>(vv, ws, tot, false)) {
    out[0] = tot[0];
    out[1] = tot[1];
  }
}

// max over free d DOFs of |(Kd - b) / diag|
__global__ void k_stag_max(size_t n, const uint8_t *__restrict__ dofm,
                           const double *__restrict__ Kd, const double *__restrict__ b,
                           const double *__restrict__ diag, double *out, RedWs ws) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    if (constrained(dofm, i, 1)) continue;
    const double r = fabs((Kd[i] - b[i]) / diag[i]);
    m = fmax(m, isnan(r) ? INFINITY : r);
  }
  double vv[1] = {m}, tot[1];
  if (vgrid_reduce<1>(vv, ws, tot, true)) out[0] = tot[0];
}

// reaction = sum of F[2n+dir] over nodes carrying the LOAD flag of direction dir
__global__ void k_reaction(size_t nn, const uint8_t *__restrict__ flags, int dir,
                           const double *__restrict__ F, double *out, RedWs ws) {
  const uint8_t bit = dir == 0 ? PF_LOAD_X : PF_LOAD_Y;
  double s = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x)
    if (flags[n] & bit) s += F[2 * n + dir];
  double vv[1] = {s}, tot[1];
  if (vgrid_reduce<1>(vv, ws, tot, false)) out[0] = tot[0];
}

// d = clamp(d, dlo, 1) on free DOFs
__global__ void k_project(size_t n, const uint8_t *__restrict__ dofm,
                          const double *__restrict__ dlo, double *__restrict__ d) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    if (constrained(dofm, i, 1)) continue;
    d[i] = fmin(fmax(d[i], dlo[i]), 1.0);
  }
}

// ---- launchers -----------------------------------------------------------------------
int red_blocks() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 64;
    cached = 2 * sms;
  }
  return cached;
}

static inline unsigned vblocks(size_t n, int cap) {
  size_t b = (n + VEC_THREADS - 1) / VEC_THREADS;
  if (b < 1) b = 1;
  if (b > (size_t)cap) b = cap;
  return (unsigned)b;
}
// reduction kernels: at most red_blocks() CTAs (and never more than the partial slots)
static inline unsigned rblocks(size_t n, int max_blocks) {
  const int cap = red_blocks() < max_blocks ? red_blocks() : max_blocks;
  return vblocks(n, cap);
}

template <class T>
void cg_init(size_t n, const T *b, T *x, T *r, T *z, T *p, const T *invd, KrylovScal *sc,
             const RedWs &ws, cudaStream_t st) {
  k_cg_init<T><<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, b, x, r, z, p, invd, sc, ws);
}
template <class T>
void cg_update(size_t n, T *x, T *r, T *z, const T *p, const T *q, const T *invd,
               KrylovScal *sc, const RedWs &ws, cudaStream_t st) {
  k_cg_update<T><<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, x, r, z, p, q, invd, sc, ws);
}
template <class T>
void cg_dir(size_t n, const T *z, T *p, const KrylovScal *sc, cudaStream_t st) {
  k_cg_dir<T><<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, z, p, sc);
}
template <class T>
void pcg_init(size_t n, const T *b, T *x, T *r, KrylovScal *sc, const RedWs &ws, cudaStream_t st) {
  k_pcg_init<T><<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, b, x, r, sc, ws);
}
template <class T>
void pcg_update(size_t n, T *x, T *r, const T *p, const T *q, KrylovScal *sc, const RedWs &ws,
                cudaStream_t st) {
  k_pcg_update<T><<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, x, r, p, q, sc, ws);
}
template <class T>
void pcg_rz(size_t n, const T *r, const T *z, T *p, int first, KrylovScal *sc, const RedWs &ws,
            cudaStream_t st) {
  k_pcg_rz<T><<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, r, z, p, first, sc, ws);
}
template <class T>
void invert(size_t n, const T *diag, T *inv, cudaStream_t st) {
  k_invert<T><<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, diag, inv);
}
void fill(size_t n, double v, double *y, cudaStream_t st) {
  k_fill<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, v, y);
}
void krylov_while(cudaGraphConditionalHandle h, KrylovScal *sc, cudaStream_t st) {
  launch_pdl(k_krylov_while, dim3(1), dim3(1), st, h, sc);
}
__global__ void k_fill_ramp_f32(size_t n, float *__restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] = 1e-3f * (float)((unsigned)(i * 2654435761u) % 1000u);
}
void fill_ramp_f32(size_t n, float *x, cudaStream_t st) {
  k_fill_ramp_f32<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, x);
}
void krylov_while_batch(cudaGraphConditionalHandle h, int n, KrylovScal *const *sc,
                        cudaStream_t st) {
  ScalSet s;
  s.n = n < PF_MAXB ? n : PF_MAXB;
  for (int i = 0; i < s.n; ++i) s.sc[i] = sc[i];
  launch_pdl(k_krylov_while_batch, dim3(1), dim3(1), st, h, s);
}
void masked_comb(size_t n, int ncomp, const uint8_t *dofm, double s, const double *a, double t,
                 const double *b, double *out, cudaStream_t st) {
  k_masked_comb<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, ncomp, dofm, s, a, t, b, out);
}
void add(size_t n, const double *x, double *y, cudaStream_t st) {
  k_add<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, x, y);
}
template <class A, class B>
void convert(size_t n, const A *a, B *b, cudaStream_t st) {
  k_convert<A, B><<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, a, b);
}
void scale_to_f32(size_t n, double s, const double *a, float *b, cudaStream_t st) {
  k_scale_to_f32<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, s, a, b);
}
void add_scaled_f32(size_t n, double s, const float *e, double *x, cudaStream_t st) {
  k_add_scaled_f32<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, s, e, x);
}
template <class T>
void coef(size_t n, double gcl, const double *H, T *c, cudaStream_t st) {
  k_coef<T><<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, gcl, H, c);
}
void lift(size_t nn, const uint8_t *flags, const uint8_t *dofm, double ubar, double *u,
          cudaStream_t st) {
  k_lift<<<vblocks(nn, 1 << 16), VEC_THREADS, 0, st>>>(nn, flags, dofm, ubar, u);
}
void norms(size_t n, int ncomp, const uint8_t *dofm, const double *v, double *out,
           const RedWs &ws, cudaStream_t st) {
  k_norms<<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, ncomp, dofm, v, out, ws);
}
void stag_max(size_t n, const uint8_t *dofm, const double *Kd, const double *b,
              const double *diag, double *out, const RedWs &ws, cudaStream_t st) {
  k_stag_max<<<rblocks(n, ws.max_blocks), VEC_THREADS, 0, st>>>(n, dofm, Kd, b, diag, out, ws);
}
void reaction(size_t nn, const uint8_t *flags, int dir, const double *F, double *out,
              const RedWs &ws, cudaStream_t st) {
  k_reaction<<<rblocks(nn, ws.max_blocks), VEC_THREADS, 0, st>>>(nn, flags, dir, F, out, ws);
}
void project(size_t n, const uint8_t *dofm, const double *dlo, double *d, cudaStream_t st) {
  k_project<<<vblocks(n, 1 << 16), VEC_THREADS, 0, st>>>(n, dofm, dlo, d);
}

#define PF_INST(T)                                                                            \
  template void cg_init<T>(size_t, const T *, T *, T *, T *, T *, const T *, KrylovScal *,   \
                           const RedWs &, cudaStream_t);                                     \
  template void cg_update<T>(size_t, T *, T *, T *, const T *, const T *, const T *,        \
                             KrylovScal *, const RedWs &, cudaStream_t);                     \
  template void cg_dir<T>(size_t, const T *, T *, const KrylovScal *, cudaStream_t);         \
  template void invert<T>(size_t, const T *, T *, cudaStream_t);                             \
  template void pcg_init<T>(size_t, const T *, T *, T *, KrylovScal *, const RedWs &,         \
                            cudaStream_t);                                                    \
  template void pcg_update<T>(size_t, T *, T *, const T *, const T *, KrylovScal *,           \
                              const RedWs &, cudaStream_t);                                   \
  template void pcg_rz<T>(size_t, const T *, const T *, T *, int, KrylovScal *, const RedWs &, \
                          cudaStream_t);                                                      \
  template void coef<T>(size_t, double, const double *, T *, cudaStream_t);
PF_INST(double)
PF_INST(float)
template void convert<double, float>(size_t, const double *, float *, cudaStream_t);
template void convert<float, double>(size_t, const float *, double *, cudaStream_t);

}  // namespace pf
