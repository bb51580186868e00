// Input / output policies of the matrix-free operator kernels (pf_ops.cu): the plain
// product y = A x and the fused stages of the multigrid-preconditioned CG.
//
// A policy forms the operand where the kernel loads it (in) and consumes the product where
// the kernel outputs it (out), so vector updates that the Krylov method and the V-cycle
// smoother need at the finest level ride along with the operator's own memory pass:
//   in(n, i, j, v)          operand at node n = (i, j), B components (constrained
//                           components are zeroed by the kernel afterwards)
//   out(n, o, c, acc)       o = (A x)_n with constrained rows zeroed, c = operand at n;
//                           adds its NR reduction terms to acc
//   fin(tot)                epilogue on the grid totals, in one thread of the last CTA
// Every node is output by exactly one thread, so out() may rewrite buffers at its own
// node; buffers read by in() are never written in the same launch.
//
// B = 2: displacement (interleaved u_x, u_y per node); B = 1: phase field.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// Both displacement components of node n (interleaved storage) in one vector load.
__device__ __forceinline__ void ld_pair(const float *x, size_t n, float &a, float &b) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(x) + n);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld_pair(const double *x, size_t n, double &a, double &b) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(x) + n);
  a = v.x;
  b = v.y;
}

// Node n's B values: read-only path (ldv), coherent path for a buffer the same thread
// rewrites in the launch (ldv_rw), store (stv).
template <class T, int B>
__device__ __forceinline__ void ldv(const T *p, size_t n, T (&v)[B]) {
  if constexpr (B == 2) {
    ld_pair(p, n, v[0], v[1]);
  } else {
    v[0] = __ldg(p + n);
  }
}
template <class T, int B>
__device__ __forceinline__ void ldv_rw(const T *p, size_t n, T (&v)[B]) {
#pragma unroll
  for (int c = 0; c < B; ++c) v[c] = p[B * n + c];
}
template <class T, int B>
__device__ __forceinline__ void stv(T *p, size_t n, const T (&v)[B]) {
  if constexpr (B == 2) {
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float2 *>(p)[n] = make_float2((float)v[0], (float)v[1]);
    } else {
      reinterpret_cast<double2 *>(p)[n] = make_double2((double)v[0], (double)v[1]);
    }
  } else {
    p[n] = v[0];
  }
}

// Epilogue for the fused matvec + dot: CG step length alpha = rz / p.q.
__device__ __forceinline__ void krylov_epilogue(int epi, KrylovScal *sc, double dot) {
  if (epi == EPI_CG_ALPHA) {
    sc->pq = dot;
    if (dot > 0.0 && isfinite(dot) && sc->rz > 0.0) {
      sc->alpha = sc->rz / dot;
    } else {
      sc->alpha = 0.0;
      sc->breakdown = 1;
    }
  }
}

// y = A x (+ x.y for the Krylov epilogue)
template <class T, int B>
struct OpApply {
  static constexpr int NR = 1;
  const T *x;
  T *y;
  KrylovScal *sc;
  int epi;
  __device__ void begin() {}
  __device__ void in(size_t n, int, int, T (&v)[B]) const { ldv<T, B>(x, n, v); }
  __device__ void out(size_t n, const T (&o)[B], const T (&c)[B], T (&acc)[1]) const {
    stv<T, B>(y, n, o);
#pragma unroll
    for (int k = 0; k < B; ++k) acc[0] += c[k] * o[k];
  }
  __device__ bool reduce() const { return epi != EPI_NONE; }
  __device__ void fin(const double (&tot)[1]) const { krylov_epilogue(epi, sc, tot[0]); }
};

// ---- PCG with the multigrid V-cycle, fine-level work fused into the operator kernel -------
// One iteration runs five operator launches (plus the restriction and the coarse levels):
//   DIR      p = z + beta p_prev at the input; q = A p; alpha = rz / p.q
//   UPD      r = r_prev - alpha q, d0 = it D^-1 r at the input; y = A d0;
//            z_a = d0 + c1 d0 + c2 D^-1 (r - y); x += alpha p; rr = r.r
//   RESID    r_l = r - A z_a                                   (restricted to level 1)
//   PROLONG  t = z_a + P x_1 at the input; r_l = r - A t; dv = it D^-1 r_l; z_b = t + dv
//   FINISH   z_b += c1 dv + c2 D^-1 (r_l - A dv); rz = r.z_b; beta = rz / rz_old;
//            r_prev = r, p_prev = p (0 after the initialisation)
// Neighbours read r and p of the previous iteration while the current ones are written, so
// each has two buffers ([0] previous, [1] current).  it, c2, c1: Chebyshev coefficients of
// level 0 (device scalars of the hierarchy).
template <class T, int B>
struct OpDir {
  static constexpr int NR = 1;
  const T *z, *pold;
  T *pnew, *q;
  KrylovScal *sc;
  T beta;
  __device__ void begin() { beta = (T)sc->beta; }
  __device__ void in(size_t n, int, int, T (&v)[B]) const {
    T zz[B], pp[B];
    ldv<T, B>(z, n, zz);
    ldv<T, B>(pold, n, pp);
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = zz[k] + beta * pp[k];
  }
  __device__ void out(size_t n, const T (&o)[B], const T (&c)[B], T (&acc)[1]) const {
    stv<T, B>(pnew, n, c);
    stv<T, B>(q, n, o);
#pragma unroll
    for (int k = 0; k < B; ++k) acc[0] += c[k] * o[k];
  }
  __device__ bool reduce() const { return true; }
  __device__ void fin(const double (&tot)[1]) const { krylov_epilogue(EPI_CG_ALPHA, sc, tot[0]); }
};

template <class T, int B, bool INIT>
struct OpUpd {
  static constexpr int NR = 1;
  const T *rold, *q, *p, *invd, *coef;
  T *rnew, *x, *za;
  KrylovScal *sc;
  T alpha, it, c2, c1;
  __device__ void begin() {
    alpha = INIT ? T(0) : (T)sc->alpha;
    it = coef[0];
    c2 = coef[1];
    c1 = coef[2];
  }
  __device__ void rn(size_t n, T (&r)[B]) const {
    ldv<T, B>(rold, n, r);
    if (!INIT) {
      T qq[B];
      ldv<T, B>(q, n, qq);
#pragma unroll
      for (int k = 0; k < B; ++k) r[k] = r[k] - alpha * qq[k];
    }
  }
  __device__ void in(size_t n, int, int, T (&v)[B]) const {
    T r[B], iv[B];
    rn(n, r);
    ldv<T, B>(invd, n, iv);
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = iv[k] * r[k] * it;
  }
  __device__ void out(size_t n, const T (&o)[B], const T (&c)[B], T (&acc)[1]) const {
    T r[B], iv[B], z[B], xv[B];
    rn(n, r);
    ldv<T, B>(invd, n, iv);
#pragma unroll
    for (int k = 0; k < B; ++k) z[k] = c[k] + (c1 * c[k] + c2 * iv[k] * (r[k] - o[k]));
    stv<T, B>(za, n, z);
    stv<T, B>(rnew, n, r);
    if (INIT) {
#pragma unroll
      for (int k = 0; k < B; ++k) xv[k] = T(0);
    } else {
      T pp[B];
      ldv<T, B>(p, n, pp);
      ldv_rw<T, B>(x, n, xv);
#pragma unroll
      for (int k = 0; k < B; ++k) xv[k] = xv[k] + alpha * pp[k];
    }
    stv<T, B>(x, n, xv);
#pragma unroll
    for (int k = 0; k < B; ++k) acc[0] += r[k] * r[k];
  }
  __device__ bool reduce() const { return true; }
  __device__ void fin(const double (&tot)[1]) const {
    sc->rr = tot[0];
    if (INIT) {
      sc->rr0 = tot[0];
      sc->it = 0;
      sc->rz = 0.0;
      sc->breakdown = 0;
      sc->alpha = 0.0;
      sc->beta = 0.0;
    }
  }
};

template <class T, int B>
struct OpResid {
  static constexpr int NR = 0;
  const T *z, *rnew;
  T *lr;
  __device__ void begin() {}
  __device__ void in(size_t n, int, int, T (&v)[B]) const { ldv<T, B>(z, n, v); }
  __device__ void out(size_t n, const T (&o)[B], const T (&)[B], T (&)[1]) const {
    T r[B];
    ldv<T, B>(rnew, n, r);
#pragma unroll
    for (int k = 0; k < B; ++k) r[k] = r[k] - o[k];
    stv<T, B>(lr, n, r);
  }
  __device__ bool reduce() const { return false; }
  __device__ void fin(const double (&)[1]) const {}
};

template <class T, int B>
struct OpProlong {
  static constexpr int NR = 0;
  const T *za, *xc, *rnew, *invd, *coef;
  const uint8_t *fm;
  int nxc, nyc;
  T *zb, *lr, *dv;
  T it;
  __device__ void begin() { it = coef[0]; }
  // t = z_a + P x_1 on the free components (bilinear interpolation, coarse node I on fine 2I)
  __device__ void in(size_t n, int ix, int iy, T (&v)[B]) const {
    ldv<T, B>(za, n, v);
    const uint8_t m = __ldg(fm + n);
    if (!m) return;
    const int px0 = ix >> 1, py0 = iy >> 1;
    const int px1 = px0 + 1 <= nxc ? px0 + 1 : nxc, py1 = py0 + 1 <= nyc ? py0 + 1 : nyc;
    const T wx1 = (ix & 1) ? T(0.5) : T(0), wx0 = T(1) - wx1;
    const T wy1 = (iy & 1) ? T(0.5) : T(0), wy0 = T(1) - wy1;
    const size_t J00 = (size_t)py0 * (nxc + 1) + px0, J01 = (size_t)py0 * (nxc + 1) + px1;
    const size_t J10 = (size_t)py1 * (nxc + 1) + px0, J11 = (size_t)py1 * (nxc + 1) + px1;
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const T w = wy0 * (wx0 * __ldg(xc + B * J00 + c) + wx1 * __ldg(xc + B * J01 + c)) +
                  wy1 * (wx0 * __ldg(xc + B * J10 + c) + wx1 * __ldg(xc + B * J11 + c));
      if ((m >> c) & 1) v[c] += w;
    }
  }
  __device__ void out(size_t n, const T (&o)[B], const T (&c)[B], T (&)[1]) const {
    T r[B], iv[B], z[B], d[B];
    ldv<T, B>(rnew, n, r);
    ldv<T, B>(invd, n, iv);
#pragma unroll
    for (int k = 0; k < B; ++k) {
      r[k] = r[k] - o[k];
      d[k] = iv[k] * r[k] * it;
      z[k] = c[k] + d[k];
    }
    stv<T, B>(zb, n, z);
    stv<T, B>(lr, n, r);
    stv<T, B>(dv, n, d);
  }
  __device__ bool reduce() const { return false; }
  __device__ void fin(const double (&)[1]) const {}
};

template <class T, int B, bool FIRST>
struct OpFinish {
  static constexpr int NR = 1;
  const T *dv, *lr, *invd, *coef, *rnew, *pnew;
  T *zb, *rprev, *pprev;
  KrylovScal *sc;
  T c2, c1;
  __device__ void begin() {
    c2 = coef[1];
    c1 = coef[2];
  }
  __device__ void in(size_t n, int, int, T (&v)[B]) const { ldv<T, B>(dv, n, v); }
  __device__ void out(size_t n, const T (&o)[B], const T (&c)[B], T (&acc)[1]) const {
    T l[B], iv[B], z[B], r[B], p[B];
    ldv<T, B>(lr, n, l);
    ldv<T, B>(invd, n, iv);
    ldv_rw<T, B>(zb, n, z);
    ldv<T, B>(rnew, n, r);
#pragma unroll
    for (int k = 0; k < B; ++k) {
      z[k] = z[k] + (c1 * c[k] + c2 * iv[k] * (l[k] - o[k]));
      acc[0] += r[k] * z[k];
    }
    stv<T, B>(zb, n, z);
    // current residual and direction become the previous ones (the first direction uses
    // p_prev = 0)
    stv<T, B>(rprev, n, r);
    if (FIRST) {
#pragma unroll
      for (int k = 0; k < B; ++k) p[k] = T(0);
    } else {
      ldv<T, B>(pnew, n, p);
    }
    stv<T, B>(pprev, n, p);
  }
  __device__ bool reduce() const { return true; }
  __device__ void fin(const double (&tot)[1]) const {
    const double old = sc->rz;
    sc->beta = (!FIRST && old > 0.0 && isfinite(tot[0])) ? tot[0] / old : 0.0;
    sc->rz = tot[0];
    if (!(tot[0] > 0.0)) sc->breakdown = 1;
  }
};

}  // namespace pf
