// Geometric multigrid kernels: fine stencil assembly, Galerkin coarse operators,
// Chebyshev smoothing, transfer operators and the dense coarsest solve.
#include <math.h>
#include <string.h>

#include <vector>

#include "pf_gmg.cuh"
#include "pf_batch.cuh"
#include "pf_spectral.cuh"

namespace pf {

namespace {

__device__ __forceinline__ double gmg_gp(int hi) {
  return hi ? 0.78867513459481288225 : 0.21132486540518711775;
}


// Max over the grid into *out (red_grid, deterministic).
__device__ void grid_max(double v, const RedWs ws, double *out) {
  double a[1] = {v}, t[1];
  if (red_grid<1>(a, ws, t, true)) *out = t[0];
}

inline unsigned nblk(size_t n, int cap = 1 << 16) {
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > (size_t)cap) b = cap;
  return (unsigned)b;
}

template <int B>
__device__ __forceinline__ size_t sidx(int k, int r, int c, size_t node, size_t nn) {
  return sten_idx<B>(k, r, c, node, nn);
}

// ---- fine stencils ---------------------------------------------------------------------
// Row block of node n of the (unmasked) Q1 elasticity tangent.
template <class T>
__global__ void k_fine_stencil_elas(GridD g, MatD mt, const T *__restrict__ d,
                                    const uint8_t *__restrict__ tens, T *__restrict__ S) {
  const int nx = g.nx, ny = g.ny;
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy, w = 0.25 * g.hx * g.hy;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    double acc[9][4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[k][q] = 0.0;
#pragma unroll
    for (int ej_off = -1; ej_off <= 0; ++ej_off)
#pragma unroll
      for (int ei_off = -1; ei_off <= 0; ++ei_off) {
        const int ei = i + ei_off, ej = j + ej_off;
        if (ei < 0 || ei >= nx || ej < 0 || ej >= ny) continue;
        const size_t e = (size_t)ej * nx + ei;
        if (g.active && !g.active[e]) continue;
        const int ax = -ei_off, ay = -ej_off;  // local coords of node n in the element
        const int a = ay * 2 + ax;
        const size_t n0 = (size_t)ej * (nx + 1) + ei;
        const double dn[4] = {(double)d[n0], (double)d[n0 + 1], (double)d[n0 + nx + 1],
                              (double)d[n0 + nx + 2]};
        const uint8_t tb = tens[e];
        for (int q = 0; q < 4; ++q) {
          const double s = gmg_gp(q & 1), t = gmg_gp(q >> 1);
          const double s1 = 1 - s, t1 = 1 - t;
          const double dq = s1 * t1 * dn[0] + s * t1 * dn[1] + s1 * t * dn[2] + s * t * dn[3];
          const double om = 1 - dq, gq = om * om + mt.eta;
          const double kv = ((tb >> q) & 1) ? gq * mt.K : mt.K;
          const double D11 = gq * 2 * mt.mu * (1 - mt.cdim) + kv;
          const double D12 = -gq * 2 * mt.mu * mt.cdim + kv;
          const double Ds = gq * mt.mu;
          const double Nx[4] = {-t1 * ihx, t1 * ihx, -t * ihx, t * ihx};
          const double Ny[4] = {-s1 * ihy, -s * ihy, s1 * ihy, s * ihy};
          for (int b = 0; b < 4; ++b) {
            const int bx = b & 1, by = b >> 1;
            const int k = (by - ay + 1) * 3 + (bx - ax + 1);
            acc[k][0] += w * (Nx[a] * D11 * Nx[b] + Ny[a] * Ds * Ny[b]);
            acc[k][1] += w * (Nx[a] * D12 * Ny[b] + Ny[a] * Ds * Nx[b]);
            acc[k][2] += w * (Ny[a] * D12 * Nx[b] + Nx[a] * Ds * Ny[b]);
            acc[k][3] += w * (Ny[a] * D11 * Ny[b] + Nx[a] * Ds * Nx[b]);
          }
        }
      }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) S[sidx<2>(k, q >> 1, q & 1, n, nn)] = (T)acc[k][q];
  }
}

template <class T>
__global__ void k_fine_stencil_damage(GridD g, const T *__restrict__ c, double kappa,
                                      T *__restrict__ S) {
  const int nx = g.nx, ny = g.ny;
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy, w = 0.25 * g.hx * g.hy;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
#pragma unroll
    for (int ej_off = -1; ej_off <= 0; ++ej_off)
#pragma unroll
      for (int ei_off = -1; ei_off <= 0; ++ei_off) {
        const int ei = i + ei_off, ej = j + ej_off;
        if (ei < 0 || ei >= nx || ej < 0 || ej >= ny) continue;
        const size_t e = (size_t)ej * nx + ei;
        if (g.active && !g.active[e]) continue;
        const int ax = -ei_off, ay = -ej_off, a = ay * 2 + ax;
        for (int q = 0; q < 4; ++q) {
          const double s = gmg_gp(q & 1), t = gmg_gp(q >> 1);
          const double s1 = 1 - s, t1 = 1 - t;
          const double N[4] = {s1 * t1, s * t1, s1 * t, s * t};
          const double Nx[4] = {-t1 * ihx, t1 * ihx, -t * ihx, t * ihx};
          const double Ny[4] = {-s1 * ihy, -s * ihy, s1 * ihy, s * ihy};
          const double cq = (double)c[4 * e + q];
          for (int b = 0; b < 4; ++b) {
            const int k = ((b >> 1) - ay + 1) * 3 + ((b & 1) - ax + 1);
            acc[k] += w * (cq * N[a] * N[b] + kappa * (Nx[a] * Nx[b] + Ny[a] * Ny[b]));
          }
        }
      }
#pragma unroll
    for (int k = 0; k < 9; ++k) S[sidx<1>(k, 0, 0, n, nn)] = (T)acc[k];
  }
}

// Level-0 free mask from the DOF mask: bit c = component c free.
template <int B>
__global__ void k_fm0(size_t nn, const uint8_t *__restrict__ dofm, uint8_t *__restrict__ fm) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const uint8_t m = dofm ? dofm[n] : 0;
    fm[n] = (B == 2) ? (uint8_t)(~m & 3) : (uint8_t)((m & 4) ? 0 : 1);
  }
}

// Inverse diagonal, free mask (diag > 0 and previously free) and Gershgorin bound of
// D^-1 A over free rows/columns.
template <class T, int B>
__global__ void k_diag_bound(int nx, int ny, const T *__restrict__ S, uint8_t *__restrict__ fm,
                             T *__restrict__ invd) {
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    uint8_t f = fm[n];
    uint8_t fnew = 0;
    for (int r = 0; r < B; ++r) {
      const double a = (double)S[sidx<B>(4, r, r, n, nn)];
      const bool free_r = ((f >> r) & 1) && a > 0.0;
      invd[B * n + r] = free_r ? (T)(1.0 / a) : T(0);
      if (free_r) fnew |= (uint8_t)(1u << r);
    }
    fm[n] = fnew;
  }
}

template <class T, int B>
__global__ void k_bound(int nx, int ny, const T *__restrict__ S, const uint8_t *__restrict__ fm,
                        RedWs ws, double *lmax) {
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  double bound = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    const uint8_t f = fm[n];
    for (int r = 0; r < B; ++r) {
      if (!((f >> r) & 1)) continue;
      double rs = 0.0;
      for (int k = 0; k < 9; ++k) {
        const int di = k % 3 - 1, dj = k / 3 - 1;
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii > nx || jj < 0 || jj > ny) continue;
        const uint8_t fn = fm[(size_t)jj * (nx + 1) + ii];
        for (int c = 0; c < B; ++c)
          if ((fn >> c) & 1) rs += fabs((double)S[sidx<B>(k, r, c, n, nn)]);
      }
      bound = fmax(bound, rs / (double)S[sidx<B>(4, r, r, n, nn)]);
    }
  }
  grid_max(bound, ws, lmax);
}

// Chebyshev coefficients of a level in its arithmetic type, from the FP64 bound:
// coef = {1/theta, 2 rho1/delta, rho1 rho0} with theta = 0.55 lmax, delta = 0.45 lmax,
// rho0 = 1/sigma = 9/11, rho1 = 1/(2 sigma - rho0) = 99/161.
template <class T>
__global__ void k_cheb_coef(const double *lmax, T *coef) {
  const double lm = *lmax > 0.0 ? *lmax : 1.0;
  const double rho0 = 9.0 / 11.0, rho1 = 99.0 / 161.0;
  coef[0] = (T)(1.0 / (0.55 * lm));
  coef[1] = (T)(2.0 * rho1 / (0.45 * lm));
  coef[2] = (T)(rho1 * rho0);
}

// Galerkin product A_c = P^T A_f P with P bilinear, rows of non-free fine DOFs removed.
template <class T, int B>
__global__ void k_rap(int nxf, int nyf, const T *__restrict__ Sf, const uint8_t *__restrict__ fmf,
                      int nxc, int nyc, T *__restrict__ Sc) {
  const size_t nnf = (size_t)(nxf + 1) * (nyf + 1);
  const size_t nnc = (size_t)(nxc + 1) * (nyc + 1);
  for (size_t I = blockIdx.x * (size_t)blockDim.x + threadIdx.x; I < nnc;
       I += (size_t)gridDim.x * blockDim.x) {
    const int Ix = (int)(I % (nxc + 1)), Iy = (int)(I / (nxc + 1));
    double acc[9][B * B];
    for (int k = 0; k < 9; ++k)
      for (int q = 0; q < B * B; ++q) acc[k][q] = 0.0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b) {
        const int ix = 2 * Ix + a, iy = 2 * Iy + b;
        if (ix < 0 || ix > nxf || iy < 0 || iy > nyf) continue;
        const double wi = (a == 0 ? 1.0 : 0.5) * (b == 0 ? 1.0 : 0.5);
        const size_t fi = (size_t)iy * (nxf + 1) + ix;
        const uint8_t mi = fmf[fi];
        if (!mi) continue;
        for (int k = 0; k < 9; ++k) {
          const int jx = ix + k % 3 - 1, jy = iy + k / 3 - 1;
          if (jx < 0 || jx > nxf || jy < 0 || jy > nyf) continue;
          const uint8_t mj = fmf[(size_t)jy * (nxf + 1) + jx];
          if (!mj) continue;
          double av[B * B];
          for (int r = 0; r < B; ++r)
            for (int c = 0; c < B; ++c)
              av[r * B + c] = (((mi >> r) & 1) && ((mj >> c) & 1))
                                  ? (double)Sf[sidx<B>(k, r, c, fi, nnf)] : 0.0;
          // coarse parents of (jx, jy)
          const int px0 = jx >> 1, py0 = jy >> 1;
          const int npx = (jx & 1) ? 2 : 1, npy = (jy & 1) ? 2 : 1;
          for (int u = 0; u < npx; ++u)
            for (int v = 0; v < npy; ++v) {
              const int Jx = px0 + u, Jy = py0 + v;
              const double wj = (npx == 2 ? 0.5 : 1.0) * (npy == 2 ? 0.5 : 1.0);
              const int kc = (Jy - Iy + 1) * 3 + (Jx - Ix + 1);
              for (int q = 0; q < B * B; ++q) acc[kc][q] += wi * wj * av[q];
            }
        }
      }
    for (int k = 0; k < 9; ++k)
      for (int q = 0; q < B * B; ++q) Sc[sidx<B>(k, q / B, q % B, I, nnc)] = (T)acc[k][q];
  }
}

// Coarse free mask before the diagonal test: a coarse DOF is a candidate if any fine
// child DOF of that component is free.
template <int B>
__global__ void k_fm_coarse(int nxf, int nyf, const uint8_t *__restrict__ fmf, int nxc, int nyc,
                            uint8_t *__restrict__ fmc) {
  const size_t nnc = (size_t)(nxc + 1) * (nyc + 1);
  for (size_t I = blockIdx.x * (size_t)blockDim.x + threadIdx.x; I < nnc;
       I += (size_t)gridDim.x * blockDim.x) {
    const int Ix = (int)(I % (nxc + 1)), Iy = (int)(I / (nxc + 1));
    uint8_t m = 0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b) {
        const int ix = 2 * Ix + a, iy = 2 * Iy + b;
        if (ix < 0 || ix > nxf || iy < 0 || iy > nyf) continue;
        m |= fmf[(size_t)iy * (nxf + 1) + ix];
      }
    fmc[I] = m;
  }
}

// (A x)_n for one node: vectors are zero on non-free DOFs at every level, so the
// neighbours' masks are not needed; out-of-grid neighbours have no stencil entry.
// xat(i) returns entry i of x, so callers choose the load path (read-only cache for
// vectors no thread rewrites during the kernel, L2 for vectors other CTAs rewrite) or
// form x on the fly.
template <class T, int B, class XAt>
__device__ __forceinline__ void sten_row_by(int nx, int ny, size_t nn, const T *__restrict__ S,
                                            size_t n, XAt xat, T (&acc)[B]) {
  // Stencil entries towards neighbours outside the grid are zero, so neighbour indices are
  // clamped into the grid instead of branched on: all loads issue back to back.
  const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
  const int im = i > 0 ? i - 1 : 0, ip = i < nx ? i + 1 : nx;
  const int jm = j > 0 ? j - 1 : 0, jp = j < ny ? j + 1 : ny;
  const int ld = nx + 1;
  const size_t m[9] = {(size_t)jm * ld + im, (size_t)jm * ld + i, (size_t)jm * ld + ip,
                       (size_t)j * ld + im,  (size_t)j * ld + i,  (size_t)j * ld + ip,
                       (size_t)jp * ld + im, (size_t)jp * ld + i, (size_t)jp * ld + ip};
  T xv[9][B];
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int c = 0; c < B; ++c) xv[k][c] = xat(B * m[k] + c);
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int c = 0; c < B; ++c)
#pragma unroll
      for (int r = 0; r < B; ++r) acc[r] += __ldg(S + sidx<B>(k, r, c, n, nn)) * xv[k][c];
}

// x is not written while the kernel runs: read-only data path.
template <class T, int B>
__device__ __forceinline__ void sten_row(int nx, int ny, size_t nn, const T *__restrict__ S,
                                         const T *__restrict__ x, size_t n, T (&acc)[B]) {
  sten_row_by<T, B>(nx, ny, nn, S, n, [x](size_t q) { return __ldg(x + q); }, acc);
}

// y = A x  (mode 0) or y = b - A x (mode 1), rows of non-free DOFs zero.
template <class T, int B>
struct StenApplyF {
  int nx, ny;
  const T *__restrict__ S;
  const uint8_t *__restrict__ fm;
  const T *__restrict__ x;
  const T *__restrict__ b;
  T *__restrict__ y;
  int mode;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    const size_t nn = (size_t)(nx + 1) * (ny + 1);
    for (size_t n = bid * (size_t)blockDim.x + threadIdx.x; n < nn;
         n += (size_t)nblk * blockDim.x) {
      T acc[B];
      sten_row<T, B>(nx, ny, nn, S, x, n, acc);
      const uint8_t f = fm[n];
#pragma unroll
      for (int r = 0; r < B; ++r) {
        T v = mode ? b[B * n + r] - acc[r] : acc[r];
        y[B * n + r] = ((f >> r) & 1) ? v : T(0);
      }
    }
  }
};
template <class T, int B>
__global__ void k_sten_apply(StenApplyF<T, B> f) {
  pdl_enter();
  f(blockIdx.x, gridDim.x);
}


// ---- fused smoothing kernels of the grid-wide stencil levels ------------------------------
// Pre-smoothing from x = 0 in one pass: d0 = it D^-1 b is formed at the neighbours, so
// x = d0 + c1 d0 + c2 D^-1 (b - A d0) needs no stored d0 or residual.
template <class T, int B>
struct StenPreF {
  int nx, ny;
  const T *__restrict__ S;
  const T *__restrict__ invd;
  const T *coef;
  const uint8_t *__restrict__ fm;
  const T *__restrict__ b;
  T *__restrict__ x;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    const T *__restrict__ invd = this->invd, *__restrict__ b = this->b;
    const size_t nn = (size_t)(nx + 1) * (ny + 1);
    const T it = coef[0], c2 = coef[1], c1 = coef[2];
    for (size_t n = bid * (size_t)blockDim.x + threadIdx.x; n < nn;
         n += (size_t)nblk * blockDim.x) {
      T acc[B];
      sten_row_by<T, B>(nx, ny, nn, S, n,
                        [=](size_t q) { return __ldg(invd + q) * __ldg(b + q) * it; }, acc);
      const uint8_t f = __ldg(fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        const T iv = __ldg(invd + i), bi = __ldg(b + i);
        const T d0 = iv * bi * it;
        const T d1 = c1 * d0 + c2 * iv * (bi - acc[c]);
        x[i] = ((f >> c) & 1) ? d0 + d1 : T(0);
      }
    }
  }
};
template <class T, int B>
__global__ void k_sten_pre(StenPreF<T, B> f) {
  pdl_enter();
  f(blockIdx.x, gridDim.x);
}

// Bilinear prolongation of the coarse correction at fine node (ix, iy), component c.
template <class T, int B>
__device__ __forceinline__ T prolong_at(int ix, int iy, int nxc, int nyc, const T *__restrict__ xc,
                                        int c) {
  const int px0 = ix >> 1, py0 = iy >> 1;
  const int px1 = px0 + 1 <= nxc ? px0 + 1 : nxc, py1 = py0 + 1 <= nyc ? py0 + 1 : nyc;
  const T wx1 = (ix & 1) ? T(0.5) : T(0), wx0 = T(1) - wx1;
  const T wy1 = (iy & 1) ? T(0.5) : T(0), wy0 = T(1) - wy1;
  const size_t J00 = (size_t)py0 * (nxc + 1) + px0, J01 = (size_t)py0 * (nxc + 1) + px1;
  const size_t J10 = (size_t)py1 * (nxc + 1) + px0, J11 = (size_t)py1 * (nxc + 1) + px1;
  return wy0 * (wx0 * __ldg(xc + B * J00 + c) + wx1 * __ldg(xc + B * J01 + c)) +
         wy1 * (wx0 * __ldg(xc + B * J10 + c) + wx1 * __ldg(xc + B * J11 + c));
}

// Coarse-grid correction and first post-smoothing step in one pass: t = x_in + P x_c on the
// free components is formed at the neighbours; r = b - A t, d = it D^-1 r, x_out = t + d.
template <class T, int B>
struct StenProlongFirstF {
  int nx, ny;
  const T *__restrict__ S;
  const T *__restrict__ invd;
  const T *coef;
  const uint8_t *__restrict__ fm;
  int nxc, nyc;
  const T *__restrict__ xc;
  const T *__restrict__ b;
  const T *__restrict__ xin;
  T *__restrict__ xout;
  T *__restrict__ r;
  T *__restrict__ d;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    const T *__restrict__ xin = this->xin, *__restrict__ xc = this->xc;
    const uint8_t *__restrict__ fm = this->fm;
    const int nxc = this->nxc, nyc = this->nyc;
    const size_t nn = (size_t)(nx + 1) * (ny + 1);
    const int ld = nx + 1;
    const T it = coef[0];
    auto t_at = [=](size_t q) {
      const size_t m = q / B;
      const int c = (int)(q - m * B);
      T v = __ldg(xin + q);
      if ((__ldg(fm + m) >> c) & 1)
        v += prolong_at<T, B>((int)(m % ld), (int)(m / ld), nxc, nyc, xc, c);
      return v;
    };
    for (size_t n = bid * (size_t)blockDim.x + threadIdx.x; n < nn;
         n += (size_t)nblk * blockDim.x) {
      T acc[B];
      sten_row_by<T, B>(nx, ny, nn, S, n, t_at, acc);
      const uint8_t f = __ldg(fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        const T ri = ((f >> c) & 1) ? __ldg(b + i) - acc[c] : T(0);
        const T di = __ldg(invd + i) * ri * it;
        r[i] = ri;
        d[i] = di;
        xout[i] = t_at(i) + di;
      }
    }
  }
};
template <class T, int B>
__global__ void k_sten_prolong_first(StenProlongFirstF<T, B> f) {
  pdl_enter();
  f(blockIdx.x, gridDim.x);
}

// Second post-smoothing step: x += c1 d + c2 D^-1 (r - A d).
template <class T, int B>
struct StenPostF {
  int nx, ny;
  const T *__restrict__ S;
  const T *__restrict__ invd;
  const T *coef;
  const uint8_t *__restrict__ fm;
  const T *__restrict__ d;
  const T *__restrict__ r;
  T *__restrict__ x;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    const size_t nn = (size_t)(nx + 1) * (ny + 1);
    const T c2 = coef[1], c1 = coef[2];
    for (size_t n = bid * (size_t)blockDim.x + threadIdx.x; n < nn;
         n += (size_t)nblk * blockDim.x) {
      T acc[B];
      sten_row<T, B>(nx, ny, nn, S, d, n, acc);
      const uint8_t f = __ldg(fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        const T ri = __ldg(r + i) - (((f >> c) & 1) ? acc[c] : T(0));
        x[i] = x[i] + (c1 * __ldg(d + i) + c2 * __ldg(invd + i) * ri);
      }
    }
  }
};
template <class T, int B>
__global__ void k_sten_post(StenPostF<T, B> f) {
  pdl_enter();
  f(blockIdx.x, gridDim.x);
}

// ---- coarse levels in one CTA --------------------------------------------------------------
template <class T>
struct CoarseLevel {
  int nx, ny;
  const T *S, *invd;
  T *x, *b, *r, *d, *y;
  const uint8_t *fm;
  const T *coef;
};
template <class T>
struct CoarseArgs {
  int nlev;                 // number of levels handled (the last one is solved densely)
  CoarseLevel<T> L[GMG_MAX_LEVELS];
  const T *b0;              // right-hand side of the first handled level
  T *x0;                    // solution of the first handled level
  const T *cinv;
  int ncoarse;
};

template <class T>
__device__ __forceinline__ T ld_(const T *p) { return *p; }
template <class T>
__device__ __forceinline__ void st_(T *p, T v) { *p = v; }

// One V-cycle over levels [0, nlev) of `a` in one CTA of COARSE_THREADS threads.  Every
// phase is a node loop over the CTA followed by a barrier; thread t owns the same nodes in
// every phase.  Chebyshev steps are fused so that each level costs three barriers on the
// way down and three on the way up:
//   down: x = d0 + c1 d0 + c2 D^-1 (b - A d0), d0 = it D^-1 b formed at the neighbours;
//         r = b - A x;  b_coarse = P^T r
//   up:   x += P x_coarse;  r = b - A x, d = it D^-1 r;  x = (x + d) + c1 d + c2 D^-1 (r - A d)
template <class T, int B>
__device__ __forceinline__ void coarse_cycle_body(const CoarseArgs<T> &a) {
  const size_t t0 = threadIdx.x, nt = blockDim.x;
  const int last = a.nlev - 1;
  for (int l = 0; l < last; ++l) {
    const CoarseLevel<T> &L = a.L[l];
    const T *b = l == 0 ? a.b0 : L.b;
    T *x = l == 0 ? a.x0 : L.x;
    const size_t nn = (size_t)(L.nx + 1) * (L.ny + 1);
    const T it = L.coef[0], c2 = L.coef[1], c1 = L.coef[2];
    const T *invd = L.invd;
    for (size_t n = t0; n < nn; n += nt) {
      T acc[B];
      sten_row_by<T, B>(L.nx, L.ny, nn, L.S, n,
                        [=](size_t q) { return __ldg(invd + q) * ld_(b + q) * it; }, acc);
      const uint8_t f = __ldg(L.fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        const T iv = __ldg(invd + i), bi = ld_(b + i);
        const T d0 = iv * bi * it;
        const T d1 = c1 * d0 + c2 * iv * (bi - acc[c]);
        st_(x + i, ((f >> c) & 1) ? d0 + d1 : T(0));
      }
    }
    __syncthreads();
    for (size_t n = t0; n < nn; n += nt) {
      T acc[B];
      const T *xr = x;
      sten_row_by<T, B>(L.nx, L.ny, nn, L.S, n, [=](size_t q) { return ld_(xr + q); }, acc);
      const uint8_t f = __ldg(L.fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        st_(L.r + i, ((f >> c) & 1) ? ld_(b + i) - acc[c] : T(0));
      }
    }
    __syncthreads();
    // restrict r -> b of level l+1
    const CoarseLevel<T> &C = a.L[l + 1];
    const size_t nnc = (size_t)(C.nx + 1) * (C.ny + 1);
    for (size_t I = t0; I < nnc; I += nt) {
      const int Ix = (int)(I % (C.nx + 1)), Iy = (int)(I / (C.nx + 1));
      T acc[B];
#pragma unroll
      for (int c = 0; c < B; ++c) acc[c] = T(0);
      for (int p = -1; p <= 1; ++p)
        for (int q = -1; q <= 1; ++q) {
          const int ix = 2 * Ix + p, iy = 2 * Iy + q;
          if (ix < 0 || ix > L.nx || iy < 0 || iy > L.ny) continue;
          const T wi = (p == 0 ? T(1) : T(0.5)) * (q == 0 ? T(1) : T(0.5));
          const size_t fi = (size_t)iy * (L.nx + 1) + ix;
#pragma unroll
          for (int c = 0; c < B; ++c) acc[c] += wi * ld_(L.r + B * fi + c);
        }
      const uint8_t mc = __ldg(C.fm + I);
#pragma unroll
      for (int c = 0; c < B; ++c) st_(C.b + B * I + c, ((mc >> c) & 1) ? acc[c] : T(0));
    }
    __syncthreads();
  }
  // dense solve on the last level: one warp per row
  {
    const CoarseLevel<T> &C = a.L[last];
    const T *b = last == 0 ? a.b0 : C.b;
    T *x = last == 0 ? a.x0 : C.x;
    const int lane = threadIdx.x & 31;
    const size_t warp = t0 >> 5, nw = nt >> 5;
    for (size_t i = warp; i < (size_t)a.ncoarse; i += nw) {
      T s = T(0);
      for (int j = lane; j < a.ncoarse; j += 32)
        s += __ldg(a.cinv + i * a.ncoarse + j) * ld_(b + j);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) st_(x + i, s);
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const CoarseLevel<T> &L = a.L[l];
    const CoarseLevel<T> &C = a.L[l + 1];
    const T *b = l == 0 ? a.b0 : L.b;
    T *x = l == 0 ? a.x0 : L.x;
    const T *xc = C.x;
    const size_t nn = (size_t)(L.nx + 1) * (L.ny + 1);
    for (size_t nf = t0; nf < nn; nf += nt) {
      const uint8_t m = __ldg(L.fm + nf);
      if (!m) continue;
      const int ix = (int)(nf % (L.nx + 1)), iy = (int)(nf / (L.nx + 1));
      const int px0 = ix >> 1, py0 = iy >> 1, npx = (ix & 1) ? 2 : 1, npy = (iy & 1) ? 2 : 1;
      T acc[B];
#pragma unroll
      for (int c = 0; c < B; ++c) acc[c] = T(0);
      for (int u = 0; u < npx; ++u)
        for (int v = 0; v < npy; ++v) {
          const T wj = (npx == 2 ? T(0.5) : T(1)) * (npy == 2 ? T(0.5) : T(1));
          const size_t J = (size_t)(py0 + v) * (C.nx + 1) + (px0 + u);
#pragma unroll
          for (int c = 0; c < B; ++c) acc[c] += wj * ld_(xc + B * J + c);
        }
#pragma unroll
      for (int c = 0; c < B; ++c)
        if ((m >> c) & 1) st_(x + B * nf + c, ld_(x + B * nf + c) + acc[c]);
    }
    __syncthreads();
    const T it = L.coef[0], c2 = L.coef[1], c1 = L.coef[2];
    const T *invd = L.invd;
    for (size_t n = t0; n < nn; n += nt) {
      T acc[B];
      const T *xr = x;
      sten_row_by<T, B>(L.nx, L.ny, nn, L.S, n, [=](size_t q) { return ld_(xr + q); }, acc);
      const uint8_t f = __ldg(L.fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        const T ri = ((f >> c) & 1) ? ld_(b + i) - acc[c] : T(0);
        st_(L.r + i, ri);
        st_(L.d + i, __ldg(invd + i) * ri * it);
      }
    }
    __syncthreads();
    for (size_t n = t0; n < nn; n += nt) {
      T acc[B];
      const T *dr = L.d;
      sten_row_by<T, B>(L.nx, L.ny, nn, L.S, n, [=](size_t q) { return ld_(dr + q); }, acc);
      const uint8_t f = __ldg(L.fm + n);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const size_t i = B * n + c;
        const T di = ld_(L.d + i);
        const T ri = ld_(L.r + i) - (((f >> c) & 1) ? acc[c] : T(0));
        const T d2 = c1 * di + c2 * __ldg(invd + i) * ri;
        st_(x + i, (ld_(x + i) + di) + d2);
      }
    }
    if (l > 0) __syncthreads();
  }
}

template <class T, int B>
__global__ void __launch_bounds__(COARSE_THREADS) k_coarse_cycle(CoarseArgs<T> a) {
  pdl_enter();
  coarse_cycle_body<T, B>(a);
}

// One simulation's coarse cycle in a batched launch: one CTA, arguments in device memory.
template <class T, int B>
struct CoarseF {
  const CoarseArgs<T> *a;
  __device__ void operator()(unsigned, unsigned) const { coarse_cycle_body<T, B>(*a); }
};

// Chebyshev on [lmax/10, lmax]: theta = 0.55 lmax, delta = 0.45 lmax, sigma = 11/9.
// first step from x = 0: d = D^-1 b / theta; x = d; r = b
template <class T>
__global__ void k_cheb_first(size_t n, const T *__restrict__ b, const T *__restrict__ invd,
                             const T *coef, T *__restrict__ x, T *__restrict__ d,
                             T *__restrict__ r) {
  const T it = coef[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T bi = b[i];
    const T di = invd[i] * bi * it;
    d[i] = di;
    x[i] = di;
    r[i] = bi;
  }
}
// first step from x != 0 with y = A x: r = b - y; d = D^-1 r / theta; x += d
template <class T>
__global__ void k_cheb_first_x(size_t n, const T *__restrict__ b, const T *__restrict__ y,
                               const T *__restrict__ invd, const T *coef, T *__restrict__ x,
                               T *__restrict__ d, T *__restrict__ r) {
  const T it = coef[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T ri = b[i] - y[i];
    const T di = invd[i] * ri * it;
    r[i] = ri;
    d[i] = di;
    x[i] += di;
  }
}
// later step with y = A d: r -= y; d = c1 d + c2 D^-1 r; x += d
template <class T>
__global__ void k_cheb_step(size_t n, const T *__restrict__ y, const T *__restrict__ invd,
                            const T *coef, T *__restrict__ x, T *__restrict__ d,
                            T *__restrict__ r) {
  const T a = coef[2], bb = coef[1];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T ri = r[i] - y[i];
    const T di = a * d[i] + bb * invd[i] * ri;
    r[i] = ri;
    d[i] = di;
    x[i] += di;
  }
}
// r = b - y
template <class T>
__global__ void k_sub(size_t n, const T *__restrict__ b, const T *__restrict__ y, T *__restrict__ r) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}

// b_c = P^T r_f over free DOFs (out-of-grid fine neighbours: clamped index, weight 0).
template <class T, int B>
struct RestrictF {
  int nxf, nyf;
  const T *__restrict__ rf;
  const uint8_t *__restrict__ fmf;
  int nxc, nyc;
  const uint8_t *__restrict__ fmc;
  T *__restrict__ bc;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    const size_t nnc = (size_t)(nxc + 1) * (nyc + 1);
    for (size_t I = bid * (size_t)blockDim.x + threadIdx.x; I < nnc;
         I += (size_t)nblk * blockDim.x) {
      const int Ix = (int)(I % (nxc + 1)), Iy = (int)(I / (nxc + 1));
      T acc[B];
#pragma unroll
      for (int c = 0; c < B; ++c) acc[c] = T(0);
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const int iy = 2 * Iy + b;
        const bool vy = iy >= 0 && iy <= nyf;
        const int iyc = iy < 0 ? 0 : (iy > nyf ? nyf : iy);
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
          const int ix = 2 * Ix + a;
          const bool v = vy && ix >= 0 && ix <= nxf;
          const int ixc = ix < 0 ? 0 : (ix > nxf ? nxf : ix);
          const T wi = v ? (a == 0 ? T(1) : T(0.5)) * (b == 0 ? T(1) : T(0.5)) : T(0);
          const size_t fi = (size_t)iyc * (nxf + 1) + ixc;
          const uint8_t m = __ldg(fmf + fi);
#pragma unroll
          for (int c = 0; c < B; ++c) {
            const T rv = __ldg(rf + B * fi + c);
            acc[c] += ((m >> c) & 1) ? wi * rv : T(0);
          }
        }
      }
      const uint8_t mc = fmc[I];
#pragma unroll
      for (int c = 0; c < B; ++c) bc[B * I + c] = ((mc >> c) & 1) ? acc[c] : T(0);
    }
  }
};
template <class T, int B>
__global__ void k_restrict(RestrictF<T, B> f) {
  pdl_enter();
  f(blockIdx.x, gridDim.x);
}

// x_f += P x_c over free fine DOFs (always four parents, out-of-grid ones weighted 0).
template <class T, int B>
__global__ void k_prolong_add(int nxf, int nyf, const uint8_t *__restrict__ fmf, int nxc,
                              const T *__restrict__ xc, T *__restrict__ xf) {
  const size_t nnf = (size_t)(nxf + 1) * (nyf + 1);
  const int nyc = (nyf + 1) / 2;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nnf;
       n += (size_t)gridDim.x * blockDim.x) {
    const uint8_t m = fmf[n];
    if (!m) continue;
    const int ix = (int)(n % (nxf + 1)), iy = (int)(n / (nxf + 1));
    const int px0 = ix >> 1, py0 = iy >> 1;
    const int px1 = px0 + 1 <= nxc ? px0 + 1 : nxc, py1 = py0 + 1 <= nyc ? py0 + 1 : nyc;
    const T wx1 = (ix & 1) ? T(0.5) : T(0), wx0 = T(1) - wx1;
    const T wy1 = (iy & 1) ? T(0.5) : T(0), wy0 = T(1) - wy1;
    const size_t J00 = (size_t)py0 * (nxc + 1) + px0, J01 = (size_t)py0 * (nxc + 1) + px1;
    const size_t J10 = (size_t)py1 * (nxc + 1) + px0, J11 = (size_t)py1 * (nxc + 1) + px1;
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const T v = wy0 * (wx0 * __ldg(xc + B * J00 + c) + wx1 * __ldg(xc + B * J01 + c)) +
                  wy1 * (wx0 * __ldg(xc + B * J10 + c) + wx1 * __ldg(xc + B * J11 + c));
      if ((m >> c) & 1) xf[B * n + c] += v;
    }
  }
}

// Dense inverse of the coarsest level in one CTA, in FP64: assemble the level's stencil
// as a dense matrix (rows of non-free DOFs: identity), symmetrise it (the Galerkin product
// is symmetric up to rounding), invert it in place by Gauss-Jordan elimination without
// pivoting (the matrix is SPD; a pivot below 1e-14 of the largest diagonal entry is lifted
// to that value), and write the inverse in T with the rows and columns of non-free DOFs
// zeroed, so the coarse correction vanishes there.  A: n x n FP64 work array; n <= 256.
constexpr int COARSE_INV_MAX = 256;
template <class T, int B>
__global__ void __launch_bounds__(1024) k_coarse_inverse(int nx, int ny, const T *__restrict__ S,
                                                         const uint8_t *__restrict__ fm, int n,
                                                         double *__restrict__ A,
                                                         T *__restrict__ cinv) {
  __shared__ double colk[COARSE_INV_MAX], rowk[COARSE_INV_MAX], red[32];
  __shared__ double pinv_s, floor_s;
  const int t = threadIdx.x, nt = blockDim.x;
  const size_t nn = (size_t)(nx + 1) * (ny + 1), n2 = (size_t)n * n;
  auto is_free = [&](int row) { return (__ldg(fm + row / B) >> (row % B)) & 1; };
  for (size_t q = t; q < n2; q += nt) A[q] = 0.0;
  __syncthreads();
  for (int row = t; row < n; row += nt) {
    const size_t node = (size_t)(row / B);
    const int r = row % B;
    if (!is_free(row)) {
      A[(size_t)row * n + row] = 1.0;
      continue;
    }
    const int i = (int)(node % (nx + 1)), j = (int)(node / (nx + 1));
    for (int k = 0; k < 9; ++k) {
      const int ii = i + k % 3 - 1, jj = j + k / 3 - 1;
      if (ii < 0 || ii > nx || jj < 0 || jj > ny) continue;
      const size_t m = (size_t)jj * (nx + 1) + ii;
      for (int c = 0; c < B; ++c)
        if ((__ldg(fm + m) >> c) & 1)
          A[(size_t)row * n + (B * m + c)] = (double)S[sten_idx<B>(k, r, c, node, nn)];
    }
  }
  __syncthreads();
  for (size_t q = t; q < n2; q += nt) {
    const size_t i = q / n, j = q % n;
    if (i < j) {
      const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = A[j * n + i] = v;
    }
  }
  __syncthreads();
  double dm = 0.0;
  for (int i = t; i < n; i += nt) dm = fmax(dm, A[(size_t)i * n + i]);
  dm = red_warp(dm, true);
  if ((t & 31) == 0) red[t >> 5] = dm;
  __syncthreads();
  if (t == 0) {
    double m = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) m = fmax(m, red[w]);
    floor_s = (m > 0.0 ? m : 1.0) * 1e-14;
  }
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    for (int i = t; i < n; i += nt) colk[i] = A[(size_t)i * n + k];
    if (t == 0) {
      double p = A[(size_t)k * n + k];
      if (!(p > floor_s)) p = floor_s;
      pinv_s = 1.0 / p;
    }
    __syncthreads();
    const double pinv = pinv_s;
    for (int j = t; j < n; j += nt) {
      const double v = (j == k ? 1.0 : A[(size_t)k * n + j]) * pinv;
      rowk[j] = v;
      A[(size_t)k * n + j] = v;
    }
    __syncthreads();
    for (size_t q = t; q < n2; q += nt) {
      const int i = (int)(q / n), j = (int)(q % n);
      if (i == k) continue;
      A[q] = (j == k ? 0.0 : A[q]) - colk[i] * rowk[j];
    }
  }
  __syncthreads();
  for (size_t q = t; q < n2; q += nt) {
    const int i = (int)(q / n), j = (int)(q % n);
    cinv[q] = (is_free(i) && is_free(j)) ? (T)A[q] : T(0);
  }
}

}  // namespace

// ---- host side ------------------------------------------------------------------------------
template <class T>
cudaError_t gmg_alloc(Gmg<T> &G, int nx, int ny, int B, const RedWs &ws, Arena &A) {
  G.B = B;
  G.ws = ws;
  int l = 0;
  int cx = nx, cy = ny;
  while (true) {
    GmgLevel<T> &L = G.lv[l];
    L.nx = cx;
    L.ny = cy;
    L.nn = (size_t)(cx + 1) * (cy + 1);
    const size_t nb = (size_t)B * L.nn;
    G.nl = l + 1;
    if (!A.take(&L.S, 9 * B * B * L.nn)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.invd, nb)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.x, nb)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.b, nb)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.r, nb)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.dv, nb)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.y, nb)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.fm, L.nn)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.lmax, 1)) return cudaErrorMemoryAllocation;
    if (!A.take(&L.coef, 4)) return cudaErrorMemoryAllocation;
    ++l;
    if ((cx <= GMG_COARSE_MAX && cy <= GMG_COARSE_MAX) || l == GMG_MAX_LEVELS) break;
    cx = (cx + 1) / 2;
    cy = (cy + 1) / 2;
  }
  G.nl = l;
  G.lc = G.nl - 1;
  for (int k = 0; k < G.nl; ++k)
    if (G.lv[k].nn <= (size_t)GMG_CTA_NODES) {
      G.lc = k;
      break;
    }
  const GmgLevel<T> &C = G.lv[l - 1];
  G.ncoarse = (int)(B * C.nn);
  if (G.ncoarse > COARSE_INV_MAX) return cudaErrorInvalidValue;
  const size_t n2 = (size_t)G.ncoarse * G.ncoarse;
  if (!A.take(&G.cinv, n2) || !A.take(&G.cwork, n2)) return cudaErrorMemoryAllocation;
  return cudaSuccess;
}

// The hierarchy's arrays belong to the owner's arena; only the batched coarse-cycle
// arguments are allocated separately.
template <class T>
void gmg_free(Gmg<T> &G) {
  for (int l = 0; l < G.nl; ++l) G.lv[l] = GmgLevel<T>();
  if (G.dca) cudaFree(G.dca);
  G.dca = nullptr;
  G.cinv = nullptr;
  G.cwork = nullptr;
  G.nl = 0;
}

template <class T, int B>
static cudaError_t gmg_setup_common(Gmg<T> &G, const GridD &g, cudaStream_t st) {
  // level 0 mask, diagonal, bound
  GmgLevel<T> &L0 = G.lv[0];
  k_fm0<B><<<nblk(L0.nn), 256, 0, st>>>(L0.nn, g.dofm, L0.fm);
  for (int l = 0; l < G.nl; ++l) {
    GmgLevel<T> &L = G.lv[l];
    if (l > 0) {
      GmgLevel<T> &F = G.lv[l - 1];
      k_rap<T, B><<<nblk(L.nn), 128, 0, st>>>(F.nx, F.ny, F.S, F.fm, L.nx, L.ny, L.S);
      k_fm_coarse<B><<<nblk(L.nn), 256, 0, st>>>(F.nx, F.ny, F.fm, L.nx, L.ny, L.fm);
    }
    k_diag_bound<T, B><<<nblk(L.nn), 256, 0, st>>>(L.nx, L.ny, L.S, L.fm, L.invd);
    k_bound<T, B><<<nblk(L.nn, red_blocks()), 256, 0, st>>>(L.nx, L.ny, L.S, L.fm, G.ws, L.lmax);
    k_cheb_coef<T><<<1, 1, 0, st>>>(L.lmax, L.coef);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // coarsest dense inverse on the device
  const GmgLevel<T> &C = G.lv[G.nl - 1];
  k_coarse_inverse<T, B><<<1, 1024, 0, st>>>(C.nx, C.ny, C.S, C.fm, G.ncoarse, G.cwork, G.cinv);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  G.ready = true;
  return cudaSuccess;
}

template <class T>
cudaError_t gmg_setup_elas(Gmg<T> &G, const GridD &g, const MatD &m, const T *d,
                           const uint8_t *tens, cudaStream_t st) {
  k_fine_stencil_elas<T><<<nblk(G.lv[0].nn), 128, 0, st>>>(g, m, d, tens, G.lv[0].S);
  return gmg_setup_common<T, 2>(G, g, st);
}

template <class T>
cudaError_t gmg_setup_elas_qp(Gmg<T> &G, const GridD &g, const double *Dq, cudaStream_t st) {
  sp_stencil<T>(g, Dq, G.lv[0].S, st);
  return gmg_setup_common<T, 2>(G, g, st);
}

template <class T>
cudaError_t gmg_setup_damage(Gmg<T> &G, const GridD &g, const T *c, double kappa,
                             cudaStream_t st) {
  k_fine_stencil_damage<T><<<nblk(G.lv[0].nn), 128, 0, st>>>(g, c, kappa, G.lv[0].S);
  return gmg_setup_common<T, 1>(G, g, st);
}

// ---- V-cycle launchers ------------------------------------------------------------------------
template <class T>
void gmg_sten_apply(const Gmg<T> &G, int l, const T *x, const T *b, T *y, int mode,
                    cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l];
  if (G.B == 2)
    launch_pdl(k_sten_apply<T, 2>, dim3(nblk(L.nn)), dim3(256), st,
               StenApplyF<T, 2>{L.nx, L.ny, L.S, L.fm, x, b, y, mode});
  else
    launch_pdl(k_sten_apply<T, 1>, dim3(nblk(L.nn)), dim3(256), st,
               StenApplyF<T, 1>{L.nx, L.ny, L.S, L.fm, x, b, y, mode});
}
template <class T>
void gmg_cheb_first(const Gmg<T> &G, int l, const T *b, T *x, T *d, T *r, cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l];
  const size_t n = (size_t)G.B * L.nn;
  k_cheb_first<T><<<nblk(n), 256, 0, st>>>(n, b, L.invd, L.coef, x, d, r);
}
template <class T>
void gmg_cheb_first_x(const Gmg<T> &G, int l, const T *b, const T *y, T *x, T *d, T *r,
                      cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l];
  const size_t n = (size_t)G.B * L.nn;
  k_cheb_first_x<T><<<nblk(n), 256, 0, st>>>(n, b, y, L.invd, L.coef, x, d, r);
}
template <class T>
void gmg_cheb_step(const Gmg<T> &G, int l, const T *y, T *x, T *d, T *r, cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l];
  const size_t n = (size_t)G.B * L.nn;
  k_cheb_step<T><<<nblk(n), 256, 0, st>>>(n, y, L.invd, L.coef, x, d, r);
}
template <class T>
void gmg_sub(size_t n, const T *b, const T *y, T *r, cudaStream_t st) {
  k_sub<T><<<nblk(n), 256, 0, st>>>(n, b, y, r);
}
template <class T>
void gmg_restrict(const Gmg<T> &G, int l, const T *rf, T *bc, cudaStream_t st) {
  const GmgLevel<T> &F = G.lv[l], &C = G.lv[l + 1];
  if (G.B == 2)
    launch_pdl(k_restrict<T, 2>, dim3(nblk(C.nn)), dim3(256), st,
               RestrictF<T, 2>{F.nx, F.ny, rf, F.fm, C.nx, C.ny, C.fm, bc});
  else
    launch_pdl(k_restrict<T, 1>, dim3(nblk(C.nn)), dim3(256), st,
               RestrictF<T, 1>{F.nx, F.ny, rf, F.fm, C.nx, C.ny, C.fm, bc});
}
template <class T>
void gmg_prolong_add(const Gmg<T> &G, int l, const T *xc, T *xf, cudaStream_t st) {
  const GmgLevel<T> &F = G.lv[l], &C = G.lv[l + 1];
  if (G.B == 2)
    k_prolong_add<T, 2><<<nblk(F.nn), 256, 0, st>>>(F.nx, F.ny, F.fm, C.nx, xc, xf);
  else
    k_prolong_add<T, 1><<<nblk(F.nn), 256, 0, st>>>(F.nx, F.ny, F.fm, C.nx, xc, xf);
}
template <class T>
void gmg_pre(const Gmg<T> &G, int l, const T *b, T *x, cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l];
  if (G.B == 2)
    launch_pdl(k_sten_pre<T, 2>, dim3(nblk(L.nn)), dim3(256), st,
               StenPreF<T, 2>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, b, x});
  else
    launch_pdl(k_sten_pre<T, 1>, dim3(nblk(L.nn)), dim3(256), st,
               StenPreF<T, 1>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, b, x});
}
template <class T>
void gmg_prolong_first(const Gmg<T> &G, int l, const T *xin, T *xout, cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l], &C = G.lv[l + 1];
  if (G.B == 2)
    launch_pdl(k_sten_prolong_first<T, 2>, dim3(nblk(L.nn)), dim3(256), st,
               StenProlongFirstF<T, 2>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm,
                                                           C.nx, C.ny, C.x, L.b, xin, xout, L.r,
                                                           L.dv});
  else
    launch_pdl(k_sten_prolong_first<T, 1>, dim3(nblk(L.nn)), dim3(256), st,
               StenProlongFirstF<T, 1>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm,
                                                           C.nx, C.ny, C.x, L.b, xin, xout, L.r,
                                                           L.dv});
}
template <class T>
void gmg_post(const Gmg<T> &G, int l, T *x, cudaStream_t st) {
  const GmgLevel<T> &L = G.lv[l];
  if (G.B == 2)
    launch_pdl(k_sten_post<T, 2>, dim3(nblk(L.nn)), dim3(256), st,
               StenPostF<T, 2>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, L.dv,
                                                  L.r, x});
  else
    launch_pdl(k_sten_post<T, 1>, dim3(nblk(L.nn)), dim3(256), st,
               StenPostF<T, 1>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, L.dv,
                                                  L.r, x});
}
template <class T>
void gmg_coarse_cycle(const Gmg<T> &G, int lc, const T *b0, T *x0, cudaStream_t st) {
  CoarseArgs<T> a;
  a.nlev = G.nl - lc;
  for (int l = lc; l < G.nl; ++l) {
    const GmgLevel<T> &L = G.lv[l];
    a.L[l - lc] = CoarseLevel<T>{L.nx, L.ny, L.S, L.invd, L.x, L.b, L.r, L.dv, L.y, L.fm, L.coef};
  }
  a.b0 = b0;
  a.x0 = x0;
  a.cinv = G.cinv;
  a.ncoarse = G.ncoarse;
  if (G.B == 2)
    launch_pdl(k_coarse_cycle<T, 2>, dim3(1), dim3(COARSE_THREADS), st, a);
  else
    launch_pdl(k_coarse_cycle<T, 1>, dim3(1), dim3(COARSE_THREADS), st, a);
}

template <class T>
int gmg_set_coarse_nodes(Gmg<T> &G, int nodes) {
  G.lc = G.nl - 1;
  for (int k = 0; k < G.nl; ++k)
    if (G.lv[k].nn <= (size_t)nodes) {
      G.lc = k;
      break;
    }
  return G.lc;
}

// ---- batched V-cycle (pf_batch.cuh) ----------------------------------------------------
template <class T>
static CoarseArgs<T> coarse_args(const Gmg<T> &G, int lc, const T *b0, T *x0) {
  CoarseArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.nlev = G.nl - lc;
  for (int l = lc; l < G.nl; ++l) {
    const GmgLevel<T> &L = G.lv[l];
    a.L[l - lc] = CoarseLevel<T>{L.nx, L.ny, L.S, L.invd, L.x, L.b, L.r, L.dv, L.y, L.fm, L.coef};
  }
  a.b0 = b0;
  a.x0 = x0;
  a.cinv = G.cinv;
  a.ncoarse = G.ncoarse;
  return a;
}

template <class T>
cudaError_t gmg_batch_prepare(Gmg<T> &G) {
  const int lc = G.lc > 1 ? G.lc : 1;
  if (lc >= G.nl) return cudaErrorInvalidValue;
  const CoarseArgs<T> a = coarse_args<T>(G, lc, G.lv[lc].b, G.lv[lc].x);
  cudaError_t e = cudaSuccess;
  if (!G.dca && (e = cudaMalloc(&G.dca, sizeof(CoarseArgs<T>))) != cudaSuccess) {
    G.dca = nullptr;
    return e;
  }
  return cudaMemcpy(G.dca, &a, sizeof(a), cudaMemcpyHostToDevice);
}

template <class T, int B>
static int restrict0_batch_b(int n, Gmg<T> *const *G, const int *const *done, cudaStream_t st) {
  Batcher<RestrictF<T, B>, 256> b;
  for (int i = 0; i < n; ++i) {
    const GmgLevel<T> &F = G[i]->lv[0], &C = G[i]->lv[1];
    b.add(RestrictF<T, B>{F.nx, F.ny, F.r, F.fm, C.nx, C.ny, C.fm, C.b}, nblk(C.nn), done[i]);
  }
  return b.launch(st);
}
template <class T>
int gmg_restrict0_batch(int n, Gmg<T> *const *G, const int *const *done, cudaStream_t st) {
  return G[0]->B == 2 ? restrict0_batch_b<T, 2>(n, G, done, st)
                      : restrict0_batch_b<T, 1>(n, G, done, st);
}

// The launch order of gmg_mid(G, 1) for every hierarchy: down through the grid levels each
// hierarchy has (level l takes the hierarchies with l < lc), the coarse cycles, and up.
template <class T, int B>
static int mid_batch_b(int n, Gmg<T> *const *G, const int *const *done, cudaStream_t st) {
  int launches = 0, lmax = 1;
  for (int i = 0; i < n; ++i) lmax = G[i]->lc > lmax ? G[i]->lc : lmax;
  for (int l = 1; l < lmax; ++l) {
    Batcher<StenPreF<T, B>, 256> pre;
    Batcher<StenApplyF<T, B>, 256> app;
    Batcher<RestrictF<T, B>, 256> res;
    for (int i = 0; i < n; ++i) {
      if (l >= G[i]->lc) continue;
      const GmgLevel<T> &L = G[i]->lv[l], &C = G[i]->lv[l + 1];
      pre.add(StenPreF<T, B>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, L.b, L.y}, nblk(L.nn), done[i]);
      app.add(StenApplyF<T, B>{L.nx, L.ny, L.S, L.fm, L.y, L.b, L.r, 1}, nblk(L.nn), done[i]);
      res.add(RestrictF<T, B>{L.nx, L.ny, L.r, L.fm, C.nx, C.ny, C.fm, C.b}, nblk(C.nn), done[i]);
    }
    launches += pre.launch(st) + app.launch(st) + res.launch(st);
  }
  {
    Batcher<CoarseF<T, B>, COARSE_THREADS> cc;
    for (int i = 0; i < n; ++i)
      cc.add(CoarseF<T, B>{static_cast<const CoarseArgs<T> *>(G[i]->dca)}, 1, done[i]);
    launches += cc.launch(st);
  }
  for (int l = lmax - 1; l >= 1; --l) {
    Batcher<StenProlongFirstF<T, B>, 256> pf;
    Batcher<StenPostF<T, B>, 256> post;
    for (int i = 0; i < n; ++i) {
      if (l >= G[i]->lc) continue;
      const GmgLevel<T> &L = G[i]->lv[l], &C = G[i]->lv[l + 1];
      pf.add(StenProlongFirstF<T, B>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, C.nx, C.ny, C.x, L.b,
                                     L.y, L.x, L.r, L.dv},
             nblk(L.nn), done[i]);
      post.add(StenPostF<T, B>{L.nx, L.ny, L.S, L.invd, L.coef, L.fm, L.dv, L.r, L.x}, nblk(L.nn),
               done[i]);
    }
    launches += pf.launch(st) + post.launch(st);
  }
  return launches;
}
template <class T>
int gmg_mid_batch(int n, Gmg<T> *const *G, const int *const *done, cudaStream_t st) {
  return G[0]->B == 2 ? mid_batch_b<T, 2>(n, G, done, st) : mid_batch_b<T, 1>(n, G, done, st);
}

#define GMG_INST(T)                                                                            \
  template cudaError_t gmg_alloc<T>(Gmg<T> &, int, int, int, const RedWs &, Arena &);          \
  template void gmg_free<T>(Gmg<T> &);                                                         \
  template cudaError_t gmg_setup_elas<T>(Gmg<T> &, const GridD &, const MatD &, const T *,     \
                                         const uint8_t *, cudaStream_t);                       \
  template cudaError_t gmg_setup_damage<T>(Gmg<T> &, const GridD &, const T *, double,         \
                                           cudaStream_t);                                      \
  template cudaError_t gmg_setup_elas_qp<T>(Gmg<T> &, const GridD &, const double *,           \
                                            cudaStream_t);                                     \
  template void gmg_sten_apply<T>(const Gmg<T> &, int, const T *, const T *, T *, int,         \
                                  cudaStream_t);                                               \
  template void gmg_cheb_first<T>(const Gmg<T> &, int, const T *, T *, T *, T *, cudaStream_t); \
  template void gmg_cheb_first_x<T>(const Gmg<T> &, int, const T *, const T *, T *, T *, T *,  \
                                    cudaStream_t);                                             \
  template void gmg_cheb_step<T>(const Gmg<T> &, int, const T *, T *, T *, T *, cudaStream_t);  \
  template void gmg_sub<T>(size_t, const T *, const T *, T *, cudaStream_t);                    \
  template void gmg_restrict<T>(const Gmg<T> &, int, const T *, T *, cudaStream_t);             \
  template cudaError_t gmg_batch_prepare<T>(Gmg<T> &);                                         \
  template int gmg_set_coarse_nodes<T>(Gmg<T> &, int);                                         \
  template int gmg_restrict0_batch<T>(int, Gmg<T> *const *, const int *const *, cudaStream_t); \
  template int gmg_mid_batch<T>(int, Gmg<T> *const *, const int *const *, cudaStream_t);       \
  template void gmg_prolong_add<T>(const Gmg<T> &, int, const T *, T *, cudaStream_t);          \
  template void gmg_coarse_cycle<T>(const Gmg<T> &, int, const T *, T *, cudaStream_t);      \
  template void gmg_pre<T>(const Gmg<T> &, int, const T *, T *, cudaStream_t);                 \
  template void gmg_prolong_first<T>(const Gmg<T> &, int, const T *, T *, cudaStream_t);       \
  template void gmg_post<T>(const Gmg<T> &, int, T *, cudaStream_t);
GMG_INST(double)
GMG_INST(float)

}  // namespace pf
