// Spectral energy split (the alternative split named in Sec. 2) on the GPU path, and the
// assembled-stencil form of the elasticity tangent that its Newton iteration needs.
//
// Pointwise law, for both plane modes (lam = K - 2 mu cdim; e1 >= e2 the in-plane
// principal strains; the out-of-plane principal strain of plane strain is 0):
//   Psi+  = lam/2 <tr>_+^2 + mu (<e1>_+^2 + <e2>_+^2)
//   sigma = g(d) [lam <tr>_+ I + 2 mu eps+] + lam <tr>_- I + 2 mu eps-,
//   eps+- = sum_i <e_i>_+- n_i (x) n_i.
// Newton tangent:
//   d sigma = lam [g H(tr) + 1 - H(tr)] tr(d eps) I + 2 mu d eps + 2 mu (g - 1) P+ d eps,
// where P+ = d eps+ / d eps keeps, in the principal frame, the two normal components with
// weights H(e1), H(e2) and the shear component with the divided difference
// (<e1>_+ - <e2>_+) / (e1 - e2) (H(e1) where e1 = e2); H(x) = 1 for x > 0 strictly.
// The fixed-stress schemes act on the two parts of Psi+: the trace part
// Psi_a = lam/2 <tr>_+^2 (S1), the second part Psi_b = mu sum <e_i>_+^2 (S2), or both
// (S3): K~ = -4 (1-d)^2/g Q with Q_S1 = 2 Psi_a, Q_S2 = 2 Psi_b, Q_S3 = 2 Psi+, and the
// prediction scales the fixed part(s) by s^2, s = 1 + 2(1-d)/g max(Delta d, 0) -- the rules
// that give the paper's VD forms for the VD parts (K/2 <tr>_+^2, mu e.e).
//
// The VD tangent is fixed by one sign bit per point, so it is applied matrix-free.  The
// spectral tangent depends on the whole strain: the u-solves assemble the per-point
// tangents into the nodal stencil of the multigrid hierarchy (9 neighbours x 2 x 2 blocks)
// and apply that: 36 stencil values per node on top of the operand and the product, where
// the matrix-free VD operator reads only d and one sign byte per element besides them.
#include <math.h>

#include "pf_fused.cuh"
#include "pf_gmg.cuh"
#include "pf_spectral.cuh"

namespace pf {

namespace {

__device__ __forceinline__ double sp_gp(int hi) {
  return hi ? 0.78867513459481288225 : 0.21132486540518711775;  // (1 +- 1/sqrt3)/2
}
__device__ __forceinline__ double sp_pos(double x) { return x > 0.0 ? x : 0.0; }
__device__ __forceinline__ double sp_neg(double x) { return x < 0.0 ? x : 0.0; }

inline unsigned sp_blocks(size_t n, size_t cap = 65536) {
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

struct SpStrain {
  double exx[4], eyy[4], exy[4];
};

__device__ __forceinline__ void sp_nodes(const GridD &g, size_t e, size_t (&n)[4]) {
  const int ei = (int)(e % g.nx), ej = (int)(e / g.nx);
  const size_t ld = (size_t)g.nx + 1;
  n[0] = (size_t)ej * ld + ei;
  n[1] = n[0] + 1;
  n[2] = n[0] + ld;
  n[3] = n[2] + 1;
}

// Strains at the four Gauss points (q = qy * 2 + qx) from the element's nodal u.
__device__ __forceinline__ void sp_strains(const GridD &g, const double *u,
                                           const size_t (&n)[4], SpStrain &S) {
  double ux[4], uy[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ux[a] = __ldg(u + 2 * n[a]);
    uy[a] = __ldg(u + 2 * n[a] + 1);
  }
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double s = sp_gp(q & 1), t = sp_gp(q >> 1);
    const double s1 = 1.0 - s, t1 = 1.0 - t;
    S.exx[q] = (t1 * (ux[1] - ux[0]) + t * (ux[3] - ux[2])) * ihx;
    S.eyy[q] = (s1 * (uy[2] - uy[0]) + s * (uy[3] - uy[1])) * ihy;
    S.exy[q] = 0.5 * ((s1 * (ux[2] - ux[0]) + s * (ux[3] - ux[1])) * ihy +
                      (t1 * (uy[1] - uy[0]) + t * (uy[3] - uy[2])) * ihx);
  }
}

__device__ __forceinline__ void sp_interp(const double *f, const size_t (&n)[4],
                                          double (&fq)[4]) {
  const double f0 = __ldg(f + n[0]), f1 = __ldg(f + n[1]), f2 = __ldg(f + n[2]),
               f3 = __ldg(f + n[3]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double s = sp_gp(q & 1), t = sp_gp(q >> 1);
    fq[q] = (1.0 - s) * (1.0 - t) * f0 + s * (1.0 - t) * f1 + (1.0 - s) * t * f2 + s * t * f3;
  }
}

// Principal strains e1 >= e2 of the symmetric 2 x 2 strain and (cos 2t, sin 2t) of the
// direction of e1; (1, 0) where e1 = e2.
struct Principal {
  double e1, e2, c2, s2;
};
__device__ __forceinline__ Principal sp_principal(double exx, double eyy, double exy) {
  const double mean = 0.5 * (exx + eyy), half = 0.5 * (exx - eyy);
  const double R = hypot(half, exy);
  Principal p;
  p.e1 = mean + R;
  p.e2 = mean - R;
  if (R > 0.0) {
    p.c2 = half / R;
    p.s2 = exy / R;
  } else {
    p.c2 = 1.0;
    p.s2 = 0.0;
  }
  return p;
}

__device__ __forceinline__ double sp_lam(const MatD &m) { return m.K - 2.0 * m.mu * m.cdim; }

// Spectral parts of Psi+: trace part pa and principal part pb.
__device__ __forceinline__ void sp_parts(const MatD &m, double exx, double eyy, double exy,
                                         double &pa, double &pb) {
  const double tp = sp_pos(exx + eyy);
  const Principal p = sp_principal(exx, eyy, exy);
  const double a = sp_pos(p.e1), b = sp_pos(p.e2);
  pa = 0.5 * sp_lam(m) * tp * tp;
  pb = m.mu * (a * a + b * b);
}

__device__ __forceinline__ double sp_Q(int scheme, double pa, double pb) {
  return scheme == PF_S1 ? 2.0 * pa
       : scheme == PF_S2 ? 2.0 * pb
       : scheme == PF_S3 ? 2.0 * (pa + pb)
                         : 0.0;
}

// Stress (sxx, syy, sxy) and Newton tangent (D00, D01, D02, D11, D12, D22) at one point
// with g = gq, for the material's split.
__device__ void point_law(const MatD &m, double gq, double exx, double eyy, double exy,
                          double (&sig)[3], double (&D)[6]) {
  const double tr = exx + eyy;
  if (m.split != PF_SPLIT_SPECTRAL) {   // VD with the indicator at the sign of tr
    const bool ip = tr > 0.0;
    const double kv = ip ? gq * m.K : m.K;
    const double tmg = 2.0 * m.mu * gq;
    sig[0] = tmg * (exx - m.cdim * tr) + kv * tr;
    sig[1] = tmg * (eyy - m.cdim * tr) + kv * tr;
    sig[2] = tmg * exy;
    D[0] = tmg * (1.0 - m.cdim) + kv;
    D[1] = -tmg * m.cdim + kv;
    D[2] = 0.0;
    D[3] = D[0];
    D[4] = 0.0;
    D[5] = m.mu * gq;
    return;
  }
  const double lam = sp_lam(m);
  const Principal p = sp_principal(exx, eyy, exy);
  const double c2 = p.c2, s2 = p.s2;
  // n1 (x) n1 = [(1 + c2)/2, s2/2; s2/2, (1 - c2)/2], n2 (x) n2 = I - n1 (x) n1,
  // n1 (x) n2 + n2 (x) n1 = [-s2, c2; c2, s2]
  const double vol = lam * (gq * sp_pos(tr) + sp_neg(tr));
  const double w1 = 2.0 * m.mu * (gq * sp_pos(p.e1) + sp_neg(p.e1));
  const double w2 = 2.0 * m.mu * (gq * sp_pos(p.e2) + sp_neg(p.e2));
  sig[0] = vol + 0.5 * (w1 * (1.0 + c2) + w2 * (1.0 - c2));
  sig[1] = vol + 0.5 * (w1 * (1.0 - c2) + w2 * (1.0 + c2));
  sig[2] = 0.5 * s2 * (w1 - w2);
  const double h1 = p.e1 > 0.0 ? 1.0 : 0.0, h2 = p.e2 > 0.0 ? 1.0 : 0.0;
  const double gap = p.e1 - p.e2;
  const double c12 = gap > 0.0 ? (sp_pos(p.e1) - sp_pos(p.e2)) / gap : h1;
  const double kv = lam * (tr > 0.0 ? gq : 1.0);
  const double tm = 2.0 * m.mu, tg = 2.0 * m.mu * (gq - 1.0);
  double col[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {   // unit Voigt strains: exx, eyy, engineering shear
    const double dxx = c == 0 ? 1.0 : 0.0, dyy = c == 1 ? 1.0 : 0.0, dxy = c == 2 ? 0.5 : 0.0;
    const double a1 = 0.5 * (1.0 + c2) * dxx + 0.5 * (1.0 - c2) * dyy + s2 * dxy;
    const double a2 = 0.5 * (1.0 - c2) * dxx + 0.5 * (1.0 + c2) * dyy - s2 * dxy;
    const double a12 = 0.5 * s2 * (dyy - dxx) + c2 * dxy;
    const double Pxx = 0.5 * (h1 * a1 * (1.0 + c2) + h2 * a2 * (1.0 - c2)) - c12 * a12 * s2;
    const double Pyy = 0.5 * (h1 * a1 * (1.0 - c2) + h2 * a2 * (1.0 + c2)) + c12 * a12 * s2;
    const double Pxy = 0.5 * s2 * (h1 * a1 - h2 * a2) + c12 * a12 * c2;
    const double trd = dxx + dyy;
    col[c][0] = kv * trd + tm * dxx + tg * Pxx;
    col[c][1] = kv * trd + tm * dyy + tg * Pyy;
    col[c][2] = tm * dxy + tg * Pxy;
  }
  D[0] = col[0][0];
  D[1] = col[1][0];
  D[2] = col[2][0];
  D[3] = col[1][1];
  D[4] = col[2][1];
  D[5] = col[2][2];
}

// ---- per-point kernels (one thread per element, FP64) ----------------------------------
__global__ void k_sp_energy(GridD g, MatD m, const double *__restrict__ u,
                            const double *__restrict__ Hprev, double *__restrict__ psi,
                            double *__restrict__ Hout) {
  const size_t ne = (size_t)g.nx * g.ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    double p[4] = {0, 0, 0, 0};
    if (live) {
      size_t n[4];
      sp_nodes(g, e, n);
      SpStrain S;
      sp_strains(g, u, n, S);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double pa, pb;
        sp_parts(m, S.exx[q], S.eyy[q], S.exy[q], pa, pb);
        p[q] = pa + pb;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Hout[4 * e + q] = fmax(__ldg(Hprev + 4 * e + q), p[q]);
      if (psi) psi[4 * e + q] = p[q];
    }
  }
}

__global__ void k_sp_fs_coeff(GridD g, MatD m, int scheme, double psi_crit,
                              const double *__restrict__ u, const double *__restrict__ d,
                              const double *__restrict__ Hprev, double *__restrict__ c_aug,
                              uint8_t *__restrict__ active, At1D at1) {
  const size_t ne = (size_t)g.nx * g.ny;
  const double floor_c = at1.on ? at1.floor : m.Gc / m.l;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    size_t n[4];
    sp_nodes(g, e, n);
    SpStrain S;
    double dq[4], dpq[4];
    if (live) {
      sp_strains(g, u, n, S);
      sp_interp(d, n, dq);
      if (at1.on) sp_interp(at1.dprev, n, dpq);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double hp = __ldg(Hprev + 4 * e + q);
      double c = at1.on ? 0.0 : floor_c + 2.0 * hp;
      uint8_t a = 0;
      if (live) {
        double pa, pb;
        sp_parts(m, S.exx[q], S.eyy[q], S.exy[q], pa, pb);
        const double ps = pa + pb;
        const double cJ = at1.on ? 2.0 * ps + (dq[q] < dpq[q] ? at1.gamma : 0.0)
                                 : floor_c + 2.0 * fmax(hp, ps);
        c = cJ;
        a = (ps > psi_crit) && (ps > hp) && (dq[q] < 0.95);
        if (a) {
          const double om = 1.0 - dq[q];
          const double gq = om * om + m.eta;
          const double lim = at1.on ? fmin(cJ, floor_c) : floor_c;
          c = fmax(cJ - 4.0 * om * om / gq * sp_Q(scheme, pa, pb), lim);
        }
      }
      c_aug[4 * e + q] = c;
      active[4 * e + q] = a;
    }
  }
}

__global__ void k_sp_fs_predict(GridD g, MatD m, int scheme, const double *__restrict__ u,
                                const double *__restrict__ d, const double *__restrict__ dd,
                                const double *__restrict__ Hprev,
                                const uint8_t *__restrict__ active, double *__restrict__ Hhalf,
                                int at1) {
  const size_t ne = (size_t)g.nx * g.ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    size_t n[4];
    sp_nodes(g, e, n);
    SpStrain S;
    double dq[4], ddq[4];
    if (live) {
      sp_strains(g, u, n, S);
      sp_interp(d, n, dq);
      sp_interp(dd, n, ddq);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double hp = __ldg(Hprev + 4 * e + q);
      double h = hp;
      if (live) {
        double pa, pb;
        sp_parts(m, S.exx[q], S.eyy[q], S.exy[q], pa, pb);
        double ps = pa + pb;
        if (active[4 * e + q]) {
          const double om = 1.0 - dq[q];
          const double gq = om * om + m.eta;
          const double ddp = ddq[q] > 0.0 ? ddq[q] : 0.0;
          const double sc = 1.0 + 2.0 * om / gq * ddp;
          const double sa = (scheme == PF_S1 || scheme == PF_S3) ? sc : 1.0;
          const double sb = (scheme == PF_S2 || scheme == PF_S3) ? sc : 1.0;
          ps = pa * sa * sa + pb * sb * sb;
        }
        h = at1 ? ps : fmax(hp, ps);
      }
      Hhalf[4 * e + q] = h;
    }
  }
}

__global__ void k_sp_points(GridD g, MatD m, const double *__restrict__ u,
                            const double *__restrict__ d, double *__restrict__ Sq,
                            double *__restrict__ Dq) {
  const size_t ne = (size_t)g.nx * g.ny, nq = 4 * ne;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    size_t n[4];
    sp_nodes(g, e, n);
    SpStrain S;
    double dq[4];
    if (live) {
      sp_strains(g, u, n, S);
      sp_interp(d, n, dq);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double sig[3] = {0.0, 0.0, 0.0}, D[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (live) {
        const double om = 1.0 - dq[q];
        point_law(m, om * om + m.eta, S.exx[q], S.eyy[q], S.exy[q], sig, D);
      }
      if (Sq)
#pragma unroll
        for (int c = 0; c < 3; ++c) Sq[c * nq + 4 * e + q] = sig[c];
      if (Dq)
#pragma unroll
        for (int k = 0; k < 6; ++k) Dq[k * nq + 4 * e + q] = D[k];
    }
  }
}

// Shape-function gradients of local node a = ay * 2 + ax at Gauss point q.
__device__ __forceinline__ void sp_grad(int a, int q, double ihx, double ihy, double &Nx,
                                        double &Ny) {
  const int ax = a & 1, ay = a >> 1;
  const double s = sp_gp(q & 1), t = sp_gp(q >> 1);
  Nx = (ax ? 1.0 : -1.0) * (ay ? t : 1.0 - t) * ihx;
  Ny = (ay ? 1.0 : -1.0) * (ax ? s : 1.0 - s) * ihy;
}

__global__ void k_sp_force(GridD g, const double *__restrict__ Sq, double *__restrict__ F) {
  const int nx = g.nx, ny = g.ny;
  const size_t nn = (size_t)(nx + 1) * (ny + 1), nq = 4 * (size_t)nx * ny;
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy, w = 0.25 * g.hx * g.hy;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    double fx = 0.0, fy = 0.0;
#pragma unroll
    for (int ej_off = -1; ej_off <= 0; ++ej_off)
#pragma unroll
      for (int ei_off = -1; ei_off <= 0; ++ei_off) {
        const int ei = i + ei_off, ej = j + ej_off;
        if (ei < 0 || ei >= nx || ej < 0 || ej >= ny) continue;
        const size_t e = (size_t)ej * nx + ei;
        if (g.active && !g.active[e]) continue;
        const int a = (-ej_off) * 2 + (-ei_off);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          double Nx, Ny;
          sp_grad(a, q, ihx, ihy, Nx, Ny);
          const double sxx = __ldg(Sq + 4 * e + q), syy = __ldg(Sq + nq + 4 * e + q),
                       sxy = __ldg(Sq + 2 * nq + 4 * e + q);
          fx += w * (Nx * sxx + Ny * sxy);
          fy += w * (Ny * syy + Nx * sxy);
        }
      }
    F[2 * n] = fx;
    F[2 * n + 1] = fy;
  }
}

// u . D v with D symmetric, packed (D00, D01, D02, D11, D12, D22).
__device__ __forceinline__ double sp_qf(const double (&D)[6], double u0, double u1, double u2,
                                        double v0, double v1, double v2) {
  return u0 * (D[0] * v0 + D[1] * v1 + D[2] * v2) + u1 * (D[1] * v0 + D[3] * v1 + D[4] * v2) +
         u2 * (D[2] * v0 + D[4] * v1 + D[5] * v2);
}

template <class T>
__global__ void k_sp_stencil(GridD g, const double *__restrict__ Dq, T *__restrict__ S) {
  const int nx = g.nx, ny = g.ny;
  const size_t nn = (size_t)(nx + 1) * (ny + 1), nq = 4 * (size_t)nx * ny;
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy, w = 0.25 * g.hx * g.hy;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    double acc[9][4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[k][c] = 0.0;
    for (int ej_off = -1; ej_off <= 0; ++ej_off)
      for (int ei_off = -1; ei_off <= 0; ++ei_off) {
        const int ei = i + ei_off, ej = j + ej_off;
        if (ei < 0 || ei >= nx || ej < 0 || ej >= ny) continue;
        const size_t e = (size_t)ej * nx + ei;
        if (g.active && !g.active[e]) continue;
        const int ax = -ei_off, ay = -ej_off, a = ay * 2 + ax;
        for (int q = 0; q < 4; ++q) {
          double D[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) D[k] = __ldg(Dq + k * nq + 4 * e + q);
          double Nxa, Nya;
          sp_grad(a, q, ihx, ihy, Nxa, Nya);
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            double Nxb, Nyb;
            sp_grad(b, q, ihx, ihy, Nxb, Nyb);
            const int k = ((b >> 1) - ay + 1) * 3 + ((b & 1) - ax + 1);
            // rows: (Nx, 0, Ny) for u_x, (0, Ny, Nx) for u_y of node a; columns likewise for b
            acc[k][0] += w * sp_qf(D, Nxa, 0.0, Nya, Nxb, 0.0, Nyb);
            acc[k][1] += w * sp_qf(D, Nxa, 0.0, Nya, 0.0, Nyb, Nxb);
            acc[k][2] += w * sp_qf(D, 0.0, Nya, Nxa, Nxb, 0.0, Nyb);
            acc[k][3] += w * sp_qf(D, 0.0, Nya, Nxa, 0.0, Nyb, Nxb);
          }
        }
      }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int c = 0; c < 4; ++c) S[sten_idx<2>(k, c >> 1, c & 1, n, nn)] = (T)acc[k][c];
  }
}

// y = P K P x (P zeroes constrained DOFs) through the stencil; x.y for the epilogue.
template <class T>
__global__ void k_sp_apply(int nx, int ny, const T *__restrict__ S,
                           const uint8_t *__restrict__ dofm, const T *__restrict__ x,
                           T *__restrict__ y, KrylovScal *sc, RedWs ws, int epi) {
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  double dot = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    T acc0 = T(0), acc1 = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ii = i + k % 3 - 1, jj = j + k / 3 - 1;
      if (ii < 0 || ii > nx || jj < 0 || jj > ny) continue;
      const size_t nb = (size_t)jj * (nx + 1) + ii;
      const uint8_t mb = dofm ? __ldg(dofm + nb) : 0;
      const T x0 = (mb & 1) ? T(0) : __ldg(x + 2 * nb);
      const T x1 = (mb & 2) ? T(0) : __ldg(x + 2 * nb + 1);
      acc0 += __ldg(S + sten_idx<2>(k, 0, 0, n, nn)) * x0 + __ldg(S + sten_idx<2>(k, 0, 1, n, nn)) * x1;
      acc1 += __ldg(S + sten_idx<2>(k, 1, 0, n, nn)) * x0 + __ldg(S + sten_idx<2>(k, 1, 1, n, nn)) * x1;
    }
    const uint8_t mn = dofm ? __ldg(dofm + n) : 0;
    const T y0 = (mn & 1) ? T(0) : acc0, y1 = (mn & 2) ? T(0) : acc1;
    y[2 * n] = y0;
    y[2 * n + 1] = y1;
    if (epi != EPI_NONE) {
      const T x0 = (mn & 1) ? T(0) : x[2 * n], x1 = (mn & 2) ? T(0) : x[2 * n + 1];
      dot += (double)x0 * (double)y0 + (double)x1 * (double)y1;
    }
  }
  if (epi != EPI_NONE) {
    double v[1] = {dot}, tot[1];
    if (red_grid<1>(v, ws, tot, false)) krylov_epilogue(epi, sc, tot[0]);
  }
}

template <class T>
__global__ void k_sp_diag(size_t nn, const T *__restrict__ S, const uint8_t *__restrict__ dofm,
                          T *__restrict__ diag) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const uint8_t mn = dofm ? dofm[n] : 0;
    diag[2 * n] = (mn & 1) ? T(0) : S[sten_idx<2>(4, 0, 0, n, nn)];
    diag[2 * n + 1] = (mn & 2) ? T(0) : S[sten_idx<2>(4, 1, 1, n, nn)];
  }
}

}  // namespace

// ---- host side ------------------------------------------------------------------------------
void point_energy(const GridD &g, const MatD &m, const double *u, const double *Hprev,
                  double *psi, double *Hout, cudaStream_t st) {
  if (m.split != PF_SPLIT_SPECTRAL) {
    qp_energy(g, m, u, Hprev, psi, Hout, st);
    return;
  }
  const size_t ne = (size_t)g.nx * g.ny;
  k_sp_energy<<<sp_blocks(ne), 256, 0, st>>>(g, m, u, Hprev, psi, Hout);
}

void point_fs_coeff(const GridD &g, const MatD &m, int scheme, double psi_crit,
                    const double *u, const double *d, const double *Hprev, double *c_aug,
                    uint8_t *active, cudaStream_t st, const At1D &at1) {
  if (m.split != PF_SPLIT_SPECTRAL) {
    fs_coeff(g, m, scheme, psi_crit, u, d, Hprev, c_aug, active, st, at1);
    return;
  }
  const size_t ne = (size_t)g.nx * g.ny;
  k_sp_fs_coeff<<<sp_blocks(ne), 256, 0, st>>>(g, m, scheme, psi_crit, u, d, Hprev, c_aug,
                                               active, at1);
}

void point_fs_predict(const GridD &g, const MatD &m, int scheme, const double *u,
                      const double *d, const double *dd, const double *Hprev,
                      const uint8_t *active, double *Hhalf, cudaStream_t st, int at1) {
  if (m.split != PF_SPLIT_SPECTRAL) {
    fs_predict(g, m, scheme, u, d, dd, Hprev, active, Hhalf, st, at1);
    return;
  }
  const size_t ne = (size_t)g.nx * g.ny;
  k_sp_fs_predict<<<sp_blocks(ne), 256, 0, st>>>(g, m, scheme, u, d, dd, Hprev, active, Hhalf,
                                                 at1);
}

void sp_points(const GridD &g, const MatD &m, const double *u, const double *d, double *Sq,
               double *Dq, cudaStream_t st) {
  const size_t ne = (size_t)g.nx * g.ny;
  k_sp_points<<<sp_blocks(ne), 128, 0, st>>>(g, m, u, d, Sq, Dq);
}

void sp_force(const GridD &g, const double *Sq, double *F, cudaStream_t st) {
  const size_t nn = (size_t)(g.nx + 1) * (g.ny + 1);
  k_sp_force<<<sp_blocks(nn), 256, 0, st>>>(g, Sq, F);
}

template <class T>
void sp_stencil(const GridD &g, const double *Dq, T *S, cudaStream_t st) {
  const size_t nn = (size_t)(g.nx + 1) * (g.ny + 1);
  k_sp_stencil<T><<<sp_blocks(nn), 128, 0, st>>>(g, Dq, S);
}

template <class T>
void sp_apply(const GridD &g, const T *S, const T *x, T *y, cudaStream_t st, KrylovScal *sc,
              const RedWs *ws, int epi) {
  const size_t nn = (size_t)(g.nx + 1) * (g.ny + 1);
  const int e = (ws && sc) ? epi : EPI_NONE;
  const RedWs w = ws ? *ws : RedWs{nullptr, nullptr, 0};
  // with the epilogue every CTA takes part in the grid reduction: at most max_blocks CTAs
  const unsigned blocks = e != EPI_NONE ? sp_blocks(nn, (size_t)w.max_blocks) : sp_blocks(nn);
  k_sp_apply<T><<<blocks, 256, 0, st>>>(g.nx, g.ny, S, g.dofm, x, y, sc, w, e);
}

template <class T>
void sp_diag(const GridD &g, const T *S, T *diag, cudaStream_t st) {
  const size_t nn = (size_t)(g.nx + 1) * (g.ny + 1);
  k_sp_diag<T><<<sp_blocks(nn), 256, 0, st>>>(nn, S, g.dofm, diag);
}

template void sp_stencil<double>(const GridD &, const double *, double *, cudaStream_t);
template void sp_stencil<float>(const GridD &, const double *, float *, cudaStream_t);
template void sp_apply<double>(const GridD &, const double *, const double *, double *,
                               cudaStream_t, KrylovScal *, const RedWs *, int);
template void sp_apply<float>(const GridD &, const float *, const float *, float *, cudaStream_t,
                              KrylovScal *, const RedWs *, int);
template void sp_diag<double>(const GridD &, const double *, double *, cudaStream_t);
template void sp_diag<float>(const GridD &, const float *, float *, cudaStream_t);

}  // namespace pf
