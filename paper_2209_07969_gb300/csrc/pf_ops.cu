// Matrix-free Q1 operators and per-Gauss-point kernels of the staggered phase-field
// method (arXiv 2209.07969), written for sm_103a.
//
// Elasticity: the tangent product, the nonlinear internal force and the fused Krylov /
// multigrid stages run in the strip kernel (k_elas_strip: a warp marches up a strip of
// node columns, neighbours by warp shuffle, no shared memory); the tangent diagonal runs
// in a tile kernel.  Phase field: K_dd products and fused stages in a tile kernel
// (k_damage_op), diagonal and right-hand side in k_damage.  Tile kernels use one 256-thread
// CTA per tile of TX x TY = 32 x 8 nodes, stage the node patch with a one-node halo in
// shared memory, compute the element values of the (TX+1) x (TY+1) touching elements (the
// halo elements are recomputed by the neighbouring CTA) and sum the four contributions of
// every owned node.  No atomics: results are deterministic and independent of the launch.
//
// Element quantities (Sec. 2 and 3.2): 2x2 Gauss points at unit coordinates
// s, t in {G0, G1} = {(1 - 1/sqrt3)/2, (1 + 1/sqrt3)/2}; N_a bilinear; weight hx hy/4.
#include <math.h>
#include <stdio.h>

#include <type_traits>

#include "pf_internal.cuh"
#include "pf_fused.cuh"
#include "pf_batch.cuh"

namespace pf {

__device__ __forceinline__ double gp_lo() { return 0.21132486540518711775; }  // (1-1/sqrt3)/2
__device__ __forceinline__ double gp_hi() { return 0.78867513459481288225; }  // (1+1/sqrt3)/2

template <class T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// ------------------------------------------------------------------------------------
// Reductions: warp shuffle -> CTA -> per-CTA partials -> grouped two-level sum in the last
// arriving CTAs (red_grid; fixed order, deterministic) -> epilogue on the totals.
// ------------------------------------------------------------------------------------

// Sums NV values over the whole grid (red_grid).  Returns true in thread 0 of the last CTA,
// with tot[] holding the totals; all other threads return false.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], const RedWs ws, double (&tot)[NV],
                                            bool is_max = false) {
  return red_grid<NV>(v, ws, tot, is_max);
}


// ------------------------------------------------------------------------------------
// Per-launch constants in the kernel's arithmetic type, computed on the host: GB300 runs
// FP64 at 1/64 of the FP32 rate, so a float kernel must not touch a double.
// ------------------------------------------------------------------------------------
template <class T>
struct ElemConst {
  T ihx, ihy, w, mu, K, cd, eta, G0, G1, kappa;
};
template <class T>
static ElemConst<T> elem_const(const GridD &g, const MatD &m, double kappa = 0.0) {
  const double a = 0.5 * (1.0 - 1.0 / sqrt(3.0)), b = 0.5 * (1.0 + 1.0 / sqrt(3.0));
  return ElemConst<T>{T(1.0 / g.hx), T(1.0 / g.hy), T(0.25 * g.hx * g.hy), T(m.mu), T(m.K),
                      T(m.cdim), T(m.eta), T(a), T(b), T(kappa)};
}

// ------------------------------------------------------------------------------------
// Elasticity: tangent apply, tangent diagonal, nonlinear internal force.
// ------------------------------------------------------------------------------------
// Element force of the Q1 elasticity element with nodal values (a0..a3 = (i,j), (i+1,j),
// (i,j+1), (i+1,j+1)): f[2a] / f[2a+1] = x / y force on node a.  RESID: nonlinear
// stress, tension bits written to tb; otherwise the frozen-indicator tangent with bits tb.
// Gauss point q has s = G[q & 1], t = G[q >> 1] with G0 + G1 = 1, so strains and the
// interpolated d separate into values per s and per t, and the force into sums over the
// two points of equal s or equal t.
template <class T, bool RESID>
__device__ __forceinline__ void elas_element(const ElemConst<T> &kc, T ux0, T ux1, T ux2, T ux3,
                                             T uy0, T uy1, T uy2, T uy3, T d0, T d1, T d2, T d3,
                                             uint8_t &tb, T (&f)[8]) {
  const T G0 = kc.G0, G1 = kc.G1, ihx = kc.ihx, ihy = kc.ihy;
  const T mu = kc.mu, K = kc.K, cd = kc.cd, eta = kc.eta;
  const T dxb = ux1 - ux0, dxt = ux3 - ux2, dyl = uy2 - uy0, dyr = uy3 - uy1;
  const T uyb = uy1 - uy0, uyt = uy3 - uy2, uxl = ux2 - ux0, uxr = ux3 - ux1;
  const T exx_lo = (G1 * dxb + G0 * dxt) * ihx, exx_hi = (G0 * dxb + G1 * dxt) * ihx;
  const T eyy_l = (G1 * dyl + G0 * dyr) * ihy, eyy_r = (G0 * dyl + G1 * dyr) * ihy;
  const T uxy_l = (G1 * uxl + G0 * uxr) * ihy, uxy_r = (G0 * uxl + G1 * uxr) * ihy;
  const T uyx_lo = (G1 * uyb + G0 * uyt) * ihx, uyx_hi = (G0 * uyb + G1 * uyt) * ihx;
  const T dbl = G1 * d0 + G0 * d1, dbr = G0 * d0 + G1 * d1;
  const T dtl = G1 * d2 + G0 * d3, dtr = G0 * d2 + G1 * d3;
  const T dqv[4] = {G1 * dbl + G0 * dtl, G1 * dbr + G0 * dtr, G0 * dbl + G1 * dtl,
                    G0 * dbr + G1 * dtr};
  const T exv[4] = {exx_lo, exx_lo, exx_hi, exx_hi};
  const T eyv[4] = {eyy_l, eyy_r, eyy_l, eyy_r};
  const T gxv[4] = {uxy_l + uyx_lo, uxy_r + uyx_lo, uxy_l + uyx_hi, uxy_r + uyx_hi};
  T P[4], Q[4], R[4], U[4];
  const T wx = kc.w * ihx, wy = kc.w * ihy;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T om = T(1) - dqv[q];
    const T gq = om * om + eta;
    const T exx = exv[q], eyy = eyv[q], tr = exx + eyy;
    T vol;
    if (RESID) {
      vol = tr > T(0) ? gq * K * tr : K * tr;
      if (tr > T(0)) tb |= (uint8_t)(1u << q);
    } else {
      vol = ((tb >> q) & 1) ? gq * K * tr : K * tr;
    }
    const T gm2 = gq * T(2) * mu;
    const T sxy = gq * mu * gxv[q];
    P[q] = wx * (gm2 * (exx - cd * tr) + vol);
    U[q] = wy * (gm2 * (eyy - cd * tr) + vol);
    Q[q] = wy * sxy;
    R[q] = wx * sxy;
  }
  // t-sums (points 0,1 have t = G0; 2,3 have t = G1), s-sums (0,2: G0; 1,3: G1)
  const T Plo = P[0] + P[1], Phi = P[2] + P[3], Rlo = R[0] + R[1], Rhi = R[2] + R[3];
  const T Ql = Q[0] + Q[2], Qr = Q[1] + Q[3], Ul = U[0] + U[2], Ur = U[1] + U[3];
  const T P1 = G1 * Plo + G0 * Phi, P2 = G0 * Plo + G1 * Phi;   // sum (1-t) P, sum t P
  const T R1 = G1 * Rlo + G0 * Rhi, R2 = G0 * Rlo + G1 * Rhi;
  const T Q1 = G1 * Ql + G0 * Qr, Q2 = G0 * Ql + G1 * Qr;       // sum (1-s) Q, sum s Q
  const T U1 = G1 * Ul + G0 * Ur, U2 = G0 * Ul + G1 * Ur;
  f[0] = -P1 - Q1;
  f[1] = -R1 - U1;
  f[2] = P1 - Q2;
  f[3] = R1 - U2;
  f[4] = -P2 + Q1;
  f[5] = -R2 + U1;
  f[6] = P2 + Q2;
  f[7] = R2 + U2;
}

// FP32 tangent element in packed FP32x2 arithmetic (sm_100 family: one FFMA2 / FADD2 /
// FMUL2 instruction does two FP32 operations).  Same operations as elas_element<float,false>
// with the Gauss points paired by equal t: lo = (q0, q1), hi = (q2, q3); .x has s = G0, .y
// has s = G1.  The kernel is issue-bound at large grids, so halving the arithmetic
// instructions shortens it.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }
__device__ __forceinline__ void elas_element_tangent_f2(const ElemConst<float> &kc, float ux0,
                                                        float ux1, float ux2, float ux3,
                                                        float uy0, float uy1, float uy2,
                                                        float uy3, float d0, float d1, float d2,
                                                        float d3, uint8_t tb, float (&f)[8]) {
  const float G0 = kc.G0, G1 = kc.G1;
  const float2 Ga = f2(G1, G0), Gb = f2(G0, G1), m1 = f2b(-1.f);
  // nodal differences: (dxb, dxt), (dyl, dyr), (uyb, uyt), (uxl, uxr)
  const float2 dx = __ffma2_rn(m1, f2(ux0, ux2), f2(ux1, ux3));
  const float2 dy = __ffma2_rn(m1, f2(uy0, uy1), f2(uy2, uy3));
  const float2 duy = __ffma2_rn(m1, f2(uy0, uy2), f2(uy1, uy3));
  const float2 dux = __ffma2_rn(m1, f2(ux0, ux1), f2(ux2, ux3));
  // (lo, hi) or (l, r) pairs of the separable strain interpolants
  const float2 exx = __fmul2_rn(__ffma2_rn(Ga, f2b(dx.x), __fmul2_rn(Gb, f2b(dx.y))), f2b(kc.ihx));
  const float2 eyy = __fmul2_rn(__ffma2_rn(Ga, f2b(dy.x), __fmul2_rn(Gb, f2b(dy.y))), f2b(kc.ihy));
  const float2 uxy = __fmul2_rn(__ffma2_rn(Ga, f2b(dux.x), __fmul2_rn(Gb, f2b(dux.y))), f2b(kc.ihy));
  const float2 uyx = __fmul2_rn(__ffma2_rn(Ga, f2b(duy.x), __fmul2_rn(Gb, f2b(duy.y))), f2b(kc.ihx));
  // d at the points: db = (dbl, dbr), dt = (dtl, dtr); lo = G1 db + G0 dt, hi = G0 db + G1 dt
  const float2 db = __ffma2_rn(Ga, f2b(d0), __fmul2_rn(Gb, f2b(d1)));
  const float2 dt = __ffma2_rn(Ga, f2b(d2), __fmul2_rn(Gb, f2b(d3)));
  const float2 dq[2] = {__ffma2_rn(f2b(G1), db, __fmul2_rn(f2b(G0), dt)),
                        __ffma2_rn(f2b(G0), db, __fmul2_rn(f2b(G1), dt))};
  const float2 exv[2] = {f2b(exx.x), f2b(exx.y)};
  const float2 gxv[2] = {__fadd2_rn(uxy, f2b(uyx.x)), __fadd2_rn(uxy, f2b(uyx.y))};
  const float2 wx = f2b(kc.w * kc.ihx), wy = f2b(kc.w * kc.ihy);
  const float2 one = f2b(1.f), eta = f2b(kc.eta), Kv = f2b(kc.K), mcd = f2b(-kc.cd);
  const float2 mu2 = f2b(2.f * kc.mu), muv = f2b(kc.mu);
  float2 P[2], Q[2], R[2], U[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 om = __ffma2_rn(m1, dq[h], one);
    const float2 gq = __ffma2_rn(om, om, eta);
    const float2 tr = __fadd2_rn(exv[h], eyy);
    const float2 gsel = f2(((tb >> (2 * h)) & 1) ? gq.x : 1.f, ((tb >> (2 * h + 1)) & 1) ? gq.y : 1.f);
    const float2 vol = __fmul2_rn(__fmul2_rn(Kv, tr), gsel);
    const float2 gm2 = __fmul2_rn(gq, mu2);
    const float2 sxy = __fmul2_rn(__fmul2_rn(gq, muv), gxv[h]);
    P[h] = __fmul2_rn(wx, __ffma2_rn(gm2, __ffma2_rn(mcd, tr, exv[h]), vol));
    U[h] = __fmul2_rn(wy, __ffma2_rn(gm2, __ffma2_rn(mcd, tr, eyy), vol));
    Q[h] = __fmul2_rn(wy, sxy);
    R[h] = __fmul2_rn(wx, sxy);
  }
  // t-sums over the pair (.x + .y), s-sums across the pairs (lo + hi)
  const float Plo = P[0].x + P[0].y, Phi = P[1].x + P[1].y;
  const float Rlo = R[0].x + R[0].y, Rhi = R[1].x + R[1].y;
  const float2 QlQr = __fadd2_rn(Q[0], Q[1]), UlUr = __fadd2_rn(U[0], U[1]);
  const float2 P12 = __ffma2_rn(Ga, f2b(Plo), __fmul2_rn(Gb, f2b(Phi)));    // (P1, P2)
  const float2 R12 = __ffma2_rn(Ga, f2b(Rlo), __fmul2_rn(Gb, f2b(Rhi)));
  const float2 Q12 = __ffma2_rn(Ga, f2b(QlQr.x), __fmul2_rn(Gb, f2b(QlQr.y)));
  const float2 U12 = __ffma2_rn(Ga, f2b(UlUr.x), __fmul2_rn(Gb, f2b(UlUr.y)));
  f[0] = -P12.x - Q12.x;
  f[1] = -R12.x - U12.x;
  f[2] = P12.x - Q12.y;
  f[3] = R12.x - U12.y;
  f[4] = -P12.y + Q12.x;
  f[5] = -R12.y + U12.x;
  f[6] = P12.y + Q12.y;
  f[7] = R12.y + U12.y;
}

// Diagonal of the elasticity tangent (Jacobi preconditioner, multigrid smoother data for
// the matrix-free level): one tile of TX x TY nodes per CTA, d staged in shared memory with
// a one-node halo, element diagonals of the (TX+1) x (TY+1) touching elements summed per
// node.
template <class T>
__global__ void __launch_bounds__(TILE_THREADS, sizeof(T) == 4 ? 8 : 4)
k_elas_diag(GridD g, ElemConst<T> kc, const T *__restrict__ d, const uint8_t *__restrict__ tens,
            T *__restrict__ y) {
  constexpr int PX = TX + 2, PY = TY + 2, EX = TX + 1, EY = TY + 1, NE = EX * EY;
  __shared__ T sd[PY * PX];
  __shared__ T ef[8][NE];
  const int nx = g.nx, ny = g.ny, ld = nx + 1;
  const int tbx = (nx + 1 + TX - 1) / TX, ntiles = tbx * ((ny + 1 + TY - 1) / TY);
  const T ihx = kc.ihx, ihy = kc.ihy, w = kc.w;
  const T mu = kc.mu, K = kc.K, cd = kc.cd, eta = kc.eta;
  const T G0 = kc.G0, G1 = kc.G1;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (tile % tbx) * TX, j0 = (tile / tbx) * TY;
    for (int t = threadIdx.x; t < PX * PY; t += TILE_THREADS) {
      const int li = t % PX, lj = t / PX;
      const int gi = i0 - 1 + li, gj = j0 - 1 + lj;
      const bool in = gi >= 0 && gi <= nx && gj >= 0 && gj <= ny;
      sd[t] = in ? ldg(d + (size_t)gj * ld + gi) : T(0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NE; t += TILE_THREADS) {
      const int le = t % EX, me = t / EX;
      const int ei = i0 - 1 + le, ej = j0 - 1 + me;
      T f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = T(0);
      bool live = ei >= 0 && ei < nx && ej >= 0 && ej < ny;
      size_t e = 0;
      if (live) {
        e = (size_t)ej * nx + ei;
        if (g.active && !ldg(g.active + e)) live = false;
      }
      if (live) {
        const int p0 = me * PX + le, p1 = p0 + 1, p2 = p0 + PX, p3 = p2 + 1;
        const T d0 = sd[p0], d1 = sd[p1], d2 = sd[p2], d3 = sd[p3];
        const uint8_t tb = ldg(tens + e);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T s = (q & 1) ? G1 : G0, tt = (q & 2) ? G1 : G0;
          const T s1 = T(1) - s, t1 = T(1) - tt;
          const T dq = s1 * t1 * d0 + s * t1 * d1 + s1 * tt * d2 + s * tt * d3;
          const T om = T(1) - dq;
          const T gq = om * om + eta;
          const T kv = ((tb >> q) & 1) ? gq * K : K;
          const T Dn = gq * T(2) * mu * (T(1) - cd) + kv;  // D00 = D11
          const T Ds = gq * mu;                              // D22
          // dN/dx: (-t1, t1, -tt, tt)*ihx ; dN/dy: (-s1, -s, s1, s)*ihy
          const T ax[4] = {t1 * ihx, t1 * ihx, tt * ihx, tt * ihx};
          const T ay[4] = {s1 * ihy, s * ihy, s1 * ihy, s * ihy};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            f[2 * a] += w * (Dn * ax[a] * ax[a] + Ds * ay[a] * ay[a]);
            f[2 * a + 1] += w * (Dn * ay[a] * ay[a] + Ds * ax[a] * ax[a]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) ef[k][t] = f[k];
    }
    __syncthreads();
    const int li = threadIdx.x % TX, lj = threadIdx.x / TX;
    const int gi = i0 + li, gj = j0 + lj;
    if (lj < TY && gi <= nx && gj <= ny) {
      const int e00 = lj * EX + li, e10 = e00 + 1, e01 = e00 + EX, e11 = e01 + 1;
      T fx = ef[6][e00] + ef[4][e10] + ef[2][e01] + ef[0][e11];
      T fy = ef[7][e00] + ef[5][e10] + ef[3][e01] + ef[1][e11];
      const size_t n = (size_t)gj * ld + gi;
      if (g.dofm) {
        const uint8_t mk = ldg(g.dofm + n);
        if (mk & 1) fx = T(0);
        if (mk & 2) fy = T(0);
      }
      y[2 * n] = fx;
      y[2 * n + 1] = fy;
    }
    __syncthreads();
  }  // tiles
}

// ------------------------------------------------------------------------------------
// Strip form of the elasticity tangent apply (the Krylov hot loop).  A warp owns 32 node
// columns and marches up SR node rows, keeping the row below in registers; the right
// neighbour's column comes by warp shuffle.  Lane k computes element (c0 + k, j) for
// k < 31 and outputs node column c0 + k for 1 <= k <= 30, so a node is read ~1.07 times
// and an element computed ~1.03 times per row step, with no shared memory or CTA
// barrier.  Node (i, j) sums a0 of its own element, a1 of the left lane's element (same
// row) and, carried from the previous row step, a2 of its own and a3 of the left lane's.
// ------------------------------------------------------------------------------------
constexpr int SW = 30;          // output node columns per warp
constexpr int STRIP_WARPS = 4;  // warps per CTA

// SR node rows per warp: short strips on small grids (more warps to hide latency), long
// strips on large ones (less halo re-reading).
// RESID: internal force of the nonlinear stress law instead of the tangent product; the
// element's tension bits are computed and stored (by the lane and row that own the element).
template <class T, int SR, class Op, bool RESID = false>
__device__ __forceinline__ void elas_strip_body(unsigned bid, unsigned nblk, const GridD &g,
                                                const ElemConst<T> &kc,
                                                const T *__restrict__ d,
                                                uint8_t *__restrict__ tens, Op op,
                                                const RedWs &ws) {
  constexpr int NR = Op::NR > 0 ? Op::NR : 1;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nx = g.nx, ny = g.ny, ld = nx + 1;
  const int nstrips = (nx + 1 + SW - 1) / SW, nchunks = (ny + 1 + SR - 1) / SR;
  const int gw = bid * STRIP_WARPS + (threadIdx.x >> 5);
  const int strip = gw % nstrips, chunk = gw / nstrips;
  op.begin();
  T acc[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) acc[k] = T(0);
  if (chunk < nchunks) {
    const int i = strip * SW - 1 + lane;
    const int r0 = chunk * SR;
    const bool col_ok = i >= 0 && i <= nx;
    auto load = [&](int j, T &vx, T &vy, T &vd) {
      vx = vy = vd = T(0);
      if (col_ok && j >= 0 && j <= ny) {
        const size_t n = (size_t)j * ld + i;
        T v[2];
        op.in(n, i, j, v);
        vx = v[0];
        vy = v[1];
        vd = ldg(d + n);
        if (g.dofm) {
          const uint8_t mk = ldg(g.dofm + n);
          if (mk & 1) vx = T(0);
          if (mk & 2) vy = T(0);
        }
      }
    };
    // Short strips (SR <= 4) load all SR + 2 input rows up front, so the chunk pays one
    // memory round trip instead of one per row; long strips stream the rows.
    constexpr int PF = SR <= 4 ? SR + 2 : 1;
    T px[PF], py[PF], pd[PF];
    if (PF > 1) {
#pragma unroll
      for (int r = 0; r < PF; ++r) load(r0 - 1 + r, px[r], py[r], pd[r]);
    }
    T cx, cy, cdv;
    if (PF > 1) {
      cx = px[0];
      cy = py[0];
      cdv = pd[0];
    } else {
      load(r0 - 1, cx, cy, cdv);
    }
    T carry_x = T(0), carry_y = T(0);
#pragma unroll
    for (int j = r0 - 1; j < r0 + SR; ++j) {
      T nxv, nyv, ndv;
      if (PF > 1) {
        nxv = px[j - r0 + 2];
        nyv = py[j - r0 + 2];
        ndv = pd[j - r0 + 2];
      } else {
        load(j + 1, nxv, nyv, ndv);
      }
      const T rx0 = __shfl_down_sync(FULL, cx, 1), ry0 = __shfl_down_sync(FULL, cy, 1);
      const T rd0 = __shfl_down_sync(FULL, cdv, 1);
      const T rx1 = __shfl_down_sync(FULL, nxv, 1), ry1 = __shfl_down_sync(FULL, nyv, 1);
      const T rd1 = __shfl_down_sync(FULL, ndv, 1);
      T f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = T(0);
      if (lane < 31 && i >= 0 && i < nx && j >= 0 && j < ny) {
        const size_t e = (size_t)j * nx + i;
        if (!g.active || ldg(g.active + e)) {
          if (RESID) {
            uint8_t tb = 0;
            elas_element<T, true>(kc, cx, rx0, nxv, rx1, cy, ry0, nyv, ry1, cdv, rd0, ndv, rd1, tb, f);
            if (tens && j >= r0 && lane >= 1) tens[e] = tb;   // tens may be NULL
          } else {
            uint8_t tb = ldg(tens + e);
            if constexpr (sizeof(T) == 4)
              elas_element_tangent_f2(kc, cx, rx0, nxv, rx1, cy, ry0, nyv, ry1, cdv, rd0, ndv, rd1,
                                      tb, f);
            else
              elas_element<T, false>(kc, cx, rx0, nxv, rx1, cy, ry0, nyv, ry1, cdv, rd0, ndv, rd1,
                                     tb, f);
          }
        }
      }
      const T lx1 = __shfl_up_sync(FULL, f[2], 1), ly1 = __shfl_up_sync(FULL, f[3], 1);
      const T lx3 = __shfl_up_sync(FULL, f[6], 1), ly3 = __shfl_up_sync(FULL, f[7], 1);
      if (j >= r0 && j <= ny && lane >= 1 && lane <= SW && col_ok) {
        T ox = f[0] + lx1 + carry_x, oy = f[1] + ly1 + carry_y;
        const size_t n = (size_t)j * ld + i;
        if (g.dofm) {
          const uint8_t mk = ldg(g.dofm + n);
          if (mk & 1) ox = T(0);
          if (mk & 2) oy = T(0);
        }
        const T o[2] = {ox, oy}, ci[2] = {cx, cy};
        op.out(n, o, ci, acc);
      }
      carry_x = f[4] + lx3;
      carry_y = f[5] + ly3;
      cx = nxv;
      cy = nyv;
      cdv = ndv;
    }
  }
  if (Op::NR > 0 && op.reduce()) {
    double v[NR], tot[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = (double)acc[k];
    if (red_grid<NR>(v, ws, tot, false, bid, nblk)) op.fin(tot);
  }
}

template <class T, int SR, class Op, bool RESID = false>
__global__ void __launch_bounds__(32 * STRIP_WARPS)
k_elas_strip(GridD g, ElemConst<T> kc, const T *__restrict__ d, uint8_t *__restrict__ tens,
             Op op, RedWs ws) {
  pdl_enter();
  elas_strip_body<T, SR, Op, RESID>(blockIdx.x, gridDim.x, g, kc, d, tens, op, ws);
}

// One simulation's share of a batched strip launch (pf_batch.cuh).
template <class T, int SR, class Op>
struct StripF {
  GridD g;
  ElemConst<T> kc;
  const T *d;
  const uint8_t *tens;
  Op op;
  RedWs ws;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    elas_strip_body<T, SR, Op, false>(bid, nblk, g, kc, d, const_cast<uint8_t *>(tens), op, ws);
  }
};

// ------------------------------------------------------------------------------------
// Evolution equation: K_dd diagonal / AT2 right-hand side (one tile of nodes per CTA,
// element values staged in shared memory) and the K_dd apply (k_damage_op below).
// ------------------------------------------------------------------------------------
enum { DM_DIAG = 1, DM_RHS = 2 };

template <class T, class C, int MODE>
__global__ void __launch_bounds__(TILE_THREADS, sizeof(T) == 4 ? 8 : 4)
k_damage(GridD g, ElemConst<T> kc, const C *__restrict__ c, T *__restrict__ y) {
  constexpr int EX = TX + 1, EY = TY + 1, NE = EX * EY;
  __shared__ T ef[4][NE];
  const int nx = g.nx, ny = g.ny, ld = nx + 1;
  const int tbx = (nx + 1 + TX - 1) / TX, ntiles = tbx * ((ny + 1 + TY - 1) / TY);
  const T ihx = kc.ihx, ihy = kc.ihy, w = kc.w;
  const T kappa = kc.kappa;
  const T G0 = kc.G0, G1 = kc.G1;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (tile % tbx) * TX, j0 = (tile / tbx) * TY;
    for (int t = threadIdx.x; t < NE; t += TILE_THREADS) {
      const int le = t % EX, me = t / EX;
      const int ei = i0 - 1 + le, ej = j0 - 1 + me;
      T f[4] = {T(0), T(0), T(0), T(0)};
      bool live = ei >= 0 && ei < nx && ej >= 0 && ej < ny;
      size_t e = 0;
      if (live) {
        e = (size_t)ej * nx + ei;
        if (g.active && !ldg(g.active + e)) live = false;
      }
      if (live) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T s = (q & 1) ? G1 : G0, tt = (q & 2) ? G1 : G0;
          const T s1 = T(1) - s, t1 = T(1) - tt;
          const T N[4] = {s1 * t1, s * t1, s1 * tt, s * tt};
          const T cq = T(ldg(c + 4 * e + q));
          if (MODE == DM_RHS) {
#pragma unroll
            for (int a = 0; a < 4; ++a) f[a] += w * T(2) * cq * N[a];
          } else {
            const T ax[4] = {t1 * ihx, t1 * ihx, tt * ihx, tt * ihx};
            const T ay[4] = {s1 * ihy, s * ihy, s1 * ihy, s * ihy};
#pragma unroll
            for (int a = 0; a < 4; ++a)
              f[a] += w * (cq * N[a] * N[a] + kappa * (ax[a] * ax[a] + ay[a] * ay[a]));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) ef[k][t] = f[k];
    }
    __syncthreads();
    const int li = threadIdx.x % TX, lj = threadIdx.x / TX;
    const int gi = i0 + li, gj = j0 + lj;
    if (lj < TY && gi <= nx && gj <= ny) {
      const int e00 = lj * EX + li, e10 = e00 + 1, e01 = e00 + EX, e11 = e01 + 1;
      T v = ef[3][e00] + ef[2][e10] + ef[1][e01] + ef[0][e11];
      const size_t n = (size_t)gj * ld + gi;
      if (MODE != DM_RHS && g.dofm && (ldg(g.dofm + n) & 4)) v = T(0);
      y[n] = v;
    }
    __syncthreads();
  }  // tiles
}

// K_dd x with an input/output policy (pf_fused.cuh, B = 1): the tile form of k_damage's
// apply, the operand formed by op.in() while the CTA stages its node patch and the product
// handed to op.out() at each owned node.
template <class T, class Op>
__device__ __forceinline__ void damage_op_body(unsigned bid, unsigned nblk, const GridD &g,
                                               const ElemConst<T> &kc, const T *__restrict__ c,
                                               Op op, const RedWs &ws) {
  constexpr int PX = TX + 2, PY = TY + 2, EX = TX + 1, EY = TY + 1, NE = EX * EY;
  constexpr int NR = Op::NR > 0 ? Op::NR : 1;
  __shared__ T sxv[PY * PX];
  __shared__ T ef[4][NE];
  const int nx = g.nx, ny = g.ny, ld = nx + 1;
  const int tbx = (nx + 1 + TX - 1) / TX, ntiles = tbx * ((ny + 1 + TY - 1) / TY);
  op.begin();
  T acc[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) acc[k] = T(0);
  const T ihx = kc.ihx, ihy = kc.ihy, w = kc.w;
  const T kappa = kc.kappa;
  const T G0 = kc.G0, G1 = kc.G1;
  for (int tile = (int)bid; tile < ntiles; tile += (int)nblk) {
    const int i0 = (tile % tbx) * TX, j0 = (tile / tbx) * TY;
    for (int t = threadIdx.x; t < PX * PY; t += TILE_THREADS) {
      const int li = t % PX, lj = t / PX;
      const int gi = i0 - 1 + li, gj = j0 - 1 + lj;
      T v[1] = {T(0)};
      if (gi >= 0 && gi <= nx && gj >= 0 && gj <= ny) {
        const size_t n = (size_t)gj * ld + gi;
        op.in(n, gi, gj, v);
        if (g.dofm && (ldg(g.dofm + n) & 4)) v[0] = T(0);
      }
      sxv[t] = v[0];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NE; t += TILE_THREADS) {
      const int le = t % EX, me = t / EX;
      const int ei = i0 - 1 + le, ej = j0 - 1 + me;
      T f[4] = {T(0), T(0), T(0), T(0)};
      bool live = ei >= 0 && ei < nx && ej >= 0 && ej < ny;
      size_t e = 0;
      if (live) {
        e = (size_t)ej * nx + ei;
        if (g.active && !ldg(g.active + e)) live = false;
      }
      if (live) {
        const int p0 = me * PX + le;
        const T x0 = sxv[p0], x1 = sxv[p0 + 1], x2 = sxv[p0 + PX], x3 = sxv[p0 + PX + 1];
        // separable form over the Gauss points (s = G[q & 1], t = G[q >> 1], G0 + G1 = 1)
        const T xbl = G1 * x0 + G0 * x1, xbr = G0 * x0 + G1 * x1;
        const T xtl = G1 * x2 + G0 * x3, xtr = G0 * x2 + G1 * x3;
        const T xq[4] = {G1 * xbl + G0 * xtl, G1 * xbr + G0 * xtr, G0 * xbl + G1 * xtl,
                         G0 * xbr + G1 * xtr};
        T m[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) m[q] = w * ldg(c + 4 * e + q) * xq[q];
        const T ml_lo = G1 * m[0] + G0 * m[1], mr_lo = G0 * m[0] + G1 * m[1];
        const T ml_hi = G1 * m[2] + G0 * m[3], mr_hi = G0 * m[2] + G1 * m[3];
        const T bx = x1 - x0, tx = x3 - x2, ly = x2 - x0, ry = x3 - x1;
        const T gx_lo = G1 * bx + G0 * tx, gx_hi = G0 * bx + G1 * tx;   // times ihx
        const T gy_l = G1 * ly + G0 * ry, gy_r = G0 * ly + G1 * ry;     // times ihy
        const T cxx = T(2) * w * kappa * ihx * ihx, cyy = T(2) * w * kappa * ihy * ihy;
        const T kx1 = cxx * (G1 * gx_lo + G0 * gx_hi), kx2 = cxx * (G0 * gx_lo + G1 * gx_hi);
        const T ky1 = cyy * (G1 * gy_l + G0 * gy_r), ky2 = cyy * (G0 * gy_l + G1 * gy_r);
        f[0] = G1 * ml_lo + G0 * ml_hi - kx1 - ky1;
        f[1] = G1 * mr_lo + G0 * mr_hi + kx1 - ky2;
        f[2] = G0 * ml_lo + G1 * ml_hi - kx2 + ky1;
        f[3] = G0 * mr_lo + G1 * mr_hi + kx2 + ky2;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) ef[k][t] = f[k];
    }
    __syncthreads();
    const int li = threadIdx.x % TX, lj = threadIdx.x / TX;
    const int gi = i0 + li, gj = j0 + lj;
    if (lj < TY && gi <= nx && gj <= ny) {
      const int e00 = lj * EX + li, e10 = e00 + 1, e01 = e00 + EX, e11 = e01 + 1;
      T o[1] = {ef[3][e00] + ef[2][e10] + ef[1][e01] + ef[0][e11]};
      const size_t n = (size_t)gj * ld + gi;
      if (g.dofm && (ldg(g.dofm + n) & 4)) o[0] = T(0);
      const T ci[1] = {sxv[(lj + 1) * PX + li + 1]};
      op.out(n, o, ci, acc);
    }
    __syncthreads();
  }  // tiles
  if (Op::NR > 0 && op.reduce()) {
    double v[NR], tot[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = (double)acc[k];
    if (red_grid<NR>(v, ws, tot, false, bid, nblk)) op.fin(tot);
  }
}

template <class T, class Op>
__global__ void __launch_bounds__(TILE_THREADS, sizeof(T) == 4 ? 8 : 4)
k_damage_op(GridD g, ElemConst<T> kc, const T *__restrict__ c, Op op, RedWs ws) {
  pdl_enter();
  damage_op_body<T, Op>(blockIdx.x, gridDim.x, g, kc, c, op, ws);
}

// One simulation's share of a batched K_dd launch (pf_batch.cuh).
template <class T, class Op>
struct DamageF {
  GridD g;
  ElemConst<T> kc;
  const T *c;
  Op op;
  RedWs ws;
  __device__ void operator()(unsigned bid, unsigned nblk) const {
    damage_op_body<T, Op>(bid, nblk, g, kc, c, op, ws);
  }
};

// ------------------------------------------------------------------------------------
// Per-Gauss-point kernels (one thread per element, FP64).
// ------------------------------------------------------------------------------------
struct QpStrain {
  double exx[4], eyy[4], exy[4];
};

__device__ __forceinline__ void element_nodes(const GridD &g, size_t e, size_t (&n)[4]) {
  const int ei = (int)(e % g.nx), ej = (int)(e / g.nx);
  const size_t ld = (size_t)g.nx + 1;
  n[0] = (size_t)ej * ld + ei;
  n[1] = n[0] + 1;
  n[2] = n[0] + ld;
  n[3] = n[2] + 1;
}

__device__ __forceinline__ void element_strains(const GridD &g, const double *u,
                                                const size_t (&n)[4], QpStrain &S) {
  double ux[4], uy[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(u) + n[a]);
    ux[a] = v.x;
    uy[a] = v.y;
  }
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double s = (q & 1) ? gp_hi() : gp_lo(), t = (q & 2) ? gp_hi() : gp_lo();
    const double s1 = 1.0 - s, t1 = 1.0 - t;
    S.exx[q] = (t1 * (ux[1] - ux[0]) + t * (ux[3] - ux[2])) * ihx;
    S.eyy[q] = (s1 * (uy[2] - uy[0]) + s * (uy[3] - uy[1])) * ihy;
    S.exy[q] = 0.5 * ((s1 * (ux[2] - ux[0]) + s * (ux[3] - ux[1])) * ihy +
                      (t1 * (uy[1] - uy[0]) + t * (uy[3] - uy[2])) * ihx);
  }
}

__device__ __forceinline__ void element_interp(const double *f, const size_t (&n)[4],
                                               double (&fq)[4]) {
  const double f0 = __ldg(f + n[0]), f1 = __ldg(f + n[1]), f2 = __ldg(f + n[2]),
               f3 = __ldg(f + n[3]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double s = (q & 1) ? gp_hi() : gp_lo(), t = (q & 2) ? gp_hi() : gp_lo();
    fq[q] = (1.0 - s) * (1.0 - t) * f0 + s * (1.0 - t) * f1 + (1.0 - s) * t * f2 + s * t * f3;
  }
}

__device__ __forceinline__ void invariants(const MatD &m, double exx, double eyy, double exy,
                                           double &tr, double &ee) {
  tr = exx + eyy;
  ee = exx * exx + eyy * eyy + 2.0 * exy * exy - m.cdim * tr * tr;
}

__device__ __forceinline__ double psi_plus(const MatD &m, double tr, double ee) {
  const double tp = tr > 0.0 ? tr : 0.0;
  return m.mu * ee + 0.5 * m.K * tp * tp;
}

__global__ void k_qp_energy(GridD g, MatD m, const double *__restrict__ u,
                            const double *__restrict__ Hprev, double *__restrict__ psi,
                            double *__restrict__ Hout) {
  const size_t ne = (size_t)g.nx * g.ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    double p[4] = {0, 0, 0, 0};
    if (live) {
      size_t n[4];
      element_nodes(g, e, n);
      QpStrain S;
      element_strains(g, u, n, S);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double tr, ee;
        invariants(m, S.exx[q], S.eyy[q], S.exy[q], tr, ee);
        p[q] = psi_plus(m, tr, ee);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Hout[4 * e + q] = fmax(__ldg(Hprev + 4 * e + q), p[q]);
      if (psi) psi[4 * e + q] = p[q];
    }
  }
}

__device__ __forceinline__ double scheme_Q(const MatD &m, int scheme, double tr, double ee) {
  const double tp = tr > 0.0 ? tr : 0.0;
  const double vol = m.K * tp * tp, dev = 2.0 * m.mu * ee;
  return scheme == PF_S1 ? vol : scheme == PF_S2 ? dev : scheme == PF_S3 ? vol + dev : 0.0;
}

// AT1 with penalty (Sec. 2): per-point arrays of the evolution equation at energy psi,
//   R_d = K(c0) d - b,  c0 = 2 psi,  b = int (2 psi - a - gamma <d - d_{n-1}>_-) N,
//   Jacobian mass coefficient cJ = 2 psi + gamma [d < d_{n-1}]  (d at the point, strict),
// with bhalf = b's integrand / 2 (damage_rhs integrates 2 (.) N).
__global__ void k_at1_coef(GridD g, const double *__restrict__ psi, const double *__restrict__ d,
                           const double *__restrict__ dprev, double a, double gamma,
                           double *__restrict__ c0, double *__restrict__ cJ,
                           double *__restrict__ bhalf) {
  const size_t ne = (size_t)g.nx * g.ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t n[4];
    element_nodes(g, e, n);
    double dq[4], dpq[4];
    element_interp(d, n, dq);
    element_interp(dprev, n, dpq);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double ps = __ldg(psi + 4 * e + q);
      const double diff = dq[q] - dpq[q];
      c0[4 * e + q] = 2.0 * ps;
      cJ[4 * e + q] = 2.0 * ps + (diff < 0.0 ? gamma : 0.0);
      bhalf[4 * e + q] = 0.5 * (2.0 * ps - a - gamma * (diff < 0.0 ? diff : 0.0));
    }
  }
}

__global__ void k_fs_coeff(GridD g, MatD m, int scheme, double psi_crit,
                           const double *__restrict__ u, const double *__restrict__ d,
                           const double *__restrict__ Hprev, double *__restrict__ c_aug,
                           uint8_t *__restrict__ active, At1D at1) {
  const size_t ne = (size_t)g.nx * g.ny;
  const double floor_c = at1.on ? at1.floor : m.Gc / m.l;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    size_t n[4];
    element_nodes(g, e, n);
    QpStrain S;
    double dq[4], dpq[4];
    if (live) {
      element_strains(g, u, n, S);
      element_interp(d, n, dq);
      if (at1.on) element_interp(at1.dprev, n, dpq);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double hp = __ldg(Hprev + 4 * e + q);
      double c = at1.on ? 0.0 : floor_c + 2.0 * hp;
      uint8_t a = 0;
      if (live) {
        double tr, ee;
        invariants(m, S.exx[q], S.eyy[q], S.exy[q], tr, ee);
        const double ps = psi_plus(m, tr, ee);
        // Jacobian mass coefficient: AT2 G_c/l + 2H; AT1 2 Psi+ (+ gamma where penalised)
        const double cJ = at1.on ? 2.0 * ps + (dq[q] < dpq[q] ? at1.gamma : 0.0)
                                 : floor_c + 2.0 * fmax(hp, ps);
        c = cJ;
        a = (ps > psi_crit) && (ps > hp) && (dq[q] < 0.95);
        if (a) {
          const double om = 1.0 - dq[q];
          const double gq = om * om + m.eta;
          const double lim = at1.on ? fmin(cJ, floor_c) : floor_c;
          c = fmax(cJ - 4.0 * om * om / gq * scheme_Q(m, scheme, tr, ee), lim);
        }
      }
      c_aug[4 * e + q] = c;
      active[4 * e + q] = a;
    }
  }
}

__global__ void k_fs_predict(GridD g, MatD m, int scheme, const double *__restrict__ u,
                             const double *__restrict__ d, const double *__restrict__ dd,
                             const double *__restrict__ Hprev,
                             const uint8_t *__restrict__ active, double *__restrict__ Hhalf,
                             int at1) {
  const size_t ne = (size_t)g.nx * g.ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool live = !g.active || g.active[e];
    size_t n[4];
    element_nodes(g, e, n);
    QpStrain S;
    double dq[4], ddq[4];
    if (live) {
      element_strains(g, u, n, S);
      element_interp(d, n, dq);
      element_interp(dd, n, ddq);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double hp = __ldg(Hprev + 4 * e + q);
      double h = hp;
      if (live) {
        double tr, ee;
        invariants(m, S.exx[q], S.eyy[q], S.exy[q], tr, ee);
        double ps = psi_plus(m, tr, ee);
        if (active[4 * e + q]) {
          const double om = 1.0 - dq[q];
          const double gq = om * om + m.eta;
          const double ddp = ddq[q] > 0.0 ? ddq[q] : 0.0;
          const double sc = 1.0 + 2.0 * om / gq * ddp;  // s = 1 + a Dd+
          const double tp = tr > 0.0 ? tr : 0.0;
          const double tpn = (scheme == PF_S1 || scheme == PF_S3) ? sc * tp : tp;
          const double een = (scheme == PF_S2 || scheme == PF_S3) ? sc * sc * ee : ee;
          ps = m.mu * een + 0.5 * m.K * tpn * tpn;
        }
        h = at1 ? ps : fmax(hp, ps);   // AT1 drives d with the (predicted) energy itself
      }
      Hhalf[4 * e + q] = h;
    }
  }
}

__global__ void k_dof_mask(int nx, int ny, const uint8_t *__restrict__ flags,
                           const uint8_t *__restrict__ active, uint8_t *__restrict__ mask) {
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1)), j = (int)(n / (nx + 1));
    bool touched = true;
    if (active) {
      touched = false;
      for (int dj = -1; dj <= 0; ++dj)
        for (int di = -1; di <= 0; ++di) {
          const int ei = i + di, ej = j + dj;
          if (ei >= 0 && ei < nx && ej >= 0 && ej < ny && active[(size_t)ej * nx + ei])
            touched = true;
        }
    }
    const uint8_t f = flags[n];
    uint8_t m = 0;
    if (!touched) {
      m = 15;
    } else {
      if (f & (PF_FIX_X | PF_LOAD_X)) m |= 1;
      if (f & (PF_FIX_Y | PF_LOAD_Y)) m |= 2;
      if (f & (PF_D_FIX1 | PF_D_FIX0)) m |= 4;
    }
    mask[n] = m;
  }
}

// ------------------------------------------------------------------------------------
// Host launch wrappers.
// ------------------------------------------------------------------------------------
static inline unsigned tile_count(const GridD &g) { return tile_blocks_x(g.nx) * tile_blocks_y(g.ny); }
static inline dim3 tile_grid(const GridD &g) { return dim3(tile_count(g)); }
// Fused-reduction launches use at most red_blocks() CTAs (each loops over tiles): one
// arrival atomic per CTA on a single counter is what limits the reduction tail.
static inline dim3 tile_grid_red(const GridD &g) {
  const unsigned t = tile_count(g), cap = (unsigned)red_blocks();
  return dim3(t < cap ? t : cap);
}
static inline unsigned elem_blocks(size_t n) {
  size_t b = (n + VEC_THREADS - 1) / VEC_THREADS;
  return (unsigned)(b < 1 ? 1 : (b > 65535u * 8u ? 65535u * 8u : b));
}

// Node rows per warp of the strip kernel.  A warp also evaluates the element row below its
// chunk: SR rows cost SR + 1 element rows.  FP32 launches are latency-bound at small sizes
// (short strips, more warps); FP64 ones are bound by the FP64 pipe, so they take long
// strips to waste little arithmetic.
template <class T>
static int strip_rows(size_t nn, int sr = 0) {
  if (sr == 2 || sr == 4 || sr == 8) return sr;   // chosen by pf_autotune
  if (sizeof(T) == 8 && nn >= (size_t)100000) return 8;
  if (nn < (size_t)1500000) return 2;
  if (nn < (size_t)6000000) return 4;
  return 8;
}
static unsigned strip_blocks(const GridD &g, int sr) {
  const unsigned strips = (unsigned)((g.nx + 1 + SW - 1) / SW);
  const unsigned warps = strips * (unsigned)((g.ny + 1 + sr - 1) / sr);
  return (warps + STRIP_WARPS - 1) / STRIP_WARPS;
}

template <class T, class Op, bool RESID = false>
static void strip_launch(const GridD &g, const MatD &m, const T *d, const uint8_t *tens_c,
                         const Op &op, const RedWs &w, cudaStream_t st, int sr_req = 0) {
  uint8_t *tens = const_cast<uint8_t *>(tens_c);  // written only by the RESID form
  const size_t nn = (size_t)(g.nx + 1) * (g.ny + 1);
  const unsigned strips = (unsigned)((g.nx + 1 + SW - 1) / SW);
  auto blocks = [&](int sr) {
    const unsigned warps = strips * (unsigned)((g.ny + 1 + sr - 1) / sr);
    return (warps + STRIP_WARPS - 1) / STRIP_WARPS;
  };
  const ElemConst<T> kc = elem_const<T>(g, m);
  const int sr = strip_rows<T>(nn, sr_req);
  if (sr == 2)
    launch_pdl(k_elas_strip<T, 2, Op, RESID>, dim3(blocks(2)), dim3(32 * STRIP_WARPS), st, g, kc, d,
               tens, op, w);
  else if (sr == 4)
    launch_pdl(k_elas_strip<T, 4, Op, RESID>, dim3(blocks(4)), dim3(32 * STRIP_WARPS), st, g, kc, d,
               tens, op, w);
  else
    launch_pdl(k_elas_strip<T, 8, Op, RESID>, dim3(blocks(8)), dim3(32 * STRIP_WARPS), st, g, kc, d,
               tens, op, w);
}

template <class T>
void elas_apply(const GridD &g, const MatD &m, const T *d, const uint8_t *tens, const T *x,
                T *y, cudaStream_t st, KrylovScal *sc, const RedWs *ws, int epi, int sr) {
  const RedWs w = ws ? *ws : RedWs{nullptr, nullptr, 0};
  const int e = ws ? epi : EPI_NONE;
  strip_launch<T>(g, m, d, tens, OpApply<T, 2>{x, y, sc, e}, w, st, sr);
}

// The input/output policy of fused stage `stage` (pf_fused.cuh) on the buffers M, handed
// to f.  B = 2: elasticity, B = 1: phase field.
template <class T, int B, class F>
static void stage_op(int stage, const MgBufs<T> &M, F &&f) {
  T *rprev = M.r[0], *rcur = M.r[1], *pprev = M.p[0], *pcur = M.p[1];
  switch (stage) {
    case FS_DIR:
      f(OpDir<T, B>{M.zb, pprev, pcur, M.q, M.sc});
      break;
    case FS_UPD:
      f(OpUpd<T, B, false>{rprev, M.q, pcur, M.invd, M.coef, rcur, M.x, M.za, M.sc});
      break;
    case FS_UPD_INIT:
      f(OpUpd<T, B, true>{M.b, nullptr, nullptr, M.invd, M.coef, rcur, M.x, M.za, M.sc});
      break;
    case FS_RESID:
      f(OpResid<T, B>{M.za, rcur, M.lr});
      break;
    case FS_PROLONG:
      f(OpProlong<T, B>{M.za, M.xc, rcur, M.invd, M.coef, M.fm, M.nxc, M.nyc, M.zb, M.lr, M.dv});
      break;
    case FS_FINISH:
      f(OpFinish<T, B, false>{M.dv, M.lr, M.invd, M.coef, rcur, pcur, M.zb, rprev, pprev, M.sc});
      break;
    case FS_FINISH_FIRST:
      f(OpFinish<T, B, true>{M.dv, M.lr, M.invd, M.coef, rcur, pcur, M.zb, rprev, pprev, M.sc});
      break;
  }
}

template <class T>
void elas_mg_stage(int stage, const GridD &g, const MatD &m, const T *d, const uint8_t *tens,
                   const MgBufs<T> &B, const RedWs &ws, cudaStream_t st, int sr) {
  stage_op<T, 2>(stage, B, [&](auto op) { strip_launch<T>(g, m, d, tens, op, ws, st, sr); });
}

// Batched form: stage `stage` for n simulations in one launch per strip height (the strip
// height follows the grid size exactly as in the single launch, so a simulation's blocks
// and reductions are the same in both).
template <class T>
int elas_mg_stage_batch(int stage, int n, const ElasStageIn<T> *in, cudaStream_t st) {
  int launches = 0;
  stage_op<T, 2>(stage, in[0].B, [&](auto op0) {
    using Op = decltype(op0);
    constexpr int TH = 32 * STRIP_WARPS;
    Batcher<StripF<T, 2, Op>, TH, 8> b2;
    Batcher<StripF<T, 4, Op>, TH, 8> b4;
    Batcher<StripF<T, 8, Op>, TH, 8> b8;
    for (int i = 0; i < n; ++i) {
      const ElasStageIn<T> &q = in[i];
      const size_t nn = (size_t)(q.g.nx + 1) * (q.g.ny + 1);
      const int sr = strip_rows<T>(nn, q.sr);
      const ElemConst<T> kc = elem_const<T>(q.g, q.m);
      const int *done = &q.B.sc->done;
      stage_op<T, 2>(stage, q.B, [&](auto op) {
        if constexpr (std::is_same<decltype(op), Op>::value) {
          if (sr == 2) {
            if (b2.L.n == PF_MAXB) { launches += b2.launch(st); b2 = {}; }
            b2.add(StripF<T, 2, Op>{q.g, kc, q.d, q.tens, op, q.ws}, strip_blocks(q.g, 2), done);
          } else if (sr == 4) {
            if (b4.L.n == PF_MAXB) { launches += b4.launch(st); b4 = {}; }
            b4.add(StripF<T, 4, Op>{q.g, kc, q.d, q.tens, op, q.ws}, strip_blocks(q.g, 4), done);
          } else {
            if (b8.L.n == PF_MAXB) { launches += b8.launch(st); b8 = {}; }
            b8.add(StripF<T, 8, Op>{q.g, kc, q.d, q.tens, op, q.ws}, strip_blocks(q.g, 8), done);
          }
        }
      });
    }
    launches += b2.launch(st) + b4.launch(st) + b8.launch(st);
  });
  return launches;
}

template <class T>
void elas_diag(const GridD &g, const MatD &m, const T *d, const uint8_t *tens, T *diag,
               cudaStream_t st) {
  k_elas_diag<T><<<tile_grid(g), TILE_THREADS, 0, st>>>(g, elem_const<T>(g, m), d, tens, diag);
}
void elas_residual(const GridD &g, const MatD &m, const double *u, const double *d, double *F,
                   uint8_t *tens, cudaStream_t st) {
  // u carries the Dirichlet values and F the forces on constrained DOFs too: no masking
  GridD gu = g;
  gu.dofm = nullptr;
  strip_launch<double, OpApply<double, 2>, true>(gu, m, d, tens,
                                                 OpApply<double, 2>{u, F, nullptr, EPI_NONE},
                                                 RedWs{nullptr, nullptr, 0}, st);
}

template <class T>
void damage_apply(const GridD &g, const T *c, double kappa, const T *x, T *y, cudaStream_t st,
                  KrylovScal *sc, const RedWs *ws, int epi) {
  const RedWs w = ws ? *ws : RedWs{nullptr, nullptr, 0};
  const int e = ws ? epi : EPI_NONE;
  launch_pdl(k_damage_op<T, OpApply<T, 1>>, tile_grid(g), dim3(TILE_THREADS), st, g,
             elem_const<T>(g, MatD{}, kappa), c, OpApply<T, 1>{x, y, sc, e}, w);
}

template <class T>
void damage_mg_stage(int stage, const GridD &g, const T *c, double kappa, const MgBufs<T> &B,
                     const RedWs &ws, cudaStream_t st) {
  const ElemConst<T> kc = elem_const<T>(g, MatD{}, kappa);
  const dim3 gt = tile_grid(g);
  stage_op<T, 1>(stage, B, [&](auto op) {
    launch_pdl(k_damage_op<T, decltype(op)>, gt, dim3(TILE_THREADS), st, g, kc, c, op, ws);
  });
}

template <class T>
int damage_mg_stage_batch(int stage, int n, const DamageStageIn<T> *in, cudaStream_t st) {
  int launches = 0;
  stage_op<T, 1>(stage, in[0].B, [&](auto op0) {
    using Op = decltype(op0);
    Batcher<DamageF<T, Op>, TILE_THREADS, sizeof(T) == 4 ? 8 : 4> b;
    for (int i = 0; i < n; ++i) {
      const DamageStageIn<T> &q = in[i];
      const ElemConst<T> kc = elem_const<T>(q.g, MatD{}, q.kappa);
      stage_op<T, 1>(stage, q.B, [&](auto op) {
        if constexpr (std::is_same<decltype(op), Op>::value) {
          if (b.L.n == PF_MAXB) { launches += b.launch(st); b = {}; }
          b.add(DamageF<T, Op>{q.g, kc, q.c, op, q.ws}, tile_count(q.g), &q.B.sc->done);
        }
      });
    }
    launches += b.launch(st);
  });
  return launches;
}

template <class T>
void damage_diag(const GridD &g, const T *c, double kappa, T *diag, cudaStream_t st) {
  k_damage<T, T, DM_DIAG><<<tile_grid(g), TILE_THREADS, 0, st>>>(
      g, elem_const<T>(g, MatD{}, kappa), c, diag);
}
void damage_rhs(const GridD &g, const double *H, double *b, cudaStream_t st) {
  k_damage<double, double, DM_RHS><<<tile_grid(g), TILE_THREADS, 0, st>>>(
      g, elem_const<double>(g, MatD{}, 0.0), H, b);
}
void qp_energy(const GridD &g, const MatD &m, const double *u, const double *Hprev,
               double *psi, double *Hout, cudaStream_t st) {
  k_qp_energy<<<elem_blocks((size_t)g.nx * g.ny), VEC_THREADS, 0, st>>>(g, m, u, Hprev, psi, Hout);
}
void fs_coeff(const GridD &g, const MatD &m, int scheme, double psi_crit, const double *u,
              const double *d, const double *Hprev, double *c_aug, uint8_t *active,
              cudaStream_t st, const At1D &at1) {
  k_fs_coeff<<<elem_blocks((size_t)g.nx * g.ny), VEC_THREADS, 0, st>>>(g, m, scheme, psi_crit, u,
                                                                        d, Hprev, c_aug, active,
                                                                        at1);
}
void fs_predict(const GridD &g, const MatD &m, int scheme, const double *u, const double *d,
                const double *dd, const double *Hprev, const uint8_t *active, double *Hhalf,
                cudaStream_t st, int at1) {
  k_fs_predict<<<elem_blocks((size_t)g.nx * g.ny), VEC_THREADS, 0, st>>>(g, m, scheme, u, d, dd,
                                                                          Hprev, active, Hhalf,
                                                                          at1);
}
void at1_coef(const GridD &g, const double *psi, const double *d, const double *dprev, double a,
              double gamma, double *c0, double *cJ, double *bhalf, cudaStream_t st) {
  k_at1_coef<<<elem_blocks((size_t)g.nx * g.ny), VEC_THREADS, 0, st>>>(g, psi, d, dprev, a, gamma,
                                                                        c0, cJ, bhalf);
}
void dof_mask(int nx, int ny, const uint8_t *flags, const uint8_t *active, uint8_t *mask,
              cudaStream_t st) {
  k_dof_mask<<<elem_blocks((size_t)(nx + 1) * (ny + 1)), VEC_THREADS, 0, st>>>(nx, ny, flags,
                                                                              active, mask);
}

template void elas_apply<double>(const GridD &, const MatD &, const double *, const uint8_t *,
                                 const double *, double *, cudaStream_t, KrylovScal *,
                                 const RedWs *, int, int);
template void elas_apply<float>(const GridD &, const MatD &, const float *, const uint8_t *,
                                const float *, float *, cudaStream_t, KrylovScal *,
                                const RedWs *, int, int);
template void elas_diag<double>(const GridD &, const MatD &, const double *, const uint8_t *,
                                double *, cudaStream_t);
template void elas_diag<float>(const GridD &, const MatD &, const float *, const uint8_t *,
                               float *, cudaStream_t);
template void elas_mg_stage<double>(int, const GridD &, const MatD &, const double *,
                                    const uint8_t *, const MgBufs<double> &, const RedWs &,
                                    cudaStream_t, int);
template int elas_mg_stage_batch<float>(int, int, const ElasStageIn<float> *, cudaStream_t);
template int damage_mg_stage_batch<float>(int, int, const DamageStageIn<float> *, cudaStream_t);
template void elas_mg_stage<float>(int, const GridD &, const MatD &, const float *,
                                   const uint8_t *, const MgBufs<float> &, const RedWs &,
                                   cudaStream_t, int);
template void damage_mg_stage<double>(int, const GridD &, const double *, double,
                                      const MgBufs<double> &, const RedWs &, cudaStream_t);
template void damage_mg_stage<float>(int, const GridD &, const float *, double,
                                     const MgBufs<float> &, const RedWs &, cudaStream_t);
template void damage_apply<double>(const GridD &, const double *, double, const double *,
                                   double *, cudaStream_t, KrylovScal *, const RedWs *, int);
template void damage_apply<float>(const GridD &, const float *, double, const float *, float *,
                                  cudaStream_t, KrylovScal *, const RedWs *, int);
template void damage_diag<double>(const GridD &, const double *, double, double *, cudaStream_t);
template void damage_diag<float>(const GridD &, const float *, double, float *, cudaStream_t);

}  // namespace pf
