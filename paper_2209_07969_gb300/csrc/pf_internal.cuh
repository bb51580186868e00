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
  int split;   // PF_SPLIT_VD or PF_SPLIT_SPECTRAL
};

// Device scalars of one Krylov solve.  The last CTA of each fused reduction updates
// them, so the host never sits between iterations; a device-side loop reads rtol2 and
// maxit (written by the host before the solve) and counts passes in it.
struct KrylovScal {
  double rz;     // r.z
  double pq;     // p.q
  double alpha;  // CG step
  double beta;   // CG direction update
  double rr;     // ||r||^2
  double rr0;    // ||r||^2 after the initialisation
  double rtol2;  // stop when rr <= rtol2 rr0
  int maxit;     // stop after maxit iterations
  int done;      // set when this solve has stopped (batched solves skip its work)
  int it;        // iterations done
  int breakdown;
};

// Reduction workspace: per-CTA partials (up to 4 values each) and the arrival counter,
// kept at zero between launches.
struct RedWs {
  double *partials;   // 4 * max_blocks doubles
  unsigned *counter;  // red_counters() arrival counters
  int max_blocks;
};
inline size_t red_counters(int) { return 2; }

// Bump allocator over one device slab: a context takes all of its arrays from a single
// allocation, so its device footprint is exactly the slab.  With no base it only counts
// (the dry run that sizes the slab and answers pf_footprint_bytes).  Every array starts
// on a 256-byte boundary.
struct Arena {
  char *base = nullptr;
  size_t used = 0, cap = 0;
  template <class T>
  bool take(T **p, size_t n) {
    const size_t b = ((n ? n : 1) * sizeof(T) + 255) & ~(size_t)255;
    if (base) {
      if (used + b > cap) return false;
      *p = reinterpret_cast<T *>(base + used);
    } else {
      *p = nullptr;
    }
    used += b;
    return true;
  }
};

// Programmatic dependent launch.  The kernels of the Krylov iteration are launched with
// programmatic stream serialization (launch_pdl) and open with pdl_enter(): the kernel's
// CTAs are dispatched while its predecessor finishes, wait there until the predecessor
// has completed and its writes are visible, then allow the next kernel to be dispatched
// in turn.  The gap between the short dependent launches of one iteration shrinks to the
// wait.  Without a programmatic launch both instructions return at once.  PF_PDL=0 in the
// environment launches everything plainly.
bool pdl_enabled();
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...) != cudaSuccess &&
      cfg.numAttrs) {
    cudaGetLastError();   // refused as a programmatic launch: launch it plainly
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
  }
}

__device__ __forceinline__ double red_warp(double v, bool is_max) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, w) : v + w;
  }
  return v;
}

// CTA-wide sum (or max) of NV values per thread; thread 0 receives the totals in v.  The
// order is fixed (xor tree in each warp, warps in index order).  sh: NV x 32 shared slots.
template <int NV>
__device__ __forceinline__ void red_cta(double (&v)[NV], double (*sh)[32], bool is_max) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = red_warp(v[k], is_max);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = sh[k][0];
      for (int w = 1; w < nw; ++w) s = is_max ? fmax(s, sh[k][w]) : s + sh[k][w];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Grid-wide sum (or max) of NV values, deterministic and without a second launch.  Every
// CTA publishes its partials and arrives on one counter; the last CTA to arrive reads all
// partials with RED_UNROLL independent loads in flight per thread and sums them in a fixed
// order.  Returns true in thread 0 of that CTA, with tot[] holding the totals; the counter
// is reset for the next launch.  Every CTA of the grid must call it.
constexpr int RED_UNROLL = 8;
// bid / nblk: the CTA's index among the nblk CTAs that take part (a batched launch runs
// several such groups, one per simulation, each with its own workspace).
template <int NV>
__device__ bool red_grid(double (&v)[NV], const RedWs ws, double (&tot)[NV], bool is_max,
                         unsigned bid, unsigned nblk) {
  __shared__ double sh[NV][32];
  __shared__ int go;
  const double none = is_max ? -INFINITY : 0.0;
  const size_t mb = (size_t)ws.max_blocks;
  red_cta<NV>(v, sh, is_max);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) ws.partials[k * mb + bid] = v[k];
    __threadfence();
    go = atomicAdd(ws.counter, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!go) return false;
  __threadfence();
  double w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a[RED_UNROLL];
#pragma unroll
    for (int u = 0; u < RED_UNROLL; ++u) a[u] = none;
    for (unsigned base = threadIdx.x; base < nblk; base += RED_UNROLL * blockDim.x) {
#pragma unroll
      for (int u = 0; u < RED_UNROLL; ++u) {
        const unsigned i = base + u * blockDim.x;
        if (i < nblk) {
          const double p = __ldcg(ws.partials + k * mb + i);
          a[u] = is_max ? fmax(a[u], p) : a[u] + p;
        }
      }
    }
    w[k] = a[0];
#pragma unroll
    for (int u = 1; u < RED_UNROLL; ++u) w[k] = is_max ? fmax(w[k], a[u]) : w[k] + a[u];
  }
  red_cta<NV>(w, sh, is_max);
  if (threadIdx.x != 0) return false;
  ws.counter[0] = 0u;
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = w[k];
  return true;
}
template <int NV>
__device__ bool red_grid(double (&v)[NV], const RedWs ws, double (&tot)[NV], bool is_max) {
  return red_grid<NV>(v, ws, tot, is_max, blockIdx.y * gridDim.x + blockIdx.x,
                      gridDim.x * gridDim.y);
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
                int epi = 0, int sr = 0);
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
// AT1 mode of the fixed-stress kernels (on = 0: AT2 with history).
struct At1D {
  int on = 0;
  const double *dprev = nullptr;  // d_{n-1} (nodal) for the penalty indicator
  double gamma = 0.0;             // penalty parameter
  double floor = 0.0;             // lower limit of the augmented coefficient, 2 G_c/(c_w l)
};
void fs_coeff(const GridD &g, const MatD &m, int scheme, double psi_crit, const double *u,
              const double *d, const double *Hprev, double *c_aug, uint8_t *active,
              cudaStream_t st, const At1D &at1 = At1D());
void fs_predict(const GridD &g, const MatD &m, int scheme, const double *u, const double *d,
                const double *dd, const double *Hprev, const uint8_t *active, double *Hhalf,
                cudaStream_t st, int at1 = 0);
// AT1 per-point arrays c0 = 2 psi, cJ, bhalf (pf_ops.cu, k_at1_coef).
void at1_coef(const GridD &g, const double *psi, const double *d, const double *dprev, double a,
              double gamma, double *c0, double *cJ, double *bhalf, cudaStream_t st);
void dof_mask(int nx, int ny, const uint8_t *flags, const uint8_t *active, uint8_t *mask,
              cudaStream_t st);

// Epilogues of the fused operator + reduction kernels.
enum { EPI_NONE = 0, EPI_CG_ALPHA = 1 };

// Buffers of the multigrid-preconditioned CG whose fine-level work runs fused into the
// operator kernel (elas_mg_stage, damage_mg_stage).  Vectors have B (nx+1)(ny+1) entries
// (B = 2: interleaved (u_x, u_y) per node; B = 1: phase field).
template <class T>
struct MgBufs {
  const T *b;              // right-hand side
  T *x;                    // iterate
  T *r[2], *p[2];          // [0]: previous iterate's residual / direction, [1]: current
  T *q, *za, *zb, *lr, *dv;  // A p; pre-smoothed z; preconditioned residual; level-0 scratch
  const T *invd, *coef;    // level-0 inverse diagonal and Chebyshev coefficients
  const uint8_t *fm;       // level-0 free-component mask
  const T *xc;             // level-1 correction
  int nxc, nyc;            // level-1 elements per direction
  KrylovScal *sc;
};
enum { FS_DIR, FS_UPD, FS_UPD_INIT, FS_RESID, FS_PROLONG, FS_FINISH, FS_FINISH_FIRST };
// One fused stage (pf_fused.cuh) on the elasticity tangent (strip kernel) or on K_dd(c)
// (tile kernel).
template <class T>
void elas_mg_stage(int stage, const GridD &g, const MatD &m, const T *d, const uint8_t *tens,
                   const MgBufs<T> &b, const RedWs &ws, cudaStream_t st, int sr = 0);
// sr: node rows per warp of the strip kernel (2, 4, 8), 0 for the grid-size rule.
template <class T>
void damage_mg_stage(int stage, const GridD &g, const T *c, double kappa, const MgBufs<T> &b,
                     const RedWs &ws, cudaStream_t st);

}  // namespace pf
