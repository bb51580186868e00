// Operator-level C ABI of libpf: single operations on caller-owned device arrays.
#include <math.h>

#include <mutex>

#include "pf_internal.cuh"
#include "pf_spectral.cuh"
#include "pf_vec.cuh"

using namespace pf;

namespace {

bool grid_ok(const pf_grid *g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->hx > 0 && g->hy > 0 &&
         (double)(g->nx + 1) * (double)(g->ny + 1) <= 4.0e8;
}
GridD to_dev(const pf_grid *g) { return GridD{g->nx, g->ny, g->hx, g->hy, g->elem_active, g->dof_mask}; }
MatD to_dev(const pf_material *m) {
  return MatD{m->mu, m->K, m->cdim, m->eta, m->Gc, m->l, m->split};
}
bool mat_ok(const pf_material *m) {
  return m && m->mu > 0 && m->K > 0 && m->cdim > 0 && m->eta >= 0 && m->Gc > 0 && m->l > 0 &&
         (m->split == PF_SPLIT_VD || m->split == PF_SPLIT_SPECTRAL);
}
size_t n_nodes(const pf_grid *g) { return (size_t)(g->nx + 1) * (g->ny + 1); }
size_t n_points(const pf_grid *g) { return 4 * (size_t)g->nx * g->ny; }
pf_status launched() { return cudaGetLastError() == cudaSuccess ? PF_OK : PF_ECUDA; }

// Scratch for a one-off reduction: partials for `blocks` CTAs, the counter and one
// result slot.  Freed by the destructor after the stream has been synchronised.
struct Scratch {
  RedWs ws{};
  double *res = nullptr;
  void *base = nullptr;
  pf_status alloc(int blocks) {
    ws.max_blocks = blocks;
    const size_t pbytes = (size_t)4 * blocks * sizeof(double);
    const size_t cbytes = red_counters(blocks) * sizeof(unsigned);
    if (cudaMalloc(&base, pbytes + cbytes + 64) != cudaSuccess) return PF_ENOMEM;
    ws.partials = (double *)base;
    ws.counter = (unsigned *)((char *)base + pbytes);
    res = (double *)((char *)base + pbytes + ((cbytes + 15) / 16) * 16);
    return cudaMemset(ws.counter, 0, cbytes) == cudaSuccess ? PF_OK : PF_ECUDA;
  }
  ~Scratch() {
    if (base) cudaFree(base);
  }
};

}  // namespace

extern "C" {

pf_status pf_op_dof_mask(int nx, int ny, const uint8_t *node_flags, const uint8_t *elem_active,
                         uint8_t *mask, void *stream) {
  if (nx < 1 || ny < 1 || !node_flags || !mask) return PF_EINVAL;
  dof_mask(nx, ny, node_flags, elem_active, mask, (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_elas_residual(const pf_grid *g, const pf_material *m, const double *u,
                              const double *d, double *F, uint8_t *tension, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !d || !F) return PF_EINVAL;
  if (m->split == PF_SPLIT_SPECTRAL) {
    double *Sq = nullptr;
    if (cudaMalloc((void **)&Sq, 3 * n_points(g) * sizeof(double)) != cudaSuccess)
      return PF_ENOMEM;
    cudaStream_t cs = (cudaStream_t)stream;
    sp_points(to_dev(g), to_dev(m), u, d, Sq, nullptr, cs);
    sp_force(to_dev(g), Sq, F, cs);
    const bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
    cudaFree(Sq);
    return ok ? PF_OK : PF_ECUDA;
  }
  elas_residual(to_dev(g), to_dev(m), u, d, F, tension, (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_elas_tangent_qp(const pf_grid *g, const pf_material *m, const double *u,
                                const double *d, double *Dq, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !d || !Dq) return PF_EINVAL;
  sp_points(to_dev(g), to_dev(m), u, d, nullptr, Dq, (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_elas_apply_qp(const pf_grid *g, int dtype, const double *Dq, const void *x,
                              void *y, void *stream) {
  if (!grid_ok(g) || !Dq || !x || !y || (dtype != PF_F64 && dtype != PF_F32)) return PF_EINVAL;
  const size_t ts = dtype == PF_F64 ? sizeof(double) : sizeof(float);
  void *S = nullptr;
  if (cudaMalloc(&S, 36 * n_nodes(g) * ts) != cudaSuccess) return PF_ENOMEM;
  cudaStream_t cs = (cudaStream_t)stream;
  const GridD gd = to_dev(g);
  if (dtype == PF_F64) {
    sp_stencil<double>(gd, Dq, (double *)S, cs);
    sp_apply<double>(gd, (const double *)S, (const double *)x, (double *)y, cs);
  } else {
    sp_stencil<float>(gd, Dq, (float *)S, cs);
    sp_apply<float>(gd, (const float *)S, (const float *)x, (float *)y, cs);
  }
  const bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
  cudaFree(S);
  return ok ? PF_OK : PF_ECUDA;
}

pf_status pf_op_elas_apply(const pf_grid *g, const pf_material *m, int dtype, const void *d,
                           const uint8_t *tension, const void *x, void *y, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !d || !tension || !x || !y) return PF_EINVAL;
  if (dtype == PF_F64)
    elas_apply<double>(to_dev(g), to_dev(m), (const double *)d, tension, (const double *)x,
                       (double *)y, (cudaStream_t)stream);
  else if (dtype == PF_F32)
    elas_apply<float>(to_dev(g), to_dev(m), (const float *)d, tension, (const float *)x,
                      (float *)y, (cudaStream_t)stream);
  else
    return PF_EINVAL;
  return launched();
}

pf_status pf_op_elas_diag(const pf_grid *g, const pf_material *m, int dtype, const void *d,
                          const uint8_t *tension, void *diag, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !d || !tension || !diag) return PF_EINVAL;
  if (dtype == PF_F64)
    elas_diag<double>(to_dev(g), to_dev(m), (const double *)d, tension, (double *)diag,
                      (cudaStream_t)stream);
  else if (dtype == PF_F32)
    elas_diag<float>(to_dev(g), to_dev(m), (const float *)d, tension, (float *)diag,
                     (cudaStream_t)stream);
  else
    return PF_EINVAL;
  return launched();
}

pf_status pf_op_damage_apply(const pf_grid *g, int dtype, const void *c, double kappa,
                             const void *x, void *y, void *stream) {
  if (!grid_ok(g) || !c || !x || !y || !(kappa >= 0)) return PF_EINVAL;
  if (dtype == PF_F64)
    damage_apply<double>(to_dev(g), (const double *)c, kappa, (const double *)x, (double *)y,
                         (cudaStream_t)stream);
  else if (dtype == PF_F32)
    damage_apply<float>(to_dev(g), (const float *)c, kappa, (const float *)x, (float *)y,
                        (cudaStream_t)stream);
  else
    return PF_EINVAL;
  return launched();
}

pf_status pf_op_damage_diag(const pf_grid *g, int dtype, const void *c, double kappa,
                            void *diag, void *stream) {
  if (!grid_ok(g) || !c || !diag || !(kappa >= 0)) return PF_EINVAL;
  if (dtype == PF_F64)
    damage_diag<double>(to_dev(g), (const double *)c, kappa, (double *)diag, (cudaStream_t)stream);
  else if (dtype == PF_F32)
    damage_diag<float>(to_dev(g), (const float *)c, kappa, (float *)diag, (cudaStream_t)stream);
  else
    return PF_EINVAL;
  return launched();
}

pf_status pf_op_damage_rhs(const pf_grid *g, const double *H, double *b, void *stream) {
  if (!grid_ok(g) || !H || !b) return PF_EINVAL;
  damage_rhs(to_dev(g), H, b, (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_qp_energy(const pf_grid *g, const pf_material *m, const double *u,
                          const double *Hprev, double *psi, double *Hout, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !Hprev || !Hout) return PF_EINVAL;
  point_energy(to_dev(g), to_dev(m), u, Hprev, psi, Hout, (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_fs_coeff(const pf_grid *g, const pf_material *m, int scheme, double psi_crit,
                         const double *u, const double *d, const double *Hprev, double *c_aug,
                         uint8_t *active, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !d || !Hprev || !c_aug || !active ||
      scheme < PF_ST || scheme > PF_S3)
    return PF_EINVAL;
  point_fs_coeff(to_dev(g), to_dev(m), scheme, psi_crit, u, d, Hprev, c_aug, active,
                 (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_fs_predict(const pf_grid *g, const pf_material *m, int scheme, const double *u,
                           const double *d, const double *dd, const double *Hprev,
                           const uint8_t *active, double *Hhalf, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !d || !dd || !Hprev || !active || !Hhalf ||
      scheme < PF_ST || scheme > PF_S3)
    return PF_EINVAL;
  point_fs_predict(to_dev(g), to_dev(m), scheme, u, d, dd, Hprev, active, Hhalf,
                   (cudaStream_t)stream);
  return launched();
}

pf_status pf_op_reaction(const pf_grid *g, const uint8_t *node_flags, const double *F, int dir,
                         double *out, void *stream) {
  if (!grid_ok(g) || !node_flags || !F || !out || (dir != 0 && dir != 1)) return PF_EINVAL;
  const size_t nn = (size_t)(g->nx + 1) * (g->ny + 1);
  Scratch s;
  pf_status st = s.alloc(4096);
  if (st != PF_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  reaction(nn, node_flags, dir, F, s.res, s.ws, cs);
  if (cudaGetLastError() != cudaSuccess) return PF_ECUDA;
  if (cudaMemcpyAsync(out, s.res, sizeof(double), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return PF_ECUDA;
  return PF_OK;
}

pf_status pf_op_stag_residual(const pf_grid *g, const pf_material *m, const double *u,
                              const double *d, const double *Hprev, double *out, void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !d || !Hprev || !out) return PF_EINVAL;
  const size_t nn = (size_t)(g->nx + 1) * (g->ny + 1), nq = (size_t)4 * g->nx * g->ny;
  GridD gd = to_dev(g);
  GridD gfull = gd;
  gfull.dofm = nullptr;
  MatD md = to_dev(m);
  Scratch s;
  pf_status st = s.alloc(4096);
  if (st != PF_OK) return st;
  double *buf = nullptr;
  if (cudaMalloc(&buf, (2 * nq + 3 * nn) * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
  double *H = buf, *c = buf + nq, *Kd = buf + 2 * nq, *b = Kd + nn, *diag = b + nn;
  cudaStream_t cs = (cudaStream_t)stream;
  point_energy(gd, md, u, Hprev, nullptr, H, cs);
  coef<double>(nq, m->Gc / m->l, H, c, cs);
  damage_rhs(gd, H, b, cs);
  damage_apply<double>(gfull, c, m->Gc * m->l, d, Kd, cs);
  damage_diag<double>(gfull, c, m->Gc * m->l, diag, cs);
  stag_max(nn, gd.dofm, Kd, b, diag, s.res, s.ws, cs);
  pf_status ret = PF_OK;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(out, s.res, sizeof(double), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    ret = PF_ECUDA;
  cudaFree(buf);
  return ret;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Allocation-free staggered residual.  Its scratch lives in file-scope device arrays
// that every GPU loading the library holds until the process exits.  Host code may not
// use the arrays' names as device addresses: the first call on a device resolves their
// addresses with cudaGetSymbolAddress while that device is current.
// ------------------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_BLOCKS = 1024;  // reduction partial slots (>= 2 CTAs per SM)
constexpr size_t NOALLOC_FIELD_DOUBLES = PF_NOALLOC_MAX_DOUBLES;
constexpr size_t NOALLOC_DOUBLES = 4 * NOALLOC_BLOCKS + 2 + NOALLOC_FIELD_DOUBLES;
constexpr size_t NOALLOC_COUNTERS = 2;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];
static __device__ __align__(256) unsigned g_noalloc_counters[NOALLOC_COUNTERS];

struct NoallocPtrs {
  double *scratch = nullptr;
  unsigned *counters = nullptr;
};
std::mutex g_noalloc_mx;
NoallocPtrs g_noalloc_dev[64];

// Device addresses of the static scratch on the current device (resolved once).
pf_status noalloc_ptrs(NoallocPtrs *out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PF_ECUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mx);
  NoallocPtrs &p = g_noalloc_dev[dev];
  if (!p.scratch) {
    void *a = nullptr, *b = nullptr;
    if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess) return PF_ECUDA;
    if (cudaGetSymbolAddress(&b, g_noalloc_counters) != cudaSuccess) return PF_ECUDA;
    p.scratch = (double *)a;
    p.counters = (unsigned *)b;
  }
  *out = p;
  return PF_OK;
}

}  // namespace

extern "C" pf_status pf_op_stag_residual_noalloc(const pf_grid *g, const pf_material *m,
                                                 const double *u, const double *d,
                                                 const double *Hprev, double *out,
                                                 void *stream) {
  if (!grid_ok(g) || !mat_ok(m) || !u || !d || !Hprev || !out) return PF_EINVAL;
  const size_t nn = (size_t)(g->nx + 1) * (g->ny + 1), nq = (size_t)4 * g->nx * g->ny;
  if (2 * nq + 3 * nn > NOALLOC_FIELD_DOUBLES) return PF_EINVAL;  // beyond the static scratch
  NoallocPtrs P;
  pf_status st = noalloc_ptrs(&P);
  if (st != PF_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  // arrival counters must start at zero; the partial sums need no clearing
  if (cudaMemsetAsync(P.counters, 0, NOALLOC_COUNTERS * sizeof(unsigned), cs) != cudaSuccess)
    return PF_ECUDA;
  RedWs ws{P.scratch, P.counters, NOALLOC_BLOCKS};
  double *res = P.scratch + 4 * NOALLOC_BLOCKS;
  double *H = res + 2, *c = H + nq, *Kd = c + nq, *b = Kd + nn, *diag = b + nn;
  GridD gd = to_dev(g);
  GridD gfull = gd;
  gfull.dofm = nullptr;
  MatD md = to_dev(m);
  point_energy(gd, md, u, Hprev, nullptr, H, cs);
  coef<double>(nq, m->Gc / m->l, H, c, cs);
  damage_rhs(gd, H, b, cs);
  damage_apply<double>(gfull, c, m->Gc * m->l, d, Kd, cs);
  damage_diag<double>(gfull, c, m->Gc * m->l, diag, cs);
  stag_max(nn, gd.dofm, Kd, b, diag, res, ws, cs);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return PF_ECUDA;
  return PF_OK;
}
