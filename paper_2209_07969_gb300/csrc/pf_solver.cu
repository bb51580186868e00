// Simulation context and the staggered drivers of libpf (C ABI in include/pf.h).
//
// Per load step (Sec. 3.1, Fig. 1, d-u order; fixed-stress d-step of Sec. 3.3-3.5):
//   lift Dirichlet values -> u-solve with d_{n-1} -> repeat {d-step; u-solve; residual}
//   -> commit H_n = max(H_{n-1}, Psi+(u_n)) and the reaction force.
// u-solve: semismooth Newton with the frozen tension indicator of every iterate; each
// Newton system is solved by Jacobi-preconditioned CG, in FP64 or as FP32 CG inside an
// FP64 iterative-refinement loop.  Every step runs on the context's stream; the host
// reads one scalar per Newton iterate, per staggered pass and every `check_every`
// Krylov iterations.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

#include "pf_batch.cuh"
#include "pf_gmg.cuh"
#include "pf_spectral.cuh"
#include "pf_internal.cuh"
#include "pf_vec.cuh"

using namespace pf;

// Multigrid hierarchies are rebuilt lazily: a hierarchy built for an earlier operator is
// still an SPD preconditioner for the current one, so it is kept until the Krylov
// iteration count of a solve grows past 1.5x (+4) the count right after the last rebuild.
struct MgState {
  int base = -1;       // iterations of the first solve after the last rebuild
  int last = 0;        // iterations of the latest solve
  int since = 0;       // solves since the last rebuild
  bool stale = true;
  bool need() const { return stale || base < 0 || last > (3 * base) / 2 + 4 || since >= 64; }
  void built() { stale = false; base = -1; since = 0; }
  void record(int it) {
    last = it;
    if (base < 0) base = it;
    ++since;
  }
};

// One Krylov solve as a single CUDA graph: the initialisation, then a conditional WHILE
// node whose body is one iteration and the condition kernel.
struct WhileGraph {
  cudaGraphExec_t exec = nullptr;
  int init_launches = 0, body_launches = 0;
  bool unsupported = false;   // building failed once: use the batched host loop
};

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  size_t n = 0;
  int every = 0;
};

struct pf_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  GridD g{};
  MatD m{};
  size_t nn = 0, ne = 0, nq = 0;
  int precision = PF_FP64, reaction_dir = 1, precond = PF_PRECOND_JACOBI, plane = 0;
  int model = PF_AT2_HISTORY;
  // AT1 (Sec. 2): a = G_c/(c_w l), kappa = 2 G_c l / c_w, gamma = 27 G_c/(64 l tol_ir^2),
  // floor = 2 G_c/(c_w l) (lower limit of the augmented coefficient)
  double at1_a = 0.0, at1_kappa = 0.0, at1_gamma = 0.0, at1_floor = 0.0;
  double *bhalf = nullptr;   // AT1 right-hand-side integrand / 2 (per Gauss point)
  pf_options opt{};
  double ubar = 0.0;
  int64_t step = 0;
  int64_t launches = 0;
  char err[512] = {0};

  // committed state and per-step work arrays (FP64)
  double *u = nullptr, *d = nullptr, *H = nullptr;   // 2N, N, Q
  double *d_prev = nullptr;                            // N
  double *F = nullptr;                                 // 2N
  double *Hk = nullptr, *cq = nullptr, *Hhalf = nullptr;  // Q
  uint8_t *act = nullptr;                              // Q
  double *bd = nullptr, *Kd = nullptr, *dd = nullptr;  // N
  uint8_t *flags = nullptr, *active = nullptr, *dofm = nullptr, *tens = nullptr;
  // Krylov workspace (FP64): 2N each (used for u and d)
  double *kb = nullptr, *kx = nullptr, *kr = nullptr, *kz = nullptr, *kp = nullptr,
         *kq = nullptr, *kinv = nullptr, *kres = nullptr;
  // FP32 copies for the inner solves
  float *fb = nullptr, *fx = nullptr, *fr = nullptr, *fz = nullptr, *fp = nullptr,
        *fq = nullptr, *finv = nullptr, *fd = nullptr, *fc = nullptr;
  double *csolve = nullptr;  // Q: coefficient of the current d-solve
  // spectral split: per-point stress (3Q) and tangent (6Q) at the last residual evaluation,
  // nodal stencils of the tangent (36 N, FP64 and, for PF_FP32_IR, FP32)
  double *sp_Sq = nullptr, *sp_Dq = nullptr, *sp_S64 = nullptr;
  float *sp_S32 = nullptr;
  KrylovScal *sc = nullptr;
  RedWs ws{};
  Gmg<double> gu, gd;        // multigrid hierarchies (FP64 mode)
  Gmg<float> gu32, gd32;     // multigrid hierarchies (FP32 inner solves)
  GraphSlot graphs[6];        // batched fallback, [slot * 2 + multigrid], [SL_FUSED(_D)]
  WhileGraph wgraphs[6];      // device-side loops, same indexing
  bool use_graphs = true;
  MgState mg_u, mg_d;
  double prof[PF_PROF_PHASES] = {0};   // host milliseconds per phase (pf_profile)
  double *dscal = nullptr;   // device scalars for norms / residual / reaction
  double *hbuf = nullptr;    // pinned host mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  char *slab = nullptr;         // the one device allocation all arrays are carved from
  pf_tuning tune{};             // launch shapes chosen by pf_autotune (0: built-in rules)
  pf_batch *batch = nullptr;   // batch this context is attached to (pf_batch_attach)
  bool batching = false;       // inside a load step whose FP32 multigrid solves are batched
  cudaEvent_t evb = nullptr;   // marks the context's work before a batched solve
};

// ---- batched solves ----------------------------------------------------------------------
// A batch (pf_batch_*) joins the FP32 multigrid Krylov solves of the contexts attached to
// it: every context runs its load step on its own host thread, and when all of them wait
// for such a solve the last to arrive launches them together: one captured CUDA graph per
// set of participants, whose kernels run each fused stage, multigrid level and coarse
// cycle of all participants in one launch (pf_batch.cuh), with a device-side loop that
// stops each participant's iteration on its own test.  Each participant's arithmetic is
// that of its own solve, so results are bit-identical alone and in any batch.
struct BatchReq {
  pf_ctx *ctx = nullptr;
  int kind = 0;                 // 0: elasticity (B = 2), 1: phase field (B = 1)
  Gmg<float> *G = nullptr;
  ElasStageIn<float> e{};
  DamageStageIn<float> dm{};
  double rtol = 0.0;
  int maxit = 0;
  int iters = 0;
  bool ok = false;
  pf_status status = PF_OK;
  bool finished = false;
};

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  int init_launches = 0, body_launches = 0;
};

struct pf_batch {
  int device = 0;
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;               // attached contexts inside a batched load step
  bool leading = false;         // a thread is running a batch
  std::vector<BatchReq *> pending;
  std::map<std::vector<uintptr_t>, BatchGraph> graphs;   // by kind and participants
  std::vector<pf_ctx *> members;
  int64_t launches = 0;         // kernel launches of batched solves
  int64_t solves = 0, groups = 0;
  int max_group = 0;
};

namespace {

// Host time of a phase; every phase ends in a stream synchronisation (a scalar read or a
// setup's host step), so host time equals device time of the phase plus launch gaps.
struct PhaseTimer {
  double *slot;
  std::chrono::steady_clock::time_point t0;
  explicit PhaseTimer(double *s) : slot(s), t0(std::chrono::steady_clock::now()) {}
  ~PhaseTimer() {
    *slot += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

pf_status set_err(pf_ctx *c, pf_status s, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return set_err(ctx, PF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKS(call)                                   \
  do {                                              \
    pf_status s_ = (call);                          \
    if (s_ != PF_OK && s_ != PF_ENOTCONV) return s_; \
  } while (0)

pf_status check_launch(pf_ctx *ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return PF_OK;
}

// Read n doubles of device scalars into the pinned mirror (synchronises the stream).
pf_status read_scalars(pf_ctx *ctx, const void *dev, int nbytes) {
  CK(cudaMemcpyAsync(ctx->hbuf, dev, nbytes, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return PF_OK;
}

GridD grid_nomask(const pf_ctx *ctx) {
  GridD g = ctx->g;
  g.dofm = nullptr;
  return g;
}

// ---- Krylov ----------------------------------------------------------------------------
// Graph slots: one captured CUDA graph per solver instance (operator x preconditioner x
// precision).  Every pointer an iteration touches is a fixed context buffer, so a graph
// captured once stays valid; operator data (d, tension bits, coefficients, multigrid
// stencils) are rewritten in place between solves.
enum { SL_U = 0, SL_D = 1, SL_COUNT = 2, SL_FUSED = 4, SL_FUSED_D = 5 };

// Runs batch() (`every` Krylov iterations) until ||r||^2 <= rtol^2 rr0, a breakdown, or
// maxit.  Each batch ends with the read-back of ||r||^2 and the breakdown flag; with graphs
// enabled the batch is captured once per slot and replayed, so the host launches once and
// synchronises once per check.
template <class Batch>
pf_status krylov_batches(pf_ctx *ctx, int sidx, int every, Batch batch, double rr0, double rtol,
                         int maxit, int *iters, bool *ok) {
  cudaStream_t st = ctx->st;
  auto run = [&]() -> int {
    const int nl = batch();
    cudaMemcpyAsync(ctx->hbuf, &ctx->sc->rr, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(ctx->hbuf + 1, &ctx->sc->breakdown, sizeof(int), cudaMemcpyDeviceToHost, st);
    return nl;
  };
  GraphSlot &S = ctx->graphs[sidx];
  if (ctx->use_graphs && (!S.exec || S.every != every)) {
    if (S.exec) cudaGraphExecDestroy(S.exec);
    S.exec = nullptr;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    S.launches = run();
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&S.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      S.exec = nullptr;
      return set_err(ctx, PF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    S.every = every;
  }
  const double target = rtol * rtol * rr0;
  int it = 0;
  *ok = false;
  while (it < maxit) {
    if (S.exec) {
      CK(cudaGraphLaunch(S.exec, st));
    } else {
      S.launches = run();
    }
    ctx->launches += S.launches;
    it += every;
    CKS(check_launch(ctx));
    CK(cudaStreamSynchronize(st));
    const double rr = ctx->hbuf[0];
    int bd;
    memcpy(&bd, ctx->hbuf + 1, sizeof(int));
    if (rr <= target) {
      *ok = true;
      break;
    }
    if (bd || !isfinite(rr)) break;
  }
  *iters = it;
  return PF_OK;
}

// Pinned host mirror of the Krylov scalars (inside the context's pinned buffer).
inline KrylovScal *host_scal(pf_ctx *ctx) { return (KrylovScal *)((char *)ctx->hbuf + 128); }

template <class Init, class Body>
cudaError_t build_while(pf_ctx *ctx, WhileGraph &W, Init init, Body body) {
  cudaStream_t st = ctx->st;
  cudaGraph_t gi = nullptr, g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  W.init_launches = init();
  if ((e = cudaStreamEndCapture(st, &gi)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  cudaGraphNode_t ni, nc;
  cudaGraphNodeParams cp = {};
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) goto done;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    goto done;
  if ((e = cudaGraphAddChildGraphNode(&ni, g, nullptr, 0, gi)) != cudaSuccess) goto done;
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&nc, g, &ni, nullptr, 1, &cp)) != cudaSuccess) goto done;
  {
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st, bg, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) goto done;
    W.body_launches = body() + 1;
    krylov_while(h, ctx->sc, st);
    if ((e = cudaStreamEndCapture(st, &bg)) != cudaSuccess) goto done;
  }
  e = cudaGraphInstantiate(&W.exec, g, 0);
  if (e != cudaSuccess) W.exec = nullptr;
done:
  if (gi) cudaGraphDestroy(gi);
  if (g) cudaGraphDestroy(g);
  return e;
}

// One Krylov solve: init() (returns its launches) sets x = 0 and the device scalars
// (rr0, it = 0), body() runs one iteration (returns its launches).  Preferred form: one
// graph launch per solve in which the iterations loop on the device (build_while) and
// the host synchronises once, with no rounding of the iteration count.  Fallback: init
// launched directly, then batches of `every` iterations with a host check after each.
template <class Init, class Body>
pf_status krylov_run(pf_ctx *ctx, int sidx, Init init, Body body, int every, double rtol,
                     int maxit, int *iters, bool *ok) {
  cudaStream_t st = ctx->st;
  WhileGraph &W = ctx->wgraphs[sidx];
  if (ctx->opt.device_loop && !W.exec && !W.unsupported) {
    if (build_while(ctx, W, init, body) != cudaSuccess || !W.exec) {
      W.unsupported = true;
      cudaGetLastError();
    }
  }
  *iters = 0;
  if (ctx->opt.device_loop && W.exec) {
    KrylovScal *hk = host_scal(ctx);
    hk->rtol2 = rtol * rtol;
    hk->maxit = maxit;
    hk->done = 0;
    CK(cudaMemcpyAsync(&ctx->sc->rtol2, &hk->rtol2, sizeof(double) + 2 * sizeof(int),
                       cudaMemcpyHostToDevice, st));
    CK(cudaGraphLaunch(W.exec, st));
    CK(cudaMemcpyAsync(hk, ctx->sc, sizeof(KrylovScal), cudaMemcpyDeviceToHost, st));
    CKS(check_launch(ctx));
    CK(cudaStreamSynchronize(st));
    ctx->launches += W.init_launches + (long long)hk->it * W.body_launches;
    if (!(hk->rr0 > 0.0)) {
      *ok = true;
      return PF_OK;
    }
    *iters = hk->it;
    *ok = hk->rr <= hk->rtol2 * hk->rr0;
    return PF_OK;
  }
  ctx->launches += init();
  CKS(check_launch(ctx));
  CKS(read_scalars(ctx, &ctx->sc->rr, sizeof(double)));
  const double rr0 = ctx->hbuf[0];
  *ok = true;
  if (!(rr0 > 0.0)) return PF_OK;
  auto batch = [&]() -> int {
    int nl = 0;
    for (int k = 0; k < every; ++k) nl += body();
    return nl;
  };
  return krylov_batches(ctx, sidx, every, batch, rr0, rtol, maxit, iters, ok);
}

// Preconditioned CG on a masked SPD operator.  apply(p, q, epi): q = A p with the fused
// dot epilogue; fine(x, y): y = A x without epilogue (multigrid smoothing).  G == nullptr
// selects Jacobi with inverse diagonal `inv`.
template <class T, class Apply, class Fine>
pf_status pcg(pf_ctx *ctx, int slot, Apply apply, Fine fine, Gmg<T> *G, size_t n, T *b, T *x,
              T *r, T *z, T *p, T *q, const T *inv, double rtol, int maxit, int *iters,
              bool *ok) {
  cudaStream_t st = ctx->st;
  auto init = [&]() -> int {
    if (!G) {
      cg_init<T>(n, b, x, r, z, p, inv, ctx->sc, ctx->ws, st);
      return 1;
    }
    pcg_init<T>(n, b, x, r, ctx->sc, ctx->ws, st);
    const int nl = gmg_vcycle<T>(*G, fine, r, z, st);
    pcg_rz<T>(n, r, z, p, 1, ctx->sc, ctx->ws, st);
    return nl + 2;
  };
  auto body = [&]() -> int {
    int nl = 1;
    apply(p, q, EPI_CG_ALPHA);
    if (G) {
      pcg_update<T>(n, x, r, p, q, ctx->sc, ctx->ws, st);
      nl += 1 + gmg_vcycle<T>(*G, fine, r, z, st);
      pcg_rz<T>(n, r, z, p, 0, ctx->sc, ctx->ws, st);
      cg_dir<T>(n, z, p, ctx->sc, st);
      nl += 2;
    } else {
      cg_update<T>(n, x, r, z, p, q, inv, ctx->sc, ctx->ws, st);
      cg_dir<T>(n, z, p, ctx->sc, st);
      nl += 2;
    }
    return nl;
  };
  const int every = ctx->opt.check_every > 0 ? ctx->opt.check_every : 8;
  return krylov_run(ctx, slot * 2 + (G ? 1 : 0), init, body, every, rtol, maxit, iters, ok);
}

// Multigrid PCG with the fine-level work fused into the operator kernel (pf_fused.cuh):
// the iteration of pcg() with the V-cycle preconditioner in five fine-level launches per
// iteration instead of sixteen.  stage(s, bufs) launches fused stage s on the fine
// operator.  Needs a hierarchy with at least one grid level above the single-CTA coarse
// cycle (G.lc >= 1).  Level-0 vectors of the hierarchy serve as the second residual and
// direction buffers and as smoother scratch.
template <class T>
MgBufs<T> mg_bufs(pf_ctx *ctx, Gmg<T> &G, const T *b, T *x, T *r, T *z, T *p, T *q) {
  GmgLevel<T> &L0 = G.lv[0];
  MgBufs<T> B;
  B.b = b;
  B.x = x;
  B.r[0] = r;
  B.r[1] = L0.b;
  B.p[0] = p;
  B.p[1] = L0.y;
  B.q = q;
  B.za = L0.x;
  B.zb = z;
  B.lr = L0.r;
  B.dv = L0.dv;
  B.invd = L0.invd;
  B.coef = L0.coef;
  B.fm = L0.fm;
  B.xc = G.lv[1].x;
  B.nxc = G.lv[1].nx;
  B.nyc = G.lv[1].ny;
  B.sc = ctx->sc;
  return B;
}

template <class T, class Stage>
pf_status pcg_mg_fused(pf_ctx *ctx, int sidx, Gmg<T> &G, Stage stage_fn, const T *b, T *x,
                       T *r, T *z, T *p, T *q, double rtol, int maxit, int *iters, bool *ok) {
  cudaStream_t st = ctx->st;
  GmgLevel<T> &L0 = G.lv[0];
  const MgBufs<T> B = mg_bufs<T>(ctx, G, b, x, r, z, p, q);
  auto stage = [&](int s) { stage_fn(s, B); };
  // residual, restriction, coarse levels and post-smoothing of the V-cycle on r[1]
  auto vcycle_rest = [&](bool first) -> int {
    stage(FS_RESID);
    gmg_restrict<T>(G, 0, L0.r, G.lv[1].b, st);
    const int nl = 2 + gmg_mid<T>(G, 1, st);
    stage(FS_PROLONG);
    stage(first ? FS_FINISH_FIRST : FS_FINISH);
    return nl + 2;
  };
  // x = 0, r = b, z = V(r), rz, beta = 0, p_prev = 0
  auto init = [&]() -> int {
    stage(FS_UPD_INIT);
    return 1 + vcycle_rest(true);
  };
  auto body = [&]() -> int {
    stage(FS_DIR);
    stage(FS_UPD);
    return 2 + vcycle_rest(false);
  };
  const int every = ctx->opt.check_every > 0 ? ctx->opt.check_every : 8;
  return krylov_run(ctx, sidx, init, body, every, rtol, maxit, iters, ok);
}

// Capture the batched solve of group g (one kind, at most PF_MAXB participants): the
// initialisation, then a conditional WHILE node whose body is one iteration of every
// participant and the batched loop condition.  Kernel order per participant is that of
// pcg_mg_fused.
cudaError_t build_batch_graph(pf_batch *b, const std::vector<BatchReq *> &g, BatchGraph &W) {
  const int n = (int)g.size();
  const int kind = g[0]->kind;
  cudaStream_t st = b->st;
  ElasStageIn<float> ein[PF_MAXB];
  DamageStageIn<float> din[PF_MAXB];
  Gmg<float> *G[PF_MAXB];
  const int *done[PF_MAXB];
  KrylovScal *sc[PF_MAXB];
  for (int i = 0; i < n; ++i) {
    ein[i] = g[i]->e;
    din[i] = g[i]->dm;
    G[i] = g[i]->G;
    sc[i] = g[i]->ctx->sc;
    done[i] = &sc[i]->done;
  }
  auto stage = [&](int s) {
    return kind == 0 ? elas_mg_stage_batch<float>(s, n, ein, st)
                     : damage_mg_stage_batch<float>(s, n, din, st);
  };
  auto vrest = [&](bool first) {
    int nl = stage(FS_RESID);
    nl += gmg_restrict0_batch<float>(n, G, done, st);
    nl += gmg_mid_batch<float>(n, G, done, st);
    nl += stage(FS_PROLONG);
    nl += stage(first ? FS_FINISH_FIRST : FS_FINISH);
    return nl;
  };
  cudaGraph_t gi = nullptr, gr = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  W.init_launches = stage(FS_UPD_INIT) + vrest(true);
  if ((e = cudaStreamEndCapture(st, &gi)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  cudaGraphNode_t ni, nc;
  cudaGraphNodeParams cp = {};
  if ((e = cudaGraphCreate(&gr, 0)) != cudaSuccess) goto done;
  if ((e = cudaGraphConditionalHandleCreate(&h, gr, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    goto done;
  if ((e = cudaGraphAddChildGraphNode(&ni, gr, nullptr, 0, gi)) != cudaSuccess) goto done;
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&nc, gr, &ni, nullptr, 1, &cp)) != cudaSuccess) goto done;
  {
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st, bg, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) goto done;
    W.body_launches = stage(FS_DIR) + stage(FS_UPD) + vrest(false) + 1;
    krylov_while_batch(h, n, sc, st);
    if ((e = cudaStreamEndCapture(st, &bg)) != cudaSuccess) goto done;
  }
  e = cudaGraphInstantiate(&W.exec, gr, 0);
  if (e != cudaSuccess) W.exec = nullptr;
done:
  if (gi) cudaGraphDestroy(gi);
  if (gr) cudaGraphDestroy(gr);
  return e;
}

// Run one group on the batch stream after each participant's earlier work, and hand each
// participant the result its own solve would give (krylov_run's device-loop branch).
void run_group(pf_batch *b, const std::vector<BatchReq *> &g) {
  cudaStream_t st = b->st;
  std::vector<uintptr_t> key;
  key.push_back((uintptr_t)g[0]->kind);
  for (BatchReq *r : g) {
    key.push_back((uintptr_t)r->ctx);
    if (r->kind == 1) {   // the captured kernels carry the gradient coefficient
      uint64_t kb;
      memcpy(&kb, &r->dm.kappa, sizeof(kb));
      key.push_back((uintptr_t)kb);
    }
  }
  BatchGraph &W = b->graphs[key];
  cudaError_t e = cudaSuccess;
  if (!W.exec) e = build_batch_graph(b, g, W);
  if (e != cudaSuccess || !W.exec) {
    cudaGetLastError();
    for (BatchReq *r : g)
      r->status = set_err(r->ctx, PF_ECUDA, "batched solve graph: %s", cudaGetErrorString(e));
    b->graphs.erase(key);
    return;
  }
  for (BatchReq *r : g) {
    KrylovScal *hk = host_scal(r->ctx);
    hk->rtol2 = r->rtol * r->rtol;
    hk->maxit = r->maxit;
    hk->done = 0;
    cudaStreamWaitEvent(st, r->ctx->evb, 0);
    cudaMemcpyAsync(&r->ctx->sc->rtol2, &hk->rtol2, sizeof(double) + 2 * sizeof(int),
                    cudaMemcpyHostToDevice, st);
  }
  cudaGraphLaunch(W.exec, st);
  for (BatchReq *r : g)
    cudaMemcpyAsync(host_scal(r->ctx), r->ctx->sc, sizeof(KrylovScal), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  int most = 0;
  for (BatchReq *r : g) {
    if (e != cudaSuccess) {
      r->status = set_err(r->ctx, PF_ECUDA, "batched solve: %s", cudaGetErrorString(e));
      continue;
    }
    const KrylovScal *hk = host_scal(r->ctx);
    most = hk->it > most ? hk->it : most;
    if (!(hk->rr0 > 0.0)) {
      r->iters = 0;
      r->ok = true;
    } else {
      r->iters = hk->it;
      r->ok = hk->rr <= hk->rtol2 * hk->rr0;
    }
  }
  std::lock_guard<std::mutex> lk(b->mu);
  b->launches += W.init_launches + (int64_t)most * W.body_launches;
  b->solves += (int64_t)g.size();
  b->groups += 1;
  b->max_group = (int)g.size() > b->max_group ? (int)g.size() : b->max_group;
}

void run_batch(pf_batch *b, const std::vector<BatchReq *> &reqs) {
  cudaSetDevice(b->device);
  for (int kind = 0; kind < 2; ++kind) {
    std::vector<BatchReq *> g;
    for (BatchReq *r : reqs) {
      if (r->kind != kind) continue;
      g.push_back(r);
      if ((int)g.size() == PF_MAXB) {
        run_group(b, g);
        g.clear();
      }
    }
    if (!g.empty()) run_group(b, g);
  }
}

// Submit one solve and wait for it.  When every context of the batch that is inside a
// load step waits for a solve, the thread that sees it runs them all.
pf_status batch_solve(pf_ctx *ctx, BatchReq &req, int *iters, bool *ok) {
  pf_batch *b = ctx->batch;
  CK(cudaEventRecord(ctx->evb, ctx->st));
  std::unique_lock<std::mutex> lk(b->mu);
  b->pending.push_back(&req);
  while (!req.finished) {
    if (!b->leading && (int)b->pending.size() >= b->active) {
      b->leading = true;
      std::vector<BatchReq *> reqs;
      reqs.swap(b->pending);
      lk.unlock();
      run_batch(b, reqs);
      lk.lock();
      for (BatchReq *r : reqs) r->finished = true;
      b->leading = false;
      b->cv.notify_all();
      continue;
    }
    b->cv.wait(lk);
  }
  lk.unlock();
  *iters = req.iters;
  *ok = req.ok;
  return req.status;
}

bool batch_eligible(const pf_ctx *c) {
  return c->precision == PF_FP32_IR && c->precond == PF_PRECOND_GMG &&
         c->m.split == PF_SPLIT_VD && c->opt.device_loop && c->gu32.lc >= 1 && c->gd32.lc >= 1;
}

// A load step of an attached context whose FP32 multigrid solves go through its batch.
struct BatchScope {
  pf_ctx *ctx;
  bool on = false;
  explicit BatchScope(pf_ctx *c) : ctx(c) {
    if (!c->batch || !batch_eligible(c)) return;
    std::lock_guard<std::mutex> lk(c->batch->mu);
    c->batch->active++;
    c->batching = on = true;
  }
  ~BatchScope() {
    if (!on) return;
    {
      std::lock_guard<std::mutex> lk(ctx->batch->mu);
      ctx->batch->active--;
      ctx->batching = false;
    }
    ctx->batch->cv.notify_all();
  }
};

template <class T>
pf_status pcg_mg_elas(pf_ctx *ctx, Gmg<T> &G, const T *d, const T *b, T *x, T *r, T *z, T *p,
                      T *q, double rtol, int maxit, int *iters, bool *ok) {
  if constexpr (std::is_same<T, float>::value) {
    if (ctx->batching) {
      BatchReq req;
      req.ctx = ctx;
      req.kind = 0;
      req.G = &G;
      req.e = ElasStageIn<float>{ctx->g, ctx->m, d, ctx->tens,
                                 mg_bufs<float>(ctx, G, b, x, r, z, p, q), ctx->ws,
                                 ctx->tune.strip_rows};
      req.rtol = rtol;
      req.maxit = maxit;
      return batch_solve(ctx, req, iters, ok);
    }
  }
  auto stage = [ctx, d](int s, const MgBufs<T> &B) {
    elas_mg_stage<T>(s, ctx->g, ctx->m, d, ctx->tens, B, ctx->ws, ctx->st,
                     sizeof(T) == 4 ? ctx->tune.strip_rows : 0);
  };
  return pcg_mg_fused<T>(ctx, SL_FUSED, G, stage, b, x, r, z, p, q, rtol, maxit, iters, ok);
}

template <class T>
pf_status pcg_mg_damage(pf_ctx *ctx, Gmg<T> &G, const T *c, double kappa, const T *b, T *x,
                        T *r, T *z, T *p, T *q, double rtol, int maxit, int *iters, bool *ok) {
  if constexpr (std::is_same<T, float>::value) {
    if (ctx->batching) {
      BatchReq req;
      req.ctx = ctx;
      req.kind = 1;
      req.G = &G;
      req.dm = DamageStageIn<float>{ctx->g, c, kappa, mg_bufs<float>(ctx, G, b, x, r, z, p, q),
                                    ctx->ws};
      req.rtol = rtol;
      req.maxit = maxit;
      return batch_solve(ctx, req, iters, ok);
    }
  }
  auto stage = [ctx, c, kappa](int s, const MgBufs<T> &B) {
    damage_mg_stage<T>(s, ctx->g, c, kappa, B, ctx->ws, ctx->st);
  };
  return pcg_mg_fused<T>(ctx, SL_FUSED_D, G, stage, b, x, r, z, p, q, rtol, maxit, iters, ok);
}

// FP32 inner solves inside FP64 iterative refinement:  x = 0; repeat {s = 2^-floor(log2
// ||r||); solve A_32 e = (s r)_32 to tol_inner; x += e / s; r = b - A_64 x; stop when
// ||r|| <= tol ||b||}.
// inner(iters, ok) solves with rhs ctx->fb into ctx->fx.
template <class ApplyD, class Inner>
pf_status refine(pf_ctx *ctx, ApplyD applyd, Inner inner, size_t n, int ncomp, const double *b,
                 double *x, double tol, int *iters, int *refines, bool *ok) {
  cudaStream_t st = ctx->st;
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), st));
  CK(cudaMemcpyAsync(ctx->kres, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  norms(n, ncomp, ctx->g.dofm, b, ctx->dscal, ctx->ws, st);
  ctx->launches++;
  CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
  const double bn = sqrt(ctx->hbuf[0]);
  *ok = true;
  if (!(bn > 0.0)) return PF_OK;
  *ok = false;
  double rn = bn;
  for (int k = 0; k < ctx->opt.max_refine; ++k) {
    // The FP32 solve sees the residual scaled to unit size: late corrections are many
    // orders of magnitude below the first one, and unscaled their FP32 dot products fall
    // into the subnormal range, where CG loses its accuracy and stalls.
    const double s = ldexp(1.0, -ilogb(rn));
    scale_to_f32(n, s, ctx->kres, ctx->fb, st);
    ctx->launches++;
    int it = 0;
    bool iok = false;
    CKS(inner(&it, &iok));
    *iters += it;
    add_scaled_f32(n, 1.0 / s, ctx->fx, x, st);
    ctx->launches++;
    (*refines)++;
    applyd(x, ctx->kq);
    masked_comb(n, ncomp, ctx->g.dofm, 1.0, b, 1.0, ctx->kq, ctx->kres, st);
    norms(n, ncomp, ctx->g.dofm, ctx->kres, ctx->dscal, ctx->ws, st);
    ctx->launches += 3;
    CKS(check_launch(ctx));
    CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
    rn = sqrt(ctx->hbuf[0]);
    if (rn <= tol * bn) {
      *ok = true;
      break;
    }
    if (!isfinite(rn) || it == 0) break;
  }
  return PF_OK;
}

// ---- lagged multigrid -----------------------------------------------------------------
// Solve with the current hierarchy; a lagged hierarchy gets a soft iteration cap, and when
// the solve misses it the hierarchy is rebuilt for the current operator and the solve
// restarted.  setup() rebuilds; solve(maxit, &it, &ok) runs one Krylov solve.
template <class Setup, class Solve>
pf_status mg_solve(pf_ctx *ctx, MgState &S, bool mg, Setup setup0, Solve solve, int *lin,
                   bool *ok) {
  double *slot = (&S == &ctx->mg_u) ? &ctx->prof[PF_PROF_U_SETUP] : &ctx->prof[PF_PROF_D_SETUP];
  auto setup = [&]() -> pf_status {
    PhaseTimer tm(slot);
    return setup0();
  };
  bool fresh = false;
  if (mg && S.need()) {
    CKS(setup());
    S.built();
    fresh = true;
  }
  const int full = ctx->opt.max_lin;
  int cap = full;
  if (mg && !fresh) {
    const int soft = 3 * (S.base > 0 ? S.base : 10) + 10;
    cap = soft < full ? soft : full;
  }
  int it = 0;
  CKS(solve(cap, &it, ok));
  *lin += it;
  if (mg && !fresh && !*ok && cap < full) {
    CKS(setup());
    S.built();
    it = 0;
    CKS(solve(full, &it, ok));
    *lin += it;
  }
  if (mg) S.record(it);
  return PF_OK;
}

// ---- u-solve ---------------------------------------------------------------------------
// Internal force F at (u, d) for the material's split; VD also writes the tension bits,
// the spectral split the per-point tangents of the next Newton correction.  Returns the
// kernel launches issued.
int u_residual(pf_ctx *ctx) {
  if (ctx->m.split == PF_SPLIT_SPECTRAL) {
    sp_points(ctx->g, ctx->m, ctx->u, ctx->d, ctx->sp_Sq, ctx->sp_Dq, ctx->st);
    sp_force(ctx->g, ctx->sp_Sq, ctx->F, ctx->st);
    return 2;
  }
  elas_residual(ctx->g, ctx->m, ctx->u, ctx->d, ctx->F, ctx->tens, ctx->st);
  return 1;
}

// Spectral split: one Newton correction with the consistent tangent at u (the per-point
// tangents of the last residual evaluation) assembled into nodal stencils, FP64 and, for
// the FP32 inner solves, FP32; the multigrid hierarchy is built from the same tangents and
// its fine level is the stencil.
pf_status newton_correction_sp(pf_ctx *ctx, double tol, int *lin, int *refines, bool *ok) {
  PhaseTimer tm(&ctx->prof[PF_PROF_U_SOLVE]);
  cudaStream_t st = ctx->st;
  const size_t n = 2 * ctx->nn;
  const bool mg = ctx->precond == PF_PRECOND_GMG;
  sp_stencil<double>(ctx->g, ctx->sp_Dq, ctx->sp_S64, st);
  ctx->launches++;
  if (ctx->precision == PF_FP64) {
    auto A = [ctx, st](const double *xx, double *yy, int epi) {
      sp_apply<double>(ctx->g, ctx->sp_S64, xx, yy, st, ctx->sc, &ctx->ws, epi);
    };
    auto Af = [ctx, st](const double *xx, double *yy) {
      sp_apply<double>(ctx->g, ctx->sp_S64, xx, yy, st);
    };
    if (!mg) {
      sp_diag<double>(ctx->g, ctx->sp_S64, ctx->kz, st);
      invert<double>(n, ctx->kz, ctx->kinv, st);
      ctx->launches += 2;
    }
    auto setup = [&]() -> pf_status {
      cudaError_t e = gmg_setup_elas_qp<double>(ctx->gu, ctx->g, ctx->sp_Dq, st);
      if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "multigrid setup: %s", cudaGetErrorString(e));
      return PF_OK;
    };
    auto solve = [&](int maxit, int *it, bool *sok) {
      return pcg<double>(ctx, SL_U, A, Af, mg ? &ctx->gu : nullptr, n, ctx->kb, ctx->kx, ctx->kr,
                         ctx->kz, ctx->kp, ctx->kq, ctx->kinv, tol, maxit, it, sok);
    };
    return mg_solve(ctx, ctx->mg_u, mg, setup, solve, lin, ok);
  }
  sp_stencil<float>(ctx->g, ctx->sp_Dq, ctx->sp_S32, st);
  ctx->launches++;
  auto Af32 = [ctx, st](const float *xx, float *yy, int epi) {
    sp_apply<float>(ctx->g, ctx->sp_S32, xx, yy, st, ctx->sc, &ctx->ws, epi);
  };
  auto Ff32 = [ctx, st](const float *xx, float *yy) {
    sp_apply<float>(ctx->g, ctx->sp_S32, xx, yy, st);
  };
  if (!mg) {
    sp_diag<float>(ctx->g, ctx->sp_S32, ctx->fz, st);
    invert<float>(n, ctx->fz, ctx->finv, st);
    ctx->launches += 2;
  }
  auto setup = [&]() -> pf_status {
    cudaError_t e = gmg_setup_elas_qp<float>(ctx->gu32, ctx->g, ctx->sp_Dq, st);
    if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "multigrid setup: %s", cudaGetErrorString(e));
    return PF_OK;
  };
  auto solve = [&](int maxit, int *it, bool *iok) {
    return pcg<float>(ctx, SL_U, Af32, Ff32, mg ? &ctx->gu32 : nullptr, n, ctx->fb, ctx->fx,
                      ctx->fr, ctx->fz, ctx->fp, ctx->fq, ctx->finv, ctx->opt.tol_inner, maxit,
                      it, iok);
  };
  auto inner = [&](int *it, bool *iok) {
    int cnt = 0;
    pf_status s2 = mg_solve(ctx, ctx->mg_u, mg, setup, solve, &cnt, iok);
    *it = cnt;
    return s2;
  };
  auto AD = [ctx, st](const double *xx, double *yy) {
    sp_apply<double>(ctx->g, ctx->sp_S64, xx, yy, st);
  };
  return refine(ctx, AD, inner, n, 2, ctx->kb, ctx->kx, tol, lin, refines, ok);
}

// One Newton correction: K_t(d, tension) kx = kb on free DOFs.
pf_status newton_correction(pf_ctx *ctx, double tol, int *lin, int *refines, bool *ok) {
  if (ctx->m.split == PF_SPLIT_SPECTRAL) return newton_correction_sp(ctx, tol, lin, refines, ok);
  PhaseTimer tm(&ctx->prof[PF_PROF_U_SOLVE]);
  cudaStream_t st = ctx->st;
  const size_t n = 2 * ctx->nn;
  const bool mg = ctx->precond == PF_PRECOND_GMG;
  if (ctx->precision == PF_FP64) {
    auto A = [ctx, st](const double *xx, double *yy, int epi) {
      elas_apply<double>(ctx->g, ctx->m, ctx->d, ctx->tens, xx, yy, st, ctx->sc, &ctx->ws, epi);
    };
    auto Af = [ctx, st](const double *xx, double *yy) {
      elas_apply<double>(ctx->g, ctx->m, ctx->d, ctx->tens, xx, yy, st);
    };
    if (!mg) {
      elas_diag<double>(ctx->g, ctx->m, ctx->d, ctx->tens, ctx->kz, st);
      invert<double>(n, ctx->kz, ctx->kinv, st);
      ctx->launches += 2;
    }
    auto setup = [&]() -> pf_status {
      cudaError_t e = gmg_setup_elas<double>(ctx->gu, ctx->g, ctx->m, ctx->d, ctx->tens, st);
      if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "multigrid setup: %s", cudaGetErrorString(e));
      return PF_OK;
    };
    auto solve = [&](int maxit, int *it, bool *sok) {
      if (mg && ctx->gu.lc >= 1)
        return pcg_mg_elas<double>(ctx, ctx->gu, ctx->d, ctx->kb, ctx->kx, ctx->kr, ctx->kz,
                                   ctx->kp, ctx->kq, tol, maxit, it, sok);
      return pcg<double>(ctx, SL_U, A, Af, mg ? &ctx->gu : nullptr, n, ctx->kb, ctx->kx, ctx->kr,
                         ctx->kz, ctx->kp, ctx->kq, ctx->kinv, tol, maxit, it, sok);
    };
    return mg_solve(ctx, ctx->mg_u, mg, setup, solve, lin, ok);
  }
  auto Af32 = [ctx, st](const float *xx, float *yy, int epi) {
    elas_apply<float>(ctx->g, ctx->m, ctx->fd, ctx->tens, xx, yy, st, ctx->sc, &ctx->ws, epi,
                      ctx->tune.strip_rows);
  };
  auto Ff32 = [ctx, st](const float *xx, float *yy) {
    elas_apply<float>(ctx->g, ctx->m, ctx->fd, ctx->tens, xx, yy, st, nullptr, nullptr, 0,
                      ctx->tune.strip_rows);
  };
  if (!mg) {
    elas_diag<float>(ctx->g, ctx->m, ctx->fd, ctx->tens, ctx->fz, st);
    invert<float>(n, ctx->fz, ctx->finv, st);
    ctx->launches += 2;
  }
  auto setup = [&]() -> pf_status {
    cudaError_t e = gmg_setup_elas<float>(ctx->gu32, ctx->g, ctx->m, ctx->fd, ctx->tens, st);
    if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "multigrid setup: %s", cudaGetErrorString(e));
    return PF_OK;
  };
  auto solve = [&](int maxit, int *it, bool *iok) {
    if (mg && ctx->gu32.lc >= 1)
      return pcg_mg_elas<float>(ctx, ctx->gu32, ctx->fd, ctx->fb, ctx->fx, ctx->fr, ctx->fz,
                                ctx->fp, ctx->fq, ctx->opt.tol_inner, maxit, it, iok);
    return pcg<float>(ctx, SL_U, Af32, Ff32, mg ? &ctx->gu32 : nullptr, n, ctx->fb, ctx->fx,
                      ctx->fr, ctx->fz, ctx->fp, ctx->fq, ctx->finv, ctx->opt.tol_inner, maxit,
                      it, iok);
  };
  auto inner = [&](int *it, bool *iok) {
    int cnt = 0;
    pf_status s2 = mg_solve(ctx, ctx->mg_u, mg, setup, solve, &cnt, iok);
    *it = cnt;
    return s2;
  };
  auto AD = [ctx, st](const double *xx, double *yy) {
    elas_apply<double>(ctx->g, ctx->m, ctx->d, ctx->tens, xx, yy, st);
  };
  return refine(ctx, AD, inner, n, 2, ctx->kb, ctx->kx, tol, lin, refines, ok);
}

pf_status solve_u(pf_ctx *ctx, int *newton, int *lin, int *refines, bool *ok) {
  cudaStream_t st = ctx->st;
  const size_t n = 2 * ctx->nn;
  double r0 = -1.0;
  *ok = false;
  if (ctx->precision == PF_FP32_IR) {
    convert<double, float>(ctx->nn, ctx->d, ctx->fd, st);
    ctx->launches++;
  }
  for (int it = 0; it <= ctx->opt.max_newton; ++it) {
    {
      PhaseTimer tm(&ctx->prof[PF_PROF_U_RESID]);
      ctx->launches += u_residual(ctx);
      norms(n, 2, ctx->g.dofm, ctx->F, ctx->dscal, ctx->ws, st);
      ctx->launches++;
      CKS(check_launch(ctx));
      CKS(read_scalars(ctx, ctx->dscal, 2 * sizeof(double)));
    }
    const double rn = sqrt(ctx->hbuf[0]), fref = sqrt(ctx->hbuf[1]);
    if (r0 < 0.0) r0 = rn;
    if (rn == 0.0 || rn <= ctx->opt.tol_nr * fmax(r0, fref)) {
      *ok = true;
      return PF_OK;
    }
    if (!isfinite(rn)) return set_err(ctx, PF_ENOTCONV, "u residual is not finite");
    if (it == ctx->opt.max_newton) break;
    // rhs = -F on free DOFs
    masked_comb(n, 2, ctx->g.dofm, -1.0, ctx->F, 0.0, nullptr, ctx->kb, st);
    ctx->launches++;
    // inexact Newton: the correction's linear residual need only stay below the Newton
    // tolerance (forcing term newton_forcing * tol_nr * ref / ||R_k||, within [tol_lin, 1e-2])
    double tol = ctx->opt.tol_lin;
    if (ctx->opt.newton_forcing > 0.0) {
      const double f = ctx->opt.newton_forcing * ctx->opt.tol_nr * fmax(r0, fref) / rn;
      tol = fmax(tol, fmin(f, 1e-2));
    }
    bool lok = false;
    CKS(newton_correction(ctx, tol, lin, refines, &lok));
    add(n, ctx->kx, ctx->u, st);
    ctx->launches++;
    (*newton)++;
    if (!lok) return set_err(ctx, PF_ENOTCONV, "u linear solve did not converge");
  }
  return set_err(ctx, PF_ENOTCONV, "Newton for u hit max_newton");
}

// ---- d-solves ----------------------------------------------------------------------------
// Solve K_dd(c) x = rhs on free DOFs (rhs constrained entries zero).  c: FP64 per Gauss
// point, copied into the fixed coefficient buffer the captured graphs read.
pf_status solve_damage(pf_ctx *ctx, const double *c, const double *rhs, double *x, int *lin,
                       int *refines, bool *ok) {
  PhaseTimer tm(&ctx->prof[PF_PROF_D_SOLVE]);
  cudaStream_t st = ctx->st;
  const size_t n = ctx->nn;
  // gradient coefficient 2 G_c l / c_w: G_c l for AT2, 3 G_c l / 4 for AT1
  const double kappa = ctx->model == PF_AT1_PENALTY ? ctx->at1_kappa : ctx->m.Gc * ctx->m.l;
  const bool mg = ctx->precond == PF_PRECOND_GMG;
  if (c != ctx->csolve)
    CK(cudaMemcpyAsync(ctx->csolve, c, ctx->nq * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (ctx->precision == PF_FP64) {
    auto A = [ctx, st, kappa](const double *xx, double *yy, int epi) {
      damage_apply<double>(ctx->g, ctx->csolve, kappa, xx, yy, st, ctx->sc, &ctx->ws, epi);
    };
    auto Af = [ctx, st, kappa](const double *xx, double *yy) {
      damage_apply<double>(ctx->g, ctx->csolve, kappa, xx, yy, st);
    };
    if (!mg) {
      damage_diag<double>(ctx->g, ctx->csolve, kappa, ctx->kz, st);
      invert<double>(n, ctx->kz, ctx->kinv, st);
      ctx->launches += 2;
    }
    CK(cudaMemcpyAsync(ctx->kb, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    auto setup = [&]() -> pf_status {
      cudaError_t e = gmg_setup_damage<double>(ctx->gd, ctx->g, ctx->csolve, kappa, st);
      if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "multigrid setup: %s", cudaGetErrorString(e));
      return PF_OK;
    };
    auto solve = [&](int maxit, int *it, bool *sok) {
      if (mg && ctx->gd.lc >= 1)
        return pcg_mg_damage<double>(ctx, ctx->gd, ctx->csolve, kappa, ctx->kb, ctx->dd, ctx->kr,
                                     ctx->kz, ctx->kp, ctx->kq, ctx->opt.tol_lin, maxit, it, sok);
      return pcg<double>(ctx, SL_D, A, Af, mg ? &ctx->gd : nullptr, n, ctx->kb, ctx->dd, ctx->kr,
                         ctx->kz, ctx->kp, ctx->kq, ctx->kinv, ctx->opt.tol_lin, maxit, it, sok);
    };
    CKS(mg_solve(ctx, ctx->mg_d, mg, setup, solve, lin, ok));
    if (x != ctx->dd) CK(cudaMemcpyAsync(x, ctx->dd, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return PF_OK;
  }
  convert<double, float>(ctx->nq, ctx->csolve, ctx->fc, st);
  ctx->launches++;
  auto Af32 = [ctx, st, kappa](const float *xx, float *yy, int epi) {
    damage_apply<float>(ctx->g, ctx->fc, kappa, xx, yy, st, ctx->sc, &ctx->ws, epi);
  };
  auto Ff32 = [ctx, st, kappa](const float *xx, float *yy) {
    damage_apply<float>(ctx->g, ctx->fc, kappa, xx, yy, st);
  };
  if (!mg) {
    damage_diag<float>(ctx->g, ctx->fc, kappa, ctx->fz, st);
    invert<float>(n, ctx->fz, ctx->finv, st);
    ctx->launches += 2;
  }
  auto setup = [&]() -> pf_status {
    cudaError_t e = gmg_setup_damage<float>(ctx->gd32, ctx->g, ctx->fc, kappa, st);
    if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "multigrid setup: %s", cudaGetErrorString(e));
    return PF_OK;
  };
  auto solve = [&](int maxit, int *it, bool *iok) {
    if (mg && ctx->gd32.lc >= 1)
      return pcg_mg_damage<float>(ctx, ctx->gd32, ctx->fc, kappa, ctx->fb, ctx->fx, ctx->fr,
                                  ctx->fz, ctx->fp, ctx->fq, ctx->opt.tol_inner, maxit, it, iok);
    return pcg<float>(ctx, SL_D, Af32, Ff32, mg ? &ctx->gd32 : nullptr, n, ctx->fb, ctx->fx,
                      ctx->fr, ctx->fz, ctx->fp, ctx->fq, ctx->finv, ctx->opt.tol_inner, maxit,
                      it, iok);
  };
  auto inner = [&](int *it, bool *iok) {
    int cnt = 0;
    pf_status s2 = mg_solve(ctx, ctx->mg_d, mg, setup, solve, &cnt, iok);
    *it = cnt;
    return s2;
  };
  auto AD = [ctx, st, kappa](const double *xx, double *yy) {
    damage_apply<double>(ctx->g, ctx->csolve, kappa, xx, yy, st);
  };
  return refine(ctx, AD, inner, n, 1, rhs, x, ctx->opt.tol_lin, lin, refines, ok);
}

// rhs = free ? b(H) - K(c) d : 0 ; then d += K_ff^-1 rhs.
pf_status d_solve_from(pf_ctx *ctx, const double *c, const double *Hdrive, int *lin,
                       int *refines, bool *ok) {
  cudaStream_t st = ctx->st;
  const size_t n = ctx->nn;
  const double kappa = ctx->m.Gc * ctx->m.l;
  damage_rhs(ctx->g, Hdrive, ctx->bd, st);
  damage_apply<double>(grid_nomask(ctx), c, kappa, ctx->d, ctx->Kd, st);
  masked_comb(n, 1, ctx->g.dofm, 1.0, ctx->bd, 1.0, ctx->Kd, ctx->bd, st);
  ctx->launches += 3;
  CKS(solve_damage(ctx, c, ctx->bd, ctx->dd, lin, refines, ok));
  add(n, ctx->dd, ctx->d, st);
  ctx->launches++;
  return PF_OK;
}

// ---- AT1 with penalty (Sec. 2) -------------------------------------------------------
// Evolution equation at per-point energy psi: R_d = K(c0) d - b (k_at1_coef writes c0 to
// Hhalf, the Jacobian coefficient cJ to cq and b's integrand / 2 to bhalf).  at1_rhs puts
// -R (free DOFs) into bd and returns ||R_free||.
pf_status at1_rhs(pf_ctx *ctx, const double *psi, double *rnorm) {
  cudaStream_t st = ctx->st;
  const size_t n = ctx->nn;
  at1_coef(ctx->g, psi, ctx->d, ctx->d_prev, ctx->at1_a, ctx->at1_gamma, ctx->Hhalf, ctx->cq,
           ctx->bhalf, st);
  damage_rhs(ctx->g, ctx->bhalf, ctx->bd, st);
  damage_apply<double>(grid_nomask(ctx), ctx->Hhalf, ctx->at1_kappa, ctx->d, ctx->Kd, st);
  masked_comb(n, 1, ctx->g.dofm, 1.0, ctx->bd, 1.0, ctx->Kd, ctx->bd, st);
  norms(n, 1, ctx->g.dofm, ctx->bd, ctx->dscal, ctx->ws, st);
  ctx->launches += 5;
  CKS(check_launch(ctx));
  CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
  *rnorm = sqrt(ctx->hbuf[0]);
  return PF_OK;
}

// ||int a N||_free: the scale of the Newton test of the AT1 evolution equation.
pf_status at1_scale(pf_ctx *ctx, double *fscale) {
  cudaStream_t st = ctx->st;
  fill(ctx->nq, 0.5 * ctx->at1_a, ctx->bhalf, st);
  damage_rhs(ctx->g, ctx->bhalf, ctx->bd, st);
  norms(ctx->nn, 1, ctx->g.dofm, ctx->bd, ctx->dscal, ctx->ws, st);
  ctx->launches += 3;
  CKS(check_launch(ctx));
  CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
  *fscale = sqrt(ctx->hbuf[0]);
  return PF_OK;
}

// Semismooth Newton for the AT1 evolution equation at per-point energy psi: solve
// K(cJ) dd = -R on the free DOFs, d += dd, until ||R_free|| <= tol_lin max(||R^0_free||,
// ||int a N||_free).  The equation is piecewise linear (the penalty), so the iterate after
// the penalised set settles is exact to the linear tolerance; stopping at tol_nr instead
// would leave a d-residual above the staggered test's tolerance.
pf_status at1_newton(pf_ctx *ctx, const double *psi, double fscale, int *lin, int *refines,
                     int *dsolves, bool *ok) {
  double r0 = -1.0;
  *ok = false;
  for (int it = 0; it <= ctx->opt.max_newton; ++it) {
    double rn;
    CKS(at1_rhs(ctx, psi, &rn));
    if (r0 < 0.0) r0 = rn;
    if (rn == 0.0 || rn <= ctx->opt.tol_lin * fmax(r0, fscale)) {
      *ok = true;
      return PF_OK;
    }
    if (!isfinite(rn)) return set_err(ctx, PF_ENOTCONV, "d residual is not finite");
    if (it == ctx->opt.max_newton) break;
    bool lok = false;
    CKS(solve_damage(ctx, ctx->cq, ctx->bd, ctx->dd, lin, refines, &lok));
    (*dsolves)++;
    add(ctx->nn, ctx->dd, ctx->d, ctx->st);
    ctx->launches++;
    if (!lok) return set_err(ctx, PF_ENOTCONV, "d linear solve did not converge");
  }
  return PF_OK;
}

// AT1 d-step.  ST: Newton with Psi+(u^k) (Hk).  S1/S2/S3 (Sec. 3.3-3.5): the first NR
// iteration with the augmented tangent gives Delta d (dd), the active energy is predicted
// from it where the softening test holds and frozen (Hk), and the NR iterations continue
// from d^k + Delta d with it.
pf_status at1_d_step(pf_ctx *ctx, int scheme, int *lin, int *refines, int *dsolves, bool *ok) {
  cudaStream_t st = ctx->st;
  // current energy into Hk (csolve takes the unused history output)
  point_energy(ctx->g, ctx->m, ctx->u, ctx->H, ctx->Hk, ctx->csolve, st);
  ctx->launches++;
  double fscale;
  CKS(at1_scale(ctx, &fscale));
  if (scheme == PF_ST) return at1_newton(ctx, ctx->Hk, fscale, lin, refines, dsolves, ok);
  const double pc = ctx->opt.psi_crit < 0.0 ? ctx->at1_a : ctx->opt.psi_crit;
  At1D at1;
  at1.on = 1;
  at1.dprev = ctx->d_prev;
  at1.gamma = ctx->at1_gamma;
  at1.floor = ctx->at1_floor;
  // augmented coefficient into csolve (solve_damage uses it in place)
  point_fs_coeff(ctx->g, ctx->m, scheme, pc, ctx->u, ctx->d, ctx->H, ctx->csolve, ctx->act, st, at1);
  ctx->launches++;
  double rn;
  CKS(at1_rhs(ctx, ctx->Hk, &rn));
  if (rn == 0.0 || rn <= ctx->opt.tol_lin * fscale) {
    *ok = true;   // already at the solution of the evolution equation
    return PF_OK;
  }
  bool ok1 = false;
  CKS(solve_damage(ctx, ctx->csolve, ctx->bd, ctx->dd, lin, refines, &ok1));
  (*dsolves)++;
  point_fs_predict(ctx->g, ctx->m, scheme, ctx->u, ctx->d, ctx->dd, ctx->H, ctx->act, ctx->Hk, st, 1);
  add(ctx->nn, ctx->dd, ctx->d, st);
  ctx->launches += 2;
  CKS(at1_newton(ctx, ctx->Hk, fscale, lin, refines, dsolves, ok));
  *ok = *ok && ok1;
  return PF_OK;
}

// AT1 staggered residual: max |R_d,i / J_ii| over free d-DOFs with Psi+(u^{k+1}) and the
// penalty at d^{k+1}.
pf_status at1_stag_residual(pf_ctx *ctx, double *out) {
  cudaStream_t st = ctx->st;
  point_energy(ctx->g, ctx->m, ctx->u, ctx->H, ctx->Hk, ctx->csolve, st);
  at1_coef(ctx->g, ctx->Hk, ctx->d, ctx->d_prev, ctx->at1_a, ctx->at1_gamma, ctx->Hhalf, ctx->cq,
           ctx->bhalf, st);
  damage_rhs(ctx->g, ctx->bhalf, ctx->bd, st);
  damage_apply<double>(grid_nomask(ctx), ctx->Hhalf, ctx->at1_kappa, ctx->d, ctx->Kd, st);
  damage_diag<double>(grid_nomask(ctx), ctx->cq, ctx->at1_kappa, ctx->kz, st);
  stag_max(ctx->nn, ctx->g.dofm, ctx->Kd, ctx->bd, ctx->kz, ctx->dscal, ctx->ws, st);
  ctx->launches += 6;
  CKS(check_launch(ctx));
  CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
  *out = ctx->hbuf[0];
  return PF_OK;
}

pf_status d_step(pf_ctx *ctx, int scheme, int *lin, int *refines, int *dsolves, bool *ok) {
  if (ctx->model == PF_AT1_PENALTY) return at1_d_step(ctx, scheme, lin, refines, dsolves, ok);
  cudaStream_t st = ctx->st;
  const double gcl = ctx->m.Gc / ctx->m.l;
  const double kappa = ctx->m.Gc * ctx->m.l;
  const size_t n = ctx->nn;
  point_energy(ctx->g, ctx->m, ctx->u, ctx->H, nullptr, ctx->Hk, st);
  ctx->launches++;
  if (scheme == PF_ST) {
    coef<double>(ctx->nq, gcl, ctx->Hk, ctx->cq, st);
    ctx->launches++;
    CKS(d_solve_from(ctx, ctx->cq, ctx->Hk, lin, refines, ok));
    (*dsolves)++;
    return PF_OK;
  }
  // S1/S2/S3: augmented first NR iteration for Delta d (Sec. 3.4) ...
  const double pc = ctx->opt.psi_crit < 0.0 ? ctx->m.Gc / (2.0 * ctx->m.l) : ctx->opt.psi_crit;
  point_fs_coeff(ctx->g, ctx->m, scheme, pc, ctx->u, ctx->d, ctx->H, ctx->Hhalf, ctx->act, st);
  coef<double>(ctx->nq, gcl, ctx->Hk, ctx->cq, st);
  damage_rhs(ctx->g, ctx->Hk, ctx->bd, st);
  damage_apply<double>(grid_nomask(ctx), ctx->cq, kappa, ctx->d, ctx->Kd, st);
  masked_comb(n, 1, ctx->g.dofm, 1.0, ctx->bd, 1.0, ctx->Kd, ctx->bd, st);  // -R_d
  ctx->launches += 5;
  bool ok1 = false;
  CKS(solve_damage(ctx, ctx->Hhalf, ctx->bd, ctx->dd, lin, refines, &ok1));
  (*dsolves)++;
  // ... predicted history (Sec. 3.3, Delta d > 0 rule of Sec. 3.5) ...
  point_fs_predict(ctx->g, ctx->m, scheme, ctx->u, ctx->d, ctx->dd, ctx->H, ctx->act, ctx->Hhalf, st);
  // ... and the frozen, linear evolution equation.
  coef<double>(ctx->nq, gcl, ctx->Hhalf, ctx->cq, st);
  ctx->launches += 2;
  CKS(d_solve_from(ctx, ctx->cq, ctx->Hhalf, lin, refines, ok));
  (*dsolves)++;
  *ok = *ok && ok1;
  return PF_OK;
}

pf_status stag_residual(pf_ctx *ctx, double *out) {
  PhaseTimer tm(&ctx->prof[PF_PROF_STAG]);
  if (ctx->model == PF_AT1_PENALTY) return at1_stag_residual(ctx, out);
  cudaStream_t st = ctx->st;
  const double gcl = ctx->m.Gc / ctx->m.l;
  const double kappa = ctx->m.Gc * ctx->m.l;
  point_energy(ctx->g, ctx->m, ctx->u, ctx->H, nullptr, ctx->Hk, st);
  coef<double>(ctx->nq, gcl, ctx->Hk, ctx->cq, st);
  damage_rhs(ctx->g, ctx->Hk, ctx->bd, st);
  damage_apply<double>(grid_nomask(ctx), ctx->cq, kappa, ctx->d, ctx->Kd, st);
  damage_diag<double>(grid_nomask(ctx), ctx->cq, kappa, ctx->kz, st);
  stag_max(ctx->nn, ctx->g.dofm, ctx->Kd, ctx->bd, ctx->kz, ctx->dscal, ctx->ws, st);
  ctx->launches += 6;
  CKS(check_launch(ctx));
  CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
  *out = ctx->hbuf[0];
  return PF_OK;
}

// Every device array of a context, in one fixed order, taken from arena A (a dry run when
// A has no base: it sizes the context's single slab and answers pf_footprint_bytes, so
// the two cannot disagree).  Only mesh fields and ctx's pointer slots are used.
bool layout(pf_ctx *ctx, const pf_mesh *mesh, Arena &A) {
  const size_t nn = (size_t)(mesh->nx + 1) * (mesh->ny + 1), ne = (size_t)mesh->nx * mesh->ny;
  const size_t nq = 4 * ne;
  const bool f32 = mesh->precision == PF_FP32_IR;
#define AL(p, n)                     \
  do {                               \
    if (!A.take(&ctx->p, (n))) return false; \
  } while (0)
  AL(u, 2 * nn); AL(d, nn); AL(H, nq); AL(d_prev, nn); AL(F, 2 * nn);
  AL(Hk, nq); AL(cq, nq); AL(Hhalf, nq); AL(act, nq);
  AL(bd, nn); AL(Kd, nn); AL(dd, nn); AL(csolve, nq);
  if (mesh->model == PF_AT1_PENALTY) AL(bhalf, nq);
  if (mesh->split == PF_SPLIT_SPECTRAL) {
    AL(sp_Sq, 3 * nq); AL(sp_Dq, 6 * nq); AL(sp_S64, 36 * nn);
    if (f32) AL(sp_S32, 36 * nn);
  }
  AL(flags, nn); AL(dofm, nn); AL(tens, ne);
  if (mesh->elem_active) AL(active, ne);
  AL(kb, 2 * nn); AL(kx, 2 * nn); AL(kr, 2 * nn); AL(kz, 2 * nn); AL(kp, 2 * nn);
  AL(kq, 2 * nn); AL(kinv, 2 * nn); AL(kres, 2 * nn);
  if (f32) {
    AL(fb, 2 * nn); AL(fx, 2 * nn); AL(fr, 2 * nn); AL(fz, 2 * nn); AL(fp, 2 * nn);
    AL(fq, 2 * nn); AL(finv, 2 * nn); AL(fd, nn); AL(fc, nq);
  }
  AL(sc, 1); AL(dscal, 8);
  {
    const size_t tiles = (size_t)tile_blocks_x(mesh->nx) * tile_blocks_y(mesh->ny);
    ctx->ws.max_blocks = (int)(tiles > 4096 ? tiles : 4096);
  }
  AL(ws.partials, 4 * (size_t)ctx->ws.max_blocks);
  AL(ws.counter, red_counters(ctx->ws.max_blocks));
#undef AL
  if (mesh->precond == PF_PRECOND_GMG) {
    cudaError_t e1, e2;
    if (!f32) {
      e1 = gmg_alloc<double>(ctx->gu, mesh->nx, mesh->ny, 2, ctx->ws, A);
      e2 = gmg_alloc<double>(ctx->gd, mesh->nx, mesh->ny, 1, ctx->ws, A);
    } else {
      e1 = gmg_alloc<float>(ctx->gu32, mesh->nx, mesh->ny, 2, ctx->ws, A);
      e2 = gmg_alloc<float>(ctx->gd32, mesh->nx, mesh->ny, 1, ctx->ws, A);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) return false;
  }
  return true;
}

void free_all(pf_ctx *c) {
  if (c->slab) cudaFree(c->slab);
  c->slab = nullptr;
  gmg_free<double>(c->gu);
  gmg_free<double>(c->gd);
  gmg_free<float>(c->gu32);
  gmg_free<float>(c->gd32);
  for (GraphSlot &g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (WhileGraph &w : c->wgraphs)
    if (w.exec) cudaGraphExecDestroy(w.exec);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  if (c->evb) cudaEventDestroy(c->evb);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

void pf_default_options(pf_options *o) {
  if (!o) return;
  o->tol_nr = 1e-7;
  o->tol_lin = 1e-10;
  o->tol_inner = 1e-3;
  o->max_newton = 50;
  o->max_stag = 1000;
  o->max_lin = 200000;
  o->max_refine = 30;
  o->psi_crit = -1.0;
  o->project = 0;
  o->check_every = 8;
  o->newton_forcing = 1e-3;
  o->device_loop = 1;
}

const char *pf_status_string(pf_status s) {
  switch (s) {
    case PF_OK: return "PF_OK";
    case PF_EINVAL: return "PF_EINVAL";
    case PF_ENOMEM: return "PF_ENOMEM";
    case PF_ENOTCONV: return "PF_ENOTCONV";
    case PF_ECUDA: return "PF_ECUDA";
    case PF_ETIMEOUT: return "PF_ETIMEOUT";
    case PF_EBUSY: return "PF_EBUSY";
  }
  return "unknown";
}

pf_status pf_material_make(double E, double nu, double Gc, double l, double k_res, int plane,
                           pf_material *out) {
  if (!out || !(E > 0) || !(nu > -1.0 && nu < 0.5) || !(Gc > 0) || !(l > 0) || !(k_res >= 0) ||
      (plane != PF_PLANE_STRAIN && plane != PF_PLANE_STRESS))
    return PF_EINVAL;
  const double mu = E / (2.0 * (1.0 + nu));
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  out->mu = mu;
  if (plane == PF_PLANE_STRAIN) {
    out->K = lam + 2.0 * mu / 3.0;
    out->cdim = 1.0 / 3.0;
  } else {
    out->K = E / (2.0 * (1.0 - nu));
    out->cdim = 0.5;
  }
  out->eta = k_res;
  out->Gc = Gc;
  out->l = l;
  out->split = PF_SPLIT_VD;
  return PF_OK;
}

pf_status pf_create(const pf_mesh *mesh, double E, double nu, double Gc, double l, double k_res,
                    pf_ctx **out) {
  if (!out) return PF_EINVAL;
  *out = nullptr;
  if (!mesh || !mesh->node_flags || mesh->nx < 1 || mesh->ny < 1 || !(mesh->Lx > 0) ||
      !(mesh->Ly > 0) || (mesh->precision != PF_FP64 && mesh->precision != PF_FP32_IR) ||
      (mesh->reaction_dir != 0 && mesh->reaction_dir != 1) ||
      (mesh->precond != PF_PRECOND_JACOBI && mesh->precond != PF_PRECOND_GMG) ||
      (mesh->model != PF_AT2_HISTORY && mesh->model != PF_AT1_PENALTY) ||
      (mesh->split != PF_SPLIT_VD && mesh->split != PF_SPLIT_SPECTRAL) ||
      !(mesh->tol_ir == mesh->tol_ir))
    return PF_EINVAL;
  if ((double)(mesh->nx + 1) * (double)(mesh->ny + 1) > 4.0e8) return PF_EINVAL;
  pf_material mat;
  if (pf_material_make(E, nu, Gc, l, k_res, mesh->plane, &mat) != PF_OK) return PF_EINVAL;
  pf_ctx *ctx = new (std::nothrow) pf_ctx();
  if (!ctx) return PF_ENOMEM;
  pf_default_options(&ctx->opt);
  cudaGetDevice(&ctx->device);
  ctx->nn = (size_t)(mesh->nx + 1) * (mesh->ny + 1);
  ctx->ne = (size_t)mesh->nx * mesh->ny;
  ctx->nq = 4 * ctx->ne;
  ctx->precision = mesh->precision;
  ctx->reaction_dir = mesh->reaction_dir;
  ctx->precond = mesh->precond;
  ctx->plane = mesh->plane;
  ctx->m = MatD{mat.mu, mat.K, mat.cdim, mat.eta, mat.Gc, mat.l, mesh->split};
  ctx->model = mesh->model;
  if (ctx->model == PF_AT1_PENALTY) {
    const double cw = 8.0 / 3.0, tir = mesh->tol_ir > 0.0 ? mesh->tol_ir : 0.01;
    ctx->at1_a = Gc / (cw * l);
    ctx->at1_kappa = 2.0 * Gc * l / cw;
    ctx->at1_gamma = 27.0 * Gc / (64.0 * l * tir * tir);
    ctx->at1_floor = 2.0 * Gc / (cw * l);
  }
  pf_status s = PF_OK;
  auto fail = [&](pf_status st) {
    free_all(ctx);
    delete ctx;
    return st;
  };
  if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess)
    return fail(PF_ECUDA);
  ctx->own_stream = true;
  const size_t nn = ctx->nn, ne = ctx->ne, nq = ctx->nq;
  {
    Arena dry;
    if (!layout(ctx, mesh, dry)) return fail(set_err(ctx, PF_EINVAL, "layout"));
    cudaError_t e = cudaMalloc((void **)&ctx->slab, dry.used);
    if (e != cudaSuccess) {
      ctx->slab = nullptr;
      cudaGetLastError();
      return fail(PF_ENOMEM);
    }
    Arena real;
    real.base = ctx->slab;
    real.cap = dry.used;
    if (!layout(ctx, mesh, real)) return fail(PF_ENOMEM);
  }
  if (cudaMallocHost((void **)&ctx->hbuf, 256) != cudaSuccess) return fail(PF_ENOMEM);
  if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess)
    return fail(PF_ECUDA);
  cudaStream_t st = ctx->st;
  bool okc = cudaMemsetAsync(ctx->ws.counter, 0, red_counters(ctx->ws.max_blocks) * sizeof(unsigned),
                             st) == cudaSuccess &&
             cudaMemsetAsync(ctx->sc, 0, sizeof(KrylovScal), st) == cudaSuccess &&
             cudaMemcpyAsync(ctx->flags, mesh->node_flags, nn, cudaMemcpyHostToDevice, st) ==
                 cudaSuccess &&
             (!mesh->elem_active ||
              cudaMemcpyAsync(ctx->active, mesh->elem_active, ne, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess) &&
             cudaMemsetAsync(ctx->u, 0, 2 * nn * sizeof(double), st) == cudaSuccess &&
             cudaMemsetAsync(ctx->H, 0, nq * sizeof(double), st) == cudaSuccess &&
             cudaMemsetAsync(ctx->tens, 0, ne, st) == cudaSuccess;
  if (!okc) return fail(PF_ECUDA);
  ctx->g = GridD{mesh->nx, mesh->ny, mesh->Lx / mesh->nx, mesh->Ly / mesh->ny, ctx->active,
                 ctx->dofm};
  dof_mask(mesh->nx, mesh->ny, ctx->flags, ctx->active, ctx->dofm, st);
  // d = 1 on D_FIX1 nodes with an active element, else 0
  {
    std::vector<double> d0(nn, 0.0);
    for (size_t i = 0; i < nn; ++i) d0[i] = (mesh->node_flags[i] & PF_D_FIX1) ? 1.0 : 0.0;
    if (mesh->elem_active) {
      const int nx = mesh->nx, ny = mesh->ny;
      for (size_t i = 0; i < nn; ++i) {
        if (d0[i] == 0.0) continue;
        const int ii = (int)(i % (nx + 1)), jj = (int)(i / (nx + 1));
        bool touched = false;
        for (int dj = -1; dj <= 0; ++dj)
          for (int di = -1; di <= 0; ++di) {
            const int ei = ii + di, ej = jj + dj;
            if (ei >= 0 && ei < nx && ej >= 0 && ej < ny && mesh->elem_active[(size_t)ej * nx + ei])
              touched = true;
          }
        if (!touched) d0[i] = 0.0;
      }
    }
    if (cudaMemcpy(ctx->d, d0.data(), nn * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return fail(PF_ECUDA);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(PF_ECUDA);
  ctx->launches = 1;
  *out = ctx;
  return PF_OK;
}

size_t pf_footprint_bytes(const pf_mesh *mesh) {
  if (!mesh || mesh->nx < 1 || mesh->ny < 1) return 0;
  std::unique_ptr<pf_ctx> tmp(new (std::nothrow) pf_ctx());
  if (!tmp) return 0;
  Arena dry;
  if (!layout(tmp.get(), mesh, dry)) return 0;
  return dry.used;
}

pf_status pf_set_options(pf_ctx *ctx, const pf_options *o) {
  if (!ctx || !o) return PF_EINVAL;
  if (!(o->tol_nr > 0) || !(o->tol_lin > 0) || !(o->tol_inner > 0) || o->max_newton < 1 ||
      o->max_stag < 1 || o->max_lin < 1 || o->max_refine < 1 || o->check_every < 1 ||
      !(o->newton_forcing >= 0) || (o->device_loop != 0 && o->device_loop != 1))
    return set_err(ctx, PF_EINVAL, "invalid options");
  ctx->opt = *o;
  return PF_OK;
}

pf_status pf_get_options(const pf_ctx *ctx, pf_options *o) {
  if (!ctx || !o) return PF_EINVAL;
  *o = ctx->opt;
  return PF_OK;
}

pf_status pf_load_step(pf_ctx *ctx, double d_ubar, int scheme, double tol,
                       pf_step_result *res) {
  if (!ctx) return PF_EINVAL;
  if (scheme < PF_ST || scheme > PF_S3 || !(tol > 0) || !isfinite(d_ubar))
    return set_err(ctx, PF_EINVAL, "invalid scheme/tol/d_ubar");
  CK(cudaSetDevice(ctx->device));
  BatchScope batch_scope(ctx);
  PhaseTimer tm_all(&ctx->prof[PF_PROF_TOTAL]);
  pf_step_result r;
  memset(&r, 0, sizeof(r));
  cudaStream_t st = ctx->st;
  CK(cudaEventRecord(ctx->ev0, st));
  ctx->ubar += d_ubar;
  r.ubar = ctx->ubar;
  lift(ctx->nn, ctx->flags, ctx->dofm, ctx->ubar, ctx->u, st);
  ctx->launches++;
  // d_{n-1}: the projection bound, and the AT1 penalty's reference
  if (ctx->opt.project || ctx->model == PF_AT1_PENALTY)
    CK(cudaMemcpyAsync(ctx->d_prev, ctx->d, ctx->nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  bool ok = false, all_ok = true;
  pf_status s = solve_u(ctx, &r.newton_u, &r.lin_u, &r.refine_steps, &ok);
  if (s != PF_OK && s != PF_ENOTCONV) return s;
  all_ok = all_ok && ok;
  double resid = INFINITY;
  for (int k = 0; k < ctx->opt.max_stag; ++k) {
    bool dok = false;
    s = d_step(ctx, scheme, &r.lin_d, &r.refine_steps, &r.d_solves, &dok);
    if (s != PF_OK && s != PF_ENOTCONV) return s;
    if (ctx->opt.project) {
      project(ctx->nn, ctx->g.dofm, ctx->d_prev, ctx->d, st);
      ctx->launches++;
    }
    s = solve_u(ctx, &r.newton_u, &r.lin_u, &r.refine_steps, &ok);
    if (s != PF_OK && s != PF_ENOTCONV) return s;
    all_ok = all_ok && ok && dok;
    s = stag_residual(ctx, &resid);
    if (s != PF_OK) return s;
    r.stag_iters = k + 1;
    if (resid <= tol) {
      r.converged = 1;
      break;
    }
    if (!isfinite(resid)) break;
  }
  r.stag_residual = resid;
  // commit history and report the reaction force
  point_energy(ctx->g, ctx->m, ctx->u, ctx->H, nullptr, ctx->Hk, st);
  ctx->launches++;
  CK(cudaMemcpyAsync(ctx->H, ctx->Hk, ctx->nq * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ctx->launches += u_residual(ctx);
  reaction(ctx->nn, ctx->flags, ctx->reaction_dir, ctx->F, ctx->dscal, ctx->ws, st);
  ctx->launches++;
  CK(cudaEventRecord(ctx->ev1, st));
  CKS(check_launch(ctx));
  CKS(read_scalars(ctx, ctx->dscal, sizeof(double)));
  r.reaction = ctx->hbuf[0];
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  r.ms = ms;
  ctx->step++;
  if (res) *res = r;
  if (!r.converged || !all_ok)
    return set_err(ctx, PF_ENOTCONV, "load step %lld: staggered residual %.3e after %d passes%s",
                   (long long)ctx->step, resid, r.stag_iters,
                   all_ok ? "" : " (an inner solve hit its cap)");
  return PF_OK;
}

pf_status pf_get_fields(pf_ctx *ctx, double *u, double *d, double *H) {
  if (!ctx) return PF_EINVAL;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->st;
  if (u) CK(cudaMemcpyAsync(u, ctx->u, 2 * ctx->nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (d) CK(cudaMemcpyAsync(d, ctx->d, ctx->nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (H) CK(cudaMemcpyAsync(H, ctx->H, ctx->nq * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PF_OK;
}

pf_status pf_set_fields(pf_ctx *ctx, const double *u, const double *d, const double *H,
                        double ubar) {
  if (!ctx || !isfinite(ubar)) return PF_EINVAL;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->st;
  if (u) CK(cudaMemcpyAsync(ctx->u, u, 2 * ctx->nn * sizeof(double), cudaMemcpyHostToDevice, st));
  if (d) CK(cudaMemcpyAsync(ctx->d, d, ctx->nn * sizeof(double), cudaMemcpyHostToDevice, st));
  if (H) CK(cudaMemcpyAsync(ctx->H, H, ctx->nq * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->ubar = ubar;
  ctx->mg_u.stale = ctx->mg_d.stale = true;
  return PF_OK;
}

static const uint64_t PF_STATE_MAGIC = 0x3130326670666670ull;  // "pffpf201"

size_t pf_state_size(const pf_ctx *ctx) {
  if (!ctx) return 0;
  return 4 * sizeof(uint64_t) + 2 * sizeof(double) +
         (3 * ctx->nn + ctx->nq) * sizeof(double);
}

pf_status pf_get_state(pf_ctx *ctx, void *buf, size_t size) {
  if (!ctx || !buf || size < pf_state_size(ctx)) return PF_EINVAL;
  uint64_t *hdr = (uint64_t *)buf;
  hdr[0] = PF_STATE_MAGIC;
  hdr[1] = ctx->nn;
  hdr[2] = ctx->nq;
  hdr[3] = (uint64_t)ctx->step;
  double *p = (double *)(hdr + 4);
  p[0] = ctx->ubar;
  p[1] = 0.0;
  return pf_get_fields(ctx, p + 2, p + 2 + 2 * ctx->nn, p + 2 + 3 * ctx->nn);
}

pf_status pf_set_state(pf_ctx *ctx, const void *buf, size_t size) {
  if (!ctx || !buf || size < pf_state_size(ctx)) return PF_EINVAL;
  const uint64_t *hdr = (const uint64_t *)buf;
  if (hdr[0] != PF_STATE_MAGIC || hdr[1] != ctx->nn || hdr[2] != ctx->nq)
    return set_err(ctx, PF_EINVAL, "state buffer does not match this mesh");
  const double *p = (const double *)(hdr + 4);
  pf_status s = pf_set_fields(ctx, p + 2, p + 2 + 2 * ctx->nn, p + 2 + 3 * ctx->nn, p[0]);
  if (s == PF_OK) ctx->step = (int64_t)hdr[3];
  return s;
}

pf_status pf_sizes(const pf_ctx *ctx, int64_t *n_nodes, int64_t *n_elems, int64_t *n_qp) {
  if (!ctx) return PF_EINVAL;
  if (n_nodes) *n_nodes = (int64_t)ctx->nn;
  if (n_elems) *n_elems = (int64_t)ctx->ne;
  if (n_qp) *n_qp = (int64_t)ctx->nq;
  return PF_OK;
}

int64_t pf_launch_count(const pf_ctx *ctx) { return ctx ? ctx->launches : 0; }

pf_status pf_profile(pf_ctx *ctx, double *ms, int n, int reset) {
  if (!ctx || (n > 0 && !ms) || n < 0) return PF_EINVAL;
  for (int i = 0; i < n && i < PF_PROF_PHASES; ++i) ms[i] = ctx->prof[i];
  if (reset)
    for (double &v : ctx->prof) v = 0.0;
  return PF_OK;
}

const char *pf_last_error(const pf_ctx *ctx) { return ctx ? ctx->err : "null context"; }

void pf_destroy(pf_ctx *ctx) {
  if (!ctx) return;
  if (ctx->batch) pf_batch_detach(ctx->batch, ctx);
  cudaSetDevice(ctx->device);
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  free_all(ctx);
  delete ctx;
}

// ---- autotuning -----------------------------------------------------------------------------
pf_status pf_get_tuning(const pf_ctx *ctx, pf_tuning *out) {
  if (!ctx || !out) return PF_EINVAL;
  *out = ctx->tune;
  return PF_OK;
}

pf_status pf_autotune(pf_ctx *ctx, pf_tuning *out) {
  if (!ctx) return PF_EINVAL;
  if (ctx->precision != PF_FP32_IR || ctx->precond != PF_PRECOND_GMG ||
      ctx->m.split != PF_SPLIT_VD)
    return set_err(ctx, PF_EINVAL, "autotune: needs FP32_IR, GMG and the VD split");
  if (ctx->step != 0 || ctx->batch)
    return set_err(ctx, PF_EBUSY, "autotune: only before the first load step, unattached");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->st;
  pf_tuning t{};
  // operands: the initial phase field and tension bits, a smooth vector
  convert<double, float>(ctx->nn, ctx->d, ctx->fd, st);
  fill_ramp_f32(2 * ctx->nn, ctx->fx, st);
  auto time_it = [&](auto launch) -> double {
    for (int k = 0; k < 3; ++k) launch();
    cudaEventRecord(ctx->ev0, st);
    for (int k = 0; k < 10; ++k) launch();
    cudaEventRecord(ctx->ev1, st);
    cudaEventSynchronize(ctx->ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    return 100.0 * ms;   // microseconds per launch
  };
  const int srs[3] = {2, 4, 8};
  double best = INFINITY;
  for (int k = 0; k < 3; ++k) {
    t.apply_us[k] = time_it([&]() {
      elas_apply<float>(ctx->g, ctx->m, ctx->fd, ctx->tens, ctx->fx, ctx->fq, st, nullptr,
                        nullptr, 0, srs[k]);
    });
    if (t.apply_us[k] < best) {
      best = t.apply_us[k];
      t.strip_rows = srs[k];
    }
  }
  Gmg<float> &G = ctx->gu32;
  cudaError_t e = gmg_setup_elas<float>(G, ctx->g, ctx->m, ctx->fd, ctx->tens, st);
  if (e != cudaSuccess) return set_err(ctx, PF_ECUDA, "autotune setup: %s", cudaGetErrorString(e));
  CK(cudaMemsetAsync(G.lv[1].b, 0, (size_t)G.B * G.lv[1].nn * sizeof(float), st));
  const int limits[3] = {300, 1100, 4300};
  best = INFINITY;
  t.coarse_nodes = GMG_CTA_NODES;
  for (int k = 0; k < 3; ++k) {
    if (gmg_set_coarse_nodes<float>(G, limits[k]) < 1) continue;   // fused path needs lc >= 1
    t.vcycle_us[k] = time_it([&]() { gmg_mid<float>(G, 1, st); });
    if (t.vcycle_us[k] < best) {
      best = t.vcycle_us[k];
      t.coarse_nodes = limits[k];
    }
  }
  gmg_set_coarse_nodes<float>(G, t.coarse_nodes);
  gmg_set_coarse_nodes<float>(ctx->gd32, t.coarse_nodes);
  ctx->mg_u.stale = true;   // the first solve rebuilds for its own operator
  CKS(check_launch(ctx));
  CK(cudaStreamSynchronize(st));
  ctx->tune = t;
  if (out) *out = t;
  return PF_OK;
}

// ---- batches (pf_batch_*) ------------------------------------------------------------------
pf_status pf_batch_create(pf_batch **out) {
  if (!out) return PF_EINVAL;
  *out = nullptr;
  pf_batch *b = new (std::nothrow) pf_batch();
  if (!b) return PF_ENOMEM;
  cudaGetDevice(&b->device);
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return PF_ECUDA;
  }
  *out = b;
  return PF_OK;
}

pf_status pf_batch_attach(pf_batch *b, pf_ctx *ctx) {
  if (!b || !ctx) return PF_EINVAL;
  if (ctx->batch)
    return ctx->batch == b ? PF_OK : set_err(ctx, PF_EBUSY, "context is attached to another batch");
  if (ctx->device != b->device)
    return set_err(ctx, PF_EINVAL, "batch and context are on different devices");
  CK(cudaSetDevice(ctx->device));
  if (ctx->precision == PF_FP32_IR && ctx->precond == PF_PRECOND_GMG) {
    if ((ctx->gu32.lc >= 1 && gmg_batch_prepare<float>(ctx->gu32) != cudaSuccess) ||
        (ctx->gd32.lc >= 1 && gmg_batch_prepare<float>(ctx->gd32) != cudaSuccess))
      return set_err(ctx, PF_ENOMEM, "batch: coarse-cycle arguments");
  }
  if (!ctx->evb && cudaEventCreateWithFlags(&ctx->evb, cudaEventDisableTiming) != cudaSuccess)
    return set_err(ctx, PF_ECUDA, "batch: event");
  std::lock_guard<std::mutex> lk(b->mu);
  b->members.push_back(ctx);
  ctx->batch = b;
  return PF_OK;
}

pf_status pf_batch_detach(pf_batch *b, pf_ctx *ctx) {
  if (!b || !ctx || ctx->batch != b) return PF_EINVAL;
  std::unique_lock<std::mutex> lk(b->mu);
  if (ctx->batching) return set_err(ctx, PF_EBUSY, "batch: context is inside a load step");
  b->cv.wait(lk, [b]() { return !b->leading; });   // graphs are in use while a batch runs
  for (auto it = b->graphs.begin(); it != b->graphs.end();) {
    bool has = false;
    for (size_t k = 1; k < it->first.size(); ++k) has = has || it->first[k] == (uintptr_t)ctx;
    if (has) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      it = b->graphs.erase(it);
    } else {
      ++it;
    }
  }
  for (size_t k = 0; k < b->members.size(); ++k)
    if (b->members[k] == ctx) {
      b->members.erase(b->members.begin() + (long)k);
      break;
    }
  ctx->batch = nullptr;
  return PF_OK;
}

pf_status pf_batch_load_step(pf_batch *b, int n, pf_ctx *const *ctx, const double *d_ubar,
                             const int *scheme, const double *tol, pf_step_result *res,
                             pf_status *status) {
  if (!b || n < 1 || !ctx || !d_ubar || !scheme || !tol) return PF_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctx[i] || ctx[i]->batch != b) return PF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctx[j] == ctx[i]) return PF_EINVAL;
  }
  std::vector<pf_status> st(n, PF_OK);
  std::vector<pf_step_result> rs(n);
  auto one = [&](int i) { st[i] = pf_load_step(ctx[i], d_ubar[i], scheme[i], tol[i], &rs[i]); };
  std::vector<std::thread> th;
  try {
    for (int i = 1; i < n; ++i) th.emplace_back(one, i);
  } catch (...) {
    for (std::thread &t : th) t.join();
    return PF_ENOMEM;
  }
  one(0);
  for (std::thread &t : th) t.join();
  pf_status worst = PF_OK;
  for (int i = 0; i < n; ++i) {
    if (res) res[i] = rs[i];
    if (status) status[i] = st[i];
    if (st[i] != PF_OK && (worst == PF_OK || worst == PF_ENOTCONV)) worst = st[i];
  }
  return worst;
}

pf_status pf_batch_stats(const pf_batch *b, int64_t *launches, int64_t *solves, int64_t *groups,
                         int *max_group) {
  if (!b) return PF_EINVAL;
  std::lock_guard<std::mutex> lk(const_cast<pf_batch *>(b)->mu);
  if (launches) *launches = b->launches;
  if (solves) *solves = b->solves;
  if (groups) *groups = b->groups;
  if (max_group) *max_group = b->max_group;
  return PF_OK;
}

void pf_batch_destroy(pf_batch *b) {
  if (!b) return;
  while (true) {
    pf_ctx *c = nullptr;
    {
      std::lock_guard<std::mutex> lk(b->mu);
      if (b->members.empty()) break;
      c = b->members.back();
    }
    if (pf_batch_detach(b, c) != PF_OK) {   // still running: drop it from the list anyway
      std::lock_guard<std::mutex> lk(b->mu);
      b->members.pop_back();
      c->batch = nullptr;
    }
  }
  for (auto &kv : b->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (b->st) {
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->st);
    cudaStreamDestroy(b->st);
  }
  delete b;
}

}  // extern "C"
