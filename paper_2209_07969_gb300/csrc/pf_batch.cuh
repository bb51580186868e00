// Batched launches: one kernel launch runs the same stage for several simulations.
//
// A stage is a functor F whose operator()(bid, nblk) does the work of CTA bid of the nblk
// CTAs the stage takes for one simulation (the body the simulation's own launch runs with
// bid = blockIdx.x, nblk = gridDim.x).  A batched launch concatenates the CTA ranges of up
// to PF_MAXB simulations: CTA b belongs to the simulation s with start[s] <= b < start[s+1]
// and runs f[s](b - start[s], start[s+1] - start[s]).  Every simulation keeps its own block
// decomposition and its own reduction workspace, so its arithmetic, including the order of
// every reduction, is the same as in its own launch: a simulation gives bit-identical
// results alone and in a batch.  A simulation whose Krylov solve has stopped (done flag
// set by the loop condition) skips the launch.
#pragma once
#include "pf_internal.cuh"

namespace pf {

constexpr int PF_MAXB = 16;   // simulations per batched launch

template <class F>
struct BatchLaunch {
  int n;
  unsigned start[PF_MAXB + 1];
  const int *done[PF_MAXB];   // per-simulation stop flag, or nullptr
  F f[PF_MAXB];
};

#ifdef __CUDACC__
template <class F, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_batch(const __grid_constant__ BatchLaunch<F> b) {
  pdl_enter();
  const unsigned blk = blockIdx.x;
  int s = 0;
  while (s + 1 < b.n && blk >= b.start[s + 1]) ++s;
  if (b.done[s] && *(volatile const int *)b.done[s]) return;
  b.f[s](blk - b.start[s], b.start[s + 1] - b.start[s]);
}

// Host side: collect (functor, CTA count, stop flag) per simulation, then launch once.
template <class F, int THREADS, int MINB = 1>
struct Batcher {
  BatchLaunch<F> L;
  Batcher() { L.n = 0; L.start[0] = 0; }
  void add(const F &f, unsigned nblk, const int *done) {
    if (nblk == 0) return;
    L.f[L.n] = f;
    L.done[L.n] = done;
    L.start[L.n + 1] = L.start[L.n] + nblk;
    ++L.n;
  }
  int launch(cudaStream_t st) {
    if (L.n == 0) return 0;
    launch_pdl(k_batch<F, THREADS, MINB>, dim3(L.start[L.n]), dim3(THREADS), st, L);
    return 1;
  }
};
#endif

// One simulation's fine-level operands of a batched fused stage (pf_ops.cu).
template <class T>
struct ElasStageIn {
  GridD g;
  MatD m;
  const T *d;
  const uint8_t *tens;
  MgBufs<T> B;
  RedWs ws;
  int sr;     // strip rows per warp (0: the grid-size rule)
};
template <class T>
struct DamageStageIn {
  GridD g;
  const T *c;
  double kappa;
  MgBufs<T> B;
  RedWs ws;
};
// Fused stage `stage` for n simulations (n >= 1); returns the launches issued.
template <class T>
int elas_mg_stage_batch(int stage, int n, const ElasStageIn<T> *in, cudaStream_t st);
template <class T>
int damage_mg_stage_batch(int stage, int n, const DamageStageIn<T> *in, cudaStream_t st);
// Device-side loop condition of a batched Krylov solve (pf_vec.cu): every simulation whose
// solve has not stopped counts its iteration and stops on the test of the single solve;
// the loop continues while any has not stopped.
void krylov_while_batch(cudaGraphConditionalHandle h, int n, KrylovScal *const *sc,
                        cudaStream_t st);

}  // namespace pf
