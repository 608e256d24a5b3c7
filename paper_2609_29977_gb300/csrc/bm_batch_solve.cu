// Batched refinement-step kernels: one CTA per tail of every system
// (forward substitution with each system's root step in its last CTA,
// backward substitution with x += d, FP64 residual with each system's
// stopping test in its last CTA). See bm_batch.cu.
#include "bm_batch.cuh"

namespace bm {
namespace {
using namespace mx;

// Per-solve reset of the control blocks.
__global__ void k_batch_reset(BInst *inst, int ninst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ninst) return;
  IRCtl *c = inst[b].m.ctl;
  c->converged = 0;
  c->iters = 0;
  c->wmax = 0u;
  c->omega_prev = 0.0;
  inst[b].m.tickets[2] = 0u;
  inst[b].m.tickets[3] = 0u;
}

__global__ void __launch_bounds__(256) k_batch_fwd(const BInst *inst, const BTail *tails, const double *const *rp,
                                                   double *const *xp, int iter) {
  __shared__ __align__(16) float sbuf[256];
  __shared__ double sR[64 * 64 + 128];
  const BTail t = tails[blockIdx.x];
  const BInst &I = inst[t.inst];
  pdl_wait();
  if (ir_done(I.m.ctl)) return;
  const double *rhs = iter == 0 ? rp[t.inst] : I.m.rho;
  switch (I.nb) {
#define X(n)                                                              \
  case n:                                                                 \
    fwd_tail<n>(I.m, rhs, t.s, 0, 1, reinterpret_cast<float(*)[n]>(sbuf)); \
    if (last_cta(&I.m.tickets[2], (unsigned)I.S)) root_step<n>(I.m, rhs, xp[t.inst], iter, sR, I.S); \
    break;
    BM_BATCH_NB_LIST(X)
#undef X
  }
}

__global__ void __launch_bounds__(256) k_batch_bwd(const BInst *inst, const BTail *tails, double *const *xp,
                                                   int iter) {
  __shared__ __align__(16) float sbuf[256];
  const BTail t = tails[blockIdx.x];
  const BInst &I = inst[t.inst];
  pdl_wait();
  if (ir_done(I.m.ctl)) return;
  switch (I.nb) {
#define X(n)                                                                           \
  case n:                                                                              \
    bwd_tail<n>(I.m, xp[t.inst], iter, t.s, 0, 1, reinterpret_cast<float(*)[n]>(sbuf)); \
    break;
    BM_BATCH_NB_LIST(X)
#undef X
  }
}

__global__ void __launch_bounds__(256) k_batch_res(const BInst *inst, const BTail *tails, const double *const *rp,
                                                   double *const *xp, int iter, int max_iter, double tol) {
  const BTail t = tails[blockIdx.x];
  const BInst &I = inst[t.inst];
  pdl_wait();
  if (ir_done(I.m.ctl)) return;
  const double *r = rp[t.inst];
  const double *x = xp[t.inst];
  switch (I.nb) {
#define X(n)                                     \
  case n:                                        \
    residual_tail<n>(I.m, r, x, t.s);            \
    break;
    BM_BATCH_NB_LIST(X)
#undef X
  }
  if (last_cta(&I.m.tickets[3], (unsigned)I.S)) residual_finish(I.m, r, x, I.nb, iter, max_iter, tol);
}

}  // namespace

void batch_launch_reset(BInst *inst, int ninst, cudaStream_t st) {
  k_batch_reset<<<(ninst + 127) / 128, 128, 0, st>>>(inst, ninst);
}

void batch_launch_solve_iteration(const BInst *inst, const BTail *tails, int ntails, const double *const *r,
                                  double *const *x, int iter, int max_iter, double tol, cudaStream_t st) {
  launch_pdl(k_batch_fwd, (unsigned)ntails, 256, 0, st, inst, tails, r, x, iter);
  launch_pdl(k_batch_bwd, (unsigned)ntails, 256, 0, st, inst, tails, x, iter);
  launch_pdl(k_batch_res, (unsigned)ntails, 256, 0, st, inst, tails, r, x, iter, max_iter, tol);
}

}  // namespace bm
