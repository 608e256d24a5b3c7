// Device tables of the batched solver (bm_batch.cu, bm_batch_solve.cu).
#pragma once

#include "bm_mixed.cuh"

namespace bm {

struct BInst {
  int S, N, nb, nr, Lc;
  MixedState m;          // FP32 tail factor, FP64 root parts, solve vectors, control block
  unsigned *tail_done;   // [S] completed factor items per tail
  unsigned *x1_done;     // completed x_1 items of the system
};

struct BSeg {            // a run of items of one (system, level) in a class queue
  long start;
  int inst, level, count;
};

struct BClass {
  int nb, nseg;
  long nitems;
  const BSeg *segs;
  unsigned long long *head;
  int team_bytes;        // shared memory per team
};

struct BTail {
  int inst, s;
};

// Block sizes of the batched form (the batched workload draws nb from
// {6, 12, 24, 48}; 4 is kept for small test systems).
#define BM_BATCH_NB_LIST(X) X(4) X(6) X(12) X(24) X(48)

void batch_launch_solve_iteration(const BInst *inst, const BTail *tails, int ntails, const double *const *r,
                                  double *const *x, int iter, int max_iter, double tol, cudaStream_t st);
void batch_launch_reset(BInst *inst, int ninst, cudaStream_t st);

}  // namespace bm
