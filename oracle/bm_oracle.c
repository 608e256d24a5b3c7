/*
 * ORACLE -- test infrastructure only. Nothing in the product path links,
 * loads or calls this file; only tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.
 *
 * Plain FP64 direct solver for the root-coupled SPD system K dx = r of
 * Sec. III-B (Eq. root_coupled_matrix, Eq. tail_block_tridiagonal), written
 * as the textbook block Cholesky in the NATURAL variable order
 * (dx^1, ..., dx^M, dx_0): each tail forward in time, the root last. This is
 * the ordering of Fig. 2(a): eliminating stage k of a tail leaves a dense
 * root row, whose blocks Z_k = W_k L_kk^{-T} are carried along the tail
 * (W_1 = C_{i,1}, W_{k+1} = -Z_k L_{k+1,k}^T). It shares nothing with the
 * GPU library: different ordering, different loops, scalar code.
 *
 * Layouts (row-major, float64): D[S][N][nb][nb] (only the lower triangle is
 * read), E[S][N-1][nb][nb] with E[s][k] the block at (stage k+2, stage k+1),
 * C[S][nr][nb], R[nr][nr], r and x of length S*N*nb + nr in natural order.
 *
 * The per-tail loops run in parallel over scenarios (OpenMP); sums across
 * scenarios are taken in index order so the result does not depend on the
 * thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((size_t)(i) * (size_t)(ld) + (size_t)(j))

/* a := lower Cholesky factor of the symmetric matrix given by the lower
 * triangle of a (n x n); upper triangle set to zero. Returns 0, or j+1 when
 * the j-th pivot is not positive / not finite. */
static int chol_lower(double *a, int n) {
  for (int j = 0; j < n; ++j) {
    double d = a[IDX(j, j, n)];
    for (int k = 0; k < j; ++k) d -= a[IDX(j, k, n)] * a[IDX(j, k, n)];
    if (!(d > 0.0) || !isfinite(d)) return j + 1;
    double ljj = sqrt(d);
    a[IDX(j, j, n)] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = a[IDX(i, j, n)];
      for (int k = 0; k < j; ++k) s -= a[IDX(i, k, n)] * a[IDX(j, k, n)];
      a[IDX(i, j, n)] = s / ljj;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) a[IDX(i, j, n)] = 0.0;
  return 0;
}

/* X := B L^{-T} for B (m x n), L lower (n x n): solve X L^T = B row by row. */
static void right_trsm_lt(const double *L, int n, const double *B, double *X, int m) {
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < n; ++j) {
      double s = B[IDX(r, j, n)];
      for (int k = 0; k < j; ++k) s -= X[IDX(r, k, n)] * L[IDX(j, k, n)];
      X[IDX(r, j, n)] = s / L[IDX(j, j, n)];
    }
}

/* y := L^{-1} b (forward substitution). */
static void trsv_l(const double *L, int n, double *y) {
  for (int i = 0; i < n; ++i) {
    double s = y[i];
    for (int k = 0; k < i; ++k) s -= L[IDX(i, k, n)] * y[k];
    y[i] = s / L[IDX(i, i, n)];
  }
}

/* x := L^{-T} y (backward substitution). */
static void trsv_lt(const double *L, int n, double *x) {
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[IDX(k, i, n)] * x[k];
    x[i] = s / L[IDX(i, i, n)];
  }
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int bmo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Natural-order factorization.
 * Outputs: Ld[S][N][nb][nb] diagonal factor blocks L_kk (lower),
 *          Lsub[S][N-1][nb][nb] L_{k+1,k},
 *          Z[S][N][nr][nb] root-row blocks,
 *          LR[nr][nr] root factor, Rt[nr][nr] root Schur complement R - sum.
 * Returns 0; or -(1 + s*N + k) on a non-positive pivot at scenario s, stage
 * index k (0-based); or -(1 + S*N) for the root.
 */
long bmo_factor(int S, int N, int nb, int nr, const double *D, const double *E,
                const double *C, const double *R, double *Ld, double *Lsub, double *Z,
                double *LR, double *Rt, int nthreads) {
  set_threads(nthreads);
  const size_t bb = (size_t)nb * nb, rb = (size_t)nr * nb, rr = (size_t)nr * nr;
  double *Upart = (double *)calloc((size_t)S * rr, sizeof(double));
  long fail = 0;
  if (!Upart) return -(long)(1 + (long)S * N) - 1;
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < S; ++s) {
    double *W = (double *)malloc(rb * sizeof(double));
    double *Us = Upart + (size_t)s * rr;
    memcpy(W, C + (size_t)s * rb, rb * sizeof(double));
    for (int k = 0; k < N; ++k) {
      double *Lkk = Ld + ((size_t)s * N + k) * bb;
      /* Lkk := D_k - L_{k,k-1} L_{k,k-1}^T (lower part) */
      const double *Dk = D + ((size_t)s * N + k) * bb;
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j <= i; ++j) {
          double v = Dk[IDX(i, j, nb)];
          if (k > 0) {
            const double *P = Lsub + ((size_t)s * (N - 1) + (k - 1)) * bb;
            for (int t = 0; t < nb; ++t) v -= P[IDX(i, t, nb)] * P[IDX(j, t, nb)];
          }
          Lkk[IDX(i, j, nb)] = v;
        }
      int info = chol_lower(Lkk, nb);
      if (info) {
#pragma omp critical
        { if (fail == 0) fail = -(long)(1 + (long)s * N + k); }
        break;
      }
      /* root row block Z_k = W L_kk^{-T}; U_s += Z_k Z_k^T */
      double *Zk = Z + ((size_t)s * N + k) * rb;
      right_trsm_lt(Lkk, nb, W, Zk, nr);
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nr; ++j) {
          double v = 0.0;
          for (int t = 0; t < nb; ++t) v += Zk[IDX(i, t, nb)] * Zk[IDX(j, t, nb)];
          Us[IDX(i, j, nr)] += v;
        }
      if (k + 1 < N) {
        /* L_{k+1,k} = E_{k+1} L_kk^{-T}; the next root-row block W = -Z_k L_{k+1,k}^T */
        double *P = Lsub + ((size_t)s * (N - 1) + k) * bb;
        right_trsm_lt(Lkk, nb, E + ((size_t)s * (N - 1) + k) * bb, P, nb);
        for (int i = 0; i < nr; ++i)
          for (int j = 0; j < nb; ++j) {
            double v = 0.0;
            for (int t = 0; t < nb; ++t) v += Zk[IDX(i, t, nb)] * P[IDX(j, t, nb)];
            W[IDX(i, j, nb)] = -v;
          }
      }
    }
    free(W);
  }
  if (fail) { free(Upart); return fail; }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nr; ++j) {
      double v = R[IDX(i >= j ? i : j, i >= j ? j : i, nr)];
      for (int s = 0; s < S; ++s) v -= Upart[(size_t)s * rr + IDX(i, j, nr)];
      Rt[IDX(i, j, nr)] = v;
      LR[IDX(i, j, nr)] = v;
    }
  free(Upart);
  if (chol_lower(LR, nr)) return -(long)(1 + (long)S * N);
  return 0;
}

/* Solve with the natural-order factor: forward tails, root, backward tails. */
void bmo_solve(int S, int N, int nb, int nr, const double *Ld, const double *Lsub,
               const double *Z, const double *LR, const double *r, double *x, int nthreads) {
  set_threads(nthreads);
  const size_t bb = (size_t)nb * nb, rb = (size_t)nr * nb;
  const size_t nt = (size_t)N * nb, n0 = (size_t)S * nt;
  double *t = (double *)calloc((size_t)S * nr, sizeof(double));
  memcpy(x, r, (n0 + nr) * sizeof(double));
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < S; ++s) {
    double *y = x + (size_t)s * nt;
    double *ts = t + (size_t)s * nr;
    for (int k = 0; k < N; ++k) {
      double *yk = y + (size_t)k * nb;
      if (k > 0) {
        const double *P = Lsub + ((size_t)s * (N - 1) + (k - 1)) * bb;
        const double *yp = y + (size_t)(k - 1) * nb;
        for (int i = 0; i < nb; ++i) {
          double v = 0.0;
          for (int j = 0; j < nb; ++j) v += P[IDX(i, j, nb)] * yp[j];
          yk[i] -= v;
        }
      }
      trsv_l(Ld + ((size_t)s * N + k) * bb, nb, yk);
      const double *Zk = Z + ((size_t)s * N + k) * rb;
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nb; ++j) ts[i] += Zk[IDX(i, j, nb)] * yk[j];
    }
  }
  double *x0 = x + n0;
  for (int i = 0; i < nr; ++i)
    for (int s = 0; s < S; ++s) x0[i] -= t[(size_t)s * nr + i];
  trsv_l(LR, nr, x0);
  trsv_lt(LR, nr, x0);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < S; ++s) {
    double *y = x + (size_t)s * nt;
    for (int k = N - 1; k >= 0; --k) {
      double *yk = y + (size_t)k * nb;
      const double *Zk = Z + ((size_t)s * N + k) * rb;
      for (int j = 0; j < nb; ++j) {
        double v = 0.0;
        for (int i = 0; i < nr; ++i) v += Zk[IDX(i, j, nb)] * x0[i];
        yk[j] -= v;
      }
      if (k + 1 < N) {
        const double *P = Lsub + ((size_t)s * (N - 1) + k) * bb;
        const double *xn = y + (size_t)(k + 1) * nb;
        for (int j = 0; j < nb; ++j) {
          double v = 0.0;
          for (int i = 0; i < nb; ++i) v += P[IDX(i, j, nb)] * xn[i];
          yk[j] -= v;
        }
      }
      trsv_lt(Ld + ((size_t)s * N + k) * bb, nb, yk);
    }
  }
  free(t);
}

/*
 * rho := r - K x in FP64 from the blocks (lower triangles of D, R read and
 * mirrored). Also returns the norms needed for the normwise backward error
 * eta = ||rho||_inf / (||K||_inf ||x||_inf + ||r||_inf):
 * out[0] = ||rho||_inf, out[1] = ||K||_inf, out[2] = ||x||_inf,
 * out[3] = ||r||_inf, out[4] = ||rho||_2, out[5] = ||r||_2.
 */
void bmo_residual(int S, int N, int nb, int nr, const double *D, const double *E,
                  const double *C, const double *R, const double *x, const double *r,
                  double *rho, double *out, int nthreads) {
  set_threads(nthreads);
  const size_t bb = (size_t)nb * nb, rb = (size_t)nr * nb;
  const size_t nt = (size_t)N * nb, n0 = (size_t)S * nt;
  const double *x0 = x + n0;
  double *rowsum = (double *)calloc(n0 + nr, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int s = 0; s < S; ++s) {
    for (int k = 0; k < N; ++k) {
      const double *Dk = D + ((size_t)s * N + k) * bb;
      const double *xk = x + (size_t)s * nt + (size_t)k * nb;
      for (int i = 0; i < nb; ++i) {
        size_t gi = (size_t)s * nt + (size_t)k * nb + i;
        double v = r[gi], a = 0.0;
        for (int j = 0; j < nb; ++j) {
          double kij = (j <= i) ? Dk[IDX(i, j, nb)] : Dk[IDX(j, i, nb)];
          v -= kij * xk[j];
          a += fabs(kij);
        }
        if (k > 0) { /* block (k, k-1) = E_k (paper, 1-based k) */
          const double *Ek = E + ((size_t)s * (N - 1) + (k - 1)) * bb;
          const double *xp = xk - nb;
          for (int j = 0; j < nb; ++j) { v -= Ek[IDX(i, j, nb)] * xp[j]; a += fabs(Ek[IDX(i, j, nb)]); }
        }
        if (k + 1 < N) { /* block (k, k+1) = E_{k+1}^T */
          const double *Ek = E + ((size_t)s * (N - 1) + k) * bb;
          const double *xn = xk + nb;
          for (int j = 0; j < nb; ++j) { v -= Ek[IDX(j, i, nb)] * xn[j]; a += fabs(Ek[IDX(j, i, nb)]); }
        }
        if (k == 0) { /* block (1, root) = C^T */
          const double *Cs = C + (size_t)s * rb;
          for (int j = 0; j < nr; ++j) { v -= Cs[IDX(j, i, nb)] * x0[j]; a += fabs(Cs[IDX(j, i, nb)]); }
        }
        rho[gi] = v;
        rowsum[gi] = a;
      }
    }
  }
  for (int i = 0; i < nr; ++i) {
    double v = r[n0 + i], a = 0.0;
    for (int j = 0; j < nr; ++j) {
      double kij = (j <= i) ? R[IDX(i, j, nr)] : R[IDX(j, i, nr)];
      v -= kij * x0[j];
      a += fabs(kij);
    }
    for (int s = 0; s < S; ++s) {
      const double *Cs = C + (size_t)s * rb;
      const double *x1 = x + (size_t)s * nt;
      for (int j = 0; j < nb; ++j) { v -= Cs[IDX(i, j, nb)] * x1[j]; a += fabs(Cs[IDX(i, j, nb)]); }
    }
    rho[n0 + i] = v;
    rowsum[n0 + i] = a;
  }
  double rn = 0, kn = 0, xn = 0, bn = 0, r2 = 0, b2 = 0;
  for (size_t i = 0; i < n0 + nr; ++i) {
    rn = fmax(rn, fabs(rho[i]));
    kn = fmax(kn, rowsum[i]);
    xn = fmax(xn, fabs(x[i]));
    bn = fmax(bn, fabs(r[i]));
    r2 += rho[i] * rho[i];
    b2 += r[i] * r[i];
  }
  out[0] = rn; out[1] = kn; out[2] = xn; out[3] = bn; out[4] = sqrt(r2); out[5] = sqrt(b2);
  free(rowsum);
}

/*
 * Schur complement of each tail onto its first stage, by eliminating the
 * stages N, N-1, ..., 2 in that order (the reversed order of Fig. 2(b)):
 * S_N = D_N, S_k = D_k - E_k^T S_{k+1}^{-1} E_k, evaluated through the
 * Cholesky factor of S_{k+1}. Out: S1[S][nb][nb] (full symmetric).
 * Returns 0 or -(1 + s*N + k) on a non-positive pivot.
 */
long bmo_tail_schur_first(int S, int N, int nb, const double *D, const double *E, double *S1,
                          int nthreads) {
  set_threads(nthreads);
  const size_t bb = (size_t)nb * nb;
  long fail = 0;
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < S; ++s) {
    double *Sk = (double *)malloc(bb * sizeof(double));
    double *G = (double *)malloc(bb * sizeof(double));
    const double *Dn = D + ((size_t)s * N + (N - 1)) * bb;
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) Sk[IDX(i, j, nb)] = (j <= i) ? Dn[IDX(i, j, nb)] : Dn[IDX(j, i, nb)];
    for (int k = N - 2; k >= 0; --k) {
      /* S_k = D_k - G^T G with G = L_{k+1}^{-1} E_k, L_{k+1} = chol(S_{k+1}) */
      if (chol_lower(Sk, nb)) {
#pragma omp critical
        { if (fail == 0) fail = -(long)(1 + (long)s * N + k + 1); }
        break;
      }
      const double *Ek = E + ((size_t)s * (N - 1) + k) * bb;
      for (int c = 0; c < nb; ++c) {
        double col[256];
        for (int i = 0; i < nb; ++i) col[i] = Ek[IDX(i, c, nb)];
        trsv_l(Sk, nb, col);
        for (int i = 0; i < nb; ++i) G[IDX(i, c, nb)] = col[i];
      }
      const double *Dk = D + ((size_t)s * N + k) * bb;
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
          double v = (j <= i) ? Dk[IDX(i, j, nb)] : Dk[IDX(j, i, nb)];
          for (int t = 0; t < nb; ++t) v -= G[IDX(t, i, nb)] * G[IDX(t, j, nb)];
          Sk[IDX(i, j, nb)] = v;
        }
    }
    memcpy(S1 + (size_t)s * bb, Sk, bb * sizeof(double));
    free(Sk);
    free(G);
  }
  return fail;
}
