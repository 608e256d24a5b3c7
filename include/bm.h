/*
 * bm.h -- C ABI of the GB300 branch-MPC direct solver.
 *
 * The solver factors and solves the SPD root-coupled system K dx = r of
 * Sec. III-B (Eq. root_coupled_matrix): S scenario tails K_i, each
 * block-tridiagonal over N stages with nb x nb blocks
 * (Eq. tail_block_tridiagonal), coupled to one shared root block R (nr x nr)
 * through a single block C_{i,1} on the first stage of every tail.
 *
 * The factorization is the two-level parallel Cholesky of Alg. 1 under the
 * tail permutation Pi_i = blkdiag(Gamma_{N-1}, I) Omega_i of Sec. IV-A, and
 * the solve is the two-level parallel forward/backward substitution of
 * Alg. 2. Everything runs in CUDA kernels on the device; there is no CPU
 * fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All matrix/vector pointers are DEVICE pointers unless the name says
 *   host, row-major, contiguous, float64, 16-byte aligned (cudaMalloc and
 *   torch allocations satisfy this).
 * - D[S][N][nb][nb]: stage blocks D_{i,k}; only the lower triangle is read.
 * - E[S][N-1][nb][nb]: E[s][k] is the paper's E_{s,k+1}, the block at
 *   (stage k+2, stage k+1) in 1-based stages (below the diagonal). For N = 1
 *   the pointer may be NULL.
 * - C[S][nr][nb]: the coupling blocks C_{i,1}; R[nr][nr]: the root block
 *   (lower triangle read).
 * - r, x[S*N*nb + nr]: natural order (dx^1, ..., dx^S, dx_0), each tail
 *   dx^i = (dx^i_1, ..., dx^i_N) (Sec. III-B).
 * - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *   default stream. Every call that launches work is asynchronous with
 *   respect to the host and ordered on that stream. Calls on one handle must
 *   be ordered (one stream, or external synchronization): the handle's
 *   workspaces are shared by its calls.
 * - Argument errors are returned synchronously. Errors found on the device
 *   (a non-positive pivot, refinement that did not converge) are recorded in
 *   a sticky status word of the handle, reset by every bm_factor, and
 *   returned by bm_query.
 */
#ifndef BM_H
#define BM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BM_VERSION 1

typedef struct bm_handle_s *bm_handle;

typedef enum {
  BM_OK = 0,
  BM_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, misaligned pointer */
  BM_ERR_NOT_SPD = 2,       /* a pivot was not positive and finite */
  BM_ERR_OOM = 3,           /* device allocation failed in bm_analyze */
  BM_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  BM_ERR_NOT_CONVERGED = 5, /* mixed precision: refinement missed tol */
  BM_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  BM_ERR_NOT_FACTORED = 7   /* bm_solve before any bm_factor */
} bm_status;

typedef enum {
  BM_PREC_FP64 = 0,    /* factor and solve in FP64 */
  BM_PREC_FP32_IR = 1  /* FP32 tails, FP64 root and FP64 refinement */
} bm_precision;

/* bm_desc.flags */
#define BM_FLAG_NO_GRAPH 1u /* launch kernels directly instead of replaying captured CUDA graphs */
/*
 * BM_PREC_FP32_IR only: how the root Schur complement R~ = R - sum_i U_i is
 * formed (Alg. 1 steps 3-4). By default (neither flag) the factor first
 * forms it from the FP32 tail factor. When that Cholesky fails, or the
 * cancellation gamma = max_j R_jj / R~_jj times the FP32 factor's pivot
 * spread rho = max over tails of (max_j L_jj / min_j L_jj)^2 times 2^-24
 * exceeds 16 (the FP32-based R~ then has no correct digit to spare), it
 * refines each tail's coupling columns X_i = K_i^{-1} C_i^T (the nr columns
 * through which the tail meets the root) with the FP32 factor and one
 * float-float residual, forms U_i = C_{i,1} X_i from them, refactors the
 * root, and the solves then use X_i for the root coupling. That indicator
 * is a heuristic: when a bm_solve's refinement without refined columns
 * ends BM_ERR_NOT_CONVERGED (stalled or out of steps), the same bm_solve
 * refines them then, refactors the root, and resumes the refinement from
 * its last residual with up to max_refine more corrections; later solves on
 * that factor use the refined columns from the start. The flags force one
 * choice (and no resumption). Setting both is BM_ERR_INVALID_ARG.
 */
#define BM_FLAG_COUPLING_REFINE 2u /* always refine the coupling columns */
#define BM_FLAG_COUPLING_FP32 4u   /* never: R~ from the FP32 tail factor alone */
/* BM_PREC_FP64: keep the default launch schedule of the tail factor instead
 * of autotuning it on the first bm_factor (see bm_schedule) */
#define BM_FLAG_NO_TUNE 8u
/* BM_PREC_FP32_IR: compute every refinement residual with FP64 arithmetic,
 * never in float-float (see bm_solve) */
#define BM_FLAG_RESIDUAL_FP64 16u

typedef struct {
  int S, N, nb, nr;   /* scenarios (the paper's M), horizon, stage block, root block */
  int precision;      /* bm_precision */
  int max_refine;     /* BM_PREC_FP32_IR: maximum refinement steps (<= 0: 10) */
  double tol;         /* BM_PREC_FP32_IR: target componentwise backward error (<= 0: 1e-10), see bm_solve */
  unsigned flags;     /* BM_FLAG_* */
} bm_desc;

typedef struct {
  int status;          /* sticky bm_status of the last bm_factor / bm_solve */
  int fail_scenario;   /* BM_ERR_NOT_SPD: 0-based scenario, -1 for the root */
  int fail_stage;      /* BM_ERR_NOT_SPD: 1-based stage k of that tail, 0 for the root */
  int iters;           /* BM_PREC_FP32_IR: refinement steps of the last solve */
  double backward_error; /* BM_PREC_FP32_IR: componentwise backward error of the returned x; FP64: -1 */
  int coupling_refined;  /* BM_PREC_FP32_IR: 1 if the coupling columns of the last bm_factor are refined
                            (by that factor, or by a later bm_solve that resumed its refinement) */
  int residual_float_float; /* BM_PREC_FP32_IR: 1 if the refinement residuals of the last bm_solve were
                               float-float, 0 if FP64 (see bm_solve) */
  int host_pipelined;  /* BM_PREC_FP64: 1 if the last bm_factor_solve_host overlapped its input copies
                          with the factor (see bm_factor_solve_host), else 0 */
} bm_info;

/* Library version (BM_VERSION). */
int bm_version(void);

/* Static string for a status code. */
const char *bm_status_string(bm_status s);

/*
 * Device bytes that bm_analyze allocates for desc (factors and workspaces),
 * or 0 for an invalid desc. The one-time analysis phase of Sec. V (fixed
 * sparsity: persistent workspaces planned once).
 */
size_t bm_workspace_bytes(const bm_desc *desc);

/*
 * One-time analysis (Sec. V): validates desc (S, N, nb, nr >= 1; nb, nr <= 64;
 * S <= 65535), plans the odd-even levels of Gamma_{N-1} (Sec. II), and
 * allocates the handle's device memory on the current device. Kernels are
 * captured into CUDA graphs lazily by the first bm_factor / bm_solve with
 * a given set of pointers. On success *out owns all of it until bm_destroy.
 * Errors: BM_ERR_INVALID_ARG, BM_ERR_OOM, BM_ERR_CUDA.
 */
bm_status bm_analyze(const bm_desc *desc, void *stream, bm_handle *out);

/*
 * Numeric factorization, Alg. 1 (steps 1-5): per tail the Cholesky factor
 * L_i of Pi_i K_i Pi_i^T (horizon-parallel, Sec. IV-B), the coupling solve
 * F_{i,1} = C_{i,1} L_{i,1}^{-T} (Theorem 1), the local Schur update
 * U_i = F_{i,1} F_{i,1}^T, the root reduction R~ = R - sum_i U_i (FP64,
 * fixed summation order) and L_R = chol(R~). Reads D, E, C, R (device);
 * the handle owns the factor. Asynchronous. In BM_PREC_FP32_IR mode D, E,
 * C, R must stay valid and unchanged until the next bm_factor or
 * bm_destroy (the refinement residual reads them).
 * Device-side failures (non-positive pivot) go to the sticky status.
 */
bm_status bm_factor(bm_handle h, const double *D, const double *E, const double *C,
                    const double *R, void *stream);

/*
 * Triangular solves, Alg. 2: tail forward substitution (Pi_i r^i, L_i^{-1}),
 * root reduction r~_0 = r_0 - sum_i F_{i,1} dy^i_1, root forward/backward
 * substitution with L_R, root propagation dy^i_1 -= F_{i,1}^T dx_0, tail
 * backward substitution and the inverse permutation. r and x are device
 * vectors of length S*N*nb + nr in natural order; x must not alias r.
 * BM_PREC_FP32_IR: iterative refinement on K with an FP64-accurate
 * residual until the componentwise backward error
 *     omega = max_i |r - K x|_i / (|K| |x| + |r|)_i     (Oettli-Prager)
 * is <= tol. The residual r - K x is computed with FP64 arithmetic, or,
 * when tol >= 1e-11 and BM_FLAG_RESIDUAL_FP64 is not set, in float-float
 * on the FP32 pipe: K and x split into hi + lo floats (K once per
 * bm_factor), exact products (Dekker's TwoProduct), Knuth's TwoSum for the
 * running sum, FP64 accumulation of every 8 terms. Its error is at most
 * beta = 4e-12 times (|K| |x|)_i, and the stopping test is then
 * omega <= tol - beta, so the returned x still has omega <= tol. A system
 * with a nonzero entry of K or x outside 2^-50..2^50 in magnitude falls
 * back to FP64 residuals (bm_info.residual_float_float says which ran).
 * It reports BM_ERR_NOT_CONVERGED (x = the last iterate) after
 * max_refine corrections, or earlier once omega fails to halve from one
 * correction to the next (stalled or diverging refinement). In the captured
 * graph the refinement iterations are a conditional loop that ends on the
 * device after the last iteration that runs; with BM_FLAG_NO_GRAPH the
 * max_refine + 1 iterations are launched and those after the stopping test
 * return at once. Both give bitwise the same x. Asynchronous.
 * Errors: BM_ERR_INVALID_ARG, BM_ERR_NOT_FACTORED, BM_ERR_CUDA.
 */
bm_status bm_solve(bm_handle h, const double *r, double *x, void *stream);

/*
 * BM_PREC_FP32_IR: rho = r - K x for the K of the last bm_factor, with the
 * arithmetic of the handle's refinement residual (float-float or FP64, see
 * bm_solve). r, x, rho: device vectors of length S*N*nb + nr in natural
 * order; rho must alias neither. Overwrites the handle's split copy of the
 * refinement iterate (the next bm_solve makes its own). Asynchronous.
 * Errors: BM_ERR_INVALID_ARG (also for BM_PREC_FP64 handles),
 * BM_ERR_NOT_FACTORED, BM_ERR_CUDA.
 */
bm_status bm_residual(bm_handle h, const double *r, const double *x, double *rho, void *stream);

/*
 * Launch schedule of the FP64 factor (not in the paper; the factor's
 * arithmetic does not depend on it): *top_level = the first odd-even level
 * of Gamma_{N-1} handled by the per-tail kernel (one CTA per tail, the
 * levels separated by block barriers; the levels before it run as grid-wide
 * launches over all tails), team_per_level[l] (32 entries, may be NULL) =
 * the lanes that process one chain position in the grid-wide launch of
 * level l (0 from top_level on). The first bm_factor of a handle takes the
 * schedule from the autotune cache (file $BM_AUTOTUNE_CACHE, else
 * ~/.cache/branch_mpc_gb300_autotune.json; key: GPU name and S, N, nb, nr)
 * or, if absent, times every compiled team size per level and top levels one
 * below and above the default on its inputs (synchronizing the stream) and
 * stores the fastest; with BM_FLAG_NO_TUNE or BM_FLAG_NO_GRAPH the default
 * rule is kept (about two warps' worth of lanes per SM sub-partition per
 * level; the first level with at most four positions per tail starts the
 * per-tail kernel). *source: 1 from the cache, 0 tuned by this handle,
 * -1 the default rule.
 * Errors: BM_ERR_NOT_FACTORED before the first bm_factor; BM_ERR_INVALID_ARG
 * for mixed-precision handles and block sizes without compiled tail kernels.
 */
bm_status bm_schedule(bm_handle h, int *top_level, int *team_per_level, int *source);

/*
 * Synchronizes stream, then reports the sticky device status of the last
 * bm_factor / bm_solve in *info (may be NULL) and returns it.
 */
bm_status bm_query(bm_handle h, void *stream, bm_info *info);

/*
 * Copies the factor of the last bm_factor into caller device buffers
 * (each may be NULL to skip). Layout, by natural 1-based stage k of tail s
 * (index [s][k-1]), with chain position p = N+1-k and level l = ctz(p) of
 * Gamma_{N-1} for k >= 2:
 *   Ld[S][N][nb][nb]: diagonal block L_pp of L_i (lower; k = 1: L_{i,1});
 *   Ll[S][N][nb][nb]: the block of L_i in row p - 2^l, column p (zero if
 *                     p <= 2^l, and for k = 1);
 *   Lr[S][N][nb][nb]: the block in row p + 2^l (or row x_1 when
 *                     p + 2^l > N-1), column p (zero for k = 1);
 *   F[S][nr][nb]: F_{i,1};  LR[nr][nr]: L_R (lower).
 * In BM_PREC_FP32_IR mode the FP32 tail factor is widened to FP64.
 * Asynchronous on stream.
 */
bm_status bm_export_factor(bm_handle h, double *Ld, double *Ll, double *Lr, double *F,
                           double *LR, void *stream);

/*
 * End-to-end convenience for callers whose data live in HOST memory:
 * copies hD, hE, hC, hR, hr to device buffers owned by the handle
 * (allocated on first use), runs bm_factor and bm_solve, copies x back to
 * hx, and synchronizes stream before returning (hx is valid on return).
 * Pinned (page-locked) host buffers give asynchronous copies. For
 * BM_PREC_FP64 handles whose nb has compiled tail kernels, with page-locked
 * inputs and S >= 2, every call after the first (which chooses the launch
 * schedule) overlaps the copies with the factor: the tails' blocks move in
 * up to 8 chunks on a second stream, and the first odd-even level of Alg. 1
 * step 1 runs on each chunk as soon as it has arrived (the tails are
 * independent until the root reduction); the other levels, the root step
 * and the solve follow once all inputs are on the device. The result is
 * bitwise that of bm_factor + bm_solve on the same data; bm_info reports
 * which form ran. Returns the sticky device status like bm_query.
 */
bm_status bm_factor_solve_host(bm_handle h, const double *hD, const double *hE,
                               const double *hC, const double *hR, const double *hr,
                               double *hx, void *stream);

/*
 * Size of the library's fixed device scratch array used by
 * bm_factor_solve_noalloc (32 MiB). Every GPU that loads the library holds
 * this much device memory until the process exits.
 */
#define BM_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * FP64 factor + solve that allocates nothing. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc (code
 * running inside an allocator or memory-pool callback, real-time loops that
 * forbid allocation after start-up, hosts that give the library a fixed
 * device-memory budget). Instead of handle-owned memory it keeps the
 * factor and all workspaces of the system in one fixed device array of
 * BM_NOALLOC_SCRATCH_BYTES that the library defines; it calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   - Inputs D, E, C, R, r and the output x are device pointers with the
 *     layouts above; x must not alias r. Result: the same x as bm_analyze +
 *     bm_factor + bm_solve in BM_PREC_FP64.
 *   - Systems whose factor and workspaces need more than the array holds
 *     (about 5 S N nb^2 doubles; e.g. S = N = 64 with nb = 12 fits) are
 *     rejected with BM_ERR_INVALID_ARG before any work, as are the size
 *     limits of bm_analyze.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and keeps it.
 *   - The work is ordered on stream; the call then synchronizes stream and
 *     returns the device status (BM_ERR_NOT_SPD on a non-positive pivot).
 *     It is synchronous and cannot be recorded into a CUDA graph: on a
 *     stream that is being captured it returns BM_ERR_INVALID_ARG without
 *     launching anything.
 *   - All calls share the one array, which keeps the last call's contents:
 *     two calls whose work overlaps on the GPU (different streams or host
 *     threads) race on it and must be serialized by the caller.
 */
bm_status bm_factor_solve_noalloc(int S, int N, int nb, int nr, const double *D, const double *E,
                                  const double *C, const double *R, const double *r, double *x,
                                  void *stream);

/*
 * Rounds n FP64 values to FP32, to nearest with ties to even, using the same
 * integer-instruction rounding that the BM_PREC_FP32_IR path applies to the
 * FP64 input blocks as it loads them (the hardware conversion instruction
 * runs on the FP64 pipe of this GPU). src, dst: device arrays of n
 * elements. Asynchronous on stream. The paper has no counterpart; it is
 * exposed so that the rounding can be checked against the hardware's.
 */
bm_status bm_round_to_fp32(const double *src, float *dst, size_t n, void *stream);

/* ---------------------------------------------------------------------------
 * Assembly front end (App. A, "Linear System Sparsity in IPM and ADMM"):
 * forms the reduced SPD matrix of a branch-MPC QP,
 *     K = P + tau I + delta^{-1} A^T A + G^T (W + delta I)^{-1} G,
 * the matrix left after eliminating the equality and inequality multipliers
 * from the regularized KKT matrix of an interior point method (Eq.
 * appendix_ipm_kkt; ADMM's Eq. appendix_admm_kkt has the same form with
 * tau = sigma, delta = 1/rho and W = 0), directly in the D, E, C, R layout
 * of bm_factor (nb = nx + nu, nr = nu).
 *
 * Stage k = 1..N of a scenario holds z_k = (x_k, u_k) (u_N pads the last
 * stage); the root is the first input u_0; the initial state is fixed. The
 * equality rows are x_1 - B_0 u_0 = A_0 x_init and
 * x_{k+1} - A_k x_k - B_k u_k = 0 (k = 1..N-1); G = I (bounds on every
 * variable). All arrays are DEVICE, row-major float64:
 *   A[S][N][nx][nx], B[S][N][nx][nu]  A_k, B_k at index k (A_0 is not read),
 *   q[S][N][nx], rw[S][N][nu]         diagonal costs of x_k and u_k (index k-1),
 *   r0w[nu]                           diagonal cost of u_0,
 *   w[S][N][nx+nu], w0[nu]            the positive diagonal W (one entry per
 *                                     variable, same order).
 * Outputs D, E, C, R (full symmetric D and R) are overwritten. Asynchronous
 * on stream. Errors: BM_ERR_INVALID_ARG (sizes, tau < 0, delta <= 0, NULL),
 * BM_ERR_CUDA. The paper has no kernel for this step; its formula is App. A's.
 * ------------------------------------------------------------------------- */
typedef struct {
  int S, N, nx, nu;   /* scenarios, horizon, state and input sizes (nx + nu <= 64) */
  double tau, delta;  /* regularizations (tau >= 0, delta > 0) */
} bm_qp_desc;

bm_status bm_assemble_reduced(const bm_qp_desc *d, const double *A, const double *B, const double *q,
                              const double *rw, const double *r0w, const double *w, const double *w0,
                              double *D, double *E, double *C, double *R, void *stream);

/* ---------------------------------------------------------------------------
 * Batched form: many independent systems of uneven S, N, nb (and nr) in one
 * object, solved with the mixed-precision method (FP32 tails, FP64 root,
 * FP64 iterative refinement). Not in the paper; every system is the one of
 * Sec. III-B and is factored and solved as in bm_factor / bm_solve.
 * ------------------------------------------------------------------------- */
typedef struct bm_batch_s *bm_batch;

/* Device bytes bm_batch_analyze allocates, or 0 if a desc is invalid
 * (precision must be BM_PREC_FP32_IR; nb in {4, 6, 12, 24, 48};
 * nr <= 64; S <= 65535). */
size_t bm_batch_workspace_bytes(const bm_desc *descs, int count);

/*
 * One-time analysis of a batch of count systems: builds the work queues of
 * the persistent factor launch (one per block size, items ordered by the
 * odd-even levels of Gamma_{N-1}, Sec. II) and allocates all factors and
 * workspaces. max_refine and tol are taken from descs[0].
 * Errors: BM_ERR_INVALID_ARG, BM_ERR_OOM, BM_ERR_CUDA.
 */
bm_status bm_batch_analyze(const bm_desc *descs, int count, void *stream, bm_batch *out);

/*
 * Factors every system of the batch (Alg. 1) in one persistent launch.
 * D, E, C, R are DEVICE arrays of count device pointers (layouts as for
 * bm_factor; E[b] may be NULL when N_b = 1); the pointed-to inputs must stay
 * valid until the next bm_batch_factor (the refinement reads them). The
 * first call on a handle autotunes the launch shape (threads per CTA, CTAs
 * per SM) by timing candidates on these inputs, synchronizing the stream,
 * unless a cached choice for the same batch signature and GPU exists
 * (cache file: $BM_AUTOTUNE_CACHE, else ~/.cache/branch_mpc_gb300_autotune.json).
 * Asynchronous afterwards. Device failures go to each system's status.
 */
bm_status bm_batch_factor(bm_batch b, const double *const *D, const double *const *E, const double *const *C,
                          const double *const *R, void *stream);

/*
 * Solves every system (Alg. 2 with FP32 tails and an FP64 root step, then
 * FP64 refinement until each system's componentwise backward error <= tol,
 * as for bm_solve); r and x are
 * DEVICE arrays of count device pointers. Asynchronous.
 */
bm_status bm_batch_solve(bm_batch b, const double *const *r, double *const *x, void *stream);

/* Synchronizes stream; fills infos[count] (may be NULL); returns the first
 * non-OK system status, or BM_OK. */
bm_status bm_batch_query(bm_batch b, void *stream, bm_info *infos);

/* The launch shape chosen by the autotuner (BM_ERR_NOT_FACTORED before the
 * first bm_batch_factor); *from_cache = 1 when it came from the cache. */
bm_status bm_batch_schedule(bm_batch b, int *threads_per_cta, int *ctas_per_sm, int *from_cache);

/* Frees everything the batch owns. */
void bm_batch_destroy(bm_batch b);

/*
 * Test entry of the bounded device wait that the batched factor uses (the
 * paper has no counterpart): one warp waits, with that same wait, on a
 * counter that nothing increments; the wait gives up after limit_cycles SM
 * clock cycles (1 .. 2^33) and records BM_ERR_TIMEOUT, which this call
 * returns after synchronizing stream. Any other return value means the wait
 * did not behave. Allocates and frees 256 bytes of device memory.
 */
bm_status bm_test_bounded_wait(unsigned long long limit_cycles, void *stream);

/* Frees everything the handle owns (synchronizes its internal stream). */
void bm_destroy(bm_handle h);

/* ---------------------------------------------------------------------------
 * Serving runtime: a request loop that admits independent branch-MPC solves
 * by device memory, runs each admitted request (one factor of Alg. 1, then
 * nrhs solves of Alg. 2 against the resident factor) on its own stream slot
 * so that the work of requests admitted at different times overlaps on the
 * GPU, and reports per-request latency. Not in the paper: the paper solves
 * one system at a time. A request is computed exactly as bm_factor /
 * bm_solve compute it alone (same kernels, same launch shapes, which depend
 * only on the request's shape), so its result does not depend on what else
 * is in flight.
 *
 * Admission is first-in first-out: the request at the head of the queue is
 * admitted as soon as a slot is free and a contiguous range of the server's
 * device arena (hbm_budget bytes, allocated once at creation) can hold
 * bm_server_request_bytes of it; requests behind a blocked head wait.
 * Memory and slot are released when the request's last copy has finished.
 * A server is driven by one host thread (no internal threads); every call
 * below advances it without blocking on the device unless it says so.
 * ------------------------------------------------------------------------- */
typedef struct bm_server_s *bm_server;

#define BM_SERVE_MAX_RHS 8
#define BM_SERVE_MAX_SLOTS 64

/* D, E, C, R, r are HOST pointers (page-locked memory recommended, else the
 * copies serialize the host), x a host output buffer; the server stages
 * them through its arena and copies x back before the request completes. */
#define BM_REQ_HOST_IO 1

/* bm_server_desc.flags: a BM_PREC_FP32_IR request whose factor or
 * refinement fails (BM_ERR_NOT_SPD or BM_ERR_NOT_CONVERGED: the FP32 tail
 * factor cannot resolve the system, e.g. when R - sum_i U_i cancels by more
 * than FP32 tails can carry) is run again with BM_PREC_FP64, ahead of the
 * queue, if its FP64 workspace fits the budget. The completion then reports
 * the FP64 run's status and fallback = 1. */
#define BM_SERVE_FP64_FALLBACK 1

typedef struct {
  size_t hbm_budget; /* bytes of device memory for admitted requests (> 0) */
  int slots;         /* requests in flight at most, 1..BM_SERVE_MAX_SLOTS; one stream each */
  int precision;     /* bm_precision, for every request of the server */
  int max_refine;    /* as bm_desc.max_refine (mixed precision) */
  int flags;         /* 0 or BM_SERVE_FP64_FALLBACK */
  double tol;        /* as bm_desc.tol */
} bm_server_desc;

typedef struct {
  unsigned long long id; /* caller's tag, returned in the completion */
  int S, N, nb, nr;      /* system shape, limits as in bm_desc */
  int nrhs;              /* right-hand sides solved against the factor, 1..BM_SERVE_MAX_RHS */
  int flags;             /* 0 or BM_REQ_HOST_IO */
  const double *D, *E, *C, *R; /* layouts as for bm_factor; E may be NULL when N = 1 */
  const double *r;       /* nrhs right-hand sides of n = S*N*nb + nr values, back to back */
  double *x;             /* nrhs solutions, same layout (must not overlap r) */
} bm_request;

typedef struct {
  unsigned long long id;
  int status;            /* first non-OK status over factor and solves (bm_status) */
  int fail_scenario;     /* as bm_info, for BM_ERR_NOT_SPD */
  int fail_stage;
  int fallback;          /* 1 if the result comes from the FP64 re-run (BM_SERVE_FP64_FALLBACK) */
  int iters[BM_SERVE_MAX_RHS];           /* refinement steps per right-hand side */
  double backward_error[BM_SERVE_MAX_RHS]; /* componentwise, per rhs (mixed; -1 for FP64) */
  /* microseconds since bm_server_create: submission (host clock), start of
   * the request's first copy or kernel, end of its factor, end of its last
   * solve/copy (device event clock) */
  double t_submit_us, t_start_us, t_factor_us, t_done_us;
} bm_completion;

typedef struct {
  unsigned long long submitted, admitted, completed, fallbacks;
  int queued, in_flight;
  size_t bytes_in_use, peak_bytes_in_use, budget;
} bm_server_stats;

/* Arena bytes a request holds while in flight (its factor workspace as
 * bm_workspace_bytes, plus the staging of its inputs and outputs under
 * BM_REQ_HOST_IO), or 0 if the request is malformed for this server. */
size_t bm_server_request_bytes(const bm_server_desc *desc, const bm_request *req);

/* Allocates the arena and the slots' streams and events.
 * Errors: BM_ERR_INVALID_ARG, BM_ERR_OOM (arena), BM_ERR_CUDA. */
bm_status bm_server_create(const bm_server_desc *desc, bm_server *out);

/* Queues a request (the caller keeps its buffers valid until its completion
 * is returned) and admits what fits. BM_ERR_INVALID_ARG: malformed request,
 * or one larger than the whole budget (it could never be admitted). */
bm_status bm_server_submit(bm_server s, const bm_request *req);

/* Retires finished requests, admits queued ones and writes up to max_out
 * completions (oldest first) to out; *n_out = how many. Does not block
 * unless wait != 0, in which case it waits until at least one completion
 * is available or nothing is queued or in flight. */
bm_status bm_server_poll(bm_server s, int wait, bm_completion *out, int max_out, int *n_out);

/* Counters of the server; may be called at any time. */
bm_status bm_server_get_stats(bm_server s, bm_server_stats *out);

/* Waits for the requests in flight, then frees everything; queued requests
 * that were never admitted are dropped. */
void bm_server_destroy(bm_server s);

#ifdef __cplusplus
}
#endif

#endif /* BM_H */
