/*
 * lrpoisson.h -- C ABI of the GB300 (sm_103a) low-rank Poisson solver.
 *
 * The method is the low-rank Poisson solve of Muravleva & Oseledets,
 * "Fast low-rank solution of the Poisson equation with application to the
 * Stokes problem" (arXiv:1306.2150):
 *
 *   A X = F,  F = U V^T  (Section 3, Eq. flr:lr), A the discrete Laplacian of
 *   the unit square with homogeneous Dirichlet conditions (Section 2, 4.1);
 *   Uh = S U, Vh = S V with S the orthonormal DST-I (Section 4.1, Eq. flr:diag);
 *   Xh[i,j] = (Uh Vh^T)[i,j] / Lambda[i,j] approximated by a cross
 *   (Section 4.2, Eq. flr:div); rounding by QR + a small SVD (Section 3);
 *   X = (S Uo) diag(s) (S Vo)^T.
 *
 * Conventions for every entry point:
 *   - All matrix pointers are DEVICE pointers owned by the caller.  Factor
 *     matrices are column-major float64 with leading dimension ld >= rows;
 *     pointers must be 16-byte aligned.
 *   - Work is enqueued on the handle's stream.  Unless LR_FLAG_ASYNC is set,
 *     a call returns after that stream has finished the work, so the output
 *     rank and status are known on return.
 *   - Errors are returned as lr_status; nothing is thrown across the ABI.
 *     lr_last_error() gives a one-line description of the last failure.
 *   - The library owns only workspace inside the handle (device memory grown
 *     on demand with cudaMalloc, pinned host memory for status), released by
 *     lr_destroy().
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef LRPOISSON_H
#define LRPOISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LR_OK = 0,
  LR_EINVAL = 1,     /* invalid argument (sizes, pointers, alignment, options) */
  LR_ENOMEM = 2,     /* device or pinned allocation failed */
  LR_ENOCONV = 3,    /* cross hit its step cap or the rank was cut to capacity;
                        the best partial result is written */
  LR_ETIMEOUT = 4,   /* reserved for a bounded device wait that ran out; no
                        kernel of this library waits on a flag (every loop
                        and barrier is bounded), so it is not returned */
  LR_ECUDA = 5,      /* a CUDA runtime call failed */
  LR_ENONFINITE = 6  /* a non-finite value reached the rounding core (in
                        LR_MIXED: entries of the frequency-space solution
                        outside the float32 range; rescale the right-hand
                        side); no factors are written */
} lr_status;

typedef enum {
  LR_FP64 = 0,       /* every step in float64 */
  LR_MIXED = 1       /* float32 transforms and row/column sampling; float64
                        pivot values, Gram accumulation and QR cores */
} lr_precision;

typedef enum {
  /* 5-point Laplacian, m interior points per direction, h = 1/(m+1):
     Lambda[i,j] = mu_i + mu_j, mu_i = (4/h^2) sin^2(i pi h / 2)
     (Section 4.2, Eq. flr:div). */
  LR_OP_5PT = 0,
  /* semi-staggered Laplacian of Section 2, Delta = B_x B_x^T + B_y B_y^T, on
     n = m+1 cells (h = 1/n): Lambda[i,j] = (l_i (4-l_j) + (4-l_i) l_j)/(16 h^2),
     l_i = 4 sin^2(i pi h / 2), the symbol of A1 (x) A2 + A2 (x) A1, A1 = G G^T,
     A2 = H H^T (Section 4.1). */
  LR_OP_SEMISTAGGERED = 1
} lr_operator;

/* Bits of lr_options.flags. */
#define LR_FLAG_ASYNC 1u   /* do not wait for the stream; read rank/status with
                              lr_get_info() after synchronising the stream */
#define LR_FLAG_TIMING 2u  /* record CUDA events between the phases of a solve
                              (lr_poisson2d, or a phase-batched
                              lr_poisson2d_batched: each phase then covers
                              every problem); read them with
                              lr_get_phase_times() */
#define LR_FLAG_GRAPH 4u   /* capture the enqueued work once as a CUDA graph
                              (keyed by every pointer, size and option) and
                              replay it on later calls with the same key */
#define LR_FLAG_CLUSTER_DST 8u /* lr_poisson2d: run both transforms with the
                                  cluster variant (one thread-block cluster
                                  per column, 8192 <= M <= 131072) for this
                                  call, whatever the tuned choice */
#define LR_FLAG_GMRES 16u      /* lr_stokes_uzawa: restarted inexact GMRES with
                                  adaptive accuracy (Section 5) instead of
                                  conjugate gradients */
#define LR_FLAG_BATCH_STREAMS 32u /* lr_poisson2d_batched: run each problem as
                                     its own launch chain over internal
                                     streams instead of the phase-batched
                                     launches */

/* Phases of lr_poisson2d timed under LR_FLAG_TIMING. */
#define LR_PHASE_FORWARD_DST 0  /* DST of the right-hand side factors      */
#define LR_PHASE_CROSS 1        /* cross approximation (one cluster launch) */
#define LR_PHASE_ROUNDING 2     /* k x k core and rotation of the skeleton  */
#define LR_PHASE_INVERSE_DST 3  /* DST of the kept factors                  */
#define LR_NUM_PHASES 4

typedef struct lr_handle_s* lr_handle;

/* A low-rank matrix X = U diag(s) V^T of size n1 x n2 (Section 3, Def. of the
 * low-rank format).  U is n1 x rmax, V is n2 x rmax (column-major, leading
 * dimension ld), s has rmax entries; the first r columns / entries are used.
 * On input s may be NULL (all ones).  On output U and V have orthonormal
 * columns and s holds the singular values in descending order. */
typedef struct {
  int n1, n2;
  int r;
  int rmax;
  int ld;
  double* U;
  double* s;
  double* V;
} lr_mat;

typedef struct {
  lr_precision prec;
  lr_operator op;
  double eps;            /* relative Frobenius tolerance of cross and rounding */
  int rmax;              /* cap on cross steps (<= 64) */
  double aca_tol_factor; /* cross stop tolerance = aca_tol_factor * eps */
  int probes;            /* residual probes after the cross stops (0 = none) */
  unsigned long long seed; /* splitmix64 seed of the probe positions */
  unsigned int flags;    /* LR_FLAG_* */
  int cluster_size;      /* CTAs per cross cluster (0 = automatic, 1..16) */
  int refine;            /* LR_MIXED only: maximum rounds of iterative
                            refinement in float64 (0 = automatic: up to 6
                            rounds when eps < 1e-7, none otherwise; -1 =
                            none).  A round forms the residual F - A X
                            exactly in float64 as a low-rank matrix, rounds
                            it with a shifted Cholesky QR, solves for the
                            correction D in mixed precision and rounds X + D
                            at eps.  Rounds stop once the correction times
                            the ratio of the last two corrections is below
                            eps / 2 relative to X, or when the corrections
                            stop shrinking.  Refined solves are synchronous. */
} lr_options;

/* Result details of the last solve on a handle. */
typedef struct {
  int status;            /* lr_status of the last solve */
  int aca_steps;         /* skeleton columns k built by the cross */
  int rank;              /* rank R kept by the rounding */
  int converged;         /* cross stop test passed */
  int cut;               /* rank cut to the output capacity */
  int probe_rounds;
  int zero_rows;         /* rows skipped because their residual was exactly 0 */
  int cluster_size;      /* CTAs used by the cross */
  int launches;          /* kernels launched by the solve */
  double norm_est;       /* cross estimate of ||Xh||_F */
  double sigma0;         /* largest singular value kept */
  int refine_rounds;     /* refinement rounds taken (LR_MIXED, eps < 1e-7);
                            after lr_stokes_uzawa: mixed velocity solves that
                            broke down in float32 and were repeated in float64 */
  int pad;
  double refine_corr;    /* sigma_0 of the last correction / sigma_0 of X */
} lr_info;

/* Defaults: LR_MIXED, LR_OP_5PT, eps 1e-6, rmax 64, aca_tol_factor 1,
 * 16 probes, seed 0, flags 0, cluster_size 0, refine 0. */
void lr_options_default(lr_options* opt);

/* Create a handle bound to a CUDA stream (cudaStream_t, NULL = legacy default
 * stream) on the current device.  Returns LR_ECUDA if no device is usable. */
lr_status lr_create(lr_handle* h, void* cuda_stream);
lr_status lr_set_stream(lr_handle h, void* cuda_stream);
/* Cap the total device workspace the handle may hold (the paper has no
 * counterpart; memory budgeting for processes that share a GPU).  bytes = 0
 * removes the cap (default).  A call whose workspace would exceed the cap
 * returns LR_ENOMEM before launching anything and leaves the handle usable;
 * workspace already held is kept.  Plan tables, captured graphs and their
 * descriptor blocks are not counted. */
lr_status lr_set_workspace_limit(lr_handle h, size_t bytes);
lr_status lr_destroy(lr_handle h);
const char* lr_last_error(lr_handle h);
const char* lr_status_string(lr_status s);

/* Orthonormal DST-I of order m applied to ncols columns (Section 4.1,
 * "DST of the factors", Eq. flr:diag): out[:,c] = S in[:,c],
 * S[i,k] = sqrt(2/(m+1)) sin(pi i k/(m+1)).  in/out are column-major float64
 * with leading dimensions ld_in, ld_out >= m; in == out is allowed.
 * prec selects float64 or float32 arithmetic.  m >= 1, ncols >= 0. */
lr_status lr_dst1(lr_handle h, int m, int ncols, const double* in, int ld_in,
                  double* out, int ld_out, lr_precision prec);

/* Low-rank Poisson solve A X = F (Sections 4.1-4.2 with the rounding of
 * Section 3).  rhs: n1 = n2 = m (1 <= m <= 131072), rank r (1..64), U, V;
 * rhs->s must be NULL (fold weights into U).
 * sol: n1 = n2 = m, capacity sol->rmax, U, s, V written; sol->r set on return
 * (synchronous mode).  The solution satisfies ||X - A^-1 F||_F <= ~2 eps
 * ||A^-1 F||_F for the default options.  Returns LR_ENOCONV with a partial
 * result if the cross needed more than opt->rmax steps or the rank exceeded
 * sol->rmax.  opt NULL means defaults. */
lr_status lr_poisson2d(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options* opt);

/* Batched low-rank Poisson solves: `batch` independent problems (host arrays
 * rhs[batch], sol[batch] of lr_mat with device pointers, each as for
 * lr_poisson2d, sizes and ranks may differ) with shared options.
 * Phase-batched form (default when every order m is at most 65536): each
 * step of the solve runs for all problems
 * in one launch -- the forward DST of every factor column, the cross of
 * every problem (one CTA, or a cluster of 2 to 16 CTAs, per problem, longest
 * problems first; cluster sizes run concurrently), the rounding cores, the
 * rotation of the skeletons and the inverse DST -- about ten launches per
 * batch.  The problem descriptors are uploaded with the work.  With
 * LR_FLAG_BATCH_STREAMS (or larger orders) each problem is instead its own
 * launch chain, dealt in decreasing order of size over 32 internal streams.
 * With LR_FLAG_GRAPH the whole batch is one replayed CUDA graph.
 * per_problem (host, may be NULL) receives each problem's status; the return
 * value is LR_OK or the first failure.  The paper solves one problem at a
 * time; batching is the data-parallel form of its Section 4.2 solve for many
 * right-hand sides. */
lr_status lr_poisson2d_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol,
                               const lr_options* opt, lr_status* per_problem);

/* Results of an asynchronous lr_poisson2d_batched (LR_FLAG_ASYNC; the paper
 * has no counterpart): once the caller has synchronised the handle's stream
 * after that call, writes sol[i].r (the kept rank of problem i) and, if
 * per_problem is not NULL, its status, as the synchronous call would have.
 * sol and per_problem are host arrays of the first `batch` problems of that
 * call; the factors themselves are already in the caller's buffers.  Returns
 * LR_OK or the first failure of those problems; LR_EINVAL if batch exceeds
 * the last batched call on this handle.  Reads the handle's status record:
 * call it before the next batched call on the same handle. */
lr_status lr_batched_status(lr_handle h, int batch, lr_mat* sol, lr_status* per_problem);

/* Rounding (recompression) of X = U diag(s) V^T in place (Section 3): QR of
 * both factors, SVD of the r x r core, truncation at relative Frobenius
 * tolerance eps, at most min(rmax, X->rmax) columns kept.  float64
 * throughout.  X->s is required: it holds the input weights (set them to 1
 * for a plain U V^T) and receives the singular values.  X->r (1..64) is
 * updated; U and V are overwritten with orthonormal columns.  Returns
 * LR_ENOCONV if more than rmax columns were needed (result cut). */
lr_status lr_truncate(lr_handle h, lr_mat* X, double eps, int rmax);

/* Maxvol row selection (Section 4.2 names maxvol as the quasi-optimal way to
 * choose the rows and columns of the cross; the algorithm is the cited one of
 * Goreinov, Oseledets, Savostyanov, Tyrtyshnikov and Zamarashkin, 2010).
 * float64 throughout.
 *
 * With B = C C[rows, :]^{-1} (the coefficients of every row of C in the basis
 * of the selected rows; B[rows, :] is the identity), repeatedly take the
 * largest |B[i, j]| (lowest column-major index j m + i on ties) and, while it
 * exceeds 1 + delta, put row i in position j -- which multiplies
 * |det C[rows, :]| by |B[i, j]| -- and update B by the rank-1 formula
 * B' = B - B[:, j] (B[i, :] - e_j^T) / B[i, j].  On return C[rows, :] is a
 * (1 + delta)-dominant submatrix unless maxswaps swaps ran out.  To refine
 * the row pivots of a cross, pass any basis of its column space (the
 * skeleton columns): B does not depend on the basis.
 *
 * C: device, m x k column-major, leading dimension ldc >= m, 1 <= k <= 64,
 *    k <= m; read only.
 * rows: host, k distinct indices in [0, m) with C[rows, :] nonsingular; on
 *    return position j holds the row whose coefficient vector is e_j.
 * nswaps, bmax (host, may be NULL): the swaps made and the final largest |B|.
 * Runs on the handle's stream and returns after it has finished; scratch
 * (m k + 4.2 K doubles) comes from the handle's workspace.
 * Returns LR_EINVAL for bad arguments or a singular C[rows, :] (rows then
 * unchanged), LR_ENONFINITE for a non-finite coefficient, LR_ENOCONV if
 * maxswaps swaps were made and max |B| still exceeds 1 + delta (rows, nswaps
 * and bmax hold the state reached), LR_ENOMEM, LR_ECUDA. */
lr_status lr_maxvol(lr_handle h, const double* C, int m, int k, int ldc, double delta, int maxswaps,
                    int* rows, int* nswaps, double* bmax);

/* Details of the last lr_poisson2d on this handle.  pivots_I / pivots_J (host,
 * may be NULL) receive up to cap cross pivot indices (0-based). */
lr_status lr_get_info(lr_handle h, lr_info* info, int* pivots_I, int* pivots_J, int cap);

/* Milliseconds of each phase (LR_PHASE_*) of the last lr_poisson2d or
 * phase-batched lr_poisson2d_batched run with LR_FLAG_TIMING, measured with
 * CUDA events on the handle's stream (in a batch, LR_PHASE_ROUNDING also
 * covers the rotation of the skeletons).  Waits for the last event.
 * n <= LR_NUM_PHASES entries are written.  LR_EINVAL if the last solve was
 * not timed. */
lr_status lr_get_phase_times(lr_handle h, double* ms, int n);

/* Low-rank Uzawa solve of the 2D Stokes problem on semi-staggered grids
 * (Section 2: Eq. flr:stprob with A = I_2 (x) Delta, B = [B_x; B_y],
 * B_x = G (x) H / (4h), B_y = H (x) G / (4h), h = 1/n; Section 5: the Uzawa
 * iteration in low-rank format).  Conjugate gradients on the Schur equation
 * (B^T A^-1 B) p = B^T A^-1 f - g (Eq. flr:schur; the paper prints it without
 * the divergence right-hand side g, elimination of u gives the -g) with every iterate in low-rank
 * format: each Schur product applies B to the factors (bidiagonal maps, rank
 * kept), runs the two velocity Poisson solves (semi-staggered kind, m = n - 1,
 * batched, opt->prec) and rounds B^T of the result; every CG update is
 * rounded in float64 at opt->eps; the CG scalars are float64.  The
 * pressure's two kernel modes (constant, checkerboard) are projected out of
 * p.  Stops when ||r|| <= tol_div ||B^T A^-1 f - g|| (r the Schur residual) or
 * after maxit iterations (LR_ENOCONV, best iterate written).
 *   d     : 2 (the only dimension built)
 *   n     : cells per direction; velocity on the (n-1) x (n-1) interior
 *           vertices, pressure on the n x n cell centres (first index x)
 *   f     : 2 body-force components, (n-1) x (n-1), rank 1..64, s = NULL
 *   g     : NULL (divergence-free, B^T u = 0) or the divergence right-hand
 *           side B^T u = g: n x n, rank 0..64, s may be NULL; rounded at
 *           eps on entry; its components along the pressure's two kernel
 *           modes cannot be met (B annihilates them) and are dropped
 *   u     : 2 velocity outputs (n-1) x (n-1), U, s, V capacity rmax
 *   p     : pressure output n x n (U, s, V capacity rmax).  On entry p->r = 0,
 *           or the rank of an initial guess held in p (resume from a saved
 *           pressure: CG restarts from r = rhs - S p, GMRES likewise)
 *   iters : CG iterations taken (may be NULL)
 *   resid : ||B^T u - g'|| / ||B^T A^-1 f - g'|| of the returned velocity,
 *           g' = g without its kernel components (may be NULL)
 *   history: host array of maxit + 1 doubles (may be NULL): ||r_k|| / ||r_0||
 *           of the CG residual for k = 0..iters (the rest untouched)
 * LR_EINVAL for bad arguments, LR_ENOCONV if tol_div was not reached or a
 * low-rank sum needed more than 64 columns.  Synchronises. */
lr_status lr_stokes_uzawa(lr_handle h, int d, int n, const lr_mat* f, const lr_mat* g, lr_mat* u, lr_mat* p,
                          double tol_div, int maxit, const lr_options* opt, int* iters, double* resid,
                          double* history);

/* A three-dimensional tensor in Tucker format (Section 3, Eq. flr:tucker):
 * A(i, j, k) = sum_{a,b,c} G(a, b, c) U[0](i, a) U[1](j, b) U[2](k, c).
 * Device pointers; factors column-major n[k] x r[k] with leading dimension
 * ld[k] (even, >= n[k], 16-byte aligned); the core in C order,
 * G[(a r[1] + b) r[2] + c].  rmax[k] is the output capacity of a solution
 * (its core must hold rmax[0] rmax[1] rmax[2] doubles, U[k] rmax[k] columns). */
typedef struct {
  int n[3];
  int r[3];
  int rmax[3];
  int ld[3];
  double* G;
  double* U[3];
} lr_tucker;

/* Low-rank 3D Poisson solve in Tucker format (Section 3, Eq. flr:tucker;
 * Sections 4.1 and 4.2 in three dimensions): A X = F for the 7-point
 * Laplacian of the unit cube with homogeneous Dirichlet conditions, n[k]
 * interior points in direction k (h_k = 1/(n[k] + 1)), F = rhs in Tucker
 * format.  X-hat = F-hat / (mu_i + mu_j + mu_k) (F-hat = G x_k (S U_k), S the
 * DST-I) is approximated by a Tucker fibre cross: each step finds a pivot by
 * alternating maximisation of the residual along fibres, adds the residual
 * fibres through it to per-mode orthonormal bases Q_k with DEIM
 * interpolation indices I_k, and takes the core by cross interpolation
 * C = X-hat(I_1, I_2, I_3) x_k Q_k(I_k, :)^-1; the stop test (the step's
 * rank-one size below tol ||C||_F twice) is confirmed by probe rounds
 * (opt->probes random fibres per mode drawn by splitmix64 from opt->seed,
 * and every fibre through the other modes' index sets), tol =
 * 0.1 aca_tol_factor eps.  Then the higher-order SVD of C, each mode
 * truncated with a tail <= eps ||C|| / sqrt(3), and the inverse DST of the
 * kept factors.  Output: sol->G, sol->U[k] (orthonormal columns), sol->r.
 * Precision: LR_FP64 throughout; LR_MIXED runs the transforms and the
 * Jacobi iterations of the rounding cores in float32 (the cross and the
 * Cholesky QR in float64) and needs eps >= 1e-7.
 * Requirements: opt->op == LR_OP_5PT (its 3D analogue), 1 <= n[k] <= 16384,
 * 1 <= r[k] <= 64, opt->rmax <= 64 cross steps.  LR_EINVAL for bad arguments, LR_ENOCONV if the cross did not
 * converge within opt->rmax steps or a rank exceeded sol->rmax (result
 * truncated), LR_ENONFINITE for a non-finite value.  Synchronises. */
lr_status lr_poisson3d_tucker(lr_handle h, const lr_tucker* rhs, lr_tucker* sol, const lr_options* opt);

/* Exponential-sum solve of the 5-point problem (Section 4.1, the known
 * approach the cross method is compared with): 1/lambda is approximated on
 * the spectrum [2 mu_1, 2 mu_m] by the sinc (trapezoidal) quadrature of
 * int exp(s - lambda e^s) ds at eps / 10, so that
 *   Xh ~ sum_q w_q (E_q Uh)(E_q Vh)^T,  E_q = diag(exp(-t_q mu)),
 * accumulated in chunks and rounded at eps in float64 (shifted Cholesky QR
 * and the core SVD, Section 3); float64 transforms.  Arguments as
 * lr_poisson2d; opt->op must be LR_OP_5PT (the semi-staggered symbol does
 * not split into a sum); nterms (may be NULL) receives the number of
 * quadrature terms.  LR_EINVAL for eps < 1e-12 or the other operator kind.
 * Synchronises. */
lr_status lr_poisson2d_expsum(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options* opt, int* nterms);

/* Full-grid solve of A X = F on the m x m grid (Section 4.1, Eq. flr:diag:
 * X = S ((S F S) / Lambda) S, the fast Poisson solver the low-rank method is
 * compared with; no truncation).  F and X are dense column-major float64
 * device matrices (leading dimensions ldf, ldx >= m, 16-byte aligned; X may
 * not alias F).  opt->prec picks the transforms' precision (LR_MIXED: float32
 * transforms), opt->op the operator kind; eps, rmax and the cross options are
 * ignored.  Work: four DST-I passes over m columns, two transposes, the
 * division by Lambda fused into the third transform's input.  Workspace:
 * about 2 m^2 + 2 M m working-precision words (M = next power of two >= 2m - 1)
 * in the handle.  Synchronises. */
lr_status lr_poisson2d_full(lr_handle h, int m, const double* F, int ldf, double* X, int ldx,
                            const lr_options* opt);

/* Autotuning of the launch shapes (the paper has no counterpart): the tiles
 * and cluster sizes a solve looks up for its order before launching.
 *
 * lr_autotune times lr_poisson2d on the caller's problem rhs (device buffers
 * as for lr_poisson2d; the trial solutions go to internal scratch) with CUDA
 * events on the handle's stream, one warm-up and `reps` timed solves per
 * candidate (median), and keeps the fastest in the handle for the order m,
 * precision and operator kind of opt.  Later solves on this handle with
 * opt->cluster_size = 0 use it.  Candidates, for orders whose transform is
 * not a single-CTA one (2m - 1 > 4096): the four-step transform's tile (1024,
 * 2048 or 4096 complex elements) and the cluster transform (one thread-block
 * cluster per column, 8192 <= M <= 131072); then the cross cluster size (1,
 * 2, 4, 8, 12, 16 CTAs, those the order admits).  Refinement is not run
 * while tuning.
 *
 * lr_autotune_batched times lr_poisson2d_batched on the given batch (its
 * sol buffers receive the trial results) for several numbers of indices per
 * cross CTA and keeps the fastest for batched solves of that precision on
 * this handle: 2048, 4096, 8192, 16384 (LR_FP64 up to 8192; default 4096)
 * for the phase-batched form, which then takes 1 to 16 CTAs per problem;
 * 1024, 2048, 4096, 8192 (default 2048) for the stream form
 * (LR_FLAG_BATCH_STREAMS in opt->flags).
 *
 * Both synchronise and return LR_EINVAL for bad arguments.  `out` (host, may
 * be NULL) receives the choice and the times. */
typedef struct {
  int cluster_size;          /* tuned CTAs per cross cluster (single solves) */
  int log_tile;              /* log2 of the tuned transform tile (0: heuristic) */
  int transform;             /* tuned transform variant: 0 four-step, 1 cluster */
  int batch_indices_per_cta; /* tuned indices per cross CTA (batched solves) */
  int candidates;            /* configurations timed */
  double ms_best;            /* median ms of the chosen configuration */
  double ms_default;         /* median ms of the untuned configuration */
} lr_tune;
lr_status lr_autotune(lr_handle h, const lr_mat* rhs, const lr_options* opt, int reps, lr_tune* out);
lr_status lr_autotune_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options* opt,
                              int reps, lr_tune* out);

/* lr_truncate without any allocation (the paper has no counterpart; this is
 * a deployment variant of lr_truncate above).  The method is the same, but
 * its Gram sums run over a fixed grid of 64 CTAs, so the summation order
 * differs from lr_truncate's: results agree up to rounding, and the kept rank
 * may differ by one where a singular value sits at the eps cutoff.
 *
 * For callers that cannot allocate device or pinned memory themselves: code
 * running inside another framework's memory pool, where a direct cudaMalloc
 * would bypass the pool's budget, and latency-critical loops, where cudaMalloc
 * may stall and cudaFree synchronises the whole device.  No handle is used
 * (creating one allocates pinned host memory) and no cudaMalloc, cudaFree or
 * allocating library routine is called.
 *
 * Scratch: one file-scope device array of 2.2 MB (Gram partials, the two
 * Gram matrices, the k x k rotations and a status record), reserved on every
 * GPU that loads the library until the process exits.  Limit: X->r <= 64
 * (larger ranks return LR_EINVAL); any number of rows.  The first call on a
 * device looks up the array's device address (with that device current), so
 * make that first call before any stream capture.
 *
 * All calls on one device share the array and it keeps the last call's
 * contents (the status record is cleared at the start of every call): calls
 * whose work overlaps on the GPU -- different streams, or different host
 * threads -- race and must be serialised by the caller.
 *
 * Arguments as lr_truncate (X->s required; U and V overwritten with
 * orthonormal columns, s with the kept singular values, X->r with the kept
 * rank), plus the CUDA stream (cudaStream_t, NULL = legacy default stream)
 * that runs the work; returns after that stream has finished it.  Returns
 * LR_EINVAL for bad arguments or X->r > 64, LR_ECUDA for a CUDA failure and
 * LR_ENOCONV if more than rmax columns were needed (result cut). */
lr_status lr_truncate_noalloc(lr_mat* X, double eps, int rmax, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LRPOISSON_H */
