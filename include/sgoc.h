/*
 * sgoc.h - C ABI of the GB300 stochastic Galerkin optimal-control solver.
 *
 * The library solves the stochastic Galerkin (SG) KKT saddle-point system of
 * distributed optimal control of  -div(k(x,xi) grad y) = u  (steady) or
 * y_t - div(k grad y) = u  (all-at-once backward Euler) on the unit square,
 * with homogeneous Dirichlet data, Q1 elements on a uniform nx x nx grid, an
 * affine coefficient k(x,xi) = kappa_0(x) + sum_{k=1..M} kappa_k(x) xi_k with
 * xi_k ~ U[-1,1] independent, and an orthonormal Legendre chaos of total degree p.
 * Reference: Li, Onwunta, Sousedik, "Stochastic Galerkin Method and Hierarchical
 * Preconditioning for PDE-constrained Optimization" (Sec. 2, Eq. (stoch-system);
 * Sec. 3, Eq. (KKT:stoch-time-dependent)).  The Krylov method is preconditioned
 * MINRES with the block-diagonal preconditioner of Eq. (stoch-prec) / Eq.
 * (precon for time), whose Schur block uses the hierarchical Gauss-Seidel sweep
 * of Alg. 1 with geometric-multigrid mean solves.
 *
 * Conventions (all entry points):
 * - Every call returns sgoc_status; no exception or abort crosses the ABI.
 *   sgoc_last_error() gives a human-readable message for the last failure of
 *   the calling thread.
 * - Memory: the library never allocates device memory.  The caller owns every
 *   device buffer (persistent problem data, workspace, vectors) and every
 *   stream; `stream` arguments are cudaStream_t values passed as void*.
 *   Host arrays passed to sgoc_problem_create are copied; the caller may free
 *   them afterwards.
 * - Layout of an SG vector: the paper's vec order (Sec. 2, Eq. (m)): interior
 *   node index fastest (nodes numbered lexicographically, x1 fastest,
 *   n = (nx-1)^2), then the chaos index alpha (graded order, see
 *   sgoc_pc_indices), then the time level.  A KKT vector is [y; u; lambda],
 *   each block of length slabs*P*n with slabs = max(nt, 1).  KKT vectors at the
 *   ABI are float64 in both precisions.
 * - Asynchrony: device work is enqueued on `stream`; calls that return results
 *   to the host (sgoc_solve) synchronize the stream before returning.
 * - Thread safety: one sgoc_problem may be used by one host thread at a time.
 */
#ifndef SGOC_H
#define SGOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SGOC_OK = 0,
  SGOC_ERR_INVALID_ARG = 1,           /* bad size, pointer or parameter */
  SGOC_ERR_UNSUPPORTED = 2,           /* valid problem outside the structured-grid scope */
  SGOC_ERR_WORKSPACE_TOO_SMALL = 3,   /* caller buffer smaller than the queried size */
  SGOC_ERR_CUDA = 4,                  /* a CUDA runtime call failed (see sgoc_last_error) */
  SGOC_ERR_NO_CONVERGENCE = 5,        /* max_iter / max_outer reached */
  SGOC_ERR_BREAKDOWN = 6,             /* Lanczos breakdown before convergence */
  SGOC_ERR_NOT_SPD = 7,               /* <v, P^{-1} v> <= 0: preconditioner not positive */
  SGOC_ERR_NAN = 8,                   /* NaN or Inf in the recurrences or the inputs */
  SGOC_ERR_NOT_UPLOADED = 9           /* device data missing: call sgoc_problem_upload */
} sgoc_status;

typedef enum {
  SGOC_FP64 = 0,        /* operator, preconditioner and Krylov vectors in float64 */
  SGOC_MIXED_FP32 = 1   /* float32 operator/preconditioner/inner MINRES vectors with
                           float64 inner products and scalars, inside float64
                           iterative refinement on the true residual */
} sgoc_precision;

/* Problem statement (Sec. 2 and Sec. 3).  All pointers are host pointers. */
typedef struct {
  int32_t nx;            /* elements per side of the unit square: a power of two, 2..4096 */
  int32_t M;             /* number of random variables / KL terms, 0..16 */
  int32_t p;             /* total degree of the chaos, 0..10; P = C(M+p, p) columns */
  const double* kappa;   /* (M+1)*nx*nx element values kappa_k(e), index (k*nx + ey)*nx + ex
                            (ex along x1); kappa_0 is the mean field and must be a positive
                            constant (the mean-operator multigrid relies on it) */
  double beta;           /* control cost beta > 0 */
  double gamma;          /* variance penalty gamma >= 0 (Eq. (problem-stoch)) */
  int32_t nt;            /* 0: steady problem; >= 1: number of backward-Euler steps */
  double T;              /* final time (nt >= 1), tau = T / nt */
  const double* yhat;    /* max(nt,1)*n target values at interior nodes; in time mode
                            slab t holds yhat(., t_{t+1}), t_k = k tau */
  const double* y0;      /* n initial-state values (time mode) or NULL for y(0) = 0 */
  int32_t chaos;         /* 0: orthonormal Legendre chaos, xi_k ~ U[-1,1], affine coefficient with
                            n_terms = M + 1 planes in kappa (kappa_k multiplies xi_k);
                            1: normalised Hermite chaos, xi_k ~ N(0,1), a coefficient expanded in
                            the chaos itself (the paper's lognormal setting, Sec. 2): n_terms =
                            C(M + 2p, 2p) planes, plane l multiplying psi_l for the multi-indices of
                            total degree <= 2p in the graded order of sgoc_pc_indices */
  double length;         /* side of the square domain (0 selects 1: the unit square; 2 for the
                            paper's [-1,1]^2): the mass matrix scales with length^2 */
} sgoc_problem_desc;

/* Solver options; sgoc_default_options fills the defaults given here. */
typedef struct {
  double tol;            /* relative residual target ||b - K x||_2 / ||b||_2 (1e-8) */
  int32_t max_iter;      /* MINRES iteration cap (FP64) / inner cap (mixed) (1000) */
  int32_t r;             /* truncation: hGS couplings use the coefficient terms 1..r-1; 1..n_terms;
                            0 selects M+1 (Sec. 2, index set I_tau; Sec. 5, r = m+1: the mean and
                            the M linear terms) */
  int32_t cheb_steps;    /* Chebyshev steps for the mass blocks (5) */
  int32_t nu_pre;        /* V-cycle pre-smoothing sweeps (2) */
  int32_t nu_post;       /* V-cycle post-smoothing sweeps (2) */
  double omega;          /* damped-Jacobi weight (0.8) */
  int32_t precision;     /* sgoc_precision (SGOC_FP64) */
  double inner_tol;      /* mixed: inner MINRES relative tolerance (1e-3) */
  int32_t max_outer;     /* mixed: refinement steps cap (20) */
  int32_t schur;         /* time mode, Schur block of the preconditioner (0):
                            0: S~ = (1/tau) Z~ (D (x) M_gamma)^{-1} Z~ with Z~ block-diagonal in
                               time (Eq. (Z hat approx), Eq. (S_tilde)): all slabs at once;
                            1: S_bar = (1/tau) Z_bar (D (x) M_gamma)^{-1} Z_bar^T with the coupled
                               Z_bar = I (x) Z~_t - C (x) M_cal (Eq. (S hat), Eq. (Z hat)): block
                               forward and backward substitution in time, one hGS sweep per step */
  int32_t krylov;        /* 0: preconditioned MINRES (needs the symmetric positive definite
                            preconditioner, the default); 1: flexible GMRES (Sec. 5), right
                            preconditioned, Arnoldi by classical Gram-Schmidt with one
                            reorthogonalisation, float64 Hessenberg and Givens scalars, restarted
                            every `restart` iterations.  In mixed precision the inner solves use
                            the same method in float32 vectors (one cycle each). */
  int32_t restart;       /* FGMRES cycle length, 1..512 (64); memory grows with it: 2*restart + 1
                            KKT vectors of the solve precision (the paper's FGMRES is unrestarted:
                            a cycle longer than the iterations needed) */
  int32_t mass_solve;    /* mass blocks 1 and 2 of the preconditioner (Sec. 5): 0 Chebyshev
                            semi-iteration with cheb_steps steps (0); 1 exact solve with the
                            (square-root-free) Cholesky factorisation of M = M1 (x) M1 */
  int32_t precond;       /* 0: block-diagonal preconditioner of Eq. (stoch-prec) / Eq. (precon
                            for time) with the hGS Schur block (0); 1: hGSoc, the hierarchical
                            Gauss-Seidel sweep over the coupled KKT system (Alg. 2-3; in time mode
                            Alg. 4, every slab independently) with level blocks
                            P~ = blkdiag(M, beta M, A~_1 M^{-1} A~_1), time
                            blkdiag(tau D_t M, beta tau D_t M, (1/tau) A^_1 (D_t M)^{-1} A^_1).  Not
                            symmetric: requires krylov = 1 (FGMRES) */
  int32_t mean_solve;    /* mean solves B ~ A~_1^{-1} of the hGS sweeps (Alg. 1) and of hGSoc:
                            0 one V(nu_pre, nu_post) multigrid cycle (0); 1 the exact inverse by fast
                            diagonalisation (the type-I sine transform diagonalises the constant-
                            stencil mean operator): four dense products with the transform on the
                            tensor cores, operands split into two bfloat16 terms (about 1e-5
                            relative).  Float32 solves only (precision SGOC_MIXED_FP32) on grids
                            of nx = 64 or 128 elements per side; otherwise SGOC_ERR_UNSUPPORTED */
} sgoc_options;

typedef struct {
  sgoc_status status;
  int32_t iterations;          /* MINRES iterations (total inner iterations in mixed mode) */
  int32_t outer_iterations;    /* refinement steps (mixed), 1 for FP64 */
  double rel_true_residual;    /* ||b - K x||_2 / ||b||_2 in float64 at exit */
  double rel_estimate;         /* last MINRES estimate |eta| / ||b||_{P^-1} */
  double ms_total;             /* wall time of the call, milliseconds */
} sgoc_result;

typedef struct sgoc_problem sgoc_problem;

/* Fill `opt` with the defaults documented in sgoc_options. */
void sgoc_default_options(sgoc_options* opt);

/* Host set-up of a problem (Sec. 2-3 problem statement): validates `desc`, builds
 * the multi-index set, the triple-product tables and the multigrid hierarchy,
 * and copies the host inputs.  opt may be NULL (defaults).  Errors:
 * INVALID_ARG for bad sizes/pointers, UNSUPPORTED for a non-constant kappa_0 or
 * a grid that is not a power of two. */
sgoc_status sgoc_problem_create(const sgoc_problem_desc* desc, const sgoc_options* opt,
                                sgoc_problem** out);
void sgoc_problem_destroy(sgoc_problem* pb);

/* n = (nx-1)^2 interior nodes, P chaos columns, slabs = max(nt,1),
 * kkt = 3*slabs*P*n entries of a KKT vector.  Any pointer may be NULL. */
sgoc_status sgoc_problem_sizes(const sgoc_problem* pb, int64_t* n, int64_t* P,
                               int64_t* slabs, int64_t* kkt);

/* Device bytes the caller must provide: `persistent` for sgoc_problem_upload and
 * `workspace` for sgoc_solve / sgoc_apply_precond at the problem's precision. */
sgoc_status sgoc_problem_device_bytes(const sgoc_problem* pb, size_t* persistent,
                                      size_t* workspace);

/* Copy the coefficient and table data into the caller's device buffer
 * d_persistent (>= persistent bytes, 256-byte aligned).  The buffer must stay
 * alive and unmodified while the problem is used. */
sgoc_status sgoc_problem_upload(sgoc_problem* pb, void* d_persistent, size_t bytes,
                                void* stream);

/* Right-hand side b of Eq. (stoch-system) / Eq. (KKT:stoch-time-dependent):
 * [M_cal yhat e_1; 0; 0] steady, [tau (D (x) M_cal) yhat; 0; -d] in time mode
 * with d = [M y0 e_1, 0, ...].  d_b: kkt float64 entries. */
sgoc_status sgoc_rhs(sgoc_problem* pb, double* d_b, void* stream);

/* Solve K x = b by preconditioned MINRES (FP64) or FP32 MINRES inside FP64
 * iterative refinement (mixed).  d_x0 (nullable) is an initial guess; d_x
 * (kkt float64) receives the solution.  d_ws: workspace of >= the queried
 * size, 256-byte aligned.  Synchronizes `stream`; fills *res (nullable). */
sgoc_status sgoc_solve(sgoc_problem* pb, void* d_ws, size_t ws_bytes, const double* d_x0,
                       double* d_x, void* stream, sgoc_result* res);

/* Solve `count` distinct problems concurrently: problem i uses workspace d_ws[i]
 * (ws_bytes[i]), initial guess d_x0[i] (d_x0 or its entries may be NULL),
 * output d_x[i] and stream streams[i] (distinct streams let the solves overlap
 * on the GPU).  The calling thread advances every unfinished solve by one unit of
 * work per sweep (one MINRES iteration, a residual check or a refinement step),
 * so all solves stay in flight together.  Results are identical to sgoc_solve of
 * each problem alone.  res (nullable) receives count results; the return value is
 * the first non-OK status (or OK).  Synchronizes every stream before returning. */
sgoc_status sgoc_solve_batch(int32_t count, sgoc_problem* const* pbs, void* const* d_ws,
                             const size_t* ws_bytes, const double* const* d_x0,
                             double* const* d_x, void* const* streams, sgoc_result* res);

/* The same solves as sgoc_solve_batch with a merged schedule: problems of one
 * shape (grid, M, p, time steps, truncation, precision and preconditioner
 * options; beta, gamma, T, the coefficient fields and targets may differ) whose
 * mean-operator V-cycles run one CTA per column (float32 up to 127 x 127 nodes,
 * float64 up to 15 x 15) are grouped, at most 8 per group, and advanced in
 * lockstep: one MINRES iteration of a group is one captured CUDA graph in which
 * every level visit of the two hGS sweeps (Alg. 1) is a single SG launch and a
 * single V-cycle launch covering the columns of all members, while each member's
 * KKT product, inner products, recurrences and Chebyshev blocks run on its own
 * graph branches.  Members that leave the lockstep for a residual check or a
 * refinement step rejoin at the next group iteration.  Results are bitwise
 * identical to sgoc_solve of each problem alone.  Problems that cannot be grouped
 * are solved as by sgoc_solve_batch.  The paper has no counterpart: batching
 * concerns this GPU code only.  Which schedule is faster depends on the shape: the
 * merged one launches fewer kernels, the independent one lets different phases
 * of different solves overlap. */
sgoc_status sgoc_solve_batch_merged(int32_t count, sgoc_problem* const* pbs, void* const* d_ws,
                                    const size_t* ws_bytes, const double* const* d_x0, double* const* d_x,
                                    void* const* streams, sgoc_result* res);

/* ---- serving: continuous batching of solves over a caller-owned device pool ----
 *
 * A server owns no device memory of its own: requests are sub-allocated (first
 * fit, 256-byte aligned) from d_pool, each needing its problem's persistent +
 * workspace bytes.  sgoc_server_submit queues a request (the problem created
 * with sgoc_problem_create, not necessarily uploaded; d_x receives the
 * solution); sgoc_server_step admits queued requests in FIFO order while a slot
 * and memory are free (uploading the problem into its pool block), advances
 * every active solve whose previous unit of work has finished by one unit (one
 * MINRES iteration, a residual check or a refinement step), retires finished
 * solves (freeing their memory and slot) and admits again.  Each active solve
 * runs on its own stream, so solves that arrived at different times overlap on
 * the GPU.  sgoc_server_poll returns finished requests with their results;
 * ms_total is then the latency from submission to completion.  A problem
 * belongs to the server from submission until it is polled; its device data is
 * released with its pool block (upload it again before using it elsewhere).
 * Results are identical to sgoc_solve of the same problem alone. */
typedef struct sgoc_server sgoc_server;
sgoc_status sgoc_server_create(void* d_pool, size_t pool_bytes, int32_t max_active,
                               sgoc_server** out);
void sgoc_server_destroy(sgoc_server* sv);
/* SGOC_ERR_WORKSPACE_TOO_SMALL when the request cannot fit even an empty pool. */
sgoc_status sgoc_server_submit(sgoc_server* sv, sgoc_problem* pb, double* d_x, uint64_t request_id);
sgoc_status sgoc_server_step(sgoc_server* sv, int32_t* n_active, int32_t* n_queued);
sgoc_status sgoc_server_poll(sgoc_server* sv, uint64_t* ids, sgoc_result* res, int32_t cap,
                             int32_t* n_done);
sgoc_status sgoc_server_stats(const sgoc_server* sv, int64_t* admitted, int64_t* completed,
                              int64_t* rejected, size_t* pool_high_water);

/* ---- tuning ----
 *
 * Kernel choice for the SG operator products of a solve.  The library has
 * several kernels for Y = sum_k K_k X G_k (Sec. 2, Eq. (gPC-A) in Kronecker
 * form); kernels 0-6 form the same products and sums in the same order, so they
 * give bitwise identical results and differ only in speed (kernel 7 agrees with
 * them to rounding; a given table of choices is deterministic).  sgoc_autotune times each
 * applicable kernel on every SG launch shape a solve of `pb` uses (the KKT
 * product, the operator alone, the right-hand side of the return visit of each
 * hGS level of Alg. 1 (d = 0..p), the right-hand side of the first visit of each
 * level (couplings to the level below only); in mixed precision also the
 * float64 true-residual product) on the
 * caller's workspace (d_ws, ws_bytes as for sgoc_solve; its contents are
 * overwritten) and stream, and records the fastest in a process-wide table keyed
 * by launch shape, which every later launch of that shape (any problem with the
 * same grid, chaos levels, truncation, slabs and precision) uses.  Without
 * tuning a built-in rule chooses.  chosen (nullable, nchosen entries, 2p + 4 used)
 * receives the kernel index per shape in the order above (0 one-phase, 1 and 2 four
 * nodes per thread on 32- and 16-node tiles, 3 two-phase float32, 4 and 5 the
 * four-node kernels built for four instead of two CTAs per SM, 6 the direct
 * kernel: a thread per node and output column, for shapes with few outputs and
 * couplings, and the only kernel for shapes whose input columns do not fit any
 * staged kernel's shared memory, e.g. float64 with P = 495; 7 the register kernel:
 * float32, Legendre chaos of the (M, p) it is compiled for ((1,1), (2,2), (3,2),
 * (3,3), (4,3)), a thread per node with every output column's sum in
 * registers; it sums a column's coupling terms in another order than 0-6 and
 * agrees with them to rounding).  Synchronizes the stream.  The paper has no
 * counterpart: it concerns this GPU code only. */
sgoc_status sgoc_autotune(sgoc_problem* pb, void* d_ws, size_t ws_bytes, int32_t* chosen,
                          int32_t nchosen, void* stream);
/* Pins kernel `variant` (0..7 as above; -1 clears the entry, restoring the
 * built-in rule) for SG launch shape `shape` of a solve of pb (0 the KKT product,
 * 1 the operator alone, 2 + d the return visit of hGS level d, 3 + p + d the
 * first visit of level d) in precision 0
 * (float64) or 1 (float32), in the same process-wide table.  The problem need
 * not be uploaded.  SGOC_ERR_UNSUPPORTED when the variant does not apply. */
sgoc_status sgoc_set_kernel(sgoc_problem* pb, int32_t precision, int32_t shape, int32_t variant);

/* ---- building blocks (used by tests and benchmarks) ---- */

/* Y = sum_{k=0}^{M} K_k X G_k (Sec. 2, Eq. (Zv) with A_l in place of A~_l),
 * applied to `nslabs` consecutive n x P panels.  precision 0: X, Y float64;
 * 1: float32.  X and Y must not overlap. */
sgoc_status sgoc_apply_operator(sgoc_problem* pb, int32_t precision, const void* d_X,
                                void* d_Y, int32_t nslabs, void* stream);
/* The same product with one given kernel variant (0..7 as listed for
 * sgoc_autotune); SGOC_ERR_UNSUPPORTED when that kernel does not apply to this
 * shape or precision.  For tests of the variants against each other. */
sgoc_status sgoc_apply_operator_variant(sgoc_problem* pb, int32_t precision, int32_t variant,
                                        const void* d_X, void* d_Y, int32_t nslabs, void* stream);

/* w = K v, the KKT matrix of Eq. (stoch-system) or Eq. (KKT:stoch-time-dependent).
 * precision 0: float64 vectors; 1: float32 vectors.  No workspace. */
sgoc_status sgoc_apply_kkt(sgoc_problem* pb, int32_t precision, const void* d_v, void* d_w,
                           void* stream);

/* z = P^{-1} r, the block preconditioner (Eq. (stoch-prec) / Eq. (precon for time))
 * in the given precision (vectors of that type). */
sgoc_status sgoc_apply_precond(sgoc_problem* pb, int32_t precision, const void* d_r,
                               void* d_z, void* d_ws, size_t ws_bytes, void* stream);

/* V = Z_hGS^{-1} R: one hierarchical Gauss-Seidel sweep (Alg. 1) over the
 * slabs of R (nslabs panels n x P), with the mean operator of the problem's mode. */
sgoc_status sgoc_apply_hgs(sgoc_problem* pb, int32_t precision, const void* d_R, void* d_V,
                           int32_t nslabs, void* d_ws, size_t ws_bytes, void* stream);

/* X = B(R) for ncols columns of length n: one V-cycle for the mean operator
 * (A~_1 of Eq. (mathcalZ) steady, A^_1 of Eq. (A_hat) in time mode). */
sgoc_status sgoc_apply_vcycle(sgoc_problem* pb, int32_t precision, const void* d_R, void* d_X,
                              int32_t ncols, void* d_ws, size_t ws_bytes, void* stream);

/* X = Chebyshev semi-iteration (cheb_steps steps) for M X = R on ncols <= 2*slabs*P
 * columns of length n (Sec. 2: the mass blocks of Eq. (stoch-prec); textbook
 * Golub-Varga weights with D = (5/4) diag(M), eigenvalue bounds [1/4, 9/4]).
 * Uses the preconditioner workspace (sgoc_problem_device_bytes sizes cover it). */
sgoc_status sgoc_apply_chebyshev(sgoc_problem* pb, int32_t precision, const void* d_R,
                                 void* d_X, int32_t ncols, void* d_ws, size_t ws_bytes,
                                 void* stream);

/* Same result as sgoc_apply_chebyshev, for callers that cannot allocate device
 * memory at the point where they need the solve (for instance a plug-in whose
 * host framework owns all device memory and hands out only the input and output
 * buffers, or a real-time path that forbids allocation after start-up): it
 * takes no workspace.  Its two iterate buffers live in a 16 MiB array built into
 * the library, which every GPU that loads the library keeps until the process
 * exits; ncols * n * sizeof(element) must not exceed 8 MiB, larger requests
 * return SGOC_ERR_INVALID_ARG, and so does a call on a device other than the one
 * the problem was uploaded to.  The first call on a device looks up the array's
 * device address with that device current and keeps it for the life of the
 * process (a cudaDeviceReset invalidates it); make that first call before any
 * stream capture.  All calls share the array and every call writes each value
 * it reads from it before reading it: calls whose kernels overlap on the GPU
 * race and must be serialized by the caller.  Allocates nothing.
 * The paper has no counterpart of this entry point. */
sgoc_status sgoc_apply_chebyshev_noalloc(sgoc_problem* pb, int32_t precision, const void* d_R,
                                         void* d_X, int32_t ncols, void* stream);

/* d_out[0] = sum_i a[i] b[i] (float64) over n entries of two device vectors of the
 * given precision (0 float64, 1 float32): the Krylov inner product of the MINRES
 * recurrences (Sec. 5: the Krylov solver's scalars stay float64 in both
 * precisions).  float64 vectors are summed in float64; float32 vectors with
 * exact float32 products and sums split by error-free transformations, whose
 * leading parts are summed in float64, which gives the float64 inner product to
 * a relative error of order 2^-48.  The order of summation is fixed, so the
 * result is reproducible bit for bit.  d_ws: device scratch of at least
 * SGOC_INNER_PRODUCT_WS_BYTES bytes (8-byte aligned); d_out: one device double;
 * d_a and d_b may be NULL when n = 0 (the result is then 0).
 * Enqueued on `stream`, no synchronization. */
#define SGOC_INNER_PRODUCT_WS_BYTES 8192
sgoc_status sgoc_inner_product(int32_t precision, const void* d_a, const void* d_b, int64_t n, void* d_ws,
                               size_t ws_bytes, double* d_out, void* stream);

/* The multi-index set, P x M int32 (host), graded by total degree and
 * lexicographically descending within a degree. */
sgoc_status sgoc_pc_indices(const sgoc_problem* pb, int32_t* host_out);

/* Non-zeros of G_k = E[xi_k Psi_a Psi_b], k = 1..M (G_0 = I is implicit):
 * host arrays of capacity *nnz on input; *nnz returns the count.  Pass NULL
 * arrays to query the count. */
sgoc_status sgoc_triple_products(const sgoc_problem* pb, int32_t* k, int32_t* a, int32_t* b,
                                 double* c, int64_t* nnz);

/* Diagnostic: number of kernels this library has launched in the process so far
 * (all problems and streams).  No counterpart in the paper. */
int64_t sgoc_kernel_launches(void);

/* Diagnostic kernel timing.  sgoc_profile_enable(1) clears the record and makes
 * every later launch record CUDA events around itself on its stream together
 * with its algorithmic bytes and flops; sgoc_profile_enable(0) stops recording.
 * sgoc_profile_query(kind, ...) waits for the recorded events of one kernel
 * class (kind in [0, SGOC_KERNEL_KINDS)) and returns the launch count, summed
 * device milliseconds, bytes and flops.  No counterpart in the paper. */
#define SGOC_KERNEL_KINDS 12
sgoc_status sgoc_profile_enable(int32_t on);
sgoc_status sgoc_profile_query(int32_t kind, int64_t* launches, double* ms, double* bytes,
                               double* flops);
const char* sgoc_kernel_kind_name(int32_t kind);

const char* sgoc_status_string(sgoc_status s);
const char* sgoc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGOC_H */
