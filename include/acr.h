/*
 * acr.h -- C ABI of the GB300 accelerated-cyclic-reduction (ACR) library.
 *
 * The library builds and applies the ACR preconditioner of Chavez,
 * Turkiyyah, Zampini and Keyes (JCAM 2017) for the block-tridiagonal
 * systems that 7-point discretisations of 3D elliptic PDEs produce
 * (Sec. 4.1: one block row per z-plane, Eq. poissonEquation, Eq. codi),
 * with every plane block held as an H-matrix (Sec. 3, Sec. 4.2), and runs
 * the FP64 Krylov iteration it preconditions (Sec. 5.3 CG, Sec. 7 GMRES).
 *
 * Conventions shared by every entry point:
 *  - Grid: nx * ny * nz interior points of the unit cube, spacing
 *    h = 1/(n+1) per axis (n = nx = ny = nz in this version), Dirichlet 0
 *    boundary.  Unknown p = ix + nx*(iy + ny*iz): x fastest, z-planes are
 *    the CR block rows.
 *  - Stencil: seven FP64 arrays of N = nx*ny*nz entries stored back to back
 *    in one device buffer of 7*N doubles, in the order
 *    c, w, e, s, n, b, t (centre, x-1, x+1, y-1, y+1, z-1, z+1).  A
 *    coefficient that points outside the domain is ignored.
 *  - All array pointers are DEVICE pointers unless a name ends in _host.
 *    The caller owns every pointer it passes; the library never frees or
 *    keeps them past the call, except the handle which the library owns.
 *  - Calls are ordered on the given stream (0 = legacy default stream)
 *    and return after queuing their work, except where noted (setup
 *    synchronises the stream; Krylov reads one scalar back per iteration).
 *  - Every call returns an acr_status.  On error nothing is leaked, output
 *    arrays hold unspecified values and a setup returns *out == NULL.
 *  - A handle is not thread-safe: use it from one host thread and one
 *    stream at a time.
 *  - There is no CPU fallback: without a CUDA device every compute call
 *    returns ACR_ERR_CUDA.
 */
#ifndef ACR_H
#define ACR_H

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ACR_OK = 0,
  ACR_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, eps/eta/leaf out of range, non-finite input */
  ACR_ERR_OOM = 2,           /* device allocation failed */
  ACR_ERR_CUDA = 3,          /* a CUDA call failed (no device, launch error, ...) */
  ACR_ERR_BREAKDOWN = 4,     /* zero pivot in a dense leaf inverse, or Krylov breakdown */
  ACR_ERR_RANK_CAP = 5,      /* a truncated block needed more than the rank cap */
  ACR_ERR_NOT_CONVERGED = 6, /* Krylov hit maxit above rtol */
  ACR_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
  ACR_ERR_UNSUPPORTED = 8    /* valid request the library does not handle (e.g. unbalanced cluster tree) */
} acr_status;

/* Arithmetic form of the H-matrix factors and of the setup / apply
 * arithmetic.  FP64: everything in double.  FP32: factors stored and
 * multiplied in float with float accumulation.  BF16: the setup runs exactly
 * as in FP32; when it ends every stored factor (dense leaves, U, V) is
 * rounded to bfloat16 (round to nearest even), halving the factor memory and
 * the bytes an apply reads; the apply multiplies in float.  The Krylov
 * iteration is FP64 in every form, and so are the Grams that decide ranks
 * (FP64-accurate float-float sums in the float forms).  The dense leaf
 * inverses and the small recompression cores are FP64 in the FP64 form; in
 * the float forms the leaf inverses are float eliminations refined to float
 * accuracy (FP64 elimination when refinement cannot get there), the Jacobi
 * cores run in float-float and the pivoted Cholesky in FP64.
 * (Reduced-precision storage is not in the paper, whose H-arithmetic is
 * double precision throughout, Sec. 5.) */
typedef enum { ACR_FP64 = 0, ACR_FP32 = 1, ACR_BF16 = 2 } acr_precision;

typedef enum { ACR_PCG = 0, ACR_GMRES = 1 } acr_krylov;

typedef struct {
  int32_t nx, ny, nz;   /* interior points per axis; this version needs nx == ny == nz */
} acr_grid;

/* Preconditioner parameters (Sec. 4.3): H_eps, the admissibility eta of
 * Eq. (admis) and the leaf size n_min; plus the storage form and the rank
 * cap of the device factors (blocks whose truncated rank exceeds it make
 * the setup fail with ACR_ERR_RANK_CAP). */
typedef struct {
  double eps;            /* blockwise relative truncation threshold, 0 < eps < 1 */
  double eta;            /* admissibility parameter, > 0 */
  int32_t leaf;          /* n_min: clusters with at most this many points are leaves */
  int32_t precision;     /* acr_precision */
  int32_t rank_cap;      /* 1..48; 0 selects the default (32) */
  int32_t flags;         /* ACR_FLAG_* bits */
  int32_t gemm_variant[16]; /* kernel shape per setup GEMM stage (index = the stage numbering of
                               acr_profile.stage_ms), 0..5 (acr_autotune_gemm); all 0 is the
                               default shape set; other values read as 0 */
} acr_options;

/* acr_options.flags: record per-kernel-class device time (CUDA events
 * around every setup launch) and counted arithmetic of the setup, readable
 * with acr_get_profile.  Adds a small per-launch host cost. */
#define ACR_FLAG_PROFILE 1

typedef struct {
  int32_t levels;            /* CR levels, ceil(log2 nz) */
  int32_t max_rank;          /* largest rank over all stored low-rank blocks */
  double avg_rank;           /* mean rank of stored low-rank blocks */
  int64_t factor_bytes;      /* bytes of stored factors (dense leaves + U,V at their ranks) */
  int64_t factor_capacity_bytes; /* bytes allocated for factors (rank_cap padding) */
  int32_t n_dense_leaves;    /* per plane H-matrix */
  int32_t n_lowrank_leaves;  /* per plane H-matrix */
  double setup_ms;           /* device time of the last setup (CUDA events) */
  double structure_ms;       /* host time spent building the block structure */
  int64_t apply_bytes;       /* bytes one acr_apply must move: every stored factor entry it
                                reads (dense leaves, U and V up to their ranks, couplings) plus
                                its FP64 vector traffic */
  int64_t apply_flops;       /* multiply-adds x 2 of one acr_apply */
  int64_t lr_truncations;    /* low-rank blocks the setup recompressed (all planes, all steps) */
  int64_t sketch_overflows;  /* of those, blocks whose stacked rank (sum of the ranks of the
                                terms summed into the block) exceeded the sketch width
                                min(rank_cap + 8, 64): their range finder was a randomized
                                approximation instead of exact */
  int64_t leaf_fp64_fallbacks; /* float storage: dense leaf inverses (all planes, all levels)
                                whose float elimination + refinement could not reach float
                                accuracy and were done by the FP64 elimination instead */
  double host_issue_ms;      /* host time the setup's device phase took to issue its work
                                (launches, copies) up to its closing event; near setup_ms when
                                the issue rate, not the device, bounds the setup */
} acr_setup_info;

/* Per-kernel-class setup statistics (ACR_FLAG_PROFILE).  flops counts the
 * arithmetic the kernels were asked to do with the ranks they met
 * (2 m n k per GEMM item, cores counted by their loop bounds). */
typedef struct {
  int64_t launches;
  double ms;                 /* summed CUDA-event time of the launches */
  double flops;
} acr_kernel_stat;

typedef struct {
  acr_kernel_stat gemm;      /* grouped small GEMMs (k_ggemm) */
  acr_kernel_stat orth;      /* pivoted-Cholesky cores (k_pchol), FP64 */
  acr_kernel_stat eig;       /* Jacobi recompression cores (k_eig; float-float for float factors) */
  acr_kernel_stat leaf_inv;  /* dense leaf inverses (k_leaf_inv; refined float for float factors) */
  acr_kernel_stat other;     /* conversion, scaling */
  /* grouped-GEMM time and counted flops per plan stage: 0 inner products
   * U^T V of phase 1, 1 term factors (H-matrix x block products, dense
   * products), 2 dense-leaf sums, 3 sketches Z^T Omega, 4 sketch Y, 5 first
   * Gram, 6 first basis, 7 second Gram, 8 second basis, 9 X^T Q, 10 B^T,
   * 11 core Gram, 12 recomposition U = Q W, V = B^T W; 13..15 unused */
  double stage_ms[16];
  double stage_flops[16];
  /* wall time (CUDA events) of each CR level's H-inversion batch and of its
   * Schur-update batch; index = level, the last plane's inversion is in
   * inv_ms[levels] */
  double inv_ms[16];
  double upd_ms[16];
} acr_profile;

typedef struct {
  int32_t iterations;        /* Krylov iterations performed */
  int32_t converged;         /* 1 if the true relative residual reached rtol */
  double rel_residual;       /* final ||f - A u||_2 / ||f||_2, FP64, computed with the 7-point SpMV */
  double solve_ms;           /* device time of the solve */
} acr_solve_info;

typedef struct acr_handle acr_handle;

/* a1, Sec. 6 Eq. (poissonEquation): stencil of -div(kappa grad u), face
 * coefficient = harmonic mean of the two nodal kappas (the node's own kappa
 * on a boundary face), scaled by 1/h^2.  kappa: N doubles (> 0, finite).
 * coef: 7*N doubles written in the stencil layout above.  Errors:
 * INVALID_ARG for NULL pointers or a bad grid. */
acr_status acr_stencil_poisson(const acr_grid* grid, const double* kappa, double* coef,
                               cudaStream_t stream);

/* a1, Sec. 7 Eq. (codi): stencil of -Lap u + beta . grad u with first-order
 * upwinding (backward difference where beta_d > 0, forward where < 0).
 * beta: 3*N doubles (beta_x, beta_y, beta_z arrays back to back). */
acr_status acr_stencil_codi(const acr_grid* grid, const double* beta, double* coef,
                            cudaStream_t stream);

/* a1 for Sec. 8, Eq. (HelmVarVel): stencil of -Lap u - sigma u with the
 * 7-point Laplacian (the paper discretises with 27-point trilinear
 * elements); sigma: N doubles, (omega / c)^2 per node.  The operator is
 * indefinite once sigma exceeds the smallest Laplacian eigenvalue. */
acr_status acr_stencil_helmholtz(const acr_grid* grid, const double* sigma, double* coef,
                                 cudaStream_t stream);

/* y = A x for the 7-point operator (FP64), x and y N doubles each, nrhs
 * vectors back to back. */
acr_status acr_spmv(const acr_grid* grid, const double* coef, const double* x, double* y,
                    int32_t nrhs, cudaStream_t stream);

/* a2-a8, Sec. 4.1-4.3: build the ACR factorisation of the operator given
 * by coef (7*N doubles, not modified, not retained).  Runs the cyclic
 * reduction levels with every plane block in H-format: H-inverse of the
 * eliminated (red) planes, Schur updates of the remaining (black) planes,
 * truncation of every low-rank block to eps relative accuracy.  Synchronises
 * `stream` before returning.  *out receives a new handle owning all factor
 * memory (release with acr_destroy).  Errors: INVALID_ARG, UNSUPPORTED,
 * OOM, CUDA, BREAKDOWN, RANK_CAP; *out is NULL then. */
acr_status acr_setup(const acr_grid* grid, const double* coef, const acr_options* opt,
                     cudaStream_t stream, acr_handle** out);

/* Autotuner of the leaf size n_min (the paper picks it by hand, Sec. 4.3;
 * no counterpart there): for every candidate leaf size, build the
 * factorisation of coef with opt (opt->leaf ignored) and solve one probe
 * system A u = A 1 from u = 0 with `method` (GMRES(restart) or PCG) to
 * rtol; time setup + solve with CUDA events on `stream`.  *best_leaf
 * receives the fastest candidate, times_ms[i] (host, n_cand doubles) the
 * time of cand[i] in ms, or -1 where that candidate failed (unsupported
 * leaf, rank cap, no convergence in 1000 iterations).  Errors: INVALID_ARG;
 * UNSUPPORTED if every candidate failed; OOM, CUDA. */
acr_status acr_autotune_leaf(const acr_grid* grid, const double* coef, const acr_options* opt,
                             int32_t method, int32_t restart, double rtol, const int32_t* cand,
                             int32_t n_cand, int32_t* best_leaf, double* times_ms,
                             cudaStream_t stream);

/* Autotuner of the setup's grouped-GEMM kernel shapes (the paper has no
 * counterpart): one profiled setup of coef with opt per shape (every stage in
 * shape 0, then every stage in shape 1, 2, 3), then per stage the fastest.
 * Shape 0: one CTA per group, 4 CTAs per SM; shape 1: for float factors 3
 * CTAs per SM with more registers (double: half the K-chunk), and the warp-
 * and CTA-per-group inner-product kernels swapped; shape 2 (float factors,
 * non-inner-product stages): one warp per group, groups with 64-column
 * outputs on the shape-0 kernel; shape 3: as 2 with those groups on the
 * tcgen05 tensor cores (split-TF32 operands); shape 4: as 2 with 32 output
 * columns per pass instead of 8; shape 5 (float factors, inner-product
 * stages): 8 x 8 output tiles per warp pass instead of 4 x 8.  variant_out
 * (host, 16 int32) receives the table to put in acr_options.gemm_variant;
 * stage_ms_out (host, 96 doubles, may be NULL) the measured stage times,
 * shape 0 to shape 5.  Errors: as acr_setup. */
acr_status acr_autotune_gemm(const acr_grid* grid, const double* coef, const acr_options* opt,
                             int32_t* variant_out, double* stage_ms_out, cudaStream_t stream);

/* a9-a10, Sec. 4.1 substitution: z = M^{-1} r, M the ACR factorisation;
 * forward then backward sweep of batched H-matrix-vector products.  r, z:
 * nrhs * N doubles (natural ordering); r is not modified; r == z is
 * allowed.  Right-hand sides are processed in groups of up to 8 that share
 * one pass over the stored factors (H-matrix times matrix), so nrhs vectors
 * cost far less than nrhs calls.  No host synchronisation. */
acr_status acr_apply(acr_handle* h, const double* r, double* z, int32_t nrhs,
                     cudaStream_t stream);

/* z = M^{-T} r: the transposed substitution (sweeps in reverse order with
 * transposed H-matrix-vector products), for adjoint solves. */
acr_status acr_apply_transpose(acr_handle* h, const double* r, double* z, int32_t nrhs,
                               cudaStream_t stream);

/* a11, Sec. 5.3 and Sec. 7: solve A u = f to ||f - A u||_2 <= rtol ||f||_2
 * with FP64 preconditioned CG (flexible, Polak-Ribiere) or GMRES(restart)
 * with right preconditioning.  coef: the 7-point operator (7*N doubles,
 * normally the one the handle was built from).  u holds x0 on entry and
 * the solution on exit.  info (host pointer, may be NULL) receives the
 * iteration count and final true residual.  nrhs (1..64) systems with the
 * same operator: f and u hold nrhs vectors N doubles apart; GMRES runs them
 * in lockstep (each its own Krylov space; the preconditioner applies,
 * SpMVs, dots and updates of all systems share launches), PCG one after
 * another; info then reports the largest iteration count and residual and
 * converged = all converged.  maxit counts lockstep iterations.  Errors:
 * NOT_CONVERGED after maxit (u holds the last iterate), BREAKDOWN. */
acr_status acr_krylov_solve(acr_handle* h, const double* coef, int32_t method, int32_t restart,
                            double rtol, int32_t maxit, const double* f, double* u,
                            int32_t nrhs, acr_solve_info* info, cudaStream_t stream);

/* Adjoint solve A^T u = f (the adjoint step of a differentiated solve; the
 * paper has no counterpart): the same Krylov iteration with the transposed
 * 7-point operator and the transposed preconditioner M^{-T}
 * (acr_apply_transpose).  Arguments, results and errors as
 * acr_krylov_solve, except that nrhs must be 1. */
acr_status acr_krylov_solve_transpose(acr_handle* h, const double* coef, int32_t method,
                                      int32_t restart, double rtol, int32_t maxit,
                                      const double* f, double* u, int32_t nrhs,
                                      acr_solve_info* info, cudaStream_t stream);

/* y = A^T x for the 7-point operator (FP64), nrhs vectors back to back. */
acr_status acr_spmv_transpose(const acr_grid* grid, const double* coef, const double* x,
                              double* y, int32_t nrhs, cudaStream_t stream);

/* Adjoint kappa-gradient of the Sec. 6 operator (Eq. poissonEquation, as
 * assembled by acr_stencil_poisson; no counterpart in the paper):
 * grad[p] = -lambda^T (dA/dkappa_p) u, N doubles each (device).  With
 * A u = f and A^T lambda = dL/du this is dL/dkappa.  Errors: INVALID_ARG,
 * CUDA. */
acr_status acr_kappa_gradient(const acr_grid* grid, const double* kappa, const double* lambda,
                              const double* u, double* grad, cudaStream_t stream);

/* Same Krylov iteration with no preconditioner (h not needed): the
 * reference for iteration counts. */
acr_status acr_krylov_solve_plain(const acr_grid* grid, const double* coef, int32_t method,
                                  int32_t restart, double rtol, int32_t maxit,
                                  const double* f, double* u, acr_solve_info* info,
                                  cudaStream_t stream);

/* Allocation-free variant of acr_krylov_solve_plain with method ACR_PCG
 * (the paper has no counterpart: this serves callers that cannot call
 * cudaMalloc where they solve, e.g. an application whose device memory is
 * fully reserved by its own pool allocator, or a latency-critical loop that
 * cannot afford the device synchronisation of cudaMalloc / cudaFree).
 * Same arguments and results as acr_krylov_solve_plain(ACR_PCG), but every
 * work vector and reduction buffer lives in one fixed 24 MiB device array
 * that the library defines at file scope; each GPU that loads the library
 * holds that array until the process exits.  Grids with more than
 * acr_noalloc_max_unknowns() unknowns (about 6.2e5, n <= 85) are rejected
 * with ACR_ERR_INVALID_ARG.  Every call looks up the array's device address
 * in the current device's context (cudaGetSymbolAddress; the first call in
 * a context also loads the library's device code there): make the first
 * call on a device before any stream capture.  Every call shares the one
 * array and keeps the previous call's contents; calls that overlap on the
 * GPU (other streams, other host threads) race with each other.  The call
 * reads a few scalars back per iteration and synchronises `stream`.
 * info->solve_ms is HOST wall time of the call here (the allocating
 * variant reports CUDA-event time); acr_alloc_count() does not change
 * across a call. */
acr_status acr_krylov_solve_plain_noalloc(const acr_grid* grid, const double* coef, double rtol,
                                          int32_t maxit, const double* f, double* u,
                                          acr_solve_info* info, cudaStream_t stream);

/* Largest number of unknowns acr_krylov_solve_plain_noalloc accepts. */
int64_t acr_noalloc_max_unknowns(void);

/* ---- Batches (Sec. 5.1-5.2 run the planes of a CR level in parallel; a
 * batch extends that data parallelism across independent problems, which the
 * paper does not do).  `count` problems, problem i on an n[i]^3 grid with the
 * 7-point operator coefs[i] (device, 7*n[i]^3 doubles, stencil layout above),
 * all with the options *opt.  Problems of equal n share every launch of the
 * setup (their planes are processed as one batch per CR level) and every
 * launch of the apply; problems of different n run on concurrent stream
 * branches.  All device memory is allocated here, sized by a counting pass of
 * the setup: refactoring and applying allocate nothing and synchronise
 * nothing, so they can be captured in a CUDA graph.  The batch keeps the
 * coefs pointers: acr_batch_refactor re-reads them, and they must stay valid
 * (and the caller may overwrite their contents between refactorisations).
 * Batch vectors hold the problems back to back in batch order (n[0]^3
 * doubles, then n[1]^3, ...).  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA,
 * BREAKDOWN, RANK_CAP (*out is NULL then).  acr_batch_create synchronises
 * `stream`. */
typedef struct acr_batch acr_batch;
acr_status acr_batch_create(int32_t count, const int32_t* n, const double* const* coefs,
                            const acr_options* opt, cudaStream_t stream, acr_batch** out);

/* Queue a new factorisation of every problem from the current contents of
 * its coefficient array (no allocation, no synchronisation).  Device errors
 * (pivot breakdown, rank cap) surface at the next acr_batch_status. */
acr_status acr_batch_refactor(acr_batch* b, cudaStream_t stream);

/* Synchronise `stream` and report the device error state of the last
 * factorisation (OK, BREAKDOWN, RANK_CAP, TIMEOUT). */
acr_status acr_batch_status(acr_batch* b, cudaStream_t stream);

/* z_i = M_i^{-1} r_i for every problem i (batch vectors, device). */
acr_status acr_batch_apply(acr_batch* b, const double* r, double* z, cudaStream_t stream);

/* Capture acr_batch_refactor followed by acr_batch_apply(r -> z) into a CUDA
 * graph owned by the batch (replacing an earlier one).  r and z (batch
 * vectors) and the coefficient arrays must stay valid while the graph is
 * used.  `stream` must not be the legacy default stream. */
acr_status acr_batch_capture(acr_batch* b, const double* r, double* z, cudaStream_t stream);

/* Launch the captured graph on `stream` (INVALID_ARG if none was captured). */
acr_status acr_batch_replay(acr_batch* b, cudaStream_t stream);

/* Krylov solve (as acr_krylov_solve, one right-hand side) of problem i with
 * its own preconditioner M_i; coef, f, u are problem i's arrays. */
acr_status acr_batch_krylov_solve(acr_batch* b, int32_t i, const double* coef, int32_t method,
                                  int32_t restart, double rtol, int32_t maxit, const double* f,
                                  double* u, acr_solve_info* info, cudaStream_t stream);

/* Setup statistics of the size class of problem i (all problems of that n
 * together, as of acr_batch_create). */
acr_status acr_batch_get_info(const acr_batch* b, int32_t i, acr_setup_info* info);

/* Release a batch, its graph and all its device memory (NULL is a no-op). */
void acr_batch_destroy(acr_batch* b);

/* Setup statistics of a handle (host struct). */
acr_status acr_get_setup_info(const acr_handle* h, acr_setup_info* info);

/* Per-kernel-class profile of the last setup; INVALID_ARG unless the
 * handle was set up with ACR_FLAG_PROFILE. */
acr_status acr_get_profile(const acr_handle* h, acr_profile* prof);

/* Host-only introspection of the plane block structure used for (n, eta,
 * leaf) (Sec. 3.1): counts[0..5] = {clusters, dense leaves, low-rank
 * leaves, sum of low-rank rows, sum of low-rank cols, tree depth}.  If
 * `leaves_host` is not NULL it receives 5 int32 per leaf block (row begin,
 * row size, col begin, col size, kind 0 = dense / 1 = low rank) in cluster
 * ordering, and `perm_host` (if not NULL) the n*n cluster-order
 * permutation.  Makes no CUDA call. */
acr_status acr_structure_query(int32_t n, double eta, int32_t leaf, int64_t* counts,
                               int32_t* leaves_host, int32_t* perm_host);

/* Number of CUDA kernels this library has launched in the process so far
 * (all handles, all threads); for accounting in benchmarks. */
int64_t acr_launch_count(void);

/* Number of device (cudaMalloc) and pinned host (cudaMallocHost) allocations
 * this library has made in the process so far; for checking which calls
 * allocate. */
int64_t acr_alloc_count(void);

/* Release a handle and all its device memory (NULL is a no-op). */
void acr_destroy(acr_handle* h);

/* Static string naming a status. */
const char* acr_status_string(acr_status s);

#ifdef __cplusplus
}
#endif
#endif /* ACR_H */
