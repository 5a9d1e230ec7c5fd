/*
 * clair.h - C ABI of the GB300 (sm_103a) library for constrained local approximate
 * ideal restriction (CLAIR) algebraic multigrid, arXiv 2307.00229.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are square CSR operators: int32 row pointers (n+1) and column indices
 *   (nnz, sorted ascending and unique within each row), float64 values.  All pointers
 *   that carry vector or matrix data are DEVICE pointers unless the name ends in _host.
 * - Inputs are borrowed: the library neither frees them nor keeps them after the call
 *   returns (a hierarchy copies what it needs).  Outputs are caller-owned buffers of the
 *   stated size.  A hierarchy (clair_h) owns every device buffer it allocates; free it
 *   with clair_free.
 * - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.  Calls
 *   that return host scalars synchronise that stream before returning.
 * - Every call returns a clair_status and never aborts; clair_last_error() gives a
 *   one-line description of the last failure on the calling thread.
 * - Index convention for C/F splittings: cf[i] = 1 for a C-point, 0 for an F-point; the
 *   coarse index of a C-point is its rank among C-points in increasing fine index.
 */
#ifndef CLAIR_H
#define CLAIR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CLAIR_OK = 0,
  CLAIR_ERR_ARG = 1,            /* invalid argument (null pointer, size, parameter) */
  CLAIR_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  CLAIR_ERR_SINGULAR_BLOCK = 3, /* a local block had a zero pivot (its weights are set to 0) */
  CLAIR_ERR_NONFINITE = 4,      /* NaN or Inf in an input or a result */
  CLAIR_ERR_NOT_CONVERGED = 5,  /* FGMRES stopped at gmres_maxit above rtol */
  CLAIR_ERR_CAPACITY = 6,       /* a size exceeded a kernel limit (e.g. local system > 4096) */
  CLAIR_ERR_UNSUPPORTED = 7     /* a parameter combination this build does not implement */
} clair_status;

enum { CLAIR_COARSEN_FC = 0, CLAIR_COARSEN_AGG = 1 };
enum { CLAIR_FP64 = 0, CLAIR_MIXED = 1 };
enum { CLAIR_INVERSE_EXACT = 0, CLAIR_INVERSE_DIAG = 1 };
enum { CLAIR_KRYLOV_FGMRES = 0, CLAIR_KRYLOV_PCG = 1 };
/* Largest number of mode vectors (columns of B). */
#define CLAIR_KMAX 4

/* Solver parameters.  Defaults (clair_params_default) follow the nonsymmetric runs of
 * Section 4.2: coarsening strength 0.25, interpolation strength 0.05, pattern degree
 * m = 2 (Algorithm 1), B = 1 smoothed by 5 CFF sweeps per level (Section 4.1), weight
 * 1/rho(D^-1 A) from 15 Arnoldi steps (Section 4), post-smoothing weight removed
 * (Section 4.2), V(1,1) cycles inside right-preconditioned FGMRES. */
typedef struct {
  double theta_coarsen;   /* strength threshold for the C/F splitting */
  double theta_interp;    /* strength threshold for the transfer patterns */
  int degree;             /* sparsity pattern degree m of Algorithm 1 (1 or 2) */
  int coarsen;            /* CLAIR_COARSEN_FC (C/F splitting, the Ruge-Stueben first pass
                             read as a parallel independent set) or CLAIR_COARSEN_AGG
                             (aggregation: roots of a distance-two independent set are the
                             C-points, Algorithm 1's base pattern T is the aggregation
                             operator; Section 3.1.3 and its footnote) */
  int b_smooth_iters;     /* CFF sweeps applied to the mode vector on each level */
  int arnoldi_iters;      /* Arnoldi steps for rho(D^-1 A) */
  int post_weighted;      /* 1: post-smoothing uses the weight too; 0: weight 1 */
  int coarse_max;         /* a level with n <= coarse_max is solved directly */
  int max_levels;         /* hard cap on the number of levels */
  int precision;          /* CLAIR_FP64 or CLAIR_MIXED (FP32 V-cycle and local solves) */
  int gmres_restart;      /* FGMRES restart length (<= 64) */
  int gmres_maxit;        /* FGMRES iteration cap */
  double rtol;            /* stop when ||f - A u||_2 <= rtol ||f||_2 (true FP64 residual) */
  uint64_t seed;          /* seed of the Arnoldi start vectors (splitmix64, seed + level) */
  int inverse;            /* block inverses of Algorithm 1: CLAIR_INVERSE_EXACT (Remark 3.2)
                             or CLAIR_INVERSE_DIAG (the local diagonal, one of the approximate
                             block inverses of Section 3.1.2) */
  int iterations;         /* Algorithm 1's loop count k (>= 1).  With the exact inverse the
                             output is the same for every k (Remark 3.2) and one pass runs */
  int symmetric;          /* 1: R = P^T, P from Algorithm 1 on A (the symmetric diffusion runs
                             of Section 4.1); 0: R from Algorithm 1 on A^T (Section 3.1.3) */
  int krylov;             /* CLAIR_KRYLOV_FGMRES (right-preconditioned flexible GMRES) or
                             CLAIR_KRYLOV_PCG (preconditioned CG: symmetric A, symmetric = 1,
                             post_weighted = 1) */
} clair_params;

typedef struct clair_hierarchy* clair_h;

/* Summary of a hierarchy (host struct filled by clair_stats). */
typedef struct {
  int levels;                 /* number of levels including the coarsest */
  int64_t n[32];              /* unknowns per level */
  int64_t nnz[32];            /* nnz(A_k) per level */
  int64_t nnz_R[32];          /* nnz(R_k) including the identity entries */
  int64_t nnz_P[32];          /* nnz(P_k) including the identity entries */
  double omega[32];           /* relaxation weight per level */
  double operator_complexity; /* sum_k nnz(A_k) / nnz(A_0) (Section 4) */
  int64_t r_rows;             /* local systems solved for R over all levels */
  int64_t p_cols;             /* local systems solved for P over all levels */
  int64_t t_hist[9];          /* local systems (R and P) with T <= 8, 16, 32, 64, 128, up to
                                 224 (FP32) / 160 (FP64), up to 4096 (entries 0-6; the last
                                 two on global tiles) */
  int64_t singular_blocks;    /* local blocks with a zero pivot */
  int64_t empty_constraints;  /* F-points skipped by the projection (no C-point or B_c = 0) */
  double setup_ms;            /* device time of the last clair_setup */
  /* Device time per phase (CUDA events on the launching stream).  Index: 0 transpose,
   * strength and splitting; 1 Arnoldi weight; 2 mode smoothing; 3 patterns; 4 local
   * gathers and solves; 5 constraint projection; 6 Galerkin product; 7 coarsest inverse;
   * 8 V-cycles; 9 FGMRES orthogonalisation and residuals. */
  double phase_ms[10];        /* of the setup (entries 0-7) */
  double solve_phase_ms[10];  /* of the last clair_solve (entries 8-9) */
  double lsolve_flops;        /* sum over local systems of (2/3) T^3 + 2 T^2 */
  double lsolve_min_bytes;    /* 12 nnz(A_k) per side (A read once) + 12 nnz(R_k) + 12 nnz(P_k) */
  int64_t lsolve_gathered;    /* A entries read by the local gathers, repeats included */
  int64_t fp64_cycle_from;    /* last clair_solve in CLAIR_MIXED: iteration from which the
                                 FP64 cycle took over (a restart cycle ended unconverged or
                                 produced a nonfinite estimate), -1 if it never did */
  int k;                      /* mode vectors (columns of B, B_P and B_R) */
  int lsolve_kind_b1;         /* configuration of the last persistent local-solve launch */
  int lsolve_kind_b3;
  int lsolve_blocks_per_sm;   /* (see clair_lsolve_config) */
  int lsolve_tuned;
  int cycle_short_lanes;      /* FP32 cycle row kernels: 2 = about eight entries per lane (one
                                 thread per row up to 16 entries), 1 = about four (one thread
                                 up to 8), 0 = lanes up to the mean row length; all three are
                                 timed on the first MIXED hierarchy of the process on each
                                 device and the fastest kept */
  int cycle64_from;           /* CLAIR_MIXED: first level whose part of the cycle runs in FP64
                                 (its largest |R| or |P| weight, or a finer level's, is above
                                 1e3: FP32 copies of such weights lose their sums to
                                 cancellation), -1 if every level runs in FP32 */
  double level_span_ms[32];   /* setup: main-stream time from the start of level k to the next */
  double level_phase_ms[32][8]; /* setup: device time of phases 0-7 (see phase_ms) per level */
} clair_stats_t;

/* Kernel launches issued by this library in this process so far (monotonic counter). */
int64_t clair_kernel_launches(void);

/* The GPU architecture the library's device code was compiled for, as nvcc's
 * __CUDA_ARCH_LIST__ value (1030 for sm_103a).  Needs no GPU. */
int clair_compiled_arch(void);

/* Execution configuration of the persistent local-solve launch (not in the paper: how
 * the batched local solves are mapped onto the GPU) for one precision on the current
 * device.  Systems of up to 64 unknowns of both sides of a level run in one persistent
 * launch; those with 8 < T <= 16 go to 16-lane groups (kind_b1 = 1) or to one warp each
 * (kind_b1 = 2); those with 32 < T <= 64 to a pair of warps (kind_b3 = 3) or to one warp
 * with two rows per lane (kind_b3 = 4); blocks_per_sm caps the resident blocks (0 = as
 * many as fit).  The first setup with a large enough level times the candidates and keeps
 * the fastest (tuned = 1).  set = 1 installs the given values (tuned is stored as given; 2
 * marks a caller's choice, which the library then keeps); set = 0 reads them.
 * CLAIR_ERR_ARG for other kinds or a negative block count. */
clair_status clair_lsolve_config(int precision, int set, int* kind_b1, int* kind_b3,
                                 int* blocks_per_sm, int* tuned);

/* Fills *p with the defaults listed above. */
clair_status clair_params_default(clair_params* p);

/* CLAIR setup (hot path, part 1): per level, strength, C/F splitting, relaxation weight,
 * mode smoothing, pattern, batched local solves and constraint projection for R (on A^T,
 * Section 3.1.3) and P (on A, Algorithm 1), then A_c = R A P (Section 1), until
 * n <= coarse_max or max_levels.
 *   n, nnz, rowptr, col, val : the fine operator A (device CSR, see conventions)
 *   k                        : number of mode vectors, 1 <= k <= CLAIR_KMAX (Eq. 3.3: the
 *                              constraint W B_c = B|_F holds for every column)
 *   B                        : device float64 [n x k], column-major (mode a at B + a n): the
 *                              near-nullspace candidates, e.g. the constant vector (k = 1)
 *   cf_marker                : NULL, or device int8 [n] with 1 = C-point, 0 = F-point: the
 *                              caller's fine-level splitting, used instead of the library's
 *                              (coarser levels are split by the library; FC coarsening only,
 *                              CLAIR_ERR_UNSUPPORTED with CLAIR_COARSEN_AGG)
 *   p                        : host parameters (NULL = defaults)
 *   out                      : receives the new hierarchy; *out = NULL on failure
 * Synchronises `stream` once per level (coarse sizes are data-dependent). */
clair_status clair_setup(int n, int nnz, const int* rowptr, const int* col,
                         const double* val, int k, const double* B, const signed char* cf_marker,
                         const clair_params* p, void* stream, clair_h* out);

/* Solve A U = F for nrhs right-hand sides (hot path, part 2): per right-hand side (and per
 * instance of a batch) an independent Krylov process in float64, all of them advancing in
 * lockstep so that they share every kernel launch: right-preconditioned FGMRES(gmres_restart)
 * (or preconditioned CG with CLAIR_KRYLOV_PCG) with one V(1,1) cycle (CFF pre, FFC post,
 * Section 4) per iteration, FP32 cycle in CLAIR_MIXED mode.  Each process stops on its own
 * true float64 residual ||f_r - A u_r||_2 <= rtol ||f_r||_2 (restarts = iterative
 * refinement).  In CLAIR_MIXED mode a restart cycle that uses all gmres_restart iterations
 * without converging, stalls (less than 2x in the worst residual estimate over 10
 * iterations) or gives a nonfinite estimate switches the rest of the solve to the FP64
 * cycle of the same hierarchy (flexible GMRES admits the change; see
 * clair_stats_t.fp64_cycle_from).
 *   f      : device float64 [nrhs x n], right-hand side r at f + r n
 *   u      : device float64 [nrhs x n]; input initial guesses, output solutions
 *   nrhs   : number of right-hand sides (>= 1)
 *   iters, relres : host arrays [nrhs] (may be NULL): iterations and final
 *            ||f_r - A u_r|| / ||f_r|| per right-hand side (for a batch, the largest over
 *            its instances; clair_solve_detail gives every instance)
 * Returns CLAIR_ERR_NOT_CONVERGED if any process reached gmres_maxit above rtol (u holds
 * the last iterates).  Synchronises `stream` once per iteration. */
clair_status clair_solve(clair_h h, const double* f, double* u, int nrhs, void* stream,
                         int* iters, double* relres);

/* Per-process results of the last clair_solve on h: *nseg = nrhs * ninst; iters_host and
 * relres_host (host arrays [nseg], may be NULL) receive, for right-hand side r and
 * instance i at index r * ninst + i, its iteration count and final relative residual. */
clair_status clair_solve_detail(clair_h h, int* nseg, int* iters_host, double* relres_host);

/* One V(1,1) cycle x = M^-1 b on level `level` (x0 = 0), in the hierarchy's precision.
 *   b, x : device float64 [n_level]. */
clair_status clair_vcycle(clair_h h, int level, const double* b, double* x, void* stream);

/* Host summary of the hierarchy. */
clair_status clair_stats(clair_h h, clair_stats_t* out);

/* Device views of level `level`, valid until clair_free.  Any output pointer may be NULL.
 * For the coarsest level only n, nnz and the A arrays are set (the others NULL / 0).
 *   A_*   : CSR of A_k (n x n)
 *   R_*   : CSR of R_k (nc x n), identity entry stored at each C-point's own column
 *   P_*   : CSR of P_k (n x nc), identity entry stored in each C-point's row
 *   cf    : int8 [n] C/F splitting;  B_P, B_R: float64 [n x k] (column-major, k from
 *           clair_stats) smoothed mode vectors for P (operator A_k) and R (operator
 *           A_k^T; equal to B_P when symmetric = 1);  omega: host scalar weight. */
clair_status clair_level_view(clair_h h, int level, int* n, int* nc, int* nnz_A,
                              const int** A_rowptr, const int** A_col, const double** A_val,
                              int* nnz_R, const int** R_rowptr, const int** R_col,
                              const double** R_val, int* nnz_P, const int** P_rowptr,
                              const int** P_col, const double** P_val,
                              const signed char** cf, const double** B_P,
                              const double** B_R, double* omega);

/* Releases every device buffer of the hierarchy.  NULL is accepted. */
clair_status clair_free(clair_h h);

/* Batched constrained local solves for given splitting and pattern (hot path steps
 * local gather, local solve, constraint projection and scatter; Eqs. 2.8 and 3.1,
 * Algorithm 1 with exact block inverses and k = 1, Remark 3.2, constraint Eq. 3.3).
 * Computes the weights of P_hat = [W; I] for Algorithm 1 run on the operator Ahat,
 * stored transposed: row i of the output is coarse point i, i.e. for Ahat = A^T this is
 * directly the CSR of the restriction R.
 *   n, Ahat_rowptr/col/val : the operator Algorithm 1 runs on (device CSR)
 *   cf                     : device int8 [n] splitting
 *   nc, Z_rowptr, Z_col    : device CSR pattern (nc x n), rows = coarse points, columns
 *                            sorted, each row containing its own C-point column (identity)
 *                            and the F-points of its local system (at most 4096 of them)
 *   B                      : device float64 [n] mode vector on the fine points
 *   precision              : CLAIR_FP64 (float64 local solves) or CLAIR_MIXED (float32)
 *   Z_val                  : device float64 [nnz] output weights (1 at identity entries)
 *   singular_out, empty_out: host counts of zero-pivot blocks and skipped F-points (NULL ok)
 * The projection needs the column view of the pattern; the call allocates it
 * (stream-ordered) and releases it before returning. */
clair_status clair_local_weights(int n, const int* Ahat_rowptr, const int* Ahat_col,
                                 const double* Ahat_val, const signed char* cf, int nc,
                                 const int* Z_rowptr, const int* Z_col, const double* B,
                                 int precision, double* Z_val, void* stream,
                                 int64_t* singular_out, int64_t* empty_out);

/* Size of the one static device scratch array used by clair_local_weights_noalloc. */
#define CLAIR_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* clair_local_weights without any device memory allocation.  The paper has no
 * counterpart: this is a deployment variant of the same computation, with the same
 * arguments, results (bit for bit: the same kernels in the same order) and error codes as
 * clair_local_weights, except that local systems of more than 128 unknowns (which need a
 * per-call tile buffer) are refused with CLAIR_ERR_CAPACITY.  Every refusal happens
 * before the call writes anything: Z_val is then left untouched.
 *
 * It exists for callers that cannot let a library allocate device memory while they run:
 * applications whose device memory is entirely reserved up front by their own pool or by
 * a framework's caching allocator (an extra cudaMalloc would either fail or bypass the
 * pool's accounting), and latency-critical loops that cannot afford cudaMalloc/cudaFree,
 * which may synchronise the device and take unbounded time.  The caller still provides
 * every input and output buffer.
 *
 * Temporaries come from one file-scope device array of CLAIR_NOALLOC_SCRATCH_BYTES
 * (32 MiB).  Every GPU that loads the library keeps that array until the process exits.
 * A call needs about 16 n + 28 nc + 16 nnz(Z) bytes plus 256-byte alignment per piece;
 * when that exceeds the limit the call returns CLAIR_ERR_CAPACITY, names the sizes, and
 * leaves Z_val untouched (use clair_local_weights for larger problems).
 * The first call on a device looks up the array's device address with that device
 * current; make that first call before starting any stream capture on the device.
 * All calls share the one array and it keeps the last call's contents (every counter is
 * cleared at the start of a call): calls that overlap on the GPU, from other streams or
 * other host threads, race on it and corrupt each other's results, so serialise them.
 * The call synchronises `stream`. */
clair_status clair_local_weights_noalloc(int n, const int* Ahat_rowptr, const int* Ahat_col,
                                         const double* Ahat_val, const signed char* cf, int nc,
                                         const int* Z_rowptr, const int* Z_col, const double* B,
                                         int precision, double* Z_val, void* stream,
                                         int64_t* singular_out, int64_t* empty_out);

/* ---- Batches of independent problems ----------------------------------------------
 * Many instances A_i u_i = f_i (not in the paper; its method applied to each instance)
 * set up and solved together as one block-diagonal operator, so every step of the setup
 * (strength, splitting, patterns, the bucketed local solves of Algorithm 1, the
 * projection, the Galerkin product) and every V-cycle kernel is one launch for the whole
 * batch.  Each instance's hierarchy equals the one clair_setup builds for it alone (up
 * to the summation order of its relaxation weight): splitting keys use instance-local
 * indices, each instance gets its own Arnoldi weight (Section 4) from its own start
 * vector, and an instance that reaches n_i <= coarse_max (or max_levels, or a splitting
 * with no C- or no F-point) is frozen: identity transfers and zero relaxation weight
 * until the batch's coarsest level, where each instance's diagonal block is inverted. */

/* Setup of a batch: A is the block-diagonal CSR of all instances, instance i owning rows
 * and columns offsets_host[i] .. offsets_host[i+1]-1.
 *   ninst, offsets_host : host int [ninst + 1], offsets_host[0] = 0, offsets_host[ninst]
 *                         = n, strictly increasing
 *   other arguments     : as clair_setup (B and cf_marker concatenated over the instances)
 * CLAIR_ERR_ARG if an entry couples two instances or the offsets are invalid;
 * CLAIR_ERR_UNSUPPORTED if arnoldi_iters > 15.  clair_solve on the result solves all
 * instances at once: one Krylov process per instance (and right-hand side), each stopping
 * at rtol relative to its own ||f_i||, all sharing the V-cycle and vector launches. */
clair_status clair_setup_batched(int ninst, const int* offsets_host, int n, int nnz,
                                 const int* rowptr, const int* col, const double* val, int k,
                                 const double* B, const signed char* cf_marker,
                                 const clair_params* p, void* stream, clair_h* out);

/* Per-instance view of level `level` of a hierarchy (a single-problem hierarchy reports
 * one instance).  Output pointers are host arrays and may be NULL:
 *   ninst        : number of instances
 *   offsets_host : int [ninst + 1], the instances' row ranges on this level
 *   omega_host   : double [ninst], relaxation weight of each instance on this level
 *   frozen_host  : int8 [ninst], 1 where the instance is frozen (its coarsest level was
 *                  reached) on this level */
clair_status clair_batch_view(clair_h h, int level, int* ninst, int* offsets_host,
                              double* omega_host, signed char* frozen_host);

/* ---- Adjoint path: gradients of a loss of the solutions -----------------------------
 * The paper solves A u = f (Section 1).  For a loss L(u_1..u_k) of several solutions, the
 * implicit-function theorem gives A^T lam_r = dL/du_r and dL/da_ij = -sum_r lam_r[i] u_r[j]
 * on the stored entries of A.  The adjoint operator A^T is nonsymmetric like A and gets
 * its own CLAIR hierarchy (R from A, P from A^T: Section 3.1.3 run on A^T). */

/* Hierarchy for A^T: transposes the fine operator of `fwd` on the device and runs
 * clair_setup on it with fwd's parameters and fwd's (unsmoothed) mode vectors.
 *   fwd : a hierarchy from clair_setup (not modified)
 *   adj : receives the new hierarchy (owned by the caller, release with clair_free);
 *         *adj = NULL on failure
 * Same errors as clair_setup; synchronises `stream`. */
clair_status clair_setup_adjoint(clair_h fwd, void* stream, clair_h* adj);

/* Operator gradient sampled on the sparsity of A:
 *   dA[e] = -sum_{r=0}^{nrhs-1} lambda[r*n + row(e)] * u[r*n + col(e)]
 * for every stored entry e of A in its CSR order (sum in increasing r, float64).
 *   n, nnz, rowptr, col : device CSR pattern of A (validated)
 *   lambda, u           : device float64 [nrhs * n], RHS-major (vector r contiguous):
 *                         the adjoint and state solutions
 *   dA                  : device float64 [nnz], written
 * CLAIR_ERR_ARG on null pointers, bad sizes or an invalid pattern. Asynchronous after
 * validation (which synchronises `stream` once). */
clair_status clair_sddmm_grad(int n, int nnz, const int* rowptr, const int* col, int nrhs,
                              const double* lambda, const double* u, double* dA, void* stream);

/* Chain rule from the entries of the 5-point first-order upwind finite-difference operator
 * of the Section 4.2 advection-diffusion problem (Eq. 4.1) to its per-node fields. The
 * grid is nside x nside interior nodes (x fastest) with spacing h and Dirichlet values
 * eliminated. The interior face between nodes k and Q carries
 * e_f = 2 e_k e_Q / (e_k + e_Q) (a boundary face carries e_k). Row k holds
 * sum_f e_f/h^2 + (|vx_k| + |vy_k|)/h on the diagonal, -e_f/h^2 on each neighbour, and
 * -max(vx_k,0)/h west, -max(-vx_k,0)/h east, -max(vy_k,0)/h south, -max(-vy_k,0)/h
 * north.
 *   eps, vx, vy          : device float64 [nside^2], the fields A was assembled from
 *   rowptr, col, nnz, dA : device CSR pattern of A and dL/da on it (e.g. from
 *                          clair_sddmm_grad)
 *   deps, dvx, dvy       : device float64 [nside^2], written: dL/d eps_k, dL/d vx_k,
 *                          dL/d vy_k. The derivative of |v| is taken as sign(v), 0 at
 *                          v = 0, where the upwind operator is not differentiable. Entries
 *                          not stored in A contribute nothing.
 * CLAIR_ERR_ARG on null pointers, bad sizes, an invalid pattern or a column outside the
 * 5-point stencil. Synchronises `stream`. */
clair_status clair_advdiff2d_param_grad(int nside, double h, const double* eps, const double* vx,
                                        const double* vy, const int* rowptr, const int* col,
                                        int nnz, const double* dA, double* deps, double* dvx,
                                        double* dvy, void* stream);

/* Sparse product C = A B (the building block of the Galerkin step A_c = (R A) P, Section
 * 1): deterministic sums (each output entry adds its products in A's row order, in
 * float64, with separate multiply and add), columns of each output row sorted, exact
 * zeros kept.  Rows are routed by their distinct-column count through shared-memory hash
 * tables of growing size and, beyond 16384 columns, a dense accumulator in global memory.
 *   m, kdim, ncols : A is m x kdim, B is kdim x ncols (device CSR, see conventions)
 *   rowptr_out     : device int [m + 1], written: C's row pointers
 *   nnz_out        : host, written: nnz(C)
 *   col_out, val_out : device buffers of at least *cap entries (cap: host, in), or NULL
 *                    to query the size only; CLAIR_ERR_CAPACITY if nnz(C) > cap
 * Synchronises `stream`. */
clair_status clair_spgemm(int m, int kdim, int ncols, const int* A_rowptr, const int* A_col,
                          const double* A_val, const int* B_rowptr, const int* B_col,
                          const double* B_val, void* stream, int* rowptr_out, int64_t* nnz_out,
                          int64_t cap, int* col_out, double* val_out);

/* One-line description of the last error on the calling thread ("" if none). */
const char* clair_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CLAIR_H */
