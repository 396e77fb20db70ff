/*
 * sfcdd -- two-level overlapping Schwarz solver on space-filling-curve
 * subdomains (Griebel, Schweitzer, Troska, "A dimension-oblivious domain
 * decomposition method based on space-filling curves", arXiv 2110.11211),
 * GB300 (sm_103a) implementation.
 *
 * Problem (Sec. 3.3, eq. dof; Sec. 4): the d-dimensional finite-difference
 * operator on the interior points k_j = 1..2^{l_j}-1 of an anisotropic grid,
 *   (A u)_k = sum_j c_j 4^{l_j} (2 u_k - u_{k-e_j} - u_{k+e_j}),  zero Dirichlet,
 * N = prod_j (2^{l_j} - 1) unknowns.
 *
 * Conventions shared by every entry point:
 *  - Vectors handed to the library are FP64, length N, in LEXICOGRAPHIC order
 *    (last axis fastest, i.e. a C-contiguous array of shape (2^{l_1}-1, ...,
 *    2^{l_d}-1)), unless the argument name ends in _curve (curve order).
 *  - Pointers whose name ends in _dev are device pointers on the current CUDA
 *    device; _host pointers are host memory.  The caller owns every buffer it
 *    passes; the library never frees them and keeps no reference after return.
 *  - The handle owns all factors, permutations and work buffers (device memory
 *    allocated in setup, freed by sfcdd_destroy).
 *  - Work is issued on the stream given in sfcdd_options (NULL = the legacy
 *    default stream) and is stream-ordered; functions that return results to
 *    host memory synchronise that stream before returning.
 *  - Return value: SFCDD_OK (0) or a negative sfcdd_status.  A handle is not
 *    thread-safe; distinct handles are independent.
 */
#ifndef SFCDD_H
#define SFCDD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfcdd_handle sfcdd_handle;

enum sfcdd_status {
  SFCDD_OK = 0,
  SFCDD_ERR_INVALID_ARG = -1,  /* d < 1, d > 8, l_j < 1, P < 2, gamma <= 0, 2 floor(gamma)+1 >= P,
                                  q outside 1..floor(N/P), a subdomain longer than N, NULL pointer */
  SFCDD_ERR_KEY_OVERFLOW = -2, /* d * max_j l_j > 64: the Hilbert key does not fit 64 bits (Sec. 4.3) */
  SFCDD_ERR_NOMEM = -3,        /* device allocation failed (dense local factors larger than free HBM) */
  SFCDD_ERR_NOT_SPD = -4,      /* non-positive Cholesky pivot; fail_index = matrix (P = coarse) */
  SFCDD_ERR_MAXIT = -5,        /* PCG did not reach rtol within maxit iterations */
  SFCDD_ERR_NAN = -6,          /* NaN / Inf in the PCG recurrences */
  SFCDD_ERR_TIMEOUT = -7,      /* a bounded device-side wait gave up (error word set by a kernel) */
  SFCDD_ERR_CUDA = -8,         /* a CUDA runtime call failed */
  SFCDD_ERR_UNSUPPORTED = -9   /* grid too large for 32-bit point codes (sum_j l_j > 31) */
};

enum sfcdd_precision { SFCDD_FP64 = 0, SFCDD_FP32 = 1, SFCDD_BF16 = 2 };
enum sfcdd_variant { SFCDD_ADDITIVE = 0, SFCDD_BALANCED = 1, SFCDD_ONE_LEVEL = 2, SFCDD_COARSE_ONLY = 3 };
enum sfcdd_weighting { SFCDD_WEIGHT_NONE = 0, SFCDD_WEIGHT_OMEGA = 1 };
enum sfcdd_method { SFCDD_METHOD_PCG = 0, SFCDD_METHOD_RICHARDSON = 1 };

typedef struct {
  const double* coeffs; /* host, length d: per-axis c_j; NULL = all ones */
  int q;                /* coarse dofs per subdomain (eq. restr); <= 0: 2^{floor(log2 floor(N/P)) - 4},
                           clamped to 1..floor(N/P) (the "four levels coarser" rule of Sec. 4) */
  int variant;          /* sfcdd_variant: eq. addSW (default), eq. balSW, eq. w1levprec, coarse term only */
  int weighting;        /* sfcdd_weighting: D_i = omega_i I with eq. omegai (default) or D_i = I */
  int precision;        /* sfcdd_precision of the local factors and local solves (FP64 default);
                           the coarse factor, the stencil and the PCG recurrences stay FP64 */
  int flexible;         /* PCG beta: 0 = r^T z ratio, 1 = Polak-Ribiere (flexible CG, Sec. 3.3),
                           < 0 = automatic (flexible for FP32 / BF16 local factors) */
  void* stream;         /* cudaStream_t for all work of this handle; NULL = legacy default stream */
  int profile;          /* != 0: time every kernel launch of setup and solves with CUDA events
                           (see sfcdd_set_profiling); 0 (default): no events */
  int local_order;      /* numbering of the unknowns inside each subdomain for its Cholesky
                           factor: 0 (default) lexicographic grid order (a fill-reducing order:
                           the factor's envelope shrinks to a band), 1 ascending curve position.
                           A_i^{-1} and therefore the preconditioner are the same either way. */
  int slabs_local;      /* work items of the local substitutions.  1, 2 or 4: row slabs per
                           64-row tile row (rows of 64, 32, 16), one CTA each, chained through
                           result slots in L2; splitting shortens the GEMV on the dependency
                           chain from one tile row to the next.  -1: one CTA per local matrix
                           sweeping all its tile rows, chained through shared memory (the
                           matrix vector must fit beside the stream ring: local matrices of
                           at most 189 tile rows with FP64 factors, 317 with FP32, 380 with
                           BF16; INVALID_ARG otherwise).
                           0 (default): -1 where the local matrices allow it, else 1.
                           sfcdd_autotune picks it by measurement. */
  int slabs_coarse;     /* the same for the coarse substitutions: 1, 2 or 4; 0 (default) = 2.
                           FP32 / BF16 local factors require 2 or 4 (INVALID_ARG otherwise). */
  int tensor_cores;     /* the panel and trailing-update tile products of the local and coarse
                           factorizations on the tensor cores (tcgen05) when 1, 2 or -1
                           (default), on CUDA cores when 0.  FP32 local factors: TF32 operands
                           with the hi/lo split, FP32 accumulation (FP32-accurate).  BF16 local
                           factors: bf16 operands with FP32 accumulation (kind::f16; FP32
                           working tiles and diagonal tiles; the BF16 factorization) when 1 or
                           -1; with 2 the FP32-accurate TF32 split, the factor rounded to bf16
                           afterwards.  FP64 factors: exact 8-bit digit slices of each row
                           (Ozaki, Ogita, Oishi and Rump's error-free splitting) multiplied as
                           bf16 with exact FP32 accumulation, combined in integers and rounded
                           once to FP64. */
  int coarse_block;     /* tiles per unit diagonal block of the coarse substitution form
                           (L = Lh blockdiag(D_J), Sec. 3.1 solves): 1, 2, 4 or 8; 0 (default)
                           = 4.  Larger blocks shorten the coarse substitutions' dependency
                           chain (nt0 / coarse_block steps) at the price of inverting larger
                           diagonal blocks in the setup. */
} sfcdd_options;

typedef struct {
  int iters;            /* PCG iterations = preconditioner applies */
  int status;           /* sfcdd_status of the call */
  int fail_index;       /* NOT_SPD: failing matrix index; TIMEOUT: kernel site */
  int reserved;
  double rel_res;       /* recurrence residual ||r_k|| / ||b|| at exit */
  double true_rel_res;  /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
  double setup_ms;      /* device time of sfcdd_setup (keys, sort, partition, factors) */
  double solve_ms;      /* device time of the PCG loop of the last solve */
} sfcdd_stats;

typedef struct {
  long long N;          /* unknowns, eq. dof */
  long long N0;         /* coarse dofs q * P */
  int d, P, q, nbits;   /* nbits = max_j l_j (curve resolution, Sec. 3.3) */
  int tile;             /* tile edge of the packed local factors */
  int precision, variant, weighting, flexible;
  long long factor_bytes; /* bytes of the local factor tiles, both substitution copies:
                             Lh (read by the forward sweep) and Lh^T with E_K (backward) */
  long long coarse_bytes; /* the same for the coarse factor (FP64) */
  double setup_ms;
} sfcdd_info;

/* Fills *opt with the defaults listed in sfcdd_options. */
void sfcdd_default_options(sfcdd_options* opt);

/* Setup phase, Algorithm 1: N from eq. (dof); Hilbert keys of all grid points
 * (Sec. 3.2, Skilling's transform at resolution max_j l_j, point k at cell
 * k_j 2^{max l - l_j}) and their radix sort into curve order (step 3); the
 * partition of eq. (sloc) and its enlargement eq. (enlarge) (steps 4-5);
 * weights eq. (omegai); dense local matrices A_i = R_i A R_i^T and their
 * Cholesky factors (Sec. 3.1, steps 6-7); coarse blocks eq. (restr), A_0 of
 * eq. (csm) and its FP64 Cholesky factor (steps 9-10).
 * levels: host array of d levels l_j >= 1.  overlap: gamma of eq. (enlarge).
 * On success *out receives a new handle.  Errors: INVALID_ARG, KEY_OVERFLOW,
 * UNSUPPORTED, NOMEM, NOT_SPD, CUDA, TIMEOUT. */
int sfcdd_setup(const int* levels, int d, int P, double overlap, sfcdd_handle** out);
int sfcdd_setup_ex(const int* levels, int d, int P, double overlap, const sfcdd_options* opt,
                   sfcdd_handle** out);

/* Solve A u = f by PCG (Sec. 3.3) preconditioned with the operator chosen in
 * the options (default eq. addSW applied as in Algorithm 2), x_0 = 0, until
 * ||r_k|| <= rtol ||f|| or maxit iterations.  f_dev, u_dev: device, length N,
 * lexicographic.  stats may be NULL.  Synchronises the handle's stream.
 * Errors: INVALID_ARG, MAXIT (u holds the last iterate), NAN, TIMEOUT, CUDA. */
int sfcdd_solve(sfcdd_handle* h, const double* f_dev, double* u_dev, double rtol, int maxit,
                sfcdd_stats* stats);

/* Same as sfcdd_solve with host buffers: copies f to the device, solves and
 * copies u back (end-to-end path). */
int sfcdd_solve_host(sfcdd_handle* h, const double* f_host, double* u_host, double rtol, int maxit,
                     sfcdd_stats* stats);

/* Adjoint of a solve, for L(u) with u = A(c)^{-1} f (no counterpart in the
 * paper; A is symmetric so the adjoint solve reuses the factors and PCG):
 *   lambda = A^{-1} gu,  dL/df = lambda,  dL/dc_j = -lambda^T (dA/dc_j) u
 * with dA/dc_j the axis-j term 4^{l_j}(2u_k - u_{k-e_j} - u_{k+e_j}).
 * u_dev: the forward solution, gu_dev: dL/du, gf_dev: receives dL/df (all
 * device, length N, lexicographic); gc_host: receives d doubles dL/dc_j.
 * Synchronises the stream.  Errors as sfcdd_solve. */
int sfcdd_solve_backward(sfcdd_handle* h, const double* u_dev, const double* gu_dev, double* gf_dev,
                         double* gc_host, double rtol, int maxit, sfcdd_stats* stats);

/* Estimates of the extreme eigenvalues lambda_min, lambda_max of C^{-1} A (the
 * numbers that give the optimal Richardson damping of eq. redrate): Ritz
 * values of the Lanczos tridiagonal formed from the coefficients of a PCG run
 * on f (at most `steps` iterations, to relative residual 1e-14).  They lie
 * inside [lambda_min, lambda_max] and converge to its ends as steps grows.
 * f_dev: device, length N, lexicographic (not modified).  Synchronises the
 * stream.  Errors: INVALID_ARG (also f = 0), NAN, TIMEOUT, CUDA. */
int sfcdd_estimate_spectrum(sfcdd_handle* h, const double* f_dev, int steps, double* lmin,
                            double* lmax);

/* Algorithm 3: the preconditioned damped linear (Richardson) iteration
 * x^{k+1} = x^k + xi C^{-1} (f - A x^k), x^0 = 0, with the handle's
 * preconditioner (additive, balanced, ...), until ||f - A x^k|| <= rtol ||f||
 * (recomputed every step) or maxit updates.  xi > 0; the optimal damping is
 * xi* = 2 / (lambda_min + lambda_max) (eq. redrate).  stats->iters = number of
 * updates.  Synchronises the stream.  Errors as sfcdd_solve. */
int sfcdd_richardson(sfcdd_handle* h, const double* f_dev, double* u_dev, double xi, double rtol,
                     int maxit, sfcdd_stats* stats);

/* The convergence protocol of Sec. 4: the homogeneous problem A x = 0 (f = 0,
 * solution 0), so every iterate x^k is its own error, measured in the energy
 * norm ||x^k||_A = sqrt(x^k^T A x^k).  Starts from x0_dev (device, length N,
 * lexicographic, not modified; the paper draws it from U[-1,1] and rescales to
 * ||x^0||_A = 1, which this relative test makes unnecessary) and iterates until
 * ||x^K||_A <= tol ||x^0||_A or maxit updates.
 *   method SFCDD_METHOD_PCG:        preconditioned CG with the handle's
 *     preconditioner; the energy norm comes from the recurrence residual,
 *     ||x^k||_A^2 = -x^k^T r^k (r^k = -A x^k), fused into the update.
 *   method SFCDD_METHOD_RICHARDSON: Algorithm 3 with damping xi > 0 (xi is
 *     ignored for PCG); the energy norm is recomputed from A x^k every step.
 * u_dev (device, length N, lexicographic) receives x^K.  stats->iters = K
 * (updates of x), stats->rel_res = ||x^K||_A / ||x^0||_A as the stopping test
 * saw it, stats->true_rel_res = the same ratio recomputed from A x^K.
 * x^0 = 0 returns at once with K = 0.  Synchronises the stream.
 * Errors: INVALID_ARG (null pointers, tol < 0, maxit < 0, unknown method,
 * xi <= 0 for Richardson), MAXIT, NAN, TIMEOUT, CUDA. */
int sfcdd_solve_homogeneous(sfcdd_handle* h, const double* x0_dev, double* u_dev, int method,
                            double xi, double tol, int maxit, sfcdd_stats* stats);

/* ---- Batched solves: many independent subgrid problems ----
 * The subproblems of the sparse-grid combination technique (Sec. 2: one
 * anisotropic full grid per level vector l, solved independently), all with the
 * same d, P, overlap and options, set up together and solved in ONE CUDA-graph
 * launch: a conditional WHILE node repeats the PCG iteration of every subgrid
 * until each has converged (its own scalars and converged flag) or maxit.
 * levels: host array nsub x d (subgrid s uses levels[s*d .. s*d+d-1]).
 * Vectors: the concatenation of the subgrids' vectors, each lexicographic, at
 * the offsets returned by sfcdd_batch_offsets (nsub + 1 entries, last = total).
 * Supported options: precision, weighting, q (<= 0: per-subgrid rule), flexible,
 * coeffs (shared), stream, slabs_local / slabs_coarse (defaults 1 and 1 for FP64,
 * 1 and 4 otherwise; slabs_local -1: one CTA per local matrix), tensor_cores,
 * variant SFCDD_ADDITIVE or SFCDD_BALANCED
 * (eq. balSW: two coarse solves and one local solve per apply; else UNSUPPORTED).
 * At most 65535 subgrids (UNSUPPORTED beyond); any number of local matrices.
 * Errors as sfcdd_setup_ex / sfcdd_solve; per_sub (nsub entries) and total may
 * be NULL; total->iters is the largest iteration count, total->fail_index the
 * number of subgrids that did not converge. */
typedef struct sfcdd_batch sfcdd_batch;
int sfcdd_batch_setup(const int* levels, int nsub, int d, int P, double overlap,
                      const sfcdd_options* opt, sfcdd_batch** out);
/* As sfcdd_batch_setup with a subdomain count per subgrid: P (host, nsub
 * entries, each >= 2 and <= that subgrid's N), e.g. eq. Pchoice,
 * P = P_hat 2^{d-1-i} for the subgrids of layer i of eq. combi. */
int sfcdd_batch_setup_each(const int* levels, const int* P, int nsub, int d, double overlap,
                           const sfcdd_options* opt, sfcdd_batch** out);
int sfcdd_batch_offsets(const sfcdd_batch* b, long long* offsets_host);
int sfcdd_batch_solve(sfcdd_batch* b, const double* f_dev, double* u_dev, double rtol, int maxit,
                      sfcdd_stats* per_sub, sfcdd_stats* total);
/* total unknowns, bytes of all factor tiles (local + coarse), setup device time */
int sfcdd_batch_info(const sfcdd_batch* b, long long* n_total, long long* factor_bytes,
                     double* setup_ms);
int sfcdd_batch_destroy(sfcdd_batch* b);

/* The combination formula eq. combi evaluated at points: for every point x_p
 *   out[p] = sum_s coef[s] * (I_s u_s)(x_p),
 * where u_s is subgrid s's solution (device, the concatenated lexicographic
 * vectors of sfcdd_batch_solve, offsets from sfcdd_batch_offsets) and I_s the
 * piecewise multilinear interpolant on its grid (nodes k_j 2^{-l_j},
 * k_j = 0..2^{l_j}, zero on the boundary nodes).  coef (host, nsub): the
 * combination coefficient of each subgrid, (-1)^i C(d-1, i) for layer i.
 * points (device, npts x d, row-major, coordinates clamped to [0, 1]);
 * out (device, npts).  One warp per point, a fixed summation order: repeated
 * calls give identical results.  Synchronises the batch's stream.
 * Errors: INVALID_ARG (null pointers, npts < 0, NaN coefficient), CUDA. */
int sfcdd_batch_combine(sfcdd_batch* b, const double* coef_host, const double* u_dev,
                        const double* points_dev, long long npts, double* out_dev);

/* y = A x (the matrix-free stencil, Sec. 4).  curve_order = 0: x, y
 * lexicographic; 1: x, y in curve order (no permutation, the hot-path form). */
int sfcdd_apply_operator(sfcdd_handle* h, const double* x_dev, double* y_dev, int curve_order);

/* z = C^{-1} g for the handle's preconditioner (Algorithm 2 for eq. addSW:
 * g_i = R_i g, A_i d_i = g_i, A_0 d_0 = R_0 g, z = R_0^T d_0 + sum_i omega_i R_i^T d_i;
 * eq. balSW adds the two coarse corrections and stencil applies of G).
 * curve_order as in sfcdd_apply_operator. */
int sfcdd_apply_precond(sfcdd_handle* h, const double* g_dev, double* z_dev, int curve_order);

/* Autotuner of the substitution shapes (what a work item of the batched
 * triangular solves covers: for the local factors a whole matrix, where its
 * vector fits the shared memory, or a row slab of 64, 32 or 16 rows; for the
 * coarse factor a row slab).  Times `reps` preconditioner applies (device time,
 * CUDA events, after two warm-up applies) for every admissible (slabs_local,
 * slabs_coarse) pair, keeps the fastest in the handle and reports it.  The
 * preconditioner's values do not depend on the choice beyond rounding (whole-
 * matrix items sum each row in another order).  Drops the captured iteration
 * graph (rebuilt by the next solve).  Synchronises the stream.
 * Errors: INVALID_ARG (reps < 1), TIMEOUT, CUDA. */
typedef struct {
  int slabs_local;      /* chosen slab count of the local substitutions (-1: whole matrices) */
  int slabs_coarse;     /* chosen slab count of the coarse substitutions */
  double apply_ms;      /* mean device time of one apply with the choice */
  int candidates;       /* configurations timed */
} sfcdd_tuning;
int sfcdd_autotune(sfcdd_handle* h, int reps, sfcdd_tuning* out);
/* The same for a batch (declared below): times `reps` pairs of batched forward
 * and backward substitutions over every subgrid for each slab pair and keeps
 * the fastest; drops the captured solve graph.  Errors as sfcdd_autotune. */
int sfcdd_batch_autotune(sfcdd_batch* b, int reps, sfcdd_tuning* out);

/* Failure-detection self-tests (no counterpart in the paper); neither faults,
 * traps nor hangs the GPU, and the handle stays usable afterwards.
 *   SFCDD_SELFTEST_WAIT_TIMEOUT: runs a forward substitution of the handle's
 *     factors whose first work item is never scheduled; the items depending on
 *     it poll result slots that nothing writes until their bounded spin (about
 *     4M polls) runs out, record SFCDD_ERR_TIMEOUT with the waiting site, and the
 *     remaining waiters stop on seeing the error word.  The result slots and work
 *     counters are restored afterwards.
 *   SFCDD_SELFTEST_BREAKDOWN: factors a host-built 64 x 64 tile with a negative
 *     pivot through the diagonal-tile factorization the setup uses; it must
 *     record SFCDD_ERR_NOT_SPD with the matrix index it was given (4242).
 * Returns the status the device recorded (the expected error code on success)
 * and *detail = its index or site; the error word is cleared again.
 * Synchronises the stream.  Errors: INVALID_ARG (unknown kind), CUDA. */
enum sfcdd_selftest_kind { SFCDD_SELFTEST_WAIT_TIMEOUT = 1, SFCDD_SELFTEST_BREAKDOWN = 2 };
int sfcdd_selftest(sfcdd_handle* h, int kind, int* detail);

/* Introspection for parity checks (all synchronise the stream). */
int sfcdd_get_info(const sfcdd_handle* h, sfcdd_info* info);
/* keys_dev: N uint64 Hilbert keys by lexicographic id (Sec. 3.2).
 * perm_dev: N int32, perm[pos] = lexicographic id at curve position pos (Alg. 1 step 3). */
int sfcdd_get_curve(const sfcdd_handle* h, unsigned long long* keys_dev, int* perm_dev);
/* Host arrays of length P: start_i, N_i of the cyclic ranges Omega_i (eq. enlarge,
 * 0-based curve positions) and omega_i (eq. omegai, or 1 for weighting NONE).
 * Any pointer may be NULL. */
int sfcdd_get_partition(const sfcdd_handle* h, long long* start_host, long long* len_host,
                        double* omega_host);
/* A0_dev: N0 x N0 FP64 row-major, receives A_0 = R_0 A R_0^T (eq. csm),
 * assembled again from the curve (the handle keeps only its factor). */
int sfcdd_get_coarse_matrix(const sfcdd_handle* h, double* A0_dev);
/* Ai_dev: N_i x N_i FP64 row-major, receives the dense local matrix A_i = R_i A R_i^T
 * in ascending cyclic curve order (Sec. 3.1). */
int sfcdd_get_local_matrix(const sfcdd_handle* h, int i, double* Ai_dev);

/* Kernel accounting.  Every kernel the library launches belongs to one class;
 * the handle counts launches per class (graph replays included).  With
 * profiling enabled the solve loop launches kernel by kernel on the handle's
 * stream with CUDA events around each launch and accumulates device time per
 * class; disabled (default) it replays a captured CUDA graph per iteration. */
enum sfcdd_kernel_class {
  SFCDD_K_KEYGEN = 0, SFCDD_K_SORT, SFCDD_K_ASSEMBLE, SFCDD_K_POTRF, SFCDD_K_TRSM, SFCDD_K_SYRK,
  SFCDD_K_COARSE_ASSEMBLE, SFCDD_K_STENCIL, SFCDD_K_UPDATE, SFCDD_K_RESTRICT, SFCDD_K_TRSV_FWD,
  SFCDD_K_TRSV_BWD, SFCDD_K_PROLONG, SFCDD_K_VECTOR, SFCDD_K_GRAD, SFCDD_K_COARSE_FACTOR,
  SFCDD_K_PCG_VECTOR, /* the fused vector phase of a PCG iteration (prolongation, p, stencil,
                         x / r update, restriction) in one cooperative launch */
  SFCDD_K_COUNT
};
int sfcdd_set_profiling(sfcdd_handle* h, int enable);
/* ms_total, launches: host arrays of SFCDD_K_COUNT entries (either may be NULL);
 * reset != 0 clears the counters after reading. */
int sfcdd_get_kernel_stats(sfcdd_handle* h, double* ms_total, long long* launches, int reset);
/* Algorithmic bytes (or FP operations) one launch of the class processes for
 * this handle: SFCDD_K_TRSV_FWD / _BWD: factor + coarse tile bytes;
 * SFCDD_K_STENCIL: 16 N; SFCDD_K_POTRF / _TRSM / _SYRK: floating-point
 * operations of that part of the local factorizations summed over all launches
 * of one setup; SFCDD_K_COARSE_FACTOR: all operations of the coarse
 * factorization.  Returns 0 for classes without a figure. */
double sfcdd_kernel_work(const sfcdd_handle* h, int kernel_class);

int sfcdd_destroy(sfcdd_handle* h);
const char* sfcdd_status_string(int status);

/* Measured FP64 FMA rate of the current device (no counterpart in the paper: a
 * measurement for reporting).  The FP64 kernels of this library (substitutions
 * with FP64 factors, the stencil, the diagonal tile factorizations) are bound
 * by the FP64 pipe, not by HBM, on this GPU; this is their measured ceiling.
 * Runs `reps` launches of an in-register FMA loop over every SM on `stream`
 * (cudaStream_t, NULL = legacy default stream), synchronises it, and writes the
 * rate in TFLOP/s (2 flops per FMA) to *tflops (host) and the mean launch time
 * in ms to *ms_per_launch (host, may be NULL).  Allocates and frees a small
 * device buffer.  Errors: INVALID_ARG (tflops NULL or reps < 1), CUDA. */
int sfcdd_measure_fp64_rate(int reps, double* tflops, double* ms_per_launch, void* stream);

/* Curve order without any device allocation.  The paper has no counterpart:
 * this is a deployment variant of the keys and sort that sfcdd_setup_ex
 * computes.  For callers that cannot call cudaMalloc: code running while a
 * stream is being captured into a CUDA graph, hosts that hand out all device
 * memory from their own pool, and latency-critical code that must not hit the
 * device synchronisation of cudaMalloc/cudaFree.
 * Outputs (caller-owned device buffers): keys_dev, N uint64 Hilbert keys by
 * lexicographic id; perm_dev, N int32 with perm[pos] = lexicographic id at
 * curve position pos -- the same values sfcdd_get_curve returns.
 * Scratch: a file-scope device array of about 6.4 MB, resident on every GPU
 * that loads the library until the process exits; N may be at most 262,144
 * (2^18) grid points, larger grids return SFCDD_ERR_INVALID_ARG with a message
 * on stderr.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current: make that first call before
 * any stream capture.  All calls share the one array, so calls that overlap on
 * the GPU (other streams, other host threads) race; serialise them.  Work is
 * issued on `stream` (cudaStream_t, NULL = legacy default stream) and is not
 * synchronised.  Errors: INVALID_ARG, KEY_OVERFLOW, UNSUPPORTED, CUDA. */
int sfcdd_curve_order_noalloc(const int* levels, int d, unsigned long long* keys_dev, int* perm_dev,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFCDD_H */
