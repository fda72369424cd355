/*
 * geneo.h — C ABI of the GenEO two-level overlapping Schwarz library (sm_103a).
 *
 * The library builds and applies the two-level additive Schwarz
 * preconditioner with the GenEO coarse space of Seelinger, Reinarz and
 * Scheichl, "A High-Performance Implementation of a Robust Preconditioner for
 * Heterogeneous Problems" (arXiv:1906.10944):
 *
 *   M^{-1}_{AS,2} = R_H^T A_H^{-1} R_H + sum_j R_j^T A_j^{-1} R_j   (Section 3,
 *   Definition 2), with R_H^T = Z, the coarse basis of Definition 4 built from
 *   the local eigenproblem Atilde_j p = lambda X_j A_j^o X_j p (eq. 5 and
 *   Section 4.3), and solves A x = b with preconditioned CG (Section 5).
 *
 * Every numeric step runs in CUDA kernels of this library on one GPU.  The
 * signatures use plain pointers and sizes only.
 *
 * Conventions shared by all entry points:
 *  - Errors are returned as geneo_status_t; no call aborts, throws or traps.
 *  - Streams: every call is ordered on the cudaStream_t it is given (0 = the
 *    legacy default stream).  geneo_setup, geneo_pcg_solve, geneo_query and
 *    geneo_get_subdomain synchronise that stream before returning.
 *    geneo_apply only enqueues work; its device-side status is reported by
 *    the next synchronising call on the same handle.
 *  - Ownership: the caller owns every input array and may free it once the
 *    call that received it returns.  geneo_setup copies what it keeps into
 *    device memory owned by the handle until geneo_destroy.
 *  - Indices are 0-based.
 */
#ifndef GENEO_H
#define GENEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GENEO_OK = 0,
  GENEO_ERR_ARG = 1,          /* invalid argument or inconsistent sizes */
  GENEO_ERR_OOM = 2,          /* device allocation failed */
  GENEO_ERR_NOT_SPD = 3,      /* non-positive pivot in a Cholesky factorisation */
  GENEO_ERR_EIG_NOCONV = 4,   /* local eigensolver reached eig_maxit (only with
                                 geneo_options_t.eig_strict = 1; otherwise the
                                 count is reported in geneo_coarse_info_t) */
  GENEO_ERR_PCG_NOCONV = 5,   /* PCG reached maxit before the tolerance */
  GENEO_ERR_BREAKDOWN = 6,    /* PCG breakdown: p^T A p <= 0 or r^T z <= 0 */
  GENEO_ERR_CUDA = 7,         /* a CUDA runtime call failed */
  GENEO_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
  GENEO_ERR_NONFINITE = 9     /* NaN or Inf met in the data (element matrices,
                                 pivots, right-hand side, PCG residual) */
} geneo_status_t;

typedef enum { GENEO_MEM_HOST = 0, GENEO_MEM_DEVICE = 1 } geneo_mem_t;

typedef enum {
  GENEO_EIG_PAPER = 0,   /* B_j = X_j A_j^o X_j, A_j^o over overlap elements (Section 4.3) */
  GENEO_EIG_FULL = 1     /* B_j = X_j Atilde_j X_j (all elements of Omega_j) */
} geneo_eig_form_t;

/* Partition of unity of Section 3 (Definition 3) when the caller gives no
 * weights: the standard piecewise-constant one of Section 4.3 (1/c_k on D_j),
 * or the smooth one Section 3 shows beside it (Sarkis): X_j(k) = d_j(k) /
 * sum_i d_i(k), d_j(k) the number of element layers between dof k and the
 * inner boundary of Omega_j (the dofs of N_j outside D_j), so X_j falls
 * linearly to zero across the overlap. */
typedef enum {
  GENEO_PU_STANDARD = 0,
  GENEO_PU_SARKIS = 1
} geneo_pu_kind_t;

typedef enum {
  GENEO_PREC_FP64 = 0,   /* all factors and local solves in FP64 */
  GENEO_PREC_FP32 = 1    /* subdomain factors in FP32; residuals, coarse
                            problem and PCG in FP64; the eigensolver's block
                            products, Gram matrices and Rayleigh-Ritz sweeps
                            and the columns of the coarse inverse in
                            double-single arithmetic (about 46 bits) */
} geneo_precision_t;

/*
 * Problem description (Section 2: a conforming FE discretisation; Section 3:
 * overlapping subdomains as unions of mesh elements).
 *
 * All arrays live where `mem` says (host or device memory of the current
 * device) and are read-only for the library.
 *
 *  n            global number of dofs.
 *  ndof_node    dofs per mesh node (1 Darcy, 3 elasticity); informational.
 *  row_ptr[n+1], col[nnz], val[nnz]
 *               CSR of the global matrix A (FP64), symmetric positive
 *               definite, column indices sorted within each row.  Rows and
 *               columns of global Dirichlet dofs are eliminated: their row
 *               and column are zero except a diagonal 1.  The pattern must
 *               contain every coupling (k, l) of two dofs of one element
 *               (explicit zeros allowed).
 *  dirichlet[n] 1 for a global Dirichlet dof, else 0.
 *  n_elem, elem_ndof
 *               number of elements and dofs per element (4 for 2D Q1, 8 for
 *               3D Q1, 24 for 3D Q1 elasticity).
 *  elem_dofs[n_elem*elem_ndof]
 *               global dof of local dof a of element e at [e*elem_ndof + a].
 *  elem_mats[n_elem*elem_ndof*elem_ndof]
 *               unconstrained element stiffness matrices, row-major per
 *               element: K_e[a][b] at [(e*elem_ndof + a)*elem_ndof + b].
 *               Their sum over all elements equals A off the Dirichlet rows.
 *  n_sub        number of overlapping subdomains N.
 *  sub_elem_ptr[N+1], sub_elem[...]
 *               elements of Omega_j, sorted ascending, at
 *               sub_elem[sub_elem_ptr[j] .. sub_elem_ptr[j+1]).
 *  sub_dof_ptr[N+1], sub_dof[...]
 *               dofs of the closure of Omega_j without global Dirichlet
 *               dofs, sorted ascending (geneo_grow_partition produces both
 *               lists from a non-overlapping partition).
 *  pu_weights   optional (NULL: the partition of unity options.pu_kind
 *               selects); otherwise the weights mu_{j,k} of Definition 3 in
 *               the layout of sub_dof: X_j(k) of dof sub_dof[t] at
 *               pu_weights[t].  They must lie in [0, 1], vanish on the dofs
 *               of N_j outside D_j (the inner boundary of Omega_j), and sum
 *               to one over the subdomains on every non-Dirichlet dof (to
 *               1e-12); else geneo_setup returns GENEO_ERR_ARG.
 *  Every subdomain must be non-empty.  Every non-Dirichlet dof must lie in
 *  the interior of at least one subdomain (overlap >= 1 element layer).
 */
typedef struct {
  int32_t mem;
  int32_t ndof_node;
  int64_t n;
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const uint8_t* dirichlet;
  int64_t n_elem;
  int32_t elem_ndof;
  int32_t n_sub;
  const int32_t* elem_dofs;
  const double* elem_mats;
  const int64_t* sub_elem_ptr;
  const int32_t* sub_elem;
  const int64_t* sub_dof_ptr;
  const int32_t* sub_dof;
  const double* pu_weights;
} geneo_problem_t;

/*
 * Options (Theorem 1 and the remark after it for the threshold; Section 4.4
 * for the shift).
 *  tau        eigenvectors with lambda < tau are taken (default 0.3).
 *  nev_max    at most this many per subdomain (default 10); 0 gives the
 *             one-level method M^{-1}_{AS,1}.
 *  fixed_nev  1: take exactly nev_max per subdomain regardless of tau.
 *  sigma      shift of the spectral transformation, nu = 1/(lambda-sigma)
 *             (default -0.01; must be negative: Atilde_j is singular on
 *             floating subdomains).
 *  eig_form   geneo_eig_form_t (default GENEO_EIG_PAPER).
 *  eig_tol    relative residual ||B x - nu K x|| / (||B x|| + nu ||K x||)
 *             at which an eigenpair counts as converged (default 1e-6).
 *  eig_maxit  iteration cap of the block eigensolver (default 100).
 *  guard      extra block vectors beyond the wanted pairs (default
 *             min(3, nev_max): on 3D Darcy 128^3 a guard of 3 needs one more
 *             iteration than 5 but less work in total).
 *  precision  geneo_precision_t (default GENEO_PREC_FP64).
 *  profile    0 (default) or 1, see geneo_coarse_info_t.prof_*.
 *  first_nev  wanted pairs of the eigensolver's narrow first pass; a
 *             subdomain whose first pass finds that many eigenvalues below
 *             tau is solved again with nev_max (default -1: min(8, nev_max);
 *             ignored with fixed_nev).
 *  seed       seed of the counter-based start vectors (SplitMix64).
 *  fp32_pivot_tol  GENEO_PREC_FP32 only: a K_j or A_j whose FP32 Cholesky
 *             meets a pivot <= this value (the bands are equilibrated to a
 *             unit diagonal) is factored and solved in FP64 instead
 *             (adaptive precision per subdomain; default 1e-4, in [0, 1)).
 *             A factorisation on the tensor cores (three-pass TF32
 *             products, error up to 12 times an FP32 FMA's) tests its
 *             pivots against 12 * fp32_pivot_tol.
 *             Those subdomains also run the eigensolver's block products
 *             and orthogonalisation in FP64 (the others in double-single
 *             arithmetic and, for the first pass, FP32).
 *  pu_kind    geneo_pu_kind_t, used when the problem gives no pu_weights
 *             (default GENEO_PU_STANDARD).
 *  eig_strict 1: geneo_setup returns GENEO_ERR_EIG_NOCONV when a subdomain's
 *             eigensolve reaches eig_maxit unconverged; 0 (default): the
 *             setup goes on with the Ritz vectors it has and reports the
 *             count in geneo_coarse_info_t.eig_unconverged.
 *  deterministic  1 (default): every reduction runs in a fixed order, so
 *             repeated calls give bitwise identical results.  0: the PCG
 *             inner products are accumulated with atomic additions (one
 *             launch fewer each); results then vary in the last bits from
 *             run to run.
 *  eig_solve_tf32  GENEO_PREC_FP32 only: 1 (default) runs the eigensolver's
 *             block solves with K_j (the shift-and-invert operator of
 *             Section 4.4) as one TF32 tensor-core pass per product instead
 *             of three (about 1e-3 relative error in K_j^{-1} R; the
 *             residuals and the convergence test stay FP64 and Rayleigh-Ritz
 *             double-single, so only the search directions change and the
 *             eigenpairs meet the same tolerance); 0 keeps FP32 accuracy in
 *             those solves.
 *  factor_kernel  GENEO_PREC_FP32 only: 0 (default) factors the bands on the
 *             fifth-generation tensor cores (tcgen05 MMAs, TMEM accumulators,
 *             tensor-map copies) when the batch's half bandwidth fits that
 *             kernel; 1 always uses the warp-level MMA kernel.
 *  autotune   1 (default): at the end of the first setup of each batch
 *             shape (precision, largest A_j band width and order, number of
 *             subdomains) in the process, the preconditioner's local solve
 *             is timed at each pipeline depth on a scratch vector and the
 *             fastest is kept for every later apply (reported in
 *             geneo_coarse_info_t.local_solve_stages); 0: the depth follows
 *             from shared memory alone.
 *  factor_bf16  GENEO_PREC_FP32 only, a precision study: 1 rounds the
 *             equilibrated matrices and every factor panel to BF16 (the
 *             fifth-generation kernel's planes hold BF16 values exactly),
 *             so the local solves and the eigensolver's shift-and-invert
 *             operator use BF16 factors (stored in FP32); matrices with a
 *             pivot at or below fp32_pivot_tol are factored in FP64 as in
 *             FP32 mode.  Widths the kernel does not take stay FP32.
 *  reserved   must be 0.
 */
typedef struct {
  double tau;
  double sigma;
  double eig_tol;
  int32_t nev_max;
  int32_t fixed_nev;
  int32_t eig_form;
  int32_t eig_maxit;
  int32_t guard;
  int32_t precision;
  int32_t profile;     /* 1: time every kernel family with CUDA events (see
                          geneo_coarse_info_t.prof_*); adds event records
                          and one synchronisation at the end of each call.
                          It creates CUDA events as it goes, so handles used
                          with geneo_pcg_solve_noalloc keep it at 0. */
  int32_t first_nev;
  uint64_t seed;
  double fp32_pivot_tol;
  int32_t pu_kind;
  int32_t eig_strict;
  int32_t deterministic;
  int32_t eig_solve_tf32;
  int32_t factor_kernel;
  int32_t autotune;
  int32_t factor_bf16;
  int32_t reserved;
} geneo_options_t;

typedef struct geneo_handle_s* geneo_handle_t;

/* Per-solve report (Section 5.3 and 5.4 report iterations and a condition
 * estimate).  resid_hist may be NULL; otherwise it receives up to
 * resid_hist_cap recursive relative residuals ||r_k||/||b|| (k = 0, 1, ...).
 * converged = 1 when the true residual ||b - A x||/||b|| met tol. */
typedef struct {
  int32_t iterations;
  int32_t converged;
  double rel_residual;       /* recursive ||r||/||b|| at exit */
  double kappa_estimate;     /* Lanczos estimate of kappa(M^{-1} A), from the
                                CG coefficients before the first replacement */
  double* resid_hist;
  int32_t resid_hist_cap;
  int32_t resid_hist_len;
  double true_residual;      /* ||b - A x||/||b|| of the returned x (FP64) */
  int32_t replacements;      /* true-residual replacements (restarts) made */
  int32_t reserved;
} geneo_solve_info_t;

/* Kernel families of geneo_coarse_info_t.prof_*. */
enum {
  GENEO_PROF_FACTOR = 0,       /* batched banded Cholesky (A_j, K_j, A_H) */
  GENEO_PROF_EIG_SOLVE = 1,    /* eigensolver block solves with K_j */
  GENEO_PROF_GRAM = 2,         /* eigensolver Gram matrices (FP64) */
  GENEO_PROF_SPMM = 3,         /* eigensolver sparse products with K_j, B_j */
  GENEO_PROF_GEMM = 4,         /* eigensolver block updates (FP64) */
  GENEO_PROF_SMALL_EIG = 5,    /* Jacobi SVQB and Rayleigh-Ritz */
  GENEO_PROF_LOCAL_SOLVE = 6,  /* preconditioner local solves L_j L_j^T u = r_j */
  GENEO_PROF_COARSE_SOLVE = 7, /* preconditioner coarse solve */
  GENEO_PROF_SPMV = 8,         /* PCG sparse matrix-vector product */
  GENEO_PROF_OTHER = 9,
  GENEO_PROF_ORTHO32 = 10,     /* eigensolver first K-orthogonalisation pass in
                                  FP32 arithmetic (FP32 factors only) */
  GENEO_PROF_COUNT = 11
};

/* Setup summary (host copies). */
typedef struct {
  int32_t n_sub;
  int32_t dim_coarse;        /* dim V_H = sum_j m_j */
  int32_t coarse_bandwidth;  /* half bandwidth of the banded A_H factor */
  int32_t eig_iterations;    /* block eigensolver iterations (max over batch) */
  int32_t block_size;        /* eigensolver block width s */
  int32_t fp64_factors_K;    /* GENEO_PREC_FP32: K_j factored in FP64 */
  int32_t fp64_factors_A;    /* GENEO_PREC_FP32: A_j factored in FP64 */
  int32_t fp64_ortho;        /* GENEO_PREC_FP32: subdomains whose eigensolver
                                products and orthogonalisation ran in FP64
                                (K_j factored in FP64, a residual that stopped
                                halving, or still iterating at iteration 30);
                                the others use double-single products */
  int32_t eig_unconverged;   /* subdomains whose eigensolve reached eig_maxit
                                unconverged (their Ritz vectors are used) */
  int32_t factor_classes;    /* GENEO_PREC_FP32: batches the K_j and A_j
                                factorisations ran in (size classes of the
                                half bandwidth, each launched as one
                                persistent kernel) */
  int64_t device_bytes;      /* device memory held by the handle */
  double setup_ms[8];        /* per phase: structure, assembly, factor,
                                eigensolve, basis, coarse matrix, coarse
                                factor, total */
  double factor_flops;       /* algorithmic flops of the batched Cholesky of
                                all A_j and K_j: sum over columns (h_c + 1)^2,
                                h_c = entries below the diagonal in column c */
  double factor_event_ms;    /* CUDA-event time of those launches */
  double eigsolve_flops;     /* algorithmic flops of the K_j^{-1} block solves
                                of the eigensolver: 2 (2 h_c + 1) per column
                                and right-hand side */
  double eigsolve_event_ms;  /* CUDA-event time of those launches */
  double apply_flops;        /* algorithmic flops of one geneo_apply */
  double apply_bytes;        /* algorithmic bytes of one geneo_apply: factors,
                                Z, the coarse factor and the vectors once */
  /* With options.profile = 1, per kernel family (index GENEO_PROF_*):
   * CUDA-event milliseconds on the launching stream, launches, and the
   * algorithmic flops and bytes of those launches (setup and every
   * apply/solve on the handle so far). */
  double prof_ms[GENEO_PROF_COUNT];
  double prof_flops[GENEO_PROF_COUNT];
  double prof_bytes[GENEO_PROF_COUNT];
  int64_t prof_launches[GENEO_PROF_COUNT];
  int32_t local_solve_stages; /* pipeline depth of the local solve (2-4) the
                                autotuner chose; 0 if it did not run */
  int32_t reserved;
} geneo_coarse_info_t;


/* Fill *opt with the defaults listed above. */
void geneo_default_options(geneo_options_t* opt);

/*
 * Build the preconditioner (Sections 3 and 4): partition of unity, local
 * Dirichlet matrices A_j, Neumann and overlap matrices, their factorisations,
 * the local eigenproblems, the coarse basis Z and A_H = Z^T A Z with its
 * factorisation.  On success *out receives a new handle.  Synchronises
 * `stream`.  On failure *out is NULL and nothing is leaked.
 */
geneo_status_t geneo_setup(const geneo_problem_t* prob, const geneo_options_t* opt,
                           void* stream, geneo_handle_t* out);

/*
 * z = M^{-1}_{AS,2} r (Section 3, Definition 2) for nrhs right-hand sides
 * stored one after another (stride n).  r_dev and z_dev are device arrays of
 * n*nrhs doubles and must not overlap.  The preconditioner is the identity on
 * global Dirichlet dofs.  Asynchronous on `stream`.
 */
geneo_status_t geneo_apply(geneo_handle_t h, const double* r_dev, double* z_dev, int32_t nrhs,
                           void* stream);

/*
 * Solve A x = b by PCG with M^{-1}_{AS,2} (Section 5; x0 = 0) for nrhs
 * right-hand sides (stride n).  Stopping rule: when the recursively updated
 * residual reaches ||r_k||_2 <= tol ||b||_2 the true residual b - A x is
 * formed; the solve has converged when that meets tol too.  Otherwise the
 * true residual replaces the recursive one and CG restarts from x, at most
 * five times and only while each replacement at least halves it (below
 * that the FP64 rounding of x, about eps ||(|A| |x|)|| / ||b||, bounds every
 * residual); the call then returns GENEO_ERR_PCG_NOCONV with the reached
 * true residual in info.  b and x are device arrays unless `mem` is
 * GENEO_MEM_HOST, in which case they are host arrays and the copies are part
 * of the call.  Several right-hand sides (nrhs >= 2) are solved together,
 * up to 8 at a time: their CG recurrences advance in lockstep so each
 * iteration reads A and the subdomain factors once for all of them, and each
 * stops on its own test (the same stopping rule); the result equals
 * separate solves up to rounding.  info may be NULL; with nrhs > 1 it
 * reports the last right-hand side (no residual history).  Synchronises
 * `stream`.
 */
geneo_status_t geneo_pcg_solve(geneo_handle_t h, const double* b, double* x, int32_t nrhs,
                               double tol, int32_t maxit, int32_t mem,
                               geneo_solve_info_t* info, void* stream);

/*
 * The same PCG solve as geneo_pcg_solve (one right-hand side, device arrays)
 * for callers that must not allocate memory during the solve: code that runs
 * under a fixed device-memory budget, inside a memory pool's own callbacks,
 * or in a request loop where a cudaMalloc would stall the device or fail.
 * The paper has no counterpart; it is a property of this library's API.
 *
 * The call allocates nothing (no cudaMalloc or cudaFree, no host heap): the
 * reduction partials, the PCG scalars and the alpha/beta history used for the
 * condition estimate live in one fixed device array inside the library
 * (73,856 bytes on every device that loads the library, held until the
 * process exits), and the vectors come from the handle, allocated by
 * geneo_setup; the host arrays of the condition estimate are sized by
 * geneo_setup too.  Limit: maxit <= 4095; larger values return
 * GENEO_ERR_ARG.  The handle's device must be current (else GENEO_ERR_ARG),
 * and its options.profile must be 0 (profiling creates CUDA events; else
 * GENEO_ERR_ARG).  The first call on a device looks up that array's device
 * address (with the handle's device current) and caches it per device
 * ordinal for the life of the process; make that first call before any
 * stream capture, and do not call the function again after a
 * cudaDeviceReset of that device.  All calls share the array and it keeps
 * the last call's contents; the scalars are cleared at the start of every
 * call.  The stopping rule and info are those of geneo_pcg_solve.  Calls whose
 * work overlaps on the GPU (on different streams, or on different handles
 * of the same device) race and must not be issued.  b_dev and x_dev are
 * device arrays of n doubles; info as in geneo_pcg_solve.  Synchronises
 * `stream`.
 */
geneo_status_t geneo_pcg_solve_noalloc(geneo_handle_t h, const double* b_dev, double* x_dev,
                                       double tol, int32_t maxit, geneo_solve_info_t* info,
                                       void* stream);

/* Setup summary; synchronises the handle's work. */
geneo_status_t geneo_query(geneo_handle_t h, geneo_coarse_info_t* info);

/*
 * Host copies of subdomain j's data, for inspection and parity tests.  Any
 * output pointer may be NULL.  Sizes first: *n_neu = |N_j|, *n_dir = |D_j|,
 * *m = m_j, *s = block width.  Then, if non-NULL and large enough (caps are
 * element counts):
 *   dir_dofs[n_dir]  global dofs of D_j (ascending)
 *   pu[n_neu]        X_j on N_j
 *   lambda[s]        Ritz values lambda (ascending; +inf where nu <= 0)
 *   Z[n_dir*m]       coarse basis block on D_j rows, column-major
 */
geneo_status_t geneo_get_subdomain(geneo_handle_t h, int32_t j, int32_t* n_neu, int32_t* n_dir,
                                   int32_t* m, int32_t* s, int32_t* dir_dofs, int64_t dir_cap,
                                   double* pu, int64_t pu_cap, double* lambda, int64_t lambda_cap,
                                   double* Z, int64_t z_cap);

/*
 * Overlapping subdomains from a non-overlapping element partition (Section 3:
 * each Omega'_j is grown by `overlap` layers; one layer adds every element
 * that shares a vertex with the current set).  Host arrays only.
 *   part[n_elem]       part of each element in [0, n_parts)
 *   elem_dofs          as in geneo_problem_t; vertices are the dofs
 *   dirichlet[n]       as in geneo_problem_t
 * Outputs are malloc'ed host arrays the caller frees with geneo_free_host:
 * *sub_elem_ptr[n_parts+1], *sub_elem, *sub_dof_ptr[n_parts+1], *sub_dof
 * (sorted lists, Dirichlet dofs excluded from the dof lists).
 */
geneo_status_t geneo_grow_partition(int64_t n, int64_t n_elem, int32_t elem_ndof,
                                    const int32_t* elem_dofs, const uint8_t* dirichlet,
                                    const int32_t* part, int32_t n_parts, int32_t overlap,
                                    int64_t** sub_elem_ptr, int32_t** sub_elem,
                                    int64_t** sub_dof_ptr, int32_t** sub_dof);

void geneo_free_host(void* p);

/* Number of CUDA kernel launches this library has made in this process
 * (all handles, all threads). */
int64_t geneo_launch_count(void);

/*
 * Sizes in bytes of geneo_problem_t, geneo_options_t, geneo_solve_info_t and
 * geneo_coarse_info_t as compiled into the library, written to out[0..3]
 * (at most n of them), so a binding can check its struct layouts.  Host
 * only; returns the number written.
 */
int32_t geneo_struct_sizes(int64_t* out, int32_t n);

/* Release all device memory of the handle (NULL is allowed).  Waits for the
 * handle's work on the stream of its last call (setup, apply or solve),
 * which must still exist, and returns the memory to the device's
 * stream-ordered pool (the library allocates from that pool and keeps freed
 * memory there for later handles). */
void geneo_destroy(geneo_handle_t h);

/* Static string describing a status code. */
const char* geneo_status_str(geneo_status_t s);

/* Details of the last error on this handle: the status code, the subdomain
 * (or matrix id, -1 if none) and the row or index where the device recorded
 * it (for GENEO_ERR_NOT_SPD: subdomain and pivot row of the failed
 * factorisation; GENEO_ERR_NONFINITE from the assembly: subdomain and
 * element).  With h = NULL: the same for the last geneo_setup call of the
 * calling thread (code 0 if it succeeded), whose handle no longer exists
 * when it failed.  Always returns GENEO_OK. */
geneo_status_t geneo_last_error(geneo_handle_t h, int32_t* code, int32_t* where, int64_t* index);

#ifdef __cplusplus
}
#endif
#endif /* GENEO_H */
