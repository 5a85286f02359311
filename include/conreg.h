/*
 * conreg.h -- C ABI of the GB300 greedy low-rank solver for the spatially
 * smoothed connectome regression
 *
 *   min_W  1/2 || (W X - Y) o Omega ||_F^2 + lambda/2 || L_y W + W L_x^T ||_F^2     (Eq. obj_fun)
 *
 * whose normal equations are the multi-term Sylvester equation
 *
 *   A(W) := lambda (W L_x^2 + 2 L_y W L_x + L_y^2 W) + sum_a diag(Omega_a) W X_a X_a^T
 *         = D := (Omega o Y) X^T                                                    (Eq. multitermSylv)
 *
 * The solution is grown as W = U Z V^T (U, V orthonormal) by rank-one ALS
 * updates (Eqs. ALS_linsys, ALS_linsys_v), each followed by a Galerkin
 * projection (Eq. Proj_Sylv): Algorithm 1 of the paper.
 *
 * Conventions for every entry point:
 *  - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *  - Pointers named *_host are host memory; the library copies inputs at the
 *    call and the caller keeps ownership.  Pointers named *_dev are device
 *    memory of the problem's GPU, read/written on the problem's stream.
 *  - Every call returns a cr_status; nothing aborts or throws across the ABI.
 *    On failure cr_last_error() describes the cause.  Device-side loops are
 *    bounded by iteration caps and report CR_ENOTCONV instead of spinning.
 *  - A problem object is used by one host thread at a time.
 */
#ifndef CONREG_H
#define CONREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CR_OK = 0,
  CR_EINVAL = 1,    /* invalid argument (sizes, NaN/Inf input, non-symmetric Laplacian, ...) */
  CR_ENOMEM = 2,    /* device allocation failed; nothing leaked */
  CR_ECUDA = 3,     /* a CUDA runtime call failed */
  CR_ENOTCONV = 4,  /* an iteration hit its cap; the best iterate is kept */
  CR_ETIMEOUT = 5,  /* a bounded device-side wait gave up (grid barrier, mbarrier) */
  CR_ERANK = 6,     /* orthogonalisation rejected a new column (rank deficient) */
  CR_ESTATE = 7     /* call not valid in the current state (e.g. rank capacity reached) */
} cr_status;

/* CR_FP64: every step in float64.  CR_MIXED: the u/v sub-solves run float32
 * PCG (double-float inner products) inside float64 iterative refinement to the
 * same pcg_tol as CR_FP64 (handing over to the float64 kernel when float32
 * cannot resolve the system); the Galerkin solve runs a float32 inner CG,
 * with BF16 tensor-core assembly of the G_a, inside float64 refinement; the
 * residual norm and stopping test stay float64. */
typedef enum { CR_FP64 = 0, CR_MIXED = 1 } cr_precision;
/* Preconditioner of the u/v PCG solves.  CR_PRECOND_MULTIGRID: two V-cycles of
 * smoothed-aggregation multigrid for L + sigma I per application (the inverse
 * of lam (L + sigma I)^2, sigma^2 = the Laplacian shift plus the mean data
 * weight over lam), hierarchy built once from L at cr_create; on the v side
 * with at most 32 injections the data term is added exactly by
 * Sherman-Morrison-Woodbury; sizes whose vectors do not fit one thread-block
 * cluster fall back to Jacobi.  CR_PRECOND_AUTO: multigrid in the float64
 * form; in the mixed form multigrid above 20,000 rows or for lambda >= 1e3
 * (where the Laplacian term dominates and Jacobi's iteration count grows),
 * Jacobi otherwise (there its many cheap float32 iterations are faster). */
typedef enum {
  CR_PRECOND_JACOBI = 0,
  CR_PRECOND_LEARNED = 1,
  CR_PRECOND_MULTIGRID = 2,
  CR_PRECOND_AUTO = 3
} cr_precond;
/* Form of the Galerkin CG (cr_options.galerkin_form).  The projection (Eq. Proj_Sylv)
 * it solves is the same in every form; the forms differ in the basis the CG runs
 * in and its preconditioner.  CR_GALERKIN_EIGEN runs the CG on Qa^T Z Qb, where
 * A1 = U^T L_y U = Qa diag(la) Qa^T and B1 = V^T L_x V = Qb diag(lb) Qb^T are
 * diagonal (fast diagonalization): the A1 Z B1 term becomes a scaling and the
 * preconditioner the operator's diagonal there.  Qa and Qb follow the greedy
 * rank by one arrowhead eigen-update per new border.  The solution is checked
 * in the original basis; if the residual is above the tolerance there, the
 * original-basis CG finishes from it. */
typedef enum {
  CR_GALERKIN_AUTO = 0,   /* the eigenbasis form wherever the persistent Galerkin kernel runs */
  CR_GALERKIN_JACOBI = 1, /* the original basis, preconditioned by diag(K) */
  CR_GALERKIN_EIGEN = 2   /* the eigenbasis form (as AUTO) */
} cr_galerkin_form;
typedef enum { CR_STOP_NONE = 0, CR_STOP_RMAX = 1, CR_STOP_DW = 2, CR_STOP_RELRES = 3, CR_STOP_RANK = 4 } cr_stop;

/* Square sparse matrix in CSR form (host memory): row i holds entries
 * rowptr[i] .. rowptr[i+1]-1 with column col[p] and value val[p]. */
typedef struct {
  int64_t n;
  const int32_t* rowptr; /* n + 1 */
  const int32_t* col;    /* rowptr[n] */
  const double* val;     /* rowptr[n] */
} cr_csr;

/* Where the descriptor's arrays live (cr_problem_desc.mem_kind). */
typedef enum { CR_MEM_HOST = 0, CR_MEM_DEVICE = 1 } cr_mem_kind;

/* Optional voxel box of one side: row i of the Laplacian is the voxel with
 * linear index box_index[i] = z*H*W + y*W + x of a D x H x W box (dims = {D, H,
 * W}); indices distinct and inside the box.  box_index = NULL: no grid. */
typedef struct {
  int32_t dims[3];
  const int32_t* box_index;
} cr_grid;

/* Problem data, Algorithm 1's input line (Sec. 1.1 and Sec. 1.4):
 *  Lx (nx x nx), Ly (ny x ny): symmetric graph Laplacians of the voxel
 *      face-adjacency graphs (Sec. 1.1).  Any symmetric CSR matrix is accepted;
 *      each row may hold at most 16 off-diagonal entries.
 *  X  (nx x ninj): injection (source) data, column a = injection a.
 *  Y  (ny x ninj): projection (target) data.
 *  Omega (ny x ninj): 1 where Y is observed, 0 on the injection site.
 *  lambda > 0: the weight of Eq. (obj_fun) (not the rescaled lambda-bar; see
 *      cr_lambda_from_bar).
 *  mem_kind: CR_MEM_HOST (0, the zero-initialised default): every array of the
 *      descriptor (the CSR arrays of Lx and Ly, X, Y, Omega, the grids' box
 *      indices) is host memory; CR_MEM_DEVICE: every one of them is device memory
 *      of the current GPU (not host, not another device: CR_EINVAL).  Either way
 *      the library copies the inputs at the call (device inputs are staged
 *      through host memory for validation) and the caller keeps ownership.
 *  grid_x, grid_y: optional voxel boxes of the two sides (cr_set_voxel_grid at
 *      creation), used by the learned preconditioner. */
typedef struct {
  int64_t nx, ny, ninj;
  cr_csr Lx, Ly;
  const double* X_host;
  int64_t ldx;
  const double* Y_host;
  int64_t ldy;
  const uint8_t* Omega_host;
  int64_t ldo;
  double lambda;
  int32_t mem_kind;
  cr_grid grid_x, grid_y;
} cr_problem_desc;

/* Solver options; call cr_options_default() first, then override fields. */
typedef struct {
  size_t struct_size;      /* sizeof(cr_options) */
  int32_t r_cap;           /* rank capacity; device memory is sized for it */
  int32_t precision;       /* cr_precision */
  int32_t precond;         /* cr_precond (u/v sub-solves) */
  double pcg_tol;          /* relative residual of the u/v PCG solves (default 1e-10) */
  int32_t pcg_maxit;       /* cap on PCG iterations per solve (default 20000) */
  double als_delta;        /* ALS stop: |‖û‖/‖v̂‖ - 1| <= als_delta (default 0.1, Sec. 2.3) */
  int32_t als_max_iter;    /* cap on ALS sweeps (default 10) */
  int32_t als_sweeps;      /* > 0: run exactly this many sweeps (deterministic comparisons) */
  int32_t galerkin_maxit;  /* cap on Galerkin CG iterations per projection (default 10 j^2 + 100) */
  int32_t residual_every;  /* cr_solve: evaluate ‖R‖_F every k steps (default 1); 0 = automatic: after each
                              check, at half the steps that relres's observed decay predicts to the target
                              (1 to 32), so sparse far from it and every step close to it */
  int32_t cluster_size;    /* PCG thread-block cluster size; 0 = automatic */
  int32_t profile;         /* != 0: time each phase with CUDA events (see cr_get_stats) */
  int32_t pcg_kernel;      /* 0 = automatic: the register-resident cluster kernel (the whole solve on
                              chip) while it applies (unit-weight Laplacian, at most 6 neighbours per
                              row, up to 1,024 rows per CTA in float64 or 2,048 in float32), else the
                              grid-wide kernel; 1 = the generic cluster kernel (grids that fit one
                              cluster); 2 = always the grid-wide kernel */
  int32_t galerkin_kernel; /* 0 = one persistent cooperative launch per projection, 1 = one launch per step */
  uint64_t seed;           /* seed of the fallback ALS start vector */
  void* stream;            /* cudaStream_t for all device work; NULL = a library-owned stream */
  /* Optional device allocator (e.g. a framework caching allocator).  When
   * alloc is NULL the library uses cudaMalloc/cudaFree. */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* alloc_ctx;
  int32_t galerkin_ctas;   /* CTA cap of the persistent Galerkin kernel; 0 = one CTA per SM.  Problems
                              that share the GPU (cr_solve_batch) cap it so that their launches co-run. */
  int32_t learned_judge;   /* how Jacobi-PCG judges the learned preconditioner (cr_set_preconditioner):
                              0 = by time (default), 1 = by iterations */
  int32_t galerkin_form;   /* cr_galerkin_form (default CR_GALERKIN_AUTO) */
} cr_options;

typedef struct {
  int32_t rank;          /* rank j after the call */
  int32_t sweeps;        /* ALS sweeps taken */
  double delta;          /* final ALS delta */
  double unorm, vnorm;   /* ‖û‖, ‖v̂‖ of the last sweep */
  int32_t pcg_iters_u;   /* total PCG iterations, u side */
  int32_t pcg_iters_v;   /* total PCG iterations, v side */
  double pcg_relres_max; /* worst final PCG relative residual */
} cr_rank1_info;

typedef struct {
  int32_t iters;   /* Galerkin CG iterations */
  double relres;   /* ‖U^T D V - K(Z)‖_F / ‖U^T D V‖_F at exit */
} cr_proj_info;

typedef struct {
  int32_t rank;        /* final rank */
  int32_t stop;        /* cr_stop */
  double relres;       /* last evaluated ‖D - A(W)‖_F / ‖D‖_F */
  double dW;           /* last ‖W_j - W_{j-1}‖_F / ‖W_j‖_F */
  double J;            /* objective of Eq. (obj_fun) at the final W */
  int64_t pcg_iters;   /* total PCG iterations */
  int64_t cg_iters;    /* total Galerkin CG iterations */
  double seconds;      /* host wall time of the call */
} cr_solve_info;

/* Phases timed when cr_options.profile != 0. */
typedef enum {
  CR_PHASE_PCG_U = 0,    /* PCG solves of Eq. (ALS_linsys) */
  CR_PHASE_PCG_V = 1,    /* PCG solves of Eq. (ALS_linsys_v) */
  CR_PHASE_RHS = 2,      /* residual products R_j v, R_j^T u and sub-problem coefficients */
  CR_PHASE_ORTH = 3,     /* orthogonalisation and projected coefficient matrices */
  CR_PHASE_GALERKIN = 4, /* Galerkin CG on Eq. (Proj_Sylv) and the masked data residual */
  CR_PHASE_RESID = 5,    /* residual norm, objective, dW */
  CR_PHASE_PCG_KERNEL = 6, /* the u side's PCG kernel launches alone (inside PCG_U) */
  CR_PHASE_BASIS = 7,    /* eigenbasis updates of the Galerkin CG's eigenbasis form (inside GALERKIN) */
  CR_PHASE_PCG_KERNEL_V = 8, /* the v side's PCG kernel launches alone (inside PCG_V) */
  CR_NPHASE = 10
} cr_phase;

typedef struct {
  int64_t launches;               /* kernels launched by the library (all problems) since the last reset */
  int64_t pcg_solves;             /* PCG solves on this problem since the last reset */
  int64_t pcg_iters;              /* their iterations */
  int64_t h2d_bytes, d2h_bytes;   /* bytes this problem copied host->device / device->host */
  double phase_ms[CR_NPHASE];     /* device time per cr_phase (profile mode; else 0) */
  int64_t phase_calls[CR_NPHASE]; /* timed intervals per phase */
  int64_t learned_solves;         /* sub-solves finished by the learned flexible CG */
  int64_t learned_fallbacks;      /* learned solves that stagnated and were finished by Jacobi-PCG */
  int64_t learned_off;            /* bit s set: the learned form is switched off for side s */
  int64_t mixed_handovers;        /* mixed-form sub-solves that float32 refinement handed to float64 */
  int64_t pcg_cluster[2];         /* CTAs per thread-block cluster of the u-side (0) and v-side (1) PCG;
                                     0 = the grid-wide kernel */
  int64_t pcg_multigrid[2];       /* levels of the multigrid preconditioner per side (0 = not in use) */
  int64_t galerkin_eigen[2];      /* projections solved in the eigenbasis form (0), of which the
                                     original-basis CG had to finish (1) */
  int64_t pcg_iters_side[2];      /* PCG iterations of the u side (0) and the v side (1) */
  double pcg_bytes_per_iter[2];   /* algorithmic bytes of one iteration of each side's PCG kernel in the
                                     form's working precision, counted as if every vector and matrix entry
                                     it touches were streamed from memory (the kernels keep them on chip) */
} cr_stats;

/* Fill *o with defaults (struct_size set).  Always succeeds for o != NULL. */
cr_status cr_options_default(cr_options* o);

/* lambda = lambda_bar * ninj / nx (Sec. 1.1). */
double cr_lambda_from_bar(double lambda_bar, int64_t ninj, int64_t nx);

/* Create a problem on the current CUDA device: validates and copies the inputs
 * (Algorithm 1, "Initialize": W_0 = 0, R_0 = D, U_0 = V_0 = []).  Fails with
 * CR_EINVAL on bad sizes, non-finite values, non-symmetric Laplacians or
 * lambda <= 0; CR_ENOMEM if device memory for rank r_cap does not fit.
 * *out is NULL on failure. */
cr_status cr_create(const cr_problem_desc* desc, const cr_options* opts, struct cr_problem** out);

/* Destroy a problem and free its device memory; NULL is a no-op. */
void cr_destroy(struct cr_problem* p);

/* One greedy rank-one step (Algorithm 1, body up to "Increment rank"): ALS
 * sweeps solving Eq. (ALS_linsys) and Eq. (ALS_linsys_v) by PCG until
 * delta <= als_delta, then orthogonalisation of u and v into U and V (j -> j+1)
 * and update of the projected coefficient matrices of Eq. (Proj_Sylv).  Z is
 * padded with a zero row/column (the warm start of the next projection).
 * CR_ESTATE if j == r_cap, CR_ERANK if u or v lies in the current span. */
cr_status cr_add_rank_one(struct cr_problem* p, cr_rank1_info* info);

/* Galerkin projection (Eq. Proj_Sylv): matrix CG on Z from the current Z until
 * ‖U^T D V - K(Z)‖_F <= tol ‖U^T D V‖_F (Algorithm 1 uses tol = tau / 2).  A tol
 * below 1e-14 (0 included) asks for the rounding floor and is taken as 1e-14. */
cr_status cr_project(struct cr_problem* p, double tol, cr_proj_info* info);

/* Stopping quantities of Algorithm 1 for W = U Z V^T: relres = ‖D - A(W)‖_F/‖D‖_F
 * (any pointer may be NULL to skip it), J = objective of Eq. (obj_fun), and
 * dW = ‖W_j - W_{j-1}‖_F / ‖W_j‖_F against the W before the last projection. */
cr_status cr_residual(struct cr_problem* p, double* relres, double* J, double* dW);

/* Algorithm 1: repeat add_rank_one + project(tau/2) + residual until j == r_max,
 * dW <= tau, or relres <= relres_target (0 disables that test). */
cr_status cr_solve(struct cr_problem* p, int32_t r_max, double tau, double relres_target, cr_solve_info* info);

/* Current rank j. */
cr_status cr_get_rank(const struct cr_problem* p, int32_t* j);

/* Copy U (ny x j), Z (j x j), V (nx x j) into caller host buffers (any may be NULL). */
cr_status cr_get_factors(struct cr_problem* p, double* U_host, int64_t ldu, double* Z_host, int64_t ldz,
                         double* V_host, int64_t ldv);

/* Opaque checkpoint of the iterate between greedy steps (Algorithm 1's loop
 * state): the rank j, U, Z, V and the Z of the step before (so that dW
 * continues), tagged with the problem's sizes and lambda.  cr_get_state with
 * buf = NULL stores the size in *bytes; otherwise *bytes must be at least that
 * size and the state is written to the host buffer buf.  cr_set_state restores
 * a state into a problem with the same ny, nx, ninj and lambda (CR_EINVAL
 * otherwise, or for a corrupt buffer; CR_ESTATE if its rank exceeds r_cap) and
 * rebuilds every projection, so that continuing from it repeats the original
 * run bit for bit. */
cr_status cr_get_state(struct cr_problem* p, void* buf, size_t* bytes);
cr_status cr_set_state(struct cr_problem* p, const void* buf, size_t bytes);

/* Replace the state by rank j factors (U, V must have orthonormal columns; the
 * library does not re-orthogonalise) and rebuild every projection: checkpoint
 * restore and step-by-step comparisons. */
cr_status cr_set_factors(struct cr_problem* p, int32_t j, const double* U_host, int64_t ldu, const double* Z_host,
                         int64_t ldz, const double* V_host, int64_t ldv);

/* out = R_j v (trans = 0; v has nx entries, out ny) or out = R_j^T u (trans = 1)
 * for R_j = D - A(U Z V^T): the right sides of Eqs. (ALS_linsys), (ALS_linsys_v). */
cr_status cr_apply_residual(struct cr_problem* p, int32_t trans, const double* in_host, double* out_host);

/* Solve Eq. (ALS_linsys): A_hat u_hat = rhs for a unit vector v (nx entries),
 * by the library's PCG to opts.pcg_tol.  rhs and u_hat have ny entries; iters
 * (may be NULL) receives the PCG iteration count.  CR_ENOTCONV at the cap. */
cr_status cr_solve_u(struct cr_problem* p, const double* v_host, const double* rhs_host, double* u_hat_host,
                     int32_t* iters);

/* Solve Eq. (ALS_linsys_v): B_hat v_hat = rhs for a unit vector u (ny entries). */
cr_status cr_solve_v(struct cr_problem* p, const double* u_host, const double* rhs_host, double* v_hat_host,
                     int32_t* iters);

/* Galerkin assembly G_a = U^T diag(Omega_a) U for every injection a (the
 * coefficient matrices of the data term of Eq. Proj_Sylv) for the current U,
 * as float32: method 0 = tensor cores (tcgen05, BF16 hi/lo split operands,
 * float32 accumulation; needs r_cap <= 128), method 1 = the float64 matrices
 * rounded to float32.  Copies G_a to G_host + a*ldg*j (j x j, leading
 * dimension ldg >= j).  Mixed form only (CR_ESTATE otherwise). */
cr_status cr_galerkin_assembly(struct cr_problem* p, int32_t method, float* G_host, int64_t ldg);

/* Counters and (profile mode) per-phase device times; reset != 0 zeroes them
 * after reading.  Synchronises the problem's stream. */
cr_status cr_get_stats(struct cr_problem* p, cr_stats* s, int32_t reset);

/* Allocation-free solve of the library's u-side ALS system, for callers that
 * cannot allocate device memory (a plug-in confined to buffers its host
 * application hands it, code that must not enter the allocator, a process whose
 * allocator belongs to another runtime).  The paper has no counterpart: it is
 * a packaging of the library's u-side PCG for such callers.
 *
 * Solves (lambda [(L + c I)^2 + (d - c^2) I] + diag(omega)) u_hat = rhs from
 * u_hat = 0 by a cluster-resident Jacobi PCG (the algorithm of cr_solve_u's
 * cluster kernels), to relative residual tol or maxit iterations.  L (n x n) is given in CSR form in device
 * memory (int32 rowptr[n+1], col[nnz], float64 val[nnz]); omega, rhs and u_hat
 * are device vectors of n entries; stream is a cudaStream_t (NULL = default).
 * *iters (host, may be NULL) receives the iteration count.
 *
 * It allocates nothing: its work vectors live in one static device array of
 * 5 x 131072 doubles (about 5 MiB) that every GPU loading the library keeps
 * until the process exits, so n may be at most 131072 (larger n: CR_EINVAL).
 * Every call looks up that array's device address in the current context
 * (with the device current); the first call on a device also loads the
 * library's device code there.  All calls share the array: calls whose kernels overlap on the GPU (other streams
 * or host threads) race and return garbage.  The call waits for `stream` to
 * finish before it returns (it reads its status words back).  Errors are
 * described by cr_last_error(NULL). */
cr_status cr_solve_u_noalloc(int64_t n, const int32_t* rowptr_dev, const int32_t* col_dev, const double* val_dev,
                             double lambda, double c, double d, const double* omega_dev, const double* rhs_dev,
                             double* u_hat_dev, double tol, int32_t maxit, int32_t* iters, void* stream);

/* Held-out (cross-validation) error of the current W = U Z V^T on mt
 * injections that the fit did not use: X_t (nx x mt, ld ldx), Y_t (ny x mt,
 * ld ldy), Omega_t (ny x mt, ld ldo), all host memory.  On return
 *   *num = sum_a |(W x_a - y_a) o omega_a|^2,   *den = sum_a |y_a o omega_a|^2,
 * the data term of Eq. (obj_fun) (times 2) evaluated on the held-out columns,
 * and its value at W = 0.  The products run on the device as V^T X_t, then
 * Z (V^T X_t), then U Z V^T X_t; the two sums are deterministic reductions.
 * The paper fixes lambda-bar by hand (Sec. 1.1); scoring held-out injections
 * is this library's criterion for the lambda x fold sweep below. */
cr_status cr_cv_error(struct cr_problem* p, int32_t mt, const double* Xt_host, int64_t ldx, const double* Yt_host,
                      int64_t ldy, const uint8_t* Omega_t_host, int64_t ldo, double* num, double* den);

/* ---- post-processing of the solution -------------------------------------- */

/* Sec. 4 (leading singular vectors of the solution): W = U Z V^T is not an SVD
 * because Z is not diagonal.  With the SVD of the core, Z = U~ S V~^T, the
 * factors U^ = U U~ (ny x j) and V^ = V V~ (nx x j) give W = U^ S V^^T.  The
 * j x j SVD runs on the host (one-sided Jacobi: Hestenes' method, accurate in
 * the relative sense of Demmel and Veselic); the n x j products run on the
 * device.  sigma receives the j singular values in descending order; U^ and
 * V^ go to caller host buffers (leading dimensions ldu >= ny, ldv >= nx).  Any
 * output may be NULL.  At rank 0 nothing is written.  Each singular pair is
 * unique up to a common sign when its singular value is simple. */
cr_status cr_svd_factors(struct cr_problem* p, double* Uhat_host, int64_t ldu, double* sigma_host,
                         double* Vhat_host, int64_t ldv);

/* Statistics of one pass over W = U Z V^T.  P(W) = max(0, W) entrywise (the
 * projection onto the nonnegative orthant, Sec. 4) when the pass is asked to
 * project, else W; W* is the reference solution of the pass (0 without one). */
typedef struct {
  int64_t entries;       /* ny * nx */
  int64_t n_negative;    /* entries of W below zero */
  double w_min, w_max;   /* smallest and largest entry of W */
  double w_fro2;         /* |W|_F^2 */
  double neg_fro2;       /* |W - max(0, W)|_F^2: squared distance of W to the nonnegative orthant */
  double ref_fro2;       /* |W*|_F^2 */
  double diff_fro2;      /* |P(W) - W*|_F^2 */
  double diff_maxabs;    /* max |P(W) - W*| over the entries */
  double rms;            /* Sec. 3: E(P(W), W*) = sqrt(diff_fro2 / (ny nx)) */
  double rel;            /* Sec. 3: E_rel(P(W), W*) = sqrt(diff_fro2 / ref_fro2); NaN when W* = 0 */
} cr_solution_stats;

/* One tiled float64 pass over W = U Z V^T (64 x 64 tiles formed on the device;
 * the whole ny x nx matrix is never held there).  nonneg != 0 projects each
 * entry onto the nonnegative orthant before it is compared or returned.  The
 * reference W* = U* Z* V*^T has rank j_ref >= 0 (0: W* = 0) and is given by
 * caller host factors: U* (ny x j_ref, ld ldur >= ny), Z* (j_ref x j_ref,
 * ld ldzr >= j_ref), V* (nx x j_ref, ld ldvr >= nx); they need not be
 * orthonormal (another rank of the same problem, a truth of low rank, ...).
 * W_host (may be NULL) receives P(W), ny x nx with ld ldw >= ny; the copy goes
 * through a device buffer of at most 256 MiB, a block of columns at a time.
 * Sums and extremes are reduced in a fixed order: repeated calls agree bit
 * for bit.  Synchronises the problem's stream. */
cr_status cr_solution_report(struct cr_problem* p, int32_t nonneg, int32_t j_ref, const double* Uref_host,
                             int64_t ldur, const double* Zref_host, int64_t ldzr, const double* Vref_host,
                             int64_t ldvr, double* W_host, int64_t ldw, cr_solution_stats* stats);

/* ---- batched lambda x fold sweep -------------------------------------------
 * Independent greedy solves (Algorithm 1) of sub-problems of one data set: a
 * member fits the injections fit_cols (columns of X, Y, Omega) with its own
 * lambda, and is scored on test_cols by cr_cv_error.  Members differ in lambda
 * and in their (uneven) injection counts. */
typedef struct {
  double lambda;             /* weight of Eq. (obj_fun) for this member */
  const int32_t* fit_cols;   /* host: injections the member fits (n_fit >= 1, each in [0, ninj)) */
  int32_t n_fit;
  const int32_t* test_cols;  /* host: held-out injections scored after the solve (may be NULL) */
  int32_t n_test;
} cr_member;

typedef struct {
  int32_t status;            /* cr_status of the member (CR_ENOTCONV: stopped early, results valid) */
  int32_t rank;              /* final rank */
  int32_t stop;              /* cr_stop */
  int32_t slot;              /* worker slot that ran the member */
  double relres, dW, J;      /* as in cr_solve_info */
  double cv_num, cv_den;     /* cr_cv_error on test_cols (0, 0 without test columns) */
  int64_t pcg_iters, cg_iters;
  double seconds;            /* host wall time of the member's solve and scoring */
} cr_member_result;

/* Solve every member: `concurrency` worker threads (0 = one per 16 SMs), each
 * with its own CUDA stream, take members longest first (largest lambda first)
 * and run create -> cr_solve(r_max, tau, relres_target) -> cr_cv_error on them,
 * so that as many greedy solves as the GPU holds run at once (each PCG solve
 * occupies one thread-block cluster).  desc holds the full data set (its
 * lambda is ignored); opts apply to every member (opts->stream, when set, is
 * the stream that the workers' streams fork from and join into, so CUDA events
 * recorded on it around the call time the whole sweep).  Each member's device
 * memory stays allocated until the sweep ends (no device-synchronising frees
 * while members run).  keep (may be NULL) receives the n_members problem
 * handles, which the caller then owns (cr_destroy); otherwise they are
 * destroyed before return.  results[k] describes members[k].  Returns CR_OK
 * when every member's status is CR_OK or CR_ENOTCONV, else the first other
 * status (all results are filled either way); CR_EINVAL for bad arguments. */
cr_status cr_solve_batch(const cr_problem_desc* desc, const cr_options* opts, const cr_member* members,
                         int32_t n_members, int32_t r_max, double tau, double relres_target, int32_t concurrency,
                         cr_member_result* results, struct cr_problem** keep);

/* ---- learned preconditioner (the paper has no counterpart: its sub-problems
 * are solved directly) ------------------------------------------------------
 * A 4-layer 3x3x3 convolutional network on the voxel box (channels 2 -> 16 ->
 * 16 -> 16 -> 1, zero padding, ReLU between layers; BF16 weights and
 * activations, float32 accumulation).  Input channel 0 is the Jacobi-scaled
 * residual D^-1 r / s on the mask voxels (s = |D^-1 r|), channel 1 the mask;
 * the preconditioner is z = D^-1 r + s net(input), used by a flexible CG
 * (Polak-Ribiere) in place of Jacobi-PCG when cr_options.precond =
 * CR_PRECOND_LEARNED.  Device buffers are float32, layout [batch][channel][z][y][x]. */
struct cr_net;

/* Number of float32 parameters (weights W_l[co][ci][27] then biases b_l, layer by layer). */
int64_t cr_net_param_count(void);

/* New network for a D x H x W box and batches of up to batch_cap volumes;
 * seeded initialisation with a zero last layer (the untrained network is Jacobi). */
cr_status cr_net_create(int32_t D, int32_t H, int32_t W, int32_t batch_cap, uint64_t seed, void* stream,
                        struct cr_net** out);
void cr_net_destroy(struct cr_net* n);
cr_status cr_net_get_params(struct cr_net* n, float* host, int64_t count);
cr_status cr_net_set_params(struct cr_net* n, const float* host, int64_t count);

/* out_dev (B x V) = net(in_dev (B x 2 x V)). */
cr_status cr_net_forward(struct cr_net* n, int32_t B, const float* in_dev, float* out_dev);

/* Loss = sum m (net(in) - target)^2 / sum m target^2 over the batch (mask_dev: V
 * bytes) and its gradient with respect to every parameter (grad_host, may be NULL). */
cr_status cr_net_gradients(struct cr_net* n, int32_t B, const float* in_dev, const float* target_dev,
                           const uint8_t* mask_dev, float* loss_host, float* grad_host);

/* One Adam step (beta1 0.9, beta2 0.999) on that loss; *loss_host (may be NULL) = loss before the step. */
cr_status cr_net_train_step(struct cr_net* n, int32_t B, const float* in_dev, const float* target_dev,
                            const uint8_t* mask_dev, float lr, float* loss_host);

/* Verification aid for the Galerkin CG's eigenbasis updates (no counterpart in
 * the paper): the device arrowhead eigen-decomposition of [diag(d) z; z^T alpha]
 * (d: n values, ascending), on host buffers: mu (n + 1, ascending) and W
 * ((n + 1)^2, column-major, columns the eigenvectors in the order of mu).
 * Allocates and frees its own device memory and stream; returns after the
 * results are copied.  EINVAL for n < 0, n > 4096 or null pointers. */
cr_status cr_arrow_check(int32_t n, const double* d, const double* z, double alpha, double* mu, double* W);

/* Verification aid for the network kernels (no counterpart in the paper): the
 * forward pass, the masked relative loss and the parameter gradients computed
 * by the same kernel templates as a cr_net, instantiated with float64 storage
 * and accumulation, on a D x H x W box (V voxels) and B samples.  All buffers
 * are host memory: params (cr_net_param_count() values, packed as in
 * cr_net_get_params), in (B x 2 x V), target (B x V), mask (V); outputs out
 * (B x V), *loss and grads (packed as params).  Allocates and frees its own
 * device memory and stream; returns after the results are copied.  EINVAL for
 * null pointers or B * V > 2^22; ENOMEM, ECUDA. */
cr_status cr_net_check_f64(int32_t D, int32_t H, int32_t W, int32_t B, const double* params, const double* in,
                           const double* target, const uint8_t* mask, double* out, double* loss, double* grads);

/* Voxel box of one side (0 = y grid of L_y, 1 = x grid of L_x): box_index_host[i]
 * is the linear index z*H*W + y*W + x of row i; dims = {D, H, W}. */
cr_status cr_set_voxel_grid(struct cr_problem* p, int32_t side, const int32_t* dims, const int32_t* box_index_host);

/* Attach a network (NULL detaches); its box must match the voxel grids.
 * Jacobi-PCG judges the network, per side: the first sub-solve after attaching
 * runs Jacobi-PCG and records its iteration count k_J and its time t_J.  Each
 * later learned solve may take at most 2 k_J + 16 flexible-CG iterations and,
 * when judging by time (cr_options.learned_judge = 0), at most 2 t_J; if it
 * has not converged by then, Jacobi-PCG finishes it from the current iterate
 * (a fallback).  By time, an attempt that falls back or takes longer than t_J
 * is a loss and two losses in a row switch the learned form off for that side;
 * by iterations, three fallbacks in a row do.  Off lasts until the next
 * attach.  cr_stats counts learned solves, fallbacks and the switched-off sides. */
cr_status cr_set_preconditioner(struct cr_problem* p, struct cr_net* net);

/* Static description of a status code. */
const char* cr_status_str(cr_status s);

/* Message of the last failure on p (or of the last failed cr_create when p is NULL). */
const char* cr_last_error(const struct cr_problem* p);

#ifdef __cplusplus
}
#endif

#endif /* CONREG_H */
