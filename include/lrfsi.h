/*
 * lrfsi -- low-rank solver for parameter-dependent stationary FSI on GB300.
 *
 * C ABI of the library built from paper_2008_10275_gb300/csrc.  It implements
 * the hot path of Benner, Richter & Weinhandl, "A Low-rank Method for
 * Parameter-dependent Fluid-structure Interaction Discretizations with
 * Hyperelasticity": the per-subset Newton step written as one matrix equation
 * (Sec. 3.4, Eq. (newton_matrix1))
 *
 *     J0 S + Jmu' S D_mu + Jnu' S D_nu = B,    S = U V^T,
 *
 * solved on the factors by the truncated, mean-preconditioned Chebyshev
 * iteration (ChebyshevT, Sec. 4 and Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status: LRFSI_OK (0) or a negative code
 *   below.  lrfsi_last_error() returns a message for the calling thread's last
 *   failure.  No function aborts, traps or prints.
 * - Vectors x in R^M use the library's DOF order (slab-major, see
 *   lrfsi_mesh_dofmap).  Tall matrices (M x r, "U factors", residual blocks)
 *   are ROW-MAJOR with a leading dimension ld >= r (element (i, j) at
 *   p[i * ld + j]).  Small parameter-side matrices (m x r, "V factors") are
 *   row-major with leading dimension ldv >= r.
 * - Pointers named *_dev are device pointers owned by the caller; pointers
 *   named *_host are host pointers owned by the caller.  The library never
 *   frees caller memory and keeps no reference to it after the call returns.
 * - Handles are created and destroyed by the library; they own their device
 *   workspace.
 * - Work is enqueued on the given stream; entry points that return host
 *   values (norms, ranks, iteration counts) synchronize that stream.
 * - All arithmetic named FP64 is IEEE binary64; the mixed mode runs the inner
 *   Chebyshev correction in binary32 inside an FP64 refinement loop.
 * - Concurrency: calls on one handle must not overlap.  Calls on different
 *   handles may run at the same time from different host threads, each on its
 *   own stream: the grouped GEMMs' workspace belongs to the calling thread
 *   (freed when it exits), the SpMM autotuner table and a mesh's lazily built
 *   nested-dissection structure are guarded by locks, and stream captures are
 *   thread-local.  lrfsi_gram_path, lrfsi_lu_mode, lrfsi_graph_mode,
 *   lrfsi_svd_cluster and lrfsi_timing are process-wide settings.  One device
 *   per process (the current device at each call).
 */
#ifndef LRFSI_H
#define LRFSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LRFSI_OK 0
#define LRFSI_EINVAL (-1)      /* bad argument (null pointer, size, option) */
#define LRFSI_ENOMEM (-2)      /* device or host allocation failed */
#define LRFSI_ECUDA (-3)       /* a CUDA runtime call failed */
#define LRFSI_ESINGULAR (-4)   /* LU pivot below threshold (reported, not trapped) */
#define LRFSI_ENOCONV (-5)     /* Newton / Chebyshev hit its iteration limit */
#define LRFSI_EBREAKDOWN (-6)  /* Cholesky-QR breakdown that the shifted retry could not fix */
#define LRFSI_ETIMEOUT (-7)    /* a bounded device wait expired */

typedef void* lrfsi_stream_t;  /* a cudaStream_t; NULL = the legacy default stream */

/* Geometry and constants of the 2D channel-with-flap problem (Sec. 2,
 * Eq. (fsi_problem_weak1); the 2D stand-in for the 3D test case of Sec. 5). */
typedef struct {
  int nx, ny;            /* cells along x and y (structured quadrilaterals) */
  double Lx, Ly;         /* channel [0, Lx] x [0, Ly] */
  double flap[4];        /* solid S = (x0, x1) x (y0, y1); x1 <= x0 means no solid */
  double rho_f;          /* fluid density */
  double lam_s;          /* first Lame parameter of the solid */
  double v_mean;         /* mean velocity of the parabolic inflow at x = 0 */
} lrfsi_problem;

typedef struct lrfsi_mesh_s* lrfsi_mesh_h;

typedef struct {
  int64_t M;             /* number of unknowns, 4 * (#Q2 nodes) + #Q1 vertices */
  int64_t nnz;           /* nonzeros of the union pattern of J0, Jmu', Jnu' */
  int nslab;             /* diagonal blocks of the block-tridiagonal ordering */
  int nmax;              /* largest slab size */
  int ncell, nsolid;     /* cells, solid cells */
} lrfsi_mesh_info_t;

/* lrfsi_mesh: build the Q2/Q2/Q1 DOF layout of the channel, the Dirichlet
 * data b_D (parabolic inflow, no-slip walls, v = 0 on the closed solid,
 * u = 0 on the outer boundary), the CSR union pattern of the affine operators
 * (Sec. 3, Eq. (pardep_matrix1)), the cell -> CSR scatter map and the slab
 * structure of the preconditioner LU; upload them to the current device.
 * Errors: LRFSI_EINVAL for nx < 1, ny < 1 or non-positive lengths;
 * LRFSI_ENOMEM / LRFSI_ECUDA on allocation failure. */
int lrfsi_mesh_create(const lrfsi_problem* prob, lrfsi_mesh_h* out);
int lrfsi_mesh_destroy(lrfsi_mesh_h mesh);
int lrfsi_mesh_info(lrfsi_mesh_h mesh, lrfsi_mesh_info_t* info);

/* DOF description (host arrays of length M): field (0 v_x, 1 v_y, 2 u_x,
 * 3 u_y, 4 p) and position of the DOF on the Q2 node grid (ix in [0, 2 nx],
 * iy in [0, 2 ny]; a Q1 vertex (a, b) sits at (2a, 2b)). */
int lrfsi_mesh_dofmap(lrfsi_mesh_h mesh, int32_t* field_host, int32_t* ix_host, int32_t* iy_host);
/* Dirichlet data b_D (host array of length M). */
int lrfsi_mesh_dirichlet(lrfsi_mesh_h mesh, double* bD_host);
/* CSR pattern copies (host; rowptr has M + 1 entries, colidx nnz). */
int lrfsi_mesh_pattern(lrfsi_mesh_h mesh, int32_t* rowptr_host, int32_t* colidx_host);

/* lrfsi_assemble_affine: at the state x, the values of J0(x), Jmu'(x), Jnu'
 * on the union pattern and the residual pieces R0(x), Rmu(x), Rnu(x) with
 *   R(x; mu, nu) = R0 + mu Rmu + nu Rnu,  J(x; mu, nu) = J0 + mu Jmu' + nu Jnu'
 * (Sec. 3, Eq. (pardep_matrix1) with the reference values mu_s = nu_f = 0;
 * Sec. 3.4, Eq. (rhs_matrix1): Rmu = A1 x + g_mu(x), Rnu = rho_f A2 x).
 * FP64, 3 x 3 Gauss quadrature per cell.
 *   x_dev    : M state (device)
 *   J3_dev   : nnz x 3 interleaved values (J0, Jmu', Jnu') per CSR entry, or NULL
 *   R3_dev   : M x 3 row-major (R0, Rmu, Rnu) per row, or NULL
 * Deterministic (cell colouring, no atomics). */
int lrfsi_assemble_affine(lrfsi_mesh_h mesh, const double* x_dev, double* J3_dev, double* R3_dev,
                          lrfsi_stream_t stream);

/* lrfsi_residual_batch: R(X_i; mu_i, nu_i) for m columns (Sec. 2,
 * Eq. (fsi_problem_weak1); Dirichlet rows X_i - b_D).
 *   X_dev   : M x m row-major states, leading dimension ldx >= m
 *   mu_dev, nu_dev : m parameters (device)
 *   R_dev   : M x m row-major output (ldr >= m), or NULL
 *   norm2_dev : m squared Euclidean norms of the columns of R, or NULL */
int lrfsi_residual_batch(lrfsi_mesh_h mesh, const double* X_dev, int ldx, int m,
                         const double* mu_dev, const double* nu_dev, double* R_dev, int ldr,
                         double* norm2_dev, lrfsi_stream_t stream);

/* ---- the four-parameter problem (Sec. 4.4): mu_s, nu_f, lambda_s, rho_f vary;
 * Eq. (matrix_fourpars1) with the reference values set to 0:
 *   J = J0 + mu Jmu' + (nu rho) Jnurho' + lam Jlam' + rho Jrho',  R likewise.
 * The mesh's own rho_f and lambda_s are not used by these entry points. */

/* lrfsi_assemble_affine4: the five affine pieces at x as two interleaved
 * triples on the CSR pattern: J3a = (J0, Jmu', Jnurho'), J3b = (Jlam', Jrho', 0)
 * (nnz x 3 each), and R3a = (R0, Rmu, Rnurho), R3b = (Rlam, Rrho, 0) (M x 3
 * row-major each); any output may be NULL.  The lambda and rho pieces are the
 * differences of assemblies at (rho_f, lambda_s) = (0, 0), (1, 0), (0, 1), exact
 * wherever no other term shares the entry and within rounding elsewhere.
 * Synchronizes the stream (temporaries). */
int lrfsi_assemble_affine4(lrfsi_mesh_h mesh, const double* x_dev, double* J3a_dev, double* J3b_dev,
                           double* R3a_dev, double* R3b_dev, lrfsi_stream_t stream);
/* lrfsi_residual_batch4: R(X_i; mu_i, nu_i, lam_i, rho_i) for m columns (as
 * lrfsi_residual_batch with lam_dev, rho_dev per column; R_dev required). */
int lrfsi_residual_batch4(lrfsi_mesh_h mesh, const double* X_dev, int ldx, int m, const double* mu_dev,
                          const double* nu_dev, const double* lam_dev, const double* rho_dev, double* R_dev,
                          int ldr, double* norm2_dev, lrfsi_stream_t stream);

/* lrfsi_residual_batch_noalloc: the same residual block and column norms as
 * lrfsi_residual_batch, computed without allocating device memory.  (No
 * counterpart in the paper: an interface for callers that cannot let a library
 * allocate -- processes whose device memory belongs to their own pool
 * allocator or fixed budget, where memory taken or returned behind that
 * allocator's back, and the device synchronisation of a cudaMalloc/cudaFree,
 * are not acceptable.)
 *   R_dev is required (M x m, ldr >= m).  The partial sums of the norms live in
 *   a library-owned device array of 2^21 doubles (16 MiB, held by every GPU
 *   that loads the library until the process exits); ceil(M / 256) * m must not
 *   exceed 2^21, else LRFSI_EINVAL.  Calls share that array: calls that
 *   overlap on the GPU (e.g. on two streams) race.  Each call overwrites every
 *   partial it reads, so no clearing is needed between calls.
 *   The first call on a device looks up the array's device address (set-up
 *   once per device, with that device current) and keeps it for the life of
 *   the process: do not use the library across cudaDeviceReset.  Make that
 *   first call before any stream capture.  R alone is computed when norm2_dev
 *   is NULL (the array is then not touched).  Enqueues work on the stream and
 *   does not synchronize. */
int lrfsi_residual_batch_noalloc(lrfsi_mesh_h mesh, const double* X_dev, int ldx, int m,
                                 const double* mu_dev, const double* nu_dev, double* R_dev, int ldr,
                                 double* norm2_dev, lrfsi_stream_t stream);

/* lrfsi_spmm: the affine operator applied to a tall factor (the SpMM of the
 * ChebyshevT residual, Sec. 4: F(U V^T) = [J0 U | Jmu' U | Jnu' U] [V | D_mu V | D_nu V]^T):
 *   Y (M x 3r, row-major, ldy >= 3r) = [J0 U | Jmu' U | Jnu' U]
 *   J3_dev : operator values, nnz x 3 interleaved on the mesh's CSR pattern
 *            (as written by lrfsi_assemble_affine)
 *   U_dev  : M x r row-major (ldu >= r)
 *   precision 0: all arrays FP64; 1: all arrays FP32 (FP32 accumulation).
 * The row/column shape of the kernel is chosen per precision and rank by
 * timing all shapes on first use (see lrfsi_spmm_tuning).  Asynchronous on the
 * stream except for that first timed use. */
int lrfsi_spmm(lrfsi_mesh_h mesh, const void* J3_dev, const void* U_dev, int ldu, int r, void* Y_dev, int ldy,
               int precision, lrfsi_stream_t stream);
/* The SpMM autotuner's table for (precision 0/1, rank bucket ceil(r / 16)
 * capped at 8): chosen shape index (-1 before the first use) and the measured
 * milliseconds of the 9 shapes (lanes per row x columns per lane: 32x1, 32x2,
 * 16x2, 16x4, 8x4, 8x8 gathering U from L2; 32x2, 16x4, 8x8 gathering from a
 * shared-memory window of U staged per block of 128 rows; 0 = not applicable). */
int lrfsi_spmm_tuning(int precision, int bucket, int* variant, float* ms9);

/* lrfsi_residual: relative residuals of the low-rank approximation
 * X = x~ 1^T + U V^T (Sec. 5.1.2): ||R(X_i; mu_i, nu_i)||_2 / ||R(b_D; mu_i, nu_i)||_2
 * for the m columns.
 *   xt_dev : M;  U_dev : M x r (ldu);  V_dev : m x r (ldv); r may be 0
 *   relres_host : m outputs (host).  Synchronizes the stream. */
int lrfsi_residual(lrfsi_mesh_h mesh, const double* xt_dev, const double* U_dev, int ldu,
                   const double* V_dev, int ldv, int r, const double* mu_dev, const double* nu_dev,
                   int m, double* relres_host, lrfsi_stream_t stream);

/* ---- Algorithm 1's parameter bookkeeping (host only: no device work, no GPU
 * needed; every array is a caller-owned host array) ---------------------- */

/* lrfsi_order_grid: the little-endian order of the grid mu_values x nu_values
 * (Sec. 3.3, Def. 1): the parameter with 1-based indices (i1, i2) goes to
 * position i1 + (i2 - 1) m1, i.e. the mu index runs fastest.  nu_fastest != 0
 * swaps the axes (position i2 + (i1 - 1) m2; used where the split of two
 * subsets must run along mu).  Outputs mu_out, nu_out have m1 m2 entries.
 * Errors: LRFSI_EINVAL for m1 < 1, m2 < 1 or NULL arrays. */
int lrfsi_order_grid(int m1, int m2, const double* mu_values_host, const double* nu_values_host,
                     int nu_fastest, double* mu_out_host, double* nu_out_host);

/* lrfsi_order_set: the order of an unstructured parameter set (the paper
 * orders grids only; this carries Def. 1 over): by nu_f, then by mu_s, equal
 * pairs in input order.  perm_host[p] = input index of the p-th parameter.
 * Errors: LRFSI_EINVAL for m < 0, NULL arrays or a NaN parameter. */
int lrfsi_order_set(int m, const double* mu_host, const double* nu_host, int32_t* perm_host);

/* lrfsi_cluster: K contiguous subsets of m ordered parameters (Eq.
 * (clustering1): |I_k| = floor(m / K) for k < K, the remainder for k = K),
 * their first positions (offsets, 0-based) and the 0-based global position of
 * each subset's upper median (Sec. 3.3: 1-based position floor(|I_k| / 2) + 1
 * within the subset).  offsets_host and medians_host may be NULL.
 * Errors: LRFSI_EINVAL unless 1 <= K <= m. */
int lrfsi_cluster(int m, int K, int32_t* sizes_host, int32_t* offsets_host, int32_t* medians_host);

/* lrfsi_medians: offsets and upper-median positions (as lrfsi_cluster) for
 * given subset sizes (uneven subsets).  Errors: LRFSI_EINVAL for K < 1 or an
 * empty subset. */
int lrfsi_medians(int K, const int32_t* sizes_host, int32_t* offsets_host, int32_t* medians_host);

/* lrfsi_partition: split K subsets into nproc contiguous blocks, balanced by
 * the per-subset weights (e.g. m_k R_k, the work of a subset step).  The K
 * subsets are independent (Sec. 2), so a process solves whole subsets.
 * first_host (nproc + 1 entries): process p owns subsets
 * [first[p], first[p + 1]); the largest block weight is the smallest possible
 * for contiguous blocks (binary search on the bound, greedy fill), and no
 * process is left without a subset while K >= nproc.
 * Errors: LRFSI_EINVAL for K < 0, nproc < 1, NULL arrays or negative weights. */
int lrfsi_partition(int K, const int64_t* weights_host, int nproc, int32_t* first_host);

/* lrfsi_lu_mode: the sparse LU of the Newton steps (Sec. 3.2) and of the
 * mean-based preconditioners (Sec. 4.2; the paper factors them with a
 * permuted sparse LU):
 *   1 (default): nested dissection -- the node grid is bisected recursively
 *      along vertex lines; every separator is a dense front, fronts of one
 *      height in the separator tree are factored together (panel LU with
 *      partial pivoting among the front's fully summed rows, explicit inverse
 *      of its pivot block, Schur complement by GEMM, extend-add into the
 *      parent), and a solve is two level-scheduled sweeps of GEMMs;
 *   0: the slab-ordered block-tridiagonal LU (dense slab blocks, block Thomas).
 * Applies to handles created (and Newton calls made) after the call.
 * mode = -1 only queries; *previous (may be NULL) receives the old mode. */
int lrfsi_lu_mode(int mode, int* previous);
/* lrfsi_lu_info: host-only analysis of the nested dissection for a problem
 * (no device work): out8 = {fronts, tree heights, largest separator, largest
 * boundary, doubles of one factorisation, FP64 flops of one factorisation,
 * FP64 flops of the slab block LU, doubles of the slab block LU}. */
int lrfsi_lu_info(const lrfsi_problem* prob, int64_t* out8);

/* lrfsi_newton_median: Newton iteration for K independent problems
 * (Sec. 3.2, Eq. (newton_step_indiv1)), batched: every iteration assembles
 * J(x_k; mu_k, nu_k), R(x_k; mu_k, nu_k), factors all K Jacobians with the
 * block-tridiagonal FP64 LU and solves.  Stops a problem when ||R||_2 <= eps
 * (absolute, as in Algorithm 1).  If the full step raises the residual norm the
 * step is halved (up to 8 times).
 *   X_dev   : K x M states (problem k at X_dev + k*M); in: start, out: result
 *   mu_host, nu_host : K parameters
 *   iters_host, res_host : K outputs (iterations, final residual norm), or NULL
 * Returns LRFSI_ENOCONV if a problem did not reach eps in max_it iterations
 * (its best iterate is left in X). */
int lrfsi_newton_median(lrfsi_mesh_h mesh, int K, double* X_dev, const double* mu_host,
                        const double* nu_host, double eps, int max_it, int* iters_host,
                        double* res_host, lrfsi_stream_t stream);

/* lrfsi_newton_median4: lrfsi_newton_median for the four-parameter problem
 * (Sec. 4.4): lam_host, rho_host (K) give lambda_s and rho_f per problem. */
int lrfsi_newton_median4(lrfsi_mesh_h mesh, int K, double* X_dev, const double* mu_host, const double* nu_host,
                         const double* lam_host, const double* rho_host, double eps, int max_it, int* iters_host,
                         double* res_host, lrfsi_stream_t stream);

/* ---- the time-dependent problem with the theta-scheme (Sec. 4.3,
 * Eq. (fsi_problem_time_weak1)).  One time step t_{i-1} -> t_i for parameter
 * (mu, nu) solves
 *   R_theta(x) = (rho_f A_t^f / dt)(x - x_prev) + theta R(x; mu, nu)
 *                + (1 - theta) R(x_prev; mu, nu) = 0,
 * A_t^f the fluid velocity mass <v, phi>_F in the fluid momentum rows.  The
 * solid is quasi-static (v = 0 on the closed solid, the stationary row
 * ownership: the weak form states no kinematic equation, so rho_s <d_t v,
 * phi>_S vanishes); b_D does not depend on time. */

/* lrfsi_mass_fluid: the values of A_t^f on the mesh's CSR pattern (nnz). */
int lrfsi_mass_fluid(lrfsi_mesh_h mesh, double* M_dev, lrfsi_stream_t stream);
/* lrfsi_newton_theta: Newton for one time step of K problems (Eq.
 * (time_indiv1)): matrix rho_f A_t^f / dt + theta J(x; mu, nu), residual
 * R_theta.  X_dev (K x M): in the start, out the solution; Xprev_dev (K x M)
 * the previous time step.  0 < theta <= 1, dt > 0.  Full Newton steps (no
 * halving: from x_prev the first step usually raises ||R_theta|| before the
 * quadratic phase).  Other arguments and errors as lrfsi_newton_median. */
int lrfsi_newton_theta(lrfsi_mesh_h mesh, int K, double* X_dev, const double* Xprev_dev, const double* mu_host,
                       const double* nu_host, double theta, double dt, double eps, int max_it, int* iters_host,
                       double* res_host, lrfsi_stream_t stream);

/* Options of the low-rank solvers (truncated Chebyshev iteration and truncated GMRES). */
typedef struct {
  double c, d;        /* half-width and centre of the spectrum of P^{-1} A (Sec. 5.1.1);
                         ChebyshevT only */
  int iters;          /* steps per cycle (paper: 6; GMREST: Arnoldi steps before a restart) */
  int cycles;         /* 1 + restarts (paper: 2) */
  int rank_cap;       /* R: maximal rank kept by the truncation */
  double tol;         /* truncation: keep the smallest r with ||s_{>r}|| <= tol ||s|| */
  double eta;         /* stop when ||B - F(S)||_F <= eta ||B||_F (0: run all steps) */
  int precision;      /* 0: FP64; 1: mixed: the inner residual B - F(S) in FP32 (SpMM
                         and GEMM, FP32 accumulation), truncated at 1e-6 (its noise
                         level); LU, Gram products, SVD and the outer loop in FP64 */
  double tol_sol;     /* lrfsi_subset_step: truncation tolerance of the accumulated solution
                         (0: 1e-6 * tol).  In the equilibrated norm a deformation error of
                         relative size e costs about 1e6 e in the unscaled relative residual,
                         so the accumulated Newton update needs a tighter tolerance than the
                         inner iteration. */
  int solver;         /* lrfsi_subset_step / _init: 0 ChebyshevT, 1 GMREST (Algorithm 1 step 3
                         allows either); lrfsi_chebyshevT and lrfsi_gmresT ignore it */
} lrfsi_cheb_options;

typedef struct {
  int steps;              /* Chebyshev steps (GMREST: Arnoldi steps) taken */
  int rank;               /* rank of the returned S */
  double rel_lin_res;     /* ||B - F(S)||_F / ||B||_F at the last evaluation */
  int max_concat_rank;    /* largest rank fed to a truncation */
} lrfsi_cheb_stats;

typedef struct lrfsi_subset_s* lrfsi_subset_h;

/* A subset handle holds K >= 1 subsets I_1..I_K (Sec. 3.3, Eq. (clustering1));
 * every operation below advances all K subsets together in batched kernels.
 * Subset k owns m_k consecutive entries of the concatenated parameter arrays
 * (offset o_k = m_1 + ... + m_{k-1}).  Per-subset tall outputs are stacked:
 * subset k's M x ld block starts at ptr + k * M * ld; per-subset V blocks are
 * stacked by rows: subset k's m_k x ldv block starts at ptr + o_k * ldv. */

/* lrfsi_subset_create: operators and preconditioners of K subsets (Sec. 3.4
 * and Sec. 4.2) at their linearisation points xt_k (the upper-median Newton
 * solutions): assembles J0, Jmu', Jnu', R0, Rmu, Rnu at xt_k and factors
 * P_k = J(xt_k; mu_bar_k, nu_bar_k) with the block-tridiagonal FP64 LU,
 * mu_bar_k / nu_bar_k the midpoints of the subset's parameter ranges.
 *   xt_dev        : K x M linearisation points (device, row k at xt_dev + k*M)
 *   mu_host, nu_host : sum m_k parameters, subsets consecutive
 *   m_host        : K subset sizes (m_k >= 1)
 *   rank_cap_host : K rank capacities R_k (1 <= R_k)
 * Errors: LRFSI_EINVAL on bad sizes, LRFSI_ESINGULAR if an LU pivot is zero. */
int lrfsi_subset_create(lrfsi_mesh_h mesh, int K, const double* xt_dev, const double* mu_host,
                        const double* nu_host, const int* m_host, const int* rank_cap_host,
                        lrfsi_subset_h* out, lrfsi_stream_t stream);
/* lrfsi_subset_create4: subsets of the four-parameter problem (Sec. 4.4,
 * Eq. (matrix_fourpars1)): operators J0, Jmu', Jnurho', Jlam', Jrho' at xt_k,
 * the mean-based preconditioner at the midpoints of the ranges of mu, nu rho,
 * lambda and rho, and in every solve the five-term operator
 *   J0 S + Jmu' S D_mu + Jnurho' S D_{nu rho} + Jlam' S D_lam + Jrho' S D_rho
 * with the rank-5 right-hand side B^{mu,nu,lambda,rho}.  lam_host, rho_host:
 * sum m_k values.  ChebyshevT only (GMREST returns LRFSI_EINVAL). */
int lrfsi_subset_create4(lrfsi_mesh_h mesh, int K, const double* xt_dev, const double* mu_host,
                         const double* nu_host, const double* lam_host, const double* rho_host, const int* m_host,
                         const int* rank_cap_host, lrfsi_subset_h* out, lrfsi_stream_t stream);
/* lrfsi_subset_create_theta: subsets of one time step (Sec. 4.3, Eq.
 * (timedep_matrix1)): at the median's time-step solutions xt_k the operators
 * (theta J0 + rho_f A_t^f / dt, theta Jmu', theta Jnu') and the mean-based
 * preconditioner of their affine sum; use with lrfsi_subset_step_theta. */
int lrfsi_subset_create_theta(lrfsi_mesh_h mesh, int K, const double* xt_dev, const double* mu_host,
                              const double* nu_host, const int* m_host, const int* rank_cap_host, double theta,
                              double dt, lrfsi_subset_h* out, lrfsi_stream_t stream);
int lrfsi_subset_destroy(lrfsi_subset_h sub);

/* lrfsi_chebyshevT: solve F_k(S_k) = B_k for every subset on the factors
 * (B_k = UB_k VB_k^T) with the truncated preconditioned Chebyshev iteration
 * (the paper's ChebyshevT; recurrence: centre d, half-width c, left
 * preconditioning by P_k, truncation after every update of the iterate, the
 * residual before preconditioning and the direction; restart = new cycle).
 *   UB_dev : K stacked M x lduB blocks;  VB_dev : stacked m_k x ldvB blocks
 *   rB_host: K right-hand-side ranks (1 <= rB_k <= lduB, ldvB)
 *   U_dev  : K stacked M x ldu output blocks (ldu >= R_k)
 *   V_dev  : stacked m_k x ldv output blocks (ldv >= R_k)
 *   rank_host : K output ranks r_k (S_k = U_k[:, :r_k] V_k[:, :r_k]^T)
 *   stats  : K entries or NULL */
int lrfsi_chebyshevT(lrfsi_subset_h sub, const double* UB_dev, int lduB, const double* VB_dev,
                     int ldvB, const int* rB_host, const lrfsi_cheb_options* opt, double* U_dev,
                     int ldu, double* V_dev, int ldv, int* rank_host, lrfsi_cheb_stats* stats,
                     lrfsi_stream_t stream);

/* lrfsi_gmresT: the same problem and arguments as lrfsi_chebyshevT, solved with
 * the truncated GMRES (the paper's GMREST, Sec. 4 Algorithm 1 step 3 and
 * Sec. 5.1, cited from [WeiBR20] without being restated; c and d are not used).
 * Restarted GMRES with right preconditioning by P_k, so that it minimises the
 * true residual ||B_k - F_k(S)||_F; Frobenius inner products computed from the
 * Gram blocks of the factors (U_a^T U_b, V_a^T V_b); classical Gram-Schmidt;
 * the truncation (tol, rank cap R_k) applied to the starting residual, to
 * F(P^{-1} V_j), to the orthogonalised vector and to the updated iterate.  A
 * cycle is `iters` Arnoldi steps; it ends early when h_{j+1,j} = 0 or the
 * least-squares residual falls to eta ||B_k||_F.  stats[k].steps counts Arnoldi
 * steps.  On first use the handle allocates the Krylov basis (2 iters tall
 * factors per subset) and widens its concatenation buffers to
 * (iters + 1) max_k R_k columns, so that every sum is truncated at once; the
 * same happens in lrfsi_subset_step / _init with opt->solver = 1.  Errors as
 * lrfsi_chebyshevT (LRFSI_ENOMEM if that allocation fails; the handle stays
 * usable). */
int lrfsi_gmresT(lrfsi_subset_h sub, const double* UB_dev, int lduB, const double* VB_dev, int ldvB,
                 const int* rB_host, const lrfsi_cheb_options* opt, double* U_dev, int ldu,
                 double* V_dev, int ldv, int* rank_host, lrfsi_cheb_stats* stats, lrfsi_stream_t stream);

/* lrfsi_subset_step: one Newton step on every subset (Sec. 3.4,
 * Eq. (rhs_matrix1), Eq. (newton_matrix1)): B_k = -(R0 1^T + Rmu mu^T + Rnu nu^T),
 * S_k = ChebyshevT(B_k) (GMREST if opt->solver = 1); then, while some
 * column's relative residual exceeds target and fewer than max_outer
 * corrections were taken, a correction in the
 * same matrix form whose right-hand side is -R(X_i; mu_i, nu_i) evaluated
 * column by column (operators and preconditioners kept at xt_k; the sum of
 * corrections is truncated with the same rule).  Result per subset:
 * X_k = xt_k 1^T + U_k V_k^T of rank r_k.
 *   relres_host : sum m_k final relative residuals (Sec. 5.1.2), or NULL
 *   outer_host  : K correction counts, or NULL
 * Returns LRFSI_ENOCONV if target > 0 was not reached by every column. */
int lrfsi_subset_step(lrfsi_subset_h sub, const lrfsi_cheb_options* opt, double target,
                      int max_outer, double* U_dev, int ldu, double* V_dev, int ldv,
                      int* rank_host, double* relres_host, int* outer_host,
                      lrfsi_stream_t stream);

/* lrfsi_subset_step_theta: one time step on every subset of a handle from
 * lrfsi_subset_create_theta: the Newton step of Eq. (timedep_matrix1) at
 * X = xt_k 1^T with the right-hand side -R_theta evaluated column by column
 * (the (***) term exactly), then chord corrections with -R_theta of the
 * current columns, until every column's ||R_theta||_2 / ||R(b_D; mu, nu)||_2
 * <= target or max_outer solves (>= 1).
 *   Xprev_dev : M x (sum m_k) row-major (ldx >= sum m_k), the previous time
 *               step's states of the columns in subset order
 * Outputs as lrfsi_subset_step (outer counts include the Newton step). */
int lrfsi_subset_step_theta(lrfsi_subset_h sub, const lrfsi_cheb_options* opt, const double* Xprev_dev, int ldx,
                            double target, int max_outer, double* U_dev, int ldu, double* V_dev, int ldv,
                            int* rank_host, double* relres_host, int* outer_host, lrfsi_stream_t stream);

/* lrfsi_subset_step_init: lrfsi_subset_step from a given start instead of the
 * first Newton step: X0_k = x~_k 1^T + U0_k V0_k^T (e.g. the learned start,
 * lrfsi_learned_factors).  The start is truncated to the rank cap (tolerance
 * tol_sol); every column whose residual norm at X0 is not below that of the
 * median solution x~_k falls back to x~_k (fallback_host, sum(m_k) ints, 1 for
 * those columns; may be NULL).  Then the chord corrections of
 * lrfsi_subset_step run until every column reaches target.
 *   U0_dev: K stacked M x ldu0 blocks; V0_dev: sum(m_k) x ldv0; r0_host (K):
 *   columns of the start factors (0 = start at x~_k).  Outputs as
 *   lrfsi_subset_step. */
int lrfsi_subset_step_init(lrfsi_subset_h sub, const lrfsi_cheb_options* opt, double target, int max_outer,
                           const double* U0_dev, int ldu0, const double* V0_dev, int ldv0, const int* r0_host,
                           double* U_dev, int ldu, double* V_dev, int ldv, int* rank_host, double* relres_host,
                           int* outer_host, int* fallback_host, lrfsi_stream_t stream);

/* lrfsi_graph_mode: how ChebyshevT (lrfsi_chebyshevT and the ChebyshevT
 * solves inside lrfsi_subset_step / _init) issues its work (Algorithm 1 step
 * 3; no counterpart in the paper: a batching choice):
 *   0: launches sized from ranks read back to the host after every truncation;
 *   1: a fixed launch sequence for all subsets of the handle -- widths fixed at
 *      the rank caps (columns beyond a rank are zero), ranks and the eta test
 *      kept on the device as flags that gate every later launch of a subset,
 *      the optional third Cholesky-QR pass gated by the flag its first pass
 *      writes; no host read inside a solve;
 *   2 (default): the sequence of mode 1 captured once per handle and option set
 *      into a CUDA graph (on a stream the handle owns, after one direct run)
 *      and replayed with one graph launch per solve.  If the capture fails the
 *      process falls back to mode 1 (counted by lrfsi_graph_counters).
 * Modes 1 and 2 equal mode 0 up to rounding (zero columns change sums only
 * by their order).  While kernel timing (lrfsi_timing) is on, mode 2 launches
 * the sequence directly.  mode = -1 only queries.  *previous (may be NULL)
 * receives the mode before the call.  Process-wide; set it between calls. */
int lrfsi_graph_mode(int mode, int* previous);
/* Graph replays, captures and capture failures since the last reset. */
int lrfsi_graph_counters(int64_t* out3, int reset);

/* lrfsi_precond_apply: Y_k = P_k^{-1} X_k with the factored mean-based
 * preconditioner of subset k (Sec. 4.2), for r_k columns.
 *   X_dev : K stacked M x ldx blocks (not modified);  Y_dev : K stacked M x ldy
 *   r_host: K column counts (0 <= r_k <= min(ldx, ldy, rank capacity + m_k)) */
int lrfsi_precond_apply(lrfsi_subset_h sub, const double* X_dev, int ldx, const int* r_host,
                        double* Y_dev, int ldy, lrfsi_stream_t stream);

/* lrfsi_truncate: the truncation operator T (Sec. 5: for an order-2 tensor
 * the best rank-<=R approximation in the Frobenius norm, Eckart-Young) of
 * X_k V_k^T for every subset: keep the smallest rank r with
 * ||s_{>r}||_2 <= tol ||s||_2, at most cap_k; returns U_k (orthonormal columns)
 * and V_k (carrying the singular values) with X_k V_k^T ~ U_k V_k^T.  The
 * inputs are used as given (no equilibration).
 *   X_dev : K stacked M x ldx blocks;  V_dev : stacked m_k x ldv blocks
 *   p_host: K input ranks (1 <= p_k <= ldx, ldv, internal capacity)
 *   U_dev : K stacked M x ldu;  Vo_dev : stacked m_k x ldvo;  rank_host: K */
int lrfsi_truncate(lrfsi_subset_h sub, const double* X_dev, int ldx, const double* V_dev, int ldv,
                   const int* p_host, double tol, const int* cap_host, double* U_dev, int ldu,
                   double* Vo_dev, int ldvo, int* rank_host, lrfsi_stream_t stream);

/* lrfsi_gram: the Gram product G = A^T B of two tall FP64 factors (the
 * CholeskyQR2 Gram of the truncation, Sec. 5; the Arnoldi products of
 * GMREST), G[i][j] = sum_l A[l][i] B[l][j].
 *   A_dev: M x p (row-major, lda >= p);  B_dev: M x q (ldb >= q); B_dev ==
 *   A_dev with ldb == lda and q == p is the symmetric product (only its upper
 *   tiles are computed);  G_dev: p x q (row-major, ldg >= q), written.
 * Path as set by lrfsi_gram_path.  The call allocates its own workspace.
 * Errors: LRFSI_EINVAL for M < 1, p or q < 1, short leading dimensions or NULL
 * pointers; LRFSI_ENOCONV if a pipeline wait of the tensor-core path ran out
 * (G is then wrong). */
int lrfsi_gram(const double* A_dev, int lda, int p, const double* B_dev, int ldb, int q, int64_t M, double* G_dev,
               int ldg, lrfsi_stream_t stream);
/* lrfsi_gemm: C = alpha A B + beta C for row-major FP64 A (m x k, lda >= k),
 * B (k x n, ldb >= n), C (m x n, ldc >= n); beta == 0 does not read C.  With
 * tensor != 0 and lrfsi_gram_path 1 a tall product (m >= 2048, k <= 400) runs
 * on the tensor cores like the Gram products: the contraction index is equilibrated (column
 * l of A and row l of B scaled by inverse powers of two), A split by rows and
 * B by columns into 8 BF16 digit slices, the 36 slice products of a 16-step
 * chunk of k accumulated exactly (FP32 in tensor memory, k <= 400 keeps every
 * level below 2^24), the 8 levels combined as two exact int64 groups and one
 * FP64 fma; the error is below 2^-53 (|A'| |B'|) scaled by the row and column
 * maxima, comparable to an FP64 GEMM's.  Otherwise FP64 FMA kernels.
 * The library uses the tensor path for the tall products inside ChebyshevT
 * and GMREST (the truncation's bases and outputs, B - F(S), the right-hand
 * side); the dense columns whose nonlinear residuals are reported are formed
 * by the FP64 kernels.  Errors as lrfsi_gram. */
int lrfsi_gemm(int m, int n, int k, const double* A_dev, int lda, const double* B_dev, int ldb, double* C_dev,
               int ldc, double alpha, double beta, int tensor, lrfsi_stream_t stream);
/* lrfsi_gram_path: how every Gram product (and every tall GEMM, see lrfsi_gemm)
 * of the library is computed:
 *   1 (default): on the BF16 tensor cores by error-free splitting (Ozaki,
 *      Ogita, Oishi, Rump 2012): each column scaled by a power of two and cut
 *      into 8 base-128 digits exact in BF16; the digit products summed over
 *      256-row windows are exact in the FP32 accumulators (tcgen05.mma into
 *      tensor memory) and added as integers; the 8 digit levels are combined
 *      in FP64.  The inputs enter as 56-bit fixed point relative to their
 *      column's largest entry: the error is that of an FP64 Gram.
 *   0: FP64 FMA kernels.
 * mode = -1 only queries; *previous (may be NULL) receives the old path. */
int lrfsi_gram_path(int path, int* previous);

/* lrfsi_svd_cluster: the thread-block cluster size of the truncation's Jacobi
 * SVD (CTAs per problem): 0 (default) chooses it from the number of problems
 * of a launch (16 up to 9 problems, 8 up to 19, 4 up to 38, else 2); 2, 4, 8
 * or 16 force it (16 only where the device co-schedules 16-CTA clusters).
 * A tuning knob: the results do not depend on it.  size = -1 only queries. */
int lrfsi_svd_cluster(int size, int* previous);

/* ---- Learned initial guess (not a method of the paper) -------------------
 * A multilayer perceptron maps the scaled parameters z = (mu_s, nu_f) in
 * [-1, 1]^2 to k coefficients of a POD basis of method-generated solutions:
 * n_in -> n_h1 -> n_h2 -> n_out with exact-erf GELU after the hidden layers,
 * BF16 weights, FP32 biases and FP32 accumulation; trained by mean squared
 * error with Adam (FP32 master weights).  Its prediction starts the median
 * Newton iteration; the plain start b_D remains the fallback.
 * Packed parameter layout (host float arrays): for each layer l, the weight
 * matrix W_l (n_{l+1} x n_l, row-major) followed by the bias b_l. */
typedef struct lrfsi_mlp_s* lrfsi_mlp_h;
int lrfsi_mlp_create(int n_in, int n_h1, int n_h2, int n_out, lrfsi_mlp_h* out);
int lrfsi_mlp_destroy(lrfsi_mlp_h mlp);
int64_t lrfsi_mlp_num_params(lrfsi_mlp_h mlp);
/* Set (and reset the Adam state) / get the FP32 master parameters (host). */
int lrfsi_mlp_set_params(lrfsi_mlp_h mlp, const float* packed_host);
int lrfsi_mlp_get_params(lrfsi_mlp_h mlp, float* packed_host);
/* Y (B x n_out) = MLP(Z (B x n_in)); device arrays, row-major. */
int lrfsi_mlp_forward(lrfsi_mlp_h mlp, const float* Z_dev, int B, float* Y_dev, lrfsi_stream_t stream);
/* Gradients of L = mean((MLP(Z) - T)^2) w.r.t. the packed parameters into
 * grad_dev (or the handle's buffer if NULL) and L into loss_dev (or NULL). */
int lrfsi_mlp_gradients(lrfsi_mlp_h mlp, const float* Z_dev, const float* T_dev, int B, float* grad_dev,
                        float* loss_dev, lrfsi_stream_t stream);
/* epochs full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8); loss_host: last loss. */
int lrfsi_mlp_train(lrfsi_mlp_h mlp, const float* Z_dev, const float* T_dev, int B, int epochs, float lr,
                    float* loss_host, lrfsi_stream_t stream);
/* lrfsi_learned_fit: build the start model from n method-generated solutions.
 *   X_dev : n solutions, problem-major (row j = solution j, length M, stride
 *           ldx >= M), e.g. the output of lrfsi_newton_median.
 *   mu_host, nu_host : their n parameters;  box = {mu_lo, mu_hi, nu_lo, nu_hi}
 *           maps the parameters to z in [-1, 1]^2.
 *   Steps (all on the device): offset = mean snapshot; field_scale = RMS of the
 *   centred snapshots per field (v_x, v_y, u_x, u_y, p); POD of the centred,
 *   field-scaled snapshots (lrfsi_pod) into Phi (M x k, ldphi); coef_scale[l] =
 *   RMS of coefficient l; then epochs Adam steps fitting MLP(z_j) to the scaled
 *   coefficients, a third each at learning rate lr, lr / 4 and lr / 16.  The MLP must be 2 -> .. -> k and
 *   hold its initial parameters.  Outputs are caller-owned device arrays
 *   (coef_scale: k, field_scale and offset: M); loss_host / sigma_host (k) may
 *   be NULL.  Synchronizes the stream. */
int lrfsi_learned_fit(lrfsi_mesh_h mesh, lrfsi_mlp_h mlp, const double* mu_host, const double* nu_host, int n,
                      const double* box, const double* X_dev, int ldx, int k, int epochs, float lr,
                      double* Phi_dev, int ldphi, double* coef_scale_dev, double* field_scale_dev,
                      double* offset_dev, float* loss_host, double* sigma_host, lrfsi_stream_t stream);
/* lrfsi_learned_start: X (B x M, problem-major, device) = offset + field_scale
 * .* (Phi (coef_scale .* MLP(z))) with Dirichlet rows set to b_D, for the B
 * parameters (host arrays, box as above).  Every column whose residual norm is
 * not below that of b_D falls back to b_D; fallback_host (B ints, or NULL)
 * receives 1 for those columns.  Synchronizes the stream. */
int lrfsi_learned_start(lrfsi_mesh_h mesh, lrfsi_mlp_h mlp, const double* mu_host, const double* nu_host, int B,
                        const double* box, const double* Phi_dev, int ldphi, int k, const double* coef_scale_dev,
                        const double* field_scale_dev, const double* offset_dev, double* X_dev,
                        int* fallback_host, lrfsi_stream_t stream);

/* lrfsi_learned_factors: the learned start of K subsets as factors relative
 * to their median solutions, X0_k - x~_k 1^T = U0_k V0_k^T with
 *   U0_k = [offset - x~_k | diag(field_scale) Phi]  (M x (k+1), Dirichlet rows 0)
 *   V0   = [1 | MLP(z) diag(coef_scale)]            (one row per parameter)
 * sizes_h (K): parameters per subset; mu_host, nu_host: all parameters in
 * subset order; xt_dev: the K median solutions (K x M, problem-major); U0_dev:
 * K stacked M x ldu0 blocks; V0_dev: sum(sizes) x ldv0 (ldu0, ldv0 >= k + 1).
 * Feed to lrfsi_subset_step_init.  Synchronizes the stream. */
int lrfsi_learned_factors(lrfsi_mesh_h mesh, lrfsi_mlp_h mlp, int K, const int* sizes_h, const double* mu_host,
                          const double* nu_host, const double* box, const double* Phi_dev, int ldphi, int k,
                          const double* coef_scale_dev, const double* field_scale_dev, const double* offset_dev,
                          const double* xt_dev, double* U0_dev, int ldu0, double* V0_dev, int ldv0,
                          lrfsi_stream_t stream);

/* lrfsi_pod: rank-k POD of the snapshot columns X (M x n, ldx): the leading k
 * left singular vectors Phi (M x k, ldphi, orthonormal columns) and the
 * coefficients C (n x k, ldc) with X ~ Phi C^T, by the same Cholesky-QR +
 * Jacobi machinery as the truncation T.  sigma_host: k singular values.
 * Directions beyond the numerical rank of X (pivoted-Cholesky remainder below
 * 1e-7 of the column norm) come back as zero columns with zero sigma. */
int lrfsi_pod(lrfsi_mesh_h mesh, const double* X_dev, int ldx, int n, int k, double* Phi_dev, int ldphi,
              double* C_dev, int ldc, double* sigma_host, lrfsi_stream_t stream);

/* Device memory held by a handle (bytes). */
size_t lrfsi_mesh_bytes(lrfsi_mesh_h mesh);
size_t lrfsi_subset_bytes(lrfsi_subset_h sub);

/* Number of kernels this library has launched in the calling process. */
/* Launch calls issued by the host since load: a direct kernel launch or a
 * graph replay counts once (lrfsi_kernel_launches counts the replay's kernels). */
uint64_t lrfsi_host_launches(void);
uint64_t lrfsi_kernel_launches(void);

/* Per-kernel-class accounting for roofline reports.  Classes:
 * 0 FP64 dense GEMM, 1 SpMM (FP64), 2 Gram products (FP64), 3 block-LU
 * factorisations (whole region, contains launches of classes 0, 8 and 9),
 * 4 FE assembly and residuals, 5 FP32 dense GEMM, 6 SpMM (FP32), 7 small
 * per-subset factorisation kernels of the truncation, 8 LU panel kernels
 * (panel factorisation and row interchanges), 9 LU diagonal-block triangular
 * solves, 10 block-LU solves (whole region, contains class-0 launches),
 * 11 the cluster SVD of the truncation (with its QR preconditioning), 12 the
 * slice products of the tensor-core Gram and GEMM kernels alone (BF16 MMA
 * FLOPs actually issued; their launches are also inside classes 13 and 14),
 * 13 FP64 GEMMs on the tensor cores by error-free splitting (whole pipeline;
 * FP64 algorithmic FLOPs), 14 FP64 Gram products the same way.  Classes 0
 * and 2 hold only the GEMMs and Gram products that run on the FP64 units.
 * For every launch the library adds the algorithmic FLOPs and
 * HBM bytes of the launch (from its shape) to the class counters; with timing
 * enabled it also brackets each launch with CUDA events on the launching
 * stream and accumulates the elapsed time when lrfsi_stats is called (which
 * synchronizes those events). */
#define LRFSI_NUM_KERNEL_CLASSES 15
typedef struct {
  uint64_t launches;
  double flops;        /* algorithmic floating-point operations */
  double bytes;        /* algorithmic bytes moved to/from HBM */
  double ms;           /* summed event time (timing enabled only) */
} lrfsi_kernel_stat;
int lrfsi_stats(int kernel_class, lrfsi_kernel_stat* out);
int lrfsi_stats_reset(void);
/* Truncation counters of this process: out6 = {truncations, SVD sweeps (sum),
 * SVD sweeps (max), SVDs stopped at the sweep limit, Cholesky-QR breakdowns,
 * retries}; reset != 0 zeroes them after reading. */
int lrfsi_truncation_counters(int64_t* out6, int reset);
int lrfsi_timing(int enable);

const char* lrfsi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LRFSI_H */
