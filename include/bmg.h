/*
 * bmg.h -- C ABI of libbmg, a GB300 (sm_103a) implementation of the bootstrap
 * multigrid (BMG) eigensolver for the P1 surface finite-element Laplace-Beltrami
 * pencil  A x = lambda M x  (Brannick & Cao, "A Bootstrap Multigrid Eigensolver").
 *
 * The paper states the problem as: given a coarse mesh, a shift mu and a tolerance,
 * compute the eigenpairs (u_{h,i}, lambda_{h,i}) near mu on a uniformly refined mesh
 * (Sec. 4.1, the paragraph after Alg. 2).  The three top-level calls follow it:
 *   bmg_assemble   coarse mesh -> refined meshes, P1 stiffness A and mass M
 *   bmg_hierarchy  prolongations P_l, Galerkin coarse operators, colourings
 *   bmg_solve      BFMG (Alg. 4) with BMG cycles (Alg. 3) -> Ritz pairs near sigma
 * The remaining calls expose the individual steps of the cycle on device buffers;
 * they exist so that each step can be checked on its own.
 *
 * Conventions
 *   - Indices are int32, 0-based.  Matrices are CSR with ascending columns; the
 *     diagonal is stored.  Dense blocks are row-major.  A block of k vectors on a
 *     level with N vertices is "k-interleaved": row-major [N][ld] with ld >= k, the
 *     k values of one vertex contiguous (ld is a multiple of 2 for 16-byte loads;
 *     columns k..ld-1 are padding that every kernel keeps at zero).
 *   - Pointers documented as "device" must be device memory of the current CUDA
 *     device; "host" pointers are ordinary host memory.  Calls that take a
 *     `stream` (a cudaStream_t passed as void*; NULL = legacy default stream)
 *     enqueue their work on it and may return before it completes, unless stated.
 *   - Ownership: a bmg_problem owns every device buffer it allocates and frees it
 *     in bmg_destroy.  Buffers passed in by the caller are never freed.
 *   - Errors: every call returns a bmg_status and never aborts the process.  On an
 *     error the outputs are unspecified (except BMG_ERR_NOT_CONVERGED, see
 *     bmg_solve), and bmg_last_error() returns a message for the calling thread.
 *   - Threads: a bmg_problem must not be used by two threads at once.
 */
#ifndef BMG_H
#define BMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BMG_OK = 0,
  BMG_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported option        */
  BMG_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has details) */
  BMG_ERR_OOM = 3,           /* device allocation failed                         */
  BMG_ERR_SINGULAR = 4,      /* enriched mass matrix rank below k                */
  BMG_ERR_NOT_CONVERGED = 5, /* cycle cap reached; best pairs are returned       */
  BMG_ERR_NONFINITE = 6,     /* NaN/Inf met in the iteration                     */
  BMG_ERR_MESH = 7,          /* input mesh not a closed manifold triangulation   */
  BMG_ERR_STATE = 8,         /* call order violated (e.g. solve before hierarchy)*/
  BMG_ERR_TIMEOUT = 9        /* a bounded wait inside a kernel expired           */
} bmg_status;

/* Smoothers of the source problems (Remark on smoothers after Alg. 1; Sec. 5.3):
 *   BMG_SMOOTH_JACOBI    damped Jacobi, omega (default 2/3)
 *   BMG_SMOOTH_MCGS      multicolour Gauss-Seidel, colours ascending
 *   BMG_SMOOTH_MCSGS     symmetric: ascending then descending colours
 *   BMG_SMOOTH_KACZMARZ  multicolour Kaczmarz, the paper's smoother for the shifted
 *      indefinite problems (Sec. 5.3, Table 2): row r projects x onto its equation,
 *      x += omega (b_r - k_r^T x) / ||k_r||^2 k_r, k_r = a_r - s m_r; the rows of one
 *      colour of a distance-2 colouring (greedy in the same priority) share no column
 *      and are projected at once, which equals the sequential sweep in (colour,
 *      index) order.  Use omega = 1 for plain Kaczmarz.                           */
typedef enum { BMG_SMOOTH_JACOBI = 0, BMG_SMOOTH_MCGS = 1, BMG_SMOOTH_MCSGS = 2,
               BMG_SMOOTH_KACZMARZ = 3 } bmg_smoother;

/* Source problem smoothed for each Ritz pair (theta_i, u_i), lambda_i = theta_i + sigma:
 *   BMG_FORM_SHIFTED:     (A - sigma M) x_i = theta_i M u_i   (Eq. pb-m-s, Alg. 3 step 3)
 *   BMG_FORM_HOMOGENEOUS: (A - lambda_i M) x_i = 0
 * Both start from x_i = u_i and have the same residual there.                       */
typedef enum { BMG_FORM_SHIFTED = 0, BMG_FORM_HOMOGENEOUS = 1 } bmg_form;

/* Arithmetic of the k-blocks during the cycles:
 *   BMG_PREC_FP64: every block, matrix value and product in float64 (the plain method).
 *   BMG_PREC_FP32: the precision form.  Blocks X, AX, MX, U, ... are stored in float32;
 *      SpMM, smoothing, transfers and the Ritz-vector expansion run in float32 with
 *      float32 copies of A, M and the Galerkin operators.  The Gram matrices are
 *      formed from the float32 blocks with error-free products and compensated sums
 *      (float64-class results), and the enriched eigensolve stays float64.  On the
 *      finest level the solve hands over to float64 cycles once every wanted pair
 *      has residual <= switch_tol or the float32 residual stops falling (3 cycles
 *      without halving), and finishes there to tol.  A tol >= switch_tol can be met
 *      in float32 alone.                                                           */
typedef enum { BMG_PREC_FP64 = 0, BMG_PREC_FP32 = 1 } bmg_precision;

typedef struct {
  int smoother;              /* bmg_smoother                                      */
  int nu;                    /* sweeps per level (SGS: forward+backward = 1)       */
  double omega;              /* Jacobi damping (ignored by Gauss-Seidel)           */
  int form;                  /* bmg_form                                          */
  int vcycle_depth;          /* max coarse levels visited after the fine sweeps   */
  int cycles_intermediate;   /* cycle cap on levels 2..L-1                         */
  double tol_intermediate;   /* early stop on levels 2..L-1 (<0: none)             */
  int max_cycles;            /* cycle cap on the finest level                      */
  int precision;             /* bmg_precision                                     */
  double switch_tol;         /* FP32 -> FP64 hand-over residual (BMG_PREC_FP32)    */
  int stop_after_cycles;     /* > 0: stop before cycle stop_after_cycles + 1 and   */
                             /*      keep the state (checkpoint, see below)        */
  int resume;                /* 1: continue from the state given to bmg_set_state  */
  int tensor_cores;          /* 1: the Gram products and the Ritz-vector expansion */
                             /*    run on the tcgen05 tensor cores from exact digit */
                             /*    slices (k <= 128; see bmg_gram_tc), 0: float64  */
                             /*    (float32) fused multiply-adds on the CUDA cores  */
  int autotune;              /* 1: row-kernel shapes timed on first use, 0: default */
  int graphs;                /* 1: cycles replayed as CUDA graphs, 0: eager launches*/
  int adaptive_shift;        /* 1: before the eigensolve of every cycle but the     */
                             /*    solve's first, the shift becomes the mean        */
                             /*    Rayleigh quotient x^T A x / x^T M x of the k     */
                             /*    columns of X (the previous shift plus the mean   */
                             /*    shifted quotient; Alg. 3 step 4, Sec. 5.3); the  */
                             /*    first cycle uses sigma.  0: sigma throughout.    */
  int selection;             /* Ritz pairs kept by every Rayleigh-Ritz (Sec. 5.2):  */
                             /*    0: the k smallest |theta| (index-updating: the   */
                             /*    enrichment follows the spectrum near the shift); */
                             /*    1: index-fixed, positions index_first ..         */
                             /*    index_first + k - 1 of the ascending Ritz values */
                             /*    (moved down when past the top of the values      */
                             /*    present); the wanted pairs are the n_wanted of   */
                             /*    the window nearest the shift.                    */
  int index_first;           /* first position of the index-fixed window (>= 0)   */
  int coarse_start;          /* 1: X0 is ignored (may be NULL) and the start block  */
                             /*    is the k eigenvectors of the level-1 problem     */
                             /*    (the Galerkin pair of level 2 on level 1) chosen */
                             /*    by `selection`, prolongated to level 2 (Alg. 4   */
                             /*    step 1); needs k <= N_1.  0: X0 as given.        */
} bmg_options;

/* Fills the defaults: Jacobi, nu=2, omega=2/3, shifted form, full depth,
 * 6 intermediate cycles, no intermediate tolerance, 200 finest cycles, float64,
 * switch_tol 1e-7 (near the float32 floor of the relative residual), no stop,
 * no resume, tensor cores, autotuned shapes and CUDA graphs on, fixed shift,
 * index-updating selection, start block X0.  autotune and
 * graphs change no result (the tests check bit-identical outputs); tensor_cores
 * changes the rounding of the products.                                          */
void bmg_default_options(bmg_options* opt);

typedef struct bmg_problem bmg_problem;

typedef struct {
  int levels;                /* hierarchy levels (finest = levels)                 */
  int cycles[32];            /* cycles run on level l+2 (levels 2..L)              */
  int total_cycles;
  int converged;             /* 1 if every wanted pair met tol                    */
  double max_resid;          /* largest wanted relative residual at exit          */
  double max_dense_err;      /* largest error estimate of the enriched eigensolve */
  int fp32_cycles;           /* cycles run with float32 blocks (all levels)       */
  int n_history;             /* entries filled below (the first 256 cycles)       */
  int history_level[256];    /* level of each cycle                               */
  int history_fp32[256];     /* 1 if the cycle ran with float32 blocks            */
  double history_resid[256]; /* largest wanted relative residual after the cycle  */
  double final_shift;        /* shift of the last cycle (sigma unless adaptive)   */
} bmg_solve_info;

/* ---------------------------------------------------------------- set-up ----- */

/* Builds the surface hierarchy from a coarse input mesh (Sec. 3; Sec. 2.1).
 *   verts [n_verts][3] host, float64: coarse vertex positions.  They are first
 *         projected onto the surface, as are all new vertices.
 *   tris  [n_tris][3]  host, int32: outward-oriented triangles of a closed
 *         two-manifold (every edge shared by exactly two triangles).
 *   refinements: number of uniform refinements R (0 <= R <= 10).
 *   amplitude, sh_coefs: surface = star-shaped sphere r(n) n with
 *         r(n) = 1 + amplitude * sum_{l<=4} c_lm Y_lm(n); sh_coefs [25] host
 *         (l = 0..4, m = -l..l), ignored when amplitude == 0 (unit sphere).
 *   stream: stream for all set-up work.  Returns after the work completes.
 * Refinement r numbers old vertices first and the midpoint of edge (i<j) as
 * N_{r-1} + rank of (i,j) among the lexicographically sorted edges; the children
 * of triangle t=(a,b,c) are (a,m_ab,m_ca), (b,m_bc,m_ab), (c,m_ca,m_bc),
 * (m_ab,m_bc,m_ca) at 4t..4t+3.  P1 stiffness and mass (Eq. bl-dis, sp-fe) are
 * assembled on every refinement >= 1.
 * Errors: BMG_ERR_INVALID_ARG, BMG_ERR_MESH, BMG_ERR_OOM, BMG_ERR_CUDA.          */
bmg_status bmg_assemble(const double* verts, int n_verts, const int* tris, int n_tris,
                        int refinements, double amplitude, const double* sh_coefs,
                        void* stream, bmg_problem** out);

/* Builds the multilevel structures on levels 1..L, level l = refinement
 * R-L+l (so `levels` = R makes refinement 1 the coarsest level): prolongations
 * P_l (Eq. proj-1: 1 at old vertices, 1/2 at both parents of a midpoint), the
 * restriction P_l^T (Sec. 3), the Galerkin operators P^T A P and P^T M P of every
 * finest level f on every coarser level (Sec. 1.1, Eq. evalapprox), and a greedy
 * colouring per level in descending (splitmix64(v), v) priority.  Synchronous.
 * Errors: BMG_ERR_INVALID_ARG (levels < 2 or > R), BMG_ERR_STATE, BMG_ERR_OOM.   */
bmg_status bmg_hierarchy(bmg_problem* p, int levels);

void bmg_destroy(bmg_problem* p);

/* Thread-local text of the last error (never NULL). */
const char* bmg_last_error(void);

/* ------------------------------------------------------------------ solve ---- */

/* BFMG (Alg. 4) on levels 2..L with BMG cycles (Alg. 3): enriched Rayleigh-Ritz
 * in V_{h_1} + span(X) (Sec. 4.1 block matrices), source-problem smoothing from
 * the finest level down (Alg. 3 step 3), prolongation of the Ritz vectors to the
 * next level.  Returns the n_wanted Ritz pairs nearest sigma on level L.
 *   k: block size (n_wanted <= k <= N_2, k <= 160, N_1 + k <= 224); sigma: shift; tol: the
 *      finest level stops when every wanted pair has
 *      ||A u - lambda M u||_2 / (||A||_1 ||u||_2) <= tol.
 *   opt: options (NULL = defaults).
 *   X0 [N_2][k] row-major float64: initial block on level 2, host memory if
 *      x0_on_device == 0, else device memory.
 *   evals [n_wanted] host: Ritz values, in selection order (|lambda - sigma|
 *      ascending, ties by value then index).
 *   evecs [N_L][n_wanted] row-major float64, host (evecs_on_device == 0) or
 *      device (== 1), or NULL: Ritz vectors, M-orthonormal.
 *   resid [n_wanted] host or NULL: relative residuals.
 *   info: optional host struct.
 * Synchronous.  Errors: BMG_ERR_INVALID_ARG, BMG_ERR_STATE, BMG_ERR_SINGULAR,
 * BMG_ERR_NONFINITE, BMG_ERR_CUDA; BMG_ERR_NOT_CONVERGED fills all outputs with the
 * last Ritz pairs.                                                               */
bmg_status bmg_solve(bmg_problem* p, int k, int n_wanted, double sigma, double tol,
                     const bmg_options* opt, const double* X0, int x0_on_device,
                     double* evals, double* evecs, int evecs_on_device, double* resid,
                     bmg_solve_info* info);

/* Batched form: n_jobs independent solves, job j = (problems[j], sigmas[j]), all with
 * the same k, n_wanted, tol and options (Sec. 4.1 problem statement, once per job).
 * The same problem may appear in several jobs (e.g. one per shift); problems of
 * different sizes mix freely.  Jobs run concurrently on up to `concurrency` streams
 * of the current device (<= 0: min(n_jobs, 64)), one host worker thread per stream,
 * so that the single-block kernels of small levels and of the enriched eigensolves
 * of different jobs overlap on the GPU.  Each job's results are those bmg_solve
 * gives for it (the same kernels and reduction orders).
 *   X0[j] [N_2][k] host; evals[j] [n_wanted] host; evecs[j] [N_L][n_wanted] host or
 *   evecs == NULL; resid[j] [n_wanted] host or resid == NULL; infos [n_jobs] or NULL.
 * Per-problem workspaces (one per job of that problem) are kept between calls.
 * Synchronous.  Returns the first failing job's status (message names the job),
 * else BMG_ERR_NOT_CONVERGED if a job hit its cycle cap, else BMG_OK.            */
bmg_status bmg_solve_batched(int n_jobs, bmg_problem* const* problems, const double* sigmas,
                             int k, int n_wanted, double tol, const bmg_options* opt,
                             const double* const* X0, double* const* evals,
                             double* const* evecs, double* const* resid,
                             bmg_solve_info* infos, int concurrency);

/* ---------------------------------------------- inspection (host outputs) --- */

/* Checkpoint and resume of bmg_solve at a cycle boundary of the BFMG loop (Alg. 4:
 * the state between two cycles is the level, the cycle count on it, the iterate block
 * on that level in the working arithmetic, the arithmetic phase of the precision form,
 * and the counters and history reported in bmg_solve_info).
 *   A bmg_solve with options.stop_after_cycles = c > 0 stops before its (c+1)-th
 *   cycle (counted over all levels), returns BMG_ERR_NOT_CONVERGED with the last
 *   cycle's Ritz values and residuals (evecs is written only if that cycle ran on
 *   the finest level) and keeps its state with the problem, for block size k.
 *   bmg_get_state copies that state into buf (host, len bytes); *used receives the
 *   size in bytes (buf may be NULL to query it).  BMG_ERR_STATE if no solve of block
 *   size k was stopped; BMG_ERR_INVALID_ARG if len is too small.
 *   bmg_set_state loads a state (host buffer) taken from this or another problem
 *   handle built from the same mesh and hierarchy; the next bmg_solve on (p, k) with
 *   options.resume = 1 and the same n_wanted, sigma, tol and options (other than
 *   stop_after_cycles and resume) continues from it, and its outputs are bit-identical
 *   to those of the uninterrupted solve.  BMG_ERR_INVALID_ARG for a malformed state
 *   or one of another hierarchy; bmg_solve with resume = 1 returns BMG_ERR_STATE
 *   without a state and BMG_ERR_INVALID_ARG if the arguments differ from the state's. */
bmg_status bmg_get_state(const bmg_problem* p, int k, void* buf, size_t len, size_t* used);
bmg_status bmg_set_state(bmg_problem* p, int k, const void* buf, size_t len);

/* Sizes of refinement r (0..R): vertices, triangles, CSR nonzeros.             */
bmg_status bmg_get_sizes(const bmg_problem* p, int refinement, int* n, int* n_tris,
                         int* nnz);
/* Mesh of refinement r: verts [n][3], tris [n_tris][3], parents [n][2] (parents
 * of refinement 0 are (v,v)).  Any output may be NULL.  Host memory.            */
bmg_status bmg_get_mesh(const bmg_problem* p, int refinement, double* verts, int* tris,
                        int* parents);
/* CSR of refinement r >= 1: row_ptr [n+1], col [nnz], a [nnz], m [nnz] (host,
 * any may be NULL).                                                             */
bmg_status bmg_get_csr(const bmg_problem* p, int refinement, int* row_ptr, int* col,
                       double* a, double* m);
/* Galerkin values of finest level f on level j < f (pattern of level j; levels
 * in 1..L as in bmg_hierarchy), host.                                           */
bmg_status bmg_get_galerkin(const bmg_problem* p, int f, int j, double* a, double* m);
/* Colouring of level l (1..L): colour [n] host; returns the colour count.        */
bmg_status bmg_get_colouring(const bmg_problem* p, int level, int* colour,
                             int* n_colours);

/* Distance-2 colouring of level l (1..L), built on first use (the Kaczmarz
 * smoother's): colour [n] host; returns the colour count.                        */
bmg_status bmg_get_colouring2(bmg_problem* p, int level, int* colour, int* n_colours);

/* ------------------------------------- individual cycle steps (device data) -- */
/* All pointers below are device memory; all calls are asynchronous on `stream`.
 * `level` is a hierarchy level (1..L); `f` selects the operator set: f == level
 * means the assembled A_l, M_l; f > level the Galerkin operators of finest level
 * f on `level`.  Blocks are k-interleaved with leading dimension ld.            */

/* [AX | MX] = [A X | M X] in one pass over the shared pattern (matrix form of
 * Eq. pb-f-aux-mat; blocks of Sec. 4.1).                                        */
bmg_status bmg_spmm(const bmg_problem* p, int f, int level, const double* X, int k,
                    int ld, double* AX, double* MX, void* stream);

/* nu sweeps of the smoother on (A - s_i M) x_i = b_i, in place on X
 * (Remark after Alg. 1; Sec. 5.3).  s [k] device shifts; B [N][ld] device right-
 * hand side or NULL for b = 0.  smoother: bmg_smoother; omega used by Jacobi.
 * Jacobi needs a work block: work [N][ld] device (caller-owned).                */
bmg_status bmg_smooth(const bmg_problem* p, int f, int level, double* X, const double* B,
                      const double* s, int k, int ld, int smoother, int nu, double omega,
                      double* work, void* stream);

/* float32 forms of the two calls above (the precision form, BMG_PREC_FP32): float32
 * blocks with ld a multiple of 4, float32 copies of the operators and float32
 * arithmetic.  s [ld] device float32 shifts (zero in the padding).               */
bmg_status bmg_spmm_f32(bmg_problem* p, int f, int level, const float* X, int k, int ld,
                        float* AX, float* MX, void* stream);
bmg_status bmg_smooth_f32(bmg_problem* p, int f, int level, float* X, const float* B,
                          const float* s, int k, int ld, int smoother, int nu, double omega,
                          float* work, void* stream);

/* Y = P_l Xc (level l-1 -> l, Eq. proj-1); with add != 0: Y += P_l Xc.          */
bmg_status bmg_prolong(const bmg_problem* p, int level, const double* Xc, double* Y,
                       int k, int ld, int add, void* stream);
/* Zc = P_l^T R (level l -> l-1).                                                 */
bmg_status bmg_restrict(const bmg_problem* p, int level, const double* R, double* Zc,
                        int k, int ld, void* stream);

/* G[i][j] = sum_r X[r][i] Y[r][j] (k x k, row-major, float64) for X, Y [n][ld],
 * 1 <= k <= 160, k <= ld <= 800.  Synchronous.                                   */
bmg_status bmg_gram(const double* X, const double* Y, int n, int k, int ld, double* G,
                    void* stream);

/* G = X^T Y for float32 blocks X, Y [n][ld] (ld a multiple of 4), float64 result:
 * each product is split exactly into two float32 parts and the sums are
 * compensated (TwoSum), so G is accurate to about 2^-46 sum_r |X[r][i] Y[r][j]|
 * before the float64 summation of the block partials.  1 <= k <= 160. Synchronous.*/
bmg_status bmg_gram_f32(const float* X, const float* Y, int n, int k, int ld, double* G,
                        void* stream);

/* The Rayleigh-Ritz block products of Sec. 4.1 (G = X^T Y, same arguments and
 * result as bmg_gram / bmg_gram_f32) on the tcgen05 tensor cores, 1 <= k <= 128.
 * Each value is turned into an integer relative to the largest exponent of its
 * column over a window of 256 rows and cut into balanced 7-bit digits (BF16 values
 * exactly); the digit products are summed exactly in float32 tensor memory and
 * combined in int64, so only the digit pairs left out and the rounding of the
 * integers contribute error: below 2^-53 (float64 blocks, 8 digits, 36 pairs) or
 * 2^-33 (float32 blocks, 5 digits, 15 pairs) of 256 max|x| max|y| per window.
 * Synchronous.  BMG_ERR_TIMEOUT if a bounded wait inside the kernel expired.     */
bmg_status bmg_gram_tc(const double* X, const double* Y, int n, int k, int ld, double* G,
                       void* stream);
bmg_status bmg_gram_tc_f32(const float* X, const float* Y, int n, int k, int ld, double* G,
                           void* stream);

/* Test of the bounded waits inside the tensor-core kernels (every wait on an
 * mbarrier gives up after a clock limit, frees the kernel's tensor memory and raises
 * an error flag).  Runs a float64 Gram of a zero 4096 x 64 block whose MMA-issuing warp
 * issues nothing, with a wait limit of about 1 ms, so that the waits for the MMA
 * commits expire.  Returns BMG_ERR_TIMEOUT, as a product call after such an expiry
 * does; BMG_ERR_CUDA if the waits did not expire.  The CUDA context stays usable
 * (the tests run a normal Gram after it).  Allocates and frees its own buffers.
 * Synchronous.                                                                      */
bmg_status bmg_tc_timeout_selftest(void* stream);

/* Ritz vectors in the enriched space V_{h1} + span X (Alg. 2 step 4; Alg. 3
 * step 5): U = Z + X Yx for X, Z, U [n][ld] device blocks (Z may be NULL: U = X Yx)
 * and Yx [k][ldy] device float64 coefficients; columns k..ld-1 of U are set to
 * those of Z (zero without Z).  tensor_cores = 0: float64 (or float32) fused
 * multiply-adds on the CUDA cores; 1: digit products on the tcgen05 tensor cores
 * with the digits and error of bmg_gram_tc, scaled per row of X and per column of
 * Yx (k <= 128).  Synchronous.  The f32 form takes float32 blocks (ld % 4 == 0).  */
bmg_status bmg_expand(const double* Z, const double* X, const double* Yx, int n, int k, int ld,
                      int ldy, double* U, int tensor_cores, void* stream);
bmg_status bmg_expand_f32(const float* Z, const float* X, const double* Yx, int n, int k,
                          int ld, int ldy, float* U, int tensor_cores, void* stream);

/* Smallest-|theta| k eigenpairs of the symmetric-semidefinite pencil
 * (Ahat - sigma Mhat) y = theta Mhat y, n x n row-major device matrices (n <= 224):
 * Mhat is scaled to unit diagonal, reduced by a Cholesky factorisation with
 * diagonal pivoting that drops pivots below 1e-12 (rank-deficient enriched
 * spaces), and the reduced standard problem is solved (Alg. 2 step 4): an FP32
 * tridiagonal start refined to FP64 accuracy.  (bmg_solve factors the enriched
 * Mhat in block form, reusing the factor of its coarse-space block.)
 * theta [k], Y [n][k] device; Y^T Mhat Y = I.  rank_out (device int or NULL)
 * receives the kept rank.  Errors: BMG_ERR_INVALID_ARG; a rank below k is
 * reported through bmg_solve as BMG_ERR_SINGULAR.                               */
bmg_status bmg_dense_eig(const double* Ahat, const double* Mhat, int n, double sigma,
                         int k, double* theta, double* Y, int* rank_out, void* stream);

/* The same product as bmg_gram for callers that must not allocate device memory:
 * a framework that has already reserved all device memory for its own pool, a
 * service held to a fixed device-memory budget, or a caller that cannot accept the
 * device-wide wait that freeing memory implies.  The paper has no counterpart; it
 * is a deployment variant.  The block partial sums live in one fixed array inside
 * the library (4 MiB, held by every GPU that loads it until the process exits).
 * The first call on each device looks up that array's device address; make that
 * first call before any stream capture.  Asynchronous on `stream`; no device
 * memory is allocated or freed.  k <= 160 and ld <= 800 (else BMG_ERR_INVALID_ARG;
 * k <= 160 is the Gram kernel's limit).  The array caps the row blocks that run at
 * once at 524288 / k^2 (20 blocks at k = 160, 128 at k = 64, against up to 304 in
 * bmg_gram), so large n at large k runs several times slower than bmg_gram.  All
 * calls share the array: calls whose work overlaps on the GPU (e.g. on two
 * streams) race and give wrong results; order them on one stream.               */
bmg_status bmg_gram_noalloc(const double* X, const double* Y, int n, int k, int ld, double* G,
                            void* stream);

/* ------------------------------------------------------------ measurement --- */
/* Kernel-class timing for benchmarks (no counterpart in the paper).  When enabled,
 * the launches of each class made by any call are bracketed by CUDA events on the
 * stream that runs them; bmg_profile_read waits for them and returns the summed
 * device time, the launch count and the algorithmic bytes and flops those launches
 * had to move / execute (formulas in the library source).  Classes:
 * 0 spmm_am, 1 smooth_sweep, 2 residual, 3 transfer, 4 gram, 5 dense_eig, 6 expand,
 * 7 small.  Process-wide state; not thread-safe.                                 */
bmg_status bmg_profile_enable(int enable);
bmg_status bmg_profile_reset(void);
bmg_status bmg_profile_read(int cls, double* total_ms, long long* launches, double* bytes,
                            double* flops);
const char* bmg_kernel_class_name(int cls);
/* Row-kernel shapes chosen by the autotuner so far (SpMM, Jacobi and residual
 * kernels: lanes per row, 16-byte chunks per lane and warps per block, picked per
 * arithmetic, block width and row count by timing the candidates on first use;
 * bmg_options.autotune = 0 keeps the default shape).  Writes at most len-1 bytes
 * of text and a terminating zero into buf; returns the full length.               */
int bmg_autotune_report(char* buf, int len);
/* Number of kernels libbmg has launched in this process.                         */
long long bmg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* BMG_H */
