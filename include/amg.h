/* amg.h -- C ABI of the GB300 aggregation AMG library.
 *
 * The library implements the method of Gandham, Esler and Zhang, "A GPU
 * Accelerated Aggregation Algebraic Multigrid Method" (arXiv 1403.1649):
 * a setup that builds aggregates from a PMIS(2) maximal independent set on the
 * graph of strong negative connections (Sec. 2.1, Alg. 1-3) and forms coarse
 * operators with a keyed-sum Galerkin product (Sec. 3.1), and a solve that uses
 * K-cycles on the top levels and V-cycles below (Alg. 4, Alg. 5, Sec. 2.2) with
 * damped Jacobi smoothing (Eq. damped Jacobi) as the preconditioner of flexible
 * CG or FGMRES (Sec. 2.2, Sec. 4).  Every step runs in the library's CUDA
 * kernels for sm_103a; there is no CPU fallback.
 *
 * General conventions
 *  - Every call returns AMG_OK (0) on success or a negative AMG_ERR_* code;
 *    no C++ exception crosses the ABI.  amg_last_error() gives a message
 *    (thread-local) for the most recent failure of the calling thread.
 *  - Pointers are plain host or device pointers; the library detects which
 *    with cudaPointerGetAttributes.  Host data is copied in/out inside the
 *    call (the copies are part of the call's cost).  Device data must be on
 *    the current device and is accessed in stream order on `stream`.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous with respect to the host only where stated; the
 *    setup and solve calls synchronise `stream` before returning because they
 *    take host-side decisions (level sizes, convergence).
 *  - Input arrays are borrowed: read during the call, never freed or kept.
 *  - A hierarchy owns all its device memory (from a stream-ordered memory pool
 *    per device that keeps freed blocks for reuse) and releases it in amg_free.
 *    A hierarchy is used by one thread at a time.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define AMG_OK 0
#define AMG_ERR_BAD_INPUT -1     /* malformed CSR, zero diagonal, bad sizes/params   */
#define AMG_ERR_CUDA -2          /* a CUDA runtime call failed (message has details) */
#define AMG_ERR_NOT_CONVERGED -3 /* max_iter reached; iters and res_hist are filled  */
#define AMG_ERR_BREAKDOWN -4     /* Krylov breakdown (p^T A p <= 0, rho <= 0, ...)   */
#define AMG_ERR_NAN -5           /* NaN/Inf in a residual norm                       */
#define AMG_ERR_SETUP -6         /* coarsening failed / coarsest level too large or
                                    not positive definite                            */
#define AMG_ERR_UNSUPPORTED -7   /* option not available for this input              */

/* precision of the preconditioner (matrix values and cycle vectors) */
#define AMG_PREC_F64 0 /* everything FP64                                              */
#define AMG_PREC_F32 1 /* FP32 values and vectors, FP32 accumulation                   */
#define AMG_PREC_BF16 2 /* BF16 matrix values, FP32 vectors and accumulation           */

/* A square sparse matrix in CSR form.  Columns ascending inside each row, the
 * diagonal present and nonzero, int32 indices, FP64 values.  Arrays may be host
 * or device pointers (all three of the same kind). */
typedef struct amg_csr {
  int32_t n;
  int64_t nnz;
  const int32_t *row_ptr; /* n+1 */
  const int32_t *col;     /* nnz */
  const double *val;      /* nnz */
} amg_csr;

typedef struct amg_params {
  double alpha;          /* strength threshold of Sec. 2.1.1 (paper: 0.25 in 2D, 0.5 in 3D) */
  uint64_t seed;         /* seeds the MIS priorities r_i of Alg. 2 and the Arnoldi start    */
  int32_t coarse_max;    /* stop coarsening when n_k <= coarse_max (exact solve below)      */
  int32_t max_levels;    /* cap on the number of levels                                     */
  int32_t kcycle_levels; /* levels k < kcycle_levels get the Krylov-accelerated coarse
                            correction of Alg. 5 (paper: the top two, Sec. 2.2)            */
  double kcycle_t;       /* threshold t of the test ||r~|| <= t ||r|| in Alg. 5            */
  int32_t omega_mode;    /* 0: omega = (4/3)/rho(D^-1 A), rho from 5 Arnoldi steps;
                            1: omega = `omega`                                             */
  double omega;
  int32_t precision;     /* AMG_PREC_* of the preconditioner                                */
  int32_t outer;         /* 0: flexible CG (CG variant of Alg. 5); 1: FGMRES(restart)
                            (GMRES variant)                                                */
  int32_t restart;       /* FGMRES restart length                                           */
  int32_t max_iter;      /* outer iteration cap of amg_solve                                */
  int32_t use_graph;     /* 1: replay one outer iteration as a captured CUDA graph          */
  int32_t smoother;      /* 0: damped Jacobi; 1: per-row polynomial smoother whose
                            coefficients are set with amg_set_poly                         */
  int32_t tail;          /* run the coarse levels (at most 4096 rows, below the K-cycle
                            levels) in one launch per visit: 1 = a cluster of 8 blocks,
                            2 = a single block; 0 = one kernel per step                    */
  int32_t pdl;           /* 1: launch setup and solve kernels with programmatic dependent
                            launch (each kernel waits on its predecessor first)            */
  int32_t autotune;      /* 1: at setup, time each level's SpMV over candidate grid sizes
                            (and, for a batch, the row tile of the per-system inner
                            products) and keep the fastest; the choice is reported in
                            amg_level_info.  Changes rounding order only                  */
  int32_t symmetric;     /* 1: A is symmetric (omega from the Lanczos form of the
                            Arnoldi process; coarsest inverse by Gauss-Jordan sweeps
                            without pivoting, A_L being SPD).  0: nonsymmetric (omega
                            from the eigenvalues of the Arnoldi Hessenberg matrix;
                            coarsest inverse with partial pivoting); needs outer = 1
                            (FGMRES, Sec. 2.2) and a single system                        */
  int32_t mis_k;         /* aggregate roots form an MIS(k), 1..8: 2 is the paper's PMIS(2)
                            (Alg. 2); k > 2 coarsens more aggressively (Sec. 2.1.2): k max
                            rounds per PMIS iteration, aggregates reach distance k        */
} amg_params;

typedef struct amg_level_info {
  int32_t n;          /* unknowns on this level                             */
  int64_t nnz;        /* nonzeros of A_k                                    */
  int32_t n_coarse;   /* n_{k+1} (0 on the coarsest level)                  */
  int32_t mis_rounds; /* PMIS iterations (k max rounds each) of this level  */
  double omega;       /* damped-Jacobi weight of this level                 */
  int32_t spmv_blocks; /* thread blocks of the level's SpMV launches that fuse inner products */
  int32_t seg_tile;    /* rows per tile of the per-system inner products of a
                          batch (0: not a batch)                              */
} amg_level_info;

typedef struct amg_solve_info {
  int32_t iters;         /* outer iterations                                 */
  int32_t status;        /* return code of the last amg_solve                */
  double final_relres;   /* ||b - A x||_2 / ||b||_2 recomputed in FP64 at exit */
  double solve_ms;       /* device time of the last solve (CUDA events)      */
  double setup_ms;       /* device time of the setup (CUDA events)           */
  int64_t kernel_launches; /* kernels of this library launched by the last solve,
                              including the one outer iteration queued after the
                              stopping one (its kernels return at once)          */
  int64_t setup_launches;  /* kernels of this library launched by the setup       */
} amg_solve_info;

typedef struct amg_hierarchy amg_hierarchy;

/* Fill *p with the defaults: alpha 0.25, seed 0, coarse_max 64, max_levels 25,
 * kcycle_levels 2, kcycle_t 0.25, omega_mode 0, omega 2/3, precision F64,
 * outer FCG, restart 30, max_iter 500, use_graph 1, smoother 0, tail 0, pdl 1,
 * autotune 0, symmetric 1, mis_k 2. */
void amg_default_params(amg_params *p);

/* Alg. 1: build the hierarchy of A on the GPU.
 * Per level: strength (Sec. 2.1.1), PMIS(2) (Alg. 2), aggregation (Sec. 2.1.2),
 * interpolation (Alg. 3), Galerkin keyed sum (Sec. 3.1), omega (Eq. damped
 * Jacobi), and finally the dense inverse of the coarsest level (the paper
 * uses SuperLU there, Sec. 3).  The aggregates, interpolation weights and coarse
 * matrices are bit-identical to a sequential FP64 evaluation of those steps.
 * Returns AMG_ERR_BAD_INPUT for a malformed CSR or zero diagonal, AMG_ERR_SETUP
 * if coarsening cannot reach a coarsest level of at most 4096 unknowns or that
 * level is not positive definite.  *out is set only on success. */
int amg_setup(const amg_csr *A, const amg_params *params, void *stream, amg_hierarchy **out);

/* Solve A x = b to ||b - A x||_2 <= tol ||b||_2 with the outer Krylov method of
 * the params, preconditioned by one K-cycle (Alg. 5) per iteration (Sec. 2.2).
 * b: n doubles; x: n doubles holding x0 on entry and the solution on exit
 * (host or device).  iters (nullable) gets the outer iterations; res_hist
 * (nullable, host, length max_iter+1) gets the relative residual norm before
 * the first and after every iteration.  The final residual is recomputed in
 * FP64 (amg_last_solve_info).  Returns AMG_ERR_NOT_CONVERGED if max_iter is
 * reached (iters, res_hist and x still filled), AMG_ERR_BREAKDOWN or
 * AMG_ERR_NAN on numerical failure. */
int amg_solve(amg_hierarchy *h, const double *b, double *x, double tol, int32_t *iters,
              double *res_hist, void *stream);

/* ---- batches of independent systems --------------------------------------
 * nsys systems of different sizes set up as one block-diagonal hierarchy: the
 * setup of Alg. 1 never couples the blocks (no strong connection between
 * them), so every level keeps each system's unknowns contiguous, and the
 * coarsest level is solved with one dense inverse per system.  Coarsening
 * continues until the largest system is at most coarse_max.  The solve runs all
 * systems in the same kernels (one captured CUDA graph per outer iteration)
 * with per-system Krylov scalars: every inner product of flexible CG and of
 * Alg. 5 is taken per system, each system has its own step lengths, branch of
 * Alg. 5 and convergence test, and a converged system stops changing.
 * Flexible CG only (params.outer must be 0). */
int amg_setup_batch(int32_t nsys, const amg_csr *As, const amg_params *params, void *stream,
                    amg_hierarchy **out);

/* b, x: the systems' right-hand sides / initial guesses concatenated in system
 * order (sum of n_s doubles each, host or device); x receives the solutions.
 * iters, relres (host, nsys entries, nullable): outer iterations and final FP64
 * relative residual ||b_s - A_s x_s|| / ||b_s|| of every system.  Returns AMG_OK
 * when every system meets tol, else the first failure code. */
int amg_solve_batch(amg_hierarchy *h, const double *b, double *x, double tol, int32_t *iters, double *relres,
                    void *stream);

/* Values-only re-setup (Sec. 3.1: the pattern of the hierarchy depends only on
 * the aggregates and the pattern of A_0, so the Galerkin products can be
 * repeated from stored summation plans, as between Newton steps).
 * val: the nnz new values of A_0 (host or device), in the CSR order of the
 * matrix given to amg_setup (for a batch: the systems' values concatenated in
 * system order); the sparsity pattern must be unchanged.  The aggregates, P and
 * every coarse pattern are kept; the coarse values are recomputed from the
 * plans, bit-identical to a full setup that finds the same aggregates; then
 * omega, the smoother data and the coarsest factorisation are refilled in
 * place (captured solves stay valid).  Polynomial coefficients set with
 * amg_set_poly or amg_apply_learned_smoother are kept: apply them again to
 * follow the new values.  The device time is reported as setup_ms.
 * Errors: AMG_ERR_BAD_INPUT (zero diagonal or non-finite value);
 * AMG_ERR_UNSUPPORTED (a level whose aggregate runs exceeded 4096 terms has no
 * plan); AMG_ERR_SETUP (coarsest matrix not positive definite). */
int amg_resetup_values(amg_hierarchy *h, const double *val, void *stream);

/* One application of the preconditioner, x = M b (Alg. 5 at level 0 from a
 * zero initial guess).  b, x: n doubles, host or device. */
int amg_precond(amg_hierarchy *h, const double *b, double *x, void *stream);

/* y = A_k x on level k with the solve-phase matrix (in the hierarchy's
 * precision).  x, y: n_k elements of the vector type of the precision (double
 * for F64, float otherwise), DEVICE pointers (host pointers: AMG_ERR_BAD_INPUT).
 * Asynchronous: the kernel is launched on `stream` itself when it is not the
 * legacy default stream (so that calls can be captured into a CUDA graph),
 * else on the hierarchy's internal stream, ordered after the caller's work. */
int amg_spmv(amg_hierarchy *h, int32_t level, const void *x, void *y, void *stream);

/* Per-row polynomial smoother coefficients of level k (n_k x 3, row major,
 * host or device doubles): the smoother applies
 * x += sum_q diag(c_q) (D^-1 A)^q D^-1 r before the coarse correction and the
 * transposed polynomial after it.  Takes effect when params.smoother == 1.
 * coef = NULL returns the level to damped Jacobi.
 * The paper lists polynomial smoothers as future work (Sec. 5). */
int amg_set_poly(amg_hierarchy *h, int32_t level, const double *coef, void *stream);

/* ---- learned per-row polynomial smoother ----------------------------------
 * The paper names polynomial smoothers as future work (Sec. 5).  Here a small
 * MLP (16 -> 64 -> 64 -> 3, tanh, FP16 weights, FP32 arithmetic) maps 16
 * scale-free features of each matrix row to the coefficients of the smoother
 * of amg_set_poly: c_q = omega_k (delta_q0 + o_q), so o = 0 is damped Jacobi.
 * The network is trained on the GPU to minimise the two-grid error reduction
 * ||T (I - G A) e||_A^2 / ||e||_A^2 measured on seeded random errors e of
 * two-level hierarchies (T = exact coarse-grid correction).
 * Parameter layout (AMG_MLP_NPARAM floats): W1[64][16] b1[64] W2[64][64]
 * b2[64] W3[3][64] b3[3]. */
#define AMG_MLP_NFEAT 16
#define AMG_MLP_NPARAM 5443

/* Features of every row of level k into feat (n_k x 16 floats, host or device). */
int amg_features(const amg_hierarchy *h, int32_t level, float *feat, void *stream);

/* out (n x 3) = MLP(feat (n x 16)); w16: AMG_MLP_NPARAM binary16 bit patterns.
 * All three arrays are DEVICE pointers.  Asynchronous on stream. */
int amg_mlp_forward(int32_t n, const uint16_t *w16, const float *feat, float *out, void *stream);

/* dparam (AMG_MLP_NPARAM doubles) = sum over rows of d<dout, MLP_w(feat)>/dw
 * evaluated at the FP32 weights w; all DEVICE pointers.  The sum over rows is
 * in a fixed order (deterministic). */
int amg_mlp_backward(int32_t n, const float *w, const float *feat, const float *dout, double *dparam,
                     void *stream);

/* Same result as amg_mlp_backward, for callers that cannot allocate device
 * memory: real-time or embedded hosts that must not enter an allocator in
 * their steady state, and hosts that have handed the whole device memory
 * budget to another framework.  The paper has no counterpart; this is a
 * service of the library.
 *  - No cudaMalloc, cudaFree or allocating library call: the work arrays live
 *    in a fixed device array of about 4.2 MB (2048 rows x (3 + 4 x 64) floats
 *    plus 64 x 4096 doubles) that every GPU loading this library keeps until
 *    the process exits.
 *  - n may be at most 2048; larger n returns AMG_ERR_BAD_INPUT with a message.
 *  - Each call looks up that array's device address on the current device
 *    (no allocation); the first call on a device also loads the module that
 *    holds it, so make that first call before any stream capture.
 *  - All calls share the array: calls whose executions overlap on the GPU (for
 *    example on two streams) race and give wrong results.  Each call writes
 *    every scratch word it reads and clears dparam itself.
 * All pointers are DEVICE pointers; asynchronous on stream. */
int amg_mlp_backward_noalloc(int32_t n, const float *w, const float *feat, const float *dout, double *dparam,
                             void *stream);

/* Two-grid error reduction of the polynomial pre-smoother with coefficients
 * coef (n_0 x 3 doubles, DEVICE) on a hierarchy with exactly two levels, over
 * nvec seeded random errors; *loss (host) gets the mean factor and dcoef
 * (DEVICE, nullable) its gradient. */
int amg_twogrid_loss(amg_hierarchy *h, const double *coef, int32_t nvec, uint64_t seed, double *loss,
                     double *dcoef, void *stream);

/* Train the MLP on two-level hierarchies hs[0..nh) with Adam for `steps`
 * steps (learning rate lr, nvec random errors per hierarchy and step).
 * w (host, AMG_MLP_NPARAM floats): initial weights in, trained weights out;
 * loss_hist (host, nullable, steps doubles): mean two-grid factor per step.
 * Every step runs on the GPU: features, MLP forward, two-grid gradient, MLP
 * backward, Adam update. */
int amg_train_smoother(amg_hierarchy *const *hs, int32_t nh, int32_t steps, double lr, int32_t nvec,
                       uint64_t seed, float *w, double *loss_hist, void *stream);

/* Evaluate the MLP (binary16 weights w16, host or device) on the rows of
 * level 0, the level whose two-grid factor the network is trained on, and
 * install the resulting per-row coefficients there; turns the polynomial
 * smoother on.  The coarser levels keep damped Jacobi (measured: on the
 * FEM and batched variable-coefficient problems the network applied to coarse
 * levels costs more SpMVs per cycle and needs as many or more iterations);
 * amg_features + amg_mlp_forward + amg_set_poly install it on any level. */
int amg_apply_learned_smoother(amg_hierarchy *h, const uint16_t *w16, void *stream);

/* Sizes per level.  levels (host, capacity cap) may be NULL to query *nlevels. */
int amg_hierarchy_info(const amg_hierarchy *h, amg_level_info *levels, int32_t cap,
                       int32_t *nlevels);

/* Copy level k of the setup to HOST arrays (any may be NULL): row_ptr (n+1),
 * col and val (nnz) of A_k in FP64; agg (n, coarse id of every node), P (n,
 * the nonzero of row i of P_k) and B (n, the near-null vector B_k).  agg and P
 * are left untouched on the coarsest level. */
int amg_export_level(const amg_hierarchy *h, int32_t level, int32_t *row_ptr, int32_t *col,
                     double *val, int32_t *agg, double *P, double *B);

/* Copy every index array of the hierarchy to the host and check it: CSR and
 * SELL ranges, aggregate ids, member lists, and for batches the per-level
 * system offsets, row-to-system map, row tiles and coarsest block offsets.
 * Returns AMG_ERR_SETUP with the first violation in amg_last_error().  A
 * diagnostic: it synchronises and copies, and runs no kernel. */
int amg_validate_hierarchy(const amg_hierarchy *h);

/* Statistics of the last setup/solve on this hierarchy. */
int amg_last_solve_info(const amg_hierarchy *h, amg_solve_info *info);

/* Cycle trace of the last amg_solve or amg_precond on this hierarchy (Alg. 4
 * and Alg. 5 as run): per level k (host arrays of capacity cap, any may be
 * NULL) visits[k] = times the cycle ran on level k (level 0: the preconditioner
 * applications; the coarsest: its exact solves), kcalls[k] = times the
 * Krylov-accelerated coarse part of Alg. 5 ran on level k, second[k] = how many
 * of those took the second inner step (||r~|| > t ||r||).  The counts come from
 * device counters read once after the solve.  Returns AMG_ERR_UNSUPPORTED for
 * batches and for the cluster tail (tail = 1, 2), which run their levels
 * without the counters, and before the first solve. */
int amg_cycle_trace(const amg_hierarchy *h, int64_t *visits, int64_t *kcalls, int64_t *second, int32_t cap,
                    int32_t *nlevels);

/* Release every device and host resource of the hierarchy (NULL is a no-op). */
void amg_free(amg_hierarchy *h);

/* Message of the calling thread's most recent failure ("" if none). */
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
