/* amg_oracle.h -- plain FP64 CPU oracle of the aggregation AMG method of
 * Gandham, Esler and Zhang, "A GPU Accelerated Aggregation Algebraic Multigrid
 * Method" (arXiv 1403.1649).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the GPU
 * product path never calls it.  It shares no code, header or helper with the
 * GPU library.
 *
 * Conventions: CSR with int32 row pointers and column indices (ascending in
 * each row, diagonal present), double values.  All arithmetic is IEEE double,
 * compiled without FMA contraction, single-threaded, in the order the paper's
 * algorithms state.
 */
#ifndef AMG_ORACLE_H
#define AMG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_params {
  double alpha;        /* strength threshold, Sec. 2.1.1 (0.25 in 2D, 0.5 in 3D)   */
  uint64_t seed;       /* MIS priorities and Arnoldi start vectors                 */
  int32_t coarse_max;  /* stop coarsening once n_k <= coarse_max                   */
  int32_t max_levels;  /* hard cap on the number of levels                         */
  int32_t kcycle_levels; /* levels k < kcycle_levels use Krylov-accelerated coarse
                            correction (Alg. 5); deeper levels use Alg. 4          */
  double kcycle_t;     /* K-cycle threshold t in ||r~|| <= t ||r||                 */
  int32_t omega_mode;  /* 0: omega = (4/3)/rho from Arnoldi; 1: fixed omega       */
  double omega;        /* used when omega_mode == 1                                */
  int32_t outer;       /* 0: flexible CG (CG variant of Alg. 5); 1: FGMRES(restart)
                          (GMRES variant)                                          */
  int32_t restart;     /* FGMRES restart length                                    */
  int32_t smoother;    /* 0: damped Jacobi; 1: per-row polynomial (coefficients
                          supplied per level through or_set_poly)                  */
  int32_t symmetric;   /* 1: A symmetric (rho from the symmetric part of H, Cholesky
                          coarsest factor); 0: nonsymmetric (rho from the
                          eigenvalues of H, LU coarsest factor; use FGMRES)        */
  int32_t mis_k;       /* roots form an MIS(k) (Sec. 2.1.2: k = 2; k > 2 coarsens
                          more aggressively); aggregates reach distance k          */
} or_params;

/* ---- individual setup steps (used directly by the pin tests) ---- */

/* Sec. 2.1.1 classic strength: C[p] = 1 iff -s_i A_ij > alpha * max(-s_i A_ij > 0). */
void or_strength(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                 double alpha, uint8_t *C);
/* #{j != i : C_ji = 1}, the strongly-influencing count of Alg. 2. */
void or_col_count(int32_t n, const int32_t *rp, const int32_t *ci, const uint8_t *C,
                  int32_t *count);
/* Neighbourhood N_i = {j != i : C_ij = 1 or C_ji = 1}, rows sorted, unique.
 * Returns the number of entries; writes at most cap entries to Scol.        */
int64_t or_sym_graph(int32_t n, const int32_t *rp, const int32_t *ci, const uint8_t *C,
                     int32_t *Sptr, int32_t *Scol, int64_t cap);
/* The random part r_i of Alg. 2, as a 32-bit integer (r_i = (h_i + 0.5) / 2^32). */
uint32_t or_mis_hash(uint64_t seed, int32_t level, int32_t i);
uint64_t or_splitmix64(uint64_t x);
/* Alg. 2 generalised to MIS(k) (Sec. 2.1.2; k = 2 is Alg. 2 as printed): k
 * rounds of max over the closed neighbourhood per iteration.  s[i] = 1 (MIS),
 * -1 (not MIS).  Returns the number of iterations. */
int32_t or_pmis(int32_t n, const int32_t *Sptr, const int32_t *Scol, const int32_t *count,
                const uint32_t *h, int8_t *s, int32_t k);
/* Aggregation: every non-MIS node joins its nearest MIS node, at distance at
 * most k (Sec. 2.1.2).  Returns n_c, or -1 if some node could not be assigned. */
int32_t or_aggregate(int32_t n, const int32_t *Sptr, const int32_t *Scol, const int32_t *count,
                     const uint32_t *h, const int8_t *s, int32_t *agg, int32_t k);
/* Alg. 3 interpolation: P[i] = B(i)/B_c(agg(i)), B_c(I) = ||B restricted to G_I||_2. */
void or_interp(int32_t n, int32_t nc, const int32_t *agg, const double *B, double *P,
               double *Bc);
/* Sec. 3.1 Galerkin product as a keyed sum.  P may be NULL (all ones).
 * Returns nnz of the coarse matrix; writes at most cap entries.            */
int64_t or_galerkin(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                    int32_t nc, const int32_t *agg, const double *P, int32_t *crp,
                    int32_t *cci, double *cval, int64_t cap);
/* Eq. (damped Jacobi): spectral-radius estimate of D^-1 A from m Arnoldi steps. */
/* largest |eigenvalue| of an upper Hessenberg m x m matrix (m <= 8, row major)
 * by the shifted QR algorithm in complex arithmetic */
double or_hess_rho(int32_t m, const double *H);
/* LU factorisation with partial pivoting (row interchanges piv), and solve */
int32_t or_lu(int32_t n, double *a, int32_t *piv);
void or_lu_solve(int32_t n, const double *lu, const int32_t *piv, double *b);
/* rho(D^-1 A) from m Arnoldi steps on |D|^-1/2 A |D|^-1/2 (Eq. damped Jacobi):
 * symmetric = 1: the largest |eigenvalue| of the symmetric part of H_m (equal to
 * H_m for symmetric A); 0: the largest |eigenvalue| of H_m itself */
double or_rho_estimate(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                       uint64_t seed, int32_t level, int32_t m, double *H_out /* m*m or NULL */,
                       int32_t symmetric);
/* eigenvalues of a symmetric m x m matrix (cyclic Jacobi), ascending */
void or_sym_eig(int32_t m, const double *a, double *w);
/* dense Cholesky in place (lower triangle); returns 0 or -1 if not SPD */
int32_t or_cholesky(int32_t n, double *a);
void or_chol_solve(int32_t n, const double *L, double *b);

/* host threads the solve stage uses: 1 in the parity build, the OpenMP thread
 * count in the CPU-baseline timing build (compiled with -fopenmp) */
int32_t or_threads(void);

/* ---- the whole method ---- */
typedef struct or_hier or_hier;

void or_default_params(or_params *p);
or_hier *or_setup(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                  const or_params *p, int32_t *err);
/* The rows [r0, r1) of level 0 and their part of every coarser level, as a
 * hierarchy of its own (the per-system view of independent systems set up
 * together as one block-diagonal matrix).  NULL with err = -2 if the rows
 * couple to other rows or an aggregate crosses the range on some level. */
or_hier *or_subsystem(const or_hier *h, int32_t r0, int32_t r1, int32_t *err);
int32_t or_nlevels(const or_hier *h);
void or_level_info(const or_hier *h, int32_t k, int32_t *n, int64_t *nnz, double *omega,
                   int32_t *mis_rounds);
/* copy level k: its matrix, and (k < L-1) its aggregates, weights P_k and B_k */
void or_level_copy(const or_hier *h, int32_t k, int32_t *rp, int32_t *ci, double *val,
                   int32_t *agg, double *P, double *B);
/* per-row polynomial smoother coefficients for level k (n_k x 3, row major) */
int32_t or_set_poly(or_hier *h, int32_t k, const double *coef);
/* one application of the preconditioner (Alg. 5 on level 0 from x = 0) */
void or_precond(or_hier *h, const double *b, double *x);
/* cycle trace of the last or_solve / or_precond: per level the cycle visits
 * (the coarsest: its exact solves), the Alg. 5 coarse parts run there, and the
 * second inner steps they took (each array h's level count long) */
void or_cycle_trace(const or_hier *h, int64_t *visits, int64_t *kcalls, int64_t *second);
/* outer Krylov solve; x holds x0 on entry.  hist gets the relative residual
 * norm after every iteration (hist[0] = initial).  Returns 0 if converged,
 * 1 if not, <0 on breakdown.                                                */
int32_t or_solve(or_hier *h, const double *b, double *x, double tol, int32_t max_iter,
                 int32_t *iters, double *hist, double *final_relres);
void or_free(or_hier *h);
/* test hook: Alg. 5 coarse part at level m, exposing the inner iterates c, d */
int32_t or_krylov2_probe(or_hier *h, int32_t m, const double *r, double *x, double *c, double *d);

/* ---- learned per-row polynomial smoother (the paper names polynomial
 *      smoothers as future work, Sec. 5; this part is the library's own) ---- */
#define OR_NFEAT 16
#define OR_HID 64
#define OR_NOUT 3
/* parameter layout (float): W1[64][16] b1[64] W2[64][64] b2[64] W3[3][64] b3[3] */
#define OR_NPARAM (OR_HID * OR_NFEAT + OR_HID + OR_HID * OR_HID + OR_HID + OR_NOUT * OR_HID + OR_NOUT)
/* 16 scale-free features of every row (see the definition in amg_oracle.c) */
void or_features(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, int32_t level,
                 float *feat);
/* MLP 16 -> 64 -> 64 -> 3 with tanh, FP16 weights (IEEE binary16 bit patterns),
 * FP32 arithmetic; out is n x 3 */
void or_mlp_forward(int32_t n, const uint16_t *w16, const float *feat, float *out);
/* FP64 forward + backward: given dL/dout (n x 3), accumulate dL/dparam (double,
 * OR_NPARAM) for weights w (double) */
void or_mlp_backward(int32_t n, const double *w, const float *feat, const double *dout, double *dparam,
                     double *out);
/* Two-grid error reduction of the pre-smoother x += sum_q diag(c_q)(D^-1 A)^q D^-1 r
 * with exact coarse solve, on nvec seeded random errors e0:
 *   L = mean_v ||T (I - G A) e0||_A^2 / ||e0||_A^2,  T = I - P A_c^-1 P^T A.
 * Uses levels 0 and 1 of a two-level hierarchy.  coef: n x 3.  dcoef (nullable)
 * gets dL/dcoef.  Returns L. */
double or_twogrid_loss(or_hier *h, const double *coef, int32_t nvec, uint64_t seed, double *dcoef);

#ifdef __cplusplus
}
#endif
#endif
