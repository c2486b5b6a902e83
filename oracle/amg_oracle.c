/* amg_oracle.c -- plain FP64 CPU oracle of aggregation AMG (arXiv 1403.1649).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark.  The GPU product path never calls it, and it
 * shares no code with the GPU library.
 *
 * Each function follows the paper's text in its own order and notation:
 *   Sec. 2.1.1  strength of connection (classic strength equation)
 *   Alg. 2      PMIS(2) with priorities v_i = #{j : C_ji = 1} + r_i
 *   Sec. 2.1.2  aggregation: every non-MIS node joins its nearest MIS node
 *   Alg. 3      unsmoothed, normalised interpolation (B_k = P_k B_{k+1}, P^T P = I)
 *   Sec. 3.1    Galerkin product as a keyed sum over (Agg(i), Agg(j))
 *   Eq. (damped Jacobi)  x <- x + omega D^-1 (b - A x), omega = (4/3)/rho(D^-1 A)
 *   Alg. 4/5    V-cycle and K-cycle; K-cycle on the top levels only (Sec. 2.2)
 *   Sec. 2.2    outer flexible CG / FGMRES
 * Readings of points the paper leaves open are stated where they are used.
 * Compiled with -ffp-contract=off: every product and sum is rounded on its own.
 */
#include "amg_oracle.h"

#include <complex.h>
#undef I /* the oracle uses I for coarse indices */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_LEVELS 40
#define OR_MAX_DENSE 8192

/* The CPU-baseline timing build (compiled again with -fopenmp) runs the row
 * loops of the solve stage on all host cores.  Its inner products add fixed
 * chunks of OR_DOT_CHUNK terms in order and then the chunk sums in order, so
 * its results do not depend on the thread count (they differ from this
 * single-threaded build by rounding only), and its restriction sums each
 * aggregate's members in ascending order as the scatter below does.  The
 * setup stays single-threaded.  The plain build (no -fopenmp) is the parity
 * reference; none of this is compiled into it. */
#ifdef _OPENMP
#include <omp.h>
#define OR_PAR _Pragma("omp parallel for schedule(static)")
#define OR_DOT_CHUNK 8192
#else
#define OR_PAR
#endif

int32_t or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* counter-based random numbers: splitmix64 (Steele, Lea, Flood 2014)        */
/* ------------------------------------------------------------------------- */
uint64_t or_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Alg. 2 draws r_i in (0,1).  We keep the 32-bit integer h_i and read
 * r_i = (h_i + 0.5)/2^32, so v_i = count_i + r_i orders exactly like the
 * integer pair (count_i, h_i); ties in h are broken by the node index, as the
 * tuple (s_i, v_i, i) of Alg. 2 does. */
uint32_t or_mis_hash(uint64_t seed, int32_t level, int32_t i) {
  return (uint32_t)(or_splitmix64(seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)(uint32_t)i) >> 32);
}

/* start vector of the Arnoldi estimate: uniform in [-1, 1) */
static double arnoldi_start(uint64_t seed, int32_t level, int32_t i) {
  uint64_t z = or_splitmix64(~seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)(uint32_t)i);
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.1.1: classic strength of connection                                */
/*   C_ij = 1  iff  -s_i A_ij > alpha * max_{j: -s_i A_ij > 0} (-s_i A_ij),  */
/*   s_i = sign(A_ii).  The diagonal never qualifies (-s_i A_ii < 0).  A row */
/*   with no entry of sign opposite to its diagonal has no strong entries.   */
/* ------------------------------------------------------------------------- */
void or_strength(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                 double alpha, uint8_t *C) {
  for (int32_t i = 0; i < n; ++i) {
    double aii = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) aii = val[p];
    double s = aii > 0.0 ? 1.0 : (aii < 0.0 ? -1.0 : 0.0);
    int have = 0;
    double mx = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      double t = -(s * val[p]);
      if (ci[p] != i && t > 0.0 && (!have || t > mx)) {
        mx = t;
        have = 1;
      }
    }
    double thr = alpha * mx;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      double t = -(s * val[p]);
      C[p] = (uint8_t)(have && ci[p] != i && t > thr);
    }
  }
}

/* Alg. 2: number of strongly influencing connections #{j : C_ji = 1} */
void or_col_count(int32_t n, const int32_t *rp, const int32_t *ci, const uint8_t *C,
                  int32_t *count) {
  memset(count, 0, sizeof(int32_t) * (size_t)n);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (C[p]) count[ci[p]]++;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* The strong neighbours N_i of Alg. 2.  Reading: the graph of C made
 * symmetric, N_i = {j != i : C_ij = 1 or C_ji = 1}, so that "distance" in
 * MIS(2) is a distance in an undirected graph. */
int64_t or_sym_graph(int32_t n, const int32_t *rp, const int32_t *ci, const uint8_t *C,
                     int32_t *Sptr, int32_t *Scol, int64_t cap) {
  int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *fill = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (C[p]) {
        off[i + 1]++;
        off[ci[p] + 1]++;
      }
  for (int32_t i = 0; i < n; ++i) off[i + 1] += off[i];
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[n] + 1));
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (C[p]) {
        int32_t j = ci[p];
        tmp[off[i] + fill[i]++] = j;
        tmp[off[j] + fill[j]++] = i;
      }
  OR_PAR
  for (int32_t i = 0; i < n; ++i) qsort(tmp + off[i], (size_t)(off[i + 1] - off[i]), sizeof(int32_t), cmp_i32);
  int64_t total = 0;
  Sptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) { /* each row sorted: drop repeats */
    int32_t *row = tmp + off[i];
    int32_t len = (int32_t)(off[i + 1] - off[i]);
    for (int32_t k = 0; k < len; ++k) {
      if (k > 0 && row[k] == row[k - 1]) continue;
      if (total < cap) Scol[total] = row[k];
      total++;
    }
    Sptr[i + 1] = (int32_t)total;
  }
  free(tmp);
  free(fill);
  free(off);
  return total;
}

/* ------------------------------------------------------------------------- */
/* Alg. 2: PMIS(2), and MIS(k) with k max rounds (Sec. 2.1.2)                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t s;     /* state: 1 MIS, 0 undecided, -1 not MIS */
  int32_t cnt;   /* #{j : C_ji = 1}                        */
  uint32_t h;    /* random part r_i as an integer          */
  int32_t i;     /* node index                             */
} tuple_t;

/* lexicographic order of (s, v, i) with v = cnt + r */
static int tuple_greater(tuple_t a, tuple_t b) {
  if (a.s != b.s) return a.s > b.s;
  if (a.cnt != b.cnt) return a.cnt > b.cnt;
  if (a.h != b.h) return a.h > b.h;
  return a.i > b.i;
}

int32_t or_pmis(int32_t n, const int32_t *Sptr, const int32_t *Scol, const int32_t *count,
                const uint32_t *h, int8_t *s, int32_t k) {
  tuple_t *T = (tuple_t *)malloc(sizeof(tuple_t) * (size_t)(n + 1));
  tuple_t *That = (tuple_t *)malloc(sizeof(tuple_t) * (size_t)(n + 1));
  for (int32_t i = 0; i < n; ++i) s[i] = 0; /* every node undecided */
  int32_t rounds = 0;
  for (;;) {
    int32_t undecided = 0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : undecided)
#endif
    for (int32_t i = 0; i < n; ++i) undecided += (s[i] == 0);
    if (undecided == 0) break;
    rounds++;
    OR_PAR
    for (int32_t i = 0; i < n; ++i) { /* T_i <- (s_i, v_i, i) */
      T[i].s = s[i];
      T[i].cnt = count[i];
      T[i].h = h[i];
      T[i].i = i;
    }
    for (int d = 1; d <= k; ++d) { /* k rounds of max over the closed neighbourhood */
      OR_PAR
      for (int32_t i = 0; i < n; ++i) {
        tuple_t t = T[i];
        for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q)
          if (tuple_greater(T[Scol[q]], t)) t = T[Scol[q]];
        That[i] = t;
      }
      tuple_t *sw = T;
      T = That;
      That = sw;
    }
    OR_PAR
    for (int32_t i = 0; i < n; ++i) { /* decide undecided nodes */
      if (s[i] != 0) continue;
      if (T[i].i == i)
        s[i] = 1;
      else if (T[i].s == 1)
        s[i] = -1;
    }
  }
  free(T);
  free(That);
  return rounds;
}

/* priority order of MIS nodes, used to break ties between equally near roots */
static int key_greater(int32_t a, int32_t b, const int32_t *count, const uint32_t *h) {
  if (count[a] != count[b]) return count[a] > count[b];
  if (h[a] != h[b]) return h[a] > h[b];
  return a > b;
}

/* Sec. 2.1.2: every non-MIS node is aggregated with its nearest MIS node.
 * Reading of the unstated tie-break: among MIS nodes at the same distance the
 * one with the largest priority (v, i) wins.  Pass 1 joins nodes adjacent to
 * a root; pass d = 2..k joins the remaining nodes through a neighbour assigned
 * by pass d-1 (for MIS(k) every node is within distance k of a root).  Roots
 * are numbered 0..n_c-1 in ascending fine index. */
int32_t or_aggregate(int32_t n, const int32_t *Sptr, const int32_t *Scol, const int32_t *count,
                     const uint32_t *h, const int8_t *s, int32_t *agg, int32_t k) {
  int32_t *r1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t *r2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int32_t i = 0; i < n; ++i) r1[i] = (s[i] == 1) ? i : -1;
  for (int32_t i = 0; i < n; ++i) {
    if (s[i] == 1) continue;
    int32_t best = -1;
    for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
      int32_t j = Scol[q];
      if (s[j] == 1 && (best < 0 || key_greater(j, best, count, h))) best = j;
    }
    r1[i] = best;
  }
  for (int32_t d = 2; d <= k; ++d) { /* r1: passes < d; r2: after pass d */
    for (int32_t i = 0; i < n; ++i) r2[i] = r1[i];
    for (int32_t i = 0; i < n; ++i) {
      if (r1[i] >= 0) continue;
      int32_t best = -1;
      for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
        int32_t j = Scol[q];
        if (s[j] != 1 && r1[j] >= 0) {
          int32_t r = r1[j];
          if (best < 0 || key_greater(r, best, count, h)) best = r;
        }
      }
      r2[i] = best;
    }
    for (int32_t i = 0; i < n; ++i) r1[i] = r2[i];
  }
  for (int32_t i = 0; i < n; ++i) r2[i] = r1[i];
  int32_t nc = 0;
  for (int32_t i = 0; i < n; ++i) cid[i] = (s[i] == 1) ? nc++ : -1;
  int32_t ok = 1;
  for (int32_t i = 0; i < n; ++i) {
    if (r2[i] < 0) {
      ok = 0;
      agg[i] = -1;
    } else {
      agg[i] = cid[r2[i]];
    }
  }
  free(r1);
  free(r2);
  free(cid);
  return ok ? nc : -1;
}

/* ------------------------------------------------------------------------- */
/* Alg. 3: interpolation.  P_k(i, Agg(i)) = B_k(i); B_{k+1}(I) is the 2-norm */
/* of row I of R_k = P_k^T (summed in ascending fine index); rows of R and    */
/* the entries of P are divided by it, so P^T P = I and B_k = P_k B_{k+1}.    */
/* ------------------------------------------------------------------------- */
void or_interp(int32_t n, int32_t nc, const int32_t *agg, const double *B, double *P,
               double *Bc) {
  double *sum = (double *)calloc((size_t)nc + 1, sizeof(double));
  uint8_t *seen = (uint8_t *)calloc((size_t)nc + 1, 1);
  for (int32_t i = 0; i < n; ++i) {
    int32_t I = agg[i];
    double t = B[i] * B[i];
    sum[I] = seen[I] ? sum[I] + t : t;
    seen[I] = 1;
  }
  for (int32_t I = 0; I < nc; ++I) Bc[I] = sqrt(sum[I]);
  for (int32_t i = 0; i < n; ++i) P[i] = B[i] / Bc[agg[i]];
  free(sum);
  free(seen);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.1: Galerkin product as a keyed sum.  For every fine nonzero A_ij   */
/* the key is (I, J) = (Agg(i), Agg(j)) and the value P_iI * A_ij * P_jJ,     */
/* scaled before sorting.  The list is sorted by key keeping the CSR order of */
/* equal keys (the order of the paper's worked example) and every run of      */
/* equal keys is summed from its first entry on.                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t I, J;
  int64_t pos;
  double v;
} gentry_t;

static int cmp_gentry(const void *a, const void *b) {
  const gentry_t *x = (const gentry_t *)a, *y = (const gentry_t *)b;
  if (x->I != y->I) return x->I < y->I ? -1 : 1;
  if (x->J != y->J) return x->J < y->J ? -1 : 1;
  return (x->pos > y->pos) - (x->pos < y->pos);
}

int64_t or_galerkin(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                    int32_t nc, const int32_t *agg, const double *P, int32_t *crp,
                    int32_t *cci, double *cval, int64_t cap) {
  int64_t nnz = rp[n];
  gentry_t *e = (gentry_t *)malloc(sizeof(gentry_t) * (size_t)(nnz + 1));
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t j = ci[p];
      e[p].I = agg[i];
      e[p].J = agg[j];
      e[p].pos = p;
      e[p].v = P ? (P[i] * val[p]) * P[j] : val[p];
    }
#ifdef _OPENMP
  { /* the same order as the one sort below: a stable counting sort of the
       entries by I (positions stay ascending), then each row's run sorted by
       (J, pos) on its own */
    int64_t *bo = (int64_t *)calloc((size_t)nc + 2, sizeof(int64_t));
    for (int64_t q = 0; q < nnz; ++q) bo[e[q].I + 1]++;
    for (int32_t I = 0; I < nc; ++I) bo[I + 1] += bo[I];
    gentry_t *e2 = (gentry_t *)malloc(sizeof(gentry_t) * (size_t)(nnz + 1));
    int64_t *fill = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    for (int64_t q = 0; q < nnz; ++q) e2[bo[e[q].I] + fill[e[q].I]++] = e[q];
    OR_PAR
    for (int32_t I = 0; I < nc; ++I) qsort(e2 + bo[I], (size_t)(bo[I + 1] - bo[I]), sizeof(gentry_t), cmp_gentry);
    free(e);
    free(fill);
    free(bo);
    e = e2;
  }
#else
  qsort(e, (size_t)nnz, sizeof(gentry_t), cmp_gentry);
#endif
  int64_t out = 0;
  for (int32_t I = 0; I <= nc; ++I) crp[I] = 0;
  int64_t q = 0;
  while (q < nnz) {
    int64_t r = q + 1;
    double sum = e[q].v;
    while (r < nnz && e[r].I == e[q].I && e[r].J == e[q].J) {
      sum = sum + e[r].v;
      r++;
    }
    if (out < cap) {
      cci[out] = e[q].J;
      cval[out] = sum;
    }
    crp[e[q].I + 1]++;
    out++;
    q = r;
  }
  for (int32_t I = 0; I < nc; ++I) crp[I + 1] += crp[I];
  free(e);
  return out;
}

/* ------------------------------------------------------------------------- */
/* eigenvalues of a small symmetric matrix: cyclic Jacobi rotations          */
/* ------------------------------------------------------------------------- */
void or_sym_eig(int32_t m, const double *a_in, double *w) {
  double a[64];
  for (int32_t k = 0; k < m * m; ++k) a[k] = a_in[k];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int32_t p = 0; p < m; ++p)
      for (int32_t q = 0; q < m; ++q) {
        tot += a[p * m + q] * a[p * m + q];
        if (p != q) off += a[p * m + q] * a[p * m + q];
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int32_t p = 0; p < m; ++p)
      for (int32_t q = p + 1; q < m; ++q) {
        double apq = a[p * m + q];
        if (apq == 0.0) continue;
        double theta = (a[q * m + q] - a[p * m + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int32_t k = 0; k < m; ++k) { /* rotate columns p, q */
          double akp = a[k * m + p], akq = a[k * m + q];
          a[k * m + p] = c * akp - s * akq;
          a[k * m + q] = s * akp + c * akq;
        }
        for (int32_t k = 0; k < m; ++k) { /* rotate rows p, q */
          double apk = a[p * m + k], aqk = a[q * m + k];
          a[p * m + k] = c * apk - s * aqk;
          a[q * m + k] = s * apk + c * aqk;
        }
      }
  }
  for (int32_t k = 0; k < m; ++k) w[k] = a[k * m + k];
  for (int32_t i = 1; i < m; ++i) /* insertion sort ascending */
    for (int32_t j = i; j > 0 && w[j] < w[j - 1]; --j) {
      double t = w[j];
      w[j] = w[j - 1];
      w[j - 1] = t;
    }
}

/* ------------------------------------------------------------------------- */
/* Eq. (damped Jacobi): rho(D^-1 A) from m (<= 5) Arnoldi steps.             */
/* Reading: the Arnoldi process runs on D^-1/2 A D^-1/2 (|D| for the root),  */
/* which is similar to D^-1 A and symmetric for symmetric A; the estimate is */
/* the largest |eigenvalue| of the symmetric part of the m x m Hessenberg.   */
/* ------------------------------------------------------------------------- */
/* Shifted QR algorithm for the eigenvalues of an upper Hessenberg matrix, in
 * complex arithmetic (Golub & Van Loan, Sec. 7.5): on the active leading block,
 * H - mu I = Q R by Givens rotations, H <- R Q + mu I, with the Wilkinson shift
 * mu (the eigenvalue of the trailing 2 x 2 block nearer to its last diagonal
 * entry); the last row deflates once |h_{n,n-1}| <= 1e-14 (|h_nn| + |h_{n-1,n-1}|)
 * (or after 200 steps).  Returns the largest modulus. */
double or_hess_rho(int32_t m, const double *Hin) {
  double complex a[8][8];
  for (int32_t i = 0; i < m; ++i)
    for (int32_t j = 0; j < m; ++j) a[i][j] = Hin[i * m + j];
  double rho = 0.0;
  int32_t n = m, iter = 0;
  while (n > 0) {
    if (n == 1) {
      if (cabs(a[0][0]) > rho) rho = cabs(a[0][0]);
      break;
    }
    const double sc = cabs(a[n - 1][n - 1]) + cabs(a[n - 2][n - 2]);
    if (cabs(a[n - 1][n - 2]) <= 1e-14 * sc || iter >= 200) {
      if (cabs(a[n - 1][n - 1]) > rho) rho = cabs(a[n - 1][n - 1]);
      n = n - 1;
      iter = 0;
      continue;
    }
    const double complex p = a[n - 2][n - 2], q = a[n - 2][n - 1], r = a[n - 1][n - 2], t = a[n - 1][n - 1];
    const double complex half = (p + t) / 2.0;
    const double complex disc = csqrt(half * half - (p * t - q * r));
    const double complex l1 = half + disc, l2 = half - disc;
    const double complex mu = cabs(l1 - t) < cabs(l2 - t) ? l1 : l2;
    double complex cs[8], sn[8];
    for (int32_t i = 0; i < n; ++i) a[i][i] = a[i][i] - mu;
    for (int32_t k = 0; k + 1 < n; ++k) { /* left rotations: R = G_{n-2} ... G_0 (H - mu I) */
      const double complex x = a[k][k], y = a[k + 1][k];
      const double nrm = sqrt(cabs(x) * cabs(x) + cabs(y) * cabs(y));
      cs[k] = nrm > 0.0 ? x / nrm : 1.0;
      sn[k] = nrm > 0.0 ? y / nrm : 0.0;
      for (int32_t j = k; j < n; ++j) {
        const double complex u = a[k][j], v = a[k + 1][j];
        a[k][j] = conj(cs[k]) * u + conj(sn[k]) * v;
        a[k + 1][j] = -sn[k] * u + cs[k] * v;
      }
    }
    for (int32_t k = 0; k + 1 < n; ++k) /* right rotations: R Q */
      for (int32_t i = 0; i <= k + 1; ++i) {
        const double complex u = a[i][k], v = a[i][k + 1];
        a[i][k] = u * cs[k] + v * sn[k];
        a[i][k + 1] = -u * conj(sn[k]) + v * conj(cs[k]);
      }
    for (int32_t i = 0; i < n; ++i) a[i][i] = a[i][i] + mu;
    iter = iter + 1;
  }
  return rho;
}

double or_rho_estimate(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                       uint64_t seed, int32_t level, int32_t m, double *H_out, int32_t symmetric) {
  if (m > n) m = n;
  if (m > 8) m = 8;
  double *dh = (double *)malloc(sizeof(double) * (size_t)n);
  double *Q = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double H[9 * 8];
  memset(H, 0, sizeof(H));
  for (int32_t i = 0; i < n; ++i) {
    double aii = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) aii = val[p];
    dh[i] = 1.0 / sqrt(fabs(aii));
  }
  double nu = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    Q[i] = arnoldi_start(seed, level, i);
    nu += Q[i] * Q[i];
  }
  nu = sqrt(nu);
  for (int32_t i = 0; i < n; ++i) Q[i] = Q[i] / nu;
  int32_t mm = m;
  for (int32_t j = 0; j < m; ++j) {
    const double *qj = Q + (size_t)j * n;
    double wn = 0.0;
    for (int32_t i = 0; i < n; ++i) { /* w = D^-1/2 A D^-1/2 q_j */
      double acc = 0.0;
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) acc += val[p] * (dh[ci[p]] * qj[ci[p]]);
      w[i] = dh[i] * acc;
      wn += w[i] * w[i];
    }
    wn = sqrt(wn);
    for (int32_t l = 0; l <= j; ++l) { /* modified Gram-Schmidt */
      const double *ql = Q + (size_t)l * n;
      double hij = 0.0;
      for (int32_t i = 0; i < n; ++i) hij += ql[i] * w[i];
      H[l * 8 + j] = hij;
      for (int32_t i = 0; i < n; ++i) w[i] = w[i] - hij * ql[i];
    }
    double hn = 0.0;
    for (int32_t i = 0; i < n; ++i) hn += w[i] * w[i];
    hn = sqrt(hn);
    H[(j + 1) * 8 + j] = hn;
    if (hn <= 1e-12 * wn || j + 1 == m) {
      mm = j + 1;
      break;
    }
    double *qn = Q + (size_t)(j + 1) * n;
    for (int32_t i = 0; i < n; ++i) qn[i] = w[i] / hn;
  }
  double T[64], ev[8];
  for (int32_t a = 0; a < mm; ++a)
    for (int32_t b = 0; b < mm; ++b) T[a * mm + b] = 0.5 * (H[a * 8 + b] + H[b * 8 + a]);
  if (H_out)
    for (int32_t a = 0; a < mm; ++a)
      for (int32_t b = 0; b < mm; ++b) H_out[a * mm + b] = H[a * 8 + b];
  double rho;
  if (symmetric) {
    or_sym_eig(mm, T, ev);
    rho = fabs(ev[0]) > fabs(ev[mm - 1]) ? fabs(ev[0]) : fabs(ev[mm - 1]);
  } else {
    for (int32_t a = 0; a < mm; ++a)
      for (int32_t b = 0; b < mm; ++b) T[a * mm + b] = H[a * 8 + b];
    rho = or_hess_rho(mm, T);
  }
  free(dh);
  free(Q);
  free(w);
  return rho;
}

/* ------------------------------------------------------------------------- */
/* dense LU with partial pivoting for a nonsymmetric coarsest level          */
/* ------------------------------------------------------------------------- */
int32_t or_lu(int32_t n, double *a, int32_t *piv) {
  for (int32_t j = 0; j < n; ++j) {
    int32_t pr = j; /* the largest |a_ij| below the diagonal, first index on ties */
    for (int32_t i = j + 1; i < n; ++i)
      if (fabs(a[(size_t)i * n + j]) > fabs(a[(size_t)pr * n + j])) pr = i;
    piv[j] = pr;
    if (!(fabs(a[(size_t)pr * n + j]) > 0.0)) return -1;
    if (pr != j)
      for (int32_t k = 0; k < n; ++k) {
        const double t = a[(size_t)j * n + k];
        a[(size_t)j * n + k] = a[(size_t)pr * n + k];
        a[(size_t)pr * n + k] = t;
      }
    for (int32_t i = j + 1; i < n; ++i) {
      const double l = a[(size_t)i * n + j] / a[(size_t)j * n + j];
      a[(size_t)i * n + j] = l;
      for (int32_t k = j + 1; k < n; ++k) a[(size_t)i * n + k] = a[(size_t)i * n + k] - l * a[(size_t)j * n + k];
    }
  }
  return 0;
}

void or_lu_solve(int32_t n, const double *lu, const int32_t *piv, double *b) {
  for (int32_t j = 0; j < n; ++j) /* the row interchanges, then L y = b, U x = y */
    if (piv[j] != j) {
      const double t = b[j];
      b[j] = b[piv[j]];
      b[piv[j]] = t;
    }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = 0; k < i; ++k) b[i] = b[i] - lu[(size_t)i * n + k] * b[k];
  for (int32_t i = n - 1; i >= 0; --i) {
    for (int32_t k = i + 1; k < n; ++k) b[i] = b[i] - lu[(size_t)i * n + k] * b[k];
    b[i] = b[i] / lu[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------------------- */
/* dense Cholesky for the coarsest level (the paper uses SuperLU, Sec. 3)    */
/* ------------------------------------------------------------------------- */
int32_t or_cholesky(int32_t n, double *a) {
  for (int32_t j = 0; j < n; ++j) {
    double d = a[(size_t)j * n + j];
    for (int32_t k = 0; k < j; ++k) d = d - a[(size_t)j * n + k] * a[(size_t)j * n + k];
    if (!(d > 0.0)) return -1;
    double ljj = sqrt(d);
    a[(size_t)j * n + j] = ljj;
    for (int32_t i = j + 1; i < n; ++i) {
      double t = a[(size_t)i * n + j];
      for (int32_t k = 0; k < j; ++k) t = t - a[(size_t)i * n + k] * a[(size_t)j * n + k];
      a[(size_t)i * n + j] = t / ljj;
    }
    for (int32_t i = 0; i < j; ++i) a[(size_t)i * n + j] = 0.0;
  }
  return 0;
}

void or_chol_solve(int32_t n, const double *L, double *b) {
  for (int32_t i = 0; i < n; ++i) { /* L y = b */
    double t = b[i];
    for (int32_t k = 0; k < i; ++k) t = t - L[(size_t)i * n + k] * b[k];
    b[i] = t / L[(size_t)i * n + i];
  }
  for (int32_t i = n - 1; i >= 0; --i) { /* L^T x = y */
    double t = b[i];
    for (int32_t k = i + 1; k < n; ++k) t = t - L[(size_t)k * n + i] * b[k];
    b[i] = t / L[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------------------- */
/* the hierarchy (Alg. 1) and the solve phase (Alg. 4, Alg. 5, Sec. 2.2)     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n, nc, mis_rounds;
  int64_t nnz;
  int32_t *rp, *ci;
  double *val;
  double *dinv;  /* 1 / A_ii                  */
  double omega;
  double *wd;    /* omega / A_ii              */
  int32_t *agg;  /* Agg_k (k < L-1)           */
  double *P;     /* P_k(i, Agg(i))            */
  double *B;     /* near-null vector B_k      */
  double *poly;  /* n x 3 smoother coefficients or NULL */
  int32_t *aptr, *amem; /* members of every aggregate, ascending (timing build only) */
  /* work vectors of this level */
  double *r, *bc, *xc, *c, *v, *rt, *d, *w, *u0, *u1;
} or_level;

struct or_hier {
  or_params p;
  int32_t L;
  or_level lev[OR_MAX_LEVELS];
  double *chol; /* dense Cholesky (symmetric) or LU (nonsymmetric) factor of A_{L-1} */
  int32_t *piv; /* LU row interchanges */
  /* cycle trace of the last solve / preconditioner application: cycle visits
   * per level, Alg. 5 coarse parts run there, second inner steps taken */
  int64_t visits[OR_MAX_LEVELS], kcalls[OR_MAX_LEVELS], second[OR_MAX_LEVELS];
};

void or_default_params(or_params *p) {
  p->alpha = 0.25;
  p->seed = 0;
  p->coarse_max = 64;
  p->max_levels = 25;
  p->kcycle_levels = 2;
  p->kcycle_t = 0.25;
  p->omega_mode = 0;
  p->omega = 2.0 / 3.0;
  p->outer = 0;
  p->restart = 30;
  p->smoother = 0;
  p->symmetric = 1;
  p->mis_k = 2;
}

static double *dalloc(size_t n) { return (double *)calloc(n + 1, sizeof(double)); }

static void level_alloc_work(or_level *l) {
  size_t n = (size_t)l->n;
  l->r = dalloc(n);
  l->bc = dalloc(n);
  l->xc = dalloc(n);
  l->c = dalloc(n);
  l->v = dalloc(n);
  l->rt = dalloc(n);
  l->d = dalloc(n);
  l->w = dalloc(n);
  l->u0 = dalloc(n);
  l->u1 = dalloc(n);
  l->dinv = dalloc(n);
  l->wd = dalloc(n);
}

static void level_free(or_level *l) {
  free(l->rp); free(l->ci); free(l->val); free(l->dinv); free(l->wd); free(l->agg);
  free(l->P); free(l->B); free(l->poly); free(l->aptr); free(l->amem);
  free(l->r); free(l->bc); free(l->xc); free(l->c); free(l->v); free(l->rt); free(l->d);
  free(l->w); free(l->u0); free(l->u1);
}

void or_free(or_hier *h) {
  if (!h) return;
  for (int32_t k = 0; k < h->L; ++k) level_free(&h->lev[k]);
  free(h->chol);
  free(h->piv);
  free(h);
}

/* input checks: ascending columns, present and nonzero diagonal */
static int32_t check_csr(int32_t n, const int32_t *rp, const int32_t *ci, const double *val) {
  if (n <= 0 || rp[0] != 0) return -2;
  for (int32_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return -2;
    int diag = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n) return -2;
      if (p > rp[i] && ci[p] <= ci[p - 1]) return -2;
      if (ci[p] == i) diag = (val[p] != 0.0);
    }
    if (!diag) return -2;
  }
  return 0;
}

/* aggregate member lists (ascending) for the restriction of the timing build */
static void build_members(or_hier *h) {
#ifdef _OPENMP
  for (int32_t q = 0; q < h->L - 1; ++q) {
    or_level *L = &h->lev[q];
    L->aptr = (int32_t *)calloc((size_t)L->nc + 1, sizeof(int32_t));
    L->amem = (int32_t *)malloc(sizeof(int32_t) * ((size_t)L->n + 1));
    for (int32_t i = 0; i < L->n; ++i) L->aptr[L->agg[i] + 1]++;
    for (int32_t I = 0; I < L->nc; ++I) L->aptr[I + 1] += L->aptr[I];
    int32_t *fill = (int32_t *)calloc((size_t)L->nc + 1, sizeof(int32_t));
    for (int32_t i = 0; i < L->n; ++i) L->amem[L->aptr[L->agg[i]] + fill[L->agg[i]]++] = i;
    free(fill);
  }
#else
  (void)h;
#endif
}

/* dense factor of the coarsest level: Cholesky (symmetric) or LU with partial
 * pivoting; 0, or -6 (too large) / -7 (not positive definite / singular) */
static int32_t factor_coarsest(or_hier *h) {
  or_level *Lc = &h->lev[h->L - 1];
  if (Lc->n > OR_MAX_DENSE) return -6;
  h->chol = dalloc((size_t)Lc->n * (size_t)Lc->n);
  for (int32_t i = 0; i < Lc->n; ++i)
    for (int32_t pp = Lc->rp[i]; pp < Lc->rp[i + 1]; ++pp)
      h->chol[(size_t)i * Lc->n + Lc->ci[pp]] = Lc->val[pp];
  if (h->p.symmetric ? or_cholesky(Lc->n, h->chol)
                     : or_lu(Lc->n, h->chol, h->piv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(Lc->n + 1))))
    return -7;
  return 0;
}

or_hier *or_setup(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                  const or_params *p, int32_t *err) {
  *err = check_csr(n, rp, ci, val);
  if (*err) return NULL;
  if (p->mis_k < 1 || p->mis_k > 8) {
    *err = -2;
    return NULL;
  }
  or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
  h->p = *p;
  or_level *l0 = &h->lev[0];
  l0->n = n;
  l0->nnz = rp[n];
  l0->rp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  l0->ci = (int32_t *)malloc(sizeof(int32_t) * ((size_t)l0->nnz + 1));
  l0->val = dalloc((size_t)l0->nnz);
  memcpy(l0->rp, rp, sizeof(int32_t) * ((size_t)n + 1));
  memcpy(l0->ci, ci, sizeof(int32_t) * (size_t)l0->nnz);
  memcpy(l0->val, val, sizeof(double) * (size_t)l0->nnz);
  l0->B = dalloc((size_t)n);
  for (int32_t i = 0; i < n; ++i) l0->B[i] = 1.0; /* reading: B_0 = 1 (constant near-null vector) */
  int32_t k = 0;
  for (;;) { /* Alg. 1 */
    or_level *L = &h->lev[k];
    if (L->n <= p->coarse_max || k + 1 >= p->max_levels || k + 1 >= OR_MAX_LEVELS) break;
    int32_t nk = L->n;
    uint8_t *C = (uint8_t *)malloc((size_t)L->nnz + 1);
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)nk);
    int32_t *Sptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nk + 1));
    uint32_t *hh = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nk);
    int8_t *s = (int8_t *)malloc((size_t)nk);
    int32_t *agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)nk);
    or_strength(nk, L->rp, L->ci, L->val, p->alpha, C);               /* C_k = strength(A_k) */
    or_col_count(nk, L->rp, L->ci, C, count);
    int64_t ns = or_sym_graph(nk, L->rp, L->ci, C, Sptr, NULL, 0);
    int32_t *Scol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns + 1));
    or_sym_graph(nk, L->rp, L->ci, C, Sptr, Scol, ns);
    for (int32_t i = 0; i < nk; ++i) hh[i] = or_mis_hash(p->seed, k, i);
    L->mis_rounds = or_pmis(nk, Sptr, Scol, count, hh, s, p->mis_k); /* Agg_k = aggregate(C_k) */
    int32_t nc = or_aggregate(nk, Sptr, Scol, count, hh, s, agg, p->mis_k);
    free(C); free(count); free(Sptr); free(Scol); free(hh); free(s);
    if (nc < 0) {
      free(agg);
      *err = -5;
      or_free(h);
      return NULL;
    }
    /* the stopping rule (coarsen while the coarse system is too large for a
       direct solve): also stop when coarsening stalls */
    if (10LL * nc >= 9LL * nk) {
      free(agg);
      break;
    }
    or_level *Cl = &h->lev[k + 1];
    L->agg = agg;
    L->nc = nc;
    L->P = dalloc((size_t)nk);
    Cl->n = nc;
    Cl->B = dalloc((size_t)nc);
    or_interp(nk, nc, agg, L->B, L->P, Cl->B);                        /* P_k, B_{k+1} */
    Cl->rp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nc + 1));
    int64_t cn = or_galerkin(nk, L->rp, L->ci, L->val, nc, agg, L->P, Cl->rp, NULL, NULL, 0);
    Cl->ci = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cn + 1));
    Cl->val = dalloc((size_t)cn);
    or_galerkin(nk, L->rp, L->ci, L->val, nc, agg, L->P, Cl->rp, Cl->ci, Cl->val, cn); /* A_{k+1} */
    Cl->nnz = cn;
    k++;
  }
  h->L = k + 1;
  for (int32_t q = 0; q < h->L; ++q) {
    or_level *L = &h->lev[q];
    level_alloc_work(L);
    for (int32_t i = 0; i < L->n; ++i)
      for (int32_t pp = L->rp[i]; pp < L->rp[i + 1]; ++pp)
        if (L->ci[pp] == i) L->dinv[i] = 1.0 / L->val[pp];
    if (q < h->L - 1) {
      L->omega = p->omega_mode == 0
                     ? (4.0 / 3.0) / or_rho_estimate(L->n, L->rp, L->ci, L->val, p->seed, q, 5, NULL, p->symmetric)
                     : p->omega;
      for (int32_t i = 0; i < L->n; ++i) {
        double aii = 1.0 / L->dinv[i];
        for (int32_t pp = L->rp[i]; pp < L->rp[i + 1]; ++pp)
          if (L->ci[pp] == i) aii = L->val[pp];
        L->wd[i] = L->omega / aii;
      }
    }
  }
  build_members(h);
  *err = factor_coarsest(h);
  if (*err) {
    or_free(h);
    return NULL;
  }
  return h;
}

/* The rows [r0, r1) of level 0 and everything below them, as a hierarchy of
 * their own.  When independent systems are set up together as one
 * block-diagonal matrix, no strong connection joins two blocks, so no
 * aggregate and no Galerkin entry crosses them and each system keeps a
 * contiguous range of rows on every level; this view is the hierarchy that
 * system is solved on.  Values are copied, nothing is recomputed except the
 * dense factor of the coarsest block (as in or_setup). */
or_hier *or_subsystem(const or_hier *h, int32_t r0, int32_t r1, int32_t *err) {
  *err = -2;
  if (r0 < 0 || r1 > h->lev[0].n || r0 >= r1) return NULL;
  or_hier *s = (or_hier *)calloc(1, sizeof(or_hier));
  s->p = h->p;
  s->L = 0;
  int32_t a = r0, b = r1;
  for (int32_t k = 0; k < h->L; ++k) {
    const or_level *L = &h->lev[k];
    or_level *S = &s->lev[k];
    s->L = k + 1;
    const int32_t n = b - a;
    const int64_t p0 = L->rp[a], p1 = L->rp[b];
    S->n = n;
    S->nnz = p1 - p0;
    S->mis_rounds = L->mis_rounds;
    S->omega = L->omega;
    S->rp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    S->ci = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S->nnz + 1));
    S->val = dalloc((size_t)S->nnz);
    S->B = dalloc((size_t)n);
    level_alloc_work(S);
    for (int32_t i = 0; i <= n; ++i) S->rp[i] = (int32_t)(L->rp[a + i] - p0);
    for (int64_t q = p0; q < p1; ++q) {
      if (L->ci[q] < a || L->ci[q] >= b) goto fail; /* the block couples to other rows */
      S->ci[q - p0] = L->ci[q] - a;
      S->val[q - p0] = L->val[q];
    }
    for (int32_t i = 0; i < n; ++i) {
      S->B[i] = L->B[a + i];
      S->dinv[i] = L->dinv[a + i];
      S->wd[i] = L->wd[a + i];
    }
    if (L->poly) {
      S->poly = dalloc((size_t)n * 3);
      memcpy(S->poly, L->poly + (size_t)a * 3, sizeof(double) * (size_t)n * 3);
    }
    if (k == h->L - 1) break;
    /* the block's aggregates: a contiguous range of coarse rows that no row
     * outside the block joins */
    int32_t lo = INT32_MAX, hi = -1;
    for (int32_t i = a; i < b; ++i) {
      if (L->agg[i] < lo) lo = L->agg[i];
      if (L->agg[i] > hi) hi = L->agg[i];
    }
    for (int32_t i = 0; i < L->n; ++i)
      if ((i < a || i >= b) && L->agg[i] >= lo && L->agg[i] <= hi) goto fail;
    S->nc = hi - lo + 1;
    S->agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->P = dalloc((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
      S->agg[i] = L->agg[a + i] - lo;
      S->P[i] = L->P[a + i];
    }
    a = lo;
    b = hi + 1;
  }
  build_members(s);
  *err = factor_coarsest(s);
  if (*err) {
    or_free(s);
    return NULL;
  }
  return s;
fail:
  or_free(s);
  *err = -2;
  return NULL;
}

int32_t or_nlevels(const or_hier *h) { return h->L; }

void or_level_info(const or_hier *h, int32_t k, int32_t *n, int64_t *nnz, double *omega,
                   int32_t *mis_rounds) {
  *n = h->lev[k].n;
  *nnz = h->lev[k].nnz;
  *omega = h->lev[k].omega;
  *mis_rounds = h->lev[k].mis_rounds;
}

void or_level_copy(const or_hier *h, int32_t k, int32_t *rp, int32_t *ci, double *val,
                   int32_t *agg, double *P, double *B) {
  const or_level *L = &h->lev[k];
  if (rp) memcpy(rp, L->rp, sizeof(int32_t) * ((size_t)L->n + 1));
  if (ci) memcpy(ci, L->ci, sizeof(int32_t) * (size_t)L->nnz);
  if (val) memcpy(val, L->val, sizeof(double) * (size_t)L->nnz);
  if (agg && L->agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->n);
  if (P && L->P) memcpy(P, L->P, sizeof(double) * (size_t)L->n);
  if (B && L->B) memcpy(B, L->B, sizeof(double) * (size_t)L->n);
}

int32_t or_set_poly(or_hier *h, int32_t k, const double *coef) {
  if (k < 0 || k >= h->L - 1) return -1;
  or_level *L = &h->lev[k];
  free(L->poly);
  L->poly = dalloc((size_t)L->n * 3);
  memcpy(L->poly, coef, sizeof(double) * (size_t)L->n * 3);
  return 0;
}

static void spmv(const or_level *L, const double *x, double *y) {
  OR_PAR
  for (int32_t i = 0; i < L->n; ++i) {
    double acc = 0.0;
    for (int32_t p = L->rp[i]; p < L->rp[i + 1]; ++p) acc += L->val[p] * x[L->ci[p]];
    y[i] = acc;
  }
}

static double dot(int32_t n, const double *a, const double *b) {
#ifdef _OPENMP
  const int32_t nch = (n + OR_DOT_CHUNK - 1) / OR_DOT_CHUNK;
  if (nch > 1) {
    double *part = (double *)malloc(sizeof(double) * (size_t)nch);
    OR_PAR
    for (int32_t c = 0; c < nch; ++c) {
      double t = 0.0;
      const int32_t e = c * OR_DOT_CHUNK + OR_DOT_CHUNK < n ? c * OR_DOT_CHUNK + OR_DOT_CHUNK : n;
      for (int32_t i = c * OR_DOT_CHUNK; i < e; ++i) t += a[i] * b[i];
      part[c] = t;
    }
    double s = 0.0;
    for (int32_t c = 0; c < nch; ++c) s += part[c];
    free(part);
    return s;
  }
#endif
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Pre-smoothing from x = 0.  Damped Jacobi: x = omega D^-1 b.  Polynomial
 * smoother with per-row coefficients c_q: x = sum_q diag(c_q) (D^-1 A)^q D^-1 b
 * (c = (omega, 0, 0) is damped Jacobi). */
static void smooth_pre(or_hier *h, int32_t k, const double *b, double *x) {
  or_level *L = &h->lev[k];
  int32_t n = L->n;
  if (!L->poly) {
    OR_PAR
    for (int32_t i = 0; i < n; ++i) x[i] = L->wd[i] * b[i];
    return;
  }
  OR_PAR
  for (int32_t i = 0; i < n; ++i) L->u0[i] = L->dinv[i] * b[i];
  spmv(L, L->u0, L->u1);
  OR_PAR
  for (int32_t i = 0; i < n; ++i) L->u1[i] = L->dinv[i] * L->u1[i];
  spmv(L, L->u1, L->r);
  OR_PAR
  for (int32_t i = 0; i < n; ++i) {
    double u2 = L->dinv[i] * L->r[i];
    x[i] = L->poly[3 * i] * L->u0[i] + L->poly[3 * i + 1] * L->u1[i] + L->poly[3 * i + 2] * u2;
  }
}

/* Post-smoothing: r = b - A x, x <- x + G^T r.  For damped Jacobi G^T r =
 * omega D^-1 r (Eq. damped Jacobi).  For the polynomial smoother the post step
 * applies the transpose of the pre step, sum_q (D^-1 A)^q D^-1 diag(c_q) r,
 * evaluated by Horner's rule, so that the cycle stays symmetric. */
static void smooth_post(or_hier *h, int32_t k, const double *b, double *x) {
  or_level *L = &h->lev[k];
  int32_t n = L->n;
  spmv(L, x, L->r);
  OR_PAR
  for (int32_t i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
  if (!L->poly) {
    OR_PAR
    for (int32_t i = 0; i < n; ++i) x[i] = x[i] + L->wd[i] * L->r[i];
    return;
  }
  OR_PAR
  for (int32_t i = 0; i < n; ++i) L->u0[i] = L->dinv[i] * (L->poly[3 * i + 2] * L->r[i]);
  spmv(L, L->u0, L->u1);
  OR_PAR
  for (int32_t i = 0; i < n; ++i)
    L->u1[i] = L->dinv[i] * L->u1[i] + L->dinv[i] * (L->poly[3 * i + 1] * L->r[i]);
  spmv(L, L->u1, L->u0);
  OR_PAR
  for (int32_t i = 0; i < n; ++i)
    x[i] = x[i] + (L->dinv[i] * L->u0[i] + L->dinv[i] * (L->poly[3 * i] * L->r[i]));
}

static void coarsest_solve(or_hier *h, const double *b, double *x) {
  int32_t n = h->lev[h->L - 1].n;
  for (int32_t i = 0; i < n; ++i) x[i] = b[i];
  if (h->piv)
    or_lu_solve(n, h->chol, h->piv, x);
  else
    or_chol_solve(n, h->chol, x);
}

static void cycle(or_hier *h, int32_t k, const double *b, double *x);

/* Alg. 5, coarse part at level m (= k+1): two inner Krylov steps with cycle(m).
 * Reading: each inner call starts from x = 0; the CG variant is used inside
 * flexible CG and the GMRES variant inside FGMRES. */
static void krylov2(or_hier *h, int32_t m, const double *r, double *x) {
  or_level *L = &h->lev[m];
  int32_t n = L->n;
  int gm = h->p.outer == 1;
  h->kcalls[m]++;
  cycle(h, m, r, L->c);
  spmv(L, L->c, L->v);
  double rho1 = gm ? dot(n, L->v, L->v) : dot(n, L->c, L->v);
  double a1 = gm ? dot(n, L->v, r) : dot(n, L->c, r);
  double s1 = a1 / rho1;
  OR_PAR
  for (int32_t i = 0; i < n; ++i) L->rt[i] = r[i] - s1 * L->v[i];
  double nrt = sqrt(dot(n, L->rt, L->rt)), nr = sqrt(dot(n, r, r));
  if (nrt <= h->p.kcycle_t * nr) {
    OR_PAR
    for (int32_t i = 0; i < n; ++i) x[i] = s1 * L->c[i];
    return;
  }
  h->second[m]++;
  cycle(h, m, L->rt, L->d);
  spmv(L, L->d, L->w);
  double gam = gm ? dot(n, L->w, L->v) : dot(n, L->d, L->v);
  double bet = gm ? dot(n, L->w, L->w) : dot(n, L->d, L->w);
  double a2 = gm ? dot(n, L->w, L->rt) : dot(n, L->d, L->rt);
  double rho2 = bet - gam * gam / rho1;
  double cc = s1 - gam * a2 / (rho1 * rho2), cd = a2 / rho2;
  OR_PAR
  for (int32_t i = 0; i < n; ++i) x[i] = cc * L->c[i] + cd * L->d[i];
}

/* Alg. 4 / Alg. 5 at level k with x = 0 on entry.  Reading of the residual
 * after prolongation ("r~_k" is not defined at level k): r_k = b_k - A_k x_k,
 * and the post-smoothing step uses b_k as its right-hand side. */
static void cycle(or_hier *h, int32_t k, const double *b, double *x) {
  h->visits[k]++;
  if (k == h->L - 1) {
    coarsest_solve(h, b, x);
    return;
  }
  or_level *L = &h->lev[k];
  or_level *C = &h->lev[k + 1];
  int32_t n = L->n;
  smooth_pre(h, k, b, x);                                  /* pre-smoothing */
  spmv(L, x, L->r);                                        /* r_k = b_k - A_k x_k */
  OR_PAR
  for (int32_t i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
#ifdef _OPENMP
  OR_PAR
  for (int32_t I = 0; I < C->n; ++I) {                     /* the same sums, per aggregate */
    double t = 0.0;
    for (int32_t q = L->aptr[I]; q < L->aptr[I + 1]; ++q) t = t + L->P[L->amem[q]] * L->r[L->amem[q]];
    C->bc[I] = t;
  }
#else
  for (int32_t I = 0; I < C->n; ++I) C->bc[I] = 0.0;       /* r_{k+1} = R_k r_k, summed in */
  for (int32_t i = 0; i < n; ++i)                          /* ascending fine index         */
    C->bc[L->agg[i]] = C->bc[L->agg[i]] + L->P[i] * L->r[i];
#endif
  if (k + 1 == h->L - 1) {
    h->visits[k + 1]++;
    coarsest_solve(h, C->bc, C->xc);                       /* exact coarse solve */
  }
  else if (k < h->p.kcycle_levels)
    krylov2(h, k + 1, C->bc, C->xc);                       /* K-cycle coarse correction */
  else
    cycle(h, k + 1, C->bc, C->xc);                         /* V-cycle recursion */
  OR_PAR
  for (int32_t i = 0; i < n; ++i) x[i] = x[i] + L->P[i] * C->xc[L->agg[i]]; /* prolongation */
  smooth_post(h, k, b, x);                                 /* post-smoothing */
}

static void trace_reset(or_hier *h) {
  for (int32_t k = 0; k < OR_MAX_LEVELS; ++k) h->visits[k] = h->kcalls[k] = h->second[k] = 0;
}

void or_cycle_trace(const or_hier *h, int64_t *visits, int64_t *kcalls, int64_t *second) {
  for (int32_t k = 0; k < h->L; ++k) {
    visits[k] = h->visits[k];
    kcalls[k] = h->kcalls[k];
    second[k] = h->second[k];
  }
}

void or_precond(or_hier *h, const double *b, double *x) {
  trace_reset(h);
  cycle(h, 0, b, x);
}

/* Flexible CG (Sec. 2.2; the K-cycle is a variable preconditioner).  Reading:
 * one-term A-orthogonalisation, beta = -(z^T q_old)/(p_old^T q_old), which
 * equals the Polak-Ribiere form z^T(r_new - r_old)/(z_old^T r_old) in exact
 * arithmetic; alpha = p^T r / p^T A p.  When the updated residual meets the
 * tolerance the true residual b - A x is recomputed; if it does not meet it
 * the iteration restarts from that residual (iterative refinement). */
static int32_t fcg(or_hier *h, const double *b, double *x, double tol, int32_t max_iter,
                   int32_t *iters, double *hist, double *final_relres) {
  or_level *L = &h->lev[0];
  int32_t n = L->n;
  double *r = dalloc((size_t)n), *z = dalloc((size_t)n), *p = dalloc((size_t)n),
         *q = dalloc((size_t)n);
  int32_t it = 0, status = 1;
  double nb = sqrt(dot(n, b, b));
  if (nb == 0.0) nb = 1.0;
  spmv(L, x, r);
  OR_PAR
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  double rel = sqrt(dot(n, r, r)) / nb;
  if (hist) hist[0] = rel;
  if (rel <= tol) status = 0;
  while (status == 1 && it < max_iter) {
    cycle(h, 0, r, z); /* restart: p = z */
    OR_PAR
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    for (;;) {
      spmv(L, p, q);
      double pq = dot(n, p, q), pr = dot(n, p, r);
      if (!(pq > 0.0)) {
        status = -1;
        break;
      }
      double alpha = pr / pq;
      OR_PAR
      for (int32_t i = 0; i < n; ++i) {
        x[i] = x[i] + alpha * p[i];
        r[i] = r[i] - alpha * q[i];
      }
      it++;
      rel = sqrt(dot(n, r, r)) / nb;
      if (hist) hist[it] = rel;
      if (rel <= tol) {
        spmv(L, x, r); /* true residual */
        OR_PAR
        for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        rel = sqrt(dot(n, r, r)) / nb;
        if (rel <= tol) status = 0;
        break;
      }
      if (it >= max_iter) break;
      cycle(h, 0, r, z);
      double beta = -dot(n, z, q) / pq;
      OR_PAR
      for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (status == -1) break;
  }
  spmv(L, x, r);
  OR_PAR
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  *final_relres = sqrt(dot(n, r, r)) / nb;
  *iters = it;
  free(r); free(z); free(p); free(q);
  return status;
}

/* Flexible GMRES(m) with modified Gram-Schmidt and Givens rotations. */
static int32_t fgmres(or_hier *h, const double *b, double *x, double tol, int32_t max_iter,
                      int32_t *iters, double *hist, double *final_relres) {
  or_level *L = &h->lev[0];
  int32_t n = L->n, m = h->p.restart;
  double *V = dalloc((size_t)n * (size_t)(m + 1)), *Z = dalloc((size_t)n * (size_t)m);
  double *r = dalloc((size_t)n), *w = dalloc((size_t)n);
  double *H = dalloc((size_t)(m + 1) * (size_t)m), *g = dalloc((size_t)m + 1);
  double *cs = dalloc((size_t)m), *sn = dalloc((size_t)m), *y = dalloc((size_t)m);
  int32_t it = 0, status = 1;
  double nb = sqrt(dot(n, b, b));
  if (nb == 0.0) nb = 1.0;
  int first = 1;
  for (;;) {
    spmv(L, x, r);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double beta = sqrt(dot(n, r, r));
    if (first && hist) hist[0] = beta / nb;
    first = 0;
    if (beta / nb <= tol) {
      status = 0;
      break;
    }
    if (it >= max_iter) break;
    for (int32_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int32_t j = 0; j <= m; ++j) g[j] = 0.0;
    g[0] = beta;
    int32_t j = 0;
    int conv = 0;
    for (; j < m && it < max_iter; ++j) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
      cycle(h, 0, vj, zj);
      spmv(L, zj, w);
      for (int32_t l = 0; l <= j; ++l) {
        double *vl = V + (size_t)l * n;
        double hl = dot(n, w, vl);
        H[l * m + j] = hl;
        for (int32_t i = 0; i < n; ++i) w[i] = w[i] - hl * vl[i];
      }
      double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (int32_t i = 0; i < n; ++i) V[(size_t)(j + 1) * n + i] = w[i] / hn;
      for (int32_t l = 0; l < j; ++l) { /* previous rotations */
        double a = H[l * m + j], bb = H[(l + 1) * m + j];
        H[l * m + j] = cs[l] * a + sn[l] * bb;
        H[(l + 1) * m + j] = -sn[l] * a + cs[l] * bb;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double den = sqrt(a * a + bb * bb);
      cs[j] = a / den;
      sn[j] = bb / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      it++;
      double rel = fabs(g[j + 1]) / nb;
      if (hist) hist[it] = rel;
      if (rel <= tol || hn == 0.0) {
        conv = 1;
        j++;
        break;
      }
    }
    for (int32_t l = j - 1; l >= 0; --l) { /* back substitution */
      double t = g[l];
      for (int32_t q = l + 1; q < j; ++q) t = t - H[l * m + q] * y[q];
      y[l] = t / H[l * m + l];
    }
    for (int32_t l = 0; l < j; ++l)
      for (int32_t i = 0; i < n; ++i) x[i] = x[i] + y[l] * Z[(size_t)l * n + i];
    (void)conv;
  }
  spmv(L, x, r);
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  *final_relres = sqrt(dot(n, r, r)) / nb;
  if (*final_relres <= tol) status = 0;
  *iters = it;
  free(V); free(Z); free(r); free(w); free(H); free(g); free(cs); free(sn); free(y);
  return status;
}

int32_t or_solve(or_hier *h, const double *b, double *x, double tol, int32_t max_iter,
                 int32_t *iters, double *hist, double *final_relres) {
  trace_reset(h);
  if (h->p.outer == 1) return fgmres(h, b, x, tol, max_iter, iters, hist, final_relres);
  return fcg(h, b, x, tol, max_iter, iters, hist, final_relres);
}

/* Test hook: run the Alg. 5 coarse part at level m on r and expose its inner
 * iterates c (first cycle) and d (second cycle, zero if not taken). */
int32_t or_krylov2_probe(or_hier *h, int32_t m, const double *r, double *x, double *c, double *d) {
  if (m <= 0 || m >= h->L - 1) return -1;
  or_level *L = &h->lev[m];
  for (int32_t i = 0; i < L->n; ++i) L->d[i] = 0.0;
  krylov2(h, m, r, x);
  memcpy(c, L->c, sizeof(double) * (size_t)L->n);
  memcpy(d, L->d, sizeof(double) * (size_t)L->n);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Learned per-row polynomial smoother.  The paper lists polynomial smoothers */
/* as future work (Sec. 5); the coefficients here come from a small MLP on    */
/* per-row features, trained to minimise the two-grid error reduction.        */
/* ------------------------------------------------------------------------- */

/* Features of row i (d = |A_ii|, t_j = -A_ij/d for j != i), all scale-free:
 *  0: 1                      1: (#off-diagonals)/8
 *  2..9: the eight largest |A_ij|/d, descending, zero-padded
 *  10: fraction of off-diagonals with the sign of A_ii
 *  11: (sum_j A_ij)/A_ii      12: level/4
 *  13: min_j t_j              14: max_j t_j
 *  15: sum_{j != i} |A_ij|/d  (sums in CSR order) */
void or_features(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, int32_t level,
                 float *feat) {
  for (int32_t i = 0; i < n; ++i) {
    double aii = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) aii = val[p];
    double d = fabs(aii), top[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double rowsum = 0.0, abssum = 0.0, tmin = 0.0, tmax = 0.0;
    int32_t noff = 0, nsame = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      rowsum = rowsum + val[p];
      if (ci[p] == i) continue;
      double a = fabs(val[p]) / d, t = -val[p] / d;
      abssum = abssum + a;
      if (noff == 0 || t < tmin) tmin = t;
      if (noff == 0 || t > tmax) tmax = t;
      if ((val[p] > 0.0 && aii > 0.0) || (val[p] < 0.0 && aii < 0.0)) nsame++;
      noff++;
      for (int k = 0; k < 8; ++k) /* insert into the descending top-8 list */
        if (a > top[k]) {
          for (int q = 7; q > k; --q) top[q] = top[q - 1];
          top[k] = a;
          break;
        }
    }
    float *f = feat + (size_t)i * OR_NFEAT;
    f[0] = 1.0f;
    f[1] = (float)((double)noff / 8.0);
    for (int k = 0; k < 8; ++k) f[2 + k] = (float)top[k];
    f[10] = noff ? (float)((double)nsame / (double)noff) : 0.0f;
    f[11] = (float)(rowsum / aii);
    f[12] = (float)((double)level / 4.0);
    f[13] = (float)tmin;
    f[14] = (float)tmax;
    f[15] = (float)abssum;
  }
}

/* IEEE binary16 -> binary32 from the bit pattern (every half is exact in float) */
static float half_to_float(uint16_t h) {
  uint32_t sign = (uint32_t)(h >> 15) << 31, ex = (h >> 10) & 0x1F, man = h & 0x3FF, bits;
  if (ex == 0) {
    if (man == 0) {
      bits = sign;
    } else { /* subnormal: normalise */
      int e = -1;
      do {
        e++;
        man <<= 1;
      } while (!(man & 0x400));
      bits = sign | ((uint32_t)(127 - 15 - e) << 23) | ((man & 0x3FF) << 13);
    }
  } else if (ex == 31) {
    bits = sign | 0x7F800000u | (man << 13);
  } else {
    bits = sign | ((ex - 15 + 127) << 23) | (man << 13);
  }
  float f;
  memcpy(&f, &bits, sizeof(f));
  return f;
}

#define W1_OFF 0
#define B1_OFF (OR_HID * OR_NFEAT)
#define W2_OFF (B1_OFF + OR_HID)
#define B2_OFF (W2_OFF + OR_HID * OR_HID)
#define W3_OFF (B2_OFF + OR_HID)
#define B3_OFF (W3_OFF + OR_NOUT * OR_HID)

void or_mlp_forward(int32_t n, const uint16_t *w16, const float *feat, float *out) {
  float w[OR_NPARAM];
  for (int k = 0; k < OR_NPARAM; ++k) w[k] = half_to_float(w16[k]);
  for (int32_t i = 0; i < n; ++i) {
    const float *f = feat + (size_t)i * OR_NFEAT;
    float h1[OR_HID], h2[OR_HID];
    for (int u = 0; u < OR_HID; ++u) {
      float z = w[B1_OFF + u];
      for (int k = 0; k < OR_NFEAT; ++k) z += w[W1_OFF + u * OR_NFEAT + k] * f[k];
      h1[u] = tanhf(z);
    }
    for (int v = 0; v < OR_HID; ++v) {
      float z = w[B2_OFF + v];
      for (int u = 0; u < OR_HID; ++u) z += w[W2_OFF + v * OR_HID + u] * h1[u];
      h2[v] = tanhf(z);
    }
    for (int q = 0; q < OR_NOUT; ++q) {
      float z = w[B3_OFF + q];
      for (int v = 0; v < OR_HID; ++v) z += w[W3_OFF + q * OR_HID + v] * h2[v];
      out[(size_t)i * OR_NOUT + q] = z;
    }
  }
}

void or_mlp_backward(int32_t n, const double *w, const float *feat, const double *dout, double *dparam,
                     double *out) {
  for (int k = 0; k < OR_NPARAM; ++k) dparam[k] = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const float *f = feat + (size_t)i * OR_NFEAT;
    double h1[OR_HID], h2[OR_HID], dz2[OR_HID];
    for (int u = 0; u < OR_HID; ++u) {
      double z = w[B1_OFF + u];
      for (int k = 0; k < OR_NFEAT; ++k) z += w[W1_OFF + u * OR_NFEAT + k] * (double)f[k];
      h1[u] = tanh(z);
    }
    for (int v = 0; v < OR_HID; ++v) {
      double z = w[B2_OFF + v];
      for (int u = 0; u < OR_HID; ++u) z += w[W2_OFF + v * OR_HID + u] * h1[u];
      h2[v] = tanh(z);
    }
    const double *g = dout + (size_t)i * OR_NOUT;
    for (int q = 0; q < OR_NOUT; ++q) {
      double z = w[B3_OFF + q];
      for (int v = 0; v < OR_HID; ++v) z += w[W3_OFF + q * OR_HID + v] * h2[v];
      if (out) out[(size_t)i * OR_NOUT + q] = z;
      dparam[B3_OFF + q] += g[q];
      for (int v = 0; v < OR_HID; ++v) dparam[W3_OFF + q * OR_HID + v] += g[q] * h2[v];
    }
    for (int v = 0; v < OR_HID; ++v) {
      double dh = 0.0;
      for (int q = 0; q < OR_NOUT; ++q) dh += w[W3_OFF + q * OR_HID + v] * g[q];
      dz2[v] = dh * (1.0 - h2[v] * h2[v]);
      dparam[B2_OFF + v] += dz2[v];
      for (int u = 0; u < OR_HID; ++u) dparam[W2_OFF + v * OR_HID + u] += dz2[v] * h1[u];
    }
    for (int u = 0; u < OR_HID; ++u) {
      double dh = 0.0;
      for (int v = 0; v < OR_HID; ++v) dh += w[W2_OFF + v * OR_HID + u] * dz2[v];
      const double dz1 = dh * (1.0 - h1[u] * h1[u]);
      dparam[B1_OFF + u] += dz1;
      for (int k = 0; k < OR_NFEAT; ++k) dparam[W1_OFF + u * OR_NFEAT + k] += dz1 * (double)f[k];
    }
  }
}

/* random error vector v of the two-grid measurement: uniform in [-1, 1) */
static double twogrid_error(uint64_t seed, int32_t v, int32_t i) {
  uint64_t z = or_splitmix64(seed ^ ((uint64_t)(uint32_t)(v + 1) << 44) ^ (uint64_t)(uint32_t)i);
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

double or_twogrid_loss(or_hier *h, const double *coef, int32_t nvec, uint64_t seed, double *dcoef) {
  if (h->L < 2) return -1.0;
  or_level *L = &h->lev[0];
  or_level *Cl = &h->lev[1];
  const int32_t n = L->n, nc = Cl->n;
  double *e0 = dalloc((size_t)n), *Ae = dalloc((size_t)n), *u0 = dalloc((size_t)n), *u1 = dalloc((size_t)n),
         *u2 = dalloc((size_t)n), *e1 = dalloc((size_t)n), *rc = dalloc((size_t)nc);
  double loss = 0.0;
  if (dcoef)
    for (int32_t i = 0; i < 3 * n; ++i) dcoef[i] = 0.0;
  for (int32_t v = 0; v < nvec; ++v) {
    for (int32_t i = 0; i < n; ++i) e0[i] = twogrid_error(seed, v, i);
    spmv(L, e0, Ae);
    const double nrm0 = dot(n, e0, Ae);
    for (int32_t i = 0; i < n; ++i) u0[i] = L->dinv[i] * Ae[i];   /* D^-1 A e0 */
    spmv(L, u0, u1);
    for (int32_t i = 0; i < n; ++i) u1[i] = L->dinv[i] * u1[i];   /* (D^-1 A) D^-1 A e0 */
    spmv(L, u1, u2);
    for (int32_t i = 0; i < n; ++i) u2[i] = L->dinv[i] * u2[i];
    for (int32_t i = 0; i < n; ++i) /* e1 = (I - G A) e0 */
      e1[i] = e0[i] - (coef[3 * i] * u0[i] + coef[3 * i + 1] * u1[i] + coef[3 * i + 2] * u2[i]);
    spmv(L, e1, Ae);                                               /* coarse correction */
    for (int32_t I = 0; I < nc; ++I) rc[I] = 0.0;
    for (int32_t i = 0; i < n; ++i) rc[L->agg[i]] = rc[L->agg[i]] + L->P[i] * Ae[i];
    or_chol_solve(nc, h->chol, rc);
    for (int32_t i = 0; i < n; ++i) e1[i] = e1[i] - L->P[i] * rc[L->agg[i]];
    spmv(L, e1, Ae);
    const double num = dot(n, e1, Ae);
    loss += num / nrm0 / nvec;
    if (dcoef) /* dL/de1 = 2 A e2 / nrm0 (A e2 is A-orthogonal to range(P)); e1 = e0 - sum c u */
      for (int32_t i = 0; i < n; ++i) {
        const double g = 2.0 * Ae[i] / nrm0 / nvec;
        dcoef[3 * i] -= g * u0[i];
        dcoef[3 * i + 1] -= g * u1[i];
        dcoef[3 * i + 2] -= g * u2[i];
      }
  }
  free(e0); free(Ae); free(u0); free(u1); free(u2); free(e1); free(rc);
  return loss;
}
