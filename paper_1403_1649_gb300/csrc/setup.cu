// setup.cu -- GPU setup of the aggregation AMG hierarchy (Alg. 1).
//
// Per level: classic strength (Sec. 2.1.1), the symmetrised strong graph,
// PMIS(2) (Alg. 2), nearest-root aggregation (Sec. 2.1.2), interpolation
// (Alg. 3), the Galerkin product as a keyed sum (Sec. 3.1), then the
// solve-phase data: SELL-32 matrix, damped-Jacobi weights with omega from an
// Arnoldi estimate (Eq. damped Jacobi), and the dense inverse of the coarsest
// level.  Every floating-point step that decides the hierarchy (strength test,
// B norms, P weights, Galerkin products and sums) is rounded operation by
// operation with __dmul_rn/__dadd_rn/__ddiv_rn/__dsqrt_rn in a fixed order, so
// the hierarchy is identical to a sequential FP64 evaluation.
#include <climits>
#include <cstdio>

#include "amg_internal.cuh"
#include "scan.cuh"

namespace amg {

// ============================================================== input checks
// bit 1: bad row pointers, bit 2: column out of range / not ascending,
// bit 4: diagonal missing or zero, bit 8: NaN/Inf value
__global__ void k_check_csr(int32_t n, int64_t nnz, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ val,
                            int *__restrict__ err) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = 0;
  int32_t p0 = rp[i], p1 = rp[i + 1];
  if (p1 < p0 || p0 < 0 || (int64_t)p1 > nnz || (i == 0 && p0 != 0) || (i == n - 1 && (int64_t)p1 != nnz)) {
    atomicOr(err, 1);
    return;
  }
  bool diag = false;
  for (int32_t p = p0; p < p1; ++p) {
    int32_t j = ci[p];
    if (j < 0 || j >= n || (p > p0 && j <= ci[p - 1])) e |= 2;
    double v = val[p];
    if (!isfinite(v)) e |= 8;
    if (j == i && v != 0.0) diag = true;
  }
  if (!diag) e |= 4;
  if (e) atomicOr(err, e);
}

// ============================================================== strength
// Sec. 2.1.1: C_ij = 1 iff -s_i A_ij > alpha * max_{j: -s_i A_ij > 0} -s_i A_ij.
// Also counts the strong entries of each row (rowcnt) and of each column
// (colcnt = #{j : C_ji = 1}, the priority count of Alg. 2).
__global__ void k_strength(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, double alpha, uint8_t *__restrict__ C,
                           int32_t *__restrict__ rowcnt, int32_t *__restrict__ colcnt) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t p0 = rp[i], p1 = rp[i + 1];
    double aii = 0.0;
    for (int32_t p = p0; p < p1; ++p)
      if (ci[p] == i) aii = val[p];
    const double s = aii > 0.0 ? 1.0 : (aii < 0.0 ? -1.0 : 0.0);
    bool have = false;
    double mx = 0.0;
    for (int32_t p = p0; p < p1; ++p) {
      double t = -__dmul_rn(s, val[p]);
      if (ci[p] != i && t > 0.0 && (!have || t > mx)) {
        mx = t;
        have = true;
      }
    }
    const double thr = __dmul_rn(alpha, mx);
    int32_t cnt = 0;
    for (int32_t p = p0; p < p1; ++p) {
      double t = -__dmul_rn(s, val[p]);
      bool strong = have && ci[p] != i && t > thr;
      C[p] = strong;
      if (strong) {
        cnt++;
        atomicAdd(&colcnt[ci[p]], 1);
      }
    }
    rowcnt[i] = cnt;
  }
}

__global__ void k_add_i32(int32_t n, const int32_t *a, const int32_t *b, int32_t *c) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] + b[i];
}

// N_i = {j != i : C_ij or C_ji}: row i of the work array holds its own strong
// columns first, then (via atomics, in any order) the rows that hold i strongly.
__global__ void k_sym_fill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const uint8_t *__restrict__ C, const int32_t *__restrict__ rowcnt,
                           const int32_t *__restrict__ off, int32_t *__restrict__ cursor,
                           int32_t *__restrict__ tmp) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t k = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (!C[p]) continue;
      const int32_t j = ci[p];
      tmp[off[i] + k++] = j;
      const int32_t q = atomicAdd(&cursor[j], 1);
      tmp[off[j] + rowcnt[j] + q] = i;
    }
  }
}

// Sort a short segment in place (insertion sort; Shell gaps for long ones).
__device__ void sort_segment(int32_t *a, int32_t len) {
  if (len > 48) {
    int gaps[] = {701, 301, 132, 57, 23, 10, 4};
    for (int g : gaps) {
      if (g >= len) continue;
      for (int32_t i = g; i < len; ++i) {
        int32_t t = a[i], j = i;
        while (j >= g && a[j - g] > t) {
          a[j] = a[j - g];
          j -= g;
        }
        a[j] = t;
      }
    }
  }
  for (int32_t i = 1; i < len; ++i) {
    int32_t t = a[i], j = i;
    while (j > 0 && a[j - 1] > t) {
      a[j] = a[j - 1];
      --j;
    }
    a[j] = t;
  }
}

__global__ void k_sort_unique(int32_t n, const int32_t *__restrict__ off, int32_t *__restrict__ tmp,
                              int32_t *__restrict__ ucount) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t *a = tmp + off[i];
    const int32_t len = off[i + 1] - off[i];
    sort_segment(a, len);
    int32_t u = 0;
    for (int32_t k = 0; k < len; ++k)
      if (k == 0 || a[k] != a[k - 1]) a[u++] = a[k];
    ucount[i] = u;
  }
}

// Structurally symmetric patterns: N_i = {j : C_ij or C_ji} is a subset of row
// i of A, so it can be marked in place (the entry (j, i) is found by binary
// search in the sorted row j) and compacted in CSR order, which is already
// ascending and duplicate-free.  A missing mirror entry sets *nonsym and the
// caller falls back to the general construction.
__global__ void k_sym_mirror(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const uint8_t *__restrict__ C, uint8_t *__restrict__ S, int32_t *__restrict__ scount,
                             int *__restrict__ nonsym) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t cnt = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t j = ci[p];
      if (j == i) {
        S[p] = 0;
        continue;
      }
      int32_t lo = rp[j], hi = rp[j + 1] - 1, q = -1;
      while (lo <= hi) {
        const int32_t mid = (lo + hi) >> 1;
        const int32_t c = ci[mid];
        if (c == i) {
          q = mid;
          break;
        }
        if (c < i) lo = mid + 1; else hi = mid - 1;
      }
      if (q < 0) atomicOr(nonsym, 1);
      const uint8_t sv = C[p] | (q >= 0 ? C[q] : (uint8_t)0);
      S[p] = sv;
      cnt += sv;
    }
    scount[i] = cnt;
  }
}

__global__ void k_sym_mirror_fill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                  const uint8_t *__restrict__ S, const int32_t *__restrict__ Sptr,
                                  int32_t *__restrict__ Scol) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t k = Sptr[i];
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (S[p]) Scol[k++] = ci[p];
  }
}

__global__ void k_compact(int32_t n, const int32_t *__restrict__ off, const int32_t *__restrict__ tmp,
                          const int32_t *__restrict__ Sptr, int32_t *__restrict__ Scol) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t len = Sptr[i + 1] - Sptr[i];
    for (int32_t k = 0; k < len; ++k) Scol[Sptr[i] + k] = tmp[off[i] + k];
  }
}

// ============================================================== PMIS(2), Alg. 2
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Priority v_i = count_i + r_i of Alg. 2 held exactly as the integer pair
// (count_i, h_i), r_i = (h_i + 1/2)/2^32, packed as count << 32 | h.
__global__ void k_mis_keys(int32_t n, const int32_t *__restrict__ colcnt, uint64_t seed, int32_t level,
                           uint64_t *__restrict__ key, int8_t *__restrict__ s) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = (uint32_t)(splitmix64(seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)(uint32_t)i) >> 32);
  key[i] = ((uint64_t)(uint32_t)colcnt[i] << 32) | h;
  s[i] = 0;
}

// tuple (s, v, i): the state occupies the top two bits of the packed word
__device__ __forceinline__ uint64_t pack_tuple(int8_t s, uint64_t key) {
  return ((uint64_t)(s + 1) << 62) | key;
}
__device__ __forceinline__ bool tuple_gt(uint64_t wa, int32_t ia, uint64_t wb, int32_t ib) {
  return wa > wb || (wa == wb && ia > ib);
}

// first max round over the closed neighbourhood, from the current states
// (also clears the round's undecided count *und_reset, which the decision fills)
__global__ void k_pmis_max1(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const int8_t *__restrict__ s, const uint64_t *__restrict__ key,
                            uint64_t *__restrict__ Tw, int32_t *__restrict__ Ti, int32_t *__restrict__ und_reset) {
  pdl_wait_and_trigger();
  if (und_reset && blockIdx.x == 0 && threadIdx.x == 0) *und_reset = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t bw = pack_tuple(s[i], key[i]);
    int32_t bi = i;
    for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
      const int32_t j = Scol[q];
      const uint64_t w = pack_tuple(s[j], key[j]);
      if (tuple_gt(w, j, bw, bi)) {
        bw = w;
        bi = j;
      }
    }
    Tw[i] = bw;
    Ti[i] = bi;
  }
}

// a middle max round of MIS(k), k > 2: (Tw, Ti) -> (Tw2, Ti2) over the closed
// neighbourhood
__global__ void k_pmis_maxk(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const uint64_t *__restrict__ Tw, const int32_t *__restrict__ Ti,
                            uint64_t *__restrict__ Tw2, int32_t *__restrict__ Ti2) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t bw = Tw[i];
    int32_t bi = Ti[i];
    for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
      const int32_t j = Scol[q];
      const uint64_t w = Tw[j];
      const int32_t wi = Ti[j];
      if (tuple_gt(w, wi, bw, bi)) {
        bw = w;
        bi = wi;
      }
    }
    Tw2[i] = bw;
    Ti2[i] = bi;
  }
}

// the last max round (none for MIS(1)), then the decision of Alg. 2 for
// undecided nodes
// The block that finishes last stores the undecided count in the mapped pinned
// host word host_out, so the host reads it after the round's event without a copy.
__global__ void k_pmis_max2_decide(int32_t n, const int32_t *__restrict__ Sptr,
                                   const int32_t *__restrict__ Scol, const uint64_t *__restrict__ Tw,
                                   const int32_t *__restrict__ Ti, int8_t *__restrict__ s,
                                   int32_t *__restrict__ undecided, bool last_max, unsigned *__restrict__ ticket,
                                   volatile int32_t *host_out) {
  pdl_wait_and_trigger();
  int32_t local = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (s[i] != 0) continue;
    uint64_t bw = Tw[i];
    int32_t bi = Ti[i];
    if (last_max)
      for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
        const int32_t j = Scol[q];
        const uint64_t w = Tw[j];
        const int32_t wi = Ti[j];
        if (tuple_gt(w, wi, bw, bi)) {
          bw = w;
          bi = wi;
        }
      }
    if (bi == i)
      s[i] = 1;
    else if ((bw >> 62) == 2)
      s[i] = -1;
    else
      local++;
  }
  local = __reduce_add_sync(0xffffffffu, local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(undecided, local);
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *host_out = atomicAdd(undecided, 0);
    *ticket = 0;
    __threadfence_system();
  }
}

// ============================================================== aggregation
__device__ __forceinline__ bool root_gt(int32_t a, int32_t b, const uint64_t *key) {
  return key[a] > key[b] || (key[a] == key[b] && a > b);
}

// Every non-MIS node joins its nearest MIS node; ties between equally near
// roots go to the larger priority (v, i).  Pass 1: roots adjacent to i.
__global__ void k_agg_pass1(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const int8_t *__restrict__ s, const uint64_t *__restrict__ key,
                            int32_t *__restrict__ r1, int32_t *__restrict__ is_root) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    is_root[i] = (s[i] == 1);
    if (s[i] == 1) {
      r1[i] = i;
      continue;
    }
    int32_t best = -1;
    for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
      const int32_t j = Scol[q];
      if (s[j] == 1 && (best < 0 || root_gt(j, best, key))) best = j;
    }
    r1[i] = best;
  }
}

// Pass d = 2..k: nodes at distance d join through a neighbour assigned by
// pass d-1 (r1: after pass d-1, r2: after pass d).
__global__ void k_agg_pass2(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const int8_t *__restrict__ s, const uint64_t *__restrict__ key,
                            const int32_t *__restrict__ r1, int32_t *__restrict__ r2) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (r1[i] >= 0) {
      r2[i] = r1[i];
      continue;
    }
    int32_t best = -1;
    for (int32_t q = Sptr[i]; q < Sptr[i + 1]; ++q) {
      const int32_t j = Scol[q];
      if (s[j] != 1 && r1[j] >= 0) {
        const int32_t r = r1[j];
        if (best < 0 || root_gt(r, best, key)) best = r;
      }
    }
    r2[i] = best;
  }
}

__global__ void k_agg_final(int32_t n, const int32_t *__restrict__ r2, const int32_t *__restrict__ cid,
                            int32_t *__restrict__ agg, int *__restrict__ err) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r = r2[i];
  if (r < 0) {
    agg[i] = -1;
    atomicOr(err, 1);
  } else {
    agg[i] = cid[r];
  }
}

// members of each aggregate, sorted ascending (the summation order of Alg. 3
// and of the keyed sum)
__global__ void k_count_members(int32_t n, const int32_t *__restrict__ agg, int32_t *__restrict__ cnt) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);  // -1: unassigned, reported by the host
}
__global__ void k_fill_members(int32_t n, const int32_t *__restrict__ agg, const int32_t *__restrict__ aptr,
                               int32_t *__restrict__ cur, int32_t *__restrict__ amem) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) {
    const int32_t I = agg[i];
    amem[aptr[I] + atomicAdd(&cur[I], 1)] = i;
  }
}
__global__ void k_sort_members(int32_t nc, const int32_t *__restrict__ aptr, int32_t *__restrict__ amem) {
  pdl_wait_and_trigger();
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x)
    sort_segment(amem + aptr[I], aptr[I + 1] - aptr[I]);
}

// ============================================================== Alg. 3
// B_{k+1}(I) = ||B_k restricted to G_I||_2 (squares summed in ascending fine
// index), P(i, I) = B_k(i) / B_{k+1}(I).
__global__ void k_interp(int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
                         const double *__restrict__ B, double *__restrict__ Bc, double *__restrict__ pw) {
  pdl_wait_and_trigger();
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    const int32_t m0 = aptr[I], m1 = aptr[I + 1];
    double sum = 0.0;
    for (int32_t m = m0; m < m1; ++m) {
      const double b = B[amem[m]];
      const double t = __dmul_rn(b, b);
      sum = (m == m0) ? t : __dadd_rn(sum, t);
    }
    const double nrm = __dsqrt_rn(sum);
    Bc[I] = nrm;
    for (int32_t m = m0; m < m1; ++m) pw[amem[m]] = __ddiv_rn(B[amem[m]], nrm);
  }
}

// ============================================================== Sec. 3.1 keyed sum
// One warp per coarse row I.  The fine entries of the rows of G_I, taken in
// ascending fine row and CSR position, are the sorted run of keys (I, *) of
// the paper's stable sort.  The warp walks the distinct coarse columns J in
// ascending order; for each it sums P_iI * A_ij * P_jJ over the run in order,
// one term at a time, so every coarse value is the sequential sum.
constexpr int kGalWarps = 8;   // warps per block of k_galerkin
constexpr int32_t kGalCapMax = 4096;         // longest run staged by k_galerkin_smem
constexpr int32_t kGalCapFirst = 160;        // run cap of its first pass (three blocks an SM)
constexpr size_t kGalSmemBudget = 200 << 10;  // its dynamic shared memory per block
constexpr int kGalCap = 320;   // entries of one coarse row staged in shared memory

template <bool FILL>
__global__ void __launch_bounds__(kGalWarps * 32) k_galerkin(
    int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ val,
    const int32_t *__restrict__ agg, const double *__restrict__ pw, int32_t *__restrict__ ccount,
    const int32_t *__restrict__ crp, int32_t *__restrict__ cci, double *__restrict__ cval, bool marked_only) {
  pdl_wait_and_trigger();
  __shared__ int32_t sJ[kGalWarps][kGalCap];
  __shared__ int32_t sK[kGalWarps][kGalCap];  // distinct coarse columns of the run
  __shared__ double sV[FILL ? kGalWarps : 1][FILL ? kGalCap : 1];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  for (int32_t I = blockIdx.x * wpb + wid; I < nc; I += gridDim.x * wpb) {
    if (marked_only && ccount[I] != -1) continue;  // done by k_galerkin_smem
    const int32_t m0 = aptr[I], m1 = aptr[I + 1];
    // length of the run of keys (I, *): all entries of the member rows
    int32_t total = 0;
    for (int32_t m = m0 + lane; m < m1; m += 32) {
      const int32_t i = amem[m];
      total += rp[i + 1] - rp[i];
    }
    total = __reduce_add_sync(0xffffffffu, total);
    if (total <= kGalCap) {
      // stage (J, P_iI * A_ij * P_jJ) in run order: one lane per member row,
      // offsets from a warp prefix sum over the member rows
      int32_t base = 0;
      for (int32_t mb = m0; mb < m1; mb += 32) {
        const int32_t m = mb + lane;
        int32_t i = 0, p0 = 0, len = 0;
        if (m < m1) {
          i = amem[m];
          p0 = rp[i];
          len = rp[i + 1] - p0;
        }
        int32_t incl = len;
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int32_t off = base + incl - len;
        const double Pi = (m < m1) ? pw[i] : 0.0;
        for (int32_t q = 0; q < len; ++q) {
          const int32_t j = ci[p0 + q];
          sJ[wid][off + q] = agg[j];
          if (FILL) sV[wid][off + q] = __dmul_rn(__dmul_rn(Pi, val[p0 + q]), pw[j]);
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
      }
      __syncwarp();
      // distinct coarse columns of the run, in order of first occurrence
      int32_t d = 0;
      for (int32_t e0 = 0; e0 < total; e0 += 32) {
        const int32_t e = e0 + lane;
        bool first = false;
        int32_t J = 0;
        if (e < total) {
          J = sJ[wid][e];
          first = true;
          for (int32_t t = 0; t < e; ++t)
            if (sJ[wid][t] == J) {
              first = false;
              break;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, first);
        if (first) sK[wid][d + __popc(b & ((1u << lane) - 1u))] = J;
        d += __popc(b);
      }
      __syncwarp();
      // ascending order: the rank of a column is the number of smaller ones
      int32_t kk[kGalCap / 32], rk[kGalCap / 32];
#pragma unroll
      for (int t = 0; t < kGalCap / 32; ++t) {
        const int32_t q = lane + 32 * t;
        kk[t] = q < d ? sK[wid][q] : INT_MAX;
        rk[t] = 0;
        if (q < d)
          for (int32_t u = 0; u < d; ++u) rk[t] += sK[wid][u] < kk[t] ? 1 : 0;
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kGalCap / 32; ++t)
        if (lane + 32 * t < d) sK[wid][rk[t]] = kk[t];
      __syncwarp();
      // each lane sums its columns' terms in run order, starting from the first
      if (FILL) {
#pragma unroll
        for (int t = 0; t < kGalCap / 32; ++t) {
          const int32_t q = lane + 32 * t;
          if (32 * t >= d) break;
          if (q < d) {
            const int32_t J = sK[wid][q];
            double sum = 0.0;
            bool have = false;
            for (int32_t e = 0; e < total; ++e)
              if (sJ[wid][e] == J) {
                sum = have ? __dadd_rn(sum, sV[wid][e]) : sV[wid][e];
                have = true;
              }
            cci[crp[I] + q] = J;
            cval[crp[I] + q] = sum;
          }
        }
      }
      if (ccount && lane == 0) ccount[I] = d;
      __syncwarp();
      continue;
    }
    // long runs: the same walk reading the member rows from global memory
    int32_t cur = -1, out = 0;
    for (;;) {
      int32_t next = INT_MAX;
      double sum = 0.0;
      bool have = false;
      for (int32_t m = m0; m < m1; ++m) {
        const int32_t i = amem[m];
        const int32_t p0 = rp[i], p1 = rp[i + 1];
        const double Pi = pw[i];
        for (int32_t pb = p0; pb < p1; pb += 32) {
          const int32_t p = pb + lane;
          int32_t J = INT_MAX, j = 0;
          if (p < p1) {
            j = ci[p];
            J = agg[j];
          }
          if (J > cur && J < next) next = J;
          if (FILL) {
            unsigned mask = __ballot_sync(0xffffffffu, J == cur);
            double v = 0.0;
            if (J == cur) v = __dmul_rn(__dmul_rn(Pi, val[p]), pw[j]);
            while (mask) {
              const int src = __ffs(mask) - 1;
              const double t = __shfl_sync(0xffffffffu, v, src);
              sum = have ? __dadd_rn(sum, t) : t;
              have = true;
              mask &= mask - 1;
            }
          }
        }
      }
      next = __reduce_min_sync(0xffffffffu, next);
      if (cur >= 0) {
        if (FILL && lane == 0) {
          cci[crp[I] + out] = cur;
          cval[crp[I] + out] = sum;
        }
        out++;
      }
      if (next == INT_MAX) break;
      cur = next;
    }
    if (ccount && lane == 0) ccount[I] = out;
  }
}

// entries of the run of keys (I, *): the summed lengths of the member rows,
// an upper bound on the number of coarse nonzeros of row I
__global__ void k_run_length(int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
                             const int32_t *__restrict__ rp, int32_t *__restrict__ len, int32_t *__restrict__ maxlen) {
  pdl_wait_and_trigger();
  int32_t mx = 0;
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    int32_t t = 0;
    for (int32_t m = aptr[I]; m < aptr[I + 1]; ++m) t += rp[amem[m] + 1] - rp[amem[m]];
    len[I] = t;
    mx = max(mx, t);
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) atomicMax(maxlen, mx);
}

// Galerkin keyed sum (Sec. 3.1), one coarse row I per warp, its run staged in
// shared memory (at most `cap` entries; longer runs are marked ccount[I] = -1 and
// left to k_galerkin).  Per row:
//  1. stage (J, (P_iI * A_ij) * P_jJ) in run order, one lane per entry;
//  2. the distinct columns J through an open-addressing hash table, ranked
//     ascending by counting;
//  3. a stable counting scatter of the terms by column: chunks of 32 entries in
//     run order, lanes of equal column ordered by lane (__match_any_sync), so
//     every column's terms end up contiguous and in run order;
//  4. one lane per column adds its terms in that order, starting from the first:
//     the order of the sequential keyed sum, bit for bit.
// Output goes to the row's upper-bound slot crp[I]; ccount[I] = number of columns.
// marked_only: a second pass with a larger cap over the rows the first left.
__global__ void __launch_bounds__(256) k_galerkin_smem(
    int32_t nc, int32_t cap, int32_t hbits, bool marked_only, const int32_t *__restrict__ aptr,
    const int32_t *__restrict__ amem,
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ val,
    const int32_t *__restrict__ agg, const double *__restrict__ pw, int32_t *__restrict__ ccount,
    const int32_t *__restrict__ crp, int32_t *__restrict__ cci, double *__restrict__ cval,
    int32_t *__restrict__ gpos, int32_t *__restrict__ grow, int32_t *__restrict__ gseg) {
  pdl_wait_and_trigger();
  extern __shared__ __align__(16) unsigned char gal_sm[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int32_t hsize = 1 << hbits, hmask = hsize - 1;
  const unsigned lt = (1u << lane) - 1u;
  const size_t per = (size_t)cap * 40 + (size_t)hsize * 8;
  double *sV = reinterpret_cast<double *>(gal_sm + per * wid);  // staged terms
  double *sW = sV + cap;                                       // terms grouped by column
  int32_t *sJ = reinterpret_cast<int32_t *>(sW + cap);          // column of each term, then its rank
  int32_t *sKey = sJ + cap;                                     // distinct columns, table order
  int32_t *sCnt = sKey + cap;                                   // per rank: count, then segment end
  int32_t *sAux = sCnt + cap;                                   // member offsets, then sorted columns
  int32_t *sPos = sAux + cap;                                   // fine CSR position of each staged term
  int32_t *sMem = sPos + cap;                                   // member (run-local) of each staged term
  int32_t *hK = sMem + cap;
  int32_t *hR = hK + hsize;
  auto slot_of = [&](int32_t J) {
    uint32_t hh = ((uint32_t)J * 2654435761u) >> (32 - hbits);
    while (hK[hh] != J) hh = (hh + 1) & hmask;
    return hh;
  };
  for (int32_t I = blockIdx.x * wpb + wid; I < nc; I += gridDim.x * wpb) {
    if (marked_only && ccount[I] != -1) continue;
    const int32_t m0 = aptr[I], m1 = aptr[I + 1], nm = m1 - m0;
    // run offsets of the member rows (warp prefix sums over chunks of 32 members);
    // each member's row, first CSR position and weight go to shared memory
    // (sKey, sCnt and sW are free until step 2)
    int32_t total = 0;
    for (int32_t mb = m0; mb < m1; mb += 32) {
      const int32_t m = mb + lane;
      int32_t len = 0, i = 0, p0 = 0;
      double pwi = 0.0;
      if (m < m1) {
        i = amem[m];
        p0 = rp[i];
        pwi = pw[i];
        len = rp[i + 1] - p0;
      }
      int32_t incl = len;
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (m < m1 && m - m0 < cap) {
        if (total + incl - len < cap) sAux[m - m0] = total + incl - len;
        sKey[m - m0] = i;
        sCnt[m - m0] = p0;
        sW[m - m0] = pwi;
      }
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (total > cap || nm > cap) {
      if (lane == 0) ccount[I] = -1;  // left to the global-memory kernel
      continue;
    }
    __syncwarp();
    // 1. stage the terms in run order, one lane per entry; four entries a lane
    // per round, so that their loads are in flight together
    for (int32_t e0 = 0; e0 < total; e0 += 4 * 32) {
      int32_t ee[4], pp[4], ii[4], jj[4];
      double pwi[4], vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ee[u] = e0 + u * 32 + lane;
        if (ee[u] < total) {
          int32_t lo = 0, hi = nm - 1;
          while (lo < hi) {  // the member whose run segment holds the entry
            const int32_t mid = (lo + hi + 1) >> 1;
            if (sAux[mid] <= ee[u]) lo = mid; else hi = mid - 1;
          }
          ii[u] = sKey[lo];
          pp[u] = sCnt[lo] + (ee[u] - sAux[lo]);
          pwi[u] = sW[lo];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ee[u] < total) {
          jj[u] = ci[pp[u]];
          vv[u] = val[pp[u]];
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ee[u] < total) {
          const int32_t j = jj[u];
          sJ[ee[u]] = agg[j];
          sV[ee[u]] = __dmul_rn(__dmul_rn(pwi[u], vv[u]), pw[j]);
          sPos[ee[u]] = pp[u];
          sMem[ee[u]] = ii[u];
        }
    }
    for (int32_t t = lane; t < hsize; t += 32) hK[t] = -1;
    __syncwarp();
    // 2. distinct columns: hash insertion, compaction, ranks by counting
    for (int32_t e = lane; e < total; e += 32) {
      const int32_t J = sJ[e];
      uint32_t hh = ((uint32_t)J * 2654435761u) >> (32 - hbits);
      for (;;) {
        const int32_t prev = atomicCAS(&hK[hh], -1, J);
        if (prev == -1 || prev == J) break;
        hh = (hh + 1) & hmask;
      }
    }
    __syncwarp();
    int32_t d = 0;
    for (int32_t t0 = 0; t0 < hsize; t0 += 32) {
      const int32_t k = hK[t0 + lane];
      const unsigned b = __ballot_sync(0xffffffffu, k != -1);
      if (k != -1) sKey[d + __popc(b & lt)] = k;
      d += __popc(b);
    }
    __syncwarp();
    for (int32_t q = lane; q < d; q += 32) {
      const int32_t K = sKey[q];
      int32_t r = 0;
      for (int32_t u = 0; u < d; ++u) r += sKey[u] < K ? 1 : 0;
      hR[slot_of(K)] = r;
      sAux[r] = K;  // sorted columns (the member offsets are no longer needed)
      sCnt[q] = 0;
    }
    __syncwarp();
    // 3. counts per column in run order, then segment starts, then the stable scatter
    for (int32_t e0 = 0; e0 < total; e0 += 32) {
      const int32_t e = e0 + lane;
      const int32_t r = e < total ? hR[slot_of(sJ[e])] : -1;
      if (e < total) sJ[e] = r;
      const unsigned grp = __match_any_sync(0xffffffffu, r);
      if (r >= 0 && (grp & lt) == 0) sCnt[r] += __popc(grp);
      __syncwarp();
    }
    {  // exclusive prefix over the d counts
      int32_t run = 0;
      for (int32_t q0 = 0; q0 < d; q0 += 32) {
        const int32_t q = q0 + lane;
        const int32_t c = q < d ? sCnt[q] : 0;
        int32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (q < d) sCnt[q] = run + incl - c;
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncwarp();
    for (int32_t e0 = 0; e0 < total; e0 += 32) {
      const int32_t e = e0 + lane;
      const int32_t r = e < total ? sJ[e] : -1;
      const unsigned grp = __match_any_sync(0xffffffffu, r);
      if (r >= 0) {
        const int32_t t = sCnt[r] + __popc(grp & lt);
        sW[t] = sV[e];
        if (gpos) {  // the summation plan: term t of the row's run, in sorted order
          gpos[crp[I] + t] = sPos[e];
          grow[crp[I] + t] = sMem[e];
        }
      }
      __syncwarp();
      if (r >= 0 && (grp & lt) == 0) sCnt[r] += __popc(grp);
      __syncwarp();
    }
    // 4. one lane per column: its terms in run order (sCnt[r] is now its segment end)
    for (int32_t q = lane; q < d; q += 32) {
      const int32_t a = q == 0 ? 0 : sCnt[q - 1], b = sCnt[q];
      double sum = sW[a];
      for (int32_t t = a + 1; t < b; ++t) sum = __dadd_rn(sum, sW[t]);
      cci[crp[I] + q] = sAux[q];
      cval[crp[I] + q] = sum;
      if (gseg) gseg[crp[I] + q] = crp[I] + a;  // first term of this coarse entry in the plan
    }
    if (lane == 0) ccount[I] = d;
    __syncwarp();
  }
}

// copy row I from its upper-bound slot to the compact coarse CSR
__global__ void k_compact_rows(int32_t nc, const int32_t *__restrict__ ub, const int32_t *__restrict__ crp,
                               const int32_t *__restrict__ tci, const double *__restrict__ tval,
                               int32_t *__restrict__ cci, double *__restrict__ cval) {
  pdl_wait_and_trigger();
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    const int32_t len = crp[I + 1] - crp[I];
    for (int32_t t = 0; t < len; ++t) {
      cci[crp[I] + t] = tci[ub[I] + t];
      cval[crp[I] + t] = tval[ub[I] + t];
    }
  }
}

// plan: segment start of row I's coarse entries, from upper-bound slots to
// compact positions; gptr[cnnz] = number of fine nonzeros
__global__ void k_compact_plan(int32_t nc, const int32_t *__restrict__ ub, const int32_t *__restrict__ crp,
                               const int32_t *__restrict__ tseg, int32_t *__restrict__ gptr, int32_t nnz_fine) {
  pdl_wait_and_trigger();
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    const int32_t len = crp[I + 1] - crp[I];
    for (int32_t t = 0; t < len; ++t) gptr[crp[I] + t] = tseg[ub[I] + t];
    if (I == nc - 1) gptr[crp[nc]] = nnz_fine;
  }
}

// values-only Galerkin product from the plan: the same terms in the same order
// as the full product, so the coarse values are bit-identical to a full setup
// that finds the same aggregates
__global__ void k_galerkin_values(int32_t cnnz, const int32_t *__restrict__ gptr, const int32_t *__restrict__ gpos,
                                  const int32_t *__restrict__ grow, const int32_t *__restrict__ ci,
                                  const double *__restrict__ val, const double *__restrict__ pw,
                                  double *__restrict__ cval) {
  pdl_wait_and_trigger();
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cnnz; q += gridDim.x * blockDim.x) {
    const int32_t a = gptr[q], b = gptr[q + 1];
    double sum = 0.0;
    for (int32_t t = a; t < b; ++t) {
      const int32_t pp = gpos[t];
      const double term = __dmul_rn(__dmul_rn(pw[grow[t]], val[pp]), pw[ci[pp]]);
      sum = t == a ? term : __dadd_rn(sum, term);
    }
    cval[q] = sum;
  }
}

// ============================================================== solve-phase data
__global__ void k_diag(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ val, double *__restrict__ diag) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) d = val[p];
  diag[i] = d;
}

// SELL-32: width of each slice = its longest row (off-diagonal entries only when
// split), rounded up to even for the pair layout of FP32 values
__global__ void k_slice_width(int32_t n, int32_t nslices, const int32_t *__restrict__ rp,
                              const int32_t *__restrict__ ci, bool split, bool pairs,
                              int64_t *__restrict__ width32) {
  pdl_wait_and_trigger();
  const int lane = threadIdx.x & 31;
  const int32_t sl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (sl >= nslices) return;
  const int32_t row = sl * kSlice + lane;
  int32_t len = 0;
  if (row < n)
    for (int32_t p = rp[row]; p < rp[row + 1]; ++p) len += (split && ci[p] == row) ? 0 : 1;
  len = __reduce_max_sync(0xffffffffu, len);
  if (pairs) len = (len + 1) & ~1;
  if (lane == 0) width32[sl] = (int64_t)len * kSlice;
}

template <class MV>
__device__ __forceinline__ MV conv_val(double v);
template <> __device__ __forceinline__ double conv_val<double>(double v) { return v; }
template <> __device__ __forceinline__ float conv_val<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 conv_val<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}

template <class MV> __device__ __forceinline__ double back_to_double(MV v);
template <> __device__ __forceinline__ double back_to_double<double>(double v) { return v; }
template <> __device__ __forceinline__ double back_to_double<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double back_to_double<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

// CSR -> SELL-32 (column-major within a slice; padding: own row, value 0).
// split: skip the diagonal entry and store sdiag[i] = a_ii + sum_j (a_ij - fl(a_ij))
// over the row's off-diagonals, in FP64 then rounded once to FP32.
// spair (FP32 values only): the entries go to the pair layout instead of scol /
// sval, entry e of the lane as half (e & 1) of int4 sptr[sl] / 2 + 32 (e / 2) + lane.
// BF16 values: entry e of the lane at sptr[sl] + 64 (e / 2) + 2 lane + (e & 1) of
// scol / sval (slice widths even).
template <class MV>
__global__ void k_build_sell(int32_t n, int32_t nslices, const int32_t *__restrict__ rp,
                             const int32_t *__restrict__ ci, const double *__restrict__ val,
                             const int64_t *__restrict__ sptr, int32_t *__restrict__ scol, MV *__restrict__ sval,
                             int4 *__restrict__ spair, float *__restrict__ sdiag) {
  pdl_wait_and_trigger();
  const int lane = threadIdx.x & 31;
  const int32_t sl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (sl >= nslices) return;
  const int32_t row = sl * kSlice + lane;
  const int64_t base = sptr[sl];
  const int32_t width = (int32_t)((sptr[sl + 1] - base) / kSlice);
  const int32_t pad_col = row < n ? row : n - 1;
  auto put = [&](int32_t e, int32_t c, MV m) {
    if constexpr (std::is_same<MV, float>::value) {
      if (spair) {
        int32_t *w = reinterpret_cast<int32_t *>(spair + (base >> 1) + (int64_t)(e >> 1) * kSlice + lane) + 2 * (e & 1);
        w[0] = c;
        w[1] = __float_as_int(m);
        return;
      }
    }
    // BF16: a lane's entries 2j and 2j+1 adjacent in both arrays
    const int64_t at = std::is_same<MV, __nv_bfloat16>::value
                           ? base + (int64_t)(e >> 1) * (2 * kSlice) + 2 * lane + (e & 1)
                           : base + (int64_t)e * kSlice + lane;
    scol[at] = c;
    sval[at] = m;
  };
  int32_t e = 0;
  double dii = 0.0, comp = 0.0;
  if (row < n)
    for (int32_t p = rp[row]; p < rp[row + 1]; ++p) {
      const int32_t c = ci[p];
      const double v = val[p];
      if (sdiag && c == row) {
        dii = v;
        continue;
      }
      const MV m = conv_val<MV>(v);
      put(e, c, m);
      if (sdiag) comp = __dadd_rn(comp, __dadd_rn(v, -back_to_double<MV>(m)));
      ++e;
    }
  for (; e < width; ++e) put(e, pad_col, conv_val<MV>(0.0));
  if (sdiag && row < n) sdiag[row] = __double2float_rn(__dadd_rn(dii, comp));
}

// ============================================================== Arnoldi omega
// ---- Arnoldi on M = |D|^-1/2 A |D|^-1/2 with three kernels per step --------
// Every kernel ends with a last-block reduction: blocks publish their partial
// sums, take a ticket, and the block that finishes last sums the partials of
// all blocks in block order (deterministic) and writes the scalars.
constexpr int kArnSlots = 8;
constexpr int kArnoldiMax = 5;  // Arnoldi steps (m <= 5, Eq. damped Jacobi)

__device__ __forceinline__ bool arn_last_block(unsigned *ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// block partials of up to kArnSlots sums -> part[slot * gridDim.x + block]
__device__ __forceinline__ void arn_block_partials(const double (&v)[kArnSlots], int ns, double *part) {
  __shared__ double sh[kArnSlots][8];
#pragma unroll
  for (int k = 0; k < kArnSlots; ++k) {
    if (k < ns) {
      const double w = warp_sum(v[k]);
      if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = w;
    }
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)ns) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sh[threadIdx.x][q];
    part[threadIdx.x * gridDim.x + blockIdx.x] = a;
  }
}

// sums of slots 0..ns-1 over all blocks, computed by the last block in a fixed
// order: warp k takes slot k (ns <= kArnSlots = the block's warps), lane l the
// blocks l, l + 32, ... in four interleaved partial sums, then a fixed tree
__device__ void arn_totals(const double *part, int ns, double *out_sh) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k < ns) {
    const double *pk = part + (size_t)k * gridDim.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned b = lane;
    for (; b + 96 < gridDim.x; b += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] += __ldcg(pk + b + 32 * u);
    }
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (b + 32 * u < gridDim.x) a[u] += __ldcg(pk + b + 32 * u);
    const double t = warp_sum((a[0] + a[1]) + (a[2] + a[3]));
    if (lane == 0) out_sh[k] = t;
  }
  __syncthreads();
}

// The products gather U = dh .* W, the unnormalised basis vector scaled by
// |D|^-1/2, so that an entry costs one FP64 fused multiply-add: the FP64 pipe
// of the part, not HBM, bounds three operations an entry.
//
// start: W = random start vector in [-1, 1), dh = |A_ii|^-1/2, U = dh .* W;
// nrm2 = ||W||^2
__global__ void __launch_bounds__(256) k_arn_start(int32_t n, uint64_t seed, int32_t level,
                                                   const double *__restrict__ diag, double *__restrict__ W,
                                                   double *__restrict__ U, double *__restrict__ dh, double *part,
                                                   double *nrm2, unsigned *ticket) {
  pdl_wait_and_trigger();
  double v[kArnSlots] = {0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t z = splitmix64(~seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)(uint32_t)i);
    const double q = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    const double di = rsqrt(fabs(diag[i]));  // a few ulp from 1 / sqrt, in fewer FP64 operations
    W[i] = q;
    dh[i] = di;
    U[i] = di * q;
    v[0] += q * q;
  }
  arn_block_partials(v, 1, part);
  if (arn_last_block(ticket)) {
    __shared__ double tot[kArnSlots];
    arn_totals(part, 1, tot);
    if (threadIdx.x == 0) {
      *nrm2 = tot[0];
      *ticket = 0;
    }
  }
}

// The inner products of step j after w = M q_j.  Arnoldi (nonsymmetric A):
// h_lj = q_l . w for l <= j, and ||w||^2.  Lanczos (symmetric A, where the
// Arnoldi matrix is tridiagonal and the recurrence needs only q_j and q_{j-1}):
// alpha_j = q_j . w and ||w||^2.
template <bool LZ>
__device__ __forceinline__ void arn_accumulate(double (&v)[kArnSlots], int j, int32_t n, int32_t i,
                                               const double *__restrict__ Q, double qi, double wi) {
  if constexpr (LZ) {
    v[0] += qi * wi;
    v[1] += wi * wi;
  } else {
#pragma unroll
    for (int l = 0; l < kArnSlots; ++l) {  // static indices: the sums stay in registers
      if (l < j) v[l] += Q[(size_t)l * n + i] * wi;
      else if (l == j) v[l] += qi * wi;
      else if (l == j + 1) v[l] += wi * wi;
    }
  }
}

// Block partials and, in the last block, the column j of H: Arnoldi h_lj
// (l <= j) and h_{j,j-1} = ||W|| = h; Lanczos alpha_j on the diagonal and
// beta_{j-1} = h on both sides of it.  wn_j = ||M q_j|| for the breakdown test.
template <bool LZ>
__device__ __forceinline__ void arn_finish(const double (&v)[kArnSlots], int j, double h, double *part, double *H,
                                           double *wn, unsigned *ticket) {
  const int ns = LZ ? 2 : j + 2;
  arn_block_partials(v, ns, part);
  if (arn_last_block(ticket)) {
    __shared__ double tot[kArnSlots];
    arn_totals(part, ns, tot);
    if (LZ) {
      if (threadIdx.x == 0) {
        H[j * 8 + j] = tot[0];
        wn[j] = sqrt(tot[1]);
        if (j > 0) H[j * 8 + (j - 1)] = H[(j - 1) * 8 + j] = h;
      }
    } else {
      if ((int)threadIdx.x <= j) H[threadIdx.x * 8 + j] = tot[threadIdx.x];
      if ((int)threadIdx.x == j + 1) wn[j] = sqrt(tot[j + 1]);
      if (threadIdx.x == 0 && j > 0) H[j * 8 + (j - 1)] = h;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// Lanczos step j, part 2: w -= alpha_j q_j + beta_{j-1} q_{j-1}; W = w,
// U = dh .* w, nrm2 = ||w||^2 (beta_j^2)
__global__ void __launch_bounds__(256) k_lz_update(int32_t n, int j, const double *__restrict__ Q,
                                                   const double *__restrict__ w, double *__restrict__ W,
                                                   double *__restrict__ U, const double *__restrict__ dh,
                                                   double *part, const double *__restrict__ H, double *nrm2,
                                                   unsigned *ticket) {
  pdl_wait_and_trigger();
  const double a = H[j * 8 + j], b = j > 0 ? H[j * 8 + (j - 1)] : 0.0;
  const double *qj = Q + (size_t)j * n, *qp = j > 0 ? Q + (size_t)(j - 1) * n : nullptr;
  double v[kArnSlots] = {0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double wi = w[i] - a * qj[i];
    if (qp) wi -= b * qp[i];
    W[i] = wi;
    U[i] = dh[i] * wi;
    v[0] += wi * wi;
  }
  arn_block_partials(v, 1, part);
  if (arn_last_block(ticket)) {
    __shared__ double tot[kArnSlots];
    arn_totals(part, 1, tot);
    if (threadIdx.x == 0) {
      *nrm2 = tot[0];
      *ticket = 0;
    }
  }
}

// step j, part 1: q_j = W / ||W||; w = M q_j = dh .* (A U) / ||W||;
// h_lj = q_l . w (l <= j), wn_j = ||w||; h_{j,j-1} = ||W|| (j > 0).
// T consecutive lanes share a row: lane t sums the row's entries t, t + T, ...
// and the T partial sums meet in a fixed shuffle tree, so that the entries of a
// row are read by neighbouring lanes.
template <int T, bool LZ>
__global__ void __launch_bounds__(256) k_arn_spmv(int32_t n, int j, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ ci, const double *__restrict__ val,
                                                  const double *__restrict__ dh, const double *__restrict__ W,
                                                  const double *__restrict__ U, double *__restrict__ Q,
                                                  double *__restrict__ w, double *part, const double *nrm2, double *H,
                                                  double *wn, unsigned *ticket) {
  pdl_wait_and_trigger();
  const double h = sqrt(*nrm2), sc = 1.0 / h;
  double *qj = Q + (size_t)j * n;
  const int t = threadIdx.x % T;
  double v[kArnSlots] = {0.0};
  const int32_t groups = (int32_t)(gridDim.x * blockDim.x / T);
  const int32_t g0 = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) / T);
  const int32_t rounds = (n + groups - 1) / groups;  // every lane of a group runs the same rounds
  for (int32_t r = 0; r < rounds; ++r) {
    const int32_t i = g0 + r * groups;
    double acc = 0.0;
    if (i < n) {
      const int32_t p1 = rp[i + 1];
      for (int32_t p = rp[i] + t; p < p1; p += 4 * T) {
        int32_t c[4];
        double a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (p + u * T < p1) {
            c[u] = __ldcs(ci + p + u * T);
            a[u] = __ldcs(val + p + u * T);
          }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (p + u * T < p1) acc += a[u] * U[c[u]];
      }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, T);
    if (i < n && t == 0) {
      const double wi = dh[i] * (sc * acc), qi = sc * W[i];
      qj[i] = qi;
      w[i] = wi;
      arn_accumulate<LZ>(v, j, n, i, Q, qi, wi);
    }
  }
  arn_finish<LZ>(v, j, h, part, H, wn, ticket);
}

// step j, part 1 on a level with an FP64 SELL-32 copy of A (one warp per slice,
// coalesced loads; the same sums in the same order as the CSR kernel above plus
// zero terms of the padding)
template <bool LZ>
__global__ void __launch_bounds__(256) k_arn_spmv_sell(int32_t n, int32_t nslices, int j,
                                                       const int64_t *__restrict__ sptr, const int32_t *__restrict__ scol,
                                                       const double *__restrict__ sval, const double *__restrict__ dh,
                                                       const double *__restrict__ W, const double *__restrict__ U,
                                                       double *__restrict__ Q,
                                                       double *__restrict__ w, double *part, const double *nrm2,
                                                       double *H, double *wn, unsigned *ticket) {
  pdl_wait_and_trigger();
  const double h = sqrt(*nrm2), sc = 1.0 / h;
  double *qj = Q + (size_t)j * n;
  const int lane = threadIdx.x & 31;
  double v[kArnSlots] = {0.0};
  for (int32_t sl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < nslices;
       sl += gridDim.x * (blockDim.x >> 5)) {
    const int64_t base = sptr[sl];
    const int32_t width = (int32_t)((sptr[sl + 1] - base) >> 5);
    double acc = 0.0;
    for (int32_t e = 0; e < width; e += 8) {  // eight entries' loads in flight, summed in order
      int32_t c[8];
      double a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < width) {
          const int64_t at = base + 32 * (int64_t)(e + u) + lane;
          c[u] = __ldcs(scol + at);
          a[u] = __ldcs(sval + at);
        }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < width) acc += a[u] * U[c[u]];
    }
    const int32_t i = sl * 32 + lane;
    if (i < n) {
      const double wi = dh[i] * (sc * acc), qi = sc * W[i];
      qj[i] = qi;
      w[i] = wi;
      arn_accumulate<LZ>(v, j, n, i, Q, qi, wi);
    }
  }
  arn_finish<LZ>(v, j, h, part, H, wn, ticket);
}

// step j, parts 2 and 3 (classical Gram-Schmidt twice): w -= sum_l c_l q_l with
// c = H[.][j] (pass 0) or the correction corr (pass 1).  Pass 0 ends with
// corr_l = q_l . w; pass 1 adds corr to H[.][j], writes W = w, U = dh .* w and
// nrm2 = ||w||^2.
__global__ void __launch_bounds__(256) k_arn_orth(int32_t n, int j, int pass, const double *__restrict__ Q,
                                                  double *__restrict__ w, double *__restrict__ W,
                                                  double *__restrict__ U, const double *__restrict__ dh,
                                                  double *part, double *H, double *corr, double *nrm2,
                                                  unsigned *ticket) {
  pdl_wait_and_trigger();
  double c[kArnoldiMax];
#pragma unroll
  for (int l = 0; l < kArnoldiMax; ++l) c[l] = l <= j ? (pass == 0 ? H[l * 8 + j] : corr[l]) : 0.0;
  double v[kArnSlots] = {0.0};
  // two rows per thread and round (i, i + stride), their loads issued together;
  // each thread still takes its rows in increasing order
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const int32_t i2 = i + stride;
    const bool two = i2 < n;
    double q1[kArnoldiMax], q2[kArnoldiMax];
    double wi = w[i], wi2 = two ? w[i2] : 0.0;
#pragma unroll
    for (int l = 0; l < kArnoldiMax; ++l)
      if (l <= j) {
        q1[l] = Q[(size_t)l * n + i];
        q2[l] = two ? Q[(size_t)l * n + i2] : 0.0;
      }
#pragma unroll
    for (int l = 0; l < kArnoldiMax; ++l)
      if (l <= j) {
        wi -= c[l] * q1[l];
        wi2 -= c[l] * q2[l];
      }
    if (pass == 0) {
      w[i] = wi;
      if (two) w[i2] = wi2;
#pragma unroll
      for (int l = 0; l < kArnoldiMax; ++l)
        if (l <= j) {
          v[l] += q1[l] * wi;
          if (two) v[l] += q2[l] * wi2;
        }
    } else {
      W[i] = wi;
      U[i] = dh[i] * wi;
      v[0] += wi * wi;
      if (two) {
        W[i2] = wi2;
        U[i2] = dh[i2] * wi2;
        v[0] += wi2 * wi2;
      }
    }
  }
  const int ns = pass == 0 ? j + 1 : 1;
  arn_block_partials(v, ns, part);
  if (arn_last_block(ticket)) {
    __shared__ double tot[kArnSlots];
    arn_totals(part, ns, tot);
    if (pass == 0) {
      if ((int)threadIdx.x <= j) corr[threadIdx.x] = tot[threadIdx.x];
    } else {
      if ((int)threadIdx.x <= j) H[threadIdx.x * 8 + j] += corr[threadIdx.x];
      if (threadIdx.x == 0) *nrm2 = tot[0];
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// Largest |eigenvalue| of a small symmetric matrix by bisection on the inertia
// of T - sigma I (Sylvester's law: the number of negative pivots of Gaussian
// elimination without pivoting equals the number of eigenvalues below sigma).

// fully unrolled over the 5 x 5 bound so that the matrix stays in registers;
// rows and columns beyond m act as an identity block (no negative pivots)
__device__ int count_below(const double (&T)[kArnoldiMax][kArnoldiMax], int m, double sigma) {
  double a[kArnoldiMax][kArnoldiMax];
#pragma unroll
  for (int r = 0; r < kArnoldiMax; ++r)
#pragma unroll
    for (int c = 0; c < kArnoldiMax; ++c)
      a[r][c] = (r < m && c < m) ? T[r][c] - (r == c ? sigma : 0.0) : (r == c ? 1.0 : 0.0);
  int neg = 0;
#pragma unroll
  for (int k = 0; k < kArnoldiMax; ++k) {
    double piv = a[k][k];
    if (piv == 0.0) piv = 1e-300;  // sigma sits on an eigenvalue of a leading block
    if (piv < 0.0) neg++;
    const double inv = 1.0 / piv;
#pragma unroll
    for (int r = k + 1; r < kArnoldiMax; ++r) {
      const double f = a[r][k] * inv;
#pragma unroll
      for (int c = k + 1; c < kArnoldiMax; ++c) a[r][c] -= f * a[k][c];
    }
  }
  return neg;
}

// H: (m+1) x 8 Hessenberg from the Arnoldi loop, wn[j] = ||M q_j||.  Applies
// the breakdown rule (h_{j+1,j} <= 1e-12 ||M q_j|| ends the process after j+1
// steps), symmetrises the leading block and sets omega = (4/3)/rho.  One warp:
// multisection, every lane tests one of 32 points of the current interval, so
// each round narrows it 33-fold (12 rounds reach double precision).
// ---- eigenvalues of a small nonsymmetric Hessenberg matrix ---------------
// complex arithmetic written from the definitions
struct cx {
  double re, im;
};
__device__ __forceinline__ cx c_add(cx a, cx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cx c_sub(cx a, cx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cx c_mul(cx a, cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cx c_conj(cx a) { return {a.re, -a.im}; }
__device__ __forceinline__ double c_abs(cx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ cx c_scale(cx a, double f) { return {a.re * f, a.im * f}; }
// principal square root: with r = |z|, sqrt(z) = s + i im/(2 s), s = sqrt((r + re)/2)
// (re >= 0); else |im|/(2 s) + i sign(im) s with s = sqrt((r - re)/2)
__device__ cx c_sqrt(cx z) {
  const double r = c_abs(z);
  if (r == 0.0) return {0.0, 0.0};
  if (z.re >= 0.0) {
    const double sq = sqrt(0.5 * (r + z.re));
    return {sq, z.im / (2.0 * sq)};
  }
  const double sq = sqrt(0.5 * (r - z.re));
  return {fabs(z.im) / (2.0 * sq), copysign(sq, z.im)};
}

// largest |eigenvalue| of the leading m x m block of H (row stride 8) by the
// shifted QR algorithm in complex arithmetic: H - mu I = Q R by Givens rotations,
// H <- R Q + mu I, Wilkinson shift from the trailing 2 x 2 block, deflation once
// |h_{n,n-1}| <= 1e-14 (|h_nn| + |h_{n-1,n-1}|) or after 200 steps
__device__ double hess_rho(int m, const double *H) {
  cx a[kArnoldiMax][kArnoldiMax];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) a[i][j] = {H[i * 8 + j], 0.0};
  double rho = 0.0;
  int n = m, iter = 0;
  while (n > 0) {
    if (n == 1) {
      rho = fmax(rho, c_abs(a[0][0]));
      break;
    }
    const double sc = c_abs(a[n - 1][n - 1]) + c_abs(a[n - 2][n - 2]);
    if (c_abs(a[n - 1][n - 2]) <= 1e-14 * sc || iter >= 200) {
      rho = fmax(rho, c_abs(a[n - 1][n - 1]));
      --n;
      iter = 0;
      continue;
    }
    const cx p = a[n - 2][n - 2], q = a[n - 2][n - 1], r = a[n - 1][n - 2], t = a[n - 1][n - 1];
    const cx half = c_scale(c_add(p, t), 0.5);
    const cx disc = c_sqrt(c_sub(c_mul(half, half), c_sub(c_mul(p, t), c_mul(q, r))));
    const cx l1 = c_add(half, disc), l2 = c_sub(half, disc);
    const cx mu = c_abs(c_sub(l1, t)) < c_abs(c_sub(l2, t)) ? l1 : l2;
    cx cs[kArnoldiMax], sn[kArnoldiMax];
    for (int i = 0; i < n; ++i) a[i][i] = c_sub(a[i][i], mu);
    for (int k = 0; k + 1 < n; ++k) {
      const cx x = a[k][k], y = a[k + 1][k];
      const double nrm = sqrt(c_abs(x) * c_abs(x) + c_abs(y) * c_abs(y));
      cs[k] = nrm > 0.0 ? cx{x.re / nrm, x.im / nrm} : cx{1.0, 0.0};
      sn[k] = nrm > 0.0 ? cx{y.re / nrm, y.im / nrm} : cx{0.0, 0.0};
      for (int j = k; j < n; ++j) {
        const cx u = a[k][j], v = a[k + 1][j];
        a[k][j] = c_add(c_mul(c_conj(cs[k]), u), c_mul(c_conj(sn[k]), v));
        a[k + 1][j] = c_add(c_mul(cx{-sn[k].re, -sn[k].im}, u), c_mul(cs[k], v));
      }
    }
    for (int k = 0; k + 1 < n; ++k)
      for (int i = 0; i <= k + 1; ++i) {
        const cx u = a[i][k], v = a[i][k + 1];
        a[i][k] = c_add(c_mul(u, cs[k]), c_mul(v, sn[k]));
        a[i][k + 1] = c_add(c_mul(cx{-u.re, -u.im}, c_conj(sn[k])), c_mul(v, c_conj(cs[k])));
      }
    for (int i = 0; i < n; ++i) a[i][i] = c_add(a[i][i], mu);
    ++iter;
  }
  return rho;
}

// One warp per level (block q: level q), so that the levels' small eigenvalue
// problems (FP64, a slow pipe on this part) run side by side in one launch.
struct OmegaJobs {
  const double *H[kMaxLevels];
  const double *wn[kMaxLevels];
  double *out[kMaxLevels];
  int m[kMaxLevels];
};

__global__ void k_omega_from_H(OmegaJobs jobs, int symmetric) {
  pdl_wait_and_trigger();
  if (threadIdx.x >= 32) return;
  const double *__restrict__ H = jobs.H[blockIdx.x];
  const double *__restrict__ wn = jobs.wn[blockIdx.x];
  double *__restrict__ omega_out = jobs.out[blockIdx.x];
  const int m = jobs.m[blockIdx.x];
  const int lane = threadIdx.x;
  int mm = m;
  for (int j = 0; j < m; ++j)
    if (H[(j + 1) * 8 + j] <= 1e-12 * wn[j] || j + 1 == m) {
      mm = j + 1;
      break;
    }
  if (!symmetric) {  // rho from the eigenvalues of the Hessenberg matrix itself
    if (lane == 0) *omega_out = (4.0 / 3.0) / hess_rho(mm, H);
    return;
  }
  double T[kArnoldiMax][kArnoldiMax];
  double g = 0.0;
#pragma unroll
  for (int a = 0; a < kArnoldiMax; ++a) {
    double rs = 0.0;
#pragma unroll
    for (int b = 0; b < kArnoldiMax; ++b) {
      T[a][b] = (a < mm && b < mm) ? 0.5 * (H[a * 8 + b] + H[b * 8 + a]) : 0.0;
      rs += fabs(T[a][b]);
    }
    g = fmax(g, rs);
  }
  g = g * (1.0 + 1e-12) + 1e-300;
  double ext[2] = {0.0, 0.0};
  // no eigenvalue below 0 (the usual case: M is positive definite): rho is the
  // largest eigenvalue and the smallest one need not be located
  const int nsides = count_below(T, mm, 0.0) == 0 ? 1 : 2;
  for (int side = 0; side < nsides; ++side) {
    // side 0: largest eigenvalue = sup{sigma : count_below(sigma) < mm}
    // side 1: smallest eigenvalue = sup{sigma : count_below(sigma) == 0}
    double lo = -g, hi = g;
    for (int it = 0; it < 40; ++it) {
      const double sig = lo + (hi - lo) * (double)(lane + 1) / 33.0;
      const int c = count_below(T, mm, sig);
      const bool below = side == 0 ? (c < mm) : (c == 0);
      // predicate is monotone in sigma: lanes 0..k-1 true, the rest false
      const unsigned bal = __ballot_sync(0xffffffffu, below);
      const int k = __popc(bal);
      const double nlo = k > 0 ? __shfl_sync(0xffffffffu, sig, k - 1) : lo;
      const double nhi = k < 32 ? __shfl_sync(0xffffffffu, sig, k < 32 ? k : 31) : hi;
      if (nlo == lo && nhi == hi) break;
      lo = nlo;
      hi = nhi;
      if (hi - lo <= 1e-16 * fmax(fabs(lo), fabs(hi))) break;
    }
    ext[side] = 0.5 * (lo + hi);
  }
  const double rho = fmax(fabs(ext[0]), fabs(ext[1]));
  if (lane == 0) *omega_out = (4.0 / 3.0) / rho;
}

// ============================================================== coarsest level
// Gauss-Jordan inverse with partial pivoting (the largest |a_ij| on or below the
// diagonal, the first index on ties) of a nonsymmetric n x n matrix, one block:
// A (destroyed) -> Ainv.  fac: n doubles of scratch.
__global__ void k_lu_inverse(int32_t n, double *__restrict__ A, double *__restrict__ Ainv, double *__restrict__ fac,
                             int *__restrict__ err) {
  pdl_wait_and_trigger();
  __shared__ double bv_s[32];
  __shared__ int bi_s[32];
  __shared__ int piv;
  __shared__ double pinv;
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) Ainv[t] = (t / n == t % n) ? 1.0 : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t j = 0; j < n; ++j) {
    double bv = -1.0;
    int bi = n;
    for (int32_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      const double v = fabs(A[(int64_t)i * n + j]);
      if (v > bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      bv_s[wid] = bv;
      bi_s[wid] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = bv_s[0];
      int i0 = bi_s[0];
      for (int q = 1; q < nw; ++q)
        if (bv_s[q] > v || (bv_s[q] == v && bi_s[q] < i0)) {
          v = bv_s[q];
          i0 = bi_s[q];
        }
      piv = i0;
      if (!(v > 0.0)) *err = 1;
    }
    __syncthreads();
    if (*err) return;
    const int32_t pr = piv;
    if (pr != j)
      for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        double t = A[(int64_t)j * n + k];
        A[(int64_t)j * n + k] = A[(int64_t)pr * n + k];
        A[(int64_t)pr * n + k] = t;
        t = Ainv[(int64_t)j * n + k];
        Ainv[(int64_t)j * n + k] = Ainv[(int64_t)pr * n + k];
        Ainv[(int64_t)pr * n + k] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) pinv = 1.0 / A[(int64_t)j * n + j];
    __syncthreads();
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
      A[(int64_t)j * n + k] *= pinv;
      Ainv[(int64_t)j * n + k] *= pinv;
    }
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) fac[i] = i == j ? 0.0 : A[(int64_t)i * n + j];
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
      const int32_t i = (int32_t)(t / n), k = (int32_t)(t % n);
      if (i == j) continue;
      A[t] -= fac[i] * A[(int64_t)j * n + k];
      Ainv[t] -= fac[i] * Ainv[(int64_t)j * n + k];
    }
    __syncthreads();
  }
}

__global__ void k_dense_from_csr(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const double *__restrict__ val, double *__restrict__ A) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t p = rp[i]; p < rp[i + 1]; ++p) A[(int64_t)i * n + ci[p]] = val[p];
}

// In-place dense Cholesky (lower) by one thread block, then the inverse
// A^-1 = L^-T L^-1 column by column (one thread per column): the blocks of a
// batch larger than the shared-memory Gauss-Jordan sweeps take.
__device__ void cholesky_inverse_body(int32_t n, double *__restrict__ A, double *__restrict__ Ainv,
                                      int *__restrict__ err);

// one thread block per system block of a batch
__global__ void k_cholesky_inverse_batched(int32_t nsys, const int32_t *__restrict__ off,
                                           const int64_t *__restrict__ boff, double *__restrict__ A,
                                           double *__restrict__ Ainv, int *__restrict__ err) {
  pdl_wait_and_trigger();
  const int32_t s = blockIdx.x;
  if (s >= nsys) return;
  cholesky_inverse_body(off[s + 1] - off[s], A + boff[s], Ainv + boff[s], err);
}

__device__ void cholesky_inverse_body(int32_t n, double *__restrict__ A, double *__restrict__ Ainv,
                                      int *__restrict__ err) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int32_t j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(int64_t)j * n + j];
      if (!(d > 0.0)) bad = 1;
      A[(int64_t)j * n + j] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    if (bad) break;
    const double ljj = A[(int64_t)j * n + j];
    for (int32_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * n + j] /= ljj;
    __syncthreads();
    const int64_t rem = n - j - 1;
    for (int64_t t = threadIdx.x; t < rem * rem; t += blockDim.x) {
      const int32_t i = j + 1 + (int32_t)(t / rem), k = j + 1 + (int32_t)(t % rem);
      if (k <= i) A[(int64_t)i * n + k] -= A[(int64_t)i * n + j] * A[(int64_t)k * n + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) *err = 1;
    return;
  }
  for (int32_t c = threadIdx.x; c < n; c += blockDim.x) {
    double *x = Ainv + (int64_t)c * n;  // column c of the inverse (A is symmetric)
    for (int32_t i = 0; i < n; ++i) {    // L y = e_c
      double t = (i == c) ? 1.0 : 0.0;
      for (int32_t k = 0; k < i; ++k) t -= A[(int64_t)i * n + k] * x[k];
      x[i] = t / A[(int64_t)i * n + i];
    }
    for (int32_t i = n - 1; i >= 0; --i) {  // L^T x = y
      double t = x[i];
      for (int32_t k = i + 1; k < n; ++k) t -= A[(int64_t)k * n + i] * x[k];
      x[i] = t / A[(int64_t)i * n + i];
    }
  }
}

// Inverse of a small SPD matrix held in shared memory by Gauss-Jordan sweeps
// (no pivoting: the pivots of an SPD matrix are the diagonals of its Schur
// complements, all positive; a pivot that is not marks the matrix as not
// positive definite).  Sweep p, with f_i = a_ip / a_pp:
//   a_ij -= f_i a_pj (i, j != p);  a_pj /= a_pp;  a_ip = -f_i;  a_pp = 1 / a_pp,
// and after n sweeps a = A^-1.  Every sweep updates the n^2 entries with all
// threads of the block (one fused multiply-add an entry), so the n sweeps cost
// 3n barriers instead of the n dependent steps per column of forward and back
// substitution.  FP64 runs at a few operations per clock per SM on this part,
// so the multiply-add count, not the barriers, sets the time.
constexpr int32_t kGjMax = 120;  // n^2 + n doubles of shared memory (113 KB)
__device__ void gj_inverse_body(int32_t n, const double *__restrict__ A, double *__restrict__ Ainv,
                                int *__restrict__ err, double *a) {
  __shared__ int bad;
  __shared__ double inv_sh;  // 1 / a_pp of the coming sweep, formed once by thread 0
  double *f = a + (size_t)n * n;
  const int32_t nn = n * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) a[t] = A[t];
  __syncthreads();
  if (threadIdx.x == 0) {
    bad = !(a[0] > 0.0);
    inv_sh = 1.0 / a[0];
  }
  __syncthreads();
  for (int32_t p = 0; p < n && !bad; ++p) {  // bad is uniform: read after a barrier
    const double inv = inv_sh;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) f[i] = a[i * n + p] * inv;
    __syncthreads();
    for (int32_t i = wid; i < n; i += nw) {  // warp per row, lanes over the columns
      if (i == p) continue;
      const double fi = f[i];
      for (int32_t j = lane; j < n; j += 32)
        if (j != p) a[i * n + j] = fma(-fi, a[p * n + j], a[i * n + j]);
    }
    __syncthreads();
    for (int32_t t = threadIdx.x; t < n; t += blockDim.x)
      if (t != p) {
        a[p * n + t] *= inv;
        a[t * n + p] = -f[t];
      }
    if (threadIdx.x == 0) {
      a[p * n + p] = inv;
      if (p + 1 < n) {  // the next pivot is final once this sweep's update is done
        const double piv = a[(p + 1) * n + p + 1];
        bad = !(piv > 0.0);
        inv_sh = 1.0 / piv;
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) *err = 1;
    return;
  }
  for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) Ainv[t] = a[t];
}

__global__ void k_gj_inverse(int32_t n, const double *__restrict__ A, double *__restrict__ Ainv,
                             int *__restrict__ err) {
  extern __shared__ double gj_a[];
  pdl_wait_and_trigger();
  gj_inverse_body(n, A, Ainv, err, gj_a);
}

// one thread block per system block of a batch
__global__ void k_gj_inverse_batched(int32_t nsys, const int32_t *__restrict__ off,
                                     const int64_t *__restrict__ boff, const double *__restrict__ A,
                                     double *__restrict__ Ainv, int *__restrict__ err) {
  extern __shared__ double gj_a[];
  pdl_wait_and_trigger();
  const int32_t s = blockIdx.x;
  if (s >= nsys) return;
  gj_inverse_body(off[s + 1] - off[s], A + boff[s], Ainv + boff[s], err, gj_a);
}

// ---- coarsest inverse across the GPU: blocked Gauss-Jordan --------------------
// The sweeps of k_gj_inverse taken kGjb pivots at a time.  With the pivot block
// P (rows and columns p0 .. p0 + kk) and B = M_PP^-1, one step is
//   M_PP <- B,  M_Pj <- B M_Pj,  M_iP <- -M_iP B,  M_ij <- M_ij - M_iP B M_Pj
// for i, j outside P; after the last block M = A^-1 (no pivoting: A is SPD, and
// so is every pivot block).  One launch per step, from src to dst (the launches
// are chained by programmatic dependent launch): a thread block owns whole
// columns and inverts the kk x kk pivot block itself, the same arithmetic in
// every block.  GB300 runs FP64 at ~2 multiply-adds per clock per SM, so the n^3
// multiply-adds of the inverse are spread over all SMs.
// err = 1: a pivot block is not positive definite.
constexpr int kGjb = 16;
constexpr int32_t kGjOneBlock = 64;  // up to this size one block in shared memory is faster

// 1/x in FP64 from an FP32 estimate and two Newton-Raphson steps
// r <- r + r (1 - x r): the relative error squares each step (2^-24 -> 2^-48 ->
// below FP64 rounding), so the result is within an ulp of 1/x; it is the same
// in every block, which is all the sweeps need.  Outside the FP32 range the
// division is taken as is.
__device__ __forceinline__ double recip_nr(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

__global__ void __launch_bounds__(256) k_gj_step(int32_t n, int32_t p0, const double *__restrict__ src,
                                                 double *__restrict__ dst, int *__restrict__ err) {
  __shared__ double sB[kGjb][kGjb + 1];  // pivot block, inverted in place
  __shared__ double sW[kGjb];            // B M_Pj of the current column
  __shared__ int bad;                    // a pivot of the block was not positive
  pdl_wait_and_trigger();
  const int tid = threadIdx.x;           // 256 threads: one per entry of the pivot block
  const int kk = min(kGjb, n - p0);
  for (int t = tid; t < kk * kk; t += blockDim.x) sB[t / kk][t % kk] = src[(int64_t)(p0 + t / kk) * n + p0 + t % kk];
  __syncthreads();
  // unblocked sweeps of the pivot block, a thread per entry: every new value
  // comes from the block before the sweep (the updates of k_gj_inverse, with the
  // pivot's reciprocal from recip_nr), so that a sweep is one short chain of
  // dependent FP64 operations and two barriers; FP64 latency, not throughput,
  // sets the time of the 16 sweeps
  if (tid == 0) bad = 0;
  {
    const int bi = tid / kGjb, bj = tid % kGjb;
    const bool mine = bi < kk && bj < kk;
    for (int p = 0; p < kk; ++p) {
      const double piv = sB[p][p];  // the same in every thread and every block
      if (!(piv > 0.0)) {
        if (tid == 0) bad = 1;
        break;
      }
      const double inv = recip_nr(piv);
      double v = 0.0;
      if (mine) {
        const double f = sB[bi][p] * inv;
        if (bi != p && bj != p) v = fma(-f, sB[p][bj], sB[bi][bj]);
        else if (bi == p && bj != p) v = sB[p][bj] * inv;
        else if (bi != p) v = -f;
        else v = inv;
      }
      __syncthreads();
      if (mine) sB[bi][bj] = v;
      __syncthreads();
    }
  }
  __syncthreads();
  if (bad) {  // the same in every block
    if (blockIdx.x == 0 && tid == 0) *err = 1;
    return;
  }
  for (int32_t j = blockIdx.x; j < n; j += gridDim.x) {
    if (j < p0 || j >= p0 + kk) {
      if (tid < kk) {  // the kGjb loads go out together (a short last block reads zeros)
        double pc[kGjb];
#pragma unroll
        for (int m = 0; m < kGjb; ++m) pc[m] = m < kk ? src[(int64_t)(p0 + m) * n + j] : 0.0;
        double w = 0.0;
#pragma unroll
        for (int m = 0; m < kGjb; ++m)
          if (m < kk) w = fma(sB[tid][m], pc[m], w);
        sW[tid] = w;
      }
      __syncthreads();
      for (int32_t i = tid; i < n; i += blockDim.x) {
        double v;
        if (i >= p0 && i < p0 + kk) {
          v = sW[i - p0];
        } else {
          const double *aip = src + (int64_t)i * n + p0;
          double a[kGjb];
#pragma unroll
          for (int l = 0; l < kGjb; ++l) a[l] = l < kk ? aip[l] : 0.0;
          v = src[(int64_t)i * n + j];
#pragma unroll
          for (int l = 0; l < kGjb; ++l)
            if (l < kk) v = fma(-a[l], sW[l], v);
        }
        dst[(int64_t)i * n + j] = v;
      }
    } else {
      const int c = j - p0;
      for (int32_t i = tid; i < n; i += blockDim.x) {
        double v;
        if (i >= p0 && i < p0 + kk) {
          v = sB[i - p0][c];
        } else {
          const double *aip = src + (int64_t)i * n + p0;
          double a[kGjb];
#pragma unroll
          for (int l = 0; l < kGjb; ++l) a[l] = l < kk ? aip[l] : 0.0;
          v = 0.0;
#pragma unroll
          for (int l = 0; l < kGjb; ++l)
            if (l < kk) v = fma(a[l], sB[l][c], v);
          v = -v;
        }
        dst[(int64_t)i * n + j] = v;
      }
    }
    __syncthreads();  // sW is rewritten by the next column
  }
}

__global__ void k_gather_i32(int32_t n, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                             int32_t *__restrict__ dst) {
  pdl_wait_and_trigger();
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// block-diagonal assembly: rows of system s shifted by (row0, nnz0)
__global__ void k_shift_rowptr(int32_t n, const int32_t *__restrict__ rp, int64_t nnz0, int32_t *__restrict__ out) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    out[i] = (int32_t)(rp[i] + nnz0);
}
__global__ void k_shift_col(int64_t nnz, const int32_t *__restrict__ ci, int32_t row0, int32_t *__restrict__ out) {
  pdl_wait_and_trigger();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    out[p] = ci[p] + row0;
}

// coarsest level of a batch: one dense block per system, copied from the CSR
__global__ void k_dense_blocks(int32_t nsys, const int32_t *__restrict__ off, const int64_t *__restrict__ boff,
                               const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const double *__restrict__ val, double *__restrict__ dense) {
  pdl_wait_and_trigger();
  const int32_t s = blockIdx.x;
  if (s >= nsys) return;
  const int32_t r0 = off[s], m = off[s + 1] - r0;
  double *D = dense + boff[s];
  for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
    for (int32_t p = rp[r0 + i]; p < rp[r0 + i + 1]; ++p) D[(int64_t)i * m + (ci[p] - r0)] = val[p];
}

__global__ void k_fill_f64(int64_t n, double *p, double v) {
  pdl_wait_and_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ============================================================== host side
namespace {

// host_pinned (128 doubles): ints [0, 2) PMIS round counts, doubles [0, levels)
// omega read-back, ints at double offset 40: setup flags (symmetry, aggregation
// error), read at the next synchronisation; int64 at double offset 64: the SELL
// entry counts of the levels (slot kMaxLevels: level 0's FP64 copy)
constexpr int kPinnedSetupFlags = 40;
constexpr int kPinnedSellEntries = 64;
static_assert(kPinnedSellEntries + kMaxLevels + 1 <= 128, "pinned scratch holds 128 doubles");

template <class T>
T read_scalar(const T *dev, cudaStream_t s) {
  T v{};
  AMG_CUDA(cudaMemcpyAsync(&v, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  return v;
}

inline unsigned blocks_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

// device arrays of one coarsening step
struct Coarsening {
  int32_t nc = 0;
  int32_t rounds = 0;
};

Coarsening coarsen_level(Hierarchy &h, int k, cudaStream_t s, int32_t *agg_out, int32_t *next_sys_off) {
  Level &L = h.lev[k];
  const int32_t n = L.n;
  const int64_t nnz = L.nnz;
  const unsigned gb = blocks_for(n);
  DevBuf<uint8_t> C(nnz);
  DevBuf<int32_t> rowcnt(n + 1), colcnt(n + 1), deg(n + 1), off(n + 1), cursor(n + 1);
  AMG_CUDA(cudaMemsetAsync(colcnt.p, 0, sizeof(int32_t) * (n + 1), s));
  AMG_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * (n + 1), s));
  AMG_COUNT(), klaunch_sm(k_strength, grid_for(n, 256), 256, 0, s, n, L.rp, L.ci, L.val, h.p.alpha, C.p, rowcnt.p,
      colcnt.p);
  AMG_LAUNCH_CHECK();
  DevBuf<int32_t> ucount(n + 1), Sptr(n + 1);
  DevBuf<int32_t> Scol;
  int32_t ns = 0;
  {  // N_i for a structurally symmetric pattern: mark in place, compact
    DevBuf<uint8_t> S(nnz);
    DevBuf<int> nonsym(1);
    AMG_CUDA(cudaMemsetAsync(nonsym.p, 0, sizeof(int), s));
    AMG_COUNT(), klaunch_sm(k_sym_mirror, grid_for(n, 256), 256, 0, s, n, L.rp, L.ci, C.p, S.p, ucount.p, nonsym.p);
    AMG_LAUNCH_CHECK();
    // The coarse levels of a structurally symmetric A_0 are structurally
    // symmetric (P^T A P keeps the pattern's symmetry): no flag to read, and the
    // graph is sized by the pattern instead of its count (no synchronisation).
    // Otherwise the flag rides on the scan's synchronisation.
    const bool known_sym = k > 0 && h.sym_pattern;
    int32_t *flag_host = reinterpret_cast<int32_t *>(h.host_pinned + kPinnedSetupFlags);
    if (known_sym) {
      exclusive_scan<int32_t, int32_t>(ucount.p, Sptr.p, n, s);
    } else {
      AMG_CUDA(cudaMemcpyAsync(flag_host, nonsym.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      exclusive_scan<int32_t, int32_t>(ucount.p, Sptr.p, n, s, &ns);
      if (k == 0) h.sym_pattern = !*flag_host;
    }
    if (known_sym || !*flag_host) {
      Scol.resize(known_sym ? (size_t)nnz + 1 : (size_t)ns + 1);
      AMG_COUNT(), klaunch_sm(k_sym_mirror_fill, grid_for(n, 256), 256, 0, s, n, L.rp, L.ci, S.p, Sptr.p, Scol.p);
      AMG_LAUNCH_CHECK();
    } else {  // general pattern: collect C rows and transposed entries, sort, deduplicate
      AMG_COUNT(), klaunch_sm(k_add_i32, gb, 256, 0, s, n, rowcnt.p, colcnt.p, deg.p);
      int32_t total = 0;
      exclusive_scan<int32_t, int32_t>(deg.p, off.p, n, s, &total);
      DevBuf<int32_t> tmp((size_t)total + 1);
      AMG_COUNT(), klaunch_sm(k_sym_fill, grid_for(n, 256), 256, 0, s, n, L.rp, L.ci, C.p, rowcnt.p, off.p, cursor.p,
          tmp.p);
      AMG_COUNT(), klaunch_sm(k_sort_unique, grid_for(n, 128), 128, 0, s, n, off.p, tmp.p, ucount.p);
      AMG_LAUNCH_CHECK();
      exclusive_scan<int32_t, int32_t>(ucount.p, Sptr.p, n, s, &ns);
      Scol.resize((size_t)ns + 1);
      AMG_COUNT(), klaunch_sm(k_compact, grid_for(n, 256), 256, 0, s, n, off.p, tmp.p, Sptr.p, Scol.p);
      AMG_LAUNCH_CHECK();
    }
  }

  // PMIS(k): k max rounds per iteration (k = 2: Alg. 2)
  const int mk = h.p.mis_k;
  DevBuf<uint64_t> key(n), Tw(n), Tw2(mk > 2 ? n : 1);
  DevBuf<int32_t> Ti(n), Ti2(mk > 2 ? n : 1), und(1);
  DevBuf<int8_t> st(n);
  AMG_COUNT(), klaunch_sm(k_mis_keys, gb, 256, 0, s, n, colcnt.p, h.p.seed, k, key.p, st.p);
  AMG_LAUNCH_CHECK();
  Coarsening out;
  {
    // Round r counts its undecided nodes into und[r % 2]; the host reads round
    // r-1's count while round r runs.  Once a round leaves no undecided node the
    // round after it changes nothing, so one speculative round is harmless.
    DevBuf<int32_t> und2(2);
    DevBuf<unsigned> ticket(1);
    AMG_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), s));
    int32_t *pin = reinterpret_cast<int32_t *>(h.host_pinned);
    int32_t *pin_dev = nullptr;  // the same words as the device sees them
    AMG_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void **>(&pin_dev), pin, 0));
    EventPair ep;  // destroyed on every exit, including a throw inside the loop
    cudaEvent_t *ev = ep.e;
    bool done = false;
    for (int round = 0; round < 100000 && !done; ++round) {
      const int b = round & 1;
      AMG_COUNT(), klaunch_sm(k_pmis_max1, grid_for(n, 256), 256, 0, s, n, Sptr.p, Scol.p, st.p, key.p, Tw.p, Ti.p,
                              und2.p + b);
      uint64_t *tw = Tw.p, *tw2 = Tw2.p;
      int32_t *ti = Ti.p, *ti2 = Ti2.p;
      for (int r = 2; r < mk; ++r) {
        AMG_COUNT(), klaunch_sm(k_pmis_maxk, grid_for(n, 256), 256, 0, s, n, Sptr.p, Scol.p, tw, ti, tw2, ti2);
        std::swap(tw, tw2);
        std::swap(ti, ti2);
      }
      AMG_COUNT(), klaunch_sm(k_pmis_max2_decide, grid_for(n, 256), 256, 0, s, n, Sptr.p, Scol.p, tw, ti, st.p,
                              und2.p + b, mk >= 2, ticket.p, (volatile int32_t *)(pin_dev + b));
      AMG_LAUNCH_CHECK();
      AMG_CUDA(cudaEventRecord(ev[b], s));
      if (round >= 1) {
        AMG_CUDA(cudaEventSynchronize(ev[b ^ 1]));
        if (pin[b ^ 1] == 0) {
          out.rounds = round;  // rounds 0..round-1 did the work
          done = true;
        }
      }
      if (!done && round + 1 >= 100000) out.rounds = round + 1;
    }
    AMG_CUDA(cudaStreamSynchronize(s));
  }
  // aggregation
  DevBuf<int32_t> r1(n), r2(n), isroot(n + 1), cid(n + 1), err(1);
  AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  AMG_COUNT(), klaunch_sm(k_agg_pass1, grid_for(n, 256), 256, 0, s, n, Sptr.p, Scol.p, st.p, key.p, r1.p, isroot.p);
  int32_t *ra = r1.p, *rb = r2.p;
  for (int d = 2; d <= mk; ++d) {  // passes 2..k
    AMG_COUNT(), klaunch_sm(k_agg_pass2, grid_for(n, 256), 256, 0, s, n, Sptr.p, Scol.p, st.p, key.p, ra, rb);
    std::swap(ra, rb);
  }
  AMG_LAUNCH_CHECK();
  int32_t nc = 0;
  exclusive_scan<int32_t, int32_t>(isroot.p, cid.p, n, s, &nc);
  AMG_COUNT(), klaunch_sm(k_agg_final, gb, 256, 0, s, n, ra, cid.p, agg_out, err.p);
  AMG_LAUNCH_CHECK();
  if (next_sys_off) {  // coarse rows of system s start at the number of roots before its first row
    AMG_COUNT(), klaunch_sm(k_gather_i32, blocks_for(h.nsys + 1), 256, 0, s, h.nsys + 1, L.sys_off, cid.p,
        next_sys_off);
    AMG_LAUNCH_CHECK();
  }
  // checked at the next synchronisation (the member kernels skip an unassigned node)
  AMG_CUDA(cudaMemcpyAsync(reinterpret_cast<int32_t *>(h.host_pinned + kPinnedSetupFlags) + 1, err.p, sizeof(int),
                           cudaMemcpyDeviceToHost, s));
  out.nc = nc;
  return out;
}

// SELL-32 layouts (slice pointers, index arrays) of every level: the slice
// widths and their scans of all levels are queued first, and one
// synchronisation reads every level's entry count (pinned words from
// kPinnedSellEntries on) before the arrays are allocated.
// pairs: entries two by two, slice widths even (FP32: stored with their
// columns in L.spair, no scol / sval; BF16: adjacent in scol and sval)
void layout_all(Hierarchy &h, cudaStream_t s) {
  const bool split = h.p.precision != AMG_PREC_F64;
  auto *ent = reinterpret_cast<int64_t *>(h.host_pinned + kPinnedSellEntries);
  auto widths = [&](Level &L, bool pairs, int64_t *&sptr, int slot) {
    DevBuf<int64_t> w32(L.nslices + 1);
    AMG_COUNT(), klaunch_sm(k_slice_width, blocks_for((int64_t)L.nslices * 32), 256, 0, s, L.n, L.nslices, L.rp,
        L.ci, pairs ? split : false, pairs, w32.p);
    AMG_LAUNCH_CHECK();
    sptr = h.arena.get<int64_t>(L.nslices + 1);
    exclusive_scan<int64_t, int64_t>(w32.p, sptr, L.nslices, s);
    AMG_CUDA(cudaMemcpyAsync(ent + slot, sptr + L.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  };
  for (int q = 0; q < h.L; ++q) {
    Level &L = h.lev[q];
    L.nslices = (L.n + kSlice - 1) / kSlice;
    widths(L, split, L.sptr, q);
  }
  if (split) widths(h.lev[0], false, h.lev[0].sptr64, kMaxLevels);  // every entry in FP64
  AMG_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < h.L; ++q) {
    Level &L = h.lev[q];
    L.sell_entries = ent[q];
    if (h.p.precision == AMG_PREC_F32) L.spair = h.arena.get<int4>(L.sell_entries / 2);
    else L.scol = h.arena.get<int32_t>(L.sell_entries);
  }
  if (split) {
    Level &L0 = h.lev[0];
    L0.sell64_entries = ent[kMaxLevels];
    L0.scol64 = h.arena.get<int32_t>(L0.sell64_entries);
    L0.sval64 = h.arena.get<double>(L0.sell64_entries);
  }
}

// SELL-32 of level L: the preconditioner's matrix in its precision and, on
// level 0, every entry in FP64 for the outer iteration (layouts from
// layout_all).  fresh: allocate the value arrays; otherwise refill the values
// of the existing layout (values-only re-setup, same pattern)
void build_solve_matrix(Hierarchy &h, Level &L, cudaStream_t s, bool fresh) {
  const int32_t n = L.n;
  const unsigned g = blocks_for((int64_t)L.nslices * 32);
  const bool split = h.p.precision != AMG_PREC_F64;
  const int64_t entries = L.sell_entries;
  if (fresh && split) L.sdiag = h.arena.get<float>(n);
  switch (h.p.precision) {
    case AMG_PREC_F64:
      if (fresh) L.sval = h.arena.get<double>(entries);
      AMG_COUNT(), klaunch_sm(k_build_sell<double>, g, 256, 0, s, n, L.nslices, L.rp, L.ci, L.val, L.sptr, L.scol,
          (double *)L.sval, nullptr, nullptr);
      break;
    case AMG_PREC_F32:
      AMG_COUNT(), klaunch_sm(k_build_sell<float>, g, 256, 0, s, n, L.nslices, L.rp, L.ci, L.val, L.sptr, nullptr,
          nullptr, L.spair, L.sdiag);
      break;
    default:
      if (fresh) L.sval = h.arena.get<__nv_bfloat16>(entries);
      AMG_COUNT(), klaunch_sm(k_build_sell<__nv_bfloat16>, g, 256, 0, s, n, L.nslices, L.rp, L.ci, L.val, L.sptr,
          L.scol, (__nv_bfloat16 *)L.sval, nullptr, L.sdiag);
  }
  AMG_LAUNCH_CHECK();
  if (&L != &h.lev[0]) return;
  if (split) {
    AMG_COUNT(), klaunch_sm(k_build_sell<double>, g, 256, 0, s, n, L.nslices, L.rp, L.ci, L.val, L.sptr64, L.scol64,
        L.sval64, nullptr, nullptr);
    AMG_LAUNCH_CHECK();
  } else {
    L.sptr64 = L.sptr;
    L.scol64 = L.scol;
    L.sval64 = (double *)L.sval;
    L.sell64_entries = L.sell_entries;
  }
}

// m = 5 Arnoldi steps on D^-1/2 A D^-1/2 for omega of Eq. (damped Jacobi):
// three kernels per step; the Hessenberg matrix goes to H (9 x 8) and the
// norms ||M q_j|| to wn (8), for k_omega_from_H.  Returns m.
int arnoldi_omega(Hierarchy &h, int k, const double *diag, double *H, double *wn, cudaStream_t s) {
  Level &L = h.lev[k];
  const int32_t n = L.n;
  const int m = n < kArnoldiMax ? n : kArnoldiMax;
  const int g = grid_for(n, 256, kRedBlocks);  // a few rows per thread; few partials to reduce
  DevBuf<double> Q((size_t)n * m), W(n), U(n), w(n), dh(n), part((size_t)kArnSlots * kRedBlocks), corr(8), nrm2(1);
  // an FP64 SELL copy of every entry: level 0 always, every level in FP64 mode
  const int64_t *sp64 = k == 0 ? L.sptr64 : (h.p.precision == AMG_PREC_F64 ? L.sptr : nullptr);
  const int32_t *sc64 = k == 0 ? L.scol64 : L.scol;
  const double *sv64 = k == 0 ? L.sval64 : static_cast<const double *>(L.sval);
  const int gs = grid_for(L.nslices, 8, kRedBlocks);
  // CSR rows: 8 lanes a row from 16 entries a row on average, else 4
  const bool wide = L.nnz >= 16 * (int64_t)n;
  const int gc = grid_for((int64_t)n * (wide ? 8 : 4), 256, kRedBlocks);
  DevBuf<unsigned> ticket(1);
  AMG_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * 72, s));
  AMG_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), s));
  AMG_COUNT(), klaunch_sm(k_arn_start, g, 256, 0, s, n, h.p.seed, k, diag, W.p, U.p, dh.p, part.p, nrm2.p, ticket.p);
  // symmetric A: the Lanczos form of the process (M = |D|^-1/2 A |D|^-1/2 is
  // symmetric, so the Arnoldi matrix is tridiagonal): one product and one
  // three-term update a step; otherwise Arnoldi with classical Gram-Schmidt twice
  const bool lz = h.p.symmetric != 0;
  for (int j = 0; j < m; ++j) {
    if (sp64) {
      if (lz)
        AMG_COUNT(), klaunch_sm(k_arn_spmv_sell<true>, gs, 256, 0, s, n, L.nslices, j, sp64, sc64, sv64, dh.p, W.p,
                                U.p, Q.p, w.p, part.p, nrm2.p, H, wn, ticket.p);
      else
        AMG_COUNT(), klaunch_sm(k_arn_spmv_sell<false>, gs, 256, 0, s, n, L.nslices, j, sp64, sc64, sv64, dh.p, W.p,
                                U.p, Q.p, w.p, part.p, nrm2.p, H, wn, ticket.p);
    } else if (wide) {
      if (lz)
        AMG_COUNT(), klaunch_sm(k_arn_spmv<8, true>, gc, 256, 0, s, n, j, L.rp, L.ci, L.val, dh.p, W.p, U.p, Q.p, w.p,
                                part.p, nrm2.p, H, wn, ticket.p);
      else
        AMG_COUNT(), klaunch_sm(k_arn_spmv<8, false>, gc, 256, 0, s, n, j, L.rp, L.ci, L.val, dh.p, W.p, U.p, Q.p, w.p,
                                part.p, nrm2.p, H, wn, ticket.p);
    } else {
      if (lz)
        AMG_COUNT(), klaunch_sm(k_arn_spmv<4, true>, gc, 256, 0, s, n, j, L.rp, L.ci, L.val, dh.p, W.p, U.p, Q.p, w.p,
                                part.p, nrm2.p, H, wn, ticket.p);
      else
        AMG_COUNT(), klaunch_sm(k_arn_spmv<4, false>, gc, 256, 0, s, n, j, L.rp, L.ci, L.val, dh.p, W.p, U.p, Q.p, w.p,
                                part.p, nrm2.p, H, wn, ticket.p);
    }
    if (lz) {
      if (j + 1 < m)  // the last step's update is not used
        AMG_COUNT(), klaunch_sm(k_lz_update, g, 256, 0, s, n, j, (const double *)Q.p, (const double *)w.p, W.p, U.p,
                                (const double *)dh.p, part.p, (const double *)H, nrm2.p, ticket.p);
      continue;
    }
    AMG_COUNT(), klaunch_sm(k_arn_orth, g, 256, 0, s, n, j, 0, Q.p, w.p, W.p, U.p, dh.p, part.p, H, corr.p, nrm2.p,
        ticket.p);
    AMG_COUNT(), klaunch_sm(k_arn_orth, g, 256, 0, s, n, j, 1, Q.p, w.p, W.p, U.p, dh.p, part.p, H, corr.p, nrm2.p,
        ticket.p);
  }
  AMG_LAUNCH_CHECK();
  return m;
}

}  // namespace

void build_hierarchy(Hierarchy &h, const amg_csr &A, cudaStream_t s) {
  const int32_t n = A.n;
  if (!h.host_pinned) h.host_pinned = pinned_scratch_get();
  // ---- level 0: copy and validate the input
  Level &L0 = h.lev[0];
  L0.n = n;
  L0.nnz = A.nnz;
  L0.rp = h.arena.get<int32_t>((size_t)n + 1);
  L0.ci = h.arena.get<int32_t>((size_t)A.nnz);
  L0.val = h.arena.get<double>((size_t)A.nnz);
  const bool dev = pointer_kind(A.row_ptr) == PTR_DEVICE;
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  AMG_CUDA(cudaMemcpyAsync(L0.rp, A.row_ptr, sizeof(int32_t) * ((size_t)n + 1), kind, s));
  AMG_CUDA(cudaMemcpyAsync(L0.ci, A.col, sizeof(int32_t) * (size_t)A.nnz, kind, s));
  AMG_CUDA(cudaMemcpyAsync(L0.val, A.val, sizeof(double) * (size_t)A.nnz, kind, s));
  {
    DevBuf<int> err(1);
    AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    AMG_COUNT(), klaunch_sm(k_check_csr, blocks_for(n), 256, 0, s, n, A.nnz, L0.rp, L0.ci, L0.val, err.p);
    AMG_LAUNCH_CHECK();
    const int e = read_scalar(err.p, s);
    if (e) {
      std::string m = "invalid CSR:";
      if (e & 1) m += " bad row pointers;";
      if (e & 2) m += " column index out of range or not ascending;";
      if (e & 4) m += " missing or zero diagonal;";
      if (e & 8) m += " non-finite value;";
      throw Error{AMG_ERR_BAD_INPUT, m};
    }
  }
  L0.B = h.arena.get<double>(n);
  AMG_COUNT(), klaunch_sm(k_fill_f64, grid_for(n, 256), 256, 0, s, n, L0.B, 1.0);  // B_0 = 1
  AMG_LAUNCH_CHECK();
  coarsen_all(h, s);
}

// Batch of nsys systems as one block-diagonal matrix.  Strength, MIS and
// aggregation never couple the blocks, and roots are numbered in ascending
// fine index, so every level keeps each system's rows contiguous.
void build_hierarchy_batch(Hierarchy &h, int32_t nsys, const amg_csr *As, cudaStream_t s) {
  if (!h.host_pinned) h.host_pinned = pinned_scratch_get();
  h.batched = true;
  h.nsys = nsys;
  Level &L0 = h.lev[0];
  std::vector<int32_t> roff(nsys + 1, 0);
  std::vector<int64_t> zoff(nsys + 1, 0);
  for (int32_t q = 0; q < nsys; ++q) {
    roff[q + 1] = roff[q] + As[q].n;
    zoff[q + 1] = zoff[q] + As[q].nnz;
  }
  if (zoff[nsys] > INT32_MAX) throw Error{AMG_ERR_BAD_INPUT, "batch has more than 2^31 nonzeros"};
  L0.n = roff[nsys];
  L0.nnz = zoff[nsys];
  L0.rp = h.arena.get<int32_t>((size_t)L0.n + 1);
  L0.ci = h.arena.get<int32_t>((size_t)L0.nnz);
  L0.val = h.arena.get<double>((size_t)L0.nnz);
  size_t maxn = 0, maxz = 0;
  for (int32_t q = 0; q < nsys; ++q) {
    maxn = std::max(maxn, (size_t)As[q].n + 1);
    maxz = std::max(maxz, (size_t)As[q].nnz);
  }
  DevBuf<int32_t> trp(maxn), tci(maxz);
  for (int32_t q = 0; q < nsys; ++q) {
    const amg_csr &A = As[q];
    const cudaMemcpyKind kind = pointer_kind(A.row_ptr) == PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    AMG_CUDA(cudaMemcpyAsync(trp.p, A.row_ptr, sizeof(int32_t) * ((size_t)A.n + 1), kind, s));
    AMG_CUDA(cudaMemcpyAsync(tci.p, A.col, sizeof(int32_t) * (size_t)A.nnz, kind, s));
    AMG_CUDA(cudaMemcpyAsync(L0.val + zoff[q], A.val, sizeof(double) * (size_t)A.nnz, kind, s));
    AMG_COUNT(), klaunch_sm(k_shift_rowptr, grid_for(A.n + 1, 256), 256, 0, s, A.n, trp.p, zoff[q], L0.rp + roff[q]);
    AMG_COUNT(), klaunch_sm(k_shift_col, grid_for(A.nnz, 256), 256, 0, s, A.nnz, tci.p, roff[q], L0.ci + zoff[q]);
    AMG_LAUNCH_CHECK();
  }
  {
    DevBuf<int> err(1);
    AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    AMG_COUNT(), klaunch_sm(k_check_csr, blocks_for(L0.n), 256, 0, s, L0.n, L0.nnz, L0.rp, L0.ci, L0.val, err.p);
    AMG_LAUNCH_CHECK();
    if (read_scalar(err.p, s)) throw Error{AMG_ERR_BAD_INPUT, "invalid CSR in the batch"};
  }
  L0.sys_off_host = roff;
  L0.sys_off = h.arena.get<int32_t>(nsys + 1);
  AMG_CUDA(cudaMemcpyAsync(L0.sys_off, roff.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, s));
  L0.B = h.arena.get<double>(L0.n);
  AMG_COUNT(), klaunch_sm(k_fill_f64, grid_for(L0.n, 256), 256, 0, s, L0.n, L0.B, 1.0);
  AMG_LAUNCH_CHECK();
  AMG_CUDA(cudaStreamSynchronize(s));
  coarsen_all(h, s);
}

void coarsen_all(Hierarchy &h, cudaStream_t s) {
  const amg_params &p = h.p;
  // ---- Alg. 1: coarsen until the level is small
  int k = 0;
  for (;;) {
    Level &L = h.lev[k];
    int32_t largest = L.n;  // a batch stops when its largest system is small
    if (h.batched) {
      largest = 0;
      for (int32_t q = 0; q < h.nsys; ++q) largest = std::max(largest, L.sys_off_host[q + 1] - L.sys_off_host[q]);
    }
    if (largest <= p.coarse_max || k + 1 >= p.max_levels || k + 1 >= kMaxLevels) break;
    int32_t *agg = h.arena.get<int32_t>(L.n);
    int32_t *next_off = h.batched ? h.arena.get<int32_t>(h.nsys + 1) : nullptr;
    Coarsening cr = coarsen_level(h, k, s, agg, next_off);
    L.mis_rounds = cr.rounds;
    if (10LL * cr.nc >= 9LL * L.n) break;  // coarsening stalled: this level is the coarsest
    const int32_t nc = cr.nc;
    if (h.batched) {
      Level &Cn = h.lev[k + 1];
      Cn.sys_off = next_off;
      Cn.sys_off_host.resize(h.nsys + 1);
      AMG_CUDA(cudaMemcpyAsync(Cn.sys_off_host.data(), next_off, sizeof(int32_t) * (h.nsys + 1),
                               cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
    }
    L.agg = agg;
    L.nc = nc;
    // members of every aggregate, ascending
    L.aptr = h.arena.get<int32_t>((size_t)nc + 1);
    L.amem = h.arena.get<int32_t>(L.n);
    {
      DevBuf<int32_t> cnt(nc + 1), cur(nc + 1);
      AMG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (nc + 1), s));
      AMG_CUDA(cudaMemsetAsync(cur.p, 0, sizeof(int32_t) * (nc + 1), s));
      AMG_COUNT(), klaunch_sm(k_count_members, blocks_for(L.n), 256, 0, s, L.n, agg, cnt.p);
      exclusive_scan<int32_t, int32_t>(cnt.p, L.aptr, nc, s);
      AMG_COUNT(), klaunch_sm(k_fill_members, blocks_for(L.n), 256, 0, s, L.n, agg, L.aptr, cur.p, L.amem);
      AMG_COUNT(), klaunch_sm(k_sort_members, grid_for(nc, 128), 128, 0, s, nc, L.aptr, L.amem);
      AMG_LAUNCH_CHECK();
    }
    Level &Cl = h.lev[k + 1];
    Cl.n = nc;
    Cl.B = h.arena.get<double>(nc);
    L.pw64 = h.arena.get<double>(L.n);
    AMG_COUNT(), klaunch_sm(k_interp, grid_for(nc, 128), 128, 0, s, nc, L.aptr, L.amem, L.B, Cl.B, L.pw64);
    AMG_LAUNCH_CHECK();
    // Galerkin keyed sum: count, offsets, fill
    Cl.rp = h.arena.get<int32_t>((size_t)nc + 1);
    {  // one walk per coarse row into upper-bound slots, then compaction
      DevBuf<int32_t> ccount(nc + 1), rlen(nc + 1), ub(nc + 1), maxlen(1);
      AMG_CUDA(cudaMemsetAsync(maxlen.p, 0, sizeof(int32_t), s));
      AMG_COUNT(), klaunch_sm(k_run_length, grid_for(nc, 256), 256, 0, s, nc, L.aptr, L.amem, L.rp, rlen.p, maxlen.p);
      AMG_LAUNCH_CHECK();
      exclusive_scan<int32_t, int32_t>(rlen.p, ub.p, nc, s);
      const int32_t mx = read_scalar(maxlen.p, s);
      if (reinterpret_cast<const int32_t *>(h.host_pinned + kPinnedSetupFlags)[1] != 0)
        throw Error{AMG_ERR_SETUP, "aggregation left a node unassigned"};
      DevBuf<int32_t> tci(L.nnz + 1);
      DevBuf<double> tval(L.nnz + 1);
      // shared-memory sort path sized by the longest run (one warp per coarse row):
      // a first pass with runs of up to kGalCapFirst entries, at a higher
      // occupancy, then the longer runs with the full cap
      const int32_t cap = std::max<int32_t>(32, std::min<int32_t>(mx, kGalCapMax));
      // the summation plan for values-only re-setup (Sec. 3.1): recorded when every
      // run fits the shared-memory path
      L.plan = mx <= cap;
      DevBuf<int32_t> tseg(L.plan ? L.nnz + 1 : 1);
      if (L.plan) {
        L.gpos = h.arena.get<int32_t>((size_t)L.nnz);
        L.grow = h.arena.get<int32_t>((size_t)L.nnz);
      }
      auto gal_pass = [&](int32_t pcap, bool marked_only) {
        int hbits = 1;  // a table larger than the run: at least one free slot
        while ((1 << hbits) <= pcap) ++hbits;
        const size_t per = (size_t)pcap * 40 + ((size_t)8 << hbits);
        const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, kGalSmemBudget / per));
        const size_t smem = per * wpb;
        AMG_CUDA(cudaFuncSetAttribute(k_galerkin_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        AMG_COUNT(), klaunch_sm(k_galerkin_smem, grid_for(nc, wpb, 152 * 64), wpb * 32, smem, s, nc, pcap, hbits,
            marked_only, L.aptr, L.amem, L.rp, L.ci, L.val, agg, L.pw64, ccount.p, ub.p, tci.p, tval.p,
            L.plan ? L.gpos : nullptr, L.plan ? L.grow : nullptr, L.plan ? tseg.p : nullptr);
        AMG_LAUNCH_CHECK();
      };
      const int32_t cap1 = std::min(cap, kGalCapFirst);
      gal_pass(cap1, false);
      if (mx > cap1) gal_pass(cap, true);
      if (mx > cap) {  // runs longer than the cap: walked from global memory
        const int gw = grid_for((int64_t)nc * 32, 256, 152 * 64);
        AMG_COUNT(), klaunch_sm(k_galerkin<true>, gw, 256, 0, s, nc, L.aptr, L.amem, L.rp, L.ci, L.val, agg, L.pw64,
            ccount.p, ub.p, tci.p, tval.p, true);
        AMG_LAUNCH_CHECK();
      }
      int32_t cnnz = 0;
      exclusive_scan<int32_t, int32_t>(ccount.p, Cl.rp, nc, s, &cnnz);
      Cl.nnz = cnnz;
      Cl.ci = h.arena.get<int32_t>(cnnz);
      Cl.val = h.arena.get<double>(cnnz);
      AMG_COUNT(), klaunch_sm(k_compact_rows, grid_for(nc, 256), 256, 0, s, nc, ub.p, Cl.rp, tci.p, tval.p, Cl.ci,
          Cl.val);
      AMG_LAUNCH_CHECK();
      if (L.plan) {
        L.gptr = h.arena.get<int32_t>((size_t)cnnz + 1);
        AMG_COUNT(), klaunch_sm(k_compact_plan, grid_for(nc, 256), 256, 0, s, nc, ub.p, Cl.rp, tseg.p, L.gptr,
            (int32_t)L.nnz);
        AMG_LAUNCH_CHECK();
      }
    }
    ++k;
  }
  h.L = k + 1;

  finish_levels(h, s, true);
}

// Solve-phase data of every level (SELL values, diagonal, omega, per-row data)
// and the coarsest factorisation.  fresh = false refills the existing buffers in
// place (values-only re-setup): captured solve graphs stay valid.
void finish_levels(Hierarchy &h, cudaStream_t s, bool fresh) {
  const amg_params &p = h.p;
  std::vector<DevBuf<double>> diag(h.L);
  DevBuf<double> Hs((size_t)kMaxLevels * 72), wns((size_t)kMaxLevels * 8);
  OmegaJobs jobs{};
  int nj = 0;
  if (fresh) layout_all(h, s);
  for (int q = 0; q < h.L; ++q) {
    Level &L = h.lev[q];
    build_solve_matrix(h, L, s, fresh);
    diag[q].resize(L.n);
    AMG_COUNT(), klaunch_sm(k_diag, blocks_for(L.n), 256, 0, s, L.n, L.rp, L.ci, L.val, diag[q].p);
    AMG_LAUNCH_CHECK();
    L.omega = p.omega;  // omega_mode 1; mode 0 reads the estimate back after the loop
    if (q < h.L - 1 && p.omega_mode == 0) {
      if (!L.omega_dev) L.omega_dev = h.arena.get<double>(1);
      jobs.H[nj] = Hs.p + (size_t)nj * 72;
      jobs.wn[nj] = wns.p + (size_t)nj * 8;
      jobs.out[nj] = L.omega_dev;
      jobs.m[nj] = arnoldi_omega(h, q, diag[q].p, Hs.p + (size_t)nj * 72, wns.p + (size_t)nj * 8, s);
      ++nj;
    }
  }
  if (nj) {  // every level's omega = (4/3) / rho in one launch
    AMG_COUNT(), klaunch_sm(k_omega_from_H, nj, 32, 0, s, jobs, p.symmetric);
    AMG_LAUNCH_CHECK();
  }
  for (int q = 0; q < h.L; ++q) make_row_data(h, h.lev[q], diag[q].p, s);  // per-row smoother data
  {  // the estimated weights back to the host, one synchronisation for all levels
    for (int q = 0; q < h.L - 1; ++q)
      if (h.lev[q].omega_dev)
        AMG_CUDA(cudaMemcpyAsync(h.host_pinned + q, h.lev[q].omega_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < h.L - 1; ++q)
      if (h.lev[q].omega_dev) h.lev[q].omega = h.host_pinned[q];
  }

  // ---- coarsest level: dense factorisation and inverse
  Level &Lc = h.lev[h.L - 1];
  if (h.batched) {  // one dense block per system
    std::vector<int64_t> boff(h.nsys + 1, 0);
    int32_t bmax = 0;
    for (int32_t q = 0; q < h.nsys; ++q) {
      const int32_t m = Lc.sys_off_host[q + 1] - Lc.sys_off_host[q];
      bmax = std::max(bmax, m);
      boff[q + 1] = boff[q] + (int64_t)m * m;
    }
    if (bmax > kMaxDense)
      throw Error{AMG_ERR_SETUP, "a system's coarsest level has " + std::to_string(bmax) + " unknowns"};
    h.bmax = bmax;
    h.nL = Lc.n;
    if (fresh) {
      h.binv = h.arena.get<double>((size_t)boff[h.nsys]);
      h.binv_off = h.arena.get<int64_t>(h.nsys + 1);
    }
    AMG_CUDA(cudaMemcpyAsync(h.binv_off, boff.data(), sizeof(int64_t) * (h.nsys + 1), cudaMemcpyHostToDevice, s));
    DevBuf<double> dense((size_t)boff[h.nsys]);
    DevBuf<int> err(1);
    AMG_CUDA(cudaMemsetAsync(dense.p, 0, sizeof(double) * (size_t)boff[h.nsys], s));
    AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    AMG_COUNT(), klaunch_sm(k_dense_blocks, h.nsys, 128, 0, s, h.nsys, Lc.sys_off, h.binv_off, Lc.rp, Lc.ci, Lc.val,
        dense.p);
    if (bmax <= kGjMax) {  // every block in shared memory
      const size_t sm = sizeof(double) * ((size_t)bmax * bmax + bmax);
      AMG_CUDA(cudaFuncSetAttribute(k_gj_inverse_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      AMG_COUNT(), klaunch_sm(k_gj_inverse_batched, h.nsys, 256, sm, s, h.nsys, (const int32_t *)Lc.sys_off,
                              (const int64_t *)h.binv_off, (const double *)dense.p, h.binv, err.p);
    } else {
      AMG_COUNT(), klaunch_sm(k_cholesky_inverse_batched, h.nsys, 256, 0, s, h.nsys, Lc.sys_off, h.binv_off, dense.p,
                              h.binv, err.p);
    }
    AMG_LAUNCH_CHECK();
    if (read_scalar(err.p, s)) throw Error{AMG_ERR_SETUP, "a system's coarsest matrix is not positive definite"};
    return;
  }
  if (Lc.n > kMaxDense)
    throw Error{AMG_ERR_SETUP, "coarsest level has " + std::to_string(Lc.n) + " unknowns (limit " +
                                   std::to_string(kMaxDense) + "); coarsening stalled"};
  h.nL = Lc.n;
  if (fresh) h.coarse_inv = h.arena.get<double>((size_t)Lc.n * Lc.n);
  {
    DevBuf<double> dense((size_t)Lc.n * Lc.n);
    DevBuf<int> err(1);
    AMG_CUDA(cudaMemsetAsync(dense.p, 0, sizeof(double) * (size_t)Lc.n * Lc.n, s));
    AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    AMG_COUNT(), klaunch_sm(k_dense_from_csr, blocks_for(Lc.n), 256, 0, s, Lc.n, Lc.rp, Lc.ci, Lc.val, dense.p);
    if (p.symmetric && Lc.n <= kGjOneBlock) {  // one block, in shared memory
      const size_t sm = sizeof(double) * ((size_t)Lc.n * Lc.n + Lc.n);
      AMG_CUDA(cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      AMG_COUNT(), klaunch_sm(k_gj_inverse, 1, 1024, sm, s, Lc.n, (const double *)dense.p, h.coarse_inv, err.p);
    } else if (p.symmetric) {  // blocked sweeps over the whole GPU, one launch per 16 pivots
      DevBuf<double> m1((size_t)Lc.n * Lc.n);
      const int nb = (Lc.n + kGjb - 1) / kGjb;
      const int grid = std::min(Lc.n, 152 * 4);  // a block per column, up to four waves of SMs
      const double *src = dense.p;
      for (int st = 0; st < nb; ++st) {  // the last step writes the inverse itself
        double *dst = (nb - 1 - st) % 2 == 0 ? h.coarse_inv : m1.p;
        AMG_COUNT(), klaunch_sm(k_gj_step, grid, 256, 0, s, Lc.n, st * kGjb, src, dst, err.p);
        src = dst;
      }
    } else {
      DevBuf<double> fac(Lc.n);
      AMG_COUNT(), klaunch_sm(k_lu_inverse, 1, 1024, 0, s, Lc.n, dense.p, h.coarse_inv, fac.p, err.p);
    }
    AMG_LAUNCH_CHECK();
    if (read_scalar(err.p, s))
      throw Error{AMG_ERR_SETUP, p.symmetric ? "coarsest level matrix is not positive definite"
                                             : "coarsest level matrix is singular"};
  }
}

// Values-only re-setup (Sec. 3.1): A_0 keeps its pattern and takes new values;
// the aggregates and P are kept (P depends on the near-null vector only), the
// coarse values come from the stored summation plans, then every level's solve
// data and the coarsest factorisation are refilled in place.
void resetup_values(Hierarchy &h, const double *val0, cudaStream_t s) {
  for (int k = 0; k + 1 < h.L; ++k)
    if (!h.lev[k].plan)
      throw Error{AMG_ERR_UNSUPPORTED, "level " + std::to_string(k) +
                                           " has aggregate runs too long for a stored Galerkin plan"};
  Level &L0 = h.lev[0];
  const cudaMemcpyKind kind = pointer_kind(val0) == PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  AMG_CUDA(cudaMemcpyAsync(L0.val, val0, sizeof(double) * (size_t)L0.nnz, kind, s));
  {
    DevBuf<int> err(1);
    AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    AMG_COUNT(), klaunch_sm(k_check_csr, blocks_for(L0.n), 256, 0, s, L0.n, L0.nnz, L0.rp, L0.ci, L0.val, err.p);
    AMG_LAUNCH_CHECK();
    if (read_scalar(err.p, s)) throw Error{AMG_ERR_BAD_INPUT, "new values: zero diagonal or non-finite value"};
  }
  for (int k = 0; k + 1 < h.L; ++k) {
    Level &L = h.lev[k], &C = h.lev[k + 1];
    AMG_COUNT(), klaunch_sm(k_galerkin_values, grid_for(C.nnz, 256, 152 * 32), 256, 0, s, (int32_t)C.nnz, L.gptr,
        L.gpos, L.grow, L.ci, L.val, L.pw64, C.val);
    AMG_LAUNCH_CHECK();
  }
  finish_levels(h, s, false);
}

}  // namespace amg
