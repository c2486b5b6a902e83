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
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] + b[i];
}

// N_i = {j != i : C_ij or C_ji}: row i of the work array holds its own strong
// columns first, then (via atomics, in any order) the rows that hold i strongly.
__global__ void k_sym_fill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const uint8_t *__restrict__ C, const int32_t *__restrict__ rowcnt,
                           const int32_t *__restrict__ off, int32_t *__restrict__ cursor,
                           int32_t *__restrict__ tmp) {
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

__global__ void k_compact(int32_t n, const int32_t *__restrict__ off, const int32_t *__restrict__ tmp,
                          const int32_t *__restrict__ Sptr, int32_t *__restrict__ Scol) {
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
__global__ void k_pmis_max1(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const int8_t *__restrict__ s, const uint64_t *__restrict__ key,
                            uint64_t *__restrict__ Tw, int32_t *__restrict__ Ti) {
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

// second max round, then the decision of Alg. 2 for undecided nodes
__global__ void k_pmis_max2_decide(int32_t n, const int32_t *__restrict__ Sptr,
                                   const int32_t *__restrict__ Scol, const uint64_t *__restrict__ Tw,
                                   const int32_t *__restrict__ Ti, int8_t *__restrict__ s,
                                   int32_t *__restrict__ undecided) {
  int32_t local = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (s[i] != 0) continue;
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
    if (bi == i)
      s[i] = 1;
    else if ((bw >> 62) == 2)
      s[i] = -1;
    else
      local++;
  }
  local = __reduce_add_sync(0xffffffffu, local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(undecided, local);
}

// ============================================================== aggregation
__device__ __forceinline__ bool root_gt(int32_t a, int32_t b, const uint64_t *key) {
  return key[a] > key[b] || (key[a] == key[b] && a > b);
}

// Every non-MIS node joins its nearest MIS node; ties between equally near
// roots go to the larger priority (v, i).  Pass 1: roots adjacent to i.
__global__ void k_agg_pass1(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const int8_t *__restrict__ s, const uint64_t *__restrict__ key,
                            int32_t *__restrict__ r1) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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

// Pass 2: nodes at distance 2 join through a neighbour assigned in pass 1.
__global__ void k_agg_pass2(int32_t n, const int32_t *__restrict__ Sptr, const int32_t *__restrict__ Scol,
                            const int8_t *__restrict__ s, const uint64_t *__restrict__ key,
                            const int32_t *__restrict__ r1, int32_t *__restrict__ r2,
                            int32_t *__restrict__ is_root) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    is_root[i] = (s[i] == 1);
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
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_fill_members(int32_t n, const int32_t *__restrict__ agg, const int32_t *__restrict__ aptr,
                               int32_t *__restrict__ cur, int32_t *__restrict__ amem) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int32_t I = agg[i];
    amem[aptr[I] + atomicAdd(&cur[I], 1)] = i;
  }
}
__global__ void k_sort_members(int32_t nc, const int32_t *__restrict__ aptr, int32_t *__restrict__ amem) {
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x)
    sort_segment(amem + aptr[I], aptr[I + 1] - aptr[I]);
}

// ============================================================== Alg. 3
// B_{k+1}(I) = ||B_k restricted to G_I||_2 (squares summed in ascending fine
// index), P(i, I) = B_k(i) / B_{k+1}(I).
__global__ void k_interp(int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
                         const double *__restrict__ B, double *__restrict__ Bc, double *__restrict__ pw) {
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
constexpr int kGalCap = 320;   // entries of one coarse row staged in shared memory

template <bool FILL>
__global__ void __launch_bounds__(kGalWarps * 32) k_galerkin(
    int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ val,
    const int32_t *__restrict__ agg, const double *__restrict__ pw, int32_t *__restrict__ ccount,
    const int32_t *__restrict__ crp, int32_t *__restrict__ cci, double *__restrict__ cval) {
  __shared__ int32_t sJ[kGalWarps][kGalCap];
  __shared__ double sV[FILL ? kGalWarps : 1][FILL ? kGalCap : 1];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  for (int32_t I = blockIdx.x * wpb + wid; I < nc; I += gridDim.x * wpb) {
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
      // walk the distinct coarse columns in ascending order; sum each in run order
      int32_t cur = -1, out = 0;
      for (;;) {
        int32_t next = INT_MAX;
        double sum = 0.0;
        bool have = false;
        for (int32_t e0 = 0; e0 < total; e0 += 32) {
          const int32_t e = e0 + lane;
          const int32_t J = e < total ? sJ[wid][e] : INT_MAX;
          if (J > cur && J < next) next = J;
          if (FILL) {
            unsigned mask = __ballot_sync(0xffffffffu, J == cur);
            const double v = (J == cur) ? sV[wid][e] : 0.0;
            while (mask) {
              const int src = __ffs(mask) - 1;
              const double t = __shfl_sync(0xffffffffu, v, src);
              sum = have ? __dadd_rn(sum, t) : t;
              have = true;
              mask &= mask - 1;
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
      if (!FILL && lane == 0) ccount[I] = out;
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
    if (!FILL && lane == 0) ccount[I] = out;
  }
}

// ============================================================== solve-phase data
__global__ void k_diag(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ val, double *__restrict__ diag) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) d = val[p];
  diag[i] = d;
}

// SELL-32: width of every slice = longest row in it
__global__ void k_slice_width(int32_t n, int32_t nslices, const int32_t *__restrict__ rp,
                              int64_t *__restrict__ width32) {
  const int lane = threadIdx.x & 31;
  const int32_t sl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (sl >= nslices) return;
  const int32_t row = sl * kSlice + lane;
  int32_t len = row < n ? rp[row + 1] - rp[row] : 0;
  len = __reduce_max_sync(0xffffffffu, len);
  if (lane == 0) width32[sl] = (int64_t)len * kSlice;
}

template <class MV>
__device__ __forceinline__ MV conv_val(double v);
template <> __device__ __forceinline__ double conv_val<double>(double v) { return v; }
template <> __device__ __forceinline__ float conv_val<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 conv_val<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}

template <class MV>
__global__ void k_build_sell(int32_t n, int32_t nslices, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ val,
                            const int64_t *__restrict__ sptr, int32_t *__restrict__ scol, MV *__restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const int32_t sl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (sl >= nslices) return;
  const int32_t row = sl * kSlice + lane;
  const int64_t base = sptr[sl];
  const int32_t width = (int32_t)((sptr[sl + 1] - base) / kSlice);
  const int32_t p0 = row < n ? rp[row] : 0;
  const int32_t len = row < n ? rp[row + 1] - p0 : 0;
  const int32_t pad_col = row < n ? row : n - 1;
  for (int32_t e = 0; e < width; ++e) {
    const int64_t at = base + (int64_t)e * kSlice + lane;
    if (e < len) {
      scol[at] = ci[p0 + e];
      sval[at] = conv_val<MV>(val[p0 + e]);
    } else {
      scol[at] = pad_col;
      sval[at] = conv_val<MV>(0.0);
    }
  }
}

// ============================================================== Arnoldi omega
__global__ void k_arnoldi_start(int32_t n, uint64_t seed, int32_t level, const double *__restrict__ diag,
                                double *__restrict__ q, double *__restrict__ dh) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t z = splitmix64(~seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)(uint32_t)i);
  q[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  dh[i] = 1.0 / sqrt(fabs(diag[i]));
}

// w = D^-1/2 A D^-1/2 q  (CSR, FP64, one thread per row)
__global__ void k_scaled_spmv(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ val, const double *__restrict__ dh,
                              const double *__restrict__ q, double *__restrict__ w) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) acc += val[p] * (dh[ci[p]] * q[ci[p]]);
    w[i] = dh[i] * acc;
  }
}

// block partial sums of a.b (grid-stride, fixed grid: deterministic)
__global__ void k_dot_part(int32_t n, const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += a[i] * b[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// out[slot] = sum of part[0..nb)  (mode 1: sqrt of the sum)
__global__ void k_fin_sum(const double *__restrict__ part, int nb, double *__restrict__ out, int mode) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) acc += part[k];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = mode == 1 ? sqrt(v) : v;
  }
}

// y -= (*h) x
__global__ void k_axpy_neg_dev(int32_t n, double *__restrict__ y, const double *__restrict__ x,
                               const double *__restrict__ h) {
  const double a = *h;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] -= a * x[i];
}
// y = x / (*nrm)
__global__ void k_div_dev(int32_t n, double *__restrict__ y, const double *__restrict__ x,
                          const double *__restrict__ nrm) {
  const double a = *nrm;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i] / a;
}

// Largest |eigenvalue| of a small symmetric matrix by bisection on the inertia
// of T - sigma I (Sylvester's law: the number of negative pivots of Gaussian
// elimination without pivoting equals the number of eigenvalues below sigma).
__device__ int count_below(const double *T, int m, double sigma) {
  double a[8][8];
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) a[r][c] = T[r * m + c] - (r == c ? sigma : 0.0);
  int neg = 0;
  for (int k = 0; k < m; ++k) {
    double piv = a[k][k];
    if (piv == 0.0) piv = 1e-300;  // sigma sits on an eigenvalue of a leading block
    if (piv < 0.0) neg++;
    for (int r = k + 1; r < m; ++r) {
      const double f = a[r][k] / piv;
      for (int c = k + 1; c < m; ++c) a[r][c] -= f * a[k][c];
    }
  }
  return neg;
}

// H: (m+1) x 8 Hessenberg from the Arnoldi loop, wn[j] = ||M q_j||.  Applies
// the breakdown rule (h_{j+1,j} <= 1e-12 ||M q_j|| ends the process after j+1
// steps), symmetrises the leading block and sets omega = (4/3)/rho.  One warp:
// multisection, every lane tests one of 32 points of the current interval, so
// each round narrows it 33-fold (12 rounds reach double precision).
__global__ void k_omega_from_H(const double *__restrict__ H, const double *__restrict__ wn, int m,
                               double *__restrict__ omega_out) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int mm = m;
  for (int j = 0; j < m; ++j)
    if (H[(j + 1) * 8 + j] <= 1e-12 * wn[j] || j + 1 == m) {
      mm = j + 1;
      break;
    }
  double T[64];
  double g = 0.0;
  for (int a = 0; a < mm; ++a) {
    double rs = 0.0;
    for (int b = 0; b < mm; ++b) {
      T[a * mm + b] = 0.5 * (H[a * 8 + b] + H[b * 8 + a]);
      rs += fabs(T[a * mm + b]);
    }
    g = fmax(g, rs);
  }
  g = g * (1.0 + 1e-12) + 1e-300;
  double ext[2];
  for (int side = 0; side < 2; ++side) {
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
__global__ void k_dense_from_csr(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const double *__restrict__ val, double *__restrict__ A) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t p = rp[i]; p < rp[i + 1]; ++p) A[(int64_t)i * n + ci[p]] = val[p];
}

// In-place dense Cholesky (lower) by one thread block, then the inverse
// A^-1 = L^-T L^-1 column by column (one thread per column).
__global__ void k_cholesky_inverse(int32_t n, double *__restrict__ A, double *__restrict__ Ainv,
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

__global__ void k_fill_f64(int64_t n, double *p, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ============================================================== host side
namespace {

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

Coarsening coarsen_level(Hierarchy &h, int k, cudaStream_t s, int32_t *agg_out) {
  Level &L = h.lev[k];
  const int32_t n = L.n;
  const int64_t nnz = L.nnz;
  const unsigned gb = blocks_for(n);
  DevBuf<uint8_t> C(nnz);
  DevBuf<int32_t> rowcnt(n + 1), colcnt(n + 1), deg(n + 1), off(n + 1), cursor(n + 1);
  AMG_CUDA(cudaMemsetAsync(colcnt.p, 0, sizeof(int32_t) * (n + 1), s));
  AMG_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * (n + 1), s));
  AMG_COUNT(), k_strength<<<grid_for(n, 256), 256, 0, s>>>(n, L.rp, L.ci, L.val, h.p.alpha, C.p, rowcnt.p, colcnt.p);
  AMG_LAUNCH_CHECK();
  AMG_COUNT(), k_add_i32<<<gb, 256, 0, s>>>(n, rowcnt.p, colcnt.p, deg.p);
  int32_t total = 0;
  exclusive_scan<int32_t, int32_t>(deg.p, off.p, n, s, &total);
  DevBuf<int32_t> tmp((size_t)total + 1), ucount(n + 1), Sptr(n + 1);
  AMG_COUNT(), k_sym_fill<<<grid_for(n, 256), 256, 0, s>>>(n, L.rp, L.ci, C.p, rowcnt.p, off.p, cursor.p, tmp.p);
  AMG_LAUNCH_CHECK();
  AMG_COUNT(), k_sort_unique<<<grid_for(n, 128), 128, 0, s>>>(n, off.p, tmp.p, ucount.p);
  AMG_LAUNCH_CHECK();
  int32_t ns = 0;
  exclusive_scan<int32_t, int32_t>(ucount.p, Sptr.p, n, s, &ns);
  DevBuf<int32_t> Scol((size_t)ns + 1);
  AMG_COUNT(), k_compact<<<grid_for(n, 256), 256, 0, s>>>(n, off.p, tmp.p, Sptr.p, Scol.p);
  AMG_LAUNCH_CHECK();

  // PMIS(2)
  DevBuf<uint64_t> key(n), Tw(n);
  DevBuf<int32_t> Ti(n), und(1);
  DevBuf<int8_t> st(n);
  AMG_COUNT(), k_mis_keys<<<gb, 256, 0, s>>>(n, colcnt.p, h.p.seed, k, key.p, st.p);
  AMG_LAUNCH_CHECK();
  Coarsening out;
  for (int round = 0; round < 100000; ++round) {
    AMG_CUDA(cudaMemsetAsync(und.p, 0, sizeof(int32_t), s));
    AMG_COUNT(), k_pmis_max1<<<grid_for(n, 256), 256, 0, s>>>(n, Sptr.p, Scol.p, st.p, key.p, Tw.p, Ti.p);
    AMG_COUNT(), k_pmis_max2_decide<<<grid_for(n, 256), 256, 0, s>>>(n, Sptr.p, Scol.p, Tw.p, Ti.p, st.p, und.p);
    AMG_LAUNCH_CHECK();
    out.rounds = round + 1;
    if (read_scalar(und.p, s) == 0) break;
  }
  // aggregation
  DevBuf<int32_t> r1(n), r2(n), isroot(n + 1), cid(n + 1), err(1);
  AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  AMG_COUNT(), k_agg_pass1<<<grid_for(n, 256), 256, 0, s>>>(n, Sptr.p, Scol.p, st.p, key.p, r1.p);
  AMG_COUNT(), k_agg_pass2<<<grid_for(n, 256), 256, 0, s>>>(n, Sptr.p, Scol.p, st.p, key.p, r1.p, r2.p, isroot.p);
  AMG_LAUNCH_CHECK();
  int32_t nc = 0;
  exclusive_scan<int32_t, int32_t>(isroot.p, cid.p, n, s, &nc);
  AMG_COUNT(), k_agg_final<<<gb, 256, 0, s>>>(n, r2.p, cid.p, agg_out, err.p);
  AMG_LAUNCH_CHECK();
  if (read_scalar(err.p, s) != 0) throw Error{AMG_ERR_SETUP, "aggregation left a node unassigned"};
  out.nc = nc;
  return out;
}

void build_solve_matrix(Hierarchy &h, Level &L, cudaStream_t s) {
  const int32_t n = L.n;
  L.nslices = (n + kSlice - 1) / kSlice;
  DevBuf<int64_t> w32(L.nslices + 1);
  AMG_COUNT(), k_slice_width<<<blocks_for((int64_t)L.nslices * 32), 256, 0, s>>>(n, L.nslices, L.rp, w32.p);
  AMG_LAUNCH_CHECK();
  L.sptr = h.arena.get<int64_t>(L.nslices + 1);
  int64_t entries = 0;
  exclusive_scan<int64_t, int64_t>(w32.p, L.sptr, L.nslices, s, &entries);
  L.sell_entries = entries;
  L.scol = h.arena.get<int32_t>(entries);
  const unsigned g = blocks_for((int64_t)L.nslices * 32);
  switch (h.p.precision) {
    case AMG_PREC_F64:
      L.sval = h.arena.get<double>(entries);
      AMG_COUNT(), k_build_sell<double><<<g, 256, 0, s>>>(n, L.nslices, L.rp, L.ci, L.val, L.sptr, L.scol, (double *)L.sval);
      break;
    case AMG_PREC_F32:
      L.sval = h.arena.get<float>(entries);
      AMG_COUNT(), k_build_sell<float><<<g, 256, 0, s>>>(n, L.nslices, L.rp, L.ci, L.val, L.sptr, L.scol, (float *)L.sval);
      break;
    default:
      L.sval = h.arena.get<__nv_bfloat16>(entries);
      AMG_COUNT(), k_build_sell<__nv_bfloat16><<<g, 256, 0, s>>>(n, L.nslices, L.rp, L.ci, L.val, L.sptr, L.scol,
                                                   (__nv_bfloat16 *)L.sval);
  }
  AMG_LAUNCH_CHECK();
  if (&L == &h.lev[0] && h.p.precision != AMG_PREC_F64) {
    L.sval64 = h.arena.get<double>(entries);
    AMG_COUNT(), k_build_sell<double><<<g, 256, 0, s>>>(n, L.nslices, L.rp, L.ci, L.val, L.sptr, L.scol, L.sval64);
    AMG_LAUNCH_CHECK();
  } else if (&L == &h.lev[0]) {
    L.sval64 = (double *)L.sval;
  }
}

// omega of Eq. (damped Jacobi) from m = 5 Arnoldi steps on D^-1/2 A D^-1/2
double estimate_omega(Hierarchy &h, int k, const double *diag, cudaStream_t s) {
  Level &L = h.lev[k];
  const int32_t n = L.n;
  const int m = n < 5 ? n : 5;
  DevBuf<double> Q((size_t)n * (m + 1)), w(n), dh(n), part(kRedBlocks), H(9 * 8), wn(8), om(1), tmp(2);
  AMG_CUDA(cudaMemsetAsync(H.p, 0, sizeof(double) * 72, s));
  const unsigned gb = blocks_for(n);
  const int gr = grid_for(n, 256, kRedBlocks);
  AMG_COUNT(), k_arnoldi_start<<<gb, 256, 0, s>>>(n, h.p.seed, k, diag, Q.p, dh.p);
  AMG_COUNT(), k_dot_part<<<gr, 256, 0, s>>>(n, Q.p, Q.p, part.p);
  AMG_COUNT(), k_fin_sum<<<1, 1024, 0, s>>>(part.p, gr, tmp.p, 1);
  AMG_COUNT(), k_div_dev<<<grid_for(n, 256), 256, 0, s>>>(n, Q.p, Q.p, tmp.p);
  AMG_LAUNCH_CHECK();
  for (int j = 0; j < m; ++j) {
    const double *qj = Q.p + (size_t)j * n;
    AMG_COUNT(), k_scaled_spmv<<<grid_for(n, 256), 256, 0, s>>>(n, L.rp, L.ci, L.val, dh.p, qj, w.p);
    AMG_COUNT(), k_dot_part<<<gr, 256, 0, s>>>(n, w.p, w.p, part.p);
    AMG_COUNT(), k_fin_sum<<<1, 1024, 0, s>>>(part.p, gr, wn.p + j, 1);
    for (int l = 0; l <= j; ++l) {  // modified Gram-Schmidt
      const double *ql = Q.p + (size_t)l * n;
      AMG_COUNT(), k_dot_part<<<gr, 256, 0, s>>>(n, ql, w.p, part.p);
      AMG_COUNT(), k_fin_sum<<<1, 1024, 0, s>>>(part.p, gr, H.p + l * 8 + j, 0);
      AMG_COUNT(), k_axpy_neg_dev<<<grid_for(n, 256), 256, 0, s>>>(n, w.p, ql, H.p + l * 8 + j);
    }
    AMG_COUNT(), k_dot_part<<<gr, 256, 0, s>>>(n, w.p, w.p, part.p);
    AMG_COUNT(), k_fin_sum<<<1, 1024, 0, s>>>(part.p, gr, H.p + (j + 1) * 8 + j, 1);
    if (j + 1 < m) AMG_COUNT(), k_div_dev<<<grid_for(n, 256), 256, 0, s>>>(n, Q.p + (size_t)(j + 1) * n, w.p, H.p + (j + 1) * 8 + j);
    AMG_LAUNCH_CHECK();
  }
  AMG_COUNT(), k_omega_from_H<<<1, 32, 0, s>>>(H.p, wn.p, m, om.p);
  AMG_LAUNCH_CHECK();
  return read_scalar(om.p, s);
}

}  // namespace

void build_hierarchy(Hierarchy &h, const amg_csr &A, cudaStream_t s) {
  const amg_params &p = h.p;
  const int32_t n = A.n;
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
    AMG_COUNT(), k_check_csr<<<blocks_for(n), 256, 0, s>>>(n, A.nnz, L0.rp, L0.ci, L0.val, err.p);
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
  AMG_COUNT(), k_fill_f64<<<grid_for(n, 256), 256, 0, s>>>(n, L0.B, 1.0);  // B_0 = 1
  AMG_LAUNCH_CHECK();

  // ---- Alg. 1: coarsen until the level is small
  int k = 0;
  for (;;) {
    Level &L = h.lev[k];
    if (L.n <= p.coarse_max || k + 1 >= p.max_levels || k + 1 >= kMaxLevels) break;
    int32_t *agg = h.arena.get<int32_t>(L.n);
    Coarsening cr = coarsen_level(h, k, s, agg);
    L.mis_rounds = cr.rounds;
    if (10LL * cr.nc >= 9LL * L.n) break;  // coarsening stalled: this level is the coarsest
    const int32_t nc = cr.nc;
    L.agg = agg;
    L.nc = nc;
    // members of every aggregate, ascending
    L.aptr = h.arena.get<int32_t>((size_t)nc + 1);
    L.amem = h.arena.get<int32_t>(L.n);
    {
      DevBuf<int32_t> cnt(nc + 1), cur(nc + 1);
      AMG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (nc + 1), s));
      AMG_CUDA(cudaMemsetAsync(cur.p, 0, sizeof(int32_t) * (nc + 1), s));
      AMG_COUNT(), k_count_members<<<blocks_for(L.n), 256, 0, s>>>(L.n, agg, cnt.p);
      exclusive_scan<int32_t, int32_t>(cnt.p, L.aptr, nc, s);
      AMG_COUNT(), k_fill_members<<<blocks_for(L.n), 256, 0, s>>>(L.n, agg, L.aptr, cur.p, L.amem);
      AMG_COUNT(), k_sort_members<<<grid_for(nc, 128), 128, 0, s>>>(nc, L.aptr, L.amem);
      AMG_LAUNCH_CHECK();
    }
    Level &Cl = h.lev[k + 1];
    Cl.n = nc;
    Cl.B = h.arena.get<double>(nc);
    L.pw64 = h.arena.get<double>(L.n);
    AMG_COUNT(), k_interp<<<grid_for(nc, 128), 128, 0, s>>>(nc, L.aptr, L.amem, L.B, Cl.B, L.pw64);
    AMG_LAUNCH_CHECK();
    // Galerkin keyed sum: count, offsets, fill
    Cl.rp = h.arena.get<int32_t>((size_t)nc + 1);
    {
      DevBuf<int32_t> ccount(nc + 1);
      const int gw = grid_for((int64_t)nc * 32, 256, 152 * 64);
      AMG_COUNT(), k_galerkin<false><<<gw, 256, 0, s>>>(nc, L.aptr, L.amem, L.rp, L.ci, L.val, agg, L.pw64, ccount.p,
                                          nullptr, nullptr, nullptr);
      AMG_LAUNCH_CHECK();
      int32_t cnnz = 0;
      exclusive_scan<int32_t, int32_t>(ccount.p, Cl.rp, nc, s, &cnnz);
      Cl.nnz = cnnz;
      Cl.ci = h.arena.get<int32_t>(cnnz);
      Cl.val = h.arena.get<double>(cnnz);
      AMG_COUNT(), k_galerkin<true><<<gw, 256, 0, s>>>(nc, L.aptr, L.amem, L.rp, L.ci, L.val, agg, L.pw64, nullptr, Cl.rp,
                                         Cl.ci, Cl.val);
      AMG_LAUNCH_CHECK();
    }
    ++k;
  }
  h.L = k + 1;

  // ---- solve-phase data of every level
  for (int q = 0; q < h.L; ++q) {
    Level &L = h.lev[q];
    build_solve_matrix(h, L, s);
    DevBuf<double> diag(L.n);
    AMG_COUNT(), k_diag<<<blocks_for(L.n), 256, 0, s>>>(L.n, L.rp, L.ci, L.val, diag.p);
    AMG_LAUNCH_CHECK();
    if (q < h.L - 1) L.omega = p.omega_mode == 0 ? estimate_omega(h, q, diag.p, s) : p.omega;
    make_row_data(h, L, diag.p, s);  // per-row smoother data in the vector type
  }

  // ---- coarsest level: dense factorisation and inverse
  Level &Lc = h.lev[h.L - 1];
  if (Lc.n > kMaxDense)
    throw Error{AMG_ERR_SETUP, "coarsest level has " + std::to_string(Lc.n) + " unknowns (limit " +
                                   std::to_string(kMaxDense) + "); coarsening stalled"};
  h.nL = Lc.n;
  h.coarse_inv = h.arena.get<double>((size_t)Lc.n * Lc.n);
  {
    DevBuf<double> dense((size_t)Lc.n * Lc.n);
    DevBuf<int> err(1);
    AMG_CUDA(cudaMemsetAsync(dense.p, 0, sizeof(double) * (size_t)Lc.n * Lc.n, s));
    AMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    AMG_COUNT(), k_dense_from_csr<<<blocks_for(Lc.n), 256, 0, s>>>(Lc.n, Lc.rp, Lc.ci, Lc.val, dense.p);
    AMG_COUNT(), k_cholesky_inverse<<<1, 1024, 0, s>>>(Lc.n, dense.p, h.coarse_inv, err.p);
    AMG_LAUNCH_CHECK();
    if (read_scalar(err.p, s)) throw Error{AMG_ERR_SETUP, "coarsest level matrix is not positive definite"};
  }
}

}  // namespace amg
