// learned.cu -- learned per-row polynomial smoother: features, MLP inference
// and training kernels, and the two-grid error-reduction gradient that the
// training minimises.  The paper lists polynomial smoothers as future work
// (Sec. 5); the network and its training are this library's own.
//
// MLP: 16 -> 64 -> 64 -> 3, tanh, FP16 weights.  Inference runs the three
// layers on the tensor cores (mma.sync, FP16 operands with FP32 accumulation,
// activations as two FP16 parts); training keeps FP32 master weights on the
// CUDA cores.  Coefficients: c_q = omega_k (delta_q0 + o_q).  The weight
// gradients are deterministic fixed-order sums over rows.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "amg_internal.cuh"

namespace amg {

constexpr int NF = 16, NH = 64, NO = 3;
constexpr int W1O = 0, B1O = NH * NF, W2O = B1O + NH, B2O = W2O + NH * NH, W3O = B2O + NH, B3O = W3O + NO * NH;
constexpr int NP = B3O + NO;
static_assert(NP == AMG_MLP_NPARAM, "parameter layout");

// ------------------------------------------------------------------ features
// Row i, d = |A_ii|, t_j = -A_ij / d (j != i):
//  0: 1   1: #off/8   2..9: eight largest |A_ij|/d descending   10: fraction of
//  off-diagonals with the sign of A_ii   11: (sum_j A_ij)/A_ii   12: level/4
//  13: min t_j   14: max t_j   15: sum |A_ij|/d.  Sums in CSR order, IEEE
//  division and addition only: identical to a sequential evaluation.
__global__ void k_features(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, int32_t level, float *__restrict__ feat) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double aii = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) aii = val[p];
    const double d = fabs(aii);
    double top[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double rowsum = 0.0, abssum = 0.0, tmin = 0.0, tmax = 0.0;
    int32_t noff = 0, nsame = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      const double v = val[p];
      rowsum = __dadd_rn(rowsum, v);
      if (ci[p] == i) continue;
      const double a = __ddiv_rn(fabs(v), d), t = __ddiv_rn(-v, d);
      abssum = __dadd_rn(abssum, a);
      if (noff == 0 || t < tmin) tmin = t;
      if (noff == 0 || t > tmax) tmax = t;
      if ((v > 0.0 && aii > 0.0) || (v < 0.0 && aii < 0.0)) nsame++;
      noff++;
#pragma unroll
      for (int k = 0; k < 8; ++k) {  // insertion into the descending list
        if (a > top[k]) {
          for (int q = 7; q > k; --q) top[q] = top[q - 1];
          top[k] = a;
          break;
        }
      }
    }
    float *f = feat + (size_t)i * NF;
    f[0] = 1.0f;
    f[1] = (float)__ddiv_rn((double)noff, 8.0);
    for (int k = 0; k < 8; ++k) f[2 + k] = (float)top[k];
    f[10] = noff ? (float)__ddiv_rn((double)nsame, (double)noff) : 0.0f;
    f[11] = (float)__ddiv_rn(rowsum, aii);
    f[12] = (float)__ddiv_rn((double)level, 4.0);
    f[13] = (float)tmin;
    f[14] = (float)tmax;
    f[15] = (float)abssum;
  }
}

// ------------------------------------------------------------------ MLP forward
template <class WT>
__device__ __forceinline__ float wload(const WT *w, int k);
template <> __device__ __forceinline__ float wload<__half>(const __half *w, int k) { return __half2float(w[k]); }
template <> __device__ __forceinline__ float wload<float>(const float *w, int k) { return w[k]; }

// out = MLP(feat); optional caches of the hidden activations for training
template <class WT>
__global__ void __launch_bounds__(256) k_mlp_forward(int32_t n, const WT *__restrict__ wg,
                                                      const float *__restrict__ feat, float *__restrict__ out,
                                                      float *__restrict__ h1c, float *__restrict__ h2c) {
  __shared__ float w[NP];
  for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = wload<WT>(wg, k);
  __syncthreads();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float f[NF], h1[NH];
#pragma unroll
    for (int k = 0; k < NF; ++k) f[k] = feat[(size_t)i * NF + k];
#pragma unroll 4
    for (int u = 0; u < NH; ++u) {
      float z = w[B1O + u];
#pragma unroll
      for (int k = 0; k < NF; ++k) z = fmaf(w[W1O + u * NF + k], f[k], z);
      h1[u] = tanhf(z);
      if (h1c) h1c[(size_t)i * NH + u] = h1[u];
    }
    float o0 = w[B3O], o1 = w[B3O + 1], o2 = w[B3O + 2];
    for (int v = 0; v < NH; ++v) {
      float z = w[B2O + v];
#pragma unroll
      for (int u = 0; u < NH; ++u) z = fmaf(w[W2O + v * NH + u], h1[u], z);
      const float h2 = tanhf(z);
      if (h2c) h2c[(size_t)i * NH + v] = h2;
      o0 = fmaf(w[W3O + v], h2, o0);
      o1 = fmaf(w[W3O + NH + v], h2, o1);
      o2 = fmaf(w[W3O + 2 * NH + v], h2, o2);
    }
    out[(size_t)i * NO] = o0;
    out[(size_t)i * NO + 1] = o1;
    out[(size_t)i * NO + 2] = o2;
  }
}

// ------------------------------------------------------------------ MLP forward on tensor cores
// Inference with the FP16 weights as given: each warp takes 16 rows and runs the
// three layers as mma.sync m16n8k16 products (FP16 operands, FP32
// accumulation), the weights as B operands from shared memory.  An activation
// (FP32) enters as the sum of two FP16 parts, hi = fp16(h) and lo = fp16(h - hi),
// each multiplied by the exact FP16 weight and accumulated in FP32: about 22
// significant bits per product, so the outputs agree with the FP32 CUDA-core
// evaluation to FP32 rounding, where FP16 activations alone would lose three
// decimal digits.  The accumulator fragment of one layer (rows g, g+8; columns
// 2t, 2t+1 of each 8-column tile) is the A-operand fragment of the next, so the
// hidden activations never leave registers.
__device__ __forceinline__ uint32_t pack_h2(__half x, __half y) {
  __half2 v = __halves2half2(x, y);
  return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ void split_h2(float x, float y, uint32_t &hi, uint32_t &lo) {
  const __half xh = __float2half_rn(x), yh = __float2half_rn(y);
  hi = pack_h2(xh, yh);
  lo = pack_h2(__float2half_rn(x - __half2float(xh)), __float2half_rn(y - __half2float(yh)));
}
// c += A (16x16, row) * B (16x8, col)
__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kTcWarps = 4;
__global__ void __launch_bounds__(32 * kTcWarps) k_mlp_forward_tc(int32_t n, const __half *__restrict__ wg,
                                                                  const float *__restrict__ feat,
                                                                  float *__restrict__ out) {
  __shared__ __align__(16) __half w[NP + 1];
  __shared__ float bias[2 * NH + NO];
  for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = wg[k];
  for (int k = threadIdx.x; k < NH; k += blockDim.x) {
    bias[k] = __half2float(wg[B1O + k]);
    bias[NH + k] = __half2float(wg[B2O + k]);
  }
  if (threadIdx.x < NO) bias[2 * NH + threadIdx.x] = __half2float(wg[B3O + threadIdx.x]);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto wpair = [&](int idx) { return *reinterpret_cast<const uint32_t *>(&w[idx]); };
  for (int32_t tile = blockIdx.x * kTcWarps + (threadIdx.x >> 5); (int64_t)tile * 16 < n;
       tile += gridDim.x * kTcWarps) {
    const int32_t ra = tile * 16 + g, rb = ra + 8;
    // layer 1: A = features (16 x 16)
    uint32_t ah[4], al[4];
    {
      auto fv = [&](int32_t r, int k) { return r < n ? feat[(size_t)r * NF + k] : 0.0f; };
      split_h2(fv(ra, 2 * t), fv(ra, 2 * t + 1), ah[0], al[0]);
      split_h2(fv(rb, 2 * t), fv(rb, 2 * t + 1), ah[1], al[1]);
      split_h2(fv(ra, 2 * t + 8), fv(ra, 2 * t + 9), ah[2], al[2]);
      split_h2(fv(rb, 2 * t + 8), fv(rb, 2 * t + 9), ah[3], al[3]);
    }
    float c[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = 8 * nt + 2 * t;
      c[nt][0] = c[nt][2] = bias[col];
      c[nt][1] = c[nt][3] = bias[col + 1];
      const int wrow = W1O + (8 * nt + g) * NF + 2 * t;
      const uint32_t b0 = wpair(wrow), b1 = wpair(wrow + 8);
      mma_16816(c[nt], ah, b0, b1);
      mma_16816(c[nt], al, b0, b1);
    }
    // tanh, then the accumulators as the A operand of the next layer (4 k-tiles)
    uint32_t hh[4][4], hl[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      split_h2(tanhf(c[2 * kk][0]), tanhf(c[2 * kk][1]), hh[kk][0], hl[kk][0]);
      split_h2(tanhf(c[2 * kk][2]), tanhf(c[2 * kk][3]), hh[kk][1], hl[kk][1]);
      split_h2(tanhf(c[2 * kk + 1][0]), tanhf(c[2 * kk + 1][1]), hh[kk][2], hl[kk][2]);
      split_h2(tanhf(c[2 * kk + 1][2]), tanhf(c[2 * kk + 1][3]), hh[kk][3], hl[kk][3]);
    }
    // layer 2: 64 x 64
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = 8 * nt + 2 * t;
      c[nt][0] = c[nt][2] = bias[NH + col];
      c[nt][1] = c[nt][3] = bias[NH + col + 1];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int wrow = W2O + (8 * nt + g) * NH + 16 * kk + 2 * t;
        const uint32_t b0 = wpair(wrow), b1 = wpair(wrow + 8);
        mma_16816(c[nt], hh[kk], b0, b1);
        mma_16816(c[nt], hl[kk], b0, b1);
      }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      split_h2(tanhf(c[2 * kk][0]), tanhf(c[2 * kk][1]), hh[kk][0], hl[kk][0]);
      split_h2(tanhf(c[2 * kk][2]), tanhf(c[2 * kk][3]), hh[kk][1], hl[kk][1]);
      split_h2(tanhf(c[2 * kk + 1][0]), tanhf(c[2 * kk + 1][1]), hh[kk][2], hl[kk][2]);
      split_h2(tanhf(c[2 * kk + 1][2]), tanhf(c[2 * kk + 1][3]), hh[kk][3], hl[kk][3]);
    }
    // layer 3: 3 outputs in the first 8-column tile (columns 3..7 zero)
    float o[4];
    o[0] = o[2] = 2 * t < NO ? bias[2 * NH + 2 * t] : 0.0f;
    o[1] = o[3] = 2 * t + 1 < NO ? bias[2 * NH + 2 * t + 1] : 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int wrow = W3O + g * NH + 16 * kk + 2 * t;
      const uint32_t b0 = g < NO ? wpair(wrow) : 0u, b1 = g < NO ? wpair(wrow + 8) : 0u;
      mma_16816(o, hh[kk], b0, b1);
      mma_16816(o, hl[kk], b0, b1);
    }
    if (ra < n) {
      if (2 * t < NO) out[(size_t)ra * NO + 2 * t] = o[0];
      if (2 * t + 1 < NO) out[(size_t)ra * NO + 2 * t + 1] = o[1];
    }
    if (rb < n) {
      if (2 * t < NO) out[(size_t)rb * NO + 2 * t] = o[2];
      if (2 * t + 1 < NO) out[(size_t)rb * NO + 2 * t + 1] = o[3];
    }
  }
}

// per-row backward: dz2 = (W3^T dout) * (1 - h2^2), dz1 = (W2^T dz2) * (1 - h1^2)
__global__ void __launch_bounds__(256) k_mlp_backward_rows(int32_t n, const float *__restrict__ wg,
                                                            const float *__restrict__ dout,
                                                            const float *__restrict__ h1c,
                                                            const float *__restrict__ h2c,
                                                            float *__restrict__ dz1, float *__restrict__ dz2) {
  __shared__ float w[NP];
  for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = wg[k];
  __syncthreads();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g0 = dout[(size_t)i * NO], g1 = dout[(size_t)i * NO + 1], g2 = dout[(size_t)i * NO + 2];
    float d2[NH];
#pragma unroll 8
    for (int v = 0; v < NH; ++v) {
      const float h2 = h2c[(size_t)i * NH + v];
      const float dh = w[W3O + v] * g0 + w[W3O + NH + v] * g1 + w[W3O + 2 * NH + v] * g2;
      d2[v] = dh * (1.0f - h2 * h2);
      dz2[(size_t)i * NH + v] = d2[v];
    }
    for (int u = 0; u < NH; ++u) {
      float dh = 0.0f;
#pragma unroll
      for (int v = 0; v < NH; ++v) dh = fmaf(w[W2O + v * NH + u], d2[v], dh);
      const float h1 = h1c[(size_t)i * NH + u];
      dz1[(size_t)i * NH + u] = dh * (1.0f - h1 * h1);
    }
  }
}

// partial[chunk][a][b] = sum over the rows of the chunk of A[r][a] * B[r][b]
// (B == nullptr: B[r][b] = 1, for the bias gradients); FP64 accumulation
constexpr int kGradChunks = 64;
__global__ void k_outer_partial(int32_t n, const float *__restrict__ A, int na, const float *__restrict__ B, int nb,
                                double *__restrict__ partial) {
  const int32_t chunk = blockIdx.x;
  const int32_t r0 = (int32_t)((int64_t)n * chunk / kGradChunks), r1 = (int32_t)((int64_t)n * (chunk + 1) / kGradChunks);
  const int nout = na * (B ? nb : 1);
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int a = B ? o / nb : o, b = B ? o % nb : 0;
    double acc = 0.0;
    for (int32_t r = r0; r < r1; ++r) acc += (double)A[(size_t)r * na + a] * (B ? (double)B[(size_t)r * nb + b] : 1.0);
    partial[(size_t)chunk * nout + o] = acc;
  }
}

__global__ void k_sum_chunks(const double *__restrict__ partial, int nout, double *__restrict__ dst) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < kGradChunks; ++c) s += partial[(size_t)c * nout + o];
    dst[o] += s;
  }
}

__global__ void k_zero_f64(int n, double *p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0.0;
}

// Adam step on the FP32 master weights (bias-corrected), gradient in FP64
__global__ void k_adam(int np, float *__restrict__ w, const double *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, int t) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    const float gk = (float)g[k];
    m[k] = b1 * m[k] + (1.0f - b1) * gk;
    v[k] = b2 * v[k] + (1.0f - b2) * gk * gk;
    w[k] -= lr * (m[k] / c1) / (sqrtf(v[k] / c2) + eps);
  }
}

// c_q = omega (delta_q0 + o_q)
__global__ void k_coef_from_out(int32_t n, const float *__restrict__ out, double omega, double *__restrict__ coef) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x)
    coef[i] = omega * ((i % 3 == 0 ? 1.0 : 0.0) + (double)out[i]);
}

// dL/do_q = omega dL/dc_q
__global__ void k_dout_from_dcoef(int32_t n, const double *__restrict__ dcoef, double omega, float *__restrict__ dout) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x)
    dout[i] = (float)(omega * dcoef[i]);
}

// ------------------------------------------------------------------ two-grid loss
__device__ __forceinline__ uint64_t smix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// random error v: uniform in [-1, 1) from the splitmix64 counter (seed, v, i)
__global__ void k_tg_error(int32_t n, uint64_t seed, int32_t v, double *__restrict__ e) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t z = smix(seed ^ ((uint64_t)(uint32_t)(v + 1) << 44) ^ (uint64_t)(uint32_t)i);
    e[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  }
}

// y = s * (A x) (s = 1/A_ii per row when dscale, else 1), FP64 CSR, thread per row
__global__ void k_csr_spmv(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
                           const double *__restrict__ dscale) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) acc += val[p] * x[ci[p]];
    y[i] = dscale ? dscale[i] * acc : acc;
  }
}

// e1 = e0 - sum_q c_q u_q
__global__ void k_tg_smooth(int32_t n, const double *__restrict__ e0, const double *__restrict__ coef,
                            const double *__restrict__ u0, const double *__restrict__ u1,
                            const double *__restrict__ u2, double *__restrict__ e1) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    e1[i] = e0[i] - (coef[3 * i] * u0[i] + coef[3 * i + 1] * u1[i] + coef[3 * i + 2] * u2[i]);
}

// coarse correction of the error: rc = P^T (A e1), xc = A_c^-1 rc, e2 = e1 - P xc
__global__ void k_tg_restrict(int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
                              const double *__restrict__ pw, const double *__restrict__ r, double *__restrict__ rc) {
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t m = aptr[I]; m < aptr[I + 1]; ++m) s += pw[amem[m]] * r[amem[m]];
    rc[I] = s;
  }
}
__global__ void k_tg_dense(int32_t nc, const double *__restrict__ Ainv, const double *__restrict__ b,
                           double *__restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nc; i += gridDim.x * (blockDim.x >> 5)) {
    double s = 0.0;
    for (int32_t j = lane; j < nc; j += 32) s += Ainv[(int64_t)i * nc + j] * b[j];
    s = warp_sum(s);
    if (lane == 0) x[i] = s;
  }
}
__global__ void k_tg_prolong(int32_t n, const int32_t *__restrict__ agg, const double *__restrict__ pw,
                             const double *__restrict__ xc, double *__restrict__ e) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) e[i] -= pw[i] * xc[agg[i]];
}

// dcoef -= (2 / (nrm0 nvec)) (A e2)_i u_q,i   (nrm0 = e0^T A e0 from slot)
__global__ void k_tg_grad(int32_t n, const double *__restrict__ Ae2, const double *__restrict__ u0,
                          const double *__restrict__ u1, const double *__restrict__ u2, const double *__restrict__ nrm0,
                          int nvec, double *__restrict__ dcoef) {
  const double s = 2.0 / (*nrm0) / nvec;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double g = s * Ae2[i];
    dcoef[3 * i] -= g * u0[i];
    dcoef[3 * i + 1] -= g * u1[i];
    dcoef[3 * i + 2] -= g * u2[i];
  }
}

__global__ void k_inv_diag(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, double *__restrict__ dinv) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) d = val[p];
    dinv[i] = 1.0 / d;
  }
}

__global__ void k_scale_vec(int32_t n, const double *__restrict__ s, const double *__restrict__ x,
                            double *__restrict__ y) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = s[i] * x[i];
}

// deterministic dot: block partials then one block
__global__ void k_ldot_part(int32_t n, const double *__restrict__ a, const double *__restrict__ b,
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
__global__ void k_ldot_fin(const double *__restrict__ part, int nb, double *__restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) acc += part[k];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}
// loss += (e2^T A e2) / nrm0 / nvec
__global__ void k_tg_accum(const double *__restrict__ num, const double *__restrict__ nrm0, int nvec,
                           double *__restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *loss += (*num) / (*nrm0) / nvec;
}

// ------------------------------------------------------------------ host side
namespace {

inline int g256(int64_t n) { return grid_for(n, 256, 152 * 16); }

void dot_dev(int32_t n, const double *a, const double *b, double *out, double *part, cudaStream_t s) {
  const int nb = grid_for(n, 256, 1216);
  AMG_COUNT(), k_ldot_part<<<nb, 256, 0, s>>>(n, a, b, part);
  AMG_COUNT(), k_ldot_fin<<<1, 256, 0, s>>>(part, nb, out);
}

}  // namespace

// Two-grid loss and gradient on a two-level hierarchy (device coef / dcoef);
// loss_dev receives the mean factor.
void twogrid_loss(Hierarchy &h, const double *coef, int nvec, uint64_t seed, double *loss_dev, double *dcoef,
                  cudaStream_t s) {
  if (h.L != 2) throw Error{AMG_ERR_BAD_INPUT, "two-grid loss needs a hierarchy with exactly two levels"};
  Level &L = h.lev[0];
  const int32_t n = L.n, nc = h.lev[1].n;
  DevBuf<double> e0(n), Ae(n), u0(n), u1(n), u2(n), e1(n), dinv(n), rc(nc), xc(nc), part(1216), sc(4);
  AMG_COUNT(), k_zero_f64<<<1, 32, 0, s>>>(1, loss_dev);
  if (dcoef) AMG_COUNT(), k_zero_f64<<<g256(3 * (int64_t)n), 256, 0, s>>>(3 * n, dcoef);
  AMG_COUNT(), k_inv_diag<<<g256(n), 256, 0, s>>>(n, L.rp, L.ci, L.val, dinv.p);  // 1/A_ii in FP64
  for (int v = 0; v < nvec; ++v) {
    AMG_COUNT(), k_tg_error<<<g256(n), 256, 0, s>>>(n, seed, v, e0.p);
    AMG_COUNT(), k_csr_spmv<<<g256(n), 256, 0, s>>>(n, L.rp, L.ci, L.val, e0.p, Ae.p, nullptr);
    dot_dev(n, e0.p, Ae.p, sc.p, part.p, s);  // nrm0
    AMG_COUNT(), k_scale_vec<<<g256(n), 256, 0, s>>>(n, dinv.p, Ae.p, u0.p);
    AMG_COUNT(), k_csr_spmv<<<g256(n), 256, 0, s>>>(n, L.rp, L.ci, L.val, u0.p, u1.p, dinv.p);
    AMG_COUNT(), k_csr_spmv<<<g256(n), 256, 0, s>>>(n, L.rp, L.ci, L.val, u1.p, u2.p, dinv.p);
    AMG_COUNT(), k_tg_smooth<<<g256(n), 256, 0, s>>>(n, e0.p, coef, u0.p, u1.p, u2.p, e1.p);
    AMG_COUNT(), k_csr_spmv<<<g256(n), 256, 0, s>>>(n, L.rp, L.ci, L.val, e1.p, Ae.p, nullptr);
    AMG_COUNT(), k_tg_restrict<<<g256(nc), 256, 0, s>>>(nc, L.aptr, L.amem, L.pw64, Ae.p, rc.p);
    AMG_COUNT(), k_tg_dense<<<grid_for(nc, 8, 152 * 16), 256, 0, s>>>(nc, h.coarse_inv, rc.p, xc.p);
    AMG_COUNT(), k_tg_prolong<<<g256(n), 256, 0, s>>>(n, L.agg, L.pw64, xc.p, e1.p);
    AMG_COUNT(), k_csr_spmv<<<g256(n), 256, 0, s>>>(n, L.rp, L.ci, L.val, e1.p, Ae.p, nullptr);
    dot_dev(n, e1.p, Ae.p, sc.p + 1, part.p, s);  // e2^T A e2
    AMG_COUNT(), k_tg_accum<<<1, 32, 0, s>>>(sc.p + 1, sc.p, nvec, loss_dev);
    if (dcoef) AMG_COUNT(), k_tg_grad<<<g256(n), 256, 0, s>>>(n, Ae.p, u0.p, u1.p, u2.p, sc.p, nvec, dcoef);
  }
  AMG_LAUNCH_CHECK();
}

void features(const Hierarchy &h, int level, float *feat_dev, cudaStream_t s) {
  const Level &L = h.lev[level];
  AMG_COUNT(), k_features<<<g256(L.n), 256, 0, s>>>(L.n, L.rp, L.ci, L.val, level, feat_dev);
  AMG_LAUNCH_CHECK();
}

void mlp_forward_half(int32_t n, const uint16_t *w16_dev, const float *feat, float *out, cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = grid_for(((int64_t)n + 15) / 16, kTcWarps, 152 * 16);
  AMG_COUNT(), k_mlp_forward_tc<<<blocks, 32 * kTcWarps, 0, s>>>(n, reinterpret_cast<const __half *>(w16_dev), feat,
                                                                 out);
  AMG_LAUNCH_CHECK();
}

// dparam += d<dout, MLP_w(feat)>/dw  (FP32 weights, device)
void mlp_backward(int32_t n, const float *w, const float *feat, const float *dout, double *dparam, cudaStream_t s,
                  bool zero) {
  DevBuf<float> out(3 * (size_t)n), h1((size_t)n * NH), h2((size_t)n * NH), dz1((size_t)n * NH), dz2((size_t)n * NH);
  DevBuf<double> partial((size_t)kGradChunks * NH * NH);
  if (zero) AMG_COUNT(), k_zero_f64<<<g256(NP), 256, 0, s>>>(NP, dparam);
  AMG_COUNT(), k_mlp_forward<float><<<g256(n), 256, 0, s>>>(n, w, feat, out.p, h1.p, h2.p);
  AMG_COUNT(), k_mlp_backward_rows<<<g256(n), 256, 0, s>>>(n, w, dout, h1.p, h2.p, dz1.p, dz2.p);
  struct Term {
    const float *A;
    int na;
    const float *B;
    int nb;
    int off;
  };
  const Term terms[] = {{dz1.p, NH, feat, NF, W1O}, {dz1.p, NH, nullptr, 1, B1O}, {dz2.p, NH, h1.p, NH, W2O},
                        {dz2.p, NH, nullptr, 1, B2O}, {dout, NO, h2.p, NH, W3O},  {dout, NO, nullptr, 1, B3O}};
  for (const Term &t : terms) {
    const int nout = t.na * (t.B ? t.nb : 1);
    AMG_COUNT(), k_outer_partial<<<kGradChunks, 256, 0, s>>>(n, t.A, t.na, t.B, t.nb, partial.p);
    AMG_COUNT(), k_sum_chunks<<<grid_for(nout, 256, 64), 256, 0, s>>>(partial.p, nout, dparam + t.off);
  }
  AMG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ fixed scratch
// MLP backward for callers that cannot allocate device memory: the work arrays
// (hidden activations, their gradients and the per-chunk weight-gradient sums)
// live in one statically sized device array that every GPU loading this
// library holds until the process exits.  Rows per call are limited to
// kFixedMaxRows; calls that overlap on the GPU share the array and race.
constexpr int32_t kFixedMaxRows = 2048;
constexpr size_t kFixedFloats = (size_t)kFixedMaxRows * (NO + 4 * NH);                // out, h1, h2, dz1, dz2
constexpr size_t kFixedBytes = kFixedFloats * sizeof(float) + (size_t)kGradChunks * NH * NH * sizeof(double);
static_assert((kFixedFloats * sizeof(float)) % 256 == 0, "double section stays 256-byte aligned");
static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedBytes];

// Address of the array on the current device.  A host may not use the symbol
// itself as a device address, so every call asks the runtime for it with the
// device current: the lookup allocates nothing, the first one on a device loads
// the module that holds the array, and nothing cached can go stale when a
// context is reset and the array moves.
static void *fixed_scratch_address() {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_scratch);
  if (e != cudaSuccess)
    throw Error{AMG_ERR_CUDA, std::string("cudaGetSymbolAddress(fixed scratch): ") + cudaGetErrorString(e)};
  return p;
}

size_t fixed_scratch_bytes() { return kFixedBytes; }
int32_t fixed_scratch_max_rows() { return kFixedMaxRows; }

void mlp_backward_fixed(int32_t n, const float *w, const float *feat, const float *dout, double *dparam,
                        cudaStream_t s) {
  if (n < 0 || n > kFixedMaxRows)
    throw Error{AMG_ERR_BAD_INPUT, "amg_mlp_backward_noalloc: n = " + std::to_string(n) + " rows exceeds the " +
                                       std::to_string(kFixedMaxRows) + "-row limit of its fixed scratch"};
  float *base = static_cast<float *>(fixed_scratch_address());
  float *out = base, *h1 = out + (size_t)NO * kFixedMaxRows, *h2 = h1 + (size_t)NH * kFixedMaxRows;
  float *dz1 = h2 + (size_t)NH * kFixedMaxRows, *dz2 = dz1 + (size_t)NH * kFixedMaxRows;
  double *partial = reinterpret_cast<double *>(base + kFixedFloats);
  // every scratch word read below is written first in the same call; only the
  // output needs clearing
  k_zero_f64<<<g256(NP), 256, 0, s>>>(NP, dparam);
  if (n > 0) {
    k_mlp_forward<float><<<g256(n), 256, 0, s>>>(n, w, feat, out, h1, h2);
    k_mlp_backward_rows<<<g256(n), 256, 0, s>>>(n, w, dout, h1, h2, dz1, dz2);
    struct Term {
      const float *A;
      int na;
      const float *B;
      int nb;
      int off;
    };
    const Term terms[] = {{dz1, NH, feat, NF, W1O}, {dz1, NH, nullptr, 1, B1O}, {dz2, NH, h1, NH, W2O},
                          {dz2, NH, nullptr, 1, B2O}, {dout, NO, h2, NH, W3O},  {dout, NO, nullptr, 1, B3O}};
    for (const Term &t : terms) {
      const int nout = t.na * (t.B ? t.nb : 1);
      k_outer_partial<<<kGradChunks, 256, 0, s>>>(n, t.A, t.na, t.B, t.nb, partial);
      k_sum_chunks<<<grid_for(nout, 256, 64), 256, 0, s>>>(partial, nout, dparam + t.off);
    }
  }
  AMG_LAUNCH_CHECK();
}

// The network is trained on the two-grid factor of level 0 and installed there;
// coarser levels keep damped Jacobi.
void apply_learned(Hierarchy &h, const uint16_t *w16_dev, cudaStream_t s) {
  for (int k = 0; k < std::min(h.L - 1, 1); ++k) {
    Level &L = h.lev[k];
    DevBuf<float> feat((size_t)L.n * NF), out((size_t)L.n * NO);
    DevBuf<double> coef((size_t)L.n * 3);
    features(h, k, feat.p, s);
    mlp_forward_half(L.n, w16_dev, feat.p, out.p, s);
    AMG_COUNT(), k_coef_from_out<<<g256(3 * (int64_t)L.n), 256, 0, s>>>(L.n, out.p, L.omega, coef.p);
    AMG_LAUNCH_CHECK();
    set_poly(h, k, coef.p, s);
  }
  h.p.smoother = 1;
  h.graph_kind = -1;
}

// Adam training of the MLP on the level-0 two-grid factor of each hierarchy
void train_smoother(Hierarchy *const *hs, int nh, int steps, double lr, int nvec, uint64_t seed, float *w_host,
                    double *loss_hist, cudaStream_t s) {
  DevBuf<float> w(NP), m(NP), v(NP);
  DevBuf<double> grad(NP), loss(1);
  AMG_CUDA(cudaMemcpyAsync(w.p, w_host, sizeof(float) * NP, cudaMemcpyHostToDevice, s));
  AMG_CUDA(cudaMemsetAsync(m.p, 0, sizeof(float) * NP, s));
  AMG_CUDA(cudaMemsetAsync(v.p, 0, sizeof(float) * NP, s));
  std::vector<DevBuf<float> *> feats(nh);
  for (int j = 0; j < nh; ++j) {
    feats[j] = new DevBuf<float>((size_t)hs[j]->lev[0].n * NF);
    features(*hs[j], 0, feats[j]->p, s);
  }
  try {
    for (int t = 1; t <= steps; ++t) {
      AMG_COUNT(), k_zero_f64<<<g256(NP), 256, 0, s>>>(NP, grad.p);
      double step_loss = 0.0;
      for (int j = 0; j < nh; ++j) {
        Hierarchy &H = *hs[j];
        const int32_t n = H.lev[0].n;
        DevBuf<float> out((size_t)n * NO), dout((size_t)n * NO);
        DevBuf<double> coef((size_t)n * 3), dcoef((size_t)n * 3);
        AMG_COUNT(), k_mlp_forward<float><<<g256(n), 256, 0, s>>>(n, w.p, feats[j]->p, out.p, nullptr, nullptr);
        AMG_COUNT(), k_coef_from_out<<<g256(3 * (int64_t)n), 256, 0, s>>>(n, out.p, H.lev[0].omega, coef.p);
        twogrid_loss(H, coef.p, nvec, seed + (uint64_t)t * 1000003ull + (uint64_t)j, loss.p, dcoef.p, s);
        AMG_COUNT(), k_dout_from_dcoef<<<g256(3 * (int64_t)n), 256, 0, s>>>(n, dcoef.p, H.lev[0].omega / nh, dout.p);
        mlp_backward(n, w.p, feats[j]->p, dout.p, grad.p, s, false);
        double lv = 0.0;
        AMG_CUDA(cudaMemcpyAsync(&lv, loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        step_loss += lv / nh;
      }
      AMG_COUNT(), k_adam<<<g256(NP), 256, 0, s>>>(NP, w.p, grad.p, m.p, v.p, (float)lr, 0.9f, 0.999f, 1e-8f, t);
      AMG_LAUNCH_CHECK();
      if (loss_hist) loss_hist[t - 1] = step_loss;
    }
    AMG_CUDA(cudaMemcpyAsync(w_host, w.p, sizeof(float) * NP, cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    for (auto *f : feats) delete f;
    throw;
  }
  for (auto *f : feats) delete f;
}

}  // namespace amg
