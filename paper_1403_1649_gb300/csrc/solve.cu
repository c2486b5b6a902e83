// solve.cu -- solve phase of the aggregation AMG method on the GPU.
//
// Preconditioner: Alg. 5 (K-cycle) on levels k < kcycle_levels and Alg. 4
// (V-cycle) below (Sec. 2.2), one damped-Jacobi pre- and post-smoothing step
// per level visit (Eq. damped Jacobi), piecewise-constant restriction (a
// segmented sum over aggregates) and prolongation (a gather), and the exact
// coarsest solve as a dense matrix-vector product with the inverse formed at
// setup.  Outer iteration: flexible CG (Sec. 2.2) in FP64.
//
// Data-dependent control stays on the device.  The branch of Alg. 5
// (||r~|| <= t ||r||) is written to a per-level predicate by a one-block
// kernel; every kernel of the second inner step reads the predicate and returns
// at once when the step is not taken.  The Krylov scalars live in device
// memory, so an outer iteration is a fixed sequence of launches that can be
// captured once as a CUDA graph and replayed.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "amg_internal.cuh"

namespace amg {

// ============================================================== kernels
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// operands of the fused dot products of the SELL kernel
enum DotOp { OP_X = 0, OP_Y = 1, OP_U1 = 2, OP_U2 = 3 };

template <class VT>
struct SellArgs {
  int32_t n, nslices;
  const int64_t *sptr;
  const int32_t *scol;
  const void *sval;
  const int4 *spair;   // FP32 values: entries as {column, value} pairs (scol / sval null)
  const float *sdiag;  // split diagonal (reduced precision), else null
  const unsigned char *live;  // batch: 0 for slices whose systems all stopped (skipped); else null
  const VT *x;    // SpMV input
  VT *out;        // output vector
  const VT *rhs;  // right-hand side (residual / smoothing epilogues)
  const VT *wd;   // omega / A_ii
  const VT *xin;  // the iterate that the post-smoothing step updates
  const VT *u1, *u2;  // extra dot operands
  double *partials;   // ndot x kRedBlocks
  int ndot;
  int dop[3][2];
  const int *pred;
  // polynomial smoother operands
  const VT *dinv;     // 1 / A_ii
  const VT *coef;     // n x 3 per-row coefficients c_0, c_1, c_2
  const VT *p0, *p1;  // earlier polynomial terms
  const VT *res;      // residual the Horner steps add back
  VT *out2;           // second output
};

// epilogues of the SELL kernel (y = A x):
//   E_Y            out = y
//   E_RESID        out = rhs - y
//   E_POST         out = xin + wd (rhs - y)                  damped Jacobi after prolongation
//   E_DSCALE       out = D^-1 y                               polynomial pre-smoother, term 1
//   E_POLYPRE      out = c0 p0 + c1 p1 + c2 D^-1 y            polynomial pre-smoother, sum
//   E_RESID_POLY   out = rhs - y, out2 = D^-1 (c2 out)        post-smoother: residual, Horner start
//   E_HORNER       out = D^-1 y + D^-1 (c1 res)               Horner middle step
//   E_HORNER_LAST  out = xin + D^-1 y + D^-1 (c0 res)         Horner last step, update
enum Epi { E_Y = 0, E_RESID = 1, E_POST = 2, E_DSCALE = 3, E_POLYPRE = 4, E_RESID_POLY = 5, E_HORNER = 6,
           E_HORNER_LAST = 7 };

template <class MV> __device__ __forceinline__ MV ld_stream(const MV *p) { return __ldcs(p); }
// FP32 matrices are stored as {column, value} pairs (Level::spair); BF16
// matrices keep separate column and value arrays with a lane's entries 2j and
// 2j+1 adjacent in each (one 8-byte column load, one 4-byte value load)
template <class MV> constexpr bool kPairs = std::is_same<MV, float>::value;
template <class MV> constexpr bool kHalfPairs = std::is_same<MV, __nv_bfloat16>::value;

// per-block partial sums of up to three dot products -> partials[k*kRedBlocks + block]
__device__ __forceinline__ void block_store_dots3(double a0, double a1, double a2, int ndot, double *partials) {
  __shared__ double sh[3][kWarps];
  const double in[3] = {a0, a1, a2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < ndot) {
      const double v = warp_sum(in[k]);
      if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < ndot) {
        double v = threadIdx.x < kWarps ? sh[k][threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partials[k * kRedBlocks + blockIdx.x] = v;
      }
    }
  }
}

template <class VT>
__device__ __forceinline__ void block_store_dots(const double (&acc)[3], int ndot, double *partials) {
  block_store_dots3(acc[0], acc[1], acc[2], ndot, partials);
}

// y = A x over SELL-32 (one warp per slice, one lane per row) with an epilogue:
//   E_Y     out = A x
//   E_RESID out = rhs - A x
//   E_POST  out = xin + wd * (rhs - A x)   (damped Jacobi after prolongation)
// and up to three fused dot products of {x_i, y_i, u1_i, u2_i} pairs.
__device__ __forceinline__ double dot_operand(int op, double x, double y, double u1, double u2) {
  return op == OP_X ? x : (op == OP_Y ? y : (op == OP_U1 ? u1 : u2));
}

// batch: live[sl] = 1 when some system with rows in slice sl still iterates.
// Rows of a stopped system are only ever read by that system, so its work can
// be skipped; a restarted system starts again from its recomputed residual.
__global__ void k_slice_live(int32_t n, int32_t nslices, const int32_t *__restrict__ sys,
                             const int *__restrict__ bact, unsigned char *__restrict__ live) {
  pdl_wait_and_trigger();
  for (int32_t sl = blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += gridDim.x * blockDim.x) {
    unsigned char v = 0;
    for (int32_t q = sys[sl * 32]; q <= sys[min(sl * 32 + 31, n - 1)]; ++q)
      if (bact[q]) {
        v = 1;
        break;
      }
    live[sl] = v;
  }
}

// Resident blocks per SM of k_sell: FP32 vectors fit in 40 registers (6 blocks
// of 256 threads), FP64 vectors need 64 (4 blocks).
template <class VT>
constexpr int sell_min_blocks() { return sizeof(VT) == 4 ? 6 : 4; }

// DOTS: the launch fuses inner products (compiled only where used, so that the
// plain SpMV does not hold their accumulators in registers)
// GATE: a batch's launch, skipping slices whose systems have all stopped
// (compiled only into the batch instantiations)
// UW: entries a row per step on small levels (0: the default below).  A level of
// a few hundred slices leaves most of the GPU idle and each warp's chain of
// dependent loads sets the time, so there every load of a coarse row (15-30
// entries) goes out in one or two steps.
// With fused inner products the FP32-vector kernel needs more than the 40
// registers of six resident blocks (it spilled there): four blocks, 64 registers.
template <class MV, class VT, bool DOTS>
constexpr int sell_launch_blocks() { return DOTS ? 4 : sell_min_blocks<VT>(); }

template <class MV, class VT, int EPI, bool DOTS, bool GATE, int UW = 0>
__global__ void __launch_bounds__(kThreads, UW ? 1 : sell_launch_blocks<MV, VT, DOTS>()) k_sell(SellArgs<VT> a) {
  pdl_wait_and_trigger();
  if (a.pred && *a.pred == 0) return;
  const int lane = threadIdx.x & 31;
  const MV *__restrict__ sval = static_cast<const MV *>(a.sval);
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  // U entries of a row per step: 6 with FP32 vectors (a 7-point row without its
  // split-off diagonal in one step, at 40 registers), 8 with FP64
  constexpr int U = UW ? UW : (sizeof(VT) == 4 ? 6 : 8);
  for (int32_t sl = blockIdx.x * kWarps + (threadIdx.x >> 5); sl < a.nslices; sl += gridDim.x * kWarps) {
    if (GATE && !a.live[sl]) continue;
    const int32_t row = sl * 32 + lane;
    VT y = VT(0), dg = VT(0), xr = VT(0);
    const bool diag = !std::is_same<MV, double>::value && a.sdiag != nullptr && row < a.n;
    // small levels (UW): the row's own operands (split diagonal, x_row and the
    // epilogue's rhs, wd, xin) go out before the slice pointers, so that the
    // warp's chain of dependent loads is the matrix and the gathers only
    VT pre_rhs = VT(0), pre_wd = VT(0), pre_xin = VT(0);
    if constexpr (UW != 0) {
      if (diag) {
        dg = (VT)ld_stream(a.sdiag + row);
        xr = __ldg(a.x + row);
      }
      if (row < a.n) {
        if (EPI == E_RESID || EPI == E_POST) pre_rhs = __ldg(a.rhs + row);
        if (EPI == E_POST) {
          pre_wd = __ldg(a.wd + row);
          pre_xin = __ldg(a.xin + row);
        }
      }
    }
    const int64_t base = a.sptr[sl];
    const int32_t width = (int32_t)((a.sptr[sl + 1] - base) >> 5);
    // otherwise the split diagonal (FP32 / BF16 values only) and x_row are loaded
    // right behind the first step's matrix loads, so that their latency overlaps
    // the gathers
    if constexpr (kPairs<MV> || kHalfPairs<MV>) {
      // FP32 values: a lane's entries 2j and 2j+1 come in one 16-byte load;
      // BF16 values: their columns in one 8-byte load and their values in one
      // 4-byte load (widths are even, U is even).  FULL: all U entries exist
      static_assert(U % 2 == 0, "pairs need an even step");
      const int4 *__restrict__ pp = a.spair + (base >> 1) + lane;
      const int2 *__restrict__ cp2 = reinterpret_cast<const int2 *>(a.scol + base) + lane;
      const __nv_bfloat162 *__restrict__ vp2 = reinterpret_cast<const __nv_bfloat162 *>(sval + base) + lane;
      auto step = [&](int32_t e, auto full, auto size) {
        constexpr bool FULL = decltype(full)::value;
        constexpr int S = decltype(size)::value;  // entries of this step
        int32_t c[S];
        float v[S];
#pragma unroll
        for (int q = 0; q < S; q += 2) {
          if (FULL || e + q < width) {
            if constexpr (kPairs<MV>) {
              const int4 pr = ld_stream(pp + 16 * (e + q));
              c[q] = pr.x;
              v[q] = __int_as_float(pr.y);
              c[q + 1] = pr.z;
              v[q + 1] = __int_as_float(pr.w);
            } else {
              const int2 cc = ld_stream(cp2 + 16 * (e + q));
              const float2 vv = __bfloat1622float2(ld_stream(vp2 + 16 * (e + q)));
              c[q] = cc.x;
              c[q + 1] = cc.y;
              v[q] = vv.x;
              v[q + 1] = vv.y;
            }
          }
        }
        if (UW == 0 && e == 0 && diag) {
          dg = (VT)ld_stream(a.sdiag + row);
          xr = __ldg(a.x + row);
        }
        VT xv[S];
#pragma unroll
        for (int q = 0; q < S; ++q)
          if (FULL || e + q < width) xv[q] = __ldg(a.x + c[q]);
#pragma unroll
        for (int q = 0; q < S; ++q)
          if (FULL || e + q < width) y += v[q] * xv[q];
      };
      // a slice of U or U + 2 entries a row (a 7-point row, a P1 FEM row) takes
      // one step without predicates, whose loads all go out before the first gather
      using UStep = std::integral_constant<int, U>;
      using U2Step = std::integral_constant<int, U + 2>;
      if (UW == 0 && width == U) {
        step(0, std::true_type{}, UStep{});
      } else if (UW == 0 && width == U + 2) {
        step(0, std::true_type{}, U2Step{});
      } else {
        for (int32_t e = 0; e < width; e += U) step(e, std::false_type{}, UStep{});
      }
    } else {
      const int32_t *__restrict__ cp = a.scol + base + lane;
      const MV *__restrict__ vp = sval + base + lane;
      for (int32_t e = 0; e < width; e += U) {
        int32_t c[U];
        MV v[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          if (e + q < width) {
            c[q] = ld_stream(cp + 32 * (e + q));
            v[q] = ld_stream(vp + 32 * (e + q));
          }
        }
        if (UW == 0 && e == 0 && diag) {
          dg = (VT)ld_stream(a.sdiag + row);
          xr = __ldg(a.x + row);
        }
        VT xv[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (e + q < width) xv[q] = __ldg(a.x + c[q]);
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (e + q < width) y += to_acc(v[q], VT(0)) * xv[q];
      }
    }
    if (diag) {
      if (width == 0) {  // a row without off-diagonal entries
        dg = (VT)a.sdiag[row];
        xr = a.x[row];
      }
      y += dg * xr;
    }
    if (row < a.n) {
      VT o;
      if (EPI == E_Y) o = y;
      else if (EPI == E_RESID) o = (UW ? pre_rhs : a.rhs[row]) - y;
      else if (EPI == E_POST)
        o = UW ? pre_xin + pre_wd * (pre_rhs - y) : a.xin[row] + a.wd[row] * (a.rhs[row] - y);
      else if (EPI == E_DSCALE) o = a.dinv[row] * y;
      else if (EPI == E_POLYPRE)
        o = a.coef[3 * row] * a.p0[row] + a.coef[3 * row + 1] * a.p1[row] + a.coef[3 * row + 2] * (a.dinv[row] * y);
      else if (EPI == E_RESID_POLY) {
        o = a.rhs[row] - y;
        a.out2[row] = a.dinv[row] * (a.coef[3 * row + 2] * o);
      } else if (EPI == E_HORNER)
        o = a.dinv[row] * y + a.dinv[row] * (a.coef[3 * row + 1] * a.res[row]);
      else
        o = a.xin[row] + (a.dinv[row] * y + a.dinv[row] * (a.coef[3 * row] * a.res[row]));
      a.out[row] = o;
      if (DOTS && a.ndot) {
        const double ox = (double)a.x[row], oy = (double)o, o1 = a.u1 ? (double)a.u1[row] : 0.0,
                     o2 = a.u2 ? (double)a.u2[row] : 0.0;
        acc0 += dot_operand(a.dop[0][0], ox, oy, o1, o2) * dot_operand(a.dop[0][1], ox, oy, o1, o2);
        if (a.ndot > 1) acc1 += dot_operand(a.dop[1][0], ox, oy, o1, o2) * dot_operand(a.dop[1][1], ox, oy, o1, o2);
        if (a.ndot > 2) acc2 += dot_operand(a.dop[2][0], ox, oy, o1, o2) * dot_operand(a.dop[2][1], ox, oy, o1, o2);
      }
    }
  }
  if (DOTS && a.ndot) block_store_dots3(acc0, acc1, acc2, a.ndot, a.partials);
}

// out = wd * rhs: damped Jacobi from a zero initial guess
template <class VT>
__global__ void k_scale(int32_t n, VT *__restrict__ out, const VT *__restrict__ wd, const VT *__restrict__ rhs,
                        const int *pred, const int32_t *sys, const int *bact) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!bact || bact[sys[i]]) out[i] = wd[i] * rhs[i];
}

// sum_{i in G_I} P(i, I) r(i) over the members amem[m0..m1) in their (ascending) order
template <class VT>
__device__ __forceinline__ VT restrict_row(int32_t m0, int32_t m1, const int32_t *__restrict__ amem,
                                          const VT *__restrict__ pw, const VT *__restrict__ r) {
  VT s = VT(0);
  for (int32_t m = m0; m < m1; ++m) {
    const int32_t i = amem[m];
    s += pw[i] * r[i];
  }
  return s;
}

// r_{k+1}(I) = sum_{i in G_I} P(i, I) r_k(i) in ascending fine index; also the
// next level's smoothing start x0 = wd_{k+1} * r_{k+1} when that level smooths.
template <class VT>
__global__ void k_restrict(int32_t nc, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
                           const VT *__restrict__ pw, const VT *__restrict__ r, VT *__restrict__ bc,
                           const VT *__restrict__ wdc, VT *__restrict__ x0c, const int *pred,
                           const int32_t *sysc, const int *bact) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    if (bact && !bact[sysc[I]]) continue;
    const VT s = restrict_row(aptr[I], aptr[I + 1], amem, pw, r);
    bc[I] = s;
    if (wdc) x0c[I] = wdc[I] * s;
  }
}

// x_k += P_k x_{k+1}: a gather through the aggregate map
template <class VT>
__global__ void k_prolong(int32_t n, const int32_t *__restrict__ agg, const VT *__restrict__ pw,
                          const VT *__restrict__ xc, VT *__restrict__ x, const int *pred, const int32_t *sys,
                          const int *bact) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!bact || bact[sys[i]]) x[i] += pw[i] * xc[agg[i]];
}

// exact coarsest solve x = A_L^-1 b (one warp per row, FP64 accumulation)
template <class VT>
__global__ void k_coarse(int32_t nL, const double *__restrict__ Ainv, const VT *__restrict__ b, VT *__restrict__ x,
                         const VT *__restrict__ wdc_unused, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const int lane = threadIdx.x & 31;
  for (int32_t i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < nL; i += gridDim.x * kWarps) {
    double s = 0.0;
    for (int32_t j = lane; j < nL; j += 32) s += Ainv[(int64_t)i * nL + j] * (double)b[j];
    s = warp_sum(s);
    if (lane == 0) x[i] = (VT)s;
  }
}

// restriction to the coarsest level and its exact solve in one launch: every
// block forms r_L = R r (as k_restrict does) in shared memory, then its warps
// take rows of x = A_L^-1 r_L (as k_coarse does)
constexpr int kFusedCoarseMax = 2048;
template <class VT>
__global__ void k_restrict_coarse(int32_t nL, const int32_t *__restrict__ aptr, const int32_t *__restrict__ amem,
                                  const VT *__restrict__ pw, const VT *__restrict__ r, const double *__restrict__ Ainv,
                                  VT *__restrict__ x, const int *pred) {
  __shared__ VT bsh[kFusedCoarseMax];
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t I = threadIdx.x; I < nL; I += blockDim.x) bsh[I] = restrict_row(aptr[I], aptr[I + 1], amem, pw, r);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int32_t i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < nL; i += gridDim.x * kWarps) {
    double s = 0.0;
    for (int32_t j = lane; j < nL; j += 32) s += Ainv[(int64_t)i * nL + j] * (double)bsh[j];
    s = warp_sum(s);
    if (lane == 0) x[i] = (VT)s;
  }
}

// sum of the first nb partials of dot k, identical in every block
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int k, int nb) {
  __shared__ double sh[kWarps];
  __shared__ double result;
  double acc = 0.0;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) acc += part[k * kRedBlocks + j];
  acc = warp_sum(acc);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) result = v;
  }
  __syncthreads();
  return result;
}

// Alg. 5 after v = A c: rho_1 and alpha_1 (CG: c^T v, c^T r; GMRES: ||v||^2, v^T r)
__global__ void k_fin_k1(const double *__restrict__ part, int nb, double *__restrict__ slots, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const double rho1 = sum_partials(part, 0, nb);
  const double a1 = sum_partials(part, 1, nb);
  if (threadIdx.x == 0) {
    slots[S_RHO1] = rho1;
    slots[S_A1] = a1;
    slots[S_S1] = a1 / rho1;
  }
}

// r~ = r - (alpha_1/rho_1) v, with ||r~||^2, ||r||^2 partials and the next
// smoothing start x0 = wd * r~
template <class VT>
__global__ void k_axpy_rt(int32_t n, const VT *__restrict__ r, const VT *__restrict__ v, VT *__restrict__ rt,
                          const VT *__restrict__ wd, VT *__restrict__ x0, const double *__restrict__ slots,
                          double *__restrict__ part, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const VT s1 = (VT)slots[S_S1];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const VT ri = r[i];
    const VT t = ri - s1 * v[i];
    rt[i] = t;
    if (wd) x0[i] = wd[i] * t;
    acc[0] += (double)t * (double)t;
    acc[1] += (double)ri * (double)ri;
  }
  block_store_dots<VT>(acc, 2, part);
}

// the test of Alg. 5: the second inner step runs iff the enclosing step runs
// and ||r~|| > t ||r||.  Never predicated, so a skipped parent clears it.
__global__ void k_decide(const double *__restrict__ part, int nb, double *__restrict__ slots, double t,
                         const int *parent, int *__restrict__ flag) {
  pdl_wait_and_trigger();
  const double nrt2 = sum_partials(part, 0, nb);
  const double nr2 = sum_partials(part, 1, nb);
  if (threadIdx.x == 0) {
    const int active = parent ? *parent : 1;
    slots[S_NRT2] = nrt2;
    slots[S_NR2] = nr2;
    const bool accept_first = sqrt(nrt2) <= t * sqrt(nr2);
    *flag = (active && !accept_first) ? 1 : 0;
    if (active && !accept_first) slots[S_TAKEN] += 1.0;  // cycle trace (one thread)
  }
}

// Alg. 5 after w = A d: gamma, beta, alpha_2, rho_2 and the combination weights
__global__ void k_fin_k3(const double *__restrict__ part, int nb, double *__restrict__ slots, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const double gam = sum_partials(part, 0, nb);
  const double bet = sum_partials(part, 1, nb);
  const double a2 = sum_partials(part, 2, nb);
  if (threadIdx.x == 0) {
    const double rho1 = slots[S_RHO1];
    const double rho2 = bet - gam * gam / rho1;
    slots[S_GAM] = gam;
    slots[S_BET] = bet;
    slots[S_A2] = a2;
    slots[S_CC] = slots[S_S1] - gam * a2 / (rho1 * rho2);
    slots[S_CD] = a2 / rho2;
  }
}

// x_{k+1} = (alpha1/rho1) c, or the two-step combination when it was taken
template <class VT>
__global__ void k_combine(int32_t n, const VT *__restrict__ c, const VT *__restrict__ d, VT *__restrict__ x,
                          const double *__restrict__ slots, const int *__restrict__ flag, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const bool two = *flag != 0;
  const VT cc = (VT)(two ? slots[S_CC] : slots[S_S1]);
  const VT cd = (VT)(two ? slots[S_CD] : 0.0);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = two ? cc * c[i] + cd * d[i] : cc * c[i];
}

// ---------------------------------------------------------------- outer FCG (FP64)
template <class VT>
__global__ void k_to_vt(int32_t n, const double *__restrict__ in, VT *__restrict__ out, const VT *__restrict__ wd,
                        VT *__restrict__ x0, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const VT v = (VT)in[i];
    out[i] = v;
    x0[i] = wd[i] * v;
  }
}

// z = (double) zin, with the partials of z^T q
template <class VT>
__global__ void k_from_vt_dot(int32_t n, const VT *__restrict__ zin, double *__restrict__ z,
                              const double *__restrict__ q, double *__restrict__ part, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = (double)zin[i];
    z[i] = v;
    acc[0] += v * q[i];
  }
  block_store_dots<double>(acc, 1, part);
}

// p = z + beta p,  beta = -(z^T q_old)/(p_old^T q_old) (0 right after a restart)
__global__ void k_fcg_p(int32_t n, const double *__restrict__ z, double *__restrict__ p,
                        const double *__restrict__ part_zq, int nb, double *__restrict__ slots,
                        const int *__restrict__ restart, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const double zq = sum_partials(part_zq, 0, nb);
  const bool rs = *restart != 0;
  const double beta = rs ? 0.0 : -zq / slots[S_PQ];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    slots[S_ZQ] = zq;
    slots[S_BETA] = beta;
  }
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = rs ? z[i] : z[i] + beta * p[i];
}

// alpha = p^T r / p^T q;  x += alpha p;  r -= alpha q;  partials of ||r||^2.
// In reduced precision also the preconditioner input (VT) and its x0.
template <class VT>
__global__ void k_fcg_update(int32_t n, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                             const double *__restrict__ q, const double *__restrict__ part_pq, int nb,
                             double *__restrict__ slots, double *__restrict__ part_rr, VT *__restrict__ rvt,
                             const VT *__restrict__ wd, VT *__restrict__ x0, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const double pq = sum_partials(part_pq, 0, nb);
  const double pr = sum_partials(part_pq, 1, nb);
  const double alpha = pr / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    slots[S_PQ] = pq;
    slots[S_PR] = pr;
    slots[S_ALPHA] = alpha;
  }
  double acc[3] = {0.0, 0.0, 0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc[0] += ri * ri;
    if (rvt) {
      const VT v = (VT)ri;
      rvt[i] = v;
      x0[i] = wd[i] * v;
    }
  }
  block_store_dots<double>(acc, 1, part_rr);
}

// end of an outer iteration: relative residual into the history, iteration
// count, convergence / breakdown status; deactivates the following launches
__global__ void k_fcg_fin(const double *__restrict__ part_rr, int nb, double *__restrict__ slots,
                          double *__restrict__ hist, int *__restrict__ it, int *__restrict__ active,
                          int *__restrict__ restart, int *__restrict__ status) {
  pdl_wait_and_trigger();
  if (*active == 0) return;
  const double tol = slots[S_TOL];
  const int max_iter = (int)slots[S_MAXIT];
  const double rr = sum_partials(part_rr, 0, nb);
  if (threadIdx.x == 0) {
    const double rel = sqrt(rr) / sqrt(slots[S_NB2]);
    const int k = *it + 1;
    *it = k;
    hist[k] = rel;
    slots[S_RR] = rr;
    slots[S_REL] = rel;
    *restart = 0;
    if (!(slots[S_PQ] > 0.0)) {
      *status = AMG_ERR_BREAKDOWN;
      *active = 0;
    } else if (!isfinite(rel)) {
      *status = AMG_ERR_NAN;
      *active = 0;
    } else if (rel <= tol) {
      *status = 1;  // recursive residual converged: the host checks the true residual
      *active = 0;
    } else if (k >= max_iter) {
      *status = AMG_ERR_NOT_CONVERGED;
      *active = 0;
    }
  }
}

// block partial dot (generic)
__global__ void k_dot64(int32_t n, const double *__restrict__ a, const double *__restrict__ b,
                        double *__restrict__ part, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc[0] += a[i] * b[i];
  block_store_dots<double>(acc, 1, part);
}

__global__ void k_store_sum(const double *__restrict__ part, int nb, double *__restrict__ dst) {
  pdl_wait_and_trigger();
  const double v = sum_partials(part, 0, nb);
  if (threadIdx.x == 0) *dst = v;
}

// r = b - A x in FP64 (level-0 SELL with FP64 values), with ||r||^2 partials
__global__ void k_residual64(int32_t n, int32_t nslices, const int64_t *__restrict__ sptr,
                             const int32_t *__restrict__ scol, const double *__restrict__ sval,
                             const double *__restrict__ x, const double *__restrict__ b, double *__restrict__ r,
                             double *__restrict__ part) {
  pdl_wait_and_trigger();
  const int lane = threadIdx.x & 31;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int32_t sl = blockIdx.x * kWarps + (threadIdx.x >> 5); sl < nslices; sl += gridDim.x * kWarps) {
    const int64_t base = sptr[sl];
    const int32_t width = (int32_t)((sptr[sl + 1] - base) >> 5);
    double y = 0.0;
    for (int32_t e = 0; e < width; ++e) {
      const int64_t at = base + 32 * e + lane;
      y += sval[at] * x[scol[at]];
    }
    const int32_t row = sl * 32 + lane;
    if (row < n) {
      const double ri = b[row] - y;
      r[row] = ri;
      acc[0] += ri * ri;
    }
  }
  block_store_dots<double>(acc, 1, part);
}

// ---------------------------------------------------------------- outer FGMRES (FP64)
constexpr int kMaxRestart = 32;

// partial dot products of w with the basis vectors V_0..V_{ncol-1}, eight
// columns per sweep over the rows
__global__ void k_mdot(int32_t n, const double *__restrict__ V, int ncol, const double *__restrict__ w,
                       double *__restrict__ part, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  __shared__ double sh[kWarps][8];
  for (int c0 = 0; c0 < ncol; c0 += 8) {
    double acc[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) acc[l] = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (c0 + l < ncol) acc[l] += V[(int64_t)(c0 + l) * n + i] * wi;
    }
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const double v = warp_sum(acc[l]);
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][l] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8 && c0 + (int)threadIdx.x < ncol) {
      double v = 0.0;
      for (int wq = 0; wq < kWarps; ++wq) v += sh[wq][threadIdx.x];
      part[(int64_t)(c0 + threadIdx.x) * kRedBlocks + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

// h_l = sum of the partials of column l; H(l, j) += h_l; hc = h
__global__ void k_fin_mdot(const double *__restrict__ part, int nb, int ncol, double *__restrict__ H, int ldh,
                           int j, double *__restrict__ hc, int accumulate, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int l = wid; l < ncol; l += blockDim.x >> 5) {
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += part[(int64_t)l * kRedBlocks + b];
    v = warp_sum(v);
    if (lane == 0) {
      hc[l] = v;
      H[l * ldh + j] = accumulate ? H[l * ldh + j] + v : v;
    }
  }
}

// w -= sum_l hc_l V_l
__global__ void k_maxpy(int32_t n, const double *__restrict__ V, int ncol, const double *__restrict__ hc,
                        double *__restrict__ w, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  __shared__ double h[kMaxRestart + 1];
  for (int l = threadIdx.x; l < ncol; l += blockDim.x) h[l] = hc[l];
  __syncthreads();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double t = w[i];
    for (int l = 0; l < ncol; ++l) t -= h[l] * V[(int64_t)l * n + i];
    w[i] = t;
  }
}

// v_{j+1} = w / ||w||, H(j+1, j) = ||w||   (norm from the partials, same in every block)
__global__ void k_fg_normalize(int32_t n, const double *__restrict__ w, double *__restrict__ vnext,
                               const double *__restrict__ part, int nb, double *__restrict__ H, int ldh, int j,
                               const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const double nrm = sqrt(sum_partials(part, 0, nb));
  if (blockIdx.x == 0 && threadIdx.x == 0) H[(j + 1) * ldh + j] = nrm;
  const double inv = nrm != 0.0 ? 1.0 / nrm : 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) vnext[i] = w[i] * inv;
}

// Givens rotations on column j of H, residual estimate |g_{j+1}| / ||b||
// into the history; deactivates the following steps when done.
// fg[0..m] = g, fg[m+1..2m] = cos, fg[2m+1..3m] = sin
__global__ void k_fg_givens(double *__restrict__ H, int ldh, int j, int m, double *__restrict__ fg,
                            double *__restrict__ slots, double *__restrict__ hist, int *__restrict__ it,
                            int *__restrict__ active, int *__restrict__ status) {
  pdl_wait_and_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0 || *active == 0) return;
  double *g = fg, *cs = fg + m + 1, *sn = fg + 2 * m + 1;
  for (int l = 0; l < j; ++l) {
    const double a = H[l * ldh + j], b = H[(l + 1) * ldh + j];
    H[l * ldh + j] = cs[l] * a + sn[l] * b;
    H[(l + 1) * ldh + j] = -sn[l] * a + cs[l] * b;
  }
  const double a = H[j * ldh + j], b = H[(j + 1) * ldh + j];
  const double den = sqrt(a * a + b * b);
  cs[j] = a / den;
  sn[j] = b / den;
  H[j * ldh + j] = den;
  const double hn = H[(j + 1) * ldh + j];
  H[(j + 1) * ldh + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  const int k = *it + 1;
  *it = k;
  const double rel = fabs(g[j + 1]) / sqrt(slots[S_NB2]);
  hist[k] = rel;
  slots[S_REL] = rel;
  if (!isfinite(rel)) {
    *status = AMG_ERR_NAN;
    *active = 0;
  } else if (rel <= slots[S_TOL] || hn == 0.0) {
    *status = 1;
    *active = 0;
  } else if (k >= (int)slots[S_MAXIT]) {
    *status = AMG_ERR_NOT_CONVERGED;
    *active = 0;
  }
}

// y = H(0:j, 0:j)^-1 g by back substitution (one thread), into fg[3m+1 ..]
__global__ void k_fg_trisolve(const double *__restrict__ H, int ldh, int j, int m, double *__restrict__ fg) {
  pdl_wait_and_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double *g = fg;
  double *y = fg + 3 * m + 1;
  for (int l = j - 1; l >= 0; --l) {
    double t = g[l];
    for (int q = l + 1; q < j; ++q) t -= H[l * ldh + q] * y[q];
    y[l] = t / H[l * ldh + l];
  }
}

// x += sum_l y_l Z_l
__global__ void k_fg_xupdate(int32_t n, double *__restrict__ x, const double *__restrict__ Z, int ncol,
                             const double *__restrict__ y) {
  pdl_wait_and_trigger();
  __shared__ double ys[kMaxRestart + 1];
  for (int l = threadIdx.x; l < ncol; l += blockDim.x) ys[l] = y[l];
  __syncthreads();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double t = x[i];
    for (int l = 0; l < ncol; ++l) t += ys[l] * Z[(int64_t)l * n + i];
    x[i] = t;
  }
}

// V_0 = r / ||r||, g = (||r||, 0, ...)
__global__ void k_fg_start(int32_t n, const double *__restrict__ r, double *__restrict__ v0,
                           const double *__restrict__ slots, int slot_rr, double *__restrict__ fg, int m) {
  pdl_wait_and_trigger();
  const double beta = sqrt(slots[slot_rr]);
  if (blockIdx.x == 0)
    for (int l = threadIdx.x; l <= m; l += blockDim.x) fg[l] = (l == 0) ? beta : 0.0;
  const double inv = beta != 0.0 ? 1.0 / beta : 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v0[i] = r[i] * inv;
}

// ---------------------------------------------------------------- batched systems
// Per-system scalars of the block-diagonal solve.  Inner products are
// segmented by system: every row tile lies inside one system; tile partials
// are summed per system in tile order (deterministic).

__global__ void k_sys_of(int32_t n, int32_t nsys, const int32_t *__restrict__ off, int32_t *__restrict__ sys) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = nsys - 1;
    while (lo < hi) {  // last system whose first row is <= i
      const int32_t mid = (lo + hi + 1) >> 1;
      if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    sys[i] = lo;
  }
}

// tile partials of up to three inner products a_d . b_d (nullptr b: a . a)
template <class VT>
__global__ void k_segdot(int32_t ntiles, const int32_t *__restrict__ tile_row, int ndot, const VT *a0,
                         const VT *b0, const VT *a1, const VT *b1, const VT *a2, const VT *b2,
                         double *__restrict__ tpart, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int32_t i = tile_row[t] + threadIdx.x; i < tile_row[t + 1]; i += blockDim.x) {
      s0 += (double)a0[i] * (double)b0[i];
      if (ndot > 1) s1 += (double)a1[i] * (double)b1[i];
      if (ndot > 2) s2 += (double)a2[i] * (double)b2[i];
    }
    __shared__ double sh[3][kWarps];
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) {
      sh[0][threadIdx.x >> 5] = s0;
      sh[1][threadIdx.x >> 5] = s1;
      sh[2][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double v = 0.0;
      for (int w = 0; w < kWarps; ++w) v += sh[threadIdx.x][w];
      if ((int)threadIdx.x < ndot) tpart[(int64_t)threadIdx.x * ntiles + t] = v;
    }
    __syncthreads();
  }
}

// dot d of system s = sum of its tiles' partials; out[(slot0 + d) * nsys + s]
__global__ void k_segfin(int32_t nsys, int32_t ntiles, const int32_t *__restrict__ sys_tile, int ndot,
                         const double *__restrict__ tpart, double *__restrict__ bslots, int slot0, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const int lane = threadIdx.x & 31;
  for (int32_t s = blockIdx.x * kWarps + (threadIdx.x >> 5); s < nsys; s += gridDim.x * kWarps) {
    for (int d = 0; d < ndot; ++d) {
      double v = 0.0;
      for (int32_t t = sys_tile[s] + lane; t < sys_tile[s + 1]; t += 32) v += tpart[(int64_t)d * ntiles + t];
      v = warp_sum(v);
      if (lane == 0) bslots[(int64_t)(slot0 + d) * nsys + s] = v;
    }
  }
}

#define BS(slot, s) bslots[(int64_t)(slot)*nsys + (s)]

// per-system status of a batch while it runs: kIterating, kUpdatedConverged
// (the updated residual met tol; the true residual is checked next), then
// AMG_OK or a negative AMG_ERR_* code once the system has stopped
constexpr int kIterating = 2;
constexpr int kUpdatedConverged = 1;

// Alg. 5 per system: s1 = alpha_1 / rho_1 (dots in S_RHO1, S_A1)
__global__ void k_bfin_k1(int32_t nsys, double *__restrict__ bslots, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x)
    BS(S_S1, s) = BS(S_A1, s) / BS(S_RHO1, s);
}

template <class VT>
__global__ void k_baxpy_rt(int32_t n, const int32_t *__restrict__ sys, int32_t nsys, const VT *__restrict__ r,
                           const VT *__restrict__ v, VT *__restrict__ rt, const VT *__restrict__ wd,
                           VT *__restrict__ x0, const double *__restrict__ bslots, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const VT t = r[i] - (VT)BS(S_S1, sys[i]) * v[i];
    rt[i] = t;
    x0[i] = wd[i] * t;
  }
}

// per-system test ||r~|| <= t ||r|| (norms squared in S_NRT2, S_NR2); flag[nsys] = any
__global__ void k_bdecide(int32_t nsys, const double *__restrict__ bslots, double t, const int *parent,
                          int *__restrict__ flag) {
  pdl_wait_and_trigger();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int active = parent ? *parent : 1;
  for (int32_t s = threadIdx.x; s < nsys; s += blockDim.x) {
    const bool second = active && !(sqrt(BS(S_NRT2, s)) <= t * sqrt(BS(S_NR2, s)));
    flag[s] = second ? 1 : 0;
    if (second) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) flag[nsys] = any;
}

__global__ void k_bfin_k3(int32_t nsys, double *__restrict__ bslots, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    const double rho1 = BS(S_RHO1, s), gam = BS(S_GAM, s), bet = BS(S_BET, s), a2 = BS(S_A2, s);
    const double rho2 = bet - gam * gam / rho1;
    BS(S_CC, s) = BS(S_S1, s) - gam * a2 / (rho1 * rho2);
    BS(S_CD, s) = a2 / rho2;
  }
}

template <class VT>
__global__ void k_bcombine(int32_t n, const int32_t *__restrict__ sys, int32_t nsys, const VT *__restrict__ c,
                           const VT *__restrict__ d, VT *__restrict__ x, const double *__restrict__ bslots,
                           const int *__restrict__ flag, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t s = sys[i];
    x[i] = flag[s] ? (VT)BS(S_CC, s) * c[i] + (VT)BS(S_CD, s) * d[i] : (VT)BS(S_S1, s) * c[i];
  }
}

// exact coarsest solve, one dense inverse per system; one warp per row
template <class VT>
__global__ void k_bcoarse(int32_t nL, const int32_t *__restrict__ sys, const int32_t *__restrict__ off,
                          const double *__restrict__ binv, const int64_t *__restrict__ boff, const VT *__restrict__ b,
                          VT *__restrict__ x, const int *pred) {
  pdl_wait_and_trigger();
  if (pred && *pred == 0) return;
  const int lane = threadIdx.x & 31;
  for (int32_t i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < nL; i += gridDim.x * kWarps) {
    const int32_t s = sys[i], r0 = off[s], m = off[s + 1] - r0;
    const double *Bi = binv + boff[s] + (int64_t)(i - r0) * m;
    double acc = 0.0;
    for (int32_t j = lane; j < m; j += 32) acc += Bi[j] * (double)b[r0 + j];
    acc = warp_sum(acc);
    if (lane == 0) x[i] = (VT)acc;
  }
}

// flexible CG per system.  bact[s]: still iterating; brs[s]: restart (beta = 0)
__global__ void k_bfcg_beta(int32_t nsys, double *__restrict__ bslots, const int *__restrict__ brs) {
  pdl_wait_and_trigger();
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x)
    BS(S_BETA, s) = brs[s] ? 0.0 : -BS(S_ZQ, s) / BS(S_PQ, s);
}

__global__ void k_bfcg_p(int32_t n, const int32_t *__restrict__ sys, int32_t nsys, const double *__restrict__ z,
                         double *__restrict__ p, const double *__restrict__ bslots) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = z[i] + BS(S_BETA, sys[i]) * p[i];
}

__global__ void k_bfcg_alpha(int32_t nsys, double *__restrict__ bslots) {
  pdl_wait_and_trigger();
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x)
    BS(S_ALPHA, s) = BS(S_PR, s) / BS(S_PQ, s);
}

__global__ void k_bfcg_update(int32_t n, const int32_t *__restrict__ sys, int32_t nsys, double *__restrict__ x,
                              double *__restrict__ r, const double *__restrict__ p, const double *__restrict__ q,
                              const double *__restrict__ bslots, const int *__restrict__ bact) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t s = sys[i];
    if (!bact[s]) continue;  // converged systems keep x and r untouched
    const double a = BS(S_ALPHA, s);
    x[i] += a * p[i];
    r[i] -= a * q[i];
  }
}

// end of an iteration: per-system relative residual, iteration count, status;
// bact[nsys] = number of systems still iterating; hist[k] (k < hist_len) gets
// the largest relative residual of pass k
__global__ void k_bfcg_fin(int32_t nsys, double *__restrict__ bslots, int *__restrict__ bact, int *__restrict__ brs,
                           int *__restrict__ bit, int *__restrict__ bstat, double tol, int max_iter,
                           double *__restrict__ hist, int hist_len, int *__restrict__ it) {
  pdl_wait_and_trigger();
  __shared__ int nact;
  __shared__ double worst;
  if (threadIdx.x == 0) {
    nact = 0;
    worst = 0.0;
  }
  __syncthreads();
  for (int32_t s = threadIdx.x; s < nsys; s += blockDim.x) {
    brs[s] = 0;
    if (!bact[s]) continue;
    const double rel = sqrt(BS(S_RR, s) / BS(S_NB2, s));
    BS(S_REL, s) = rel;
    const int k = bit[s] + 1;
    bit[s] = k;
    atomicMax(reinterpret_cast<unsigned long long *>(&worst), __double_as_longlong(isfinite(rel) ? rel : 1e300));
    if (!(BS(S_PQ, s) > 0.0)) {
      bstat[s] = AMG_ERR_BREAKDOWN;
      bact[s] = 0;
    } else if (!isfinite(rel)) {
      bstat[s] = AMG_ERR_NAN;
      bact[s] = 0;
    } else if (rel <= tol) {
      bstat[s] = kUpdatedConverged;
      bact[s] = 0;
    } else if (k >= max_iter) {
      bstat[s] = AMG_ERR_NOT_CONVERGED;
      bact[s] = 0;
    } else {
      atomicAdd(&nact, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bact[nsys] = nact;
    const int k = *it + 1;
    *it = k;
    if (k < hist_len) hist[k] = worst;
  }
}

#undef BS

template <class VT>
__global__ void k_convert_row_data(int32_t n, const double *__restrict__ diag, double omega_host,
                                   const double *__restrict__ omega_dev, const double *__restrict__ pw64,
                                   VT *__restrict__ wd, VT *__restrict__ dinv, VT *__restrict__ pw) {
  pdl_wait_and_trigger();
  const double omega = omega_dev ? *omega_dev : omega_host;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    wd[i] = (VT)(omega / diag[i]);
    dinv[i] = (VT)(1.0 / diag[i]);
    if (pw64) pw[i] = (VT)pw64[i];
  }
}

template <class VT>
__global__ void k_copy_cast(int32_t n, const double *__restrict__ in, VT *__restrict__ out) {
  pdl_wait_and_trigger();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (VT)in[i];
}

// ============================================================== host engine
namespace {

inline int ew_grid(int64_t n) { return grid_for(n, kThreads, kRedBlocks); }
void prepare_batched(Hierarchy &h, cudaStream_t s);
template <class MV, class VT>
void autotune_t(Hierarchy &h, cudaStream_t s);
// Grid of a level's SpMV launches: one wave of resident blocks (6 per SM with
// FP32 vectors, 4 with FP64) unless the autotuner chose another size (at most
// kRedBlocks, the capacity of the partial-sum buffers).  The FP64 products of the
// outer iteration on level 0 use the FP64 kernel's wave whatever the precision.
template <class VT>
inline int default_sell_grid(const Level &L) {
  return grid_for((int64_t)L.nslices, kWarps, sell_min_blocks<VT>() * 152);
}
inline int sell_grid(const Level &L) { return L.sell_blocks; }
// launches without inner products have no partial-sum buffer to fill, so the
// autotuner may give them up to one warp per slice; by default they take the
// same wave of resident blocks (one warp per slice measured slower on the 128^3
// level 0: 34.4 against 27.4 us under ncu)
inline int full_plain_grid(const Level &L) { return grid_for((int64_t)L.nslices, kWarps, 1 << 30); }
inline int plain_grid(const Level &L) { return L.sell_plain_blocks; }
// levels of at most kSmallSlices slices (fewer warps than the GPU holds at a
// quarter of its occupancy) run the products with kSmallU entries a step, with
// FP32 vectors (measured: no gain with FP64 vectors)
constexpr int32_t kSmallSlices = 2048;
constexpr int kSmallU = 16;
inline int outer_grid(const Level &L0) { return default_sell_grid<double>(L0); }

template <class MV, class VT>
struct Engine {
  Hierarchy &h;
  cudaStream_t s;
  int64_t launches = 0;
  bool gmres_variant;

  Engine(Hierarchy &hh, cudaStream_t ss) : h(hh), s(ss) { gmres_variant = h.p.outer == 1; }

  VT *V(void *p) { return static_cast<VT *>(p); }
  // batch: the system map of a level and the systems still iterating (null otherwise)
  const int32_t *bsys(const Level &L) const { return h.batched ? L.sys_of : nullptr; }
  const int *bact() const { return h.batched ? h.bactive : nullptr; }

  void check() {
    ++launches;
    AMG_LAUNCH_CHECK();
  }

  SellArgs<VT> sell_args(int k, const VT *x, VT *out, const int *pred) {
    const Level &L = h.lev[k];
    SellArgs<VT> a{};
    a.n = L.n;
    a.nslices = L.nslices;
    a.sptr = L.sptr;
    a.scol = L.scol;
    a.sval = L.sval;
    a.spair = L.spair;
    a.sdiag = L.sdiag;
    if (h.batched) a.live = L.slive;
    a.x = x;
    a.out = out;
    a.pred = pred;
    a.partials = L.partials;
    return a;
  }

  template <int EPI>
  void sell(const SellArgs<VT> &a, int k) {
    // fused inner products: after the plain product (Alg. 5) and on the last
    // post-smoothing step of level 0 (z^T q of the outer flexible CG)
    if (h.batched) {  // no fused inner products in a batch: they are per system (segdot)
      if (a.ndot) throw Error{AMG_ERR_UNSUPPORTED, "batched SpMV was given fused inner products"};
      klaunch(k_sell<MV, VT, EPI, false, true>, plain_grid(h.lev[k]), kThreads, s, a);
      check();
      return;
    }
    const bool small = sizeof(VT) == 4 && h.lev[k].nslices <= kSmallSlices;
    if constexpr (EPI == E_Y || EPI == E_POST || EPI == E_HORNER_LAST) {
      if (a.ndot) {
        if constexpr (EPI == E_Y && sizeof(VT) == 4)
          if (small) {
            klaunch(k_sell<MV, VT, EPI, true, false, kSmallU>, sell_grid(h.lev[k]), kThreads, s, a);
            check();
            return;
          }
        klaunch(k_sell<MV, VT, EPI, true, false>, sell_grid(h.lev[k]), kThreads, s, a);
        check();
        return;
      }
    } else {
      if (a.ndot) throw Error{AMG_ERR_UNSUPPORTED, "SpMV epilogue without fused inner products was given some"};
    }
    if constexpr ((EPI == E_Y || EPI == E_RESID || EPI == E_POST) && sizeof(VT) == 4)
      if (small) {
        klaunch(k_sell<MV, VT, EPI, false, false, kSmallU>, plain_grid(h.lev[k]), kThreads, s, a);
        check();
        return;
      }
    klaunch(k_sell<MV, VT, EPI, false, false>, plain_grid(h.lev[k]), kThreads, s, a);
    check();
  }

  // out = approximately A_k^-1 rhs with a zero initial guess (Alg. 4/5).
  // If x0_ready, lev[k].tmp already holds wd_k * rhs.
  void cycle(int k, const VT *rhs, VT *out, bool x0_ready, const int *pred) {
    Level &L = h.lev[k];
    if (k == h.L - 1) {
      if (h.batched)
        klaunch(k_bcoarse<VT>, grid_for(h.nL, kWarps, 152 * 8), kThreads, s, h.nL, (const int32_t *)L.sys_of,
                (const int32_t *)L.sys_off, (const double *)h.binv, (const int64_t *)h.binv_off, rhs, out, pred);
      else
        klaunch(k_coarse<VT>, grid_for(h.nL, kWarps, 152), kThreads, s, h.nL, h.coarse_inv, rhs, out, nullptr, pred);
      check();
      return;
    }
    Level &C = h.lev[k + 1];
    VT *tmp = V(L.tmp);
    const bool poly = h.p.smoother == 1 && L.poly != nullptr && !L.poly_off;
    if (poly) {  // x = sum_q diag(c_q) (D^-1 A)^q D^-1 b
      klaunch(k_scale<VT>, ew_grid(L.n), kThreads, s, L.n, V(L.u0), V(L.dinv), rhs, pred, bsys(L), bact());
      check();
      SellArgs<VT> a = sell_args(k, V(L.u0), V(L.u1), pred);
      a.dinv = V(L.dinv);
      sell<E_DSCALE>(a, k);
      a = sell_args(k, V(L.u1), tmp, pred);
      a.dinv = V(L.dinv);
      a.coef = V(L.poly);
      a.p0 = V(L.u0);
      a.p1 = V(L.u1);
      sell<E_POLYPRE>(a, k);
    } else if (!x0_ready) {
      klaunch(k_scale<VT>, ew_grid(L.n), kThreads, s, L.n, tmp, V(L.wd), rhs, pred, bsys(L), bact());  // pre-smoothing
      check();
    }
    {  // r_k = b_k - A_k x_k
      SellArgs<VT> a = sell_args(k, tmp, V(L.r), pred);
      a.rhs = rhs;
      sell<E_RESID>(a, k);
    }
    const bool coarse_is_last = (k + 1 == h.L - 1);
    const bool tail = (k + 1 == h.tail_t);
    // single systems: the restriction to the coarsest level and its solve in one launch
    const bool fuse_coarse = coarse_is_last && !tail && !h.batched && h.nL <= kFusedCoarseMax;
    if (fuse_coarse) {
      klaunch(k_restrict_coarse<VT>, grid_for(h.nL, kWarps, 152), kThreads, s, h.nL, L.aptr, L.amem, V(L.pw),
              V(L.r), h.coarse_inv, V(C.xc), pred);
      check();
    } else {
      // r_{k+1} = R_k r_k  (and x0 of level k+1 when it smooths)
      klaunch(k_restrict<VT>, ew_grid(L.nc), kThreads, s, L.nc, L.aptr, L.amem, V(L.pw), V(L.r), V(C.bc),
              (coarse_is_last || tail) ? nullptr : V(C.wd), V(C.tmp), pred, bsys(C), bact());
      check();
    }
    if (tail) {  // levels k+1..L-1 in one cluster launch
      TailArgs ta{};
      ta.t = k + 1;
      ta.L = h.L;
      ta.mode = k < h.p.kcycle_levels ? 1 : 0;
      ta.nL = h.nL;
      ta.gmres = gmres_variant ? 1 : 0;
      ta.kt = h.p.kcycle_t;
      ta.Ainv = h.coarse_inv;
      ta.lev = h.tail_dev;
      ta.pred = pred;
      tail_launch<MV, VT>(ta, h.p.tail == 2 ? 1 : 8, s);
      ++launches;
    } else if (coarse_is_last) {
      if (!fuse_coarse) cycle(k + 1, V(C.bc), V(C.xc), true, pred);  // exact coarse solve
    } else if (k < h.p.kcycle_levels) {
      krylov2(k + 1, pred);  // Alg. 5 coarse correction
    } else {
      cycle(k + 1, V(C.bc), V(C.xc), true, pred);  // Alg. 4 recursion
    }
    // x_k += P_k x_{k+1}
    klaunch(k_prolong<VT>, ew_grid(L.n), kThreads, s, L.n, L.agg, V(L.pw), V(C.xc), tmp, pred, bsys(L), bact());
    check();
    // r_k = b_k - A_k x_k;  x_k += omega D^-1 r_k  (or the transposed polynomial)
    SellArgs<VT> a = sell_args(k, tmp, out, pred);
    a.rhs = rhs;
    a.wd = V(L.wd);
    a.xin = tmp;
    if (poly) {
      SellArgs<VT> b = sell_args(k, tmp, V(L.r), pred);
      b.rhs = rhs;
      b.dinv = V(L.dinv);
      b.coef = V(L.poly);
      b.out2 = V(L.u0);
      sell<E_RESID_POLY>(b, k);
      b = sell_args(k, V(L.u0), V(L.u1), pred);
      b.dinv = V(L.dinv);
      b.coef = V(L.poly);
      b.res = V(L.r);
      sell<E_HORNER>(b, k);
      a.x = V(L.u1);
      a.dinv = V(L.dinv);
      a.coef = V(L.poly);
      a.res = V(L.r);
    }
    if (k == 0 && std::is_same<VT, double>::value && zq_fuse) {
      a.ndot = 1;  // z^T q for the outer flexible CG
      a.dop[0][0] = OP_Y;
      a.dop[0][1] = OP_U1;
      a.u1 = (const VT *)h.q;
      a.partials = h.lev[0].partials + 4 * kRedBlocks;
    }
    if (poly)
      sell<E_HORNER_LAST>(a, k);
    else
      sell<E_POST>(a, k);
  }
  bool zq_fuse = false;

  // per-system inner products of the batch into bslots[slot0 ..]
  void segdot(int k, int ndot, const VT *a0, const VT *b0, const VT *a1, const VT *b1, const VT *a2, const VT *b2,
              int slot0, const int *pred) {
    Level &L = h.lev[k];
    klaunch(k_segdot<VT>, grid_for(L.ntiles, 1, 152 * 8), kThreads, s, L.ntiles, (const int32_t *)L.tile_row, ndot,
            a0, b0, a1, b1, a2, b2, L.tpart, pred);
    klaunch(k_segfin, grid_for(h.nsys, kWarps, 152), kThreads, s, (int32_t)h.nsys, L.ntiles,
            (const int32_t *)L.sys_tile, ndot, (const double *)L.tpart, L.bslots, slot0, pred);
    launches += 2;
    AMG_LAUNCH_CHECK();
  }

  // Alg. 5 coarse part at level m for every system of a batch, with per-system
  // scalars; the second inner step runs when any system needs it
  void krylov2_batched(int m, const int *pred) {
    Level &L = h.lev[m];
    const int32_t ns = h.nsys;
    cycle(m, V(L.bc), V(L.c), true, pred);
    sell<E_Y>(sell_args(m, V(L.c), V(L.v), pred), m);
    if (gmres_variant)
      segdot(m, 2, V(L.v), V(L.v), V(L.v), V(L.bc), nullptr, nullptr, S_RHO1, pred);
    else
      segdot(m, 2, V(L.c), V(L.v), V(L.c), V(L.bc), nullptr, nullptr, S_RHO1, pred);
    klaunch(k_bfin_k1, grid_for(ns, kThreads, 152), kThreads, s, ns, L.bslots, pred);
    klaunch(k_baxpy_rt<VT>, ew_grid(L.n), kThreads, s, L.n, (const int32_t *)L.sys_of, ns, (const VT *)V(L.bc),
            (const VT *)V(L.v), V(L.rt), (const VT *)V(L.wd), V(L.tmp), (const double *)L.bslots, pred);
    segdot(m, 2, V(L.rt), V(L.rt), V(L.bc), V(L.bc), nullptr, nullptr, S_NRT2, pred);
    klaunch(k_bdecide, 1, 1024, s, ns, (const double *)L.bslots, h.p.kcycle_t, pred, L.bflag);
    launches += 3;
    AMG_LAUNCH_CHECK();
    const int *any = L.bflag + ns;
    cycle(m, V(L.rt), V(L.d), true, any);
    sell<E_Y>(sell_args(m, V(L.d), V(L.w), any), m);
    if (gmres_variant)
      segdot(m, 3, V(L.w), V(L.v), V(L.w), V(L.w), V(L.w), V(L.rt), S_GAM, any);
    else
      segdot(m, 3, V(L.d), V(L.v), V(L.d), V(L.w), V(L.d), V(L.rt), S_GAM, any);
    klaunch(k_bfin_k3, grid_for(ns, kThreads, 152), kThreads, s, ns, L.bslots, any);
    klaunch(k_bcombine<VT>, ew_grid(L.n), kThreads, s, L.n, (const int32_t *)L.sys_of, ns, (const VT *)V(L.c),
            (const VT *)V(L.d), V(L.xc), (const double *)L.bslots, (const int *)L.bflag, pred);
    launches += 2;
    AMG_LAUNCH_CHECK();
  }

  // Alg. 5 coarse part at level m: rhs = bc[m], result in xc[m]; lev[m].tmp holds wd*bc.
  void krylov2(int m, const int *pred) {
    if (h.batched) {
      krylov2_batched(m, pred);
      return;
    }
    Level &L = h.lev[m];
    const int nb = sell_grid(L);
    // c = cycle(m, r)
    cycle(m, V(L.bc), V(L.c), true, pred);
    {  // v = A c; dots
      SellArgs<VT> a = sell_args(m, V(L.c), V(L.v), pred);
      a.ndot = 2;
      a.u1 = V(L.bc);
      if (gmres_variant) {  // rho1 = v^T v, alpha1 = v^T r
        a.dop[0][0] = OP_Y; a.dop[0][1] = OP_Y; a.dop[1][0] = OP_Y; a.dop[1][1] = OP_U1;
      } else {               // rho1 = c^T v, alpha1 = c^T r
        a.dop[0][0] = OP_X; a.dop[0][1] = OP_Y; a.dop[1][0] = OP_X; a.dop[1][1] = OP_U1;
      }
      sell<E_Y>(a, m);
    }
    // One-block kernels take the scalars: with programmatic dependent launch
    // their launch costs less than every block of the vector kernel summing the
    // partials itself.
    klaunch(k_fin_k1, 1, kThreads, s, L.partials, nb, L.slots, pred);
    check();
    const int ng = ew_grid(L.n);
    klaunch(k_axpy_rt<VT>, ng, kThreads, s, L.n, V(L.bc), V(L.v), V(L.rt), V(L.wd), V(L.tmp), L.slots,
            L.partials + 3 * kRedBlocks, pred);
    check();
    klaunch(k_decide, 1, kThreads, s, L.partials + 3 * kRedBlocks, ng, L.slots, h.p.kcycle_t, pred, L.flag);
    check();
    // second inner step, predicated on the decision
    cycle(m, V(L.rt), V(L.d), true, L.flag);
    {
      SellArgs<VT> a = sell_args(m, V(L.d), V(L.w), L.flag);
      a.ndot = 3;
      a.u1 = V(L.v);
      a.u2 = V(L.rt);
      if (gmres_variant) {  // gamma = w^T v, beta = w^T w, alpha2 = w^T r~
        a.dop[0][0] = OP_Y; a.dop[0][1] = OP_U1;
        a.dop[1][0] = OP_Y; a.dop[1][1] = OP_Y;
        a.dop[2][0] = OP_Y; a.dop[2][1] = OP_U2;
      } else {               // gamma = d^T v, beta = d^T w, alpha2 = d^T r~
        a.dop[0][0] = OP_X; a.dop[0][1] = OP_U1;
        a.dop[1][0] = OP_X; a.dop[1][1] = OP_Y;
        a.dop[2][0] = OP_X; a.dop[2][1] = OP_U2;
      }
      sell<E_Y>(a, m);
    }
    klaunch(k_fin_k3, 1, kThreads, s, L.partials, nb, L.slots, L.flag);
    check();
    klaunch(k_combine<VT>, ng, kThreads, s, L.n, V(L.c), V(L.d), V(L.xc), L.slots, L.flag, pred);
    check();
  }

  // z = M r for the FP64 outer iteration
  void precond(const double *r, double *z, const int *pred, bool with_zq) {
    Level &L0 = h.lev[0];
    if (std::is_same<VT, double>::value) {
      zq_fuse = with_zq;
      cycle(0, (const VT *)r, (VT *)z, false, pred);
      zq_fuse = false;
      if (with_zq && h.L == 1) {
        klaunch(k_dot64, ew_grid(L0.n), kThreads, s, L0.n, z, h.q, L0.partials + 4 * kRedBlocks, pred);
        check();
      }
    } else {
      klaunch(k_to_vt<VT>, ew_grid(L0.n), kThreads, s, L0.n, r, V(h.pre_in), V(L0.wd), V(L0.tmp), pred);
      check();
      cycle(0, V(h.pre_in), V(h.pre_out), true, pred);
      klaunch(k_from_vt_dot<VT>, ew_grid(L0.n), kThreads, s, L0.n, V(h.pre_out), z, h.q,
                                                           L0.partials + 4 * kRedBlocks, pred);
      check();
    }
  }

  // one flexible-CG iteration of every system of a batch (graph-capturable)
  void fcg_iteration_batched(double tol) {
    Level &L0 = h.lev[0];
    const int32_t ns = h.nsys, n = L0.n;
    const int ng = ew_grid(n);
    int *bact = h.bactive, *brs = h.bactive + ns + 1;
    for (int k = 0; k < h.L; ++k) {  // slices of the systems still iterating
      Level &L = h.lev[k];
      klaunch(k_slice_live, grid_for(L.nslices, kThreads, 152 * 4), kThreads, s, L.n, L.nslices,
              (const int32_t *)L.sys_of, (const int *)bact, L.slive);
      ++launches;
    }
    // z = M r
    precond(h.r, h.z, nullptr, false);
    Engine<double, double> e64(h, s);
    e64.segdot(0, 1, h.z, h.q, nullptr, nullptr, nullptr, nullptr, S_ZQ, nullptr);
    launches += e64.launches;
    klaunch(k_bfcg_beta, grid_for(ns, kThreads, 152), kThreads, s, ns, L0.bslots, (const int *)brs);
    klaunch(k_bfcg_p, ng, kThreads, s, n, (const int32_t *)L0.sys_of, ns, (const double *)h.z, h.pdir,
            (const double *)L0.bslots);
    {  // q = A p in FP64
      SellArgs<double> a{};
      a.n = n;
      a.nslices = L0.nslices;
      a.sptr = L0.sptr64;
      a.scol = L0.scol64;
      a.sval = L0.sval64;
      a.x = h.pdir;
      a.out = h.q;
      a.live = L0.slive;
      klaunch(k_sell<double, double, E_Y, false, true>, outer_grid(L0), kThreads, s, a);
    }
    launches += 3;
    e64.launches = 0;
    e64.segdot(0, 2, h.pdir, h.q, h.pdir, h.r, nullptr, nullptr, S_PQ, nullptr);
    klaunch(k_bfcg_alpha, grid_for(ns, kThreads, 152), kThreads, s, ns, L0.bslots);
    klaunch(k_bfcg_update, ng, kThreads, s, n, (const int32_t *)L0.sys_of, ns, h.x, h.r, (const double *)h.pdir,
            (const double *)h.q, (const double *)L0.bslots, (const int *)bact);
    e64.segdot(0, 1, h.r, h.r, nullptr, nullptr, nullptr, nullptr, S_RR, nullptr);
    launches += e64.launches + 2;
    klaunch(k_bfcg_fin, 1, 1024, s, ns, L0.bslots, bact, brs, h.bit, h.bit + ns, tol, h.p.max_iter, h.hist,
            h.p.max_iter + 8, h.it_dev);
    ++launches;
    AMG_LAUNCH_CHECK();
  }

  // one flexible-CG iteration, all on the device (graph-capturable)
  void fcg_iteration(int *active, int *restart) {
    Level &L0 = h.lev[0];
    double *part = L0.partials;
    const int ng = ew_grid(L0.n);
    const int nsg = outer_grid(L0);  // FP64 q = A p and its two inner products
    const int nzq = (std::is_same<VT, double>::value && h.L > 1) ? sell_grid(L0) : ng;  // z^T q of the cycle
    // z = M r (+ z^T q partials)
    precond(h.r, h.z, active, true);
    // p = z + beta p
    klaunch(k_fcg_p, ng, kThreads, s, L0.n, h.z, h.pdir, part + 4 * kRedBlocks, nzq, L0.slots, restart, active);
    check();
    {  // q = A p (FP64), p^T q, p^T r
      SellArgs<double> a{};
      a.n = L0.n;
      a.nslices = L0.nslices;
      a.sptr = L0.sptr64;
      a.scol = L0.scol64;
      a.sval = L0.sval64;
      a.x = h.pdir;
      a.out = h.q;
      a.u1 = h.r;
      a.ndot = 2;
      a.dop[0][0] = OP_X; a.dop[0][1] = OP_Y;
      a.dop[1][0] = OP_X; a.dop[1][1] = OP_U1;
      a.partials = part + 5 * kRedBlocks;
      a.pred = active;
      klaunch(k_sell<double, double, E_Y, true, false>, nsg, kThreads, s, a);
      check();
    }
    // x, r update (+ the next preconditioner input in reduced precision)
    const bool red = !std::is_same<VT, double>::value;
    klaunch(k_fcg_update<VT>, ng, kThreads, s, L0.n, h.x, h.r, h.pdir, h.q, part + 5 * kRedBlocks, nsg, L0.slots,
                                             part + 7 * kRedBlocks, nullptr, V(L0.wd), V(L0.tmp), active);
    check();
    (void)red;
    klaunch(k_fcg_fin, 1, kThreads, s, part + 7 * kRedBlocks, ng, L0.slots, h.hist, h.it_dev, active, restart,
                                     h.status_dev);
    check();
  }
};

template <class MV, class VT>
void alloc_level_vectors(Hierarchy &h, Level &L, int k) {
  const size_t n = (size_t)L.n;
  auto vec = [&]() { return (void *)h.arena.get<VT>(n + 1); };
  L.r = vec();
  L.bc = vec();
  L.xc = vec();
  L.tmp = vec();
  L.u0 = vec();
  L.u1 = vec();
  if (k >= 1) {
    L.c = vec();
    L.v = vec();
    L.rt = vec();
    L.d = vec();
    L.w = vec();
  }
  if (L.sell_blocks <= 0) L.sell_blocks = default_sell_grid<VT>(L);
  if (L.sell_plain_blocks <= 0) L.sell_plain_blocks = L.sell_blocks;
  L.slots = h.arena.get<double>(kNumSlots);
  L.flag = h.arena.get<int>(4);
  L.partials = h.arena.get<double>((size_t)kRedBlocks * 8);
  AMG_CUDA(cudaMemsetAsync(L.slots, 0, sizeof(double) * kNumSlots, current_stream()));
  AMG_CUDA(cudaMemsetAsync(L.flag, 0, sizeof(int) * 4, current_stream()));
  AMG_CUDA(cudaMemsetAsync(L.partials, 0, sizeof(double) * kRedBlocks * 8, current_stream()));
}

// First level t of the cluster tail: at most kTailMaxRows rows, not the
// coarsest, every level in t..L-3 below the K-cycle levels (the tail runs
// V-cycles only), and no polynomial smoother on those levels.
void configure_tail(Hierarchy &h, cudaStream_t s) {
  h.tail_t = -1;
  if (!h.p.tail || h.batched) return;  // the cluster tail has no per-system scalars
  for (int t = 1; t <= h.L - 2; ++t) {
    if (h.lev[t].n > kTailMaxRows) continue;
    bool ok = true;
    for (int k = t; k <= h.L - 3; ++k) ok = ok && k >= h.p.kcycle_levels;
    for (int k = t; k < h.L - 1; ++k) ok = ok && !(h.p.smoother == 1 && h.lev[k].poly && !h.lev[k].poly_off);
    if (ok) {
      h.tail_t = t;
      break;
    }
  }
  if (h.tail_t < 0) return;
  std::vector<TailLevel> tl(h.L);
  for (int k = 0; k < h.L; ++k) {
    const Level &L = h.lev[k];
    TailLevel &T = tl[k];
    T.n = L.n;
    T.nslices = L.nslices;
    T.nc = L.nc;
    T.sptr = L.sptr;
    T.scol = L.scol;
    T.sval = L.sval;
    T.spair = L.spair;
    T.sdiag = L.sdiag;
    T.wd = L.wd;
    T.pw = L.pw;
    T.agg = L.agg;
    T.aptr = L.aptr;
    T.amem = L.amem;
    T.bc = L.bc;
    T.xc = L.xc;
    T.r = L.r;
    T.c = L.c;
    T.v = L.v;
    T.rt = L.rt;
    T.d = L.d;
    T.w = L.w;
  }
  if (!h.tail_dev) h.tail_dev = h.arena.get<TailLevel>(kMaxLevels);
  AMG_CUDA(cudaMemcpyAsync(h.tail_dev, tl.data(), sizeof(TailLevel) * h.L, cudaMemcpyHostToDevice, s));
  AMG_CUDA(cudaStreamSynchronize(s));
}

template <class MV, class VT>
void prepare_t(Hierarchy &h, cudaStream_t s) {
  for (int k = 0; k < h.L; ++k) alloc_level_vectors<MV, VT>(h, h.lev[k], k);
  const size_t n = (size_t)h.lev[0].n;
  h.x = h.arena.get<double>(n);
  h.b = h.arena.get<double>(n);
  h.r = h.arena.get<double>(n);
  h.z = h.arena.get<double>(n);
  h.pdir = h.arena.get<double>(n);
  h.q = h.arena.get<double>(n);
  h.pre_in = h.arena.get<VT>(n);
  h.pre_out = h.arena.get<VT>(n);
  h.hist = h.arena.get<double>((size_t)h.p.max_iter + 8);
  h.it_dev = h.arena.get<int>(8);
  h.status_dev = h.it_dev + 4;
  AMG_CUDA(cudaMemsetAsync(h.q, 0, sizeof(double) * n, s));
  AMG_CUDA(cudaMemsetAsync(h.pdir, 0, sizeof(double) * n, s));
  if (h.p.outer == 1) {
    const int m = h.p.restart;
    h.V = h.arena.get<double>(n * (size_t)(m + 1));
    h.Z = h.arena.get<double>(n * (size_t)m);
    h.H = h.arena.get<double>((size_t)(m + 1) * m);
    h.fg = h.arena.get<double>(4 * (size_t)m + 2);
    h.hc = h.arena.get<double>(kMaxRestart + 2);
    h.gpart = h.arena.get<double>((size_t)(kMaxRestart + 1) * kRedBlocks);
    AMG_CUDA(cudaMemsetAsync(h.H, 0, sizeof(double) * (m + 1) * m, s));
  }
  if (!h.host_pinned) h.host_pinned = pinned_scratch_get();
  if (h.batched) prepare_batched(h, s);
  configure_tail(h, s);
  if (h.p.autotune) autotune_t<MV, VT>(h, s);
}

template <class VT>
void make_row_data_t(Hierarchy &h, Level &L, const double *diag, cudaStream_t s) {
  if (!L.wd) {  // refilled in place by a values-only re-setup
    L.wd = h.arena.get<VT>((size_t)L.n + 1);
    L.dinv = h.arena.get<VT>((size_t)L.n + 1);
    L.pw = h.arena.get<VT>((size_t)L.n + 1);
  }
  klaunch(k_convert_row_data<VT>, ew_grid(L.n), kThreads, s, L.n, diag, L.omega, (const double *)L.omega_dev,
          L.pw64, (VT *)L.wd, (VT *)L.dinv, (VT *)L.pw);
  AMG_LAUNCH_CHECK();
}

__global__ void k_set_state(int *it, int *active, int *restart, int *status, int it_v, int active_v,
                            int restart_v, int status_v) {
  pdl_wait_and_trigger();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (it_v >= 0) *it = it_v;
    *active = active_v;
    *restart = restart_v;
    *status = status_v;
  }
}

__global__ void k_set_slot(double *slots, int idx, double v) {
  pdl_wait_and_trigger();
  if (threadIdx.x == 0 && blockIdx.x == 0) slots[idx] = v;
}

// Copy n doubles between user memory (host or device) and device memory.
void copy_in(double *dst_dev, const double *src, int32_t n, cudaStream_t s) {
  const cudaMemcpyKind k = pointer_kind(src) == PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  AMG_CUDA(cudaMemcpyAsync(dst_dev, src, sizeof(double) * (size_t)n, k, s));
}
void copy_out(double *dst, const double *src_dev, int32_t n, cudaStream_t s) {
  const cudaMemcpyKind k = pointer_kind(dst) == PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  AMG_CUDA(cudaMemcpyAsync(dst, src_dev, sizeof(double) * (size_t)n, k, s));
}

// ||b - A x||^2 into slots[dst] (FP64)
void true_residual(Hierarchy &h, int dst, cudaStream_t s, int64_t &launches) {
  Level &L0 = h.lev[0];
  const int nsg = outer_grid(L0);
  klaunch(k_residual64, nsg, kThreads, s, L0.n, L0.nslices, L0.sptr64, L0.scol64, L0.sval64, h.x, h.b, h.r,
                                        L0.partials + 7 * kRedBlocks);
  klaunch(k_store_sum, 1, kThreads, s, L0.partials + 7 * kRedBlocks, nsg, L0.slots + dst);
  launches += 2;
  AMG_LAUNCH_CHECK();
}

// cycle trace: clear the per-level counts of second inner steps before a solve
void trace_reset(Hierarchy &h, cudaStream_t s) {
  for (int k = 0; k < h.L; ++k) klaunch(k_set_slot, 1, 32, s, h.lev[k].slots, S_TAKEN, 0.0);
  AMG_LAUNCH_CHECK();
  h.trace_ok = false;
}

// after a solve with `apps` preconditioner applications: the counts of second
// steps, and from them the visits of every level (Alg. 5 at level m runs the
// cycle of m once, twice when its second step is taken; Alg. 4 recurses once)
void trace_collect(Hierarchy &h, int64_t apps, cudaStream_t s) {
  std::vector<double> pin(h.L, 0.0);
  for (int k = 0; k < h.L; ++k)
    AMG_CUDA(cudaMemcpyAsync(&pin[k], h.lev[k].slots + S_TAKEN, sizeof(double), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < kMaxLevels; ++k) h.visits[k] = h.kcalls[k] = h.second[k] = 0;
  h.visits[0] = apps;
  for (int k = 0; k + 1 < h.L; ++k) {
    const int m = k + 1;
    if (m < h.L - 1 && k < h.p.kcycle_levels && h.tail_t != m) {
      h.kcalls[m] = h.visits[k];
      h.second[m] = (int64_t)pin[m];
      h.visits[m] = h.visits[k] + h.second[m];
    } else {
      h.visits[m] = h.visits[k];
    }
  }
  h.trace_ok = h.tail_t < 0;  // the cluster tail runs its levels without the counters
}

template <class MV, class VT>
int run_solve_t(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *res_hist,
                cudaStream_t s) {
  Level &L0 = h.lev[0];
  const int32_t n = L0.n;
  Engine<MV, VT> eng(h, s);
  int64_t launches = 0;
  int *active = h.it_dev + 1, *restart = h.it_dev + 2;
  copy_in(h.b, b, n, s);
  copy_in(h.x, x, n, s);
  trace_reset(h, s);
  // ||b||^2 and the initial residual
  klaunch(k_dot64, ew_grid(n), kThreads, s, n, h.b, h.b, L0.partials + 6 * kRedBlocks, nullptr);
  klaunch(k_store_sum, 1, kThreads, s, L0.partials + 6 * kRedBlocks, ew_grid(n), L0.slots + S_NB2);
  launches += 2;
  AMG_LAUNCH_CHECK();
  true_residual(h, S_RR, s, launches);
  klaunch(k_set_slot, 1, 32, s, L0.slots, S_TOL, tol);
  klaunch(k_set_slot, 1, 32, s, L0.slots, S_MAXIT, (double)h.p.max_iter);
  AMG_CUDA(cudaMemcpyAsync(h.host_pinned, L0.slots, sizeof(double) * kNumSlots, cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  double nb2 = h.host_pinned[S_NB2];
  const double rr0 = h.host_pinned[S_RR];
  const bool zero_b = !(nb2 > 0.0);
  if (zero_b) nb2 = 1.0, klaunch(k_set_slot, 1, 32, s, L0.slots, S_NB2, 1.0);
  double rel = std::sqrt(rr0 / nb2);
  std::vector<double> hist(1, rel);
  int status = AMG_OK;
  int it = 0;
  if (!std::isfinite(rel)) status = AMG_ERR_NAN;
  else if (rel > tol) {
    klaunch(k_set_state, 1, 32, s, h.it_dev, active, restart, h.status_dev, 0, 1, 1, 0);
    AMG_CUDA(cudaMemcpyAsync(h.hist, &hist[0], sizeof(double), cudaMemcpyHostToDevice, s));
    AMG_LAUNCH_CHECK();
    // capture one outer iteration as a graph
    int64_t per_iter = 0;
    if (h.p.use_graph && h.graph_kind != 0) {
      if (h.graph_exec) {
        cudaGraphExecDestroy(h.graph_exec);
        cudaGraphDestroy(h.graph);
        h.graph_exec = nullptr;
      }
      AMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      eng.fcg_iteration(active, restart);
      AMG_CUDA(cudaStreamEndCapture(s, &h.graph));
      AMG_CUDA(cudaGraphInstantiate(&h.graph_exec, h.graph, 0));
      h.graph_kind = 0;
      h.graph_launches = eng.launches;
      eng.launches = 0;
    }
    per_iter = h.graph_launches;
    auto enqueue = [&]() {
      if (h.p.use_graph) {
        AMG_CUDA(cudaGraphLaunch(h.graph_exec, s));
        launches += per_iter;
      } else {
        eng.fcg_iteration(active, restart);
      }
    };
    // The next iteration is queued before this one's state is read, so the GPU
    // does not wait for the host between iterations; once an iteration stops
    // (*active = 0) every kernel of the next one returns at once.
    int *st_host = reinterpret_cast<int *>(h.host_pinned + 32);  // two slots of 8 ints
    EventPair ep;  // destroyed on every exit, including a throw inside the loop
    cudaEvent_t *evs = ep.e;
    auto launch_iter = [&](int slot) {
      enqueue();
      AMG_CUDA(cudaMemcpyAsync(st_host + 8 * slot, h.it_dev, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaEventRecord(evs[slot], s));
    };
    int slot = 0;
    launch_iter(slot);
    for (;;) {
      launch_iter(slot ^ 1);
      AMG_CUDA(cudaEventSynchronize(evs[slot]));
      const int dst = st_host[8 * slot + 4];
      it = st_host[8 * slot];
      if (dst == 0) {  // still iterating
        slot ^= 1;
        continue;
      }
      AMG_CUDA(cudaStreamSynchronize(s));  // the queued iteration ran and did nothing
      if (dst == 1) {  // updated residual meets tol: check the true residual
        true_residual(h, S_TRUE_RR, s, launches);
        AMG_CUDA(cudaMemcpyAsync(h.host_pinned, L0.slots, sizeof(double) * kNumSlots, cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        const double rel_true = std::sqrt(h.host_pinned[S_TRUE_RR] / nb2);
        if (rel_true <= tol) {
          status = AMG_OK;
          break;
        }
        if (it >= h.p.max_iter) {
          status = AMG_ERR_NOT_CONVERGED;
          break;
        }
        // iterative refinement: restart flexible CG from the true residual
        klaunch(k_set_state, 1, 32, s, h.it_dev, active, restart, h.status_dev, -1, 1, 1, 0);
        AMG_LAUNCH_CHECK();
        slot = 0;
        launch_iter(slot);
        continue;
      }
      status = dst;
      break;
    }
    AMG_CUDA(cudaStreamSynchronize(s));
    hist.resize((size_t)it + 1);
    if (it > 0)
      AMG_CUDA(cudaMemcpyAsync(&hist[1], h.hist + 1, sizeof(double) * (size_t)it, cudaMemcpyDeviceToHost, s));
  }
  launches += eng.launches;
  // final FP64 residual
  true_residual(h, S_TRUE_RR, s, launches);
  AMG_CUDA(cudaMemcpyAsync(h.host_pinned, L0.slots, sizeof(double) * kNumSlots, cudaMemcpyDeviceToHost, s));
  copy_out(x, h.x, n, s);
  AMG_CUDA(cudaStreamSynchronize(s));
  h.info.final_relres = zero_b ? std::sqrt(h.host_pinned[S_TRUE_RR]) : std::sqrt(h.host_pinned[S_TRUE_RR] / nb2);
  trace_collect(h, it, s);
  h.info.iters = it;
  h.info.status = status;
  h.info.kernel_launches = launches;
  if (iters) *iters = it;
  if (res_hist) std::memcpy(res_hist, hist.data(), sizeof(double) * hist.size());
  return status;
}

// Flexible GMRES(m) (Sec. 2.2, Sec. 4): the Arnoldi basis is orthogonalised by
// classical Gram-Schmidt with one reorthogonalisation (two multi-dot passes), in
// FP64; the K-cycle uses the GMRES variant of Alg. 5.  Every restart starts from
// the true FP64 residual.
template <class MV, class VT>
int run_fgmres_t(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *res_hist,
                 cudaStream_t s) {
  Level &L0 = h.lev[0];
  const int32_t n = L0.n;
  const int m = h.p.restart;
  Engine<MV, VT> eng(h, s);
  int64_t launches = 0;
  int *active = h.it_dev + 1;
  copy_in(h.b, b, n, s);
  copy_in(h.x, x, n, s);
  trace_reset(h, s);
  const int ng = ew_grid(n);
  klaunch(k_dot64, ng, kThreads, s, n, h.b, h.b, L0.partials + 6 * kRedBlocks, nullptr);
  klaunch(k_store_sum, 1, kThreads, s, L0.partials + 6 * kRedBlocks, ng, L0.slots + S_NB2);
  klaunch(k_set_slot, 1, 32, s, L0.slots, S_TOL, tol);
  klaunch(k_set_slot, 1, 32, s, L0.slots, S_MAXIT, (double)h.p.max_iter);
  klaunch(k_set_state, 1, 32, s, h.it_dev, active, h.it_dev + 2, h.status_dev, 0, 1, 0, 0);
  launches += 5;
  AMG_LAUNCH_CHECK();
  double *w = h.q;
  int it = 0, status = AMG_ERR_NOT_CONVERGED;
  std::vector<double> hist;
  double nb2 = 1.0;
  bool first = true;
  int *st_host = reinterpret_cast<int *>(h.host_pinned + 32);
  for (;;) {
    true_residual(h, S_RR, s, launches);
    AMG_CUDA(cudaMemcpyAsync(h.host_pinned, L0.slots, sizeof(double) * kNumSlots, cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (first) {
      nb2 = h.host_pinned[S_NB2];
      if (!(nb2 > 0.0)) {
        nb2 = 1.0;
        klaunch(k_set_slot, 1, 32, s, L0.slots, S_NB2, 1.0);
        ++launches;
      }
      hist.push_back(std::sqrt(h.host_pinned[S_RR] / nb2));
      first = false;
    }
    const double rel = std::sqrt(h.host_pinned[S_RR] / nb2);
    if (!std::isfinite(rel)) { status = AMG_ERR_NAN; break; }
    if (rel <= tol) { status = AMG_OK; break; }
    if (it >= h.p.max_iter) { status = AMG_ERR_NOT_CONVERGED; break; }
    klaunch(k_fg_start, ng, kThreads, s, n, h.r, h.V, L0.slots, S_RR, h.fg, m);
    klaunch(k_set_state, 1, 32, s, h.it_dev, active, h.it_dev + 2, h.status_dev, -1, 1, 0, 0);
    launches += 2;
    AMG_LAUNCH_CHECK();
    int jused = 0, dst = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = h.V + (size_t)j * n, *zj = h.Z + (size_t)j * n;
      const int64_t before = eng.launches;
      eng.precond(vj, zj, active, false);
      {  // w = A z_j in FP64
        SellArgs<double> a{};
        a.n = n;
        a.nslices = L0.nslices;
        a.sptr = L0.sptr64;
        a.scol = L0.scol64;
        a.sval = L0.sval64;
        a.x = zj;
        a.out = w;
        a.pred = active;
        klaunch(k_sell<double, double, E_Y, false, false>, outer_grid(L0), kThreads, s, a);
        eng.check();
      }
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        klaunch(k_mdot, ng, kThreads, s, n, h.V, j + 1, w, h.gpart, active);
        klaunch(k_fin_mdot, 1, 1024, s, h.gpart, ng, j + 1, h.H, m, j, h.hc, pass, active);
        klaunch(k_maxpy, ng, kThreads, s, n, h.V, j + 1, h.hc, w, active);
        eng.launches += 3;
        AMG_LAUNCH_CHECK();
      }
      klaunch(k_dot64, ng, kThreads, s, n, w, w, L0.partials + 6 * kRedBlocks, active);
      klaunch(k_fg_normalize, ng, kThreads, s, n, w, h.V + (size_t)(j + 1) * n, L0.partials + 6 * kRedBlocks, ng,
                                             h.H, m, j, active);
      klaunch(k_fg_givens, 1, 32, s, h.H, m, j, m, h.fg, L0.slots, h.hist, h.it_dev, active, h.status_dev);
      eng.launches += 3;
      AMG_LAUNCH_CHECK();
      (void)before;
      AMG_CUDA(cudaMemcpyAsync(st_host, h.it_dev, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
      it = st_host[0];
      dst = st_host[4];
      jused = j + 1;
      if (dst != 0) break;
    }
    klaunch(k_fg_trisolve, 1, 32, s, h.H, m, jused, m, h.fg);
    klaunch(k_fg_xupdate, ng, kThreads, s, n, h.x, h.Z, jused, h.fg + 3 * m + 1);
    launches += 2;
    AMG_LAUNCH_CHECK();
    if (dst == AMG_ERR_NAN) { status = AMG_ERR_NAN; break; }
  }
  hist.resize((size_t)it + 1);
  if (it > 0)
    AMG_CUDA(cudaMemcpyAsync(&hist[1], h.hist + 1, sizeof(double) * (size_t)it, cudaMemcpyDeviceToHost, s));
  launches += eng.launches;
  AMG_CUDA(cudaMemcpyAsync(h.host_pinned, L0.slots, sizeof(double) * kNumSlots, cudaMemcpyDeviceToHost, s));
  copy_out(x, h.x, n, s);
  AMG_CUDA(cudaStreamSynchronize(s));
  h.info.final_relres = std::sqrt(h.host_pinned[S_RR] / nb2);
  trace_collect(h, it, s);
  h.info.iters = it;
  h.info.status = status;
  h.info.kernel_launches = launches;
  if (iters) *iters = it;
  if (res_hist) std::memcpy(res_hist, hist.data(), sizeof(double) * hist.size());
  return status;
}

__global__ void k_bset(int32_t nsys, const double *__restrict__ bslots, double tol, int *__restrict__ bact,
                       int *__restrict__ bit) {
  pdl_wait_and_trigger();
  // bact[0..nsys) active, bact[nsys] count, bact[nsys+1 ..] restart flags; bit: iters, status
  __shared__ int nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int32_t s = threadIdx.x; s < nsys; s += blockDim.x) {
    const double rel = sqrt(bslots[(int64_t)S_RR * nsys + s] / bslots[(int64_t)S_NB2 * nsys + s]);
    const int a = rel > tol ? 1 : 0;
    bact[s] = a;
    bact[nsys + 1 + s] = 1;
    bit[s] = 0;
    bit[nsys + s] = a ? kIterating : AMG_OK;
    if (a) atomicAdd(&nact, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) bact[nsys] = nact;
}

// restart the systems whose updated residual met tol but whose true residual did not
__global__ void k_brestart(int32_t nsys, const double *__restrict__ bslots, double tol, int max_iter,
                           int *__restrict__ bact, int *__restrict__ bit) {
  pdl_wait_and_trigger();
  __shared__ int nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int32_t s = threadIdx.x; s < nsys; s += blockDim.x) {
    const double rel = sqrt(bslots[(int64_t)S_TRUE_RR * nsys + s] / bslots[(int64_t)S_NB2 * nsys + s]);
    int &st = bit[nsys + s];
    if (st == kUpdatedConverged) st = rel <= tol ? AMG_OK : (bit[s] >= max_iter ? AMG_ERR_NOT_CONVERGED : kIterating);
    if (st == kIterating) {
      bact[s] = 1;
      bact[nsys + 1 + s] = 1;
      atomicAdd(&nact, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) bact[nsys] = nact;
}

__global__ void k_fix_zero_norm(int32_t nsys, double *__restrict__ bslots) {
  pdl_wait_and_trigger();
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x)
    if (!(bslots[(int64_t)S_NB2 * nsys + s] > 0.0)) bslots[(int64_t)S_NB2 * nsys + s] = 1.0;
}

template <class MV, class VT>
int run_solve_batch_t(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *relres,
                      cudaStream_t s) {
  Level &L0 = h.lev[0];
  const int32_t n = L0.n, ns = h.nsys;
  Engine<MV, VT> eng(h, s);
  Engine<double, double> e64(h, s);
  int64_t launches = 0;
  copy_in(h.b, b, n, s);
  copy_in(h.x, x, n, s);
  e64.segdot(0, 1, h.b, h.b, nullptr, nullptr, nullptr, nullptr, S_NB2, nullptr);
  klaunch(k_fix_zero_norm, grid_for(ns, kThreads, 152), kThreads, s, ns, L0.bslots);
  klaunch(k_residual64, outer_grid(L0), kThreads, s, n, L0.nslices, (const int64_t *)L0.sptr64,
          (const int32_t *)L0.scol64, (const double *)L0.sval64, (const double *)h.x, (const double *)h.b, h.r,
          L0.partials + 7 * kRedBlocks);
  e64.segdot(0, 1, h.r, h.r, nullptr, nullptr, nullptr, nullptr, S_RR, nullptr);
  klaunch(k_bset, 1, 1024, s, ns, (const double *)L0.bslots, tol, h.bactive, h.bit);
  AMG_CUDA(cudaMemsetAsync(h.it_dev, 0, sizeof(int), s));
  launches += 3;
  AMG_LAUNCH_CHECK();
  // capture one iteration of all systems
  if (h.graph_exec) {
    cudaGraphExecDestroy(h.graph_exec);
    cudaGraphDestroy(h.graph);
    h.graph_exec = nullptr;
  }
  if (h.p.use_graph) {
    AMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    eng.fcg_iteration_batched(tol);
    AMG_CUDA(cudaStreamEndCapture(s, &h.graph));
    AMG_CUDA(cudaGraphInstantiate(&h.graph_exec, h.graph, 0));
    h.graph_launches = eng.launches;
    eng.launches = 0;
    h.graph_kind = -1;  // not the single-system iteration
  }
  int *pin = reinterpret_cast<int *>(h.host_pinned + 32);
  int rounds = 0;
  for (;;) {
    AMG_CUDA(cudaMemcpyAsync(pin, h.bactive + ns, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (pin[0] > 0 && rounds < 100 * h.p.max_iter) {
      if (h.p.use_graph) {
        AMG_CUDA(cudaGraphLaunch(h.graph_exec, s));
        launches += h.graph_launches;
      } else {
        eng.fcg_iteration_batched(tol);
      }
      ++rounds;
      continue;
    }
    // every system stopped: check the true residuals, restart those that miss tol
    klaunch(k_residual64, outer_grid(L0), kThreads, s, n, L0.nslices, (const int64_t *)L0.sptr64,
            (const int32_t *)L0.scol64, (const double *)L0.sval64, (const double *)h.x, (const double *)h.b, h.r,
            L0.partials + 7 * kRedBlocks);
    e64.segdot(0, 1, h.r, h.r, nullptr, nullptr, nullptr, nullptr, S_TRUE_RR, nullptr);
    klaunch(k_brestart, 1, 1024, s, ns, (const double *)L0.bslots, tol, h.p.max_iter, h.bactive, h.bit);
    launches += 2;
    AMG_CUDA(cudaMemcpyAsync(pin, h.bactive + ns, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (pin[0] == 0 || rounds >= 100 * h.p.max_iter) break;
  }
  launches += eng.launches + e64.launches;
  std::vector<int> bit(2 * ns);
  std::vector<double> sl((size_t)kNumSlots * ns);
  AMG_CUDA(cudaMemcpyAsync(bit.data(), h.bit, sizeof(int) * 2 * ns, cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaMemcpyAsync(sl.data(), L0.bslots, sizeof(double) * kNumSlots * ns, cudaMemcpyDeviceToHost, s));
  copy_out(x, h.x, n, s);
  AMG_CUDA(cudaStreamSynchronize(s));
  int status = AMG_OK, maxit = 0;
  double worst = 0.0;
  for (int32_t q = 0; q < ns; ++q) {
    const double rel = std::sqrt(sl[(size_t)S_TRUE_RR * ns + q] / sl[(size_t)S_NB2 * ns + q]);
    if (iters) iters[q] = bit[q];
    if (relres) relres[q] = rel;
    maxit = std::max(maxit, bit[q]);
    worst = std::max(worst, rel);
    const int st = bit[ns + q];
    if (st != AMG_OK && status == AMG_OK) status = st < 0 ? st : AMG_ERR_NOT_CONVERGED;
  }
  h.info.iters = maxit;
  h.info.final_relres = worst;
  h.info.status = status;
  h.info.kernel_launches = launches;
  return status;
}

// row tiles of level L for the per-system inner products: every tile lies in
// one system and holds at most `tile` rows
void build_tiles(Hierarchy &h, Level &L, int32_t tile, cudaStream_t s) {
  const int32_t ns = h.nsys;
  std::vector<int32_t> trow, stile(ns + 1, 0);
  for (int32_t q = 0; q < ns; ++q) {
    stile[q] = (int32_t)trow.size();
    for (int32_t r = L.sys_off_host[q]; r < L.sys_off_host[q + 1]; r += tile) trow.push_back(r);
  }
  stile[ns] = (int32_t)trow.size();
  L.ntiles = (int32_t)trow.size();
  L.seg_tile = tile;
  trow.push_back(L.n);
  L.tile_row = h.arena.get<int32_t>(trow.size());
  L.sys_tile = h.arena.get<int32_t>(ns + 1);
  L.tpart = h.arena.get<double>(3 * (size_t)L.ntiles + 1);
  AMG_CUDA(cudaMemcpyAsync(L.tile_row, trow.data(), sizeof(int32_t) * trow.size(), cudaMemcpyHostToDevice, s));
  AMG_CUDA(cudaMemcpyAsync(L.sys_tile, stile.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice, s));
  AMG_CUDA(cudaStreamSynchronize(s));  // trow / stile leave scope
}

// per-level system map, row tiles and per-system scalars of a batch
void prepare_batched(Hierarchy &h, cudaStream_t s) {
  const int32_t ns = h.nsys;
  constexpr int32_t kTile = 2048;
  for (int k = 0; k < h.L; ++k) {
    Level &L = h.lev[k];
    L.sys_of = h.arena.get<int32_t>((size_t)L.n + 1);
    klaunch(k_sys_of, ew_grid(L.n), kThreads, s, L.n, ns, (const int32_t *)L.sys_off, L.sys_of);
    L.slive = h.arena.get<unsigned char>((size_t)L.nslices + 1);
    AMG_CUDA(cudaMemsetAsync(L.slive, 1, (size_t)L.nslices + 1, s));
    build_tiles(h, L, kTile, s);
    L.bslots = h.arena.get<double>((size_t)kNumSlots * ns);
    L.bflag = h.arena.get<int>((size_t)ns + 1);
    AMG_CUDA(cudaMemsetAsync(L.bslots, 0, sizeof(double) * kNumSlots * ns, s));
    AMG_CUDA(cudaMemsetAsync(L.bflag, 0, sizeof(int) * (ns + 1), s));
  }
  h.bit = h.arena.get<int>(2 * (size_t)ns);
  h.bactive = h.arena.get<int>(2 * (size_t)ns + 2);
  AMG_LAUNCH_CHECK();
}

// Autotuner of the launch shapes (setup time).  For every level the SpMV is
// timed with CUDA events over candidate grid sizes (multiples of the 152 SMs up
// to one warp per slice) and the smallest grid within 3 % of the fastest is
// kept, for the launches that fuse inner products among the grids within the
// partial-sum capacity; for a batch, the row tile of the per-system inner products is chosen
// the same way.  The shapes change the grouping of partial sums only.
template <class MV, class VT>
void autotune_t(Hierarchy &h, cudaStream_t s) {
  Engine<MV, VT> eng(h, s);
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](auto &&launch) {
    for (int r = 0; r < 2; ++r) launch();
    AMG_CUDA(cudaEventRecord(e0, s));
    constexpr int kReps = 5;
    for (int r = 0; r < kReps; ++r) launch();
    AMG_CUDA(cudaEventRecord(e1, s));
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms / kReps;
  };
  auto pick = [](const std::vector<std::pair<int, float>> &t) {  // smallest within 3 % of the best
    float best = t[0].second;
    for (auto &c : t) best = std::min(best, c.second);
    for (auto &c : t)
      if (c.second <= 1.03f * best) return c.first;
    return t[0].first;
  };
  try {
    for (int k = 0; k < h.L; ++k) {
      Level &L = h.lev[k];
      DevBuf<VT> x((size_t)L.n + 1), y((size_t)L.n + 1);
      AMG_CUDA(cudaMemsetAsync(x.p, 0, sizeof(VT) * (L.n + 1), s));
      // the plain product at each grid; launches with fused inner products take
      // the best grid within the partial-sum capacity
      const int gfull = full_plain_grid(L);
      std::vector<std::pair<int, float>> t, tr;
      for (int g : {152, 304, 608, 912, 1216, 2432, 4864, 1 << 30}) {
        const int gg = std::min(g, gfull);
        if (!t.empty() && t.back().first == gg) continue;
        L.sell_plain_blocks = gg;
        const SellArgs<VT> a = eng.sell_args(k, x.p, y.p, nullptr);
        t.push_back({gg, time_it([&] { eng.template sell<E_Y>(a, k); })});
        if (gg <= kRedBlocks) tr.push_back(t.back());
      }
      L.sell_plain_blocks = pick(t);
      L.sell_blocks = pick(tr);
      if (h.batched && k < h.L - 1) {
        std::vector<std::pair<int, float>> tt;
        for (int tile : {1024, 2048, 4096, 8192}) {
          build_tiles(h, L, tile, s);
          tt.push_back({tile, time_it([&] {
                          eng.segdot(k, 2, x.p, x.p, y.p, y.p, nullptr, nullptr, S_RHO1, nullptr);
                        })});
        }
        build_tiles(h, L, pick(tt), s);
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  AMG_CUDA(cudaEventDestroy(e0));
  AMG_CUDA(cudaEventDestroy(e1));
}

template <class MV, class VT>
void run_precond_t(Hierarchy &h, const double *b, double *x, cudaStream_t s) {
  Engine<MV, VT> eng(h, s);
  const int32_t n = h.lev[0].n;
  if (!h.batched) trace_reset(h, s);
  copy_in(h.r, b, n, s);
  eng.precond(h.r, h.z, nullptr, false);
  copy_out(x, h.z, n, s);
  AMG_CUDA(cudaStreamSynchronize(s));
  if (!h.batched) trace_collect(h, 1, s);
  h.info.kernel_launches = eng.launches;
}

template <class MV, class VT>
void run_spmv_t(Hierarchy &h, int k, const void *x, void *y, cudaStream_t s) {
  Engine<MV, VT> eng(h, s);
  SellArgs<VT> a = eng.sell_args(k, static_cast<const VT *>(x), static_cast<VT *>(y), nullptr);
  eng.template sell<E_Y>(a, k);
}

}  // namespace

#define AMG_DISPATCH(prec, CALL)                                   \
  switch (prec) {                                                  \
    case AMG_PREC_F64: { using MV = double; using VT = double; CALL; break; } \
    case AMG_PREC_F32: { using MV = float; using VT = float; CALL; break; }   \
    default: { using MV = __nv_bfloat16; using VT = float; CALL; break; }     \
  }

void set_poly(Hierarchy &h, int level, const double *coef, cudaStream_t s) {
  Level &L = h.lev[level];
  if (!coef) {  // back to damped Jacobi on this level (the buffer stays for a later set)
    L.poly_off = true;
    configure_tail(h, s);
    h.graph_kind = -1;
    return;
  }
  L.poly_off = false;
  const size_t cnt = (size_t)L.n * 3;
  DevBuf<double> tmp(cnt);
  const cudaMemcpyKind kind = pointer_kind(coef) == PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  AMG_CUDA(cudaMemcpyAsync(tmp.p, coef, sizeof(double) * cnt, kind, s));
  if (h.p.precision == AMG_PREC_F64) {
    if (!L.poly) L.poly = h.arena.get<double>(cnt);
    AMG_CUDA(cudaMemcpyAsync(L.poly, tmp.p, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s));
  } else {
    if (!L.poly) L.poly = h.arena.get<float>(cnt);
    klaunch(k_copy_cast<float>, ew_grid((int64_t)cnt), kThreads, s, (int32_t)cnt, tmp.p, (float *)L.poly);
    AMG_LAUNCH_CHECK();
  }
  AMG_CUDA(cudaStreamSynchronize(s));
  configure_tail(h, s);
  h.graph_kind = -1;  // the captured iteration no longer matches: capture again
}

void make_row_data(Hierarchy &h, Level &L, const double *diag, cudaStream_t s) {
  if (h.p.precision == AMG_PREC_F64)
    make_row_data_t<double>(h, L, diag, s);
  else
    make_row_data_t<float>(h, L, diag, s);
}

void prepare_solve(Hierarchy &h, cudaStream_t s) {
  AMG_DISPATCH(h.p.precision, (prepare_t<MV, VT>(h, s)));
}

int run_solve_batch(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *relres,
                    cudaStream_t s) {
  int rc = 0;
  AMG_DISPATCH(h.p.precision, (rc = run_solve_batch_t<MV, VT>(h, b, x, tol, iters, relres, s)));
  return rc;
}

int run_solve(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *res_hist,
              cudaStream_t s) {
  int rc = 0;
  if (h.p.outer == 1) {
    AMG_DISPATCH(h.p.precision, (rc = run_fgmres_t<MV, VT>(h, b, x, tol, iters, res_hist, s)));
  } else {
    AMG_DISPATCH(h.p.precision, (rc = run_solve_t<MV, VT>(h, b, x, tol, iters, res_hist, s)));
  }
  return rc;
}

void run_precond(Hierarchy &h, const double *b, double *x, cudaStream_t s) {
  AMG_DISPATCH(h.p.precision, (run_precond_t<MV, VT>(h, b, x, s)));
}

void run_spmv(Hierarchy &h, int level, const void *x, void *y, cudaStream_t s) {
  AMG_DISPATCH(h.p.precision, (run_spmv_t<MV, VT>(h, level, x, y, s)));
}

}  // namespace amg
