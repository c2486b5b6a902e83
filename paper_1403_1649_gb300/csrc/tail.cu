// tail.cu -- the coarse tail of the cycle in one thread-block-cluster launch.
//
// Below the first two levels every level is small (tens of thousands of rows
// and less), so a kernel per step is dominated by launch and memory latency.
// This kernel runs, for levels t..L-1, either one V-cycle (Alg. 4) or the whole
// Krylov-accelerated coarse part of Alg. 5 at level t (two V-cycles, the inner
// products, the test ||r~|| <= t ||r|| and the combination) inside a single
// cluster of CL blocks (CL = 8, or CL = 1: one block, which needs no co-scheduled
// SMs).  Phases are separated by cluster barriers;
// inner products are reduced through distributed shared memory in a fixed rank
// order, so every block computes the same value and takes the same branch.
// Vectors written inside the kernel are read with ld.global.cg (L2), never
// through a possibly stale L1 line.
#include <cooperative_groups.h>

#include "amg_internal.cuh"

namespace cg = cooperative_groups;

namespace amg {

constexpr int kTailThreads = 1024;
constexpr int kTailWarps = kTailThreads / 32;

template <class T> __device__ __forceinline__ T ldc(const T *p) { return __ldcg(p); }
__device__ __forceinline__ float to_vt(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ float to_vt(float v, float) { return v; }
__device__ __forceinline__ double to_vt(double v, double) { return v; }

struct TailCtx {
  cg::cluster_group cl;
  int nblocks, rank, gtid, gsize, gwarp, nwarps, lane;
  int buf;
};

// cluster-wide sum of v[0..nv): block reduction, publish, cluster barrier, sum
// of the blocks' partials in rank order (identical in every block)
__device__ void cluster_sum(TailCtx &c, double v0, double v1, double v2, double out[3]) {
  __shared__ double s_warp[kTailWarps][3];
  __shared__ double s_red[2][4];
  const int wid = threadIdx.x >> 5;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  v2 = warp_sum(v2);
  if (c.lane == 0) {
    s_warp[wid][0] = v0;
    s_warp[wid][1] = v1;
    s_warp[wid][2] = v2;
  }
  __syncthreads();
  if (wid == 0) {
    double a0 = c.lane < kTailWarps ? s_warp[c.lane][0] : 0.0;
    double a1 = c.lane < kTailWarps ? s_warp[c.lane][1] : 0.0;
    double a2 = c.lane < kTailWarps ? s_warp[c.lane][2] : 0.0;
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (c.lane == 0) {
      s_red[c.buf][0] = a0;
      s_red[c.buf][1] = a1;
      s_red[c.buf][2] = a2;
    }
  }
  c.cl.sync();
  out[0] = out[1] = out[2] = 0.0;
  for (int r = 0; r < c.nblocks; ++r) {
    const double *peer = c.cl.map_shared_rank(&s_red[c.buf][0], r);
    out[0] += peer[0];
    out[1] += peer[1];
    out[2] += peer[2];
  }
  c.buf ^= 1;
}

// y = sum_e A(row, e) * xf(col) over the SELL slice of this warp
template <class MV, class VT, class XF>
__device__ __forceinline__ VT sell_row(const TailLevel &L, int32_t sl, int lane, XF xf) {
  const int64_t base = L.sptr[sl];
  const int32_t width = (int32_t)((L.sptr[sl + 1] - base) >> 5);
  const int32_t *cp = L.scol + base + lane;
  const MV *vp = static_cast<const MV *>(L.sval) + base + lane;
  const int4 *pp = L.spair + (base >> 1) + lane;  // FP32 values: {column, value} pairs
  VT y = VT(0);
  for (int32_t e = 0; e < width; e += 4) {
    int32_t cc[4];
    MV vv[4];
    if constexpr (std::is_same<MV, float>::value) {
#pragma unroll
      for (int q = 0; q < 4; q += 2)
        if (e + q < width) {
          const int4 pr = pp[16 * (e + q)];
          cc[q] = pr.x;
          vv[q] = __int_as_float(pr.y);
          cc[q + 1] = pr.z;
          vv[q + 1] = __int_as_float(pr.w);
        }
    } else if constexpr (std::is_same<MV, __nv_bfloat16>::value) {  // entries 2j, 2j+1 adjacent
#pragma unroll
      for (int q = 0; q < 4; q += 2)
        if (e + q < width) {
          const int64_t at = base + 32 * (int64_t)(e + q) + 2 * lane;
          cc[q] = L.scol[at];
          cc[q + 1] = L.scol[at + 1];
          vv[q] = static_cast<const MV *>(L.sval)[at];
          vv[q + 1] = static_cast<const MV *>(L.sval)[at + 1];
        }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (e + q < width) {
          cc[q] = cp[32 * (e + q)];
          vv[q] = vp[32 * (e + q)];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (e + q < width) y += to_vt(vv[q], VT(0)) * xf(cc[q]);
  }
  const int32_t row = sl * 32 + lane;
  if (L.sdiag && row < L.n) y += (VT)L.sdiag[row] * xf(row);
  return y;
}

// one V-cycle (Alg. 4) from level t with a zero initial guess: out = M_t rhs
template <class MV, class VT>
__device__ void tail_vcycle(TailCtx &c, const TailArgs &a, const VT *rhs_t, VT *out_t) {
  const int L = a.L;
  // down: residual after the Jacobi pre-smoothing x0 = wd * rhs, then restriction
  for (int k = a.t; k < L - 1; ++k) {
    const TailLevel &Lk = a.lev[k];
    const VT *rhs = k == a.t ? rhs_t : static_cast<const VT *>(Lk.bc);
    const VT *wd = static_cast<const VT *>(Lk.wd);
    VT *r = static_cast<VT *>(Lk.r);
    for (int32_t sl = c.gwarp; sl < Lk.nslices; sl += c.nwarps) {
      const VT y = sell_row<MV, VT>(Lk, sl, c.lane, [&](int32_t j) { return wd[j] * ldc(rhs + j); });
      const int32_t row = sl * 32 + c.lane;
      if (row < Lk.n) r[row] = ldc(rhs + row) - y;
    }
    c.cl.sync();
    const TailLevel &Lc = a.lev[k + 1];
    const VT *pw = static_cast<const VT *>(Lk.pw);
    VT *bc = static_cast<VT *>(Lc.bc);
    for (int32_t I = c.gtid; I < Lk.nc; I += c.gsize) {
      VT s = VT(0);
      for (int32_t m = Lk.aptr[I]; m < Lk.aptr[I + 1]; ++m) {
        const int32_t i = Lk.amem[m];
        s += pw[i] * ldc(r + i);
      }
      bc[I] = s;
    }
    c.cl.sync();
  }
  {  // exact coarsest solve (dense inverse), one warp per row
    const TailLevel &Lc = a.lev[L - 1];
    const VT *b = L - 1 == a.t ? rhs_t : static_cast<const VT *>(Lc.bc);
    VT *x = L - 1 == a.t ? out_t : static_cast<VT *>(Lc.xc);
    for (int32_t i = c.gwarp; i < a.nL; i += c.nwarps) {
      double s = 0.0;
      for (int32_t j = c.lane; j < a.nL; j += 32) s += a.Ainv[(int64_t)i * a.nL + j] * (double)ldc(b + j);
      s = warp_sum(s);
      if (c.lane == 0) x[i] = (VT)s;
    }
    c.cl.sync();
  }
  // up: x = x0 + P x_{k+1} (formed on the fly), then x += wd * (rhs - A x)
  for (int k = L - 2; k >= a.t; --k) {
    const TailLevel &Lk = a.lev[k];
    const VT *rhs = k == a.t ? rhs_t : static_cast<const VT *>(Lk.bc);
    VT *out = k == a.t ? out_t : static_cast<VT *>(Lk.xc);
    const VT *wd = static_cast<const VT *>(Lk.wd);
    const VT *pw = static_cast<const VT *>(Lk.pw);
    const VT *xn = static_cast<const VT *>(a.lev[k + 1].xc);
    auto xk = [&](int32_t j) { return wd[j] * ldc(rhs + j) + pw[j] * ldc(xn + Lk.agg[j]); };
    for (int32_t sl = c.gwarp; sl < Lk.nslices; sl += c.nwarps) {
      const VT y = sell_row<MV, VT>(Lk, sl, c.lane, xk);
      const int32_t row = sl * 32 + c.lane;
      if (row < Lk.n) {
        const VT xi = xk(row);
        out[row] = xi + wd[row] * (ldc(rhs + row) - y);
      }
    }
    c.cl.sync();
  }
}

template <class MV, class VT, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kTailThreads, 1) k_tail(TailArgs a) {
  pdl_wait_and_trigger();  // launched like the other solve kernels (programmatic dependent launch)
  if (a.pred && *a.pred == 0) return;  // uniform: every block reads the same flag
  TailCtx c{cg::this_cluster()};
  c.nblocks = CL;
  c.rank = (int)c.cl.block_rank();
  c.gtid = c.rank * kTailThreads + threadIdx.x;
  c.gsize = CL * kTailThreads;
  c.lane = threadIdx.x & 31;
  c.gwarp = c.gtid >> 5;
  c.nwarps = c.gsize >> 5;
  c.buf = 0;
  const TailLevel &T = a.lev[a.t];
  if (a.mode == 0) {
    tail_vcycle<MV, VT>(c, a, static_cast<const VT *>(T.bc), static_cast<VT *>(T.xc));
    return;
  }
  // Alg. 5 coarse part at level t (rhs r = bc_t, result in xc_t)
  const VT *r = static_cast<const VT *>(T.bc);
  VT *cv = static_cast<VT *>(T.c), *v = static_cast<VT *>(T.v), *rt = static_cast<VT *>(T.rt);
  VT *dv = static_cast<VT *>(T.d), *w = static_cast<VT *>(T.w), *x = static_cast<VT *>(T.xc);
  tail_vcycle<MV, VT>(c, a, r, cv);
  double s3[3];
  {  // v = A c; rho_1, alpha_1
    double p0 = 0.0, p1 = 0.0;
    for (int32_t sl = c.gwarp; sl < T.nslices; sl += c.nwarps) {
      const VT y = sell_row<MV, VT>(T, sl, c.lane, [&](int32_t j) { return ldc(cv + j); });
      const int32_t row = sl * 32 + c.lane;
      if (row < T.n) {
        v[row] = y;
        const double ci = (double)ldc(cv + row), ri = (double)ldc(r + row);
        if (a.gmres) {
          p0 += (double)y * (double)y;
          p1 += (double)y * ri;
        } else {
          p0 += ci * (double)y;
          p1 += ci * ri;
        }
      }
    }
    cluster_sum(c, p0, p1, 0.0, s3);
  }
  const double rho1 = s3[0], a1 = s3[1], s1 = a1 / rho1;
  {  // r~ = r - (alpha_1/rho_1) v and the two norms
    double p0 = 0.0, p1 = 0.0;
    for (int32_t i = c.gtid; i < T.n; i += c.gsize) {
      const VT ri = ldc(r + i);
      const VT t = ri - (VT)s1 * ldc(v + i);
      rt[i] = t;
      p0 += (double)t * (double)t;
      p1 += (double)ri * (double)ri;
    }
    cluster_sum(c, p0, p1, 0.0, s3);
  }
  if (sqrt(s3[0]) <= a.kt * sqrt(s3[1])) {
    for (int32_t i = c.gtid; i < T.n; i += c.gsize) x[i] = (VT)s1 * ldc(cv + i);
    c.cl.sync();  // no block leaves while a peer may still read its shared memory
    return;
  }
  tail_vcycle<MV, VT>(c, a, rt, dv);
  {  // w = A d; gamma, beta, alpha_2
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int32_t sl = c.gwarp; sl < T.nslices; sl += c.nwarps) {
      const VT y = sell_row<MV, VT>(T, sl, c.lane, [&](int32_t j) { return ldc(dv + j); });
      const int32_t row = sl * 32 + c.lane;
      if (row < T.n) {
        w[row] = y;
        const double di = (double)ldc(dv + row), vi = (double)ldc(v + row), ti = (double)ldc(rt + row);
        if (a.gmres) {
          p0 += (double)y * vi;
          p1 += (double)y * (double)y;
          p2 += (double)y * ti;
        } else {
          p0 += di * vi;
          p1 += di * (double)y;
          p2 += di * ti;
        }
      }
    }
    cluster_sum(c, p0, p1, p2, s3);
  }
  const double gam = s3[0], bet = s3[1], a2 = s3[2];
  const double rho2 = bet - gam * gam / rho1;
  const VT cc = (VT)(s1 - gam * a2 / (rho1 * rho2)), cd = (VT)(a2 / rho2);
  for (int32_t i = c.gtid; i < T.n; i += c.gsize) x[i] = cc * ldc(cv + i) + cd * ldc(dv + i);
  c.cl.sync();  // no block leaves while a peer may still read its shared memory
}

template <class MV, class VT>
void tail_launch(const TailArgs &a, int blocks, cudaStream_t s) {
  if (blocks == 1)
    klaunch(k_tail<MV, VT, 1>, 1, kTailThreads, s, a);
  else
    klaunch(k_tail<MV, VT, 8>, 8, kTailThreads, s, a);
  AMG_LAUNCH_CHECK();
}

template void tail_launch<double, double>(const TailArgs &, int, cudaStream_t);
template void tail_launch<float, float>(const TailArgs &, int, cudaStream_t);
template void tail_launch<__nv_bfloat16, float>(const TailArgs &, int, cudaStream_t);

}  // namespace amg
