// amg_internal.cuh -- shared declarations of the GB300 aggregation AMG library.
//
// Device data layout (per level k of the hierarchy, all in HBM):
//   setup CSR   rp[n+1] int32, ci[nnz] int32, val[nnz] f64   (bit-exact level matrix)
//   solve SELL  slices of 32 rows, column-major inside a slice: entry e of row
//               32*s + l sits at sptr[s] + 32*e + l; padding has col = own row,
//               value 0.  Values in the preconditioner precision (f64/f32/bf16);
//               in f32/bf16 the diagonal is split off into sdiag[n] f32.
//   agg[n]      coarse id of every node;  pw[n] the nonzero of row i of P_k
//   aptr[nc+1], amem[n]   members of every aggregate in ascending fine index
//   wd[n]       omega / A_ii  (damped Jacobi, Eq. damped Jacobi)
//   vectors     cycle work vectors in the vector type of the precision
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/amg.h"

namespace amg {

// ---------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};

void set_last_error(const std::string &m);

#define AMG_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e__ = (call);                                                                 \
    if (e__ != cudaSuccess)                                                                   \
      throw ::amg::Error{AMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__) +   \
                                           " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"}; \
  } while (0)

#define AMG_LAUNCH_CHECK() AMG_CUDA(cudaGetLastError())

// kernels launched by the calling thread (setup statistics)
int64_t &launch_counter();
#define AMG_COUNT() (++::amg::launch_counter())

// two timing-free events, destroyed with their owner (also when a call throws)
struct EventPair {
  cudaEvent_t e[2] = {nullptr, nullptr};
  EventPair() {
    try {
      AMG_CUDA(cudaEventCreateWithFlags(&e[0], cudaEventDisableTiming));
      AMG_CUDA(cudaEventCreateWithFlags(&e[1], cudaEventDisableTiming));
    } catch (...) {
      release();
      throw;
    }
  }
  ~EventPair() { release(); }
  void release() {
    for (cudaEvent_t &x : e)
      if (x) cudaEventDestroy(x), x = nullptr;
  }
  EventPair(const EventPair &) = delete;
  EventPair &operator=(const EventPair &) = delete;
};

// ---------------------------------------------------------------- device memory
// Device memory comes from one stream-ordered pool per device that keeps freed
// blocks (release threshold = unlimited), so repeated setups do not pay for
// cudaMalloc/cudaFree and never synchronise the device to free scratch.
cudaMemPool_t device_pool();
// a recycled 64-double pinned host buffer and a recycled non-blocking stream of
// the current device; returned by amg_free
double *pinned_scratch_get();
void pinned_scratch_put(double *p);
cudaStream_t stream_get();
void stream_put(cudaStream_t st);
// stream of the API call in progress on this thread (allocation order)
cudaStream_t &current_stream();

inline void *pool_alloc(size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  AMG_CUDA(cudaMallocFromPoolAsync(&p, bytes, device_pool(), current_stream()));
  return p;
}
inline void pool_free(void *p) {
  if (p) cudaFreeAsync(p, current_stream());
}

// All allocations of a hierarchy go through one arena so that amg_free
// releases everything, also after a failure half way through setup.
struct Arena {
  std::vector<void *> blocks;
  void *alloc(size_t bytes) {
    void *p = pool_alloc(bytes);
    blocks.push_back(p);
    return p;
  }
  template <class T>
  T *get(size_t n) { return static_cast<T *>(alloc(n * sizeof(T))); }
  void release() {
    for (void *p : blocks) pool_free(p);
    blocks.clear();
  }
};

// Temporary device buffer returned to the pool at scope exit (setup scratch).
template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  explicit DevBuf(size_t count) { resize(count); }
  void resize(size_t count) {
    pool_free(p);
    n = count;
    p = static_cast<T *>(pool_alloc((count ? count : 1) * sizeof(T)));
  }
  ~DevBuf() { pool_free(p); }
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
};

// ---------------------------------------------------------------- levels
constexpr int kSlice = 32;          // SELL slice height = warp width
constexpr int kMaxLevels = 32;
constexpr int kMaxDense = 4096;     // largest coarsest level factorised densely
constexpr int kRedBlocks = 1216;    // 8 x 152 SMs: grid of the reduction kernels
constexpr int kNumSlots = 32;       // Krylov scalars per level

// scalar slots of a level (double) used by the K-cycle coarse step at that level
enum Slot {
  S_RHO1 = 0, S_A1, S_S1, S_NRT2, S_NR2, S_GAM, S_BET, S_A2, S_CC, S_CD,
  S_TAKEN,  // second inner steps of Alg. 5 taken at this level in the current solve
  // outer Krylov (level 0 only)
  S_PQ = 12, S_PR, S_ALPHA, S_BETA, S_RR, S_NB2, S_REL, S_ZQ, S_TRUE_RR, S_TOL, S_MAXIT,
};

struct Level {
  int32_t n = 0, nc = 0, mis_rounds = 0;
  int64_t nnz = 0;
  double omega = 0.0;
  double *omega_dev = nullptr;  // the estimated weight on the device (omega_mode 0)
  // setup CSR (FP64, exact)
  int32_t *rp = nullptr, *ci = nullptr;
  double *val = nullptr;
  double *B = nullptr;  // near-null vector B_k
  // transfer
  int32_t *agg = nullptr, *aptr = nullptr, *amem = nullptr;
  double *pw64 = nullptr;  // P weights in FP64 (exported)
  // summation plan of the Galerkin product into level k+1 (Sec. 3.1): coarse
  // nonzero q sums the terms gptr[q] .. gptr[q+1]-1, term t being
  // (P_i * A_ij) * P_j with fine CSR position gpos[t] and fine row i = grow[t]
  bool plan = false;
  int32_t *gpos = nullptr, *grow = nullptr, *gptr = nullptr;
  // solve-phase matrix (SELL-32).  FP64: every entry of A.  FP32 / BF16: the
  // off-diagonal entries only, rounded, with the diagonal in sdiag (FP32) as
  // a_ii plus the rounding errors of the row's off-diagonals, so that row sums
  // stay exact and the rounded matrix stays spectrally equivalent to A.
  int32_t nslices = 0;
  int32_t sell_blocks = 0;    // grid of this level's SpMV launches with fused inner products
                              // (set at prepare, autotuned; at most kRedBlocks)
  int32_t sell_plain_blocks = 0;  // grid of the launches without inner products (default: a
                                  // warp per slice)
  int32_t seg_tile = 0;       // batch: rows per tile of the per-system inner products
  int64_t sell_entries = 0;
  int64_t *sptr = nullptr;
  int32_t *scol = nullptr;
  void *sval = nullptr;
  // FP32 values: the entries as pairs instead of scol / sval (both null).  Entry
  // e of lane l in slice sl is {column, value bits} in half (e & 1) of
  // spair[sptr[sl] / 2 + 32 (e / 2) + l], so that a lane reads two entries with
  // one 16-byte load; slice widths are even.
  int4 *spair = nullptr;
  float *sdiag = nullptr;
  // level 0 only: every entry in FP64 for the outer Krylov method and the true
  // residual (the same arrays as sptr / scol / sval in FP64 mode)
  int64_t *sptr64 = nullptr;
  int32_t *scol64 = nullptr;
  double *sval64 = nullptr;
  int64_t sell64_entries = 0;
  // solve-phase vectors and per-row data in the vector type
  void *wd = nullptr, *dinv = nullptr, *pw = nullptr, *poly = nullptr;
  bool poly_off = false;  // the level's polynomial was cleared: damped Jacobi
  void *r = nullptr, *bc = nullptr, *xc = nullptr, *c = nullptr, *v = nullptr, *rt = nullptr,
       *d = nullptr, *w = nullptr, *tmp = nullptr, *u0 = nullptr, *u1 = nullptr;
  double *slots = nullptr;    // kNumSlots doubles
  int *flag = nullptr;        // predicate of the second inner step of Alg. 5 at this level
  double *partials = nullptr; // kRedBlocks * 8 doubles
  // batched systems (block-diagonal hierarchy): system s owns rows
  // [sys_off[s], sys_off[s+1]) on every level; row tiles never cross systems
  int32_t *sys_off = nullptr, *sys_of = nullptr;
  unsigned char *slive = nullptr;  // per slice: some system in it still iterates
  std::vector<int32_t> sys_off_host;
  int32_t ntiles = 0;
  int32_t *tile_row = nullptr, *sys_tile = nullptr;  // ntiles+1 row starts; nsys+1 first tiles
  double *bslots = nullptr;   // kNumSlots x nsys per-system scalars
  int *bflag = nullptr;       // nsys second-step flags, then "any"
  double *tpart = nullptr;    // 3 x ntiles tile partial sums
};

// Per-level view used by the cluster kernel that runs the coarse tail of the
// cycle (levels t..L-1) in one launch.
struct TailLevel {
  int32_t n, nslices, nc;
  const int64_t *sptr;
  const int32_t *scol;
  const void *sval;
  const int4 *spair;   // FP32 values: entries as pairs (scol / sval null)
  const float *sdiag;  // split diagonal of a reduced-precision level (else null)
  const void *wd, *pw;
  const int32_t *agg, *aptr, *amem;
  void *bc, *xc, *r, *c, *v, *rt, *d, *w;
};

struct TailArgs {
  int t, L, mode, nL, gmres;  // mode 0: V-cycle at t; 1: Alg. 5 coarse part at t
  double kt;                  // K-cycle threshold
  const double *Ainv;         // coarsest inverse
  const TailLevel *lev;       // device array indexed by level
  const int *pred;
};

struct Hierarchy {
  amg_params p{};
  int L = 0;
  // batched mode: nsys independent systems in one block-diagonal hierarchy
  bool batched = false;
  bool sym_pattern = false;  // A_0 is structurally symmetric (found on level 0)
  int nsys = 1;
  double *binv = nullptr;        // coarsest level: per-system dense inverses, back to back
  int64_t *binv_off = nullptr;   // nsys+1 offsets into binv
  int32_t bmax = 0;              // largest coarsest block
  int *bit = nullptr;            // per-system iteration counts, then per-system status
  int *bactive = nullptr;        // per-system "still iterating", [nsys] = number active
  int tail_t = -1;                 // first level of the cluster tail (-1: none)
  TailLevel *tail_dev = nullptr;   // device copy of the per-level views
  Level lev[kMaxLevels];
  double *coarse_inv = nullptr;  // dense inverse of A_{L-1}, n_L x n_L, FP64
  int32_t nL = 0;
  Arena arena;
  // outer Krylov work (FP64, level 0)
  double *x = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *pdir = nullptr, *q = nullptr;
  double *hist = nullptr;   // device residual history
  int *it_dev = nullptr;    // device iteration counter
  int *status_dev = nullptr;
  // FGMRES
  double *V = nullptr, *Z = nullptr, *H = nullptr, *fg = nullptr, *hc = nullptr, *gpart = nullptr;
  // precision bridging vectors at level 0 of the preconditioner
  void *pre_in = nullptr, *pre_out = nullptr;
  // statistics
  amg_solve_info info{};
  int64_t launches = 0;
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_kind = -1;
  int64_t graph_launches = 0;     // kernels in one replay of the captured iteration
  double *host_pinned = nullptr;  // small pinned staging buffer
  bool poly_set[kMaxLevels] = {};
  // cycle trace of the last solve or preconditioner application: per level the
  // cycle visits, the Krylov-accelerated coarse parts of Alg. 5 run there, and
  // how many of those took the second inner step
  int64_t visits[kMaxLevels] = {}, kcalls[kMaxLevels] = {}, second[kMaxLevels] = {};
  bool trace_ok = false;
};

// ---------------------------------------------------------------- helpers
inline int grid_for(int64_t items, int per_block, int cap = 152 * 32) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1 };
PtrKind pointer_kind(const void *p);

// setup.cu
void build_hierarchy(Hierarchy &h, const amg_csr &A, cudaStream_t s);
void build_hierarchy_batch(Hierarchy &h, int32_t nsys, const amg_csr *As, cudaStream_t s);
void coarsen_all(Hierarchy &h, cudaStream_t s);
void finish_levels(Hierarchy &h, cudaStream_t s, bool fresh);
void resetup_values(Hierarchy &h, const double *val0, cudaStream_t s);
// solve.cu: per-row smoother data (omega/A_ii, 1/A_ii, P weights) in the vector type
void make_row_data(Hierarchy &h, Level &L, const double *diag, cudaStream_t s);
// solve.cu
void prepare_solve(Hierarchy &h, cudaStream_t s);
int run_solve(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *res_hist,
              cudaStream_t s);
void run_precond(Hierarchy &h, const double *b, double *x, cudaStream_t s);
int run_solve_batch(Hierarchy &h, const double *b, double *x, double tol, int32_t *iters, double *relres,
                    cudaStream_t s);
void run_spmv(Hierarchy &h, int level, const void *x, void *y, cudaStream_t s);
void set_poly(Hierarchy &h, int level, const double *coef_dev, cudaStream_t s);

// learned.cu
void twogrid_loss(Hierarchy &h, const double *coef, int nvec, uint64_t seed, double *loss_dev, double *dcoef,
                  cudaStream_t s);
void features(const Hierarchy &h, int level, float *feat_dev, cudaStream_t s);
void mlp_forward_half(int32_t n, const uint16_t *w16_dev, const float *feat, float *out, cudaStream_t s);
void mlp_backward(int32_t n, const float *w, const float *feat, const float *dout, double *dparam, cudaStream_t s,
                  bool zero);
void apply_learned(Hierarchy &h, const uint16_t *w16_dev, cudaStream_t s);
void train_smoother(Hierarchy *const *hs, int nh, int steps, double lr, int nvec, uint64_t seed, float *w_host,
                    double *loss_hist, cudaStream_t s);
void mlp_backward_fixed(int32_t n, const float *w, const float *feat, const float *dout, double *dparam,
                        cudaStream_t s);
size_t fixed_scratch_bytes();
int32_t fixed_scratch_max_rows();

// tail.cu
template <class MV, class VT>
void tail_launch(const TailArgs &a, int blocks, cudaStream_t s);
// Largest first level of the cluster tail.  Eight SMs of a cluster run a level
// of ~1.5k rows in a few microseconds per phase, where one full-GPU kernel per
// step is bound by launch latency; a 17k-row level is faster on all 152 SMs.
constexpr int kTailMaxRows = 4096;

// ---------------------------------------------------------------- launches
// Solve kernels are launched with programmatic dependent launch: each kernel
// may be scheduled while its predecessor in the stream still runs, waits in
// griddepcontrol.wait until the predecessor has completed and its writes are
// visible, and at once lets its own successor launch.  This hides the launch
// latency of the many short kernels of a multigrid cycle.
bool &pdl_enabled();  // thread-local, set from the hierarchy's parameters

template <typename... KArgs, typename... Args>
inline void klaunch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// the same with dynamic shared memory (the setup kernels)
template <class... KArgs, class... Args>
inline void klaunch_sm(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

__device__ __forceinline__ void pdl_wait_and_trigger() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- device utilities
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T> struct VecOf;
template <> struct VecOf<double> { using type = double; };

__device__ __forceinline__ double to_acc(double v, double) { return v; }
__device__ __forceinline__ float to_acc(float v, float) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ double to_acc(float v, double) { return (double)v; }

}  // namespace amg
