// capi.cu -- the C ABI of include/amg.h: argument checks, stream handoff,
// error translation (no exception crosses the boundary).
#include <cstring>
#include <mutex>

#include "amg_internal.cuh"

struct amg_hierarchy {
  amg::Hierarchy h;
  cudaStream_t stream = nullptr;  // internal non-blocking stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
};

namespace amg {

static thread_local std::string g_last_error;

void set_last_error(const std::string &m) { g_last_error = m; }

int64_t &launch_counter() {
  static thread_local int64_t n = 0;
  return n;
}

cudaStream_t &current_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}

bool &pdl_enabled() {
  static thread_local bool on = true;
  return on;
}

// Pinned 64-double staging buffers and streams of freed hierarchies are kept
// for the next one: page-locking host memory and creating streams cost more
// than a small setup.
namespace {
std::mutex g_recycle_mu;
std::vector<double *> g_pinned_free;
std::vector<cudaStream_t> g_stream_free[64];  // per device
int current_device() {
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error{AMG_ERR_CUDA, "device index out of range"};
  return dev;
}
}  // namespace

cudaStream_t stream_get() {
  const int dev = current_device();
  {
    std::lock_guard<std::mutex> lk(g_recycle_mu);
    if (!g_stream_free[dev].empty()) {
      cudaStream_t st = g_stream_free[dev].back();
      g_stream_free[dev].pop_back();
      return st;
    }
  }
  cudaStream_t st = nullptr;
  AMG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  return st;
}
void stream_put(cudaStream_t st) {  // kept only when idle and not capturing
  if (!st) return;
  int dev = 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 ||
      cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone ||
      cudaStreamQuery(st) != cudaSuccess) {
    if (cap == cudaStreamCaptureStatusActive) {
      cudaGraph_t g = nullptr;
      if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    cudaStreamDestroy(st);
    return;
  }
  std::lock_guard<std::mutex> lk(g_recycle_mu);
  g_stream_free[dev].push_back(st);
}

double *pinned_scratch_get() {
  {
    std::lock_guard<std::mutex> lk(g_recycle_mu);
    if (!g_pinned_free.empty()) {
      double *p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return p;
    }
  }
  double *p = nullptr;
  AMG_CUDA(cudaMallocHost(&p, 128 * sizeof(double)));  // layout: see kPinnedSetupFlags
  return p;
}
void pinned_scratch_put(double *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_recycle_mu);
  g_pinned_free.push_back(p);
}

cudaMemPool_t device_pool() {
  static cudaMemPool_t pools[64] = {};
  static std::mutex mu;  // threads of one process create each device's pool once
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error{AMG_ERR_CUDA, "device index out of range"};
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    AMG_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = UINT64_MAX;
    AMG_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = p;
  }
  return pools[dev];
}

PtrKind pointer_kind(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? PTR_DEVICE : PTR_HOST;
}

}  // namespace amg

namespace {

// run f; translate exceptions to status codes
template <class F>
int guarded(F &&f) {
  try {
    amg::g_last_error.clear();
    return f();
  } catch (const amg::Error &e) {
    amg::set_last_error(e.msg);
    return e.code;
  } catch (const std::exception &e) {
    amg::set_last_error(e.what());
    return AMG_ERR_CUDA;
  }
}

// make the internal stream wait for the caller's stream
void enter(amg_hierarchy *H, void *user) {
  amg::current_stream() = H->stream;
  amg::pdl_enabled() = H->h.p.pdl != 0;
  AMG_CUDA(cudaEventRecord(H->ev_in, (cudaStream_t)user));
  AMG_CUDA(cudaStreamWaitEvent(H->stream, H->ev_in, 0));
}
// and the caller's stream for the internal one
void leave(amg_hierarchy *H, void *user) {
  AMG_CUDA(cudaEventRecord(H->ev_out, H->stream));
  AMG_CUDA(cudaStreamWaitEvent((cudaStream_t)user, H->ev_out, 0));
}

int check_params(const amg_params *p) {
  if (!p) return AMG_ERR_BAD_INPUT;
  if (!(p->alpha >= 0.0 && p->alpha < 1.0) || p->coarse_max < 1 || p->max_levels < 1 || p->kcycle_levels < 0 ||
      p->precision < 0 || p->precision > 2 || p->outer < 0 || p->outer > 1 || p->max_iter < 1 ||
      p->restart < 1 || p->omega_mode < 0 || p->omega_mode > 1 || p->smoother < 0 || p->smoother > 1 ||
      p->tail < 0 || p->tail > 2 || p->autotune < 0 || p->autotune > 1 || p->symmetric < 0 || p->symmetric > 1 ||
      p->mis_k < 1 || p->mis_k > 8) {
    amg::set_last_error("invalid amg_params");
    return AMG_ERR_BAD_INPUT;
  }
  return AMG_OK;
}

template <class T>
std::vector<T> fetch(const T *dev, size_t n) {
  std::vector<T> v(n);
  if (n && dev) AMG_CUDA(cudaMemcpy(v.data(), dev, sizeof(T) * n, cudaMemcpyDeviceToHost));
  return v;
}
void expect(bool ok, int k, const char *what) {
  if (!ok) throw amg::Error{AMG_ERR_SETUP, "level " + std::to_string(k) + ": " + what};
}

}  // namespace

extern "C" {

void amg_default_params(amg_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->alpha = 0.25;
  p->seed = 0;
  p->coarse_max = 64;
  p->max_levels = 25;
  p->kcycle_levels = 2;
  p->kcycle_t = 0.25;
  p->omega_mode = 0;
  p->omega = 2.0 / 3.0;
  p->precision = AMG_PREC_F64;
  p->outer = 0;
  p->restart = 30;
  p->max_iter = 500;
  p->use_graph = 1;
  p->smoother = 0;
  p->tail = 0;
  p->pdl = 1;
  p->autotune = 0;
  p->symmetric = 1;
  p->mis_k = 2;
}

int amg_setup(const amg_csr *A, const amg_params *params, void *stream, amg_hierarchy **out) {
  if (!A || !out || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)) || A->n <= 0 || A->nnz < A->n ||
      A->nnz > (int64_t)INT32_MAX) {
    amg::set_last_error("amg_setup: null pointer or bad sizes");
    return AMG_ERR_BAD_INPUT;
  }
  int rc = check_params(params);
  if (rc) return rc;
  if (params->symmetric == 0 && params->outer != 1) {
    amg::set_last_error("amg_setup: a nonsymmetric system needs FGMRES (outer = 1)");
    return AMG_ERR_BAD_INPUT;
  }
  if (params->outer == 1 && params->restart > 32) {
    amg::set_last_error("amg_setup: FGMRES restart length is limited to 32");
    return AMG_ERR_BAD_INPUT;
  }
  *out = nullptr;
  amg_hierarchy *H = new amg_hierarchy();
  rc = guarded([&]() {
    H->stream = amg::stream_get();
    AMG_CUDA(cudaEventCreateWithFlags(&H->ev_in, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreateWithFlags(&H->ev_out, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreate(&H->t0));
    AMG_CUDA(cudaEventCreate(&H->t1));
    H->h.p = *params;
    enter(H, stream);
    AMG_CUDA(cudaEventRecord(H->t0, H->stream));
    const int64_t l0 = amg::launch_counter();
    amg::build_hierarchy(H->h, *A, H->stream);
    amg::prepare_solve(H->h, H->stream);
    H->h.info.setup_launches = amg::launch_counter() - l0;
    AMG_CUDA(cudaEventRecord(H->t1, H->stream));
    AMG_CUDA(cudaEventSynchronize(H->t1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, H->t0, H->t1));
    H->h.info.setup_ms = ms;
    leave(H, stream);
    return AMG_OK;
  });
  if (rc != AMG_OK) {
    amg_free(H);
    return rc;
  }
  *out = H;
  return AMG_OK;
}

int amg_solve(amg_hierarchy *H, const double *b, double *x, double tol, int32_t *iters, double *res_hist,
              void *stream) {
  if (!H || !b || !x || !(tol >= 0.0)) {
    amg::set_last_error("amg_solve: null pointer or negative tolerance");
    return AMG_ERR_BAD_INPUT;
  }
  return guarded([&]() {
    enter(H, stream);
    AMG_CUDA(cudaEventRecord(H->t0, H->stream));
    int rc = amg::run_solve(H->h, b, x, tol, iters, res_hist, H->stream);
    AMG_CUDA(cudaEventRecord(H->t1, H->stream));
    AMG_CUDA(cudaEventSynchronize(H->t1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, H->t0, H->t1));
    H->h.info.solve_ms = ms;
    leave(H, stream);
    if (rc == AMG_ERR_NOT_CONVERGED) amg::set_last_error("amg_solve: max_iter reached before tol");
    if (rc == AMG_ERR_BREAKDOWN) amg::set_last_error("amg_solve: Krylov breakdown (p^T A p <= 0)");
    if (rc == AMG_ERR_NAN) amg::set_last_error("amg_solve: non-finite residual");
    return rc;
  });
}

int amg_setup_batch(int32_t nsys, const amg_csr *As, const amg_params *params, void *stream,
                    amg_hierarchy **out) {
  if (nsys < 1 || !As || !out) {
    amg::set_last_error("amg_setup_batch: bad arguments");
    return AMG_ERR_BAD_INPUT;
  }
  for (int32_t q = 0; q < nsys; ++q)
    if (!As[q].row_ptr || !As[q].col || !As[q].val || As[q].n <= 0 || As[q].nnz < As[q].n) {
      amg::set_last_error("amg_setup_batch: system " + std::to_string(q) + " has null pointers or bad sizes");
      return AMG_ERR_BAD_INPUT;
    }
  int rc = check_params(params);
  if (rc) return rc;
  if (params->outer != 0 || params->symmetric != 1) {
    amg::set_last_error("amg_setup_batch: batches are symmetric systems solved by flexible CG (outer = 0)");
    return AMG_ERR_UNSUPPORTED;
  }
  *out = nullptr;
  amg_hierarchy *H = new amg_hierarchy();
  rc = guarded([&]() {
    H->stream = amg::stream_get();
    AMG_CUDA(cudaEventCreateWithFlags(&H->ev_in, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreateWithFlags(&H->ev_out, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreate(&H->t0));
    AMG_CUDA(cudaEventCreate(&H->t1));
    H->h.p = *params;
    enter(H, stream);
    AMG_CUDA(cudaEventRecord(H->t0, H->stream));
    const int64_t l0 = amg::launch_counter();
    amg::build_hierarchy_batch(H->h, nsys, As, H->stream);
    amg::prepare_solve(H->h, H->stream);
    H->h.info.setup_launches = amg::launch_counter() - l0;
    AMG_CUDA(cudaEventRecord(H->t1, H->stream));
    AMG_CUDA(cudaEventSynchronize(H->t1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, H->t0, H->t1));
    H->h.info.setup_ms = ms;
    leave(H, stream);
    return AMG_OK;
  });
  if (rc != AMG_OK) {
    amg_free(H);
    return rc;
  }
  *out = H;
  return AMG_OK;
}

int amg_solve_batch(amg_hierarchy *H, const double *b, double *x, double tol, int32_t *iters, double *relres,
                    void *stream) {
  if (!H || !b || !x || !(tol >= 0.0) || !H->h.batched) {
    amg::set_last_error("amg_solve_batch: null pointer, negative tolerance or not a batch hierarchy");
    return AMG_ERR_BAD_INPUT;
  }
  return guarded([&]() {
    enter(H, stream);
    AMG_CUDA(cudaEventRecord(H->t0, H->stream));
    const int rc = amg::run_solve_batch(H->h, b, x, tol, iters, relres, H->stream);
    AMG_CUDA(cudaEventRecord(H->t1, H->stream));
    AMG_CUDA(cudaEventSynchronize(H->t1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, H->t0, H->t1));
    H->h.info.solve_ms = ms;
    leave(H, stream);
    if (rc != AMG_OK) amg::set_last_error("amg_solve_batch: some system did not converge");
    return rc;
  });
}

int amg_resetup_values(amg_hierarchy *H, const double *val, void *stream) {
  if (!H || !val) {
    amg::set_last_error("amg_resetup_values: null argument");
    return AMG_ERR_BAD_INPUT;
  }
  return guarded([&]() {
    enter(H, stream);
    AMG_CUDA(cudaEventRecord(H->t0, H->stream));
    amg::resetup_values(H->h, val, H->stream);
    AMG_CUDA(cudaEventRecord(H->t1, H->stream));
    AMG_CUDA(cudaEventSynchronize(H->t1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, H->t0, H->t1));
    H->h.info.setup_ms = ms;
    leave(H, stream);
    return AMG_OK;
  });
}

int amg_precond(amg_hierarchy *H, const double *b, double *x, void *stream) {
  if (!H || !b || !x) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    enter(H, stream);
    amg::run_precond(H->h, b, x, H->stream);
    leave(H, stream);
    return AMG_OK;
  });
}

int amg_spmv(amg_hierarchy *H, int32_t level, const void *x, void *y, void *stream) {
  if (!H || !x || !y || level < 0 || level >= H->h.L) {
    amg::set_last_error("amg_spmv: bad arguments");
    return AMG_ERR_BAD_INPUT;
  }
  if (amg::pointer_kind(x) != amg::PTR_DEVICE || amg::pointer_kind(y) != amg::PTR_DEVICE) {
    amg::set_last_error("amg_spmv: x and y must be device pointers");
    return AMG_ERR_BAD_INPUT;
  }
  return guarded([&]() {
    if (stream) {  // no allocation: launch straight on the caller's stream (graph-capturable)
      amg::current_stream() = (cudaStream_t)stream;
      amg::pdl_enabled() = H->h.p.pdl != 0;
      amg::run_spmv(H->h, level, x, y, (cudaStream_t)stream);
      return AMG_OK;
    }
    enter(H, stream);  // legacy default stream: run on the hierarchy's stream
    amg::run_spmv(H->h, level, x, y, H->stream);
    leave(H, stream);
    return AMG_OK;
  });
}

int amg_set_poly(amg_hierarchy *H, int32_t level, const double *coef, void *stream) {
  if (!H || level < 0 || level >= H->h.L - 1) {
    amg::set_last_error("amg_set_poly: bad level (the coarsest level has no smoother) or null hierarchy");
    return AMG_ERR_BAD_INPUT;
  }
  return guarded([&]() {
    enter(H, stream);
    amg::set_poly(H->h, level, coef, H->stream);
    leave(H, stream);
    return AMG_OK;
  });
}

int amg_features(const amg_hierarchy *H, int32_t level, float *feat, void *stream) {
  if (!H || !feat || level < 0 || level >= H->h.L) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    amg_hierarchy *Hm = const_cast<amg_hierarchy *>(H);
    enter(Hm, stream);
    const size_t cnt = (size_t)H->h.lev[level].n * AMG_MLP_NFEAT;
    if (amg::pointer_kind(feat) == amg::PTR_DEVICE) {
      amg::features(H->h, level, feat, Hm->stream);
    } else {
      amg::DevBuf<float> tmp(cnt);
      amg::features(H->h, level, tmp.p, Hm->stream);
      AMG_CUDA(cudaMemcpyAsync(feat, tmp.p, sizeof(float) * cnt, cudaMemcpyDeviceToHost, Hm->stream));
      AMG_CUDA(cudaStreamSynchronize(Hm->stream));
    }
    leave(Hm, stream);
    return AMG_OK;
  });
}

int amg_mlp_forward(int32_t n, const uint16_t *w16, const float *feat, float *out, void *stream) {
  if (n < 0 || !w16 || !feat || !out) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    amg::mlp_forward_half(n, w16, feat, out, (cudaStream_t)stream);
    return AMG_OK;
  });
}

int amg_mlp_backward(int32_t n, const float *w, const float *feat, const float *dout, double *dparam, void *stream) {
  if (n < 0 || !w || !feat || !dout || !dparam) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    amg::current_stream() = (cudaStream_t)stream;
    amg::mlp_backward(n, w, feat, dout, dparam, (cudaStream_t)stream, true);
    return AMG_OK;
  });
}

int amg_mlp_backward_noalloc(int32_t n, const float *w, const float *feat, const float *dout, double *dparam,
                             void *stream) {
  if (n < 0 || !w || !feat || !dout || !dparam) {
    amg::set_last_error("amg_mlp_backward_noalloc: null pointer or negative n");
    return AMG_ERR_BAD_INPUT;
  }
  return guarded([&]() {
    amg::mlp_backward_fixed(n, w, feat, dout, dparam, (cudaStream_t)stream);
    return AMG_OK;
  });
}

int amg_twogrid_loss(amg_hierarchy *H, const double *coef, int32_t nvec, uint64_t seed, double *loss, double *dcoef,
                     void *stream) {
  if (!H || !coef || !loss || nvec < 1) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    enter(H, stream);
    amg::DevBuf<double> l(1);
    amg::twogrid_loss(H->h, coef, nvec, seed, l.p, dcoef, H->stream);
    AMG_CUDA(cudaMemcpyAsync(loss, l.p, sizeof(double), cudaMemcpyDeviceToHost, H->stream));
    AMG_CUDA(cudaStreamSynchronize(H->stream));
    leave(H, stream);
    return AMG_OK;
  });
}

int amg_train_smoother(amg_hierarchy *const *hs, int32_t nh, int32_t steps, double lr, int32_t nvec, uint64_t seed,
                       float *w, double *loss_hist, void *stream) {
  if (!hs || nh < 1 || steps < 0 || !w || nvec < 1) return AMG_ERR_BAD_INPUT;
  for (int j = 0; j < nh; ++j)
    if (!hs[j] || hs[j]->h.L != 2) {
      amg::set_last_error("amg_train_smoother: every hierarchy needs exactly two levels");
      return AMG_ERR_BAD_INPUT;
    }
  return guarded([&]() {
    enter(hs[0], stream);
    std::vector<amg::Hierarchy *> v(nh);
    for (int j = 0; j < nh; ++j) v[j] = &hs[j]->h;
    amg::train_smoother(v.data(), nh, steps, lr, nvec, seed, w, loss_hist, hs[0]->stream);
    leave(hs[0], stream);
    return AMG_OK;
  });
}

int amg_apply_learned_smoother(amg_hierarchy *H, const uint16_t *w16, void *stream) {
  if (!H || !w16) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    enter(H, stream);
    amg::DevBuf<uint16_t> w(AMG_MLP_NPARAM);
    const cudaMemcpyKind k =
        amg::pointer_kind(w16) == amg::PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    AMG_CUDA(cudaMemcpyAsync(w.p, w16, sizeof(uint16_t) * AMG_MLP_NPARAM, k, H->stream));
    amg::apply_learned(H->h, w.p, H->stream);
    AMG_CUDA(cudaStreamSynchronize(H->stream));
    leave(H, stream);
    return AMG_OK;
  });
}

int amg_hierarchy_info(const amg_hierarchy *H, amg_level_info *levels, int32_t cap, int32_t *nlevels) {
  if (!H) return AMG_ERR_BAD_INPUT;
  if (nlevels) *nlevels = H->h.L;
  if (levels)
    for (int k = 0; k < H->h.L && k < cap; ++k) {
      const amg::Level &L = H->h.lev[k];
      levels[k].n = L.n;
      levels[k].nnz = L.nnz;
      levels[k].n_coarse = (k + 1 < H->h.L) ? L.nc : 0;
      levels[k].mis_rounds = L.mis_rounds;
      levels[k].omega = L.omega;
      levels[k].spmv_blocks = L.sell_blocks;
      levels[k].seg_tile = H->h.batched ? L.seg_tile : 0;
    }
  return AMG_OK;
}

int amg_export_level(const amg_hierarchy *H, int32_t level, int32_t *row_ptr, int32_t *col, double *val,
                     int32_t *agg, double *P, double *B) {
  if (!H || level < 0 || level >= H->h.L) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    const amg::Level &L = H->h.lev[level];
    const bool last = level == H->h.L - 1;
    if (row_ptr) AMG_CUDA(cudaMemcpy(row_ptr, L.rp, sizeof(int32_t) * ((size_t)L.n + 1), cudaMemcpyDeviceToHost));
    if (col) AMG_CUDA(cudaMemcpy(col, L.ci, sizeof(int32_t) * (size_t)L.nnz, cudaMemcpyDeviceToHost));
    if (val) AMG_CUDA(cudaMemcpy(val, L.val, sizeof(double) * (size_t)L.nnz, cudaMemcpyDeviceToHost));
    if (agg && !last) AMG_CUDA(cudaMemcpy(agg, L.agg, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToHost));
    if (P && !last) AMG_CUDA(cudaMemcpy(P, L.pw64, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToHost));
    if (B) AMG_CUDA(cudaMemcpy(B, L.B, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToHost));
    return AMG_OK;
  });
}

int amg_validate_hierarchy(const amg_hierarchy *H) {
  if (!H) return AMG_ERR_BAD_INPUT;
  return guarded([&]() {
    const amg::Hierarchy &h = H->h;
    AMG_CUDA(cudaStreamSynchronize(H->stream));
    for (int k = 0; k < h.L; ++k) {
      const amg::Level &L = h.lev[k];
      const bool last = k == h.L - 1;
      auto rp = fetch(L.rp, (size_t)L.n + 1);
      auto ci = fetch(L.ci, (size_t)L.nnz);
      expect(rp[0] == 0 && rp[L.n] == L.nnz, k, "row pointer ends");
      for (int32_t i = 0; i < L.n; ++i) expect(rp[i] <= rp[i + 1], k, "row pointers not monotone");
      for (int32_t c : ci) expect(c >= 0 && c < L.n, k, "column out of range");
      auto sp = fetch(L.sptr, (size_t)L.nslices + 1);
      expect(sp[0] == 0 && sp[L.nslices] == L.sell_entries, k, "SELL pointer ends");
      const int64_t unit = h.p.precision != AMG_PREC_F64 ? 64 : 32;  // pairs: slice widths are even
      for (int32_t q = 0; q < L.nslices; ++q)
        expect(sp[q] <= sp[q + 1] && (sp[q + 1] - sp[q]) % unit == 0, k, "SELL slice");
      if (L.spair) {  // {column, value bits} pairs: the columns are the even words
        auto pw = fetch(reinterpret_cast<const int32_t *>(L.spair), 2 * (size_t)L.sell_entries);
        for (size_t q = 0; q < pw.size(); q += 2) expect(pw[q] >= 0 && pw[q] < L.n, k, "SELL column out of range");
      } else {
        auto sc = fetch(L.scol, (size_t)L.sell_entries);
        for (int32_t c : sc) expect(c >= 0 && c < L.n, k, "SELL column out of range");
      }
      if (k == 0 && L.sptr64 != L.sptr) {
        auto sp64 = fetch(L.sptr64, (size_t)L.nslices + 1);
        auto sc64 = fetch(L.scol64, (size_t)L.sell64_entries);
        expect(sp64[0] == 0 && sp64[L.nslices] == L.sell64_entries, k, "FP64 SELL pointer ends");
        for (int32_t c : sc64) expect(c >= 0 && c < L.n, k, "FP64 SELL column out of range");
      }
      if (!last) {
        auto agg = fetch(L.agg, (size_t)L.n);
        auto ap = fetch(L.aptr, (size_t)L.nc + 1);
        auto am = fetch(L.amem, (size_t)L.n);
        expect(L.nc == h.lev[k + 1].n, k, "coarse size");
        for (int32_t a : agg) expect(a >= 0 && a < L.nc, k, "aggregate id out of range");
        expect(ap[0] == 0 && ap[L.nc] == L.n, k, "member pointer ends");
        std::vector<char> seen(L.n, 0);
        for (int32_t I = 0; I < L.nc; ++I)
          for (int32_t m = ap[I]; m < ap[I + 1]; ++m) {
            expect(am[m] >= 0 && am[m] < L.n && !seen[am[m]] && agg[am[m]] == I, k, "member lists");
            seen[am[m]] = 1;
          }
      }
      if (h.batched) {
        auto so = fetch(L.sys_off, (size_t)h.nsys + 1);
        expect(so == L.sys_off_host, k, "system offsets differ between host and device");
        expect(so[0] == 0 && so[h.nsys] == L.n, k, "system offset ends");
        for (int q = 0; q < h.nsys; ++q) expect(so[q] < so[q + 1], k, "empty or unordered system");
        auto sy = fetch(L.sys_of, (size_t)L.n);
        for (int q = 0; q < h.nsys; ++q)
          for (int32_t i = so[q]; i < so[q + 1]; ++i) expect(sy[i] == q, k, "row-to-system map");
        auto tr = fetch(L.tile_row, (size_t)L.ntiles + 1);
        auto st = fetch(L.sys_tile, (size_t)h.nsys + 1);
        expect(st[0] == 0 && st[h.nsys] == L.ntiles && tr[L.ntiles] == L.n, k, "tile ends");
        for (int q = 0; q < h.nsys; ++q)
          for (int32_t t = st[q]; t < st[q + 1]; ++t)
            expect(tr[t] >= so[q] && tr[t] < tr[t + 1] && tr[t + 1] <= so[q + 1], k, "tile crosses a system");
        if (!last && k + 1 < h.L) {
          auto agg = fetch(L.agg, (size_t)L.n);
          const auto &sn = h.lev[k + 1].sys_off_host;
          for (int q = 0; q < h.nsys; ++q)
            for (int32_t i = so[q]; i < so[q + 1]; ++i)
              expect(agg[i] >= sn[q] && agg[i] < sn[q + 1], k, "aggregate leaves its system");
        }
      }
    }
    if (h.batched) {
      const amg::Level &Lc = h.lev[h.L - 1];
      auto bo = fetch(h.binv_off, (size_t)h.nsys + 1);
      for (int q = 0; q < h.nsys; ++q) {
        const int64_t m = Lc.sys_off_host[q + 1] - Lc.sys_off_host[q];
        expect(bo[q + 1] - bo[q] == m * m, h.L - 1, "coarsest block offsets");
      }
      expect(h.nL == Lc.n, h.L - 1, "coarsest size");
    }
    return AMG_OK;
  });
}

int amg_cycle_trace(const amg_hierarchy *H, int64_t *visits, int64_t *kcalls, int64_t *second, int32_t cap,
                    int32_t *nlevels) {
  if (!H) return AMG_ERR_BAD_INPUT;
  const amg::Hierarchy &h = H->h;
  if (nlevels) *nlevels = h.L;
  if (h.batched || !h.trace_ok) {
    amg::set_last_error("amg_cycle_trace: no trace (batch, cluster tail, or no solve yet)");
    return AMG_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < h.L && k < cap; ++k) {
    if (visits) visits[k] = h.visits[k];
    if (kcalls) kcalls[k] = h.kcalls[k];
    if (second) second[k] = h.second[k];
  }
  return AMG_OK;
}

int amg_last_solve_info(const amg_hierarchy *H, amg_solve_info *info) {
  if (!H || !info) return AMG_ERR_BAD_INPUT;
  *info = H->h.info;
  return AMG_OK;
}

void amg_free(amg_hierarchy *H) {
  if (!H) return;
  if (H->stream) cudaStreamSynchronize(H->stream);
  if (H->h.graph_exec) cudaGraphExecDestroy(H->h.graph_exec);
  if (H->h.graph) cudaGraphDestroy(H->h.graph);
  amg::current_stream() = H->stream;
  H->h.arena.release();
  if (H->stream) cudaStreamSynchronize(H->stream);
  amg::pinned_scratch_put(H->h.host_pinned);
  if (H->ev_in) cudaEventDestroy(H->ev_in);
  if (H->ev_out) cudaEventDestroy(H->ev_out);
  if (H->t0) cudaEventDestroy(H->t0);
  if (H->t1) cudaEventDestroy(H->t1);
  amg::stream_put(H->stream);
  delete H;
}

const char *amg_last_error(void) { return amg::g_last_error.c_str(); }

}  // extern "C"
