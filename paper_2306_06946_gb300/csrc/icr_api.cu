// libicr host side: the C ABI declared in include/icr.h.
//
// This file validates inputs, derives the symbolic schedule of the
// supernodal factor once per system (children, etree levels, the row maps of
// every supernode into its parent's front) and manages the scene's device
// buffers.  All per-step arithmetic runs in the kernels of icr_kernels.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "icr_internal.h"

struct icr_ctx : icr::Ctx {};
struct icr_scene : icr::Scene {};

namespace icr {

static thread_local std::string g_err = "no error";

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int cuda_fail(cudaError_t e, const char* where) {
  set_error("%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
  return ICR_ECUDA;
}

int dalloc(Scene* s, DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.p && b.bytes >= bytes) return ICR_OK;
  dfree(s, b);
  Ctx* c = s->ctx;
  if (c->fail_alloc_after >= 0 && c->fail_alloc_after-- == 0) {
    set_error("allocation of %zu bytes failed (injected by icr_ctx_inject_alloc_failure)", bytes);
    return ICR_ENOMEM;
  }
  if (c->budget && c->in_use + bytes > c->budget) {
    set_error("allocation of %zu bytes exceeds the context HBM budget (%llu of %llu in use)", bytes,
              (unsigned long long)c->in_use, (unsigned long long)c->budget);
    return ICR_ENOMEM;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return ICR_ENOMEM;
  }
  b.bytes = bytes;
  static std::atomic<uint64_t> generation{0};
  b.gen = ++generation;
  c->in_use += bytes;
  ++s->alloc_epoch;
  return ICR_OK;
}

void dfree(Scene* s, DBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    s->ctx->in_use -= b.bytes;
    ++s->alloc_epoch;   // a captured graph that read this buffer is stale
  }
  b.p = nullptr;
  b.bytes = 0;
}

}  // namespace icr

using namespace icr;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static int check_scene(icr_scene* s) {
  if (!s) {
    set_error("scene is NULL");
    return ICR_EINVAL;
  }
  if (s->evicted) {
    set_error("the scene is evicted: icr_scene_readmit it first");
    return ICR_ESTATE;
  }
  return ICR_OK;
}

static int set_device(Scene* s) {
  CK(cudaSetDevice(s->ctx->device));
  return ICR_OK;
}

// Copy `count` host doubles into a device buffer of the scene's precision.
static int upload_T(Scene* s, DBuf& dst, const double* src, size_t count) {
  if (count == 0) return ICR_OK;
  if (s->prec == ICR_FP64) {
    CK(cudaMemcpyAsync(dst.p, src, count * sizeof(double), cudaMemcpyHostToDevice, s->ctx->stream));
  } else {
    std::vector<float> tmp(count);
    for (size_t i = 0; i < count; ++i) tmp[i] = (float)src[i];
    // pageable source: the call returns once tmp has been staged, so tmp may go
    CK(cudaMemcpyAsync(dst.p, tmp.data(), count * sizeof(float), cudaMemcpyHostToDevice, s->ctx->stream));
  }
  return ICR_OK;
}

template <class V>
static int upload(Scene* s, DBuf& dst, const V* src, size_t count) {
  if (count == 0) return ICR_OK;
  CK(cudaMemcpyAsync(dst.p, src, count * sizeof(V), cudaMemcpyHostToDevice, s->ctx->stream));
  return ICR_OK;
}

// Host doubles (rows x cols, dense) into a device matrix with leading dimension ld.
static int upload_T_2d(Scene* s, DBuf& dst, int64_t ld, const double* src, size_t rows, size_t cols) {
  if (rows == 0 || cols == 0) return ICR_OK;
  const size_t es = s->tsize;
  std::vector<unsigned char> tmp(rows * cols * es);
  if (s->prec == ICR_FP64)
    std::memcpy(tmp.data(), src, tmp.size());
  else
    for (size_t i = 0; i < rows * cols; ++i) ((float*)tmp.data())[i] = (float)src[i];
  CK(cudaMemcpy2DAsync(dst.p, ld * es, tmp.data(), cols * es, cols * es, rows, cudaMemcpyHostToDevice,
                       s->ctx->stream));
  CK(cudaStreamSynchronize(s->ctx->stream));
  return ICR_OK;
}

// Device matrix with leading dimension ld -> host doubles (synchronises).
static int download_T_2d(Scene* s, const DBuf& src, int64_t ld, double* dst, size_t rows, size_t cols) {
  if (rows == 0 || cols == 0) return ICR_OK;
  const size_t es = s->tsize;
  std::vector<unsigned char> tmp(rows * cols * es);
  CK(cudaMemcpy2DAsync(tmp.data(), cols * es, src.p, ld * es, cols * es, rows, cudaMemcpyDeviceToHost,
                       s->ctx->stream));
  CK(cudaStreamSynchronize(s->ctx->stream));
  if (s->prec == ICR_FP64)
    std::memcpy(dst, tmp.data(), tmp.size());
  else
    for (size_t i = 0; i < rows * cols; ++i) dst[i] = ((float*)tmp.data())[i];
  return ICR_OK;
}

// Device buffer of the scene's precision -> host doubles (synchronises).
static int download_T(Scene* s, const DBuf& src, double* dst, size_t count) {
  if (count == 0) return ICR_OK;
  if (s->prec == ICR_FP64) {
    CK(cudaMemcpyAsync(dst, src.p, count * sizeof(double), cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(cudaStreamSynchronize(s->ctx->stream));
  } else {
    std::vector<float> tmp(count);
    CK(cudaMemcpyAsync(tmp.data(), src.p, count * sizeof(float), cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(cudaStreamSynchronize(s->ctx->stream));
    for (size_t i = 0; i < count; ++i) dst[i] = tmp[i];
  }
  return ICR_OK;
}

// Solve operator of every supernode, from its factor panel (FP64):
//   G_s = [ L_ss^-1 ; L[R_s, s] L_ss^-1 ],  (w + r) x w, column-major,
// so that the forward solve of a front is X_s = L_ss^-1 F_top and
// U_s = F_R - (L_Rs L_ss^-1) F_top, and the backward solve is
// dq_s = G_s^T [y_s ; -dq_R].  Supernodes are spread over host threads.
static void compute_G(int ns, const std::vector<int32_t>& sp, const std::vector<int64_t>& rp,
                      const std::vector<int64_t>& vp, const double* Lp, std::vector<double>& G) {
  G.assign(vp[ns], 0.0);
  std::atomic<int> next(0);
  auto work = [&]() {
    std::vector<double> z;
    for (int k = next++; k < ns; k = next++) {
      const int w = sp[k + 1] - sp[k];
      const int64_t r = rp[k + 1] - rp[k];
      const int64_t ld = w + r;
      const double* L = Lp + vp[k];
      double* Gk = G.data() + vp[k];
      // L_ss^-1, one column at a time: z = L^-1 e_j by column-oriented substitution
      z.assign(w, 0.0);
      for (int j = 0; j < w; ++j) {
        std::fill(z.begin(), z.end(), 0.0);
        z[j] = 1.0;
        for (int c = j; c < w; ++c) {
          const double zc = z[c];
          if (zc == 0.0) continue;
          const double* Lc = L + (int64_t)c * ld;
          for (int i = c + 1; i < w; ++i) z[i] -= Lc[i] * zc;
        }
        double* Gj = Gk + (int64_t)j * ld;
        for (int i = j; i < w; ++i) Gj[i] = z[i];
        // P[:, j] = sum_{c >= j} L[R, c] Z[c, j]
        double* Pj = Gj + w;
        for (int c = j; c < w; ++c) {
          const double zc = z[c];
          if (zc == 0.0) continue;
          const double* Lc = L + (int64_t)c * ld + w;
          for (int64_t i = 0; i < r; ++i) Pj[i] += Lc[i] * zc;
        }
      }
    }
  };
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (unsigned t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
}

namespace icr {
int check_step_graph(Scene* s, const char* where) {
  if (!s->step_graph) {
    set_error("%s: no captured step (icr_step_capture)", where);
    return ICR_ESTATE;
  }
  if (!s->has_mapping || s->obst_kind == 0) {
    set_error("%s: the step needs a mapping and an obstacle", where);
    return ICR_ESTATE;
  }
  if (s->graph_epoch != s->alloc_epoch || s->graph_m != s->m || s->graph_obst != s->obst_kind ||
      !same_params(s->graph_params, s->params)) {
    set_error("%s: the captured step is stale (buffers, contact count, obstacle or parameters changed); "
              "capture it again", where);
    return ICR_ESTATE;
  }
  return ICR_OK;
}

int prof_mark(Scene* s, const char* name, bool after) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s->ctx->stream, &cs);
  if (e != cudaSuccess) return cuda_fail(e, "profile: cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) return ICR_OK;
  Profiler* P = s->prof;
  if (!after) {
    cudaEvent_t a = P->take(), b = P->take();
    if (!a || !b) {
      set_error("profile: cudaEventCreate failed");
      return ICR_ECUDA;
    }
    P->recs.push_back({name, a, b});
    e = cudaEventRecord(a, s->ctx->stream);
  } else {
    e = cudaEventRecord(P->recs.back().b, s->ctx->stream);
  }
  return e == cudaSuccess ? ICR_OK : cuda_fail(e, "profile: cudaEventRecord");
}

int check_device_error(Scene* s) {
  if (!s->dev_err.p) return ICR_OK;
  int h = 0;
  CK(cudaMemcpyAsync(&h, s->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, s->ctx->stream));
  CK(cudaStreamSynchronize(s->ctx->stream));
  if (h) {
    CK(cudaMemsetAsync(s->dev_err.p, 0, sizeof(int), s->ctx->stream));
    set_error("a bounded device-side wait ran out (tensor-core contraction); W_H is incomplete");
    return ICR_ETIMEOUT;
  }
  return ICR_OK;
}
}  // namespace icr

extern "C" {

const char* icr_last_error(void) { return g_err.c_str(); }

int icr_ctx_create(icr_ctx** out, int device, void* cuda_stream, uint64_t hbm_budget_bytes) {
  if (!out) {
    set_error("out is NULL");
    return ICR_EINVAL;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) {
    set_error("device %d out of range (%d devices)", device, ndev);
    return ICR_EINVAL;
  }
  CK(cudaSetDevice(device));
  icr_ctx* c = new (std::nothrow) icr_ctx();
  if (!c) {
    set_error("out of host memory");
    return ICR_ENOMEM;
  }
  c->device = device;
  e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaDeviceGetAttribute(MultiProcessorCount)");
  }
  c->stream = (cudaStream_t)cuda_stream;
  c->budget = hbm_budget_bytes;
  *out = c;
  return ICR_OK;
}

int icr_ctx_destroy(icr_ctx* ctx) {
  if (!ctx) return ICR_OK;
  if (ctx->scenes > 0) {
    ctx->destroyed = true;   // freed by the last icr_scene_destroy
    return ICR_OK;
  }
  delete ctx;
  return ICR_OK;
}

int icr_ctx_set_wait_limit(icr_ctx* ctx, uint64_t pipeline_wait_ns) {
  if (!ctx) {
    set_error("NULL context");
    return ICR_EINVAL;
  }
  ctx->wait_ns = pipeline_wait_ns;
  return ICR_OK;
}

int icr_ctx_inject_alloc_failure(icr_ctx* ctx, int64_t after) {
  if (!ctx || after < -1) {
    set_error("inject_alloc_failure: need a context and after >= -1");
    return ICR_EINVAL;
  }
  ctx->fail_alloc_after = after;
  return ICR_OK;
}

int icr_ctx_bytes_in_use(const icr_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) {
    set_error("NULL argument");
    return ICR_EINVAL;
  }
  *out = ctx->in_use;
  return ICR_OK;
}

static int check_params(const icr_params* p) {
  if (!p) {
    set_error("params is NULL");
    return ICR_EINVAL;
  }
  if (p->precision != ICR_FP32 && p->precision != ICR_FP64) {
    set_error("unknown precision %d", p->precision);
    return ICR_EINVAL;
  }
  if (p->n_sweeps < 0 || !std::isfinite(p->tol)) {
    set_error("n_sweeps must be >= 0 and tol finite");
    return ICR_EINVAL;
  }
  if (p->contraction < ICR_CONTRACT_AUTO || p->contraction > ICR_CONTRACT_BF16) {
    set_error("unknown contraction mode %d", p->contraction);
    return ICR_EINVAL;
  }
  if (p->warm_start != 0 && p->warm_start != 1) {
    set_error("warm_start must be 0 or 1");
    return ICR_EINVAL;
  }
  if (p->w_update < ICR_W_FP32 || p->w_update > ICR_W_BF16) {
    set_error("unknown W update mode %d", p->w_update);
    return ICR_EINVAL;
  }
  if (!(p->newton_tol >= 0) || !std::isfinite(p->newton_tol)) {
    set_error("newton_tol must be finite and >= 0");
    return ICR_EINVAL;
  }
  return ICR_OK;
}

int icr_scene_create(icr_ctx* ctx, icr_scene** out, const icr_params* params) {
  if (!ctx || !out) {
    set_error("NULL argument");
    return ICR_EINVAL;
  }
  RET(check_params(params));
  icr_scene* s = new (std::nothrow) icr_scene();
  if (!s) {
    set_error("out of host memory");
    return ICR_ENOMEM;
  }
  s->ctx = ctx;
  ctx->scenes++;
  s->params = *params;
  s->prec = params->precision;
  s->tsize = s->prec == ICR_FP64 ? 8 : 4;
  *out = s;
  return ICR_OK;
}

int icr_scene_destroy(icr_scene* s) {
  if (!s) return ICR_OK;
  if (s->batches > 0) {
    set_error("scene_destroy: the scene is held by %d batch(es); destroy them first", s->batches);
    return ICR_ESTATE;
  }
  cudaSetDevice(s->ctx->device);
  cudaStreamSynchronize(s->ctx->stream);
  std::vector<std::pair<DBuf*, bool>> all;
  scene_buffers(s, all);
  for (auto& b : all) dfree(s, *b.first);
  for (auto& sv : s->saved) cudaFreeHost(sv.host);
  s->saved.clear();
  if (s->stage_dev.p) {
    cudaFree(s->stage_dev.p);
    s->ctx->in_use -= s->stage_dev.bytes;
  }
  for (int k = 0; k < 2; ++k) {
    if (s->stage_host[k]) cudaFreeHost(s->stage_host[k]);
    if (s->stage_ev[k]) cudaEventDestroy(s->stage_ev[k]);
  }
  if (s->step_graph) cudaGraphExecDestroy(s->step_graph);
  delete s->prof;
  icr_ctx* c = static_cast<icr_ctx*>(s->ctx);
  delete s;
  if (--c->scenes == 0 && c->destroyed) delete c;
  return ICR_OK;
}

int icr_set_params(icr_scene* s, const icr_params* params) {
  RET(check_scene(s));
  RET(check_params(params));
  if (params->precision != s->prec) {
    set_error("precision is fixed when the scene is created");
    return ICR_EINVAL;
  }
  if (params->contraction != s->params.contraction) s->tuned = false;
  s->params = *params;
  return ICR_OK;
}

static int upload_tc_super(Scene* s);

int icr_set_system(icr_scene* s, int32_t n, int32_t ns, const int32_t* super_ptr, const int64_t* rowpat_ptr,
                   const int32_t* rowpat, const int64_t* val_ptr, const double* Lp, const double* D,
                   const int32_t* parent) {
  RET(check_scene(s));
  if (n <= 0 || n % 3 != 0 || ns <= 0 || ns > n / 3 || !super_ptr || !rowpat_ptr || !val_ptr || !Lp || !D ||
      !parent || (rowpat_ptr[ns] > 0 && !rowpat)) {
    set_error("set_system: bad sizes or NULL arrays (n=%d nsuper=%d)", n, ns);
    return ICR_EINVAL;
  }
  if (super_ptr[0] != 0 || super_ptr[ns] != n || rowpat_ptr[0] != 0 || val_ptr[0] != 0) {
    set_error("set_system: super_ptr must run from 0 to n and offsets start at 0");
    return ICR_EINVAL;
  }
  std::vector<int32_t> sp(super_ptr, super_ptr + ns + 1), par(parent, parent + ns);
  std::vector<int64_t> rp(rowpat_ptr, rowpat_ptr + ns + 1), vp(val_ptr, val_ptr + ns + 1);
  int wmax = 0, rmax = 0;
  for (int k = 0; k < ns; ++k) {
    int w = sp[k + 1] - sp[k];
    if (w <= 0 || sp[k] % 3 != 0 || sp[k + 1] % 3 != 0) {
      set_error("set_system: supernode %d has columns [%d,%d): must be non-empty and hold whole nodes", k, sp[k],
                sp[k + 1]);
      return ICR_EINVAL;
    }
    int64_t r = rp[k + 1] - rp[k];
    if (r < 0 || r > n) {
      set_error("set_system: rowpat_ptr not non-decreasing at %d", k);
      return ICR_EINVAL;
    }
    if (vp[k + 1] - vp[k] != (int64_t)w * (w + r)) {
      set_error("set_system: panel %d has %lld values, expected (w+r)*w = %lld", k,
                (long long)(vp[k + 1] - vp[k]), (long long)w * (w + r));
      return ICR_EINVAL;
    }
    for (int64_t i = rp[k]; i < rp[k + 1]; ++i) {
      int row = rowpat[i];
      if (row < sp[k + 1] || row >= n || (i > rp[k] && row <= rowpat[i - 1])) {
        set_error("set_system: below-diagonal rows of supernode %d must be ascending in [%d,%d)", k, sp[k + 1], n);
        return ICR_EINVAL;
      }
    }
    if (r == 0) {
      if (par[k] != -1) {
        set_error("set_system: supernode %d has no below-diagonal rows but parent %d", k, par[k]);
        return ICR_EINVAL;
      }
    } else {
      int first = rowpat[rp[k]];
      int p = par[k];
      if (p <= k || p >= ns || first < sp[p] || first >= sp[p + 1]) {
        set_error("set_system: parent of supernode %d must own its first below-diagonal row %d", k, first);
        return ICR_EINVAL;
      }
    }
    wmax = std::max(wmax, w);
    rmax = std::max(rmax, (int)r);
  }
  for (int i = 0; i < n; ++i) {
    if (!(std::isfinite(D[i]) && D[i] > 0)) {
      set_error("set_system: pivot D[%d] = %g is not finite and positive", i, D[i]);
      return ICR_ENOTSPD;
    }
  }
  for (int64_t i = 0; i < vp[ns]; ++i) {
    if (!std::isfinite(Lp[i])) {
      set_error("set_system: Lpanels[%lld] is not finite", (long long)i);
      return ICR_EINVAL;
    }
  }
  // children, etree levels (height above the leaves), row maps into parent fronts
  std::vector<int32_t> nchild(ns, 0), level(ns, 0);
  for (int k = 0; k < ns; ++k)
    if (par[k] >= 0) nchild[par[k]]++;
  std::vector<int32_t> cptr(ns + 1, 0);
  for (int k = 0; k < ns; ++k) cptr[k + 1] = cptr[k] + nchild[k];
  std::vector<int32_t> clist(std::max(1, cptr[ns])), fill(cptr.begin(), cptr.end() - 1);
  for (int k = 0; k < ns; ++k)
    if (par[k] >= 0) clist[fill[par[k]]++] = k;
  for (int k = 0; k < ns; ++k)
    if (par[k] >= 0) level[par[k]] = std::max(level[par[k]], level[k] + 1);
  std::vector<int32_t> relidx(std::max<int64_t>(1, rp[ns]), 0);
  for (int k = 0; k < ns; ++k) {
    int p = par[k];
    if (p < 0) continue;
    int wp = sp[p + 1] - sp[p];
    const int32_t* Rp = rowpat + rp[p];
    int64_t rpn = rp[p + 1] - rp[p];
    for (int64_t i = rp[k]; i < rp[k + 1]; ++i) {
      int row = rowpat[i];
      if (row < sp[p + 1]) {
        relidx[i] = row - sp[p];
      } else {
        const int32_t* it = std::lower_bound(Rp, Rp + rpn, row);
        if (it == Rp + rpn || *it != row) {
          set_error("set_system: row %d of supernode %d is neither a column nor a below-diagonal row of its parent %d",
                    row, k, p);
          return ICR_EINVAL;
        }
        relidx[i] = wp + (int)(it - Rp);
      }
    }
  }
  // front-row contribution lists: for every row of every front, the
  // (child, child update row) pairs the extend-add sums into it, children in
  // ascending order; the child's row is stored as its row in the front
  // storage (the child's first front row + w_child + its update row)
  std::vector<int64_t> frp0(ns + 1, 0);
  for (int k = 0; k < ns; ++k) frp0[k + 1] = frp0[k] + (sp[k + 1] - sp[k]) + (rp[k + 1] - rp[k]);
  if (frp0[ns] >= (int64_t)INT32_MAX) {
    set_error("set_system: %lld front rows exceed the 32-bit row index", (long long)frp0[ns]);
    return ICR_EINVAL;
  }
  std::vector<int32_t> cptr_rows(frp0[ns] + 1, 0), crow_child(std::max<int64_t>(1, rp[ns])),
      crow_row(std::max<int64_t>(1, rp[ns]));
  for (int k = 0; k < ns; ++k)
    if (par[k] >= 0)
      for (int64_t i = rp[k]; i < rp[k + 1]; ++i) cptr_rows[frp0[par[k]] + relidx[i] + 1]++;
  for (int64_t i = 0; i < frp0[ns]; ++i) cptr_rows[i + 1] += cptr_rows[i];
  {
    std::vector<int32_t> fillr(cptr_rows.begin(), cptr_rows.end() - 1);
    for (int k = 0; k < ns; ++k)
      if (par[k] >= 0)
        for (int64_t i = rp[k]; i < rp[k + 1]; ++i) {
          const int64_t slot = fillr[frp0[par[k]] + relidx[i]]++;
          crow_child[slot] = k;
          crow_row[slot] = (int32_t)(frp0[k] + (sp[k + 1] - sp[k]) + (i - rp[k]));
        }
  }
  int nlev = 0;
  for (int k = 0; k < ns; ++k) nlev = std::max(nlev, level[k] + 1);
  std::vector<Level> levs(nlev);
  for (int k = 0; k < ns; ++k) levs[level[k]].count++;
  std::vector<int32_t> llist(ns);
  {
    int off = 0;
    for (auto& L : levs) {
      L.first = off;
      off += L.count;
      L.count = 0;
    }
    for (int k = 0; k < ns; ++k) {
      Level& L = levs[level[k]];
      llist[L.first + L.count++] = k;
      L.wmax = std::max(L.wmax, sp[k + 1] - sp[k]);
      L.rmax = std::max<int>(L.rmax, (int)(rp[k + 1] - rp[k]));
    }
  }
  std::vector<int64_t> frp(ns + 1, 0);
  for (int k = 0; k < ns; ++k) frp[k + 1] = frp[k] + (sp[k + 1] - sp[k]) + (rp[k + 1] - rp[k]);
  std::vector<int32_t> dsup(n), nsup(n / 3);
  for (int k = 0; k < ns; ++k)
    for (int j = sp[k]; j < sp[k + 1]; ++j) dsup[j] = k;
  for (int j = 0; j < n / 3; ++j) nsup[j] = dsup[3 * j];
  std::vector<double> dinv(n), dis(n);
  for (int i = 0; i < n; ++i) {
    dinv[i] = 1.0 / D[i];
    dis[i] = 1.0 / std::sqrt(D[i]);
  }

  std::vector<double> Gpanels;
  compute_G(ns, sp, rp, vp, Lp, Gpanels);

  RET(set_device(s));
  CK(cudaStreamSynchronize(s->ctx->stream));
  // from here buffers are replaced: a failure part way leaves no system
  s->has_system = false;
  s->has_mapping = s->has_WH = s->has_W = s->has_dirs = s->has_lam = false;
  s->obst_kind = 0;
  RET(dalloc(s, s->super_ptr, (ns + 1) * sizeof(int32_t)));
  RET(dalloc(s, s->rowpat_ptr, (ns + 1) * sizeof(int64_t)));
  RET(dalloc(s, s->rowpat, std::max<int64_t>(1, rp[ns]) * sizeof(int32_t)));
  RET(dalloc(s, s->val_ptr, (ns + 1) * sizeof(int64_t)));
  RET(dalloc(s, s->G, vp[ns] * s->tsize));
  RET(dalloc(s, s->dinv, n * sizeof(double)));
  RET(dalloc(s, s->dinvsqrt, n * sizeof(double)));
  RET(dalloc(s, s->parent, ns * sizeof(int32_t)));
  RET(dalloc(s, s->child_ptr, (ns + 1) * sizeof(int32_t)));
  RET(dalloc(s, s->child_list, clist.size() * sizeof(int32_t)));
  RET(dalloc(s, s->relidx, relidx.size() * sizeof(int32_t)));
  RET(dalloc(s, s->level_list, ns * sizeof(int32_t)));
  RET(dalloc(s, s->node_super, (n / 3) * sizeof(int32_t)));
  RET(dalloc(s, s->dof_super, n * sizeof(int32_t)));
  RET(dalloc(s, s->fr_ptr, (ns + 1) * sizeof(int64_t)));
  RET(dalloc(s, s->ctr_ptr, cptr_rows.size() * sizeof(int32_t)));
  RET(dalloc(s, s->ctr_child, crow_child.size() * sizeof(int32_t)));
  RET(dalloc(s, s->ctr_row, crow_row.size() * sizeof(int32_t)));
  RET(upload(s, s->super_ptr, sp.data(), ns + 1));
  RET(upload(s, s->rowpat_ptr, rp.data(), ns + 1));
  if (rp[ns]) RET(upload(s, s->rowpat, rowpat, rp[ns]));
  RET(upload(s, s->val_ptr, vp.data(), ns + 1));
  RET(upload_T(s, s->G, Gpanels.data(), vp[ns]));
  RET(upload(s, s->dinv, dinv.data(), n));
  RET(upload(s, s->dinvsqrt, dis.data(), n));
  RET(upload(s, s->parent, par.data(), ns));
  RET(upload(s, s->child_ptr, cptr.data(), ns + 1));
  RET(upload(s, s->child_list, clist.data(), clist.size()));
  RET(upload(s, s->relidx, relidx.data(), relidx.size()));
  RET(upload(s, s->level_list, llist.data(), ns));
  RET(upload(s, s->node_super, nsup.data(), n / 3));
  RET(upload(s, s->dof_super, dsup.data(), n));
  RET(upload(s, s->fr_ptr, frp.data(), ns + 1));
  RET(upload(s, s->ctr_ptr, cptr_rows.data(), cptr_rows.size()));
  RET(upload(s, s->ctr_child, crow_child.data(), crow_child.size()));
  RET(upload(s, s->ctr_row, crow_row.data(), crow_row.size()));
  if (s->prec == ICR_FP32) {
    // G_s of the supernodes wide enough for the tensor-core forward solve, as
    // 3xTF32 operand blocks of 128 rows x TC_KT columns (TC_BLOCK_BYTES each)
    std::vector<int64_t> goff(ns + 1, -1);
    std::vector<int32_t> blocks;
    int64_t nb = 0;
    for (int k = 0; k < ns; ++k) {
      const int w = sp[k + 1] - sp[k];
      if (w < TC_GEMM_MIN_W) continue;
      const int nrows = w + (int)(rp[k + 1] - rp[k]);
      const int nrt = (nrows + TC_TILE - 1) / TC_TILE, nk = (w + TC_KT - 1) / TC_KT;
      goff[k] = nb;
      for (int rt = 0; rt < nrt; ++rt)
        for (int kt = 0; kt < nk; ++kt) {
          blocks.push_back(k);
          blocks.push_back(rt);
          blocks.push_back(kt);
        }
      nb += (int64_t)nrt * nk;
    }
    RET(dalloc(s, s->gpk_off, (ns + 1) * sizeof(int64_t)));
    RET(upload(s, s->gpk_off, goff.data(), ns + 1));
    RET(dalloc(s, s->Gpk, std::max<int64_t>(1, nb) * TC_BLOCK_BYTES));
    if (nb) {
      DBuf list;
      RET(dalloc(s, list, blocks.size() * sizeof(int32_t)));
      const int rc = upload(s, list, blocks.data(), blocks.size());
      const int rc2 = rc == ICR_OK ? launch_pack_g(s, (const int32_t*)list.p, (int)(nb)) : rc;
      cudaStreamSynchronize(s->ctx->stream);
      dfree(s, list);
      if (rc2 != ICR_OK) return rc2;
    }
  }
  CK(cudaStreamSynchronize(s->ctx->stream));

  s->n = n;
  s->ns = ns;
  s->n_nodes = n / 3;
  s->h_super_ptr = sp;
  s->h_parent = par;
  s->h_rowpat_ptr = rp;
  s->h_val_ptr = vp;
  s->h_fr_ptr = frp;
  s->levels = levs;
  s->h_level_list = llist;
  s->tc_level.assign(nlev, 0);
  for (int l = 0; l < nlev; ++l) s->tc_level[l] = levs[l].wmax >= TC_GEMM_MIN_W ? 1 : 0;
  s->tuned = false;
  RET(dalloc(s, s->tc_super, ns));
  RET(upload_tc_super(s));
  {
    std::vector<int32_t> lf(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) lf[l + 1] = levs[l].first + levs[l].count;
    RET(dalloc(s, s->level_first, (nlev + 1) * sizeof(int32_t)));
    RET(upload(s, s->level_first, lf.data(), nlev + 1));
  }
  s->total_front_rows = frp[ns];
  s->wmax = wmax;
  s->rmax = rmax;
  s->has_system = true;
  s->has_mapping = s->has_WH = s->has_W = s->has_dirs = s->has_lam = false;
  return ICR_OK;
}

// the checks of icr_set_mapping
static int check_mapping(const Scene* s, int32_t m, const int32_t* nodes, const double* bary) {
  if (!s->has_system) {
    set_error("set_mapping: call icr_set_system first");
    return ICR_ESTATE;
  }
  if (m < 0 || m > 32768 || (m > 0 && (!nodes || !bary))) {
    set_error("set_mapping: m = %d must be in [0, 32768] with non-NULL arrays", m);
    return ICR_EINVAL;
  }
  for (int a = 0; a < m; ++a) {
    double sum = 0;
    for (int i = 0; i < 4; ++i) {
      int nd = nodes[4 * a + i];
      double b = bary[4 * a + i];
      if (nd < 0 || nd >= s->n_nodes) {
        set_error("set_mapping: node id %d of contact %d out of range [0,%d)", nd, a, s->n_nodes);
        return ICR_EINVAL;
      }
      if (!(std::isfinite(b) && b >= 0)) {
        set_error("set_mapping: weight %g of contact %d is negative or not finite", b, a);
        return ICR_EINVAL;
      }
      sum += b;
    }
    if (std::fabs(sum - 1.0) > 1e-12) {
      set_error("set_mapping: weights of contact %d sum to %.17g, not 1", a, sum);
      return ICR_EINVAL;
    }
  }
  return ICR_OK;
}

int icr_set_mapping(icr_scene* s, int32_t m, const int32_t* nodes, const double* bary) {
  RET(check_scene(s));
  RET(check_mapping(s, m, nodes, bary));
  RET(set_device(s));
  const int ns = s->ns;
  const int words = std::max(1, (m + 31) / 32);
  const int64_t ldx = std::max<int64_t>(32, ((3 * (int64_t)m + 31) / 32) * 32);
  const int64_t ldw = std::max<int64_t>(96, ((3 * (int64_t)m + 95) / 96) * 96);
  const size_t T = s->tsize;
  const size_t mm = std::max(1, m);
  // from here buffers are replaced: a failure part way leaves no mapping
  s->has_mapping = s->has_WH = s->has_W = s->has_dirs = s->has_lam = false;
  s->obst_kind = 0;
  RET(dalloc(s, s->nodes, 4 * mm * sizeof(int32_t)));
  RET(dalloc(s, s->bary, 4 * mm * T));
  RET(dalloc(s, s->bitmap, (size_t)ns * words * sizeof(uint32_t)));
  RET(dalloc(s, s->wprefix, (size_t)ns * words * sizeof(int32_t)));
  RET(dalloc(s, s->qcount, ns * sizeof(int32_t)));
  RET(dalloc(s, s->plan, ((size_t)PLAN_LISTS * (ns + 1) + 3 + 2 * s->levels.size()) * sizeof(int32_t)));
  RET(dalloc(s, s->qidx, (size_t)ns * mm * sizeof(int32_t)));
  RET(dalloc(s, s->qpos, (size_t)ns * mm * sizeof(int32_t)));
  RET(dalloc(s, s->qinv, (size_t)ns * mm * sizeof(int32_t)));
  RET(dalloc(s, s->X, (size_t)s->total_front_rows * ldx * T));
  RET(dalloc(s, s->Ftop, (size_t)s->n * ldx * T));
  RET(dalloc(s, s->WH, 9 * mm * mm * T));
  RET(dalloc(s, s->W, 3 * mm * (size_t)ldw * T));
  RET(dalloc(s, s->C, 9 * mm * T));
  RET(dalloc(s, s->delta, 3 * mm * T));
  RET(dalloc(s, s->mu, mm * T));
  RET(dalloc(s, s->lam, 3 * mm * T));
  RET(dalloc(s, s->lam0, 3 * mm * T));
  RET(dalloc(s, s->p, 3 * mm * sizeof(double)));
  RET(dalloc(s, s->p0, 3 * mm * sizeof(double)));
  RET(dalloc(s, s->u, 6 * mm * sizeof(double)));   // u (3m) then the last increment dp (3m)
  RET(dalloc(s, s->uk, 3 * mm * T));
  RET(dalloc(s, s->wblk, mm * ((mm + (s->prec == ICR_FP64 ? 15 : 31)) / (s->prec == ICR_FP64 ? 16 : 32)) * T));
  RET(dalloc(s, s->y, s->n * T));
  RET(dalloc(s, s->dq, s->n * T));
  RET(dalloc(s, s->stats, sizeof(PgsDevStats)));
  RET(dalloc(s, s->dev_err, sizeof(int)));
  RET(dalloc(s, s->newton, 2 * sizeof(int32_t)));
  RET(dalloc(s, s->pgsb, 2 * mm * T));
  RET(dalloc(s, s->WH16, s->prec == ICR_FP32 ? 9 * mm * mm * 2 : 16));
  if (s->prec == ICR_FP32) {
    // tensor-core operand blocks: per supernode ceil(3m/128) column tiles x
    // ceil(w/TC_KT) row chunks of TC_BLOCK_BYTES (two TF32 planes)
    const int tmax = std::max(1, (int)((3 * (int64_t)m + 127) / 128));
    if (tmax != s->tc_tmax || !s->tc_boff.p) {   // the block offsets depend on the tile count only
      std::vector<int64_t> boff(ns + 1, 0);
      for (int k = 0; k < ns; ++k)
        boff[k + 1] = boff[k] + (int64_t)tmax * ((s->h_super_ptr[k + 1] - s->h_super_ptr[k] + TC_KT - 1) / TC_KT);
      RET(dalloc(s, s->tc_boff, (ns + 1) * sizeof(int64_t)));
      RET(upload(s, s->tc_boff, boff.data(), ns + 1));
      CK(cudaStreamSynchronize(s->ctx->stream));   // boff is a local vector
      RET(dalloc(s, s->Ypk, (size_t)boff[ns] * TC_BLOCK_BYTES));
      s->tc_tmax = tmax;
    }
  }
  if (m) {
    RET(upload(s, s->nodes, nodes, 4 * (size_t)m));
    RET(upload_T(s, s->bary, bary, 4 * (size_t)m));
  }
  cudaStream_t st = s->ctx->stream;
  // W's padding columns stay zero (update_W writes the 3m x 3m part); a new
  // mapping resets the contact state in one launch
  if (s->W_zeroed != s->W.gen || s->W_zeroed_ld != ldw || s->W_zeroed_rows != 3 * (int64_t)mm) {
    CK(cudaMemsetAsync(s->W.p, 0, 3 * mm * (size_t)ldw * T, st));
    s->W_zeroed = s->W.gen;
    s->W_zeroed_ld = ldw;
    s->W_zeroed_rows = 3 * (int64_t)mm;
  }
  RET(launch_reset_contacts(s, (int)mm));
  s->m = m;
  s->words = words;
  s->ldx = ldx;
  s->ldw = ldw;
  s->has_mapping = true;
  s->has_WH = s->has_W = s->has_dirs = s->has_lam = false;
  s->obst_kind = 0;
  s->tuned = false;
  return ICR_OK;
}

static int need_mapping(Scene* s, const char* who) {
  if (!s->has_mapping) {
    set_error("%s: call icr_set_mapping first", who);
    return ICR_ESTATE;
  }
  return ICR_OK;
}

int icr_set_proximity(icr_scene* s, const double* p) {
  RET(check_scene(s));
  RET(need_mapping(s, "set_proximity"));
  if (s->m && !p) {
    set_error("set_proximity: p is NULL");
    return ICR_EINVAL;
  }
  for (int i = 0; i < 3 * s->m; ++i)
    if (!std::isfinite(p[i])) {
      set_error("set_proximity: p[%d] is not finite", i);
      return ICR_EINVAL;
    }
  RET(set_device(s));
  RET(upload(s, s->p, p, 3 * (size_t)s->m));
  if (s->m)
    CK(cudaMemcpyAsync(s->p0.p, s->p.p, 3 * (size_t)s->m * sizeof(double), cudaMemcpyDeviceToDevice,
                       s->ctx->stream));
  return ICR_OK;
}

int icr_reset_proximity(icr_scene* s) {
  RET(check_scene(s));
  RET(need_mapping(s, "reset_proximity"));
  RET(set_device(s));
  if (s->m) {
    CK(cudaMemcpyAsync(s->p.p, s->p0.p, 3 * (size_t)s->m * sizeof(double), cudaMemcpyDeviceToDevice,
                       s->ctx->stream));
    CK(cudaMemsetAsync(s->u.p, 0, 6 * (size_t)s->m * sizeof(double), s->ctx->stream));
  }
  return ICR_OK;
}

int icr_scene_launches(icr_scene* s, uint64_t* out) {
  RET(check_scene(s));
  if (!out) {
    set_error("out is NULL");
    return ICR_EINVAL;
  }
  *out = s->launches;
  return ICR_OK;
}

static int check_directions(const double* C, int m) {
  for (int a = 0; a < m; ++a) {
    const double* B = C + 9 * a;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double d = B[3 * i] * B[3 * j] + B[3 * i + 1] * B[3 * j + 1] + B[3 * i + 2] * B[3 * j + 2];
        if (!(std::fabs(d - (i == j ? 1.0 : 0.0)) <= 1e-6)) {
          set_error("update_directions: block %d is not orthonormal (row %d . row %d = %g)", a, i, j, d);
          return ICR_EINVAL;
        }
      }
  }
  return ICR_OK;
}

int icr_update_directions(icr_scene* s, const double* C, const double* delta, const double* mu) {
  RET(check_scene(s));
  RET(need_mapping(s, "update_directions"));
  const int m = s->m;
  if (m && (!C || !delta)) {
    set_error("update_directions: C and delta must not be NULL");
    return ICR_EINVAL;
  }
  RET(check_directions(C, m));
  for (int i = 0; i < 3 * m; ++i)
    if (!std::isfinite(delta[i])) {
      set_error("update_directions: delta[%d] is not finite", i);
      return ICR_EINVAL;
    }
  if (mu)
    for (int a = 0; a < m; ++a)
      if (!(std::isfinite(mu[a]) && mu[a] >= 0)) {
        set_error("update_directions: mu[%d] = %g must be finite and >= 0", a, mu[a]);
        return ICR_EINVAL;
      }
  RET(set_device(s));
  RET(upload_T(s, s->C, C, 9 * (size_t)m));
  RET(upload_T(s, s->delta, delta, 3 * (size_t)m));
  if (mu) RET(upload_T(s, s->mu, mu, (size_t)m));
  s->has_dirs = true;
  s->has_W = false;
  return ICR_OK;
}

int icr_set_obstacle_plane(icr_scene* s, int32_t n_iters, const double* normals, const double* anchors) {
  RET(check_scene(s));
  RET(need_mapping(s, "set_obstacle_plane"));
  const int m = s->m;
  if (n_iters <= 0 || (m && (!normals || !anchors))) {
    set_error("set_obstacle_plane: n_iters must be > 0 and arrays non-NULL");
    return ICR_EINVAL;
  }
  for (size_t i = 0; i < (size_t)n_iters * m; ++i) {
    const double* v = normals + 3 * i;
    double nn = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (!(std::fabs(nn - 1.0) <= 1e-6)) {
      set_error("set_obstacle_plane: normal %zu is not a unit vector", i);
      return ICR_EINVAL;
    }
  }
  for (int i = 0; i < 3 * m; ++i)
    if (!std::isfinite(anchors[i])) {
      set_error("set_obstacle_plane: anchor coordinate %d is not finite", i);
      return ICR_EINVAL;
    }
  RET(set_device(s));
  s->obst_kind = 0;   // until the new obstacle is in place
  RET(dalloc(s, s->obst_normals, std::max<size_t>(1, (size_t)n_iters * m * 3) * sizeof(double)));
  RET(dalloc(s, s->obst_anchors, std::max<size_t>(1, (size_t)m * 3) * sizeof(double)));
  RET(upload(s, s->obst_normals, normals, (size_t)n_iters * m * 3));
  RET(upload(s, s->obst_anchors, anchors, (size_t)m * 3));
  s->obst_kind = 1;
  s->obst_iters = n_iters;
  return ICR_OK;
}

// the checks of icr_set_obstacle_spheres for m contacts
static int check_spheres(int m, int32_t n_spheres, const double* spheres, const int32_t* contact_sphere,
                         const double* anchors) {
  if (n_spheres <= 0 || !spheres || (m && (!anchors || !contact_sphere))) {
    set_error("set_obstacle_spheres: need n_spheres > 0, the spheres, each contact's sphere and anchors");
    return ICR_EINVAL;
  }
  for (int i = 0; i < n_spheres; ++i) {
    const double* q = spheres + 4 * i;
    if (!(std::isfinite(q[0]) && std::isfinite(q[1]) && std::isfinite(q[2]) && q[3] > 0 && std::isfinite(q[3]))) {
      set_error("set_obstacle_spheres: sphere %d needs a finite centre and a positive radius", i);
      return ICR_EINVAL;
    }
  }
  for (int a = 0; a < m; ++a)
    if (contact_sphere[a] < 0 || contact_sphere[a] >= n_spheres) {
      set_error("set_obstacle_spheres: contact %d names sphere %d of %d", a, contact_sphere[a], n_spheres);
      return ICR_EINVAL;
    }
  for (int i = 0; i < 3 * m; ++i)
    if (!std::isfinite(anchors[i])) {
      set_error("set_obstacle_spheres: anchor coordinate %d is not finite", i);
      return ICR_EINVAL;
    }
  return ICR_OK;
}

int icr_set_obstacle_spheres(icr_scene* s, int32_t n_spheres, const double* spheres, const int32_t* contact_sphere,
                             const double* anchors) {
  RET(check_scene(s));
  RET(need_mapping(s, "set_obstacle_spheres"));
  const int m = s->m;
  RET(check_spheres(m, n_spheres, spheres, contact_sphere, anchors));
  RET(set_device(s));
  s->obst_kind = 0;   // until the new obstacle is in place
  RET(dalloc(s, s->obst_anchors, std::max<size_t>(1, (size_t)m * 3) * sizeof(double)));
  RET(dalloc(s, s->obst_spheres, (size_t)n_spheres * 4 * sizeof(double)));
  RET(dalloc(s, s->obst_of, std::max<size_t>(1, (size_t)m) * sizeof(int32_t)));
  RET(upload(s, s->obst_anchors, anchors, (size_t)m * 3));
  RET(upload(s, s->obst_spheres, spheres, (size_t)n_spheres * 4));
  if (m) RET(upload(s, s->obst_of, contact_sphere, (size_t)m));
  s->obst_kind = 2;
  s->obst_iters = 0;
  return ICR_OK;
}

int icr_set_step_inputs(icr_scene* s, int32_t m, const int32_t* nodes, const double* bary, const double* p0,
                        const double* mu, int32_t n_spheres, const double* spheres, const int32_t* contact_sphere,
                        const double* anchors) {
  RET(check_scene(s));
  const bool fast = s->has_mapping && m > 0 && m == s->m && n_spheres > 0 && s->obst_kind == 2 &&
                    s->obst_spheres.bytes >= (size_t)n_spheres * 4 * sizeof(double) &&
                    s->W_zeroed == s->W.gen && s->W_zeroed_ld == s->ldw && s->W_zeroed_rows == 3 * (int64_t)m;
  if (!fast) {
    RET(icr_set_mapping(s, m, nodes, bary));
    RET(icr_set_proximity(s, p0));
    RET(icr_set_obstacle_spheres(s, n_spheres, spheres, contact_sphere, anchors));
    return icr_set_field(s, ICR_FIELD_MU, mu, (size_t)m * sizeof(double));
  }
  RET(check_mapping(s, m, nodes, bary));
  if (!p0 || !mu) {
    set_error("set_step_inputs: p0 and mu must not be NULL");
    return ICR_EINVAL;
  }
  for (int i = 0; i < 3 * m; ++i)
    if (!std::isfinite(p0[i])) {
      set_error("set_proximity: p[%d] is not finite", i);
      return ICR_EINVAL;
    }
  RET(check_spheres(m, n_spheres, spheres, contact_sphere, anchors));
  for (int a = 0; a < m; ++a)
    if (!std::isfinite(mu[a])) {
      set_error("set_field: value %d is not finite", a);
      return ICR_EINVAL;
    }
  RET(set_device(s));
  // staging layout (bytes, 16-byte aligned parts): nodes, sphere ids, bary, mu, p0, anchors, spheres
  const size_t T = s->tsize;
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  int64_t off[7];
  off[0] = 0;
  off[1] = (int64_t)al((size_t)off[0] + 16 * (size_t)m);
  off[2] = (int64_t)al((size_t)off[1] + 4 * (size_t)m);
  off[3] = (int64_t)al((size_t)off[2] + 4 * T * (size_t)m);
  off[4] = (int64_t)al((size_t)off[3] + T * (size_t)m);
  off[5] = (int64_t)al((size_t)off[4] + 24 * (size_t)m);
  off[6] = (int64_t)al((size_t)off[5] + 24 * (size_t)m);
  const size_t total = al((size_t)off[6] + 32 * (size_t)n_spheres);
  if (s->stage_bytes < total) {
    for (int k = 0; k < 2; ++k) {
      if (s->stage_used[k]) CK(cudaEventSynchronize(s->stage_ev[k]));
      if (s->stage_host[k]) cudaFreeHost(s->stage_host[k]);
      s->stage_host[k] = nullptr;
      s->stage_used[k] = false;
      if (!s->stage_ev[k]) CK(cudaEventCreateWithFlags(&s->stage_ev[k], cudaEventDisableTiming));
    }
    CK(cudaStreamSynchronize(s->ctx->stream));   // the device buffer may be in use
    if (s->stage_dev.p) {
      cudaFree(s->stage_dev.p);
      s->ctx->in_use -= s->stage_dev.bytes;
      s->stage_dev.p = nullptr;
      s->stage_dev.bytes = 0;
      s->stage_bytes = 0;
    }
    // outside dalloc: a captured step graph does not read it, so it stays valid
    Ctx* c = s->ctx;
    if (c->budget && c->in_use + total > c->budget) {
      set_error("set_step_inputs: staging %zu bytes exceeds the context HBM budget", total);
      return ICR_ENOMEM;
    }
    CK(cudaMalloc(&s->stage_dev.p, total));
    s->stage_dev.bytes = total;
    s->ctx->in_use += total;
    for (int k = 0; k < 2; ++k) CK(cudaHostAlloc((void**)&s->stage_host[k], total, cudaHostAllocDefault));
    s->stage_bytes = total;
  }
  const int slot = s->stage_slot;
  s->stage_slot ^= 1;
  if (s->stage_used[slot]) CK(cudaEventSynchronize(s->stage_ev[slot]));   // its last copy has left
  unsigned char* h = s->stage_host[slot];
  std::memcpy(h + off[0], nodes, 16 * (size_t)m);
  std::memcpy(h + off[1], contact_sphere, 4 * (size_t)m);
  if (s->prec == ICR_FP64) {
    std::memcpy(h + off[2], bary, 32 * (size_t)m);
    std::memcpy(h + off[3], mu, 8 * (size_t)m);
  } else {
    float* b = (float*)(h + off[2]);
    for (int i = 0; i < 4 * m; ++i) b[i] = (float)bary[i];
    float* u = (float*)(h + off[3]);
    for (int i = 0; i < m; ++i) u[i] = (float)mu[i];
  }
  std::memcpy(h + off[4], p0, 24 * (size_t)m);
  std::memcpy(h + off[5], anchors, 24 * (size_t)m);
  std::memcpy(h + off[6], spheres, 32 * (size_t)n_spheres);
  CK(cudaMemcpyAsync(s->stage_dev.p, h, total, cudaMemcpyHostToDevice, s->ctx->stream));
  CK(cudaEventRecord(s->stage_ev[slot], s->ctx->stream));
  s->stage_used[slot] = true;
  RET(launch_unpack_inputs(s, n_spheres, off));
  // the state icr_set_mapping leaves, then the obstacle's
  s->has_WH = s->has_W = s->has_dirs = s->has_lam = false;
  s->tuned = false;
  s->obst_kind = 2;
  s->obst_iters = 0;
  return ICR_OK;
}

int icr_set_obstacle_sphere(icr_scene* s, const double* center, double radius, const double* anchors) {
  RET(check_scene(s));
  if (!center) {
    set_error("set_obstacle_sphere: need a centre");
    return ICR_EINVAL;
  }
  const double q[4] = {center[0], center[1], center[2], radius};
  std::vector<int32_t> of(std::max(0, s->m), 0);
  return icr_set_obstacle_spheres(s, 1, q, of.data(), anchors);
}

int icr_linearize(icr_scene* s, int32_t k) {
  RET(check_scene(s));
  RET(need_mapping(s, "linearize"));
  if (s->obst_kind == 0) {
    set_error("linearize: no obstacle set");
    return ICR_ESTATE;
  }
  if (s->obst_kind == 1 && (k < 0 || k >= s->obst_iters)) {
    set_error("linearize: iteration %d outside the %d plane normal sets", k, s->obst_iters);
    return ICR_EINVAL;
  }
  RET(set_device(s));
  RET(launch_linearize(s, k));
  s->has_dirs = true;
  s->has_W = false;
  return ICR_OK;
}

int icr_build_WH(icr_scene* s) {
  RET(check_scene(s));
  RET(need_mapping(s, "build_WH"));
  RET(set_device(s));
  RET(launch_build_WH(s));
  s->has_WH = true;
  s->has_W = false;
  return ICR_OK;
}

int icr_update_W(icr_scene* s) {
  RET(check_scene(s));
  if (!s->has_WH || !s->has_dirs) {
    set_error("update_W: needs icr_build_WH and directions first");
    return ICR_ESTATE;
  }
  RET(set_device(s));
  RET(launch_update_W(s));
  s->has_W = true;
  return ICR_OK;
}

int icr_solve_friction(icr_scene* s, int warm_start, icr_pgs_stats* stats) {
  RET(check_scene(s));
  if (!s->has_W) {
    set_error("solve_friction: needs W (icr_update_W or icr_set_field)");
    return ICR_ESTATE;
  }
  RET(set_device(s));
  RET(launch_pgs(s, warm_start ? 1 : 0, stats ? 1 : 0));
  s->has_lam = true;
  if (!stats) return ICR_OK;
  RET(check_device_error(s));
  PgsDevStats d;
  CK(cudaMemcpyAsync(&d, s->stats.p, sizeof(d), cudaMemcpyDeviceToHost, s->ctx->stream));
  CK(cudaStreamSynchronize(s->ctx->stream));
  stats->sweeps = d.sweeps;
  stats->n_separated = d.n_sep;
  stats->n_stick = d.n_stick;
  stats->n_slip = d.n_slip;
  stats->eps = d.eps;
  double r[4];
  for (int i = 0; i < 4; ++i) std::memcpy(&r[i], &d.res_bits[i], sizeof(double));
  stats->res_normal = r[0];
  stats->res_cone = r[1];
  stats->res_stick = r[2];
  stats->res_slip = r[3];
  stats->sweeps_s_only = d.s_only;
  stats->deferred_folds = d.folds;
  stats->rechecks = d.rechecks;
  stats->joins = d.joins;
  if (s->params.tol > 0 && d.eps > s->params.tol && s->m > 0) {
    set_error("solve_friction: eps %g above tol %g after %d sweeps", d.eps, s->params.tol, d.sweeps);
    return ICR_ENOCONV;
  }
  return ICR_OK;
}

int icr_update_proximity(icr_scene* s, double* dp_out) {
  RET(check_scene(s));
  if (!s->has_lam || !s->has_dirs || !s->has_WH) {
    set_error("update_proximity: needs W_H, directions and a solve first");
    return ICR_ESTATE;
  }
  RET(set_device(s));
  RET(launch_update_proximity(s));
  if (dp_out && s->m) {
    CK(cudaMemcpyAsync(dp_out, (double*)s->u.p + 3 * (size_t)s->m, 3 * (size_t)s->m * sizeof(double),
                       cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(cudaStreamSynchronize(s->ctx->stream));
  }
  return ICR_OK;
}

int icr_correct_motion(icr_scene* s, double* dq_out, int reset) {
  RET(check_scene(s));
  if (!s->has_WH) {
    set_error("correct_motion: needs icr_build_WH first");
    return ICR_ESTATE;
  }
  RET(set_device(s));
  RET(launch_correct_motion(s));
  if (dq_out) RET(download_T(s, s->dq, dq_out, s->n));
  if (reset && s->m) CK(cudaMemsetAsync(s->u.p, 0, 3 * (size_t)s->m * sizeof(double), s->ctx->stream));
  return ICR_OK;
}

int icr_profile_begin(icr_scene* s) {
  RET(check_scene(s));
  if (!s->prof) s->prof = new (std::nothrow) Profiler();
  if (!s->prof) {
    set_error("profile_begin: out of host memory");
    return ICR_ENOMEM;
  }
  s->prof->recycle();
  return ICR_OK;
}

int icr_profile_end(icr_scene* s, icr_kernel_time* out, int32_t max_out, int32_t* n_out) {
  RET(check_scene(s));
  if (!s->prof) {
    set_error("profile_end: no icr_profile_begin before");
    return ICR_ESTATE;
  }
  if (max_out < 0 || (max_out > 0 && !out) || !n_out) {
    set_error("profile_end: need max_out >= 0, out for max_out entries and n_out");
    return ICR_EINVAL;
  }
  RET(set_device(s));
  CK(cudaStreamSynchronize(s->ctx->stream));
  Profiler* P = s->prof;
  s->prof = nullptr;   // launches of the aggregation below (none) and later ones are not timed
  std::vector<icr_kernel_time> agg;
  int rc = ICR_OK;
  for (const auto& r : P->recs) {
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "profile_end: cudaEventElapsedTime");
      break;
    }
    size_t i = 0;
    while (i < agg.size() && std::strncmp(agg[i].name, r.name, sizeof(agg[i].name) - 1) != 0) ++i;
    if (i == agg.size()) {
      icr_kernel_time k{};
      std::snprintf(k.name, sizeof(k.name), "%s", r.name);
      agg.push_back(k);
    }
    agg[i].launches += 1;
    agg[i].total_ms += ms;
  }
  P->recycle();
  s->prof = nullptr;
  delete P;
  if (rc != ICR_OK) return rc;
  *n_out = (int32_t)agg.size();
  for (int32_t i = 0; i < std::min<int32_t>(max_out, (int32_t)agg.size()); ++i) out[i] = agg[i];
  return ICR_OK;
}

int icr_build_info(icr_scene* s, icr_build_info_t* out) {
  RET(check_scene(s));
  if (!out) {
    set_error("build_info: out must not be NULL");
    return ICR_EINVAL;
  }
  if (!s->has_WH) {
    set_error("build_info: needs icr_build_WH first");
    return ICR_ESTATE;
  }
  RET(set_device(s));
  *out = icr_build_info_t{};
  out->levels = (int32_t)s->levels.size();
  out->prox_split = 3 * (size_t)s->m * s->tsize > 48 * 1024 ? 1 : 0;
  if (s->m == 0) return ICR_OK;
  const int ns = s->ns, nlev = (int)s->levels.size();
  const size_t words = (size_t)PLAN_LISTS * (ns + 1) + 3 + 2 * (size_t)nlev;
  std::vector<int32_t> plan(words);
  std::vector<int32_t> qc(ns);
  CK(cudaMemcpyAsync(plan.data(), s->plan.p, words * sizeof(int32_t), cudaMemcpyDeviceToHost, s->ctx->stream));
  CK(cudaMemcpyAsync(qc.data(), s->qcount.p, ns * sizeof(int32_t), cudaMemcpyDeviceToHost, s->ctx->stream));
  CK(cudaStreamSynchronize(s->ctx->stream));
  auto P = [&](int list, int pos) { return plan[(size_t)list * (ns + 1) + pos]; };
  const int32_t* splits = plan.data() + (size_t)PLAN_LISTS * (ns + 1) + 2 + nlev;
  out->gemm_tc_split_max = 1;
  for (int li = 0; li < nlev; ++li) {
    const Level& lv = s->levels[li];
    const int units = P(PLAN_GTC, lv.first + lv.count) - P(PLAN_GTC, lv.first);
    if (units > 0) {
      ++out->tc_levels;
      out->gemm_tc_split_max = std::max(out->gemm_tc_split_max, splits[li]);
    }
  }
  // algorithmic flops of each engine, with the planner's rules (k_plan): the
  // forward solve of front s costs 3q (w^2 + 2 w r) (triangular solve on the
  // w x w block, product with the r x w block below), the contraction
  // w c (c + 1) for c = 3q columns (upper triangle of Y_s^T Y_s)
  int mode = s->params.contraction;
  if (s->prec == ICR_FP64) mode = ICR_CONTRACT_SIMT;
  if (mode == ICR_CONTRACT_AUTO) mode = ICR_CONTRACT_TF32X3;
  const bool simt = mode == ICR_CONTRACT_SIMT;
  for (int li = 0; li < nlev; ++li) {
    const Level& lv = s->levels[li];
    for (int p = lv.first; p < lv.first + lv.count; ++p) {
      const int sn = s->h_level_list[p];
      const double q = qc[sn], c = 3.0 * q;
      if (q == 0) continue;
      const double w = s->h_super_ptr[sn + 1] - s->h_super_ptr[sn];
      const double r = (double)(s->h_rowpat_ptr[sn + 1] - s->h_rowpat_ptr[sn]);
      const double fwd = c * (w * w + 2.0 * w * r), con = w * c * (c + 1.0);
      const bool tcg = !simt && s->tc_level[li] == FWD_TC && w >= TC_GEMM_MIN_W && c >= TC_GEMM_MIN_COLS;
      (tcg ? out->flops_front_tc : out->flops_front_simt) += fwd;
      (!simt && c >= 64 ? out->flops_contract_tc : out->flops_contract_simt) += con;
    }
  }
  out->gemm_tc_units = P(PLAN_GTC, ns);
  out->gemm_simt_units = P(PLAN_GEMM, ns);
  out->contract_tc_units = P(PLAN_TC, ns);
  out->contract_tc_split = out->contract_tc_units > 0 ? splits[nlev] : 1;
  out->contract_simt_units = P(PLAN_SIMT, ns);
  for (int i = 0; i < ns; ++i) out->reach_nnz += qc[i];
  for (uint8_t f : s->tc_level) out->short_tile_levels += f == FWD_SIMT_SHORT ? 1 : 0;
  return ICR_OK;
}

// the per-level forward-solve engine flags, per supernode, for the planner
static int upload_tc_super(Scene* s) {
  std::vector<uint8_t> f(s->ns, 0);
  for (size_t l = 0; l < s->levels.size(); ++l)
    for (int i = 0; i < s->levels[l].count; ++i) f[s->h_level_list[s->levels[l].first + i]] = s->tc_level[l];
  CK(cudaMemcpy(s->tc_super.p, f.data(), f.size(), cudaMemcpyHostToDevice));
  return ICR_OK;
}

static int autotune(Scene* s, double* level_ms, int max_levels) {
  const int nlev = (int)s->levels.size();
  cudaStream_t st = s->ctx->stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    set_error("autotune: the scene's stream is being captured");
    return ICR_ESTATE;
  }
  std::vector<cudaEvent_t> ev(nlev + 1, nullptr);
  for (auto& e : ev) {
    const cudaError_t rc = cudaEventCreate(&e);
    if (rc != cudaSuccess) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return cuda_fail(rc, "autotune: cudaEventCreate");
    }
  }
  auto done = [&](int rc) {
    s->level_events = nullptr;
    for (auto& x : ev) cudaEventDestroy(x);
    return rc;
  };
  // every level on one tile shape (the tensor cores only where a level has a
  // front wide enough; its narrower fronts then take 64-row CUDA-core tiles)
  auto configure = [&](int cfg) {
    for (int l = 0; l < nlev; ++l)
      s->tc_level[l] = cfg == FWD_TC ? (s->levels[l].wmax >= TC_GEMM_MIN_W ? FWD_TC : FWD_SIMT) : cfg;
    return upload_tc_super(s);
  };
  const int mode = s->params.contraction;
  const bool tc_ok = s->prec == ICR_FP32 && mode != ICR_CONTRACT_SIMT;
  const int ncfg = tc_ok ? FWD_TILES : FWD_TILES - 1;
  const int cfgs[FWD_TILES] = {FWD_SIMT, FWD_SIMT_SHORT, FWD_TC};
  // per level and tile shape, the median of REPS timed builds; the shapes
  // alternate so that clock and cache drift affect them alike
  constexpr int REPS = 5;
  std::vector<double> samp[FWD_TILES];
  for (auto& v : samp) v.assign((size_t)nlev * REPS, 0.0);
  for (int rep = -1; rep < REPS; ++rep) {
    for (int ci = 0; ci < ncfg; ++ci) {
      const int cfg = cfgs[ci];
      int rc = configure(cfg);
      if (rc != ICR_OK) return done(rc);
      s->level_events = rep >= 0 ? ev.data() : nullptr;   // rep -1 warms up
      rc = launch_build_WH(s);
      if (rc != ICR_OK) return done(rc);
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return done(cuda_fail(e, "autotune: build"));
      if (rep < 0) continue;
      for (int l = 0; l < nlev; ++l) {
        float ms = 0.f;
        const cudaError_t e2 = cudaEventElapsedTime(&ms, ev[l], ev[l + 1]);
        if (e2 != cudaSuccess) return done(cuda_fail(e2, "autotune: cudaEventElapsedTime"));
        samp[cfg][(size_t)l * REPS + rep] = ms;
      }
    }
  }
  // per level: the faster CUDA-core tile, replaced by the tensor cores when
  // they win by 3 %
  for (int l = 0; l < nlev; ++l) {
    double med[FWD_TILES];
    for (int ci = 0; ci < FWD_TILES; ++ci) {
      const int cfg = cfgs[ci];
      if (ci >= ncfg) {
        med[cfg] = med[FWD_SIMT];
        continue;
      }
      std::vector<double> v(samp[cfg].begin() + (size_t)l * REPS, samp[cfg].begin() + (size_t)(l + 1) * REPS);
      std::nth_element(v.begin(), v.begin() + REPS / 2, v.end());
      med[cfg] = v[REPS / 2];
    }
    const int simt = med[FWD_SIMT_SHORT] < med[FWD_SIMT] ? FWD_SIMT_SHORT : FWD_SIMT;
    const bool wide = tc_ok && s->levels[l].wmax >= TC_GEMM_MIN_W;
    s->tc_level[l] = wide && med[FWD_TC] < 0.97 * med[simt] ? FWD_TC : simt;
    if (level_ms && l < max_levels) {
      level_ms[3 * l] = med[FWD_SIMT];
      level_ms[3 * l + 1] = med[FWD_SIMT_SHORT];
      level_ms[3 * l + 2] = wide ? med[FWD_TC] : med[FWD_SIMT];
    }
  }
  const int rc = upload_tc_super(s);
  if (rc != ICR_OK) return done(rc);

  s->tuned = true;
  s->has_WH = true;   // every tuning build formed W_H
  RET(check_device_error(s));
  return done(ICR_OK);
}

int icr_set_forward_plan(icr_scene* s, const uint8_t* tc_levels, int32_t n_levels) {
  RET(check_scene(s));
  if (!s->has_system) {
    set_error("set_forward_plan: call icr_set_system first");
    return ICR_ESTATE;
  }
  const int nlev = (int)s->levels.size();
  if (n_levels != nlev || !tc_levels) {
    set_error("set_forward_plan: tc_levels must hold one flag per etree level (%d)", nlev);
    return ICR_EINVAL;
  }
  for (int l = 0; l < nlev; ++l)
    if (tc_levels[l] >= FWD_TILES) {
      set_error("set_forward_plan: tile %d of level %d is not 0, 1 or 2", tc_levels[l], l);
      return ICR_EINVAL;
    }
  RET(set_device(s));
  for (int l = 0; l < nlev; ++l)
    s->tc_level[l] = tc_levels[l] == FWD_TC ? (s->levels[l].wmax >= TC_GEMM_MIN_W ? FWD_TC : FWD_SIMT) : tc_levels[l];
  RET(upload_tc_super(s));
  s->tuned = true;
  return ICR_OK;
}

int icr_forward_levels(icr_scene* s, int32_t* n_levels) {
  RET(check_scene(s));
  if (!s->has_system || !n_levels) {
    set_error("forward_levels: needs a system and an output");
    return s->has_system ? ICR_EINVAL : ICR_ESTATE;
  }
  *n_levels = (int32_t)s->levels.size();
  return ICR_OK;
}

int icr_autotune(icr_scene* s, int32_t* tc_levels, double* level_ms, int32_t max_levels) {
  RET(check_scene(s));
  RET(need_mapping(s, "autotune"));
  RET(set_device(s));
  if (max_levels < 0 || (max_levels > 0 && !level_ms)) {
    set_error("autotune: level_ms needs room for 3 x max_levels doubles");
    return ICR_EINVAL;
  }
  const int mode = s->params.contraction;
  const bool tc_ok = s->prec == ICR_FP32 && mode != ICR_CONTRACT_SIMT;
  if (s->m > 0) RET(autotune(s, level_ms, max_levels));
  s->tuned = true;
  if (tc_levels) {
    int n = 0;
    for (uint8_t f : s->tc_level) n += tc_ok && f == FWD_TC ? 1 : 0;
    *tc_levels = n;
  }
  return ICR_OK;
}

}  // extern "C"

int icr::step_enqueue(Scene* s, int n_newton) {
  if (!s->has_mapping || !s->has_system) {
    set_error("step: needs icr_set_system and icr_set_mapping");
    return ICR_ESTATE;
  }
  if (s->obst_kind == 0) {
    set_error("step: needs an obstacle (icr_set_obstacle_plane / icr_set_obstacle_sphere)");
    return ICR_ESTATE;
  }
  if (n_newton < 0 || (s->obst_kind == 1 && n_newton > s->obst_iters)) {
    set_error("step: %d Newton iterations not available for this obstacle", n_newton);
    return ICR_EINVAL;
  }
  if (s->m) {
    RET(dcopy(s, s->p.p, s->p0.p, 3 * (size_t)s->m * sizeof(double), "copy p0"));
    RET(dzero(s, s->u.p, 6 * (size_t)s->m * sizeof(double), "memset u"));
  }
  RET(launch_build_WH(s));
  s->has_WH = true;
  const size_t lam_bytes = 3 * (size_t)s->m * s->tsize;
  // newton_tol: from iteration 2 on, the kernels of an iteration return at
  // entry once the FP64 check after the previous linearisation ended the loop
  const bool nstop = s->params.newton_tol > 0 && n_newton > 1 && s->m;
  if (nstop) RET(dzero(s, s->newton.p, 2 * sizeof(int32_t), "memset newton"));
  struct StopGuard {
    Scene* s;
    ~StopGuard() { s->step_stop = nullptr; }
  } guard{s};
  s->last_newton = n_newton;
  s->last_newton_tol = nstop;
  for (int k = 0; k < n_newton; ++k) {
    if (k == 1 && nstop) s->step_stop = (const int*)s->newton.p;
    RET(launch_linearize(s, k));
    if (k >= 1 && nstop) RET(launch_newton_check(s));
    RET(launch_update_W(s));
    if (k == 0 && s->params.warm_start && s->m) {
      // Newton iteration 1 starts from the previous time step's iteration-1 solution
      RET(dcopy(s, s->lam.p, s->lam0.p, lam_bytes, "copy lam0"));
      RET(launch_pgs(s, 1, 0));
      RET(dcopy(s, s->lam0.p, s->lam.p, lam_bytes, "copy lam"));
    } else {
      RET(launch_pgs(s, 0, 0));
    }
    RET(launch_update_proximity(s));
  }
  s->step_stop = nullptr;
  RET(launch_correct_motion(s));
  if (s->m) RET(dzero(s, s->u.p, 3 * (size_t)s->m * sizeof(double), "memset u"));
  s->has_dirs = s->has_W = s->has_lam = true;
  return ICR_OK;
}

extern "C" {

static int field_size(Scene* s, int32_t f, size_t* count, size_t* elem) {
  const size_t m = s->m;
  *elem = sizeof(double);
  switch (f) {
    case ICR_FIELD_WH:
    case ICR_FIELD_W: *count = 9 * m * m; break;
    case ICR_FIELD_LAMBDA:
    case ICR_FIELD_LAMBDA0:
    case ICR_FIELD_DELTA:
    case ICR_FIELD_P:
    case ICR_FIELD_U: *count = 3 * m; break;
    case ICR_FIELD_C: *count = 9 * m; break;
    case ICR_FIELD_MU: *count = m; break;
    case ICR_FIELD_DQ: *count = s->n; break;
    case ICR_FIELD_REACH_PTR:
      *count = s->ns + 1;
      *elem = sizeof(int32_t);
      break;
    case ICR_FIELD_REACH_IDX: {
      *elem = sizeof(int32_t);
      std::vector<int32_t> qc(s->ns);
      cudaMemcpyAsync(qc.data(), s->qcount.p, s->ns * sizeof(int32_t), cudaMemcpyDeviceToHost, s->ctx->stream);
      cudaError_t e = cudaStreamSynchronize(s->ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "field_size");
      size_t tot = 0;
      for (int v : qc) tot += v;
      *count = tot;
      break;
    }
    default: set_error("unknown field %d", f); return ICR_EINVAL;
  }
  return ICR_OK;
}

int icr_step(icr_scene* s, int32_t n_newton) {
  RET(check_scene(s));
  RET(set_device(s));
  return step_enqueue(s, n_newton);
}

// Capture step_enqueue into the scene's graph; with `warm_up` one plain step
// runs first so that every kernel is set up (per-device attributes) before
// capture.  A readmitted scene has run its kernels before and is captured
// without it, which leaves its warm start untouched.
static int capture_step(Scene* s, int32_t n_newton, bool warm_up) {
  cudaStream_t st = s->ctx->stream;
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) {
    set_error("step_capture: the context needs its own CUDA stream to capture a graph");
    return ICR_EINVAL;
  }
  if (warm_up) {
    RET(step_enqueue(s, n_newton));
    CK(cudaStreamSynchronize(st));
  }
  if (s->step_graph) {
    cudaGraphExecDestroy(s->step_graph);
    s->step_graph = nullptr;
  }
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const uint64_t before = s->launches;
  const int rc = step_enqueue(s, n_newton);
  s->graph_kernels = s->launches - before;   // recorded into the graph, not launched
  s->launches = before;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != ICR_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  s->graph_epoch = s->alloc_epoch;
  s->graph_m = s->m;
  s->graph_obst = s->obst_kind;
  s->graph_newton = n_newton;
  s->graph_params = s->params;
  const cudaError_t e2 = cudaGraphInstantiate(&s->step_graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    s->step_graph = nullptr;
    return cuda_fail(e2, "cudaGraphInstantiate");
  }
  return ICR_OK;
}

int icr_step_capture(icr_scene* s, int32_t n_newton) {
  RET(check_scene(s));
  RET(set_device(s));
  if (!s->tuned) RET(icr_autotune(s, nullptr, nullptr, 0));
  return capture_step(s, n_newton, true);
}

}  // extern "C"

// ---------------------------------------------------------------- eviction
namespace icr {
void scene_buffers(Scene* s, std::vector<std::pair<DBuf*, bool>>& out) {
  DBuf* keep[] = {&s->super_ptr, &s->rowpat_ptr, &s->rowpat, &s->val_ptr, &s->G, &s->dinv, &s->dinvsqrt,
                  &s->parent, &s->child_ptr, &s->child_list, &s->relidx, &s->level_list, &s->node_super,
                  &s->dof_super, &s->fr_ptr, &s->ctr_ptr, &s->ctr_child, &s->ctr_row, &s->nodes, &s->bary,
                  &s->C, &s->delta, &s->mu, &s->lam, &s->lam0, &s->p, &s->p0, &s->u, &s->dq, &s->tc_boff,
                  &s->obst_normals, &s->obst_anchors, &s->obst_spheres, &s->obst_of, &s->Gpk, &s->gpk_off,
                  &s->tc_super, &s->level_first, &s->newton};
  DBuf* scratch[] = {&s->bitmap, &s->wprefix, &s->qcount, &s->qidx, &s->qpos, &s->qinv, &s->X, &s->Ftop,
                     &s->WH, &s->W, &s->uk, &s->y, &s->plan, &s->Ypk, &s->wblk, &s->stats, &s->dev_err,
                     &s->WH16, &s->pgsb};
  out.clear();
  for (DBuf* b : keep) out.push_back({b, true});
  for (DBuf* b : scratch) out.push_back({b, false});
}

int scene_evict(Scene* s) {
  if (s->evicted) return ICR_OK;
  CK(cudaSetDevice(s->ctx->device));
  RET(check_device_error(s));   // synchronises; a pending device error is reported, not dropped
  std::vector<std::pair<DBuf*, bool>> all;
  scene_buffers(s, all);
  std::vector<Scene::Saved> saved;
  auto undo = [&]() {
    for (auto& sv : saved) cudaFreeHost(sv.host);
  };
  for (auto& b : all) {
    if (!b.second || !b.first->p) continue;
    void* h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, b.first->bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      undo();
      return cuda_fail(e, "scene_evict: cudaHostAlloc");
    }
    saved.push_back({b.first, h, b.first->bytes});
    e = cudaMemcpyAsync(h, b.first->p, b.first->bytes, cudaMemcpyDeviceToHost, s->ctx->stream);
    if (e != cudaSuccess) {
      undo();
      return cuda_fail(e, "scene_evict: copy to host");
    }
  }
  cudaError_t e = cudaStreamSynchronize(s->ctx->stream);
  if (e != cudaSuccess) {
    undo();
    return cuda_fail(e, "scene_evict: synchronize");
  }
  // the scene gives up every device byte: buffers, the input staging buffer, its graph
  s->evicted_sizes.clear();
  uint64_t bytes = 0;
  for (auto& b : all) {
    s->evicted_sizes.push_back({b.first, b.first->bytes});
    bytes += b.first->bytes;
    dfree(s, *b.first);
  }
  if (s->stage_dev.p) {
    for (int k = 0; k < 2; ++k)
      if (s->stage_used[k]) cudaEventSynchronize(s->stage_ev[k]);
    cudaFree(s->stage_dev.p);
    s->ctx->in_use -= s->stage_dev.bytes;
    s->stage_dev.p = nullptr;
    s->stage_dev.bytes = 0;
    for (int k = 0; k < 2; ++k) {
      if (s->stage_host[k]) cudaFreeHost(s->stage_host[k]);
      s->stage_host[k] = nullptr;
      s->stage_used[k] = false;
    }
    s->stage_bytes = 0;
  }
  s->recapture = s->step_graph != nullptr;
  if (s->step_graph) {
    cudaGraphExecDestroy(s->step_graph);
    s->step_graph = nullptr;
  }
  s->saved = std::move(saved);
  s->resident_bytes = bytes;
  s->evicted = true;
  return ICR_OK;
}

int scene_readmit(Scene* s) {
  if (!s->evicted) return ICR_OK;
  CK(cudaSetDevice(s->ctx->device));
  Ctx* c = s->ctx;
  if (c->budget && c->in_use + s->resident_bytes > c->budget) {
    set_error("readmit: %llu bytes exceed the context HBM budget (%llu of %llu in use)",
              (unsigned long long)s->resident_bytes, (unsigned long long)c->in_use, (unsigned long long)c->budget);
    return ICR_ENOMEM;
  }
  for (auto& b : s->evicted_sizes) {
    if (b.second == 0) continue;
    const int rc = dalloc(s, *b.first, b.second);
    if (rc != ICR_OK) {   // back to the evicted state: nothing is kept on the device
      for (auto& f : s->evicted_sizes) dfree(s, *f.first);
      return rc;
    }
  }
  cudaStream_t st = s->ctx->stream;
  for (auto& sv : s->saved) CK(cudaMemcpyAsync(sv.b->p, sv.host, sv.bytes, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(s->dev_err.p, 0, s->dev_err.bytes, st));
  // W's padding columns must read zero (icr_update_W writes the 3m x 3m part only)
  CK(cudaMemsetAsync(s->W.p, 0, s->W.bytes, st));
  s->W_zeroed = s->W.gen;
  s->W_zeroed_ld = s->ldw;
  s->W_zeroed_rows = 3 * (int64_t)std::max(1, s->m);
  CK(cudaStreamSynchronize(st));
  for (auto& sv : s->saved) cudaFreeHost(sv.host);
  s->saved.clear();
  s->evicted = false;
  s->has_WH = s->has_W = false;   // rebuilt by the next step
  if (s->recapture) {
    s->recapture = false;
    RET(capture_step(s, s->graph_newton, false));
  }
  return ICR_OK;
}
}  // namespace icr

extern "C" {

int icr_scene_evict(icr_scene* s) {
  if (!s) {
    set_error("scene is NULL");
    return ICR_EINVAL;
  }
  return scene_evict(s);
}

int icr_scene_readmit(icr_scene* s) {
  if (!s) {
    set_error("scene is NULL");
    return ICR_EINVAL;
  }
  return scene_readmit(s);
}

int icr_scene_residency(icr_scene* s, int32_t* resident, uint64_t* device_bytes) {
  if (!s || !resident || !device_bytes) {
    set_error("scene_residency: NULL argument");
    return ICR_EINVAL;
  }
  *resident = s->evicted ? 0 : 1;
  if (s->evicted) {
    *device_bytes = s->resident_bytes;
  } else {
    std::vector<std::pair<DBuf*, bool>> all;
    scene_buffers(s, all);
    uint64_t b = s->stage_dev.bytes;
    for (auto& x : all) b += x.first->bytes;
    *device_bytes = b;
  }
  return ICR_OK;
}

int icr_step_launch(icr_scene* s) {
  RET(check_scene(s));
  RET(check_step_graph(s, "step_launch"));
  RET(set_device(s));
  CK(cudaGraphLaunch(s->step_graph, s->ctx->stream));
  s->launches += s->graph_kernels;
  s->last_newton = s->graph_newton;
  s->last_newton_tol = s->graph_params.newton_tol > 0 && s->graph_newton > 1 && s->graph_m > 0;
  return ICR_OK;
}

int icr_newton_iterations(icr_scene* s, int32_t* out) {
  RET(check_scene(s));
  if (!out) {
    set_error("newton_iterations: out is NULL");
    return ICR_EINVAL;
  }
  if (!s->last_newton_tol) {
    *out = s->last_newton;
    return ICR_OK;
  }
  RET(set_device(s));
  int32_t nw[2] = {0, 0};
  CK(cudaMemcpyAsync(nw, s->newton.p, sizeof(nw), cudaMemcpyDeviceToHost, s->ctx->stream));
  CK(cudaStreamSynchronize(s->ctx->stream));
  *out = 1 + nw[1];
  return ICR_OK;
}

int icr_sync(icr_scene* s) {
  RET(check_scene(s));
  RET(set_device(s));
  CK(cudaStreamSynchronize(s->ctx->stream));
  return check_device_error(s);
}

int icr_field_bytes(icr_scene* s, int32_t field, size_t* out) {
  RET(check_scene(s));
  RET(need_mapping(s, "field_bytes"));
  if (!out) {
    set_error("out is NULL");
    return ICR_EINVAL;
  }
  size_t c, e;
  RET(field_size(s, field, &c, &e));
  *out = c * e;
  return ICR_OK;
}

int icr_get(icr_scene* s, int32_t field, void* dst, size_t bytes) {
  RET(check_scene(s));
  RET(need_mapping(s, "get"));
  RET(set_device(s));
  RET(check_device_error(s));
  size_t c, e;
  RET(field_size(s, field, &c, &e));
  if (bytes != c * e || (c && !dst)) {
    set_error("get: field %d needs %zu bytes, got %zu", field, c * e, bytes);
    return ICR_EINVAL;
  }
  if (c == 0) return ICR_OK;
  cudaStream_t st = s->ctx->stream;
  switch (field) {
    case ICR_FIELD_WH: return download_T(s, s->WH, (double*)dst, c);
    case ICR_FIELD_W: return download_T_2d(s, s->W, s->ldw, (double*)dst, 3 * (size_t)s->m, 3 * (size_t)s->m);
    case ICR_FIELD_LAMBDA: return download_T(s, s->lam, (double*)dst, c);
    case ICR_FIELD_LAMBDA0: return download_T(s, s->lam0, (double*)dst, c);
    case ICR_FIELD_DELTA: return download_T(s, s->delta, (double*)dst, c);
    case ICR_FIELD_C: return download_T(s, s->C, (double*)dst, c);
    case ICR_FIELD_MU: return download_T(s, s->mu, (double*)dst, c);
    case ICR_FIELD_DQ: return download_T(s, s->dq, (double*)dst, c);
    case ICR_FIELD_P:
      CK(cudaMemcpyAsync(dst, s->p.p, bytes, cudaMemcpyDeviceToHost, st));
      break;
    case ICR_FIELD_U:
      CK(cudaMemcpyAsync(dst, s->u.p, bytes, cudaMemcpyDeviceToHost, st));
      break;
    case ICR_FIELD_REACH_PTR:
    case ICR_FIELD_REACH_IDX: {
      std::vector<int32_t> qc(s->ns), qi((size_t)s->ns * std::max(1, s->m));
      CK(cudaMemcpyAsync(qc.data(), s->qcount.p, s->ns * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(qi.data(), s->qidx.p, qi.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      int32_t* out = (int32_t*)dst;
      if (field == ICR_FIELD_REACH_PTR) {
        out[0] = 0;
        for (int k = 0; k < s->ns; ++k) out[k + 1] = out[k] + qc[k];
      } else {
        size_t o = 0;
        for (int k = 0; k < s->ns; ++k)
          for (int j = 0; j < qc[k]; ++j) out[o++] = qi[(size_t)k * s->m + j];
      }
      return ICR_OK;
    }
  }
  CK(cudaStreamSynchronize(st));
  return ICR_OK;
}

int icr_set_field(icr_scene* s, int32_t field, const double* src, size_t bytes) {
  RET(check_scene(s));
  RET(need_mapping(s, "set_field"));
  RET(set_device(s));
  size_t c, e;
  RET(field_size(s, field, &c, &e));
  if (bytes != c * e || (c && !src) || e != sizeof(double)) {
    set_error("set_field: field %d needs %zu bytes of doubles, got %zu", field, c * e, bytes);
    return ICR_EINVAL;
  }
  for (size_t i = 0; i < c; ++i)
    if (!std::isfinite(src[i])) {
      set_error("set_field: value %zu is not finite", i);
      return ICR_EINVAL;
    }
  switch (field) {
    case ICR_FIELD_W:
      RET(upload_T_2d(s, s->W, s->ldw, src, 3 * (size_t)s->m, 3 * (size_t)s->m));
      RET(launch_wcoup(s));
      s->has_W = true;
      break;
    case ICR_FIELD_WH: RET(upload_T(s, s->WH, src, c)); s->has_WH = true; break;
    case ICR_FIELD_LAMBDA: RET(upload_T(s, s->lam, src, c)); s->has_lam = true; break;
    case ICR_FIELD_LAMBDA0: RET(upload_T(s, s->lam0, src, c)); break;
    case ICR_FIELD_DELTA: RET(upload_T(s, s->delta, src, c)); break;
    case ICR_FIELD_C:
      RET(check_directions(src, s->m));
      RET(upload_T(s, s->C, src, c));
      s->has_dirs = true;
      break;
    case ICR_FIELD_MU: RET(upload_T(s, s->mu, src, c)); break;
    case ICR_FIELD_P: RET(upload(s, s->p, src, c)); break;
    case ICR_FIELD_U: RET(upload(s, s->u, src, c)); break;
    default: set_error("set_field: field %d cannot be set", field); return ICR_EINVAL;
  }
  return ICR_OK;
}

}  // extern "C"
