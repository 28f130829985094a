// The C ABI of libxc (include/xc.h): argument validation, plan lifetime, the
// host-buffer path and statistics.  No C++ exception crosses this boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "xc_internal.h"

namespace xc {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return XC_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(XC_ERR_ALLOC, std::string(what) + ": " + cudaGetErrorString(e));
  }
  return fail(XC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int plan_alloc(Plan* p, void** ptr, size_t bytes) {
  void* d = nullptr;
  const cudaError_t e = cudaMalloc(&d, bytes == 0 ? 1 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(XC_ERR_ALLOC, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  p->allocations.push_back(d);
  *ptr = d;
  return XC_OK;
}

static std::atomic<int64_t> g_launches{0};

const char* kernel_name(int id) {
  static const char* names[K_COUNT] = {"fwd_fft",       "fwd_sparse", "adj_sparse", "adj_fft",  "adj_tail",
                                       "fwd_reduce",    "adj_transpose", "pair_scale", "row_scale",
                                       "fft_in_2d",     "sparse_2d",  "fft_out_2d", "combine_2d"};
  return (id >= 0 && id < K_COUNT) ? names[id] : "unknown";
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t take_event(Plan* p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void launch_begin(Plan* p, int kernel, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!p->timing) return;
  Plan::Pending pd{kernel, take_event(p), take_event(p)};
  if (pd.start) cudaEventRecord(pd.start, s);
  p->pending.push_back(pd);
}

void launch_end(Plan* p, int kernel, cudaStream_t s) {
  (void)kernel;
  if (!p->timing || p->pending.empty()) return;
  if (p->pending.back().stop) cudaEventRecord(p->pending.back().stop, s);
}

static void release_events(Plan* p) {
  for (auto& pd : p->pending) {
    if (pd.start) cudaEventDestroy(pd.start);
    if (pd.stop) cudaEventDestroy(pd.stop);
  }
  p->pending.clear();
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  p->event_pool.clear();
}

int ensure_scratch_kept(Plan* p, int64_t nrhs) {
  if (nrhs <= p->scratch_nrhs || p->batch_refs == 0 || !p->scratch) return ensure_scratch(p, nrhs);
  void* old = p->scratch;
  p->scratch = nullptr;        // ensure_scratch then allocates without freeing
  const int rc = ensure_scratch(p, nrhs);
  if (p->scratch) p->retired.push_back(old);
  else p->scratch = old;       // the growth failed: the old buffer stays in use
  return rc;
}

static void free_plan(Plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  release_events(p);
  for (void* d : p->allocations) cudaFree(d);
  for (void* d : p->retired) cudaFree(d);
  delete p->d2;
  if (p->scratch) cudaFree(p->scratch);
  if (p->stage) cudaFree(p->stage);
  delete p;
}

static int validate_vectors(const Plan* p, const void* a, const void* b, int64_t nrhs, int64_t ld) {
  if (!p) return fail(XC_ERR_ARG, "plan is NULL");
  if (nrhs < 0) return fail(XC_ERR_ARG, "nrhs < 0");
  if (nrhs == 0) return XC_OK;
  if (!a || !b) return fail(XC_ERR_ARG, "vector pointer is NULL");
  if (ld < p->N) return fail(XC_ERR_ARG, "ld < N");
  if (nrhs > 65535LL * 8) return fail(XC_ERR_UNSUPPORTED, "nrhs above 524280");
  if (ld > (int64_t(1) << 40) / nrhs) return fail(XC_ERR_ARG, "nrhs * ld too large");
  // the [nrhs][ld] arrays, up to the last used element, must not overlap
  const uintptr_t span = uintptr_t((nrhs - 1) * ld + p->N) * p->io_bytes();
  const uintptr_t ua = reinterpret_cast<uintptr_t>(a), ub = reinterpret_cast<uintptr_t>(b);
  if (ua < ub + span && ub < ua + span) return fail(XC_ERR_ARG, "input and output must not overlap");
  return XC_OK;
}

}  // namespace xc

using xc::fail;

extern "C" {

void xc_params_default(xc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nodes = XC_NODES_GAUSS;
  p->normalise = XC_RAW;
  p->precision = XC_FP64;
  p->scheme = XC_SCHEME_AUTO;
}

int xc_plan_create(xc_plan_t* out, int family, const xc_params* params, int64_t N, double eps) {
  if (!out) return fail(XC_ERR_ARG, "out is NULL");
  *out = nullptr;
  xc_params prm;
  if (params) prm = *params;
  else xc_params_default(&prm);
  if (family < XC_CHEBYSHEV_T || family > XC_KERNEL_A2) return fail(XC_ERR_ARG, "unknown family");
  const bool index_kernel = family == XC_KERNEL_A1 || family == XC_KERNEL_A2;
  if (index_kernel && prm.scheme == XC_SCHEME_AUTO) prm.scheme = XC_SCHEME_2D;
  const bool two_d = prm.scheme == XC_SCHEME_2D;
  const bool cplx = family == XC_EXP || family == XC_LAGUERRE_SPECTRAL;
  const bool trig = family == XC_CHEBYSHEV_T || family == XC_SINE || family == XC_COS_POWER || cplx;
  if (N < 2 || N > (int64_t(1) << 20)) return fail(XC_ERR_ARG, "N must lie in [2, 2^20]");
  if (!(eps >= 0.0) || !(eps < 1.0)) return fail(XC_ERR_ARG, "eps must lie in [0, 1)");
  if (prm.precision < XC_FP64 || prm.precision > XC_FP64_PAIR) return fail(XC_ERR_ARG, "unknown precision");
  if (prm.nodes != XC_NODES_GAUSS && prm.nodes != XC_NODES_USER) return fail(XC_ERR_ARG, "unknown node set");
  if (prm.nodes == XC_NODES_USER && !prm.user_nodes) return fail(XC_ERR_ARG, "user_nodes is NULL");
  if (prm.normalise != XC_RAW && prm.normalise != XC_ORTHONORMAL) return fail(XC_ERR_ARG, "unknown normalisation");
  if (prm.normalise == XC_ORTHONORMAL && prm.nodes == XC_NODES_USER)
    return fail(XC_ERR_ARG, "the orthonormal variant needs Gauss nodes");
  if (family == XC_JACOBI && !(prm.alpha > -1.0 && prm.beta > -1.0)) return fail(XC_ERR_ARG, "Jacobi needs alpha, beta > -1");
  if (prm.scheme < XC_SCHEME_AUTO || prm.scheme > XC_SCHEME_2D) return fail(XC_ERR_ARG, "unknown scheme");
  double x0 = 0.0, h = 1.0;
  if (two_d) {
    if (!(index_kernel || family == XC_LAGUERRE_FN || family == XC_HERMITE_FN))
      return fail(XC_ERR_UNSUPPORTED, "the 2-D scheme takes Laguerre / Hermite functions or the index kernels");
    if (prm.precision != XC_FP64 && prm.precision != XC_FP32)
      return fail(XC_ERR_UNSUPPORTED, "the 2-D scheme runs in XC_FP64 or XC_FP32");
    if (prm.normalise != XC_RAW) return fail(XC_ERR_UNSUPPORTED, "the 2-D scheme takes the raw matrix");
    if (!index_kernel) {
      // equispaced nodes x_i = x0 + i h, h > 0: the rows extend with the same step
      if (prm.nodes != XC_NODES_USER || !prm.user_nodes)
        return fail(XC_ERR_ARG, "the 2-D scheme needs equispaced user nodes");
      x0 = prm.user_nodes[0];
      h = (prm.user_nodes[N - 1] - x0) / double(N - 1);
      if (!(h > 0.0)) return fail(XC_ERR_ARG, "the 2-D scheme needs increasing equispaced nodes");
      for (int64_t i = 0; i < N; ++i) {
        const double want = x0 + h * double(i);
        if (std::fabs(prm.user_nodes[i] - want) > 1e-12 * std::fmax(std::fabs(want), h * double(N)))
          return fail(XC_ERR_ARG, "the 2-D scheme needs equispaced user nodes");
      }
    }
  } else if (index_kernel) {
    return fail(XC_ERR_ARG, "the index kernels take XC_SCHEME_2D");
  }
  if (prm.scheme == XC_SCHEME_TWO_SIDED && !trig)
    return fail(XC_ERR_ARG, "the two-sided extension needs a trigonometric family");
  if (prm.normalise == XC_ORTHONORMAL && (family == XC_SINE || family == XC_COS_POWER))
    return fail(XC_ERR_UNSUPPORTED, "the orthonormal variant is defined for the polynomial families");
  if (prm.power < 0 || prm.power > 16) return fail(XC_ERR_ARG, "power must lie in [0, 16]");
  if (prm.eps2 < 0.0 || prm.eps2 >= 1.0 || prm.eps_window < 0.0 || prm.eps_window >= 1.0 || prm.tail_max < 0)
    return fail(XC_ERR_ARG, "eps2 / eps_window / tail_max out of range");
  if (prm.precompute != XC_PRECOMPUTE_AUTO && prm.precompute != XC_PRECOMPUTE_FFT)
    return fail(XC_ERR_ARG, "unknown precompute mode");
  if (family == XC_LAGUERRE_SPECTRAL && !(prm.alpha > 0.0 && prm.beta > 0.0))
    return fail(XC_ERR_ARG, "the spectral Laguerre matrix needs eta = alpha > 0 and T = beta > 0");
  if (family == XC_LAGUERRE_SPECTRAL && prm.nodes == XC_NODES_USER)
    return fail(XC_ERR_ARG, "the spectral Laguerre matrix has its own angles (no user nodes)");
  if (cplx && prm.precision != XC_FP64 && prm.precision != XC_FP32)
    return fail(XC_ERR_UNSUPPORTED, "complex families run in XC_FP64 or XC_FP32");
  if (cplx && prm.scheme == XC_SCHEME_BLOCKS)
    return fail(XC_ERR_UNSUPPORTED, "complex families take the two-sided extension");
  if (cplx && prm.normalise == XC_ORTHONORMAL)
    return fail(XC_ERR_UNSUPPORTED, "the orthonormal variant is defined for the polynomial families");

  xc::Plan* p = new (std::nothrow) xc::Plan();
  if (!p) return fail(XC_ERR_ALLOC, "host allocation failed");
  p->N = N;
  p->family = family;
  p->params = prm;
  p->params.user_nodes = nullptr;
  // only the Jacobi family (alpha, beta) and the spectral Laguerre matrix (eta, T) have parameters
  if (family != XC_JACOBI && family != XC_LAGUERRE_SPECTRAL) p->params.alpha = p->params.beta = 0.0;
  p->cplx = cplx;
  p->x0 = x0;
  p->h = h;
  p->precision = prm.precision;
  p->normalise = prm.normalise;
  p->scheme = prm.scheme == XC_SCHEME_AUTO ? (trig ? XC_SCHEME_TWO_SIDED : XC_SCHEME_BLOCKS) : prm.scheme;
  if (family == XC_COS_POWER && p->params.power == 0) p->params.power = 2;
  p->eps = eps;
  p->eps2 = prm.eps2 > 0 ? prm.eps2 : (p->io64() ? 1e-3 : 1e-1);
  if (prm.nodes == XC_NODES_USER) p->nodes_host.assign(prm.user_nodes, prm.user_nodes + N);
  int rc = XC_OK;
  if (two_d) {
    // zeta as for any block; the 2-D decomposition is made on the device side
    const double ew = eps > 0 ? eps : (prm.eps_window > 0 ? prm.eps_window : 1e-14);
    p->sch.eps_window = ew;
    p->sch.zeta = xc::zeta_of_eps_host(ew);
  } else {
    rc = xc::make_schedule(N, eps, p->eps2, p->scheme == XC_SCHEME_TWO_SIDED, prm.eps_window,
                           prm.tail_max > 0 ? prm.tail_max : 20, &p->sch);
  }
  if (rc == XC_OK) {
    p->zeta = p->sch.zeta;
    rc = xc::build_plan_device(p);
  }
  if (rc == XC_OK) rc = xc::ensure_scratch(p, 1);
  if (rc != XC_OK) {
    const std::string msg = xc_last_error_message();
    xc::free_plan(p);
    return fail(rc, msg);
  }
  *out = reinterpret_cast<xc_plan_t>(p);
  return XC_OK;
}

int xc_plan_destroy(xc_plan_t plan) {
  xc::free_plan(reinterpret_cast<xc::Plan*>(plan));
  return XC_OK;
}

int xc_plan_reserve(xc_plan_t plan, int64_t nrhs) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p) return fail(XC_ERR_ARG, "plan is NULL");
  if (nrhs < 0) return fail(XC_ERR_ARG, "nrhs < 0");
  return xc::ensure_scratch_kept(p, nrhs);
}

int xc_apply(xc_plan_t plan, const void* x_dev, void* y_dev, int64_t nrhs, int64_t ld, void* stream) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  XC_TRY(xc::validate_vectors(p, x_dev, y_dev, nrhs, ld));
  if (nrhs == 0) return XC_OK;
  XC_TRY(xc::ensure_scratch_kept(p, nrhs));
  p->last_stream = static_cast<cudaStream_t>(stream);
  return xc::launch_apply(p, x_dev, y_dev, nrhs, ld, static_cast<cudaStream_t>(stream));
}

int xc_apply_adjoint(xc_plan_t plan, const void* y_dev, void* x_dev, int64_t nrhs, int64_t ld, void* stream) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  XC_TRY(xc::validate_vectors(p, y_dev, x_dev, nrhs, ld));
  if (nrhs == 0) return XC_OK;
  XC_TRY(xc::ensure_scratch_kept(p, nrhs));
  p->last_stream = static_cast<cudaStream_t>(stream);
  return xc::launch_apply_adjoint(p, y_dev, x_dev, nrhs, ld, static_cast<cudaStream_t>(stream));
}

int xc_apply_noalloc(xc_plan_t plan, const void* x_dev, void* y_dev, int64_t nrhs, int64_t ld, void* stream) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  XC_TRY(xc::validate_vectors(p, x_dev, y_dev, nrhs, ld));
  if (nrhs == 0) return XC_OK;
  if (p->cplx || p->d2) return fail(XC_ERR_UNSUPPORTED, "xc_apply_noalloc takes 1-D real plans only");
  p->last_stream = static_cast<cudaStream_t>(stream);
  return xc::launch_apply_noalloc(p, x_dev, y_dev, nrhs, ld, static_cast<cudaStream_t>(stream));
}

int xc_apply_host(xc_plan_t plan, int adjoint, const void* in_host, void* out_host, int64_t nrhs, int64_t ld,
                  void* stream) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  XC_TRY(xc::validate_vectors(p, in_host, out_host, nrhs, ld));
  if (nrhs == 0) return XC_OK;
  const int64_t elems = nrhs * ld;
  if (elems > p->stage_elems) {
    if (p->stage) {
      cudaDeviceSynchronize();
      cudaFree(p->stage);
      p->stage = nullptr;
      p->stage_elems = 0;
    }
    void* d = nullptr;
    if (cudaMalloc(&d, size_t(2 * elems) * p->io_bytes()) != cudaSuccess) {
      cudaGetLastError();
      return fail(XC_ERR_ALLOC, "staging allocation failed");
    }
    p->stage = d;
    p->stage_elems = elems;
  }
  XC_TRY(xc::ensure_scratch_kept(p, nrhs));
  auto st = static_cast<cudaStream_t>(stream);
  p->last_stream = st;
  char* din = static_cast<char*>(p->stage);
  char* dout = din + size_t(p->stage_elems) * p->io_bytes();
  // Only the N used elements of each row move: the caller's padding columns
  // [N, ld) of out_host are left as they are (as xc_apply leaves them).
  const size_t eb = p->io_bytes();
  if (ld == p->N) {
    const size_t bytes = size_t(elems) * eb;
    XC_CUDA(cudaMemcpyAsync(din, in_host, bytes, cudaMemcpyHostToDevice, st));
  } else {
    XC_CUDA(cudaMemcpy2DAsync(din, size_t(ld) * eb, in_host, size_t(ld) * eb, size_t(p->N) * eb, size_t(nrhs),
                              cudaMemcpyHostToDevice, st));
  }
  if (adjoint) XC_TRY(xc::launch_apply_adjoint(p, din, dout, nrhs, ld, st));
  else XC_TRY(xc::launch_apply(p, din, dout, nrhs, ld, st));
  if (ld == p->N) {
    XC_CUDA(cudaMemcpyAsync(out_host, dout, size_t(elems) * eb, cudaMemcpyDeviceToHost, st));
  } else {
    XC_CUDA(cudaMemcpy2DAsync(out_host, size_t(ld) * eb, dout, size_t(ld) * eb, size_t(p->N) * eb, size_t(nrhs),
                              cudaMemcpyDeviceToHost, st));
  }
  XC_CUDA(cudaStreamSynchronize(st));
  return XC_OK;
}

int xc_plan_info(xc_plan_t plan, xc_plan_stats* out) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p || !out) return fail(XC_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->N = p->N;
  out->family = p->family;
  out->precision = p->precision;
  out->scheme = p->scheme;
  out->normalise = p->normalise;
  out->eps = p->eps;
  out->eps2 = p->eps2;
  out->zeta = p->zeta;
  out->nblocks = int(p->blocks.size());
  for (size_t i = 0; i < p->blocks.size(); ++i) {
    out->L[i] = p->blocks[i].L;
    out->off[i] = p->blocks[i].off;
    out->j_lo[i] = p->blocks[i].j_lo;
    out->j_hi[i] = p->blocks[i].j_hi;
    out->nnz[i] = p->nnz[i];
    out->stored[i] = p->stored[i];
    out->maxabs[i] = p->maxabs[i];
  }
  out->m_tail = p->m_tail;
  out->matrix_bytes = p->matrix_bytes;
  out->adjoint_bytes = p->adjoint_bytes;
  out->closed_form_blocks = p->closed_form_blocks;
  if (p->d2) {
    out->nblocks = 0;
    out->blocks2d = p->d2->nb;
    out->dense2d = int(p->d2->rects_host.size());
    out->nnz2d = p->d2->kept;
    out->dense_elems2d = p->d2->dense_elems;
  }
  return XC_OK;
}

int xc_get_nodes(xc_plan_t plan, double* host_out) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p || !host_out) return fail(XC_ERR_ARG, "NULL argument");
  std::copy(p->nodes_host.begin(), p->nodes_host.end(), host_out);
  return XC_OK;
}

int xc_dense_matrix(xc_plan_t plan, void* A_dev, int64_t lda, void* stream) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p || !A_dev) return fail(XC_ERR_ARG, "NULL argument");
  if (lda < p->N) return fail(XC_ERR_ARG, "lda < N");
  return xc::dense_matrix_device(p, A_dev, lda, static_cast<cudaStream_t>(stream));
}

int xc_timing_enable(xc_plan_t plan, int enable) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p) return fail(XC_ERR_ARG, "plan is NULL");
  p->timing = enable != 0;
  if (p->t_ms.empty()) {
    p->t_ms.assign(xc::K_COUNT, 0.0);
    p->t_launches.assign(xc::K_COUNT, 0);
  }
  return XC_OK;
}

int xc_timing_read(xc_plan_t plan, xc_kernel_time* out, int max, int* count) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p || !count || (max > 0 && !out)) return fail(XC_ERR_ARG, "NULL argument");
  if (p->t_ms.empty()) {
    p->t_ms.assign(xc::K_COUNT, 0.0);
    p->t_launches.assign(xc::K_COUNT, 0);
  }
  for (auto& pd : p->pending) {
    float ms = 0.0f;
    if (pd.start && pd.stop) {
      XC_CUDA(cudaEventSynchronize(pd.stop));
      XC_CUDA(cudaEventElapsedTime(&ms, pd.start, pd.stop));
    }
    p->t_ms[pd.kernel] += ms;
    p->t_launches[pd.kernel] += 1;
    if (pd.start) p->event_pool.push_back(pd.start);
    if (pd.stop) p->event_pool.push_back(pd.stop);
  }
  p->pending.clear();
  int n = 0;
  for (int k = 0; k < xc::K_COUNT; ++k) {
    if (p->t_launches[k] == 0) continue;
    if (n < max) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, xc::kernel_name(k), sizeof(out[n].name) - 1);
      out[n].launches = p->t_launches[k];
      out[n].total_ms = p->t_ms[k];
    }
    ++n;
  }
  *count = std::min(n, max);
  p->t_ms.assign(xc::K_COUNT, 0.0);
  p->t_launches.assign(xc::K_COUNT, 0);
  return XC_OK;
}

int64_t xc_launch_count(void) { return xc::g_launches.load(); }

int xc_sync_status(xc_plan_t plan) {
  auto* p = reinterpret_cast<xc::Plan*>(plan);
  if (!p) return fail(XC_ERR_ARG, "plan is NULL");
  XC_CUDA(cudaStreamSynchronize(p->last_stream));
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

const char* xc_strerror(int code) {
  switch (code) {
    case XC_OK: return "ok";
    case XC_ERR_ARG: return "invalid argument";
    case XC_ERR_ALLOC: return "allocation failed";
    case XC_ERR_CUDA: return "CUDA error";
    case XC_ERR_TIMEOUT: return "device wait timed out";
    case XC_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown error";
  }
}

const char* xc_last_error_message(void) { return xc::g_last_error.c_str(); }

}  // extern "C"
