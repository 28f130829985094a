// Many plans in one persistent launch per direction.
//
// A batch groups plans of one precision (uneven N, families and numbers of
// right-hand sides).  Binding I/O buffers builds, per direction, one device
// task list over all plans:
//   forward   phase 1: FFT of (plan, block, RHS)              [fwd_fft_body]
//             phase 2: band product of (plan, 8 row slices, RPW RHS) + tail;
//                      for plans with long bands, of (plan, 8 band chunks,
//                      RPW RHS) into partial sums               [fwd_unit_item]
//             phase 3: (long-band plans) partials + tail of (plan, 256 rows,
//                      32 RHS)                                  [fwd_reduce_row]
//   adjoint   phase 1: transposed band product of (plan, 8 chunks, RPW RHS),
//                      and the dense tail of (plan, RHS)
//             phase 2: inverse FFT of (plan, block, RHS)
// Every CTA of a persistent grid takes tasks from a device counter in list
// order; all phase-1 tasks precede all phase-2 tasks (and those all phase-3
// tasks), and within a phase the costliest tasks come first.  A phase-2 task
// of plan p waits until every phase-1 task of p has finished: phase-1 tasks
// increment done[p] when they end; a phase-2 task reads done[p] with acquire
// semantics and waits, for a bounded number of sleeps, until it reaches
// need[p].  Phase-3 tasks wait in the same way on done[nplans + p], which the
// chunked phase-2 tasks increment.  Because every task of a phase has been
// taken (and so is running) before any task of the next phase starts, the
// waits end; if one does not end within the limit, the status word records a
// timeout, the remaining tasks are skipped and the host reads XC_ERR_TIMEOUT.
// The last CTA to finish resets the counters, so a launch needs no memset and
// can be captured in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "xc_fft.cuh"
#include "xc_internal.h"
#include "xc_items.cuh"

namespace xc {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
enum TaskKind {
  T_FWD_FFT = 0, T_FWD_SPARSE = 1, T_ADJ_SPARSE = 2, T_ADJ_FFT = 3, T_ADJ_TAIL = 4, T_FWD_UNIT = 5, T_FWD_REDUCE = 6
};
constexpr int kReduceRhs = 32;   // right-hand sides per phase-3 task

struct BatchPlanDev {
  const BlockDev* blocks;
  int nblocks;
  int nslices;
  int64_t N, m_tail, total_chunks;
  const void* tail;
  const void* rowscale;
  const void* colscale;
  const int2* t_items;
  const int* t_cbase;
  const int4* fu_units;      // chunked forward (nullptr: direct band product)
  const int* fu_order;
  const int* fu_ubase;
  int64_t total_units;
  int64_t spec_per_rhs;      // the unit partials follow the spectra in scratch
  void* scratch;
  const void* x;
  void* y;
  int64_t nrhs, ld;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait for done >= need.  Returns 1 when satisfied, 0 on timeout or
// when an earlier wait of this launch already failed (status != 0).
__device__ int wait_for(const unsigned* done, unsigned need, long long limit, unsigned* status) {
  for (long long it = 0;; ++it) {
    if (ld_acquire(done) >= need) return 1;
    if (*(volatile unsigned*)status != 0u) return 0;
    if (it >= limit) {
      atomicCAS(status, 0u, 1u);
      return 0;
    }
    __nanosleep(256);
  }
}

template <typename T, int RPW, bool COMP>
__global__ void __launch_bounds__(kBatchThreads)
    batch_kernel(const BatchPlanDev* __restrict__ plans, const int4* __restrict__ tasks, int64_t ntasks,
                 unsigned* ctrl, const unsigned* __restrict__ need, unsigned* done, int nplans, long long wait_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  __shared__ unsigned s_task;
  __shared__ int s_ok;
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* next = &ctrl[0];
  unsigned* finished = &ctrl[1];
  unsigned* status = &ctrl[2];
  for (;;) {
    if (tid == 0) s_task = atomicAdd(next, 1u);
    __syncthreads();
    const int64_t t = s_task;
    if (t >= ntasks) break;
    const int4 tk = tasks[t];
    const BatchPlanDev& P = plans[tk.y];
    const BlockDev* blocks = P.blocks;
    if (tid == 0) {
      if (tk.x == T_FWD_SPARSE || tk.x == T_FWD_UNIT || tk.x == T_ADJ_FFT)
        s_ok = wait_for(&done[tk.y], need[tk.y], wait_limit, status);
      else if (tk.x == T_FWD_REDUCE)
        s_ok = wait_for(&done[nplans + tk.y], need[nplans + tk.y], wait_limit, status);
      else
        s_ok = *(volatile unsigned*)status == 0u;
    }
    __syncthreads();
    if (s_ok) {
      const T* rs = static_cast<const T*>(P.rowscale);
      const T* cs = static_cast<const T*>(P.colscale);
      switch (tk.x) {
        case T_FWD_FFT:
          fwd_fft_body<T>(blocks[tk.z], tk.w, static_cast<const T*>(P.x), P.ld, cs,
                          static_cast<cx<T>*>(P.scratch), P.nrhs, s, tid, kBatchThreads);
          break;
        case T_FWD_SPARSE: {
          const int64_t slice = int64_t(tk.z) + warp;
          if (slice < P.nslices)
            fwd_sparse_item<T, RPW, COMP>(blocks, P.nblocks, P.N, static_cast<const T*>(P.x), P.ld,
                                          static_cast<T*>(P.y), static_cast<const cx<T>*>(P.scratch), P.nrhs, rs, cs,
                                          static_cast<const T*>(P.tail), P.m_tail, slice, int64_t(tk.w) * RPW, lane);
          break;
        }
        case T_FWD_UNIT: {
          const int64_t k = int64_t(tk.z) + warp;
          if (k < P.total_units) {
            const int u = P.fu_order[k];
            fwd_unit_item<T, RPW, COMP>(blocks, static_cast<const cx<T>*>(P.scratch), P.nrhs,
                                        static_cast<cx<T>*>(P.scratch) + P.spec_per_rhs * P.nrhs, P.fu_units[u], u,
                                        int64_t(tk.w) * RPW, lane);
          }
          break;
        }
        case T_FWD_REDUCE: {
          const int64_t n = int64_t(tk.z) * kBatchThreads + tid;
          if (n < P.N) {
            const int64_t r1 = min(P.nrhs, int64_t(tk.w) + kReduceRhs);
            for (int64_t r = tk.w; r < r1; ++r)
              fwd_reduce_row<T, COMP>(P.N, static_cast<const T*>(P.x), P.ld, static_cast<T*>(P.y),
                                      static_cast<const cx<T>*>(P.scratch) + P.spec_per_rhs * P.nrhs, P.nrhs,
                                      P.fu_ubase, rs, cs, static_cast<const T*>(P.tail), P.m_tail, n, r);
          }
          break;
        }
        case T_ADJ_SPARSE: {
          const int64_t item = int64_t(tk.z) + warp;
          if (item < P.total_chunks)
            adj_sparse_item<T, RPW, COMP>(blocks, P.nblocks, static_cast<const T*>(P.y), P.ld, nullptr, 0,
                                          static_cast<cx<T>*>(P.scratch), P.nrhs, rs, P.t_cbase, P.t_items[item],
                                          int64_t(tk.w) * RPW, lane);
          break;
        }
        case T_ADJ_FFT:
          adj_fft_body<T>(blocks[tk.z], tk.w, static_cast<const cx<T>*>(P.scratch), P.t_cbase, P.nrhs,
                          static_cast<T*>(const_cast<void*>(P.x)), P.ld, cs, s, tid, kBatchThreads);
          break;
        default:  // T_ADJ_TAIL
          for (int64_t m = warp; m < P.m_tail; m += kBatchWarps)
            adj_tail_warp<T, COMP>(P.N, m, tk.w, static_cast<const T*>(P.tail), static_cast<const T*>(P.y), P.ld,
                                   static_cast<T*>(const_cast<void*>(P.x)), rs, cs, lane);
          break;
      }
    }
    if (tk.x == T_FWD_FFT || tk.x == T_ADJ_SPARSE || tk.x == T_FWD_UNIT) {
      __syncthreads();                        // every thread's results are written
      if (tid == 0) {
        __threadfence();
        atomicAdd(&done[tk.x == T_FWD_UNIT ? nplans + tk.y : tk.y], 1u);
      }
    }
    __syncthreads();                          // s_task / s_ok are reused
  }
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(finished, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int p = tid; p < 2 * nplans; p += kBatchThreads) done[p] = 0u;
    __syncthreads();
    if (tid == 0) {
      *next = 0u;
      *finished = 0u;
    }
  }
}

}  // namespace

struct Batch {
  std::vector<Plan*> plans;
  int precision = XC_FP64;
  BatchPlanDev* dplans = nullptr;
  int4* tasks[2] = {nullptr, nullptr};
  int64_t ntasks[2] = {0, 0};
  unsigned* need[2] = {nullptr, nullptr};
  unsigned* ctrl = nullptr;      // [0] next task, [1] finished CTAs, [2] status
  unsigned* done = nullptr;      // [2 * nplans]: phase-1, phase-2 completions per plan
  std::vector<int> extra_need;   // fault injection (tests)
  long long wait_limit = 1LL << 22;   // sleeps of ~256 ns: about a second
  int rpw[2] = {0, 0};           // right-hand sides per band item, per direction (0 = not bound)
  bool tuned = false;
  size_t smem = 0;
  int64_t max_n = 0;
  std::vector<const void*> x;
  std::vector<void*> y;
  std::vector<int64_t> nrhs, ld;
  std::vector<void*> allocs;
  ~Batch() {
    cudaDeviceSynchronize();
    for (void* d : allocs) cudaFree(d);
  }
  int alloc(void** ptr, size_t bytes) {
    if (cudaMalloc(ptr, bytes == 0 ? 1 : bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(XC_ERR_ALLOC, "batch allocation failed");
    }
    allocs.push_back(*ptr);
    return XC_OK;
  }
};

namespace {

// Task lists of both directions for the bound right-hand sides, with rpw_f
// (forward) and rpw_a (adjoint) right-hand sides per band item.
int build_tasks(Batch* b, int rpw_f, int rpw_a) {
  const int np = int(b->plans.size());
  std::vector<std::pair<double, int4>> ph1, ph2, ph3;
  std::vector<unsigned> need_f(2 * size_t(np), 0), need_a(2 * size_t(np), 0);
  // forward
  for (int p = 0; p < np; ++p) {
    const Plan* P = b->plans[p];
    const int64_t R = b->nrhs[p];
    if (R == 0) continue;
    for (size_t i = 0; i < P->blocks.size(); ++i) {
      const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
      for (int64_t r = 0; r < R; ++r) {
        ph1.push_back({c, int4{T_FWD_FFT, p, int(i), int(r)}});
        ++need_f[p];
      }
    }
    const int rpw = rpw_f;
    const int64_t groups = (R + rpw - 1) / rpw;
    if (P->fwd_chunked) {
      for (int64_t k0 = 0; k0 < P->total_units; k0 += kBatchWarps) {
        const double c = double(P->unit_len[k0]);   // longest first
        for (int64_t g = 0; g < groups; ++g) {
          ph2.push_back({c * rpw, int4{T_FWD_UNIT, p, int(k0), int(g)}});
          ++need_f[np + p];
        }
      }
      for (int64_t n0 = 0; n0 < P->N; n0 += kBatchThreads)
        for (int64_t r0 = 0; r0 < R; r0 += kReduceRhs)
          ph3.push_back({0.0, int4{T_FWD_REDUCE, p, int(n0 / kBatchThreads), int(r0)}});
      continue;
    }
    for (int64_t s0 = 0; s0 < P->nslices; s0 += kBatchWarps) {
      double c = 0;
      for (int64_t s = s0; s < std::min<int64_t>(P->nslices, s0 + kBatchWarps); ++s)
        c = std::max(c, double(P->slice_cost[s] + P->m_tail));
      for (int64_t g = 0; g < groups; ++g) ph2.push_back({c * rpw, int4{T_FWD_SPARSE, p, int(s0), int(g)}});
    }
  }
  auto order = [](std::vector<std::pair<double, int4>>& v) {
    std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b2) { return a.first > b2.first; });
  };
  order(ph1);
  order(ph2);
  std::vector<int4> fwd;
  for (auto& e : ph1) fwd.push_back(e.second);
  for (auto& e : ph2) fwd.push_back(e.second);
  for (auto& e : ph3) fwd.push_back(e.second);
  // adjoint
  ph1.clear();
  ph2.clear();
  for (int p = 0; p < np; ++p) {
    const Plan* P = b->plans[p];
    const int64_t R = b->nrhs[p];
    if (R == 0) continue;
    const int rpw = rpw_a;
    const int64_t groups = (R + rpw - 1) / rpw;
    for (int64_t i0 = 0; i0 < P->total_chunks; i0 += kBatchWarps) {
      double c = 0;
      for (int64_t i = i0; i < std::min<int64_t>(P->total_chunks, i0 + kBatchWarps); ++i)
        c = std::max(c, double(P->item_len[i]));
      for (int64_t g = 0; g < groups; ++g) {
        ph1.push_back({c * rpw, int4{T_ADJ_SPARSE, p, int(i0), int(g)}});
        ++need_a[p];
      }
    }
    if (P->m_tail > 0)
      for (int64_t r = 0; r < R; ++r) ph1.push_back({double(P->N * P->m_tail) / 32.0, int4{T_ADJ_TAIL, p, 0, int(r)}});
    for (size_t i = 0; i < P->blocks.size(); ++i) {
      const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
      for (int64_t r = 0; r < R; ++r) ph2.push_back({c, int4{T_ADJ_FFT, p, int(i), int(r)}});
    }
  }
  order(ph1);
  order(ph2);
  std::vector<int4> adj;
  for (auto& e : ph1) adj.push_back(e.second);
  for (auto& e : ph2) adj.push_back(e.second);

  for (int p = 0; p < np; ++p) {
    need_f[p] += unsigned(b->extra_need[p]);
    need_a[p] += unsigned(b->extra_need[p]);
  }
  const std::vector<int4>* lists2[2] = {&fwd, &adj};
  const std::vector<unsigned>* needs[2] = {&need_f, &need_a};
  for (int d = 0; d < 2; ++d) {
    if (int64_t(lists2[d]->size()) > b->ntasks[d] || b->tasks[d] == nullptr) {
      void* ptr = nullptr;
      XC_TRY(b->alloc(&ptr, std::max<size_t>(1, lists2[d]->size()) * sizeof(int4)));
      b->tasks[d] = static_cast<int4*>(ptr);
    }
    b->ntasks[d] = int64_t(lists2[d]->size());
    if (!lists2[d]->empty())
      XC_CUDA(cudaMemcpy(b->tasks[d], lists2[d]->data(), lists2[d]->size() * sizeof(int4), cudaMemcpyHostToDevice));
    XC_CUDA(cudaMemcpy(b->need[d], needs[d]->data(), 2 * size_t(np) * sizeof(unsigned), cudaMemcpyHostToDevice));
  }
  b->rpw[0] = rpw_f;
  b->rpw[1] = rpw_a;
  return XC_OK;
}

template <typename T, bool COMP, int RPW>
int launch_batch_rpw(Batch* b, int dir, cudaStream_t st) {
  auto fn = batch_kernel<T, RPW, COMP>;
  if (b->smem > 48 * 1024)
    XC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(b->smem)));
  int dev = 0, sms = 0, per_sm = 0;
  XC_CUDA(cudaGetDevice(&dev));
  XC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  XC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(fn), kBatchThreads,
                                                        b->smem));
  if (per_sm < 1) return fail(XC_ERR_UNSUPPORTED, "batch kernel does not fit on an SM");
  const int64_t grid = std::min<int64_t>(int64_t(sms) * per_sm, std::max<int64_t>(1, b->ntasks[dir]));
  count_launch();
  fn<<<unsigned(grid), kBatchThreads, b->smem, st>>>(b->dplans, b->tasks[dir], b->ntasks[dir], b->ctrl, b->need[dir],
                                                      b->done, int(b->plans.size()), b->wait_limit);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

template <typename T, bool COMP>
int launch_batch_t(Batch* b, int dir, cudaStream_t st) {
  switch (b->rpw[dir]) {
    case 1: return launch_batch_rpw<T, COMP, 1>(b, dir, st);
    case 2: return launch_batch_rpw<T, COMP, 2>(b, dir, st);
    case 4: return launch_batch_rpw<T, COMP, 4>(b, dir, st);
    default: return launch_batch_rpw<T, COMP, 8>(b, dir, st);
  }
}

int launch_batch(Batch* b, int dir, cudaStream_t st) {
  if (b->ntasks[dir] == 0) return XC_OK;
  switch (b->precision) {
    case XC_FP64: return launch_batch_t<double, false>(b, dir, st);
    case XC_FP32: return launch_batch_t<float, false>(b, dir, st);
    default: return launch_batch_t<float, true>(b, dir, st);
  }
}

// Tuning cache: batch signature -> chosen right-hand sides per item (forward, adjoint).
std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;

std::string signature(const Batch* b) {
  std::string sig = std::to_string(b->precision) + ":" + std::to_string(b->plans.size());
  int64_t nnz = 0, rhs = 0, len = 0;
  for (size_t p = 0; p < b->plans.size(); ++p) {
    for (int64_t v : b->plans[p]->nnz) nnz += v;
    rhs += b->nrhs[p];
    len += b->plans[p]->N;
  }
  return sig + ":" + std::to_string(nnz) + ":" + std::to_string(rhs) + ":" + std::to_string(len);
}

}  // namespace

}  // namespace xc

using xc::fail;

extern "C" {

int xc_batch_create(xc_batch_t* out, const xc_plan_t* plans, int nplans) {
  if (!out) return fail(XC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!plans || nplans < 1) return fail(XC_ERR_ARG, "need at least one plan");
  auto* b = new (std::nothrow) xc::Batch();
  if (!b) return fail(XC_ERR_ALLOC, "host allocation failed");
  for (int i = 0; i < nplans; ++i) {
    auto* p = reinterpret_cast<xc::Plan*>(plans[i]);
    if (!p) {
      delete b;
      return fail(XC_ERR_ARG, "plan " + std::to_string(i) + " is NULL");
    }
    if (i > 0 && p->precision != b->precision) {
      delete b;
      return fail(XC_ERR_ARG, "all plans of a batch need the same precision");
    }
    b->precision = p->precision;
    b->plans.push_back(p);
    b->max_n = std::max(b->max_n, p->max_n);
  }
  b->smem = size_t(b->max_n) * 2 * (b->precision == XC_FP64 ? 8 : 4);
  b->extra_need.assign(nplans, 0);
  void* ptr = nullptr;
  int rc = b->alloc(&ptr, 4 * sizeof(unsigned));
  if (rc == XC_OK) {
    b->ctrl = static_cast<unsigned*>(ptr);
    rc = b->alloc(&ptr, 2 * size_t(nplans) * sizeof(unsigned));
  }
  if (rc == XC_OK) {
    b->done = static_cast<unsigned*>(ptr);
    rc = b->alloc(&ptr, 2 * size_t(nplans) * sizeof(unsigned));
  }
  if (rc == XC_OK) {
    b->need[0] = static_cast<unsigned*>(ptr);
    rc = b->alloc(&ptr, 2 * size_t(nplans) * sizeof(unsigned));
  }
  if (rc == XC_OK) {
    b->need[1] = static_cast<unsigned*>(ptr);
    rc = b->alloc(&ptr, size_t(nplans) * sizeof(xc::BatchPlanDev));
  }
  if (rc == XC_OK) {
    b->dplans = static_cast<xc::BatchPlanDev*>(ptr);
    if (cudaMemset(b->ctrl, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b->done, 0, 2 * size_t(nplans) * sizeof(unsigned)) != cudaSuccess)
      rc = xc::cuda_check(cudaGetLastError(), "cudaMemset");
  }
  if (rc != XC_OK) {
    const std::string msg = xc_last_error_message();
    delete b;
    return fail(rc, msg);
  }
  *out = reinterpret_cast<xc_batch_t>(b);
  return XC_OK;
}

int xc_batch_bind(xc_batch_t batch, const void* const* x_dev, void* const* y_dev, const int64_t* nrhs,
                  const int64_t* ld) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b || !x_dev || !y_dev || !nrhs || !ld) return fail(XC_ERR_ARG, "NULL argument");
  const int np = int(b->plans.size());
  std::vector<xc::BatchPlanDev> host(np);
  b->x.assign(x_dev, x_dev + np);
  b->y.assign(y_dev, y_dev + np);
  b->nrhs.assign(nrhs, nrhs + np);
  b->ld.assign(ld, ld + np);
  for (int i = 0; i < np; ++i) {
    xc::Plan* p = b->plans[i];
    if (nrhs[i] < 0 || nrhs[i] > (int64_t(1) << 24)) return fail(XC_ERR_ARG, "nrhs out of range");
    if (nrhs[i] > 0 && (!x_dev[i] || !y_dev[i] || x_dev[i] == y_dev[i] || ld[i] < p->N))
      return fail(XC_ERR_ARG, "bad buffers for plan " + std::to_string(i));
    XC_TRY(xc::ensure_scratch(p, std::max<int64_t>(1, nrhs[i])));
    xc::BatchPlanDev& d = host[i];
    std::memset(&d, 0, sizeof(d));
    d.blocks = static_cast<const xc::BlockDev*>(p->scratch_desc);
    d.nblocks = int(p->blocks.size());
    d.nslices = int(p->nslices);
    d.N = p->N;
    d.m_tail = p->m_tail;
    d.total_chunks = p->total_chunks;
    d.tail = p->tail;
    d.rowscale = p->rowscale;
    d.colscale = p->colscale;
    d.t_items = p->t_items;
    d.t_cbase = p->t_cbase;
    if (p->fwd_chunked) {
      d.fu_units = p->fu_units;
      d.fu_order = p->fu_order;
      d.fu_ubase = p->fu_ubase;
      d.total_units = p->total_units;
    }
    d.spec_per_rhs = p->spec_per_rhs;
    d.scratch = p->scratch;
    d.x = x_dev[i];
    d.y = y_dev[i];
    d.nrhs = nrhs[i];
    d.ld = ld[i];
  }
  XC_CUDA(cudaMemcpy(b->dplans, host.data(), size_t(np) * sizeof(xc::BatchPlanDev), cudaMemcpyHostToDevice));
  const int dflt = b->precision == XC_FP64 ? 2 : 8;
  std::pair<int, int> rpw{b->rpw[0] > 0 ? b->rpw[0] : dflt, b->rpw[1] > 0 ? b->rpw[1] : dflt};
  {
    std::lock_guard<std::mutex> lock(xc::g_tune_mutex);
    auto it = xc::g_tune_cache.find(xc::signature(b));
    if (it != xc::g_tune_cache.end()) rpw = it->second;
  }
  return xc::build_tasks(b, rpw.first, rpw.second);
}

int xc_batch_apply(xc_batch_t batch, int adjoint, void* stream) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b) return fail(XC_ERR_ARG, "batch is NULL");
  if (b->rpw[0] == 0) return fail(XC_ERR_ARG, "bind the batch's buffers first");
  return xc::launch_batch(b, adjoint ? 1 : 0, static_cast<cudaStream_t>(stream));
}

int xc_batch_tune(xc_batch_t batch, void* stream) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b) return fail(XC_ERR_ARG, "batch is NULL");
  if (b->rpw[0] == 0) return fail(XC_ERR_ARG, "bind the batch's buffers first");
  auto st = static_cast<cudaStream_t>(stream);
  // the trial launches overwrite x (adjoint) and y (forward): keep copies
  const size_t eb = b->precision == XC_FP64 ? 8 : 4;
  std::vector<void*> saved;
  struct Restore {
    std::vector<void*>* v;
    ~Restore() {
      for (void* d : *v) cudaFree(d);
    }
  } restore{&saved};
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const size_t bytes = size_t(b->nrhs[i]) * size_t(b->ld[i]) * eb;
    for (const void* src : {b->x[i], static_cast<const void*>(b->y[i])}) {
      void* d = nullptr;
      if (bytes > 0) {
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
          cudaGetLastError();
          return fail(XC_ERR_ALLOC, "tuner copy of the bound buffers failed");
        }
        saved.push_back(d);
        XC_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyDeviceToDevice, st));
      } else {
        saved.push_back(nullptr);
      }
    }
  }
  // each direction is timed on its own: the forward and adjoint band
  // products favour different numbers of right-hand sides per item
  cudaEvent_t ev[3];
  for (auto& e : ev) XC_CUDA(cudaEventCreate(&e));
  int best[2] = {b->rpw[0], b->rpw[1]};
  float best_ms[2] = {1e30f, 1e30f};
  for (int cand : {1, 2, 4, 8}) {
    XC_TRY(xc::build_tasks(b, cand, cand));
    XC_TRY(xc::launch_batch(b, 0, st));   // warm
    XC_TRY(xc::launch_batch(b, 1, st));
    float ms[2] = {0, 0};
    for (int rep = 0; rep < 3; ++rep) {
      XC_CUDA(cudaEventRecord(ev[0], st));
      XC_TRY(xc::launch_batch(b, 0, st));
      XC_CUDA(cudaEventRecord(ev[1], st));
      XC_TRY(xc::launch_batch(b, 1, st));
      XC_CUDA(cudaEventRecord(ev[2], st));
      XC_CUDA(cudaEventSynchronize(ev[2]));
      float f = 0, a = 0;
      XC_CUDA(cudaEventElapsedTime(&f, ev[0], ev[1]));
      XC_CUDA(cudaEventElapsedTime(&a, ev[1], ev[2]));
      ms[0] += f;
      ms[1] += a;
    }
    for (int d = 0; d < 2; ++d)
      if (ms[d] < best_ms[d]) {
        best_ms[d] = ms[d];
        best[d] = cand;
      }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const size_t bytes = size_t(b->nrhs[i]) * size_t(b->ld[i]) * eb;
    if (bytes == 0) continue;
    XC_CUDA(cudaMemcpyAsync(const_cast<void*>(b->x[i]), saved[2 * i], bytes, cudaMemcpyDeviceToDevice, st));
    XC_CUDA(cudaMemcpyAsync(b->y[i], saved[2 * i + 1], bytes, cudaMemcpyDeviceToDevice, st));
  }
  XC_CUDA(cudaStreamSynchronize(st));
  XC_TRY(xc::build_tasks(b, best[0], best[1]));
  b->tuned = true;
  std::lock_guard<std::mutex> lock(xc::g_tune_mutex);
  xc::g_tune_cache[xc::signature(b)] = {best[0], best[1]};
  return XC_OK;
}

int xc_batch_info(xc_batch_t batch, xc_batch_stats* out) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b || !out) return fail(XC_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->nplans = int(b->plans.size());
  out->rhs_per_item = b->rpw[0];
  out->rhs_per_item_adjoint = b->rpw[1];
  out->tuned = b->tuned ? 1 : 0;
  out->tasks_forward = b->ntasks[0];
  out->tasks_adjoint = b->ntasks[1];
  out->shared_bytes = int64_t(b->smem);
  for (const xc::Plan* p : b->plans) {
    out->matrix_bytes += p->matrix_bytes;
    out->adjoint_bytes += p->adjoint_bytes;
  }
  return XC_OK;
}

int xc_batch_status(xc_batch_t batch, void* stream) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b) return fail(XC_ERR_ARG, "batch is NULL");
  auto st = static_cast<cudaStream_t>(stream);
  unsigned status = 0;
  XC_CUDA(cudaMemcpyAsync(&status, &b->ctrl[2], sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  XC_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    XC_CUDA(cudaMemsetAsync(&b->ctrl[2], 0, sizeof(unsigned), st));
    XC_CUDA(cudaStreamSynchronize(st));
    return fail(XC_ERR_TIMEOUT, "a phase wait of the batch kernel gave up; results of that launch are incomplete");
  }
  return XC_OK;
}

int xc_batch_debug_set(xc_batch_t batch, int plan, int extra_need, int64_t wait_limit) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b) return fail(XC_ERR_ARG, "batch is NULL");
  if (plan < 0 || plan >= int(b->plans.size()) || extra_need < 0 || wait_limit < 1)
    return fail(XC_ERR_ARG, "bad debug setting");
  b->extra_need[plan] = extra_need;
  b->wait_limit = wait_limit;
  if (b->rpw[0] > 0) return xc::build_tasks(b, b->rpw[0], b->rpw[1]);
  return XC_OK;
}

int xc_batch_destroy(xc_batch_t batch) {
  delete reinterpret_cast<xc::Batch*>(batch);
  return XC_OK;
}

}  // extern "C"
