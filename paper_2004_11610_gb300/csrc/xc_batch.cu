// Many plans in one persistent launch per direction.
//
// A batch groups plans of one precision (uneven N, families and numbers of
// right-hand sides).  Binding I/O buffers builds, per direction, three device
// work lists over all plans:
//   forward   A: FFT of (plan, block, RHS), one CTA each        [fwd_fft_body]
//             B: band product of (plan, row slice, RPW RHS) + tail, or for
//                plans with long bands of (plan, band chunk, RPW RHS) into
//                partial sums; one warp each         [fwd_sparse_item / fwd_unit_item]
//             C: (long-band plans) partials + tail of (plan, 32 rows), one
//                warp each                                      [fwd_reduce_row]
//   adjoint   B: transposed band product of (plan, chunk, RPW RHS) and the
//                dense tail of (plan, column, RHS), one warp each
//             C: inverse FFT of (plan, block, RHS), one CTA each
// Plans whose window (lockstep) layouts are tight -- Hermite functions, the
// bulk of the 1000-plan workload's band values -- run their band products as
// lockstep items instead (fwd_lock_item / fwd_lock_unit / adj_lock_item): the
// warp's 32 rows (bins) walk the same bin (row), the forward spectra are
// written bin-major (bin k of RHS r at k * rp + r, rp = nrhs rounded up to
// 8) into a scratch buffer owned by the batch, and each lane owns a block of
// RL rows (bins) x 8 right-hand sides, so that every band and spectrum value
// it loads feeds several multiply-adds.  The tuner decides per direction
// whether such plans use them.
// FP32 plans whose bands are nearly dense over 128 rows (64 bins) also have
// tensor windows; with lockstep 2 their band products leave the persistent
// launch for tensor-core launches of their own (xc_window.cuh): forward, the
// persistent launch makes their spectra (bin-major), fwd_tail_kernel puts
// their dense tails' sums in y, and tc_window_kernel<NP, false> adds the band
// sums; adjoint, adj_yt_kernel writes their row-scaled right-hand sides
// row-major, tc_window_kernel<NP, true> writes one chunk partial per bin
// slice, and the persistent launch that follows runs their tails and inverse
// FFTs.
// Every CTA of a persistent grid works through A (CTA tasks from a device
// counter), then its warps take B items one by one from a second counter,
// then -- after a CTA barrier -- it works through C (CTA tasks or warp items).
// Warps thus never wait for the slowest warp of their CTA inside B, where the
// items are of very uneven length.  Within each list the costliest entries
// come first.  An entry of plan p in B waits until all A tasks of p have
// finished (done[p] reaches need[p]); an entry in C waits for all B items of
// p (done[nplans + p] reaches need[nplans + p]).  The finishing task or item
// increments the counter after a fence; the waiter reads it with acquire
// semantics, sleeping between reads, for a bounded number of reads.  Because
// a CTA enters B only when A is exhausted -- every A task has been taken by a
// running CTA -- and C only when B is exhausted, the waits end; if one does
// not end within the limit, the status word records a timeout, the remaining
// work of the launch is skipped and the host reads XC_ERR_TIMEOUT.  The last
// CTA to finish resets the counters, so a launch needs no memset and can be
// captured in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <type_traits>
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
#include "xc_lock.cuh"
#include "xc_window.cuh"

namespace xc {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
enum TaskKind {
  T_FWD_FFT = 0, T_FWD_SPARSE = 1, T_ADJ_SPARSE = 2, T_ADJ_FFT = 3, T_ADJ_TAIL = 4, T_FWD_UNIT = 5, T_FWD_REDUCE = 6,
  T_FWD_LOCK = 7, T_FWD_LUNIT = 8, T_ADJ_LOCK = 9
};
// control words: next entry of lists A, B, C; finished CTAs; status
enum { C_NEXT_A = 0, C_NEXT_B = 1, C_NEXT_C = 2, C_FINISHED = 3, C_STATUS = 4, C_WORDS = 8 };

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
  // lockstep items (lock_f: forward, lock_a: adjoint); their spectra and
  // partial sums live in lscratch (forward: spectra [bin][rp] of every block,
  // then the unit partials; adjoint: the chunk partials)
  int lock_f, lock_a, rp, rl;   // rp: bin-major spectrum row (nrhs rounded up to 8); rl: rows per lane
  void* lscratch;
  const int4* lk_units;
  const int* lk_ubase;
  const int2* lk_items;
  const int* lk_cbase;
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

// One CTA task (an FFT of one block and RHS).
template <typename T>
__device__ __forceinline__ void run_cta_task(const BatchPlanDev& P, int4 tk, cx<T>* s, int tid) {
  const T* cs = static_cast<const T*>(P.colscale);
  if (tk.x == T_FWD_FFT) {
    if (P.lock_f)
      fwd_fft_body<T>(P.blocks[tk.z], tk.w, static_cast<const T*>(P.x), P.ld, cs, static_cast<cx<T>*>(P.lscratch),
                      P.nrhs, s, tid, kBatchThreads, nullptr, P.rp);
    else
      fwd_fft_body<T>(P.blocks[tk.z], tk.w, static_cast<const T*>(P.x), P.ld, cs, static_cast<cx<T>*>(P.scratch),
                      P.nrhs, s, tid, kBatchThreads);
  } else {  // T_ADJ_FFT
    adj_fft_body<T>(P.blocks[tk.z], tk.w, static_cast<const cx<T>*>(P.lock_a ? P.lscratch : P.scratch),
                    P.lock_a ? P.lk_cbase : P.t_cbase, P.nrhs, static_cast<T*>(const_cast<void*>(P.x)), P.ld, cs, s,
                    tid, kBatchThreads);
  }
}

// Batch tail item: columns [m0, m0 + kTailCols) of x (those below m_tail)
// for right-hand side r, x_m = colscale_m sum_n tail[m][n] rowscale_n y_n;
// the lanes stride over the rows with one sum per column (in the order of
// adj_tail_warp), then a warp reduction per column.  Eight columns per item
// keep the batch's list short (one item per column and RHS made the
// bookkeeping of the adjoint launch cost as much as a third of it).
constexpr int kTailCols = 8;

template <typename T, bool COMP>
__device__ void adj_tail_cols(int64_t N, int64_t m_tail, int64_t m0, int64_t r, const T* __restrict__ tail,
                              const T* __restrict__ y, int64_t ld, T* __restrict__ x, const T* __restrict__ rowscale,
                              const T* __restrict__ colscale, int lane) {
  const int nc = int(m_tail - m0 < kTailCols ? m_tail - m0 : kTailCols);
  Acc<T, COMP> acc[kTailCols];
  for (int64_t n = lane; n < N; n += 32) {
    const T yv = y[r * ld + n] * (rowscale ? rowscale[n] : T(1));
#pragma unroll
    for (int c = 0; c < kTailCols; ++c)
      if (c < nc) acc[c].add(tail[(m0 + c) * N + n], yv);
  }
#pragma unroll
  for (int c = 0; c < kTailCols; ++c) {
    if (c >= nc) break;
    T v = acc[c].value();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) x[r * ld + m0 + c] = v * (colscale ? colscale[m0 + c] : T(1));
  }
}

// Forward dense tails of the plans whose band products run in the window
// launches (xc_window.cuh): one warp per entry (plan, row slice), lane = row
// 32 slice + lane, all right-hand sides in groups of 8; y[r][n] = sum_m
// tail[m][n] colscale_m x[r][m], unscaled -- the window epilogue adds the
// band sums and applies the row scale.  A launch of its own: as an item of
// the persistent kernel it cost that kernel's 80-register instantiations a
// quarter of their speed.
__global__ void __launch_bounds__(256) fwd_tail_kernel(const BatchPlanDev* __restrict__ plans,
                                                       const int2* __restrict__ entries, int64_t n) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; e < n;
       e += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const int2 en = entries[e];
    const BatchPlanDev& P = plans[en.x];
    const int64_t row = int64_t(en.y) * 32 + lane;
    if (row >= P.N) continue;
    const float* tail = static_cast<const float*>(P.tail);
    const float* x = static_cast<const float*>(P.x);
    const float* cs = static_cast<const float*>(P.colscale);
    float* y = static_cast<float*>(P.y);
    for (int64_t r0 = 0; r0 < P.nrhs; r0 += 8) {
      const int nq = int(P.nrhs - r0 < 8 ? P.nrhs - r0 : 8);
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int64_t m = 0; m < P.m_tail; ++m) {
        const float tv = tail[m * P.N + row] * (cs ? cs[m] : 1.f);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nq) acc[q] = fmaf(tv, x[(r0 + q) * P.ld + m], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < nq) y[(r0 + q) * P.ld + row] = acc[q];
    }
  }
}

// Row-scaled right-hand sides of the plans whose adjoint band products run in
// the window launches, stored row-major for them: yt[n][r] = y[r][n]
// rowscale_n, one warp per entry (plan, row slice), lane = row.  The pad
// columns r >= nrhs and the pad rows past N stay zero from the allocation.
__global__ void __launch_bounds__(256) adj_yt_kernel(const WinPlan* __restrict__ plans,
                                                     const int2* __restrict__ entries, int64_t n) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; e < n;
       e += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const int2 en = entries[e];
    const WinPlan& P = plans[en.x];
    const int64_t row = int64_t(en.y) * 32 + lane;
    if (row >= P.N) continue;
    const float rs = P.rowscale ? P.rowscale[row] : 1.f;
    float* out = P.yt + row * P.rp;
    for (int64_t r = 0; r < P.nrhs; ++r) out[r] = P.y[r * P.ld + row] * rs;
  }
}

// Lockstep forward items of a plan: RL = P.rl rows per lane (1, 2 or 4;
// 8 RL right-hand sides per item).
template <typename T, bool COMP>
__device__ __noinline__ void run_lock_item(const BatchPlanDev& P, int4 tk, int lane, unsigned char* ring) {
  const T* rs = static_cast<const T*>(P.rowscale);
  const T* cs = static_cast<const T*>(P.colscale);
  const cx<T>* sp = static_cast<const cx<T>*>(P.lscratch);
  auto go = [&](auto rl) {
    constexpr int RL = decltype(rl)::value;
    fwd_lock_item<T, RL, COMP>(P.blocks, P.nblocks, P.N, static_cast<const T*>(P.x), P.ld, static_cast<T*>(P.y), sp,
                               P.rp, P.nrhs, rs, cs, static_cast<const T*>(P.tail), P.m_tail, tk.z,
                               int64_t(tk.w) * lock_rhs<RL>(), lane, ring);
  };
  if constexpr (!COMP) {
    if (P.rl == 4) {
      go(std::integral_constant<int, 4>{});
      return;
    }
  }
  if (P.rl == 2) go(std::integral_constant<int, 2>{});
  else go(std::integral_constant<int, 1>{});
}

template <typename T, bool COMP>
__device__ __noinline__ void run_lock_unit(const BatchPlanDev& P, int4 tk, int lane, unsigned char* ring) {
  const cx<T>* sp = static_cast<const cx<T>*>(P.lscratch);
  cx<T>* part = static_cast<cx<T>*>(P.lscratch) + P.spec_per_rhs * P.rp;
  auto go = [&](auto rl) {
    constexpr int RL = decltype(rl)::value;
    fwd_lock_unit<T, RL, COMP>(P.blocks, sp, P.rp, P.nrhs, part, P.lk_units[tk.z], tk.z,
                               int64_t(tk.w) * lock_rhs<RL>(), lane, ring);
  };
  if constexpr (!COMP) {
    if (P.rl == 4) {
      go(std::integral_constant<int, 4>{});
      return;
    }
  }
  if (P.rl == 2) go(std::integral_constant<int, 2>{});
  else go(std::integral_constant<int, 1>{});
}

// Lockstep adjoint items: RL bins per lane, so that the real and imaginary
// sums of RL bins x 8 RHS stay in registers: 2, and 1 with compensation (4
// bins x 8 and 2 bins x 16 right-hand sides per lane, in the kernels with
// 128 registers per thread, ran no faster).
template <int RPW, bool COMP>
__host__ __device__ constexpr int adj_lock_rl() { return COMP ? 1 : 2; }

template <typename T, bool COMP, int RL>
__device__ __noinline__ void run_lock_adj(const BatchPlanDev& P, int4 tk, int lane, unsigned char* ring) {
  adj_lock_item<T, RL, COMP>(P.blocks, P.nblocks, static_cast<const T*>(P.y), P.ld,
                             static_cast<cx<T>*>(P.lscratch), P.nrhs, static_cast<const T*>(P.rowscale), P.lk_cbase,
                             P.lk_items[tk.z], int64_t(tk.w) * lock_rhs<RL>(), lane, ring);
}

// One warp item.
template <typename T, int RPW, bool COMP>
__device__ __forceinline__ void run_warp_item(const BatchPlanDev& P, int4 tk, int lane, unsigned char* ring) {
  const T* rs = static_cast<const T*>(P.rowscale);
  const T* cs = static_cast<const T*>(P.colscale);
  switch (tk.x) {
    case T_FWD_SPARSE:
      fwd_sparse_item<T, RPW, COMP>(P.blocks, P.nblocks, P.N, static_cast<const T*>(P.x), P.ld, static_cast<T*>(P.y),
                                    static_cast<const cx<T>*>(P.scratch), P.nrhs, rs, cs,
                                    static_cast<const T*>(P.tail), P.m_tail, tk.z, int64_t(tk.w) * RPW, lane);
      break;
    case T_FWD_UNIT: {
      const int u = P.fu_order[tk.z];
      fwd_unit_item<T, RPW, COMP>(P.blocks, static_cast<const cx<T>*>(P.scratch), P.nrhs,
                                  static_cast<cx<T>*>(P.scratch) + P.spec_per_rhs * P.nrhs, P.fu_units[u], u,
                                  int64_t(tk.w) * RPW, lane);
      break;
    }
    case T_FWD_REDUCE: {
      const int64_t n = int64_t(tk.z) * 32 + lane;
      const cx<T>* part = P.lock_f ? static_cast<const cx<T>*>(P.lscratch) + P.spec_per_rhs * P.rp
                                   : static_cast<const cx<T>*>(P.scratch) + P.spec_per_rhs * P.nrhs;
      if (n < P.N)
        for (int64_t r = 0; r < P.nrhs; ++r)
          fwd_reduce_row<T, COMP>(P.N, static_cast<const T*>(P.x), P.ld, static_cast<T*>(P.y), part, P.nrhs,
                                  P.lock_f ? P.lk_ubase : P.fu_ubase, rs, cs, static_cast<const T*>(P.tail), P.m_tail,
                                  n, r);
      break;
    }
    // lockstep items exist for FP32 batches only
    case T_FWD_LOCK:
      if constexpr (sizeof(T) == 4) run_lock_item<T, COMP>(P, tk, lane, ring);
      break;
    case T_FWD_LUNIT:
      if constexpr (sizeof(T) == 4) run_lock_unit<T, COMP>(P, tk, lane, ring);
      break;
    case T_ADJ_LOCK:
      if constexpr (sizeof(T) == 4) run_lock_adj<T, COMP, adj_lock_rl<RPW, COMP>()>(P, tk, lane, ring);
      break;
    case T_ADJ_SPARSE:
      adj_sparse_item<T, RPW, COMP>(P.blocks, P.nblocks, static_cast<const T*>(P.y), P.ld, nullptr, 0,
                                    static_cast<cx<T>*>(P.scratch), P.nrhs, rs, P.t_cbase, P.t_items[tk.z], kAdjChunk,
                                    int64_t(tk.w) * RPW, lane);
      break;
    default:  // T_ADJ_TAIL: columns [tk.z, tk.z + kTailCols), RHS tk.w
      adj_tail_cols<T, COMP>(P.N, P.m_tail, tk.z, tk.w, static_cast<const T*>(P.tail), static_cast<const T*>(P.y),
                             P.ld, static_cast<T*>(const_cast<void*>(P.x)), rs, cs, lane);
      break;
  }
}

// Which completion counter an entry waits for (-1: none) and which one it
// increments (-1: none): index p (after the A tasks of plan p) or nplans + p
// (after its B items).
__device__ __forceinline__ int waits_on(int kind, int plan, int nplans) {
  if (kind == T_FWD_SPARSE || kind == T_FWD_UNIT || kind == T_FWD_LOCK || kind == T_FWD_LUNIT) return plan;
  if (kind == T_FWD_REDUCE || kind == T_ADJ_FFT) return nplans + plan;
  return -1;
}
__device__ __forceinline__ int counts_in(int kind, int plan, int nplans) {
  if (kind == T_FWD_FFT) return plan;
  if (kind == T_FWD_SPARSE || kind == T_FWD_UNIT || kind == T_ADJ_SPARSE || kind == T_ADJ_TAIL ||
      kind == T_FWD_LOCK || kind == T_FWD_LUNIT || kind == T_ADJ_LOCK)
    return nplans + plan;
  return -1;
}

// A list worked through by whole CTAs.
template <typename T>
__device__ void cta_list(const BatchPlanDev* __restrict__ plans, const int4* __restrict__ list, int64_t n,
                         unsigned* next, const unsigned* __restrict__ need, unsigned* done, int nplans,
                         long long wait_limit, unsigned* status, cx<T>* s, unsigned* s_task, int* s_ok) {
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) *s_task = atomicAdd(next, 1u);
    __syncthreads();
    const int64_t t = *s_task;
    if (t >= n) break;
    const int4 tk = list[t];
    if (tid == 0) {
      const int w = waits_on(tk.x, tk.y, nplans);
      *s_ok = w >= 0 ? wait_for(&done[w], need[w], wait_limit, status) : (*(volatile unsigned*)status == 0u);
    }
    __syncthreads();
    if (*s_ok) run_cta_task<T>(plans[tk.y], tk, s, tid);
    const int c = counts_in(tk.x, tk.y, nplans);
    if (c >= 0) {
      __syncthreads();                        // every thread's results are written
      if (tid == 0) {
        __threadfence();
        atomicAdd(&done[c], 1u);
      }
    }
    __syncthreads();                          // s_task / s_ok are reused
  }
}

// A list worked through by single warps, one entry per atomic on the list
// counter.  (Taking four consecutive entries per atomic, with the completions
// of a plan's entries added at once, made the 1000-plan batch slower: the
// right-hand-side groups of one band chunk, which sit next to each other in
// the list, then run one after another on one warp instead of side by side
// on four, and the list's end balances worse.)
template <typename T, int RPW, bool COMP>
__device__ void warp_list(const BatchPlanDev* __restrict__ plans, const int4* __restrict__ list, int64_t n,
                          unsigned* next, const unsigned* __restrict__ need, unsigned* done, int nplans,
                          long long wait_limit, unsigned* status, unsigned char* ring) {
  const int lane = threadIdx.x & 31;
  int pend_c = -1;
  unsigned pend = 0;
  auto flush = [&]() {
    if (pend_c >= 0 && pend > 0) {
      __syncwarp();                           // every lane's results are written
      if (lane == 0) {
        __threadfence();
        atomicAdd(&done[pend_c], pend);
      }
    }
    pend = 0;
  };
  for (;;) {
    unsigned t0 = 0;
    if (lane == 0) t0 = atomicAdd(next, 1u);
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    if (int64_t(t0) >= n) break;
    {
      const int64_t t = t0;
      const int4 tk = list[t];
      int ok = 0;
      if (lane == 0) {
        const int w = waits_on(tk.x, tk.y, nplans);
        ok = w >= 0 ? wait_for(&done[w], need[w], wait_limit, status) : (*(volatile unsigned*)status == 0u);
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok) run_warp_item<T, RPW, COMP>(plans[tk.y], tk, lane, ring);
      const int c = counts_in(tk.x, tk.y, nplans);
      if (c != pend_c) {
        flush();
        pend_c = c;
      }
      if (c >= 0) ++pend;
    }
    flush();
  }
}

// Three CTAs per SM where the accumulators fit in 80 registers (the shared
// FFT buffer of the largest plans allows about three as well), two otherwise.
template <typename T, int RPW, bool COMP>
__global__ void __launch_bounds__(kBatchThreads, RPW * sizeof(T) >= 32 ? 2 : 3)
    batch_kernel(const BatchPlanDev* __restrict__ plans, const int4* __restrict__ listA, int64_t nA,
                 const int4* __restrict__ listB, int64_t nB, const int4* __restrict__ listC, int64_t nC,
                 int c_by_warps, unsigned* ctrl, const unsigned* __restrict__ need, unsigned* done, int nplans,
                 long long wait_limit, int smem_ring) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  __shared__ unsigned s_task;
  __shared__ int s_ok;
  __shared__ int s_last;
  const int tid = threadIdx.x;
  unsigned* status = &ctrl[C_STATUS];
  cta_list<T>(plans, listA, nA, &ctrl[C_NEXT_A], need, done, nplans, wait_limit, status, s, &s_task, &s_ok);
  // the band phase: each warp's staging ring in the FFT buffer, idle until phase C
  unsigned char* ring = smem_ring ? smem_raw + (tid >> 5) * kRingBytes : nullptr;
  warp_list<T, RPW, COMP>(plans, listB, nB, &ctrl[C_NEXT_B], need, done, nplans, wait_limit, status, ring);
  __syncthreads();
  if (c_by_warps)
    warp_list<T, RPW, COMP>(plans, listC, nC, &ctrl[C_NEXT_C], need, done, nplans, wait_limit, status, nullptr);
  else
    cta_list<T>(plans, listC, nC, &ctrl[C_NEXT_C], need, done, nplans, wait_limit, status, s, &s_task, &s_ok);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl[C_FINISHED], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int p = tid; p < 2 * nplans; p += kBatchThreads) done[p] = 0u;
    __syncthreads();
    if (tid == 0) {
      ctrl[C_NEXT_A] = 0u;
      ctrl[C_NEXT_B] = 0u;
      ctrl[C_NEXT_C] = 0u;
      ctrl[C_FINISHED] = 0u;
    }
  }
}

}  // namespace

struct Batch {
  std::vector<Plan*> plans;
  int precision = XC_FP64;
  BatchPlanDev* dplans = nullptr;
  // per direction (0 forward, 1 adjoint): work lists A, B, C
  int4* list[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int64_t nlist[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int64_t cap[2][3] = {{0, 0, 0}, {0, 0, 0}};
  unsigned* need[2] = {nullptr, nullptr};   // [2 * nplans]: A tasks, B items per plan
  unsigned* ctrl = nullptr;      // C_WORDS control words
  unsigned* done = nullptr;      // [2 * nplans]: finished A tasks, B items per plan
  std::vector<int> extra_need;   // fault injection (tests)
  long long wait_limit = 1LL << 22;   // sleeps of ~256 ns: about a second
  int rpw[2] = {0, 0};           // right-hand sides per band item, per direction (0 = not bound)
  int lock[2] = {1, 1};          // lockstep items for the plans that have them, per direction
  float tune_ms[2][12];           // the tuner's timings, entry 4 * lockstep + log2(rpw); -1: not tried
  // forward tensor-window launches (xc_window.cuh), one per class of
  // spectrum row length rp <= 16, 32, 64: the plans' descriptors and the
  // tasks (plan, row group) of each class
  // (per direction: the window launches of the forward band products and of
  // the adjoint's)
  WinPlan* dwin[2] = {nullptr, nullptr};
  std::vector<WinPlan> hwin[2];
  int4* wlist[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int64_t nw[2][3] = {{0, 0, 0}, {0, 0, 0}}, wcap[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int2* tlist = nullptr;         // (plan, row slice) entries of fwd_tail_kernel
  int64_t ntail = 0, tcap = 0;
  int2* ylist = nullptr;         // (plan, row slice) entries of adj_yt_kernel
  int64_t nyt = 0, ycap = 0;
  std::vector<void*> ytbuf;      // per plan: the adjoint windows' row-scaled right-hand sides (nullptr: none)
  std::vector<int64_t> ytbuf_bytes;
  int tens_plans[2] = {0, 0};
  bool ring = false;             // the kernel's shared memory holds the warps' staging rings
  bool tuned = false;
  std::vector<BatchPlanDev> host;   // device copies of these are in dplans
  std::vector<void*> lscratch;   // per plan: the batch's lockstep scratch (nullptr: none)
  std::vector<int64_t> lscratch_bytes;
  size_t smem = 0;
  int64_t max_n = 0;
  std::vector<const void*> x;
  std::vector<void*> y;
  std::vector<int64_t> nrhs, ld;
  std::vector<void*> allocs;
  bool holds_refs = false;       // counted in each plan's batch_refs (after the first bind)
  ~Batch() {
    cudaDeviceSynchronize();
    for (void* d : allocs) cudaFree(d);
    if (holds_refs)
      for (Plan* p : plans) --p->batch_refs;
  }
  int alloc(void** ptr, size_t bytes) {
    if (cudaMalloc(ptr, bytes == 0 ? 1 : bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(XC_ERR_ALLOC, "batch allocation failed");
    }
    allocs.push_back(*ptr);
    return XC_OK;
  }
  int64_t entries(int dir) const { return nlist[dir][0] + nlist[dir][1] + nlist[dir][2]; }
};

namespace {

using Entry = std::pair<double, int4>;   // (cost estimate, entry)

// Whether plan p of the batch runs its forward band product on the tensor
// cores (xc_window.cuh) when the schedule asks for it: an XC_FP32 plan with
// tensor windows, lockstep scratch and at most 64 right-hand sides.
bool tensor_capable(const Batch* b, int p) {
  const Plan* P = b->plans[p];
  return b->precision == XC_FP32 && P->tens_ok && b->lscratch[p] != nullptr && b->nrhs[p] > 0 && b->nrhs[p] <= 64;
}
// The same for the adjoint band product (transposed tensor windows).
bool tensor_t_capable(const Batch* b, int p) {
  const Plan* P = b->plans[p];
  return b->precision == XC_FP32 && P->tens_t_ok && b->lscratch[p] != nullptr && b->ytbuf[p] != nullptr &&
         b->nrhs[p] > 0 && b->nrhs[p] <= 64;
}

// Work lists of both directions for the bound right-hand sides, with rpw_f
// (forward) and rpw_a (adjoint) right-hand sides per band item; lock_f /
// lock_a: the plans that have lockstep scratch use lockstep items in that
// direction, and with lock_f = 2 the plans with tensor windows run their
// forward band products in the window launches (tasks = row groups, one
// list per class of spectrum row length).  Uploads the plan descriptors
// with the matching flags.
int build_tasks(Batch* b, int rpw_f, int rpw_a, int lock_f, int lock_a) {
  const int np = int(b->plans.size());
  b->rpw[0] = b->rpw[1] = 0;   // unbound until every list is in place (a failure leaves it so)
  std::vector<Entry> L[2][3];
  std::vector<std::pair<double, int4>> W[2][3];
  std::vector<int2> tails, yts;
  std::vector<unsigned> need[2] = {std::vector<unsigned>(2 * size_t(np), 0), std::vector<unsigned>(2 * size_t(np), 0)};
  for (int d = 0; d < 2; ++d) {
    b->hwin[d].assign(np, WinPlan{});
    b->tens_plans[d] = 0;
  }
  for (int p = 0; p < np; ++p) {
    const Plan* P = b->plans[p];
    BatchPlanDev& H = b->host[p];
    const bool tens = lock_f == 2 && tensor_capable(b, p);
    // tensor plans keep the lockstep (bin-major) spectra of their FFTs
    H.lock_f = tens || (lock_f && b->lscratch[p] != nullptr && P->lock_f_ok);
    const bool tens_a = lock_a == 2 && tensor_t_capable(b, p);
    // tensor adjoint plans write one chunk partial per bin slice, which the
    // inverse FFTs read as they read the lockstep items' partials
    H.lock_a = tens_a || (lock_a && b->lscratch[p] != nullptr && P->lock_t_ok);
    H.lk_cbase = tens_a ? P->tw_tcbase : P->lk_cbase;
    const int64_t R = b->nrhs[p];
    if (R == 0) continue;
    if (tens) {
      for (size_t i = 0; i < P->blocks.size(); ++i) {
        const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
        for (int64_t r = 0; r < R; ++r) {
          L[0][0].push_back({c, int4{T_FWD_FFT, p, int(i), int(r)}});
          ++need[0][p];
        }
      }
      // the dense tail's sums go to y first (fwd_tail_kernel)
      if (P->m_tail > 0)
        for (int64_t s0 = 0; s0 < P->nslices; ++s0) tails.push_back(int2{p, int(s0)});
      const int cls = H.rp <= 16 ? 0 : H.rp <= 32 ? 1 : 2;
      for (int64_t g = 0; g < P->tens_groups; ++g) {
        int tiles = 0;
        for (size_t i = 0; i < P->blocks.size(); ++i) tiles += P->tw_nkb_h[i][g];
        W[0][cls].push_back({double(tiles), int4{p, 0, int(g), 0}});
      }
      WinPlan& w = b->hwin[0][p];
      w.blocks = P->win_blocks;
      w.nblocks = int(P->blocks.size());
      w.rp = H.rp;
      w.N = P->N;
      w.nrhs = R;
      w.ld = b->ld[p];
      w.y = static_cast<float*>(b->y[p]);
      w.spec = static_cast<const cx<float>*>(b->lscratch[p]);
      w.tail_in_y = P->m_tail > 0 ? 1 : 0;
      w.rowscale = static_cast<const float*>(P->rowscale);
      ++b->tens_plans[0];
    } else if (H.lock_f) {
      for (size_t i = 0; i < P->blocks.size(); ++i) {
        const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
        for (int64_t r = 0; r < R; ++r) {
          L[0][0].push_back({c, int4{T_FWD_FFT, p, int(i), int(r)}});
          ++need[0][p];
        }
      }
      // a lockstep item covers 8 RL right-hand sides (RL rows per lane)
      const int64_t lr = 8 * int64_t(H.rl);
      const int64_t gf = (R + lr - 1) / lr;
      if (P->fwd_chunked) {
        for (int64_t k = 0; k < P->lk_total_units; ++k)
          for (int64_t g = 0; g < gf; ++g) {
            L[0][1].push_back({double(P->lk_unit_len[k]) * double(lr), int4{T_FWD_LUNIT, p, int(k), int(g)}});
            ++need[0][np + p];
          }
        for (int64_t s0 = 0; s0 < P->nslices; ++s0)
          L[0][2].push_back({double(R) * double(P->m_tail + 4), int4{T_FWD_REDUCE, p, int(s0), 0}});
      } else {
        for (int64_t s0 = 0; s0 < P->nslices; ++s0) {
          int64_t w = 0;
          for (size_t i = 0; i < P->blocks.size(); ++i) w += P->hf_len[i][s0];
          for (int64_t g = 0; g < gf; ++g) {
            L[0][1].push_back({double(w + P->m_tail) * double(lr), int4{T_FWD_LOCK, p, int(s0), int(g)}});
            ++need[0][np + p];
          }
        }
      }
    }
    if (tens_a) {
      // adjoint on the tensor cores: yt, then every bin group's window
      // product (groups without tiles write zeros), the tails and inverse FFTs
      for (int64_t s0 = 0; s0 < P->nslices; ++s0) yts.push_back(int2{p, int(s0)});
      const int cls = H.rp <= 16 ? 0 : H.rp <= 32 ? 1 : 2;
      for (size_t i = 0; i < P->blocks.size(); ++i)
        for (size_t g = 0; g < P->tw_t_nkb_h[i].size(); ++g)
          W[1][cls].push_back({double(P->tw_t_nkb_h[i][g]) + 0.5, int4{p, int(i), int(g), 0}});
      for (int64_t m = 0; m < P->m_tail; m += kTailCols)
        for (int64_t r = 0; r < R; ++r) {
          L[1][1].push_back({double(P->N) / 32.0 * double(std::min<int64_t>(kTailCols, P->m_tail - m)),
                             int4{T_ADJ_TAIL, p, int(m), int(r)}});
          ++need[1][np + p];
        }
      for (size_t i = 0; i < P->blocks.size(); ++i) {
        const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
        for (int64_t r = 0; r < R; ++r) L[1][2].push_back({c, int4{T_ADJ_FFT, p, int(i), int(r)}});
      }
      WinPlan& w = b->hwin[1][p];
      w.blocks = P->win_blocks_t;
      w.nblocks = int(P->blocks.size());
      w.rp = H.rp;
      w.N = P->N;
      w.nrhs = R;
      w.ld = b->ld[p];
      w.y = static_cast<float*>(b->y[p]);
      w.rowscale = static_cast<const float*>(P->rowscale);
      w.yt = static_cast<float*>(b->ytbuf[p]);
      w.part = static_cast<cx<float>*>(b->lscratch[p]);
      ++b->tens_plans[1];
    } else if (H.lock_a) {
      // adjoint lockstep items: RL bins x 8 RHS per lane, 8 RL right-hand sides per item
      const int64_t la = b->precision == XC_FP32_COMPENSATED ? 8 : 16;
      const int64_t ga = (R + la - 1) / la;
      for (int64_t i = 0; i < P->lk_total_chunks; ++i)
        for (int64_t g = 0; g < ga; ++g) {
          L[1][1].push_back({double(P->lk_item_len[i]) * double(la), int4{T_ADJ_LOCK, p, int(i), int(g)}});
          ++need[1][np + p];
        }
      for (int64_t m = 0; m < P->m_tail; m += kTailCols)
        for (int64_t r = 0; r < R; ++r) {
          L[1][1].push_back({double(P->N) / 32.0 * double(std::min<int64_t>(kTailCols, P->m_tail - m)),
                             int4{T_ADJ_TAIL, p, int(m), int(r)}});
          ++need[1][np + p];
        }
      for (size_t i = 0; i < P->blocks.size(); ++i) {
        const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
        for (int64_t r = 0; r < R; ++r) L[1][2].push_back({c, int4{T_ADJ_FFT, p, int(i), int(r)}});
      }
    }
    if (H.lock_f && H.lock_a) continue;
    // forward (row-per-lane items)
    if (!H.lock_f) {
    for (size_t i = 0; i < P->blocks.size(); ++i) {
      const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
      for (int64_t r = 0; r < R; ++r) {
        L[0][0].push_back({c, int4{T_FWD_FFT, p, int(i), int(r)}});
        ++need[0][p];
      }
    }
    const int64_t gf = (R + rpw_f - 1) / rpw_f;
    if (P->fwd_chunked) {
      for (int64_t k = 0; k < P->total_units; ++k)
        for (int64_t g = 0; g < gf; ++g) {
          L[0][1].push_back({double(P->unit_len[k]) * rpw_f, int4{T_FWD_UNIT, p, int(k), int(g)}});
          ++need[0][np + p];
        }
      for (int64_t s0 = 0; s0 < P->nslices; ++s0)
        L[0][2].push_back({double(R) * double(P->m_tail + 4), int4{T_FWD_REDUCE, p, int(s0), 0}});
    } else {
      for (int64_t s0 = 0; s0 < P->nslices; ++s0)
        for (int64_t g = 0; g < gf; ++g) {
          L[0][1].push_back({double(P->slice_cost[s0] + P->m_tail) * rpw_f, int4{T_FWD_SPARSE, p, int(s0), int(g)}});
          ++need[0][np + p];
        }
    }
    }
    // adjoint
    if (H.lock_a) continue;
    const int64_t ga = (R + rpw_a - 1) / rpw_a;
    for (int64_t i = 0; i < P->total_chunks; ++i)
      for (int64_t g = 0; g < ga; ++g) {
        L[1][1].push_back({double(P->item_len[i]) * rpw_a, int4{T_ADJ_SPARSE, p, int(i), int(g)}});
        ++need[1][np + p];
      }
    for (int64_t m = 0; m < P->m_tail; m += kTailCols)
      for (int64_t r = 0; r < R; ++r) {
        L[1][1].push_back({double(P->N) / 32.0 * double(std::min<int64_t>(kTailCols, P->m_tail - m)),
                           int4{T_ADJ_TAIL, p, int(m), int(r)}});
        ++need[1][np + p];
      }
    for (size_t i = 0; i < P->blocks.size(); ++i) {
      const double c = double(P->blocks[i].n) * std::log2(double(P->blocks[i].n) + 1.0);
      for (int64_t r = 0; r < R; ++r) L[1][2].push_back({c, int4{T_ADJ_FFT, p, int(i), int(r)}});
    }
  }
  for (int p = 0; p < np; ++p) {
    need[0][p] += unsigned(b->extra_need[p]);       // forward B items wait for A
    need[1][np + p] += unsigned(b->extra_need[p]);  // adjoint C tasks wait for B
  }
  for (int d = 0; d < 2; ++d) {
    for (int l = 0; l < 3; ++l) {
      auto& v = L[d][l];
      std::stable_sort(v.begin(), v.end(), [](const Entry& a, const Entry& c) { return a.first > c.first; });
      std::vector<int4> flat(v.size());
      for (size_t k = 0; k < v.size(); ++k) flat[k] = v[k].second;
      if (int64_t(flat.size()) > b->cap[d][l] || b->list[d][l] == nullptr) {
        void* ptr = nullptr;
        XC_TRY(b->alloc(&ptr, std::max<size_t>(1, flat.size()) * sizeof(int4)));
        b->list[d][l] = static_cast<int4*>(ptr);
        b->cap[d][l] = int64_t(std::max<size_t>(1, flat.size()));
      }
      b->nlist[d][l] = int64_t(flat.size());
      if (!flat.empty())
        XC_CUDA(cudaMemcpy(b->list[d][l], flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    XC_CUDA(cudaMemcpy(b->need[d], need[d].data(), 2 * size_t(np) * sizeof(unsigned), cudaMemcpyHostToDevice));
  }
  for (int d = 0; d < 2; ++d)
    for (int c = 0; c < 3; ++c) {
      auto& v = W[d][c];
      std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& e) { return a.first > e.first; });
      std::vector<int4> flat(v.size());
      for (size_t k = 0; k < v.size(); ++k) flat[k] = v[k].second;
      if (int64_t(flat.size()) > b->wcap[d][c] || b->wlist[d][c] == nullptr) {
        void* ptr = nullptr;
        XC_TRY(b->alloc(&ptr, std::max<size_t>(1, flat.size()) * sizeof(int4)));
        b->wlist[d][c] = static_cast<int4*>(ptr);
        b->wcap[d][c] = int64_t(std::max<size_t>(1, flat.size()));
      }
      b->nw[d][c] = int64_t(flat.size());
      if (!flat.empty())
        XC_CUDA(cudaMemcpy(b->wlist[d][c], flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
  if (int64_t(yts.size()) > b->ycap || b->ylist == nullptr) {
    void* ptr = nullptr;
    XC_TRY(b->alloc(&ptr, std::max<size_t>(1, yts.size()) * sizeof(int2)));
    b->ylist = static_cast<int2*>(ptr);
    b->ycap = int64_t(std::max<size_t>(1, yts.size()));
  }
  b->nyt = int64_t(yts.size());
  if (!yts.empty())
    XC_CUDA(cudaMemcpy(b->ylist, yts.data(), yts.size() * sizeof(int2), cudaMemcpyHostToDevice));
  if (int64_t(tails.size()) > b->tcap || b->tlist == nullptr) {
    void* ptr = nullptr;
    XC_TRY(b->alloc(&ptr, std::max<size_t>(1, tails.size()) * sizeof(int2)));
    b->tlist = static_cast<int2*>(ptr);
    b->tcap = int64_t(std::max<size_t>(1, tails.size()));
  }
  b->ntail = int64_t(tails.size());
  if (!tails.empty())
    XC_CUDA(cudaMemcpy(b->tlist, tails.data(), tails.size() * sizeof(int2), cudaMemcpyHostToDevice));
  for (int d = 0; d < 2; ++d)
    if (b->tens_plans[d] > 0) {
      if (b->dwin[d] == nullptr) {
        void* ptr = nullptr;
        XC_TRY(b->alloc(&ptr, size_t(np) * sizeof(WinPlan)));
        b->dwin[d] = static_cast<WinPlan*>(ptr);
      }
      XC_CUDA(cudaMemcpy(b->dwin[d], b->hwin[d].data(), size_t(np) * sizeof(WinPlan), cudaMemcpyHostToDevice));
    }
  XC_CUDA(cudaMemcpy(b->dplans, b->host.data(), size_t(np) * sizeof(BatchPlanDev), cudaMemcpyHostToDevice));
  b->rpw[0] = rpw_f;
  b->rpw[1] = rpw_a;
  b->lock[0] = lock_f;
  b->lock[1] = lock_a;
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
  // every CTA is resident (the waits rely on it); no more CTAs than the work needs
  const int64_t work = std::max<int64_t>({b->nlist[dir][0], (b->nlist[dir][1] + kBatchWarps - 1) / kBatchWarps,
                                          b->nlist[dir][2], int64_t(1)});
  const int64_t grid = std::min<int64_t>(int64_t(sms) * per_sm, work);
  count_launch();
  fn<<<unsigned(grid), kBatchThreads, b->smem, st>>>(b->dplans, b->list[dir][0], b->nlist[dir][0], b->list[dir][1],
                                                      b->nlist[dir][1], b->list[dir][2], b->nlist[dir][2],
                                                      dir == 0 ? 1 : 0, b->ctrl, b->need[dir], b->done,
                                                      int(b->plans.size()), b->wait_limit, b->ring ? 1 : 0);
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

template <int NP, bool ADJ>
int launch_window(Batch* b, int cls, cudaStream_t st) {
  using C = WinCfg<NP>;
  auto fn = tc_window_kernel<NP, ADJ>;
  const int d = ADJ ? 1 : 0;
  // one CTA per SM: each allocates all of the SM's tensor memory
  const int smem = std::max(C::SMEM, 116 * 1024);
  XC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int dev = 0, sms = 0;
  XC_CUDA(cudaGetDevice(&dev));
  XC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t grid = std::min<int64_t>(sms, b->nw[d][cls]);
  count_launch();
  fn<<<unsigned(grid), kWinThreads, smem, st>>>(b->dwin[d], b->wlist[d][cls], int(b->nw[d][cls]),
                                                &b->ctrl[C_STATUS]);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

template <bool ADJ>
int launch_windows(Batch* b, cudaStream_t st) {
  const int d = ADJ ? 1 : 0;
  if (b->nw[d][0] > 0) XC_TRY((launch_window<16, ADJ>(b, 0, st)));
  if (b->nw[d][1] > 0) XC_TRY((launch_window<32, ADJ>(b, 1, st)));
  if (b->nw[d][2] > 0) XC_TRY((launch_window<64, ADJ>(b, 2, st)));
  return XC_OK;
}

int launch_batch(Batch* b, int dir, cudaStream_t st) {
  // adjoint band products of the tensor plans first: their row-scaled
  // right-hand sides, then the window products, whose partials the inverse
  // FFTs of the persistent launch read
  if (dir == 1 && b->tens_plans[1] > 0) {
    if (b->nyt > 0) {
      count_launch();
      adj_yt_kernel<<<unsigned(std::min<int64_t>((b->nyt + 7) / 8, 4096)), 256, 0, st>>>(b->dwin[1], b->ylist,
                                                                                      b->nyt);
      XC_CUDA(cudaGetLastError());
    }
    XC_TRY(launch_windows<true>(b, st));
  }
  if (b->entries(dir) > 0) {
    switch (b->precision) {
      case XC_FP64: XC_TRY((launch_batch_t<double, false>(b, dir, st))); break;
      case XC_FP32: XC_TRY((launch_batch_t<float, false>(b, dir, st))); break;
      default: XC_TRY((launch_batch_t<float, true>(b, dir, st))); break;
    }
  }
  // forward band products of the tensor plans, after their FFTs (and their
  // dense tails, which the window epilogue adds)
  if (dir == 0 && b->tens_plans[0] > 0) {
    if (b->ntail > 0) {
      count_launch();
      fwd_tail_kernel<<<unsigned(std::min<int64_t>((b->ntail + 7) / 8, 4096)), 256, 0, st>>>(b->dplans, b->tlist,
                                                                                          b->ntail);
      XC_CUDA(cudaGetLastError());
    }
    XC_TRY(launch_windows<false>(b, st));
  }
  return XC_OK;
}

// Tuning cache: batch signature -> chosen (right-hand sides per item, lockstep
// items on) per direction: {rpw_f, rpw_a, lock_f, lock_a}.
std::mutex g_tune_mutex;
std::map<std::string, std::array<int, 4>> g_tune_cache;

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
    if (p->max_csize > 1) {
      delete b;
      return fail(XC_ERR_UNSUPPORTED, "plan " + std::to_string(i) + " has blocks whose FFT needs a CTA cluster");
    }
    if (p->precision == XC_FP64_PAIR) {
      delete b;
      return fail(XC_ERR_UNSUPPORTED, "batches take XC_FP64, XC_FP32 or XC_FP32_COMPENSATED plans");
    }
    if (p->cplx || p->d2) {
      delete b;
      return fail(XC_ERR_UNSUPPORTED, "plan " + std::to_string(i) + ": batches take real 1-D plans");
    }
    if (i > 0 && p->precision != b->precision) {
      delete b;
      return fail(XC_ERR_ARG, "all plans of a batch need the same precision");
    }
    if (std::find(b->plans.begin(), b->plans.end(), p) != b->plans.end()) {
      delete b;   // two entries would share the plan's scratch
      return fail(XC_ERR_ARG, "plan " + std::to_string(i) + " appears twice in the batch");
    }
    b->precision = p->precision;
    b->plans.push_back(p);
    b->max_n = std::max(b->max_n, p->max_n);
  }
  b->smem = size_t(b->max_n) * 2 * (b->precision == XC_FP64 ? 8 : 4);
  // FP32 batches: room for every warp's staging ring of the lockstep items
  b->ring = b->precision != XC_FP64;
  if (b->ring) b->smem = std::max(b->smem, size_t(xc::kBatchWarps) * size_t(xc::kRingBytes));
  std::fill(&b->tune_ms[0][0], &b->tune_ms[0][0] + 2 * 12, -1.f);
  b->extra_need.assign(nplans, 0);
  b->lscratch.assign(nplans, nullptr);
  b->ytbuf.assign(nplans, nullptr);
  b->ytbuf_bytes.assign(nplans, 0);
  b->lscratch_bytes.assign(nplans, 0);
  void* ptr = nullptr;
  int rc = b->alloc(&ptr, xc::C_WORDS * sizeof(unsigned));
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
    if (cudaMemset(b->ctrl, 0, xc::C_WORDS * sizeof(unsigned)) != cudaSuccess ||
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
  // every argument is checked before the batch changes: a refused bind
  // leaves the previous binding in force
  for (int i = 0; i < np; ++i) {
    const xc::Plan* p = b->plans[i];
    if (nrhs[i] < 0 || nrhs[i] > (int64_t(1) << 24)) return fail(XC_ERR_ARG, "nrhs out of range");
    if (nrhs[i] > 0 && (!x_dev[i] || !y_dev[i] || x_dev[i] == y_dev[i] || ld[i] < p->N))
      return fail(XC_ERR_ARG, "bad buffers for plan " + std::to_string(i));
  }
  for (int i = 0; i < np; ++i) XC_TRY(xc::ensure_scratch_kept(b->plans[i], std::max<int64_t>(1, nrhs[i])));
  if (!b->holds_refs) {
    for (xc::Plan* p : b->plans) ++p->batch_refs;
    b->holds_refs = true;
  }
  // lockstep layouts and the batch's lockstep scratch (FP32 plans: the FP64
  // band products are bound by the FP64 pipe, where the windows' stored
  // zeros would only add work)
  for (int i = 0; i < np; ++i) {
    xc::Plan* p = b->plans[i];
    if (b->precision == XC_FP64 || nrhs[i] == 0) continue;
    XC_TRY(xc::ensure_lockstep(p));
    if (!p->lock_f_ok && !p->lock_t_ok && !p->tens_ok && !p->tens_t_ok) continue;
    const int64_t rp = (nrhs[i] + 7) / 8 * 8;
    // forward: bin-major spectra, the lockstep unit partials, and 16 bins
    // of zeros past the spectra (a tensor window's last tile may reach 15
    // bins past its block's spectrum)
    const int64_t fwd = p->lock_f_ok || p->tens_ok
                            ? p->spec_per_rhs * rp + p->lk_total_units * 32 * nrhs[i] + xc::kWinBins * rp
                            : 0;
    // adjoint: the chunk partials (lockstep chunks, or one per bin slice)
    const int64_t adj = p->lock_t_ok || p->tens_t_ok
                            ? std::max<int64_t>(p->lk_total_chunks, p->total_tslices) * 32 * nrhs[i]
                            : 0;
    const int64_t bytes = std::max<int64_t>(fwd, adj) * int64_t(sizeof(xc::cx<float>));
    if (b->lscratch[i] == nullptr || b->lscratch_bytes[i] < bytes) {
      void* ptr = nullptr;
      XC_TRY(b->alloc(&ptr, size_t(bytes)));   // kept until the batch goes (a launch may still use the old one)
      XC_CUDA(cudaMemset(ptr, 0, size_t(bytes)));   // the pad column of odd nrhs stays zero
      b->lscratch[i] = ptr;
      b->lscratch_bytes[i] = bytes;
    }
    if (p->tens_t_ok && nrhs[i] <= 64) {
      // row-scaled right-hand sides of the adjoint windows, [N + 32][rp]: a
      // window's last tile may reach 31 rows past N (zeros)
      const int64_t ybytes = (p->N + 32) * rp * int64_t(sizeof(float));
      if (b->ytbuf[i] == nullptr || b->ytbuf_bytes[i] < ybytes) {
        void* ptr = nullptr;
        XC_TRY(b->alloc(&ptr, size_t(ybytes)));
        XC_CUDA(cudaMemset(ptr, 0, size_t(ybytes)));
        b->ytbuf[i] = ptr;
        b->ytbuf_bytes[i] = ybytes;
      }
    }
  }
  std::vector<xc::BatchPlanDev>& host = b->host;
  host.assign(np, xc::BatchPlanDev{});
  for (int i = 0; i < np; ++i) {
    xc::Plan* p = b->plans[i];
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
    d.rp = int((nrhs[i] + 7) / 8 * 8);
    // rows per lane: 8 RL right-hand sides per item (FP32 up to 4; two with
    // compensation, whose accumulators take twice the registers)
    d.rl = nrhs[i] > 16 && b->precision == XC_FP32 ? 4 : nrhs[i] > 8 ? 2 : 1;
    d.lscratch = b->lscratch[i];
    d.lk_units = p->lk_units;
    d.lk_ubase = p->lk_ubase;
    d.lk_items = p->lk_items;
    d.lk_cbase = p->lk_cbase;
  }
  b->x.assign(x_dev, x_dev + np);
  b->y.assign(y_dev, y_dev + np);
  b->nrhs.assign(nrhs, nrhs + np);
  b->ld.assign(ld, ld + np);
  const int dflt = b->precision == XC_FP64 ? 2 : 8;
  std::array<int, 4> cfg{b->rpw[0] > 0 ? b->rpw[0] : dflt, b->rpw[1] > 0 ? b->rpw[1] : dflt, b->lock[0], b->lock[1]};
  {
    std::lock_guard<std::mutex> lock(xc::g_tune_mutex);
    auto it = xc::g_tune_cache.find(xc::signature(b));
    if (it != xc::g_tune_cache.end()) cfg = it->second;
  }
  return xc::build_tasks(b, cfg[0], cfg[1], cfg[2], cfg[3]);
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
  int best_lock[2] = {b->lock[0], b->lock[1]};
  float best_ms[2] = {1e30f, 1e30f};
  bool any_lock = false, any_tens = false;
  for (size_t p = 0; p < b->plans.size(); ++p) {
    any_lock = any_lock || b->lscratch[p] != nullptr;
    any_tens = any_tens || xc::tensor_capable(b, int(p)) || xc::tensor_t_capable(b, int(p));
  }
  // lockstep 2: tensor windows forward (lockstep items in the adjoint)
  for (int lk = any_tens ? 2 : any_lock ? 1 : 0; lk >= 0; --lk)
  for (int cand : {1, 2, 4, 8}) {
    XC_TRY(xc::build_tasks(b, cand, cand, lk, lk));
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
    const int slot = 4 * lk + (cand == 1 ? 0 : cand == 2 ? 1 : cand == 4 ? 2 : 3);
    for (int d = 0; d < 2; ++d) b->tune_ms[d][slot] = ms[d];
    for (int d = 0; d < 2; ++d)
      if (ms[d] < best_ms[d]) {
        best_ms[d] = ms[d];
        best[d] = cand;
        best_lock[d] = lk;
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
  XC_TRY(xc::build_tasks(b, best[0], best[1], best_lock[0], best_lock[1]));
  b->tuned = true;
  std::lock_guard<std::mutex> lock(xc::g_tune_mutex);
  xc::g_tune_cache[xc::signature(b)] = {best[0], best[1], best_lock[0], best_lock[1]};
  return XC_OK;
}

int xc_batch_schedule(xc_batch_t batch, int rpw_forward, int rpw_adjoint, int lockstep_forward,
                      int lockstep_adjoint) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b) return fail(XC_ERR_ARG, "batch is NULL");
  if (b->rpw[0] == 0) return fail(XC_ERR_ARG, "bind the batch's buffers first");
  for (int r : {rpw_forward, rpw_adjoint})
    if (r != 1 && r != 2 && r != 4 && r != 8) return fail(XC_ERR_ARG, "right-hand sides per item: 1, 2, 4 or 8");
  return xc::build_tasks(b, rpw_forward, rpw_adjoint, lockstep_forward == 2 ? 2 : lockstep_forward ? 1 : 0,
                         lockstep_adjoint == 2 ? 2 : lockstep_adjoint ? 1 : 0);
}

int xc_batch_info(xc_batch_t batch, xc_batch_stats* out) {
  auto* b = reinterpret_cast<xc::Batch*>(batch);
  if (!b || !out) return fail(XC_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->nplans = int(b->plans.size());
  out->rhs_per_item = b->rpw[0];
  out->rhs_per_item_adjoint = b->rpw[1];
  out->tuned = b->tuned ? 1 : 0;
  out->tasks_forward = b->entries(0);
  out->tasks_adjoint = b->entries(1);
  out->lockstep_forward = b->lock[0];
  out->lockstep_adjoint = b->lock[1];
  for (int k = 0; k < 12; ++k) {
    out->tune_ms_forward[k] = b->tune_ms[0][k];
    out->tune_ms_adjoint[k] = b->tune_ms[1][k];
  }
  out->tensor_plans = b->tens_plans[0];
  out->tensor_plans_adjoint = b->tens_plans[1];
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (i < b->host.size() && (b->host[i].lock_f || b->host[i].lock_a)) ++out->lockstep_plans;
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
  XC_CUDA(cudaMemcpyAsync(&status, &b->ctrl[xc::C_STATUS], sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  XC_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    XC_CUDA(cudaMemsetAsync(&b->ctrl[xc::C_STATUS], 0, sizeof(unsigned), st));
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
  if (b->rpw[0] > 0) return xc::build_tasks(b, b->rpw[0], b->rpw[1], b->lock[0], b->lock[1]);
  return XC_OK;
}

int xc_batch_destroy(xc_batch_t batch) {
  delete reinterpret_cast<xc::Batch*>(batch);
  return XC_OK;
}

}  // extern "C"
