// Execution stage (the hot path) of Algorithms 1-4: the single-plan kernels
// and their launches (device bodies in xc_items.cuh).
//
// Forward, y = A x (Algorithm 1 step 2 / Algorithm 3):
//   fwd_fft_kernel     per (block, RHS): extend the input with zero extra
//                      components (eqs. (Fe1), (Fe3)), multiply by W^{-1},
//                      real FFT -> half spectrum F_k = sum_j u_j exp(-2 pi i jk/L)
//   fwd_sparse_kernel  per (32-row slice, RHS group): y_n = sum over blocks of
//                      sum_k Re(C_nk conj(F_k)) over the row's band, plus the
//                      dense tail; C = g_k A_e W F / sqrt(L) is stored with the
//                      unitary and half-spectrum factors folded in, so that
//                      Re(C conj F) = Re C Re F + Im C Im F.
// Adjoint, x = A^T y (Algorithm 2 step 2 / Algorithm 4):
//   adj_sparse_kernel  per (32-bin slice, RHS group): z_k = sum_n CT_kn y_n
//   adj_fft_kernel     per (block, RHS): real inverse FFT of z, W^{-1}, keep the
//                      real components [j_lo, j_hi), discard the extra ones (eq. (Fe2))
//   adj_tail_kernel    the first m_tail entries from the dense tail.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "xc_fft.cuh"
#include "xc_internal.h"
#include "xc_items.cuh"

namespace xc {

namespace {

constexpr int kFftThreads = 256;
constexpr int kSparseWarps = 4;

// ------------------------------------------------------------ forward FFT
// (pexp: per-RHS exponents of FP32-pair plans, whose spectra go out as pairs)
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    fwd_fft_kernel(const BlockDev* __restrict__ blocks, const T* __restrict__ x, int64_t ld,
                   const T* __restrict__ colscale, cx<T>* __restrict__ spec, int64_t nrhs,
                   const int* __restrict__ pexp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fwd_fft_body<T>(blocks[blockIdx.y], blockIdx.x, x, ld, colscale, spec, nrhs, reinterpret_cast<cx<T>*>(smem_raw),
                  threadIdx.x, blockDim.x, pexp);
}

// The same for one block whose n-point array is split over a cluster of
// csize CTAs (rank q holds [q n/csize, (q+1) n/csize)); butterflies reach the
// other parts through distributed shared memory, a cluster barrier separates
// the passes.  Grid: nrhs * csize CTAs, cluster dimension (csize, 1, 1).
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    fwd_fft_cluster_kernel(const BlockDev* __restrict__ block, const T* __restrict__ x, int64_t ld,
                           const T* __restrict__ colscale, cx<T>* __restrict__ spec, int64_t nrhs,
                           const int* __restrict__ pexp) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int csize = int(cluster.num_blocks());
  const int rank = int(cluster.block_rank());
  const BlockDev& b = *block;
  ClusterMem<T> mem;
  mem.per = b.n / csize;
  for (int q = 0; q < 8; ++q) mem.base[q] = q < csize ? cluster.map_shared_rank(s, q) : s;
  cluster.sync();   // every CTA of the cluster runs before any remote access
  fwd_fft_run<T>(b, blockIdx.x / csize, x, ld, colscale, spec, nrhs, mem, rank * int(blockDim.x) + int(threadIdx.x),
                 csize * int(blockDim.x), [&] { cluster.sync(); }, pexp);
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------- work distribution
// The sparse kernels run a persistent grid (every CTA resident).  Each warp
// takes items -- (slice, group of RPW right-hand sides) -- from a device
// counter, longest slices first, until the list is exhausted; the last warp to
// finish resets the counter pair for the next launch.  This keeps all SMs busy
// to the end even though band widths differ from slice to slice.
__device__ __forceinline__ int64_t take_item(unsigned* next, int lane) {
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(next, 1u);
  return int64_t(__shfl_sync(0xffffffffu, t, 0));
}

__device__ __forceinline__ void retire_warp(unsigned* next, unsigned* done, unsigned total_warps, int lane) {
  if (lane == 0) {
    __threadfence();                              // this warp's last take precedes its retirement
    if (atomicAdd(done, 1u) == total_warps - 1) {
      atomicExch(next, 0u);
      atomicExch(done, 0u);
    }
  }
}

// ------------------------------------------------------- forward sparse
template <typename T, int RPW, bool COMP>
__global__ void __launch_bounds__(32 * kSparseWarps)
    fwd_sparse_kernel(const BlockDev* __restrict__ blocks, int nblocks, int64_t N, const T* __restrict__ x,
                      int64_t ld, T* __restrict__ y, const cx<T>* __restrict__ spec, int64_t nrhs,
                      const T* __restrict__ rowscale, const T* __restrict__ colscale, const T* __restrict__ tail,
                      int64_t m_tail, const int* __restrict__ order, unsigned* counters, int sg) {
  // item = (slice, supergroup of sg groups of RPW right-hand sides)
  const int lane = threadIdx.x & 31;
  const int64_t nsup = ((nrhs + RPW - 1) / RPW + sg - 1) / sg;
  const int64_t total = ((N + 31) / 32) * nsup;
  for (;;) {
    const int64_t t = take_item(&counters[0], lane);
    if (t >= total) break;
    fwd_sparse_item<T, RPW, COMP>(blocks, nblocks, N, x, ld, y, spec, nrhs, rowscale, colscale, tail, m_tail,
                                  order[t / nsup], (t % nsup) * int64_t(sg) * RPW, lane, sg);
  }
  retire_warp(&counters[0], &counters[1], gridDim.x * kSparseWarps, lane);
}

// Chunked forward (plans with long bands): item = (unit, supergroup).
template <typename T, int RPW, bool COMP>
__global__ void __launch_bounds__(32 * kSparseWarps)
    fwd_unit_kernel(const BlockDev* __restrict__ blocks, const cx<T>* __restrict__ spec, int64_t nrhs,
                    cx<T>* __restrict__ part, const int4* __restrict__ units, const int* __restrict__ order,
                    int64_t total_units, unsigned* counters, int sg) {
  const int lane = threadIdx.x & 31;
  const int64_t nsup = ((nrhs + RPW - 1) / RPW + sg - 1) / sg;
  const int64_t total = total_units * nsup;
  for (;;) {
    const int64_t t = take_item(&counters[0], lane);
    if (t >= total) break;
    const int u = order[t / nsup];
    fwd_unit_item<T, RPW, COMP>(blocks, spec, nrhs, part, units[u], u, (t % nsup) * int64_t(sg) * RPW, lane, sg);
  }
  retire_warp(&counters[0], &counters[1], gridDim.x * kSparseWarps, lane);
}

// Thread per (row, RHS); grid.y strides over the right-hand sides.
template <typename T, bool COMP>
__global__ void fwd_reduce_kernel(int64_t N, const T* __restrict__ x, int64_t ld, T* __restrict__ y,
                                  const cx<T>* __restrict__ part, int64_t nrhs, const int* __restrict__ ubase,
                                  const T* __restrict__ rowscale, const T* __restrict__ colscale,
                                  const T* __restrict__ tail, int64_t m_tail) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  for (int64_t r = blockIdx.y; r < nrhs; r += gridDim.y)
    fwd_reduce_row<T, COMP>(N, x, ld, y, part, nrhs, ubase, rowscale, colscale, tail, m_tail, n, r);
}

// ------------------------------------------------------- adjoint sparse
// Chunking keeps bins that are covered by thousands of rows (the small last
// blocks, high frequencies of the Laguerre functions) from becoming one long
// serial loop; the adjoint FFT adds the chunks of each bin in chunk order
// (deterministic, no atomics).
template <typename T, int RPW, bool COMP, bool YT>
__global__ void __launch_bounds__(32 * kSparseWarps)
    adj_sparse_kernel(const BlockDev* __restrict__ blocks, int nblocks, int64_t N, const T* __restrict__ y,
                      int64_t ld, const T* __restrict__ yt, int64_t ldt, cx<T>* __restrict__ part, int64_t nrhs, const T* __restrict__ rowscale,
                      const int2* __restrict__ items, const int* __restrict__ cbase, int64_t total_chunks,
                      int chunk, unsigned* counters, int sg) {
  (void)N;
  const int lane = threadIdx.x & 31;
  const int64_t nsup = ((nrhs + RPW - 1) / RPW + sg - 1) / sg;
  const int64_t total = total_chunks * nsup;
  for (;;) {
    const int64_t t = take_item(&counters[2], lane);
    if (t >= total) break;
    adj_sparse_item<T, RPW, COMP, YT, true>(blocks, nblocks, y, ld, yt, ldt, part, nrhs, rowscale, cbase,
                                      items[t / nsup], chunk, (t % nsup) * int64_t(sg) * RPW, lane, sg);
  }
  retire_warp(&counters[2], &counters[3], gridDim.x * kSparseWarps, lane);
}

// ------------------------------------------------ FP64 plans in FP32 pairs
// Per right-hand side r: e[r] = the binary exponent of max_n |v[r][n] rs[n]|
// (0 for a zero vector), so that v 2^-e[r] lies below 1 in magnitude; with
// `out`, also out[r][n] = pair(v[r][n] rs[n] 2^-e[r]).  One CTA per RHS.
__global__ void __launch_bounds__(256)
    pair_scale_kernel(const double* __restrict__ v, int64_t ld, int64_t N, const double* __restrict__ rs,
                      int* __restrict__ e, float2* __restrict__ out) {
  __shared__ double red[8];
  __shared__ int s_e;
  const int64_t r = blockIdx.x;
  const double* __restrict__ vr = v + r * ld;
  double m = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) m = fmax(m, fabs(vr[n] * (rs ? rs[n] : 1.0)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) mm = fmax(mm, red[i]);
    int ex = 0;
    if (mm > 0.0) frexp(mm, &ex);
    s_e = ex;
    e[r] = ex;
  }
  __syncthreads();
  if (out) {
    const int ex = -s_e;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) out[r * N + n] = to_pair(ldexp(vr[n] * (rs ? rs[n] : 1.0), ex));
  }
}

template <int RPW>
__global__ void __launch_bounds__(32 * kSparseWarps)
    fwd_sparse_pair_kernel(const BlockDev* __restrict__ blocks, int nblocks, int64_t N, const double* __restrict__ x,
                           int64_t ld, double* __restrict__ y, const PairCx* __restrict__ spec, int64_t nrhs,
                           const int* __restrict__ pexp, const double* __restrict__ rowscale,
                           const double* __restrict__ colscale, const double* __restrict__ tail, int64_t m_tail,
                           const int* __restrict__ order, unsigned* counters, int sg) {
  const int lane = threadIdx.x & 31;
  const int64_t nsup = ((nrhs + RPW - 1) / RPW + sg - 1) / sg;
  const int64_t total = ((N + 31) / 32) * nsup;
  for (;;) {
    const int64_t t = take_item(&counters[0], lane);
    if (t >= total) break;
    fwd_sparse_item_pair<RPW>(blocks, nblocks, N, x, ld, y, spec, nrhs, pexp, rowscale, colscale, tail, m_tail,
                              order[t / nsup], (t % nsup) * int64_t(sg) * RPW, lane, sg);
  }
  retire_warp(&counters[0], &counters[1], gridDim.x * kSparseWarps, lane);
}

template <int RPW>
__global__ void __launch_bounds__(32 * kSparseWarps)
    fwd_unit_pair_kernel(const BlockDev* __restrict__ blocks, const PairCx* __restrict__ spec, int64_t nrhs,
                         const int* __restrict__ pexp, cx<double>* __restrict__ part, const int4* __restrict__ units,
                         const int* __restrict__ order, int64_t total_units, unsigned* counters, int sg) {
  const int lane = threadIdx.x & 31;
  const int64_t nsup = ((nrhs + RPW - 1) / RPW + sg - 1) / sg;
  const int64_t total = total_units * nsup;
  for (;;) {
    const int64_t t = take_item(&counters[0], lane);
    if (t >= total) break;
    const int u = order[t / nsup];
    fwd_unit_item_pair<RPW>(blocks, spec, nrhs, pexp, part, units[u], u, (t % nsup) * int64_t(sg) * RPW, lane, sg);
  }
  retire_warp(&counters[0], &counters[1], gridDim.x * kSparseWarps, lane);
}

template <int RPW>
__global__ void __launch_bounds__(32 * kSparseWarps)
    adj_sparse_pair_kernel(const BlockDev* __restrict__ blocks, int nblocks, int64_t N,
                           const float2* __restrict__ yp, const int* __restrict__ pexp, cx<double>* __restrict__ part,
                           int64_t nrhs, const int2* __restrict__ items, const int* __restrict__ cbase,
                           int64_t total_chunks, int chunk, unsigned* counters, int sg) {
  const int lane = threadIdx.x & 31;
  const int64_t nsup = ((nrhs + RPW - 1) / RPW + sg - 1) / sg;
  const int64_t total = total_chunks * nsup;
  for (;;) {
    const int64_t t = take_item(&counters[2], lane);
    if (t >= total) break;
    adj_sparse_item_pair<RPW>(blocks, nblocks, yp, N, pexp, part, nrhs, cbase, items[t / nsup], chunk,
                              (t % nsup) * int64_t(sg) * RPW, lane, sg);
  }
  retire_warp(&counters[2], &counters[3], gridDim.x * kSparseWarps, lane);
}

// y [nrhs][ld] -> yt [N][ldt] (zero columns beyond nrhs).
template <typename T>
__global__ void __launch_bounds__(256)
    transpose_kernel(const T* __restrict__ y, int64_t ld, int64_t N, int64_t nrhs, T* __restrict__ yt, int64_t ldt) {
  __shared__ T tile[32][33];
  for (int64_t rb = blockIdx.y; rb * 32 < ldt; rb += gridDim.y) {
    transpose_tile<T>(y, ld, N, nrhs, yt, ldt, int64_t(blockIdx.x) * 32, rb * 32, tile, threadIdx.x, threadIdx.y);
    __syncthreads();                       // the tile is refilled next
  }
}

// Resident CTAs of kSparseWarps warps per SM for a kernel, and the SM count:
// queried once per kernel and host thread (the queries cost microseconds,
// which small applies would otherwise pay at every launch).
int resident_ctas(const void* fn, int* per_sm, int* sms) {
  static thread_local int cached_sms = 0;
  static thread_local std::unordered_map<const void*, int> cache;
  if (cached_sms == 0) {
    int dev = 0;
    XC_CUDA(cudaGetDevice(&dev));
    XC_CUDA(cudaDeviceGetAttribute(&cached_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  auto it = cache.find(fn);
  if (it == cache.end()) {
    int n = 0;
    XC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * kSparseWarps, 0));
    it = cache.emplace(fn, n < 1 ? 1 : n).first;
  }
  *per_sm = it->second;
  *sms = cached_sms;
  return XC_OK;
}

// Persistent grid: as many CTAs as can be resident, but no more than the
// items need.  Every resident warp takes part (warps that find the list empty
// retire at once); the dynamic schedule balances SMs and their schedulers.
// With many items a warp is meant to take about items_per_warp of them; with
// few, every item gets a warp of its own.
int persistent_grid(const void* fn, int64_t items, unsigned* grid, int items_per_warp = 1) {
  int per_sm = 1, sms = 1;
  XC_TRY(resident_ctas(fn, &per_sm, &sms));
  const int64_t resident = int64_t(sms) * per_sm;
  if (items < resident * kSparseWarps * items_per_warp) items_per_warp = 1;
  const int64_t per_cta = int64_t(kSparseWarps) * items_per_warp;
  const int64_t need = (items + per_cta - 1) / per_cta;
  *grid = unsigned(std::min<int64_t>(resident, std::max<int64_t>(1, need)));
  return XC_OK;
}

// ------------------------------------------------------------ adjoint FFT
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    adj_fft_kernel(const BlockDev* __restrict__ blocks, const cx<T>* __restrict__ part, const int* __restrict__ cbase,
                   int64_t nrhs, T* __restrict__ x, int64_t ld, const T* __restrict__ colscale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  adj_fft_body<T>(blocks[blockIdx.y], blockIdx.x, part, cbase, nrhs, x, ld, colscale,
                  reinterpret_cast<cx<T>*>(smem_raw), threadIdx.x, blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    adj_fft_cluster_kernel(const BlockDev* __restrict__ block, const cx<T>* __restrict__ part,
                           const int* __restrict__ cbase, int64_t nrhs, T* __restrict__ x, int64_t ld,
                           const T* __restrict__ colscale) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int csize = int(cluster.num_blocks());
  const int rank = int(cluster.block_rank());
  const BlockDev& b = *block;
  ClusterMem<T> mem;
  mem.per = b.n / csize;
  for (int q = 0; q < 8; ++q) mem.base[q] = q < csize ? cluster.map_shared_rank(s, q) : s;
  cluster.sync();
  adj_fft_run<T>(b, blockIdx.x / csize, part, cbase, nrhs, x, ld, colscale, mem,
                 rank * int(blockDim.x) + int(threadIdx.x), csize * int(blockDim.x), [&] { cluster.sync(); });
  cluster.sync();
}

// ------------------------------------------------------------ adjoint tail
// Warp per (m, RHS).
template <typename T, bool COMP>
__global__ void adj_tail_kernel(int64_t N, int64_t m_tail, const T* __restrict__ tail, const T* __restrict__ y,
                                int64_t ld, T* __restrict__ x, const T* __restrict__ rowscale,
                                const T* __restrict__ colscale) {
  const int64_t m = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= m_tail) return;
  adj_tail_warp<T, COMP>(N, m, blockIdx.y, tail, y, ld, x, rowscale, colscale, threadIdx.x & 31);
}

// Right-hand-side groups per item: enough items for ~4 per resident warp,
// and no more groups per item than that, so that short bands (FP32 plans,
// small blocks) amortise each item's bookkeeping over several groups.
int supergroup(const void* fn, int64_t units, int64_t ngroups) {
  int per_sm = 1, sms = 1;
  if (resident_ctas(fn, &per_sm, &sms) != XC_OK) {
    cudaGetLastError();
    return 1;
  }
  const int64_t warps = int64_t(sms) * per_sm * kSparseWarps;
  const int64_t want_items = 4 * warps;
  const int64_t have = std::max<int64_t>(1, units * ngroups);
  if (have <= want_items) return 1;
  return int(std::min<int64_t>(ngroups, (have + want_items - 1) / want_items));
}

// ------------------------------------------------------------------ launch
template <typename T>
int set_dynamic_smem(const void* fn, size_t smem) {
  static thread_local std::unordered_map<const void*, size_t> configured;
  size_t& done = configured[fn];
  if (smem > 48 * 1024 && smem > done) {
    XC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    done = smem;
  }
  return XC_OK;
}

// The FFTs of all blocks (forward: input -> spectra; adjoint: chunk partials
// -> output).  One launch over (RHS, block) when every block fits one CTA;
// otherwise one launch per block, clusters for the long ones.
template <typename T>
int launch_fft(Plan* p, bool forward, const void* in, void* out, int64_t nrhs, int64_t ld, cudaStream_t st,
               const int* pexp = nullptr) {
  const BlockDev* bd = static_cast<const BlockDev*>(p->scratch_desc);
  const int kid = forward ? K_FWD_FFT : K_ADJ_FFT;
  const T* cs = static_cast<const T*>(p->colscale);
  auto one_cta = [&](const BlockDev* d, unsigned nb, size_t smem) -> int {
    dim3 grid(unsigned(nrhs), nb);
    if (forward) {
      XC_TRY(set_dynamic_smem<T>(reinterpret_cast<const void*>(fwd_fft_kernel<T>), smem));
      fwd_fft_kernel<T><<<grid, kFftThreads, smem, st>>>(d, static_cast<const T*>(in), ld, cs,
                                                          static_cast<cx<T>*>(out), nrhs, pexp);
    } else {
      XC_TRY(set_dynamic_smem<T>(reinterpret_cast<const void*>(adj_fft_kernel<T>), smem));
      adj_fft_kernel<T><<<grid, kFftThreads, smem, st>>>(d, static_cast<const cx<T>*>(in), p->s_cbase, nrhs,
                                                          static_cast<T*>(out), ld, cs);
    }
    XC_CUDA(cudaGetLastError());
    return XC_OK;
  };
  launch_begin(p, kid, st);
  if (p->max_csize == 1) {
    XC_TRY(one_cta(bd, unsigned(p->blocks.size()), size_t(p->max_n) * sizeof(cx<T>)));
  } else {
    for (size_t i = 0; i < p->blocks.size(); ++i) {
      const BlockDev& b = p->blocks[i];
      if (b.a_csize == 1) {
        XC_TRY(one_cta(bd + i, 1u, size_t(b.n) * sizeof(cx<T>)));
        continue;
      }
      const size_t smem = size_t(b.n / b.a_csize) * sizeof(cx<T>);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(nrhs * b.a_csize));
      cfg.blockDim = dim3(kFftThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = unsigned(b.a_csize);
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (forward) {
        XC_TRY(set_dynamic_smem<T>(reinterpret_cast<const void*>(fwd_fft_cluster_kernel<T>), smem));
        XC_CUDA(cudaLaunchKernelEx(&cfg, fwd_fft_cluster_kernel<T>, bd + i, static_cast<const T*>(in), ld, cs,
                                   static_cast<cx<T>*>(out), nrhs, pexp));
      } else {
        XC_TRY(set_dynamic_smem<T>(reinterpret_cast<const void*>(adj_fft_cluster_kernel<T>), smem));
        XC_CUDA(cudaLaunchKernelEx(&cfg, adj_fft_cluster_kernel<T>, bd + i, static_cast<const cx<T>*>(in),
                                   static_cast<const int*>(p->s_cbase), nrhs, static_cast<T*>(out), ld, cs));
      }
    }
  }
  launch_end(p, kid, st);
  return XC_OK;
}

template <typename T, bool COMP, int RPW>
int launch_sparse_fwd_rpw(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const void* fn = reinterpret_cast<const void*>(fwd_sparse_kernel<T, RPW, COMP>);
  unsigned grid = 1;
  // forward items cannot be split along the band, so each warp should see
  // several of them for the dynamic schedule to balance the tail
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  const int sg = supergroup(fn, p->nslices, ngroups);
  XC_TRY(persistent_grid(fn, p->nslices * ((ngroups + sg - 1) / sg), &grid, 4));
  launch_begin(p, K_FWD_SPARSE, st);
  fwd_sparse_kernel<T, RPW, COMP><<<grid, 32 * kSparseWarps, 0, st>>>(
      static_cast<const BlockDev*>(p->scratch_desc), int(p->blocks.size()), p->N, static_cast<const T*>(x), ld,
      static_cast<T*>(y), static_cast<const cx<T>*>(p->scratch), nrhs, static_cast<const T*>(p->rowscale),
      static_cast<const T*>(p->colscale), static_cast<const T*>(p->tail), p->m_tail, p->f_order, p->counters, sg);
  launch_end(p, K_FWD_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

template <typename T, bool COMP, int RPW>
int launch_unit_fwd_rpw(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const void* fn = reinterpret_cast<const void*>(fwd_unit_kernel<T, RPW, COMP>);
  unsigned grid = 1;
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  const int sg = supergroup(fn, p->total_units, ngroups);
  XC_TRY(persistent_grid(fn, p->total_units * ((ngroups + sg - 1) / sg), &grid, 4));
  cx<T>* spec = static_cast<cx<T>*>(p->scratch);
  cx<T>* part = spec + p->spec_per_rhs * nrhs;
  launch_begin(p, K_FWD_SPARSE, st);
  fwd_unit_kernel<T, RPW, COMP><<<grid, 32 * kSparseWarps, 0, st>>>(
      static_cast<const BlockDev*>(p->scratch_desc), spec, nrhs, part, p->fu_units, p->fu_order, p->total_units,
      p->counters, sg);
  launch_end(p, K_FWD_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  dim3 rgrid(unsigned((p->N + 255) / 256), unsigned(std::min<int64_t>(nrhs, 65535)));
  launch_begin(p, K_FWD_REDUCE, st);
  fwd_reduce_kernel<T, COMP><<<rgrid, 256, 0, st>>>(p->N, static_cast<const T*>(x), ld, static_cast<T*>(y), part,
                                                    nrhs, p->fu_ubase, static_cast<const T*>(p->rowscale),
                                                    static_cast<const T*>(p->colscale),
                                                    static_cast<const T*>(p->tail), p->m_tail);
  launch_end(p, K_FWD_REDUCE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

template <typename T, bool COMP, int RPW>
int launch_sparse_adj_rpw(Plan* p, const void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  if (p->s_total_chunks == 0) return XC_OK;
  // blocks whose bins start far apart read a transposed copy of y (columns
  // beyond nrhs zero), where a step reads each lane's RPW values of one row
  // as one vector; with fewer than 4 right-hand sides per item the vector
  // is too short to pay for the transposition and for the shorter reuse of
  // each cache line (4 rows per 128-byte line instead of 32)
  const int64_t ldt = yt_ld(nrhs);
  T* yt = nullptr;
  if (p->any_yt && RPW >= 4) {
    yt = reinterpret_cast<T*>(static_cast<cx<T>*>(p->scratch) + p->s_total_chunks * 32 * nrhs);
    launch_begin(p, K_ADJ_TRANSPOSE, st);
    const int64_t rtiles = (ldt + 31) / 32;
    transpose_kernel<T><<<dim3(unsigned((p->N + 31) / 32), unsigned(std::min<int64_t>(rtiles, 65535))), dim3(32, 8),
                          0, st>>>(static_cast<const T*>(y), ld, p->N, nrhs, yt, ldt);
    launch_end(p, K_ADJ_TRANSPOSE, st);
    XC_CUDA(cudaGetLastError());
  }
  const void* fn = reinterpret_cast<const void*>(adj_sparse_kernel<T, RPW, COMP, true>);
  unsigned grid = 1;
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  const int sg = supergroup(fn, p->s_total_chunks, ngroups);
  XC_TRY(persistent_grid(fn, p->s_total_chunks * ((ngroups + sg - 1) / sg), &grid));
  launch_begin(p, K_ADJ_SPARSE, st);
  adj_sparse_kernel<T, RPW, COMP, true><<<grid, 32 * kSparseWarps, 0, st>>>(
      static_cast<const BlockDev*>(p->scratch_desc), int(p->blocks.size()), p->N, static_cast<const T*>(y), ld, yt,
      ldt, static_cast<cx<T>*>(p->scratch), nrhs, static_cast<const T*>(p->rowscale), p->s_items, p->s_cbase,
      p->s_total_chunks, p->s_chunk, p->counters, sg);
  launch_end(p, K_ADJ_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

// Right-hand sides per item.  FP64 is bound by the FP64 pipe, where reusing a
// band value over more right-hand sides buys nothing and finer items balance
// better.  FP32 gains from the reuse, but only while the items still outnumber
// the resident warps about twice: plans with few slices and long bands
// (Hermite and Laguerre functions) otherwise leave most of the GPU idle.
int choose_rpw(int preferred, int64_t units, int64_t nrhs) {
  static thread_local int64_t warps = 0;
  if (warps == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    warps = int64_t(sms) * 32;   // a typical resident count for these kernels
  }
  int r = preferred;
  while (r > 1 && (r > nrhs || units * ((nrhs + r - 1) / r) < 2 * warps)) r /= 2;
  return r;
}

template <typename T, bool COMP>
int launch_sparse_fwd(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const int pref = sizeof(T) == 8 ? 1 : 8;
  if (p->fwd_chunked) {
    switch (choose_rpw(pref, p->total_units, nrhs)) {
      case 8: return launch_unit_fwd_rpw<T, COMP, 8>(p, x, y, nrhs, ld, st);
      case 4: return launch_unit_fwd_rpw<T, COMP, 4>(p, x, y, nrhs, ld, st);
      case 2: return launch_unit_fwd_rpw<T, COMP, 2>(p, x, y, nrhs, ld, st);
      default: return launch_unit_fwd_rpw<T, COMP, 1>(p, x, y, nrhs, ld, st);
    }
  }
  switch (choose_rpw(pref, p->nslices, nrhs)) {
    case 8: return launch_sparse_fwd_rpw<T, COMP, 8>(p, x, y, nrhs, ld, st);
    case 4: return launch_sparse_fwd_rpw<T, COMP, 4>(p, x, y, nrhs, ld, st);
    case 2: return launch_sparse_fwd_rpw<T, COMP, 2>(p, x, y, nrhs, ld, st);
    default: return launch_sparse_fwd_rpw<T, COMP, 1>(p, x, y, nrhs, ld, st);
  }
}

template <typename T, bool COMP>
int launch_sparse_adj(Plan* p, const void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  switch (choose_rpw(sizeof(T) == 8 ? 2 : 8, p->s_total_chunks, nrhs)) {
    case 8: return launch_sparse_adj_rpw<T, COMP, 8>(p, y, nrhs, ld, st);
    case 4: return launch_sparse_adj_rpw<T, COMP, 4>(p, y, nrhs, ld, st);
    case 2: return launch_sparse_adj_rpw<T, COMP, 2>(p, y, nrhs, ld, st);
    default: return launch_sparse_adj_rpw<T, COMP, 1>(p, y, nrhs, ld, st);
  }
}

template <typename T, bool COMP>
int apply_impl(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  if (!p->blocks.empty()) XC_TRY(launch_fft<T>(p, true, x, p->scratch, nrhs, ld, st));
  return launch_sparse_fwd<T, COMP>(p, x, y, nrhs, ld, st);
}

template <typename T, bool COMP>
int adjoint_impl(Plan* p, const void* y, void* x, int64_t nrhs, int64_t ld, cudaStream_t st) {
  if (!p->blocks.empty()) {
    XC_TRY(launch_sparse_adj<T, COMP>(p, y, nrhs, ld, st));
    XC_TRY(launch_fft<T>(p, false, p->scratch, x, nrhs, ld, st));
  }
  if (p->m_tail > 0) {
    dim3 grid(unsigned((p->m_tail + 7) / 8), unsigned(nrhs));
    launch_begin(p, K_ADJ_TAIL, st);
    adj_tail_kernel<T, COMP><<<grid, 256, 0, st>>>(p->N, p->m_tail, static_cast<const T*>(p->tail),
                                                   static_cast<const T*>(y), ld, static_cast<T*>(x),
                                                   static_cast<const T*>(p->rowscale),
                                                   static_cast<const T*>(p->colscale));
    launch_end(p, K_ADJ_TAIL, st);
    XC_CUDA(cudaGetLastError());
  }
  return XC_OK;
}

// ------------------------------------------------ FP64 plans in FP32 pairs
int* pair_exponents(Plan* p) { return reinterpret_cast<int*>(static_cast<char*>(p->scratch) + p->pexp_off); }

template <int RPW>
int launch_pair_fwd_rpw(Plan* p, const double* x, double* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const BlockDev* bd = static_cast<const BlockDev*>(p->scratch_desc);
  const PairCx* spec = static_cast<const PairCx*>(p->scratch);
  int* pexp = pair_exponents(p);
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  unsigned grid = 1;
  if (p->fwd_chunked) {
    const void* fn = reinterpret_cast<const void*>(fwd_unit_pair_kernel<RPW>);
    const int sg = supergroup(fn, p->total_units, ngroups);
    XC_TRY(persistent_grid(fn, p->total_units * ((ngroups + sg - 1) / sg), &grid, 4));
    cx<double>* part = static_cast<cx<double>*>(p->scratch) + p->spec_per_rhs * nrhs;
    launch_begin(p, K_FWD_SPARSE, st);
    fwd_unit_pair_kernel<RPW><<<grid, 32 * kSparseWarps, 0, st>>>(bd, spec, nrhs, pexp, part, p->fu_units,
                                                                   p->fu_order, p->total_units, p->counters, sg);
    launch_end(p, K_FWD_SPARSE, st);
    XC_CUDA(cudaGetLastError());
    dim3 rgrid(unsigned((p->N + 255) / 256), unsigned(std::min<int64_t>(nrhs, 65535)));
    launch_begin(p, K_FWD_REDUCE, st);
    fwd_reduce_kernel<double, false><<<rgrid, 256, 0, st>>>(p->N, x, ld, y, part, nrhs, p->fu_ubase,
                                                            static_cast<const double*>(p->rowscale),
                                                            static_cast<const double*>(p->colscale),
                                                            static_cast<const double*>(p->tail), p->m_tail);
    launch_end(p, K_FWD_REDUCE, st);
    XC_CUDA(cudaGetLastError());
    return XC_OK;
  }
  const void* fn = reinterpret_cast<const void*>(fwd_sparse_pair_kernel<RPW>);
  const int sg = supergroup(fn, p->nslices, ngroups);
  XC_TRY(persistent_grid(fn, p->nslices * ((ngroups + sg - 1) / sg), &grid, 4));
  launch_begin(p, K_FWD_SPARSE, st);
  fwd_sparse_pair_kernel<RPW><<<grid, 32 * kSparseWarps, 0, st>>>(
      bd, int(p->blocks.size()), p->N, x, ld, y, spec, nrhs, pexp, static_cast<const double*>(p->rowscale),
      static_cast<const double*>(p->colscale), static_cast<const double*>(p->tail), p->m_tail, p->f_order,
      p->counters, sg);
  launch_end(p, K_FWD_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

int apply_pair(Plan* p, const void* xv, void* yv, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const double* x = static_cast<const double*>(xv);
  double* y = static_cast<double*>(yv);
  int* pexp = pair_exponents(p);
  launch_begin(p, K_PAIR_SCALE, st);
  pair_scale_kernel<<<unsigned(nrhs), 256, 0, st>>>(x, ld, p->N, nullptr, pexp, nullptr);
  launch_end(p, K_PAIR_SCALE, st);
  XC_CUDA(cudaGetLastError());
  if (!p->blocks.empty()) XC_TRY(launch_fft<double>(p, true, x, p->scratch, nrhs, ld, st, pexp));
  switch (choose_rpw(8, p->fwd_chunked ? p->total_units : p->nslices, nrhs)) {
    case 8: return launch_pair_fwd_rpw<8>(p, x, y, nrhs, ld, st);
    case 4: return launch_pair_fwd_rpw<4>(p, x, y, nrhs, ld, st);
    case 2: return launch_pair_fwd_rpw<2>(p, x, y, nrhs, ld, st);
    default: return launch_pair_fwd_rpw<1>(p, x, y, nrhs, ld, st);
  }
}

template <int RPW>
int launch_pair_adj_rpw(Plan* p, const float2* yp, int64_t nrhs, cudaStream_t st) {
  if (p->s_total_chunks == 0) return XC_OK;
  const void* fn = reinterpret_cast<const void*>(adj_sparse_pair_kernel<RPW>);
  unsigned grid = 1;
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  const int sg = supergroup(fn, p->s_total_chunks, ngroups);
  XC_TRY(persistent_grid(fn, p->s_total_chunks * ((ngroups + sg - 1) / sg), &grid));
  launch_begin(p, K_ADJ_SPARSE, st);
  adj_sparse_pair_kernel<RPW><<<grid, 32 * kSparseWarps, 0, st>>>(
      static_cast<const BlockDev*>(p->scratch_desc), int(p->blocks.size()), p->N, yp, pair_exponents(p),
      static_cast<cx<double>*>(p->scratch), nrhs, p->s_items, p->s_cbase, p->s_total_chunks, p->s_chunk,
      p->counters, sg);
  launch_end(p, K_ADJ_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

int adjoint_pair(Plan* p, const void* yv, void* xv, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const double* y = static_cast<const double*>(yv);
  if (!p->blocks.empty()) {
    float2* yp = reinterpret_cast<float2*>(static_cast<cx<double>*>(p->scratch) + p->s_total_chunks * 32 * nrhs);
    launch_begin(p, K_PAIR_SCALE, st);
    pair_scale_kernel<<<unsigned(nrhs), 256, 0, st>>>(y, ld, p->N, static_cast<const double*>(p->rowscale),
                                                      pair_exponents(p), yp);
    launch_end(p, K_PAIR_SCALE, st);
    XC_CUDA(cudaGetLastError());
    switch (choose_rpw(8, p->s_total_chunks, nrhs)) {
      case 8: XC_TRY(launch_pair_adj_rpw<8>(p, yp, nrhs, st)); break;
      case 4: XC_TRY(launch_pair_adj_rpw<4>(p, yp, nrhs, st)); break;
      case 2: XC_TRY(launch_pair_adj_rpw<2>(p, yp, nrhs, st)); break;
      default: XC_TRY(launch_pair_adj_rpw<1>(p, yp, nrhs, st)); break;
    }
    XC_TRY(launch_fft<double>(p, false, p->scratch, xv, nrhs, ld, st));
  }
  if (p->m_tail > 0) {
    dim3 grid(unsigned((p->m_tail + 7) / 8), unsigned(nrhs));
    launch_begin(p, K_ADJ_TAIL, st);
    adj_tail_kernel<double, false><<<grid, 256, 0, st>>>(p->N, p->m_tail, static_cast<const double*>(p->tail), y,
                                                         ld, static_cast<double*>(xv),
                                                         static_cast<const double*>(p->rowscale),
                                                         static_cast<const double*>(p->colscale));
    launch_end(p, K_ADJ_TAIL, st);
    XC_CUDA(cudaGetLastError());
  }
  return XC_OK;
}

}  // namespace

// ------------------------------------------------------ allocation-free apply
// Spectrum scratch for xc_apply_noalloc: one fixed array in device memory,
// shared by every call on a device.  Host code must not use the symbol's
// host-side name as a device address; the device address is looked up once
// per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[XC_NOALLOC_SCRATCH_BYTES];
// The work counters of the allocation-free sparse launch ({next, done}, reset
// by the launch's last warp): its own pair, so that it never shares a pair
// with xc_apply / xc_apply_adjoint on the same plan.  Zero at module load.
static __device__ __align__(16) unsigned g_noalloc_counters[4];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};
void* g_noalloc_ctr[kMaxDevices] = {};

// Device addresses of g_noalloc_scratch and g_noalloc_counters on the current
// device (looked up on the first call per device).
int noalloc_scratch(void** out, unsigned** counters) {
  int dev = 0;
  XC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(XC_ERR_UNSUPPORTED, "device index beyond 64");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    void* ctr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&ctr, g_noalloc_counters);
    if (e != cudaSuccess || ptr == nullptr || ctr == nullptr) {
      cudaGetLastError();
      return fail(XC_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                                   cudaGetErrorString(e));
    }
    g_noalloc_ctr[dev] = ctr;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  *counters = static_cast<unsigned*>(g_noalloc_ctr[dev]);
  return XC_OK;
}

template <typename T, bool COMP>
int apply_noalloc_impl(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st, void* spec,
                       unsigned* counters) {
  const BlockDev* bd = static_cast<const BlockDev*>(p->scratch_desc);
  if (!p->blocks.empty()) {
    const size_t smem = size_t(p->max_n) * sizeof(cx<T>);
    if (smem > 48 * 1024)
      XC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fwd_fft_kernel<T>),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    dim3 grid(unsigned(nrhs), unsigned(p->blocks.size()));
    count_launch();
    fwd_fft_kernel<T><<<grid, kFftThreads, smem, st>>>(bd, static_cast<const T*>(x), ld,
                                                        static_cast<const T*>(p->colscale),
                                                        static_cast<cx<T>*>(spec), nrhs, nullptr);
    XC_CUDA(cudaGetLastError());
  }
  constexpr int RPW = 8;
  unsigned grid = 1;
  XC_TRY(persistent_grid(reinterpret_cast<const void*>(fwd_sparse_kernel<T, RPW, COMP>),
                         p->nslices * ((nrhs + RPW - 1) / RPW), &grid));
  count_launch();
  fwd_sparse_kernel<T, RPW, COMP><<<grid, 32 * kSparseWarps, 0, st>>>(
      bd, int(p->blocks.size()), p->N, static_cast<const T*>(x), ld, static_cast<T*>(y),
      static_cast<const cx<T>*>(spec), nrhs, static_cast<const T*>(p->rowscale),
      static_cast<const T*>(p->colscale), static_cast<const T*>(p->tail), p->m_tail, p->f_order, counters, 1);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

}  // namespace

int launch_apply_noalloc(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const double need = double(p->spec_per_rhs) * double(nrhs) * double(2 * p->elem_bytes());
  if (need > double(XC_NOALLOC_SCRATCH_BYTES))
    return fail(XC_ERR_UNSUPPORTED, "xc_apply_noalloc needs " + std::to_string(int64_t(need)) +
                                        " bytes of spectrum scratch, above its fixed " +
                                        std::to_string(int64_t(XC_NOALLOC_SCRATCH_BYTES)) +
                                        "-byte array; split the right-hand sides");
  if (p->scratch_desc == nullptr) return fail(XC_ERR_ARG, "plan has no device descriptors");
  if (p->precision == XC_FP64_PAIR) return fail(XC_ERR_UNSUPPORTED, "xc_apply_noalloc does not take XC_FP64_PAIR plans");
  if (p->max_csize > 1) return fail(XC_ERR_UNSUPPORTED, "xc_apply_noalloc does not take plans with cluster FFTs");
  void* spec = nullptr;
  unsigned* counters = nullptr;
  XC_TRY(noalloc_scratch(&spec, &counters));
  switch (p->precision) {
    case XC_FP64: return apply_noalloc_impl<double, false>(p, x, y, nrhs, ld, st, spec, counters);
    case XC_FP32: return apply_noalloc_impl<float, false>(p, x, y, nrhs, ld, st, spec, counters);
    default: return apply_noalloc_impl<float, true>(p, x, y, nrhs, ld, st, spec, counters);
  }
}

namespace {

int grow_scratch(Plan* p, int64_t nrhs, size_t bytes) {
  void* fresh = nullptr;
  if (cudaMalloc(&fresh, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(XC_ERR_ALLOC, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
  }
  if (p->scratch) {
    // a previous apply may still use the old buffer on its stream
    cudaDeviceSynchronize();
    cudaFree(p->scratch);
  }
  p->scratch = fresh;
  p->scratch_nrhs = nrhs;
  return XC_OK;
}

}  // namespace

int ensure_scratch(Plan* p, int64_t nrhs) {
  if (p->scratch_desc == nullptr) {
    void* d = nullptr;
    XC_TRY(plan_alloc(p, &d, std::max<size_t>(1, p->blocks.size()) * sizeof(BlockDev)));
    if (!p->blocks.empty())
      XC_CUDA(cudaMemcpy(d, p->blocks.data(), p->blocks.size() * sizeof(BlockDev), cudaMemcpyHostToDevice));
    p->scratch_desc = d;
  }
  if (nrhs <= p->scratch_nrhs) return XC_OK;
  const size_t cbytes = 2 * p->elem_bytes();
  if (p->cplx) return grow_scratch(p, nrhs, complex_scratch_bytes(p, nrhs));
  if (p->d2) return grow_scratch(p, nrhs, d2_scratch_bytes(p, nrhs));
  // forward: spectra (+ unit partials); adjoint: chunk partials + transposed
  // y.  The directions share the buffer (one at a time).
  const int64_t fwd = p->spec_per_rhs + (p->fwd_chunked ? p->total_units * 32 : 0);
  const size_t fwd_bytes = size_t(fwd) * size_t(nrhs) * cbytes;
  const int64_t chunks = std::max(p->total_chunks, p->s_total_chunks);
  const size_t adj_bytes = size_t(chunks) * 32 * size_t(nrhs) * cbytes +
                           (p->any_yt ? size_t(p->N) * size_t(yt_ld(nrhs)) * p->elem_bytes() : 0);
  size_t bytes = std::max<size_t>({cbytes, fwd_bytes, adj_bytes});
  if (p->precision == XC_FP64_PAIR) {
    // adjoint input pairs after the chunk partials, then the per-RHS exponents
    const size_t adj_pair = size_t(chunks) * 32 * size_t(nrhs) * cbytes + size_t(p->N) * size_t(nrhs) * 8;
    bytes = (std::max(bytes, adj_pair) + 255) / 256 * 256;
    p->pexp_off = bytes;
    bytes += size_t(nrhs) * sizeof(int);
  }
  return grow_scratch(p, nrhs, bytes);
}

int launch_apply(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  XC_TRY(ensure_scratch(p, nrhs));
  if (p->cplx) return launch_apply_complex(p, x, y, nrhs, ld, st);
  if (p->d2) return launch_apply_2d(p, x, y, nrhs, ld, st, false);
  switch (p->precision) {
    case XC_FP64: return apply_impl<double, false>(p, x, y, nrhs, ld, st);
    case XC_FP64_PAIR: return apply_pair(p, x, y, nrhs, ld, st);
    case XC_FP32: return apply_impl<float, false>(p, x, y, nrhs, ld, st);
    default: return apply_impl<float, true>(p, x, y, nrhs, ld, st);
  }
}

int launch_apply_adjoint(Plan* p, const void* y, void* x, int64_t nrhs, int64_t ld, cudaStream_t st) {
  XC_TRY(ensure_scratch(p, nrhs));
  if (p->cplx) return launch_adjoint_complex(p, y, x, nrhs, ld, st);
  if (p->d2) return launch_apply_2d(p, y, x, nrhs, ld, st, true);
  switch (p->precision) {
    case XC_FP64: return adjoint_impl<double, false>(p, y, x, nrhs, ld, st);
    case XC_FP64_PAIR: return adjoint_pair(p, y, x, nrhs, ld, st);
    case XC_FP32: return adjoint_impl<float, false>(p, y, x, nrhs, ld, st);
    default: return adjoint_impl<float, true>(p, y, x, nrhs, ld, st);
  }
}

}  // namespace xc
