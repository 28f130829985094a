// Execution stage of the complex families (exp(i m theta_n) and the spectral
// Laguerre matrix of eq. (lag_matrix)): Algorithms 1 and 2 with a complex
// matrix and complex vectors, one two-sided block, no real part taken.
//
// Forward, y = A x:
//   c_fwd_fft_kernel     per RHS: u = W^{-1} x^{[1]} (complex, eq. (Fe1)),
//                        v_k = sum_j u_j exp(+2 pi i jk / L) over the full
//                        spectrum (the unnormalised F* of Algorithm 1 step 2.1;
//                        the stored matrix carries the 1/L), followed by a
//                        periodic copy of the first c_vpad bins
//   c_fwd_sparse_kernel  per (32-row slice, RHS group): y_n = f_n sum_j S_nj v_{k0_n + j}
//                        over the row's circular band (f_n: the row factor of
//                        the spectral Laguerre matrix, else 1)
// Adjoint, x = A^T y (plain transpose):
//   c_row_scale_kernel   y_n f_n into scratch (spectral Laguerre matrix only)
//   c_adj_sparse_kernel  per (32-bin slice, RHS group): z_k = sum_i S_{n0_k + i, k} y_{n0_k + i}
//                        over the bin's circular run of rows
//   c_adj_fft_kernel     per RHS: x_j = w_j^{-1} sum_k z_k exp(+2 pi i jk / L),
//                        the real components [j_lo, j_hi) kept (eq. (Fe2))
//
// The L-point complex transforms reuse the n = L/2 point packed real FFT of
// the real families twice: a complex sequence is the pair of its real and
// imaginary parts, two real sequences, which the two CTAs of a cluster
// transform one each, exchanging the results through distributed shared
// memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "xc_fft.cuh"
#include "xc_internal.h"

namespace xc {

namespace {

namespace cg = cooperative_groups;

constexpr int kCfftThreads = 512;   // per CTA; two CTAs (a cluster) per transform
constexpr int kCsparseThreads = 128;
constexpr int kCAdjChunk = 64;      // rows per adjoint item (long bin runs are cut)

template <typename T>
__device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}

// ---------------------------------------------------------------- forward FFT
// A cluster of two CTAs per RHS: rank 0 transforms the real parts, rank 1 the
// imaginary parts (n = L/2 complex values each); after a cluster barrier both
// read the two spectra through distributed shared memory and write half of
// the bins each.
template <typename T>
__global__ void __launch_bounds__(kCfftThreads) c_fwd_fft_kernel(BlockDev b, const cx<T>* __restrict__ x,
                                                                 int64_t ld, cx<T>* __restrict__ v, int64_t Lv,
                                                                 int vpad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int n = b.n, L = b.L;
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int64_t r = blockIdx.x / 2;
  const T* __restrict__ invw = static_cast<const T*>(b.invw);
  const cx<T>* __restrict__ tw = static_cast<const cx<T>*>(b.tw);
  const cx<T>* __restrict__ xr = x + r * ld;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int j0 = 2 * j, j1 = 2 * j + 1;
    cx<T> u0{T(0), T(0)}, u1{T(0), T(0)};
    if (j0 >= b.j_lo && j0 < b.j_hi) u0 = scal(invw[j0], xr[j0 - b.off]);
    if (j1 >= b.j_lo && j1 < b.j_hi) u1 = scal(invw[j1], xr[j1 - b.off]);
    s[b.perm[j]] = rank == 0 ? cx<T>{u0.re, u1.re} : cx<T>{u0.im, u1.im};
  }
  __syncthreads();
  fft_inplace<T>(s, n, b.p, b.radix, tw, threadIdx.x, blockDim.x);
  cluster.sync();   // both packed spectra are complete
  const cx<T>* sa = cluster.map_shared_rank(s, 0);
  const cx<T>* sb = cluster.map_shared_rank(s, 1);
  cx<T>* __restrict__ vr = v + r * Lv;
  // with A = DFT(re u), B = DFT(im u) (exp(-2 pi i jk / L), Hermitian):
  // v_k = conj(A_k) + i conj(B_k), v_{L-k} = A_k + i B_k
  auto put = [&](int k, cx<T> val) {
    vr[k] = val;
    if (k < vpad) vr[L + k] = val;
  };
  auto emit = [&](int k, cx<T> A, cx<T> B) {
    put(k, cx<T>{A.re + B.im, B.re - A.im});
    if (k > 0 && k < n) put(L - k, cx<T>{A.re - B.im, A.im + B.re});
  };
  for (int k = rank * int(blockDim.x) + int(threadIdx.x); k <= n / 2; k += 2 * int(blockDim.x)) {
    cx<T> Ak, Ank, Bk, Bnk;
    r2c_split(sa, n, k, tw, &Ak, &Ank);
    r2c_split(sb, n, k, tw, &Bk, &Bnk);
    emit(k, Ak, Bk);
    if (n - k != k) emit(n - k, Ank, Bnk);
  }
  cluster.sync();   // no CTA leaves while its partner may still read its shared memory
}

// ------------------------------------------------------------- forward band
template <typename T, int RPW>
__global__ void __launch_bounds__(kCsparseThreads) c_fwd_sparse_kernel(BlockDev b, int64_t N,
                                                                       const cx<T>* __restrict__ v, int64_t Lv,
                                                                       int64_t nrhs, int64_t ngroups,
                                                                       const cx<T>* __restrict__ rowscale,
                                                                       cx<T>* __restrict__ y, int64_t ld) {
  const int64_t item = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= int64_t(b.nslices) * ngroups) return;
  const int s = int(item / ngroups);
  const int64_t r0 = (item % ngroups) * RPW;
  const int64_t row = int64_t(s) * 32 + lane;
  const int W = b.f_width[s];
  const cx<T>* __restrict__ val = static_cast<const cx<T>*>(b.f_val) + b.f_off[s] + lane;
  const int k0 = row < N ? b.f_k0[row] : 0;
  const cx<T>* vb[RPW];
#pragma unroll
  for (int q = 0; q < RPW; ++q) vb[q] = v + (r0 + q < nrhs ? r0 + q : nrhs - 1) * Lv + k0;
  cx<T> acc[RPW];
#pragma unroll
  for (int q = 0; q < RPW; ++q) acc[q] = cx<T>{T(0), T(0)};
  for (int j = 0; j < W; ++j) {
    const cx<T> a = val[int64_t(j) * 32];
#pragma unroll
    for (int q = 0; q < RPW; ++q) cfma(acc[q], a, vb[q][j]);
  }
  if (row >= N) return;
  const cx<T> f = rowscale ? rowscale[row] : cx<T>{T(1), T(0)};
#pragma unroll
  for (int q = 0; q < RPW; ++q)
    if (r0 + q < nrhs) y[(r0 + q) * ld + row] = rowscale ? cmul(f, acc[q]) : acc[q];
}

// --------------------------------------------------------------- adjoint
template <typename T>
__global__ void c_row_scale_kernel(const cx<T>* __restrict__ y, int64_t ld, int64_t N, int64_t nrhs,
                                   const cx<T>* __restrict__ rowscale, cx<T>* __restrict__ ys) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N * nrhs) return;
  const int64_t r = i / N, n = i % N;
  ys[i] = cmul(rowscale[n], y[r * ld + n]);
}

// One warp per (chunk of at most kCAdjChunk rows of a 32-bin slice, RHS
// group): partial sums of z_k over the chunk's rows, stored per chunk; the
// adjoint FFT adds a bin's chunks in chunk order (no atomics, a fixed order).
// items[g] = (slice, chunk within the slice) with g = cbase[slice] + chunk.
template <typename T, int RPW>
__global__ void __launch_bounds__(kCsparseThreads) c_adj_sparse_kernel(BlockDev b, int64_t N,
                                                                       const int2* __restrict__ items,
                                                                       int64_t nitems, const cx<T>* __restrict__ y,
                                                                       int64_t ldy, int64_t nrhs, int64_t ngroups,
                                                                       cx<T>* __restrict__ part) {
  const int64_t item = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= nitems * ngroups) return;
  const int64_t g = item / ngroups;
  const int2 it = items[g];
  const int s = it.x;
  const int64_t r0 = (item % ngroups) * RPW;
  const int k = s * 32 + lane;
  const int W = b.t_width[s];
  const int i0 = it.y * kCAdjChunk;
  const int i1 = min(W, i0 + kCAdjChunk);
  const cx<T>* __restrict__ val = static_cast<const cx<T>*>(b.t_val) + b.t_off[s] + lane;
  const int64_t n0 = k < b.L ? b.t_n0[k] : 0;
  const cx<T>* yb[RPW];
#pragma unroll
  for (int q = 0; q < RPW; ++q) yb[q] = y + (r0 + q < nrhs ? r0 + q : nrhs - 1) * ldy;
  cx<T> acc[RPW];
#pragma unroll
  for (int q = 0; q < RPW; ++q) acc[q] = cx<T>{T(0), T(0)};
  int64_t nn = (n0 + i0) % N;
  for (int i = i0; i < i1; ++i) {
    const cx<T> a = val[int64_t(i) * 32];
#pragma unroll
    for (int q = 0; q < RPW; ++q) cfma(acc[q], a, yb[q][nn]);
    if (++nn == N) nn = 0;   // circular run of rows
  }
#pragma unroll
  for (int q = 0; q < RPW; ++q)
    if (r0 + q < nrhs) part[(g * nrhs + r0 + q) * 32 + lane] = acc[q];
}

// z_k of RHS r: the chunk partials of bin k's slice, in chunk order
template <typename T>
__device__ __forceinline__ cx<T> gather_z(const cx<T>* __restrict__ part, const int* __restrict__ cbase, int k,
                                          int64_t r, int64_t nrhs) {
  const int s = k >> 5;
  cx<T> z{T(0), T(0)};
  for (int c = cbase[s]; c < cbase[s + 1]; ++c) z = z + part[(int64_t(c) * nrhs + r) * 32 + (k & 31)];
  return z;
}

// Cluster of two CTAs per RHS: rank 0 transforms P_k = (z_k + conj z_{L-k}) / 2,
// rank 1 Q_k = (z_k - conj z_{L-k}) / (2i), both Hermitian, so that
// sum_k z_k exp(+2 pi i jk / L) = p_j + i q_j with p, q the real inverse
// transforms of P and Q (packed as in the real adjoint); each rank then writes
// half of the outputs, reading p and q through distributed shared memory.
template <typename T>
__global__ void __launch_bounds__(kCfftThreads) c_adj_fft_kernel(BlockDev b, const cx<T>* __restrict__ part,
                                                                 const int* __restrict__ cbase, int64_t nrhs,
                                                                 cx<T>* __restrict__ x, int64_t ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int n = b.n, L = b.L;
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int64_t r = blockIdx.x / 2;
  const T* __restrict__ invw = static_cast<const T*>(b.invw);
  const cx<T>* __restrict__ tw = static_cast<const cx<T>*>(b.tw);
  const T h = T(0.5);
  // each bin pair (k, n - k) once: this CTA takes every other pair, forms
  // both P and Q, and stores them packed into rank 0's (P) and rank 1's (Q)
  // shared memory
  cx<T>* dp = cluster.map_shared_rank(s, 0);
  cx<T>* dq = cluster.map_shared_rank(s, 1);
  cluster.sync();   // the partner runs before its shared memory is written
  for (int k = rank * int(blockDim.x) + int(threadIdx.x); k <= n / 2; k += 2 * int(blockDim.x)) {
    const cx<T> zk = gather_z(part, cbase, k, r, nrhs);
    const cx<T> zLk = conj(gather_z(part, cbase, k == 0 ? 0 : L - k, r, nrhs));
    const cx<T> znk = gather_z(part, cbase, n - k, r, nrhs);
    const cx<T> zLnk = conj(gather_z(part, cbase, L - (n - k), r, nrhs));
    cx<T> Pk = scal(h, zk + zLk), Qk = scal(h, mul_mi(zk - zLk));
    cx<T> Pnk = scal(h, znk + zLnk), Qnk = scal(h, mul_mi(znk - zLnk));
    if (k == 0) {   // P_0, P_n, Q_0, Q_n enter as real numbers
      Pk.im = Pnk.im = Qk.im = Qnk.im = T(0);
    }
    const int pk = b.perm[k], pnk = b.perm[n - k];
    const bool two = k != 0 && n - k != k;
    cx<T> Zk, Znk;
    c2r_merge(Pk, Pnk, k, tw, &Zk, &Znk);
    dp[pk] = conj(Zk);   // inverse FFT as conj(FFT(conj(Z)))
    if (two) dp[pnk] = conj(Znk);
    c2r_merge(Qk, Qnk, k, tw, &Zk, &Znk);
    dq[pk] = conj(Zk);
    if (two) dq[pnk] = conj(Znk);
  }
  cluster.sync();   // both packed spectra are in place
  fft_inplace<T>(s, n, b.p, b.radix, tw, threadIdx.x, blockDim.x);
  cluster.sync();   // p and q are complete
  const cx<T>* sp = cluster.map_shared_rank(s, 0);
  const cx<T>* sq = cluster.map_shared_rank(s, 1);
  cx<T>* __restrict__ xr = x + r * ld;
  for (int j = rank * int(blockDim.x) + int(threadIdx.x); j < n; j += 2 * int(blockDim.x)) {
    const cx<T> P = sp[j], Q = sq[j];
    const int j0 = 2 * j, j1 = 2 * j + 1;
    if (j0 >= b.j_lo && j0 < b.j_hi) xr[j0 - b.off] = cx<T>{P.re * invw[j0], Q.re * invw[j0]};
    if (j1 >= b.j_lo && j1 < b.j_hi) xr[j1 - b.off] = cx<T>{-P.im * invw[j1], -Q.im * invw[j1]};
  }
  cluster.sync();   // no CTA leaves while its partner may still read its shared memory
}

// ------------------------------------------------------------------ launches
int64_t spectrum_ld(const Plan* p) { return int64_t(p->blocks[0].L) + p->c_vpad; }

// right-hand sides per warp item: as many as the spread over 4 items per
// warp slot of the GPU allows
int choose_crpw(int64_t slices, int64_t nrhs) {
  int rpw = 8;
  while (rpw > 1 && (rpw > nrhs || slices * ((nrhs + rpw - 1) / rpw) < 152 * 32)) rpw /= 2;
  return rpw;
}

template <typename T>
int set_fft_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) XC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return XC_OK;
}

template <typename T, int RPW>
int fwd_sparse_rpw(Plan* p, const cx<T>* v, cx<T>* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const BlockDev& b = p->blocks[0];
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  const int64_t warps = int64_t(b.nslices) * ngroups;
  const unsigned grid = unsigned((warps * 32 + kCsparseThreads - 1) / kCsparseThreads);
  launch_begin(p, K_FWD_SPARSE, st);
  c_fwd_sparse_kernel<T, RPW><<<grid, kCsparseThreads, 0, st>>>(b, p->N, v, spectrum_ld(p), nrhs, ngroups,
                                                               static_cast<const cx<T>*>(p->rowscale), y, ld);
  launch_end(p, K_FWD_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

template <typename T, int RPW>
int adj_sparse_rpw(Plan* p, const cx<T>* y, int64_t ldy, cx<T>* part, int64_t nrhs, cudaStream_t st) {
  const BlockDev& b = p->blocks[0];
  const int64_t ngroups = (nrhs + RPW - 1) / RPW;
  const int64_t warps = p->c_nchunks * ngroups;
  if (warps == 0) return XC_OK;
  const unsigned grid = unsigned((warps * 32 + kCsparseThreads - 1) / kCsparseThreads);
  launch_begin(p, K_ADJ_SPARSE, st);
  c_adj_sparse_kernel<T, RPW><<<grid, kCsparseThreads, 0, st>>>(b, p->N, p->c_items, p->c_nchunks, y, ldy, nrhs,
                                                               ngroups, part);
  launch_end(p, K_ADJ_SPARSE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

// Launch a two-CTA cluster per right-hand side.
template <typename K, typename... Args>
int launch_pair_cluster(K kernel, int64_t nrhs, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(2 * nrhs));
  cfg.blockDim = dim3(kCfftThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  XC_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
  return XC_OK;
}

template <typename T>
int apply_complex(Plan* p, const void* xv, void* yv, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const BlockDev& b = p->blocks[0];
  const auto* x = static_cast<const cx<T>*>(xv);
  auto* y = static_cast<cx<T>*>(yv);
  auto* v = static_cast<cx<T>*>(p->scratch);
  const size_t smem = size_t(b.n) * sizeof(cx<T>);
  XC_TRY(set_fft_smem<T>(reinterpret_cast<const void*>(c_fwd_fft_kernel<T>), smem));
  launch_begin(p, K_FWD_FFT, st);
  const int rc = launch_pair_cluster(c_fwd_fft_kernel<T>, nrhs, smem, st, b, x, ld, v, spectrum_ld(p), p->c_vpad);
  launch_end(p, K_FWD_FFT, st);
  XC_TRY(rc);
  switch (choose_crpw(b.nslices, nrhs)) {
    case 8: return fwd_sparse_rpw<T, 8>(p, v, y, nrhs, ld, st);
    case 4: return fwd_sparse_rpw<T, 4>(p, v, y, nrhs, ld, st);
    case 2: return fwd_sparse_rpw<T, 2>(p, v, y, nrhs, ld, st);
    default: return fwd_sparse_rpw<T, 1>(p, v, y, nrhs, ld, st);
  }
}

template <typename T>
int adjoint_complex(Plan* p, const void* yv, void* xv, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const BlockDev& b = p->blocks[0];
  const auto* y = static_cast<const cx<T>*>(yv);
  auto* x = static_cast<cx<T>*>(xv);
  auto* part = static_cast<cx<T>*>(p->scratch);           // [chunk][nrhs][32]
  cx<T>* ys = part + p->c_nchunks * nrhs * 32;             // [nrhs][N] (row factor applied)
  const cx<T>* yin = y;
  int64_t ldy = ld;
  if (p->rowscale) {
    const int64_t tot = nrhs * p->N;
    launch_begin(p, K_ROW_SCALE, st);
    c_row_scale_kernel<T><<<unsigned((tot + 255) / 256), 256, 0, st>>>(
        y, ld, p->N, nrhs, static_cast<const cx<T>*>(p->rowscale), ys);
    launch_end(p, K_ROW_SCALE, st);
    XC_CUDA(cudaGetLastError());
    yin = ys;
    ldy = p->N;
  }
  switch (choose_crpw(p->c_nchunks, nrhs)) {
    case 8: XC_TRY((adj_sparse_rpw<T, 8>(p, yin, ldy, part, nrhs, st))); break;
    case 4: XC_TRY((adj_sparse_rpw<T, 4>(p, yin, ldy, part, nrhs, st))); break;
    case 2: XC_TRY((adj_sparse_rpw<T, 2>(p, yin, ldy, part, nrhs, st))); break;
    default: XC_TRY((adj_sparse_rpw<T, 1>(p, yin, ldy, part, nrhs, st))); break;
  }
  const size_t smem = size_t(b.n) * sizeof(cx<T>);
  XC_TRY(set_fft_smem<T>(reinterpret_cast<const void*>(c_adj_fft_kernel<T>), smem));
  launch_begin(p, K_ADJ_FFT, st);
  const int rc = launch_pair_cluster(c_adj_fft_kernel<T>, nrhs, smem, st, b, static_cast<const cx<T>*>(part),
                                     static_cast<const int*>(p->c_cbase), nrhs, x, ld);
  launch_end(p, K_ADJ_FFT, st);
  XC_TRY(rc);
  return XC_OK;
}

}  // namespace

size_t complex_scratch_bytes(const Plan* p, int64_t nrhs) {
  const int64_t L = p->blocks.empty() ? 0 : p->blocks[0].L;
  // forward: the spectra; adjoint: the chunk partials, then the row-scaled input
  const int64_t per_rhs = std::max<int64_t>(L + p->c_vpad, p->c_nchunks * 32 + p->N);
  return std::max<size_t>(256, size_t(per_rhs) * size_t(nrhs) * 2 * p->elem_bytes());
}

int launch_apply_complex(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  if (p->io64()) return apply_complex<double>(p, x, y, nrhs, ld, st);
  return apply_complex<float>(p, x, y, nrhs, ld, st);
}

int launch_adjoint_complex(Plan* p, const void* y, void* x, int64_t nrhs, int64_t ld, cudaStream_t st) {
  if (p->io64()) return adjoint_complex<double>(p, y, x, nrhs, ld, st);
  return adjoint_complex<float>(p, y, x, nrhs, ld, st);
}

}  // namespace xc
