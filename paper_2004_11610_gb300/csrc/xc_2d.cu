// Execution stage of the 2-D block scheme (eq. (comp_2d), Sections 4.2 and
// 5.3): for every block, y_e = W_r^{-1} F* D̈ F* W_c^{-1} x^{[1]} on the block's
// valid rows, plus the dense rectangles.  The adjoint is the transpose,
// x_e = W_c^{-1} F* D̈^T F* W_r^{-1} y^{[1]}.  One direction is four launches:
//   d2_in_kernel       per (RHS, block): the input side's extension, W^{-1} and
//                      real FFT -> half spectrum U (DFT with exp(-2 pi i jk / L)),
//                      stored bin-major ([bin][RHS]) like the product's output
//   d2_sparse_kernel   per (output bin of a block, RHS), one warp (lanes over
//                      the row's entries; with 16 or more RHS d2_sparse_rhs_kernel,
//                      lanes over 32 RHS): z = sum a conj(U_k) + sum c U_k over the
//                      bin's two CSR segments (F* x = conj(U) for real x; the c
//                      terms carry the other half of the spectrum through the
//                      Hermitian symmetries)
//   d2_out_kernel      per (RHS, block): real inverse FFT of z, W^{-1}, the
//                      block's valid outputs into its partial buffer
//   d2_combine_kernel  per (output index, RHS), one warp: the partials of the blocks
//                      that cover the index and the dense rectangles, added
//                      in a fixed order (blocks by index, then rectangles).
#include <cuda_runtime.h>

#include <algorithm>

#include "xc_fft.cuh"
#include "xc_internal.h"
#include "xc_items.cuh"

namespace xc {

namespace {

constexpr int kD2FftThreads = 256;

// Spectra are stored bin-major, [spec_off + k][nrhs]: the 32 lanes of a CSR
// warp (32 consecutive RHS) read one contiguous line per entry.
template <typename T>
__global__ void __launch_bounds__(kD2FftThreads)
    d2_in_kernel(const BlockDev* __restrict__ devs, const T* __restrict__ x, int64_t ld, cx<T>* __restrict__ spec,
                 int64_t nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const BlockDev& b = devs[blockIdx.y];
  const int64_t r = blockIdx.x;
  const int n = b.n;
  const T* __restrict__ invw = static_cast<const T*>(b.invw);
  const cx<T>* __restrict__ tw = static_cast<const cx<T>*>(b.tw);
  const T* __restrict__ xr = x + r * ld;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int j0 = 2 * j, j1 = 2 * j + 1;
    const T u0 = (j0 >= b.j_lo && j0 < b.j_hi) ? xr[j0 - b.off] * invw[j0] : T(0);
    const T u1 = (j1 >= b.j_lo && j1 < b.j_hi) ? xr[j1 - b.off] * invw[j1] : T(0);
    s[b.perm[j]] = cx<T>{u0, u1};
  }
  __syncthreads();
  fft_inplace<T>(s, n, b.p, b.radix, tw, threadIdx.x, blockDim.x);
  cx<T>* __restrict__ out = spec + b.spec_off * nrhs + r;
  for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
    cx<T> Uk, Unk;
    r2c_split_vals(s[k], s[k == 0 ? 0 : n - k], k, tw, &Uk, &Unk);
    out[int64_t(k) * nrhs] = Uk;
    if (n - k != k) out[int64_t(n - k) * nrhs] = Unk;
  }
}

template <typename T>
__global__ void d2_sparse_kernel(const BlockDev* __restrict__ in, const BlockDev* __restrict__ out,
                                 const int64_t* __restrict__ ptr, const int* __restrict__ idx,
                                 const cx<T>* __restrict__ a, const int* __restrict__ row_blk, const int* __restrict__ row_loc, int64_t rows,
                                 const cx<T>* __restrict__ spec, cx<T>* __restrict__ z, int64_t nrhs) {
  const int64_t item = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= rows * nrhs) return;
  const int64_t row = item / nrhs, r = item % nrhs;
  const int b = row_blk[row];
  const BlockDev& bi = in[b];
  const cx<T>* __restrict__ U = spec + bi.spec_off * nrhs + r;
  T re = T(0), im = T(0);
  for (int64_t e = ptr[2 * row] + lane; e < ptr[2 * row + 1]; e += 32) {   // a conj(u)
    const cx<T> u = U[int64_t(idx[e]) * nrhs];
    const cx<T> ae = a[e];
    re += ae.re * u.re + ae.im * u.im;
    im += ae.im * u.re - ae.re * u.im;
  }
  for (int64_t e = ptr[2 * row + 1] + lane; e < ptr[2 * row + 2]; e += 32) {   // c u
    const cx<T> u = U[int64_t(idx[e]) * nrhs];
    const cx<T> ce = a[e];
    re += ce.re * u.re - ce.im * u.im;
    im += ce.re * u.im + ce.im * u.re;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    const BlockDev& bo = out[b];
    z[(bo.spec_off + row_loc[row]) * nrhs + r] = cx<T>{re, im};
  }
}

// The same product with the lanes over 32 right-hand sides (rhs0 + lane):
// one warp per (output bin, group of 32 RHS) walks the bin's CSR row once.
template <typename T>
__global__ void d2_sparse_rhs_kernel(const BlockDev* __restrict__ in, const BlockDev* __restrict__ out,
                                     const int64_t* __restrict__ ptr, const int* __restrict__ idx,
                                     const cx<T>* __restrict__ a, const int* __restrict__ row_blk, const int* __restrict__ row_loc, int64_t rows,
                                     const cx<T>* __restrict__ spec, cx<T>* __restrict__ z, int64_t nrhs) {
  const int64_t groups = (nrhs + 31) / 32;
  const int64_t item = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= rows * groups) return;
  const int64_t row = item / groups;
  const int64_t r = (item % groups) * 32 + lane;
  const int64_t rr = r < nrhs ? r : nrhs - 1;
  const int b = row_blk[row];
  const BlockDev& bi = in[b];
  const cx<T>* __restrict__ U = spec + bi.spec_off * nrhs + rr;
  T re = T(0), im = T(0);
  for (int64_t e = ptr[2 * row]; e < ptr[2 * row + 1]; ++e) {   // a conj(u)
    const cx<T> u = U[int64_t(idx[e]) * nrhs];
    const cx<T> ae = a[e];
    re += ae.re * u.re + ae.im * u.im;
    im += ae.im * u.re - ae.re * u.im;
  }
  for (int64_t e = ptr[2 * row + 1]; e < ptr[2 * row + 2]; ++e) {   // c u
    const cx<T> u = U[int64_t(idx[e]) * nrhs];
    const cx<T> ce = a[e];
    re += ce.re * u.re - ce.im * u.im;
    im += ce.re * u.im + ce.im * u.re;
  }
  if (r < nrhs) {
    const BlockDev& bo = out[b];
    z[(bo.spec_off + row_loc[row]) * nrhs + r] = cx<T>{re, im};
  }
}

template <typename T>
__global__ void __launch_bounds__(kD2FftThreads)
    d2_out_kernel(const BlockDev* __restrict__ devs, const cx<T>* __restrict__ z, const int64_t* __restrict__ part_off,
                  T* __restrict__ part, int64_t nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const BlockDev& b = devs[blockIdx.y];
  const int64_t r = blockIdx.x;
  const int n = b.n;
  const int* __restrict__ perm = b.perm;
  const cx<T>* __restrict__ tw = static_cast<const cx<T>*>(b.tw);
  const T* __restrict__ invw = static_cast<const T*>(b.invw);
  const cx<T>* __restrict__ zr = z + b.spec_off * nrhs + r;
  for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
    cx<T> Uk = zr[int64_t(k) * nrhs], Unk = zr[int64_t(n - k) * nrhs];
    if (k == 0) {   // U_0 and U_n enter as real numbers
      Uk.im = T(0);
      Unk.im = T(0);
    }
    cx<T> Zk, Znk;
    c2r_merge(Uk, Unk, k, tw, &Zk, &Znk);
    s[perm[k]] = conj(Zk);   // inverse FFT as conj(FFT(conj(Z)))
    if (k != 0 && n - k != k) s[perm[n - k]] = conj(Znk);
  }
  __syncthreads();
  fft_inplace<T>(s, n, b.p, b.radix, tw, threadIdx.x, blockDim.x);
  const int valid = b.j_hi - b.j_lo;
  T* __restrict__ pr = part + part_off[blockIdx.y] * nrhs + r * valid;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const cx<T> v = s[j];
    const int j0 = 2 * j, j1 = 2 * j + 1;
    if (j0 >= b.j_lo && j0 < b.j_hi) pr[j0 - b.j_lo] = v.re * invw[j0];
    if (j1 >= b.j_lo && j1 < b.j_hi) pr[j1 - b.j_lo] = -v.im * invw[j1];
  }
}

// forward (rows = true): y[o] = sum of block partials + sum_j D[o][j] x[j]
// over the dense rectangles holding row o; adjoint: x[o] = ... + sum_i D[i][o] y[i].
// One warp per (o, RHS): lanes split each rectangle's line, then a fixed-order
// reduction; the block partials are added by lane 0 in list order.
template <typename T, bool ROWS>
__global__ void d2_combine_kernel(const BlockDev* __restrict__ out, const int* __restrict__ comb_ptr,
                                  const int* __restrict__ comb_ent, const int64_t* __restrict__ part_off,
                                  const T* __restrict__ part, const D2Rect* __restrict__ rects,
                                  const T* __restrict__ dense, const T* __restrict__ in, T* __restrict__ res,
                                  int64_t N, int64_t nrhs, int64_t ld) {
  const int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= N * nrhs) return;
  const int64_t r = t / N, o = t % N;
  const T* __restrict__ v = in + r * ld;
  T acc = T(0), blk = T(0);
  for (int e = comb_ptr[o]; e < comb_ptr[o + 1]; ++e) {
    const int id = comb_ent[e];
    if (id >= 0) {
      if (lane == 0) {
        const BlockDev& b = out[id];
        const int valid = b.j_hi - b.j_lo;
        const int64_t lo = int64_t(b.j_lo) - b.off;   // matrix index of the first valid output
        blk += part[part_off[id] * nrhs + r * valid + (o - lo)];
      }
    } else {
      const D2Rect q = rects[~id];
      const int64_t w = q.c1 - q.c0;
      const T* __restrict__ d = dense + q.off;
      if (ROWS) {
        const T* __restrict__ dr = d + (o - q.r0) * w;
        for (int64_t j = lane; j < w; j += 32) acc += dr[j] * v[q.c0 + j];
      } else {
        for (int64_t i = lane; i < q.r1 - q.r0; i += 32) acc += d[i * w + (o - q.c0)] * v[q.r0 + i];
      }
    }
  }
  for (int k = 16; k > 0; k >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, k);
  if (lane == 0) res[r * ld + o] = blk + acc;
}

int set_smem_2d(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) XC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return XC_OK;
}

template <typename T>
int run_dir(Plan* p, const D2Dir& D, bool rows, const T* x, T* y, int64_t nrhs, int64_t ld, cudaStream_t st) {
  const D2Plan* d2 = p->d2;
  const int nb = d2->nb;
  auto* spec = static_cast<cx<T>*>(p->scratch);
  cx<T>* z = spec + D.spec_in * nrhs;
  T* part = reinterpret_cast<T*>(z + D.spec_out * nrhs);
  const auto* in = static_cast<const BlockDev*>(D.in_dev);
  const auto* out = static_cast<const BlockDev*>(D.out_dev);
  if (nb > 0) {
    const size_t smi = size_t(D.max_n_in) * sizeof(cx<T>);
    XC_TRY(set_smem_2d(reinterpret_cast<const void*>(d2_in_kernel<T>), smi));
    launch_begin(p, K_2D_FFT_IN, st);
    d2_in_kernel<T><<<dim3(unsigned(nrhs), unsigned(nb)), kD2FftThreads, smi, st>>>(in, x, ld, spec, nrhs);
    launch_end(p, K_2D_FFT_IN, st);
    XC_CUDA(cudaGetLastError());
    launch_begin(p, K_2D_SPARSE, st);
    if (nrhs >= 16) {
      const int64_t warps = D.rows * ((nrhs + 31) / 32);
      d2_sparse_rhs_kernel<T><<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(
          in, out, D.ptr, D.idx, static_cast<const cx<T>*>(D.a), D.row_blk,
          D.row_loc, D.rows, spec, z, nrhs);
    } else {
      const int64_t warps = D.rows * nrhs;
      d2_sparse_kernel<T><<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(
          in, out, D.ptr, D.idx, static_cast<const cx<T>*>(D.a), D.row_blk,
          D.row_loc, D.rows, spec, z, nrhs);
    }
    launch_end(p, K_2D_SPARSE, st);
    XC_CUDA(cudaGetLastError());
    const size_t smo = size_t(D.max_n_out) * sizeof(cx<T>);
    XC_TRY(set_smem_2d(reinterpret_cast<const void*>(d2_out_kernel<T>), smo));
    launch_begin(p, K_2D_FFT_OUT, st);
    d2_out_kernel<T><<<dim3(unsigned(nrhs), unsigned(nb)), kD2FftThreads, smo, st>>>(out, z, D.part_off, part,
                                                                                     nrhs);
    launch_end(p, K_2D_FFT_OUT, st);
    XC_CUDA(cudaGetLastError());
  }
  const int64_t tot = p->N * nrhs * 32;   // one warp per (output, RHS)
  launch_begin(p, K_2D_COMBINE, st);
  if (rows)
    d2_combine_kernel<T, true><<<unsigned((tot + 255) / 256), 256, 0, st>>>(
        out, D.comb_ptr, D.comb_ent, D.part_off, part, d2->rects, static_cast<const T*>(d2->dense), x, y, p->N,
        nrhs, ld);
  else
    d2_combine_kernel<T, false><<<unsigned((tot + 255) / 256), 256, 0, st>>>(
        out, D.comb_ptr, D.comb_ent, D.part_off, part, d2->rects, static_cast<const T*>(d2->dense), x, y, p->N,
        nrhs, ld);
  launch_end(p, K_2D_COMBINE, st);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

}  // namespace

size_t d2_scratch_bytes(const Plan* p, int64_t nrhs) {
  const D2Plan* d2 = p->d2;
  const size_t e = p->elem_bytes();
  size_t per = 0;
  for (const D2Dir* D : {&d2->fwd, &d2->adj})
    per = std::max(per, size_t(D->spec_in + D->spec_out) * 2 * e + size_t(D->parts) * e);
  return std::max<size_t>(256, per * size_t(nrhs) + 256);
}

int launch_apply_2d(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t st, bool adjoint) {
  const D2Dir& D = adjoint ? p->d2->adj : p->d2->fwd;
  if (nrhs > 65535) return fail(XC_ERR_UNSUPPORTED, "the 2-D scheme takes up to 65535 right-hand sides per call");
  if (p->io64())
    return run_dir<double>(p, D, !adjoint, static_cast<const double*>(x), static_cast<double*>(y), nrhs, ld, st);
  return run_dir<float>(p, D, !adjoint, static_cast<const float*>(x), static_cast<float*>(y), nrhs, ld, st);
}

}  // namespace xc
