// Device bodies of the execution stage, shared by the single-plan kernels
// (xc_apply.cu) and the many-plan persistent kernel (xc_batch.cu).
//
// Forward, y = A x (Algorithm 1 step 2 / Algorithm 3):
//   fwd_fft_body      one (block, RHS): extend the input with zero extra
//                     components (eqs. (Fe1), (Fe3)), multiply by W^{-1}, real
//                     FFT -> half spectrum F_k = sum_j u_j exp(-2 pi i jk / L)
//   fwd_sparse_item   one (32-row slice, RPW right-hand sides): y_n = sum over
//                     blocks of sum_k Re(C_nk conj(F_k)) over the row's band,
//                     plus the dense tail; C = g_k A_e W F / sqrt(L) carries the
//                     unitary and half-spectrum factors, so
//                     Re(C conj F) = Re C Re F + Im C Im F.
//   fwd_unit_item     the same over one chunk of a slice's band (plans with
//                     long bands), partial sums out
//   fwd_reduce_row    one (row, RHS): adds a chunked slice's partials and the
//                     dense tail.
// Adjoint, x = A^T y (Algorithm 2 step 2 / Algorithm 4):
//   transpose_tile    y [rhs][row] -> yt [row][rhs] for the adjoint products
//   adj_sparse_item   one (chunk of rows of a 32-bin slice, RPW RHS): partial
//                     sums of z_k = sum_n CT_kn y_n
//   adj_fft_body      one (block, RHS): add the chunk partials, real inverse
//                     FFT, W^{-1}, keep [j_lo, j_hi) and discard the extra
//                     components (eq. (Fe2))
//   adj_tail_warp     one (m, RHS): x_m from the dense tail.
#pragma once

#include <cuda_runtime.h>

#include "xc_fft.cuh"
#include "xc_internal.h"

namespace xc {

// Plain or compensated (TwoProduct + TwoSum) sum of products.
template <typename T, bool COMP>
struct Acc {
  T s = 0, c = 0;
  __device__ __forceinline__ void add(T a, T b) {
    if constexpr (!COMP) {
      s = fma(a, b, s);
    } else {
      const T p = a * b;
      const T e = fma(a, b, -p);          // a*b = p + e exactly
      const T t = s + p;                  // TwoSum(s, p)
      const T bb = t - s;
      const T err = (s - (t - bb)) + (p - bb);
      s = t;
      c += err + e;
    }
  }
  // adds a partial sum given as a (sum, compensation) pair
  __device__ __forceinline__ void add_pair(T ps, T pc) {
    if constexpr (!COMP) {
      s += ps;
    } else {
      const T t = s + ps;
      const T bb = t - s;
      const T err = (s - (t - bb)) + (ps - bb);
      s = t;
      c += err + pc;
    }
  }
  __device__ __forceinline__ T value() const { return COMP ? s + c : s; }
};

// ------------------------------------------------------ FP32 pairs
// XC_FP64_PAIR plans keep FP64 vectors and FFTs but store band values and
// spectra as pairs of FP32 numbers, v = hi + lo with |lo| <= ulp(hi)/2
// (48-bit significands), and run the band products on the FP32 pipes: a
// product a*b of pairs is hi*hi exactly (TwoProduct by FMA) plus the cross
// terms hi*lo + lo*hi, and the sum is accumulated with TwoSum, its errors
// collected in a second FP32 word.  The result matches FP64 accumulation to a
// few units of 2^-48 of the summed magnitudes, independently of the band
// length, while the FP32 pipes run 64 times the FP64 rate on this GPU.
struct __align__(16) PairCx {
  float re_hi, re_lo, im_hi, im_lo;
};

__device__ __forceinline__ float2 to_pair(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - double(hi)));
}
__device__ __forceinline__ PairCx to_pair(double re, double im) {
  const float2 a = to_pair(re), b = to_pair(im);
  return PairCx{a.x, a.y, b.x, b.y};
}

struct AccPair {
  float s = 0.f, c = 0.f;
  // += (ah + al) (bh + bl)
  __device__ __forceinline__ void add(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);               // ah*bh = p + e exactly
    const float x = fmaf(ah, bl, al * bh);          // cross terms
    const float t = s + p;                           // TwoSum(s, p)
    const float bb = t - s;
    const float err = (s - (t - bb)) + (p - bb);
    s = t;
    c += err + (e + x);
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// ------------------------------------------------------ band streaming
// A band value is read once per item: in the single-plan FP32 adjoint
// product (STREAM) it is loaded evict-first, so that it does not displace the
// right-hand-side lines that the slice's other rows re-read from L1 (Legendre
// N = 32768, 128 RHS: adjoint 0.43 -> 0.33 ms).  Elsewhere the normal load is
// kept: FP64 items of other right-hand-side groups re-read the same values
// from L1 (evict-first cost the FP64 adjoint 58 %), and the batch kernel's
// adjoint ran 2 % slower with it.
template <typename T>
__device__ __forceinline__ cx<T> load_band(const cx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    const float2 t = __ldcs(reinterpret_cast<const float2*>(p));
    return cx<T>{t.x, t.y};
  } else {
    const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    return cx<T>{t.x, t.y};
  }
}

// Band rows [j0, j1) of a slice whose value (j, lane) sits at base[j*32 + lane]:
// step(j) is called for every row in order, four rows per unrolled iteration
// so that their loads are in flight together.  (An L2 bulk prefetch of the
// item's values ahead of the loop was measured: about 4% faster on the
// 1000-plan batch, up to 1.6x slower on single plans whose bands already sit
// in L2; not used.)
template <typename T, typename Step>
__device__ __forceinline__ void band_rows(int j0, int j1, Step&& step) {
#pragma unroll 4
  for (int j = j0; j < j1; ++j) step(j);
}

// Forward band product of rows [j0, j1) for RPW right-hand sides: lane = row,
// acc[q] += Re C Re F + Im C Im F with F the spectrum of RHS q from bin k0 + j.
template <typename T, int RPW, bool COMP>
__device__ __forceinline__ void fwd_band(const cx<T>* __restrict__ base, int lane, const cx<T>* __restrict__ F,
                                         int H, int j0, int j1, int nq, Acc<T, COMP> (&acc)[RPW]) {
  const cx<T>* __restrict__ val = base + lane;
  if (nq == RPW) {
    band_rows<T>(j0, j1, [&](int j) {
      const cx<T> c = val[j * 32];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const cx<T> f = F[q * H + j];
        acc[q].add(c.re, f.re);
        acc[q].add(c.im, f.im);
      }
    });
  } else {
    band_rows<T>(j0, j1, [&](int j) {
      const cx<T> c = val[j * 32];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (q < nq) {
          const cx<T> f = F[q * H + j];
          acc[q].add(c.re, f.re);
          acc[q].add(c.im, f.im);
        }
      }
    });
  }
}

// ------------------------------------------------------------ forward FFT
// With `pair_exp` (FP64 plans whose band products run in FP32 pairs), the
// spectrum is written as pairs (see PairCx) scaled by 2^-pair_exp[r].
// `mem` is this CTA's shared memory (LocalMem) or a cluster's distributed
// shared memory (ClusterMem) for blocks too long for one CTA; `sync` is the
// matching barrier; tid / nthreads count over all CTAs that share the array.
// With rp > 0 the spectrum goes out bin-major, bin k of RHS r at
// spec + spec_off * rp + k * rp + r (the layout of the lockstep band items);
// otherwise RHS-major, spec + spec_off * nrhs + r * H + k.
template <typename T, class M, class Sync>
__device__ void fwd_fft_run(const BlockDev& b, int64_t r, const T* __restrict__ x, int64_t ld,
                            const T* __restrict__ colscale, cx<T>* __restrict__ spec, int64_t nrhs, const M& mem,
                            int tid, int nthreads, Sync sync, const int* __restrict__ pair_exp, int rp = 0) {
  const int n = b.n, j_lo = b.j_lo, j_hi = b.j_hi, off = b.off;
  const T* __restrict__ invw = static_cast<const T*>(b.invw);
  const int* __restrict__ perm = b.perm;
  const cx<T>* __restrict__ tw = static_cast<const cx<T>*>(b.tw);
  const T* __restrict__ xr = x + r * ld;
  for (int j = tid; j < n; j += nthreads) {
    const int j0 = 2 * j, j1 = 2 * j + 1;
    T u0 = T(0), u1 = T(0);
    if (j0 >= j_lo && j0 < j_hi) {
      T v = xr[j0 - off];
      if (colscale) v *= colscale[j0 - off];
      u0 = v * invw[j0];
    }
    if (j1 >= j_lo && j1 < j_hi) {
      T v = xr[j1 - off];
      if (colscale) v *= colscale[j1 - off];
      u1 = v * invw[j1];
    }
    mem.at(perm[j]) = cx<T>{u0, u1};
  }
  sync();
  fft_run<T>(mem, n, b.p, b.radix, tw, tid, nthreads, sync);
  cx<T>* out = spec + b.spec_off * nrhs + r * int64_t(n + 1);
  if constexpr (sizeof(T) == 8) {
    if (pair_exp) {
      const int e = -pair_exp[r];
      PairCx* po = reinterpret_cast<PairCx*>(out);
      for (int k = tid; k <= n / 2; k += nthreads) {
        cx<T> Uk, Unk;
        r2c_split_vals(mem.at(k), mem.at(k == 0 ? 0 : n - k), k, tw, &Uk, &Unk);
        po[k] = to_pair(ldexp(Uk.re, e), ldexp(Uk.im, e));
        if (n - k != k) po[n - k] = to_pair(ldexp(Unk.re, e), ldexp(Unk.im, e));
      }
      return;
    }
  }
  if (rp > 0) {
    cx<T>* bo = spec + b.spec_off * rp + r;
    for (int k = tid; k <= n / 2; k += nthreads) {
      cx<T> Uk, Unk;
      r2c_split_vals(mem.at(k), mem.at(k == 0 ? 0 : n - k), k, tw, &Uk, &Unk);
      bo[int64_t(k) * rp] = Uk;
      if (n - k != k) bo[int64_t(n - k) * rp] = Unk;
    }
    return;
  }
  for (int k = tid; k <= n / 2; k += nthreads) {
    cx<T> Uk, Unk;
    r2c_split_vals(mem.at(k), mem.at(k == 0 ? 0 : n - k), k, tw, &Uk, &Unk);
    out[k] = Uk;
    if (n - k != k) out[n - k] = Unk;
  }
}

template <typename T>
__device__ void fwd_fft_body(const BlockDev& b, int64_t r, const T* __restrict__ x, int64_t ld,
                             const T* __restrict__ colscale, cx<T>* __restrict__ spec, int64_t nrhs, cx<T>* s,
                             int tid, int nthreads, const int* __restrict__ pair_exp = nullptr, int rp = 0) {
  fwd_fft_run<T>(b, r, x, ld, colscale, spec, nrhs, LocalMem<T>{s}, tid, nthreads, [] { __syncthreads(); },
                 pair_exp, rp);
}

// ------------------------------------------------------- forward sparse
// Lane = row.  Each band value is loaded once (coalesced across the slice)
// and used for the RPW right-hand sides; the spectra are gathered through L1.
// `groups` consecutive groups of RPW right-hand sides starting at r_begin are
// processed one after the other (the slice's band layout is read once).
template <typename T, int RPW, bool COMP>
__device__ void fwd_sparse_item(const BlockDev* __restrict__ blocks, int nblocks, int64_t N,
                                const T* __restrict__ x, int64_t ld, T* __restrict__ y,
                                const cx<T>* __restrict__ spec, int64_t nrhs, const T* __restrict__ rowscale,
                                const T* __restrict__ colscale, const T* __restrict__ tail, int64_t m_tail,
                                int64_t slice, int64_t r_begin, int lane, int groups = 1) {
  const int64_t n = slice * 32 + lane;
  for (int grp = 0; grp < groups; ++grp) {
  const int64_t r0 = r_begin + int64_t(grp) * RPW;
  if (r0 >= nrhs) break;
  const int nq = int(nrhs - r0 < RPW ? nrhs - r0 : RPW);
  Acc<T, COMP> acc[RPW];
  for (int i = 0; i < nblocks; ++i) {
    const BlockDev& b = blocks[i];
    const int W = b.f_width[slice];
    const int k0 = b.f_k0[n];
    const int H = b.H;
    fwd_band<T, RPW, COMP>(static_cast<const cx<T>*>(b.f_val) + b.f_off[slice], lane,
                           spec + b.spec_off * nrhs + r0 * H + k0, H, 0, W, nq, acc);
  }
  if (n < N) {
    for (int64_t m = 0; m < m_tail; ++m) {
      const T tv = tail[m * N + n];
      const T cs = colscale ? colscale[m] : T(1);
#pragma unroll
      for (int q = 0; q < RPW; ++q)
        if (q < nq) acc[q].add(tv, x[(r0 + q) * ld + m] * cs);
    }
    const T rs = rowscale ? rowscale[n] : T(1);
#pragma unroll
    for (int q = 0; q < RPW; ++q)
      if (q < nq) y[(r0 + q) * ld + n] = acc[q].value() * rs;
  }
  }
}

// ------------------------------------------- forward sparse, chunked bands
// Plans whose bands run to thousands of bins (Hermite and Laguerre functions)
// have few row slices with long serial loops; their bands are cut into units
// (block, slice, chunk of kFwdChunk band rows).  A unit writes the partial
// sums of its rows as (sum, compensation) pairs to part[u][rhs][lane];
// fwd_reduce_row adds the units of a slice in unit order (deterministic).
template <typename T, int RPW, bool COMP>
__device__ void fwd_unit_item(const BlockDev* __restrict__ blocks, const cx<T>* __restrict__ spec, int64_t nrhs,
                              cx<T>* __restrict__ part, int4 unit, int64_t u, int64_t r_begin, int lane,
                              int groups = 1) {
  const BlockDev& b = blocks[unit.x];
  const int64_t slice = unit.y;
  const int64_t n = slice * 32 + lane;
  const int j0 = unit.z * kFwdChunk, j1 = j0 + unit.w;
  const int k0 = b.f_k0[n];
  const int H = b.H;
  const cx<T>* __restrict__ base = static_cast<const cx<T>*>(b.f_val) + b.f_off[slice];
  for (int grp = 0; grp < groups; ++grp) {
    const int64_t r0 = r_begin + int64_t(grp) * RPW;
    if (r0 >= nrhs) break;
    const int nq = int(nrhs - r0 < RPW ? nrhs - r0 : RPW);
    Acc<T, COMP> acc[RPW];
    fwd_band<T, RPW, COMP>(base, lane, spec + b.spec_off * nrhs + r0 * H + k0, H, j0, j1, nq, acc);
    cx<T>* out = part + (u * nrhs + r0) * 32 + lane;
#pragma unroll
    for (int q = 0; q < RPW; ++q)
      if (q < nq) out[q * 32] = cx<T>{acc[q].s, acc[q].c};
  }
}

// y_n for one (row n < N, RHS r) of a chunked plan: the unit partials of the
// row's slice in unit order, plus the dense tail, times the row scaling.
template <typename T, bool COMP>
__device__ __forceinline__ void fwd_reduce_row(int64_t N, const T* __restrict__ x, int64_t ld, T* __restrict__ y,
                                               const cx<T>* __restrict__ part, int64_t nrhs,
                                               const int* __restrict__ ubase, const T* __restrict__ rowscale,
                                               const T* __restrict__ colscale, const T* __restrict__ tail,
                                               int64_t m_tail, int64_t n, int64_t r) {
  const int64_t slice = n >> 5;
  const int lane = int(n & 31);
  Acc<T, COMP> acc;
  for (int64_t u = ubase[slice], u1 = ubase[slice + 1]; u < u1; ++u) {
    const cx<T> v = part[(u * nrhs + r) * 32 + lane];
    acc.add_pair(v.re, v.im);
  }
  for (int64_t m = 0; m < m_tail; ++m)
    acc.add(tail[m * N + n], x[r * ld + m] * (colscale ? colscale[m] : T(1)));
  y[r * ld + n] = acc.value() * (rowscale ? rowscale[n] : T(1));
}

// ------------------------------------------------------- adjoint sparse
// RPW consecutive values from p, which is aligned to RPW * sizeof(T) bytes
// (vector loads of up to 16 bytes).
template <typename T, int RPW>
__device__ __forceinline__ void load_rhs(const T* __restrict__ p, T (&v)[RPW]) {
  constexpr int bytes = RPW * int(sizeof(T));
  if constexpr (bytes >= 16) {
    constexpr int per = 16 / int(sizeof(T));
#pragma unroll
    for (int q = 0; q < RPW; q += per) {
      if constexpr (sizeof(T) == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p + q));
        v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
      } else {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p + q));
        v[q] = t.x; v[q + 1] = t.y;
      }
    }
  } else if constexpr (bytes == 8 && sizeof(T) == 4) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int q = 0; q < RPW; ++q) v[q] = __ldg(p + q);
  }
}

// Rows [j0, j1) of one bin-slice chunk for RPW right-hand sides from r0.
// y is read row-major by right-hand side ([rhs][ld]) or, with YT, from its
// transpose yt[row][ldt] (ldt a multiple of 8, columns beyond nrhs zero),
// where one lane's RPW values of a row are adjacent and a step reads one
// vector per lane.
template <typename T, int RPW, bool COMP, bool YT, bool STREAM>
__device__ __forceinline__ void adj_chunk_rows(const cx<T>* __restrict__ base, int lane, int64_t n0, int j0, int j1,
                                               const T* __restrict__ y, int64_t ld, int64_t r0, int nq,
                                               const T* __restrict__ rowscale, Acc<T, COMP> (&re)[RPW],
                                               Acc<T, COMP> (&im)[RPW]) {
  const cx<T>* __restrict__ val = base + lane;
  band_rows<T>(j0, j1, [&](int j) {
    const cx<T> c = (STREAM && sizeof(T) == 4) ? load_band(val + j * 32) : val[j * 32];
    const int64_t row = n0 + j;
    const T rs = rowscale ? rowscale[row] : T(1);
    if constexpr (YT) {
      T v[RPW];
      load_rhs<T, RPW>(y + row * ld + r0, v);
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        re[q].add(c.re, v[q] * rs);
        im[q].add(c.im, v[q] * rs);
      }
    } else {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (q < nq) {
          const T v = y[(r0 + q) * ld + row] * rs;
          re[q].add(c.re, v);
          im[q].add(c.im, v);
        }
      }
    }
  });
}

// Item (global bin slice g, chunk c): lane = bin k; the partial sum over rows
// [c*chunk, (c+1)*chunk) of the slice goes to part[chunk][rhs][lane].
// Blocks marked t_yt (their bins start at rows far apart, so that a step of
// scalar loads touches up to 32 sectors per right-hand side) read the
// transposed copy yt when USE_YT and yt is given; the others read y, where
// neighbouring bins share cache lines over many steps.
template <typename T, int RPW, bool COMP, bool USE_YT = false, bool STREAM = false>
__device__ void adj_sparse_item(const BlockDev* __restrict__ blocks, int nblocks, const T* __restrict__ y,
                                int64_t ld, const T* __restrict__ yt, int64_t ldt, cx<T>* __restrict__ part,
                                int64_t nrhs, const T* __restrict__ rowscale, const int* __restrict__ cbase, int2 it,
                                int chunk, int64_t r_begin, int lane, int groups = 1) {
  int i = 0;
  while (i < nblocks - 1 && it.x >= blocks[i].t_gbase + blocks[i].tslices) ++i;
  const BlockDev& b = blocks[i];
  const int gl = it.x - b.t_gbase;
  const int64_t k = int64_t(gl) * 32 + lane;
  const int W = b.t_width[gl];
  const int j0 = it.y * chunk;
  const int j1 = min(W, j0 + chunk);
  const int n0 = b.t_n0[k];
  const cx<T>* __restrict__ base = static_cast<const cx<T>*>(b.t_val) + b.t_off[gl];
  const int64_t cb = cbase[it.x];
  const bool from_yt = USE_YT && b.t_yt && yt != nullptr;
  for (int grp = 0; grp < groups; ++grp) {
    const int64_t r0 = r_begin + int64_t(grp) * RPW;
    if (r0 >= nrhs) break;
    const int nq = int(nrhs - r0 < RPW ? nrhs - r0 : RPW);
    Acc<T, COMP> re[RPW], im[RPW];
    if constexpr (USE_YT) {
      if (from_yt)
        adj_chunk_rows<T, RPW, COMP, true, STREAM>(base, lane, n0, j0, j1, yt, ldt, r0, nq, rowscale, re, im);
      else
        adj_chunk_rows<T, RPW, COMP, false, STREAM>(base, lane, n0, j0, j1, y, ld, r0, nq, rowscale, re, im);
    } else {
      adj_chunk_rows<T, RPW, COMP, false, STREAM>(base, lane, n0, j0, j1, y, ld, r0, nq, rowscale, re, im);
    }
    cx<T>* out = part + ((cb + it.y) * nrhs + r0) * 32 + lane;
#pragma unroll
    for (int q = 0; q < RPW; ++q)
      if (q < nq) out[q * 32] = cx<T>{re[q].value(), im[q].value()};
  }
}

// yt[n][ldt] = y[r][n] for r < nrhs, 0 for nrhs <= r < ldt: a 32 x 32 tile per
// CTA of 32 x 8 threads through shared memory (coalesced on both sides).
template <typename T>
__device__ __forceinline__ void transpose_tile(const T* __restrict__ y, int64_t ld, int64_t N, int64_t nrhs,
                                               T* __restrict__ yt, int64_t ldt, int64_t n_base, int64_t r_base,
                                               T (*tile)[33], int tx, int ty) {
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r_base + i, n = n_base + tx;
    tile[i][tx] = (r < nrhs && n < N) ? y[r * ld + n] : T(0);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int64_t n = n_base + i, r = r_base + tx;
    if (n < N && r < ldt) yt[n * ldt + r] = tile[tx][i];
  }
}

// ------------------------------------------- band products in FP32 pairs
// Forward band rows [j0, j1) for RPW right-hand sides, pairs (values, spectra).
template <int RPW>
__device__ __forceinline__ void fwd_band_pair(const PairCx* __restrict__ base, int lane,
                                              const PairCx* __restrict__ F, int H, int j0, int j1, int nq,
                                              AccPair (&acc)[RPW]) {
  const PairCx* __restrict__ val = base + lane;
  band_rows<double>(j0, j1, [&](int j) {
    const PairCx c = val[j * 32];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      if (q < nq) {
        const PairCx f = F[q * H + j];
        acc[q].add(c.re_hi, c.re_lo, f.re_hi, f.re_lo);
        acc[q].add(c.im_hi, c.im_lo, f.im_hi, f.im_lo);
      }
    }
  });
}

// fwd_sparse_item for pair plans: the band sums scaled back by 2^e[r] (the
// spectra were scaled by 2^-e[r]), the dense tail and the output in FP64.
template <int RPW>
__device__ void fwd_sparse_item_pair(const BlockDev* __restrict__ blocks, int nblocks, int64_t N,
                                     const double* __restrict__ x, int64_t ld, double* __restrict__ y,
                                     const PairCx* __restrict__ spec, int64_t nrhs, const int* __restrict__ pexp,
                                     const double* __restrict__ rowscale, const double* __restrict__ colscale,
                                     const double* __restrict__ tail, int64_t m_tail, int64_t slice, int64_t r_begin,
                                     int lane, int groups = 1) {
  const int64_t n = slice * 32 + lane;
  for (int grp = 0; grp < groups; ++grp) {
    const int64_t r0 = r_begin + int64_t(grp) * RPW;
    if (r0 >= nrhs) break;
    const int nq = int(nrhs - r0 < RPW ? nrhs - r0 : RPW);
    AccPair acc[RPW];
    for (int i = 0; i < nblocks; ++i) {
      const BlockDev& b = blocks[i];
      const int W = b.f_width[slice];
      const int k0 = b.f_k0[n];
      const int H = b.H;
      fwd_band_pair<RPW>(static_cast<const PairCx*>(b.f_val) + b.f_off[slice], lane,
                         spec + b.spec_off * nrhs + r0 * H + k0, H, 0, W, nq, acc);
    }
    if (n < N) {
      const double rs = rowscale ? rowscale[n] : 1.0;
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (q < nq) {
          double t = ldexp(acc[q].value(), pexp[r0 + q]);
          for (int64_t m = 0; m < m_tail; ++m)
            t = fma(tail[m * N + n], x[(r0 + q) * ld + m] * (colscale ? colscale[m] : 1.0), t);
          y[(r0 + q) * ld + n] = t * rs;
        }
      }
    }
  }
}

// fwd_unit_item for pair plans: the partial goes out as one FP64 value (in
// the `re` word of the plan's partial array), already scaled back.
template <int RPW>
__device__ void fwd_unit_item_pair(const BlockDev* __restrict__ blocks, const PairCx* __restrict__ spec,
                                   int64_t nrhs, const int* __restrict__ pexp, cx<double>* __restrict__ part,
                                   int4 unit, int64_t u, int64_t r_begin, int lane, int groups = 1) {
  const BlockDev& b = blocks[unit.x];
  const int64_t slice = unit.y;
  const int64_t n = slice * 32 + lane;
  const int j0 = unit.z * kFwdChunk, j1 = j0 + unit.w;
  const int k0 = b.f_k0[n];
  const int H = b.H;
  const PairCx* __restrict__ base = static_cast<const PairCx*>(b.f_val) + b.f_off[slice];
  for (int grp = 0; grp < groups; ++grp) {
    const int64_t r0 = r_begin + int64_t(grp) * RPW;
    if (r0 >= nrhs) break;
    const int nq = int(nrhs - r0 < RPW ? nrhs - r0 : RPW);
    AccPair acc[RPW];
    fwd_band_pair<RPW>(base, lane, spec + b.spec_off * nrhs + r0 * H + k0, H, j0, j1, nq, acc);
    cx<double>* out = part + (u * nrhs + r0) * 32 + lane;
#pragma unroll
    for (int q = 0; q < RPW; ++q)
      if (q < nq) out[q * 32] = cx<double>{ldexp(acc[q].value(), pexp[r0 + q]), 0.0};
  }
}

// adj_sparse_item for pair plans: y arrives as pairs yp[r][n] scaled by
// 2^-e[r]; the chunk partials go out in FP64, scaled back.
template <int RPW>
__device__ void adj_sparse_item_pair(const BlockDev* __restrict__ blocks, int nblocks,
                                     const float2* __restrict__ yp, int64_t N, const int* __restrict__ pexp,
                                     cx<double>* __restrict__ part, int64_t nrhs, const int* __restrict__ cbase,
                                     int2 it, int chunk, int64_t r_begin, int lane, int groups = 1) {
  int i = 0;
  while (i < nblocks - 1 && it.x >= blocks[i].t_gbase + blocks[i].tslices) ++i;
  const BlockDev& b = blocks[i];
  const int gl = it.x - b.t_gbase;
  const int64_t k = int64_t(gl) * 32 + lane;
  const int W = b.t_width[gl];
  const int j0 = it.y * chunk;
  const int j1 = min(W, j0 + chunk);
  const int64_t n0 = b.t_n0[k];
  const PairCx* __restrict__ val = static_cast<const PairCx*>(b.t_val) + b.t_off[gl] + lane;
  const int64_t cb = cbase[it.x];
  for (int grp = 0; grp < groups; ++grp) {
    const int64_t r0 = r_begin + int64_t(grp) * RPW;
    if (r0 >= nrhs) break;
    const int nq = int(nrhs - r0 < RPW ? nrhs - r0 : RPW);
    AccPair re[RPW], im[RPW];
    band_rows<double>(j0, j1, [&](int j) {
      const PairCx c = val[j * 32];
      const int64_t row = n0 + j;
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (q < nq) {
          const float2 v = yp[(r0 + q) * N + row];
          re[q].add(c.re_hi, c.re_lo, v.x, v.y);
          im[q].add(c.im_hi, c.im_lo, v.x, v.y);
        }
      }
    });
    cx<double>* out = part + ((cb + it.y) * nrhs + r0) * 32 + lane;
#pragma unroll
    for (int q = 0; q < RPW; ++q)
      if (q < nq) {
        const int e = pexp[r0 + q];
        out[q * 32] = cx<double>{ldexp(re[q].value(), e), ldexp(im[q].value(), e)};
      }
  }
}

// ------------------------------------------------------------ adjoint FFT
// Sum of the chunk partials of bin k of a block for right-hand side r.
template <typename T>
__device__ __forceinline__ cx<T> gather_bin(const cx<T>* __restrict__ part, const int* __restrict__ cbase,
                                            int gbase, int k, int64_t r, int64_t nrhs) {
  const int g = gbase + (k >> 5);
  const int c0 = cbase[g], c1 = cbase[g + 1];
  cx<T> u{T(0), T(0)};
  for (int c = c0; c < c1; ++c) u = u + part[(int64_t(c) * nrhs + r) * 32 + (k & 31)];
  return u;
}

template <typename T, class M, class Sync>
__device__ void adj_fft_run(const BlockDev& b, int64_t r, const cx<T>* __restrict__ part,
                            const int* __restrict__ cbase, int64_t nrhs, T* __restrict__ x, int64_t ld,
                            const T* __restrict__ colscale, const M& mem, int tid, int nthreads, Sync sync) {
  const int n = b.n, j_lo = b.j_lo, j_hi = b.j_hi, off = b.off;
  const int* __restrict__ perm = b.perm;
  const cx<T>* __restrict__ tw = static_cast<const cx<T>*>(b.tw);
  const T* __restrict__ invw = static_cast<const T*>(b.invw);
  for (int k = tid; k <= n / 2; k += nthreads) {
    cx<T> Uk = gather_bin(part, cbase, b.t_gbase, k, r, nrhs);
    cx<T> Unk = gather_bin(part, cbase, b.t_gbase, n - k, r, nrhs);
    if (k == 0) {
      Uk.im = T(0);    // U_0 and U_n enter as real numbers
      Unk.im = T(0);
    }
    cx<T> Zk, Znk;
    c2r_merge(Uk, Unk, k, tw, &Zk, &Znk);
    // inverse FFT as conj(FFT(conj(Z)))
    mem.at(perm[k]) = conj(Zk);
    if (k != 0 && n - k != k) mem.at(perm[n - k]) = conj(Znk);
  }
  sync();
  fft_run<T>(mem, n, b.p, b.radix, tw, tid, nthreads, sync);
  T* __restrict__ xr = x + r * ld;
  for (int j = tid; j < n; j += nthreads) {
    const cx<T> v = mem.at(j);
    const int j0 = 2 * j, j1 = 2 * j + 1;
    if (j0 >= j_lo && j0 < j_hi) {
      T u = v.re * invw[j0];
      if (colscale) u *= colscale[j0 - off];
      xr[j0 - off] = u;
    }
    if (j1 >= j_lo && j1 < j_hi) {
      T u = -v.im * invw[j1];
      if (colscale) u *= colscale[j1 - off];
      xr[j1 - off] = u;
    }
  }
}

template <typename T>
__device__ void adj_fft_body(const BlockDev& b, int64_t r, const cx<T>* __restrict__ part,
                             const int* __restrict__ cbase, int64_t nrhs, T* __restrict__ x, int64_t ld,
                             const T* __restrict__ colscale, cx<T>* s, int tid, int nthreads) {
  adj_fft_run<T>(b, r, part, cbase, nrhs, x, ld, colscale, LocalMem<T>{s}, tid, nthreads, [] { __syncthreads(); });
}

// ------------------------------------------------------------ adjoint tail
// One warp: x_m = colscale_m sum_n tail[m][n] rowscale_n y_n for one RHS.
template <typename T, bool COMP>
__device__ void adj_tail_warp(int64_t N, int64_t m, int64_t r, const T* __restrict__ tail, const T* __restrict__ y,
                              int64_t ld, T* __restrict__ x, const T* __restrict__ rowscale,
                              const T* __restrict__ colscale, int lane) {
  Acc<T, COMP> acc;
  for (int64_t n = lane; n < N; n += 32) acc.add(tail[m * N + n], y[r * ld + n] * (rowscale ? rowscale[n] : T(1)));
  T v = acc.value();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) x[r * ld + m] = v * (colscale ? colscale[m] : T(1));
}

}  // namespace xc
