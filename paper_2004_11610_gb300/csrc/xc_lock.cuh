// Lockstep (window) band items of the many-plan batch (xc_batch.cu): the
// band products of plans whose window layouts are tight, register-blocked and
// fed through a per-warp staging ring in shared memory.
#pragma once

#include <cuda_runtime.h>

#include "xc_fft.cuh"
#include "xc_internal.h"
#include "xc_items.cuh"

namespace xc {

// ------------------------------------------- lockstep (window) band items
// The batch's items for plans whose window layouts are tight (see BlockDev).
// In the window layout the 32 rows of a slice (forward) or the 32 bins of a
// bin slice (adjoint) step through the same bin (row), so the band product of
// a window position is a small dense outer product, and each lane can own a
// block of it: RL rows (bins) x 8 right-hand sides, register-blocked like a
// GEMM micro-kernel.  Per window position a lane loads its RL band values and
// 8 right-hand-side values and does 16 RL multiply-adds, where the row-per-lane
// items load one right-hand-side value for every two: the loads, not the
// arithmetic, limit those (every value a lane uses must reach its registers).
// Lane = rg + (32 / RL) qg: row (bin) group rg of RL, right-hand-side group qg
// of 8.  Stored zeros outside a lane's band leave its sums unchanged, and each
// row's nonzero terms come in ascending bin order, as in fwd_sparse_item.

// Right-hand sides per lockstep item: RL groups of 8.
template <int RL>
__host__ __device__ constexpr int lock_rhs() { return 8 * RL; }

// RL complex band values of consecutive rows from p (16-byte aligned for RL >= 2).
template <typename T, int RL>
__device__ __forceinline__ void load_rl(const cx<T>* __restrict__ p, cx<T> (&c)[RL]) {
  if constexpr (sizeof(T) == 4 && RL % 2 == 0) {
#pragma unroll
    for (int i = 0; i < RL; i += 2) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p + i));
      c[i] = cx<T>{t.x, t.y};
      c[i + 1] = cx<T>{t.z, t.w};
    }
  } else {
#pragma unroll
    for (int i = 0; i < RL; ++i) c[i] = p[i];
  }
}

// ---- per-warp staging ring (batch band phase)
// The lockstep loops are latency-bound with loads issued from registers (a
// warp waits on every window position's loads).  In the batch they stage
// each window position's band values and right-hand-side values in a ring
// of kRingStages slots of this warp's part of the CTA's shared memory
// (idle during the band phase) with asynchronous copies, kRingStages - 1
// positions ahead of the arithmetic.
constexpr int kRingStages = 8;
constexpr int kRingSlot = 512;   // bytes per position: 256 band values + up to 256 RHS values
constexpr int kRingBytes = kRingStages * kRingSlot;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// RL complex values from shared memory (16-byte aligned for RL >= 2).
template <int RL>
__device__ __forceinline__ void lds_rl(const cx<float>* p, cx<float> (&c)[RL]) {
  if constexpr (RL % 2 == 0) {
#pragma unroll
    for (int i = 0; i < RL; i += 2) {
      const float4 t = *reinterpret_cast<const float4*>(p + i);
      c[i] = cx<float>{t.x, t.y};
      c[i + 1] = cx<float>{t.z, t.w};
    }
  } else {
#pragma unroll
    for (int i = 0; i < RL; ++i) c[i] = p[i];
  }
}

// Window positions [w0, w1) of forward slice `slice` of block b through the
// warp's ring (FP32): position w's 32 band values (256 bytes) and the 8 RL
// spectrum values of the item's right-hand sides (64 RL bytes) are copied
// by the lanes as 16-byte pieces; each lane then reads its RL band values
// and its 8 spectrum values from shared memory.
template <int RL, bool COMP>
__device__ __forceinline__ void lock_band_fwd_ring(const BlockDev& b, int64_t slice, int lane, int rg, int qg,
                                                   const cx<float>* __restrict__ F, int rp, int64_t r0, int w0,
                                                   int w1, unsigned char* ring, Acc<float, COMP> (&acc)[RL][8]) {
  constexpr int NF = RL * 4;   // lanes copying the 8 RL spectrum values (16 bytes each)
  // lane l < 16 copies bytes [16 l, 16 l + 16) of the position's band values,
  // lane 16 + m the m-th 16 bytes of its spectrum values (right-hand sides
  // r0 + 2m and r0 + 2m + 1): one source pointer and one stride per lane,
  // destination slot + 16 l.  Spectrum rows hold rp values: the lanes past
  // them copy nothing (an item of 8 RL right-hand sides can reach past rp,
  // and past the last bin's row that would read beyond the spectra), and
  // the slots they leave stale feed only sums of right-hand sides >= rp,
  // which are never written.
  const bool copier = lane < 16 || (lane < 16 + NF && r0 + 2 * (lane - 16) < rp);
  const unsigned char* src =
      lane < 16 ? reinterpret_cast<const unsigned char*>(static_cast<const cx<float>*>(b.lf_val) + b.lf_off[slice]) +
                      lane * 16
                : reinterpret_cast<const unsigned char*>(F + b.spec_off * rp + int64_t(b.lf_lo[slice]) * rp + r0) +
                      (lane - 16) * 16;
  const int64_t stride = lane < 16 ? 256 : int64_t(rp) * 8;
  src += int64_t(w0) * stride;
  unsigned char* const dst0 = ring + lane * 16;
  int wi = w0;   // next position to copy
  auto issue = [&](int slot) {
    if (copier && wi < w1) cp_async16(dst0 + slot * kRingSlot, src);
    src += stride;
    ++wi;
    cp_async_commit();   // one group per position, empty past the end
  };
#pragma unroll
  for (int st = 0; st < kRingStages - 1; ++st) issue(st);
  int slot = 0;
  for (int w = w0; w < w1; ++w) {
    issue(slot == 0 ? kRingStages - 1 : slot - 1);
    cp_async_wait<kRingStages - 1>();   // position w's group has landed (this lane's copies)
    __syncwarp();                       // ... and every lane's
    const unsigned char* sl = ring + slot * kRingSlot;
    cx<float> c[RL];
    lds_rl<RL>(reinterpret_cast<const cx<float>*>(sl) + rg * RL, c);
#pragma unroll
    for (int h = 0; h < 8; h += 4) {
      cx<float> g[4];
      lds_rl<4>(reinterpret_cast<const cx<float>*>(sl + 256) + qg * 8 + h, g);
#pragma unroll
      for (int i = 0; i < RL; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[i][h + q].add(c[i].re, g[q].re);
          acc[i][h + q].add(c[i].im, g[q].im);
        }
    }
    __syncwarp();                       // the slot is refilled by the next iteration's copy
    slot = slot + 1 == kRingStages ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  __syncwarp();
}

// Window positions [w0, w1) of forward slice `slice` of block b: F points at
// the block's bin-major spectra (bin k of RHS r at k * rp + r, rp a multiple
// of 8), right-hand sides [r0 + 8 qg, r0 + 8 qg + 8).
template <typename T, int RL, bool COMP>
__device__ __forceinline__ void lock_band_fwd(const BlockDev& b, int64_t slice, int rg, int qg,
                                              const cx<T>* __restrict__ F, int rp, int64_t r0, int w0, int w1,
                                              Acc<T, COMP> (&acc)[RL][8]) {
  const cx<T>* __restrict__ val = static_cast<const cx<T>*>(b.lf_val) + b.lf_off[slice] + rg * RL;
  const cx<T>* __restrict__ f =
      F + b.spec_off * rp + int64_t(b.lf_lo[slice]) * rp + r0 + 8 * qg;
#pragma unroll 1
  for (int w = w0; w < w1; ++w) {
    cx<T> c[RL];
    load_rl<T, RL>(val + w * 32, c);
    const cx<T>* __restrict__ fw = f + int64_t(w) * rp;
    // the 8 right-hand sides in two halves, so that only 4 spectrum values
    // are live beside the accumulators
#pragma unroll
    for (int h = 0; h < 8; h += 4) {
      cx<T> g[4];
      load_rl<T, 4>(fw + h, g);
#pragma unroll
      for (int i = 0; i < RL; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[i][h + q].add(c[i].re, g[q].re);
          acc[i][h + q].add(c[i].im, g[q].im);
        }
    }
  }
}

// Forward item (row slice, right-hand sides [r_begin, r_begin + 8 RL)) of a
// plan without chunked bands: every block's window, then the dense tail;
// writes y.  The sums are those of xc_apply's fwd_sparse_item.
template <typename T, int RL, bool COMP>
__device__ void fwd_lock_item(const BlockDev* __restrict__ blocks, int nblocks, int64_t N, const T* __restrict__ x,
                              int64_t ld, T* __restrict__ y, const cx<T>* __restrict__ spec, int rp, int64_t nrhs,
                              const T* __restrict__ rowscale, const T* __restrict__ colscale,
                              const T* __restrict__ tail, int64_t m_tail, int64_t slice, int64_t r_begin, int lane,
                              unsigned char* ring = nullptr) {
  constexpr int NG = 32 / RL;   // row groups
  const int rg = lane % NG, qg = lane / NG;
  const int64_t rq = r_begin + 8 * qg;        // this lane's first right-hand side
  Acc<T, COMP> acc[RL][8];
  for (int i = 0; i < nblocks; ++i) {
    const BlockDev& b = blocks[i];
    if constexpr (sizeof(T) == 4) {
      if (ring) {   // every lane takes part in the copies, whatever its right-hand sides
        lock_band_fwd_ring<RL, COMP>(b, slice, lane, rg, qg, spec, rp, r_begin, 0, b.lf_len[slice], ring, acc);
        continue;
      }
    }
    if (rq < nrhs) lock_band_fwd<T, RL, COMP>(b, slice, rg, qg, spec, rp, r_begin, 0, b.lf_len[slice], acc);
  }
  if (rq >= nrhs) return;
  const int nq = int(nrhs - rq < 8 ? nrhs - rq : 8);
#pragma unroll
  for (int i = 0; i < RL; ++i) {
    const int64_t n = slice * 32 + rg * RL + i;
    if (n >= N) continue;
    for (int64_t m = 0; m < m_tail; ++m) {
      const T tv = tail[m * N + n];
      const T cs = colscale ? colscale[m] : T(1);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < nq) acc[i][q].add(tv, x[(rq + q) * ld + m] * cs);
    }
    const T rs = rowscale ? rowscale[n] : T(1);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < nq) y[(rq + q) * ld + n] = acc[i][q].value() * rs;
  }
}

// Forward unit (block, slice, window positions [unit.z, unit.z + unit.w)) of
// a plan with chunked bands, right-hand sides [r_begin, r_begin + 8 RL):
// partial sums to part[u][rhs][row], as fwd_unit_item.
template <typename T, int RL, bool COMP>
__device__ void fwd_lock_unit(const BlockDev* __restrict__ blocks, const cx<T>* __restrict__ spec, int rp,
                              int64_t nrhs, cx<T>* __restrict__ part, int4 unit, int64_t u, int64_t r_begin,
                              int lane, unsigned char* ring = nullptr) {
  constexpr int NG = 32 / RL;
  const int rg = lane % NG, qg = lane / NG;
  const int64_t rq = r_begin + 8 * qg;
  Acc<T, COMP> acc[RL][8];
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (ring) {   // every lane takes part in the copies
      lock_band_fwd_ring<RL, COMP>(blocks[unit.x], unit.y, lane, rg, qg, spec, rp, r_begin, unit.z, unit.z + unit.w,
                                   ring, acc);
      done = true;
    }
  }
  if (rq >= nrhs) return;
  if (!done)
    lock_band_fwd<T, RL, COMP>(blocks[unit.x], unit.y, rg, qg, spec, rp, r_begin, unit.z, unit.z + unit.w, acc);
  const int nq = int(nrhs - rq < 8 ? nrhs - rq : 8);
#pragma unroll
  for (int i = 0; i < RL; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < nq) part[(u * nrhs + rq + q) * 32 + rg * RL + i] = cx<T>{acc[i][q].s, acc[i][q].c};
}

// adj_lock_item through the warp's ring (FP32): per window row the 32 bins'
// band values (16-byte pieces) and the 8 RL right-hand-side values of y at
// that row (4-byte pieces) are staged kRingStages - 1 rows ahead.
template <int RL, bool COMP>
__device__ void adj_lock_item_ring(const BlockDev* __restrict__ blocks, int nblocks, const float* __restrict__ y,
                                   int64_t ld, cx<float>* __restrict__ part, int64_t nrhs,
                                   const float* __restrict__ rowscale, const int* __restrict__ cbase, int2 it,
                                   int64_t r_begin, int lane, unsigned char* ring) {
  constexpr int NG = 32 / RL;
  constexpr int NY = 8 * RL;   // right-hand sides of the item, one copying lane each (lanes 16 ..)
  static_assert(NY <= 16, "lanes 16..31 copy the item's right-hand-side values");
  const int bg = lane % NG, qg = lane / NG;
  const int64_t rq = r_begin + 8 * qg;
  int i = 0;
  while (i < nblocks - 1 && it.x >= blocks[i].t_gbase + blocks[i].tslices) ++i;
  const BlockDev& b = blocks[i];
  const int gl = it.x - b.t_gbase;
  const int len = b.lt_len[gl];
  const int w0 = it.y * kAdjChunk;
  const int w1 = min(len, w0 + kAdjChunk);
  const int64_t lo = b.lt_lo[gl];
  // lane l < 16 copies bytes [16 l, 16 l + 16) of the row's band values,
  // lane 16 + q the row's value of right-hand side r_begin + q (when it exists)
  const int yq = lane - 16;
  const bool copies_y = yq >= 0 && yq < NY && r_begin + yq < nrhs;
  const unsigned char* bsrc =
      reinterpret_cast<const unsigned char*>(static_cast<const cx<float>*>(b.lt_val) + b.lt_off[gl]) + lane * 16 +
      int64_t(w0) * 256;
  const float* ysrc = y + (r_begin + (copies_y ? yq : 0)) * ld + lo + w0;
  unsigned char* const dst0 = lane < 16 ? ring + lane * 16 : ring + 256 + yq * 4;
  int wi = w0;
  auto issue = [&](int slot) {
    if (wi < w1) {
      if (lane < 16) cp_async16(dst0 + slot * kRingSlot, bsrc);
      else if (copies_y) cp_async4(dst0 + slot * kRingSlot, ysrc);
    }
    bsrc += 256;
    ++ysrc;
    ++wi;
    cp_async_commit();
  };
  Acc<float, COMP> re[RL][8], im[RL][8];
#pragma unroll
  for (int st = 0; st < kRingStages - 1; ++st) issue(st);
  int slot = 0;
  for (int w = w0; w < w1; ++w) {
    issue(slot == 0 ? kRingStages - 1 : slot - 1);
    cp_async_wait<kRingStages - 1>();
    __syncwarp();
    const unsigned char* sl = ring + slot * kRingSlot;
    cx<float> c[RL];
    lds_rl<RL>(reinterpret_cast<const cx<float>*>(sl) + bg * RL, c);
    const float rs = rowscale ? rowscale[lo + w] : 1.f;
    const float* yv = reinterpret_cast<const float*>(sl + 256) + qg * 8;
#pragma unroll
    for (int h = 0; h < 8; h += 4) {
      const float4 t = *reinterpret_cast<const float4*>(yv + h);
      const float v[4] = {t.x * rs, t.y * rs, t.z * rs, t.w * rs};
#pragma unroll
      for (int k = 0; k < RL; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          re[k][h + q].add(c[k].re, v[q]);
          im[k][h + q].add(c[k].im, v[q]);
        }
    }
    __syncwarp();
    slot = slot + 1 == kRingStages ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  __syncwarp();
  if (rq >= nrhs) return;
  const int nq = int(nrhs - rq < 8 ? nrhs - rq : 8);
  cx<float>* out = part + (cbase[it.x] + it.y) * nrhs * 32;
#pragma unroll
  for (int k = 0; k < RL; ++k)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < nq) out[(rq + q) * 32 + bg * RL + k] = cx<float>{re[k][q].value(), im[k][q].value()};
}

// Adjoint item (global bin slice it.x, chunk it.y of kAdjChunk window rows),
// right-hand sides [r_begin, r_begin + 8 RL): lane = (bin group of RL, RHS
// group of 8); per window row its RL band values (contiguous) and the 8
// right-hand-side values of y at that row.  Partial sums to
// part[(cbase[it.x] + it.y)][rhs][bin], as adj_sparse_item.
template <typename T, int RL, bool COMP>
__device__ void adj_lock_item(const BlockDev* __restrict__ blocks, int nblocks, const T* __restrict__ y, int64_t ld,
                              cx<T>* __restrict__ part, int64_t nrhs, const T* __restrict__ rowscale,
                              const int* __restrict__ cbase, int2 it, int64_t r_begin, int lane,
                              unsigned char* ring = nullptr) {
  constexpr int NG = 32 / RL;
  const int bg = lane % NG, qg = lane / NG;
  const int64_t rq = r_begin + 8 * qg;
  if constexpr (sizeof(T) == 4) {
    if (ring) {
      adj_lock_item_ring<RL, COMP>(blocks, nblocks, y, ld, part, nrhs, rowscale, cbase, it, r_begin, lane, ring);
      return;
    }
  }
  if (rq >= nrhs) return;
  int i = 0;
  while (i < nblocks - 1 && it.x >= blocks[i].t_gbase + blocks[i].tslices) ++i;
  const BlockDev& b = blocks[i];
  const int gl = it.x - b.t_gbase;
  const int len = b.lt_len[gl];
  const int w0 = it.y * kAdjChunk;
  const int w1 = min(len, w0 + kAdjChunk);
  const int64_t lo = b.lt_lo[gl];
  const cx<T>* __restrict__ val = static_cast<const cx<T>*>(b.lt_val) + b.lt_off[gl] + bg * RL;
  const int nq = int(nrhs - rq < 8 ? nrhs - rq : 8);
  const T* __restrict__ yq = y + rq * ld;
  Acc<T, COMP> re[RL][8], im[RL][8];
#pragma unroll 1
  for (int w = w0; w < w1; ++w) {
    cx<T> c[RL];
    load_rl<T, RL>(val + w * 32, c);
    const int64_t row = lo + w;
    const T rs = rowscale ? rowscale[row] : T(1);
#pragma unroll
    for (int h = 0; h < 8; h += 4) {   // right-hand sides in two halves (fewer live values)
      T v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = h + q < nq ? __ldg(yq + (h + q) * ld + row) * rs : T(0);
#pragma unroll
      for (int k = 0; k < RL; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          re[k][h + q].add(c[k].re, v[q]);
          im[k][h + q].add(c[k].im, v[q]);
        }
    }
  }
  cx<T>* out = part + (cbase[it.x] + it.y) * nrhs * 32;
#pragma unroll
  for (int k = 0; k < RL; ++k)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < nq) out[(rq + q) * 32 + bg * RL + k] = cx<T>{re[k][q].value(), im[k][q].value()};
}

}  // namespace xc
