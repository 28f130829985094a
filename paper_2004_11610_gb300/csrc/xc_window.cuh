// Forward band products of FP32 plans with dense windows on the tensor cores
// (the many-plan batch, xc_batch.cu).
//
// Plans whose bands are wide and move slowly from row to row (Hermite
// functions: over a thousand stored bins per row) store, besides their band
// layouts, tensor windows: per group of 128 rows and block, the union of the
// rows' stored bins [lo, lo + 16 nkb), as nkb tiles of 128 rows x 16 bins
// (WinBlock).  Over one window the band product of Algorithm 1 (step
// 3: y_n = sum_k Re(A_nk conj-folded . F_k)) is a dense contraction,
//   y[n][r] = sum_k  A[n][2k] F[k][r].re + A[n][2k+1] F[k][r].im,
// with K = 32 FP32 values per tile (16 bins, real and imaginary parts
// interleaved) and the spectra F in the bin-major layout of the lockstep
// items (bin k of RHS r at spec + (spec_off + k) rp + r).  Zeros stored
// outside a row's band leave its sum unchanged.
//
// Precision: 3xTF32 as in the dense comparator (xc_dense.cu): A = A_hi + A_lo
// and F = F_hi + F_lo split exactly into TF32 numbers, the product summed as
// A_hi F_hi + A_lo F_hi + A_hi F_lo; each tile's products start a fresh
// tensor-memory accumulator (the tensor core truncates when it adds), which
// the epilogue adds to FP32 registers with round-to-nearest additions.  The
// split is made on the SM, so the band tiles cross HBM once, as FP32: the
// band operand goes to tensor memory (read there by the MMAs, which would
// otherwise fetch the 128 x 8 operand from shared memory for every narrow
// product), the spectra to shared memory.
//
// Kernel: persistent, one CTA per SM, tasks (plan, row group) taken in
// a fixed order (task blockIdx.x + i gridDim.x), each task the tiles of all
// blocks of its row group.  480 threads:
//   warp 0     producer: per tile one bulk copy of the 16 KB band tile and
//              one of the 16 bins x rp spectrum values (contiguous in the
//              bin-major layout) into a ring of STAGES stages
//   warp 1     allocates all 512 tensor-memory columns: per stage 32
//              columns of A_hi and 32 of A_lo (lane = band row), and two
//              accumulator buffers of 3 NP columns; its first thread
//              issues, per K step of 8, tcgen05.mma kind::tf32 with A in
//              tensor memory, M = 128, N = 2 NP: A_hi x [F_hi; F_lo] into
//              columns [0, 2 NP)
//   warp 14    the second issuer: N = NP, A_lo x F_hi into [2 NP, 3 NP) --
//              two threads issuing into separate accumulators, since one
//              thread issuing these narrow products back to back left the
//              tensor pipe idle about two thirds of the time; both commit
//              to the stage and buffer barriers, which count two arrivals
//   warps 2-9  converters: warp w, lane l splits half (w - 2) / 4 of band
//              row 32 (w % 4) + l (its tensor-memory lane) and stores hi and
//              lo to the stage's tensor-memory columns, and the threads
//              together write F_hi / F_lo as K-major 128-byte swizzled rows
//              of the right-hand sides (zero past rp) to shared memory, then
//              release the stage to the MMA threads (two converter warps per
//              scheduler: the split is bound by latency, not arithmetic)
//   warps 10-13 epilogue: warp w owns tensor-memory lanes 32 (w % 4) .. + 31
//              = rows of the group; per tile it loads the 3 NP columns and
//              adds the three parts to its NP sums; after a task's last tile
//              it adds the dense tail's sum, which the persistent launch has
//              left in y (plans with a tail), scales by rowscale_n and
//              stores y[r][n]
// Every mbarrier wait is bounded; a wait that runs out sets the batch's
// status word (XC_ERR_TIMEOUT for xc_batch_status), waits (bounded) for the
// copies and products in flight, frees the tensor memory and returns.
//
// The adjoint (ADJ = true; Algorithm 2, step 1: U_k = sum_n A_nk y_n of the
// stored bands, before the inverse FFT) runs the same pipeline on the
// transposed windows: a task is (plan, block, group of 64 bins), a tile is
// M = 128 rows = the real parts of the 64 bins' values, then their imaginary
// parts, over K = 32 rows of y; the right-hand sides come from yt, the
// row-scaled right-hand sides stored row-major ([row][rp], written by a small
// launch before), so a tile's 32 rows x rp values are again one bulk copy.
// The epilogue writes each bin's sums as the one chunk partial of its bin
// slice ([slice][rhs][32] complex), which the inverse-FFT tasks of the
// persistent launch add up as they do the lockstep items' partials.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "xc_internal.h"
#include "xc_tc.cuh"

namespace xc {

// Rows of a tensor window group (= UMMA M) and bins per tile (16 bins = 32
// FP32 values = one 128-byte swizzle row).
constexpr int kWinRows = 128;
constexpr int kWinBins = 16;
constexpr int kWinTileFloats = kWinRows * 2 * kWinBins;   // 4096

// One plan of a window launch (device copy per plan of the batch).
struct WinPlan {
  const WinBlock* blocks;
  int nblocks;
  int rp;                       // spectrum (yt) row length (nrhs rounded up to 8), <= NP of the launch
  int64_t N, nrhs, ld;
  float* y;                     // forward: [nrhs][ld] output, holding the dense tail's sum (unscaled)
                                // when tail_in_y; adjoint: the [nrhs][ld] input
  const cx<float>* spec;        // forward: bin-major spectra of all blocks
  int tail_in_y;
  const float* rowscale;
  float* yt;                    // adjoint: [N + 32][rp] row-scaled right-hand sides (pad rows zero)
  cx<float>* part;              // adjoint: chunk partials [slice][nrhs][32], one chunk per bin slice
};

template <int NP>
struct WinCfg {
  static constexpr int A_BYTES = kWinTileFloats * 4;   // 16 KB: the band tile as copied
  static constexpr int BT_BYTES = 2 * NP * 128;        // F_hi rows then F_lo rows, K-major
  static constexpr int BR_BYTES = kWinBins * NP * 8;   // raw spectra: 16 bins x up to NP complex values
  static constexpr int STAGE = A_BYTES + BT_BYTES + BR_BYTES;
  // stages of the shared-memory ring = stages of the band operand in tensor
  // memory (a deeper ring, with the band stages released separately, ran
  // slower)
  static constexpr int STAGES = NP <= 32 ? 4 : 2;
  static constexpr int SMEM = STAGES * STAGE + 1024 /* alignment */ + 256 /* barriers */;
  static constexpr int TMEM_COLS = 512;
  static constexpr int A_COLS = 64;                    // per stage: A_hi [0, 32), A_lo [32, 64)
  static constexpr int D_COL = STAGES * A_COLS;        // accumulators [D_COL + 3 NP buf, + 3 NP)
  static_assert(NP % 16 == 0 && 2 * NP <= 256, "UMMA N for M = 128");
  static_assert(D_COL + 6 * NP <= TMEM_COLS, "tensor memory");
  static_assert(STAGE % 1024 == 0, "1024-byte aligned stages");
  static_assert((3 * STAGES + 4) * 8 + 4 <= 256, "barrier space");
};

constexpr int kWinConvThreads = 256;
constexpr int kWinThreads = 64 + kWinConvThreads + 128 + 32;   // + the second MMA issuer (last warp)

template <int NP, bool ADJ>
__global__ void __launch_bounds__(kWinThreads, 1)
    tc_window_kernel(const WinPlan* __restrict__ plans, const int4* __restrict__ tasks, int ntasks, unsigned* status) {
  using namespace tc;
  using C = WinCfg<NP>;
  constexpr int S = C::STAGES;
  // (a name of its own: extern shared arrays of one name are one symbol in a
  // translation unit, and a 1024-byte alignment here would add 1 KB of static
  // shared memory to the batch kernel -- enough, at three CTAs per SM, to
  // take a step of the shared-memory carveout from its L1)
  extern __shared__ __align__(16) unsigned char win_smem[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(win_smem) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  // barriers: full[S], conv[S], empty[S], tfull[2], tempty[2]; then the tensor-memory address
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * C::STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 4);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tile0 = smem_u32(smem);
  auto a_t = [&](int s) { return tile0 + uint32_t(s * C::STAGE); };                         // band tile
  auto b_t = [&](int s) { return tile0 + uint32_t(s * C::STAGE + C::A_BYTES); };             // F_hi; F_lo
  auto b_raw = [&](int s) { return tile0 + uint32_t(s * C::STAGE + C::A_BYTES + C::BT_BYTES); };
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto conv = [&](int s) { return smem_u32(&bars[S + s]); };
  auto empty = [&](int s) { return smem_u32(&bars[2 * S + s]); };
  auto tfull = [&](int b) { return smem_u32(&bars[3 * S + b]); };
  auto tempty = [&](int b) { return smem_u32(&bars[3 * S + 2 + b]); };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), kWinConvThreads);
      mbar_init(empty(s), 2);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 2);
      mbar_init(tempty(b), 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), uint32_t(C::TMEM_COLS));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort = &s_abort;
  int zero_flag = 0;
  volatile int* no_abort = &zero_flag;
  auto give_up = [&]() {
    s_abort = 1;
    atomicCAS(status, 0u, 1u);
  };
  // tiles of a task: forward all blocks' tiles of its row group, adjoint
  // the tiles of its block's bin group
  auto task_tiles = [&](const WinPlan& P, int4 tk) {
    if constexpr (ADJ) return P.blocks[tk.y].nkb[tk.z];
    int n = 0;
    for (int bi = 0; bi < P.nblocks; ++bi) n += P.blocks[bi].nkb[tk.z];
    return n;
  };

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      int kbi = 0;   // tiles issued by this CTA
      bool ok = true;
      for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
        const int4 tk = tasks[t];
        const WinPlan& P = plans[tk.x];
        const uint32_t braw_bytes = uint32_t(kWinBins * P.rp * 8);   // = 32 rows x rp values of yt
        for (int bi = ADJ ? tk.y : 0; bi < (ADJ ? tk.y + 1 : P.nblocks) && ok; ++bi) {
          const WinBlock& b = P.blocks[bi];
          const int nkb = b.nkb[tk.z];
          const int64_t lo = b.lo[tk.z];
          const float* a_src = b.val + b.off[tk.z] * kWinTileFloats;
          for (int kb = 0; kb < nkb; ++kb) {
            const int s = kbi % S;
            if (!mbar_wait(empty(s), (uint32_t(kbi / S) & 1u) ^ 1u, abort)) {
              if (!*abort) give_up();
              ok = false;
              break;
            }
            mbar_expect_tx(full(s), uint32_t(C::A_BYTES) + braw_bytes);
            bulk_load(a_t(s), a_src + int64_t(kb) * kWinTileFloats, uint32_t(C::A_BYTES), full(s));
            if constexpr (ADJ)
              bulk_load(b_raw(s), P.yt + (lo + int64_t(kb) * 2 * kWinBins) * P.rp, braw_bytes, full(s));
            else
              bulk_load(b_raw(s), P.spec + (b.spec_off + lo + int64_t(kb) * kWinBins) * P.rp, braw_bytes, full(s));
            ++kbi;
          }
        }
      }
      // copies still in flight land before the CTA leaves
      for (int k = kbi > S ? kbi - S : 0; k < kbi; ++k)
        if (!mbar_wait(full(k % S), uint32_t(k / S) & 1u, no_abort) && !*abort) give_up();
    }
  } else if (warp == 1 || warp == kWinThreads / 32 - 1) {
    // ---------------------------------------------------------- MMA issuers
    // warp 1: A_hi x [F_hi; F_lo] into columns [0, 2 NP); the last warp:
    // A_lo x F_hi into [2 NP, 3 NP) -- two issuing threads, each committing
    // to the stage and buffer barriers (which count two arrivals)
    const bool second = warp != 1;
    if (lane == 0) {
      constexpr uint32_t idesc2 = tf32_idesc(kWinRows, 2 * NP);   // A_hi x [F_hi; F_lo]
      constexpr uint32_t idesc1 = tf32_idesc(kWinRows, NP);       // A_lo x F_hi
      int kbi = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
        const int4 tk = tasks[t];
        const int nk = task_tiles(plans[tk.x], tk);
        for (int k = 0; k < nk; ++k) {
          const int s = kbi % S, buf = kbi & 1;
          if (!mbar_wait(tempty(buf), (uint32_t(kbi >> 1) & 1u) ^ 1u, abort) ||
              !mbar_wait(conv(s), uint32_t(kbi / S) & 1u, abort)) {
            if (!*abort) give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + uint32_t(C::D_COL + buf * 3 * NP);
          const uint32_t a = tmem + uint32_t(s * C::A_COLS);
          if (!second) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)   // K step of 8 FP32 values = 32 bytes inside the swizzled row
              umma_tf32_ts(d, a + uint32_t(kk * 8), sw128_desc(b_t(s) + uint32_t(kk * 32)), idesc2,
                           kk != 0 ? 1u : 0u);
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              umma_tf32_ts(d + uint32_t(2 * NP), a + uint32_t(32 + kk * 8), sw128_desc(b_t(s) + uint32_t(kk * 32)),
                           idesc1, kk != 0 ? 1u : 0u);
          }
          umma_commit(empty(s));
          umma_commit(tfull(buf));
          ++kbi;
        }
      }
      // no product may still run when the tensor memory is freed
      for (int k = kbi > 2 ? kbi - 2 : 0; k < kbi; ++k)
        if (!mbar_wait(tfull(k & 1), uint32_t(k >> 1) & 1u, no_abort) && !*abort) give_up();
    }
  } else if (warp < 2 + kWinConvThreads / 32) {
    // ---------------------------------------------------------- converters
    const int ct = threadIdx.x - 64;
    // band row = this thread's tensor-memory lane; K columns [16 half, 16 half + 16)
    const int row = 32 * (warp & 3) + lane, half = (warp - 2) >> 2;
    const uint32_t a_lane = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(16 * half);
    int kbi = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
      const int4 tk = tasks[t];
      const WinPlan& P = plans[tk.x];
      const int nk = task_tiles(P, tk);
      const int rp = P.rp;
      for (int k = 0; k < nk; ++k) {
        const int s = kbi % S;
        // one lane waits, the warp follows (the tensor-memory stores are warp-collective)
        int ready = 0;
        if (lane == 0) {
          ready = mbar_wait(full(s), uint32_t(kbi / S) & 1u, abort) ? 1 : 0;
          if (!ready && !*abort) give_up();
        }
        if (!__shfl_sync(0xffffffffu, ready, 0)) {
          ok = false;
          break;
        }
        // band row, K values 16 half .. + 15 (chunk c of the copied tile row
        // at position c ^ (row & 7)), split into the stage's tensor memory
        const float4* ar = reinterpret_cast<const float4*>(smem + (a_t(s) - tile0) + row * 128);
        float hv[16], lv[16];
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) {
          const float4 v = ar[(4 * half + c0) ^ (row & 7)];
          split_tf32(v.x, &hv[4 * c0], &lv[4 * c0]);
          split_tf32(v.y, &hv[4 * c0 + 1], &lv[4 * c0 + 1]);
          split_tf32(v.z, &hv[4 * c0 + 2], &lv[4 * c0 + 2]);
          split_tf32(v.w, &hv[4 * c0 + 3], &lv[4 * c0 + 3]);
        }
        // (the stage's previous products are done: the producer waited for
        // them before copying this tile)
        tc_fence_after();
        tmem_st16(a_lane + uint32_t(s * C::A_COLS), hv);
        tmem_st16(a_lane + uint32_t(s * C::A_COLS + 32), lv);
        // right-hand sides: K-major rows n of [F_hi; F_lo]; chunk c = bins 2c,
        // 2c+1 (forward spectra, complex) or rows 4c .. 4c+3 (adjoint yt)
        const float* raw = reinterpret_cast<const float*>(smem + (b_raw(s) - tile0));
        unsigned char* bt = smem + (b_t(s) - tile0);
        for (int i = ct; i < NP * 8; i += kWinConvThreads) {
          const int n = i >> 3, c = i & 7;
          float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
          if (n < rp) {
            if constexpr (ADJ) {
              f.x = raw[(4 * c) * rp + n];
              f.y = raw[(4 * c + 1) * rp + n];
              f.z = raw[(4 * c + 2) * rp + n];
              f.w = raw[(4 * c + 3) * rp + n];
            } else {
              const float2 f0 = reinterpret_cast<const float2*>(raw)[(2 * c) * rp + n];
              const float2 f1 = reinterpret_cast<const float2*>(raw)[(2 * c + 1) * rp + n];
              f = make_float4(f0.x, f0.y, f1.x, f1.y);
            }
          }
          float4 h, l;
          split_tf32(f.x, &h.x, &l.x);
          split_tf32(f.y, &h.y, &l.y);
          split_tf32(f.z, &h.z, &l.z);
          split_tf32(f.w, &h.w, &l.w);
          const int sw = (c ^ (n & 7)) * 16;
          *reinterpret_cast<float4*>(bt + n * 128 + sw) = h;
          *reinterpret_cast<float4*>(bt + (NP + n) * 128 + sw) = l;
        }
        __syncwarp();
        tmem_wait_st();       // the band values are in tensor memory
        tc_fence_before();
        fence_async_smem();   // the tensor core reads the spectrum tiles through the async proxy
        mbar_arrive(conv(s));
        ++kbi;
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;   // tensor-memory lanes [32 q, 32 q + 32) = rows of the group (warps 10-13: 2, 3, 0, 1)
    int kbi = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
      const int4 tk = tasks[t];
      const WinPlan& P = plans[tk.x];
      const int nk = task_tiles(P, tk);
      float acc[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[j] = 0.f;
      for (int k = 0; k < nk; ++k) {
        const int buf = kbi & 1;
        int ready = 0;   // one lane waits, the warp follows (tcgen05.ld is warp-collective)
        if (lane == 0) {
          ready = mbar_wait(tfull(buf), uint32_t(kbi >> 1) & 1u, abort) ? 1 : 0;
          if (!ready && !*abort) give_up();
        }
        ready = __shfl_sync(0xffffffffu, ready, 0);
        if (!ready) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + (uint32_t(q * 32) << 16) + uint32_t(C::D_COL + buf * 3 * NP);
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16) {
          float vh[16], vl[16], vm[16];
          tmem_ld16(base + uint32_t(c0), vh);            // A_hi F_hi
          tmem_ld16(base + uint32_t(NP + c0), vl);       // A_hi F_lo
          tmem_ld16(base + uint32_t(2 * NP + c0), vm);   // A_lo F_hi
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[c0 + j] += vh[j] + (vl[j] + vm[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty(buf));
        ++kbi;
      }
      if (!ok) break;
      if constexpr (ADJ) {
        // lane m = 32 q + lane: bin 64 g + (m & 63) of the block, real part
        // (m < 64) or imaginary part; its bin slice's one chunk partial
        const WinBlock& b = P.blocks[tk.y];
        const int m = q * 32 + lane, bl = m & 63;
        const int sl = 2 * tk.z + (bl >> 5);
        if (sl < b.tslices) {
          float* out = reinterpret_cast<float*>(P.part + (int64_t(b.gbase) + sl) * P.nrhs * 32) +
                       2 * (bl & 31) + (m >> 6);
          const int nq = int(P.nrhs < NP ? P.nrhs : NP);
#pragma unroll
          for (int j = 0; j < NP; ++j)
            if (j < nq) out[int64_t(j) * 64] = acc[j];
        }
        continue;
      }
      const int64_t n = int64_t(tk.z) * kWinRows + q * 32 + lane;
      if (n < P.N) {
        const int nq = int(P.nrhs < NP ? P.nrhs : NP);
        float* yn = P.y + n;
        if (P.tail_in_y) {
#pragma unroll
          for (int j = 0; j < NP; ++j)
            if (j < nq) acc[j] += yn[j * P.ld];
        }
        const float rs = P.rowscale ? P.rowscale[n] : 1.f;
#pragma unroll
        for (int j = 0; j < NP; ++j)
          if (j < nq) yn[j * P.ld] = acc[j] * rs;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, uint32_t(C::TMEM_COLS));
  }
}

}  // namespace xc
