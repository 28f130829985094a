// The direct dense product y = A x that the extra-component method replaces
// (Section 1: the matrix-vector product with eq. (cheb_matrix) /
// eq. (Jac_matrix); Section 5 compares the method with it), computed on the
// tensor cores (tcgen05, sm_103a) at FP32 accuracy.
//
// Precision: 3xTF32.  Every FP32 operand v is split into v = hi + lo with hi
// = v rounded to TF32 (10 explicit mantissa bits) and lo = (v - hi) rounded
// to TF32; the product a b is accumulated as hi_a hi_b + hi_a lo_b + lo_a hi_b
// (the lo_a lo_b term is below 2^-22 |a b|) in FP32 in tensor memory.  Both
// halves are exact TF32 numbers, so the result does not depend on how the
// tensor core reduces a wider FP32 operand.  The matrix is split once, when
// the comparator is created (and a transposed copy made for A^T y, so that
// both products read K-major operands); right-hand sides are split per call.
//
// Accumulation: the tensor core rounds toward zero when it adds a product
// sum into its FP32 accumulator, so over a long K loop the truncations add up
// with one sign (a CPU model of the arithmetic gives 6e-5 relative at
// K = 4096, against 6e-7 for FP32 round-to-nearest).  Each k-block (32
// columns, twelve MMAs) therefore starts a fresh accumulator in tensor
// memory, and the epilogue warps add it to FP32 registers with
// round-to-nearest additions (the model: 4.7e-7), while the tensor core fills
// the other of two accumulator buffers.
//
// Kernel (one 128 x BN output tile per CTA, the full K loop):
//   warp 0     TMA producer: per k-block of 32 columns, the four tiles
//              A_hi, A_lo (128 x 32) and X_hi, X_lo (BN x 32), 128-byte
//              swizzled, into a ring of STAGES stages (mbarriers full/empty)
//   warp 1     allocates 2 BN columns of tensor memory; one thread issues
//              tcgen05.mma kind::tf32 (M = 128, N = BN, K = 8), three per
//              k-step, into accumulator buffer (k-block & 1), and commits
//              each stage back to the producer and each buffer to the
//              epilogue
//   warps 2-9  epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. +31
//              (output rows) and half (w - 2) / 4 of the BN columns; per
//              k-block tcgen05.ld of its buffer, FP32 additions into
//              registers, then releases the buffer; at the end it stores
//              y[r][m] -- 32 consecutive m per warp and column
// Every mbarrier wait is bounded (about two seconds of global time); a wait
// that runs out records XC_ERR_TIMEOUT in the comparator's status word,
// waits (bounded) for the loads and products it has in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "xc_internal.h"
#include "xc_tc.cuh"

namespace xc {

namespace {

constexpr int kBM = 128;        // output rows (matrix rows) per tile = UMMA M
constexpr int kBK = 32;         // FP32 columns per k-block: one 128-byte swizzled row
constexpr int kUK = 8;          // K of one kind::tf32 MMA
constexpr int kEpiWarps = 8;    // two per tensor-memory lane quadrant
constexpr int kThreads = 32 * (2 + kEpiWarps);

enum { DS_OK = 0, DS_TIMEOUT = 1 };

template <int BN>
struct Cfg {
  static constexpr int A_BYTES = kBM * kBK * 4;                  // 16 KB
  static constexpr int B_BYTES = BN * kBK * 4;                   // BN x 128 B
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE < 8 ? (200 * 1024) / STAGE : 8;
  static constexpr int SMEM = STAGES * STAGE + 1024 /* alignment */ + 256 /* barriers */;
  static constexpr int TMEM_COLS = 2 * BN;    // two accumulator buffers (a power of two, <= 512)
  static_assert(STAGES >= 2, "two stages at least");
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "UMMA N for M = 128");
};

using namespace tc;

// Instruction descriptor of the comparator's products (M = 128, N = BN).
template <int BN>
__host__ __device__ constexpr uint32_t tf32_idesc() {
  return tc::tf32_idesc(kBM, BN);
}

// ------------------------------------------------------------ split kernels
// hi[r][k], lo[r][k] (row stride ldo) from v[r][k] (row stride ldi), k < K.
__global__ void split_kernel(const float* __restrict__ v, int64_t ldi, int64_t rows, int64_t K, float* __restrict__ hi,
                             float* __restrict__ lo, int64_t ldo) {
  const int64_t total = rows * K;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / K, k = i - r * K;
    float h, l;
    split_tf32(v[r * ldi + k], &h, &l);
    hi[r * ldo + k] = h;
    lo[r * ldo + k] = l;
  }
}

// The split of A^T: hi[k][m], lo[k][m] (row stride ldo) from A[m][k] (row
// stride lda), a 32 x 32 tile per CTA of 32 x 8 threads through shared memory.
__global__ void split_transpose_kernel(const float* __restrict__ A, int64_t lda, int64_t M, int64_t K,
                                       float* __restrict__ hi, float* __restrict__ lo, int64_t ldo) {
  __shared__ float tile[32][33];
  const int64_t m0 = int64_t(blockIdx.y) * 32, k0 = int64_t(blockIdx.x) * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t m = m0 + i, k = k0 + threadIdx.x;
    tile[i][threadIdx.x] = (m < M && k < K) ? A[m * lda + k] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t k = k0 + i, m = m0 + threadIdx.x;
    if (k < K && m < M) {
      float h, l;
      split_tf32(tile[threadIdx.x][i], &h, &l);
      hi[k * ldo + m] = h;
      lo[k * ldo + m] = l;
    }
  }
}

// ------------------------------------------------------------ GEMM kernel
// y[r][m] = sum_k A[m][k] x[r][k] for m < M, r < R (A given as A_hi + A_lo,
// x as X_hi + X_lo through the four tensor maps).  Grid: (ceil(R / BN),
// ceil(M / 128)); blockIdx.x runs over the right-hand-side tiles so that the
// CTAs reading one A row block are launched together.
template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    gemm3xtf32_kernel(const __grid_constant__ CUtensorMap map_ah, const __grid_constant__ CUtensorMap map_al,
                      const __grid_constant__ CUtensorMap map_xh, const __grid_constant__ CUtensorMap map_xl,
                      int64_t M, int64_t K, int64_t R, float* __restrict__ y, int64_t ldy, int* __restrict__ status) {
  using C = Cfg<BN>;
  constexpr int S = C::STAGES;
  constexpr int HALF = BN / 2;   // accumulator columns per epilogue warp
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // tiles at a 1024-byte aligned base (the 128-byte swizzle pattern repeats every 1024 bytes)
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  // barriers: full[S], empty[S], tfull[2], tempty[2]; then the tensor-memory address
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * C::STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 4);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN;
  const int64_t m0 = int64_t(blockIdx.y) * kBM;
  const int nk = int((K + kBK - 1) / kBK);
  const uint32_t tile0 = smem_u32(smem);
  auto a_hi = [&](int s) { return tile0 + uint32_t(s * C::STAGE); };
  auto a_lo = [&](int s) { return tile0 + uint32_t(s * C::STAGE + C::A_BYTES); };
  auto x_hi = [&](int s) { return tile0 + uint32_t(s * C::STAGE + 2 * C::A_BYTES); };
  auto x_lo = [&](int s) { return tile0 + uint32_t(s * C::STAGE + 2 * C::A_BYTES + C::B_BYTES); };
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[S + s]); };
  auto tfull = [&](int b) { return smem_u32(&bars[2 * S + b]); };
  auto tempty = [&](int b) { return smem_u32(&bars[2 * S + 2 + b]); };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), uint32_t(C::TMEM_COLS));   // the whole warp: two buffers
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort = &s_abort;
  int zero_flag = 0;
  volatile int* no_abort = &zero_flag;
  auto give_up = [&]() {
    s_abort = 1;
    atomicExch(status, DS_TIMEOUT);
  };

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        const uint32_t ph = uint32_t(kb / S) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort)) {
          if (!*abort) give_up();
          break;
        }
        mbar_expect_tx(full(s), uint32_t(C::STAGE));
        const int kc = kb * kBK;
        tma_load_2d(a_hi(s), &map_ah, full(s), kc, int(m0));
        tma_load_2d(a_lo(s), &map_al, full(s), kc, int(m0));
        tma_load_2d(x_hi(s), &map_xh, full(s), kc, n0);
        tma_load_2d(x_lo(s), &map_xl, full(s), kc, n0);
        issued = kb + 1;
      }
      // a load still in flight must land before the CTA leaves, whatever
      // happened to its consumer
      for (int kb = issued > S ? issued - S : 0; kb < issued; ++kb)
        if (!mbar_wait(full(kb % S), uint32_t(kb / S) & 1u, no_abort) && !*abort) give_up();
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc<BN>();
      int committed = 0;   // k-blocks whose products were issued and committed
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S, buf = kb & 1;
        // the buffer is free once the epilogue has drained its previous k-block
        if (!mbar_wait(tempty(buf), (uint32_t(kb >> 1) & 1u) ^ 1u, abort) ||
            !mbar_wait(full(s), uint32_t(kb / S) & 1u, abort)) {
          if (!*abort) give_up();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(buf * BN);
#pragma unroll
        for (int kk = 0; kk < kBK / kUK; ++kk) {
          const uint32_t off = uint32_t(kk * kUK * 4);   // 32 bytes per K step inside the swizzled row
          const uint64_t ah = sw128_desc(a_hi(s) + off), al = sw128_desc(a_lo(s) + off);
          const uint64_t xh = sw128_desc(x_hi(s) + off), xl = sw128_desc(x_lo(s) + off);
          umma_tf32(d, ah, xh, idesc, kk != 0 ? 1u : 0u);   // a fresh accumulator per k-block
          umma_tf32(d, ah, xl, idesc, 1u);
          umma_tf32(d, al, xh, idesc, 1u);
        }
        umma_commit(empty(s));     // the stage is free once these products have read it
        umma_commit(tfull(buf));   // and the buffer holds this k-block's sum
        committed = kb + 1;
      }
      // no product may still run when the tensor memory is freed: the last
      // commit of each buffer completes only after its products
      for (int kb = committed > 2 ? committed - 2 : 0; kb < committed; ++kb)
        if (!mbar_wait(tfull(kb & 1), uint32_t(kb >> 1) & 1u, no_abort) && !*abort) give_up();
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;             // tensor-memory lanes [32 q, 32 q + 32) = output rows
    const int half = (warp - 2) >> 2;   // columns [half * HALF, half * HALF + HALF)
    float acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int buf = kb & 1;
      // one lane waits and the warp follows its verdict (tcgen05.ld is warp-collective)
      int ready = 0;
      if (lane == 0) {
        ready = mbar_wait(tfull(buf), uint32_t(kb >> 1) & 1u, abort) ? 1 : 0;
        if (!ready && !*abort) give_up();
      }
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * BN + half * HALF);
#pragma unroll
      for (int c0 = 0; c0 < HALF; c0 += 32) {
        float v[32];
        tmem_ld32(base + uint32_t(c0), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[c0 + j] += v[j];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(buf));
    }
    if (ok) {
      const int64_t m = m0 + q * 32 + lane;
      if (m < M) {
#pragma unroll
        for (int j = 0; j < HALF; ++j) {
          const int64_t r = int64_t(n0) + half * HALF + j;
          if (r < R) y[r * ldy + m] = acc[j];
        }
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

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of a row-major FP32 array [rows][ld] (the first `cols` columns
// used), box = 32 columns x box_rows rows, 128-byte swizzle, zero fill
// outside.  ld * 4 must be a multiple of 16 and the base 16-byte aligned.
int make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(XC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 4) % 16 != 0)
    return fail(XC_ERR_ARG, "tensor map base or row stride not 16-byte aligned");
  const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 4};
  const cuuint32_t box[2] = {cuuint32_t(kBK), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(XC_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
  return XC_OK;
}

int64_t round4(int64_t v) { return (v + 3) / 4 * 4; }

}  // namespace

struct Dense {
  int64_t M = 0, K = 0;
  int64_t ldk = 0, ldm = 0;           // row strides of the split A [M][ldk] and A^T [K][ldm]
  float* a_hi = nullptr;              // [M][ldk]
  float* a_lo = nullptr;
  float* t_hi = nullptr;              // [K][ldm] (A^T)
  float* t_lo = nullptr;
  float* x_hi = nullptr;              // [nrhs][ldx] split right-hand sides
  float* x_lo = nullptr;
  int64_t x_elems = 0;
  int* status = nullptr;
  CUtensorMap map_a[2][2];            // [transpose][hi, lo]
  ~Dense() {
    cudaDeviceSynchronize();
    for (void* p : {static_cast<void*>(a_hi), static_cast<void*>(a_lo), static_cast<void*>(t_hi),
                    static_cast<void*>(t_lo), static_cast<void*>(x_hi), static_cast<void*>(x_lo),
                    static_cast<void*>(status)})
      if (p) cudaFree(p);
  }
};

namespace {

int dev_alloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes == 0 ? 16 : bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(XC_ERR_ALLOC, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  return XC_OK;
}

template <int BN>
int launch_gemm(Dense* d, int tr, int64_t R, float* y, int64_t ldy, cudaStream_t st) {
  using C = Cfg<BN>;
  const int64_t M = tr ? d->K : d->M;
  const int64_t K = tr ? d->M : d->K;
  const int64_t ldx = tr ? d->ldm : d->ldk;
  CUtensorMap mxh, mxl;
  XC_TRY(make_map(&mxh, d->x_hi, R, K, ldx, BN));
  XC_TRY(make_map(&mxl, d->x_lo, R, K, ldx, BN));
  auto fn = gemm3xtf32_kernel<BN>;
  XC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               C::SMEM));
  const dim3 grid(unsigned((R + BN - 1) / BN), unsigned((M + kBM - 1) / kBM));
  count_launch();
  fn<<<grid, kThreads, C::SMEM, st>>>(d->map_a[tr][0], d->map_a[tr][1], mxh, mxl, M, K, R, y, ldy, d->status);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

}  // namespace

int dense_create(Dense** out, const float* A, int64_t M, int64_t K, int64_t lda, cudaStream_t st) {
  auto* d = new (std::nothrow) Dense();
  if (!d) return fail(XC_ERR_ALLOC, "host allocation failed");
  d->M = M;
  d->K = K;
  d->ldk = round4(K);
  d->ldm = round4(M);
  auto run = [&]() -> int {
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->a_hi), size_t(M) * d->ldk * 4));
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->a_lo), size_t(M) * d->ldk * 4));
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->t_hi), size_t(K) * d->ldm * 4));
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->t_lo), size_t(K) * d->ldm * 4));
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->status), sizeof(int)));
    XC_CUDA(cudaMemsetAsync(d->status, 0, sizeof(int), st));
    count_launch();
    split_kernel<<<1024, 256, 0, st>>>(A, lda, M, K, d->a_hi, d->a_lo, d->ldk);
    XC_CUDA(cudaGetLastError());
    count_launch();
    split_transpose_kernel<<<dim3(unsigned((K + 31) / 32), unsigned((M + 31) / 32)), dim3(32, 8), 0, st>>>(
        A, lda, M, K, d->t_hi, d->t_lo, d->ldm);
    XC_CUDA(cudaGetLastError());
    XC_TRY(make_map(&d->map_a[0][0], d->a_hi, M, K, d->ldk, kBM));
    XC_TRY(make_map(&d->map_a[0][1], d->a_lo, M, K, d->ldk, kBM));
    XC_TRY(make_map(&d->map_a[1][0], d->t_hi, K, M, d->ldm, kBM));
    XC_TRY(make_map(&d->map_a[1][1], d->t_lo, K, M, d->ldm, kBM));
    XC_CUDA(cudaStreamSynchronize(st));
    return XC_OK;
  };
  const int rc = run();
  if (rc != XC_OK) {
    const std::string msg = xc_last_error_message();
    delete d;
    return fail(rc, msg);
  }
  *out = d;
  return XC_OK;
}

int dense_apply(Dense* d, int tr, const float* in, float* out, int64_t R, int64_t ld, cudaStream_t st) {
  const int64_t M = tr ? d->K : d->M;   // output length
  const int64_t K = tr ? d->M : d->K;   // input length
  const int64_t ldx = tr ? d->ldm : d->ldk;
  if (R == 0) return XC_OK;
  const int64_t need = R * ldx;
  if (need > d->x_elems) {
    cudaStreamSynchronize(st);   // a previous call may still read the old buffers
    cudaFree(d->x_hi);
    cudaFree(d->x_lo);
    d->x_hi = d->x_lo = nullptr;
    d->x_elems = 0;
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->x_hi), size_t(need) * 4));
    XC_TRY(dev_alloc(reinterpret_cast<void**>(&d->x_lo), size_t(need) * 4));
    d->x_elems = need;
  }
  count_launch();
  split_kernel<<<1024, 256, 0, st>>>(in, ld, R, K, d->x_hi, d->x_lo, ldx);
  XC_CUDA(cudaGetLastError());
  (void)M;
  if (R > 128) return launch_gemm<256>(d, tr, R, out, ld, st);
  if (R > 64) return launch_gemm<128>(d, tr, R, out, ld, st);
  return launch_gemm<64>(d, tr, R, out, ld, st);
}

int dense_status(Dense* d, cudaStream_t st) {
  int h = 0;
  XC_CUDA(cudaMemcpyAsync(&h, d->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  XC_CUDA(cudaStreamSynchronize(st));
  if (h != 0) {
    XC_CUDA(cudaMemsetAsync(d->status, 0, sizeof(int), st));
    XC_CUDA(cudaStreamSynchronize(st));
    return fail(XC_ERR_TIMEOUT, "a wait of the dense tensor-core product gave up; its output is incomplete");
  }
  return XC_OK;
}

}  // namespace xc

using xc::fail;

extern "C" {

int xc_dense_create(xc_dense_t* out, const float* A_dev, int64_t M, int64_t K, int64_t lda, void* stream) {
  if (!out) return fail(XC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!A_dev) return fail(XC_ERR_ARG, "A_dev is NULL");
  if (M < 1 || K < 1 || lda < K || M > (int64_t(1) << 31) - 256 || K > (int64_t(1) << 31) - 256)
    return fail(XC_ERR_ARG, "need 1 <= M, K < 2^31 - 256 and lda >= K");
  xc::Dense* d = nullptr;
  XC_TRY(xc::dense_create(&d, A_dev, M, K, lda, static_cast<cudaStream_t>(stream)));
  *out = reinterpret_cast<xc_dense_t>(d);
  return XC_OK;
}

int xc_dense_apply(xc_dense_t dense, int transpose, const float* in_dev, float* out_dev, int64_t nrhs, int64_t ld,
                   void* stream) {
  auto* d = reinterpret_cast<xc::Dense*>(dense);
  if (!d) return fail(XC_ERR_ARG, "dense is NULL");
  if (nrhs < 0 || nrhs > (int64_t(1) << 31) - 256) return fail(XC_ERR_ARG, "nrhs out of range");
  if (nrhs == 0) return XC_OK;
  if (!in_dev || !out_dev) return fail(XC_ERR_ARG, "NULL vector");
  const int64_t n_in = transpose ? d->M : d->K, n_out = transpose ? d->K : d->M;
  if (ld < std::max(n_in, n_out)) return fail(XC_ERR_ARG, "ld below the vector length");
  const auto* a = reinterpret_cast<const char*>(in_dev);
  const auto* b = reinterpret_cast<const char*>(out_dev);
  const int64_t span_in = ((nrhs - 1) * ld + n_in) * 4, span_out = ((nrhs - 1) * ld + n_out) * 4;
  if (a < b + span_out && b < a + span_in) return fail(XC_ERR_ARG, "in_dev and out_dev overlap");
  return xc::dense_apply(d, transpose ? 1 : 0, in_dev, out_dev, nrhs, ld, static_cast<cudaStream_t>(stream));
}

int xc_dense_status(xc_dense_t dense, void* stream) {
  auto* d = reinterpret_cast<xc::Dense*>(dense);
  if (!d) return fail(XC_ERR_ARG, "dense is NULL");
  return xc::dense_status(d, static_cast<cudaStream_t>(stream));
}

int xc_dense_destroy(xc_dense_t dense) {
  delete reinterpret_cast<xc::Dense*>(dense);
  return XC_OK;
}

}  // extern "C"
