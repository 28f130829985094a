// Internal declarations of libxc: the plan, per-block descriptors passed to
// kernels, and the error plumbing shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "xc.h"

namespace xc {

constexpr int kMaxPasses = 24;   // radix passes of one FFT (n <= 2^24)
constexpr int kSlice = 32;       // rows (forward) or spectrum bins (adjoint) per band slice

// Set the thread's last error message and return `code`.
int fail(int code, const std::string& msg);
// Map a CUDA status to XC_ERR_CUDA with context; XC_OK if cudaSuccess.
int cuda_check(cudaError_t e, const char* what);

#define XC_CUDA(...)                                                  \
  do {                                                                \
    int _rc = ::xc::cuda_check((__VA_ARGS__), #__VA_ARGS__);          \
    if (_rc != XC_OK) return _rc;                                     \
  } while (0)

#define XC_TRY(...)                   \
  do {                                \
    int _rc = (__VA_ARGS__);          \
    if (_rc != XC_OK) return _rc;     \
  } while (0)

// ------------------------------------------------------------ host parameters
// (xc_params.cpp) The host side of the precomputation stage, step 1.1 of
// Algorithms 1-4: zeta, the extra-component counts and the block schedule.
double bessel_i0_host(double z);
double kaiser_value_host(double j, int64_t length, double zeta);
double zeta_of_eps_host(double eps1);
bool is_fft_friendly(int64_t length);
int64_t fft_friendly_at_least(int64_t length);
// Smallest s >= 1 with w_s^{zeta, L-1} >= eps2 (Section 2.2), or -1.
int64_t extra_count(int64_t m, double zeta, double eps2, bool two_sided);
// Factor n into radices 8, 4, 2, 3, 5, 7 (product == n); returns pass count or -1.
int fft_radices(int64_t n, int* radix);

struct BlockShape {
  int64_t L, off, j_lo, j_hi;
};
struct Schedule {
  double zeta = 0, eps_window = 0;
  std::vector<BlockShape> blocks;
  int64_t m_tail = 0;
};
int make_schedule(int64_t N, double eps, double eps2, bool two_sided, double eps_window,
                  int tail_max, Schedule* out);

// ----------------------------------------------------------- device descriptor
// One block of the compressed operator as the apply kernels see it.  Value
// pointers are untyped; the kernels cast them to the plan's precision.
struct BlockDev {
  int L, n, H;               // FFT length, n = L/2 complex points, H = n + 1 bins
  int a_csize;               // CTAs sharing the apply FFT (1, or a cluster of 2..8 for long blocks)
  int off, j_lo, j_hi;       // extended column j <-> matrix column j - off; input in [j_lo, j_hi)
  int p;                     // radix passes
  int radix[kMaxPasses];
  const int* perm;           // [n] digit-reversed position of input index j
  const void* tw;            // [L] complex exp(-2 pi i k / L), plan precision
  const void* invw;          // [L] 1 / w_j^{zeta, L-1}, plan precision
  // forward band layout: slices of 32 rows; row n reads bins [k0[n], k0[n] + width[slice])
  int nslices;
  const int* f_k0;           // [N]
  const int* f_width;        // [nslices]
  const int64_t* f_off;      // [nslices] element offset of the slice's values
  const void* f_val;         // complex values, value (slice, j, lane) at f_off[s] + j*32 + lane
  // adjoint band layout: slices of 32 bins; bin k reads rows [n0[k], n0[k] + width[slice])
  int tslices;
  const int* t_n0;           // [H]
  const int* t_width;        // [tslices]
  const int64_t* t_off;      // [tslices]
  const void* t_val;
  int t_yt;                  // 1: the adjoint product reads the transposed right-hand sides
  int64_t spec_off;          // offset (complex elements) of this block's spectrum per unit nrhs
  int t_gbase;               // index of this block's first bin slice in the plan-wide slice list
  // Window ("lockstep") copies of the two band layouts, used by batches (null
  // until ensure_lockstep builds them).  Forward: row slice s covers the bins
  // [lf_lo[s], lf_lo[s] + lf_len[s]) -- the union of its 32 rows' bands --
  // and value (s, bin k, lane) sits at lf_off[s] + (k - lf_lo[s]) * 32 + lane,
  // zero where k is outside the lane's band; all 32 rows of a warp then step
  // through the same bin.  Adjoint: bin slice s covers the rows [lt_lo[s],
  // lt_lo[s] + lt_len[s]) in the same way.
  const int* lf_lo;
  const int* lf_len;
  const int64_t* lf_off;
  const void* lf_val;
  const int* lt_lo;
  const int* lt_len;
  const int64_t* lt_off;
  const void* lt_val;
};

// Tensor windows of one block (FP32 plans, batches; built by ensure_lockstep,
// kept apart from BlockDev, which every band item reads): group g of 128 rows
// covers the bins [lo[g], lo[g] + 16 nkb[g]) in nkb[g] tiles of 128 rows x 16
// bins from tile off[g] of val; a tile is 128 rows of 32 FP32 values (real
// and imaginary parts of 16 bins, zero outside the row's stored band), the
// 16-byte chunk c of row r stored at chunk c ^ (r & 7) (the 128-byte
// swizzled K-major layout of the tensor core's operands; xc_window.cuh).
//
// Adjoint windows (the transposed layout): group g of 64 bins (bin slices 2g,
// 2g + 1) covers the rows [lo[g], lo[g] + 32 nkb[g]) in tiles of 128 rows x
// 32 FP32 values: row m holds the real (m < 64) or imaginary part of bin
// 64 g + (m & 63)'s values at 32 consecutive rows of y, swizzled the same way.
struct WinBlock {
  const int* lo;
  const int* nkb;
  const int64_t* off;
  const float* val;
  int64_t spec_off;          // = BlockDev::spec_off
  int gbase, tslices;        // = BlockDev::t_gbase, tslices (adjoint)
};

// Rows per chunk of a transposed (bin) slice in the adjoint product: long
// slices are cut into chunks whose partial sums the adjoint FFT adds up.
// Plans with few rows in all take shorter chunks (down to kAdjChunkMin), so
// that even one right-hand side spreads over enough warps.
constexpr int kAdjChunk = 256;
constexpr int kAdjChunkMin = 32;
constexpr int64_t kAdjTargetChunks = 512;

// Band rows per chunk of a row slice in the forward product of plans with long
// bands; a reduction kernel adds the chunks of each slice.
constexpr int kFwdChunk = 256;

// A plan's window (lockstep) layouts are used by batches when they store at
// most this many times the elements of the band layouts (Hermite functions:
// about 1.05-1.2; Legendre / Jacobi / Chebyshev: 1.5-4).
constexpr double kLockRatio = 1.25;

// The tensor windows (128 rows) of an FP32 plan are built when they store at
// most this many times the elements of its band layout (2.0, which adds the
// smaller Hermite plans, gave the 1000-plan batch no gain).
constexpr double kTensorRatio = 1.5;

// ---------------------------------------------------------- 2-D block scheme
// One direction of the 2-D scheme (forward: input side = columns, output side
// = rows; adjoint: the other way round).  Block b's input transform is
// described by in_host[b] (a BlockDev whose j_lo/j_hi/off select the valid
// inputs), its output transform by out_host[b]; the compressed product of all
// blocks is one CSR over the output half-spectrum bins with two segments per
// bin, entries (k, a) adding a conj(U_k), then entries (k, c) adding c U_k
// (U: the input half spectrum, DFT with exp(-...)).
struct D2Dir {
  std::vector<BlockDev> in_host, out_host;
  void* in_dev = nullptr;              // BlockDev[nb]
  void* out_dev = nullptr;             // BlockDev[nb]
  int64_t spec_in = 0, spec_out = 0;   // complex elements per RHS over all blocks
  int64_t parts = 0;                   // real elements per RHS: every block's valid outputs
  int64_t rows = 0, nnz = 0;           // CSR rows (output bins of all blocks) and entries
  int64_t* ptr = nullptr;              // [2 rows + 1]: bin r's a terms [ptr[2r], ptr[2r+1]), c terms to ptr[2r+2]
  int* idx = nullptr;                  // [nnz] input bin
  void* a = nullptr;                   // [nnz] complex values, plan precision
  int* row_blk = nullptr;              // [rows] block of the row
  int* row_loc = nullptr;              // [rows] output bin within the block
  int64_t* part_off = nullptr;         // [nb] per-RHS offset of the block's valid outputs
  int max_n_in = 0, max_n_out = 0;
  // combine: output index o gets entries comb_ent[comb_ptr[o] .. comb_ptr[o+1]):
  // b >= 0 a block's partial, ~d a dense rectangle
  int* comb_ptr = nullptr;             // [N + 1]
  int* comb_ent = nullptr;
};
struct D2Rect {
  int r0, r1, c0, c1;
  int64_t off;                         // row-major values [r1 - r0][c1 - c0] at dense + off
};
struct D2Plan {
  int nb = 0;
  D2Dir fwd, adj;
  std::vector<D2Rect> rects_host;
  D2Rect* rects = nullptr;
  void* dense = nullptr;               // plan precision
  double* lam = nullptr;               // Lambda table of A^[1]
  int64_t dense_elems = 0, kept = 0;
};

// ------------------------------------------------------------------- the plan
struct Plan {
  int64_t N = 0;
  int family = 0, precision = 0, scheme = 0, normalise = 0;
  xc_params params{};
  double eps = 0, eps2 = 0, zeta = 0;
  Schedule sch;
  std::vector<BlockDev> blocks;        // device descriptors (pointers into plan memory)
  std::vector<int64_t> nnz, stored;
  std::vector<double> maxabs;
  int64_t m_tail = 0;
  int closed_form_blocks = 0;          // blocks whose rows came from the Appendix A closed form
  void* tail = nullptr;                // [m_tail][N] plan precision
  void* rowscale = nullptr;            // [N] or null (raw)
  void* colscale = nullptr;            // [N] or null (raw)
  double* nodes_dev = nullptr;         // [N] FP64
  double* rc_dev = nullptr;            // [3 nrc] recurrence coefficients (one-sided families)
  int64_t nrc = 0;
  std::vector<double> nodes_host;
  // work lists of the sparse kernels, longest item first: forward = row slices
  // (cost = summed band widths over blocks), adjoint = bin slices of all blocks
  int* f_order = nullptr;              // [nslices]
  int2* t_items = nullptr;             // [total_chunks]: (global bin slice, chunk), longest chunk first
  // the adjoint items of single-plan applies: the same as t_items / t_cbase,
  // or (small plans) a cut into shorter chunks of s_chunk rows
  int s_chunk = kAdjChunk;
  int64_t s_total_chunks = 0;
  int2* s_items = nullptr;
  int* s_cbase = nullptr;
  int* t_cbase = nullptr;              // [total_tslices + 1]: first chunk of each bin slice
  int64_t total_chunks = 0;
  std::vector<int64_t> slice_cost;     // host: summed forward band width of each row slice
  // forward chunking (plans with long bands): units (block, slice, chunk, rows)
  bool fwd_chunked = false;
  int4* fu_units = nullptr;            // [total_units]
  int* fu_order = nullptr;             // [total_units], longest first
  int* fu_ubase = nullptr;             // [nslices + 1]: first unit of each slice (units of a slice are consecutive)
  int64_t total_units = 0;
  bool any_yt = false;                 // some block reads the transposed right-hand sides
  std::vector<int> unit_len;           // host: rows of each unit (in fu_order order)
  std::vector<int> item_len;           // host: rows of each adjoint chunk, in t_items order
  int64_t nslices = 0, total_tslices = 0;
  unsigned* counters = nullptr;        // [4]: {next, done} for the forward and the adjoint sparse kernel
  int64_t spec_per_rhs = 0;            // complex elements of all blocks' spectra per RHS
  int64_t max_n = 0;                   // largest n of a block whose apply FFT runs in one CTA
  int max_csize = 1;                   // largest apply cluster of any block
  // complex families: one two-sided block over the full spectrum, circular
  // bands (xc_complex.cu); the forward spectra carry a periodic copy of their
  // first c_vpad bins after bin L-1 so that no band read wraps
  bool cplx = false;
  int c_vpad = 0;
  // XC_SCHEME_2D (xc_2d.cu); node spacing of the equispaced nodes
  D2Plan* d2 = nullptr;
  double x0 = 0, h = 0;
  // adjoint items of the complex block: (bin slice, chunk of 64 rows), item
  // g = c_cbase[slice] + chunk
  int2* c_items = nullptr;
  int* c_cbase = nullptr;              // [tslices + 1]
  int64_t c_nchunks = 0;
  int64_t matrix_bytes = 0, adjoint_bytes = 0;
  // window ("lockstep") layouts for batches (ensure_lockstep): host copies of
  // each block's windows, the elements they store, and the work lists over
  // them -- forward units (block, slice, first window position, length) with
  // the first unit of each slice, adjoint chunks (global bin slice, chunk of
  // kAdjChunk window rows) with the first chunk of each bin slice
  std::vector<std::vector<int>> hf_lo, hf_len, ht_lo, ht_len;
  int64_t lock_f_elems = 0, lock_t_elems = 0;
  bool lock_built = false;
  bool lock_f_ok = false, lock_t_ok = false;   // the windows cost at most kLockRatio x the band layouts
  // tensor windows (forward, XC_FP32 plans): built when they cost at most
  // kTensorRatio x the band layout; per block the tiles of each row group
  bool tens_ok = false;
  int64_t tens_elems = 0;
  int64_t tens_groups = 0;
  std::vector<std::vector<int>> tw_nkb_h;   // [block][group]
  WinBlock* win_blocks = nullptr;           // device copy, one per block
  // the same for the adjoint (groups of 64 bins per block), and the chunk
  // base of its partials (one chunk per bin slice: 0, 1, ..., total_tslices)
  bool tens_t_ok = false;
  int64_t tens_t_elems = 0;
  std::vector<std::vector<int>> tw_t_nkb_h;   // [block][group]
  WinBlock* win_blocks_t = nullptr;
  int* tw_tcbase = nullptr;
  int4* lk_units = nullptr;
  int* lk_ubase = nullptr;
  int64_t lk_total_units = 0;
  std::vector<int> lk_unit_len;
  int2* lk_items = nullptr;
  int* lk_cbase = nullptr;
  int64_t lk_total_chunks = 0;
  std::vector<int> lk_item_len;
  // device copy of `blocks` (read by the kernels), scratch spectra, host-path staging
  void* scratch_desc = nullptr;
  void* scratch = nullptr;
  int64_t scratch_nrhs = 0;
  // batches whose binding holds a pointer to `scratch` (xc_batch_bind);
  // while there are any, a growth keeps the old buffer in `retired` (freed
  // with the plan) instead of freeing it under the batch
  int batch_refs = 0;
  std::vector<void*> retired;
  size_t pexp_off = 0;                 // XC_FP64_PAIR: byte offset of the per-RHS exponents in scratch
  void* stage = nullptr;
  int64_t stage_elems = 0;
  std::vector<void*> allocations;      // everything cudaMalloc'ed for the plan
  cudaStream_t last_stream = nullptr;
  // per-kernel timing (xc_timing_enable)
  bool timing = false;
  struct Pending { int kernel; cudaEvent_t start, stop; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<int64_t> t_launches;
  std::vector<double> t_ms;
  bool io64() const { return precision == XC_FP64 || precision == XC_FP64_PAIR; }   // FP64 vectors, FFTs, tail
  size_t elem_bytes() const { return io64() ? 8 : 4; }   // one real value
  size_t io_bytes() const { return (cplx ? 2 : 1) * elem_bytes(); }   // one vector element
};

// Device allocation recorded in the plan (freed by xc_plan_destroy).
int plan_alloc(Plan* p, void** ptr, size_t bytes);

// Kernel identities for the launch counter and the per-kernel timing.
enum KernelId {
  K_FWD_FFT = 0, K_FWD_SPARSE, K_ADJ_SPARSE, K_ADJ_FFT, K_ADJ_TAIL, K_FWD_REDUCE, K_ADJ_TRANSPOSE, K_PAIR_SCALE,
  K_ROW_SCALE, K_2D_FFT_IN, K_2D_SPARSE, K_2D_FFT_OUT, K_2D_COMBINE, K_COUNT
};

// Row stride of the transposed adjoint input: nrhs rounded up to 8.
inline int64_t yt_ld(int64_t nrhs) { return (nrhs + 7) / 8 * 8; }
const char* kernel_name(int id);
// Bracket one launch: begin() before it, end() after it (counts the launch and,
// when timing is on, records events on the stream).
void launch_begin(Plan* p, int kernel, cudaStream_t s);
void launch_end(Plan* p, int kernel, cudaStream_t s);
// Count one launch without any event work (used by the allocation-free apply).
void count_launch();
// The allocation-free forward apply (xc_apply.cu).
int launch_apply_noalloc(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t s);

// ------------------------------------------------------------------- kernels
// (xc_plan.cu) precomputation
int build_plan_device(Plan* p);
int dense_matrix_device(const Plan* p, void* A, int64_t lda, cudaStream_t s);
// (xc_apply.cu) execution
int ensure_scratch(Plan* p, int64_t nrhs);
// (xc_abi.cpp) ensure_scratch for calls made while batches may point at the
// scratch: a buffer that has to grow is retired rather than freed
int ensure_scratch_kept(Plan* p, int64_t nrhs);
int launch_apply(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t s);
int launch_apply_adjoint(Plan* p, const void* y, void* x, int64_t nrhs, int64_t ld, cudaStream_t s);
// (xc_plan.cu) the window layouts of a real 1-D plan's blocks, built once;
// uploads the updated block descriptors
int ensure_lockstep(Plan* p);
// (xc_2d.cu) execution of the 2-D block scheme
size_t d2_scratch_bytes(const Plan* p, int64_t nrhs);
int launch_apply_2d(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t s, bool adjoint);
// (xc_complex.cu) execution of the complex families
size_t complex_scratch_bytes(const Plan* p, int64_t nrhs);
int launch_apply_complex(Plan* p, const void* x, void* y, int64_t nrhs, int64_t ld, cudaStream_t s);
int launch_adjoint_complex(Plan* p, const void* y, void* x, int64_t nrhs, int64_t ld, cudaStream_t s);

}  // namespace xc
