/*
 * xc.h -- C ABI of libxc, the GB300 (sm_103a) implementation of the
 * execution stage of the extra-component method for fast matrix-vector
 * products with special-function matrices (A. V. Terekhov, "An extra-component
 * method for evaluating fast matrix-vector multiplication with special
 * functions").
 *
 * The matrix is A[n, m] = phi_m(x_n), n = 0..N-1 (node), m = 0..N-1 (degree),
 * eq. (cheb_matrix) for the Chebyshev family and eq. (Jac_matrix) for the
 * orthogonal polynomials; Section 4 for the Laguerre functions.
 *
 *   xc_apply          y = A x      (Algorithm 1 for the two-sided Chebyshev
 *                                    family, Algorithm 3 for the block method)
 *   xc_apply_adjoint  x = A^T y    (Algorithm 2 / Algorithm 4)
 *
 * Conventions shared by every entry point
 *   - Return value: XC_OK (0) or a negative XC_ERR_* code.  No C++ exception
 *     crosses this boundary.  xc_strerror() names a code; xc_last_error_message()
 *     gives the text of the most recent failure on the calling thread.
 *   - Vectors are row-major [nrhs][ld] with ld >= N: right-hand side r occupies
 *     elements r*ld .. r*ld+N-1.  Their element type is the plan's I/O type:
 *     double for XC_FP64 and XC_FP64_PAIR plans, float for XC_FP32 and
 *     XC_FP32_COMPENSATED.
 *     The complex families (XC_EXP, XC_LAGUERRE_SPECTRAL) take complex
 *     vectors: an element is two consecutive values (re, im) of the I/O type,
 *     and ld, N and every element count are in complex elements.
 *   - Pointers named *_dev are device pointers owned by the caller; pointers
 *     named *_host are host pointers owned by the caller.  The plan owns every
 *     other buffer (compressed matrices, windows, twiddles, scratch).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Apply
 *     calls are asynchronous on that stream.  Calls on one plan must not
 *     overlap on the GPU: the plan's scratch is shared by its calls.
 *   - A plan is immutable after xc_plan_create, apart from the scratch growth
 *     done by xc_plan_reserve / the first apply with a larger nrhs.
 */
#ifndef XC_H_
#define XC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- error codes */
#define XC_OK               0
#define XC_ERR_ARG         -1   /* invalid argument (null pointer, N < 2, eps < 0, ...) */
#define XC_ERR_ALLOC       -2   /* device or host allocation failed */
#define XC_ERR_CUDA        -3   /* a CUDA runtime call or kernel launch failed */
#define XC_ERR_TIMEOUT     -4   /* a bounded device-side wait gave up */
#define XC_ERR_UNSUPPORTED -5   /* valid request outside what the library implements */

/* ---------------------------------------------------------------- families */
typedef enum {
  XC_CHEBYSHEV_T = 0,  /* T_m(x) = cos(m arccos x); two-sided extension (Section 2) */
  XC_LEGENDRE    = 1,  /* P_m(x); block method (Section 3, alpha = beta = 0) */
  XC_JACOBI      = 2,  /* P_m^{(alpha,beta)}(x); block method (Section 3) */
  XC_LAGUERRE_FN = 3,  /* l_m(x) = exp(-x/2) L_m(x) (Section 4); block method */
  XC_HERMITE_FN  = 4,  /* orthonormal Hermite functions psi_m(x); block method */
  XC_SINE        = 5,  /* sin(m theta_n), theta_n = arccos x_n (Section 2.2 names the sin and exp
                          matrices beside eq. (cheb_matrix)); two-sided extension */
  XC_COS_POWER   = 6,  /* cos^s(m theta_n), s = xc_params.power (eq. (cosd2)); two-sided extension */
  XC_EXP         = 7,  /* exp(i m theta_n), complex matrix and vectors (Section 2.2 names the exp
                          matrix beside eq. (cheb_matrix)).  The nodes are the angles theta_n
                          themselves: Gauss nodes = the midpoints (2n + 1 - N) pi / N of N equal
                          arcs (discretely orthogonal), user nodes = any real angles.  Two-sided
                          extension, one block. */
  XC_LAGUERRE_SPECTRAL = 8,  /* the spectral Laguerre matrix C of eq. (lag_matrix) (Section 4),
                          read as C[j, m] = (-eta/2 - i k_j)^m / (eta/2 - i k_j)^(m+1)
                          = exp(i m psi_j) / (eta/2 - i k_j), k_j = 2 pi j / T,
                          psi_j = 2 arctan(2 k_j / eta) - pi; eta = alpha > 0, T = beta > 0.
                          The exp part is compressed (an XC_EXP plan at the angles psi_j, which
                          xc_get_nodes returns), the factor 1/(eta/2 - i k_j) is applied to the
                          rows outside it.  xc_apply_adjoint gives C^T F (Fourier coefficients
                          to Laguerre coefficients).  Complex vectors. */
  XC_KERNEL_A1   = 9,  /* A^[1] of Section 5.3 (entries of the row and column indices):
                          Lambda(j)/pi on row 0, (2/pi) Lambda(j-i) Lambda(j+i) for 0 < i <= j,
                          0 below the diagonal, Lambda(z) = Gamma(z+1/2)/Gamma(z+1);
                          XC_SCHEME_2D only */
  XC_KERNEL_A2   = 10  /* A^[2] of Section 5.3: (i cos(log i^2) - j cos(log j^2)) / (i - j)^2,
                          0 on the diagonal (k cos(log k^2) read as 0 at k = 0); XC_SCHEME_2D only */
} xc_family;

/* node sets */
#define XC_NODES_GAUSS 0   /* Gauss nodes of the family (Chebyshev, sine, cos^s: x_n = cos((2n+1)pi/(2N))) */
#define XC_NODES_USER  1   /* caller-supplied nodes (user_nodes) */

/* normalisation */
#define XC_RAW         0   /* A[n,m] = phi_m(x_n) */
#define XC_ORTHONORMAL 1   /* sqrt(lambda_n / chi_m) phi_m(x_n): orthogonal at Gauss nodes (Section 5.2);
                              the threshold is taken on this matrix's compressed rows,
                              lambda_n |a|^2 > eps1^2 max(lambda |a|^2), so the accuracy
                              does not fall with the Jacobi alpha, beta */

/* apply precision */
#define XC_FP64             0   /* FP64 FFT, FP64 sparse product */
#define XC_FP32             1   /* FP32 FFT, FP32 sparse product */
#define XC_FP32_COMPENSATED 2   /* FP32 FFT; sparse product and dense tail accumulated
                                   with error-free transformations (TwoProduct/TwoSum) */
#define XC_FP64_PAIR        3   /* FP64 vectors, FFTs and dense tail; band values and spectra as
                                   pairs of FP32 (hi + lo, 48-bit significands), band products on the
                                   FP32 pipes accumulated with TwoProduct/TwoSum.  I/O type double.
                                   Single-plan applies only (not xc_batch_*, not xc_apply_noalloc). */

/* extension scheme */
#define XC_SCHEME_AUTO      0   /* two-sided for the trigonometric families, block method otherwise */
#define XC_SCHEME_TWO_SIDED 1   /* Algorithms 1-2; trigonometric families (Chebyshev, sine, cos^s) only */
#define XC_SCHEME_BLOCKS    2   /* Algorithms 3-4 */
#define XC_SCHEME_2D        3   /* the 2-D compression F W D W F (eq. (comp_2d)) in its block
                                   scheme (Sections 4.2, 5.3): rectangles of the matrix, each
                                   extended below and to the right, compressed along both
                                   dimensions; the rows and columns whose window is below eps2
                                   form further rectangles, thin ones (a side <= tail_max) are
                                   dense.  XC_LAGUERRE_FN / XC_HERMITE_FN at equispaced user nodes
                                   (x_i = x_0 + i h, extended with the same step) and
                                   XC_KERNEL_A1 / XC_KERNEL_A2; XC_FP64 or XC_FP32; real vectors.
                                   Blocks up to L <= 28928 along each side (N up to about 19000);
                                   at most 65535 right-hand sides per apply (else
                                   XC_ERR_UNSUPPORTED).  The error bound is eps1 / eps2^2 (two
                                   window divisions): take eps2 larger than for 1-D plans. */

/* precomputation of the compressed rows */
#define XC_PRECOMPUTE_AUTO 0   /* Appendix A closed form for XC_CHEBYSHEV_T at its Gauss nodes with
                                  eps > 0 (blocks of a few hundred columns and more), FFT of the
                                  generated rows otherwise */
#define XC_PRECOMPUTE_FFT  1   /* always the FFT of the generated rows (Algorithm 1 step 1.3 as written) */

typedef struct {
  double alpha, beta;        /* Jacobi parameters (> -1); eta and T (> 0) of XC_LAGUERRE_SPECTRAL;
                                ignored by the other families */
  int nodes;                 /* XC_NODES_GAUSS | XC_NODES_USER */
  const double* user_nodes;  /* host, N entries, copied at create; used when nodes == XC_NODES_USER */
  int normalise;             /* XC_RAW | XC_ORTHONORMAL (orthonormal needs Gauss nodes and a
                                polynomial family: not XC_SINE / XC_COS_POWER) */
  double eps2;               /* window floor of the first real component; 0 => 1e-3 (FP64) or 1e-1 (FP32) */
  double eps_window;         /* eps that fixes zeta when eps == 0; 0 => 1e-14 */
  int precision;             /* XC_FP64 | XC_FP32 | XC_FP32_COMPENSATED | XC_FP64_PAIR */
  int scheme;                /* XC_SCHEME_* */
  int tail_max;              /* blocks are added while m_i > tail_max; 0 => 20 */
  int precompute;            /* XC_PRECOMPUTE_* */
  int power;                 /* s of XC_COS_POWER, 1..16; 0 => 2 */
} xc_params;

/* Fill *p with the defaults listed above (Gauss nodes, raw, FP64, auto scheme). */
void xc_params_default(xc_params* p);

typedef struct xc_plan* xc_plan_t;

/*
 * xc_plan_create -- precomputation stage of Algorithms 1-4 (step 1 of each).
 *   family  an xc_family value
 *   p       parameters (NULL => defaults); user_nodes is copied
 *   N       matrix order, 2 <= N <= 2^20
 *   eps     eps1 of the paper: elements of the compressed matrix with
 *           |a| <= eps * max|A_e W F| (per block) are dropped, and the Kaiser
 *           shape zeta solves 1/I0(zeta) = eps (Section 2.2).  eps == 0 keeps
 *           every element and takes zeta from p->eps_window.
 * Runs on the current CUDA device and synchronises it.  On success *out owns
 * all device memory of the plan; on failure *out is NULL and nothing leaks.
 * Complex families: precision XC_FP64 or XC_FP32, the two-sided scheme, raw
 * normalisation, and a block length L whose L/2 complex FP64 values fit one
 * CTA's shared memory (L <= 28928; L / N is about 1.46 at eps1 = 1e-10,
 * eps2 = 1e-3 and 1.9 at eps1 = 1e-6, eps2 = 0.1, so N up to about 19800 and
 * 15000); otherwise XC_ERR_UNSUPPORTED.  Such plans are applied by
 * xc_apply / xc_apply_adjoint / xc_apply_host only (xc_apply_noalloc and
 * the batches return XC_ERR_UNSUPPORTED).
 */
int xc_plan_create(xc_plan_t* out, int family, const xc_params* p, int64_t N, double eps);

/* Release every resource of the plan (NULL is accepted).  Synchronises the device. */
int xc_plan_destroy(xc_plan_t plan);

/*
 * xc_plan_reserve -- allocate the scratch needed by applies with up to nrhs
 * right-hand sides, so that later applies allocate nothing.
 */
int xc_plan_reserve(xc_plan_t plan, int64_t nrhs);

/*
 * xc_apply -- y = A x (Algorithm 1 step 2 / Algorithm 3): per block, extend the
 * input with zero extra components (eq. (Fe1) / (Fe3)), divide by the window,
 * FFT, multiply by the compressed matrix; add the dense tail.  Plans whose
 * bands (summed over blocks) exceed 512 bins in some 32-row slice sum each
 * row's band in chunks of 256 bins and add the chunks in a fixed order; the
 * summation order is a property of the plan, so a column's result does not
 * depend on nrhs, on the stream or on batching.
 *   x_dev  device, [nrhs][ld] of the plan's I/O type (read only)
 *   y_dev  device, [nrhs][ld] (columns [0, N) of each row written, the rest
 *          untouched); its elements up to the last used one, ((nrhs-1) ld + N)
 *          of them, must not overlap those of x_dev (XC_ERR_ARG)
 *   nrhs   number of right-hand sides (0 is a no-op; at most 524280)
 *   ld     leading dimension in elements, N <= ld, nrhs * ld <= 2^40
 */
int xc_apply(xc_plan_t plan, const void* x_dev, void* y_dev, int64_t nrhs, int64_t ld, void* stream);
/* (xc_apply and xc_apply_adjoint share the plan's scratch and the work
 * counters of its sparse kernels, which each launch's last warp resets: two
 * calls on one plan must not overlap on the GPU, or items are skipped and
 * outputs left unwritten.  Order them on one stream, or use one plan per
 * stream.) */

/*
 * xc_apply_adjoint -- x = A^T y (Algorithm 2 step 2 / Algorithm 4): per block,
 * multiply by the transposed compressed matrix, inverse FFT, divide by the
 * window and discard the extra components (eq. (Fe2)); the dense tail writes
 * the first m_tail entries.  Exactly the transpose of xc_apply's operator
 * (for the complex families the plain transpose, not the conjugate one).
 * Same argument conventions as xc_apply (y_dev is read, x_dev written).
 */
int xc_apply_adjoint(xc_plan_t plan, const void* y_dev, void* x_dev, int64_t nrhs, int64_t ld, void* stream);

/*
 * xc_apply_noalloc -- the same y = A x as xc_apply, for callers that must not
 * allocate device memory: code running where cudaMalloc is forbidden or
 * unsafe (inside a memory-pool-managed runtime that owns every allocation,
 * real-time paths where an allocation could stall, or hosts that budget
 * device memory up front).  The paper has no counterpart; this is an
 * interface convenience of the library.
 *
 * The spectra that xc_apply keeps in the plan's scratch are placed instead in
 * one fixed device array inside the library, XC_NOALLOC_SCRATCH_BYTES large,
 * which every GPU that loads the library holds until the process exits.  The
 * call allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * routine.  It needs (sum over blocks of L_i/2 + 1) * nrhs complex elements
 * of the plan's precision; larger requests return XC_ERR_UNSUPPORTED before
 * anything is launched (split the right-hand sides into several calls).
 * Every row's band is summed in one pass (plans with long bands included:
 * no chunk partials, which would need more scratch), so results equal
 * xc_apply's to rounding, not bit for bit, on such plans.
 *
 * Refused with XC_ERR_UNSUPPORTED, before anything is launched:
 *   - XC_FP64_PAIR plans;
 *   - the complex families (XC_EXP, XC_LAGUERRE_SPECTRAL) and XC_SCHEME_2D plans;
 *   - plans with a block whose FFT needs a thread-block cluster, i.e. whose
 *     L/2 complex values exceed one CTA's shared memory: L > 28928 in FP64,
 *     L > 57856 in FP32 (block method: N above about 23000 in FP64 at
 *     eps2 = 1e-3 and about 43000 in FP32 at eps2 = 1e-1).
 *
 *   - The first call on a device looks up that device's address of the array
 *     (once per device, with the device current); make that first call before
 *     any stream capture on the device.
 *   - All calls share the one array, and one pair of work counters of the
 *     sparse kernel beside it (also a fixed device array, reset by each
 *     launch's last warp); the array keeps the last call's contents.  Every
 *     element a call reads was written earlier in the same call, so nothing
 *     needs clearing, but calls that overlap on the GPU (different streams,
 *     or different plans at the same time) race on the array and on the
 *     counters: order them, e.g. on one stream.  A call does not share
 *     scratch or counters with xc_apply / xc_apply_adjoint on the same plan.
 * Arguments as for xc_apply.
 */
#define XC_NOALLOC_SCRATCH_BYTES (16ll << 20)
int xc_apply_noalloc(xc_plan_t plan, const void* x_dev, void* y_dev, int64_t nrhs, int64_t ld, void* stream);

/*
 * xc_apply_host -- end-to-end forward or adjoint apply on HOST buffers:
 * copies the input to the device, applies, copies the result back and
 * synchronises the stream.  adjoint = 0: out = A in; adjoint = 1: out = A^T in.
 * in_host / out_host: [nrhs][ld] of the plan's I/O type (pinned memory gives
 * full copy bandwidth); only the first N elements of each row are read from
 * in_host and written to out_host, the padding [N, ld) of out_host keeps its
 * contents.  Uses device staging owned by the plan.
 */
int xc_apply_host(xc_plan_t plan, int adjoint, const void* in_host, void* out_host,
                  int64_t nrhs, int64_t ld, void* stream);

/* Per-block statistics reported by xc_plan_info. */
#define XC_MAX_BLOCKS 16
typedef struct {
  int64_t N;
  int family, precision, scheme, normalise;
  double eps, eps2, zeta;
  int nblocks;
  int64_t L[XC_MAX_BLOCKS];          /* FFT length of block i */
  int64_t off[XC_MAX_BLOCKS];        /* extended column j holds matrix column j - off */
  int64_t j_lo[XC_MAX_BLOCKS];       /* real input occupies extended columns [j_lo, j_hi) */
  int64_t j_hi[XC_MAX_BLOCKS];
  int64_t nnz[XC_MAX_BLOCKS];        /* kept elements in the half spectrum k = 0..L/2 (complex
                                        families: in the full spectrum) */
  int64_t stored[XC_MAX_BLOCKS];     /* stored band elements incl. explicit zeros (forward layout) */
  double maxabs[XC_MAX_BLOCKS];      /* max |A_e W F| of the block */
  int64_t m_tail;                    /* dense tail columns [0, m_tail) */
  int64_t matrix_bytes;              /* device bytes of the compressed matrices + tail (forward) */
  int64_t adjoint_bytes;             /* device bytes of the transposed copies */
  int closed_form_blocks;            /* blocks whose rows the Appendix A closed form built
                                        (the others: FFT of the generated rows) */
  /* XC_SCHEME_2D plans (the per-block arrays above then stay empty, nblocks = 0): */
  int blocks2d;                      /* compressed 2-D blocks */
  int dense2d;                       /* dense rectangles */
  int64_t nnz2d;                     /* kept elements of the compressed blocks (full spectra) */
  int64_t dense_elems2d;             /* elements of the dense rectangles */
} xc_plan_stats;

/* Copy the plan's parameters and per-block statistics into *out. */
int xc_plan_info(xc_plan_t plan, xc_plan_stats* out);

/* Copy the plan's N nodes (FP64, the order of the rows of A) into host_out
 * (the angles for XC_EXP / XC_LAGUERRE_SPECTRAL, the row indices for the index
 * kernels). */
int xc_get_nodes(xc_plan_t plan, double* host_out);

/*
 * xc_dense_matrix -- write the plain N x N matrix (with the plan's
 * normalisation) to A_dev, row-major with leading dimension lda >= N, in the
 * plan's I/O type.  Generated on the device by the same recurrences as the
 * precompute; used by the dense-GEMM comparison.
 */
int xc_dense_matrix(xc_plan_t plan, void* A_dev, int64_t lda, void* stream);

/* ---------------------------------------------------------------- batches
 * Many plans (uneven N, families, numbers of right-hand sides; one precision)
 * applied by one persistent kernel launch per direction.  The launch works
 * through a device task list over all plans: phase 1 (forward: the FFTs;
 * adjoint: the transposed band products and dense tails), then phase 2
 * (forward: the band products and tails; adjoint: the inverse FFTs), then,
 * for the forward products of long-band plans, phase 3 (the sums of their
 * chunk partials, as in xc_apply).  A task of a phase waits, with a bounded
 * number of sleeps, until all tasks of the plan's previous phase have
 * finished; a wait that runs out sets the
 * batch's status to XC_ERR_TIMEOUT (read by xc_batch_status) instead of
 * hanging.  This is the batched form of Algorithms 1-4; the paper itself
 * applies one matrix at a time.
 */
typedef struct xc_batch* xc_batch_t;
typedef struct {
  int nplans;
  int rhs_per_item;          /* right-hand sides per forward band-product task (tuned) */
  int tuned;                 /* 1 after xc_batch_tune */
  int rhs_per_item_adjoint;  /* right-hand sides per adjoint band-product task (tuned) */
  int64_t tasks_forward, tasks_adjoint;
  int64_t shared_bytes;      /* dynamic shared memory of the persistent kernel */
  int64_t matrix_bytes, adjoint_bytes;   /* summed over the plans */
  int lockstep_forward;      /* 1: plans with tight windows use lockstep band items forward; 2: tensor
                                windows where plans have them (tuned) */
  int lockstep_adjoint;      /* the same for the adjoint */
  int lockstep_plans;        /* plans that run lockstep items in at least one direction */
  /* the tuner's timings (ms, summed over 3 launches) per candidate schedule,
   * entry 4 * lockstep + log2(right-hand sides per item); -1 where not tried */
  float tune_ms_forward[12], tune_ms_adjoint[12];
  int tensor_plans;          /* plans whose forward band products run on the tensor cores */
  int tensor_plans_adjoint;  /* the same for the adjoint band products */
} xc_batch_stats;

/* Group nplans distinct plans (host array of handles; all of one precision;
 * a plan listed twice is XC_ERR_ARG).  The batch refers to the plans, which
 * must outlive it. */
int xc_batch_create(xc_batch_t* out, const xc_plan_t* plans, int nplans);
/* Bind the I/O buffers: x_dev[i], y_dev[i] are device pointers to
 * [nrhs[i]][ld[i]] arrays of plan i's type (ld[i] >= N_i; nrhs[i] = 0 skips the
 * plan).  The forward apply reads x and writes y, the adjoint reads y and
 * writes x.  Allocates the plans' scratch and builds the task lists
 * (synchronous).  All arguments are checked first: a refused bind leaves the
 * previous binding in force.  The binding points at each plan's scratch; a
 * later single-plan apply (or bind of another batch) that needs more scratch
 * allocates a new buffer and the plan keeps the one the batch uses until the
 * plan is destroyed, so the binding stays valid.  If building the task lists
 * fails the batch is left unbound (xc_batch_apply returns XC_ERR_ARG). */
int xc_batch_bind(xc_batch_t b, const void* const* x_dev, void* const* y_dev, const int64_t* nrhs, const int64_t* ld);
/* One persistent launch over all bound plans (adjoint = 0: y = A x for every
 * plan; 1: x = A^T y), and, forward, up to three tensor-core launches for
 * the plans whose band products run on tensor windows (below).
 * Asynchronous on `stream`; allocates nothing and does not synchronise, so
 * it can be captured in a CUDA graph and replayed.  Launches of one batch,
 * and of batches sharing a plan, must not overlap. */
int xc_batch_apply(xc_batch_t b, int adjoint, void* stream);
/* Autotuner: times the bound problem with 1, 2, 4 and 8 right-hand sides per
 * band-product task, with tensor windows forward (where plans have them),
 * with lockstep items and with neither (forward + adjoint, 3 repetitions
 * each), and keeps the fastest per direction; the choice is cached per batch
 * shape for later binds in the process.  Synchronises `stream`; the bound
 * buffers are restored afterwards.
 *
 * Lockstep items: a bind of an FP32 batch builds, for plans whose bands
 * line up across the 32 rows of a slice (the union of the rows' bands, and
 * of the bins' row runs, at most 1.25 times the stored bands: Hermite
 * functions), window copies of both band layouts; their band products then
 * walk one bin (row) per step for the whole warp, and their spectra are
 * stored bin-major in scratch owned by the batch.  Plans with long bands sum
 * them in window pieces whose grouping differs from xc_apply's, so those
 * results equal xc_apply's to rounding, not bit for bit.
 *
 * Tensor windows: a bind of an XC_FP32 batch also builds, for plans whose
 * bands over groups of 128 rows (adjoint: the rows of groups of 64 bins)
 * cost at most 1.5 times their stored bands, 16 KB tiles of the band
 * layouts; with lockstep 2 the band products of those plans with at most 64
 * right-hand sides run as dense 3xTF32 tensor-core products over the tiles
 * (tcgen05, FP32 accuracy, xc_window.cuh): forward after the persistent
 * launch has made their spectra, adjoint before it, which then runs their
 * inverse FFTs.  Their results equal xc_apply's to FP32 rounding. */
int xc_batch_tune(xc_batch_t b, void* stream);
/* Set the schedule by hand instead of tuning it: right-hand sides per band
 * item (1, 2, 4 or 8) and lockstep items on (1) or off (0), per direction;
 * lockstep 2 runs the band products of the plans with tensor windows on the
 * tensor cores in that direction (lockstep items for the other plans that
 * have them).
 * Rebuilds the task lists (synchronous); XC_ERR_ARG before a bind. */
int xc_batch_schedule(xc_batch_t b, int rpw_forward, int rpw_adjoint, int lockstep_forward, int lockstep_adjoint);
int xc_batch_info(xc_batch_t b, xc_batch_stats* out);
/* Synchronise `stream` and report XC_ERR_TIMEOUT if a phase wait of an
 * earlier launch gave up (then clear it); XC_OK otherwise.  While the status
 * is set, later launches skip their tasks. */
int xc_batch_status(xc_batch_t b, void* stream);
/* Fault injection for tests: plan `plan` needs `extra_need` more phase-1
 * completions than exist (so its phase-2 waits run out), and every wait gives
 * up after wait_limit sleeps of ~256 ns.  extra_need = 0 restores the plan. */
int xc_batch_debug_set(xc_batch_t b, int plan, int extra_need, int64_t wait_limit);
int xc_batch_destroy(xc_batch_t b);

/* ------------------------------------------------- direct dense product
 * The product the method replaces: y = A x with the plain matrix A (Section
 * 1, eq. (cheb_matrix) / eq. (Jac_matrix); Section 5 compares the method with
 * it), as a dense GEMM on the tensor cores (tcgen05) at FP32 accuracy:
 * every FP32 value v = hi + lo with hi, lo exact TF32 numbers (hi = v rounded
 * to TF32, lo = v - hi rounded to TF32), products accumulated as
 * hi hi + hi lo + lo hi in FP32 ("3xTF32"; the dropped lo lo term is below
 * 2^-22 of each product).  The benchmark times it beside the method; it is a
 * comparator, not part of the method.
 */
typedef struct xc_dense* xc_dense_t;
/* Copy A_dev (device, FP32, row-major [M][lda], lda >= K) into the
 * comparator: its split A and the split of A^T (both K-major for the tensor
 * cores), 16 M K bytes of device memory owned by the comparator.  A_dev is
 * not referenced afterwards.  Synchronises `stream`. */
int xc_dense_create(xc_dense_t* out, const float* A_dev, int64_t M, int64_t K, int64_t lda, void* stream);
/* transpose = 0: out[r][m] = sum_k A[m][k] in[r][k]  (m < M, k < K);
 * transpose = 1: out[r][k] = sum_m A[m][k] in[r][m].
 * in_dev, out_dev: device FP32 [nrhs][ld], ld >= max(M, K), not overlapping
 * (XC_ERR_ARG); only the first M (or K) entries of each output row are
 * written.  Asynchronous on `stream`; the first call with a larger nrhs
 * allocates the split right-hand sides (8 nrhs max(M, K) bytes, kept).  Calls
 * on one comparator must not overlap on the GPU.  A device wait that runs out
 * (about two seconds) is reported by xc_dense_status. */
int xc_dense_apply(xc_dense_t dense, int transpose, const float* in_dev, float* out_dev, int64_t nrhs, int64_t ld,
                   void* stream);
/* Synchronise `stream`; XC_ERR_TIMEOUT (then cleared) if a wait inside an
 * earlier xc_dense_apply gave up, XC_OK otherwise. */
int xc_dense_status(xc_dense_t dense, void* stream);
int xc_dense_destroy(xc_dense_t dense);

/*
 * Per-kernel timing.  While enabled, every kernel the plan launches is
 * bracketed by two CUDA events recorded on the launch stream; xc_timing_read
 * synchronises those events and returns, per kernel name, the number of
 * launches and their summed device time since the previous read (then resets).
 * Timing adds two event records per launch; leave it off for throughput runs.
 */
typedef struct {
  char name[32];      /* kernel name, e.g. "fwd_sparse" */
  int64_t launches;
  double total_ms;
} xc_kernel_time;
int xc_timing_enable(xc_plan_t plan, int enable);
/* out: caller array of max entries; *count receives the number filled. */
int xc_timing_read(xc_plan_t plan, xc_kernel_time* out, int max, int* count);

/* Total number of kernels launched by this library in the process so far. */
int64_t xc_launch_count(void);

/*
 * xc_sync_status -- synchronise the plan's last stream and report any error
 * recorded by the device since the last call (XC_OK if none).
 */
int xc_sync_status(xc_plan_t plan);

const char* xc_strerror(int code);
const char* xc_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* XC_H_ */
