// Precomputation stage of Algorithms 1-4 on the device, in FP64:
//   nodes (closed form, or Sturm bisection + Newton on the three-term
//   recurrence), the Kaiser window and its reciprocal, FFT twiddles, the rows of
//   the extended matrix A_e by recurrence (step 1.2), their real FFTs giving the
//   compressed matrix A_e W F (eq. (A_comp), step 1.3), the per-block maximum,
//   the threshold |a| > eps1 * max|A_e W F|, and the banded storage of the kept
//   elements for the forward and the transposed (adjoint) product.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "xc_fft.cuh"
#include "xc_internal.h"
#include "xc_items.cuh"

namespace xc {

namespace {

// ------------------------------------------------------- family evaluation
struct GenParams {
  int family;
  int64_t N;
  double alpha, beta;
  const double* x;      // nodes
  int cheb_exact;       // trigonometric family at x_n = cos((2n+1) pi / (2N)): exact angles
  int power;            // s of the cos^s family
  // three-term recurrence phi_{m+1} = (rc[3m] + rc[3m+1] x) phi_m - rc[3m+2] phi_{m-1}
  // for m < nrc (null for the trigonometric families)
  const double* rc = nullptr;
  int64_t nrc = 0;
  int cpart = 0;        // complex families: 0 = real part cos(m theta), 1 = imaginary part sin(m theta)
  // orthonormal variant: lambda_n, the squared row scale, which weights the
  // threshold (null: unweighted)
  const double* rw = nullptr;
};

__host__ __device__ __forceinline__ bool is_complex_family(int family) {
  return family == XC_EXP || family == XC_LAGUERRE_SPECTRAL;
}

__host__ __device__ __forceinline__ bool is_trig(int family) {
  return family == XC_CHEBYSHEV_T || family == XC_SINE || family == XC_COS_POWER || family == XC_EXP ||
         family == XC_LAGUERRE_SPECTRAL;
}

// exp(-a) for a >= 0 as mant * 2^expo, with the argument split
// a = q ln2 - r (q integer, ln2 = hi + lo, q * hi exact: the published
// Cody-Waite additive range reduction) so that the result keeps full
// relative accuracy even when exp(-a) is far below the FP64 range; the
// reduced exp(-r) is CUDA's own exp.  a_lo carries a low-order part of the
// argument (exact products).
__device__ void exp_neg_split(double a_hi, double a_lo, double* mant, int* expo) {
  const double ln2_hi = 0.6931471803691238;          // ln 2 to 32 significant bits
  const double ln2_lo = 1.9082149292705877e-10;      // ln 2 - ln2_hi
  const double inv_ln2 = 1.4426950408889634;
  const double q = rint(a_hi * inv_ln2);
  // exp(-a) = 2^{-q} exp(q ln2 - a)
  const double r = ((q * ln2_hi - a_hi) + q * ln2_lo) - a_lo;
  double m = exp(r);
  int e2 = 0;
  m = frexp(m, &e2);
  *mant = m;
  *expo = e2 - int(q);
}

// Emit phi_m(x_n) for m in [m_lo, m_hi) to `emit(m, value)` in increasing m.
template <class F>
__device__ void gen_values(const GenParams& g, int64_t n, int64_t m_lo, int64_t m_hi, F emit) {
  const double x = g.x[n];
  if (is_complex_family(g.family)) {
    // exp(i m theta_n), one part at a time; the node is the angle itself
    if (g.cheb_exact) {
      // theta_n = pi (2n + 1 - N) / N: angle pi k / N with k = m (2n + 1 - N) mod 2N
      const int64_t per = 2 * g.N;
      int64_t num = (2 * n + 1 - g.N) % per;
      if (num < 0) num += per;
      for (int64_t m = m_lo; m < m_hi; ++m) {
        int64_t mm = m % per;
        if (mm < 0) mm += per;
        int64_t k = mm * num % per;
        double sign = 1.0;
        if (k > g.N) {                                 // angle in (pi, 2 pi): sin odd
          k = per - k;
          sign = -1.0;
        }
        const double a = double(k) / double(g.N);      // in [0, 1]
        emit(m, g.cpart ? sign * sinpi(a) : cospi(a));
      }
    } else {
      for (int64_t m = m_lo; m < m_hi; ++m) {
        double sn, c;
        sincos(double(m) * x, &sn, &c);
        emit(m, g.cpart ? sn : c);
      }
    }
    return;
  }
  if (is_trig(g.family)) {
    // cos(m theta), sin(m theta) or cos^s(m theta) of the row's angle
    auto finish = [&](double c, double sn) {
      if (g.family == XC_SINE) return sn;
      if (g.family == XC_COS_POWER) {
        double v = c;
        for (int i = 1; i < g.power; ++i) v *= c;
        return v;
      }
      return c;
    };
    if (g.cheb_exact) {
      // angle = pi m (2n+1) / (2N); period 4N in m (2n+1)
      const int64_t num = 2 * n + 1, per = 4 * g.N;
      for (int64_t m = m_lo; m < m_hi; ++m) {
        int64_t k = (m % per) * num % per;
        if (k < 0) k += per;
        double sign = 1.0;
        if (k > per / 2) {                             // angle in (pi, 2 pi): cos even, sin odd
          k = per - k;
          sign = -1.0;
        }
        const double a = double(k) / double(2 * g.N);  // in [0, 1]
        emit(m, finish(cospi(a), g.family == XC_SINE ? sign * sinpi(a) : 0.0));
      }
    } else {
      const double th = acos(fmin(1.0, fmax(-1.0, x)));
      for (int64_t m = m_lo; m < m_hi; ++m) {
        double sn, c;
        sincos(double(m) * th, &sn, &c);
        emit(m, finish(c, sn));
      }
    }
    return;
  }
  // one-sided families start at m = 0
  if (g.family == XC_LEGENDRE || g.family == XC_JACOBI) {
    const double a = g.family == XC_JACOBI ? g.alpha : 0.0;
    const double b = g.family == XC_JACOBI ? g.beta : 0.0;
    double pm1 = 1.0;
    double p = (a + 1.0) + (a + b + 2.0) * (x - 1.0) * 0.5;
    if (m_lo <= 0 && 0 < m_hi) emit(0, pm1);
    if (m_lo <= 1 && 1 < m_hi) emit(1, p);
    for (int64_t m = 1; m + 1 < m_hi; ++m) {
      double pn;
      if (m < g.nrc) {
        pn = (g.rc[3 * m] + g.rc[3 * m + 1] * x) * p - g.rc[3 * m + 2] * pm1;
      } else {
        const double c = 2.0 * m + a + b;
        const double a1 = 2.0 * (m + 1) * (m + a + b + 1) * c;
        const double a2 = (c + 1) * (a * a - b * b);
        const double a3 = c * (c + 1) * (c + 2);
        const double a4 = 2.0 * (m + a) * (m + b) * (c + 2);
        pn = ((a2 + a3 * x) * p - a4 * pm1) / a1;
      }
      pm1 = p;
      p = pn;
      if (m + 1 >= m_lo) emit(m + 1, p);
    }
    return;
  }
  // Laguerre / Hermite functions: scaled recurrence with a power-of-two exponent
  double mant;
  int expo;
  double pm1, p;
  if (g.family == XC_LAGUERRE_FN) {
    exp_neg_split(0.5 * x, 0.0, &mant, &expo);           // exp(-x/2)
    pm1 = mant;
    p = (1.0 - x) * mant;
  } else {
    const double xx = x * x;
    const double xx_lo = fma(x, x, -xx);                 // x^2 = xx + xx_lo exactly
    exp_neg_split(0.5 * xx, 0.5 * xx_lo, &mant, &expo);  // exp(-x^2/2)
    mant *= 0.7511255444649425;                          // pi^(-1/4)
    pm1 = mant;
    p = 1.4142135623730951 * x * mant;
  }
  // values times 2^expo: one multiply while 2^expo is a normal number
  double sc = ldexp(1.0, expo);
  bool sc_ok = expo >= -1000 && expo <= 1000;
  auto scaled = [&](double v) { return sc_ok ? v * sc : ldexp(v, expo); };
  if (m_lo <= 0 && 0 < m_hi) emit(0, scaled(pm1));
  if (m_lo <= 1 && 1 < m_hi) emit(1, scaled(p));
  for (int64_t m = 1; m + 1 < m_hi; ++m) {
    double pn;
    if (m < g.nrc)
      pn = (g.rc[3 * m] + g.rc[3 * m + 1] * x) * p - g.rc[3 * m + 2] * pm1;
    else if (g.family == XC_LAGUERRE_FN)
      pn = ((2.0 * m + 1.0 - x) * p - double(m) * pm1) / double(m + 1);
    else
      pn = sqrt(2.0 / double(m + 1)) * x * p - sqrt(double(m) / double(m + 1)) * pm1;
    pm1 = p;
    p = pn;
    const double big = fmax(fabs(p), fabs(pm1));
    if (big > 0x1p+500) {
      p *= 0x1p-500;
      pm1 *= 0x1p-500;
      expo += 500;
      sc = ldexp(1.0, expo);
      sc_ok = expo >= -1000 && expo <= 1000;
    } else if (big < 0x1p-500 && big > 0.0) {
      p *= 0x1p+500;
      pm1 *= 0x1p+500;
      expo -= 500;
      sc = ldexp(1.0, expo);
      sc_ok = expo >= -1000 && expo <= 1000;
    }
    if (m + 1 >= m_lo) emit(m + 1, scaled(p));
  }
}

// ---------------------------------------------------------------- nodes
// Number of eigenvalues of the symmetric tridiagonal matrix (d, e) below lam
// (Sturm count through the LDL^T pivots).
__device__ int sturm_count(const double* d, const double* e2, int64_t N, double lam) {
  int cnt = 0;
  double q = d[0] - lam;
  if (q == 0.0) q = -1e-300;
  cnt += q < 0.0;
  for (int64_t i = 1; i < N; ++i) {
    q = (d[i] - lam) - e2[i - 1] / q;
    if (q == 0.0) q = -1e-300;
    cnt += q < 0.0;
  }
  return cnt;
}

// Sturm counts at G+1 points of [lo, hi], spaced like the zeros: uniform in
// theta for lo + h (1 - cos(pi u)) (polynomials on [-1, 1], Hermite
// functions), uniform in sqrt(x - lo) for the Laguerre functions, whose zeros
// crowd near 0.  The ends are set to 0 and N: [lo, hi] strictly contains the
// spectrum.
__global__ void grid_count_kernel(const double* d, const double* e2, int64_t N, double lo, double hi,
                                  int square, int64_t G, double* grid, int* counts) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > G) return;
  const double u = double(i) / double(G);
  const double x = square ? lo + (hi - lo) * u * u : lo + 0.5 * (hi - lo) * (1.0 - cospi(u));
  grid[i] = x;
  counts[i] = i == 0 ? 0 : i == G ? int(N) : sturm_count(d, e2, N, x);
}
// (p_N, p_{N-1}) at x by the family's recurrence; a common scale factor may
// remain (it cancels in the Newton ratio).
__device__ void last_two(int family, int64_t N, double a, double b, double x, double* pN, double* pN1) {
  double pm1 = 1.0, p;
  if (family == XC_LEGENDRE || family == XC_JACOBI) {
    p = (a + 1.0) + (a + b + 2.0) * (x - 1.0) * 0.5;
    for (int64_t m = 1; m < N; ++m) {
      const double c = 2.0 * m + a + b;
      const double pn = ((c + 1) * ((c + 2) * c * x + a * a - b * b) * p - 2.0 * (m + a) * (m + b) * (c + 2) * pm1) /
                        (2.0 * (m + 1) * (m + a + b + 1) * c);
      pm1 = p;
      p = pn;
    }
  } else if (family == XC_LAGUERRE_FN) {
    p = 1.0 - x;
    for (int64_t m = 1; m < N; ++m) {
      const double pn = ((2.0 * m + 1.0 - x) * p - double(m) * pm1) / double(m + 1);
      pm1 = p;
      p = pn;
      if (fabs(p) > 0x1p+500) { p *= 0x1p-500; pm1 *= 0x1p-500; }
    }
  } else {
    p = 1.4142135623730951 * x;
    for (int64_t m = 1; m < N; ++m) {
      const double pn = sqrt(2.0 / double(m + 1)) * x * p - sqrt(double(m) / double(m + 1)) * pm1;
      pm1 = p;
      p = pn;
      if (fabs(p) > 0x1p+500) { p *= 0x1p-500; pm1 *= 0x1p-500; }
    }
  }
  *pN = p;
  *pN1 = pm1;
}

// phi_N / phi_N' from the derivative identities of each family.
__device__ double newton_ratio(int family, int64_t N, double a, double b, double x) {
  double pN, pN1;
  last_two(family, N, a, b, x, &pN, &pN1);
  double d;
  if (family == XC_LEGENDRE || family == XC_JACOBI) {
    const double c = 2.0 * N + a + b;
    d = (double(N) * ((a - b) - c * x) * pN + 2.0 * (N + a) * (N + b) * pN1) / (c * (1.0 - x * x));
  } else if (family == XC_LAGUERRE_FN) {
    d = double(N) * (pN - pN1) / x;
  } else {
    d = sqrt(2.0 * double(N)) * pN1 - x * pN;
  }
  return pN / d;
}

// p_N(x) / p_N'(x) for the monic polynomials of the Jacobi matrix (d, e2):
// p_{m+1} = (x - d_m) p_m - e2_{m-1} p_{m-1}, differentiated alongside; *f
// gets p_N up to a positive factor (both are rescaled by powers of two).
__device__ double monic_ratio(const double* d, const double* e2, int64_t N, double x, double* f) {
  double p0 = 0.0, p1 = 1.0, q0 = 0.0, q1 = 0.0;
  for (int64_t m = 0; m < N; ++m) {
    const double t = x - d[m];
    const double e = m > 0 ? e2[m - 1] : 0.0;
    const double p2 = t * p1 - e * p0;
    const double q2 = p1 + t * q1 - e * q0;
    p0 = p1; p1 = p2; q0 = q1; q1 = q2;
    const double big = fmax(fabs(p1), fabs(q1));
    if (big > 0x1p+500) {
      p0 *= 0x1p-500; p1 *= 0x1p-500; q0 *= 0x1p-500; q1 *= 0x1p-500;
    } else if (big < 0x1p-500 && big > 0.0) {
      p0 *= 0x1p+500; p1 *= 0x1p+500; q0 *= 0x1p+500; q1 *= 0x1p+500;
    }
  }
  *f = p1;
  return p1 / q1;
}

// The k-th smallest zero: bracket it between the grid points where the Sturm
// count passes k, bisect (Sturm counts) until the bracket holds this zero
// alone, then Newton on the recurrence, kept inside the bracket (a step that
// leaves it bisects instead; every iterate shrinks the bracket by the sign of
// phi_N).  Both loops are bounded.
__global__ void isolate_newton_kernel(const double* d, const double* e2, int64_t N, const double* grid,
                                      const int* counts, int64_t G, double* out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int64_t lo = 0, hi = G;  // counts[lo] <= k < counts[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (counts[mid] > k) hi = mid;
    else lo = mid;
  }
  double a = grid[lo], b = grid[hi];
  int ca = counts[lo], cb = counts[hi];
  for (int it = 0; it < 64 && !(ca == k && cb == k + 1); ++it) {
    const double mid = 0.5 * (a + b);
    if (mid <= a || mid >= b) break;
    const int cm = sturm_count(d, e2, N, mid);
    if (cm > k) { b = mid; cb = cm; }
    else { a = mid; ca = cm; }
  }
  double fa;
  monic_ratio(d, e2, N, a, &fa);
  const double tiny = 1e-6 * (b - a);  // absolute scale for a zero at x = 0
  double x = 0.5 * (a + b);
  bool clipped = false;
  for (int it = 0; it < 40; ++it) {
    double f;
    const double r = monic_ratio(d, e2, N, x, &f);
    if (f == 0.0) break;
    if (fabs(r) <= 1e-10 * fmax(fabs(x), tiny)) {  // quadratic: the error is now far below rounding
      x -= r;
      break;
    }
    if ((f < 0.0) == (fa < 0.0)) a = x;
    else b = x;
    double xn = x - r;
    if (!(xn > a && xn < b)) {
      // Overshoot: try the bracket end it passed (a zero right at an end
      // otherwise costs one bisection per bit), then bisect.
      const double end = xn <= a ? a : b;
      xn = (!clipped && x != end) ? end : 0.5 * (a + b);
      clipped = !clipped && xn == end;
    } else {
      clipped = false;
    }
    x = xn;
    if (b - a <= 4e-16 * fmax(fabs(a), fabs(b))) break;
  }
  out[k] = x;
}

// Zeros of the Jacobi polynomials with |alpha| = |beta| = 1/2 in closed form
// (Chebyshev polynomials of the four kinds), ascending.
__global__ void jacobi_half_nodes_kernel(int64_t N, double al, double be, double* x) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double j = double(N - k);  // theta_j descending in k
  double t;
  if (al < 0 && be < 0) t = (2.0 * j - 1.0) / (2.0 * double(N));         // first kind
  else if (al > 0 && be > 0) t = j / double(N + 1);                      // second kind
  else if (al > 0) t = 2.0 * j / (2.0 * double(N) + 1.0);                // fourth kind
  else t = (2.0 * j - 1.0) / (2.0 * double(N) + 1.0);                    // third kind
  x[k] = cospi(t);
}

// Final Newton step(s) on the family's own recurrence.
__global__ void newton_kernel(int family, int64_t N, double a, double b, int steps, double* x) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double v = x[k];
  for (int it = 0; it < steps; ++it) v -= newton_ratio(family, N, a, b, v);
  x[k] = v;
}

__global__ void cheb_nodes_kernel(int64_t N, double* x) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n < N) x[n] = cospi(double(2 * n + 1) / double(2 * N));
}

// Christoffel numbers times exp(x) / exp(x^2) for the Laguerre / Hermite
// functions (the discrete inner product of the functions themselves).
__global__ void weights_kernel(GenParams g, double* lam) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const double x = g.x[n];
  const int64_t N = g.N;
  if (g.family == XC_CHEBYSHEV_T) {
    lam[n] = 3.141592653589793 / double(N);
    return;
  }
  if (g.family == XC_LEGENDRE || g.family == XC_JACOBI) {
    const double a = g.family == XC_JACOBI ? g.alpha : 0.0, b = g.family == XC_JACOBI ? g.beta : 0.0;
    double pN, pN1;
    last_two(g.family, N, a, b, x, &pN, &pN1);
    const double c = 2.0 * N + a + b;
    const double d = (double(N) * ((a - b) - c * x) * pN + 2.0 * (N + a) * (N + b) * pN1) / (c * (1.0 - x * x));
    const double lg = lgamma(N + a + 1.0) + lgamma(N + b + 1.0) - lgamma(N + a + b + 1.0) - lgamma(N + 1.0) +
                      (a + b + 1.0) * 0.6931471805599453;
    lam[n] = exp(lg) / ((1.0 - x * x) * d * d);
    return;
  }
  // functions: the needed value phi_{N+1} (Laguerre) or phi_{N-1} (Hermite)
  const int64_t want = g.family == XC_LAGUERRE_FN ? N + 1 : N - 1;
  double v = 0.0;
  gen_values(g, n, want, want + 1, [&](int64_t, double val) { v = val; });
  lam[n] = g.family == XC_LAGUERRE_FN ? x / ((N + 1.0) * (N + 1.0) * v * v) : 1.0 / (double(N) * v * v);
}

// rowscale = sqrt(lambda_n); colscale = 1/sqrt(chi_m) for the polynomials
__global__ void scales_kernel(GenParams g, const double* lam, void* rowscale, void* colscale, int fp64) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const double rs = sqrt(lam[i]);
  double chi = 1.0;
  const double m = double(i);
  if (g.family == XC_CHEBYSHEV_T) {
    chi = i == 0 ? 3.141592653589793 : 1.5707963267948966;
  } else if (g.family == XC_LEGENDRE) {
    chi = 2.0 / (2.0 * m + 1.0);
  } else if (g.family == XC_JACOBI) {
    const double a = g.alpha, b = g.beta;
    double lg;
    if (i == 0)
      lg = (a + b + 1.0) * 0.6931471805599453 + lgamma(a + 1.0) + lgamma(b + 1.0) - lgamma(a + b + 2.0);
    else
      lg = (a + b + 1.0) * 0.6931471805599453 - log(2.0 * m + a + b + 1.0) + lgamma(m + a + 1.0) +
           lgamma(m + b + 1.0) - lgamma(m + a + b + 1.0) - lgamma(m + 1.0);
    chi = exp(lg);
  }
  const double cs = 1.0 / sqrt(chi);
  if (fp64) {
    static_cast<double*>(rowscale)[i] = rs;
    static_cast<double*>(colscale)[i] = cs;
  } else {
    static_cast<float*>(rowscale)[i] = float(rs);
    static_cast<float*>(colscale)[i] = float(cs);
  }
}

// -------------------------------------------------- window, twiddles, tables
__device__ double bessel_i0_dev(double z) {
  const double q = 0.25 * z * z;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 4000; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

// w_j^{zeta, L-1} (FP64) and 1/w_j in the plan precision.
template <typename T>
__global__ void window_kernel(int64_t L, double zeta, double* w, T* invw) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= L) return;
  const double t = 2.0 * double(j) / double(L - 1) - 1.0;
  const double a = sqrt(fmax(0.0, 1.0 - t * t));
  const double v = bessel_i0_dev(zeta * a) / bessel_i0_dev(zeta);
  w[j] = v;
  invw[j] = T(1.0 / v);
}

// exp(-2 pi i k / L), k < L, reduced to the first octant for accuracy.
template <typename T>
__global__ void twiddle_kernel(int64_t L, cx<T>* tw) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= L) return;
  double s, c;
  sincospi(2.0 * double(k) / double(L), &s, &c);
  tw[k] = cx<T>{T(c), T(-s)};
}

// ------------------------------------------------------------ row spectra
// G[j * C + c] = phi_{j - off}(x_{row0 + c}) * w_j for j < L (column-major
// chunk of C rows).
__global__ void gen_rows_kernel(GenParams g, int64_t row0, int64_t C, int64_t L, int64_t off,
                                const double* w, double* G) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= C || row0 + c >= g.N) return;
  gen_values(g, row0 + c, -off, L - off, [&](int64_t m, double v) {
    const int64_t j = m + off;
    G[j * C + c] = v * w[j];
  });
}

// One CTA per row of the chunk: real FFT of length L = 2n of the windowed row,
// S[row][k] = U_k / L for k = 0..n, and the block maximum of |S|^2 (times
// rw[row] where row weights are given).
__global__ void __launch_bounds__(256) row_fft_kernel(const double* G, int64_t C, int64_t row0, int64_t N,
                                                      BlockDev b, const cx<double>* tw, cx<double>* S,
                                                      unsigned long long* maxsq_bits, const double* rw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<double>* s = reinterpret_cast<cx<double>*>(smem_raw);
  __shared__ double red[8];
  const int64_t c = blockIdx.x;
  const int64_t row = row0 + c;
  if (row >= N) return;
  const int n = b.n;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    s[b.perm[j]] = cx<double>{G[int64_t(2 * j) * C + c], G[int64_t(2 * j + 1) * C + c]};
  __syncthreads();
  fft_inplace<double>(s, n, b.p, b.radix, tw, threadIdx.x, blockDim.x);
  const double scale = 1.0 / double(b.L);
  const double wt = rw ? rw[row] : 1.0;
  cx<double>* out = S + row * int64_t(n + 1);
  double local = 0.0;
  for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
    cx<double> Uk, Unk;
    r2c_split(s, n, k, tw, &Uk, &Unk);
    Uk = scal(scale, Uk);
    Unk = scal(scale, Unk);
    out[k] = Uk;
    out[n - k] = Unk;
    local = fmax(local, wt * fmax(Uk.re * Uk.re + Uk.im * Uk.im, Unk.re * Unk.re + Unk.im * Unk.im));
  }
  for (int o = 16; o > 0; o >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
    // non-negative doubles order like their bit patterns
    atomicMax(maxsq_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

// The same row transform for lengths whose FP64 array exceeds one CTA's shared
// memory: a cluster of `csize` CTAs per row holds the n-point array split in
// equal parts (rank r owns [r*per, (r+1)*per)); butterflies reach the other
// parts through distributed shared memory, and a cluster barrier separates the
// passes.  Launched with cluster dimension (csize, 1, 1), grid = rows * csize.
__global__ void __launch_bounds__(256) row_fft_cluster_kernel(const double* G, int64_t C, int64_t row0, int64_t N,
                                                              BlockDev b, const cx<double>* tw, cx<double>* S,
                                                              unsigned long long* maxsq_bits, int csize,
                                                              const double* rw) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<double>* s = reinterpret_cast<cx<double>*>(smem_raw);
  __shared__ double red[8];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int64_t c = blockIdx.x / csize;
  const int64_t row = row0 + c;
  const int n = b.n;
  ClusterMem<double> mem;
  mem.per = n / csize;
  for (int r = 0; r < 8; ++r) mem.base[r] = r < csize ? cluster.map_shared_rank(s, r) : s;
  const int tid = rank * int(blockDim.x) + int(threadIdx.x);
  const int nthreads = csize * int(blockDim.x);
  const bool live = row < N;            // the whole cluster shares one row: uniform
  cluster.sync();                       // every CTA of the cluster runs before any remote access
  if (live)
    for (int j = tid; j < n; j += nthreads)
      mem.at(b.perm[j]) = cx<double>{G[int64_t(2 * j) * C + c], G[int64_t(2 * j + 1) * C + c]};
  cluster.sync();
  fft_run<double>(mem, n, b.p, b.radix, tw, tid, nthreads, [&] { cluster.sync(); });
  const double scale = 1.0 / double(b.L);
  double local = 0.0;
  if (live) {
    const double wt = rw ? rw[row] : 1.0;
    cx<double>* out = S + row * int64_t(n + 1);
    for (int k = tid; k <= n / 2; k += nthreads) {
      cx<double> Uk, Unk;
      r2c_split_vals(mem.at(k), mem.at(k == 0 ? 0 : n - k), k, tw, &Uk, &Unk);
      Uk = scal(scale, Uk);
      Unk = scal(scale, Unk);
      out[k] = Uk;
      out[n - k] = Unk;
      local = fmax(local, wt * fmax(Uk.re * Uk.re + Uk.im * Uk.im, Unk.re * Unk.re + Unk.im * Unk.im));
    }
  }
  for (int o = 16; o > 0; o >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0 && live) {
    double m = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
    atomicMax(maxsq_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------- Appendix A (Chebyshev rows)
// sin(pi a / d) and cos(pi a / d) for integers a and d > 0: a is reduced
// exactly modulo 2d and reflected into [-d/2, d/2] (sin(pi - x) = sin x,
// cos(pi - x) = -cos x) first, so the only rounding is in the final quotient
// and sincospi, and the sine keeps its relative accuracy next to every zero.
__device__ __forceinline__ void sincospi_ratio(int64_t a, int64_t d, double* s, double* c) {
  int64_t r = a % (2 * d);
  if (r < 0) r += 2 * d;
  if (r >= d) r -= 2 * d;
  double sign_c = 1.0;
  if (2 * r > d) {
    r = d - r;
    sign_c = -1.0;
  } else if (2 * r < -d) {
    r = -d - r;
    sign_c = -1.0;
  }
  sincospi(double(r) / double(d), s, c);
  *c *= sign_c;
}

// xw[m + M] = sum_{j<L} w_j exp(-2 pi i j m / L) for |m| <= M: the few DFT
// components of the Kaiser window that carry it (one CTA per m).
__global__ void __launch_bounds__(256) window_dft_kernel(const double* w, int64_t L, int M, cx<double>* xw) {
  __shared__ double red[2][8];
  const int64_t m = int64_t(blockIdx.x) - M;
  double re = 0.0, im = 0.0;
  for (int64_t j = threadIdx.x; j < L; j += blockDim.x) {
    double sn, cs;
    sincospi_ratio(2 * ((j * m) % L), L, &sn, &cs);
    re += w[j] * cs;
    im -= w[j] * sn;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = re;
    red[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    xw[blockIdx.x] = cx<double>{a, b};
  }
}

constexpr int kCfMaxM = 32;   // window components |m| <= M
constexpr int kCfMaxB = 64;   // bins |k - k_c| <= B computed per row

// The candidate bins of row `row` of a Chebyshev block: within B of the
// row's peak k_c = round(theta L / (2 pi)), clipped to [0, n].
__host__ __device__ __forceinline__ void cf_window(int64_t row, int64_t N, int64_t L, int n, int B, int64_t* klo,
                                                   int64_t* khi) {
  const int64_t t = (2 * row + 1) * L;   // theta L / (2 pi) = t / (4N)
  const int64_t kc = (t + 2 * N) / (4 * N);
  *klo = kc - B < 0 ? 0 : kc - B;
  *khi = kc + B > n ? int64_t(n) : kc + B;
}

// Appendix A: S[row][k] = U_k / L for the extended Chebyshev row
// a_j = cos((j - off) theta), theta = (2 row + 1) pi / (2N), j < L, where
// U = DFT(a . w).  By the convolution theorem (eq. (conv_appendix)),
// U_k = L^{-1} sum_m xw_m Ahat_{k-m} with Ahat the row's own DFT, which has a
// closed form (eqs. (y1), (y3)): writing cos as two exponentials,
//   Ahat_q = e^{-i pi q (L-1)/L} [e^{i theta c} D_+ + e^{-i theta c} D_-] / 2,
//   c = (L - 1 - 2 off) / 2,  D_+- = (-1)^q sin(L theta/2) / sin(theta/2 -+ pi q/L),
// and D_+- = L (-1)^{p (L-1)} where the sine below vanishes (theta/2 -+ pi q/L = pi p).
// Only |m| <= M enter (the window's spectrum is concentrated there) and only
// the candidate bins are computed; S is zero elsewhere.  One CTA per row.
__global__ void __launch_bounds__(128) cheb_rows_closed_kernel(int64_t N, int64_t L, int64_t off, int n, int M,
                                                               int B, const cx<double>* xw, cx<double>* S,
                                                               unsigned long long* maxsq_bits, const double* rw) {
  __shared__ cx<double> ah[2 * kCfMaxB + 2 * kCfMaxM + 1];
  __shared__ cx<double> xs[2 * kCfMaxM + 1];
  __shared__ double red[4];
  const int64_t row = blockIdx.x;
  int64_t klo, khi;
  cf_window(row, N, L, n, B, &klo, &khi);
  const int64_t q0 = klo - M;
  const int Q = int(khi - klo) + 2 * M + 1;
  for (int i = threadIdx.x; i <= 2 * M; i += blockDim.x) xs[i] = xw[i];
  const int64_t t = (2 * row + 1) * L;
  double sin_lt, cos_lt;
  sincospi_ratio(t, 4 * N, &sin_lt, &cos_lt);            // L theta / 2 = pi t / (4N)
  double sc, cc;
  sincospi_ratio((2 * row + 1) * (L - 1 - 2 * off), 4 * N, &sc, &cc);   // theta c
  const int64_t P = 4 * N * L;                           // theta/2 -+ pi q/L = pi (t -+ 4Nq) / P
  for (int i = threadIdx.x; i < Q; i += blockDim.x) {
    const int64_t q = q0 + i;
    const double sg = (q & 1) ? -1.0 : 1.0;
    double d[2];
    for (int h = 0; h < 2; ++h) {
      const int64_t a = h == 0 ? t - 4 * N * q : t + 4 * N * q;
      if (a % P == 0) {
        const int64_t p = a / P;
        d[h] = ((p & 1) && ((L - 1) & 1)) ? -double(L) : double(L);
      } else {
        double sn, cs;
        sincospi_ratio(a, P, &sn, &cs);
        d[h] = sg * sin_lt / sn;
      }
    }
    double sq, cq;
    sincospi_ratio(-(q * (L - 1)), L, &sq, &cq);
    // e^{i theta c} D_+ + e^{-i theta c} D_-
    const cx<double> v{0.5 * cc * (d[0] + d[1]), 0.5 * sc * (d[0] - d[1])};
    ah[i] = cx<double>{cq * v.re - sq * v.im, cq * v.im + sq * v.re};
  }
  __syncthreads();
  const double scale = 1.0 / (double(L) * double(L));
  const double wt = rw ? rw[row] : 1.0;
  double local = 0.0;
  for (int64_t k = klo + threadIdx.x; k <= khi; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int i = 0; i <= 2 * M; ++i) {
      const cx<double> a = xs[i], b = ah[k - (i - M) - q0];
      re += a.re * b.re - a.im * b.im;
      im += a.re * b.im + a.im * b.re;
    }
    re *= scale;
    im *= scale;
    S[row * int64_t(n + 1) + k] = cx<double>{re, im};
    local = fmax(local, wt * (re * re + im * im));
  }
  for (int o = 16; o > 0; o >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
    atomicMax(maxsq_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

// The real blocks' threshold test: |v|^2, times the row weight where there
// are weights, above thr.
__device__ __forceinline__ bool kept_row(cx<double> v, double thr, const double* rw, int64_t row) {
  const double m = v.re * v.re + v.im * v.im;
  return (rw ? rw[row] * m : m) > thr;
}

// One warp per row: first/last kept bin and the number of kept bins.
__global__ void extents_kernel(const cx<double>* S, int64_t N, int64_t H, double thr, int* kfirst, int* klast,
                               int* count, const double* rw) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  int lo = INT_MAX, hi = -1, cnt = 0;
  for (int64_t k = lane; k < H; k += 32) {
    if (kept_row(S[row * H + k], thr, rw, row)) {
      lo = min(lo, int(k));
      hi = max(hi, int(k));
      ++cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if (lane == 0) {
    kfirst[row] = hi >= 0 ? lo : 0;
    klast[row] = hi;
    count[row] = cnt;
  }
}

// A stored band value in the plan's format: cx<T>, or (pair, T = double) the
// FP32 pair split of each part in the same 16 bytes.
template <typename T>
__device__ __forceinline__ void store_value(cx<T>* dst, cx<double> v, int pair) {
  if constexpr (sizeof(T) == 8) {
    if (pair) {
      *reinterpret_cast<PairCx*>(dst) = to_pair(v.re, v.im);
      return;
    }
  }
  *dst = cx<T>{T(v.re), T(v.im)};
}

// Forward band values: slice s, position j, lane -> row 32 s + lane, bin
// k0[row] + j; kept elements times g_k (2 inside the half spectrum, 1 at k = 0
// and k = n), everything else zero.
template <typename T>
__global__ void fill_forward_kernel(const cx<double>* S, int64_t N, int n, double thr, const int* k0,
                                    const int* width, const int64_t* off, int nslices, cx<T>* val, int pair,
                                    const double* rw) {
  const int s = blockIdx.y;
  if (s >= nslices) return;
  const int W = width[s];
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;   // j * 32 + lane
  if (idx >= int64_t(W) * 32) return;
  const int lane = int(idx & 31);
  const int j = int(idx >> 5);
  const int64_t row = int64_t(s) * 32 + lane;
  cx<double> v{0.0, 0.0};
  if (row < N) {
    const int k = k0[row] + j;
    const cx<double> a = S[row * int64_t(n + 1) + k];
    if (kept_row(a, thr, rw, row)) v = scal((k == 0 || k == n) ? 1.0 : 2.0, a);
  }
  store_value(val + off[s] + idx, v, pair);
}

// Transposed band values: slice s of bins, lane -> bin 32 s + lane, row n0[bin] + j.
template <typename T>
__global__ void fill_adjoint_kernel(const cx<double>* S, int64_t N, int n, double thr, const int* n0,
                                    const int* width, const int64_t* off, int tslices, cx<T>* val, int pair,
                                    const double* rw) {
  const int s = blockIdx.y;
  if (s >= tslices) return;
  const int W = width[s];
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(W) * 32) return;
  const int lane = int(idx & 31);
  const int j = int(idx >> 5);
  const int64_t k = int64_t(s) * 32 + lane;
  cx<double> v{0.0, 0.0};
  if (k <= n) {
    const int64_t row = n0[k] + j;
    const cx<double> a = S[row * int64_t(n + 1) + k];
    if (kept_row(a, thr, rw, row)) v = a;
  }
  store_value(val + off[s] + idx, v, pair);
}

// ---------------------------------------------------- complex families
// Full spectrum of the complex row exp(i (j - off) theta) w_j from the half
// spectra of its real part (Sc) and imaginary part (Ss), each the DFT of a
// real row and so Hermitian: S_k = Sc_k + i Ss_k with Sc_{L-k} = conj(Sc_k).
__device__ __forceinline__ cx<double> full_bin(const cx<double>* __restrict__ Sc, const cx<double>* __restrict__ Ss,
                                               int64_t row, int n, int k) {
  const int64_t H = n + 1;
  cx<double> a, b;
  if (k <= n) {
    a = Sc[row * H + k];
    b = Ss[row * H + k];
  } else {
    a = conj(Sc[row * H + (2 * n - k)]);
    b = conj(Ss[row * H + (2 * n - k)]);
  }
  return cx<double>{a.re - b.im, a.im + b.re};
}

__device__ __forceinline__ double sq(cx<double> v) { return v.re * v.re + v.im * v.im; }

// max |S|^2 over the block (non-negative doubles order like their bits)
__global__ void c_max_kernel(const cx<double>* Sc, const cx<double>* Ss, int64_t N, int n,
                             unsigned long long* maxsq_bits) {
  const int64_t L = 2 * int64_t(n);
  double local = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N * L; i += int64_t(gridDim.x) * blockDim.x)
    local = fmax(local, sq(full_bin(Sc, Ss, i / L, n, int(i % L))));
  for (int o = 16; o > 0; o >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxsq_bits, static_cast<unsigned long long>(__double_as_longlong(local)));
}

// Smallest circular interval [start, start + width) of 0..len-1 around the
// reference `ref` that holds every index whose offset from ref lies in
// [dmin, dmax] (offsets taken in [-len/2, len/2)).
__device__ __forceinline__ int circ_offset(int64_t i, int64_t ref, int64_t len) {
  int64_t d = (i - ref) % len;
  if (d < 0) d += len;
  if (d >= (len + 1) / 2) d -= len;
  return int(d);
}

// One warp per row: the row's peak bin, then the circular band of its kept
// bins around the peak (start k0 in [0, L), width), and the kept count.
__global__ void c_extents_kernel(const cx<double>* Sc, const cx<double>* Ss, int64_t N, int n, double thr,
                                 int* k0, int* width, int* count) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  const int L = 2 * n;
  double best = -1.0;
  int bk = 0;
  for (int k = lane; k < L; k += 32) {
    const double m = sq(full_bin(Sc, Ss, row, n, k));
    if (m > best) { best = m; bk = k; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
    if (ob > best || (ob == best && ok < bk)) { best = ob; bk = ok; }
  }
  int dmin = INT_MAX, dmax = INT_MIN, cnt = 0;
  for (int k = lane; k < L; k += 32) {
    if (sq(full_bin(Sc, Ss, row, n, k)) > thr) {
      const int d = circ_offset(k, bk, L);
      dmin = min(dmin, d);
      dmax = max(dmax, d);
      ++cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if (lane == 0) {
    k0[row] = cnt > 0 ? int(((bk + dmin) % L + L) % L) : 0;
    width[row] = cnt > 0 ? dmax - dmin + 1 : 0;
    count[row] = cnt;
  }
}

// One thread per bin (consecutive bins in a warp read consecutive values):
// the bin's peak row, then the circular run of rows around it that holds its
// kept elements (start n0 in [0, N), width).
__global__ void c_col_extents_kernel(const cx<double>* Sc, const cx<double>* Ss, int64_t N, int n, double thr,
                                     int* n0, int* width) {
  const int k = int(int64_t(blockIdx.x) * blockDim.x + threadIdx.x);
  if (k >= 2 * n) return;
  double best = -1.0;
  int64_t br = 0;
  for (int64_t r = 0; r < N; ++r) {
    const double m = sq(full_bin(Sc, Ss, r, n, k));
    if (m > best) { best = m; br = r; }
  }
  int dmin = INT_MAX, dmax = INT_MIN;
  for (int64_t r = 0; r < N; ++r) {
    if (sq(full_bin(Sc, Ss, r, n, k)) > thr) {
      const int d = circ_offset(r, br, N);
      dmin = min(dmin, d);
      dmax = max(dmax, d);
    }
  }
  const bool any = dmax >= dmin;
  n0[k] = any ? int(((br + dmin) % N + N) % N) : 0;
  width[k] = any ? dmax - dmin + 1 : 0;
}

// Band values of the complex block, forward layout: slice s, band position j,
// lane -> row 32 s + lane, bin (k0 + j) mod L; zero outside the row's band or
// where the element is dropped.
template <typename T>
__global__ void c_fill_forward_kernel(const cx<double>* Sc, const cx<double>* Ss, int64_t N, int n, double thr,
                                      const int* k0, const int* rwidth, const int* width, const int64_t* off,
                                      int nslices, cx<T>* val) {
  const int s = blockIdx.y;
  if (s >= nslices) return;
  const int W = width[s];
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;   // j * 32 + lane
  if (idx >= int64_t(W) * 32) return;
  const int lane = int(idx & 31);
  const int j = int(idx >> 5);
  const int64_t row = int64_t(s) * 32 + lane;
  cx<double> v{0.0, 0.0};
  if (row < N && j < rwidth[row]) {
    const int L = 2 * n;
    const int k = (k0[row] + j) % L;
    const cx<double> a = full_bin(Sc, Ss, row, n, k);
    if (sq(a) > thr) v = a;
  }
  val[off[s] + idx] = cx<T>{T(v.re), T(v.im)};
}

// Transposed band values: slice s of bins, lane -> bin 32 s + lane, row
// (n0 + i) mod N.
template <typename T>
__global__ void c_fill_adjoint_kernel(const cx<double>* Sc, const cx<double>* Ss, int64_t N, int n, double thr,
                                      const int* n0, const int* bwidth, const int* width, const int64_t* off,
                                      int tslices, cx<T>* val) {
  const int s = blockIdx.y;
  if (s >= tslices) return;
  const int W = width[s];
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;   // i * 32 + lane
  if (idx >= int64_t(W) * 32) return;
  const int lane = int(idx & 31);
  const int i = int(idx >> 5);
  const int k = s * 32 + lane;
  cx<double> v{0.0, 0.0};
  if (k < 2 * n && i < bwidth[k]) {
    const int64_t row = (int64_t(n0[k]) + i) % N;
    const cx<double> a = full_bin(Sc, Ss, row, n, k);
    if (sq(a) > thr) v = a;
  }
  val[off[s] + idx] = cx<T>{T(v.re), T(v.im)};
}

// The plain complex matrix (comparison path): one thread per element, the
// row factor of the spectral Laguerre matrix included.
template <typename T>
__global__ void c_dense_kernel(GenParams g, const cx<T>* rowscale, cx<T>* A, int64_t lda) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = blockIdx.y;
  if (m >= g.N || n >= g.N) return;
  double re = 0.0, im = 0.0;
  GenParams gc = g;
  gc.cpart = 0;
  gen_values(gc, n, m, m + 1, [&](int64_t, double v) { re = v; });
  gc.cpart = 1;
  gen_values(gc, n, m, m + 1, [&](int64_t, double v) { im = v; });
  cx<T> a{T(re), T(im)};
  if (rowscale) a = cmul(rowscale[n], a);
  A[n * lda + m] = a;
}

// ------------------------------------------------------- 2-D block scheme
// Lambda(z) = Gamma(z + 1/2) / Gamma(z + 1) from a table (built on the host by
// the recurrence Lambda(z) = Lambda(z - 1) (2z - 1) / (2z) in long double).
__device__ __forceinline__ double kernel_a1(int64_t i, int64_t j, const double* lam) {
  if (i > j) return 0.0;
  if (i == 0) return lam[j] * 0.3183098861837907;          // 1/pi
  return 0.6366197723675814 * lam[j - i] * lam[j + i];      // 2/pi
}

__device__ __forceinline__ double kernel_a2(int64_t i, int64_t j) {
  if (i == j) return 0.0;
  auto g = [](int64_t k) { return k > 0 ? double(k) * cos(2.0 * log(double(k))) : 0.0; };
  const double d = double(i - j);
  return (g(i) - g(j)) / (d * d);
}

// W_r D_e W_c of a 2-D block, column-major for the row FFT: G[j * C + i] =
// D(r0 + i, c0 + j) wr[i] wc[j], i < Lr (= C), j < Lc.  Functions at nodes:
// one thread per row i (recurrence over the degrees; g.x holds the block's
// row nodes); index kernels: one thread per element.
__global__ void gen2d_rows_kernel(GenParams g, int64_t Lr, int64_t c0, int64_t Lc, const double* wr,
                                  const double* wc, double* G) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Lr) return;
  const double a = wr[i];
  gen_values(g, i, c0, c0 + Lc, [&](int64_t m, double v) { G[(m - c0) * Lr + i] = v * a * wc[m - c0]; });
}

__global__ void gen2d_kernel_elems(int kind, int64_t r0, int64_t Lr, int64_t c0, int64_t Lc, const double* wr,
                                   const double* wc, const double* lam, double* G) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= Lr || j >= Lc) return;
  const double v = kind == XC_KERNEL_A1 ? kernel_a1(r0 + i, c0 + j, lam) : kernel_a2(r0 + i, c0 + j);
  G[j * Lr + i] = v * wr[i] * wc[j];
}

// S[i][q] (Lr x Hc complex) -> the real and imaginary parts as rows q of
// length Lr for the second row FFT: Re[i * Hc + q], Im[i * Hc + q].
__global__ void split2d_kernel(const cx<double>* S, int64_t Lr, int64_t Hc, double* Re, double* Im) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= Lr * Hc) return;
  Re[e] = S[e].re;
  Im[e] = S[e].im;
}

// Entries of a rectangle [r0, r1) x [c0, c1), row i at out + i * ldo, in the
// plan precision (g.x holds the rectangle's row nodes).
template <typename T>
__global__ void rect2d_kernel(GenParams g, int kind, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                              const double* lam, T* out, int64_t ldo) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= r1 - r0) return;
  const int64_t w = c1 - c0;
  if (kind == XC_KERNEL_A1 || kind == XC_KERNEL_A2) {
    for (int64_t j = 0; j < w; ++j)
      out[i * ldo + j] = T(kind == XC_KERNEL_A1 ? kernel_a1(r0 + i, c0 + j, lam) : kernel_a2(r0 + i, c0 + j));
  } else {
    gen_values(g, i, c0, c1, [&](int64_t m, double v) { out[i * ldo + (m - c0)] = T(v); });
  }
}

// Dense tail [m][N] and the plain matrix (comparison path).
template <typename T>
__global__ void tail_kernel(GenParams g, int64_t m_tail, T* tail) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  gen_values(g, n, 0, m_tail, [&](int64_t m, double v) { tail[m * g.N + n] = T(v); });
}

// 32 rows per CTA (one warp); each lane walks its row's recurrence once and
// the values are staged through shared memory 32 columns at a time so that
// every row of A is written contiguously.  Lanes past the last row evaluate
// row N-1 without writing, keeping the warp in lockstep.
template <typename T>
__global__ void dense_kernel(GenParams g, const T* rowscale, const T* colscale, T* A, int64_t lda) {
  __shared__ T tile[32][33];
  const int64_t n0 = int64_t(blockIdx.x) * 32;
  const int lane = threadIdx.x;
  const int64_t N = g.N;
  const int64_t n = n0 + lane < N ? n0 + lane : N - 1;
  gen_values(g, n, 0, N, [&](int64_t m, double v) {
    tile[lane][m & 31] = T(v);
    if ((m & 31) == 31 || m == N - 1) {
      __syncwarp();
      const int64_t mb = m & ~int64_t(31);
      for (int r = 0; r < 32; ++r) {
        const int64_t row = n0 + r;
        const int64_t col = mb + lane;
        if (row < N && col <= m) {
          T val = tile[r][lane];
          if (rowscale) val = val * rowscale[row] * colscale[col];
          A[row * lda + col] = val;
        }
      }
      __syncwarp();
    }
  });
}

}  // namespace

// The plain N x N matrix with the plan's normalisation (comparison path).
int dense_matrix_device(const Plan* p, void* A, int64_t lda, cudaStream_t s) {
  GenParams g{p->family, p->N, p->params.alpha, p->params.beta, p->nodes_dev,
              is_trig(p->family) && p->family != XC_LAGUERRE_SPECTRAL && p->params.nodes == XC_NODES_GAUSS,
              p->params.power, p->rc_dev, p->nrc};
  if (p->d2) {
    // the whole index square as one rectangle
    g.x = p->nodes_dev;
    const unsigned gr = unsigned((p->N + 31) / 32);
    if (p->io64())
      rect2d_kernel<double><<<gr, 32, 0, s>>>(g, p->family, 0, p->N, 0, p->N, p->d2->lam, static_cast<double*>(A), lda);
    else
      rect2d_kernel<float><<<gr, 32, 0, s>>>(g, p->family, 0, p->N, 0, p->N, p->d2->lam, static_cast<float*>(A), lda);
    XC_CUDA(cudaGetLastError());
    return XC_OK;
  }
  if (p->cplx) {
    const dim3 grid(unsigned((p->N + 127) / 128), unsigned(p->N));
    if (p->io64())
      c_dense_kernel<double><<<grid, 128, 0, s>>>(g, static_cast<const cx<double>*>(p->rowscale),
                                                   static_cast<cx<double>*>(A), lda);
    else
      c_dense_kernel<float><<<grid, 128, 0, s>>>(g, static_cast<const cx<float>*>(p->rowscale),
                                                  static_cast<cx<float>*>(A), lda);
    XC_CUDA(cudaGetLastError());
    return XC_OK;
  }
  const unsigned grid = unsigned((p->N + 31) / 32);
  if (p->io64())
    dense_kernel<double><<<grid, 32, 0, s>>>(g, static_cast<const double*>(p->rowscale),
                                              static_cast<const double*>(p->colscale), static_cast<double*>(A), lda);
  else
    dense_kernel<float><<<grid, 32, 0, s>>>(g, static_cast<const float*>(p->rowscale),
                                             static_cast<const float*>(p->colscale), static_cast<float*>(A), lda);
  XC_CUDA(cudaGetLastError());
  return XC_OK;
}

namespace {

// Host helpers ----------------------------------------------------------------

// Jacobi matrix of the family's monic recurrence (Golub-Welsch) for the Sturm
// bisection; e2 holds the squared off-diagonals.
void jacobi_matrix(int family, int64_t N, double a, double b, std::vector<double>* d, std::vector<double>* e2) {
  d->assign(N, 0.0);
  e2->assign(N > 1 ? N - 1 : 1, 0.0);
  for (int64_t k = 0; k < N; ++k) {
    const double kk = double(k);
    if (family == XC_LEGENDRE) {
      (*d)[k] = 0.0;
      if (k >= 1) (*e2)[k - 1] = kk * kk / (4.0 * kk * kk - 1.0);
    } else if (family == XC_JACOBI) {
      const double c = 2.0 * kk + a + b;
      (*d)[k] = k == 0 ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (c * (c + 2.0));
      if (k == 1)  // the factor 1 + a + b cancelled (0/0 when a + b = -1)
        (*e2)[0] = 4.0 * (1.0 + a) * (1.0 + b) / ((2.0 + a + b) * (2.0 + a + b) * (3.0 + a + b));
      else if (k > 1)
        (*e2)[k - 1] = 4.0 * kk * (kk + a) * (kk + b) * (kk + a + b) / (c * c * (c + 1.0) * (c - 1.0));
    } else if (family == XC_LAGUERRE_FN) {
      (*d)[k] = 2.0 * kk + 1.0;
      if (k >= 1) (*e2)[k - 1] = kk * kk;
    } else {
      (*d)[k] = 0.0;
      if (k >= 1) (*e2)[k - 1] = kk / 2.0;
    }
  }
}

// Coefficients (alpha_m, beta_m, gamma_m) of phi_{m+1} = (alpha_m + beta_m x)
// phi_m - gamma_m phi_{m-1}, m = 1..M-1, of the one-sided families: the
// three-term recurrences of the Jacobi polynomials, the Laguerre polynomials
// and the normalised Hermite functions with their divisions done once.
std::vector<double> recurrence_table(int family, double a, double b, int64_t M) {
  std::vector<double> t(size_t(3 * M), 0.0);
  for (int64_t m = 1; m < M; ++m) {
    const double mm = double(m);
    double al, be, ga;
    if (family == XC_LEGENDRE || family == XC_JACOBI) {
      const double c = 2.0 * mm + a + b;
      const double a1 = 2.0 * (mm + 1) * (mm + a + b + 1) * c;
      al = (c + 1) * (a * a - b * b) / a1;
      be = c * (c + 1) * (c + 2) / a1;
      ga = 2.0 * (mm + a) * (mm + b) * (c + 2) / a1;
    } else if (family == XC_LAGUERRE_FN) {
      al = (2.0 * mm + 1.0) / (mm + 1.0);
      be = -1.0 / (mm + 1.0);
      ga = mm / (mm + 1.0);
    } else {
      al = 0.0;
      be = std::sqrt(2.0 / (mm + 1.0));
      ga = std::sqrt(mm / (mm + 1.0));
    }
    t[size_t(3 * m)] = al;
    t[size_t(3 * m + 1)] = be;
    t[size_t(3 * m + 2)] = ga;
  }
  return t;
}

// Digit-reversed position of each input index (see xc_fft.cuh).
std::vector<int> digit_reversal(int n, int p, const int* radix) {
  std::vector<int> perm(n);
  for (int j = 0; j < n; ++j) {
    int rem = j, pos = 0, mult = 1;
    // j = t_p + r_p (t_{p-1} + r_{p-1} (...)); position = t_1 + r_1 (t_2 + ...)
    std::vector<int> t(p);
    for (int q = p - 1; q >= 0; --q) {
      t[q] = rem % radix[q];
      rem /= radix[q];
    }
    for (int q = 0; q < p; ++q) {
      pos += t[q] * mult;
      mult *= radix[q];
    }
    perm[j] = pos;
  }
  return perm;
}

template <typename T>
int upload(Plan* p, const std::vector<T>& v, T** out) {
  void* d = nullptr;
  XC_TRY(plan_alloc(p, &d, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty()) XC_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = static_cast<T*>(d);
  return XC_OK;
}

struct DevBuf {  // scratch freed at scope exit
  void* ptr = nullptr;
  ~DevBuf() {
    if (ptr) cudaFree(ptr);
  }
};

int alloc_tmp(DevBuf* b, size_t bytes) {
  if (cudaMalloc(&b->ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    b->ptr = nullptr;
    return fail(XC_ERR_ALLOC, "temporary device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  return XC_OK;
}

int set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) XC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return XC_OK;
}

template <typename T>
int build_block(Plan* p, int bi, const GenParams& g, const BlockShape& shp) {
  BlockDev& b = p->blocks[bi];
  std::memset(&b, 0, sizeof(b));
  const int64_t N = p->N;
  b.L = int(shp.L);
  b.n = int(shp.L / 2);
  b.H = b.n + 1;
  b.off = int(shp.off);
  b.j_lo = int(shp.j_lo);
  b.j_hi = int(shp.j_hi);
  b.p = fft_radices(b.n, b.radix);
  if (b.p < 0) return fail(XC_ERR_UNSUPPORTED, "FFT length not 2^a 3^b 5^c 7^d");
  const int n = b.n, H = b.H;
  const size_t smem = size_t(n) * sizeof(cx<double>);
  int dev = 0, optin = 0;
  XC_CUDA(cudaGetDevice(&dev));
  XC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // single CTA when the FP64 array fits its shared memory, else a cluster
  int csize = 1;
  if (smem + 1024 > size_t(optin)) {
    csize = 0;
    for (int cand = 2; cand <= 8; ++cand)
      if (n % cand == 0 && size_t(n / cand) * sizeof(cx<double>) + 1024 <= size_t(optin)) {
        csize = cand;
        break;
      }
    if (csize == 0)
      return fail(XC_ERR_UNSUPPORTED, "block length L = " + std::to_string(b.L) +
                                          " exceeds an 8-CTA cluster FFT of the precompute");
  }
  // the apply FFT runs in one CTA in the plan precision, or for long blocks
  // on a cluster of up to 8 CTAs that split the array (distributed shared
  // memory)
  b.a_csize = 0;
  for (int cand = 1; cand <= 8 && b.a_csize == 0; ++cand)
    if (n % cand == 0 && size_t(n / cand) * sizeof(cx<T>) + 1024 <= size_t(optin)) b.a_csize = cand;
  if (b.a_csize == 0)
    return fail(XC_ERR_UNSUPPORTED, "block length L = " + std::to_string(b.L) +
                                        " exceeds an 8-CTA cluster FFT of the apply in this precision");

  // permutation, window, twiddles
  std::vector<int> perm = digit_reversal(n, b.p, b.radix);
  int* perm_d = nullptr;
  XC_TRY(upload(p, perm, &perm_d));
  b.perm = perm_d;
  DevBuf w64;
  XC_TRY(alloc_tmp(&w64, size_t(b.L) * sizeof(double)));
  void *invw = nullptr, *tw = nullptr;
  XC_TRY(plan_alloc(p, &invw, size_t(b.L) * sizeof(T)));
  XC_TRY(plan_alloc(p, &tw, size_t(b.L) * sizeof(cx<T>)));
  const unsigned gL = unsigned((b.L + 255) / 256);
  window_kernel<T><<<gL, 256>>>(b.L, p->zeta, static_cast<double*>(w64.ptr), static_cast<T*>(invw));
  twiddle_kernel<T><<<gL, 256>>>(b.L, static_cast<cx<T>*>(tw));
  XC_CUDA(cudaGetLastError());
  b.invw = invw;
  b.tw = tw;
  // FP64 twiddles for the precompute FFT
  DevBuf tw64;
  XC_TRY(alloc_tmp(&tw64, size_t(b.L) * sizeof(cx<double>)));
  twiddle_kernel<double><<<gL, 256>>>(b.L, static_cast<cx<double>*>(tw64.ptr));
  XC_CUDA(cudaGetLastError());

  // compressed rows: S[N][H] FP64 complex
  DevBuf Sbuf, maxbuf;
  const size_t s_bytes = size_t(N) * size_t(H) * sizeof(cx<double>);
  if (s_bytes > (size_t(64) << 30)) return fail(XC_ERR_UNSUPPORTED, "compressed block exceeds 64 GiB during precompute");
  XC_TRY(alloc_tmp(&Sbuf, s_bytes));
  XC_TRY(alloc_tmp(&maxbuf, sizeof(unsigned long long)));
  XC_CUDA(cudaMemset(maxbuf.ptr, 0, sizeof(unsigned long long)));
  // Rows by the FFT of the generated, windowed rows (Algorithm 1 step 1.3).
  auto fft_rows = [&]() -> int {
    int64_t C = std::max<int64_t>(1, std::min<int64_t>(N, (int64_t(1) << 30) / (int64_t(b.L) * 8)));
    DevBuf Gbuf;
    XC_TRY(alloc_tmp(&Gbuf, size_t(C) * size_t(b.L) * sizeof(double)));
    const size_t csmem = size_t(n / csize) * sizeof(cx<double>);
    if (csize == 1) XC_TRY(set_smem(reinterpret_cast<const void*>(row_fft_kernel), smem));
    else XC_TRY(set_smem(reinterpret_cast<const void*>(row_fft_cluster_kernel), csmem));
    for (int64_t row0 = 0; row0 < N; row0 += C) {
      const int64_t rows = std::min<int64_t>(C, N - row0);
      // one thread per row, 32 per CTA so that the rows spread over every SM
      gen_rows_kernel<<<unsigned((rows + 31) / 32), 32>>>(g, row0, C, b.L, b.off, static_cast<double*>(w64.ptr),
                                                          static_cast<double*>(Gbuf.ptr));
      if (csize == 1) {
        row_fft_kernel<<<unsigned(rows), 256, smem>>>(static_cast<double*>(Gbuf.ptr), C, row0, N, b,
                                                       static_cast<cx<double>*>(tw64.ptr),
                                                       static_cast<cx<double>*>(Sbuf.ptr),
                                                       static_cast<unsigned long long*>(maxbuf.ptr), g.rw);
      } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(rows * csize));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = csmem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = unsigned(csize);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        XC_CUDA(cudaLaunchKernelEx(&cfg, row_fft_cluster_kernel, static_cast<const double*>(Gbuf.ptr), C, row0, N,
                                   b, static_cast<const cx<double>*>(tw64.ptr), static_cast<cx<double>*>(Sbuf.ptr),
                                   static_cast<unsigned long long*>(maxbuf.ptr), csize, g.rw));
      }
      XC_CUDA(cudaGetLastError());
    }
    XC_CUDA(cudaDeviceSynchronize());
    return XC_OK;
  };
  // Chebyshev rows at Chebyshev-Gauss angles by the Appendix A closed form:
  // the window's DFT components |m| <= cf_M (main lobe plus a margin; the
  // truncation error is under a tenth of eps1 * max|A_e W F|), the bins within
  // cf_B of each row's peak.  eps == 0 keeps every element, and short blocks
  // (where |m| <= cf_M would reach around the circle) are cheap to transform:
  // FFT rows then.
  const int cf_M = std::min(kCfMaxM, int(std::ceil(p->zeta / 3.141592653589793)) + 10);
  const int cf_B = std::min(kCfMaxB, cf_M + 24);
  const bool closed_ok = g.family == XC_CHEBYSHEV_T && g.cheb_exact && p->eps > 0 &&
                         p->params.precompute == XC_PRECOMPUTE_AUTO && b.L >= 8 * (2 * cf_M + 1);
  auto closed_rows = [&]() -> int {
    DevBuf xw;
    XC_TRY(alloc_tmp(&xw, size_t(2 * cf_M + 1) * sizeof(cx<double>)));
    window_dft_kernel<<<unsigned(2 * cf_M + 1), 256>>>(static_cast<double*>(w64.ptr), b.L, cf_M,
                                                       static_cast<cx<double>*>(xw.ptr));
    XC_CUDA(cudaMemset(Sbuf.ptr, 0, s_bytes));
    cheb_rows_closed_kernel<<<unsigned(N), 128>>>(N, b.L, b.off, n, cf_M, cf_B, static_cast<cx<double>*>(xw.ptr),
                                                  static_cast<cx<double>*>(Sbuf.ptr),
                                                  static_cast<unsigned long long*>(maxbuf.ptr), g.rw);
    XC_CUDA(cudaGetLastError());
    XC_CUDA(cudaDeviceSynchronize());
    return XC_OK;
  };
  bool closed = closed_ok;
  if (closed) XC_TRY(closed_rows());
  else XC_TRY(fft_rows());
  unsigned long long bits = 0;
  double maxsq = 0.0, thr = -1.0;
  auto read_threshold = [&]() -> int {
    XC_CUDA(cudaMemcpy(&bits, maxbuf.ptr, sizeof(bits), cudaMemcpyDeviceToHost));
    std::memcpy(&maxsq, &bits, sizeof(maxsq));
    thr = p->eps > 0 ? (p->eps * p->eps) * maxsq : -1.0;
    return XC_OK;
  };
  XC_TRY(read_threshold());
  p->maxabs[bi] = std::sqrt(maxsq);
  const int pair = p->precision == XC_FP64_PAIR ? 1 : 0;
  // stored values reach 2 max|S| (the half-spectrum factor): keep them well
  // inside the FP32 range
  if (pair && !(2.0 * std::sqrt(maxsq) < 1e30))
    return fail(XC_ERR_UNSUPPORTED, "band values exceed the FP32 range of XC_FP64_PAIR; use XC_FP64");

  // extents of the kept elements per row
  DevBuf kf, kl, cnt;
  XC_TRY(alloc_tmp(&kf, size_t(N) * sizeof(int)));
  XC_TRY(alloc_tmp(&kl, size_t(N) * sizeof(int)));
  XC_TRY(alloc_tmp(&cnt, size_t(N) * sizeof(int)));
  std::vector<int> kfirst(N), klast(N), count(N);
  auto extents = [&]() -> int {
    extents_kernel<<<unsigned((N * 32 + 255) / 256), 256>>>(static_cast<cx<double>*>(Sbuf.ptr), N, H, thr,
                                                            static_cast<int*>(kf.ptr), static_cast<int*>(kl.ptr),
                                                            static_cast<int*>(cnt.ptr), g.rw);
    XC_CUDA(cudaGetLastError());
    XC_CUDA(cudaMemcpy(kfirst.data(), kf.ptr, size_t(N) * sizeof(int), cudaMemcpyDeviceToHost));
    XC_CUDA(cudaMemcpy(klast.data(), kl.ptr, size_t(N) * sizeof(int), cudaMemcpyDeviceToHost));
    XC_CUDA(cudaMemcpy(count.data(), cnt.ptr, size_t(N) * sizeof(int), cudaMemcpyDeviceToHost));
    return XC_OK;
  };
  XC_TRY(extents());
  if (closed) {
    // a kept element on the edge of a row's candidate bins means its band may
    // reach beyond them: build the block from the FFT rows instead
    bool edge = false;
    for (int64_t r = 0; r < N && !edge; ++r) {
      if (klast[r] < 0) continue;
      int64_t klo, khi;
      cf_window(r, N, b.L, n, cf_B, &klo, &khi);
      edge = (klo > 0 && kfirst[r] <= klo) || (khi < n && klast[r] >= khi);
    }
    if (edge) {
      closed = false;
      XC_CUDA(cudaMemset(maxbuf.ptr, 0, sizeof(unsigned long long)));
      XC_TRY(fft_rows());
      XC_TRY(read_threshold());
      p->maxabs[bi] = std::sqrt(maxsq);
      XC_TRY(extents());
    }
  }
  if (closed) ++p->closed_form_blocks;
  int64_t nnz = 0;
  for (int64_t r = 0; r < N; ++r) nnz += count[r];
  p->nnz[bi] = nnz;

  // forward layout: slices of 32 rows, width = widest band in the slice; the
  // band start is moved left where needed so that k0 + width <= H
  const int nslices = int((N + kSlice - 1) / kSlice);
  std::vector<int> fwidth(nslices, 0), fk0(size_t(nslices) * kSlice, 0);
  std::vector<int64_t> foff(nslices, 0);
  int64_t total = 0;
  for (int s = 0; s < nslices; ++s) {
    int W = 0;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t r = int64_t(s) * kSlice + l;
      if (r < N && klast[r] >= 0) W = std::max(W, klast[r] - kfirst[r] + 1);
    }
    fwidth[s] = W;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t r = int64_t(s) * kSlice + l;
      fk0[size_t(s) * kSlice + l] = (r < N && klast[r] >= 0) ? std::min(kfirst[r], H - W) : 0;
    }
    foff[s] = total;
    total += int64_t(W) * kSlice;
  }
  p->stored[bi] = total;
  // adjoint layout: slices of 32 bins; bin k covers the rows whose band holds it
  const int tslices = int((H + kSlice - 1) / kSlice);
  std::vector<int> nlo(H, INT_MAX), nhi(H, -1);
  for (int64_t r = 0; r < N; ++r)
    for (int k = kfirst[r]; k <= klast[r]; ++k) {
      nlo[k] = std::min<int>(nlo[k], int(r));
      nhi[k] = std::max<int>(nhi[k], int(r));
    }
  std::vector<int> twidth(tslices, 0), tn0(size_t(tslices) * kSlice, 0);
  std::vector<int64_t> toff(tslices, 0);
  int64_t ttotal = 0;
  for (int s = 0; s < tslices; ++s) {
    int W = 0;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t k = int64_t(s) * kSlice + l;
      if (k < H && nhi[k] >= 0) W = std::max(W, nhi[k] - nlo[k] + 1);
    }
    twidth[s] = W;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t k = int64_t(s) * kSlice + l;
      tn0[size_t(s) * kSlice + l] = (k < H && nhi[k] >= 0) ? int(std::min<int64_t>(nlo[k], N - W)) : 0;
    }
    toff[s] = ttotal;
    ttotal += int64_t(W) * kSlice;
  }
  // Transposed right-hand sides for the adjoint product of FP32 plans where
  // the 32 bins of a slice start at rows far apart: the width-weighted mean
  // number of distinct 32-byte sectors among their first rows is 8 or more,
  // so that a step of scalar loads would gather from as many sectors per
  // right-hand side and the row-major y lines would not survive in L1.  (The
  // FP64 product is bound by the FP64 pipe, not by these loads.)
  int use_yt = 0;
  if (sizeof(T) == 4) {
    const int rows_per_sector = 32 / int(sizeof(T));
    double wsum = 0, swsum = 0;
    for (int s = 0; s < tslices; ++s) {
      int sec[kSlice], ns = 0;
      for (int l = 0; l < kSlice && int64_t(s) * kSlice + l < H; ++l) {
        const int sid = tn0[size_t(s) * kSlice + l] / rows_per_sector;
        bool seen = false;
        for (int q = 0; q < ns; ++q) seen = seen || sec[q] == sid;
        if (!seen) sec[ns++] = sid;
      }
      wsum += twidth[s];
      swsum += double(twidth[s]) * ns;
    }
    use_yt = wsum > 0 && swsum / wsum >= 8.0;
  }

  // adjoint items: each slice's run cut into chunks of 64 rows
  constexpr int kChunk = 64;
  std::vector<int2> citems;
  std::vector<int> cbase(tslices + 1, 0);
  for (int sl = 0; sl < tslices; ++sl) {
    cbase[sl] = int(citems.size());
    for (int c = 0; c * kChunk < twidth[sl]; ++c) citems.push_back(int2{sl, c});
  }
  cbase[tslices] = int(citems.size());
  p->c_nchunks = int64_t(citems.size());
  XC_TRY(upload(p, citems, &p->c_items));
  XC_TRY(upload(p, cbase, &p->c_cbase));
  // windows of the lockstep layouts (ensure_lockstep): per row slice the
  // union of its rows' bands, per bin slice the union of its bins' row runs
  {
    auto& flo = p->hf_lo[bi];
    auto& flen = p->hf_len[bi];
    flo.assign(nslices, 0);
    flen.assign(nslices, 0);
    for (int s = 0; s < nslices; ++s) {
      int lo = INT_MAX, hi = -1;
      for (int l = 0; l < kSlice; ++l) {
        const int64_t r = int64_t(s) * kSlice + l;
        if (r < N && klast[r] >= 0) {
          lo = std::min(lo, fk0[size_t(s) * kSlice + l]);
          hi = std::max(hi, fk0[size_t(s) * kSlice + l] + fwidth[s]);
        }
      }
      if (hi > lo) {
        flo[s] = lo;
        flen[s] = hi - lo;
      }
    }
    auto& tlo = p->ht_lo[bi];
    auto& tlen = p->ht_len[bi];
    tlo.assign(tslices, 0);
    tlen.assign(tslices, 0);
    for (int s = 0; s < tslices; ++s) {
      int lo = INT_MAX, hi = -1;
      for (int l = 0; l < kSlice; ++l) {
        const int64_t k = int64_t(s) * kSlice + l;
        if (k < H && nhi[k] >= 0) {
          lo = std::min(lo, tn0[size_t(s) * kSlice + l]);
          hi = std::max(hi, tn0[size_t(s) * kSlice + l] + twidth[s]);
        }
      }
      if (hi > lo) {
        tlo[s] = lo;
        tlen[s] = hi - lo;
      }
    }
  }
  int *fk0_d, *fw_d, *tn0_d, *tw_d;
  int64_t *foff_d, *toff_d;
  XC_TRY(upload(p, fk0, &fk0_d));
  XC_TRY(upload(p, fwidth, &fw_d));
  XC_TRY(upload(p, foff, &foff_d));
  XC_TRY(upload(p, tn0, &tn0_d));
  XC_TRY(upload(p, twidth, &tw_d));
  XC_TRY(upload(p, toff, &toff_d));
  void *fval = nullptr, *tval = nullptr;
  XC_TRY(plan_alloc(p, &fval, size_t(std::max<int64_t>(total, 1)) * sizeof(cx<T>)));
  XC_TRY(plan_alloc(p, &tval, size_t(std::max<int64_t>(ttotal, 1)) * sizeof(cx<T>)));
  int maxW = 0, maxTW = 0;
  for (int v : fwidth) maxW = std::max(maxW, v);
  for (int v : twidth) maxTW = std::max(maxTW, v);
  if (maxW > 0) {
    dim3 grid(unsigned((int64_t(maxW) * kSlice + 255) / 256), unsigned(nslices));
    fill_forward_kernel<T><<<grid, 256>>>(static_cast<cx<double>*>(Sbuf.ptr), N, n, thr, fk0_d, fw_d, foff_d,
                                          nslices, static_cast<cx<T>*>(fval), pair, g.rw);
  }
  if (maxTW > 0) {
    dim3 grid(unsigned((int64_t(maxTW) * kSlice + 255) / 256), unsigned(tslices));
    fill_adjoint_kernel<T><<<grid, 256>>>(static_cast<cx<double>*>(Sbuf.ptr), N, n, thr, tn0_d, tw_d, toff_d,
                                          tslices, static_cast<cx<T>*>(tval), pair, g.rw);
  }
  XC_CUDA(cudaGetLastError());
  XC_CUDA(cudaDeviceSynchronize());
  b.nslices = nslices;
  b.f_k0 = fk0_d;
  b.f_width = fw_d;
  b.f_off = foff_d;
  b.f_val = fval;
  b.tslices = tslices;
  b.t_n0 = tn0_d;
  b.t_width = tw_d;
  b.t_off = toff_d;
  b.t_val = tval;
  b.t_yt = use_yt;
  p->any_yt = p->any_yt || use_yt;
  p->matrix_bytes += total * int64_t(sizeof(cx<T>)) + int64_t(N) * 4;
  p->adjoint_bytes += ttotal * int64_t(sizeof(cx<T>)) + int64_t(H) * 4;
  return XC_OK;
}

// The single two-sided block of a complex family (Section 2.2 with a complex
// matrix): the extended rows exp(i (j - off) theta_n) w_j are transformed as
// their real and imaginary parts (two real row FFTs), which give the full
// spectrum S = A_e W F / sqrt(L) (up to the 1/sqrt(L) the apply folds in);
// each row keeps one circular band around its peak bin theta_n L / (2 pi),
// each bin one circular run of rows.
template <typename T>
int build_block_complex(Plan* p, const GenParams& g, const BlockShape& shp) {
  BlockDev& b = p->blocks[0];
  std::memset(&b, 0, sizeof(b));
  const int64_t N = p->N;
  b.L = int(shp.L);
  b.n = int(shp.L / 2);
  b.H = b.n + 1;
  b.off = int(shp.off);
  b.j_lo = int(shp.j_lo);
  b.j_hi = int(shp.j_hi);
  b.a_csize = 1;
  b.p = fft_radices(b.n, b.radix);
  if (b.p < 0) return fail(XC_ERR_UNSUPPORTED, "FFT length not 2^a 3^b 5^c 7^d");
  const int n = b.n, H = b.H, L = b.L;
  int dev = 0, optin = 0;
  XC_CUDA(cudaGetDevice(&dev));
  XC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t smem = size_t(n) * sizeof(cx<double>);
  // the FP64 row FFT of the precompute and each CTA of the apply's two-CTA
  // transforms hold n = L/2 complex values
  if (smem + 1024 > size_t(optin) || size_t(n) * sizeof(cx<T>) + 1024 > size_t(optin))
    return fail(XC_ERR_UNSUPPORTED, "complex block length L = " + std::to_string(L) +
                                        " exceeds one CTA's shared memory for L/2 values");
  std::vector<int> perm = digit_reversal(n, b.p, b.radix);
  int* perm_d = nullptr;
  XC_TRY(upload(p, perm, &perm_d));
  b.perm = perm_d;
  DevBuf w64;
  XC_TRY(alloc_tmp(&w64, size_t(L) * sizeof(double)));
  void *invw = nullptr, *tw = nullptr;
  XC_TRY(plan_alloc(p, &invw, size_t(L) * sizeof(T)));
  XC_TRY(plan_alloc(p, &tw, size_t(L) * sizeof(cx<T>)));
  const unsigned gL = unsigned((L + 255) / 256);
  window_kernel<T><<<gL, 256>>>(L, p->zeta, static_cast<double*>(w64.ptr), static_cast<T*>(invw));
  twiddle_kernel<T><<<gL, 256>>>(L, static_cast<cx<T>*>(tw));
  b.invw = invw;
  b.tw = tw;
  DevBuf tw64;
  XC_TRY(alloc_tmp(&tw64, size_t(L) * sizeof(cx<double>)));
  twiddle_kernel<double><<<gL, 256>>>(L, static_cast<cx<double>*>(tw64.ptr));
  XC_CUDA(cudaGetLastError());

  // half spectra of the real and imaginary parts of every row
  const size_t s_bytes = size_t(N) * size_t(H) * sizeof(cx<double>);
  if (2 * s_bytes > (size_t(64) << 30)) return fail(XC_ERR_UNSUPPORTED, "compressed block exceeds 64 GiB during precompute");
  DevBuf Sc, Ss, maxbuf;
  XC_TRY(alloc_tmp(&Sc, s_bytes));
  XC_TRY(alloc_tmp(&Ss, s_bytes));
  XC_TRY(alloc_tmp(&maxbuf, sizeof(unsigned long long)));
  XC_TRY(set_smem(reinterpret_cast<const void*>(row_fft_kernel), smem));
  {
    const int64_t C = std::max<int64_t>(1, std::min<int64_t>(N, (int64_t(1) << 30) / (int64_t(L) * 8)));
    DevBuf Gbuf;
    XC_TRY(alloc_tmp(&Gbuf, size_t(C) * size_t(L) * sizeof(double)));
    for (int part = 0; part < 2; ++part) {
      GenParams gp = g;
      gp.cpart = part;
      cx<double>* S = static_cast<cx<double>*>(part == 0 ? Sc.ptr : Ss.ptr);
      for (int64_t row0 = 0; row0 < N; row0 += C) {
        const int64_t rows = std::min<int64_t>(C, N - row0);
        gen_rows_kernel<<<unsigned((rows + 31) / 32), 32>>>(gp, row0, C, L, b.off, static_cast<double*>(w64.ptr),
                                                            static_cast<double*>(Gbuf.ptr));
        row_fft_kernel<<<unsigned(rows), 256, smem>>>(static_cast<double*>(Gbuf.ptr), C, row0, N, b,
                                                       static_cast<cx<double>*>(tw64.ptr), S,
                                                       static_cast<unsigned long long*>(maxbuf.ptr), nullptr);
        XC_CUDA(cudaGetLastError());
      }
    }
  }
  const cx<double>* scp = static_cast<const cx<double>*>(Sc.ptr);
  const cx<double>* ssp = static_cast<const cx<double>*>(Ss.ptr);
  XC_CUDA(cudaMemset(maxbuf.ptr, 0, sizeof(unsigned long long)));
  c_max_kernel<<<unsigned(std::min<int64_t>(152 * 16, (N * L + 255) / 256)), 256>>>(
      scp, ssp, N, n, static_cast<unsigned long long*>(maxbuf.ptr));
  XC_CUDA(cudaGetLastError());
  unsigned long long bits = 0;
  double maxsq = 0.0;
  XC_CUDA(cudaMemcpy(&bits, maxbuf.ptr, sizeof(bits), cudaMemcpyDeviceToHost));
  std::memcpy(&maxsq, &bits, sizeof(maxsq));
  const double thr = p->eps > 0 ? (p->eps * p->eps) * maxsq : -1.0;
  p->maxabs[0] = std::sqrt(maxsq);

  // circular row bands and bin runs
  DevBuf k0d, rwd, cntd, n0d, bwd;
  XC_TRY(alloc_tmp(&k0d, size_t(N) * sizeof(int)));
  XC_TRY(alloc_tmp(&rwd, size_t(N) * sizeof(int)));
  XC_TRY(alloc_tmp(&cntd, size_t(N) * sizeof(int)));
  XC_TRY(alloc_tmp(&n0d, size_t(L) * sizeof(int)));
  XC_TRY(alloc_tmp(&bwd, size_t(L) * sizeof(int)));
  c_extents_kernel<<<unsigned((N * 32 + 255) / 256), 256>>>(scp, ssp, N, n, thr, static_cast<int*>(k0d.ptr),
                                                            static_cast<int*>(rwd.ptr), static_cast<int*>(cntd.ptr));
  c_col_extents_kernel<<<unsigned((L + 127) / 128), 128>>>(scp, ssp, N, n, thr, static_cast<int*>(n0d.ptr),
                                                           static_cast<int*>(bwd.ptr));
  XC_CUDA(cudaGetLastError());
  std::vector<int> k0(N), rw(N), cnt(N), bw(L), n0(L);
  XC_CUDA(cudaMemcpy(k0.data(), k0d.ptr, size_t(N) * sizeof(int), cudaMemcpyDeviceToHost));
  XC_CUDA(cudaMemcpy(rw.data(), rwd.ptr, size_t(N) * sizeof(int), cudaMemcpyDeviceToHost));
  XC_CUDA(cudaMemcpy(cnt.data(), cntd.ptr, size_t(N) * sizeof(int), cudaMemcpyDeviceToHost));
  XC_CUDA(cudaMemcpy(n0.data(), n0d.ptr, size_t(L) * sizeof(int), cudaMemcpyDeviceToHost));
  XC_CUDA(cudaMemcpy(bw.data(), bwd.ptr, size_t(L) * sizeof(int), cudaMemcpyDeviceToHost));
  int64_t nnz = 0;
  for (int64_t r = 0; r < N; ++r) nnz += cnt[r];
  p->nnz[0] = nnz;

  // forward: slices of 32 rows, width = widest band of the slice
  const int nslices = int((N + kSlice - 1) / kSlice);
  std::vector<int> fwidth(nslices, 0);
  std::vector<int64_t> foff(nslices, 0);
  int64_t total = 0;
  int vpad = 0;
  for (int sl = 0; sl < nslices; ++sl) {
    int W = 0;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t r = int64_t(sl) * kSlice + l;
      if (r < N) W = std::max(W, rw[r]);
    }
    fwidth[sl] = W;
    foff[sl] = total;
    total += int64_t(W) * kSlice;
    vpad = std::max(vpad, W);
  }
  p->stored[0] = total;
  p->c_vpad = vpad;
  // adjoint: slices of 32 bins, width = longest run of the slice
  const int tslices = (L + kSlice - 1) / kSlice;
  std::vector<int> twidth(tslices, 0);
  std::vector<int64_t> toff(tslices, 0);
  int64_t ttotal = 0;
  for (int sl = 0; sl < tslices; ++sl) {
    int W = 0;
    for (int l = 0; l < kSlice; ++l) {
      const int k = sl * kSlice + l;
      if (k < L) W = std::max(W, bw[k]);
    }
    twidth[sl] = W;
    toff[sl] = ttotal;
    ttotal += int64_t(W) * kSlice;
  }
  // adjoint items: each slice's run cut into chunks of 64 rows
  constexpr int kChunk = 64;
  std::vector<int2> citems;
  std::vector<int> cbase(tslices + 1, 0);
  for (int sl = 0; sl < tslices; ++sl) {
    cbase[sl] = int(citems.size());
    for (int c = 0; c * kChunk < twidth[sl]; ++c) citems.push_back(int2{sl, c});
  }
  cbase[tslices] = int(citems.size());
  p->c_nchunks = int64_t(citems.size());
  XC_TRY(upload(p, citems, &p->c_items));
  XC_TRY(upload(p, cbase, &p->c_cbase));
  int *fk0_d, *fw_d, *tn0_d, *tw_d;
  int64_t *foff_d, *toff_d;
  XC_TRY(upload(p, k0, &fk0_d));
  XC_TRY(upload(p, fwidth, &fw_d));
  XC_TRY(upload(p, foff, &foff_d));
  XC_TRY(upload(p, n0, &tn0_d));
  XC_TRY(upload(p, twidth, &tw_d));
  XC_TRY(upload(p, toff, &toff_d));
  void *fval = nullptr, *tval = nullptr;
  XC_TRY(plan_alloc(p, &fval, size_t(std::max<int64_t>(1, total)) * sizeof(cx<T>)));
  XC_TRY(plan_alloc(p, &tval, size_t(std::max<int64_t>(1, ttotal)) * sizeof(cx<T>)));
  int maxW = 0, maxTW = 0;
  for (int w : fwidth) maxW = std::max(maxW, w);
  for (int w : twidth) maxTW = std::max(maxTW, w);
  if (maxW > 0)
    c_fill_forward_kernel<T><<<dim3(unsigned((int64_t(maxW) * 32 + 255) / 256), unsigned(nslices)), 256>>>(
        scp, ssp, N, n, thr, fk0_d, static_cast<int*>(rwd.ptr), fw_d, foff_d, nslices, static_cast<cx<T>*>(fval));
  if (maxTW > 0)
    c_fill_adjoint_kernel<T><<<dim3(unsigned((int64_t(maxTW) * 32 + 255) / 256), unsigned(tslices)), 256>>>(
        scp, ssp, N, n, thr, tn0_d, static_cast<int*>(bwd.ptr), tw_d, toff_d, tslices, static_cast<cx<T>*>(tval));
  XC_CUDA(cudaGetLastError());
  XC_CUDA(cudaDeviceSynchronize());
  b.nslices = nslices;
  b.f_k0 = fk0_d;
  b.f_width = fw_d;
  b.f_off = foff_d;
  b.f_val = fval;
  b.tslices = tslices;
  b.t_n0 = tn0_d;
  b.t_width = tw_d;
  b.t_off = toff_d;
  b.t_val = tval;
  b.spec_off = 0;
  p->matrix_bytes += total * int64_t(sizeof(cx<T>)) + int64_t(N) * 4;
  p->adjoint_bytes += ttotal * int64_t(sizeof(cx<T>)) + int64_t(L) * 4;
  return XC_OK;
}

// One transform side (length L) of a 2-D block: the apply's descriptor in the
// plan precision (permutation, twiddles, 1/w) and the FP64 window and
// twiddles of the precompute.
template <typename T>
int make_side(Plan* p, int64_t L, BlockDev* d, DevBuf* w64, DevBuf* tw64) {
  std::memset(d, 0, sizeof(*d));
  d->L = int(L);
  d->n = int(L / 2);
  d->H = d->n + 1;
  d->a_csize = 1;
  d->p = fft_radices(d->n, d->radix);
  if (d->p < 0) return fail(XC_ERR_UNSUPPORTED, "FFT length not 2^a 3^b 5^c 7^d");
  std::vector<int> perm = digit_reversal(d->n, d->p, d->radix);
  int* perm_d = nullptr;
  XC_TRY(upload(p, perm, &perm_d));
  d->perm = perm_d;
  void *invw = nullptr, *tw = nullptr;
  XC_TRY(plan_alloc(p, &invw, size_t(L) * sizeof(T)));
  XC_TRY(plan_alloc(p, &tw, size_t(L) * sizeof(cx<T>)));
  XC_TRY(alloc_tmp(w64, size_t(L) * sizeof(double)));
  XC_TRY(alloc_tmp(tw64, size_t(L) * sizeof(cx<double>)));
  const unsigned gL = unsigned((L + 255) / 256);
  window_kernel<T><<<gL, 256>>>(L, p->zeta, static_cast<double*>(w64->ptr), static_cast<T*>(invw));
  twiddle_kernel<T><<<gL, 256>>>(L, static_cast<cx<T>*>(tw));
  twiddle_kernel<double><<<gL, 256>>>(L, static_cast<cx<double>*>(tw64->ptr));
  XC_CUDA(cudaGetLastError());
  d->invw = invw;
  d->tw = tw;
  return XC_OK;
}

struct Blk2 {
  int64_t r0, Lr, vr0, r1, c0, Lc, vc0, c1;
};

// Cover the N x N index square by the valid rectangles of 2-D blocks and
// dense rectangles: a rectangle takes a block whose first sr rows and sc
// columns (window below eps2) are left to two further rectangles; a side of
// at most `tail` makes it dense.  lower_zero (A^[1], zero for i > j): a
// rectangle wholly below the diagonal, and a block whose valid part is, is
// left out (it adds exactly zero; its extension would bring in the jump).
void decompose_2d(int64_t N, double zeta, double eps2, int64_t tail, bool lower_zero, std::vector<Blk2>* blocks,
                  std::vector<D2Rect>* rects) {
  std::vector<std::array<int64_t, 4>> todo{{0, N, 0, N}};
  while (!todo.empty()) {
    const std::array<int64_t, 4> t = todo.back();
    todo.pop_back();
    const int64_t r0 = t[0], r1 = t[1], c0 = t[2], c1 = t[3];
    const int64_t mr = r1 - r0, mc = c1 - c0;
    if (mr <= 0 || mc <= 0) continue;
    if (lower_zero && r0 >= c1) continue;
    const D2Rect whole{int(r0), int(r1), int(c0), int(c1), 0};
    if (mr <= tail || mc <= tail) {
      rects->push_back(whole);
      continue;
    }
    int64_t sr = extra_count(mr, zeta, eps2, false), sc = extra_count(mc, zeta, eps2, false);
    if (sr < 0 || sc < 0) {
      rects->push_back(whole);
      continue;
    }
    const int64_t Lr = fft_friendly_at_least(mr + sr), Lc = fft_friendly_at_least(mc + sc);
    sr = Lr - mr;
    sc = Lc - mc;
    if (sr >= mr || sc >= mc) {
      rects->push_back(whole);
      continue;
    }
    if (!(lower_zero && r0 + sr >= c1)) blocks->push_back(Blk2{r0, Lr, r0 + sr, r1, c0, Lc, c0 + sc, c1});
    todo.push_back({r0, r0 + sr, c0, c1});
    todo.push_back({r0 + sr, r1, c0, c0 + sc});
  }
}

// Combine lists of the 2-D scheme: output index o (a row for the forward
// product, a column for the adjoint) takes the partials of the blocks whose
// valid outputs hold it (entry b), then the dense rectangles that cover it
// (entry ~d).
void combine_lists_2d(int64_t N, const std::vector<Blk2>& blks, const std::vector<D2Rect>& rects, bool rows,
                      std::vector<int>* ptr, std::vector<int>* flat) {
  std::vector<std::vector<int>> ent(static_cast<size_t>(N));
  for (size_t bi = 0; bi < blks.size(); ++bi) {
    const Blk2& b = blks[bi];
    const int64_t lo = rows ? b.vr0 : b.vc0;
    const int64_t hi = rows ? b.r1 : b.c1;
    for (int64_t o = lo; o < hi; ++o) ent[static_cast<size_t>(o)].push_back(static_cast<int>(bi));
  }
  for (size_t d = 0; d < rects.size(); ++d) {
    const int lo = rows ? rects[d].r0 : rects[d].c0;
    const int hi = rows ? rects[d].r1 : rects[d].c1;
    for (int o = lo; o < hi; ++o) ent[static_cast<size_t>(o)].push_back(~static_cast<int>(d));
  }
  ptr->assign(static_cast<size_t>(N) + 1, 0);
  flat->clear();
  for (int64_t o = 0; o < N; ++o) {
    (*ptr)[static_cast<size_t>(o)] = static_cast<int>(flat->size());
    flat->insert(flat->end(), ent[static_cast<size_t>(o)].begin(), ent[static_cast<size_t>(o)].end());
  }
  (*ptr)[static_cast<size_t>(N)] = static_cast<int>(flat->size());
}

// The 2-D block scheme's precompute.  Per block: W_r D_e W_c generated on the
// device, FFT of every row along the columns (row_fft_kernel), then of every
// column along the rows (its real and imaginary parts as two real row
// transforms), giving S = DFT2(W_r D_e W_c) / (Lr Lc) = D̈ / sqrt(Lr Lc) for
// row bins p < Lr and column bins q <= Lc/2; the other columns follow from
// S[p][Lc - q] = conj(S[(Lr - p) % Lr][q]) (real D_e).  Elements with
// |S|^2 <= eps1^2 max|S|^2 are dropped and each direction's product is stored
// as a CSR over its output half-spectrum bins.
template <typename T>
int build_plan_2d(Plan* p) {
  const int64_t N = p->N;
  const bool kernel = p->family == XC_KERNEL_A1 || p->family == XC_KERNEL_A2;
  auto* d2 = new (std::nothrow) D2Plan();
  if (!d2) return fail(XC_ERR_ALLOC, "host allocation failed");
  p->d2 = d2;
  std::vector<Blk2> blks;
  const int64_t tail = p->params.tail_max > 0 ? p->params.tail_max : 20;
  decompose_2d(N, p->zeta, p->eps2, tail, p->family == XC_KERNEL_A1, &blks, &d2->rects_host);
  const int nb = int(blks.size());
  d2->nb = nb;
  int64_t mmax = N + 2, rmax = N;
  for (const auto& b : blks) {
    mmax = std::max(mmax, b.c0 + b.Lc + 2);
    rmax = std::max(rmax, b.r0 + b.Lr);
  }
  int dev = 0, optin = 0;
  XC_CUDA(cudaGetDevice(&dev));
  XC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  for (const auto& b : blks)
    if (size_t(std::max(b.Lr, b.Lc) / 2) * sizeof(cx<double>) + 1024 > size_t(optin))
      return fail(XC_ERR_UNSUPPORTED, "2-D block side above one CTA's shared memory for L/2 FP64 values");
  // generation helpers: recurrence coefficients (functions) or the Lambda
  // table (A^[1]), node arrays per block
  GenParams g{p->family, N, 0.0, 0.0, nullptr, 0, 0};
  XC_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->nodes_dev), size_t(N) * sizeof(double)));
  XC_CUDA(cudaMemcpy(p->nodes_dev, p->nodes_host.data(), size_t(N) * sizeof(double), cudaMemcpyHostToDevice));
  const double* lamp = nullptr;
  if (kernel) {
    const int64_t K = 2 * std::max(mmax, rmax) + 4;
    std::vector<double> lam(K);
    long double v = 1.7724538509055160272981674833411452L;   // sqrt(pi) = Lambda(0)
    for (int64_t z = 0; z < K; ++z) {
      if (z > 0) v = v * (2.0L * z - 1.0L) / (2.0L * z);
      lam[z] = double(v);
    }
    double* lamd = nullptr;
    XC_TRY(upload(p, lam, &lamd));
    d2->lam = lamd;
    lamp = lamd;
  } else {
    const std::vector<double> rc = recurrence_table(p->family, 0.0, 0.0, mmax + 1);
    XC_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->rc_dev), rc.size() * sizeof(double)));
    XC_CUDA(cudaMemcpy(p->rc_dev, rc.data(), rc.size() * sizeof(double), cudaMemcpyHostToDevice));
    p->nrc = mmax + 1;
    g.rc = p->rc_dev;
    g.nrc = p->nrc;
  }
  auto node_array = [&](int64_t r0, int64_t rows, DevBuf* buf) -> int {
    std::vector<double> x(rows);
    for (int64_t i = 0; i < rows; ++i) x[i] = p->x0 + p->h * double(r0 + i);
    XC_TRY(alloc_tmp(buf, size_t(rows) * sizeof(double)));
    XC_CUDA(cudaMemcpy(buf->ptr, x.data(), size_t(rows) * sizeof(double), cudaMemcpyHostToDevice));
    return XC_OK;
  };

  d2->fwd.in_host.resize(nb);
  d2->fwd.out_host.resize(nb);
  d2->adj.in_host.resize(nb);
  d2->adj.out_host.resize(nb);
  // per output bin two segments: the a terms (with conj(U)), then the c terms
  struct Csr {
    std::vector<int64_t> ptr{0};
    std::vector<int> idx, blk, loc;
    std::vector<cx<T>> val;
  } fcsr, acsr;
  int64_t kept_total = 0;
  int64_t fspec_in = 0, fspec_out = 0, aspec_in = 0, aspec_out = 0, fparts = 0, aparts = 0;
  std::vector<int64_t> fpart_off(nb), apart_off(nb);
  for (int bi = 0; bi < nb; ++bi) {
    const Blk2& B = blks[bi];
    BlockDev col, row;
    DevBuf wc64, twc64, wr64, twr64;
    XC_TRY(make_side<T>(p, B.Lc, &col, &wc64, &twc64));
    XC_TRY(make_side<T>(p, B.Lr, &row, &wr64, &twr64));
    const int64_t Lr = B.Lr, Lc = B.Lc, Hr = row.H, Hc = col.H;
    // W_r D_e W_c, column-major [Lc][Lr]
    DevBuf G;
    XC_TRY(alloc_tmp(&G, size_t(Lr) * size_t(Lc) * sizeof(double)));
    if (kernel) {
      gen2d_kernel_elems<<<dim3(unsigned((Lr + 127) / 128), unsigned(Lc)), 128>>>(
          p->family, B.r0, Lr, B.c0, Lc, static_cast<double*>(wr64.ptr), static_cast<double*>(wc64.ptr), lamp,
          static_cast<double*>(G.ptr));
    } else {
      DevBuf xn;
      XC_TRY(node_array(B.r0, Lr, &xn));
      GenParams gb = g;
      gb.x = static_cast<double*>(xn.ptr);
      gen2d_rows_kernel<<<unsigned((Lr + 31) / 32), 32>>>(gb, Lr, B.c0, Lc, static_cast<double*>(wr64.ptr),
                                                          static_cast<double*>(wc64.ptr),
                                                          static_cast<double*>(G.ptr));
      XC_CUDA(cudaDeviceSynchronize());
    }
    XC_CUDA(cudaGetLastError());
    // along the columns: S1[i][q], q <= Lc/2 (scaled 1/Lc)
    DevBuf S1, dummy;
    XC_TRY(alloc_tmp(&S1, size_t(Lr) * size_t(Hc) * sizeof(cx<double>)));
    XC_TRY(alloc_tmp(&dummy, sizeof(unsigned long long)));
    XC_TRY(set_smem(reinterpret_cast<const void*>(row_fft_kernel),
                    size_t(std::max(col.n, row.n)) * sizeof(cx<double>)));
    row_fft_kernel<<<unsigned(Lr), 256, size_t(col.n) * sizeof(cx<double>)>>>(
        static_cast<double*>(G.ptr), Lr, 0, Lr, col, static_cast<cx<double>*>(twc64.ptr),
        static_cast<cx<double>*>(S1.ptr), static_cast<unsigned long long*>(dummy.ptr), nullptr);
    XC_CUDA(cudaGetLastError());
    // along the rows: real and imaginary parts of every column bin q
    DevBuf Re, Im, A, Bm;
    XC_TRY(alloc_tmp(&Re, size_t(Lr) * size_t(Hc) * sizeof(double)));
    XC_TRY(alloc_tmp(&Im, size_t(Lr) * size_t(Hc) * sizeof(double)));
    split2d_kernel<<<unsigned((Lr * Hc + 255) / 256), 256>>>(static_cast<cx<double>*>(S1.ptr), Lr, Hc,
                                                              static_cast<double*>(Re.ptr),
                                                              static_cast<double*>(Im.ptr));
    XC_TRY(alloc_tmp(&A, size_t(Hc) * size_t(Hr) * sizeof(cx<double>)));
    XC_TRY(alloc_tmp(&Bm, size_t(Hc) * size_t(Hr) * sizeof(cx<double>)));
    const size_t rsm = size_t(row.n) * sizeof(cx<double>);
    row_fft_kernel<<<unsigned(Hc), 256, rsm>>>(static_cast<double*>(Re.ptr), Hc, 0, Hc, row,
                                                static_cast<cx<double>*>(twr64.ptr), static_cast<cx<double>*>(A.ptr),
                                                static_cast<unsigned long long*>(dummy.ptr), nullptr);
    row_fft_kernel<<<unsigned(Hc), 256, rsm>>>(static_cast<double*>(Im.ptr), Hc, 0, Hc, row,
                                                static_cast<cx<double>*>(twr64.ptr), static_cast<cx<double>*>(Bm.ptr),
                                                static_cast<unsigned long long*>(dummy.ptr), nullptr);
    XC_CUDA(cudaGetLastError());
    std::vector<cx<double>> Ah(size_t(Hc) * size_t(Hr)), Bh(size_t(Hc) * size_t(Hr));
    XC_CUDA(cudaMemcpy(Ah.data(), A.ptr, Ah.size() * sizeof(cx<double>), cudaMemcpyDeviceToHost));
    XC_CUDA(cudaMemcpy(Bh.data(), Bm.ptr, Bh.size() * sizeof(cx<double>), cudaMemcpyDeviceToHost));
    // S(p, q) for p < Lr, q <= Lc/2: A_full + i B_full along p
    auto S = [&](int64_t pp, int64_t q) {
      cx<double> a, b;
      if (pp <= Lr / 2) {
        a = Ah[size_t(q) * Hr + pp];
        b = Bh[size_t(q) * Hr + pp];
      } else {
        a = Ah[size_t(q) * Hr + (Lr - pp)];
        b = Bh[size_t(q) * Hr + (Lr - pp)];
        a.im = -a.im;
        b.im = -b.im;
      }
      return cx<double>{a.re - b.im, a.im + b.re};
    };
    auto sq = [](cx<double> v) { return v.re * v.re + v.im * v.im; };
    double maxsq = 0.0;
    for (int64_t pp = 0; pp < Lr; ++pp)
      for (int64_t q = 0; q < Hc; ++q) maxsq = std::max(maxsq, sq(S(pp, q)));
    const double thr = p->eps > 0 ? (p->eps * p->eps) * maxsq : -1.0;
    for (int64_t pp = 0; pp < Lr; ++pp)
      for (int64_t q = 0; q < Hc; ++q)
        if (sq(S(pp, q)) > thr) kept_total += (q > 0 && q < Lc / 2) ? 2 : 1;
    auto cvt = [](cx<double> v) { return cx<T>{T(v.re), T(v.im)}; };
    // forward: z_p = sum_q a conj(U_q) + c U_q, a = S(p, q), c = conj(S(-p, q)) (0 < q < Lc/2)
    for (int64_t pp = 0; pp < Hr; ++pp) {
      for (int64_t q = 0; q < Hc; ++q) {
        const cx<double> a = S(pp, q);
        if (sq(a) > thr) {
          fcsr.idx.push_back(int(q));
          fcsr.val.push_back(cvt(a));
        }
      }
      fcsr.ptr.push_back(int64_t(fcsr.idx.size()));
      for (int64_t q = 1; q < (Lc + 1) / 2; ++q) {
        const cx<double> m = S((Lr - pp) % Lr, q);
        if (sq(m) > thr) {
          fcsr.idx.push_back(int(q));
          fcsr.val.push_back(cvt(cx<double>{m.re, -m.im}));
        }
      }
      fcsr.ptr.push_back(int64_t(fcsr.idx.size()));
      fcsr.blk.push_back(bi);
      fcsr.loc.push_back(int(pp));
    }
    // adjoint: z_q = sum_p a conj(U_p) + c U_p, a = S(p, q), c = S(Lr - p, q) (0 < p < Lr/2)
    for (int64_t q = 0; q < Hc; ++q) {
      for (int64_t pp = 0; pp < Hr; ++pp) {
        const cx<double> a = S(pp, q);
        if (sq(a) > thr) {
          acsr.idx.push_back(int(pp));
          acsr.val.push_back(cvt(a));
        }
      }
      acsr.ptr.push_back(int64_t(acsr.idx.size()));
      for (int64_t pp = 1; pp < (Lr + 1) / 2; ++pp) {
        const cx<double> c = S(Lr - pp, q);
        if (sq(c) > thr) {
          acsr.idx.push_back(int(pp));
          acsr.val.push_back(cvt(c));
        }
      }
      acsr.ptr.push_back(int64_t(acsr.idx.size()));
      acsr.blk.push_back(bi);
      acsr.loc.push_back(int(q));
    }
    // descriptors: the column side takes the forward inputs and the adjoint
    // outputs, the row side the forward outputs and the adjoint inputs
    col.off = -int(B.c0);
    col.j_lo = int(B.vc0 - B.c0);
    col.j_hi = int(B.c1 - B.c0);
    row.off = -int(B.r0);
    row.j_lo = int(B.vr0 - B.r0);
    row.j_hi = int(B.r1 - B.r0);
    d2->fwd.in_host[bi] = col;
    d2->fwd.in_host[bi].spec_off = fspec_in;
    d2->fwd.out_host[bi] = row;
    d2->fwd.out_host[bi].spec_off = fspec_out;
    d2->adj.in_host[bi] = row;
    d2->adj.in_host[bi].spec_off = aspec_in;
    d2->adj.out_host[bi] = col;
    d2->adj.out_host[bi].spec_off = aspec_out;
    fspec_in += Hc;
    fspec_out += Hr;
    aspec_in += Hr;
    aspec_out += Hc;
    fpart_off[bi] = fparts;
    fparts += B.r1 - B.vr0;
    apart_off[bi] = aparts;
    aparts += B.c1 - B.vc0;
    d2->fwd.max_n_in = std::max(d2->fwd.max_n_in, col.n);
    d2->fwd.max_n_out = std::max(d2->fwd.max_n_out, row.n);
    d2->adj.max_n_in = std::max(d2->adj.max_n_in, row.n);
    d2->adj.max_n_out = std::max(d2->adj.max_n_out, col.n);
  }
  d2->kept = kept_total;
  // device copies
  auto put_dir = [&](D2Dir& D, Csr& C, int64_t spec_in, int64_t spec_out, int64_t parts,
                     const std::vector<int64_t>& part_off) -> int {
    D.spec_in = spec_in;
    D.spec_out = spec_out;
    D.parts = parts;
    D.rows = int64_t(C.blk.size());
    D.nnz = int64_t(C.idx.size());
    XC_TRY(upload(p, D.in_host, reinterpret_cast<BlockDev**>(&D.in_dev)));
    XC_TRY(upload(p, D.out_host, reinterpret_cast<BlockDev**>(&D.out_dev)));
    XC_TRY(upload(p, C.ptr, &D.ptr));
    XC_TRY(upload(p, C.idx, &D.idx));
    XC_TRY(upload(p, C.blk, &D.row_blk));
    XC_TRY(upload(p, C.loc, &D.row_loc));
    cx<T>* v = nullptr;
    XC_TRY(upload(p, C.val, &v));
    D.a = v;
    XC_TRY(upload(p, part_off, &D.part_off));
    return XC_OK;
  };
  XC_TRY(put_dir(d2->fwd, fcsr, fspec_in, fspec_out, fparts, fpart_off));
  XC_TRY(put_dir(d2->adj, acsr, aspec_in, aspec_out, aparts, apart_off));
  // dense rectangles
  int64_t dense_elems = 0;
  for (auto& r : d2->rects_host) {
    r.off = dense_elems;
    dense_elems += int64_t(r.r1 - r.r0) * (r.c1 - r.c0);
  }
  d2->dense_elems = dense_elems;
  XC_TRY(plan_alloc(p, &d2->dense, size_t(std::max<int64_t>(1, dense_elems)) * sizeof(T)));
  for (const auto& r : d2->rects_host) {
    DevBuf xn;
    GenParams gr = g;
    if (!kernel) {
      XC_TRY(node_array(r.r0, r.r1 - r.r0, &xn));
      gr.x = static_cast<double*>(xn.ptr);
    }
    rect2d_kernel<T><<<unsigned((r.r1 - r.r0 + 31) / 32), 32>>>(gr, p->family, r.r0, r.r1, r.c0, r.c1, lamp,
                                                                 static_cast<T*>(d2->dense) + r.off, r.c1 - r.c0);
    XC_CUDA(cudaGetLastError());
    XC_CUDA(cudaDeviceSynchronize());
  }
  XC_TRY(upload(p, d2->rects_host, &d2->rects));
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<int> ptr, flat;
    combine_lists_2d(N, blks, d2->rects_host, dir == 0, &ptr, &flat);
    D2Dir& D = dir == 0 ? d2->fwd : d2->adj;
    XC_TRY(upload(p, ptr, &D.comb_ptr));
    XC_TRY(upload(p, flat, &D.comb_ent));
  }
  p->matrix_bytes = d2->fwd.nnz * int64_t(sizeof(cx<T>) + sizeof(int)) + dense_elems * int64_t(sizeof(T));
  p->adjoint_bytes = d2->adj.nnz * int64_t(sizeof(cx<T>) + sizeof(int));
  return XC_OK;
}

}  // namespace

int build_plan_device(Plan* p) {
  const int64_t N = p->N;
  const unsigned gN = unsigned((N + 127) / 128);
  if (p->scheme == XC_SCHEME_2D) {
    // nodes: the equispaced nodes (functions) or the row indices (index kernels)
    p->nodes_host.resize(N);
    for (int64_t i = 0; i < N; ++i) p->nodes_host[i] = p->x0 + p->h * double(i);
    if (p->io64()) return build_plan_2d<double>(p);
    return build_plan_2d<float>(p);
  }
  XC_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->nodes_dev), size_t(N) * sizeof(double)));
  const bool user = p->params.nodes == XC_NODES_USER;
  if (p->cplx) {
    // the nodes of the complex families are angles: the arc midpoints
    // (2n + 1 - N) pi / N, the caller's angles, or the psi_j of the spectral
    // Laguerre matrix, 2 arctan(2 k_j / eta) - pi with k_j = 2 pi j / T
    if (p->family == XC_LAGUERRE_SPECTRAL) {
      p->nodes_host.resize(N);
      for (int64_t j = 0; j < N; ++j) {
        const double k = 2.0 * 3.141592653589793 * double(j) / p->params.beta;
        p->nodes_host[j] = 2.0 * std::atan(2.0 * k / p->params.alpha) - 3.141592653589793;
      }
    } else if (!user) {
      p->nodes_host.resize(N);
      for (int64_t j = 0; j < N; ++j) p->nodes_host[j] = 3.141592653589793 * double(2 * j + 1 - N) / double(N);
    }
    XC_CUDA(cudaMemcpy(p->nodes_dev, p->nodes_host.data(), size_t(N) * sizeof(double), cudaMemcpyHostToDevice));
  } else if (user) {
    XC_CUDA(cudaMemcpy(p->nodes_dev, p->nodes_host.data(), size_t(N) * sizeof(double), cudaMemcpyHostToDevice));
  } else if (is_trig(p->family)) {
    cheb_nodes_kernel<<<gN, 128>>>(N, p->nodes_dev);
  } else {
    std::vector<double> d, e2;
    jacobi_matrix(p->family, N, p->params.alpha, p->params.beta, &d, &e2);
    double lo = 1e300, hi = -1e300;  // Gershgorin interval
    for (int64_t k = 0; k < N; ++k) {
      const double r = (k > 0 ? std::sqrt(e2[k - 1]) : 0.0) + (k + 1 < N ? std::sqrt(e2[k]) : 0.0);
      lo = std::min(lo, d[k] - r);
      hi = std::max(hi, d[k] + r);
    }
    const double al = p->params.alpha, be = p->params.beta;
    if (p->family == XC_JACOBI && std::fabs(al) == 0.5 && std::fabs(be) == 0.5) {
      jacobi_half_nodes_kernel<<<gN, 128>>>(N, al, be, p->nodes_dev);
    } else {
      const double pad = 1e-3 * (hi - lo) + 1e-300;
      lo -= pad;
      hi += pad;
      const int64_t G = 4 * N;
      DevBuf dd, de, grid, counts;
      XC_TRY(alloc_tmp(&dd, d.size() * sizeof(double)));
      XC_TRY(alloc_tmp(&de, e2.size() * sizeof(double)));
      XC_TRY(alloc_tmp(&grid, size_t(G + 1) * sizeof(double)));
      XC_TRY(alloc_tmp(&counts, size_t(G + 1) * sizeof(int)));
      XC_CUDA(cudaMemcpy(dd.ptr, d.data(), d.size() * sizeof(double), cudaMemcpyHostToDevice));
      XC_CUDA(cudaMemcpy(de.ptr, e2.data(), e2.size() * sizeof(double), cudaMemcpyHostToDevice));
      const double* dp = static_cast<double*>(dd.ptr);
      const double* ep = static_cast<double*>(de.ptr);
      double* gp = static_cast<double*>(grid.ptr);
      int* cp = static_cast<int*>(counts.ptr);
      grid_count_kernel<<<unsigned((G + 128) / 128), 128>>>(dp, ep, N, lo, hi, p->family == XC_LAGUERRE_FN, G, gp,
                                                            cp);
      isolate_newton_kernel<<<gN, 128>>>(dp, ep, N, gp, cp, G, p->nodes_dev);
      XC_CUDA(cudaGetLastError());
      XC_CUDA(cudaDeviceSynchronize());
    }
    newton_kernel<<<gN, 128>>>(p->family, N, al, be, 1, p->nodes_dev);
    XC_CUDA(cudaGetLastError());
    XC_CUDA(cudaDeviceSynchronize());
  }
  XC_CUDA(cudaGetLastError());
  p->nodes_host.resize(N);
  XC_CUDA(cudaMemcpy(p->nodes_host.data(), p->nodes_dev, size_t(N) * sizeof(double), cudaMemcpyDeviceToHost));

  GenParams g{p->family, N, p->params.alpha, p->params.beta, p->nodes_dev,
              is_trig(p->family) && p->family != XC_LAGUERRE_SPECTRAL && !user, p->params.power};
  if (p->cplx) {
    const bool fp64c = p->io64();
    if (p->family == XC_LAGUERRE_SPECTRAL) {
      // row factor 1 / (eta/2 - i k_j) = (eta/2 + i k_j) / ((eta/2)^2 + k_j^2)
      std::vector<double> rf(size_t(2 * N));
      const double h = 0.5 * p->params.alpha;
      for (int64_t j = 0; j < N; ++j) {
        const double k = 2.0 * 3.141592653589793 * double(j) / p->params.beta;
        const double d = h * h + k * k;
        rf[size_t(2 * j)] = h / d;
        rf[size_t(2 * j + 1)] = k / d;
      }
      XC_TRY(plan_alloc(p, &p->rowscale, size_t(N) * 2 * p->elem_bytes()));
      if (fp64c) {
        XC_CUDA(cudaMemcpy(p->rowscale, rf.data(), rf.size() * sizeof(double), cudaMemcpyHostToDevice));
      } else {
        std::vector<float> rff(rf.begin(), rf.end());
        XC_CUDA(cudaMemcpy(p->rowscale, rff.data(), rff.size() * sizeof(float), cudaMemcpyHostToDevice));
      }
    }
    p->blocks.resize(1);
    p->nnz.assign(1, 0);
    p->stored.assign(1, 0);
    p->maxabs.assign(1, 0.0);
    if (fp64c) XC_TRY(build_block_complex<double>(p, g, p->sch.blocks[0]));
    else XC_TRY(build_block_complex<float>(p, g, p->sch.blocks[0]));
    p->spec_per_rhs = p->blocks[0].L + p->c_vpad;
    p->max_n = p->blocks[0].n;
    p->m_tail = 0;
    return XC_OK;
  }
  if (!is_trig(p->family)) {
    // recurrence coefficients for every degree the rows, weights and dense
    // comparison reach
    int64_t M = N + 2;
    for (const auto& shp : p->sch.blocks) M = std::max<int64_t>(M, int64_t(shp.L) - int64_t(shp.off));
    const std::vector<double> rc = recurrence_table(p->family, p->params.alpha, p->params.beta, M + 1);
    XC_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->rc_dev), rc.size() * sizeof(double)));
    XC_CUDA(cudaMemcpy(p->rc_dev, rc.data(), rc.size() * sizeof(double), cudaMemcpyHostToDevice));
    p->nrc = M + 1;
    g.rc = p->rc_dev;
    g.nrc = p->nrc;
  }
  const bool fp64 = p->io64();
  DevBuf lam;   // orthonormal variant: lambda_n, also the row weights of the blocks' thresholds
  if (p->normalise == XC_ORTHONORMAL) {
    XC_TRY(alloc_tmp(&lam, size_t(N) * sizeof(double)));
    XC_TRY(plan_alloc(p, &p->rowscale, size_t(N) * p->elem_bytes()));
    XC_TRY(plan_alloc(p, &p->colscale, size_t(N) * p->elem_bytes()));
    weights_kernel<<<gN, 128>>>(g, static_cast<double*>(lam.ptr));
    scales_kernel<<<gN, 128>>>(g, static_cast<double*>(lam.ptr), p->rowscale, p->colscale, fp64 ? 1 : 0);
    XC_CUDA(cudaGetLastError());
    XC_CUDA(cudaDeviceSynchronize());
    g.rw = static_cast<const double*>(lam.ptr);
  }

  const int nb = int(p->sch.blocks.size());
  p->blocks.resize(nb);
  p->hf_lo.assign(nb, {});
  p->hf_len.assign(nb, {});
  p->ht_lo.assign(nb, {});
  p->ht_len.assign(nb, {});
  p->nnz.assign(nb, 0);
  p->stored.assign(nb, 0);
  p->maxabs.assign(nb, 0.0);
  p->spec_per_rhs = 0;
  p->max_n = 0;
  for (int i = 0; i < nb; ++i) {
    if (fp64) XC_TRY(build_block<double>(p, i, g, p->sch.blocks[i]));
    else XC_TRY(build_block<float>(p, i, g, p->sch.blocks[i]));
    p->blocks[i].spec_off = p->spec_per_rhs;
    p->spec_per_rhs += p->blocks[i].H;
    if (p->blocks[i].a_csize == 1) p->max_n = std::max<int64_t>(p->max_n, p->blocks[i].n);
    p->max_csize = std::max(p->max_csize, p->blocks[i].a_csize);
  }
  // work lists for the sparse kernels (longest first); widths come back from the device
  p->nslices = (N + kSlice - 1) / kSlice;
  std::vector<int64_t> fcost(p->nslices, 0);
  std::vector<std::pair<int64_t, int>> tcost;
  int64_t gbase = 0;
  std::vector<std::vector<int>> fwidths(nb);
  for (int i = 0; i < nb; ++i) {
    std::vector<int> w(p->blocks[i].nslices), tw(p->blocks[i].tslices);
    XC_CUDA(cudaMemcpy(w.data(), p->blocks[i].f_width, w.size() * sizeof(int), cudaMemcpyDeviceToHost));
    XC_CUDA(cudaMemcpy(tw.data(), p->blocks[i].t_width, tw.size() * sizeof(int), cudaMemcpyDeviceToHost));
    fwidths[i] = w;
    for (size_t s2 = 0; s2 < w.size(); ++s2) fcost[s2] += w[s2];
    for (size_t s2 = 0; s2 < tw.size(); ++s2) tcost.push_back({tw[s2], int(gbase + int64_t(s2))});
    gbase += int64_t(tw.size());
  }
  p->total_tslices = gbase;
  // adjoint items: every bin slice cut into chunks of kAdjChunk rows (the
  // batch's items and, for plans with enough of them, the single-plan ones);
  // a plan that would give fewer than kAdjTargetChunks such chunks also gets
  // a second cut with shorter chunks (a power of two, at least kAdjChunkMin)
  // for single-plan applies, so that even one right-hand side spreads over
  // enough warps
  std::vector<int64_t> twidths(gbase, 0);
  for (const auto& tc : tcost) twidths[tc.second] = tc.first;
  auto make_chunks = [&](int chunk, std::vector<int2>* titems, std::vector<int>* cbase,
                         std::vector<int>* lens) -> int64_t {
    std::vector<std::pair<int, int2>> items;   // (rows, (g, chunk))
    cbase->assign(size_t(gbase) + 1, 0);
    int64_t run = 0;
    for (int64_t g = 0; g < gbase; ++g) {
      const int64_t W = twidths[g];
      const int64_t nch = W > 0 ? (W + chunk - 1) / chunk : 1;
      (*cbase)[g] = int(run);
      for (int64_t c = 0; c < nch; ++c)
        items.push_back({int(std::min<int64_t>(chunk, std::max<int64_t>(0, W - c * chunk))), int2{int(g), int(c)}});
      run += nch;
    }
    (*cbase)[gbase] = int(run);
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<int, int2>& a, const std::pair<int, int2>& b) { return a.first > b.first; });
    titems->resize(items.size());
    lens->resize(items.size());
    for (size_t k = 0; k < items.size(); ++k) {
      (*titems)[k] = items[k].second;
      (*lens)[k] = items[k].first;
    }
    return run;
  };
  std::vector<int2> titems;
  std::vector<int> cbase;
  p->total_chunks = make_chunks(kAdjChunk, &titems, &cbase, &p->item_len);
  p->slice_cost = fcost;
  XC_TRY(upload(p, titems, &p->t_items));
  XC_TRY(upload(p, cbase, &p->t_cbase));
  {
    int64_t rows = 0;
    for (int64_t W : twidths) rows += W;
    int chunk = kAdjChunk;
    while (chunk > kAdjChunkMin && rows / chunk < kAdjTargetChunks) chunk /= 2;
    p->s_chunk = chunk;
    if (chunk == kAdjChunk) {
      p->s_items = p->t_items;
      p->s_cbase = p->t_cbase;
      p->s_total_chunks = p->total_chunks;
    } else {
      std::vector<int2> si;
      std::vector<int> sc, sl;
      p->s_total_chunks = make_chunks(chunk, &si, &sc, &sl);
      XC_TRY(upload(p, si, &p->s_items));
      XC_TRY(upload(p, sc, &p->s_cbase));
    }
  }
  {
    int64_t gb = 0;
    for (int i = 0; i < nb; ++i) {
      p->blocks[i].t_gbase = int(gb);
      gb += p->blocks[i].tslices;
    }
  }
  // forward chunking when some slice's bands (summed over blocks) are long:
  // units (block, slice, chunk) of up to kFwdChunk rows, slice-major
  {
    int64_t longest = 0;
    for (int64_t c : fcost) longest = std::max(longest, c);
    p->fwd_chunked = longest > 2 * kFwdChunk;
    if (p->fwd_chunked) {
      std::vector<int4> units;
      std::vector<int> ubase(size_t(p->nslices) + 1, 0);
      for (int64_t s2 = 0; s2 < p->nslices; ++s2) {
        ubase[s2] = int(units.size());
        for (int i = 0; i < nb; ++i) {
          const int W = fwidths[i][s2];
          for (int c = 0; c * kFwdChunk < W; ++c)
            units.push_back(int4{i, int(s2), c, std::min(kFwdChunk, W - c * kFwdChunk)});
        }
      }
      ubase[p->nslices] = int(units.size());
      std::vector<int> uorder(units.size());
      for (size_t u = 0; u < units.size(); ++u) uorder[u] = int(u);
      std::stable_sort(uorder.begin(), uorder.end(), [&](int a, int b2) { return units[a].w > units[b2].w; });
      p->unit_len.resize(units.size());
      for (size_t u = 0; u < units.size(); ++u) p->unit_len[u] = units[uorder[u]].w;
      p->total_units = int64_t(units.size());
      XC_TRY(upload(p, units, &p->fu_units));
      XC_TRY(upload(p, uorder, &p->fu_order));
      XC_TRY(upload(p, ubase, &p->fu_ubase));
    }
  }
  std::vector<int> forder(p->nslices);
  for (int64_t s2 = 0; s2 < p->nslices; ++s2) forder[s2] = int(s2);
  std::stable_sort(forder.begin(), forder.end(), [&](int a, int b) { return fcost[a] > fcost[b]; });
  XC_TRY(upload(p, forder, &p->f_order));
  XC_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->counters), 4 * sizeof(unsigned)));
  XC_CUDA(cudaMemset(p->counters, 0, 4 * sizeof(unsigned)));

  p->m_tail = p->sch.m_tail;
  if (p->m_tail > 0) {
    XC_TRY(plan_alloc(p, &p->tail, size_t(p->m_tail) * size_t(N) * p->elem_bytes()));
    if (fp64) tail_kernel<double><<<gN, 128>>>(g, p->m_tail, static_cast<double*>(p->tail));
    else tail_kernel<float><<<gN, 128>>>(g, p->m_tail, static_cast<float*>(p->tail));
    XC_CUDA(cudaGetLastError());
    p->matrix_bytes += p->m_tail * N * int64_t(p->elem_bytes());
  }
  XC_CUDA(cudaDeviceSynchronize());
  return XC_OK;
}

// ------------------------------------------------------ lockstep layouts
// Window copy of a band layout (forward or adjoint, the same shape): slice s
// of the band layout holds value (j, lane) at off[s] + j * 32 + lane for the
// lane's rows (bins) start[s * 32 + lane] + j, j < width[s]; its window copy
// holds (w, lane) at woff[s] + w * 32 + lane for position wlo[s] + w,
// w < wlen[s], and zero where the lane's band does not reach.  One thread
// per window element.
template <typename T>
__global__ void window_copy_kernel(const cx<T>* __restrict__ val, const int* __restrict__ start,
                                   const int* __restrict__ width, const int64_t* __restrict__ off,
                                   const int* __restrict__ wlo, const int* __restrict__ wlen,
                                   const int64_t* __restrict__ woff, int nslices, cx<T>* __restrict__ out) {
  const int s = blockIdx.y;
  if (s >= nslices) return;
  const int64_t len = int64_t(wlen[s]) * kSlice;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x) {
    const int w = int(e / kSlice), lane = int(e % kSlice);
    const int j = wlo[s] + w - start[size_t(s) * kSlice + lane];
    out[woff[s] + e] = (j >= 0 && j < width[s]) ? val[off[s] + int64_t(j) * kSlice + lane] : cx<T>{T(0), T(0)};
  }
}

// Tensor-window tiles of one block (forward, FP32 plans; the layout of
// BlockDev::tw_*): blockIdx.y = row group g; element e = (tile kb, row r,
// 16-byte chunk c) of the group's tiles, chunk c = bins lo + 16 kb + 2c and
// + 1 of row 128 g + r (real, imaginary parts), stored at chunk c ^ (r & 7)
// of the tile row; zero outside the row's stored band and for rows >= N.
__global__ void tensor_tile_kernel(const cx<float>* __restrict__ fval, const int* __restrict__ fk0,
                                   const int* __restrict__ fwidth, const int64_t* __restrict__ foff, int64_t N,
                                   const int* __restrict__ glo, const int* __restrict__ gnkb,
                                   const int64_t* __restrict__ goff, float* __restrict__ out) {
  const int g = blockIdx.y;
  const int64_t total = int64_t(gnkb[g]) * 1024;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int kb = int(e >> 10), r = int(e >> 3) & 127, c = int(e & 7);
    const int64_t row = int64_t(g) * 128 + r;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < N) {
      const int64_t s = row >> 5;
      const int w = fwidth[s];
      const int j = glo[g] + 16 * kb + 2 * c - fk0[row];
      const cx<float>* base = fval + foff[s] + (row & 31);
      if (j >= 0 && j < w) {
        const cx<float> a = base[int64_t(j) * 32];
        v.x = a.re;
        v.y = a.im;
      }
      if (j + 1 >= 0 && j + 1 < w) {
        const cx<float> a = base[int64_t(j + 1) * 32];
        v.z = a.re;
        v.w = a.im;
      }
    }
    reinterpret_cast<float4*>(out + (goff[g] + kb) * 4096 + int64_t(r) * 32)[c ^ (r & 7)] = v;
  }
}

// Adjoint tensor-window tiles of one block (the layout of WinBlock, adjoint):
// blockIdx.y = bin group g; element e = (tile kb, row m, 16-byte chunk c) of
// the group's tiles, chunk c = rows lo + 32 kb + 4c .. + 3 of component m >> 6
// of bin 64 g + (m & 63), stored at chunk c ^ (m & 7); zero outside the bin's
// stored run of rows and for bins >= H.
__global__ void tensor_tile_t_kernel(const cx<float>* __restrict__ tval, const int* __restrict__ tn0,
                                     const int* __restrict__ twidth, const int64_t* __restrict__ toff, int H,
                                     const int* __restrict__ glo, const int* __restrict__ gnkb,
                                     const int64_t* __restrict__ goff, float* __restrict__ out) {
  const int g = blockIdx.y;
  const int64_t total = int64_t(gnkb[g]) * 1024;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int kb = int(e >> 10), m = int(e >> 3) & 127, c = int(e & 7);
    const int k = 64 * g + (m & 63);
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (k < H) {
      const int s = k >> 5;
      const int w = twidth[s];
      const cx<float>* base = tval + toff[s] + (k & 31);
      const int j0 = glo[g] + 32 * kb + 4 * c - tn0[k];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (j0 + i >= 0 && j0 + i < w) {
          const cx<float> a = base[int64_t(j0 + i) * 32];
          v[i] = (m >> 6) ? a.im : a.re;
        }
    }
    reinterpret_cast<float4*>(out + (goff[g] + kb) * 4096 + int64_t(m) * 32)[c ^ (m & 7)] =
        make_float4(v[0], v[1], v[2], v[3]);
  }
}

namespace {

template <typename T>
int build_lockstep(Plan* p) {
  const int nb = int(p->blocks.size());
  int64_t fstored = 0, tstored = 0, fwin = 0, twin = 0;
  for (int i = 0; i < nb; ++i) {
    fstored += p->stored[i];
    for (int v : p->hf_len[i]) fwin += int64_t(v) * kSlice;
    for (int v : p->ht_len[i]) twin += int64_t(v) * kSlice;
  }
  for (int i = 0; i < nb; ++i) {
    const BlockDev& b = p->blocks[i];
    std::vector<int> tw(b.tslices);
    XC_CUDA(cudaMemcpy(tw.data(), b.t_width, tw.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int v : tw) tstored += int64_t(v) * kSlice;
  }
  p->lock_f_ok = fstored > 0 && double(fwin) <= kLockRatio * double(fstored);
  p->lock_t_ok = tstored > 0 && double(twin) <= kLockRatio * double(tstored);
  p->lock_f_elems = p->lock_f_ok ? fwin : 0;
  p->lock_t_elems = p->lock_t_ok ? twin : 0;
  for (int i = 0; i < nb; ++i) {
    BlockDev& b = p->blocks[i];
    for (int dir = 0; dir < 2; ++dir) {
      if (!(dir == 0 ? p->lock_f_ok : p->lock_t_ok)) continue;
      const std::vector<int>& lo = dir == 0 ? p->hf_lo[i] : p->ht_lo[i];
      const std::vector<int>& len = dir == 0 ? p->hf_len[i] : p->ht_len[i];
      const int ns = int(lo.size());
      std::vector<int64_t> woff(ns, 0);
      int64_t tot = 0;
      int maxlen = 0;
      for (int s = 0; s < ns; ++s) {
        woff[s] = tot;
        tot += int64_t(len[s]) * kSlice;
        maxlen = std::max(maxlen, len[s]);
      }
      int *lo_d, *len_d;
      int64_t* off_d;
      void* val = nullptr;
      XC_TRY(upload(p, lo, &lo_d));
      XC_TRY(upload(p, len, &len_d));
      XC_TRY(upload(p, woff, &off_d));
      XC_TRY(plan_alloc(p, &val, size_t(std::max<int64_t>(tot, 1)) * sizeof(cx<T>)));
      if (maxlen > 0 && ns > 0) {
        const dim3 grid(unsigned(std::min<int64_t>((int64_t(maxlen) * kSlice + 255) / 256, 4096)), unsigned(ns));
        if (dir == 0)
          window_copy_kernel<T><<<grid, 256>>>(static_cast<const cx<T>*>(b.f_val), b.f_k0, b.f_width, b.f_off, lo_d,
                                               len_d, off_d, ns, static_cast<cx<T>*>(val));
        else
          window_copy_kernel<T><<<grid, 256>>>(static_cast<const cx<T>*>(b.t_val), b.t_n0, b.t_width, b.t_off, lo_d,
                                               len_d, off_d, ns, static_cast<cx<T>*>(val));
        XC_CUDA(cudaGetLastError());
      }
      if (dir == 0) {
        b.lf_lo = lo_d;
        b.lf_len = len_d;
        b.lf_off = off_d;
        b.lf_val = val;
      } else {
        b.lt_lo = lo_d;
        b.lt_len = len_d;
        b.lt_off = off_d;
        b.lt_val = val;
      }
    }
  }
  // forward units over the windows (plans with long bands): per slice, per
  // block, window positions cut into pieces of kFwdChunk; slice-major
  if (p->lock_f_ok && p->fwd_chunked) {
    std::vector<int4> units;
    std::vector<int> ubase(size_t(p->nslices) + 1, 0);
    for (int64_t s2 = 0; s2 < p->nslices; ++s2) {
      ubase[s2] = int(units.size());
      for (int i = 0; i < nb; ++i) {
        const int W = s2 < int64_t(p->hf_len[i].size()) ? p->hf_len[i][s2] : 0;
        for (int c = 0; c * kFwdChunk < W; ++c)
          units.push_back(int4{i, int(s2), c * kFwdChunk, std::min(kFwdChunk, W - c * kFwdChunk)});
      }
    }
    ubase[p->nslices] = int(units.size());
    p->lk_total_units = int64_t(units.size());
    p->lk_unit_len.resize(units.size());
    for (size_t u = 0; u < units.size(); ++u) p->lk_unit_len[u] = units[u].w;
    XC_TRY(upload(p, units, &p->lk_units));
    XC_TRY(upload(p, ubase, &p->lk_ubase));
  }
  // adjoint chunks over the windows: (global bin slice, chunk of kAdjChunk rows)
  if (p->lock_t_ok) {
    std::vector<int2> items;
    std::vector<int> cbase(size_t(p->total_tslices) + 1, 0);
    int64_t run = 0, g = 0;
    p->lk_item_len.clear();
    for (int i = 0; i < nb; ++i)
      for (size_t s2 = 0; s2 < p->ht_len[i].size(); ++s2, ++g) {
        const int W = p->ht_len[i][s2];
        const int nch = W > 0 ? (W + kAdjChunk - 1) / kAdjChunk : 1;
        cbase[g] = int(run);
        for (int c = 0; c < nch; ++c) {
          items.push_back(int2{int(g), c});
          p->lk_item_len.push_back(std::min(kAdjChunk, std::max(0, W - c * kAdjChunk)));
        }
        run += nch;
      }
    cbase[g] = int(run);
    p->lk_total_chunks = run;
    XC_TRY(upload(p, items, &p->lk_items));
    XC_TRY(upload(p, cbase, &p->lk_cbase));
  }
  // tensor windows (forward, XC_FP32 plans): row group g = slices 4g .. 4g+3,
  // window = the union of their slice windows, rounded up to whole tiles
  if constexpr (sizeof(T) == 4) {
    if (p->precision == XC_FP32 && fstored > 0) {
      const int64_t groups = (p->N + 127) / 128;
      std::vector<std::vector<int>> glo(nb, std::vector<int>(groups, 0)), gnkb(nb, std::vector<int>(groups, 0));
      int64_t tiles = 0;
      for (int i = 0; i < nb; ++i)
        for (int64_t g = 0; g < groups; ++g) {
          int lo = INT_MAX, hi = -1;
          for (int64_t s = 4 * g; s < std::min<int64_t>(4 * g + 4, int64_t(p->hf_len[i].size())); ++s)
            if (p->hf_len[i][s] > 0) {
              lo = std::min(lo, p->hf_lo[i][s]);
              hi = std::max(hi, p->hf_lo[i][s] + p->hf_len[i][s]);
            }
          if (hi > lo) {
            glo[i][g] = lo;
            gnkb[i][g] = (hi - lo + 15) / 16;
            tiles += gnkb[i][g];
          }
        }
      const int64_t elems = tiles * 128 * 16;
      p->tens_ok = double(elems) <= kTensorRatio * double(fstored);
      p->tens_elems = p->tens_ok ? elems : 0;
      p->tens_groups = p->tens_ok ? groups : 0;
      if (p->tens_ok) {
        p->tw_nkb_h = gnkb;
        std::vector<WinBlock> wb(nb);
        void* val = nullptr;
        XC_TRY(plan_alloc(p, &val, size_t(std::max<int64_t>(tiles, 1)) * 4096 * sizeof(float)));
        int64_t t0 = 0;
        for (int i = 0; i < nb; ++i) {
          BlockDev& b = p->blocks[i];
          std::vector<int64_t> goff(groups, 0);
          int maxk = 0;
          for (int64_t g = 0; g < groups; ++g) {
            goff[g] = t0;
            t0 += gnkb[i][g];
            maxk = std::max(maxk, gnkb[i][g]);
          }
          int *lo_d, *nkb_d;
          int64_t* off_d;
          XC_TRY(upload(p, glo[i], &lo_d));
          XC_TRY(upload(p, gnkb[i], &nkb_d));
          XC_TRY(upload(p, goff, &off_d));
          if (maxk > 0) {
            const dim3 grid(unsigned(std::min<int64_t>((int64_t(maxk) * 1024 + 255) / 256, 4096)), unsigned(groups));
            tensor_tile_kernel<<<grid, 256>>>(static_cast<const cx<float>*>(b.f_val), b.f_k0, b.f_width, b.f_off,
                                              p->N, lo_d, nkb_d, off_d, static_cast<float*>(val));
            XC_CUDA(cudaGetLastError());
          }
          wb[i] = WinBlock{lo_d, nkb_d, off_d, static_cast<const float*>(val), b.spec_off, b.t_gbase, b.tslices};
        }
        XC_TRY(upload(p, wb, &p->win_blocks));
      }
    }
    // adjoint: bin group g of a block = bin slices 2g, 2g + 1, window = the
    // union of their row runs, rounded up to whole tiles of 32 rows
    if (p->precision == XC_FP32 && tstored > 0) {
      std::vector<std::vector<int>> glo(nb), gnkb(nb);
      int64_t tiles = 0;
      for (int i = 0; i < nb; ++i) {
        const int64_t ts = int64_t(p->ht_len[i].size());
        const int64_t groups = (ts + 1) / 2;
        glo[i].assign(groups, 0);
        gnkb[i].assign(groups, 0);
        for (int64_t g = 0; g < groups; ++g) {
          int lo = INT_MAX, hi = -1;
          for (int64_t s = 2 * g; s < std::min<int64_t>(2 * g + 2, ts); ++s)
            if (p->ht_len[i][s] > 0) {
              lo = std::min(lo, p->ht_lo[i][s]);
              hi = std::max(hi, p->ht_lo[i][s] + p->ht_len[i][s]);
            }
          if (hi > lo) {
            glo[i][g] = lo;
            gnkb[i][g] = (hi - lo + 31) / 32;
            tiles += gnkb[i][g];
          }
        }
      }
      const int64_t elems = tiles * 64 * 32;   // complex values per tile: 64 bins x 32 rows
      p->tens_t_ok = double(elems) <= kTensorRatio * double(tstored);
      p->tens_t_elems = p->tens_t_ok ? elems : 0;
      if (p->tens_t_ok) {
        p->tw_t_nkb_h = gnkb;
        std::vector<WinBlock> wb(nb);
        void* val = nullptr;
        XC_TRY(plan_alloc(p, &val, size_t(std::max<int64_t>(tiles, 1)) * 4096 * sizeof(float)));
        int64_t t0 = 0;
        for (int i = 0; i < nb; ++i) {
          const BlockDev& b = p->blocks[i];
          const int64_t groups = int64_t(glo[i].size());
          std::vector<int64_t> goff(std::max<int64_t>(groups, 1), 0);
          int maxk = 0;
          for (int64_t g = 0; g < groups; ++g) {
            goff[g] = t0;
            t0 += gnkb[i][g];
            maxk = std::max(maxk, gnkb[i][g]);
          }
          int *lo_d, *nkb_d;
          int64_t* off_d;
          XC_TRY(upload(p, glo[i], &lo_d));
          XC_TRY(upload(p, gnkb[i], &nkb_d));
          XC_TRY(upload(p, goff, &off_d));
          if (maxk > 0) {
            const dim3 grid(unsigned(std::min<int64_t>((int64_t(maxk) * 1024 + 255) / 256, 4096)), unsigned(groups));
            tensor_tile_t_kernel<<<grid, 256>>>(static_cast<const cx<float>*>(b.t_val), b.t_n0, b.t_width, b.t_off,
                                                b.H, lo_d, nkb_d, off_d, static_cast<float*>(val));
            XC_CUDA(cudaGetLastError());
          }
          wb[i] = WinBlock{lo_d, nkb_d, off_d, static_cast<const float*>(val), 0, b.t_gbase, b.tslices};
        }
        XC_TRY(upload(p, wb, &p->win_blocks_t));
        std::vector<int> cb(size_t(p->total_tslices) + 1);
        for (size_t i = 0; i < cb.size(); ++i) cb[i] = int(i);
        XC_TRY(upload(p, cb, &p->tw_tcbase));
      }
    }
  }
  XC_CUDA(cudaDeviceSynchronize());
  return XC_OK;
}

}  // namespace

int ensure_lockstep(Plan* p) {
  if (p->lock_built) return XC_OK;
  if (p->cplx || p->d2 || p->blocks.empty()) {
    p->lock_built = true;
    return XC_OK;
  }
  if (p->io64()) XC_TRY(build_lockstep<double>(p));
  else XC_TRY(build_lockstep<float>(p));
  if (p->scratch_desc)
    XC_CUDA(cudaMemcpy(p->scratch_desc, p->blocks.data(), p->blocks.size() * sizeof(BlockDev), cudaMemcpyHostToDevice));
  p->lock_built = true;
  return XC_OK;
}

}  // namespace xc
