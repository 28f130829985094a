// Host side of the precomputation stage, step 1.1 of Algorithms 1-4:
// zeta(eps1) by Newton's method, the extra-component counts s(eps2, zeta), the
// FFT-friendly block lengths and the block schedule of the block method
// (Section 3).  Only scalars and a handful of integers are computed here; the
// matrices themselves are built on the device (xc_plan.cu).
#include <cmath>
#include <string>

#include "xc_internal.h"

namespace xc {

// I0 by its power series sum_k (z^2/4)^k / (k!)^2 (Kaiser window, Section 2.1).
double bessel_i0_host(double z) {
  const double q = 0.25 * z * z;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 4000; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

static double bessel_i1_host(double z) {
  const double q = 0.25 * z * z;
  double term = 0.5 * z, sum = term;
  for (int k = 1; k < 4000; ++k) {
    term *= q / (double(k) * double(k + 1));
    sum += term;
    if (std::fabs(term) <= 1e-18 * std::fabs(sum)) break;
  }
  return sum;
}

// Window value w_j^{zeta, length-1}: a window of `length` samples whose end
// points equal 1/I0(zeta).
double kaiser_value_host(double j, int64_t length, double zeta) {
  const double t = 2.0 * j / double(length - 1) - 1.0;
  const double a = std::sqrt(std::fmax(0.0, 1.0 - t * t));
  return bessel_i0_host(zeta * a) / bessel_i0_host(zeta);
}

// Newton's method on I0(zeta) - 1/eps1 = 0 started at zeta0 = 50 (Section 2.2).
// The function is convex and increasing, so the iterates decrease
// monotonically to the root from the right.
double zeta_of_eps_host(double eps1) {
  const double target = 1.0 / eps1;
  double z = 50.0;
  for (int it = 0; it < 500; ++it) {
    double zn = z - (bessel_i0_host(z) - target) / bessel_i1_host(z);
    if (zn <= 0.0) zn = 0.5 * z;
    if (std::fabs(zn - z) <= 1e-15 * std::fabs(z)) return zn;
    z = zn;
  }
  return z;
}

// FFT-friendly: even, >= 8, and length/2 = 2^a 3^b 5^c 7^d.
bool is_fft_friendly(int64_t length) {
  if (length < 8 || (length & 1)) return false;
  int64_t n = length / 2;
  for (int64_t p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

int64_t fft_friendly_at_least(int64_t length) {
  int64_t n = length < 8 ? 8 : length;
  while (!is_fft_friendly(n)) ++n;
  return n;
}

int fft_radices(int64_t n, int* radix) {
  int p = 0;
  // odd radices first, then the powers of two as radix-8/4/2 passes
  for (int r : {7, 5, 3}) {
    while (n % r == 0) {
      if (p >= kMaxPasses) return -1;
      radix[p++] = r;
      n /= r;
    }
  }
  for (int r : {8, 4, 2}) {
    while (n % r == 0) {
      if (p >= kMaxPasses) return -1;
      radix[p++] = r;
      n /= r;
    }
  }
  return n == 1 ? p : -1;
}

// Smallest s >= 1 with w_s^{zeta, L-1} >= eps2, L = m + 2s (two-sided) or m + s
// (one-sided): the extra components keep the window of every real component
// at eps2 or above (Section 2.2, sequential search over s).
int64_t extra_count(int64_t m, double zeta, double eps2, bool two_sided) {
  for (int64_t s = 1; s <= 50 * m + 100; ++s) {
    const int64_t length = two_sided ? m + 2 * s : m + s;
    if (kaiser_value_host(double(s), length, zeta) >= eps2) return s;
  }
  return -1;
}

int make_schedule(int64_t N, double eps, double eps2, bool two_sided, double eps_window,
                  int tail_max, Schedule* out) {
  Schedule sch;
  sch.eps_window = eps > 0 ? eps : (eps_window > 0 ? eps_window : 1e-14);
  if (!(sch.eps_window < 1.0)) return fail(XC_ERR_ARG, "eps (or eps_window) must be < 1");
  sch.zeta = zeta_of_eps_host(sch.eps_window);
  if (two_sided) {
    const int64_t s = extra_count(N, sch.zeta, eps2, true);
    if (s < 0) return fail(XC_ERR_ARG, "no extra-component count meets eps2");
    int64_t L = fft_friendly_at_least(N + 2 * s);
    int64_t left = (L - N) / 2;
    // odd L - N can leave the left pad at s while L grew: re-check the floor
    while (kaiser_value_host(double(left), L, sch.zeta) < eps2) {
      L = fft_friendly_at_least(L + 1);
      left = (L - N) / 2;
    }
    sch.blocks.push_back({L, left, left, left + N});
    sch.m_tail = 0;
  } else {
    int64_t m = N;
    while (m > tail_max) {
      int64_t s = extra_count(m, sch.zeta, eps2, false);
      if (s < 0 || s >= m) break;
      const int64_t L = fft_friendly_at_least(m + s);
      s = L - m;
      if (s >= m) break;
      sch.blocks.push_back({L, 0, s, m});
      m = s;
    }
    sch.m_tail = m;
  }
  if (sch.blocks.size() > XC_MAX_BLOCKS) return fail(XC_ERR_UNSUPPORTED, "more than XC_MAX_BLOCKS blocks");
  *out = sch;
  return XC_OK;
}

}  // namespace xc
