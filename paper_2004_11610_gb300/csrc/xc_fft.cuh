// Shared-memory FFT building blocks for libxc (device code).
//
// The transform of every block is the unitary DFT of eq. (fourier); the real
// inputs of the method (Section 5.1: the matrix rows and the vectors are real)
// are handled as an n = L/2 point complex FFT of the packed sequence
// z_j = u_{2j} + i u_{2j+1} followed by the standard even/odd split.
//
// The complex FFT is an in-place mixed-radix decimation-in-time transform in
// shared memory: inputs are written in digit-reversed order (a per-length
// permutation table), then pass q combines r_q sub-transforms of length
// m_{q-1} = r_1 ... r_{q-1}.  One thread owns one radix-r butterfly of a pass,
// so a pass needs no synchronisation inside it, only a barrier between passes.
#pragma once

#include <cuda_runtime.h>

namespace xc {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {  // a * conj(b)
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> scal(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> mul_mi(cx<T> a) { return {a.im, -a.re}; }   // -i * a
template <typename T>
__device__ __forceinline__ cx<T> mul_pi(cx<T> a) { return {-a.im, a.re}; }   // +i * a

// cos / sin of 2 pi k / R for the odd-radix kernels (k = 0..R-1).
template <int R> struct RootTable;
template <> struct RootTable<3> {
  static __device__ __forceinline__ double c(int k) { return k == 0 ? 1.0 : -0.5; }
  static __device__ __forceinline__ double s(int k) {
    return k == 0 ? 0.0 : (k == 1 ? 0.8660254037844386467637 : -0.8660254037844386467637);
  }
};
template <> struct RootTable<5> {
  static __device__ __forceinline__ double c(int k) {
    const double v[5] = {1.0, 0.3090169943749474241023, -0.8090169943749474241023,
                         -0.8090169943749474241023, 0.3090169943749474241023};
    return v[k];
  }
  static __device__ __forceinline__ double s(int k) {
    const double v[5] = {0.0, 0.9510565162951535721164, 0.5877852522924731291687,
                         -0.5877852522924731291687, -0.9510565162951535721164};
    return v[k];
  }
};
template <> struct RootTable<7> {
  static __device__ __forceinline__ double c(int k) {
    const double v[7] = {1.0, 0.623489801858733530525, -0.2225209339563144042889,
                         -0.9009688679024191262361, -0.9009688679024191262361,
                         -0.2225209339563144042889, 0.623489801858733530525};
    return v[k];
  }
  static __device__ __forceinline__ double s(int k) {
    const double v[7] = {0.0, 0.7818314824680298087084, 0.9749279121818236070181,
                         0.4338837391175581204758, -0.4338837391175581204758,
                         -0.9749279121818236070181, -0.7818314824680298087084};
    return v[k];
  }
};

// Forward DFT of odd size R (exp(-2 pi i k t / R)) on a[0..R-1], in place.
template <int R, typename T>
__device__ __forceinline__ void dft_odd(cx<T>* a) {
  constexpr int H = (R - 1) / 2;
  cx<T> S[H], D[H];
#pragma unroll
  for (int t = 1; t <= H; ++t) {
    S[t - 1] = a[t] + a[R - t];
    D[t - 1] = a[t] - a[R - t];
  }
  cx<T> y0 = a[0];
#pragma unroll
  for (int t = 0; t < H; ++t) y0 = y0 + S[t];
  cx<T> out[R];
  out[0] = y0;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    cx<T> P = a[0], Q = mk<T>(T(0), T(0));
#pragma unroll
    for (int t = 1; t <= H; ++t) {
      const int kt = (k * t) % R;
      const T c = T(RootTable<R>::c(kt)), s = T(RootTable<R>::s(kt));
      P = P + scal(c, S[t - 1]);
      Q = Q + scal(s, D[t - 1]);
    }
    out[k] = P + mul_mi(Q);       // P - i Q
    out[R - k] = P + mul_pi(Q);   // P + i Q
  }
#pragma unroll
  for (int k = 0; k < R; ++k) a[k] = out[k];
}

template <typename T>
__device__ __forceinline__ void dft2(cx<T>* a) {
  const cx<T> t = a[0] - a[1];
  a[0] = a[0] + a[1];
  a[1] = t;
}

template <typename T>
__device__ __forceinline__ void dft4(cx<T>& a0, cx<T>& a1, cx<T>& a2, cx<T>& a3) {
  const cx<T> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = a1 - a3;
  a0 = t0 + t2;
  a2 = t0 - t2;
  a1 = t1 + mul_mi(t3);
  a3 = t1 + mul_pi(t3);
}

template <typename T>
__device__ __forceinline__ void dft8(cx<T>* a) {
  cx<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  cx<T> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const T h = T(0.7071067811865475244008);
  const cx<T> w1 = {h * (o1.re + o1.im), h * (o1.im - o1.re)};   // exp(-i pi/4) o1
  const cx<T> w2 = mul_mi(o2);                                    // exp(-i pi/2) o2
  const cx<T> w3 = {h * (o3.im - o3.re), -h * (o3.re + o3.im)};   // exp(-3 i pi/4) o3
  a[0] = e0 + o0;
  a[4] = e0 - o0;
  a[1] = e1 + w1;
  a[5] = e1 - w1;
  a[2] = e2 + w2;
  a[6] = e2 - w2;
  a[3] = e3 + w3;
  a[7] = e3 - w3;
}

template <int R, typename T>
__device__ __forceinline__ void dft_small(cx<T>* a) {
  if constexpr (R == 2) dft2(a);
  else if constexpr (R == 4) dft4(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 8) dft8(a);
  else dft_odd<R, T>(a);
}

// Element access for the FFT passes: the array lives either in this CTA's
// shared memory, or spread over the shared memories of a thread-block cluster
// (rank r holds elements [r*per, (r+1)*per)), reached through distributed
// shared memory.
template <typename T>
struct LocalMem {
  cx<T>* s;
  __device__ __forceinline__ cx<T>& at(int e) const { return s[e]; }
};

template <typename T>
struct ClusterMem {
  cx<T>* base[8];
  int per;
  __device__ __forceinline__ cx<T>& at(int e) const {
    const int r = e / per;
    return base[r][e - r * per];
  }
};

// One radix-R pass over the n-point array (in place).  tw is the length-L
// table exp(-2 pi i k / L) with L = 2n; the twiddle exp(-2 pi i k t / m) of
// sub-length m is tw[2 k t (n/m)].
template <int R, typename T, class M>
__device__ __forceinline__ void fft_pass(const M& mem, int n, int m_prev, const cx<T>* __restrict__ tw, int tid,
                                         int nthreads) {
  const int m = m_prev * R;
  const int nbf = n / R;
  const int tw_step = 2 * (n / m);
  for (int w = tid; w < nbf; w += nthreads) {
    const int k = w % m_prev;
    const int base = (w / m_prev) * m + k;
    cx<T> a[R];
#pragma unroll
    for (int t = 0; t < R; ++t) a[t] = mem.at(base + t * m_prev);
    if (m_prev > 1) {
#pragma unroll
      for (int t = 1; t < R; ++t) a[t] = cmul(a[t], tw[k * t * tw_step]);
    }
    dft_small<R, T>(a);
#pragma unroll
    for (int t = 0; t < R; ++t) mem.at(base + t * m_prev) = a[t];
  }
}

// All passes of the in-place forward FFT (exp(-2 pi i jk/n)) of digit-reversed
// data; `sync` is the barrier between passes (CTA or cluster) and ends the run.
template <typename T, class M, class Sync>
__device__ void fft_run(const M& mem, int n, int p, const int* radix, const cx<T>* __restrict__ tw, int tid,
                        int nthreads, Sync sync) {
  int m_prev = 1;
  for (int q = 0; q < p; ++q) {
    const int r = radix[q];
    switch (r) {
      case 2: fft_pass<2, T>(mem, n, m_prev, tw, tid, nthreads); break;
      case 3: fft_pass<3, T>(mem, n, m_prev, tw, tid, nthreads); break;
      case 4: fft_pass<4, T>(mem, n, m_prev, tw, tid, nthreads); break;
      case 5: fft_pass<5, T>(mem, n, m_prev, tw, tid, nthreads); break;
      case 7: fft_pass<7, T>(mem, n, m_prev, tw, tid, nthreads); break;
      default: fft_pass<8, T>(mem, n, m_prev, tw, tid, nthreads); break;
    }
    m_prev *= r;
    sync();
  }
}

// In-place FFT in this CTA's shared memory.  Ends with a barrier.
template <typename T>
__device__ void fft_inplace(cx<T>* s, int n, int p, const int* radix, const cx<T>* __restrict__ tw, int tid,
                            int nthreads) {
  fft_run<T>(LocalMem<T>{s}, n, p, radix, tw, tid, nthreads, [] { __syncthreads(); });
}

// Even/odd split after the packed FFT: from Z = FFT_n(u_even + i u_odd) give
// the half spectrum U_k = sum_j u_j exp(-2 pi i jk / L), k = 0..n, as the pair
// (U_k, U_{n-k}) for 0 <= k <= n/2.  For k = 0 the second value is U_n.
template <typename T>
__device__ __forceinline__ void r2c_split_vals(cx<T> Zk, cx<T> Znk, int k, const cx<T>* __restrict__ tw, cx<T>* Uk,
                                               cx<T>* Unk) {
  const T half = T(0.5);
  const cx<T> E = scal(half, Zk + conj(Znk));
  const cx<T> O = scal(half, mul_mi(Zk - conj(Znk)));   // (Zk - conj Znk) / (2i)
  const cx<T> P = cmul(tw[k], O);
  *Uk = E + P;
  *Unk = conj(E - P);
}

template <typename T>
__device__ __forceinline__ void r2c_split(const cx<T>* s, int n, int k, const cx<T>* __restrict__ tw, cx<T>* Uk,
                                          cx<T>* Unk) {
  r2c_split_vals(s[k], s[k == 0 ? 0 : n - k], k, tw, Uk, Unk);
}

// Inverse of r2c_split up to the packing: from a half spectrum U_0..U_n
// (imaginary parts of U_0, U_n ignored) give Z_k and Z_{n-k} with
// sum_k Z_k exp(+2 pi i jk / n) = u_{2j} + i u_{2j+1}, where
// u_j = Re sum_{k=0..n} c_k U_k exp(2 pi i jk / L), c_0 = c_n = 1, c_k = 2 else.
template <typename T>
__device__ __forceinline__ void c2r_merge(cx<T> Uk, cx<T> Unk, int k, const cx<T>* __restrict__ tw,
                                          cx<T>* Zk, cx<T>* Znk) {
  const cx<T> A = Uk + conj(Unk);
  const cx<T> B = Uk - conj(Unk);
  const cx<T> Q = cmulc(B, tw[k]);   // exp(+2 pi i k / L) * B
  *Zk = A + mul_pi(Q);
  *Znk = conj(A) + mul_pi(conj(Q));
}

}  // namespace xc
