"""Window, parameter selection and block schedule of the extra-component method.

Test infrastructure only (see the package docstring).  All arithmetic in FP64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------- Bessel I0/I1

def bessel_i0(z):
    """Modified Bessel function I0 by its defining power series
    I0(z) = sum_k (z^2/4)^k / (k!)^2 (Section 2.1, Kaiser window definition).

    Works elementwise on arrays; terms are summed until they no longer change
    the FP64 sum.  All terms are positive, so there is no cancellation.
    """
    z = np.asarray(z, dtype=np.float64)
    q = 0.25 * z * z
    term = np.ones_like(z)
    total = np.ones_like(z)
    k = 0
    while True:
        k += 1
        term = term * q / (k * k)
        total = total + term
        if np.all(term <= 1e-18 * total) or k > 2000:
            break
    return total


def bessel_i1(z):
    """I1(z) = sum_k (z/2)^(2k+1) / (k! (k+1)!), the derivative of I0."""
    z = np.asarray(z, dtype=np.float64)
    q = 0.25 * z * z
    term = 0.5 * z
    total = term.copy()
    k = 0
    while True:
        k += 1
        term = term * q / (k * (k + 1))
        total = total + term
        if np.all(np.abs(term) <= 1e-18 * np.abs(total) + 1e-300) or k > 2000:
            break
    return total


# -------------------------------------------------------------- Kaiser window

def kaiser_value(j, length: int, zeta: float):
    """Kaiser window value w_j^{zeta, length-1} (Section 2.1):

        w_n^{zeta,N} = I0(zeta * sqrt(1 - (2n/N - 1)^2)) / I0(zeta),  0 <= n <= N,

    evaluated with N = length - 1 so that a window of `length` samples has both
    end points equal to 1/I0(zeta).  (Reading: the paper's W_M is (M+1)x(M+1)
    for an (M+1)-column matrix, so an L-column block uses w^{zeta, L-1}.)
    """
    j = np.asarray(j, dtype=np.float64)
    t = 2.0 * j / (length - 1) - 1.0
    arg = np.sqrt(np.maximum(0.0, 1.0 - t * t))
    return bessel_i0(zeta * arg) / bessel_i0(zeta)


def kaiser_window(length: int, zeta: float) -> np.ndarray:
    """The full window (w_0, ..., w_{length-1}) of the diagonal matrix W."""
    return kaiser_value(np.arange(length), length, zeta)


# ------------------------------------------------------------ zeta(eps1)

def zeta_of_eps(eps1: float, zeta0: float = 50.0) -> float:
    """Kaiser shape parameter zeta(eps1) solving 1/I0(zeta) = eps1 by Newton's
    method from the initial guess zeta0 = 50 (Section 2.2, text after eq. (Fe2)).

    Reading: Newton is applied to the equivalent form I0(zeta) - 1/eps1 = 0,
    which is convex and increasing, so the iteration started to the right of the
    root (zeta0 = 50) decreases monotonically to it.  (The literal form
    1/I0(zeta) - eps1 diverges from zeta0 = 50.)
    """
    if not (0.0 < eps1 < 1.0):
        raise ValueError("eps1 must lie in (0, 1)")
    target = 1.0 / eps1
    z = float(zeta0)
    for _ in range(500):
        f = float(bessel_i0(z)) - target
        step = f / float(bessel_i1(z))
        z_new = z - step
        if z_new <= 0.0:
            z_new = 0.5 * z
        if abs(z_new - z) <= 1e-15 * abs(z):
            z = z_new
            break
        z = z_new
    return z


# ------------------------------------------------------------ s(eps2, zeta)

def extra_count(m: int, zeta: float, eps2: float, two_sided: bool) -> int:
    """Smallest number s >= 1 of extra components whose first real component
    keeps a window value of at least eps2 (Section 2.2: s is found by a
    sequential search over s = 1, 2, 3, ...).

    Reading of the garbled inequality: the paper asks for the smallest s with
    "w_s^{zeta,M+2s} < eps2", which s = 1 satisfies trivially; the reading
    used here is w_s^{zeta, L-1} >= eps2, i.e. the division by W^{-1} amplifies
    no real component by more than 1/eps2.  The window length L is M + 2s for
    the two-sided extension (Algorithms 1-2) and m + s for a block of the block
    method, which is extended on the right only (Section 3).
    """
    s = 1
    while True:
        length = m + 2 * s if two_sided else m + s
        if kaiser_value(s, length, zeta) >= eps2:
            return s
        s += 1
        if s > 50 * m + 100:
            raise RuntimeError("no extra-component count satisfies eps2")


# ------------------------------------------------------- FFT-friendly lengths

def is_fft_friendly(length: int) -> bool:
    """Lengths the implementation accepts for its FFTs: even, at least 8, and
    length/2 a product of 2, 3, 5 and 7 only.  (Section 5.1 asks for an
    extended size whose FFT is fast; this is the build's choice of such sizes.)
    """
    if length < 8 or length % 2:
        return False
    n = length // 2
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def fft_friendly_at_least(length: int) -> int:
    """Smallest FFT-friendly length >= `length` (s is enlarged to reach it;
    Section 5.1 notes a slightly larger s only costs a few extra components)."""
    n = max(int(length), 8)
    while not is_fft_friendly(n):
        n += 1
    return n


# ------------------------------------------------------------ block schedule

@dataclass
class Block:
    """One compressed block.  Extended column j (0 <= j < L) holds the matrix
    column m = j - off; the real input occupies j in [j_lo, j_hi), the rest of
    the extended vector is zero (eqs. (Fe1), (Fe3))."""
    L: int
    off: int
    j_lo: int
    j_hi: int


@dataclass
class Schedule:
    zeta: float
    eps1: float          # threshold (0 means: keep every element)
    eps_window: float    # the eps that fixed zeta
    eps2: float
    blocks: list = field(default_factory=list)
    m_tail: int = 0      # dense tail columns [0, m_tail)


def schedule(N: int, eps: float, eps2: float, two_sided: bool,
             eps_window: float = 0.0, tail_max: int = 20) -> Schedule:
    """Parameters and blocks for an N-column matrix (Algorithms 1-4).

    * zeta from eps1 = eps (or eps_window, default 1e-14, when eps == 0, in
      which case nothing is thresholded).
    * Two-sided (trigonometric rows, Algorithm 1/2): one block of length
      L = N + 2s rounded up to an FFT-friendly size; the left pad is
      s = (L - N) // 2, the right pad L - N - s >= s; if rounding left the
      floor w_s >= eps2 unmet (odd L - N), the next friendly size is taken.
    * One-sided (orthogonal polynomials and functions, Algorithms 3/4,
      Section 3): block i covers columns [0, m_i) extended on the right to
      L_i = m_i + s_i columns; its first s_i inputs are zeroed and the next
      block covers columns [0, s_i).  Blocks are added while m_i > tail_max;
      the remaining m_tail columns are multiplied directly (Section 3, last
      step, a direct product).  Reading: tail_max = 20 reproduces the
      number of blocks in Table 1.
    """
    ew = eps if eps > 0 else (eps_window if eps_window > 0 else 1e-14)
    z = zeta_of_eps(ew)
    sch = Schedule(zeta=z, eps1=eps, eps_window=ew, eps2=eps2)
    if two_sided:
        s = extra_count(N, z, eps2, True)
        L = fft_friendly_at_least(N + 2 * s)
        left = (L - N) // 2
        # with odd L - N the left pad can stay at s while L grew by one, which
        # lowers w_s; move to the next friendly size until the floor holds
        while kaiser_value(left, L, z) < eps2:
            L = fft_friendly_at_least(L + 1)
            left = (L - N) // 2
        sch.blocks.append(Block(L=L, off=left, j_lo=left, j_hi=left + N))
        sch.m_tail = 0
        return sch
    m = N
    while m > tail_max:
        s = extra_count(m, z, eps2, False)
        if s >= m:
            break
        L = fft_friendly_at_least(m + s)
        s = L - m
        if s >= m:
            break
        sch.blocks.append(Block(L=L, off=0, j_lo=s, j_hi=m))
        m = s
    sch.m_tail = m
    return sch
