"""Special-function families: nodes, quadrature weights and matrix entries.

Test infrastructure only (see the package docstring).  FP64 throughout; where
an intermediate value leaves the FP64 exponent range (Laguerre functions at
large nodes, Hermite functions far from the origin) the three-term recurrence
carries an explicit power-of-two exponent per node, and the initial values
exp(-x/2), exp(-x^2/2) are evaluated with mpmath at 40 digits.

Matrix convention (eqs. (cheb_matrix), (Jac_matrix)): A[n, m] = phi_m(x_n),
row n = node, column m = degree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import mpmath
import numpy as np
import scipy.linalg
from scipy.special import gammaln

FAMILIES = ("chebyshev", "legendre", "jacobi", "laguerre", "hermite", "sine", "cospow", "exp", "lagspec")
ONE_SIDED = ("legendre", "jacobi", "laguerre", "hermite")
# trigonometric families, all at the angles theta_n of the Chebyshev-Gauss
# points: cos(m theta_n) (Chebyshev T), sin(m theta_n) (Section 2.2 names the
# sin and exp matrices beside eq. (cheb_matrix)) and cos^s(m theta_n)
# (eq. (cosd2)); all are defined for negative m and take the two-sided extension
TRIG = ("chebyshev", "sine", "cospow")
# complex families (complex matrix, complex vectors): exp(i m theta_n) at
# angles theta_n (the nodes are the angles themselves), and the spectral
# Laguerre matrix C of eq. (lag_matrix), C[j, m] = exp(i m psi_j) / (eta/2 -
# i k_j), k_j = 2 pi j / T, whose exp part is an exp matrix at the angles psi_j
# and whose 1 / (eta/2 - i k_j) is a row factor outside the compression
# (Section 4: Algorithms 1 and 2 apply to the exp elements unchanged).  Both
# are defined for negative m: two-sided extension.
COMPLEX = ("exp", "lagspec")
TWO_SIDED = TRIG + COMPLEX


@dataclass
class Spec:
    """A family at a node set.  For the Chebyshev family at its default
    Chebyshev-Gauss points the angles theta_n = (2n+1) pi / (2N) are kept as
    exact rationals (`cheb_num` / `cheb_den`) so that cos(m theta_n) can be
    reduced exactly."""
    family: str
    N: int
    x: np.ndarray
    alpha: float = 0.0
    beta: float = 0.0
    cheb_num: np.ndarray | None = None
    cheb_den: int = 0
    power: int = 2            # s of the cos^s family

    @property
    def is_complex(self) -> bool:
        return self.family in COMPLEX


# ------------------------------------------------------------------ recurrences

def _legendre_rows(x, m_hi):
    """P_m(x_n), m in [0, m_hi): (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}."""
    out = np.empty((x.size, m_hi))
    p_prev = np.ones_like(x)
    out[:, 0] = p_prev
    if m_hi == 1:
        return out
    p = x.copy()
    out[:, 1] = p
    for m in range(1, m_hi - 1):
        p_next = ((2 * m + 1) * x * p - m * p_prev) / (m + 1)
        p_prev, p = p, p_next
        out[:, m + 1] = p
    return out


def _jacobi_coeffs(m, a, b):
    """Coefficients of 2(m+1)(m+a+b+1)(2m+a+b) P_{m+1}
    = (2m+a+b+1)[(2m+a+b+2)(2m+a+b) x + a^2 - b^2] P_m - 2(m+a)(m+b)(2m+a+b+2) P_{m-1}."""
    c = 2 * m + a + b
    a1 = 2.0 * (m + 1) * (m + a + b + 1) * c
    a2 = (c + 1) * (a * a - b * b)
    a3 = c * (c + 1) * (c + 2)
    a4 = 2.0 * (m + a) * (m + b) * (c + 2)
    return a1, a2, a3, a4


def _jacobi_rows(x, m_hi, a, b):
    """Jacobi polynomials P_m^{(a,b)}(x_n), m in [0, m_hi), by the standard
    three-term recurrence; P_1 = (a+1) + (a+b+2)(x-1)/2."""
    out = np.empty((x.size, m_hi))
    p_prev = np.ones_like(x)
    out[:, 0] = p_prev
    if m_hi == 1:
        return out
    p = (a + 1.0) + (a + b + 2.0) * (x - 1.0) / 2.0
    out[:, 1] = p
    for m in range(1, m_hi - 1):
        a1, a2, a3, a4 = _jacobi_coeffs(m, a, b)
        p_next = ((a2 + a3 * x) * p - a4 * p_prev) / a1
        p_prev, p = p, p_next
        out[:, m + 1] = p
    return out


def _mant_exp(values_mp):
    """Split mpmath numbers into (FP64 mantissa in [0.5, 1), int exponent)."""
    mant = np.empty(len(values_mp))
    expo = np.empty(len(values_mp), dtype=np.int64)
    for i, v in enumerate(values_mp):
        m, e = mpmath.frexp(v)
        mant[i] = float(m)
        expo[i] = int(e)
    return mant, expo


_BIG = 2.0 ** 400
_SMALL = 2.0 ** -400


def _rescale(p_prev, p, expo):
    """Keep the pair (p_{m-1}, p_m) inside the FP64 range by exact powers of two."""
    big = np.maximum(np.abs(p_prev), np.abs(p))
    hi = big > _BIG
    if np.any(hi):
        p_prev[hi] *= _SMALL
        p[hi] *= _SMALL
        expo[hi] += 400
    lo = (big < _SMALL) & (big > 0)
    if np.any(lo):
        p_prev[lo] *= _BIG
        p[lo] *= _BIG
        expo[lo] -= 400


def laguerre_exp_start(x):
    """exp(-x/2) for every node as (mantissa, exponent), at 40 digits."""
    with mpmath.workdps(40):
        return _mant_exp([mpmath.exp(-mpmath.mpf(float(v)) / 2) for v in x])


def hermite_exp_start(x):
    """pi^(-1/4) exp(-x^2/2) for every node as (mantissa, exponent), at 40 digits."""
    with mpmath.workdps(40):
        c = mpmath.pi ** mpmath.mpf(-0.25)
        return _mant_exp([c * mpmath.exp(-mpmath.mpf(float(v)) ** 2 / 2) for v in x])


def _laguerre_fn_rows(x, m_hi):
    """Laguerre functions l_m(x) = exp(-x/2) L_m(x) (Section 4), m in [0, m_hi):
    (m+1) L_{m+1} = (2m+1-x) L_m - m L_{m-1}, L_0 = 1, L_1 = 1 - x, carried on
    the scaled values with a per-node power-of-two exponent."""
    out = np.empty((x.size, m_hi))
    mant, expo = laguerre_exp_start(x)
    p_prev = mant.copy()
    out[:, 0] = np.ldexp(p_prev, expo)
    if m_hi == 1:
        return out
    p = (1.0 - x) * mant
    out[:, 1] = np.ldexp(p, expo)
    for m in range(1, m_hi - 1):
        p_next = ((2 * m + 1 - x) * p - m * p_prev) / (m + 1)
        p_prev, p = p, p_next
        _rescale(p_prev, p, expo)
        out[:, m + 1] = np.ldexp(p, expo)
    return out


def _hermite_fn_rows(x, m_hi):
    """Orthonormal Hermite functions psi_m(x) = H_m(x) exp(-x^2/2) / sqrt(2^m m! sqrt(pi)):
    psi_{m+1} = sqrt(2/(m+1)) x psi_m - sqrt(m/(m+1)) psi_{m-1},
    psi_0 = pi^(-1/4) exp(-x^2/2), psi_1 = sqrt(2) x psi_0."""
    out = np.empty((x.size, m_hi))
    mant, expo = hermite_exp_start(x)
    p_prev = mant.copy()
    out[:, 0] = np.ldexp(p_prev, expo)
    if m_hi == 1:
        return out
    p = math.sqrt(2.0) * x * mant
    out[:, 1] = np.ldexp(p, expo)
    for m in range(1, m_hi - 1):
        p_next = math.sqrt(2.0 / (m + 1)) * x * p - math.sqrt(m / (m + 1.0)) * p_prev
        p_prev, p = p, p_next
        _rescale(p_prev, p, expo)
        out[:, m + 1] = np.ldexp(p, expo)
    return out


def values(spec: Spec, m_lo: int, m_hi: int, rows=None) -> np.ndarray:
    """Matrix entries phi_m(x_n) for the selected rows and m in [m_lo, m_hi).

    Only the Chebyshev family accepts m_lo < 0: T_m(x) = cos(m arccos x) is
    defined for negative m (the left extra columns of eq. (extd_f_e)).
    """
    x = spec.x if rows is None else spec.x[np.asarray(rows)]
    fam = spec.family
    if fam in COMPLEX:
        # exp(i m theta_n); exact angle reduction when theta_n = pi num_n / den
        m = np.arange(m_lo, m_hi, dtype=np.int64)
        if spec.cheb_num is not None:
            num = spec.cheb_num if rows is None else spec.cheb_num[np.asarray(rows)]
            k = np.mod(np.outer(num.astype(np.int64), m), 2 * spec.cheb_den)
            ang = np.pi * k / spec.cheb_den
        else:
            ang = np.outer(x, m.astype(np.float64))
        return np.exp(1j * ang)
    if fam in TRIG:
        m = np.arange(m_lo, m_hi, dtype=np.int64)
        if spec.cheb_num is not None:
            num = spec.cheb_num if rows is None else spec.cheb_num[np.asarray(rows)]
            period = 2 * spec.cheb_den  # angle = pi * num * m / den, period 2*den in num*m
            k = np.mod(np.outer(num.astype(np.int64), m), period)
            ang = np.pi * k / spec.cheb_den
        else:
            ang = np.outer(np.arccos(np.clip(x, -1.0, 1.0)), m.astype(np.float64))
        if fam == "sine":
            return np.sin(ang)
        c = np.cos(ang)
        return c ** spec.power if fam == "cospow" else c
    if m_lo < 0:
        raise ValueError("only the trigonometric families extend to negative degrees")
    if fam == "legendre":
        full = _legendre_rows(x, m_hi)
    elif fam == "jacobi":
        full = _jacobi_rows(x, m_hi, spec.alpha, spec.beta)
    elif fam == "laguerre":
        full = _laguerre_fn_rows(x, m_hi)
    elif fam == "hermite":
        full = _hermite_fn_rows(x, m_hi)
    else:
        raise ValueError(f"unknown family {fam!r}")
    return full[:, m_lo:m_hi]


# ------------------------------------------------------------- nodes & weights

def _golub_welsch(diag, off):
    """Eigenvalues of the symmetric tridiagonal Jacobi matrix (ascending)."""
    return scipy.linalg.eigh_tridiagonal(diag, off, eigvals_only=True)


def _jacobi_matrix(family, N, a=0.0, b=0.0):
    k = np.arange(N, dtype=np.float64)
    if family == "legendre":
        diag = np.zeros(N)
        kk = k[1:]
        off = kk / np.sqrt(4 * kk * kk - 1)
    elif family == "jacobi":
        c = 2 * k + a + b
        diag = np.empty(N)
        with np.errstate(invalid="ignore", divide="ignore"):
            diag[:] = (b * b - a * a) / (c * (c + 2))
        diag[0] = (b - a) / (a + b + 2)
        kk = k[1:]
        c1 = 2 * kk + a + b
        with np.errstate(invalid="ignore", divide="ignore"):
            off = np.sqrt(4 * kk * (kk + a) * (kk + b) * (kk + a + b)
                          / (c1 * c1 * (c1 + 1) * (c1 - 1)))
        if N > 1:   # k = 1 with the factor 1 + a + b cancelled (0/0 when a + b = -1)
            off[0] = np.sqrt(4 * (1 + a) * (1 + b) / ((2 + a + b) ** 2 * (3 + a + b)))
    elif family == "laguerre":
        diag = 2 * k + 1
        off = k[1:]
    elif family == "hermite":
        diag = np.zeros(N)
        off = np.sqrt(k[1:] / 2)
    else:
        raise ValueError(family)
    return diag, off


def _last_two(spec_family, x, N, a, b):
    """(phi_N, phi_{N-1}) at x for the degree-N Newton step, as values whose
    common scale cancels in phi_N / phi_N'."""
    if spec_family == "legendre":
        p_prev, p = np.ones_like(x), x.copy()
        for m in range(1, N):
            p_prev, p = p, ((2 * m + 1) * x * p - m * p_prev) / (m + 1)
        return p, p_prev
    if spec_family == "jacobi":
        p_prev, p = np.ones_like(x), (a + 1.0) + (a + b + 2.0) * (x - 1.0) / 2.0
        for m in range(1, N):
            a1, a2, a3, a4 = _jacobi_coeffs(m, a, b)
            p_prev, p = p, ((a2 + a3 * x) * p - a4 * p_prev) / a1
        return p, p_prev
    # functions: run the scaled recurrence and read the last two values unscaled
    if spec_family == "laguerre":
        mant = np.ones_like(x)
        p_prev, p = mant.copy(), (1.0 - x) * mant
        expo = np.zeros(x.size, dtype=np.int64)
        for m in range(1, N):
            p_next = ((2 * m + 1 - x) * p - m * p_prev) / (m + 1)
            p_prev, p = p, p_next
            _rescale(p_prev, p, expo)
        return p, p_prev
    if spec_family == "hermite":
        p_prev, p = np.ones_like(x), math.sqrt(2.0) * x
        expo = np.zeros(x.size, dtype=np.int64)
        for m in range(1, N):
            p_next = math.sqrt(2.0 / (m + 1)) * x * p - math.sqrt(m / (m + 1.0)) * p_prev
            p_prev, p = p, p_next
            _rescale(p_prev, p, expo)
        return p, p_prev
    raise ValueError(spec_family)


def _newton_step(family, x, N, a, b):
    """One Newton correction phi_N(x) / phi_N'(x) using the derivative identities
    of each family (no scale factor survives the ratio)."""
    pN, pN1 = _last_two(family, x, N, a, b)
    if family == "legendre":
        d = N * (x * pN - pN1) / (x * x - 1.0)
    elif family == "jacobi":
        c = 2 * N + a + b
        d = (N * ((a - b) - c * x) * pN + 2.0 * (N + a) * (N + b) * pN1) / (c * (1.0 - x * x))
    elif family == "laguerre":
        # Laguerre polynomials: x L_N' = N (L_N - L_{N-1}); the exp factor of
        # the functions is common to both terms and cancels.
        d = N * (pN - pN1) / x
    elif family == "hermite":
        # Hermite functions (up to a common positive factor): psi_N' = sqrt(2N) psi_{N-1} - x psi_N
        d = math.sqrt(2.0 * N) * pN1 - x * pN
    else:
        raise ValueError(family)
    return pN / d


def gauss_nodes(family: str, N: int, alpha: float = 0.0, beta: float = 0.0) -> np.ndarray:
    """Gauss nodes of the family's orthogonality weight (ascending, except the
    Chebyshev-Gauss points which follow x_n = cos((2n+1) pi / (2N))).

    Golub-Welsch eigenvalues, then three Newton corrections on the degree-N
    recurrence value (Section 5.2 uses Gauss-Jacobi quadrature nodes; Laguerre
    and Hermite function nodes are the Gauss-Laguerre / Gauss-Hermite nodes).
    """
    if family in TRIG:
        n = np.arange(N)
        return np.cos((2 * n + 1) * np.pi / (2 * N))
    diag, off = _jacobi_matrix(family, N, alpha, beta)
    x = _golub_welsch(diag, off)
    for _ in range(3):
        x = x - _newton_step(family, x, N, alpha, beta)
    return np.sort(x)


def exp_default_angles(N: int):
    """Default angles of the exp family: the midpoints theta_n = (2n + 1 - N)
    pi / N of N equal arcs of (-pi, pi), at which the exp functions of degrees
    0..N-1 are discretely orthogonal; returned as (numerator, denominator) of
    theta_n / pi."""
    return 2 * np.arange(N, dtype=np.int64) + 1 - N, N


def lagspec_angles(N: int, eta: float, period: float) -> np.ndarray:
    """psi_j of the spectral Laguerre matrix: exp(i psi_j) = (-eta/2 - i k_j) /
    (eta/2 - i k_j), k_j = 2 pi j / T, j = 0..N-1.  The quotient is
    -(eta/2 + i k)^2 / |eta/2 + i k|^2, so psi_j = 2 arctan(2 k_j / eta) - pi,
    in [-pi, 0) and increasing with j."""
    k = 2.0 * np.pi * np.arange(N) / period
    return 2.0 * np.arctan(2.0 * k / eta) - np.pi


def lagspec_row_factor(N: int, eta: float, period: float) -> np.ndarray:
    """1 / (eta/2 - i k_j), the row factor of the spectral Laguerre matrix."""
    k = 2.0 * np.pi * np.arange(N) / period
    return 1.0 / (eta / 2.0 - 1j * k)


def make_spec(family: str, N: int, alpha: float = 0.0, beta: float = 0.0, x=None, power: int = 2) -> Spec:
    """A family at its Gauss nodes (or at user nodes x); `power` is the s of
    the cos^s family.  exp: x are angles (default `exp_default_angles`);
    lagspec: alpha = eta, beta = T (the angles follow from them)."""
    if family == "lagspec":
        if not (alpha > 0 and beta > 0):
            raise ValueError("the spectral Laguerre matrix needs eta > 0 and T > 0")
        return Spec(family, N, lagspec_angles(N, alpha, beta), alpha, beta)
    if x is not None:
        return Spec(family, N, np.asarray(x, dtype=np.float64), alpha, beta, power=power)
    if family == "exp":
        num, den = exp_default_angles(N)
        return Spec(family, N, np.pi * num / den, alpha, beta, cheb_num=num, cheb_den=den)
    if family in TRIG:
        n = np.arange(N, dtype=np.int64)
        return Spec(family, N, gauss_nodes(family, N), alpha, beta,
                    cheb_num=2 * n + 1, cheb_den=2 * N, power=power)
    return Spec(family, N, gauss_nodes(family, N, alpha, beta), alpha, beta)


def quadrature_weights(spec: Spec) -> np.ndarray:
    """Gauss weights adjusted so that sum_n lam_n phi_m(x_n) phi_k(x_n) equals the
    continuous inner product of phi_m and phi_k (exact for m + k <= 2N - 1):
    Christoffel numbers of the weight function, multiplied by exp(x) / exp(x^2)
    for the Laguerre / Hermite functions, whose weight is inside phi."""
    fam, N, x, a, b = spec.family, spec.N, spec.x, spec.alpha, spec.beta
    if fam == "chebyshev":
        return np.full(N, np.pi / N)
    if fam == "legendre":
        pN, pN1 = _last_two(fam, x, N, a, b)
        d = N * (x * pN - pN1) / (x * x - 1.0)
        return 2.0 / ((1.0 - x * x) * d * d)
    if fam == "jacobi":
        pN, pN1 = _last_two(fam, x, N, a, b)
        c = 2 * N + a + b
        d = (N * ((a - b) - c * x) * pN + 2.0 * (N + a) * (N + b) * pN1) / (c * (1.0 - x * x))
        lg = (gammaln(N + a + 1) + gammaln(N + b + 1) - gammaln(N + a + b + 1) - gammaln(N + 1)
              + (a + b + 1) * math.log(2.0))
        return math.exp(lg) / ((1.0 - x * x) * d * d)
    if fam == "laguerre":
        l_next = values(spec, N + 1, N + 2)[:, 0]      # l_{N+1}(x_n)
        return x / ((N + 1.0) ** 2 * l_next * l_next)
    if fam == "hermite":
        psi = values(spec, N - 1, N)[:, 0]             # psi_{N-1}(x_n)
        return 1.0 / (N * psi * psi)
    raise ValueError(fam)


def column_norms_sq(spec: Spec, m_hi: int) -> np.ndarray:
    """Squared norms chi_m of the basis functions in the weighted L2 space
    (chi_m of eq. (int_jacobi), read as the squared norm so that the normalised
    matrix of Section 5.2 is orthogonal)."""
    fam, a, b = spec.family, spec.alpha, spec.beta
    m = np.arange(m_hi, dtype=np.float64)
    if fam == "chebyshev":
        out = np.full(m_hi, np.pi / 2)
        out[0] = np.pi
        return out
    if fam == "legendre":
        return 2.0 / (2 * m + 1)
    if fam == "jacobi":
        lg = np.empty(m_hi)
        lg[0] = (a + b + 1) * math.log(2.0) + gammaln(a + 1) + gammaln(b + 1) - gammaln(a + b + 2)
        mm = m[1:]
        lg[1:] = ((a + b + 1) * math.log(2.0) - np.log(2 * mm + a + b + 1)
                  + gammaln(mm + a + 1) + gammaln(mm + b + 1)
                  - gammaln(mm + a + b + 1) - gammaln(mm + 1))
        return np.exp(lg)
    if fam in ("laguerre", "hermite"):
        return np.ones(m_hi)
    raise ValueError(fam)


def scalings(spec: Spec, normalise: bool):
    """(rowscale, colscale) with Q = diag(rowscale) A diag(colscale).

    Raw: both ones.  Orthonormal (Section 5.2): rowscale = sqrt(lam_n),
    colscale = 1/sqrt(chi_m), which makes Q orthogonal at Gauss nodes.
    """
    N = spec.N
    if spec.family == "lagspec" and not normalise:
        return lagspec_row_factor(N, spec.alpha, spec.beta), np.ones(N)
    if not normalise:
        return np.ones(N), np.ones(N)
    if spec.family in ("sine", "cospow") + COMPLEX:
        raise ValueError("the orthonormal variant is defined for the orthogonal polynomial families")
    return np.sqrt(quadrature_weights(spec)), 1.0 / np.sqrt(column_norms_sq(spec, N))


def dense_matrix(spec: Spec, normalise: bool = False, rows=None) -> np.ndarray:
    """The plain N x N matrix (or the selected rows) that defines the result."""
    A = values(spec, 0, spec.N, rows)
    if spec.family == "lagspec":
        r = lagspec_row_factor(spec.N, spec.alpha, spec.beta)
        A = (r if rows is None else r[np.asarray(rows)])[:, None] * A
    if normalise:
        r, c = scalings(spec, True)
        if rows is not None:
            r = r[np.asarray(rows)]
        A = r[:, None] * A * c[None, :]
    return A
