"""The extra-component method, step by step, and the dense products it replaces.

Test infrastructure only (see the package docstring).  FP64 throughout.

Notation follows the paper: the unitary DFT F of eq. (fourier)
(F[j,k] = L^{-1/2} exp(-2 pi i jk / L)), the Kaiser window matrix W, the
extended matrix A_e, the compressed matrix  A_e W F  (eq. (A_comp)), and the
identities (comp1) / (comp2):

    forward   y    = Ä_e F* W^{-1} x^{[1]}          (Algorithm 1, step 2.2)
    adjoint   x^[2] = W^{-1} F* Ä_e^T y  then discard the extra components
                                                    (Algorithm 2, steps 2.1-2.2)

applied per block and summed (Algorithms 3 and 4, Section 3), plus the dense
tail.  numpy's FFT is used as the multiplication by sqrt(L) F / sqrt(L) F*:
F u = fft(u) / sqrt(L) and F* u = ifft(u) * sqrt(L).

Reading (the method reaches a real result only up to truncation): the real part
is taken after each block's product, in both directions, which makes the
adjoint the exact transpose of the thresholded forward operator.

Rows are processed in chunks so that a full-size block never has to be held as
a dense N x L complex matrix; the kept elements are stored as a scipy CSR
matrix (a library sparse matrix-vector product is the multiplication step).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sps

from . import families as fam_mod
from . import special


@dataclass
class OracleBlock:
    L: int
    off: int
    j_lo: int
    j_hi: int
    window: np.ndarray            # w_j^{zeta, L-1}, j = 0..L-1
    maxsq: float                  # max |Ä_e|^2 over the whole block (orthonormal: of lam_n |ä|^2)
    kept: sps.csr_matrix          # thresholded Ä_e restricted to `rows`, full spectrum
    nnz_half: np.ndarray | None = None   # kept elements per row with k <= L/2


@dataclass
class OraclePlan:
    spec: fam_mod.Spec
    schedule: special.Schedule
    normalise: bool
    rows: np.ndarray              # the rows whose compressed entries are stored
    rowscale: np.ndarray
    colscale: np.ndarray
    blocks: list = field(default_factory=list)
    tail: np.ndarray | None = None   # raw A[rows, 0:m_tail]


def default_eps2(precision: str) -> float:
    """The eps2 used when the caller passes none.  FP64: 1e-3, the paper's value
    for its 1e-10 experiments (Section 5.2).  FP32 paths: 1e-1.  Section 2.2
    puts the accuracy at eps1/eps2: with eps1 = 1e-7 the adjoint, whose
    truncation error W^{-1} amplifies after the product, needs eps2 ~ 0.1 to stay
    below 1e-5, and the FP32 FFT rounding is amplified by up to 1/eps2 as well;
    Section 5.1 notes that more extra components than needed only cost a little."""
    return 1e-3 if precision == "fp64" else 1e-1


def compress_rows(spec, blk: special.Block, zeta: float, rows) -> np.ndarray:
    """Rows of the compressed block Ä_e = A_e W F (eq. (A_comp), Algorithm 1
    step 1.3 without the threshold): A_e[n, j] = phi_{j-off}(x_n), j < L."""
    A_e = fam_mod.values(spec, -blk.off, blk.L - blk.off, rows)
    w = special.kaiser_window(blk.L, zeta)
    return np.fft.fft(A_e * w[None, :], axis=1) / np.sqrt(blk.L)


def _sinpi_ratio(num, den: int):
    """sin(pi * num / den) for integer arrays num, with num reduced exactly
    modulo 2 den and reflected into [-den/2, den/2] (sin(pi - x) = sin x)
    first, so that the only rounding is in the final quotient and sine and the
    result keeps its relative accuracy next to every zero."""
    r = np.mod(np.asarray(num, dtype=object), 2 * den).astype(np.int64)
    r = np.where(r >= den, r - 2 * den, r)                 # [-den, den)
    r = np.where(2 * r > den, den - r, r)
    r = np.where(2 * r < -den, -den - r, r)
    return np.sin(np.pi * r.astype(np.float64) / den)


def _cospi_ratio(num, den: int):
    r = np.mod(np.asarray(num, dtype=object), 2 * den).astype(np.int64)
    return np.cos(np.pi * r.astype(np.float64) / den)


def chebyshev_row_dft(n: int, N: int, L: int, off: int, q) -> np.ndarray:
    """Appendix A, eqs. (y1)/(y3): the DFT sum_{j<L} cos((j - off) theta_n)
    exp(-2 pi i j q / L) of an extended Chebyshev row in closed form, theta_n =
    (2n+1) pi / (2N).  Writing cos as two exponentials, each part is a
    geometric series sum_j exp(i j phi) = exp(i (L-1) phi / 2) sin(L phi / 2) /
    sin(phi / 2) with phi = +-theta - 2 pi q / L.  Every angle is a rational
    multiple of pi; numerators are reduced exactly before the sines are taken,
    and the series is L where phi is a multiple of 2 pi."""
    q = np.asarray(q, dtype=np.int64)
    P = 4 * N * L                                   # phi / 2 = pi a / P
    t = (2 * n + 1) * L                             # L theta / 2 = pi t / (4N)
    sin_lt = float(_sinpi_ratio(np.array([t]), 4 * N)[0])
    sign_q = np.where(q % 2 == 0, 1.0, -1.0)

    def dirichlet_ratio(a):
        """sin(L phi/2) / sin(phi/2) for phi/2 = pi a / P, sin(L phi/2) = (-1)^q sin(L theta/2)."""
        den = _sinpi_ratio(a, P)
        res = np.mod(a.astype(object), P) == 0
        p = (a.astype(object) // P)
        lim = np.array([L * (1.0 if (int(pp) * (L - 1)) % 2 == 0 else -1.0) for pp in p])
        with np.errstate(divide="ignore", invalid="ignore"):
            val = sign_q * sin_lt / den
        return np.where(res.astype(bool), lim, val)

    s_plus = dirichlet_ratio(t - 4 * N * q)         # phi = theta - 2 pi q / L
    s_minus = dirichlet_ratio(t + 4 * N * q)        # -phi for phi = -theta - 2 pi q / L (the ratio is even)
    c2 = (2 * n + 1) * (L - 1 - 2 * off)            # theta (L - 1 - 2 off) / 2 = pi c2 / (4N)
    e_c = complex(float(_cospi_ratio(np.array([c2]), 4 * N)[0]), float(_sinpi_ratio(np.array([c2]), 4 * N)[0]))
    ph = -(q * (L - 1))                             # -pi q (L - 1) / L
    e_q = _cospi_ratio(ph, L) + 1j * _sinpi_ratio(ph, L)
    return e_q * 0.5 * (e_c * s_plus + np.conj(e_c) * s_minus)


def compress_rows_appendix_a(spec, blk: special.Block, zeta: float, rows, M: int) -> np.ndarray:
    """Rows of the compressed Chebyshev block by Appendix A: the DFT of the
    windowed row is the circular convolution (eq. (conv_appendix)) of the
    window's DFT with the row's closed-form DFT; only the window components
    |m| <= M enter (the Kaiser spectrum is concentrated there).  Same
    normalisation as compress_rows: fft(A_e w) / sqrt(L)."""
    assert spec.family == "chebyshev"
    N, L, off = spec.N, blk.L, blk.off
    w = special.kaiser_window(L, zeta)
    j = np.arange(L, dtype=np.int64)
    ms = np.arange(-M, M + 1)
    xw = np.array([np.sum(w * np.exp(-2j * np.pi * ((j * m) % L) / L)) for m in ms])
    k = np.arange(L)
    q = np.arange(-M, L + M)
    out = np.empty((len(rows), L), dtype=complex)
    for r, n in enumerate(rows):
        a_hat = chebyshev_row_dft(int(n), N, L, off, q)
        u = np.zeros(L, dtype=complex)
        for i, m in enumerate(ms):
            u += xw[i] * a_hat[k - m + M]
        out[r] = u / L / np.sqrt(L)
    return out


def build(spec, eps: float, eps2: float | None = None, precision: str = "fp64",
          normalise: bool = False, eps_window: float = 0.0, tail_max: int = 20,
          two_sided: bool | None = None, rows=None, chunk: int = 256) -> OraclePlan:
    """Precomputation stage of Algorithms 1-4.

    Per block: zeta(eps1) and s(eps2, zeta) (step 1.1), the extended matrix
    (step 1.2), the compressed matrix and the elements with |ä| > eps1 *
    max|Ä_e| kept (step 1.3).  The maximum is taken over the whole block.
    The comparison is made on squared magnitudes, |ä|^2 > eps1^2 * max|ä|^2, which
    is the same test in exact arithmetic.  With eps == 0 every element is kept.

    The orthonormal variant (Section 5.2) applies B = diag(sqrt(lam)) A
    diag(1/sqrt(chi)); its rows are those of A times sqrt(lam_n), and so are
    the rows of its compressed matrix (the window and the DFT act along the
    rows).  The threshold is taken on those: lam_n |ä|^2 > eps1^2 max(lam |ä|^2).
    Thresholding A's own compressed matrix instead loses the rows of small
    polynomial values that carry most of the weight, and the accuracy of the
    forward transform would fall with alpha and beta, which Section 5.2 says
    it does not.

    `rows` restricts what is stored (the maximum still runs over all rows), so
    that sampled outputs of a full-size plan can be computed.
    """
    if eps2 is None:
        eps2 = default_eps2(precision)
    if two_sided is None:
        two_sided = spec.family in fam_mod.TWO_SIDED
    N = spec.N
    sch = special.schedule(N, eps, eps2, two_sided, eps_window, tail_max)
    rows = np.arange(N) if rows is None else np.asarray(rows)
    r, c = fam_mod.scalings(spec, normalise)
    plan = OraclePlan(spec, sch, normalise, rows, r, c)
    lam = fam_mod.quadrature_weights(spec) if normalise else None   # row weights of the threshold

    def weighted(comp, sel):
        mag = comp.real ** 2 + comp.imag ** 2
        return mag if lam is None else lam[sel][:, None] * mag

    for b in sch.blocks:
        maxsq = 0.0
        for lo in range(0, N, chunk):
            sel = np.arange(lo, min(N, lo + chunk))
            comp = compress_rows(spec, b, sch.zeta, sel)
            maxsq = max(maxsq, float(np.max(weighted(comp, sel))))
        thr = (eps * eps) * maxsq
        pieces = []
        nnz_half = []
        for lo in range(0, rows.size, chunk):
            sel = rows[lo:lo + chunk]
            comp = compress_rows(spec, b, sch.zeta, sel)
            mag = weighted(comp, sel)
            keep = mag > thr if eps > 0 else np.ones_like(mag, dtype=bool)
            nnz_half.append(np.count_nonzero(keep[:, : b.L // 2 + 1], axis=1))
            pieces.append(sps.csr_matrix(np.where(keep, comp, 0.0)))
        kept = sps.vstack(pieces).tocsr()
        plan.blocks.append(OracleBlock(b.L, b.off, b.j_lo, b.j_hi,
                                       special.kaiser_window(b.L, sch.zeta), maxsq, kept,
                                       np.concatenate(nnz_half)))
    if sch.m_tail > 0:
        plan.tail = fam_mod.values(spec, 0, sch.m_tail, rows)
    return plan


def _as_2d(v, complex_=False):
    v = np.asarray(v, dtype=np.complex128 if complex_ or np.iscomplexobj(v) else np.float64)
    return (v[None, :], True) if v.ndim == 1 else (v, False)


def apply(plan: OraclePlan, x) -> np.ndarray:
    """y = A x by Algorithm 1 (one two-sided block) or Algorithm 3 (blocks +
    dense tail).  x has shape (N,) or (R, N); the result covers plan.rows.

    Per block: x^{[1]} of eq. (Fe1)/(Fe3) (zeros outside [j_lo, j_hi)), then
    Ä_e F* W^{-1} x^{[1]} (step 2.2), real part, summed over the blocks.
    Complex families: complex x and y, no real part taken.
    """
    cplx = plan.spec.is_complex
    X, flat = _as_2d(x, cplx)
    Xs = X * plan.colscale[None, :]
    R = X.shape[0]
    Y = np.zeros((R, plan.rows.size), dtype=np.complex128 if cplx else np.float64)
    for b in plan.blocks:
        x1 = np.zeros((R, b.L), dtype=Xs.dtype)
        x1[:, b.j_lo:b.j_hi] = Xs[:, b.j_lo - b.off:b.j_hi - b.off]
        u = x1 / b.window[None, :]
        v = np.fft.ifft(u, axis=1) * np.sqrt(b.L)          # F* W^{-1} x^{[1]}
        prod = (b.kept @ v.T).T                            # Ä_e (F* W^{-1} x^{[1]})
        Y += prod if cplx else np.real(prod)
    if plan.tail is not None:
        Y += Xs[:, : plan.tail.shape[1]] @ plan.tail.T     # direct product, last block
    Y *= plan.rowscale[plan.rows][None, :]
    return Y[0] if flat else Y


def apply_adjoint(plan: OraclePlan, y) -> np.ndarray:
    """x = A^T y by Algorithm 2 (two-sided) or Algorithm 4 (blocks + tail).

    Per block: x^{[2]} = W^{-1} F* Ä_e^T y (step 2.1, plain transpose), real
    part, then the extra components outside [j_lo, j_hi) are discarded
    (step 2.2, eq. (Fe2)); each block writes its own slice of x.
    Requires a plan built over all rows.  Complex families: the plain
    transpose (not the conjugate transpose), no real part taken.
    """
    if plan.rows.size != plan.spec.N:
        raise ValueError("the adjoint needs every row of the compressed matrix")
    cplx = plan.spec.is_complex
    Y, flat = _as_2d(y, cplx)
    Ys = Y * plan.rowscale[None, :]
    R = Y.shape[0]
    Xh = np.zeros((R, plan.spec.N), dtype=np.complex128 if cplx else np.float64)
    for b in plan.blocks:
        z = (b.kept.T @ Ys.T).T                            # Ä_e^T y
        x2 = np.fft.ifft(z, axis=1) * np.sqrt(b.L) / b.window[None, :]   # W^{-1} F* (.)
        part = x2[:, b.j_lo:b.j_hi]
        Xh[:, b.j_lo - b.off:b.j_hi - b.off] = part if cplx else np.real(part)
    if plan.tail is not None:
        Xh[:, : plan.tail.shape[1]] = Ys @ plan.tail
    Xh *= plan.colscale[None, :]
    return Xh[0] if flat else Xh


def dense_apply(spec, x, normalise: bool = False, rows=None, chunk: int = 1024) -> np.ndarray:
    """The definition y = A x (A of eq. (cheb_matrix) / (Jac_matrix)), rows of A
    generated in chunks by the recurrences; x has shape (N,) or (R, N)."""
    X, flat = _as_2d(x, spec.is_complex)
    rows = np.arange(spec.N) if rows is None else np.asarray(rows)
    Y = np.empty((X.shape[0], rows.size), dtype=np.complex128 if spec.is_complex else np.float64)
    for lo in range(0, rows.size, chunk):
        sel = rows[lo:lo + chunk]
        A = fam_mod.dense_matrix(spec, normalise, sel)
        Y[:, lo:lo + sel.size] = X @ A.T
    return Y[0] if flat else Y


def dense_apply_adjoint(spec, y, normalise: bool = False, chunk: int = 1024) -> np.ndarray:
    """The definition x = A^T y, accumulated over chunks of rows of A."""
    Y, flat = _as_2d(y, spec.is_complex)
    Xh = np.zeros((Y.shape[0], spec.N), dtype=np.complex128 if spec.is_complex else np.float64)
    for lo in range(0, spec.N, chunk):
        sel = np.arange(lo, min(spec.N, lo + chunk))
        A = fam_mod.dense_matrix(spec, normalise, sel)
        Xh += Y[:, sel] @ A
    return Xh[0] if flat else Xh


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 over all entries."""
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    b = b.astype(np.complex128 if np.iscomplexobj(b) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
