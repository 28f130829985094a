"""The two-dimensional compression D̈ = F W_M D W_N F (eq. (comp_2d)) and its
block scheme (Sections 4.2 and 5.3), step by step -- test infrastructure only
(see the package docstring).  FP64 throughout.

The matrix D[i, m] = phi_m(x_i) of a one-sided family (Laguerre or Hermite
functions) at equispaced nodes x_i = x0 + i h.  Its rows (nodes) and columns
(degrees) are extended below the last row and to the right of the last column (Section 6: the
functions stay defined and decay there), never before the first row or
column.  A block is a rectangle of rows [r0, r1) and columns [c0, c1) of D:

- extended rectangle: rows r0 .. r0 + Lr - 1, columns c0 .. c0 + Lc - 1 with
  Lr = (r1 - r0) + sr, Lc = (c1 - c0) + sc, the extra counts of the 1-D block
  method (Section 3) taken along each dimension;
- compressed matrix D̈ = F_Lr W_Lr D_e W_Lc F_Lc (unitary DFTs, Kaiser windows
  w^{zeta, L-1}), elements with |d| <= eps1 max|D̈| dropped (per block);
- product: y_e = W_Lr^{-1} F* D̈ F* W_Lc^{-1} x^{[1]}, where x^{[1]} holds the
  inputs of the block's valid columns [c0 + sc, c1) and zeros elsewhere; the
  valid rows [r0 + sr, r1) of Re(y_e) are added to y; the other rows (window
  below eps2, or extension rows) are discarded.

The first sr rows and sc columns of a block are left out because the window
there is below eps2 (dividing by it would amplify the truncation error by more
than 1/eps2; Section 5.3 names these divisions by near-zero window values).
They are covered by two more rectangles, [r0, r0 + sr) x [c0, c1) and
[r0 + sr, r1) x [c0, c0 + sc), decomposed the same way: the "additional
matrices of various orders" of Section 5.3.  Rectangles with a side of at most
`tail` rows or columns are multiplied densely.

Readings (the paper shows the decomposition only as a figure):
- the recursion above, both remainders decomposed by the same rule;
- the same eps1 (threshold and zeta) and eps2 for every block;
- a rectangle is dense when a side is <= tail (default 20, the 1-D tail) or
  when an extra count reaches the side it extends;
- A^[1] is zero below its diagonal (its definition in Section 5.3): a
  rectangle that lies wholly there, and a block whose valid part does, is
  left out -- it adds exactly zero to every output.  Its extension would
  otherwise bring the diagonal's jump into the block and keep nearly every
  element of a block whose valid part is zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sps
from scipy.special import gammaln

from . import families as fam_mod
from . import special


def lam(z):
    """Lambda(z) = Gamma(z + 1/2) / Gamma(z + 1) (Section 5.3)."""
    return np.exp(gammaln(np.asarray(z, dtype=np.float64) + 0.5) - gammaln(np.asarray(z, dtype=np.float64) + 1.0))


def kernel_a1(i, j):
    """A^[1] of Section 5.3: Lambda(j)/pi on row 0, (2/pi) Lambda(j-i)
    Lambda(j+i) for 0 < i <= j, zero below the diagonal."""
    i, j = np.broadcast_arrays(np.asarray(i, dtype=np.int64), np.asarray(j, dtype=np.int64))
    out = np.zeros(i.shape)
    up = i <= j
    d = np.where(up, j - i, 0)
    out = np.where(up & (i == 0), lam(j) / np.pi, out)
    out = np.where(up & (i > 0), (2.0 / np.pi) * lam(d) * lam(j + i), out)
    return out


def kernel_a2(i, j):
    """A^[2] of Section 5.3: (i cos(log i^2) - j cos(log j^2)) / (i - j)^2
    off the diagonal, zero on it (k cos(log k^2) is read as 0 at k = 0, its
    limit)."""
    i, j = np.broadcast_arrays(np.asarray(i, dtype=np.float64), np.asarray(j, dtype=np.float64))

    def g(k):
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(k > 0, k * np.cos(np.log(np.where(k > 0, k, 1.0) ** 2)), 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(i != j, (g(i) - g(j)) / np.where(i != j, (i - j) ** 2, 1.0), 0.0)


KERNELS = {"a1": kernel_a1, "a2": kernel_a2}


@dataclass
class Spec2D:
    """A one-sided family at the equispaced nodes x_i = x0 + i h, i >= 0, or
    one of the index kernels A^[1], A^[2] of Section 5.3 (entries f(i, j) of
    the row and column indices, defined beyond N in both directions)."""
    family: str
    N: int
    x0: float = 0.0
    h: float = 1.0

    def nodes(self, lo: int, hi: int) -> np.ndarray:
        return self.x0 + self.h * np.arange(lo, hi, dtype=np.float64)

    def values(self, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
        """Entries for rows [r0, r1) and columns [c0, c1)."""
        if self.family in KERNELS:
            i = np.arange(r0, r1)[:, None]
            j = np.arange(c0, c1)[None, :]
            return KERNELS[self.family](i, j)
        sp = fam_mod.make_spec(self.family, r1 - r0, x=self.nodes(r0, r1))
        return fam_mod.values(sp, c0, c1)


@dataclass
class Block2D:
    r0: int
    Lr: int
    vr0: int          # valid rows [vr0, vr1) (matrix indices)
    vr1: int
    c0: int
    Lc: int
    vc0: int          # valid columns [vc0, vc1)
    vc1: int
    wr: np.ndarray = None
    wc: np.ndarray = None
    maxsq: float = 0.0
    kept: sps.csr_matrix = None   # thresholded D̈ (Lr x Lc, complex)


@dataclass
class Dense2D:
    r0: int
    r1: int
    c0: int
    c1: int
    values: np.ndarray = None


@dataclass
class Plan2D:
    spec: Spec2D
    eps: float
    eps2: float
    zeta: float
    blocks: list = field(default_factory=list)
    dense: list = field(default_factory=list)


def supported(family: str) -> bool:
    """Matrices whose entries stay defined below and to the right: Laguerre
    and Hermite functions at equispaced nodes, the index kernels."""
    return family in ("laguerre", "hermite") or family in KERNELS


def zero_below_diagonal(family: str) -> bool:
    """A^[1] vanishes for i > j (Section 5.3)."""
    return family == "a1"


def decompose(N: int, zeta: float, eps2: float, tail: int = 20, lower_zero: bool = False):
    """Cover the N x N index square by the valid rectangles of 2-D blocks and
    dense rectangles (each (row, column) exactly once; with `lower_zero`,
    rectangles and valid parts wholly below the diagonal are left out, so
    entries there are covered at most once).  Returns (blocks as
    (r0, Lr, vr0, r1, c0, Lc, vc0, c1), dense rectangles as (r0, r1, c0, c1))."""
    blocks, dense = [], []
    todo = [(0, N, 0, N)]
    while todo:
        r0, r1, c0, c1 = todo.pop()
        mr, mc = r1 - r0, c1 - c0
        if mr <= 0 or mc <= 0:
            continue
        if lower_zero and r0 >= c1:      # every row index above every column index
            continue
        if mr <= tail or mc <= tail:
            dense.append((r0, r1, c0, c1))
            continue
        sr = special.extra_count(mr, zeta, eps2, False)
        sc = special.extra_count(mc, zeta, eps2, False)
        Lr = special.fft_friendly_at_least(mr + sr)
        Lc = special.fft_friendly_at_least(mc + sc)
        sr, sc = Lr - mr, Lc - mc
        if sr >= mr or sc >= mc:
            dense.append((r0, r1, c0, c1))
            continue
        if not (lower_zero and r0 + sr >= c1):
            blocks.append((r0, Lr, r0 + sr, r1, c0, Lc, c0 + sc, c1))
        todo.append((r0, r0 + sr, c0, c1))
        todo.append((r0 + sr, r1, c0, c0 + sc))
    return blocks, dense


def compress_block(spec: Spec2D, b: Block2D) -> np.ndarray:
    """D̈ = F W_Lr D_e W_Lc F with unitary DFTs (numpy's FFT along both axes)."""
    De = spec.values(b.r0, b.r0 + b.Lr, b.c0, b.c0 + b.Lc)
    A = b.wr[:, None] * De * b.wc[None, :]
    return np.fft.fft(np.fft.fft(A, axis=1), axis=0) / np.sqrt(b.Lr * b.Lc)


def build(spec: Spec2D, eps: float, eps2: float = 1e-3, tail: int = 20,
          eps_window: float = 0.0) -> Plan2D:
    """Precomputation: the decomposition, each block's compressed matrix with
    the per-block threshold |d|^2 > eps1^2 max|d|^2 (eps1 = 0 keeps all), and
    the dense rectangles."""
    if not supported(spec.family):
        raise ValueError("the 2-D scheme extends rows downwards: Laguerre or Hermite functions")
    zeta = special.zeta_of_eps(eps if eps > 0 else (eps_window or 1e-14))
    plan = Plan2D(spec, eps, eps2, zeta)
    blocks, dense = decompose(spec.N, zeta, eps2, tail, zero_below_diagonal(spec.family))
    for (r0, Lr, vr0, r1, c0, Lc, vc0, c1) in blocks:
        b = Block2D(r0, Lr, vr0, r1, c0, Lc, vc0, c1, special.kaiser_window(Lr, zeta),
                    special.kaiser_window(Lc, zeta))
        Dd = compress_block(spec, b)
        mag = Dd.real ** 2 + Dd.imag ** 2
        b.maxsq = float(mag.max())
        keep = mag > (eps * eps) * b.maxsq if eps > 0 else np.ones_like(mag, dtype=bool)
        b.kept = sps.csr_matrix(np.where(keep, Dd, 0.0))
        plan.blocks.append(b)
    for (r0, r1, c0, c1) in dense:
        plan.dense.append(Dense2D(r0, r1, c0, c1, spec.values(r0, r1, c0, c1)))
    return plan


def _as_2d(v):
    v = np.asarray(v, dtype=np.float64)
    return (v[None, :], True) if v.ndim == 1 else (v, False)


def apply(plan: Plan2D, x) -> np.ndarray:
    """y = D x: per block, y[valid rows] += Re(W^{-1} F* D̈ F* W^{-1} x^{[1]})
    on the valid rows; plus the dense rectangles."""
    X, flat = _as_2d(x)
    R, N = X.shape[0], plan.spec.N
    Y = np.zeros((R, N))
    for b in plan.blocks:
        x1 = np.zeros((R, b.Lc))
        x1[:, b.vc0 - b.c0:b.vc1 - b.c0] = X[:, b.vc0:b.vc1]
        v = np.fft.ifft(x1 / b.wc[None, :], axis=1) * np.sqrt(b.Lc)      # F* W^{-1} x^{[1]}
        z = (b.kept @ v.T).T                                               # D̈ (.)
        ye = np.fft.ifft(z, axis=1) * np.sqrt(b.Lr) / b.wr[None, :]        # W^{-1} F* (.)
        Y[:, b.vr0:b.vr1] += np.real(ye[:, b.vr0 - b.r0:b.vr1 - b.r0])
    for d in plan.dense:
        Y[:, d.r0:d.r1] += X[:, d.c0:d.c1] @ d.values.T
    return Y[0] if flat else Y


def apply_adjoint(plan: Plan2D, y) -> np.ndarray:
    """x = D^T y, the plain transpose of `apply`'s operator:
    D_e^T = W^{-1} F* D̈^T F* W^{-1} (F symmetric), valid rows of the block in,
    valid columns out."""
    Y, flat = _as_2d(y)
    R, N = Y.shape[0], plan.spec.N
    X = np.zeros((R, N))
    for b in plan.blocks:
        y1 = np.zeros((R, b.Lr))
        y1[:, b.vr0 - b.r0:b.vr1 - b.r0] = Y[:, b.vr0:b.vr1]
        v = np.fft.ifft(y1 / b.wr[None, :], axis=1) * np.sqrt(b.Lr)
        z = (b.kept.T @ v.T).T
        xe = np.fft.ifft(z, axis=1) * np.sqrt(b.Lc) / b.wc[None, :]
        X[:, b.vc0:b.vc1] += np.real(xe[:, b.vc0 - b.c0:b.vc1 - b.c0])
    for d in plan.dense:
        X[:, d.c0:d.c1] += Y[:, d.r0:d.r1] @ d.values
    return X[0] if flat else X


def dense_matrix(spec: Spec2D) -> np.ndarray:
    return spec.values(0, spec.N, 0, spec.N)


def stored_fraction(plan: Plan2D) -> float:
    """Kept compressed elements plus dense elements, relative to N^2."""
    kept = sum(b.kept.nnz for b in plan.blocks)
    dense = sum((d.r1 - d.r0) * (d.c1 - d.c0) for d in plan.dense)
    return (kept + dense) / float(plan.spec.N) ** 2
