"""FP64 parity bound of the CUDA path against the oracle's method (a test
helper, computed from the oracle plan and the inputs only).

Both sides run Algorithms 1-4 in FP64, independently: the plan's compressed
matrix K is computed twice (different recurrences, row FFTs and rounding),
and the apply rounds differently.  The relative l2 gap between the two
results is bounded by three terms:

  apply rounding   u ||S|| / ||y||: the FFT of W^-1 x and the band sums,
                   S = |K| (|v| + rms(v)) log2 L per block (forward), with
                   v = F* W^-1 x; for the adjoint the inverse transform of
                   z = K^T y and its window division,
                   S_j = (log2 L ||z|| + || |K|^T |y| ||) / (sqrt(L) w_j);
  precompute       rho u ||V|| / ||y||, V = |K| |v| (forward) or
                   || |K|^T |y| || / (sqrt(L) w_j) (adjoint): entries of K
                   that differ by a few rho units in the last place on the two
                   sides.  rho = 8 for the stable recurrences; the Laguerre
                   functions' recurrence at Gauss-Laguerre nodes (x up to
                   about 4N) loses accuracy in proportion to N on both sides,
                   rho = N / 2 (measured gaps at N = 4096: 2.8e-11 forward,
                   3.8e-11 adjoint, about a third of the bound);
  threshold        8 eps1: elements within rounding of eps1 max|K| kept on
                   one side only (each moves an output by about
                   eps1 max|K| |v_k|), and the closed-form (Appendix A)
                   Chebyshev rows, whose window spectrum is truncated at
                   0.1 eps1 max|K|.
"""
import math

import numpy as np

U64 = 2.0 ** -53


def _rho(spec):
    return spec.N / 2.0 if spec.family == "laguerre" else 8.0


def forward_bound(ora, X, y_ref):
    """Relative l2 bound of the forward apply (X: (R, N) real inputs)."""
    X = np.atleast_2d(X) * ora.colscale[None, :]
    R = X.shape[0]
    S = np.zeros((R, ora.rows.size))
    V = np.zeros_like(S)
    for b in ora.blocks:
        x1 = np.zeros((R, b.L))
        x1[:, b.j_lo:b.j_hi] = X[:, b.j_lo - b.off:b.j_hi - b.off]
        v = np.fft.ifft(x1 / b.window[None, :], axis=1) * np.sqrt(b.L)
        av = np.abs(v)
        rms = np.linalg.norm(v, axis=1, keepdims=True) / np.sqrt(b.L)
        K = abs(b.kept)
        S += (K @ (av + rms).T).T * math.log2(b.L)
        V += (K @ av.T).T
    if ora.tail is not None:
        T = np.abs(ora.tail)
        S += np.abs(X[:, :T.shape[1]]) @ T.T * math.log2(max(2, T.shape[1]))
    S *= np.abs(ora.rowscale[ora.rows])[None, :]
    V *= np.abs(ora.rowscale[ora.rows])[None, :]
    ny = np.linalg.norm(y_ref)
    return U64 * np.linalg.norm(S) / ny + _rho(ora.spec) * U64 * np.linalg.norm(V) / ny + 8 * ora_eps(ora)


def adjoint_bound(ora, Y, x_ref):
    """Relative l2 bound of the adjoint apply (Y: (R, N) real inputs)."""
    Y = np.atleast_2d(Y) * ora.rowscale[None, :]
    R = Y.shape[0]
    S = np.zeros((R, ora.spec.N))
    V = np.zeros_like(S)
    for b in ora.blocks:
        z = (b.kept.T @ Y.T).T
        az = (abs(b.kept).T @ np.abs(Y).T).T
        nz = np.linalg.norm(z, axis=1, keepdims=True)
        naz = np.linalg.norm(az, axis=1, keepdims=True)
        iw = 1.0 / (np.sqrt(b.L) * b.window[b.j_lo:b.j_hi])[None, :]
        S[:, b.j_lo - b.off:b.j_hi - b.off] += (math.log2(b.L) * nz + naz) * iw
        V[:, b.j_lo - b.off:b.j_hi - b.off] += naz * iw
    if ora.tail is not None:
        T = np.abs(ora.tail)
        S[:, :T.shape[1]] += (np.abs(Y) @ T) * math.log2(ora.spec.N)
    S *= np.abs(ora.colscale)[None, :]
    V *= np.abs(ora.colscale)[None, :]
    nx = np.linalg.norm(x_ref)
    return U64 * np.linalg.norm(S) / nx + _rho(ora.spec) * U64 * np.linalg.norm(V) / nx + 8 * ora_eps(ora)


def ora_eps(ora):
    return ora.schedule.eps1


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
