"""Pins for oracle/method.py: the identities (comp1)/(comp2), brute force on
tiny cases, the exact-transpose property of Algorithms 2/4, the accuracy and
compression the paper reports, the Appendix A closed forms, and planted
mistakes that these pins must catch."""
import json
import math
import os

import numpy as np
import pytest

from oracle import families as F
from oracle import method as M
from oracle import special as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CLAIMS = json.load(open(os.path.join(GOLDEN, "paper_claims.json")))


def _spec(fam, N):
    if fam == "jacobi":
        return F.make_spec(fam, N, 0.5, -0.5)
    if fam == "lagspec":
        return F.make_spec(fam, N, 50.0, 2.0)     # eta, T
    return F.make_spec(fam, N)


def identity_error(fam, N, two_sided=None, normalise=False, seed=0):
    """eps = 0 keeps every element, so Ä_e F* W^{-1} x^{[1]} = A x exactly
    (eq. (comp1)); the FP64 result differs by rounding amplified by W^{-1}."""
    sp = _spec(fam, N)
    P = M.build(sp, 0.0, eps2=1e-3, two_sided=two_sided, normalise=normalise)
    x = np.random.default_rng(seed).uniform(-1, 1, (2, N))
    y = M.apply(P, x)
    yd = M.dense_apply(sp, x, normalise)
    xa = M.apply_adjoint(P, y)
    xd = M.dense_apply_adjoint(sp, y, normalise)
    return max(M.rel_l2(y, yd), M.rel_l2(xa, xd))


@pytest.mark.parametrize("fam", F.FAMILIES)
@pytest.mark.parametrize("N", [48, 203])
def test_eps0_method_equals_dense(fam, N):
    assert identity_error(fam, N) < 2e-13


def test_eps0_block_scheme_for_chebyshev_and_orthonormal():
    assert identity_error("chebyshev", 130, two_sided=False) < 2e-13
    assert identity_error("legendre", 150, normalise=True) < 2e-13


def operator_matrices(fam, N, eps, two_sided=None):
    """Explicit matrices of the forward and adjoint operators, column by column."""
    sp = _spec(fam, N)
    P = M.build(sp, eps, eps2=1e-3, two_sided=two_sided)
    I = np.eye(N)
    fwd = M.apply(P, I).T            # column m = A e_m
    adj = M.apply_adjoint(P, I).T    # column n = A^T e_n
    return sp, fwd, adj


@pytest.mark.parametrize("fam", F.FAMILIES)
def test_brute_force_tiny(fam):
    """N <= 64: the whole forward operator at eps = 0 equals A entrywise, and
    the adjoint operator is its transpose (also for eps > 0).  Entrywise
    rounding: an FFT of length L loses ~u log2 L relative to the largest input,
    which W^{-1} has amplified by up to 1/eps2 = 1e3: tol = 8 u log2(L) / eps2."""
    u = 2.0 ** -53
    for N in (21, 40, 64):
        sp, fwd, adj = operator_matrices(fam, N, 0.0)
        A = F.dense_matrix(sp)
        tol = 8 * u * math.log2(4 * N) / 1e-3 * np.abs(A).max()
        assert np.abs(fwd - A).max() <= tol
        assert np.abs(adj - A.T).max() <= tol
        sp, fwd, adj = operator_matrices(fam, N, 1e-6)
        assert np.abs(adj - fwd.T).max() <= 8 * u * math.log2(4 * N) / 1e-3 * np.abs(fwd).max()


@pytest.mark.parametrize("fam", F.FAMILIES)
def test_adjoint_dot_product_identity(fam):
    """Algorithm 2 uses the transposed compressed matrix (step 1.3), so
    <A x, y> = <x, A^T y> holds for the thresholded operator to rounding."""
    N = 300
    sp = _spec(fam, N)
    P = M.build(sp, 1e-8, eps2=1e-3)
    g = np.random.default_rng(3)
    x, y = g.standard_normal((4, N)), g.standard_normal((4, N))
    Ax, Aty = M.apply(P, x), M.apply_adjoint(P, y)
    lhs, rhs = np.sum(Ax * y, axis=1), np.sum(x * Aty, axis=1)
    scale = np.sum(np.abs(Ax * y), axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-14 * scale)


@pytest.mark.parametrize("case", CLAIMS["jacobi_bw"]["cases"])
def test_legendre_accuracy_and_bandwidth_section52(case):
    """Section 5.2: bw = 20 at (1e-10, 1e-3) and 16 at (1e-6, 1e-4); the
    achieved error stays below the eps1/eps2 level of Section 2.2 and every row
    keeps at most rho = 25 elements (Section 2.1)."""
    N = 1024
    sp = _spec("legendre", N)
    P = M.build(sp, case["eps1"], eps2=case["eps2"])
    x = np.random.default_rng(1).uniform(0, 1, (3, N))
    err = M.rel_l2(M.apply(P, x), M.dense_apply(sp, x))
    assert err <= case["eps1"] / case["eps2"]
    for b in P.blocks:
        assert b.nnz_half.max() <= min(case["bw"] + 2, CLAIMS["rho_max"]["value"])


@pytest.mark.parametrize("case", CLAIMS["chebyshev_bw"]["cases"])
def test_chebyshev_bandwidth_section51(case):
    """Section 5.1: about bw = 16 stored diagonals for 1e-8 and 24 for 1e-15,
    independent of N; rho <= 25."""
    for N in (512, 2048):
        sp = _spec("chebyshev", N)
        P = M.build(sp, case["accuracy"], eps2=1e-3)
        (b,) = P.blocks
        bw = float(np.median(b.nnz_half))
        assert abs(bw - case["bw"]) <= 3
        assert b.nnz_half.max() <= CLAIMS["rho_max"]["value"] + 1


@pytest.mark.parametrize("case", CLAIMS["jacobi_bw"]["cases"])
@pytest.mark.parametrize("fam,alpha,beta", [("legendre", 0.0, 0.0), ("jacobi", 0.5, -0.5)])
def test_block_nnz_does_not_depend_on_the_block_order(case, fam, alpha, beta):
    """Section 5.2: the compressed N x N_i submatrix of every block keeps a
    number of elements of the order of bw N whatever N_i is.  Per block of
    order N_i >= 4 bw (below that the half spectrum itself has fewer than 2 bw
    bins), kept elements per row (half spectrum) lie within 15 % of the first
    block's and between bw/3 and bw, for N = 2048 and 4096 (orders ~N down to
    ~100)."""
    for N in (2048, 4096):
        sp = F.make_spec(fam, N, alpha=alpha, beta=beta)
        P = M.build(sp, case["eps1"], eps2=case["eps2"])
        per_row = [b.nnz_half.sum() / N for b in P.blocks if b.L >= 4 * case["bw"]]
        assert len(per_row) >= 2
        assert all(abs(r - per_row[0]) <= 0.15 * per_row[0] for r in per_row)
        assert all(case["bw"] / 3 <= r <= case["bw"] for r in per_row)


@pytest.mark.parametrize("eps2", [1e-3, 1e-2])
def test_chebyshev_extension_doubles_from_1e8_to_1e15(eps2):
    """Section 5.1: the two-sided extension takes s ~ N/4 extra columns on each
    side for accuracy 1e-8 and s ~ N/2 for 1e-15, twice as many.  The paper
    does not give its eps2; for a fixed eps2 the ratio s(1e-15) / s(1e-8) is
    within 10 % of two, for N = 512 .. 8192."""
    c = {c_["accuracy"]: c_["s_over_N"] for c_ in CLAIMS["chebyshev_bw"]["cases"]}
    for N in (512, 2048, 8192):
        s = {}
        for acc in (1e-8, 1e-15):
            (b,) = S.schedule(N, acc, eps2, True, 0.0, 20).blocks
            s[acc] = (b.L - N) / 2
        assert abs(s[1e-15] / s[1e-8] - c[1e-15] / c[1e-8]) <= 0.1 * c[1e-15] / c[1e-8]


def test_forward_accuracy_tracks_eps():
    sp = _spec("chebyshev", 1000)
    x = np.random.default_rng(2).uniform(0, 1, (2, 1000))
    yd = M.dense_apply(sp, x)
    errs = [M.rel_l2(M.apply(M.build(sp, e, eps2=1e-3), x), yd) for e in (1e-6, 1e-9, 1e-12)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9


def test_orthonormal_round_trip():
    """Section 5.2: B^{-1} = B^T for the normalised Gauss matrix, so the
    adjoint undoes the forward apply up to the method's error."""
    N = 512
    sp = _spec("legendre", N)
    P = M.build(sp, 1e-12, eps2=1e-3, normalise=True)
    x = np.random.default_rng(4).standard_normal((2, N))
    assert M.rel_l2(M.apply_adjoint(P, M.apply(P, x)), x) < 1e-9


def test_orthonormal_jacobi_accuracy_does_not_change_with_alpha_beta():
    """Section 5.2: the accuracy of the forward (and transposed) orthonormal
    Jacobi transform stays the same as alpha or beta grow (Gauss-Jacobi nodes,
    eps1 = 1e-10, eps2 = 1e-3): every error under eps1/eps2 and all within a
    factor of ten of each other."""
    N = 512
    x = np.random.default_rng(7).uniform(0, 1, (3, N))
    errs = []
    # alpha, beta > -1 anywhere (Section 5.2 widens the range beyond |alpha|, |beta| < 1/2)
    for a, b in ((0.0, 0.0), (0.5, -0.5), (1.5, 0.3), (-0.7, 2.0), (3.0, 3.0), (5.0, 1.0), (-0.9, -0.9),
                 (-0.9, 3.0), (8.0, 8.0)):
        sp = F.make_spec("jacobi", N, alpha=a, beta=b)
        P = M.build(sp, 1e-10, eps2=1e-3, normalise=True)
        errs.append(M.rel_l2(M.apply(P, x), M.dense_apply(sp, x, normalise=True)))
        errs.append(M.rel_l2(M.apply_adjoint(P, x), M.dense_apply_adjoint(sp, x, normalise=True)))
    assert max(errs) <= 1e-10 / 1e-3
    assert max(errs) <= 10 * min(errs)


# ------------------------------------------------------- Appendix A closed forms

def y_cos(theta, N):
    """eq. (y1): L^{-1/2} sum_j cos(j theta) w^{jk}, w = exp(-2 pi i / N)."""
    om = np.exp(-2j * np.pi * np.arange(N) / N)
    c, s = math.cos(N * theta), math.sin(N * theta)
    num = om * (((c - 1) * math.cos(theta) + math.sin(theta) * s) - (c - 1) * om)
    return num / (om * om - 2 * om * math.cos(theta) + 1) / math.sqrt(N)


def y_sin(theta, N):
    """eq. (y2)."""
    om = np.exp(-2j * np.pi * np.arange(N) / N)
    c, s = math.cos(N * theta), math.sin(N * theta)
    num = om * ((math.sin(theta) * (c - 1) - math.cos(theta) * s) + s * om)
    return num / (-om * om + 2 * om * math.cos(theta) - 1) / math.sqrt(N)


def y_exp(theta, N):
    """eq. (y3)."""
    om = np.exp(-2j * np.pi * np.arange(N) / N)
    return (np.exp(1j * N * theta) - 1) / (np.exp(1j * theta) * om - 1) / math.sqrt(N)


def test_appendix_a_closed_forms_against_sums():
    """Reading: eq. (y3) holds as printed with w = exp(-2 pi i / N); eqs. (y1)
    and (y2) as printed equal the sums taken with the conjugate root
    exp(+2 pi i / N) (for real rows: the complex conjugate of the stated DFT)."""
    N = 64
    j = np.arange(N)
    om = np.exp(-2j * np.pi * np.outer(j, j) / N)
    for theta in (0.3, 1.1, 2.9):
        assert np.allclose(y_cos(theta, N), np.conj(om @ np.cos(j * theta)) / 8, atol=1e-13)
        assert np.allclose(y_sin(theta, N), np.conj(om @ np.sin(j * theta)) / 8, atol=1e-13)
        assert np.allclose(y_exp(theta, N), om @ np.exp(1j * j * theta) / 8, atol=1e-13)
        assert not np.allclose(y_cos(theta, N), om @ np.cos(j * theta) / 8, atol=1e-3)


def test_compressed_chebyshev_rows_match_appendix_a_convolution():
    """Appendix A: a compressed row F(a . w) equals the convolution (eq.
    (conv_appendix)) of the closed-form DFT of the trigonometric row with the
    DFT of the Kaiser window.  The two-sided row a_j = cos((j - s) theta) is
    (e^{i(j-s)theta} + e^{-i(j-s)theta}) / 2, so eq. (y3) gives its DFT."""
    N = 200
    sp = _spec("chebyshev", N)
    sch = S.schedule(N, 1e-8, 1e-3, True)
    (blk,) = sch.blocks
    L = blk.L
    rows = [0, 37, 120, 199]
    comp = M.compress_rows(sp, blk, sch.zeta, rows)
    w_hat = np.fft.fft(S.kaiser_window(L, sch.zeta)) / math.sqrt(L)
    for r, n in enumerate(rows):
        theta = (2 * n + 1) * math.pi / (2 * N)
        a_hat = 0.5 * (np.exp(-1j * blk.off * theta) * y_exp(theta, L)
                       + np.exp(1j * blk.off * theta) * y_exp(-theta, L))
        k = np.arange(L)
        conv = np.array([np.sum(a_hat * w_hat[(q - k) % L]) for q in range(L)]) / math.sqrt(L)
        assert np.abs(conv - comp[r]).max() < 1e-11 * np.abs(comp[r]).max()


def test_chebyshev_row_dft_closed_form_against_sums():
    """The closed-form DFT of an extended Chebyshev row (two geometric series
    with exactly reduced angles) equals the direct sum, including a row and a
    length where one of the series is resonant (theta/2 = pi q / L)."""
    for N, L, off, n in ((64, 80, 8, 5), (64, 81, 8, 63), (100, 160, 30, 0), (8, 16, 0, 1), (4, 8, 2, 0),
                         (6, 12, 3, 1)):
        q = np.arange(-5, L + 5)
        j = np.arange(L)
        th = (2 * n + 1) * math.pi / (2 * N)
        direct = np.array([np.sum(np.cos((j - off) * th) * np.exp(-2j * np.pi * j * qq / L)) for qq in q])
        cf = M.chebyshev_row_dft(n, N, L, off, q)
        assert np.abs(cf - direct).max() <= 1e-13 * np.abs(direct).max(), (N, L, off, n)


@pytest.mark.parametrize("N,eps,two_sided", [(512, 1e-14, True), (300, 1e-10, True), (1000, 1e-8, True),
                                             (4096, 1e-12, True), (700, 1e-10, False)])
def test_appendix_a_truncated_rows_match_fft_rows(N, eps, two_sided):
    """Appendix A with only the window components |m| <= ceil(zeta/pi) + 10:
    the rows agree with the FFT of the windowed rows to under a tenth of
    eps1 * max|Ä| (the Kaiser spectrum outside its main lobe sits at about
    eps1), i.e. below the threshold that decides which elements are kept."""
    sp = _spec("chebyshev", N)
    sch = S.schedule(N, eps, 1e-3, two_sided)
    blk = sch.blocks[0]
    rows = [0, 1, N // 3, N // 2, N - 2, N - 1]
    comp = M.compress_rows(sp, blk, sch.zeta, rows)
    Mw = int(math.ceil(sch.zeta / math.pi)) + 10
    cf = M.compress_rows_appendix_a(sp, blk, sch.zeta, rows, Mw)
    assert np.abs(cf - comp).max() <= max(0.1 * eps, 4e-15) * np.abs(comp).max()


@pytest.mark.parametrize("N", [256, 1000])
def test_appendix_a_needs_about_24_convolutions_at_1e15(N):
    """Appendix A: about 24 convolutions per row give an accuracy of order
    1e-15.  With 25 window components (|m| <= 12) the truncated closed-form
    rows of a two-sided Chebyshev block at accuracy 1e-15 equal the FFT rows
    to 4e-15 of the block maximum; with 17 they do not reach 1e-10."""
    sp = _spec("chebyshev", N)
    sch = S.schedule(N, 1e-15, 1e-3, True)
    blk = sch.blocks[0]
    rows = [0, 1, N // 3, N // 2, N - 2, N - 1]
    comp = M.compress_rows(sp, blk, sch.zeta, rows)
    mx = np.abs(M.compress_rows(sp, blk, sch.zeta, np.arange(N))).max()
    assert np.abs(M.compress_rows_appendix_a(sp, blk, sch.zeta, rows, 12) - comp).max() <= 4e-15 * mx
    assert np.abs(M.compress_rows_appendix_a(sp, blk, sch.zeta, rows, 8) - comp).max() > 1e-10 * mx


# ------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each mutation of the oracle must make one of the pins above fail."""
    # 1. forward DFT used where F* belongs: the identity (comp1) breaks
    real_ifft = np.fft.ifft
    monkeypatch.setattr(M.np.fft, "ifft", lambda a, axis=-1: np.fft.fft(a, axis=axis) / a.shape[axis])
    assert identity_error("legendre", 48) > 1e-3
    monkeypatch.setattr(M.np.fft, "ifft", real_ifft)
    assert identity_error("legendre", 48) < 2e-13

    # 2. conjugate transpose in the adjoint: the exact-transpose property breaks
    real_adjoint = M.apply_adjoint

    def adjoint_conj(plan, y):
        for b in plan.blocks:
            b.kept = b.kept.conj()
        try:
            return real_adjoint(plan, y)
        finally:
            for b in plan.blocks:
                b.kept = b.kept.conj()

    monkeypatch.setattr(M, "apply_adjoint", adjoint_conj)
    sp, fwd, adj = operator_matrices("chebyshev", 40, 1e-6)
    assert np.abs(adj - fwd.T).max() > 1e-3 * np.abs(fwd).max()
    monkeypatch.setattr(M, "apply_adjoint", real_adjoint)

    # 3. a wrong recurrence coefficient in the Legendre family: the scipy values
    #    pin and the orthogonality pin break
    real_rows = F._legendre_rows

    def bad_rows(x, m_hi):
        out = real_rows(x, m_hi)
        out[:, 2:] *= 1.0 + 1e-9
        return out

    monkeypatch.setattr(F, "_legendre_rows", bad_rows)
    sp = F.make_spec("legendre", 64)
    Q = F.dense_matrix(sp, normalise=True)
    assert np.abs(Q.T @ Q - np.eye(64)).max() > 1e-10
    monkeypatch.setattr(F, "_legendre_rows", real_rows)

    # 4. window evaluated as w^{zeta, L} instead of w^{zeta, L-1}: the Kaiser
    #    pin against scipy breaks
    import scipy.signal
    bad = S.kaiser_value(np.arange(64), 65, 20.0)
    assert not np.allclose(bad, scipy.signal.windows.kaiser(64, 20.0, sym=True), rtol=1e-6)
