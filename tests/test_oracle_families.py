"""Pins for oracle/families.py: nodes, weights and matrix entries against
independent libraries (numpy, scipy, mpmath), closed forms and Gauss-quadrature
orthogonality."""
import math

import mpmath
import numpy as np
import pytest
import scipy.fft
import scipy.special

from oracle import families as F


@pytest.mark.parametrize("N", [5, 17, 64, 100])
def test_nodes_match_numpy_gauss_rules(N):
    assert np.allclose(F.gauss_nodes("legendre", N), np.polynomial.legendre.leggauss(N)[0],
                       rtol=0, atol=4e-16)
    # the FP64 recurrence fixes L_N near its small roots to ~1e-15 absolute
    assert np.allclose(F.gauss_nodes("laguerre", N), np.polynomial.laguerre.laggauss(N)[0],
                       rtol=4e-15, atol=2e-15)
    assert np.allclose(F.gauss_nodes("hermite", N), np.polynomial.hermite.hermgauss(N)[0],
                       rtol=0, atol=4e-15)


def test_laguerre_hermite_extreme_nodes_against_mpmath():
    """Newton on the FP64 recurrence fixes a root to about N u (1 + |x|)
    absolutely: the recurrence value carries an absolute error of order N u."""
    N = 200
    tol = lambda r: 2 * N * 1.1e-16 * (1 + abs(r))
    x = F.gauss_nodes("laguerre", N)
    with mpmath.workdps(40):
        for i in (0, 1, N // 2, N - 1):
            r = mpmath.findroot(lambda t: mpmath.exp(-t / 2) * mpmath.laguerre(N, 0, t), mpmath.mpf(x[i]),
                                tol=1e-60, verify=False)
            assert abs(x[i] - float(r)) <= tol(float(r))
    x = F.gauss_nodes("hermite", N)
    with mpmath.workdps(40):
        for i in (0, N // 2, N - 1):
            r = mpmath.findroot(lambda t: mpmath.exp(-t * t / 2) * mpmath.hermite(N, t) / mpmath.sqrt(
                    mpmath.mpf(2) ** N * mpmath.factorial(N)), mpmath.mpf(x[i]), tol=1e-60, verify=False)
            assert abs(x[i] - float(r)) <= tol(float(r))


@pytest.mark.parametrize("ab", [(0.5, -0.5), (1.0, 1.0), (-0.3, 2.5), (0.0, 0.0), (-0.5, -0.5), (-0.3, -0.7)])
def test_jacobi_nodes_match_scipy_roots(ab):
    a, b = ab
    for N in (7, 60):
        ref = scipy.special.roots_jacobi(N, a, b)[0]
        assert np.allclose(F.gauss_nodes("jacobi", N, a, b), np.sort(ref), rtol=0, atol=1e-14)


def test_jacobi_half_minus_half_nodes_closed_form():
    # P_N^{(1/2,-1/2)}(cos t) is proportional to sin((N+1/2)t)/sin(t/2): zeros t_k = 2k pi/(2N+1)
    for N in (31, 1000):
        k = np.arange(1, N + 1)
        ref = np.sort(np.cos(2 * k * np.pi / (2 * N + 1)))
        assert np.allclose(F.gauss_nodes("jacobi", N, 0.5, -0.5), ref, rtol=0, atol=2e-15)


def test_jacobi_nodes_of_the_chebyshev_kinds_closed_form():
    """alpha = beta = -1/2 and 1/2 are the Chebyshev polynomials of the first and
    second kind, alpha = -1/2, beta = 1/2 the third kind: zeros cos((2k-1) pi /
    (2N)), cos(k pi / (N+1)) and cos((2k-1) pi / (2N+1)).  alpha + beta = -1
    makes the k = 1 entry of the Jacobi matrix a removable 0/0."""
    for N in (2, 31, 1000):
        k = np.arange(1, N + 1)
        for (a, b), t in (((-0.5, -0.5), (2 * k - 1) / (2 * N)), ((0.5, 0.5), k / (N + 1)),
                          ((-0.5, 0.5), (2 * k - 1) / (2 * N + 1))):
            ref = np.sort(np.cos(t * np.pi))
            assert np.allclose(F.gauss_nodes("jacobi", N, a, b), ref, rtol=0, atol=2e-15), (a, b, N)


def test_chebyshev_gauss_points():
    N = 12
    x = F.gauss_nodes("chebyshev", N)
    assert np.allclose(x, np.cos((2 * np.arange(N) + 1) * np.pi / (2 * N)), atol=0)


def test_polynomial_values_match_scipy():
    x = np.linspace(-1, 1, 37)
    sp = F.Spec("legendre", 37, x)
    m = 120
    V = F.values(sp, 0, m)
    ref = np.stack([scipy.special.eval_legendre(k, x) for k in range(m)], axis=1)
    assert np.allclose(V, ref, rtol=1e-12, atol=1e-13)
    for a, b in ((0.5, -0.5), (1.5, 0.25)):
        sp = F.Spec("jacobi", 37, x, a, b)
        V = F.values(sp, 3, m)
        ref = np.stack([scipy.special.eval_jacobi(k, a, b, x) for k in range(3, m)], axis=1)
        assert np.allclose(V, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_jacobi_half_minus_half_closed_form():
    # P_n^{(1/2,-1/2)}(cos t) = binom(2n, n)/4^n * sin((n+1/2) t) / sin(t/2)
    t = np.linspace(0.05, 3.1, 29)
    sp = F.Spec("jacobi", t.size, np.cos(t), 0.5, -0.5)
    n = np.arange(200)
    V = F.values(sp, 0, 200)
    c = np.exp(scipy.special.gammaln(2 * n + 1) - 2 * scipy.special.gammaln(n + 1) - n * math.log(4))
    ref = c[None, :] * np.sin((n[None, :] + 0.5) * t[:, None]) / np.sin(t[:, None] / 2)
    assert np.allclose(V, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_laguerre_function_values():
    x = np.array([0.0, 0.1, 1.0, 7.5, 30.0])
    sp = F.Spec("laguerre", x.size, x)
    V = F.values(sp, 0, 60)
    ref = np.stack([scipy.special.eval_laguerre(k, x) * np.exp(-x / 2) for k in range(60)], axis=1)
    assert np.allclose(V, ref, rtol=1e-11, atol=1e-13)
    # far outside the FP64 range of exp(-x/2) (x ~ 4N at N = 4096): mpmath at 50 digits
    x = np.array([1500.0, 9000.0, 16300.0])
    sp = F.Spec("laguerre", x.size, x)
    cols = [300, 2300, 4090]
    V = F.values(sp, 0, 4091)
    with mpmath.workdps(60):
        for i, xv in enumerate(x):
            for m in cols:
                ref = mpmath.exp(-mpmath.mpf(xv) / 2) * mpmath.laguerre(m, 0, mpmath.mpf(xv))
                assert abs(V[i, m] - float(ref)) <= 1e-12 * max(abs(float(ref)), 1e-300) + 1e-300


def test_hermite_function_values():
    x = np.array([-3.0, -0.2, 0.0, 1.3, 5.0])
    sp = F.Spec("hermite", x.size, x)
    V = F.values(sp, 0, 40)
    ref = np.stack([scipy.special.eval_hermite(k, x) * np.exp(-x * x / 2)
                    / math.sqrt(2.0 ** k * math.factorial(k) * math.sqrt(math.pi)) for k in range(40)],
                   axis=1)
    assert np.allclose(V, ref, rtol=1e-11, atol=1e-13)
    x = np.array([40.0, 90.0])
    sp = F.Spec("hermite", x.size, x)
    V = F.values(sp, 0, 4200)
    with mpmath.workdps(80):
        for i, xv in enumerate(x):
            for m in (1000, 4199):
                X = mpmath.mpf(xv)
                ref = (mpmath.hermite(m, X) * mpmath.exp(-X * X / 2)
                       / mpmath.sqrt(mpmath.mpf(2) ** m * mpmath.factorial(m) * mpmath.sqrt(mpmath.pi)))
                assert abs(V[i, m] - float(ref)) <= 1e-11 * max(abs(float(ref)), 1e-300) + 1e-300


def test_chebyshev_exact_angles():
    N = 4096
    sp = F.make_spec("chebyshev", N)
    rows = [0, 1, 777, 4095]
    V = F.values(sp, -900, 5000, rows)
    with mpmath.workdps(40):
        for i, n in enumerate(rows):
            for m in (-900, -1, 0, 1, 2500, 4999):
                ref = mpmath.cos(m * (2 * n + 1) * mpmath.pi / (2 * N))
                assert abs(V[i, m + 900] - float(ref)) < 5e-16


def test_chebyshev_dense_matvec_is_dct3():
    # At Chebyshev-Gauss points y_n = sum_k x_k cos(k(2n+1)pi/(2N)) = (DCT-III(x)_n + x_0)/2
    N = 300
    sp = F.make_spec("chebyshev", N)
    x = np.random.default_rng(5).standard_normal(N)
    y = F.dense_matrix(sp) @ x
    ref = (scipy.fft.dct(x, type=3) + x[0]) / 2
    assert np.allclose(y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("N", [5, 30, 90])
def test_weights_match_numpy(N):
    for fam, ref in (("legendre", np.polynomial.legendre.leggauss(N)),
                     ("laguerre", np.polynomial.laguerre.laggauss(N)),
                     ("hermite", np.polynomial.hermite.hermgauss(N))):
        sp = F.make_spec(fam, N)
        lam = F.quadrature_weights(sp)
        w = ref[1]
        if fam == "laguerre":
            w = w * np.exp(ref[0])
        if fam == "hermite":
            w = w * np.exp(ref[0] ** 2)
        assert np.allclose(lam, w, rtol=1e-12)
    for a, b in ((0.5, -0.5), (1.0, 2.0)):
        sp = F.make_spec("jacobi", N, a, b)
        assert np.allclose(F.quadrature_weights(sp), scipy.special.roots_jacobi(N, a, b)[1], rtol=1e-12)


@pytest.mark.parametrize("fam,N", [("chebyshev", 256), ("legendre", 512), ("jacobi", 400),
                                   ("laguerre", 300), ("hermite", 300)])
def test_orthonormal_matrix_is_orthogonal(fam, N):
    """Section 5.2: with Gauss quadrature the normalised matrix is orthogonal.
    The smallest Gauss-Laguerre nodes are fixed only to ~N u absolutely by the
    FP64 recurrence (relative ~1e-13), which bounds the Laguerre case."""
    sp = F.make_spec(fam, N, 0.5, -0.5) if fam == "jacobi" else F.make_spec(fam, N)
    Q = F.dense_matrix(sp, normalise=True)
    err = np.abs(Q.T @ Q - np.eye(N)).max()
    assert err < (5e-11 if fam == "laguerre" else 2e-12)


# ------------------------------------------------- sine and cos^s families

@pytest.mark.parametrize("N", [8, 63, 256])
def test_sine_matvec_is_a_dst(N):
    """sum_m x_m sin(m theta_n), theta_n = (2n+1) pi / (2N), m < N, is half of
    scipy's DST-III of (x_1, ..., x_{N-1}, 0)."""
    sp = F.make_spec("sine", N)
    x = np.random.default_rng(N).standard_normal(N)
    y = F.dense_matrix(sp) @ x
    xs = np.concatenate([x[1:], [0.0]])
    assert np.allclose(y, scipy.fft.dst(xs, type=3) / 2, rtol=0, atol=1e-12 * np.abs(x).sum())


@pytest.mark.parametrize("N", [16, 100])
def test_sine_discrete_orthogonality(N):
    """sum_n sin(m theta_n) sin(k theta_n) = (N/2) delta_mk for 1 <= m, k < N."""
    S = F.dense_matrix(F.make_spec("sine", N))[:, 1:]
    assert np.abs(S.T @ S - (N / 2) * np.eye(N - 1)).max() < 1e-11 * N


@pytest.mark.parametrize("s", [1, 2, 3, 5])
def test_cospow_is_a_sum_of_chebyshev_matrices(s):
    """cos^s(m theta) = 2^-s sum_k C(s, k) cos((s - 2k) m theta): the cos^s
    matrix equals the binomial combination of Chebyshev matrices at the nodes
    cos((s - 2k) theta_n) (generated through arccos, not the exact angles)."""
    N = 97
    sp = F.make_spec("cospow", N, power=s)
    th = (2 * np.arange(N) + 1) * np.pi / (2 * N)
    acc = np.zeros((N, N))
    for k in range(s + 1):
        acc += math.comb(s, k) * F.dense_matrix(F.make_spec("chebyshev", N, x=np.cos((s - 2 * k) * th)))
    assert np.abs(F.dense_matrix(sp) - acc / 2 ** s).max() < 1e-12
