"""Pins of the oracle's complex families: the exp matrix exp(i m theta_n) and
the spectral Laguerre matrix C of eq. (lag_matrix).

What fixes them independently of the oracle's own formulas:
- at theta_n = 2 pi n / N the exp matrix is N times numpy's inverse DFT;
- at the default angles (midpoints of N equal arcs) the exp matrix is
  discretely orthogonal (E^H E = N I);
- exact angle reduction agrees with a 50-digit evaluation at large degrees;
- C[j, m] equals the power form (-eta/2 - i k)^m / (eta/2 - i k)^{m+1}
  (repeated complex multiplication) and, independently, the Laplace transform
  of the Laguerre function, (1/eta) int_0^inf exp(i k t) eta l_m(eta t) dt
  (numerical quadrature of scipy's Laguerre polynomials);
- the method with eps1 = 0 reproduces the dense product (the identity of
  eqs. (comp1)/(comp2)); with eps1 > 0 its error is of order eps1;
- the adjoint is the plain transpose (bilinear identity, no conjugation);
- at tiny N the method applied to the identity rebuilds the matrix entrywise;
- planted mistakes (the sign of psi, a conjugated row factor, a conjugate
  transpose, shifted default angles) fail a pin.
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.integrate
import scipy.special

from oracle import families as F
from oracle import method as M


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_exp_at_dft_angles_is_an_inverse_dft():
    N = 50
    spec = F.make_spec("exp", N, x=2 * np.pi * np.arange(N) / N)
    X = crandn(np.random.default_rng(1), 3, N)
    ref = N * np.fft.ifft(X, axis=1)
    assert np.abs(M.dense_apply(spec, X) - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(M.dense_apply_adjoint(spec, X) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_exp_default_angles_are_discretely_orthogonal():
    N = 64
    spec = F.make_spec("exp", N)
    E = F.dense_matrix(spec)
    assert np.allclose(E.conj().T @ E, N * np.eye(N), atol=1e-11)
    assert np.all(np.diff(spec.x) > 0) and spec.x[0] > -np.pi and spec.x[-1] < np.pi


def test_exp_exact_angle_reduction_at_large_degrees():
    N = 1001
    spec = F.make_spec("exp", N)
    rows = np.array([0, 17, 500, 1000])
    m_lo = 10 ** 6
    got = F.values(spec, m_lo, m_lo + 5, rows)
    with mpmath.workdps(50):
        for i, n in enumerate(rows):
            th = mpmath.pi * (2 * int(n) + 1 - N) / N
            for j in range(5):
                ref = complex(mpmath.exp(1j * (m_lo + j) * th))
                assert abs(got[i, j] - ref) <= 2e-15   # unreduced m theta would be ~1e-10 off


@pytest.mark.parametrize("eta,T", [(2500.0, 4.0), (3.0, 10.0), (50.0, 2.0)])
def test_lagspec_entries_equal_the_power_form(eta, T):
    N = 300
    C = F.dense_matrix(F.make_spec("lagspec", N, alpha=eta, beta=T))
    k = 2 * np.pi * np.arange(N) / T
    a, b = -eta / 2 - 1j * k, eta / 2 - 1j * k
    q = 1.0 / b
    u = 2.0 ** -53
    for m in range(N):
        # both forms carry a phase error of order m u (m psi rounded; m products)
        assert np.abs(C[:, m] - q).max() <= (8 + 8 * m) * u * np.abs(q).max(), m
        q = q * a / b


def test_lagspec_entries_are_laplace_transforms_of_laguerre_functions():
    eta, T = 3.0, 10.0
    C = F.dense_matrix(F.make_spec("lagspec", 8, alpha=eta, beta=T))
    for j in range(4):
        kj = 2 * np.pi * j / T
        for m in range(6):
            f = lambda t, part: part(np.exp(1j * kj * t)) * eta * math.exp(-eta * t / 2) * \
                scipy.special.eval_laguerre(m, eta * t)
            re = scipy.integrate.quad(f, 0, 80.0 / eta, args=(np.real,), limit=400, epsabs=1e-13)[0]
            im = scipy.integrate.quad(f, 0, 80.0 / eta, args=(np.imag,), limit=400, epsabs=1e-13)[0]
            assert abs(C[j, m] - (re + 1j * im) / eta) <= 1e-10, (j, m)


def test_lagspec_angles_increase_over_the_lower_half_circle():
    psi = F.make_spec("lagspec", 500, alpha=50.0, beta=2.0).x
    assert psi[0] == -np.pi and np.all(np.diff(psi) > 0) and psi[-1] < 0


def specs():
    rng = np.random.default_rng(5)
    return [
        ("exp default", F.make_spec("exp", 200)),
        ("exp random angles", F.make_spec("exp", 150, x=np.sort(rng.uniform(-np.pi, np.pi, 150)))),
        ("lagspec", F.make_spec("lagspec", 180, alpha=50.0, beta=2.0)),
        ("lagspec narrow", F.make_spec("lagspec", 160, alpha=2500.0, beta=4.0)),
    ]


@pytest.mark.parametrize("name,spec", specs())
def test_complex_method_without_threshold_is_the_dense_product(name, spec):
    rng = np.random.default_rng(7)
    plan = M.build(spec, 0.0, eps2=1e-3)
    assert len(plan.blocks) == 1 and plan.blocks[0].L >= spec.N
    X = crandn(rng, 3, spec.N)
    assert M.rel_l2(M.apply(plan, X), M.dense_apply(spec, X)) <= 1e-11
    assert M.rel_l2(M.apply_adjoint(plan, X), M.dense_apply_adjoint(spec, X)) <= 1e-11


@pytest.mark.parametrize("name,spec", specs())
@pytest.mark.parametrize("eps,eps2", [(1e-6, 1e-3), (1e-10, 1e-3), (1e-8, 1e-2)])
def test_complex_method_error_is_of_order_eps(name, spec, eps, eps2):
    """Section 2.2 bounds the error by eps1 / eps2 (the same bound holds, and
    is reached to within a factor of a few, for the Chebyshev matrix)."""
    rng = np.random.default_rng(8)
    plan = M.build(spec, eps, eps2=eps2)
    X = crandn(rng, 4, spec.N)
    assert M.rel_l2(M.apply(plan, X), M.dense_apply(spec, X)) <= 0.1 * eps / eps2
    assert M.rel_l2(M.apply_adjoint(plan, X), M.dense_apply_adjoint(spec, X)) <= 0.1 * eps / eps2
    # one band per row around the row's angle: a few dozen elements at most
    nnz = np.diff(plan.blocks[0].kept.indptr)
    assert nnz.max() <= 40 and nnz.min() >= 1


def test_complex_adjoint_is_the_plain_transpose():
    spec = F.make_spec("lagspec", 150, alpha=50.0, beta=2.0)
    plan = M.build(spec, 1e-8, eps2=1e-3)
    rng = np.random.default_rng(9)
    x, y = crandn(rng, spec.N), crandn(rng, spec.N)
    lhs = np.sum(y * M.apply(plan, x))
    rhs = np.sum(M.apply_adjoint(plan, y) * x)
    assert abs(lhs - rhs) <= 1e-13 * np.abs(M.apply(plan, x)).sum() * np.abs(y).max()


@pytest.mark.parametrize("fam", ["exp", "lagspec"])
def test_complex_method_rebuilds_tiny_matrices_entrywise(fam):
    for N in (1, 2, 5, 24):
        spec = F.make_spec(fam, N, alpha=40.0, beta=3.0) if fam == "lagspec" else F.make_spec("exp", N)
        plan = M.build(spec, 0.0, eps2=1e-3)
        A = M.apply(plan, np.eye(N, dtype=np.complex128)).T      # column m = A e_m
        ref = F.dense_matrix(spec)
        assert np.abs(A - ref).max() <= 1e-11 * np.abs(ref).max(), N


# ------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each mutation of the complex oracle must make one of the pins above fail."""
    eta, T, N = 50.0, 2.0, 40
    k = 2 * np.pi * np.arange(N) / T

    def power_form_error():
        C = F.dense_matrix(F.make_spec("lagspec", N, alpha=eta, beta=T))
        a, b = -eta / 2 - 1j * k, eta / 2 - 1j * k
        ref = np.stack([a ** m / b ** (m + 1) for m in range(N)], axis=1)
        return np.abs(C - ref).max() / np.abs(ref).max()

    assert power_form_error() < 1e-12

    # 1. psi with the wrong sign (exp(-i m psi)): the power-form pin breaks
    real_angles = F.lagspec_angles
    monkeypatch.setattr(F, "lagspec_angles", lambda n, e, p: -real_angles(n, e, p))
    assert power_form_error() > 1e-3
    monkeypatch.setattr(F, "lagspec_angles", real_angles)

    # 2. the row factor conjugated, 1/(eta/2 + i k): the power-form pin breaks
    real_factor = F.lagspec_row_factor
    monkeypatch.setattr(F, "lagspec_row_factor", lambda n, e, p: np.conj(real_factor(n, e, p)))
    assert power_form_error() > 1e-3
    monkeypatch.setattr(F, "lagspec_row_factor", real_factor)
    assert power_form_error() < 1e-12

    # 3. conjugate transpose in the adjoint: the bilinear transpose pin breaks
    spec = F.make_spec("lagspec", 150, alpha=50.0, beta=2.0)
    plan = M.build(spec, 1e-8, eps2=1e-3)
    rng = np.random.default_rng(9)
    x, y = crandn(rng, spec.N), crandn(rng, spec.N)
    lhs = np.sum(y * M.apply(plan, x))
    for b in plan.blocks:
        b.kept = b.kept.conj()
    assert abs(lhs - np.sum(M.apply_adjoint(plan, y) * x)) > 1e-6 * abs(lhs)

    # 4. default exp angles shifted by half an arc (2 n - N instead of
    #    2 n + 1 - N): still orthogonal, but the first angle reaches -pi, which
    #    the angle pin rules out
    real_default = F.exp_default_angles
    monkeypatch.setattr(F, "exp_default_angles", lambda n: (real_default(n)[0] - 1, n))
    x0 = F.make_spec("exp", 64).x[0]
    monkeypatch.setattr(F, "exp_default_angles", real_default)
    assert not x0 > -np.pi
