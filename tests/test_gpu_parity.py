"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Both sides build the plan independently from the same nodes: the Chebyshev
family uses its exact Chebyshev-Gauss angles on both sides; the other families
hand the oracle's Gauss nodes to the library as user nodes, so the matrices are
defined at identical FP64 points (the library's own Gauss nodes are checked
separately against the oracle's).

Tolerances:
  FP64   relative l2 within the bound of tests/fp64_bounds.py, computed from
         the oracle plan and the inputs: the apply's rounding u ||S|| / ||y||
         (S = |K| (|v| + rms v) log2 L, the absolute-value apply), the two
         sides' independent precompute of K (rho u || |K| |v| || / ||y||) and
         8 eps1 for elements within rounding of the threshold; the observed
         error and the bound are printed.  Config 1 (Legendre N = 512,
         eps = 1e-14) gets a bound of about 8e-13, so a defect of 1e-12 of
         the output fails it.  Besides, elementwise relative to max |y|:
         64 u log2(L) / eps2 + 10 eps (FFT rounding of the input amplified by
         up to 1/eps2 through W^{-1}, plus threshold flips).
  FP32   the FFT rounding of Section 2.2's W^{-1}-amplified input dominates:
         relative l2 <= max(10 eps, 1e-5) against the FP64 oracle method.
"""
import functools
import math

import numpy as np
import pytest

from fp64_bounds import adjoint_bound, forward_bound
from oracle import families as F
from oracle import method as M
from paper_2004_11610_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc as mod
    return mod


def spec_for(fam, N, alpha=0.5, beta=-0.5):
    return F.make_spec(fam, N, alpha, beta) if fam == "jacobi" else F.make_spec(fam, N)


@functools.lru_cache(maxsize=32)
def oracle_plan(fam, N, eps, eps2, normalise=False, scheme="auto", alpha=0.5, beta=-0.5):
    sp = spec_for(fam, N, alpha, beta)
    two = None if scheme == "auto" else scheme == "two_sided"
    return M.build(sp, eps, eps2=eps2, normalise=normalise, two_sided=two)


def gpu_plan(xc, fam, N, eps, precision, eps2, normalise=False, scheme="auto", alpha=0.5, beta=-0.5):
    ora = oracle_plan(fam, N, eps, eps2, normalise, scheme, alpha, beta)
    nodes = None if fam == "chebyshev" or normalise else ora.spec.x
    return ora, xc.Plan(fam, N, eps, precision=precision, alpha=alpha, beta=beta, nodes=nodes,
                        normalise=normalise, eps2=eps2, scheme=scheme)


def assert_fp64(ora, X, out, ref, adjoint=False, label=""):
    """out (GPU) against ref (oracle) within the FP64 bound (relative l2)."""
    bound = (adjoint_bound if adjoint else forward_bound)(ora, X, ref)
    err = M.rel_l2(out, ref)
    print(f"fp64 {label} {'adjoint' if adjoint else 'forward'}: rel-l2 {err:.2e} <= bound {bound:.2e}")
    assert err <= bound, (err, bound)


def fp64_tol(ora, eps):
    Lmax = max([b.L for b in ora.blocks] + [8])
    return 64 * U64 * math.log2(Lmax) / ora.schedule.eps2 + 10 * eps


def check_schedule(ora, plan):
    info = plan.info()
    assert info["L"] == [b.L for b in ora.schedule.blocks]
    assert info["j_lo"] == [b.j_lo for b in ora.schedule.blocks]
    assert info["j_hi"] == [b.j_hi for b in ora.schedule.blocks]
    assert info["off"] == [b.off for b in ora.schedule.blocks]
    assert info["m_tail"] == ora.schedule.m_tail
    assert info["zeta"] == pytest.approx(ora.schedule.zeta, rel=1e-13)
    for nnz, b in zip(info["nnz"], ora.blocks):
        total = int(b.nnz_half.sum())
        assert abs(nnz - total) <= max(2, total // 1000)
    return info


def run_both(xc, plan, ora, X, adjoint=False):
    dt = torch.float64 if plan.precision in ("fp64", "fp64pair") else torch.float32
    Xd = torch.from_numpy(X).to("cuda", dt)
    out = plan.apply_adjoint(Xd) if adjoint else plan.apply(Xd)
    torch.cuda.synchronize()
    plan.sync_status()
    ref = M.apply_adjoint(ora, X) if adjoint else M.apply(ora, X)
    return out.double().cpu().numpy(), ref


def max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES_FP64 = [
    ("legendre", 512, 1e-14), ("legendre", 333, 1e-10), ("chebyshev", 256, 1e-12), ("chebyshev", 301, 1e-8),
    ("jacobi", 400, 1e-10), ("laguerre", 256, 1e-10), ("hermite", 200, 1e-10), ("legendre", 97, 0.0),
    ("chebyshev", 64, 0.0),
]


@pytest.mark.parametrize("fam,N,eps", CASES_FP64)
@pytest.mark.parametrize("nrhs", [1, 3, 9])
def test_fp64_forward_and_adjoint_match_oracle(xc, fam, N, eps, nrhs):
    ora, plan = gpu_plan(xc, fam, N, eps, "fp64", 1e-3)
    with plan:
        check_schedule(ora, plan)
        X = inputs.uniform_pm1(N, nrhs, 11)
        y, y_ref = run_both(xc, plan, ora, X)
        tol = fp64_tol(ora, eps)
        assert max_rel(y, y_ref) <= tol
        assert_fp64(ora, X, y, y_ref, label=f"{fam} N={N} eps={eps} R={nrhs}")
        Y = inputs.normal(N, nrhs, 12)
        xa, xa_ref = run_both(xc, plan, ora, Y, adjoint=True)
        assert max_rel(xa, xa_ref) <= tol
        assert_fp64(ora, Y, xa, xa_ref, adjoint=True, label=f"{fam} N={N} eps={eps} R={nrhs}")


@pytest.mark.parametrize("fam,N,eps", [("legendre", 512, 1e-14), ("chebyshev", 1000, 1e-12), ("laguerre", 700, 1e-12),
                                       ("hermite", 400, 1e-10), ("jacobi", 333, 1e-10), ("legendre", 64, 0.0)])
@pytest.mark.parametrize("nrhs", [1, 9])
def test_fp64_pair_matches_oracle(xc, fam, N, eps, nrhs):
    """XC_FP64_PAIR (FP64 vectors and FFTs, band products in FP32 pairs with
    error-free accumulation) meets the FP64 tolerances."""
    ora, plan = gpu_plan(xc, fam, N, eps, "fp64pair", 1e-3)
    with plan:
        check_schedule(ora, plan)
        tol = fp64_tol(ora, eps)
        X = inputs.uniform_pm1(N, nrhs, 13)
        y, y_ref = run_both(xc, plan, ora, X)
        assert max_rel(y, y_ref) <= tol
        Y = inputs.normal(N, nrhs, 14)
        xa, xa_ref = run_both(xc, plan, ora, Y, adjoint=True)
        assert max_rel(xa, xa_ref) <= tol
        # far from unit scale: the per-RHS power-of-two scaling keeps the pairs in range
        y2, y2_ref = run_both(xc, plan, ora, X * 1e200)
        assert max_rel(y2, y2_ref) <= tol
        xa2, xa2_ref = run_both(xc, plan, ora, Y * 1e-200, adjoint=True)
        assert max_rel(xa2, xa2_ref) <= tol


@pytest.mark.parametrize("fam,N,eps", [("legendre", 700, 1e-7), ("jacobi", 515, 1e-7), ("chebyshev", 640, 1e-7),
                                       ("hermite", 300, 1e-7)])
@pytest.mark.parametrize("precision", ["fp32", "fp32c"])
def test_fp32_paths_match_oracle(xc, fam, N, eps, precision):
    ora, plan = gpu_plan(xc, fam, N, eps, precision, 3e-2)
    with plan:
        check_schedule(ora, plan)
        X = inputs.uniform_pm1(N, 17, 21)
        y, y_ref = run_both(xc, plan, ora, X)
        assert M.rel_l2(y, y_ref) <= max(10 * eps, 1e-5)
        xa, xa_ref = run_both(xc, plan, ora, X, adjoint=True)
        assert M.rel_l2(xa, xa_ref) <= max(10 * eps, 1e-5)


@pytest.mark.parametrize("fam,N,precision,nrhs,kernel", [
    ("legendre", 4096, "fp32c", 512, "adj_transpose"),   # bins far apart: transposed right-hand sides
    ("legendre", 4096, "fp32", 512, "adj_transpose"),
    ("hermite", 1500, "fp32", 48, "fwd_reduce"),         # long bands: chunked forward product
    ("laguerre", 1200, "fp64", 5, "fwd_reduce"),
])
def test_wide_and_long_band_paths_match_oracle(xc, fam, N, precision, nrhs, kernel):
    """Many right-hand sides (the adjoint reads a transposed copy of y for
    blocks whose bins start far apart) and long bands (the forward product is
    summed in chunks and reduced): the kernel that marks the path runs, and the
    results match the oracle."""
    eps = 1e-7 if precision != "fp64" else 1e-10
    ora, plan = gpu_plan(xc, fam, N, eps, precision, 1e-3 if precision == "fp64" else 3e-2)
    with plan:
        plan.timing_enable(True)
        plan.timing_read()
        X = inputs.uniform_pm1(N, nrhs, 23)
        y, y_ref = run_both(xc, plan, ora, X)
        Y = inputs.normal(N, nrhs, 24)
        xa, xa_ref = run_both(xc, plan, ora, Y, adjoint=True)
        ran = plan.timing_read()
        plan.timing_enable(False)
        assert kernel in ran
        if precision == "fp64":
            tol = fp64_tol(ora, eps)
            assert max_rel(y, y_ref) <= tol and max_rel(xa, xa_ref) <= tol
            assert_fp64(ora, X, y, y_ref, label=f"{fam} N={N}")
            assert_fp64(ora, Y, xa, xa_ref, adjoint=True, label=f"{fam} N={N}")
        else:
            assert M.rel_l2(y, y_ref) <= max(10 * eps, 1e-5)
            assert M.rel_l2(xa, xa_ref) <= max(10 * eps, 1e-5)


def test_orthonormal_and_block_scheme_variants(xc):
    ora, plan = gpu_plan(xc, "legendre", 256, 1e-12, "fp64", 1e-3, normalise=True)
    with plan:
        X = inputs.normal(256, 4, 31)
        y, y_ref = run_both(xc, plan, ora, X)
        assert max_rel(y, y_ref) <= fp64_tol(ora, 1e-12)
        assert_fp64(ora, X, y, y_ref, label="orthonormal legendre")
        xa, xa_ref = run_both(xc, plan, ora, X, adjoint=True)
        assert max_rel(xa, xa_ref) <= fp64_tol(ora, 1e-12)
        assert_fp64(ora, X, xa, xa_ref, adjoint=True, label="orthonormal legendre")
    ora, plan = gpu_plan(xc, "chebyshev", 200, 1e-10, "fp64", 1e-3, scheme="blocks")
    with plan:
        check_schedule(ora, plan)
        X = inputs.normal(200, 2, 32)
        y, y_ref = run_both(xc, plan, ora, X)
        assert max_rel(y, y_ref) <= fp64_tol(ora, 1e-10)


@pytest.mark.parametrize("alpha,beta", [(3.0, 3.0), (5.0, 1.0), (-0.7, 2.0)])
def test_orthonormal_jacobi_keeps_its_accuracy_for_large_alpha_beta(xc, alpha, beta):
    """The orthonormal variant thresholds the row-weighted compressed matrix
    (Section 5.2: the forward accuracy does not change with alpha and beta):
    same kept elements as the oracle, products equal to the oracle's and
    within the eps1/eps2 level of the dense orthonormal matrix."""
    N, eps = 512, 1e-10
    ora, plan = gpu_plan(xc, "jacobi", N, eps, "fp64", 1e-3, normalise=True, alpha=alpha, beta=beta)
    with plan:
        check_schedule(ora, plan)
        X = inputs.uniform_pm1(N, 3, 33)
        y, y_ref = run_both(xc, plan, ora, X)
        assert max_rel(y, y_ref) <= fp64_tol(ora, eps)
        xa, xa_ref = run_both(xc, plan, ora, X, adjoint=True)
        assert max_rel(xa, xa_ref) <= fp64_tol(ora, eps)
        Q = F.dense_matrix(ora.spec, normalise=True)
        assert M.rel_l2(y, X @ Q.T) <= eps / 1e-3 and M.rel_l2(xa, X @ Q) <= eps / 1e-3


@pytest.mark.parametrize("N", [2, 3, 8, 20, 21, 33])
def test_tiny_and_dense_only_plans(xc, N):
    """N <= tail_max: no compressed block, the whole product is the dense tail."""
    for fam in ("legendre", "chebyshev"):
        ora, plan = gpu_plan(xc, fam, N, 1e-10, "fp64", 1e-3)
        with plan:
            check_schedule(ora, plan)
            X = inputs.uniform_pm1(N, 2, 41)
            y, y_ref = run_both(xc, plan, ora, X)
            assert max_rel(y, y_ref) <= fp64_tol(ora, 1e-10)
            assert_fp64(ora, X, y, y_ref, label=f"{fam} N={N} dense only")
            xa, xa_ref = run_both(xc, plan, ora, X, adjoint=True)
            assert max_rel(xa, xa_ref) <= fp64_tol(ora, 1e-10)
            assert_fp64(ora, X, xa, xa_ref, adjoint=True, label=f"{fam} N={N} dense only")


def test_gauss_nodes_match_oracle(xc):
    for fam, N in (("legendre", 1000), ("jacobi", 777), ("laguerre", 500), ("hermite", 600), ("chebyshev", 300)):
        sp = spec_for(fam, N)
        with xc.Plan(fam, N, 1e-8, alpha=0.5, beta=-0.5) as plan:
            x = plan.nodes()
        tol = 4 * N * U64 * (1 + np.abs(sp.x))
        assert np.all(np.abs(x - sp.x) <= tol), fam


@pytest.mark.parametrize("fam,N,alpha,beta", [
    ("legendre", 4096, 0.0, 0.0), ("legendre", 4097, 0.0, 0.0), ("jacobi", 3000, 0.3, -0.7),
    ("jacobi", 2000, 2.5, 1.0), ("jacobi", 1500, -0.5, 0.5), ("jacobi", 1500, 0.5, 0.5),
    ("jacobi", 1500, -0.5, -0.5), ("jacobi", 1200, -0.3, -0.7), ("laguerre", 4096, 0.0, 0.0), ("hermite", 4096, 0.0, 0.0),
    ("hermite", 4095, 0.0, 0.0), ("legendre", 2, 0.0, 0.0), ("laguerre", 2, 0.0, 0.0), ("hermite", 3, 0.0, 0.0)])
def test_gauss_nodes_of_every_kind_match_oracle(xc, fam, N, alpha, beta):
    """Nodes from the Sturm-count grid and bracketed Newton (and the closed
    forms of the Jacobi polynomials with |alpha| = |beta| = 1/2) against the
    oracle's Golub-Welsch eigenvalues: every node, including the ones at the
    ends of the spectrum and at x = 0."""
    sp = F.make_spec(fam, N, alpha=alpha, beta=beta)
    with xc.Plan(fam, N, 1e-8, alpha=alpha, beta=beta, precision="fp32") as plan:
        x = plan.nodes()
    assert np.all(np.diff(x) > 0)
    assert np.all(np.abs(x - sp.x) <= 4 * N * U64 * (1 + np.abs(sp.x))), fam


def test_leading_dimension_and_host_path(xc):
    ora, plan = gpu_plan(xc, "legendre", 300, 1e-10, "fp64", 1e-3)
    with plan:
        X = inputs.uniform_pm1(300, 5, 51)
        big = torch.zeros((5, 320), dtype=torch.float64, device="cuda")
        big[:, :300] = torch.from_numpy(X).cuda()
        out = torch.full((5, 320), 7.0, dtype=torch.float64, device="cuda")
        import ctypes
        rc = xc._lib.xc_apply(plan.handle, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(out.data_ptr()), 5, 320,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        # output overlapping the input's rows: refused before any launch
        rc = xc._lib.xc_apply(plan.handle, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr() + 8 * 320),
                              5, 320, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == xc.XC_ERR_ARG
        y_ref = M.apply(ora, X)
        o = out.cpu().numpy()
        assert max_rel(o[:, :300], y_ref) <= fp64_tol(ora, 1e-10)
        assert np.all(o[:, 300:] == 7.0)           # padding untouched
        ys = plan.apply(big[:, :300])              # strided input: the output takes its strides
        torch.cuda.synchronize()
        assert ys.stride() == (320, 1)
        assert max_rel(ys.cpu().numpy(), y_ref) <= fp64_tol(ora, 1e-10)
        yh = plan.apply_host(X)
        assert max_rel(yh, y_ref) <= fp64_tol(ora, 1e-10)
        xh = plan.apply_host(X, adjoint=True)
        assert max_rel(xh, M.apply_adjoint(ora, X)) <= fp64_tol(ora, 1e-10)
        # host buffers with ld = 320 > N: only the first N columns move
        wide = np.zeros((5, 320))
        wide[:, :300] = X
        wout = np.full((5, 320), 7.0)
        plan.apply_host(wide, out=wout)
        assert max_rel(wout[:, :300], y_ref) <= fp64_tol(ora, 1e-10) and np.all(wout[:, 300:] == 7.0)
        with pytest.raises(ValueError):
            plan.apply_host(wide, out=np.empty((5, 300)))


def test_dense_matrix_matches_oracle(xc):
    for fam, N, norm in (("legendre", 200, False), ("chebyshev", 150, False), ("laguerre", 180, False),
                         ("hermite", 160, True), ("jacobi", 170, True)):
        sp = spec_for(fam, N)
        A_ref = F.dense_matrix(sp, normalise=norm)
        nodes = None if (fam == "chebyshev" or norm) else sp.x
        with xc.Plan(fam, N, 1e-8, alpha=0.5, beta=-0.5, nodes=nodes, normalise=norm) as plan:
            A = plan.dense_matrix().cpu().numpy()
        tol = 1e-12 if not norm else 1e-10
        assert np.abs(A - A_ref).max() <= tol * np.abs(A_ref).max(), fam


@pytest.mark.parametrize("fam", ["legendre", "chebyshev", "laguerre"])
def test_adjoint_is_the_exact_transpose_on_gpu(xc, fam):
    """<A x, y> = <x, A^T y> for the GPU operator itself (any size)."""
    N = 1500
    with xc.Plan(fam, N, 1e-9) as plan:
        g = np.random.default_rng(7)
        X = torch.from_numpy(g.standard_normal((4, N))).cuda()
        Y = torch.from_numpy(g.standard_normal((4, N))).cuda()
        Ax = plan.apply(X)
        Aty = plan.apply_adjoint(Y)
        lhs = (Ax * Y).sum(dim=1)
        rhs = (X * Aty).sum(dim=1)
        scale = (Ax * Y).abs().sum(dim=1)
        assert torch.all((lhs - rhs).abs() <= 1e-12 * scale)


def test_invalid_calls_return_errors(xc):
    import ctypes
    with xc.Plan("legendre", 64, 1e-8) as plan:
        x = torch.zeros((2, 64), dtype=torch.float64, device="cuda")
        st = ctypes.c_void_p(0)
        assert xc._lib.xc_apply(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 2, 64,
                                st) == xc.XC_ERR_ARG
        y = torch.zeros_like(x)
        assert xc._lib.xc_apply(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 2, 10,
                                st) == xc.XC_ERR_ARG
        assert xc._lib.xc_apply(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 0, 64,
                                st) == xc.XC_OK


@pytest.mark.parametrize("fam,N,eps,power,precision", [
    ("sine", 512, 1e-12, 0, "fp64"), ("sine", 1001, 1e-8, 0, "fp64"), ("cospow", 600, 1e-10, 2, "fp64"),
    ("cospow", 400, 1e-10, 3, "fp64"), ("sine", 700, 1e-7, 0, "fp32"), ("cospow", 500, 1e-7, 4, "fp32c"),
    ("sine", 2048, 1e-12, 0, "fp64pair"),
])
def test_sine_and_cos_power_families_match_oracle(xc, fam, N, eps, power, precision):
    """The sin(m theta_n) and cos^s(m theta_n) matrices (Section 2.2, eq.
    (cosd2)) through the same two-sided method as the Chebyshev family."""
    eps2 = 1e-3 if precision in ("fp64", "fp64pair") else 3e-2
    ora = M.build(F.make_spec(fam, N, power=power or 2), eps, eps2=eps2)
    with xc.Plan(fam, N, eps, precision=precision, eps2=eps2, power=power) as plan:
        check_schedule(ora, plan)
        X = inputs.uniform_pm1(N, 3, 51)
        y, y_ref = run_both(xc, plan, ora, X)
        xa, xa_ref = run_both(xc, plan, ora, X, adjoint=True)
        if precision in ("fp64", "fp64pair"):
            tol = fp64_tol(ora, eps)
            assert max_rel(y, y_ref) <= tol and max_rel(xa, xa_ref) <= tol
        else:
            assert M.rel_l2(y, y_ref) <= max(10 * eps, 1e-5)
            assert M.rel_l2(xa, xa_ref) <= max(10 * eps, 1e-5)
        # the method approximates the plain product to about eps1 / eps2
        y_d = M.dense_apply(ora.spec, X)
        assert M.rel_l2(y, y_d) <= max(10 * eps / eps2, 1e-5)
