"""GPU parity of the complex families (exp(i m theta_n) and the spectral
Laguerre matrix C of eq. (lag_matrix)) against the FP64 oracle, through the C
ABI: forward and plain-transpose adjoint, element by element, on the same
seeded inputs; the row bands and bin runs wrap around the spectrum, so the
cases include angles on both sides of +-pi, unsorted angles, several tiles and
ragged tails; plus the full-size sampled check, the bilinear transpose
identity, the dense matrix, the host path, autograd and the refusals."""
import math

import numpy as np
import pytest

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


def cinput(N, R, seed):
    return inputs.complex_normal(N, R, seed)


def run(plan, X, adjoint=False):
    dt = torch.complex128 if plan.precision == "fp64" else torch.complex64
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda", dt)
    out = plan.apply_adjoint(Xd) if adjoint else plan.apply(Xd)
    torch.cuda.synchronize()
    plan.sync_status()
    return out.to(torch.complex128).cpu().numpy()


def max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def oracle_spec(plan, fam, N, nodes=None, eta=0.0, T=0.0):
    """The oracle's spec at the plan's own angles where they come from a
    floating-point formula (spectral Laguerre), after checking them."""
    if fam == "lagspec":
        got = plan.nodes()
        ref = F.lagspec_angles(N, eta, T)
        assert np.abs(got - ref).max() <= 8 * U64 * math.pi
        return F.Spec("lagspec", N, got, eta, T)
    if nodes is not None:
        return F.make_spec("exp", N, x=nodes)
    return F.make_spec("exp", N)


def angles(kind, N, seed=3):
    rng = np.random.default_rng(seed)
    if kind == "sorted":
        return np.sort(rng.uniform(-math.pi, math.pi, N))
    if kind == "unsorted":
        return rng.uniform(-math.pi, math.pi, N)
    if kind == "wide":            # beyond (-pi, pi): the same rows, other branches
        return np.sort(rng.uniform(-3 * math.pi, 3 * math.pi, N))
    if kind == "dft":
        return 2 * math.pi * np.arange(N) / N
    return None


CASES = [  # family, N, eps, nodes kind, eta, T
    ("exp", 64, 1e-12, None, 0, 0), ("exp", 300, 1e-10, None, 0, 0), ("exp", 1001, 1e-14, None, 0, 0),
    ("exp", 777, 1e-12, "sorted", 0, 0), ("exp", 500, 1e-10, "unsorted", 0, 0), ("exp", 400, 1e-10, "wide", 0, 0),
    ("exp", 256, 1e-12, "dft", 0, 0), ("exp", 200, 0.0, None, 0, 0), ("exp", 2, 1e-10, None, 0, 0),
    ("lagspec", 649, 1e-10, None, 2500.0, 4.0), ("lagspec", 1000, 1e-12, None, 50.0, 2.0),
    ("lagspec", 97, 1e-8, None, 3.0, 10.0), ("lagspec", 3000, 1e-10, None, 50.0, 0.5),
]


@pytest.mark.parametrize("fam,N,eps,kind,eta,T", CASES)
@pytest.mark.parametrize("nrhs", [1, 5, 33])
def test_fp64_matches_oracle(xc, fam, N, eps, kind, eta, T, nrhs):
    nodes = angles(kind, N)
    with xc.Plan(fam, N, eps, precision="fp64", nodes=nodes, eta=eta, period=T) as plan:
        spec = oracle_spec(plan, fam, N, nodes, eta, T)
        ora = M.build(spec, eps, eps2=1e-3)
        info = plan.info()
        assert info["L"] == [b.L for b in ora.blocks] and info["nblocks"] == 1
        assert info["nnz"][0] == ora.blocks[0].kept.nnz or eps > 0
        assert abs(info["nnz"][0] - ora.blocks[0].kept.nnz) <= max(4, ora.blocks[0].kept.nnz // 1000)
        X = cinput(N, nrhs, 11)
        Y = cinput(N, nrhs, 12)
        tol = 64 * U64 * math.log2(ora.blocks[0].L) / 1e-3 + 10 * eps
        assert max_rel(run(plan, X), M.apply(ora, X)) <= tol
        assert max_rel(run(plan, Y, True), M.apply_adjoint(ora, Y)) <= tol


@pytest.mark.parametrize("fam,N,eps,eta,T", [("exp", 1500, 1e-6, 0, 0), ("lagspec", 1200, 1e-6, 40.0, 2.0),
                                             ("exp", 333, 1e-5, 0, 0)])
def test_fp32_matches_oracle(xc, fam, N, eps, eta, T):
    with xc.Plan(fam, N, eps, precision="fp32", eta=eta, period=T) as plan:
        spec = oracle_spec(plan, fam, N, None, eta, T)
        ora = M.build(spec, eps, eps2=plan.info()["eps2"])
        X = cinput(N, 9, 21)
        assert M.rel_l2(run(plan, X), M.apply(ora, X)) <= max(10 * eps, 1e-5)
        assert M.rel_l2(run(plan, X, True), M.apply_adjoint(ora, X)) <= max(10 * eps, 1e-5)
        # and against the plain product
        assert M.rel_l2(run(plan, X), M.dense_apply(spec, X)) <= max(10 * eps, 2e-5)


def test_full_size_sampled_rows_and_transpose_identity(xc):
    """N = 19000 exp plan at FP64 (L = 27648, near the limit of 28928 set by
    L/2 FP64 values per CTA): sampled rows of the forward product against the
    oracle built on those rows, and the bilinear identity
    y . (A x) = (A^T y) . x on all of it."""
    N, eps, R = 19000, 1e-10, 8
    with xc.Plan("exp", N, eps, precision="fp64") as plan:
        spec = F.make_spec("exp", N)
        rows = np.sort(np.random.default_rng(4).choice(N, 48, replace=False))
        rows = np.unique(np.concatenate([rows, [0, 31, 32, N - 1]]))
        ora = M.build(spec, eps, eps2=1e-3, rows=rows)
        X = cinput(N, R, 31)
        y = run(plan, X)
        ref = M.apply(ora, X)
        assert max_rel(y[:, rows], ref) <= 64 * U64 * math.log2(ora.blocks[0].L) / 1e-3 + 10 * eps
        Y = cinput(N, R, 32)
        xa = run(plan, Y, True)
        lhs = np.sum(Y * y, axis=1)
        rhs = np.sum(xa * X, axis=1)
        scale = np.abs(Y).sum(axis=1) * np.abs(y).max(axis=1)
        assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)


def test_dense_matrix_host_path_and_leading_dimension(xc):
    N = 150
    with xc.Plan("lagspec", N, 1e-12, eta=50.0, period=2.0) as plan:
        spec = F.Spec("lagspec", N, plan.nodes(), 50.0, 2.0)
        A = plan.dense_matrix().cpu().numpy()
        ref = F.dense_matrix(spec)
        assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()
        X = cinput(N, 3, 41)
        dev = run(plan, X)
        host = plan.apply_host(X)
        assert np.array_equal(dev, host)
        hosta = plan.apply_host(X, adjoint=True)
        assert np.array_equal(run(plan, X, True), hosta)
        # ld > N: a strided view of a wider buffer
        wide = torch.zeros((3, N + 17), dtype=torch.complex128, device="cuda")
        wide[:, :N] = torch.from_numpy(X).to("cuda")
        out = torch.zeros_like(wide)
        plan.apply(wide[:, :N], out=out[:, :N])
        torch.cuda.synchronize()
        assert np.array_equal(out[:, :N].cpu().numpy(), dev)
        assert torch.count_nonzero(out[:, N:]).item() == 0


def test_autograd_gives_the_conjugate_transpose(xc):
    N = 64
    with xc.Plan("exp", N, 0.0, precision="fp64") as plan:
        A = F.dense_matrix(F.make_spec("exp", N))
        x = torch.from_numpy(cinput(N, 2, 51)).to("cuda").requires_grad_(True)
        w = torch.from_numpy(cinput(N, 2, 52)).to("cuda")
        y = xc.xc_apply_autograd(x, plan)
        loss = torch.real(torch.sum(torch.conj(w) * y))
        loss.backward()
        ref = w.cpu().numpy() @ A.conj()          # rows of A^H w
        assert np.abs(x.grad.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


def test_complex_plans_refuse_what_they_do_not_support(xc):
    with xc.Plan("exp", 128, 1e-8) as plan:
        with pytest.raises(xc.XcError) as e:
            xc.Batch([plan])
        assert e.value.code == xc.XC_ERR_UNSUPPORTED
        X = torch.zeros((1, 128), dtype=torch.complex128, device="cuda")
        with pytest.raises(xc.XcError) as e:
            plan.apply_noalloc(X, torch.empty_like(X))
        assert e.value.code == xc.XC_ERR_UNSUPPORTED
        with pytest.raises(ValueError):
            plan.apply(X.conj())
    for kw, code in ((dict(precision="fp32c"), xc.XC_ERR_UNSUPPORTED),
                     (dict(precision="fp64pair"), xc.XC_ERR_UNSUPPORTED),
                     (dict(scheme="blocks"), xc.XC_ERR_UNSUPPORTED),
                     (dict(normalise=True), xc.XC_ERR_UNSUPPORTED)):
        with pytest.raises(xc.XcError) as e:
            xc.Plan("exp", 100, 1e-8, **kw)
        assert e.value.code == code, kw
    with pytest.raises(xc.XcError) as e:
        xc.Plan("lagspec", 100, 1e-8, eta=0.0, period=2.0)
    assert e.value.code == xc.XC_ERR_ARG
    with pytest.raises(xc.XcError) as e:   # L/2 FP64 values above one CTA's shared memory
        xc.Plan("exp", 30000, 1e-8)
    assert e.value.code == xc.XC_ERR_UNSUPPORTED


def test_bench_size_spectral_laguerre(xc):
    """The bench's spectral Laguerre workload (eta = 2500, T = 4, N = 8192,
    eps1 = 1e-12, FP64): forward and transpose of 3 right-hand sides against
    the oracle at the plan's angles."""
    N, eps, eta, T = 8192, 1e-12, 2500.0, 4.0
    with xc.Plan("lagspec", N, eps, precision="fp64", eta=eta, period=T) as plan:
        spec = oracle_spec(plan, "lagspec", N, None, eta, T)
        ora = M.build(spec, eps, eps2=1e-3)
        X = cinput(N, 3, 71)
        tol = 64 * U64 * math.log2(ora.blocks[0].L) / 1e-3 + 10 * eps
        assert max_rel(run(plan, X), M.apply(ora, X)) <= tol
        assert max_rel(run(plan, X, True), M.apply_adjoint(ora, X)) <= tol
