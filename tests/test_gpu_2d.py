"""GPU parity of the 2-D block scheme (eq. (comp_2d), Sections 4.2 and 5.3)
against the FP64 oracle through the C ABI: forward and transpose on seeded
inputs for Laguerre / Hermite functions at equispaced nodes and the index
kernels A^[1], A^[2]; the decomposition's counts, the dense matrix, the host
path and the refusals."""
import numpy as np
import pytest

from oracle import method as M
from oracle import method2d as M2
from paper_2004_11610_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc as mod
    return mod


def spec_of(fam, N, eta=None, x0=None, h=None):
    if fam == "laguerre":     # the Laguerre transform's points t_i = 12 (i + 1) / (N - 1), x = eta t
        h = 12.0 * eta / (N - 1)
        return M2.Spec2D("laguerre", N, h, h)
    if fam == "hermite":
        return M2.Spec2D("hermite", N, x0, h)
    return M2.Spec2D(fam, N)


def make(xc, spec, eps, precision="fp64", eps2=0.0):
    nodes = spec.nodes(0, spec.N) if spec.family in ("laguerre", "hermite") else None
    return xc.Plan(spec.family, spec.N, eps, precision=precision, nodes=nodes, scheme="2d", eps2=eps2)


def run(plan, X, adjoint=False):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda", dt)
    out = plan.apply_adjoint(Xd) if adjoint else plan.apply(Xd)
    torch.cuda.synchronize()
    plan.sync_status()
    return out.double().cpu().numpy()


def max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [  # family, N, eps, spec parameters
    ("laguerre", 300, 1e-10, dict(eta=20.0)), ("laguerre", 1000, 1e-10, dict(eta=100.0)),
    ("hermite", 260, 1e-9, dict(x0=-12.0, h=0.09)), ("a1", 240, 1e-8, {}), ("a2", 250, 1e-8, {}),
    ("a2", 1024, 1e-10, {}), ("a2", 150, 0.0, {}), ("laguerre", 64, 0.0, dict(eta=5.0)),
    ("a1", 21, 1e-8, {}), ("a1", 1024, 1e-8, {}),
]


@pytest.mark.parametrize("fam,N,eps,kw", CASES)
@pytest.mark.parametrize("nrhs", [1, 6])
def test_fp64_matches_oracle(xc, fam, N, eps, kw, nrhs):
    spec = spec_of(fam, N, **kw)
    with make(xc, spec, eps, eps2=1e-3) as plan:
        ora = M2.build(spec, eps, eps2=1e-3)
        info = plan.info()
        assert info["blocks2d"] == len(ora.blocks) and info["dense2d"] == len(ora.dense)
        kept = sum(b.kept.nnz for b in ora.blocks)
        if eps == 0:   # every element (the oracle's sparse matrix leaves out exact zeros)
            assert info["nnz2d"] == sum(b.Lr * b.Lc for b in ora.blocks)
        assert abs(info["nnz2d"] - kept) <= max(8, kept // 1000)
        assert info["dense_elems2d"] == sum((d.r1 - d.r0) * (d.c1 - d.c0) for d in ora.dense)
        X = inputs.normal(N, nrhs, 61)
        Y = inputs.normal(N, nrhs, 62)
        tol = 1e-10 + 10 * eps
        assert max_rel(run(plan, X), M2.apply(ora, X)) <= tol
        assert max_rel(run(plan, Y, True), M2.apply_adjoint(ora, Y)) <= tol


@pytest.mark.parametrize("fam,N,eps,kw", [("laguerre", 600, 1e-5, dict(eta=50.0)), ("a2", 700, 1e-5, {}),
                                          ("hermite", 400, 1e-5, dict(x0=-15.0, h=0.075))])
def test_fp32_matches_oracle(xc, fam, N, eps, kw):
    spec = spec_of(fam, N, **kw)
    with make(xc, spec, eps, precision="fp32") as plan:
        ora = M2.build(spec, eps, eps2=plan.info()["eps2"])
        X = inputs.normal(N, 5, 63)
        assert M.rel_l2(run(plan, X), M2.apply(ora, X)) <= max(10 * eps, 1e-4)
        assert M.rel_l2(run(plan, X, True), M2.apply_adjoint(ora, X)) <= max(10 * eps, 1e-4)


def test_dense_matrix_host_path_and_leading_dimension(xc):
    for spec in (spec_of("laguerre", 200, eta=30.0), spec_of("a1", 150), spec_of("a2", 160)):
        with make(xc, spec, 1e-10) as plan:
            A = plan.dense_matrix().cpu().numpy()
            ref = M2.dense_matrix(spec)
            assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max(), spec.family
            X = inputs.normal(spec.N, 3, 64)
            dev = run(plan, X)
            assert np.array_equal(plan.apply_host(X), dev)
            assert np.array_equal(plan.apply_host(X, adjoint=True), run(plan, X, True))
            wide = torch.zeros((3, spec.N + 9), dtype=torch.float64, device="cuda")
            wide[:, :spec.N] = torch.from_numpy(X).to("cuda")
            out = torch.zeros_like(wide)
            plan.apply(wide[:, :spec.N], out=out[:, :spec.N])
            torch.cuda.synchronize()
            assert np.array_equal(out[:, :spec.N].cpu().numpy(), dev)
            assert torch.count_nonzero(out[:, spec.N:]).item() == 0


def test_2d_plans_refuse_what_they_do_not_support(xc):
    spec = spec_of("a2", 128)
    with make(xc, spec, 1e-8) as plan:
        with pytest.raises(xc.XcError) as e:
            xc.Batch([plan])
        assert e.value.code == xc.XC_ERR_UNSUPPORTED
        X = torch.zeros((1, 128), dtype=torch.float64, device="cuda")
        with pytest.raises(xc.XcError) as e:
            plan.apply_noalloc(X, torch.empty_like(X))
        assert e.value.code == xc.XC_ERR_UNSUPPORTED
    x = np.linspace(0.5, 40.0, 200)
    x[7] += 1e-3                       # not equispaced
    with pytest.raises(xc.XcError) as e:
        xc.Plan("laguerre", 200, 1e-8, nodes=x, scheme="2d")
    assert e.value.code == xc.XC_ERR_ARG
    with pytest.raises(xc.XcError) as e:
        xc.Plan("a1", 100, 1e-8, scheme="blocks")
    assert e.value.code == xc.XC_ERR_ARG
    with pytest.raises(xc.XcError) as e:
        xc.Plan("a2", 100, 1e-8, precision="fp32c")
    assert e.value.code == xc.XC_ERR_UNSUPPORTED
    with pytest.raises(xc.XcError) as e:
        xc.Plan("legendre", 100, 1e-8, nodes=np.linspace(-0.9, 0.9, 100), scheme="2d")
    assert e.value.code == xc.XC_ERR_UNSUPPORTED


def test_a1_leaves_out_the_rectangles_below_its_diagonal(xc):
    """A^[1] is zero below its diagonal: the plan holds exactly the oracle's
    blocks and dense rectangles, none of them wholly below the diagonal, and
    still gives the dense product at eps1 = 0."""
    spec = spec_of("a1", 600)
    with make(xc, spec, 0.0, eps2=1e-3) as plan:
        ora = M2.build(spec, 0.0, eps2=1e-3)
        info = plan.info()
        assert info["blocks2d"] == len(ora.blocks) and info["dense2d"] == len(ora.dense)
        stored = info["nnz2d"] + info["dense_elems2d"]
        assert stored == sum(b.Lr * b.Lc for b in ora.blocks) + sum((d.r1 - d.r0) * (d.c1 - d.c0) for d in ora.dense)
        X = inputs.normal(600, 3, 66)
        D = M2.dense_matrix(spec)
        assert max_rel(run(plan, X), X @ D.T) <= 1e-10
        assert max_rel(run(plan, X, True), X @ D) <= 1e-10


def test_bench_size_laguerre_transform(xc):
    """The bench's 2-D workload (eta = 100, N = 4096, eps1 = 1e-10, FP64): the
    whole forward and transposed products of 4 right-hand sides against the
    oracle."""
    spec = spec_of("laguerre", 4096, eta=100.0)
    with make(xc, spec, 1e-10, eps2=1e-3) as plan:
        ora = M2.build(spec, 1e-10, eps2=1e-3)
        assert plan.info()["blocks2d"] == len(ora.blocks)
        X = inputs.normal(4096, 4, 65)
        assert max_rel(run(plan, X), M2.apply(ora, X)) <= 1e-10 + 10 * 1e-10
        assert max_rel(run(plan, X, True), M2.apply_adjoint(ora, X)) <= 1e-10 + 10 * 1e-10
