"""Full-size parity (the workloads' own sizes and launch configuration) and the
autograd path.

Each case builds the oracle plan (FP64, full precompute), feeds both sides the
same seeded inputs and compares
  * against the oracle's method: the FP64 relative-l2 bound of
    fp64_bounds.py (and the elementwise tolerance of test_gpu_parity.py), or
    the FP32 relative-l2 bound max(10 eps, 1e-5);
  * against the plain dense product: the method's own accuracy, bounded by
    eps1/eps2 (Section 2.2) for FP64 and by max(10 eps, 1e-5) for FP32.
Forward outputs are compared on a sample of rows (the dense product computes
those rows only); adjoint outputs in full.
"""
import math

import numpy as np
import pytest

from fp64_bounds import adjoint_bound, forward_bound
from oracle import families as F
from oracle import method as M
from paper_2004_11610_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc as mod
    return mod


def spec_for(fam, N, params):
    return F.make_spec(fam, N, params.get("alpha", 0.0), params.get("beta", 0.0))


def sample_rows(N, k=257):
    g = np.random.default_rng(N)
    rows = np.unique(np.concatenate([[0, 1, N // 2, N - 2, N - 1], g.integers(0, N, k)]))
    return rows


def run_workload(xc, name, nrhs_cap=None, adjoint=True):
    wl = inputs.WORKLOADS[name]
    prec = wl["precision"]
    out = []
    for i, (fam, N, params) in enumerate(wl["plans"]):
        sp = spec_for(fam, N, params)
        ora = M.build(sp, wl["eps"], precision=prec)
        nodes = None if fam == "chebyshev" else sp.x
        R = wl["nrhs"] if nrhs_cap is None else min(nrhs_cap, wl["nrhs"])
        X = inputs.draw(wl["dist"], N, R, 5, i)
        with xc.Plan(fam, N, wl["eps"], precision=prec, nodes=nodes, alpha=params.get("alpha", 0.0),
                     beta=params.get("beta", 0.0)) as plan:
            info = plan.info()
            assert info["L"] == [b.L for b in ora.schedule.blocks]
            dt = plan.torch_dtype
            Xd = torch.from_numpy(X).to("cuda", dt)
            Y = plan.apply(Xd).double().cpu().numpy()
            XA = plan.apply_adjoint(Xd).double().cpu().numpy() if adjoint else None
            torch.cuda.synchronize()
            plan.sync_status()
        rows = sample_rows(N)
        y_full = M.apply(ora, X)
        y_m = y_full[:, rows]
        y_d = M.dense_apply(sp, X, rows=rows)
        res = {"fam": fam, "N": N, "ora": ora, "y": Y[:, rows], "y_m": y_m, "y_d": y_d, "prec": prec,
               "eps": wl["eps"]}
        if prec == "fp64":
            res["fwd_rel"] = M.rel_l2(Y, y_full)
            res["fwd_bound"] = forward_bound(ora, X, y_full)
        if adjoint:
            res.update(xa=XA, xa_m=M.apply_adjoint(ora, X), xa_d=M.dense_apply_adjoint(sp, X))
            if prec == "fp64":
                res["adj_bound"] = adjoint_bound(ora, X, res["xa_m"])
        out.append(res)
    return out


def check(res):
    eps = res["eps"]
    if res["prec"] == "fp64":
        ora = res["ora"]
        Lmax = max([b.L for b in ora.blocks] + [8])
        tol = 64 * U64 * math.log2(Lmax) / ora.schedule.eps2 + 10 * eps
        assert np.abs(res["y"] - res["y_m"]).max() <= tol * np.abs(res["y_m"]).max()
        assert M.rel_l2(res["y"], res["y_d"]) <= eps / ora.schedule.eps2
        print(f"fp64 {res['fam']} N={res['N']} forward: rel-l2 {res['fwd_rel']:.2e} <= bound {res['fwd_bound']:.2e}")
        assert res["fwd_rel"] <= res["fwd_bound"]
        if "xa" in res:
            assert np.abs(res["xa"] - res["xa_m"]).max() <= tol * np.abs(res["xa_m"]).max()
            assert M.rel_l2(res["xa"], res["xa_d"]) <= eps / ora.schedule.eps2
            ea = M.rel_l2(res["xa"], res["xa_m"])
            print(f"fp64 {res['fam']} N={res['N']} adjoint: rel-l2 {ea:.2e} <= bound {res['adj_bound']:.2e}")
            assert ea <= res["adj_bound"]
    else:
        tol = max(10 * eps, 1e-5)
        assert M.rel_l2(res["y"], res["y_m"]) <= tol
        assert M.rel_l2(res["y"], res["y_d"]) <= tol
        if "xa" in res:
            assert M.rel_l2(res["xa"], res["xa_m"]) <= tol
            assert M.rel_l2(res["xa"], res["xa_d"]) <= tol


def test_legendre512_fp64_eps1e14_full(xc):
    """Legendre N=512, eps=1e-14, one RHS: relative l2 <= 1e-12 against the dense product."""
    (res,) = run_workload(xc, "legendre512_fp64")
    check(res)
    assert M.rel_l2(res["y"], res["y_d"]) <= 1e-12
    assert M.rel_l2(res["xa"], res["xa_d"]) <= 1e-12


def test_chebyshev_laguerre4096_fp64_full(xc):
    for res in run_workload(xc, "cheb_lag4096_fp64"):
        check(res)


def test_legendre_jacobi16384_fp32c_full(xc):
    """All 256 right-hand sides: the launch shapes the benchmark times."""
    for res in run_workload(xc, "leg_jac16384_fp32c"):
        check(res)


def test_legendre32768_fp32_full_uses_cluster_precompute(xc):
    """The first block (L_1 = 44100) is too long for one CTA's FP64 FFT: the
    precompute runs it on a thread-block cluster (distributed shared memory)."""
    for res in run_workload(xc, "legendre32768_fp32"):
        check(res)


# ----------------------------------------------------------------- autograd

def test_autograd_matches_finite_differences_fp64(xc):
    """Central finite differences with step 1e-3 in FP64 at N = 256 (the loss
    is linear in x, so they agree with the adjoint to rounding)."""
    N = 256
    with xc.Plan("legendre", N, 1e-12, precision="fp64") as plan:
        x = torch.from_numpy(inputs.normal(N, 2, 61)).cuda().requires_grad_(True)
        w = torch.from_numpy(inputs.normal(N, 2, 62)).cuda()
        loss = (xc.xc_apply_autograd(x, plan) * w).sum()
        loss.backward()
        g = x.grad.detach().cpu().numpy()
        h = 1e-3
        with torch.no_grad():
            for r, i in [(0, 0), (0, 17), (1, 100), (1, 255), (0, 128)]:
                e = torch.zeros_like(x)
                e[r, i] = h
                lp = float((plan.apply(x + e) * w).sum())
                lm = float((plan.apply(x - e) * w).sum())
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[r, i]) <= 1e-9 * max(1.0, abs(g[r, i]))
        sp = F.make_spec("legendre", N)
        ref = M.dense_apply_adjoint(sp, w.cpu().numpy())
        assert M.rel_l2(g, ref) <= 1e-12 / 1e-3


def test_autograd_legendre32768_fp32_against_dense_transpose(xc):
    """Legendre N=32768, FP32 forward and backward through the autograd
    function at the workload's 128 right-hand sides; the gradient equals the
    dense transpose product A^T g."""
    N, R = 32768, 128
    sp = F.make_spec("legendre", N)
    with xc.Plan("legendre", N, 1e-7, precision="fp32", nodes=sp.x) as plan:
        x = torch.from_numpy(inputs.normal(N, R, 63)).to("cuda", torch.float32).requires_grad_(True)
        gout = torch.from_numpy(inputs.normal(N, R, 64)).to("cuda", torch.float32)
        y = xc.xc_apply_autograd(x, plan)
        y.backward(gout)
        grad = x.grad.double().cpu().numpy()
    ref = M.dense_apply_adjoint(sp, gout.double().cpu().numpy())
    assert M.rel_l2(grad, ref) <= 1e-5


@pytest.mark.parametrize("N,eps,precision", [(30000, 1e-10, "fp64"), (30000, 1e-10, "fp64pair"),
                                             (60000, 1e-7, "fp32")])
def test_long_blocks_run_the_apply_fft_on_a_cluster(xc, N, eps, precision):
    """Chebyshev blocks too long for one CTA's shared memory in the plan
    precision (n = L/2 complex points above ~14.5 k in FP64, ~29 k in FP32):
    the apply FFTs split the array over a thread-block cluster.  Checked
    against the plain dense product (the method's own accuracy, eps1/eps2) and
    the exact-transpose property of the adjoint."""
    eps2 = 1e-3 if precision != "fp32" else 1e-1
    with xc.Plan("chebyshev", N, eps, precision=precision, eps2=eps2) as plan:
        info = plan.info()
        dt = torch.float64 if precision != "fp32" else torch.float32
        esize = 16 if precision != "fp32" else 8
        assert info["L"][0] // 2 * esize > 227 * 1024          # one CTA could not hold it
        A = plan.dense_matrix()
        X = torch.from_numpy(inputs.normal(N, 4, 61)).to("cuda", dt)
        y = plan.apply(X)
        y_d = X @ A.T
        bound = max(10 * eps / eps2, 1e-5) if precision == "fp32" else 10 * eps / eps2
        assert float(torch.linalg.norm(y.double() - y_d.double()) / torch.linalg.norm(y_d.double())) <= bound
        Y = torch.from_numpy(inputs.normal(N, 4, 62)).to("cuda", dt)
        xa = plan.apply_adjoint(Y)
        xa_d = Y @ A
        assert float(torch.linalg.norm(xa.double() - xa_d.double()) / torch.linalg.norm(xa_d.double())) <= bound
        # <A x, y> = <x, A^T y> for the method's own operators
        lhs = (y.double() * Y.double()).sum(dim=1)
        rhs = (X.double() * xa.double()).sum(dim=1)
        scale = (y.double() * Y.double()).abs().sum(dim=1)
        tol = 1e-12 if precision != "fp32" else 1e-5
        assert bool(((lhs - rhs).abs() <= tol * scale).all())
        del A
