"""The Appendix A precompute on the GPU: Chebyshev plans at Chebyshev-Gauss
nodes build their compressed rows from the closed-form row DFT convolved with
the window's DFT instead of an FFT per row.

Checked against the FP64 oracle built the plain way (FFT of every windowed row)
with the tolerances of the other parity tests, and against the library's own
FFT precompute (XC_PRECOMPUTE_FFT): the kept elements may differ only where an
element lies within the closed form's truncation error (under 0.1 eps1 *
max|Ä|) of the threshold, which moves an output by about eps1 of its scale.
"""
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


def run(plan, X, adjoint=False):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    Xd = torch.from_numpy(X).to("cuda", dt)
    out = plan.apply_adjoint(Xd) if adjoint else plan.apply(Xd)
    torch.cuda.synchronize()
    plan.sync_status()
    return out.double().cpu().numpy()


def max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [  # N, eps, precision, scheme
    (256, 1e-12, "fp64", "auto"), (301, 1e-8, "fp64", "auto"), (512, 1e-14, "fp64", "auto"),
    (4096, 1e-12, "fp64", "auto"), (1000, 1e-10, "fp64", "blocks"), (700, 1e-7, "fp32", "auto"),
    (2, 1e-10, "fp64", "auto"), (33, 1e-6, "fp64", "auto"),
]


@pytest.mark.parametrize("N,eps,precision,scheme", CASES)
def test_closed_form_rows_match_oracle(xc, N, eps, precision, scheme):
    eps2 = 1e-3 if precision == "fp64" else 3e-2
    ora = M.build(F.make_spec("chebyshev", N), eps, eps2=eps2,
                  two_sided=None if scheme == "auto" else scheme == "two_sided")
    with xc.Plan("chebyshev", N, eps, precision=precision, eps2=eps2, scheme=scheme) as plan:
        info = plan.info()
        if N >= 256:   # the first (longest) block at least; short blocks take FFT rows
            assert info["closed_form_blocks"] >= 1
            if scheme == "auto":
                assert info["closed_form_blocks"] == info["nblocks"] == 1
        assert info["L"] == [b.L for b in ora.schedule.blocks]
        X = inputs.uniform_pm1(N, 5, 41)
        Y = inputs.normal(N, 5, 42)
        y, xa = run(plan, X), run(plan, Y, adjoint=True)
        y_ref, xa_ref = M.apply(ora, X), M.apply_adjoint(ora, Y)
        if precision == "fp64":
            Lmax = max([b.L for b in ora.blocks] + [8])
            tol = 64 * U64 * math.log2(Lmax) / ora.schedule.eps2 + 10 * eps
            assert max_rel(y, y_ref) <= tol and max_rel(xa, xa_ref) <= tol
        else:
            assert M.rel_l2(y, y_ref) <= max(10 * eps, 1e-5)
            assert M.rel_l2(xa, xa_ref) <= max(10 * eps, 1e-5)


@pytest.mark.parametrize("N,eps", [(1024, 1e-12), (3000, 1e-9)])
def test_closed_form_and_fft_precompute_agree(xc, N, eps):
    with xc.Plan("chebyshev", N, eps) as a, xc.Plan("chebyshev", N, eps, precompute="fft") as b:
        ia, ib = a.info(), b.info()
        assert ia["closed_form_blocks"] == 1 and ib["closed_form_blocks"] == 0
        assert ia["L"] == ib["L"]
        for na, nb in zip(ia["nnz"], ib["nnz"]):
            assert abs(na - nb) <= max(4, nb // 500)
        for ma, mb in zip(ia["maxabs"], ib["maxabs"]):
            assert ma == pytest.approx(mb, rel=1e-13)
        X = inputs.normal(N, 4, 43)
        assert max_rel(run(a, X), run(b, X)) <= 4 * eps
        assert max_rel(run(a, X, True), run(b, X, True)) <= 4 * eps


def test_eps_zero_and_user_nodes_take_the_fft_rows(xc):
    with xc.Plan("chebyshev", 640, 0.0) as p:
        assert p.info()["closed_form_blocks"] == 0
    x = np.cos((2 * np.arange(500) + 1) * np.pi / 1000)
    with xc.Plan("chebyshev", 500, 1e-10, nodes=x) as p:
        assert p.info()["closed_form_blocks"] == 0
    with xc.Plan("legendre", 300, 1e-10) as p:
        assert p.info()["closed_form_blocks"] == 0
