"""xc_apply_noalloc: the forward apply for callers that cannot allocate device
memory (for example code running under an allocator that owns all device
memory, or latency-critical paths where cudaMalloc could stall).  Its spectra
live in a fixed array inside the library instead of the plan's scratch.

The test calls the entry point through the C ABI twice in a row, with
different inputs, and compares each result with xc_apply's on the same input
and with the FP64 oracle's method on the same nodes (FP64: the tolerances of
the parity tests; FP32: relative l2 <= max(10 eps, 1e-5)).  One
case has bands long enough that xc_apply sums them in chunks, while this
entry point sums each row in one pass.  It also checks that an oversized
request is refused before anything runs.  This file is named so that pytest
collects it last.
"""
import ctypes
import math

import numpy as np
import pytest

from fp64_bounds import forward_bound
from oracle import families as F
from oracle import method as M
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


def call_noalloc(xc, plan, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return xc._lib.xc_apply_noalloc(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    x.shape[0], x.stride(0), stream)


def fp64_tol(ora, eps):
    """The FP64 parity tolerance of the oracle-parity tests, relative to max |y|."""
    Lmax = max([b.L for b in ora.blocks] + [8])
    return 64 * 2.0 ** -53 * math.log2(Lmax) / ora.schedule.eps2 + 10 * eps


@pytest.mark.parametrize("fam,N,eps,precision,nrhs,chunked", [
    ("legendre", 1000, 1e-10, "fp64", 5, False),
    ("chebyshev", 777, 1e-12, "fp64", 9, False),
    ("laguerre", 300, 1e-10, "fp64", 3, False),
    ("laguerre", 1500, 1e-10, "fp64", 4, True),
    ("jacobi", 2048, 1e-7, "fp32", 17, False),
    ("hermite", 500, 1e-7, "fp32c", 8, False),
])
def test_noalloc_matches_apply_and_oracle_on_two_calls(xc, fam, N, eps, precision, nrhs, chunked):
    prec = "fp32" if precision == "fp32c" else precision
    sp = F.make_spec(fam, N, 0.5, -0.5) if fam == "jacobi" else F.make_spec(fam, N)
    ora = M.build(sp, eps, precision=prec)
    nodes = None if fam == "chebyshev" else sp.x
    with xc.Plan(fam, N, eps, precision=precision, alpha=0.5, beta=-0.5, nodes=nodes) as plan:
        dt = plan.torch_dtype
        plan.timing_enable(True)
        for call in range(2):
            X = inputs.normal(N, nrhs, 70 + call)
            x = torch.from_numpy(X).to("cuda", dt)
            y_ref = plan.apply(x)
            y = torch.full_like(x, float("nan"))
            assert call_noalloc(xc, plan, x, y) == xc.XC_OK
            torch.cuda.synchronize()
            plan.sync_status()
            yd = y.double()
            err = float((yd - y_ref.double()).abs().max() / y_ref.double().abs().max())
            Y = yd.cpu().numpy()
            y_m = M.apply(ora, X)
            if precision == "fp64":
                assert err <= 1e-12, (call, err)
                assert np.abs(Y - y_m).max() <= fp64_tol(ora, eps) * np.abs(y_m).max()
                assert M.rel_l2(Y, y_m) <= forward_bound(ora, X, y_m)
            else:
                assert err <= 1e-5, (call, err)
                assert M.rel_l2(Y, y_m) <= max(10 * eps, 1e-5)
        # xc_apply of this plan cuts its bands into chunks exactly when `chunked`
        assert ("fwd_reduce" in plan.timing_read()) == chunked
        plan.timing_enable(False)


def test_noalloc_rejects_requests_beyond_its_array(xc):
    with xc.Plan("legendre", 4096, 1e-8) as plan:
        info = plan.info()
        per_rhs = sum(L // 2 + 1 for L in info["L"]) * 16
        nrhs = (16 << 20) // per_rhs + 1
        x = torch.zeros((nrhs, 4096), dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        launches = xc.xc_launch_count()
        assert call_noalloc(xc, plan, x, y) == xc.XC_ERR_UNSUPPORTED
        assert "split the right-hand sides" in xc._lib.xc_last_error_message().decode()
        assert xc.xc_launch_count() == launches
        assert call_noalloc(xc, plan, x[: nrhs - 1], y[: nrhs - 1]) == xc.XC_OK
        torch.cuda.synchronize()
