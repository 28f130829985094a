"""xc_apply_noalloc: the forward apply for callers that cannot allocate device
memory (for example code running under an allocator that owns all device
memory, or latency-critical paths where cudaMalloc could stall).  Its spectra
live in a fixed array inside the library instead of the plan's scratch.

The test calls the entry point through the C ABI twice in a row, with
different inputs, and compares each result with xc_apply's on the same input
(the same kernels run, so the tolerance of the parity tests is generous here).
It also checks that an oversized request is refused before anything runs.
This file is named so that pytest collects it last.
"""
import ctypes

import pytest

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


@pytest.mark.parametrize("fam,N,eps,precision,nrhs", [
    ("legendre", 1000, 1e-10, "fp64", 5),
    ("chebyshev", 777, 1e-12, "fp64", 9),
    ("laguerre", 300, 1e-10, "fp64", 3),
    ("jacobi", 2048, 1e-7, "fp32", 17),
    ("hermite", 500, 1e-7, "fp32c", 8),
])
def test_noalloc_matches_apply_on_two_calls(xc, fam, N, eps, precision, nrhs):
    with xc.Plan(fam, N, eps, precision=precision, alpha=0.5, beta=-0.5) as plan:
        dt = plan.torch_dtype
        tol = 1e-12 if precision == "fp64" else 1e-5
        for call in range(2):
            x = torch.from_numpy(inputs.normal(N, nrhs, 70 + call)).to("cuda", dt)
            y_ref = plan.apply(x)
            y = torch.full_like(x, float("nan"))
            assert call_noalloc(xc, plan, x, y) == xc.XC_OK
            torch.cuda.synchronize()
            plan.sync_status()
            err = float((y.double() - y_ref.double()).abs().max() / y_ref.double().abs().max())
            assert err <= tol, (call, err)


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
