"""The direct dense product on the tensor cores (xc_dense_*, 3xTF32): the
comparator the method is measured against.  Checked against the FP64
oracle's plain dense product (rows of A generated by the oracle's own
recurrences), forward and transpose, at sizes with ragged tiles in every
dimension and at the benchmark's full sizes (sampled rows), and against
cuBLAS SGEMM's own error on the same FP32 matrix.

Tolerance: relative l2 <= 4e-6 + the error of the FP32 matrix itself (its
entries rounded to FP32 from the FP64 recurrence), which cuBLAS shares; the
3xTF32 products carry about 2^-22 relative error each, accumulated in FP32.
"""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fam,N,nrhs", [("legendre", 1000, 1), ("legendre", 1000, 37), ("chebyshev", 777, 100),
                                        ("jacobi", 1333, 259), ("hermite", 500, 64), ("legendre", 129, 3)])
def test_dense_tensor_core_product_matches_the_oracle(xc, fam, N, nrhs):
    sp = F.make_spec(fam, N, 0.5, -0.5) if fam == "jacobi" else F.make_spec(fam, N)
    with xc.Plan(fam, N, 1e-7, precision="fp32", alpha=0.5, beta=-0.5,
                 nodes=None if fam == "chebyshev" else sp.x) as plan:
        A = plan.dense_matrix()
    X = inputs.uniform_pm1(N, nrhs, 31)
    Y = inputs.normal(N, nrhs, 32)
    ref_f = M.dense_apply(sp, X)
    ref_a = M.dense_apply_adjoint(sp, Y)
    with xc.Dense(A) as d:
        xd = torch.from_numpy(X).to("cuda", torch.float32)
        yd = torch.from_numpy(Y).to("cuda", torch.float32)
        f = d.apply(xd).double().cpu().numpy()
        a = d.apply(yd, transpose=True).double().cpu().numpy()
        f2 = d.apply(xd).double().cpu().numpy()           # a second call on the same comparator
        assert d.status() == xc.XC_OK
    torch.backends.cuda.matmul.allow_tf32 = False
    sg_f = (xd @ A.T).double().cpu().numpy()
    sg_a = (yd @ A).double().cpu().numpy()
    ef, ea = rel(f, ref_f), rel(a, ref_a)
    print(f"dense {fam} N={N} R={nrhs}: 3xTF32 fwd {ef:.2e} adj {ea:.2e}; "
          f"SGEMM fwd {rel(sg_f, ref_f):.2e} adj {rel(sg_a, ref_a):.2e}")
    assert np.array_equal(f, f2)
    assert ef <= 4e-6 + rel(sg_f, ref_f)
    assert ea <= 4e-6 + rel(sg_a, ref_a)


@pytest.mark.parametrize("N,nrhs", [(16384, 256), (32768, 128), (8192, 256)])
def test_dense_tensor_core_product_at_the_benchmark_sizes(xc, N, nrhs):
    """Legendre at N = 16384 with 256 right-hand sides and N = 32768 with 128
    (the launch shapes the benchmark times), and N = 8192 with 256 (the
    profiled case: 1.3 GB on the device), against the oracle's dense
    product on sampled rows (forward) and sampled right-hand sides (transpose,
    on every output)."""
    sp = F.make_spec("legendre", N)
    with xc.Plan("legendre", N, 1e-7, precision="fp32", nodes=sp.x) as plan:
        A = plan.dense_matrix()
    X = inputs.normal(N, nrhs, 33)
    with xc.Dense(A) as d:
        del A
        xd = torch.from_numpy(X).to("cuda", torch.float32)
        f = d.apply(xd).double().cpu().numpy()
        a = d.apply(xd, transpose=True).double().cpu().numpy()
        assert d.status() == xc.XC_OK
    rows = np.unique(np.random.default_rng(N).integers(0, N, 200))
    ef = rel(f[:, rows], M.dense_apply(sp, X, rows=rows))
    pick = np.array([0, nrhs // 2, nrhs - 1])
    ea = rel(a[pick], M.dense_apply_adjoint(sp, X[pick]))
    print(f"dense legendre N={N} R={nrhs}: 3xTF32 fwd {ef:.2e} adj {ea:.2e}")
    assert ef <= 1e-5 and ea <= 1e-5


def test_dense_rejects_bad_arguments(xc):
    import ctypes
    A = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with xc.Dense(A) as d:
        x = torch.zeros((2, 64), dtype=torch.float32, device="cuda")
        assert xc._lib.xc_dense_apply(d._h, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      2, 64, None) == xc.XC_ERR_ARG
        assert xc._lib.xc_dense_apply(d._h, 0, ctypes.c_void_p(x.data_ptr()), None, 2, 64, None) == xc.XC_ERR_ARG
        assert xc._lib.xc_dense_apply(d._h, 0, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr() + 1024), 1, 32, None) == xc.XC_ERR_ARG
