"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/xc.h declares, and rejects invalid arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xc.h")


@pytest.fixture(scope="module")
def xc():
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc as mod
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("xc_plan_create", "xc_apply", "xc_apply_adjoint", "xc_plan_destroy", "xc_plan_info",
                     "xc_get_nodes", "xc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(xc):
    lib = ctypes.CDLL(xc._LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(xc.EXPORTED)


def test_invalid_arguments_are_rejected_on_the_host(xc):
    h = ctypes.c_void_p()
    p = xc.xc_params()
    xc._lib.xc_params_default(ctypes.byref(p))
    create = xc._lib.xc_plan_create
    assert create(ctypes.byref(h), 99, ctypes.byref(p), 64, 1e-8) == xc.XC_ERR_ARG
    assert create(ctypes.byref(h), 1, ctypes.byref(p), 1, 1e-8) == xc.XC_ERR_ARG
    assert create(ctypes.byref(h), 1, ctypes.byref(p), 64, -1.0) == xc.XC_ERR_ARG
    assert create(ctypes.byref(h), 1, ctypes.byref(p), 64, 1.5) == xc.XC_ERR_ARG
    assert create(None, 1, ctypes.byref(p), 64, 1e-8) == xc.XC_ERR_ARG
    p.precision = 7
    assert create(ctypes.byref(h), 1, ctypes.byref(p), 64, 1e-8) == xc.XC_ERR_ARG
    xc._lib.xc_params_default(ctypes.byref(p))
    p.nodes = 1      # user nodes without a pointer
    assert create(ctypes.byref(h), 1, ctypes.byref(p), 64, 1e-8) == xc.XC_ERR_ARG
    xc._lib.xc_params_default(ctypes.byref(p))
    p.alpha = -1.5
    assert create(ctypes.byref(h), 2, ctypes.byref(p), 64, 1e-8) == xc.XC_ERR_ARG
    xc._lib.xc_params_default(ctypes.byref(p))
    p.scheme = 1     # two-sided needs the Chebyshev family
    assert create(ctypes.byref(h), 1, ctypes.byref(p), 64, 1e-8) == xc.XC_ERR_ARG
    assert not h.value
    msg = xc._lib.xc_last_error_message().decode()
    assert "two-sided" in msg
    assert xc._lib.xc_apply(None, None, None, 1, 64, None) == xc.XC_ERR_ARG
    assert xc._lib.xc_strerror(xc.XC_ERR_TIMEOUT) == b"device wait timed out"


def test_structure_layouts_match_the_header(xc):
    # offsets fixed by the C layout of include/xc.h (LP64)
    assert ctypes.sizeof(xc.xc_params) == 80
    assert xc.xc_plan_stats.L.offset == 56
    assert ctypes.sizeof(xc.xc_plan_stats) == 56 + 7 * 8 * 16 + 24 + 32


def test_ctypes_mirrors_match_a_c_compiler(xc, tmp_path):
    """Every field offset and struct size of the Python mirrors equals what a
    C compiler makes of include/xc.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [xc.xc_params, xc.xc_plan_stats, xc.xc_kernel_time, xc.xc_batch_stats]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "xc.h"', "int main(void) {"]
    expect = []
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(st))
        for field in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field[0]}));')
            expect.append(getattr(st, field[0]).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_batch_arguments_are_checked_on_the_host(xc):
    h = ctypes.c_void_p()
    assert xc._lib.xc_batch_create(None, None, 1) == xc.XC_ERR_ARG
    assert xc._lib.xc_batch_create(ctypes.byref(h), None, 1) == xc.XC_ERR_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert xc._lib.xc_batch_create(ctypes.byref(h), arr, 0) == xc.XC_ERR_ARG
    assert xc._lib.xc_batch_create(ctypes.byref(h), arr, 2) == xc.XC_ERR_ARG
    assert not h.value
    assert xc._lib.xc_batch_apply(None, 0, None) == xc.XC_ERR_ARG
    assert xc._lib.xc_batch_debug_set(None, 0, 0, 1) == xc.XC_ERR_ARG


class _FakeCudaTensor:
    """Just enough of a CUDA tensor for the binding's argument checks (which
    run before anything reaches the library)."""

    def __init__(self, shape, stride, dtype):
        self.shape, self._stride, self.dtype, self.is_cuda = tuple(shape), tuple(stride), dtype, True

    def dim(self):
        return len(self.shape)

    def stride(self, i):
        return self._stride[i]

    def is_complex(self):
        return False


def test_binding_checks_the_output_against_the_input(xc):
    """One leading dimension serves input and output at the boundary: the
    binding refuses an output of another shape or row stride (a shorter output
    would be written past its end) and passes N as the leading dimension of a
    single vector."""
    torch = pytest.importorskip("torch")
    plan = object.__new__(xc.Plan)
    plan.N, plan.precision, plan.is_complex = 100, "fp64", False
    f64 = torch.float64
    x = _FakeCudaTensor((4, 100), (128, 1), f64)
    assert plan._pair(x, _FakeCudaTensor((4, 100), (128, 1), f64), "x", "out") == 128
    with pytest.raises(ValueError):
        plan._pair(x, _FakeCudaTensor((3, 100), (128, 1), f64), "x", "out")
    with pytest.raises(ValueError):
        plan._pair(x, _FakeCudaTensor((4, 100), (100, 1), f64), "x", "out")
    with pytest.raises(ValueError):
        plan._pair(x, _FakeCudaTensor((4, 100), (1, 4), f64), "x", "out")
    with pytest.raises(TypeError):
        plan._pair(x, _FakeCudaTensor((4, 100), (128, 1), torch.float32), "x", "out")
    one = _FakeCudaTensor((1, 100), (7, 1), f64)
    assert plan._pair(one, _FakeCudaTensor((1, 100), (100, 1), f64), "x", "out") == 100
