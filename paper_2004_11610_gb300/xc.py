"""ctypes binding of libxc (C ABI in include/xc.h).

Argument marshalling only: every step of the apply runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream; raw device
pointers and the stream handle are what cross the boundary.  Importing this
module fails loudly when libxc.so has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libxc.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libxc.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(_LIB_PATH)

# ------------------------------------------------------------------ constants
XC_OK, XC_ERR_ARG, XC_ERR_ALLOC, XC_ERR_CUDA, XC_ERR_TIMEOUT, XC_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
FAMILY = {"chebyshev": 0, "legendre": 1, "jacobi": 2, "laguerre": 3, "hermite": 4, "sine": 5, "cospow": 6,
          "exp": 7, "lagspec": 8, "a1": 9, "a2": 10}
COMPLEX_FAMILIES = ("exp", "lagspec")
PRECISION = {"fp64": 0, "fp32": 1, "fp32c": 2, "fp64pair": 3}
SCHEME = {"auto": 0, "two_sided": 1, "blocks": 2, "2d": 3}
XC_MAX_BLOCKS = 16


class xc_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("nodes", ctypes.c_int),
                ("user_nodes", ctypes.POINTER(ctypes.c_double)), ("normalise", ctypes.c_int),
                ("eps2", ctypes.c_double), ("eps_window", ctypes.c_double), ("precision", ctypes.c_int),
                ("scheme", ctypes.c_int), ("tail_max", ctypes.c_int), ("precompute", ctypes.c_int),
                ("power", ctypes.c_int)]


_I64x = ctypes.c_int64 * XC_MAX_BLOCKS


class xc_plan_stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("family", ctypes.c_int), ("precision", ctypes.c_int),
                ("scheme", ctypes.c_int), ("normalise", ctypes.c_int), ("eps", ctypes.c_double),
                ("eps2", ctypes.c_double), ("zeta", ctypes.c_double), ("nblocks", ctypes.c_int),
                ("L", _I64x), ("off", _I64x), ("j_lo", _I64x), ("j_hi", _I64x), ("nnz", _I64x),
                ("stored", _I64x), ("maxabs", ctypes.c_double * XC_MAX_BLOCKS), ("m_tail", ctypes.c_int64),
                ("matrix_bytes", ctypes.c_int64), ("adjoint_bytes", ctypes.c_int64), ("closed_form_blocks", ctypes.c_int),
                ("blocks2d", ctypes.c_int), ("dense2d", ctypes.c_int), ("nnz2d", ctypes.c_int64),
                ("dense_elems2d", ctypes.c_int64)]


class xc_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class xc_batch_stats(ctypes.Structure):
    _fields_ = [("nplans", ctypes.c_int), ("rhs_per_item", ctypes.c_int), ("tuned", ctypes.c_int),
                ("rhs_per_item_adjoint", ctypes.c_int), ("tasks_forward", ctypes.c_int64), ("tasks_adjoint", ctypes.c_int64),
                ("shared_bytes", ctypes.c_int64), ("matrix_bytes", ctypes.c_int64),
                ("adjoint_bytes", ctypes.c_int64), ("lockstep_forward", ctypes.c_int),
                ("lockstep_adjoint", ctypes.c_int), ("lockstep_plans", ctypes.c_int), ("tune_ms_forward", ctypes.c_float * 12),
                ("tune_ms_adjoint", ctypes.c_float * 12), ("tensor_plans", ctypes.c_int),
                ("tensor_plans_adjoint", ctypes.c_int)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "xc_params_default": (None, [ctypes.POINTER(xc_params)]),
    "xc_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(xc_params), _I64,
                                      ctypes.c_double]),
    "xc_plan_destroy": (ctypes.c_int, [_P]),
    "xc_plan_reserve": (ctypes.c_int, [_P, _I64]),
    "xc_apply": (ctypes.c_int, [_P, _P, _P, _I64, _I64, _P]),
    "xc_apply_adjoint": (ctypes.c_int, [_P, _P, _P, _I64, _I64, _P]),
    "xc_apply_host": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _I64, _I64, _P]),
    "xc_apply_noalloc": (ctypes.c_int, [_P, _P, _P, _I64, _I64, _P]),
    "xc_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(xc_plan_stats)]),
    "xc_get_nodes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "xc_dense_matrix": (ctypes.c_int, [_P, _P, _I64, _P]),
    "xc_sync_status": (ctypes.c_int, [_P]),
    "xc_timing_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "xc_timing_read": (ctypes.c_int, [_P, ctypes.POINTER(xc_kernel_time), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "xc_launch_count": (ctypes.c_int64, []),
    "xc_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int]),
    "xc_batch_bind": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I64),
                                     ctypes.POINTER(_I64)]),
    "xc_batch_apply": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "xc_batch_tune": (ctypes.c_int, [_P, _P]),
    "xc_batch_schedule": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "xc_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(xc_batch_stats)]),
    "xc_batch_status": (ctypes.c_int, [_P, _P]),
    "xc_batch_debug_set": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _I64]),
    "xc_batch_destroy": (ctypes.c_int, [_P]),
    "xc_dense_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _I64, _I64, _I64, _P]),
    "xc_dense_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _I64, _I64, _P]),
    "xc_dense_status": (ctypes.c_int, [_P, _P]),
    "xc_dense_destroy": (ctypes.c_int, [_P]),
    "xc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "xc_last_error_message": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_SIGS)


class XcError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.xc_last_error_message().decode(errors="replace")
        super().__init__(f"{where}: {_lib.xc_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def _check(code: int, where: str) -> None:
    if code != XC_OK:
        raise XcError(code, where)


def _stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------- plans

class Plan:
    """A compressed operator for A[n, m] = phi_m(x_n) (xc_plan_create).

    family     'chebyshev' | 'legendre' | 'jacobi' | 'laguerre' | 'hermite' | 'sine' | 'cospow'
               | 'exp' | 'lagspec' (complex: complex128 / complex64 tensors) | 'a1' | 'a2'
               (index kernels of Section 5.3, scheme '2d')
    scheme     'auto' | 'two_sided' | 'blocks' | '2d' (2-D compression; Laguerre / Hermite
               functions at equispaced `nodes`, or 'a1' / 'a2')
    N          order of the square matrix
    eps        eps1: threshold and Kaiser shape (0 keeps every element)
    precision  'fp64' | 'fp32' | 'fp32c' (FP32 with compensated accumulation) | 'fp64pair'
    nodes      optional host array of N nodes (default: the family's Gauss nodes;
               'exp': angles)
    eta, period  the spectral Laguerre matrix's eta and T (stored as alpha, beta)
    """

    def __init__(self, family: str, N: int, eps: float, precision: str = "fp64", alpha: float = 0.0,
                 beta: float = 0.0, nodes=None, normalise: bool = False, eps2: float = 0.0,
                 eps_window: float = 0.0, scheme: str = "auto", tail_max: int = 0, precompute: str = "auto",
                 power: int = 0, eta: float | None = None, period: float | None = None):
        p = xc_params()
        _lib.xc_params_default(ctypes.byref(p))
        if eta is not None:
            alpha = eta
        if period is not None:
            beta = period
        p.alpha, p.beta = float(alpha), float(beta)
        self._nodes_keep = None
        if nodes is not None:
            arr = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64))
            if arr.shape != (N,):
                raise ValueError("nodes must have shape (N,)")
            self._nodes_keep = arr
            p.nodes = 1
            p.user_nodes = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.normalise = 1 if normalise else 0
        p.eps2, p.eps_window = float(eps2), float(eps_window)
        p.precision = PRECISION[precision]
        p.scheme = SCHEME[scheme]
        p.tail_max = int(tail_max)
        p.precompute = {"auto": 0, "fft": 1}[precompute]
        p.power = int(power)
        h = _P()
        _check(_lib.xc_plan_create(ctypes.byref(h), FAMILY[family], ctypes.byref(p), int(N), float(eps)),
               "xc_plan_create")
        self._h = h
        self.family, self.N, self.eps, self.precision = family, int(N), float(eps), precision
        self.is_complex = family in COMPLEX_FAMILIES
        wide = precision in ("fp64", "fp64pair")
        if self.is_complex:
            self.np_dtype = np.complex128 if wide else np.complex64
        else:
            self.np_dtype = np.float64 if wide else np.float32

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.xc_plan_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def torch_dtype(self):
        import torch
        wide = self.precision in ("fp64", "fp64pair")
        if self.is_complex:
            return torch.complex128 if wide else torch.complex64
        return torch.float64 if wide else torch.float32

    # -- queries
    def info(self) -> dict:
        st = xc_plan_stats()
        _check(_lib.xc_plan_info(self._h, ctypes.byref(st)), "xc_plan_info")
        nb = st.nblocks
        return {
            "N": st.N, "family": st.family, "precision": st.precision, "scheme": st.scheme,
            "normalise": st.normalise, "eps": st.eps, "eps2": st.eps2, "zeta": st.zeta, "nblocks": nb,
            "L": list(st.L[:nb]), "off": list(st.off[:nb]), "j_lo": list(st.j_lo[:nb]),
            "j_hi": list(st.j_hi[:nb]), "nnz": list(st.nnz[:nb]), "stored": list(st.stored[:nb]),
            "maxabs": list(st.maxabs[:nb]), "m_tail": st.m_tail, "matrix_bytes": st.matrix_bytes,
            "adjoint_bytes": st.adjoint_bytes, "closed_form_blocks": st.closed_form_blocks,
            "blocks2d": st.blocks2d, "dense2d": st.dense2d, "nnz2d": st.nnz2d, "dense_elems2d": st.dense_elems2d,
        }

    def nodes(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.float64)
        _check(_lib.xc_get_nodes(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "xc_get_nodes")
        return out

    def reserve(self, nrhs: int) -> None:
        _check(_lib.xc_plan_reserve(self._h, int(nrhs)), "xc_plan_reserve")

    # -- device applies (torch tensors)
    def _check_tensor(self, t, name):
        import torch
        if not t.is_cuda or t.dtype != self.torch_dtype:
            raise TypeError(f"{name} must be a CUDA tensor of dtype {self.torch_dtype}")
        if t.is_complex() and t.is_conj():
            raise ValueError(f"{name} has PyTorch's lazy conjugate bit set: pass t.resolve_conj()")
        if t.dim() != 2 or t.shape[1] != self.N or t.stride(1) != 1:
            raise ValueError(f"{name} must have shape (nrhs, N) with unit column stride")
        return t

    @staticmethod
    def _like(t):
        """An output with the input's shape and strides (the boundary takes one
        leading dimension for both; empty_like would make a strided input's
        output contiguous)."""
        import torch
        return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=t.device)

    def _pair(self, a, b, na, nb):
        """Checks the input and output tensors of an apply (one leading
        dimension serves both) and returns that leading dimension."""
        self._check_tensor(a, na)
        self._check_tensor(b, nb)
        if b.shape != a.shape:
            raise ValueError(f"{nb} must have the shape of {na}")
        if a.shape[0] <= 1:
            return self.N
        if b.stride(0) != a.stride(0):
            raise ValueError(f"{nb} must have the row stride of {na}")
        return a.stride(0)

    def apply(self, x, out=None, stream=None):
        """y = A x for x of shape (nrhs, N) (xc_apply)."""
        x = self._check_tensor(x if x.dim() == 2 else x[None, :], "x")
        y = self._like(x) if out is None else out
        ld = self._pair(x, y, "x", "out")
        _check(_lib.xc_apply(self._h, _P(x.data_ptr()), _P(y.data_ptr()), x.shape[0], ld,
                             _stream_handle(stream)), "xc_apply")
        return y

    def apply_adjoint(self, y, out=None, stream=None):
        """x = A^T y for y of shape (nrhs, N) (xc_apply_adjoint; the plain
        transpose for the complex families)."""
        y = self._check_tensor(y if y.dim() == 2 else y[None, :], "y")
        x = self._like(y) if out is None else out
        ld = self._pair(y, x, "y", "out")
        _check(_lib.xc_apply_adjoint(self._h, _P(y.data_ptr()), _P(x.data_ptr()), y.shape[0], ld,
                                     _stream_handle(stream)), "xc_apply_adjoint")
        return x

    def apply_noalloc(self, x, out, stream=None):
        """y = A x without any device allocation (xc_apply_noalloc): the
        spectra go to the library's fixed device array instead of the plan's
        scratch.  `out` must be supplied; calls must not overlap on the GPU."""
        ld = self._pair(x, out, "x", "out")
        _check(_lib.xc_apply_noalloc(self._h, _P(x.data_ptr()), _P(out.data_ptr()), x.shape[0], ld,
                                     _stream_handle(stream)), "xc_apply_noalloc")
        return out

    # -- host path
    def apply_host(self, v, adjoint: bool = False, out=None, stream=None):
        """Forward or adjoint apply on host arrays (xc_apply_host): copies in,
        applies, copies out and synchronises.  `v` is (nrhs, ld) with ld >= N
        (the first N columns are the vectors); `out`, if given, is a writeable
        C-contiguous array of the same dtype and shape, whose columns beyond N
        are left as they are."""
        v = np.ascontiguousarray(v, dtype=self.np_dtype)
        if v.ndim == 1:
            v = v[None, :]
        if out is None:
            res = np.empty_like(v)
        else:
            res = out
            if not (isinstance(res, np.ndarray) and res.dtype == v.dtype and res.shape == v.shape
                    and res.flags.c_contiguous and res.flags.writeable):
                raise ValueError("out must be a writeable C-contiguous array of the input's dtype and shape")
        s = ctypes.c_void_p(0) if stream is None else _stream_handle(stream)
        _check(_lib.xc_apply_host(self._h, 1 if adjoint else 0, _P(v.ctypes.data), _P(res.ctypes.data),
                                  v.shape[0], v.shape[1], s), "xc_apply_host")
        return res

    def dense_matrix(self, stream=None):
        """The plain N x N matrix on the device (xc_dense_matrix)."""
        import torch
        A = torch.empty((self.N, self.N), dtype=self.torch_dtype, device="cuda")
        _check(_lib.xc_dense_matrix(self._h, _P(A.data_ptr()), self.N, _stream_handle(stream)),
               "xc_dense_matrix")
        return A

    def timing_enable(self, enable: bool = True) -> None:
        """Bracket every launch of this plan with CUDA events (xc_timing_enable)."""
        _check(_lib.xc_timing_enable(self._h, 1 if enable else 0), "xc_timing_enable")

    def timing_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last read (xc_timing_read)."""
        arr = (xc_kernel_time * 16)()
        n = ctypes.c_int()
        _check(_lib.xc_timing_read(self._h, arr, 16, ctypes.byref(n)), "xc_timing_read")
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}

    def sync_status(self) -> None:
        _check(_lib.xc_sync_status(self._h), "xc_sync_status")


# -------------------------------------------------------------------- batches

class Batch:
    """Many plans of one precision applied by one persistent launch per
    direction (xc_batch_*).  Bind device tensors once; `apply` then launches
    without allocating or synchronising (CUDA-graph capturable)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (_P * len(self.plans))(*[p.handle.value for p in self.plans])
        h = _P()
        _check(_lib.xc_batch_create(ctypes.byref(h), arr, len(self.plans)), "xc_batch_create")
        self._h = h
        self._bound = None

    def bind(self, xs, ys):
        """xs[i], ys[i]: CUDA tensors (nrhs_i, N_i) of plan i's dtype."""
        n = len(self.plans)
        if len(xs) != n or len(ys) != n:
            raise ValueError("one x and one y tensor per plan")
        lds = [p._pair(a, b, "x", "y") for p, a, b in zip(self.plans, xs, ys)]
        xp = (_P * n)(*[a.data_ptr() for a in xs])
        yp = (_P * n)(*[b.data_ptr() for b in ys])
        nr = (_I64 * n)(*[a.shape[0] for a in xs])
        ld = (_I64 * n)(*lds)
        _check(_lib.xc_batch_bind(self._h, xp, yp, nr, ld), "xc_batch_bind")
        self._bound = (list(xs), list(ys))

    def apply(self, adjoint: bool = False, stream=None):
        _check(_lib.xc_batch_apply(self._h, 1 if adjoint else 0, _stream_handle(stream)), "xc_batch_apply")

    def tune(self, stream=None):
        _check(_lib.xc_batch_tune(self._h, _stream_handle(stream)), "xc_batch_tune")

    def schedule(self, rpw_forward: int, rpw_adjoint: int, lockstep_forward: bool, lockstep_adjoint: bool):
        """Set the schedule by hand (xc_batch_schedule) instead of tuning it."""
        _check(_lib.xc_batch_schedule(self._h, rpw_forward, rpw_adjoint, int(lockstep_forward),
                                      int(lockstep_adjoint)), "xc_batch_schedule")

    def set_lockstep(self, forward: bool, adjoint: bool):
        """Lockstep items on or off per direction, keeping the right-hand sides per item."""
        st = self.info()
        self.schedule(st["rhs_per_item"], st["rhs_per_item_adjoint"], forward, adjoint)

    def info(self) -> dict:
        st = xc_batch_stats()
        _check(_lib.xc_batch_info(self._h, ctypes.byref(st)), "xc_batch_info")
        return {k: list(v) if isinstance(v, ctypes.Array) else v
                for k, v in ((k, getattr(st, k)) for k, _ in xc_batch_stats._fields_)}

    def status(self, stream=None) -> int:
        """XC_OK or XC_ERR_TIMEOUT (cleared on read)."""
        return int(_lib.xc_batch_status(self._h, _stream_handle(stream)))

    def debug_set(self, plan: int, extra_need: int, wait_limit: int) -> None:
        _check(_lib.xc_batch_debug_set(self._h, plan, extra_need, wait_limit), "xc_batch_debug_set")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.xc_batch_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------- dense comparator

class Dense:
    """The direct product y = A x with the plain FP32 matrix on the tensor
    cores, 3xTF32 (xc_dense_*): the comparator the method is measured
    against.  `A` is a CUDA float32 tensor (M, K); it is copied (split into
    TF32 halves, with a transposed copy) at construction."""

    def __init__(self, A, stream=None):
        import torch
        if not A.is_cuda or A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
            raise TypeError("A must be a 2-D CUDA float32 tensor with unit column stride")
        self.M, self.K = int(A.shape[0]), int(A.shape[1])
        h = _P()
        _check(_lib.xc_dense_create(ctypes.byref(h), _P(A.data_ptr()), self.M, self.K, A.stride(0),
                                    _stream_handle(stream)), "xc_dense_create")
        self._h = h

    def apply(self, x, transpose: bool = False, out=None, stream=None):
        """out[r] = A x[r] (transpose: A^T x[r]) for x of shape (nrhs, K) (or (nrhs, M))."""
        import torch
        n_in, n_out = (self.M, self.K) if transpose else (self.K, self.M)
        if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2 or x.shape[1] != n_in or x.stride(1) != 1:
            raise ValueError(f"x must be a CUDA float32 tensor of shape (nrhs, {n_in})")
        if n_in != n_out and x.shape[0] > 1:
            raise ValueError("rectangular comparators take one right-hand side per call")
        ld = x.stride(0) if x.shape[0] > 1 else max(n_in, n_out)
        if out is None:
            out = torch.empty_strided((x.shape[0], n_out), (ld, 1), dtype=torch.float32, device=x.device)
        elif out.shape != (x.shape[0], n_out) or out.stride(1) != 1 or (x.shape[0] > 1 and out.stride(0) != ld):
            raise ValueError("out must match x's shape and row stride")
        _check(_lib.xc_dense_apply(self._h, 1 if transpose else 0, _P(x.data_ptr()), _P(out.data_ptr()),
                                   x.shape[0], ld, _stream_handle(stream)), "xc_dense_apply")
        return out

    def status(self, stream=None) -> int:
        """XC_OK or XC_ERR_TIMEOUT (a device wait of an earlier apply gave up; cleared on read)."""
        return int(_lib.xc_dense_status(self._h, _stream_handle(stream)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.xc_dense_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------- autograd

def _autograd():
    import torch

    class XcApply(torch.autograd.Function):
        """y = A x with the gradient A^T g (the hand-written adjoint apply);
        complex plans: A^H g = conj(A^T conj(g)), PyTorch's convention for the
        gradient of a complex linear map."""

        @staticmethod
        def forward(ctx, x, plan):
            ctx.plan = plan
            return plan.apply(x.contiguous())

        @staticmethod
        def backward(ctx, g):
            if ctx.plan.is_complex:   # conj_physical: the kernels read memory, not the conj bit
                return torch.conj_physical(ctx.plan.apply_adjoint(torch.conj_physical(g).contiguous())), None
            return ctx.plan.apply_adjoint(g.contiguous()), None

    return XcApply


def xc_launch_count() -> int:
    """Kernels launched by libxc in this process (xc_launch_count)."""
    return int(_lib.xc_launch_count())


def xc_apply_autograd(x, plan: Plan):
    """Differentiable y = A x (torch.autograd.Function with the adjoint apply as backward)."""
    return _autograd().apply(x, plan)
