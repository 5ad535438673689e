"""Thin ctypes binding of the C ABI in ``include/afieti.h``.

The Python names equal the C names; this module only marshals arguments
(torch CUDA tensors -> device pointers, the current torch stream -> the
stream argument).  Every computation runs in ``libafieti.so``; there is no
fallback: if the library is missing, importing the binding fails."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

AFI_OK, AFI_EINVAL, AFI_ENOMEM, AFI_ECUDA, AFI_ESINGULAR, AFI_ENOT_CONVERGED, AFI_EBREAKDOWN, \
    AFI_ETIMEOUT = range(8)
AFI_FD_FP64, AFI_FD_FP32, AFI_FD_TF32, AFI_FD_BF16 = range(4)
PRECISIONS = {"fp64": AFI_FD_FP64, "fp32": AFI_FD_FP32, "tf32": AFI_FD_TF32, "bf16": AFI_FD_BF16}
(AFI_OP_STIFFNESS, AFI_OP_B, AFI_OP_BT, AFI_OP_PCHI, AFI_OP_PU, AFI_OP_PA_INV, AFI_OP_SCHUR,
 AFI_OP_PS, AFI_OP_PRECOND, AFI_OP_SADDLE) = range(10)

EXPORTED = ["af_ieti_setup", "fd_apply", "ieti_solve", "ieti_solve_adjoint", "afi_lame_grad",
            "afi_load_vector", "afi_apply", "afi_set_precision", "afi_sizes", "afi_memory",
            "af_ieti_destroy", "afi_status_string", "afi_last_error", "afi_kernel_launches",
            "afi_fd_apply_static", "afi_selftest_bounded_wait", "afi_apply_batch"]


class afi_problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("npatch", C.c_int), ("degree", C.POINTER(C.c_int)),
                ("nel", C.POINTER(C.c_int)), ("ctrl", C.POINTER(C.c_double)),
                ("lame", C.POINTER(C.c_double)), ("dirichlet_face", C.POINTER(C.c_ubyte))]


class afi_options(C.Structure):
    _fields_ = [("prec", C.c_int), ("tol", C.c_double), ("maxit", C.c_int),
                ("use_graph", C.c_int), ("variant", C.c_int)]


class afi_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres_est", C.c_double), ("relres_true", C.c_double),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("t_fd_setup_ms", C.c_double), ("fp64_restarts", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AfiError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {afi_status_string(status)} ({afi_last_error()})")


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load libafieti.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} not built: run __graft_entry__.build() first")
        _build.build()
    lib = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.c_void_p, C.c_int
    lib.af_ieti_setup.argtypes = [C.POINTER(afi_problem), C.POINTER(afi_options), C.POINTER(vp)]
    lib.fd_apply.argtypes = [vp, ip, dp, dp, ip, vp]
    lib.ieti_solve.argtypes = [vp, dp, dp, dp, ip, C.POINTER(afi_info), vp]
    lib.ieti_solve_adjoint.argtypes = [vp, dp, dp, dp, ip, C.POINTER(afi_info), vp]
    lib.afi_lame_grad.argtypes = [vp, dp, dp, dp, vp]
    lib.afi_load_vector.argtypes = [vp, dp, dp, vp]
    lib.afi_apply.argtypes = [vp, ip, dp, dp, vp]
    lib.afi_apply_batch.argtypes = [vp, ip, dp, dp, ip, vp]
    lib.afi_set_precision.argtypes = [vp, ip]
    lib.afi_sizes.argtypes = [vp, C.POINTER(C.c_long), C.POINTER(C.c_long)]
    lib.afi_memory.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.af_ieti_destroy.argtypes = [vp]
    lib.af_ieti_destroy.restype = None
    lib.afi_status_string.argtypes = [ip]
    lib.afi_status_string.restype = C.c_char_p
    lib.afi_last_error.argtypes = []
    lib.afi_last_error.restype = C.c_char_p
    lib.afi_fd_apply_static.argtypes = [ip, ip, ip, dp, dp, dp, dp, dp, dp,
                                         C.POINTER(C.c_double), C.c_double, C.c_double, dp, dp,
                                         ip, vp]
    lib.afi_selftest_bounded_wait.argtypes = [C.c_longlong, C.POINTER(C.c_longlong)]
    lib.afi_kernel_launches.argtypes = []
    lib.afi_kernel_launches.restype = C.c_longlong
    for name in EXPORTED:
        if name not in ("af_ieti_destroy", "afi_status_string", "afi_last_error",
                        "afi_kernel_launches"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def afi_status_string(status: int) -> str:
    return load().afi_status_string(int(status)).decode()


def afi_last_error() -> str:
    return load().afi_last_error().decode()


def afi_kernel_launches() -> int:
    return int(load().afi_kernel_launches())


def afi_selftest_bounded_wait(polls: int):
    """Run the bounded-wait failure path once; returns (status, polls used)."""
    used = C.c_longlong(0)
    status = load().afi_selftest_bounded_wait(int(polls), C.byref(used))
    return int(status), int(used.value)


def _check(status, where, allow=()):
    if status != AFI_OK and status not in allow:
        raise AfiError(status, where)
    return status


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda or not t.is_contiguous() or t.dtype.itemsize != 8:
            raise ValueError("expected a contiguous FP64 CUDA tensor")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Problem:
    """Host-side afi_problem with its arrays kept alive."""

    def __init__(self, prob):
        self.src = prob
        self.degree = np.ascontiguousarray(prob.degree, dtype=np.int32)
        self.nel = np.ascontiguousarray(prob.nel.reshape(-1), dtype=np.int32)
        self.ctrl = np.ascontiguousarray(prob.ctrl_flat(), dtype=np.float64)
        self.lame = np.ascontiguousarray(prob.lame.reshape(-1), dtype=np.float64)
        self.dface = np.ascontiguousarray(prob.dirichlet_face.reshape(-1), dtype=np.uint8)
        self.c = afi_problem(prob.dim, prob.npatch,
                             self.degree.ctypes.data_as(C.POINTER(C.c_int)),
                             self.nel.ctypes.data_as(C.POINTER(C.c_int)),
                             self.ctrl.ctypes.data_as(C.POINTER(C.c_double)),
                             self.lame.ctypes.data_as(C.POINTER(C.c_double)),
                             self.dface.ctypes.data_as(C.POINTER(C.c_ubyte)))


AFI_VARIANT_LOCAL_ONLY = 1
AFI_VARIANT_FD_SLAB = 2
AFI_VARIANT_STENCIL_F64 = 4
AFI_VARIANT_FORCE_RESTART = 8
AFI_VARIANT_EXACT = 16
AFI_VARIANT_GEO = 32
AFI_VARIANT_FD_FIXED = 64
AFI_VARIANT_MATRIX_FREE = 128


def af_ieti_setup(prob, prec="fp64", tol=1e-8, maxit=2000, use_graph=False, variant=0):
    """Create a context for a afi_workloads.Problem; returns the handle (int)."""
    lib = load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    opt = afi_options(PRECISIONS.get(prec, prec) if isinstance(prec, str) else int(prec),
                      float(tol), int(maxit), 1 if use_graph else 0, int(variant))
    h = C.c_void_p()
    _check(lib.af_ieti_setup(C.byref(P.c), C.byref(opt), C.byref(h)), "af_ieti_setup")
    return h.value


def fd_apply(ctx, interior, r, s, nrhs=1, stream=None):
    return _check(load().fd_apply(C.c_void_p(ctx), int(interior), _ptr(r), _ptr(s), int(nrhs),
                                  _stream(stream)), "fd_apply")


def ieti_solve(ctx, f, u, lam=None, nrhs=1, stream=None, allow_not_converged=False):
    info = afi_info()
    allow = (AFI_ENOT_CONVERGED,) if allow_not_converged else ()
    st = load().ieti_solve(C.c_void_p(ctx), _ptr(f), _ptr(u), _ptr(lam), int(nrhs), C.byref(info),
                           _stream(stream))
    _check(st, "ieti_solve", allow)
    return info.as_dict()


def ieti_solve_adjoint(ctx, g, z, zlam=None, nrhs=1, stream=None):
    info = afi_info()
    st = load().ieti_solve_adjoint(C.c_void_p(ctx), _ptr(g), _ptr(z), _ptr(zlam), int(nrhs),
                                   C.byref(info), _stream(stream))
    _check(st, "ieti_solve_adjoint")
    return info.as_dict()


def afi_lame_grad(ctx, u, z, grad, stream=None):
    return _check(load().afi_lame_grad(C.c_void_p(ctx), _ptr(u), _ptr(z), _ptr(grad),
                                       _stream(stream)), "afi_lame_grad")


def afi_load_vector(ctx, coef, f, stream=None):
    return _check(load().afi_load_vector(C.c_void_p(ctx), _ptr(coef), _ptr(f), _stream(stream)),
                  "afi_load_vector")


def afi_apply(ctx, op, x, y, stream=None):
    return _check(load().afi_apply(C.c_void_p(ctx), int(op), _ptr(x), _ptr(y), _stream(stream)),
                  "afi_apply")


def afi_apply_batch(ctx, op, x, y, nrhs, stream=None):
    return _check(load().afi_apply_batch(C.c_void_p(ctx), int(op), _ptr(x), _ptr(y), int(nrhs),
                                         _stream(stream)), "afi_apply_batch")


def afi_set_precision(ctx, prec):
    p = PRECISIONS.get(prec, prec) if isinstance(prec, str) else int(prec)
    return _check(load().afi_set_precision(C.c_void_p(ctx), int(p)), "afi_set_precision")


def afi_sizes(ctx):
    n, m = C.c_long(), C.c_long()
    _check(load().afi_sizes(C.c_void_p(ctx), C.byref(n), C.byref(m)), "afi_sizes")
    return n.value, m.value


def afi_memory(ctx):
    a, b = C.c_longlong(), C.c_longlong()
    _check(load().afi_memory(C.c_void_p(ctx), C.byref(a), C.byref(b)), "afi_memory")
    return a.value, b.value


def afi_fd_apply_static(n, U, D, coef, shift, scale, r, s, nblk=1, stream=None):
    """Allocation-free FD on nblk tensors of shape n = (n1, n2, n3); U, D are
    lists of device tensors (U[2], D[2] may be None when n3 == 1)."""
    cf = (C.c_double * 3)(*[float(x) for x in coef])
    u3 = _ptr(U[2]) if len(U) > 2 and U[2] is not None else None
    d3 = _ptr(D[2]) if len(D) > 2 and D[2] is not None else None
    return _check(load().afi_fd_apply_static(int(n[0]), int(n[1]), int(n[2]), _ptr(U[0]),
                                             _ptr(U[1]), u3, _ptr(D[0]), _ptr(D[1]), d3, cf,
                                             float(shift), float(scale), _ptr(r), _ptr(s),
                                             int(nblk), _stream(stream)), "afi_fd_apply_static")


def af_ieti_destroy(ctx):
    if ctx:
        load().af_ieti_destroy(C.c_void_p(ctx))
