"""Thin Python binding of the C ABI in ``include/hps.h`` (ctypes).

The functions carry the C names (``hps_nodes``, ``hps_build``, ``hps_solve``,
``hps_root_R``, ``hps_leaf_ops``, ``hps_info``, ``hps_status``, ``hps_free``)
and only marshal arguments: arrays are passed as raw pointers (numpy arrays
as host pointers, torch tensors as their data pointers), streams as
``cudaStream_t`` handles.  Every step of the method runs in the library's
CUDA kernels; there is no fallback.  Loading fails loudly if
``_lib/libhps.so`` has not been built (``python -m paper_1812_07167_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhps.so")

HPS_OK, HPS_EINVAL, HPS_ENOMEM, HPS_ESINGULAR, HPS_ETIMEOUT, HPS_ECUDA, HPS_ENOTSUP, HPS_ETOOBIG = range(8)
HPS_NOALLOC_WORKSPACE_BYTES = 16 << 20
HPS_FP64 = 0
HPS_MIXED = 1
HPS_LEAF_LU = 0
HPS_LEAF_INVERSE = 1

# every entry point include/hps.h declares
EXPORTS = ("hps_nodes", "hps_build", "hps_build_batch", "hps_rebuild", "hps_solve", "hps_solve_batch", "hps_reserve", "hps_solve_noalloc",
           "hps_root_R", "hps_leaf_ops", "hps_zgemm", "hps_zinv", "hps_check_wait", "hps_fp64_rate", "hps_tune", "hps_plan", "hps_info", "hps_build_times", "hps_build_product_times", "hps_status", "hps_free", "hps_strerror")


class hps_desc(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("mx", ctypes.c_int), ("my", ctypes.c_int),
        ("p", ctypes.c_int), ("q", ctypes.c_int),
        ("kappa", ctypes.c_double),
        ("eta_re", ctypes.c_double), ("eta_im", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("fp64_levels", ctypes.c_int), ("refine_steps", ctypes.c_int),
        ("fp64_native", ctypes.c_int),
        ("leaf_form", ctypes.c_int),
    ]


class hps_info_t(ctypes.Structure):
    _fields_ = [
        ("leaves", ctypes.c_int), ("levels", ctypes.c_int),
        ("n_leaf", ctypes.c_int), ("n_bdry", ctypes.c_int),
        ("dof", ctypes.c_longlong), ("operator_bytes", ctypes.c_longlong),
        ("build_flops", ctypes.c_longlong), ("solve_flops", ctypes.c_longlong),
        ("solve_bytes", ctypes.c_longlong),
        ("build_launches", ctypes.c_int), ("solve_launches", ctypes.c_int),
        ("build_scratch_bytes", ctypes.c_longlong), ("solve_ws_bytes_per_rhs", ctypes.c_longlong),
    ]


class HPSError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {hps_strerror(code)} (code {code})")
        self.code = code


_lib = None


def lib():
    """The loaded libhps (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhps is not built ({LIB_PATH} missing); run "
                               "python -m paper_1812_07167_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        D = ctypes.POINTER(hps_desc)
        L.hps_nodes.argtypes = [D, P, P]
        L.hps_build.argtypes = [D, P, P, ctypes.POINTER(ctypes.c_void_p)]
        L.hps_build_batch.argtypes = [ctypes.c_int, D, P, P, ctypes.POINTER(ctypes.c_void_p)]
        L.hps_rebuild.argtypes = [ctypes.c_int, P, P, P]
        L.hps_tune.argtypes = [ctypes.c_int, D, P, ctypes.POINTER(ctypes.c_int)]
        L.hps_solve.argtypes = [P, P, P, P, ctypes.c_int, P]
        L.hps_solve_noalloc.argtypes = [P, P, P, P, ctypes.c_int, P]
        L.hps_solve_batch.argtypes = [P, ctypes.c_int, P, P, P, P, P]
        L.hps_reserve.argtypes = [P, ctypes.c_int]
        L.hps_zgemm.argtypes = [ctypes.c_int] * 4 + [P, P, P, ctypes.c_int, P]
        L.hps_zinv.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), P]
        L.hps_check_wait.argtypes = [ctypes.c_int, P]
        L.hps_fp64_rate.argtypes = [P, P]
        L.hps_root_R.argtypes = [P, P, ctypes.c_int, P]
        L.hps_leaf_ops.argtypes = [P, ctypes.c_int, P, P, P, P]
        L.hps_info.argtypes = [P, ctypes.POINTER(hps_info_t)]
        L.hps_plan.argtypes = [D, ctypes.POINTER(hps_info_t)]
        L.hps_build_times.argtypes = [P, P, ctypes.c_int]
        L.hps_build_product_times.argtypes = [P, P, P, ctypes.c_int]
        L.hps_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.hps_free.argtypes = [P]
        L.hps_strerror.argtypes = [ctypes.c_int]
        L.hps_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def hps_strerror(code: int) -> str:
    return lib().hps_strerror(int(code)).decode()


@dataclass
class Problem:
    """Parameters of one problem (the fields of hps_desc)."""
    m: int
    p: int
    kappa: float
    eta: complex
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    precision: int = HPS_FP64
    fp64_levels: int = 0
    refine_steps: int = 0
    fp64_native: int = 0
    my: int = 0  # leaves along y (0: the same as m, the leaves along x)
    leaf_form: int = HPS_LEAF_LU  # leaf operators as LU factors, or HPS_LEAF_INVERSE: as B^-1
    q: int = 0  # boundary data points per leaf edge: 0 / p-2 Chebyshev, else Gauss-Legendre

    @property
    def ny(self) -> int:
        return self.my or self.m

    @property
    def qe(self) -> int:
        """Boundary data points per leaf edge."""
        return self.q or self.p - 2

    @property
    def nbi(self) -> int:
        """Boundary data points of a leaf."""
        return 4 * self.qe

    def desc(self) -> hps_desc:
        eta = complex(self.eta)
        return hps_desc(self.x0, self.x1, self.y0, self.y1, self.m, self.ny, self.p, self.qe,
                        float(self.kappa), eta.real, eta.imag, int(self.precision),
                        int(self.fp64_levels), int(self.refine_steps), int(self.fp64_native),
                        int(self.leaf_form))

    @property
    def n(self) -> int:
        return self.p * self.p - 4

    @property
    def nb(self) -> int:
        return 4 * (self.p - 2)

    @property
    def ni(self) -> int:
        return (self.p - 2) ** 2

    @property
    def leaves(self) -> int:
        return self.m * self.ny

    @property
    def nbdry(self) -> int:
        return 2 * (self.m + self.ny) * self.qe


def _ptr(a) -> int:
    """Raw pointer of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libhps must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors passed to libhps must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(code: int, what: str):
    if code != HPS_OK:
        raise HPSError(code, what)


def hps_nodes(pr: Problem):
    """(leaf_xy [leaves, p^2-4, 2], bdry_xy [2 (mx + my) (p-2), 2]) as numpy arrays."""
    lxy = np.zeros((pr.leaves, pr.n, 2))
    bxy = np.zeros((pr.nbdry, 2))
    d = pr.desc()
    _check(lib().hps_nodes(ctypes.byref(d), _ptr(lxy), _ptr(bxy)), "hps_nodes")
    return lxy, bxy


class Handle:
    """A built solver (owns device memory until free())."""

    def __init__(self, ptr: int, pr: Problem):
        self.ptr = ptr
        self.pr = pr

    def info(self) -> hps_info_t:
        out = hps_info_t()
        _check(lib().hps_info(self.ptr, ctypes.byref(out)), "hps_info")
        return out

    def free(self):
        if self.ptr:
            lib().hps_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hps_plan(pr: Problem) -> hps_info_t:
    """Sizes of the solver hps_build would create, without building it."""
    d = pr.desc()
    out = hps_info_t()
    _check(lib().hps_plan(ctypes.byref(d), ctypes.byref(out)), "hps_plan")
    return out


def hps_build(pr: Problem, c, stream=None) -> Handle:
    """Build the solver; c is [leaves, (p-2)^2] float64 (numpy or torch)."""
    d = pr.desc()
    h = ctypes.c_void_p()
    _check(lib().hps_build(ctypes.byref(d), _ptr(c), _stream(stream), ctypes.byref(h)), "hps_build")
    return Handle(h.value, pr)


def hps_build_batch(problems, cs, stream=None) -> list:
    """Build several problems together (same p, precision and fp64_levels);
    one Handle per problem, in the given order."""
    k = len(problems)
    if len(cs) != k:
        raise ValueError("hps_build_batch: one c per problem")
    if k == 0:
        return []
    descs = (hps_desc * k)(*[pr.desc() for pr in problems])
    cp = (ctypes.c_void_p * k)(*[_ptr(c) for c in cs])
    out = (ctypes.c_void_p * k)()
    _check(lib().hps_build_batch(k, descs, cp, _stream(stream), out), "hps_build_batch")
    return [Handle(out[i], problems[i]) for i in range(k)]


def hps_tune(problems, stream=None) -> int:
    """Measure the kernel choices of these problems' builds (kept for the
    process); returns the number of shapes measured."""
    k = len(problems)
    descs = (hps_desc * max(k, 1))(*[pr.desc() for pr in problems])
    n = ctypes.c_int(0)
    _check(lib().hps_tune(k, descs, _stream(stream), ctypes.byref(n)), "hps_tune")
    return n.value


def hps_rebuild(handles, cs, stream=None):
    """New coefficients for every handle of one build (replayed as a CUDA graph
    after the first call)."""
    k = len(handles)
    hp = (ctypes.c_void_p * max(k, 1))(*[h.ptr for h in handles])
    cp = (ctypes.c_void_p * max(k, 1))(*[_ptr(c) for c in cs])
    _check(lib().hps_rebuild(k, hp, cp, _stream(stream)), "hps_rebuild")
    return handles


def hps_solve(h: Handle, s, t, u, nrhs: int, stream=None):
    """u[nrhs, leaves, p^2-4] (complex128) from s and t (numpy or torch)."""
    _check(lib().hps_solve(h.ptr, _ptr(s), _ptr(t), _ptr(u), int(nrhs), _stream(stream)), "hps_solve")
    return u


def hps_solve_batch(h: Handle, s_list, t_list, u_list, nrhs_list, stream=None):
    """One solve pass over several requests' right-hand sides side by side
    (each request's arrays in the hps_solve layouts)."""
    k = len(nrhs_list)
    if not (len(s_list) == len(t_list) == len(u_list) == k):
        raise ValueError("hps_solve_batch: one s, t, u and nrhs per request")
    arr = ctypes.c_void_p * max(k, 1)
    sp = arr(*[_ptr(x) for x in s_list])
    tp = arr(*[_ptr(x) for x in t_list])
    up = arr(*[_ptr(x) for x in u_list])
    nr = (ctypes.c_int * max(k, 1))(*[int(x) for x in nrhs_list])
    _check(lib().hps_solve_batch(h.ptr, k, sp, tp, up, nr, _stream(stream)), "hps_solve_batch")
    return u_list


def hps_zgemm(A, B, C, emulated: int, stream=None):
    """C[b] = A[b] B[b] for complex128 device tensors shaped [batch, K, M],
    [batch, N, K], [batch, N, M] (column-major matrices stored transposed)."""
    batch, K, M = A.shape
    N = B.shape[1]
    _check(lib().hps_zgemm(M, N, K, batch, _ptr(A), _ptr(B), _ptr(C), int(emulated), _stream(stream)),
           "hps_zgemm")
    return C


def hps_zinv(A, Ainv, mode: int = 0, stream=None):
    """Ainv[b] = A[b]^-1 for complex128 device tensors shaped [batch, n, n]
    (column-major matrices stored transposed; the inverse of the transpose is
    the transpose of the inverse, so row-major input works the same).
    Returns (code, bad): HPS_OK or HPS_ESINGULAR with the index of a matrix
    that had a zero pivot column; raises for every other code."""
    batch, n, n2 = A.shape
    if n2 != n or tuple(Ainv.shape) != (batch, n, n):
        raise ValueError("A and Ainv must be [batch, n, n]")
    bad = ctypes.c_int(-1)
    code = lib().hps_zinv(n, batch, _ptr(A), _ptr(Ainv), int(mode), ctypes.byref(bad), _stream(stream))
    if code not in (HPS_OK, HPS_ESINGULAR):
        raise HPSError(code, "hps_zinv")
    return code, bad.value


def hps_check_wait(limit_ms: int, stream=None) -> int:
    """Run the products' bounded wait on a barrier nothing completes; returns
    the status code (HPS_ETIMEOUT expected)."""
    return lib().hps_check_wait(int(limit_ms), _stream(stream))


def hps_fp64_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s."""
    out = ctypes.c_double(0.0)
    _check(lib().hps_fp64_rate(ctypes.byref(out), _stream(stream)), "hps_fp64_rate")
    return out.value


def hps_reserve(h: Handle, nrhs: int):
    """Allocate the handle's solve workspace for up to nrhs right-hand sides now."""
    _check(lib().hps_reserve(h.ptr, int(nrhs)), "hps_reserve")


def hps_solve_noalloc(h: Handle, s, t, u, nrhs: int, stream=None):
    """hps_solve without allocation: s, t, u must be device tensors; the scratch
    is the library's fixed workspace (see include/hps.h)."""
    _check(lib().hps_solve_noalloc(h.ptr, _ptr(s), _ptr(t), _ptr(u), int(nrhs), _stream(stream)),
           "hps_solve_noalloc")
    return u


def hps_root_R(h: Handle, R, stream=None, gauss_basis: bool = False):
    _check(lib().hps_root_R(h.ptr, _ptr(R), int(bool(gauss_basis)), _stream(stream)), "hps_root_R")
    return R


def hps_leaf_ops(h: Handle, leaf: int, Psi=None, Y=None, Gam=None, stream=None):
    _check(lib().hps_leaf_ops(h.ptr, int(leaf), _ptr(Psi), _ptr(Y), _ptr(Gam), _stream(stream)),
           "hps_leaf_ops")
    return Psi, Y, Gam


def hps_build_product_times(h: Handle):
    """(ms, bf16 flops) of each tensor-core product kernel of the build."""
    ms = np.zeros(256)
    fl = np.zeros(256)
    n = lib().hps_build_product_times(h.ptr, _ptr(ms), _ptr(fl), len(ms))
    if n < 0:
        raise HPSError(-n, "hps_build_product_times")
    return ms[:n].copy(), fl[:n].copy()


def hps_build_times(h: Handle):
    """Device milliseconds of [leaf kernel, merge level 0, 1, ...] of the build."""
    out = np.zeros(64)
    n = lib().hps_build_times(h.ptr, _ptr(out), len(out))
    if n < 0:
        raise HPSError(-n, "hps_build_times")
    return out[:n].copy()


def hps_status(h: Handle, stream=None):
    """(code, level, box) after waiting for the handle's work on the stream."""
    lev = ctypes.c_int(-1)
    box = ctypes.c_int(-1)
    code = lib().hps_status(h.ptr, _stream(stream), ctypes.byref(lev), ctypes.byref(box))
    return code, lev.value, box.value


def hps_free(h: Handle):
    h.free()
