"""Python handle on the plain FP64 CPU oracle (``hps_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library and never loads it.

The C file follows the paper (arXiv:1812.07167) step by step: Sec. 2.1 for the
leaf operators, Sec. 2.2 for the merge, Algorithm 1 for the build, Algorithm 2
for the solve, plus a dense solve of the global collocation system whose
solution the HPS build+solve reproduces up to rounding.  This module only
marshals numpy arrays (row-major, complex128) to and from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``hps_oracle.c`` with gcc into ``oracle/_build/liboracle.so``.

    ``HPS_ORACLE_LIB`` names an already built variant instead (the mutation
    tests load deliberately broken copies this way)."""
    if os.environ.get("HPS_ORACLE_LIB"):
        return os.environ["HPS_ORACLE_LIB"]
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Desc(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("mx", ctypes.c_int), ("my", ctypes.c_int), ("p", ctypes.c_int),
        ("kappa", ctypes.c_double),
        ("eta_re", ctypes.c_double), ("eta_im", ctypes.c_double),
        ("first_vertical", ctypes.c_int),
        ("gauss_q", ctypes.c_int),
    ]


@dataclass
class Problem:
    """Problem description: rectangle, m x my leaves (my = m unless given),
    p Chebyshev nodes per side; q > 0 puts the boundary data on q
    Gauss-Legendre nodes per leaf edge (0: the p-2 corner-free Chebyshev
    edge nodes of the paper's scheme)."""
    m: int
    p: int
    kappa: float
    eta: complex
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    my: int = 0
    q: int = 0

    @property
    def mx(self) -> int:
        return self.m

    @property
    def ny(self) -> int:
        return self.my or self.m

    @property
    def e(self) -> int:
        return self.p - 2

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
    def qe(self) -> int:
        """Boundary-data points per leaf edge."""
        return self.q or self.p - 2

    @property
    def nbi(self) -> int:
        """Boundary-data points of a leaf (its interface with its neighbours)."""
        return 4 * self.qe

    @property
    def nbdry(self) -> int:
        return 2 * (self.m + self.ny) * self.qe


def _lib_handle():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.ora_cheb.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]
        lib.ora_nodes.argtypes = [ctypes.POINTER(_Desc), P, P]
        lib.ora_leaf.argtypes = [ctypes.POINTER(_Desc), P, P, P, P, P, P, P, P]
        lib.ora_build.argtypes = [ctypes.POINTER(_Desc), P, ctypes.c_int]
        lib.ora_build.restype = ctypes.c_void_p
        lib.ora_status.argtypes = [P]
        lib.ora_solve.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int]
        lib.ora_root_R.argtypes = [P, P]
        lib.ora_tree_leaf.argtypes = [P, ctypes.c_int, P, P, P]
        lib.ora_free.argtypes = [P]
        lib.ora_brute.argtypes = [ctypes.POINTER(_Desc), P, P, P, P]
        lib.ora_max_threads.restype = ctypes.c_int
        lib.ora_gauss_nodes.argtypes = [ctypes.c_int, P]
        lib.ora_edge_interp.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
        lib.ora_cond_W.argtypes = [P, ctypes.c_int]
        lib.ora_cond_W.restype = ctypes.c_double
        _lib = lib
    return _lib


def _desc(pr: Problem, first_vertical: bool = False) -> _Desc:
    eta = complex(pr.eta)
    return _Desc(pr.x0, pr.x1, pr.y0, pr.y1, pr.m, pr.ny, pr.p, pr.kappa, eta.real, eta.imag,
                 1 if first_vertical else 0, int(pr.q))


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_lib_handle().ora_max_threads())


def cheb(p: int, a: float = -1.0, b: float = 1.0):
    """Chebyshev nodes (increasing) on [a, b] and the differentiation matrix."""
    x = np.zeros(p)
    D = np.zeros((p, p))
    _lib_handle().ora_cheb(p, a, b, _ptr(x), _ptr(D))
    return x, D


def gauss_nodes(q: int) -> np.ndarray:
    """The q Gauss-Legendre nodes on [-1, 1], increasing."""
    z = np.zeros(q)
    if _lib_handle().ora_gauss_nodes(int(q), _ptr(z)):
        raise ValueError("q < 1")
    return z


def edge_interp(p: int, q: int):
    """(P [q, p-2], Q [p-2, q]): interpolation from an edge's corner-free
    Chebyshev nodes to its q Gauss nodes and back."""
    Pm = np.zeros((q, p - 2))
    Qm = np.zeros((p - 2, q))
    if _lib_handle().ora_edge_interp(int(p), int(q), _ptr(Pm), _ptr(Qm)):
        raise ValueError("bad p or q")
    return Pm, Qm


def nodes(pr: Problem):
    """(leaf_xy [leaves, n, 2], bdry_xy [4 m e, 2]) in the public layouts."""
    lxy = np.zeros((pr.leaves, pr.n, 2))
    bxy = np.zeros((pr.nbdry, 2))
    d = _desc(pr)
    if _lib_handle().ora_nodes(ctypes.byref(d), _ptr(lxy), _ptr(bxy)):
        raise ValueError("invalid problem")
    return lxy, bxy


def leaf(pr: Problem, c_int: np.ndarray, with_matrices: bool = False):
    """Leaf operators (Psi, Y, R, Gamma[, B, F, G]) for interior samples c."""
    c_int = np.ascontiguousarray(c_int, dtype=np.float64)
    n, nb, ni = pr.n, pr.nb, pr.ni
    Psi = np.zeros((n, nb), complex)
    Y = np.zeros((n, ni), complex)
    R = np.zeros((nb, nb), complex)
    Gam = np.zeros((nb, ni), complex)
    B = np.zeros((n, n), complex)
    F = np.zeros((nb, n), complex)
    G = np.zeros((nb, n), complex)
    d = _desc(pr)
    st = _lib_handle().ora_leaf(ctypes.byref(d), _ptr(c_int), _ptr(Psi), _ptr(Y), _ptr(R),
                                _ptr(Gam), _ptr(B), _ptr(F), _ptr(G))
    if st < 0:
        raise ValueError("invalid problem")
    if with_matrices:
        return Psi, Y, R, Gam, B, F, G
    return Psi, Y, R, Gam


class Tree:
    """An oracle build (Algorithm 1); free with close() or use as a context."""

    def __init__(self, pr: Problem, c: np.ndarray, nthreads: int = 1, first_vertical: bool = False):
        self.pr = pr
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(pr.leaves, pr.ni)
        self._d = _desc(pr, first_vertical)
        self._h = _lib_handle().ora_build(ctypes.byref(self._d), _ptr(c), int(nthreads))
        if not self._h:
            raise ValueError("invalid problem")
        self.status = int(_lib_handle().ora_status(self._h))

    def solve(self, s: np.ndarray, t: np.ndarray, nthreads: int = 1) -> np.ndarray:
        pr = self.pr
        s = np.ascontiguousarray(s, dtype=np.complex128).reshape(-1, pr.leaves, pr.ni)
        nrhs = s.shape[0]
        t = np.ascontiguousarray(t, dtype=np.complex128).reshape(nrhs, pr.nbdry)
        u = np.zeros((nrhs, pr.leaves, pr.n), complex)
        _lib_handle().ora_solve(self._h, _ptr(s), _ptr(t), _ptr(u), nrhs, int(nthreads))
        return u

    def root_R(self) -> np.ndarray:
        R = np.zeros((self.pr.nbdry, self.pr.nbdry), complex)
        if _lib_handle().ora_root_R(self._h, _ptr(R)):
            raise RuntimeError("root R not available")
        return R

    def cond_W(self):
        """Per merge level from the root down, the largest 1-norm condition
        number of the interface matrices W = I - R33b R33a (Sec. 2.2)."""
        out = []
        lev = 0
        while True:
            v = float(_lib_handle().ora_cond_W(self._h, lev))
            if v < 0:
                return out
            out.append(v)
            lev += 1

    def leaf_ops(self, pub: int):
        """(Psi [n, nbi], Y [n, ni], Gamma [nbi, ni]) of a leaf as the build
        stores them (on the Gauss nodes when q > 0)."""
        pr = self.pr
        Psi = np.zeros((pr.n, pr.nbi), complex)
        Y = np.zeros((pr.n, pr.ni), complex)
        Gam = np.zeros((pr.nbi, pr.ni), complex)
        if _lib_handle().ora_tree_leaf(self._h, int(pub), _ptr(Psi), _ptr(Y), _ptr(Gam)):
            raise IndexError(pub)
        return Psi, Y, Gam

    def close(self):
        if self._h:
            _lib_handle().ora_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def brute(pr: Problem, c: np.ndarray, s: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Dense solve of the global collocation system for one right-hand side."""
    c = np.ascontiguousarray(c, dtype=np.float64).reshape(pr.leaves, pr.ni)
    s = np.ascontiguousarray(s, dtype=np.complex128).reshape(pr.leaves, pr.ni)
    t = np.ascontiguousarray(t, dtype=np.complex128).reshape(pr.nbdry)
    u = np.zeros((pr.leaves, pr.n), complex)
    d = _desc(pr)
    st = _lib_handle().ora_brute(ctypes.byref(d), _ptr(c), _ptr(s), _ptr(t), _ptr(u))
    if st:
        raise np.linalg.LinAlgError(f"singular global system (status {st})")
    return u
