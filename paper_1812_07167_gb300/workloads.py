"""Seeded synthetic inputs for the 2-D Helmholtz impedance problem.

    -Laplace(u) - kappa^2 c(x) u = s   in the rectangle Omega,
    du/dnu + i eta u = t               on its boundary        (Eq. (1))

This module holds no arithmetic of the HPS method: it evaluates problem data
(the coefficient c, the body load s, the boundary data t and, where one
exists, the exact solution) at coordinates the caller passes in.  Both the
CUDA path and the CPU oracle take their inputs from here.

Randomness comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: value k of stream ``seed`` is SplitMix64's output for the state
``seed * 2**32 + k``.

The paper's own workload (Sec. 4) is a manufactured plane-wave solution on the
unit square with a Gaussian bump in c; no public dataset is involved.  The
workloads below have that shape at the sizes the solver is measured on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(state: int) -> int:
    """One SplitMix64 output for the given 64-bit state (after its increment)."""
    z = (state + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles in [0, 1) from stream ``seed`` (53 high bits)."""
    base = ((int(seed) & 0xFFFFFFFF) << 32) + int(offset)
    z = np.arange(count, dtype=np.uint64) + np.uint64(base & _M64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# outward unit normals of the sides in the public boundary order S, E, N, W
_NORMALS = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])


def boundary_sides(m: int, p: int, my: Optional[int] = None, per_edge: Optional[int] = None) -> np.ndarray:
    """Side index (0 S, 1 E, 2 N, 3 W) of each public outer-boundary node of
    an m x my leaf grid (my = m unless given), with per_edge nodes on each
    leaf edge (p - 2 unless given)."""
    my = m if not my else my
    e = per_edge or p - 2
    return np.concatenate([np.full(m * e, 0), np.full(my * e, 1), np.full(m * e, 2), np.full(my * e, 3)])


@dataclass
class Workload:
    """A problem instance: parameters plus the functions that define its data."""
    name: str
    m: int
    p: int
    kappa: float
    eta: complex
    c: Callable[[np.ndarray, np.ndarray], np.ndarray]
    s: Callable[[np.ndarray, np.ndarray], np.ndarray]
    # t(x, y, side) -> values; side indexes _NORMALS
    t: Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray]
    u_exact: Optional[Callable[[np.ndarray, np.ndarray], np.ndarray]] = None
    domain: tuple = (0.0, 1.0, 0.0, 1.0)
    notes: dict = field(default_factory=dict)
    my: int = 0  # leaves along y (0: m)

    def sample(self, leaf_xy: np.ndarray, bdry_xy: np.ndarray):
        """(c_int [leaves, e^2], s [leaves, e^2], t [4 m e]) at the given nodes.

        ``leaf_xy`` is [leaves, p^2-4, 2] in the public per-leaf order (edges
        first, then the (p-2)^2 interior nodes); ``bdry_xy`` is [4 m e, 2].
        """
        nb = 4 * (self.p - 2)
        xi = leaf_xy[:, nb:, 0]
        yi = leaf_xy[:, nb:, 1]
        c = np.asarray(self.c(xi, yi), dtype=np.float64)
        s = np.asarray(self.s(xi, yi), dtype=np.complex128)
        my = self.my or self.m
        side = boundary_sides(self.m, self.p, self.my, per_edge=len(bdry_xy) // (2 * (self.m + my)))
        t = np.asarray(self.t(bdry_xy[:, 0], bdry_xy[:, 1], side), dtype=np.complex128)
        return c, s, t


def _plane_wave(kappa: float, angle: float):
    d = np.array([math.cos(angle), math.sin(angle)])

    def u(x, y):
        return np.exp(1j * kappa * (d[0] * x + d[1] * y))

    def dudn(x, y, side):
        nrm = _NORMALS[side]
        return 1j * kappa * (d[0] * nrm[..., 0] + d[1] * nrm[..., 1]) * u(x, y)

    return u, dudn


def plane_wave_bump(m: int = 4, p: int = 16, kappa: float = 20.0, eta: Optional[complex] = None,
                    angle: float = 0.3) -> Workload:
    """Manufactured plane wave through a Gaussian dip in c.

    c = 1 - 0.5 exp(-50 |x - (0.5, 0.5)|^2), u = exp(i kappa (x cos a + y sin a)),
    s = kappa^2 (1 - c) u (so that -Lap u - kappa^2 c u = s), t = du/dnu + i eta u.
    Defaults: 4 x 4 leaves, p = 16, kappa = eta = 20.
    """
    eta = kappa if eta is None else eta
    u, dudn = _plane_wave(kappa, angle)

    def c(x, y):
        return 1.0 - 0.5 * np.exp(-50.0 * ((x - 0.5) ** 2 + (y - 0.5) ** 2))

    def s(x, y):
        return kappa ** 2 * (1.0 - c(x, y)) * u(x, y)

    def t(x, y, side):
        return dudn(x, y, side) + 1j * eta * u(x, y)

    return Workload("plane_wave_bump", m, p, kappa, eta, c, s, t, u_exact=u)


def gaussian_sources(seed: int, count: int = 8, width: float = 0.01):
    """Sum of ``count`` Gaussians exp(-|x - x_k|^2 / w^2) with unit complex
    amplitudes exp(i theta_k) and centres uniform in [0.1, 0.9]^2."""
    r = uniform(seed, 3 * count)
    cx = 0.1 + 0.8 * r[0::3]
    cy = 0.1 + 0.8 * r[1::3]
    amp = np.exp(2j * math.pi * r[2::3])

    def s(x, y):
        out = np.zeros(np.broadcast(x, y).shape, dtype=np.complex128)
        for k in range(count):
            out += amp[k] * np.exp(-((x - cx[k]) ** 2 + (y - cy[k]) ** 2) / width ** 2)
        return out

    return s, (cx, cy, amp)


def point_sources(m: int = 16, p: int = 16, kappa: float = 80.0, eta: Optional[complex] = None,
                  seed: int = 1) -> Workload:
    """Periodic medium with 8 narrow Gaussian sources and zero boundary data.

    c = 1 + 0.3 sin(4 pi x) cos(6 pi y); s = 8 seeded Gaussians of width 0.01
    with unit complex amplitudes; t = 0.  Defaults: 16 x 16 leaves, p = 16,
    kappa = eta = 80 (65,536 tensor nodes, 64,512 unknowns).
    """
    eta = kappa if eta is None else eta
    s, params = gaussian_sources(seed)

    def c(x, y):
        return 1.0 + 0.3 * np.sin(4 * math.pi * x) * np.cos(6 * math.pi * y)

    def t(x, y, side):
        return np.zeros(np.shape(x), dtype=np.complex128)

    return Workload("point_sources", m, p, kappa, eta, c, s, t,
                    notes={"sources": [list(map(float, v)) if np.isrealobj(v) else
                                       [complex(z) for z in v] for v in params]})


def random_medium(seed: int, modes: int = 32, kmax: int = 8, total: float = 0.5):
    """Smooth random field 1 + sum_k a_k cos(2 pi (kx x + ky y) + phi_k) with
    integer wave vectors in [-kmax, kmax]^2, a_k proportional to 1/(1+|k|^2)
    and sum |a_k| = total, so c stays in [1 - total, 1 + total]."""
    r = uniform(seed, 3 * modes, offset=1 << 20)
    kx = np.floor(r[0::3] * (2 * kmax + 1)).astype(int) - kmax
    ky = np.floor(r[1::3] * (2 * kmax + 1)).astype(int) - kmax
    phi = 2 * math.pi * r[2::3]
    a = 1.0 / (1.0 + kx ** 2 + ky ** 2)
    a = a * (total / a.sum())

    def c(x, y):
        out = np.ones(np.broadcast(x, y).shape)
        for k in range(modes):
            out += a[k] * np.cos(2 * math.pi * (kx[k] * x + ky[k] * y) + phi[k])
        return out

    return c


def random_medium_sources(m: int, p: int = 16, kappa: float = 300.0, eta: Optional[complex] = None,
                          seed: int = 2) -> Workload:
    """Random smooth medium (32 Fourier modes, c in [0.5, 1.5]) with 8 seeded
    Gaussian sources and zero boundary data."""
    eta = kappa if eta is None else eta
    c = random_medium(seed)
    s, _ = gaussian_sources(seed + 1000)

    def t(x, y, side):
        return np.zeros(np.shape(x), dtype=np.complex128)

    return Workload("random_medium_sources", m, p, kappa, eta, c, s, t)


def polynomial_solution(m: int, p: int, kappa: float, eta: complex, seed: int = 7,
                        c: Optional[Callable] = None, domain=(0.0, 1.0, 0.0, 1.0),
                        my: Optional[int] = None, deg: Optional[int] = None) -> Workload:
    """Manufactured solution that is a polynomial of degree p-1 (or deg) in x and in y.

    u(x, y) = sum_{a,b <= p-1} C_ab X^a Y^b with X, Y the coordinates scaled to
    [-1, 1] over the domain and seeded complex coefficients that decay with
    degree.  s = -Lap u - kappa^2 c u and t = du/dnu + i eta u are evaluated
    from the exact derivatives, so every collocation, impedance and interface
    condition of the discretisation holds exactly for u at the nodes.
    """
    x0, x1, y0, y1 = domain
    deg = p - 1 if deg is None else deg
    r = uniform(seed, 2 * (deg + 1) ** 2, offset=1 << 24)
    C = (r[0::2] - 0.5 + 1j * (r[1::2] - 0.5)).reshape(deg + 1, deg + 1)
    decay = np.array([[0.7 ** (a + b) for b in range(deg + 1)] for a in range(deg + 1)])
    C = C * decay
    sx, sy = 2.0 / (x1 - x0), 2.0 / (y1 - y0)
    if c is None:
        cfun = random_medium(seed, modes=6, kmax=3, total=0.4)
    else:
        cfun = c

    def _ev(x, y, dx=0, dy=0):
        X = sx * (np.asarray(x) - x0) - 1.0
        Y = sy * (np.asarray(y) - y0) - 1.0
        out = np.zeros(np.broadcast(X, Y).shape, dtype=np.complex128)
        for a in range(deg + 1):
            if a < dx:
                continue
            fa = math.perm(a, dx) * sx ** dx
            Xa = X ** (a - dx)
            for b in range(deg + 1):
                if b < dy:
                    continue
                fb = math.perm(b, dy) * sy ** dy
                out += C[a, b] * fa * fb * Xa * Y ** (b - dy)
        return out

    def u(x, y):
        return _ev(x, y)

    def s(x, y):
        return -(_ev(x, y, 2, 0) + _ev(x, y, 0, 2)) - kappa ** 2 * cfun(x, y) * _ev(x, y)

    def t(x, y, side):
        nrm = _NORMALS[side]
        return nrm[..., 0] * _ev(x, y, 1, 0) + nrm[..., 1] * _ev(x, y, 0, 1) + 1j * eta * _ev(x, y)

    return Workload("polynomial_solution", m, p, kappa, eta, cfun, s, t, u_exact=u, domain=domain,
                    my=my or m)


def random_data(m: int, p: int, kappa: float, eta: complex, seed: int, nrhs: int = 1,
                my: Optional[int] = None):
    """Unstructured seeded data: c in [0.5, 1.5] at the (p-2)^2 interior nodes of
    each leaf of an m x my grid (my = m unless given), complex s (same nodes)
    and t (outer boundary), values in the unit box.  Returned as
    (c [leaves, e^2], s [nrhs, leaves, e^2], t [nrhs, 2 (m + my) e])."""
    e = p - 2
    my = m if not my else my
    L = m * my
    nb = 2 * (m + my) * e
    r = uniform(seed, L * e * e + 2 * nrhs * (L * e * e + nb), offset=1 << 28)
    k = 0
    c = 0.5 + r[k:k + L * e * e].reshape(L, e * e)
    k += L * e * e
    ns = nrhs * L * e * e
    s = (r[k:k + ns] - 0.5 + 1j * (r[k + ns:k + 2 * ns] - 0.5)).reshape(nrhs, L, e * e)
    k += 2 * ns
    nt = nrhs * nb
    t = (r[k:k + nt] - 0.5 + 1j * (r[k + nt:k + 2 * nt] - 0.5)).reshape(nrhs, nb)
    return c, s, t


def request_stream(seed: int, count: int, rate: float, solve_frac: float = 0.9, nrhs_max: int = 64,
                   build_m=(16, 32, 64), kappa_range=(20.0, 200.0)):
    """Arrival schedule of the serving workload (scheduling data only).

    Arrivals form a Poisson process of ``rate`` requests per second
    (exponential gaps of mean 1/rate; ``rate = 0`` puts every arrival at 0,
    a backlog).  Each request is a solve with probability ``solve_frac``,
    carrying nrhs uniform in 1..nrhs_max right-hand sides, else a build of
    m x m leaves with m uniform in ``build_m`` and kappa uniform in
    ``kappa_range``.  The draws other than the gaps do not depend on the
    rate, so schedules at different loads hold the same requests.  Returns a
    list of dicts with keys arrival, kind, nrhs, m, kappa, seed.
    """
    r = uniform(seed, 4 * count, offset=1 << 40)
    gap = -np.log1p(-r[0::4])
    arrival = np.cumsum(gap) / rate if rate > 0 else np.zeros(count)
    out = []
    for k in range(count):
        if r[4 * k + 1] < solve_frac:
            out.append(dict(arrival=float(arrival[k]), kind="solve",
                            nrhs=1 + int(r[4 * k + 2] * nrhs_max), m=0, kappa=0.0, seed=seed * 1000 + k))
        else:
            lo, hi = kappa_range
            out.append(dict(arrival=float(arrival[k]), kind="build", nrhs=0,
                            m=int(build_m[int(r[4 * k + 2] * len(build_m))]),
                            kappa=float(lo + (hi - lo) * r[4 * k + 3]), seed=seed * 1000 + k))
    return out


def ragged_batch(count: int = 32, seed0: int = 100, p: int = 16, ms=(8, 16, 32), kappa_range=(20.0, 200.0)):
    """Independent problems of different sizes for batched builds: problem k
    (seed seed0 + k) has m x m leaves with m uniform in ``ms``, kappa = eta
    uniform in ``kappa_range`` and the random smooth medium of that seed
    (32 Fourier modes, c in [0.5, 1.5]).  Returns a list of (m, kappa, c)."""
    out = []
    lo, hi = kappa_range
    for k in range(count):
        r = uniform(seed0 + k, 2, offset=1 << 44)
        out.append((int(ms[int(r[0] * len(ms))]), float(lo + (hi - lo) * r[1]), random_medium(seed0 + k)))
    return out
