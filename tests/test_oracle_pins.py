"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties the oracle to something fixed by the paper (arXiv:1812.07167)
or by mathematics: textbook closed forms, exact reproduction of polynomial
solutions, a different algorithm (the dense global collocation solve),
spectral convergence, and the isometry / reciprocity of the ItI map.
"""
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as Ch
from numpy.polynomial import legendre as Lg

import oracle as O
from _geometry import coincident_pairs
from paper_1812_07167_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _problem(wl):
    x0, x1, y0, y1 = wl.domain
    return O.Problem(wl.m, wl.p, wl.kappa, wl.eta, x0, x1, y0, y1)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# ---------------------------------------------------------------- Sec. 2.1


@pytest.mark.parametrize("N,name", [(1, "cheb_D_N1.txt"), (2, "cheb_D_N2.txt")])
def test_cheb_matches_textbook_example(N, name):
    """Trefethen's worked N = 1 and N = 2 matrices (the paper's Sec. 2.1 source)."""
    x, D = O.cheb(N + 1)
    assert np.allclose(x, np.cos(np.pi * np.arange(N, -1, -1) / N), atol=1e-15)
    np.testing.assert_allclose(D, _load_golden(name), atol=1e-14)


@pytest.mark.parametrize("p", [4, 9, 16, 21])
def test_cheb_closed_form_entries(p):
    """Corner and interior diagonal entries from their closed forms (the
    oracle's diagonal uses the negative-sum rule instead)."""
    N = p - 1
    x, D = O.cheb(p)
    assert D[0, 0] == pytest.approx(-(2 * N * N + 1) / 6.0, rel=1e-12)
    assert D[N, N] == pytest.approx((2 * N * N + 1) / 6.0, rel=1e-12)
    for j in range(1, N):
        assert D[j, j] == pytest.approx(-x[j] / (2 * (1 - x[j] ** 2)), abs=1e-11 * N * N)


@pytest.mark.parametrize("p,a,b", [(5, -1.0, 1.0), (16, 0.25, 0.3125), (20, -3.0, 2.0)])
def test_cheb_differentiates_polynomials_exactly(p, a, b):
    rng = np.random.default_rng(p)
    coef = rng.standard_normal(p)  # degree p-1 in the Chebyshev basis of [a, b]
    x, D = O.cheb(p, a, b)
    s = 2 * (x - a) / (b - a) - 1
    f = Ch.chebval(s, coef)
    df = Ch.chebval(s, Ch.chebder(coef)) * 2 / (b - a)
    np.testing.assert_allclose(D @ f, df, atol=1e-11 * np.abs(df).max() * p * p)


def test_leaf_operators_satisfy_their_definitions():
    """B [Psi Y] = I (Eqs. hmgsolnopdef, prtsolnopdef), R = G Psi, Gamma = G Y,
    and the corner-free node count n = p^2 - 4 (Sec. 2.1)."""
    pr = O.Problem(1, 10, 7.0, 4.0 + 1.0j, 0.0, 0.5, 0.0, 0.25)
    rng = np.random.default_rng(3)
    c = 0.5 + rng.random(pr.ni)
    Psi, Y, R, Gam, B, F, G = O.leaf(pr, c, with_matrices=True)
    assert B.shape == (96, 96) and Psi.shape == (96, 32) and Y.shape == (96, 64)
    X = np.hstack([Psi, Y])
    assert np.abs(B @ X - np.eye(pr.n)).max() < 1e-9
    np.testing.assert_allclose(R, G @ Psi, atol=1e-12 * np.abs(R).max())
    np.testing.assert_allclose(Gam, G @ Y, atol=1e-12 * np.abs(Gam).max())
    # F and G differ only by 2 i eta on the boundary diagonal
    D = F - G
    assert np.allclose(D[:, :pr.nb], 2j * pr.eta * np.eye(pr.nb))
    assert np.allclose(D[:, pr.nb:], 0)


def test_leaf_normal_derivative_signs():
    """N applied to u = x (resp. y) gives the outward normal's x (y) component
    on each side: south (0,-1), east (1,0), north (0,1), west (-1,0)."""
    pr = O.Problem(1, 8, 1.0, 1.0)
    _, _, _, _, _, F, G = O.leaf(pr, np.ones(pr.ni), with_matrices=True)
    N = 0.5 * (F + G)
    lxy, _ = O.nodes(pr)
    x, y = lxy[0, :, 0], lxy[0, :, 1]
    e = pr.e
    nx = np.repeat([0, 1, 0, -1], e)
    ny = np.repeat([-1, 0, 1, 0], e)
    np.testing.assert_allclose((N @ x).real, nx, atol=1e-12)
    np.testing.assert_allclose((N @ y).real, ny, atol=1e-12)


# ------------------------------------------------ exactness and brute force


@pytest.mark.parametrize(
    "m,p,kappa,eta,domain",
    [
        (1, 6, 3.0, 2.0, (0.0, 1.0, 0.0, 1.0)),
        (2, 8, 5.0, 3.0 - 1.0j, (0.0, 1.0, 0.0, 1.0)),
        (4, 8, 9.0, 9.0, (-1.0, 1.0, 0.5, 1.0)),
        (4, 12, 20.0, 20.0, (0.0, 1.0, 0.0, 1.0)),
        (8, 6, 12.0, 0.5 + 2.0j, (0.0, 2.0, 0.0, 1.0)),
    ],
)
def test_polynomial_solution_reproduced_to_rounding(m, p, kappa, eta, domain):
    """A polynomial of degree p-1 in x and y satisfies every discrete equation
    exactly, so the HPS solution equals it at all nodes up to rounding.  This
    pins the leaf operators, the normal signs, the merge formulas and the
    index bookkeeping end to end."""
    wl = W.polynomial_solution(m, p, kappa, eta, domain=domain)
    pr = _problem(wl)
    lxy, bxy = O.nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    with O.Tree(pr, c) as T:
        assert T.status == 0
        u = T.solve(s[None], t[None])[0]
    ue = wl.u_exact(lxy[..., 0], lxy[..., 1])
    assert _rel(u, ue) < 1e-10


@pytest.mark.parametrize(
    "m,p,kappa,eta",
    [(1, 8, 10.0, 10.0), (2, 8, 6.0, 2.0 + 1.0j), (2, 12, 15.0, 15.0), (4, 8, 25.0, 25.0), (4, 10, 12.0, 3.0)],
)
def test_hps_equals_dense_global_solve(m, p, kappa, eta):
    """HPS (Algorithms 1 and 2) solves the same global collocation system as
    a dense LU of all leaf rows plus the interface conditions of Sec. 2.2."""
    pr = O.Problem(m, p, kappa, eta)
    c, s, t = W.random_data(m, p, kappa, eta, seed=11 + m + p)
    ub = O.brute(pr, c, s[0], t[0])
    with O.Tree(pr, c) as T:
        u = T.solve(s, t)[0]
    assert _rel(u, ub) < 1e-12  # the brute-force bar; measured 2e-15 ... 4.9e-13


def test_merge_order_does_not_change_the_solution():
    """Pairing south/north leaves first instead of west/east gives a different
    tree over the same global system, hence the same u up to rounding."""
    pr = O.Problem(4, 10, 14.0, 14.0)
    c, s, t = W.random_data(4, 10, 14.0, 14.0, seed=5, nrhs=2)
    with O.Tree(pr, c) as A, O.Tree(pr, c, first_vertical=True) as B:
        ua = A.solve(s, t)
        ub = B.solve(s, t)
        Ra, Rb = A.root_R(), B.root_R()
    assert _rel(ua, ub) < 1e-11
    assert _rel(Ra, Rb) < 1e-11


# ------------------------------------------------ rectangular leaf grids


@pytest.mark.parametrize("mx,my,p", [(2, 1, 8), (1, 2, 8), (4, 2, 6), (2, 8, 6), (1, 4, 8)])
def test_rectangular_grid_polynomial_reproduced(mx, my, p):
    """mx != my leaf grids (merges alternate, then the longer axis takes the
    remaining ones): the polynomial solution is still reproduced at every
    node, on a domain whose aspect ratio differs from the grid's."""
    wl = W.polynomial_solution(mx, p, 9.0, 4.0 - 1.0j, domain=(0.0, 1.5, -0.5, 0.5), my=my)
    pr = O.Problem(mx, p, wl.kappa, wl.eta, 0.0, 1.5, -0.5, 0.5, my=my)
    lxy, bxy = O.nodes(pr)
    assert lxy.shape[0] == mx * my and bxy.shape[0] == 2 * (mx + my) * (p - 2)
    c, s, t = wl.sample(lxy, bxy)
    with O.Tree(pr, c) as T:
        assert T.status == 0
        u = T.solve(s[None], t[None])[0]
    assert _rel(u, wl.u_exact(lxy[..., 0], lxy[..., 1])) < 1e-10


@pytest.mark.parametrize("mx,my", [(2, 1), (1, 2), (4, 2), (2, 4)])
def test_rectangular_grid_equals_dense_global_solve(mx, my):
    pr = O.Problem(mx, 8, 12.0, 12.0, my=my)
    c, s, t = W.random_data(mx, 8, 12.0, 12.0, seed=40 + mx * 10 + my, my=my)
    ub = O.brute(pr, c, s[0], t[0])
    with O.Tree(pr, c) as T:
        u = T.solve(s, t)[0]
    assert _rel(u, ub) < 1e-12  # the brute-force bar; measured 2e-15 ... 4.9e-13


def test_rectangular_grid_nodes_cover_the_domain():
    pr = O.Problem(4, 6, 5.0, 5.0, 0.0, 2.0, 0.0, 0.5, my=1)
    lxy, bxy = O.nodes(pr)
    # every leaf inside the domain, leaves side by side along x
    assert lxy[..., 0].min() == 0.0 and lxy[..., 0].max() == 2.0
    assert lxy[..., 1].min() == 0.0 and lxy[..., 1].max() == 0.5
    cols = sorted({round(float(lxy[l, :, 0].min()), 12) for l in range(4)})
    assert cols == [0.0, 0.5, 1.0, 1.5]
    # outer boundary: S then E then N then W, 4 + 1 + 4 + 1 leaf edges of 4 nodes
    assert np.all(bxy[:16, 1] == 0.0) and np.all(bxy[16:20, 0] == 2.0)
    assert np.all(bxy[20:36, 1] == 0.5) and np.all(bxy[36:, 0] == 0.0)


def test_rectangular_merge_order_does_not_change_the_solution():
    pr = O.Problem(4, 8, 10.0, 10.0, my=2)
    c, s, t = W.random_data(4, 8, 10.0, 10.0, seed=6, nrhs=2, my=2)
    with O.Tree(pr, c) as A, O.Tree(pr, c, first_vertical=True) as B:
        ua, ub = A.solve(s, t), B.solve(s, t)
        Ra, Rb = A.root_R(), B.root_R()
    assert _rel(ua, ub) < 1e-11
    assert _rel(Ra, Rb) < 1e-11


def test_threads_change_no_arithmetic():
    pr = O.Problem(4, 8, 11.0, 11.0)
    c, s, t = W.random_data(4, 8, 11.0, 11.0, seed=9, nrhs=3)
    with O.Tree(pr, c, nthreads=1) as A, O.Tree(pr, c, nthreads=4) as B:
        assert np.array_equal(A.solve(s, t, 1), B.solve(s, t, 4))
        assert np.array_equal(A.root_R(), B.root_R())


def test_solve_is_linear_in_s_and_t():
    pr = O.Problem(2, 8, 9.0, 9.0)
    c, s, t = W.random_data(2, 8, 9.0, 9.0, seed=21, nrhs=2)
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    with O.Tree(pr, c) as T:
        u = T.solve(s, t)
        ul = T.solve(a * s[:1] + b * s[1:], a * t[:1] + b * t[1:])[0]
    assert _rel(ul, a * u[0] + b * u[1]) < 1e-12


def test_leaf_identity_in_the_tree():
    """Remark in Sec. 2.1: u = Psi t + Y s on each leaf, with t the leaf's
    incoming impedance data; checked through F u = t and the interior rows."""
    pr = O.Problem(2, 8, 6.0, 6.0)
    c, s, t = W.random_data(2, 8, 6.0, 6.0, seed=4)
    with O.Tree(pr, c) as T:
        u = T.solve(s, t)[0]
        for leaf in range(pr.leaves):
            Psi, Y, R, Gam, B, F, G = O.leaf(pr, c[leaf], with_matrices=True)
            r = B @ u[leaf]
            np.testing.assert_allclose(r[pr.nb:], s[0, leaf], atol=1e-9 * np.abs(s).max())
            Psi2, Y2, Gam2 = T.leaf_ops(leaf)
            np.testing.assert_array_equal(Psi2, Psi)
            np.testing.assert_array_equal(Gam2, Gam)
            # outgoing data: G u = R t + Gamma s with t = F u the incoming data
            tl = r[:pr.nb]
            np.testing.assert_allclose(G @ u[leaf], R @ tl + Gam @ s[0, leaf],
                                       atol=1e-12 * np.abs(G @ u[leaf]).max())  # ~2e-14 measured


def test_interface_condition_number_of_two_leaves():
    """cond_1(W) reported for the one merge of a 2 x 1 grid equals that of
    W = I - R33b R33a assembled here from the two leaves' own ItI operators:
    I3 is the west leaf's east edge and the east leaf's west edge (nodes
    [e, 2e) and [3e, 4e) of the [S, E, N, W] order, both running upwards)."""
    for kappa, eta in ((10.0, 10.0), (25.0, 4.0 - 3.0j)):
        pr = O.Problem(2, 10, kappa, eta, my=1)
        c, _, _ = W.random_data(2, 10, kappa, eta, seed=17, my=1)
        e = pr.e
        Ra = O.leaf(pr, c[0])[2]
        Rb = O.leaf(pr, c[1])[2]
        Wm = np.eye(e) - Rb[3 * e:, 3 * e:] @ Ra[e:2 * e, e:2 * e]
        with O.Tree(pr, c) as T:
            cw = T.cond_W()
        assert len(cw) == 1
        assert cw[0] == pytest.approx(np.linalg.cond(Wm, 1), rel=1e-8)


def test_interface_condition_numbers_per_level():
    pr = O.Problem(4, 8, 20.0, 20.0)
    c, _, _ = W.random_data(4, 8, 20.0, 20.0, seed=2)
    with O.Tree(pr, c) as T:
        cw = T.cond_W()
    assert len(cw) == 4 and all(v >= 1.0 for v in cw)


def test_duplicate_interface_values_agree():
    """Subtracting the two impedance-matching rows of a shared edge node
    (Sec. 2.2) leaves 2 i eta (u_alpha - u_beta) = 0, so for eta != 0 both
    copies of every interface node carry the same value to rounding."""
    pr = O.Problem(4, 10, 13.0, 5.0 - 2.0j, 0.0, 1.0, -0.5, 0.5)
    c, s, t = W.random_data(4, 10, 13.0, 5.0 - 2.0j, seed=31, nrhs=2)
    lxy, _ = O.nodes(pr)
    (la, lb), (na, nb) = coincident_pairs(lxy)
    # 4 x 4 leaves: 24 interior leaf edges of p - 2 nodes each
    assert la.size == 24 * (pr.p - 2)
    with O.Tree(pr, c) as T:
        u = T.solve(s, t)
    d = np.abs(u[:, la, na] - u[:, lb, nb]).max()
    assert d < 1e-11 * np.abs(u).max()
    # and it is a property of the solution, not of the data: a single leaf's
    # own solve does not have it
    assert np.abs(u[:, la, na]).max() > 1e-3 * np.abs(u).max()


# --------------------------------------------------------- convergence, ItI


def test_plane_wave_converges_spectrally():
    """Manufactured plane wave through a Gaussian dip (4 x 4 leaves, kappa =
    eta = 20): the nodal error falls by orders of magnitude as p grows (the
    trend of the paper's accuracy study, Sec. 4.1)."""
    errs = {}
    for p in (8, 12, 16):
        wl = W.plane_wave_bump(m=4, p=p)
        pr = _problem(wl)
        lxy, bxy = O.nodes(pr)
        c, s, t = wl.sample(lxy, bxy)
        with O.Tree(pr, c) as T:
            u = T.solve(s[None], t[None])[0]
        errs[p] = np.abs(u - wl.u_exact(lxy[..., 0], lxy[..., 1])).max()
    assert errs[8] > 1e2 * errs[12] > 1e4 * errs[16]
    assert errs[16] < 1e-9


def _interp(xs, xt, a, b):
    s = lambda x: 2 * (x - a) / (b - a) - 1
    return Ch.chebvander(s(xt), len(xs) - 1) @ np.linalg.inv(Ch.chebvander(s(xs), len(xs) - 1))


def _edge_mass(pr, h):
    """Gauss-Legendre quadrature of |f|^2 over one edge, acting on the values
    at the p-2 corner-free Chebyshev edge nodes (q = p - 2 Gauss points)."""
    xc, _ = O.cheb(pr.p, 0.0, h)
    g, w = Lg.leggauss(pr.e)
    P = _interp(xc[1:-1], (g + 1) * h / 2, 0.0, h)
    return P.conj().T @ np.diag(w * h / 2) @ P


@pytest.mark.parametrize("p,tol", [(12, 1e-5), (16, 1e-7)])
def test_root_ItI_is_an_isometry_and_reciprocal(p, tol):
    """For real kappa, c, eta, Green's identity makes the ItI map an L2
    isometry, and reciprocity makes it symmetric in the bilinear L2 pairing
    (Definition of the ItI map, Sec. 2).  Checked on smooth incoming data."""
    m = 4
    wl = W.plane_wave_bump(m=m, p=p)
    pr = _problem(wl)
    lxy, bxy = O.nodes(pr)
    c, _, _ = wl.sample(lxy, bxy)
    with O.Tree(pr, c) as T:
        R = T.root_R()
    M = np.kron(np.eye(4 * m), _edge_mass(pr, 1.0 / m))
    side = W.boundary_sides(m, p)
    F = []
    for k, ang in enumerate(np.linspace(0.1, 2.9, 5)):
        u, dudn = W._plane_wave(20.0 * (0.5 + 0.2 * k), ang)
        F.append(dudn(bxy[:, 0], bxy[:, 1], side) + 1j * 20.0 * u(bxy[:, 0], bxy[:, 1]))
    F = np.array(F).T
    G = R @ F
    nf = np.real(np.einsum("ik,ij,jk->k", F.conj(), M, F))
    ng = np.real(np.einsum("ik,ij,jk->k", G.conj(), M, G))
    assert np.max(np.abs(ng - nf) / nf) < tol
    S = F.T @ M @ R @ F
    assert np.abs(S - S.T).max() / np.abs(S).max() < 10 * tol


@pytest.mark.parametrize("eta", [20.0 - 5.0j, 3.0 + 8.0j])
def test_root_ItI_is_reciprocal_for_complex_eta(eta):
    """Reciprocity needs no real eta: R = (Lambda - i eta)(Lambda + i eta)^-1
    with a symmetric Dirichlet-to-Neumann map Lambda is symmetric in the
    bilinear L2 pairing for any eta (the isometry is lost, the symmetry is
    not).  Checked on smooth data at p = 16."""
    m, p = 4, 16
    wl = W.plane_wave_bump(m=m, p=p, eta=eta)
    pr = _problem(wl)
    lxy, bxy = O.nodes(pr)
    c, _, _ = wl.sample(lxy, bxy)
    with O.Tree(pr, c) as T:
        R = T.root_R()
    M = np.kron(np.eye(4 * m), _edge_mass(pr, 1.0 / m))
    side = W.boundary_sides(m, p)
    F = []
    for k, ang in enumerate(np.linspace(0.1, 2.9, 5)):
        u, dudn = W._plane_wave(20.0 * (0.5 + 0.2 * k), ang)
        F.append(dudn(bxy[:, 0], bxy[:, 1], side) + 1j * eta * u(bxy[:, 0], bxy[:, 1]))
    F = np.array(F).T
    S = F.T @ M @ R @ F
    assert np.abs(S - S.T).max() / np.abs(S).max() < 1e-7  # 3.4e-9 and 3.0e-9 measured
