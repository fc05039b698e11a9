"""Pins of the oracle's Gauss-Legendre interface mode (boundary data on q
Gauss-Legendre nodes per leaf edge, reached from the leaves' corner-free
Chebyshev edge nodes by polynomial interpolation), each against something
the oracle does not compute itself:

* the nodes against numpy's Gauss-Legendre rule;
* the interpolation matrices against direct evaluation of polynomials;
* the hierarchical build + solve against the dense global system of the same
  discretisation (unknowns: every leaf's nodal values and its incoming data on
  the Gauss nodes of its edges);
* for q >= p-2: the same solution as the paper's Chebyshev-edge scheme when the
  boundary data agree (an exact polynomial change of basis on every edge);
* for q < p-2: a polynomial of degree q-1 in x and in y is reproduced at every
  node (its traces lie in the interface space), while one of degree q+1 is
  not.
"""
import numpy as np
import pytest

import oracle as O
from paper_1812_07167_gb300 import workloads as W


def _cheb_edge(p):
    # corner-free Chebyshev nodes of the reference edge [-1, 1], increasing
    j = np.arange(1, p - 1)
    return -np.cos(np.pi * j / (p - 1))


def _lagrange_matrix(src, dst):
    """L[i, j] = the j-th Lagrange basis polynomial of the nodes src at dst[i],
    through a Vandermonde solve in the Legendre basis (numpy)."""
    V = np.polynomial.legendre.legvander(src, len(src) - 1)
    Vd = np.polynomial.legendre.legvander(dst, len(src) - 1)
    return Vd @ np.linalg.inv(V)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 7, 14, 16, 25])
def test_gauss_nodes_match_numpy(q):
    z = O.gauss_nodes(q)
    assert np.all(np.diff(z) > 0)
    assert np.abs(z - np.polynomial.legendre.leggauss(q)[0]).max() < 1e-14


@pytest.mark.parametrize("p,q", [(8, 3), (8, 6), (8, 9), (12, 7), (16, 14), (16, 16)])
def test_edge_interpolation_is_exact_on_polynomials(p, q):
    e = p - 2
    Pm, Qm = O.edge_interp(p, q)
    ce, zg = _cheb_edge(p), np.polynomial.legendre.leggauss(q)[0]
    rng = np.random.default_rng(p * 31 + q)
    # degree e-1 polynomial: its Chebyshev-node samples give its Gauss-node values
    a = rng.standard_normal(e)
    assert np.abs(Pm @ np.polynomial.polynomial.polyval(ce, a) - np.polynomial.polynomial.polyval(zg, a)).max() < 1e-11
    # degree q-1 polynomial: its Gauss-node samples give its Chebyshev-node values
    b = rng.standard_normal(q)
    assert np.abs(Qm @ np.polynomial.polynomial.polyval(zg, b) - np.polynomial.polynomial.polyval(ce, b)).max() < 1e-11
    # and the same matrices as an independent Vandermonde construction
    assert np.abs(Pm - _lagrange_matrix(ce, zg)).max() < 1e-9
    assert np.abs(Qm - _lagrange_matrix(zg, ce)).max() < 1e-9


@pytest.mark.parametrize("m,my,p,q", [(1, 1, 8, 4), (2, 2, 8, 4), (2, 2, 8, 9), (4, 4, 6, 3), (2, 1, 10, 5),
                                      (1, 2, 6, 6)])
def test_gauss_hps_equals_dense_global_solve(m, my, p, q):
    pr = O.Problem(m, p, 7.0, 5.0 - 2.0j, my=my, q=q)
    rng = np.random.default_rng(m + 10 * p + q)
    c = 0.5 + rng.random((pr.leaves, pr.ni))
    s = rng.standard_normal((pr.leaves, pr.ni)) + 1j * rng.standard_normal((pr.leaves, pr.ni))
    t = rng.standard_normal(pr.nbdry) + 1j * rng.standard_normal(pr.nbdry)
    with O.Tree(pr, c) as T:
        assert T.status == 0
        u = T.solve(s[None], t[None])[0]
    ub = O.brute(pr, c, s, t)
    assert np.abs(u - ub).max() / np.abs(ub).max() < 1e-12


@pytest.mark.parametrize("m,p,q", [(2, 8, 6), (2, 8, 9), (4, 6, 4), (4, 6, 7), (2, 10, 12)])
def test_gauss_q_at_least_p_minus_2_is_the_chebyshev_scheme(m, p, q):
    prg, prn = O.Problem(m, p, 7.0, 7.0, q=q), O.Problem(m, p, 7.0, 7.0)
    rng = np.random.default_rng(q)
    c = 0.5 + rng.random((prn.leaves, prn.ni))
    s = rng.standard_normal((prn.leaves, prn.ni)) + 0j
    tn = rng.standard_normal(prn.nbdry) + 1j * rng.standard_normal(prn.nbdry)
    # the same boundary data: the Chebyshev-node values' interpolant at the Gauss nodes
    P = _lagrange_matrix(_cheb_edge(p), np.polynomial.legendre.leggauss(q)[0])
    tg = (P @ tn.reshape(-1, p - 2).T).T.reshape(-1)
    with O.Tree(prg, c) as T:
        ug = T.solve(s[None], tg[None])[0]
    with O.Tree(prn, c) as T:
        un = T.solve(s[None], tn[None])[0]
    assert np.abs(ug - un).max() / np.abs(un).max() < 1e-12


@pytest.mark.parametrize("m,my,p,q", [(2, 2, 10, 5), (4, 4, 8, 3), (2, 2, 12, 7), (2, 1, 8, 4)])
def test_gauss_polynomial_of_degree_q_minus_1_is_exact(m, my, p, q):
    pr = O.Problem(m, p, 9.0, 4.0 - 1.0j, my=my, q=q)
    lxy, bxy = O.nodes(pr)
    ok = W.polynomial_solution(m, p, 9.0, 4.0 - 1.0j, deg=q - 1, my=my)
    c, s, t = ok.sample(lxy, bxy)
    with O.Tree(pr, c) as T:
        u = T.solve(s[None], t[None])[0]
    ue = ok.u_exact(lxy[..., 0], lxy[..., 1])
    assert np.abs(u - ue).max() / np.abs(ue).max() < 1e-12
    # one degree too many for the interface space: no longer exact
    bad = W.polynomial_solution(m, p, 9.0, 4.0 - 1.0j, deg=q + 1, my=my)
    c, s, t = bad.sample(lxy, bxy)
    with O.Tree(pr, c) as T:
        u = T.solve(s[None], t[None])[0]
    ue = bad.u_exact(lxy[..., 0], lxy[..., 1])
    assert np.abs(u - ue).max() / np.abs(ue).max() > 1e-6


def test_gauss_boundary_nodes():
    pr = O.Problem(2, 8, 5.0, 5.0, 0.0, 2.0, 0.0, 1.0, my=1, q=5)
    _, bxy = O.nodes(pr)
    z = np.polynomial.legendre.leggauss(5)[0]
    # south side: two leaf edges of width 1, the Gauss nodes of each
    assert np.allclose(bxy[:5, 0], 0.5 * (z + 1)) and np.allclose(bxy[5:10, 0], 1 + 0.5 * (z + 1))
    assert np.allclose(bxy[:10, 1], 0.0)
    # east side: one leaf edge of height 1 at x = 2
    assert np.allclose(bxy[10:15, 0], 2.0) and np.allclose(bxy[10:15, 1], 0.5 * (z + 1))
    assert bxy.shape == (2 * (2 + 1) * 5, 2)
